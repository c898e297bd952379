"""CPU tests of the tiled kernel's schedule (host logic; no GPU needed).

The C ABI builds a pass's stage list and coefficient rows exactly as the
stepper does.  Against the oracle's own matrices (built by a different
method), every input of the other parity must stream by once, every output
must be finalised once and only after every input it couples to through Mx
or My (eq. central_differences, section 5.5) has streamed by, and the
coefficient rows must hold -Mx/dx and -My/dy of those couplings, each
value twice (one per point of an f32x2 pair)."""
import numpy as np
import pytest

from oracle import pn_oracle as O

ORDERS = [1, 2, 3, 4, 5, 8, 13, 22, 39, 63]


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1211_2205_gb300 import capi as c
    return c


@pytest.mark.parametrize("N", ORDERS)
@pytest.mark.parametrize("parity", [0, 1])
def test_inputs_stream_before_the_outputs_they_reach(capi, N, parity):
    Mx, My, order = O.system_matrices("pn2d", N)
    n = len(order)
    st, co, fi = capi.tiled_schedule(N, parity)
    seen, done = set(), []
    for s in st:
        for k in s[:2]:
            if k >= 0:
                assert order[k] % 2 != parity and k not in seen
                seen.add(int(k))
        for j in s[2:]:
            if j >= 0:
                assert order[j] % 2 == parity and j not in done
                need = set(np.nonzero(Mx[j])[0]) | set(np.nonzero(My[j])[0])
                assert need <= seen, (int(j), sorted(need - seen))
                done.append(int(j))
    assert seen == {k for k in range(n) if order[k] % 2 != parity}
    assert set(done) == {j for j in range(n) if order[j] % 2 == parity}
    assert [int(j) for j in fi if j >= 0] == done
    # one coefficient row pair (R, I) per stage that streams an input
    assert co.shape[0] == 2 * sum(1 for s in st if s[0] >= 0)


@pytest.mark.parametrize("N", [7, 8, 13])
def test_frozen_top_order_is_never_finalised(capi, N):
    """A closure sets the order-N moments: the pass of their parity leaves
    them out (no stage loads or writes them); the other pass still reads
    them as inputs."""
    Mx, My, order = O.system_matrices("pn2d", N)
    st, co, fi = capi.tiled_schedule(N, N % 2, frozen_top=True)
    outs = {int(j) for s in st for j in s[2:] if j >= 0}
    assert outs == {j for j in range(len(order)) if order[j] % 2 == N % 2 and order[j] < N}
    st, co, fi = capi.tiled_schedule(N, 1 - N % 2, frozen_top=True)
    ins = {int(k) for s in st for k in s[:2] if k >= 0}
    assert {j for j in range(len(order)) if order[j] == N} <= ins


@pytest.mark.parametrize("N", ORDERS)
@pytest.mark.parametrize("parity", [0, 1])
def test_coefficient_rows_are_the_oracles_couplings(capi, N, parity):
    dx, dy = 0.3, 0.7
    Mx, My, order = O.system_matrices("pn2d", N)
    comps = O.real_moments(N)
    index = {c: i for i, c in enumerate(comps)}
    st, co, fi = capi.tiled_schedule(N, parity, dx=dx, dy=dy)
    used = np.zeros((2, len(comps), len(comps)), dtype=bool)
    r = 0
    for s in st:
        if s[0] < 0:
            continue
        for kind_pos in (0, 1):
            row = co[r]
            r += 1
            k = int(s[kind_pos])
            if k < 0:
                assert not row.any()
                continue
            kind, lp, m = comps[k]
            q = (lp - m) // 2
            other = "I" if kind == "R" else "R"
            # targets in reach (Lemma 2): order lp-1 with q-1, q; order lp+1 with q, q+1
            for t, (L, Q) in enumerate(((lp - 1, q - 1), (lp - 1, q), (lp + 1, q), (lp + 1, q + 1))):
                for part, (tkind, M, h) in enumerate(((kind, Mx, dx), (other, My, dy))):
                    pair = row[8 * part + 2 * t: 8 * part + 2 * t + 2]
                    assert pair[0] == pair[1]
                    j = index.get((tkind, L, L - 2 * Q)) if 0 <= Q and L - 2 * Q >= 0 else None
                    want = 0.0 if j is None else -M[j, k] / h
                    assert pair[0] == np.float32(want), (k, t, part)
                    if j is not None and M[j, k] != 0:
                        used[part, j, k] = True
    assert r == co.shape[0]
    # every coupling between the two parities appears in some row
    for part, M in enumerate((Mx, My)):
        cross = (M != 0) & (order[:, None] % 2 == parity) & (order[None, :] % 2 != parity)
        assert np.array_equal(used[part], cross)


def test_schedule_rejects_bad_arguments(capi):
    with pytest.raises(capi.StarmapError):
        capi.tiled_schedule(0, 1)
    with pytest.raises(capi.StarmapError):
        capi.tiled_schedule(64, 1)
    with pytest.raises(capi.StarmapError):
        capi.tiled_schedule(5, 2)
