"""CPU tests of the C-ABI library: it loads without a GPU, exports every
function include/starmap.h declares, and its host mathematics (moment
matrices, grid placement, lambda_max, E) agrees with the oracle."""
import os

import numpy as np
import pytest

from oracle import pn_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1211_2205_gb300 import capi as c
    return c


def test_library_exports_every_declared_symbol(capi):
    L = capi.lib()
    names = capi.exported_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(L, name), name


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 13, 39])
def test_host_matrices_match_oracle(capi, N):
    Mx, My, grid, order, lam = capi.host_matrices(capi.PN2D, N)
    Ox, Oy = O.pn_matrices(N)
    np.testing.assert_allclose(Mx, Ox, atol=1e-15)
    np.testing.assert_allclose(My, Oy, atol=1e-15)
    code = {(1, 1): 0, (2, 1): 1, (1, 2): 2, (2, 2): 3}
    assert list(grid) == [code[g] for g in O.assign_grids(Ox, Oy)]
    assert list(order) == list(O.moment_orders(N))
    assert abs(lam - O.lambda_max(Ox)) <= 1e-13


@pytest.mark.parametrize("N", [1, 4, 9, 39])
def test_host_slab_matrices_match_oracle(capi, N):
    Mx, My, grid, order, lam = capi.host_matrices(capi.SLAB, N)
    np.testing.assert_array_equal(Mx, O.slab_matrix(N))
    assert not My.any()
    assert list(grid) == [l % 2 for l in range(N + 1)]
    assert abs(lam - O.lambda_max(O.slab_matrix(N))) <= 1e-13


def test_host_expm1div_matches_oracle(capi):
    c = np.concatenate([-np.logspace(-10, 2, 200), np.logspace(-10, 2, 200), [0.0, 2e-4, -2e-4]])
    np.testing.assert_allclose(capi.host_expm1div(c), O.expm1div(c), rtol=5e-16, atol=0)  # libm ulps


def test_host_matrices_reject_bad_order(capi):
    with pytest.raises(capi.StarmapError):
        capi.host_matrices(capi.PN2D, 64)


def test_create_without_gpu_fails_cleanly(capi):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(capi.StarmapError) as ei:
        capi.Stepper(N=3, ax=(0, 1, 0, 1), n=(8, 8))
    assert ei.value.code == capi.E_CUDA


@pytest.mark.parametrize("N", [8, 39])
def test_grid_placement_follows_kind_and_parity(capi, N):
    """Section 4.1: R_l^m with even l on G11, odd l on G21; I_l^m with odd l
    on G12, even l on G22 -- the placement the closure kernels are unrolled
    over (the first 45 components of any P_N with N >= 8)."""
    _, _, grid, order, _ = capi.host_matrices(capi.PN2D, N)
    kinds = [k for (k, _, _) in O.real_moments(N)]
    for j in range(len(kinds)):
        l = order[j]
        want = (0 if l % 2 == 0 else 1) if kinds[j] == "R" else (2 if l % 2 == 1 else 3)
        assert grid[j] == want, j


def test_binding_declares_every_header_function(capi):
    """The binding gives every function of include/starmap.h a ctypes
    signature, and declares none the header lacks."""
    import re
    src = open(os.path.join(ROOT, "paper_1211_2205_gb300", "capi.py")).read()
    declared = set(re.findall(r'"(starmap_[a-z0-9_]+)": \(', src))
    assert declared == set(capi.exported_functions())


def test_health_verdict(capi):
    """The health check's decision: the L2 norm may reach growth * (start +
    t * |q|) and not beyond; a NaN or Inf anywhere is non-finite."""
    v = capi.health_verdict
    assert v(1.0, 1.0, 0.0, 0.0, 1.0) == capi.OK
    assert v(1.0, 1.05, 0.0, 0.0, 1.05) == capi.OK
    assert v(1.0, 1.0500001, 0.0, 0.0, 1.05) == capi.E_GROWTH
    assert v(2.0, 2.0 + 0.5 * 3.0, 0.5, 3.0, 1.0) == capi.OK          # the source's share
    assert v(2.0, 2.0 + 0.5 * 3.0 + 1e-9, 0.5, 3.0, 1.0) == capi.E_GROWTH
    assert v(1.0, 0.2, 1.0, 0.0, 1.05) == capi.OK                      # decay is always fine
    assert v(1.0, float("nan"), 0.1, 0.0, 1.05) == capi.E_NONFINITE
    assert v(1.0, float("inf"), 0.1, 0.0, 1.05) == capi.E_NONFINITE
    assert v(1.0, 1.0, 0.1, 0.0, 1.05, 3) == capi.E_NONFINITE
