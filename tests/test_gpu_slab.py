"""The spatial split over several GPUs, emulated on one GPU: each rank's
window is its own library handle and the halo exchange runs through the
C ABI's row pack / unpack (device to device).  Nothing waits on another
handle: the exchange is host-ordered between step calls.  On a dyadic grid
the stitched owned rows equal the single-domain library run bit for bit
(same kernels, same arithmetic per point, the same step calls), and that
run matches the FP64 oracle."""
import math

import numpy as np
import pytest

from helpers import assert_parity, oracle_run
from paper_1211_2205_gb300 import capi, inputs, slab

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _problem(periodic_y, precision, N):
    ax = (-0.5, 0.5, -1.0, 1.0)                   # 64 x 128 cells: spacing 1/64
    L = ax[3] - ax[2]

    def wrap(f):
        return lambda t, x, y: f(t, x, ax[2] + np.mod(y - ax[2], L))

    rng = inputs.SplitMix64(4100 + N)
    ic = []
    for j in range((N + 1) * (N + 2) // 2):
        c = rng.uniforms(3)
        ic.append((j, wrap(inputs.gaussian_std(-0.3 + 0.6 * c[0], -0.7 + 1.4 * c[1], 0.1 + 0.1 * c[2],
                                               mass=(-1) ** j))))
    return inputs.Problem(name="slab", N=N, ax=ax, n=(64, 128),
                          bc=("periodic", "periodic" if periodic_y else "extrapolation"), precision=precision,
                          sigma_a=wrap(lambda t, x, y: 0.3 + 0.2 * np.cos(math.pi * y) * np.sin(3 * x)),
                          sigma_s0=wrap(lambda t, x, y: 1.5 + np.sin(math.pi * y + 2 * x)),
                          sources=[(0, wrap(inputs.gaussian_std(0.1, 0.2, 0.15)))], ic=ic, nsteps=11)


def _grid_of(s):
    return [s.moment_info(j)["grid"] for j in range(s.ncomp)]


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("precision,kernel,N", [("fp64", "gather", 4), ("fp32", "tiled", 7)])
def test_emulated_ranks_equal_the_single_domain_run(periodic, precision, kernel, N):
    p = _problem(periodic, precision, N)
    k, ranks = 3, 3
    ref = capi.Stepper(N=p.N, ax=p.ax, n=p.n, bc=p.bc, precision=precision, kernel=kernel, schedule="merged")
    glob = slab.global_samples(p, _grid_of(ref))
    plan = slab.SlabPlan(p.n[1], periodic, ranks, k)
    engines = [slab.LibraryEngine(plan, r, p, ref.dt, kernel=kernel) for r in range(ranks)]
    for e in engines:
        e.load(glob)
    for g in range(4):
        ref.set_material(g, glob.sigma_a[g], glob.sigma_s0[g])
    for j, q in glob.sources.items():
        ref.set_source(j, q)
    for j, u in glob.ic.items():
        ref.set_moment(j, u)
    moved = slab.run(plan, engines, p.nsteps, lambda: slab.exchange_local(plan, engines))
    assert moved > 0
    done = 0
    while done < p.nsteps:                      # the same step calls as the ranks
        ref.step(min(k, p.nsteps - done))
        done += min(k, p.nsteps - done)
    want = [ref.moments(j) for j in range(ref.ncomp)]
    got = [np.concatenate([e.owned(j) for e in engines], axis=0) for j in range(ref.ncomp)]
    for j in range(ref.ncomp):
        assert got[j].shape == want[j].shape
        assert np.array_equal(got[j], want[j]), j
    # owned-row diagnostics summed over the ranks = the whole grid's
    mass = sum(e.owned_sums()[0] for e in engines) * ref.grid_info(0)[4] * ref.grid_info(0)[5]
    m_ref, _, _ = ref.diagnostics()
    assert mass == pytest.approx(m_ref, rel=1e-12, abs=1e-14)
    # and the single-domain run is the method: against the oracle
    _, oref = oracle_run(p, ref, nsteps=p.nsteps)
    assert_parity(want, oref, 1e-12 if precision == "fp64" else 1e-5, precision)


def test_pack_and_unpack_rows_round_trip():
    p = _problem(True, "fp32", 3)
    s = capi.Stepper.from_problem(p, kernel="tiled")
    K = [0] * 4
    for j in range(s.ncomp):
        K[s.moment_info(j)["grid"]] += 1
    for g in range(4):
        nx, ny, *_ = s.grid_info(g)
        buf = torch.empty(K[g] * 5 * nx, dtype=torch.float32, device="cuda")
        s.pack_rows(g, 7, 5, buf.data_ptr(), buf.numel() * 4)
        s.sync()
        a = buf.cpu().numpy().reshape(K[g], 5, nx)
        comps = [j for j in range(s.ncomp) if s.moment_info(j)["grid"] == g]
        for c, j in enumerate(comps):
            assert np.array_equal(a[c], s.moments(j)[7:12].astype(np.float32))
        buf.mul_(-2.0)
        torch.cuda.synchronize()
        s.unpack_rows(g, ny - 5, 5, buf.data_ptr(), buf.numel() * 4)
        s.sync()
        for c, j in enumerate(comps):
            assert np.array_equal(s.moments(j)[ny - 5:], -2.0 * a[c])
    with pytest.raises(capi.StarmapError) as e:
        s.pack_rows(0, 125, 5, buf.data_ptr(), buf.numel() * 4)
    assert e.value.code == capi.E_ARG
