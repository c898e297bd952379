"""GPU parity of the tiled (TMA-staged, order-streamed) FP32 kernel against
the FP64 oracle (rel-L2 <= 1e-5) and against the gather kernel."""
import math

import numpy as np
import pytest

from helpers import assert_parity, check_dt, gpu_run, oracle_run, rel_l2
from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi, inputs
from test_gpu_parity import _random_problem

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.mark.parametrize("kernel", ["tiled_tall", "tiled_short"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 13])
@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("extrapolation", "extrapolation"),
                                ("periodic", "extrapolation"), ("extrapolation", "periodic")])
def test_tiled_vs_oracle_ragged(N, bc, kernel):
    """70 x 45 grid: two 64-wide tile columns (the second ragged) and 5 or
    9 tile rows (the last ragged), every boundary combination, both tile
    heights."""
    p = _random_problem(N, (70, 45), bc, "fp32", 300 + N, 7)
    for sched in ("literal", "merged"):
        s, got = gpu_run(p, schedule=sched, kernel=kernel)
        assert s.kernel == "tiled" and s.tile_rows == (10 if kernel == "tiled_tall" else 5)
        o, ref = oracle_run(p, s)
        assert_parity(got, ref, FP32_TOL, "fp32", sched)


@pytest.mark.parametrize("N", [3, 9, 22])
def test_tile_heights_agree(N):
    """Both tile heights compute the same arithmetic per point: bit for bit."""
    p = _random_problem(N, (83, 37), ("periodic", "extrapolation"), "fp32", 500 + N, 5)
    a, ga = gpu_run(p, kernel="tiled_tall", schedule="merged")
    b, gb = gpu_run(p, kernel="tiled_short", schedule="merged")
    for x, y in zip(ga, gb):
        assert np.array_equal(x, y)


def test_tiled_anisotropic():
    p = _random_problem(6, (41, 33), ("extrapolation", "periodic"), "fp32", 17, 6, aniso=True)
    s, got = gpu_run(p, kernel="tiled")
    o, ref = oracle_run(p, s)
    assert_parity(got, ref, FP32_TOL, "fp32")


def test_tiled_matches_gather():
    p = _random_problem(9, (64, 40), ("periodic", "extrapolation"), "fp32", 23, 10)
    a, ga = gpu_run(p, kernel="tiled", schedule="merged")
    b, gb = gpu_run(p, kernel="gather", schedule="merged")
    assert rel_l2(ga, gb) <= 2e-6


def test_tiled_checkerboard_to_time():
    """P_13 checkerboard, 72 x 72, interpolated output at t = 0.8."""
    p = inputs.checkerboard_p13(n=72, t_final=0.8, precision="fp32")
    s, got = gpu_run(p, t_final=0.8, kernel="tiled", schedule="merged")
    o, ref = oracle_run(p, s, t_final=0.8)
    assert_parity(got, ref, FP32_TOL, "fp32")


def test_tiled_large_order():
    """P_39 on a 40 x 36 periodic grid (all 820 moments, several tiles)."""
    p = _random_problem(39, (40, 36), ("periodic", "periodic"), "fp32", 39, 3)
    s, got = gpu_run(p, kernel="tiled", schedule="merged")
    o, ref = oracle_run(p, s)
    assert_parity(got, ref, FP32_TOL, "fp32")


def test_tiled_mass_conservation_fp32():
    p = _random_problem(7, (64, 64), ("periodic", "periodic"), "fp32", 55, 1)
    p.sigma_a = lambda t, x, y: 0 * x
    p.sources = []
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    m0, _, _ = s.diagnostics()
    s.step(50)
    m1, _, bad = s.diagnostics()
    assert bad == 0
    assert abs(m1 - m0) <= 1e-5 * abs(m0)


def _window_problem(p, i0, j0, cells):
    """Sub-problem on cells x cells cells starting at cell (i0, j0) of p,
    same spacing and material, periodic wrap (valid in the window interior
    while the wrap error has not travelled in)."""
    x0, x1, y0, y1 = p.ax
    hx = (x1 - x0) / p.n[0]
    hy = (y1 - y0) / p.n[1]
    ax = (x0 + i0 * hx, x0 + (i0 + cells) * hx, y0 + j0 * hy, y0 + (j0 + cells) * hy)
    return inputs.Problem(**{**p.__dict__, "ax": ax, "n": (cells, cells), "bc": ("periodic", "periodic")})


@pytest.mark.parametrize("nsteps", [4])
def test_full_size_random_p39_sampled(nsteps):
    """The bench configuration (P_39, 1024 x 1024, FP32, merged schedule,
    tiled kernel): a 16 x 16 window of the result (all 820 moments) against
    the oracle run on the window plus a halo of 1.5 cells per step."""
    p = inputs.random_p39()
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    s.step(nsteps)
    halo = int(math.ceil(1.5 * nsteps)) + 3
    w = 16
    i0, j0 = 600 - halo, 300 - halo            # window cell origin (includes the Gaussian's tail)
    sub = _window_problem(p, i0, j0, w + 2 * halo)
    o = O.solver_from_problem(sub, dt=check_dt(s, p))
    o.run(nsteps)
    got, ref = [], []
    for j in range(s.ncomp):
        # on every periodic grid, window point k is point i0 + k of the full grid
        got.append(s.moments_window(j, i0 + halo, j0 + halo, w, w))
        sub_u = o.U[j].T                       # (ny, nx) on the window grid
        ref.append(sub_u[halo: halo + w, halo: halo + w])
    assert_parity(got, ref, FP32_TOL, "fp32")


def test_full_size_random_p39_sampled_across_periodic_edge():
    """The bench configuration again, with the sampled window straddling the
    periodic x boundary at mid height (the boundary copies refreshed after
    every pass at full size): the window sub-problem continues past x = 1
    with its fields evaluated at the wrapped points; the pulse's tail there
    (~1e-22) is well inside FP32's normal range."""
    p = inputs.random_p39()
    nsteps = 4
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    s.step(nsteps)
    halo = int(math.ceil(1.5 * nsteps)) + 3
    w = 16
    i0, j0 = p.n[0] - w // 2 - halo, p.n[1] // 2 - halo
    x0, x1, y0, y1 = p.ax

    def wrapped(f):
        # f at the point of the periodic domain that (x, y) stands for
        return lambda t, x, y: f(t, x0 + np.mod(x - x0, x1 - x0), y0 + np.mod(y - y0, y1 - y0))

    sub = _window_problem(p, i0, j0, w + 2 * halo)
    sub = inputs.Problem(**{**sub.__dict__, "sigma_a": wrapped(p.sigma_a), "sigma_s0": wrapped(p.sigma_s0),
                            "ic": [(k, wrapped(f)) for k, f in p.ic]})
    o = O.solver_from_problem(sub, dt=check_dt(s, p))
    o.run(nsteps)
    xa = i0 + halo                          # first window column on the full grid
    left = p.n[0] - xa                      # columns before the wrap
    got, ref = [], []
    for j in range(s.ncomp):
        a = s.moments_window(j, xa, j0 + halo, left, w)
        b = s.moments_window(j, 0, j0 + halo, w - left, w)
        got.append(np.concatenate([a, b], axis=1))
        ref.append(o.U[j].T[halo: halo + w, halo: halo + w])
    assert min(np.abs(r).max() for r in ref[:1]) > 1e-30
    assert_parity(got, ref, FP32_TOL, "fp32")


def test_state_beyond_32bit_offsets():
    """P_39 FP32 on 3300 x 3300: every grid holds more than 2^31 values, so
    the highest components of G11, G21 and G12 start beyond 32-bit element
    offsets from their grid's base (36 GB of state).  Each component from
    local index 186 up gets its own bump next to the bench pulse; a 16 x 16
    window of all 820 moments after 2 steps against the oracle on the window
    plus a halo, and the high components on their own."""
    n, nsteps = 3300, 2
    p = inputs.random_p39(n=n, nsteps=nsteps)
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    assert s.kernel == "tiled"
    assert s.state_bytes() // 4 > 4 * 2 ** 31            # more than 2^31 values per grid on average
    h = (p.ax[1] - p.ax[0]) / n
    halo = int(math.ceil(1.5 * nsteps)) + 3
    w = 16
    i0, j0 = n // 2 + 200 - halo, n // 2 - 100 - halo
    xc, yc = p.ax[0] + (i0 + halo + w / 2) * h, p.ax[2] + (j0 + halo + w / 2) * h
    rng = inputs.SplitMix64(3300)
    seen, high, bumps = [0, 0, 0, 0], [], []
    for j in range(s.ncomp):
        g = s.moment_info(j)["grid"]
        if seen[g] >= 186:
            c = rng.uniforms(3)
            sd = (4 + 4 * c[2]) * h
            f = inputs.gaussian_std(xc + (c[0] - 0.5) * 8 * h, yc + (c[1] - 0.5) * 8 * h, sd,
                                    mass=(-1) ** j * 2 * math.pi * sd * sd)
            X, Y = s.grid_coords(g)
            s.set_moment(j, f(0.0, X, Y))
            high.append(j)
            bumps.append((j, f))
        seen[g] += 1
    assert len(high) >= 60
    s.step(nsteps)
    sub = _window_problem(p, i0, j0, w + 2 * halo)
    sub = inputs.Problem(**{**sub.__dict__, "ic": list(p.ic) + bumps})
    o = O.solver_from_problem(sub, dt=check_dt(s, p))
    o.run(nsteps)
    got = [s.moments_window(j, i0 + halo, j0 + halo, w, w) for j in range(s.ncomp)]
    ref = [o.U[j].T[halo: halo + w, halo: halo + w] for j in range(s.ncomp)]
    s.close()
    assert min(float(np.abs(ref[j]).max()) for j in high) > 1e-3
    assert_parity(got, ref, FP32_TOL, "fp32")
    assert_parity([got[j] for j in high], [ref[j] for j in high], FP32_TOL, "fp32")


def test_full_size_checkerboard_p13_sampled():
    """The P_13 checkerboard workload at full size (512 x 512, FP32,
    extrapolation boundaries, source block, tiled kernel, merged schedule):
    a 16 x 16 window across the source block's edge at x = 4 against the
    oracle on the window plus a halo.  The window problem wraps
    periodically, so on a grid with nodes along an axis its node k lies
    between full cells i0 + k and i0 + k + 1, which is node i0 + k + 1 of
    the full grid (extrapolation: node m lies between cells m - 1 and m)."""
    p = inputs.checkerboard_p13()
    nsteps = 4
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    s.step(nsteps)
    halo = int(math.ceil(1.5 * nsteps)) + 3
    w = 16
    i0, j0 = 285 - halo, 250 - halo
    sub = _window_problem(p, i0, j0, w + 2 * halo)
    o = O.solver_from_problem(sub, dt=check_dt(s, p))
    o.run(nsteps)
    got, ref = [], []
    for j in range(s.ncomp):
        g = s.moment_info(j)["grid"]
        xo = i0 + halo + (1 if g & 1 else 0)
        yo = j0 + halo + (1 if g & 2 else 0)
        got.append(s.moments_window(j, xo, yo, w, w))
        ref.append(o.U[j].T[halo: halo + w, halo: halo + w])
    assert np.abs(ref[0]).max() > 1e-3
    assert_parity(got, ref, FP32_TOL, "fp32")


@pytest.mark.parametrize("kernel", ["auto", "tiled"])
def test_highest_orders_run_on_short_tiles(kernel):
    """At N = 61 the partial sums and tables of the 10-row tiles leave no
    room for a ring: kernel "auto" and "tiled" run the 5-row tiles at one
    CTA per SM (and match the oracle), an explicit "tiled_tall" is refused."""
    p = inputs.Problem(name="p61", N=61, ax=(0.0, 1.0, 0.0, 1.0), n=(12, 10), bc=("periodic", "extrapolation"),
                       precision="fp32", sigma_a=lambda t, x, y: 0.3 + 0 * x,
                       sigma_s0=lambda t, x, y: 1.0 + 0.5 * np.sin(6 * x) * np.cos(4 * y),
                       ic=[(0, inputs.gaussian_std(0.5, 0.45, 0.15))], nsteps=2)
    s = capi.Stepper.from_problem(p, schedule="merged", kernel=kernel)
    assert s.kernel == "tiled" and s.tile_rows == 5
    s.step(2)
    got = [s.moments(j) for j in range(s.ncomp)]
    o, ref = oracle_run(p, s, nsteps=2)
    assert_parity(got, ref, FP32_TOL, "fp32")
    with pytest.raises(capi.StarmapError) as e:
        capi.Stepper.from_problem(p, kernel="tiled_tall")
    assert e.value.code == capi.E_UNSUPPORTED
