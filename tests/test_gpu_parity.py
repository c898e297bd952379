"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs.  Bars: rel-L2 over all moments <= 1e-12 in FP64 and
<= 1e-5 in FP32 (the tolerances of the FP64/FP32 precision policy)."""
import math

import numpy as np
import pytest

from helpers import assert_parity, gpu_run, oracle_run, rel_l2
from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def _random_problem(N, n, bc, precision, seed, nsteps, system="pn2d", aniso=False):
    ax = (-0.3, 1.2, 0.1, 1.4)
    rng = inputs.SplitMix64(seed)
    sa = inputs.piecewise_blocks(rng, 5, 0.0, 3.0, ax)
    ss = inputs.smooth_log_field(seed + 1, 6, -1.0, 1.0, ax)
    ncomp = (N + 1) * (N + 2) // 2 if system == "pn2d" else N + 1
    ic = []
    for j in range(ncomp):
        c = rng.uniforms(3)
        ic.append((j, inputs.gaussian_std(ax[0] + 0.3 + c[0], ax[2] + 0.3 + c[1], 0.15 + 0.1 * c[2], mass=(-1) ** j)))
    src = [(0, inputs.gaussian_std(0.4, 0.7, 0.1))]
    if ncomp > 2:
        src.append((2, inputs.gaussian_std(0.6, 0.5, 0.2, mass=0.3)))
    return inputs.Problem(name="random", N=N, ax=ax, n=n, bc=bc, precision=precision, system=system,
                          sigma_a=sa, sigma_s0=ss, sources=src, ic=ic, nsteps=nsteps,
                          sigma_sl_factor=[0.7 ** l for l in range(N + 1)] if aniso else None)


@pytest.mark.parametrize("schedule", ["literal", "merged"])
def test_gaussian_p5_fp64_full_config(schedule):
    """P_5, FP64, 64x64 periodic, sigma_s0 = 1, Gaussian pulse, 100 steps."""
    p = inputs.gaussian_p5()
    s, got = gpu_run(p, schedule=schedule, kernel="gather")
    o, ref = oracle_run(p, s)
    assert abs(s.dt - 0.0167566) < 1e-6
    assert_parity(got, ref, FP64_TOL, "fp64")


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("extrapolation", "extrapolation"),
                                ("periodic", "extrapolation"), ("extrapolation", "periodic")])
@pytest.mark.parametrize("N", [1, 4, 7])
def test_random_media_fp64_ragged(bc, N):
    """Random media and sources on a 37x29 grid (several 128-wide rows and a
    ragged tail), every boundary combination, FP64."""
    p = _random_problem(N, (37, 29), bc, "fp64", 100 + N, 9)
    for sched in ("literal", "merged"):
        s, got = gpu_run(p, schedule=sched, kernel="gather")
        o, ref = oracle_run(p, s)
        assert_parity(got, ref, FP64_TOL, "fp64", sched)


def test_anisotropic_scattering_fp64():
    p = _random_problem(5, (24, 30), ("extrapolation", "periodic"), "fp64", 7, 8, aniso=True)
    s, got = gpu_run(p, kernel="gather")
    o, ref = oracle_run(p, s)
    assert_parity(got, ref, FP64_TOL, "fp64")


@pytest.mark.parametrize("bc", ["periodic", "extrapolation"])
def test_slab_fp64(bc):
    N = 7
    p = _random_problem(N, (47, 1), (bc, "periodic"), "fp64", 3, 12, system="slab")
    s, got = gpu_run(p, kernel="gather")
    o, ref = oracle_run(p, s)
    assert_parity(got, ref, FP64_TOL, "fp64")


def test_fp32_gather_checkerboard_reduced():
    """P_13 checkerboard on 72x72 (no grid point on a block edge) to t = 0.8,
    FP32 against the FP64 oracle."""
    p = inputs.checkerboard_p13(n=72, t_final=0.8, precision="fp32")
    s, got = gpu_run(p, t_final=0.8, kernel="gather")
    o, ref = oracle_run(p, s, t_final=0.8)
    assert_parity(got, ref, FP32_TOL, "fp32")


def test_advance_to_interpolates():
    p = inputs.gaussian_p5(n=40)
    t_out = 0.37
    s, got = gpu_run(p, t_final=t_out, kernel="gather")
    o, ref = oracle_run(p, s, t_final=t_out)
    assert_parity(got, ref, FP64_TOL, "fp64")
    assert s.time >= t_out and s.time - s.dt < t_out


def test_diagnostics_match_oracle():
    p = _random_problem(4, (33, 31), ("periodic", "extrapolation"), "fp64", 21, 6)
    s, got = gpu_run(p, kernel="gather")
    o, ref = oracle_run(p, s)
    mass, l2, bad = s.diagnostics()
    assert bad == 0
    assert abs(mass - o.mass()) <= 1e-12 * abs(o.l2norm())
    assert abs(l2 - o.l2norm()) <= 1e-12 * o.l2norm()


def test_diagnostics_flag_nonfinite():
    p = inputs.gaussian_p5(n=16, nsteps=1)
    s = capi.Stepper.from_problem(p)
    u = s.moments(3)
    u[2, 5] = np.nan
    s.set_moment(3, u)
    mass, l2, bad = s.diagnostics()
    assert bad == 1


def test_mass_conserved_on_gpu():
    p = _random_problem(6, (40, 36), ("periodic", "periodic"), "fp64", 5, 20)
    p.sigma_a = lambda t, x, y: 0 * x
    p.sources = []
    s = capi.Stepper.from_problem(p, kernel="gather")
    m0, _, _ = s.diagnostics()
    s.step(20)
    m1, _, _ = s.diagnostics()
    assert abs(m1 - m0) <= 1e-13 * abs(m0)


def test_checkpoint_resume_bitwise():
    p = _random_problem(5, (32, 32), ("extrapolation", "periodic"), "fp32", 9, 10)
    a = capi.Stepper.from_problem(p, schedule="merged")
    a.step(10)
    ref = [a.moments(j) for j in range(a.ncomp)]
    b = capi.Stepper.from_problem(p, schedule="merged")
    b.step(4)
    snap = b.get_state()
    c = capi.Stepper.from_problem(p, schedule="merged")
    c.set_state(snap)
    assert c.steps_done == 4 and abs(c.time - b.time) == 0
    c.step(6)
    got = [c.moments(j) for j in range(c.ncomp)]
    # merged schedule: (4 + 6) steps equal 10 steps up to the rounding of the
    # split odd pass; the literal schedule is bitwise
    assert rel_l2(got, ref) <= 1e-6
    d = capi.Stepper.from_problem(p, schedule="literal")
    d.step(4)
    e = capi.Stepper.from_problem(p, schedule="literal")
    e.set_state(d.get_state())
    e.step(6)
    d.step(6)
    for j in range(d.ncomp):
        assert np.array_equal(d.moments(j), e.moments(j))


def test_invalid_arguments_are_errors():
    with pytest.raises(capi.StarmapError) as ei:
        capi.Stepper(N=3, ax=(0, 1, 0, 1), n=(8, 8), cn=0.9)
    assert ei.value.code == capi.E_CFL
    with pytest.raises(capi.StarmapError):
        capi.Stepper(N=0, ax=(0, 1, 0, 1), n=(8, 8))
    s = capi.Stepper(N=3, ax=(0, 1, 0, 1), n=(8, 8))
    with pytest.raises(capi.StarmapError):
        s.set_moment(0, np.zeros(5))
    with pytest.raises(capi.StarmapError):
        s.moments(99)
    with pytest.raises(capi.StarmapError):
        s.output(0)
