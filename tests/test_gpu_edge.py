"""Edge cases of the GPU path against the FP64 oracle: grids of one to a few
points (a single tile, mostly outside the grid; the node grids of an
extrapolation axis one point longer), zero steps, and the homogeneous state
whose exact evolution is the relaxation ODE of every moment."""
import math

import numpy as np
import pytest

from helpers import assert_parity, check_dt, gpu_run, oracle_run
from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi, inputs
from test_gpu_parity import _random_problem

pytestmark = pytest.mark.gpu

BCS = [("periodic", "periodic"), ("extrapolation", "extrapolation"), ("periodic", "extrapolation")]


@pytest.mark.parametrize("kernel,precision,tol", [("gather", "fp64", 1e-12), ("tiled_tall", "fp32", 1e-5),
                                                  ("tiled_short", "fp32", 1e-5)])
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [(1, 1), (2, 1), (1, 3), (3, 2)])
def test_tiny_grids_match_oracle(n, bc, kernel, precision, tol):
    p = _random_problem(3, n, bc, precision, 900 + 7 * n[0] + n[1], 6)
    for sched in ("literal", "merged"):
        s, got = gpu_run(p, schedule=sched, kernel=kernel)
        o, ref = oracle_run(p, s)
        s.close()
        assert_parity(got, ref, tol, precision, sched)


@pytest.mark.parametrize("kernel,precision", [("gather", "fp64"), ("tiled", "fp32")])
def test_zero_steps_leave_the_state(kernel, precision):
    p = _random_problem(5, (20, 13), ("periodic", "extrapolation"), precision, 71, 0)
    s = capi.Stepper.from_problem(p, kernel=kernel)
    before = [s.moments(j) for j in range(s.ncomp)]
    s.step(0)
    assert s.steps_done == 0 and s.time == 0.0
    for j in range(s.ncomp):
        assert np.array_equal(s.moments(j), before[j])
    s.advance_to(0.0)
    for j in range(s.ncomp):
        assert np.array_equal(s.output(j), before[j])
    s.close()


@pytest.mark.parametrize("kernel,precision,tol", [("gather", "fp64", 1e-13), ("tiled", "fp32", 2e-6)])
def test_homogeneous_state_follows_the_relaxation_ode(kernel, precision, tol):
    """Constant state and medium on a periodic grid: no differences, so each
    moment follows u' = -c_l u + q exactly (section 2, eq. sub_step_solution):
    the GPU against the closed form directly, not through the oracle."""
    N, sa, s0 = 6, 0.8, 1.7
    ncomp = (N + 1) * (N + 2) // 2
    rng = inputs.SplitMix64(43)
    u0 = rng.uniforms(ncomp) * 2 - 1
    q = {0: 0.9, 2: -0.4, 7: 0.25}
    const = lambda v: (lambda t, x, y: v + 0 * x)  # noqa: E731
    p = inputs.Problem(name="homogeneous", N=N, ax=(0.0, 1.0, 0.0, 1.0), n=(70, 23), bc=("periodic", "periodic"),
                       precision=precision, sigma_a=const(sa), sigma_s0=const(s0),
                       sources=[(j, const(v)) for j, v in q.items()],
                       ic=[(j, const(u0[j])) for j in range(ncomp)], nsteps=9)
    for sched in ("literal", "merged"):
        s, got = gpu_run(p, schedule=sched, kernel=kernel)
        t = p.nsteps * check_dt(s, p)
        order = O.moment_orders(N)
        for j in range(ncomp):
            c = sa if order[j] == 0 else sa + s0
            e = math.exp(-c * t)
            want = e * u0[j] + q.get(j, 0.0) * (1.0 - e) / c
            assert np.max(np.abs(got[j] - want)) <= tol * max(1.0, abs(want)), (sched, j)
        s.close()


@pytest.mark.parametrize("kernel,precision", [("gather", "fp64"), ("tiled_tall", "fp32"), ("tiled_short", "fp32")])
@pytest.mark.parametrize("schedule", ["literal", "merged"])
def test_finite_speed_gives_exact_zeros(kernel, precision, schedule):
    """A source in one cell and a zero initial state: information moves at
    most two cells per step (odd half, even pair, odd half), so after 6 steps
    every moment is exactly 0 further than 13 cells from the source (one
    more for the node grids) -- no halo, ghost or out-of-range box value may
    leak in.  Scaling the source scales the result (linearity)."""
    n = 40
    cell = 1.0 / n

    def problem(alpha):
        box = lambda t, x, y: alpha * ((np.abs(x - 0.5 - 0.5 * cell) < 0.4 * cell) &  # noqa: E731
                                       (np.abs(y - 0.5 - 0.5 * cell) < 0.4 * cell)).astype(float)
        return inputs.Problem(name="point", N=3, ax=(0.0, 1.0, 0.0, 1.0), n=(n, n), bc=("extrapolation", "periodic"),
                              precision=precision, sigma_a=lambda t, x, y: 0 * x,
                              sigma_s0=lambda t, x, y: 0.5 + 0 * x, sources=[(0, box)], ic=[], nsteps=6)

    s, got = gpu_run(problem(1.0), schedule=schedule, kernel=kernel)
    s.close()
    s2, scaled = gpu_run(problem(-3.5), schedule=schedule, kernel=kernel)
    s2.close()
    assert got[0][n // 2, n // 2] != 0
    jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")   # (y, x) like the moments
    far = np.maximum(np.abs(ii - n // 2), np.abs(jj - n // 2)) > 14
    tol = 1e-14 if precision == "fp64" else 2e-6
    for j, (u, v) in enumerate(zip(got, scaled)):
        assert np.all(u[far[:u.shape[0], :u.shape[1]]] == 0.0), j
        scale = float(np.max(np.abs(u))) + 1e-300
        assert np.max(np.abs(v + 3.5 * u)) <= tol * 3.5 * scale, j
