"""Time-dependent material and sources on the GPU (the method freezes them
at each step's midpoint, section 5.5): the manufactured solution of
section 6.1 -- P_3 on [0,1]^2, Sigma_a = t cos(2 pi y), Sigma_sl = 0.9^l,
R_0^0 = e^-t sin^2(2 pi x), every other moment 0 -- stepped through the C
ABI with the data re-sampled at t + dt/2 before every step.  The results
equal the FP64 oracle's (FP64 to 1e-12, FP32 to 1e-5) and converge to the
exact solution at second order."""
import math

import numpy as np
import pytest

from helpers import assert_parity, check_dt
from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


def _exact(t, x, y):
    return math.exp(-t) * np.sin(2 * math.pi * x) ** 2 + 0 * y


def _sigma_a(t, x, y):
    return t * np.cos(2 * math.pi * y) + 0 * x


def mms_problem(n, precision="fp64"):
    """The manufactured problem: the sources make R_0^0 = e^-t sin^2(2 pi x)
    with all other moments zero an exact solution of the P_3 system
    (q_R00 = d_t R00 + c_0 R00, q_R11 = Mx[R11, R00] d_x R00 with
    Mx[R11, R00] = 1/sqrt(3))."""
    q0 = lambda t, x, y: -math.exp(-t) * np.sin(2 * math.pi * x) ** 2 + _sigma_a(t, x, y) * _exact(t, x, y)
    q1 = lambda t, x, y: (1 / math.sqrt(3)) * 2 * math.pi * math.exp(-t) * np.sin(4 * math.pi * x) + 0 * y
    return inputs.Problem(name=f"mms_p3_{n}", N=3, ax=(0.0, 1.0, 0.0, 1.0), n=(n, n), bc=("periodic", "periodic"),
                          cn=0.5, precision=precision, sigma_a=_sigma_a, sigma_s0=lambda t, x, y: 1.0 + 0 * x,
                          sigma_sl_factor=[0.9 ** l for l in range(4)], sources=[(0, q0), (1, q1)],
                          ic=[(0, _exact)], time_dependent=True)


def _run_gpu(p, t_final, kernel="auto"):
    s = capi.Stepper.from_problem(p, kernel=kernel, schedule="literal")
    d = check_dt(s, p)                         # the library's own step rule equals the oracle's
    s.close()
    nsteps = int(math.ceil(t_final / d - 1e-9))
    dt = t_final / nsteps                      # the final time on a step: both sides use this one
    s = capi.Stepper.from_problem(p, kernel=kernel, schedule="literal", dt=dt)
    s.set_time_dependence(p)                   # the library samples at every step's midpoint
    s.step(nsteps)
    out = [s.moments(j) for j in range(s.ncomp)]
    info = [s.moment_info(j) for j in range(s.ncomp)]
    coords = [s.grid_coords(i["grid"]) for i in info]
    s.close()
    return out, coords, dt, nsteps


@pytest.mark.parametrize("precision,kernel,tol", [("fp64", "auto", 1e-12), ("fp32", "tiled", 1e-5)])
def test_time_dependent_matches_oracle(precision, kernel, tol):
    p = mms_problem(24, precision)
    got, _, dt, nsteps = _run_gpu(p, 0.1, kernel)
    o = O.solver_from_problem(p, dt=dt)
    o.run(nsteps)
    ref = [u.T for u in o.U]
    assert_parity(got, ref, tol, precision)


def test_mms_second_order_on_gpu():
    """Observed orders between successive resolutions 32, 64, 128, 256 in
    the L1, L2 and max norms of the error against the exact solution."""
    errs = []
    for n in (32, 64, 128, 256):
        got, coords, _, _ = _run_gpu(mms_problem(n), 0.5)
        e = [u - (_exact(0.5, X, Y) if j == 0 else 0 * X) for j, (u, (X, Y)) in enumerate(zip(got, coords))]
        flat = np.concatenate([v.ravel() for v in e])
        errs.append((np.mean(np.abs(flat)), math.sqrt(np.mean(flat ** 2)), np.max(np.abs(flat))))
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 1.9) and np.all(orders < 2.1), orders


def test_time_dependence_callback_errors_and_off():
    """A failing callback stops the step with E_ARG; with the callback off
    the material and sources stay as last sampled; a merged-schedule
    handle steps time-dependent problems as the literal schedule does."""
    p = mms_problem(16, "fp64")
    s = capi.Stepper.from_problem(p, kernel="gather", schedule="merged")
    s.set_time_dependence(p)
    s.step(3)
    lit = capi.Stepper.from_problem(p, kernel="gather", schedule="literal")
    lit.set_time_dependence(p)
    lit.step(3)
    for j in range(s.ncomp):
        assert np.array_equal(s.moments(j), lit.moments(j))
    bad = inputs.Problem(**{**p.__dict__, "sigma_a": lambda t, x, y: 1 / 0})
    s.set_time_dependence(bad)
    with pytest.raises(capi.StarmapError) as e:
        s.step(1)
    assert e.value.code == capi.E_ARG and s.steps_done == 3
    s.set_time_dependence(None)
    s.step(1)
    assert s.steps_done == 4
