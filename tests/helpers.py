"""Shared helpers of the GPU parity tests: run a Problem through the C ABI
and through the oracle on the same seeded inputs, and compare.

The oracle always computes its own time step (the section 4.5 rule in
``pn_oracle.time_step``); the library's step size is checked against it and
never handed to the oracle.  Where a test deliberately runs two systems at
one common step size (a closure against P_39, windows of a larger grid),
that step size also comes from the oracle (``oracle_dt``)."""
import math

import numpy as np

from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi

# The library computes lambda_max by bisection on a Sturm sequence, the
# oracle with LAPACK's general eigenvalue routine, whose error grows with the
# matrix size (1.7e-14 relative at N = 39, an 820 x 820 matrix); the CPU
# tests hold the two lambda_max to 1e-13.
DT_RTOL = 1e-13

# Unit round-off of the stored precision.
UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}

# Per-component bar: ||g_j - r_j|| <= tol * ||r_j|| + FLOOR_ULPS[p] * u * ||r||,
# with ||r|| the norm of all components together and u the unit round-off.
# The floor lets a component that is tiny (or zero) in exact arithmetic
# carry the rounding noise of its larger neighbours.  FP32: 4 units of the
# whole state's round-off (the parity suite needs at most 0.62).  FP64: the
# two sides' step sizes agree only to DT_RTOL, which moves every component
# by up to ~1e-14 of the state: 64 units (the suite needs at most 31).
FLOOR_ULPS = {"fp32": 4.0, "fp64": 64.0}


def gpu_run(problem, nsteps=None, t_final=None, **over):
    """Run through the C ABI; returns (stepper, list of (ny, nx) arrays)."""
    s = capi.Stepper.from_problem(problem, **over)
    if t_final is not None:
        s.advance_to(t_final)
        out = [s.output(j) for j in range(s.ncomp)]
    else:
        s.step(problem.nsteps if nsteps is None else nsteps)
        out = [s.moments(j) for j in range(s.ncomp)]
    return s, out


def oracle_dt(problem) -> float:
    """The oracle's own step size for ``problem`` (section 4.5 rule)."""
    Mx, _, _ = O.system_matrices(problem.system, problem.N)
    return O.time_step(Mx, problem.ax, problem.n, problem.cn)


def check_dt(s, problem) -> float:
    """Assert that the stepper's step size equals the oracle's; return it."""
    d = oracle_dt(problem)
    assert abs(s.dt - d) <= DT_RTOL * d, (s.dt, d)
    return d


def oracle_run(problem, s=None, nsteps=None, t_final=None, **over):
    """Run the oracle with its own step size (or an explicit common ``dt=``
    from ``over``); when a stepper ``s`` is given, first check that its step
    size equals the oracle's.  Returns (solver, list of (ny, nx) arrays)."""
    o = O.solver_from_problem(problem, **over)
    if s is not None and "dt" not in over:
        assert abs(s.dt - o.dt) <= DT_RTOL * o.dt, (s.dt, o.dt)
    if t_final is not None:
        U = o.run_to(t_final)
    else:
        o.run(problem.nsteps if nsteps is None else nsteps)
        U = o.U
    return o, [u.T.copy() for u in U]


def rel_l2(got, ref):
    """rel-L2 over all components together (pooled)."""
    num = sum(float(np.sum((np.asarray(g, dtype=np.float64) - r) ** 2)) for g, r in zip(got, ref))
    den = sum(float(np.sum(np.asarray(r, dtype=np.float64) ** 2)) for r in ref)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


def component_ratios(got, ref, tol, precision):
    """Per component j: ||g_j - r_j|| / (tol ||r_j|| + FLOOR_ULPS u ||r||);
    every entry must be <= 1."""
    u = UNIT_ROUNDOFF[precision] * FLOOR_ULPS[precision]
    err = np.array([math.sqrt(float(np.sum((np.asarray(g, dtype=np.float64) - r) ** 2)))
                    for g, r in zip(got, ref)])
    nrm = np.array([math.sqrt(float(np.sum(np.asarray(r, dtype=np.float64) ** 2))) for r in ref])
    pooled = math.sqrt(float(np.sum(nrm ** 2)))
    bar = tol * nrm + u * pooled
    return np.where(bar > 0, err / np.where(bar > 0, bar, 1.0), np.where(err > 0, np.inf, 0.0))


def assert_parity(got, ref, tol, precision, what=""):
    """Pooled rel-L2 <= tol, and every component within its own bar (see
    ``component_ratios``).  Returns the pooled rel-L2."""
    r = rel_l2(got, ref)
    assert r <= tol, f"{what} pooled rel-L2 {r:.3e} > {tol:.1e}"
    ratios = component_ratios(got, ref, tol, precision)
    worst = int(np.argmax(ratios))
    assert ratios[worst] <= 1.0, (f"{what} component {worst}: error "
                                  f"{ratios[worst]:.3g} x its bar (pooled rel-L2 {r:.3e})")
    return r
