"""Shared helpers of the GPU parity tests: run a Problem through the C ABI
and through the oracle on the same seeded inputs, and compare."""
import math

import numpy as np

from oracle import pn_oracle as O
from paper_1211_2205_gb300 import capi


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


def oracle_run(problem, dt, nsteps=None, t_final=None, **over):
    """Run the oracle with the given dt; returns (solver, list of (ny, nx))."""
    o = O.solver_from_problem(problem, dt=dt, **over)
    if t_final is not None:
        U = o.run_to(t_final)
    else:
        o.run(problem.nsteps if nsteps is None else nsteps)
        U = o.U
    return o, [u.T.copy() for u in U]


def rel_l2(got, ref):
    num = sum(float(np.sum((np.asarray(g, dtype=np.float64) - r) ** 2)) for g, r in zip(got, ref))
    den = sum(float(np.sum(r ** 2)) for r in ref)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)
