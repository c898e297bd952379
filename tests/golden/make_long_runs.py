"""Writes the stored FP64 oracle results of the two full-length runs used by
``tests/test_gpu_long_runs.py``.  It calls only the oracle and the seeded
input module; nothing here touches the CUDA library.

Runs (the workloads' own run lengths):

* ``long_checkerboard_p13.npz``: the P_13 checkerboard of section 6.3 at
  512 x 512 on [0,7]^2 with extrapolation boundaries, stepped to t = 3.2
  (462 steps of the fixed step size, output interpolated linearly in time
  as in section 5.8);
* ``long_random_p39_256.npz``: P_39 on the random scattering medium, 256 x
  256 periodic on [-1,1]^2, 200 steps.

Each file keeps, besides the step size and step counts,
* R_0^0 on its whole grid at the final time;
* every component on the sub-lattice [OFF::STRIDE, OFF::STRIDE] of its own
  grid array (indexed [iy, ix]) at the final time;
* every component on a coarser sub-lattice at intermediate step counts,
  for the error-against-run-length curve;
* every component's L2 norm over its whole grid at the final time.

Usage: ``python tests/golden/make_long_runs.py [p13|p39 ...]`` (about 20
minutes per run on one core).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pn_oracle as O                     # noqa: E402
from paper_1211_2205_gb300 import inputs              # noqa: E402

OFF, STRIDE = 3, 16            # final-time sub-lattice
SNAP_OFF, SNAP_STRIDE = 7, 32  # intermediate sub-lattices


def _sub(u, off, stride):
    return np.ascontiguousarray(u.T[off::stride, off::stride])   # [iy, ix]


def _run(o, snap_steps, final, t_final=None):
    """Step the oracle, keeping the coarse sub-lattice at each snapshot step;
    return (snapshots, final list of [iy, ix] arrays)."""
    snaps = {}
    for k in snap_steps:
        o.run(k - o.nsteps_done)
        snaps[k] = [_sub(u, SNAP_OFF, SNAP_STRIDE) for u in o.U]
        print(f"  step {k}  t={o.t:.6f}", flush=True)
    if t_final is not None:
        U = o.run_to(t_final)
    else:
        o.run(final - o.nsteps_done)
        U = o.U
    return snaps, [u.T.copy() for u in U]


def _save(path, o, snaps, final_u, extra):
    data = dict(dt=np.float64(o.dt), steps_done=np.int64(o.nsteps_done),
                r00=final_u[0], off=np.int64(OFF), stride=np.int64(STRIDE),
                snap_off=np.int64(SNAP_OFF), snap_stride=np.int64(SNAP_STRIDE),
                norms=np.array([np.sqrt(np.sum(u * u)) for u in final_u]),
                snap_steps=np.array(sorted(snaps), dtype=np.int64), **extra)
    for j, u in enumerate(final_u):
        data[f"c{j}"] = np.ascontiguousarray(u[OFF::STRIDE, OFF::STRIDE])
    for k, us in snaps.items():
        for j, u in enumerate(us):
            data[f"s{k}_{j}"] = u
    np.savez_compressed(path, **data)


def make_p13():
    p = inputs.checkerboard_p13()                    # 512^2, to t = 3.2
    o = O.solver_from_problem(p)
    t0 = time.time()
    snaps, final_u = _run(o, [58, 116, 231], None, t_final=p.t_final)
    print(f"p13: {o.nsteps_done} steps in {time.time() - t0:.0f} s", flush=True)
    _save(os.path.join(HERE, "long_checkerboard_p13.npz"), o, snaps, final_u,
          dict(t_final=np.float64(p.t_final)))


def make_p39():
    p = inputs.random_p39(n=256)                     # 200 steps
    o = O.solver_from_problem(p)
    t0 = time.time()
    snaps, final_u = _run(o, [25, 50, 100], p.nsteps)
    print(f"p39: {o.nsteps_done} steps in {time.time() - t0:.0f} s", flush=True)
    _save(os.path.join(HERE, "long_random_p39_256.npz"), o, snaps, final_u,
          dict(t_final=np.float64(o.t)))


if __name__ == "__main__":
    which = sys.argv[1:] or ["p13", "p39"]
    for w in which:
        {"p13": make_p13, "p39": make_p39}[w]()
