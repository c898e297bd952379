"""The spatial split over several GPUs (paper_1211_2205_gb300/slab.py), on
the CPU: the index logic of the slabs, windows and halo segments, and a
world-size-2 run over torch.distributed (gloo) whose ranks step their
windows with the FP64 oracle and swap halos with the module's own
exchange.  On dyadic grids the windows' coordinates, spacings and material
samples are the global ones to the last bit, so the stitched owned rows
must equal the single-domain oracle run bit for bit."""
import math
import os
import socket

import numpy as np
import pytest

from oracle import pn_oracle as O
from paper_1211_2205_gb300 import inputs
from paper_1211_2205_gb300.slab import Y_NODE, SlabPlan, exchange_dist, grid_coordinates, run

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("ny,ranks,k", [(64, 2, 3), (96, 3, 2), (50, 4, 1), (40, 1, 5)])
def test_plan_partitions_rows_and_segments_line_up(periodic, ny, ranks, k):
    p = SlabPlan(ny, periodic, ranks, k)
    for g in range(4):
        owners = np.zeros(p.global_rows(g), dtype=int)
        for r in range(ranks):
            w0, w1 = p.owned(r, g)
            assert 0 <= w0 < w1 <= p.window_rows(r, g)
            for w in range(w0, w1):
                owners[p.global_row(r, w)] += 1
                assert p.owner_of(g, p.global_row(r, w)) == r
            # the halo: H rows beyond the slab on each side, or the domain's edge
            if ranks > 1:
                assert w0 == p.H or (not periodic and p.lo[r] == 0 and w0 == 0)
                # (an extrapolation node grid has one node row more above its cells)
                extra = 1 if Y_NODE[g] and not periodic else 0
                assert p.window_rows(r, g) - w1 == p.H + extra or (not periodic and p.hi[r] == ny)
        assert np.all(owners == 1)                      # every global row owned exactly once
    for r in range(ranks):
        covered = {g: set() for g in range(4)}
        for seg in p.recv_segments(r):
            assert seg.owner != r
            s0, s1 = p.owned(seg.owner, seg.g)
            assert s0 <= seg.src_row and seg.src_row + seg.rows <= s1
            for i in range(seg.rows):
                assert p.global_row(r, seg.row + i) == p.global_row(seg.owner, seg.src_row + i)
                covered[seg.g].add(seg.row + i)
        for g in range(4):
            w0, w1 = p.owned(r, g)
            assert covered[g] == set(range(p.window_rows(r, g))) - set(range(w0, w1))
        sent = [(rr, seg) for rr, seg in p.send_segments(r)]
        assert all(seg.owner == r for _, seg in sent)
    assert sum(len(p.send_segments(r)) for r in range(ranks)) == sum(len(p.recv_segments(r)) for r in range(ranks))


def test_plan_rejects_thin_slabs():
    with pytest.raises(ValueError):
        SlabPlan(20, True, 4, 2)          # 5-row slabs, halo 6


def test_grid_coordinates_follow_the_staggering():
    p = inputs.Problem(name="c", N=1, ax=(0.0, 1.0, -1.0, 1.0), n=(4, 8), bc=("periodic", "extrapolation"))
    X, Y = grid_coordinates(p, 3)
    assert X.shape == (9, 4)                              # node rows 0..8 (extrapolation), node columns 1..4
    assert X[0, 0] == 0.25 and X[0, -1] == 1.0 and Y[0, 0] == -1.0 and Y[-1, 0] == 1.0
    X, Y = grid_coordinates(p, 0)
    assert X[0, 0] == 0.125 and Y[0, 0] == -0.875


# ----------------------------------------------------------------- gloo run
def _problem(periodic_y):
    """P_3 on [0, 0.75] x [0, 1], 24 x 32 cells (dyadic spacing 1/32):
    smooth material, a source, every component with a pulse."""
    ax = (0.0, 0.75, 0.0, 1.0)
    L = ax[3] - ax[2]

    def wrap(f):
        return lambda t, x, y: f(t, x, ax[2] + np.mod(y - ax[2], L))

    sa = wrap(lambda t, x, y: 0.5 + 0.4 * np.sin(2 * math.pi * y) * np.cos(3 * x))
    ss = wrap(lambda t, x, y: 1.0 + 0.5 * np.cos(2 * math.pi * y + x))
    ic = [(j, wrap(inputs.gaussian_std(0.2 + 0.05 * j, 0.3 + 0.04 * j, 0.12, mass=(-1) ** j)))
          for j in range(10)]
    return inputs.Problem(name="slab", N=3, ax=ax, n=(24, 32),
                          bc=("extrapolation", "periodic" if periodic_y else "extrapolation"),
                          sigma_a=sa, sigma_s0=ss, sources=[(0, wrap(inputs.gaussian_std(0.4, 0.6, 0.1)))],
                          ic=ic, nsteps=9)


class OracleEngine:
    """A window stepped by the FP64 oracle; rows as CPU tensors laid out
    [component][row][x] like the library's pack / unpack."""
    dtype = torch.float64
    device = torch.device("cpu")

    def __init__(self, plan, r, problem, dt):
        wp = plan.window_problem(problem, r)
        self.o = O.solver_from_problem(wp, dt=dt)
        self.comps = {g: [] for g in range(4)}
        for j, (gx, gy) in enumerate(self.o.grid):
            self.comps[(gx == 2) + 2 * (gy == 2)].append(j)
        self.plan, self.r = plan, r

    def row_elems(self, g, rows):
        nx = self.o.U[self.comps[g][0]].shape[0] if self.comps[g] else 0
        return len(self.comps[g]) * rows * nx

    def rows(self, g, y0, rows):
        a = np.stack([self.o.U[j][:, y0:y0 + rows].T for j in self.comps[g]])
        return torch.from_numpy(np.ascontiguousarray(a).ravel())

    def set_rows(self, g, y0, rows, buf):
        nx = self.o.U[self.comps[g][0]].shape[0]
        a = buf.numpy().reshape(len(self.comps[g]), rows, nx)
        for c, j in enumerate(self.comps[g]):
            self.o.U[j][:, y0:y0 + rows] = a[c].T

    def step(self, k):
        self.o.run(k)

    def sync(self):
        pass

    def owned(self, j):
        gx, gy = self.o.grid[j]
        w0, w1 = self.plan.owned(self.r, (gx == 2) + 2 * (gy == 2))
        return self.o.U[j].T[w0:w1]


def _rank_main(rank, world, port, periodic, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem(periodic)
        Mx, _, _ = O.system_matrices("pn2d", prob.N)
        dt = O.time_step(Mx, prob.ax, prob.n, prob.cn)
        plan = SlabPlan(prob.n[1], periodic, world, 2)
        eng = OracleEngine(plan, rank, prob, dt)
        moved = run(plan, [eng], prob.nsteps, lambda: exchange_dist(plan, rank, eng))
        owned = [torch.from_numpy(np.ascontiguousarray(eng.owned(j))) for j in range(eng.o.ncomp)]
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(([o.numpy() for o in owned], moved), gathered, dst=0)
        if rank == 0:
            np.save(out_path, np.array(gathered, dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("periodic", [True, False])
def test_two_ranks_over_gloo_equal_the_single_domain_oracle(periodic, tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "owned.npy")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, periodic, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs)
    gathered = np.load(out, allow_pickle=True)
    prob = _problem(periodic)
    ref = O.solver_from_problem(prob)
    ref.run(prob.nsteps)
    moved = [m for _, m in gathered]
    assert all(m > 0 for m in moved)
    for j in range(ref.ncomp):
        stitched = np.concatenate([owned[j] for owned, _ in gathered], axis=0)
        want = ref.U[j].T
        assert stitched.shape == want.shape
        assert np.array_equal(stitched, want), j
