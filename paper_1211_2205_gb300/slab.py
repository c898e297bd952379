"""Spatial split of one problem over several GPUs: slabs of cell rows in y,
each rank stepping a window of its slab plus a halo, with halo exchanges.

The method is explicit with finite speed: one full step (odd half, even
pair, odd half) moves information by at most two cells (the domain of
dependence of section 4's staggered stencils).  So a rank that holds its
slab plus H >= 2k + 2 rows on each side can run k steps on its own: the
rows near its window's edges go wrong (the window's own boundary copies
stand in for the neighbours' data), but the error travels at most 2k rows
and never reaches the slab.  After the k steps the ranks swap the halo
rows, which their neighbours own, and every rank again holds the exact
state of its window.  One exchange per k steps, of H rows of every
component on each cut face, point to point (NCCL send/recv into local
buffers, unpacked by a device copy), no collective on the data path; the
FP64 diagnostics sum each rank's owned rows (one all-reduce of three
numbers).

Windows are ordinary problems of the library (or of any engine with the
same row interface): the same x extent, the cell rows [lo, hi) of the
global grid in y, the global boundary type in y (periodic windows wrap,
extrapolation windows end at the domain's edge when they reach it), the
global step size, and material, sources and initial data sliced from the
global grid's samples.  Row k of every window grid is global row lo + k
(mod ny when periodic) of the same grid:
    cell rows:                  y = y0 + (lo + k + 1/2) dy
    node rows, periodic:        y = y0 + (lo + k + 1) dy   (global index lo + k mod ny)
    node rows, extrapolation:   y = y0 + (lo + k) dy       (global index lo + k, 0..ny)
Ownership partitions every grid's global rows: rank r owns [a_r, b_r), the
last rank also the top node row of an extrapolation node grid.

This module holds the index logic and the orchestration; the arithmetic
runs in the engines (the library's kernels on the GPU).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import inputs

Y_NODE = (False, False, True, True)        # grid g = G11, G21, G12, G22: rows on nodes?


@dataclasses.dataclass(frozen=True)
class Segment:
    """Rows [row, row + rows) of grid g in the receiver's window, owned by
    rank `owner`, where they are rows [src_row, src_row + rows) of its window."""
    owner: int
    g: int
    row: int
    rows: int
    src_row: int


class SlabPlan:
    """Index logic of the split of ny cell rows over `ranks` slabs with
    `steps` steps between exchanges (halo 2 * steps + 2 rows)."""

    def __init__(self, ny: int, periodic_y: bool, ranks: int, steps: int):
        if ranks < 1 or steps < 1:
            raise ValueError("ranks and steps per exchange must be positive")
        self.ny, self.periodic, self.ranks, self.k = int(ny), bool(periodic_y), int(ranks), int(steps)
        self.H = 2 * self.k + 2
        self.a = [r * self.ny // ranks for r in range(ranks)]
        self.b = [(r + 1) * self.ny // ranks for r in range(ranks)]
        if ranks > 1 and min(b - a for a, b in zip(self.a, self.b)) < self.H:
            raise ValueError(f"slabs of fewer than {self.H} rows: use fewer ranks or fewer steps per exchange")
        self.lo, self.hi = [], []
        for r in range(ranks):
            if ranks == 1:
                lo, hi = 0, self.ny
            elif self.periodic:
                lo, hi = self.a[r] - self.H, self.b[r] + self.H
            else:
                lo, hi = max(self.a[r] - self.H, 0), min(self.b[r] + self.H, self.ny)
            self.lo.append(lo)
            self.hi.append(hi)

    # -- sizes and ownership --------------------------------------------
    def global_rows(self, g: int) -> int:
        return self.ny + (1 if Y_NODE[g] and not self.periodic else 0)

    def window_cells(self, r: int) -> int:
        return self.hi[r] - self.lo[r]

    def window_rows(self, r: int, g: int) -> int:
        return self.window_cells(r) + (1 if Y_NODE[g] and not self.periodic else 0)

    def owner_of(self, g: int, grow: int) -> int:
        """Rank owning global row `grow` (already wrapped) of grid g."""
        if grow == self.ny:                    # top node row of an extrapolation node grid
            return self.ranks - 1
        for r in range(self.ranks):
            if self.a[r] <= grow < self.b[r]:
                return r
        raise IndexError(grow)

    def owned(self, r: int, g: int) -> Tuple[int, int]:
        """Window rows [w0, w1) of rank r that it owns in grid g."""
        a, b = self.a[r], self.b[r]
        if Y_NODE[g] and not self.periodic and r == self.ranks - 1:
            b = self.ny + 1
        return a - self.lo[r], b - self.lo[r]

    def global_row(self, r: int, wrow: int) -> int:
        v = self.lo[r] + wrow
        return v % self.ny if self.periodic else v

    # -- the exchange ------------------------------------------------------
    def recv_segments(self, r: int) -> List[Segment]:
        """The rows of rank r's window that other ranks own, as contiguous
        runs per owner, grid by grid in increasing window row."""
        out = []
        if self.ranks == 1:
            return out
        for g in range(4):
            w0, w1 = self.owned(r, g)
            runs = []
            for w in list(range(0, w0)) + list(range(w1, self.window_rows(r, g))):
                grow = self.global_row(r, w)
                s = self.owner_of(g, grow)
                src = grow - self.lo[s]                 # inside the rows s owns
                if runs and runs[-1][0] == s and runs[-1][1] + runs[-1][2] == w and runs[-1][3] + runs[-1][2] == src:
                    runs[-1][2] += 1
                else:
                    runs.append([s, w, 1, src])
            out += [Segment(owner=s, g=g, row=w, rows=n, src_row=src) for s, w, n, src in runs]
        return out

    def send_segments(self, s: int) -> List[Tuple[int, Segment]]:
        """What rank s sends: (receiver, segment) in the order the receiver
        lists them."""
        return [(r, seg) for r in range(self.ranks) for seg in self.recv_segments(r) if seg.owner == s]

    def window_problem(self, problem: inputs.Problem, r: int) -> inputs.Problem:
        """Rank r's window as a problem: the global problem with the
        window's y extent (`LibraryEngine.load` uploads sliced global
        samples, not the field functions)."""
        x0, x1, y0, y1 = problem.ax
        dy = (y1 - y0) / problem.n[1]
        ax = (x0, x1, y0 + self.lo[r] * dy, y0 + self.hi[r] * dy)
        return inputs.Problem(**{**problem.__dict__, "ax": ax, "n": (problem.n[0], self.window_cells(r))})

    def slice_rows(self, r: int, g: int, global_array: np.ndarray) -> np.ndarray:
        """Rows of rank r's window cut from an array [row][x] of grid g's
        global samples (wrapped when periodic)."""
        idx = [self.global_row(r, w) for w in range(self.window_rows(r, g))]
        return np.ascontiguousarray(global_array[idx])


def exchange_local(plan: SlabPlan, engines: Sequence) -> int:
    """Every rank's halo from its owners, all ranks in this process (the
    emulation of a multi-GPU run on one device); returns bytes moved."""
    moved = 0
    for r in range(plan.ranks):
        for seg in plan.recv_segments(r):
            buf = engines[seg.owner].rows(seg.g, seg.src_row, seg.rows)
            engines[seg.owner].sync()            # packed on the owner's stream
            engines[r].set_rows(seg.g, seg.row, seg.rows, buf)
            engines[r].sync()                    # unpacked before the buffer is released
            moved += buf.numel() * buf.element_size()
    return moved


def exchange_dist(plan: SlabPlan, rank: int, engine, group=None) -> int:
    """This rank's part of the halo exchange over torch.distributed:
    one message per neighbour pair and direction (the segments of every
    grid concatenated), point to point; returns bytes received."""
    import torch
    import torch.distributed as dist
    sends: Dict[int, list] = {}
    for r, seg in plan.send_segments(rank):
        sends.setdefault(r, []).append(engine.rows(seg.g, seg.src_row, seg.rows))
    recv_segs: Dict[int, List[Segment]] = {}
    for seg in plan.recv_segments(rank):
        recv_segs.setdefault(seg.owner, []).append(seg)
    engine.sync()
    ops, bufs = [], {}
    for s, segs in sorted(recv_segs.items()):
        n = sum(engine.row_elems(seg.g, seg.rows) for seg in segs)
        bufs[s] = torch.empty(n, dtype=engine.dtype, device=engine.device)
        ops.append(dist.P2POp(dist.irecv, bufs[s], s, group))
    for r, parts in sorted(sends.items()):
        ops.append(dist.P2POp(dist.isend, torch.cat(parts), r, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    if engine.device.type == "cuda":
        torch.cuda.synchronize()                 # received on torch's streams, unpacked on the engine's
    got = 0
    for s, segs in sorted(recv_segs.items()):
        off = 0
        for seg in segs:
            n = engine.row_elems(seg.g, seg.rows)
            engine.set_rows(seg.g, seg.row, seg.rows, bufs[s][off:off + n])
            off += n
        got += bufs[s].numel() * bufs[s].element_size()
    engine.sync()
    return got


class LibraryEngine:
    """A rank's window stepped by the library (its own stream); rows move
    through torch device tensors with the C ABI's pack / unpack calls."""

    def __init__(self, plan: SlabPlan, r: int, problem: inputs.Problem, dt: float, schedule: str = "merged",
                 kernel: str = "auto", device: str = "cuda", stream=None):
        import torch
        from . import capi
        self.plan, self.r = plan, r
        wp = plan.window_problem(problem, r)
        self.s = capi.Stepper(N=wp.N, ax=wp.ax, n=wp.n, bc=wp.bc, cn=wp.cn, precision=wp.precision,
                              system=wp.system, dt=dt, schedule=schedule, kernel=kernel, stream=stream)
        self.dtype = torch.float32 if wp.precision == "fp32" else torch.float64
        self.device = torch.device(device)
        self.nx = [self.s.grid_info(g)[0] for g in range(4)]
        self.K = [0, 0, 0, 0]
        for j in range(self.s.ncomp):
            self.K[self.s.moment_info(j)["grid"]] += 1

    def load(self, glob: "GlobalSamples"):
        """Material, sources and initial state sliced from the global samples."""
        s, r, plan = self.s, self.r, self.plan
        if glob.sl_factor is not None:
            s.set_scattering_factors(glob.sl_factor)
        for g in range(4):
            if self.nx[g] == 0:
                continue
            s.set_material(g, plan.slice_rows(r, g, glob.sigma_a[g]), plan.slice_rows(r, g, glob.sigma_s0[g]))
        for j, q in glob.sources.items():
            s.set_source(j, plan.slice_rows(r, glob.grid[j], q))
        for j, u in glob.ic.items():
            s.set_moment(j, plan.slice_rows(r, glob.grid[j], u))

    def row_elems(self, g: int, rows: int) -> int:
        return self.K[g] * rows * self.nx[g]

    def rows(self, g: int, y0: int, rows: int):
        import torch
        buf = torch.empty(self.row_elems(g, rows), dtype=self.dtype, device=self.device)
        self.s.pack_rows(g, y0, rows, buf.data_ptr(), buf.numel() * buf.element_size())
        return buf

    def set_rows(self, g: int, y0: int, rows: int, buf):
        self.s.unpack_rows(g, y0, rows, buf.data_ptr(), buf.numel() * buf.element_size())

    def step(self, n: int):
        self.s.step(n)

    def sync(self):
        self.s.sync()

    def owned(self, j: int) -> np.ndarray:
        g = self.s.moment_info(j)["grid"]
        w0, w1 = self.plan.owned(self.r, g)
        return self.s.moments(j)[w0:w1]

    def owned_updates(self) -> int:
        """Moment-cell updates per step of the rows this rank owns."""
        total = 0
        for j in range(self.s.ncomp):
            info = self.s.moment_info(j)
            w0, w1 = self.plan.owned(self.r, info["grid"])
            total += (w1 - w0) * info["nx"]
        return total

    def owned_sums(self):
        """FP64 sums over the owned rows: (sum of R_0^0, sum of squares, non-finite count)."""
        mass, sq, bad = 0.0, 0.0, 0
        for j in range(self.s.ncomp):
            u = self.owned(j)
            fin = np.isfinite(u)
            bad += int(u.size - fin.sum())
            v = np.where(fin, u, 0.0)
            sq += float(np.sum(v * v))
            if j == 0:
                mass += float(np.sum(v))
        return mass, sq, bad


def grid_coordinates(problem: inputs.Problem, g: int) -> Tuple[np.ndarray, np.ndarray]:
    """Coordinates (X, Y), arrays [row][x], of the points of grid g of the
    global problem (eq. grid11 / staggered_grids; the library's layout)."""
    def axis(d, node):
        lo, hi = problem.ax[2 * d], problem.ax[2 * d + 1]
        n = problem.n[d]
        h = (hi - lo) / n
        if not node:
            return lo + (np.arange(n) + 0.5) * h
        if problem.bc[d] == "periodic":
            return lo + (np.arange(n) + 1.0) * h
        return lo + np.arange(n + 1) * h
    xs, ys = axis(0, g & 1), axis(1, g & 2)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return X, Y


def global_samples(problem: inputs.Problem, grid_of) -> "GlobalSamples":
    """Material, sources and initial data of `problem` sampled at the
    global grids' points; grid_of[j] is component j's grid."""
    sa, ss = [], []
    for g in range(4):
        X, Y = grid_coordinates(problem, g)
        sa.append(np.ascontiguousarray(np.broadcast_to(problem.sigma_a(0.0, X, Y), X.shape), dtype=np.float64)
                  if problem.sigma_a else np.zeros_like(X))
        ss.append(np.ascontiguousarray(np.broadcast_to(problem.sigma_s0(0.0, X, Y), X.shape), dtype=np.float64)
                  if problem.sigma_s0 else np.zeros_like(X))
    src, ic = {}, {}
    for j, q in problem.sources:
        X, Y = grid_coordinates(problem, grid_of[j])
        src[j] = src.get(j, 0.0) + np.broadcast_to(q(0.0, X, Y), X.shape)
    for j, f in problem.ic:
        X, Y = grid_coordinates(problem, grid_of[j])
        ic[j] = np.ascontiguousarray(np.broadcast_to(f(0.0, X, Y), X.shape), dtype=np.float64)
    return GlobalSamples(sigma_a=sa, sigma_s0=ss, sources={j: np.ascontiguousarray(v) for j, v in src.items()},
                         ic=ic, grid=list(grid_of), sl_factor=problem.sigma_sl_factor)


@dataclasses.dataclass
class GlobalSamples:
    """Material, sources and initial data sampled on the global grids
    (arrays [row][x] per grid; per component for sources and ic)."""
    sigma_a: List[np.ndarray]
    sigma_s0: List[np.ndarray]
    sources: Dict[int, np.ndarray]
    ic: Dict[int, np.ndarray]
    grid: List[int]
    sl_factor: object = None


def run(plan: SlabPlan, engines: Sequence, nsteps: int, exchange) -> int:
    """nsteps steps in chunks of plan.k with an exchange after each chunk
    but the last; returns the bytes exchanged."""
    moved, done = 0, 0
    while done < nsteps:
        k = min(plan.k, nsteps - done)
        for e in engines:
            e.step(k)
        done += k
        if done < nsteps:
            moved += exchange()
    return moved
