"""Learned order-8 closure of P_7: training data from high-order runs of the
method, training on the GPU with the library's own network kernels, and
the error-matched comparison with plain P_N.

Every numerical step runs in libstarmap.so (the P_N passes, the closure
kernel, feature extraction, forward/backward/Adam); this module only
orchestrates: it allocates device buffers with torch, draws seeded
minibatch orders with numpy and times runs with CUDA events.

Workflow
--------
1. ``generate``: for each training medium (``inputs.closure_medium``) run
   plain P_{N_ref} (default P_39) from the initial pulses and, at evenly
   spaced time levels, extract per cell the 38 network inputs and the
   order-8 moments divided by the local RMS scale (the regression target).
2. ``train``: minibatch Adam on the mean squared error of the scaled
   targets (cosine learning-rate decay).
3. ``evaluate``: on held-out media, run P_{N_ref} as the reference, plain
   P_N for N in ``orders`` and P_7 with the trained closure, all with the
   same dt (the P_{N_ref} bound) and step count; report the relative L2
   error of R_0^0 against the reference and the device time of each run.
   The error-matched speedup is time(P_N*) / time(closure) for the lowest
   N* whose error is at most the closure's.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import capi, inputs

N_BASE = 7


def lambda_max(N: int) -> float:
    return capi.host_matrices(capi.PN2D, N)[4]


def common_dt(problem: inputs.Problem, N_ref: int) -> float:
    """cn * min(dx, dy) / lambda_max of P_{N_ref}: stable for every N <= N_ref."""
    h = min((problem.ax[1] - problem.ax[0]) / problem.n[0], (problem.ax[3] - problem.ax[2]) / problem.n[1])
    return problem.cn * h / lambda_max(N_ref)


def init_params(seed: int, scale_out: float = 0.1) -> np.ndarray:
    """Parameters with N(0, 1/fan_in) weights and zero biases; the output
    layer scaled by scale_out (a small initial closure)."""
    rng = np.random.default_rng(seed)
    H, I, O = capi.MLP_HIDDEN, capi.MLP_INPUTS, capi.MLP_OUTPUTS
    p = {
        "W1": rng.normal(0, 1 / math.sqrt(I), (H, I)),
        "b1": np.zeros(H),
        "W2": rng.normal(0, 1 / math.sqrt(H), (H, H)),
        "b2": np.zeros(H),
        "W3": scale_out * rng.normal(0, 1 / math.sqrt(H), (O, H)),
        "b3": np.zeros(O),
    }
    return capi.params_from_dict(p)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the closure workflow runs on the GPU (CUDA device required)")
    return torch


@dataclass
class SampleSet:
    X: object            # torch [S, 38] float32 (device)
    T: object            # torch [S, 9] float32 (device): order-8 moments / scale
    index: np.ndarray    # int32 indices of the samples used for training
    count: int           # len(index)
    seeds: List[int]
    snapshots: int
    n: int
    N_ref: int


def _set_ic(s: capi.Stepper, problem: inputs.Problem):
    for j, f in problem.ic:
        X, Y = s.grid_coords(s.moment_info(j)["grid"])
        s.set_moment(j, np.broadcast_to(f(0.0, X, Y), X.shape))


MEDIA = {"periodic": inputs.closure_medium, "c5": inputs.closure_c5}


def generate(seeds: Sequence[int], n: int = 512, N_ref: int = 39, snapshots: int = 8,
             t_final: float = 0.5, rel_floor: float = 1e-4, media: str = "periodic") -> SampleSet:
    """Training samples from plain P_{N_ref} runs on the media of `seeds`.
    Cells whose moment scale s lies below rel_floor times the largest s of
    their snapshot are left out: there the moments are round-off far from
    the pulses, and the network's prediction s * y is negligible anyway."""
    torch = _torch()
    M = n * n
    total = len(seeds) * snapshots * M
    X = torch.empty((total, capi.MLP_INPUTS), device="cuda", dtype=torch.float32)
    T = torch.empty((total, capi.MLP_OUTPUTS), device="cuda", dtype=torch.float32)
    scale = torch.empty(M, device="cuda", dtype=torch.float32)
    off = 0
    keep = []
    for seed in seeds:
        p = MEDIA[media](seed, n=n, N=N_ref, t_final=t_final)
        dt = common_dt(p, N_ref)
        nsteps = int(round(t_final / dt))
        marks = [int(round((k + 1) * nsteps / snapshots)) for k in range(snapshots)]
        s = capi.Stepper.from_problem(p, dt=dt, schedule="merged")
        done = 0
        torch.cuda.synchronize()
        for mk in marks:
            s.step(mk - done)
            done = mk
            s.closure_samples(X[off:off + M], scale, T[off:off + M])
            s.sync()                     # the samples are written on the stepper's stream
            sc = scale.cpu().numpy()
            keep.append(off + np.nonzero(sc >= rel_floor * sc.max())[0].astype(np.int64))
            off += M
        s.sync()
        s.close()
    torch.cuda.synchronize()
    index = np.concatenate(keep).astype(np.int32)
    return SampleSet(X=X, T=T, index=index, count=int(index.size), seeds=list(seeds), snapshots=snapshots, n=n,
                     N_ref=N_ref)


@dataclass
class TrainResult:
    params: np.ndarray
    losses: List[float] = field(default_factory=list)    # full-batch-free running minibatch losses
    steps: int = 0


def train(data: SampleSet, steps: int = 48000, batch: int = 8192, lr0: float = 2e-3, lr1: float = 2e-5,
          seed: int = 0, log_every: int = 200, noise: float = 0.05, engine: str = "tcgen05") -> TrainResult:
    """Minibatch Adam with cosine decay from lr0 to lr1.  noise: standard
    deviation of Gaussian noise added to the 36 normalised moment inputs,
    drawn afresh for every pass over the samples (the closed run feeds the
    network states with errors of its own; noise in training makes it
    tolerate them).  engine: kernels of the loss gradient ("tcgen05" or
    "mma_sync")."""
    torch = _torch()
    net = capi.Network(init_params(seed))
    net.set_engine(engine)
    loss = torch.zeros(1, device="cuda")
    res = TrainResult(params=np.empty(0))
    # the kept samples on the device once; each epoch's order is drawn there
    index = torch.from_numpy(np.ascontiguousarray(data.index, dtype=np.int32)).cuda()
    idx = torch.empty_like(index)
    pos = data.count
    X = torch.empty_like(data.X) if noise > 0 else data.X
    epoch = 0
    torch.cuda.synchronize()
    for it in range(steps):
        if pos + batch > data.count:
            net.shuffle(index, data.count, (seed << 20) + epoch, idx)
            if noise > 0:
                net.perturb_inputs(data.X, X, data.X.shape[0], capi.MLP_INPUTS - 2, noise,
                                   (seed << 20) + epoch)
            epoch += 1
            torch.cuda.synchronize()
            pos = 0
        lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * it / max(1, steps - 1)))
        net.train_step(X, data.T, batch, lr, loss=loss if (it % log_every == 0) else None,
                       idx=idx[pos:pos + batch])
        pos += batch
        if it % log_every == 0:
            net.sync()
            res.losses.append(float(loss.item()))
    net.sync()
    res.params = net.params
    res.steps = steps
    net.close()
    return res


def mean_loss(params: np.ndarray, data: SampleSet, limit: Optional[int] = None) -> float:
    """Mean squared error of the network on (a prefix of) a sample set."""
    torch = _torch()
    net = capi.Network(params)
    B = data.count if limit is None else min(limit, data.count)
    idx = torch.from_numpy(data.index[:B].copy()).cuda()
    g = torch.empty(capi.MLP_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    net.loss_grad(data.X, data.T, B, g, loss, idx=idx)
    net.sync()
    v = float(loss.item())
    net.close()
    return v


@dataclass
class RunResult:
    N: int
    closure: bool
    R00: np.ndarray
    ms: float
    steps: int
    e2e_ms: float = float("nan")      # host clock: initial moments uploaded, steps, R_0^0 read back
    h2d_bytes: int = 0
    d2h_bytes: int = 0


def run_case(problem: inputs.Problem, N: int, dt: float, nsteps: int, params: Optional[np.ndarray] = None,
             repeats: int = 1, closure_schedule: str = "merged") -> RunResult:
    """Run P_N (params None) or P_7 with the closure network from the
    problem's initial condition for nsteps steps of size dt; device time of
    the stepping (after one untimed warm-up run) on a dedicated stream, and
    the same run end to end on the host clock: state cleared, initial
    moments uploaded from host arrays, the steps, R_0^0 read back."""
    torch = _torch()
    stream = torch.cuda.Stream()
    closure = params is not None
    q = inputs.Problem(**{**problem.__dict__, "N": N})
    s = capi.Stepper.from_problem(q, dt=dt, stream=stream.cuda_stream,
                                  schedule=closure_schedule if closure else "merged",
                                  closure="mlp8" if closure else "none")
    if closure:
        s.set_closure(params)
    ic_host = []
    for j, f in q.ic:
        X, Y = s.grid_coords(s.moment_info(j)["grid"])
        ic_host.append((j, np.ascontiguousarray(np.broadcast_to(f(0.0, X, Y), X.shape), dtype=np.float64)))
    times, e2e = [], []
    for r in range(repeats + 1):
        s.clear()
        for j, a0 in ic_host:
            s.set_moment(j, a0)
        s.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            s.step(nsteps)
            b.record(stream)
        s.sync()
        b.synchronize()
        if r > 0:
            times.append(a.elapsed_time(b))
    for r in range(repeats):
        t0 = time.perf_counter()
        s.clear()
        for j, a0 in ic_host:
            s.set_moment(j, a0)
        s.step(nsteps)
        R00 = s.moments(0)
        e2e.append((time.perf_counter() - t0) * 1e3)
    R00 = s.moments(0)
    s.close()
    return RunResult(N=N, closure=closure, R00=R00, ms=float(np.median(times)), steps=nsteps,
                     e2e_ms=float(np.median(e2e)) if e2e else float("nan"),
                     h2d_bytes=sum(a0.nbytes for _, a0 in ic_host), d2h_bytes=R00.size * 8)


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    return float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-300))


def evaluate(params: np.ndarray, seeds: Sequence[int], n: int = 512, orders: Sequence[int] = (7, 9, 11, 13, 15),
             N_ref: int = 39, t_final: float = 0.5, repeats: int = 1,
             closure_schedules: Sequence[str] = ("merged",), compare: Optional[Sequence[int]] = None,
             media: str = "periodic") -> Dict:
    """Errors of R_0^0 against P_{N_ref} and device times, per held-out
    medium; the error-matched speedup is taken among the orders `compare`
    (default: all of `orders`) and among all of `orders` ("strict")."""
    cases = []
    for seed in seeds:
        p = MEDIA[media](seed, n=n, N=N_ref, t_final=t_final)
        dt = common_dt(p, N_ref)
        nsteps = int(round(t_final / dt))
        ref = run_case(p, N_ref, dt, nsteps)
        row = {"seed": seed, "dt": dt, "steps": nsteps, "ref_ms": ref.ms, "plain": {}}
        for N in orders:
            r = run_case(p, N, dt, nsteps, repeats=repeats)
            row["plain"][N] = {"err": rel_l2(r.R00, ref.R00), "ms": r.ms, "e2e_ms": r.e2e_ms,
                               "h2d_bytes": r.h2d_bytes, "d2h_bytes": r.d2h_bytes}
        for k, sched in enumerate(closure_schedules):
            r = run_case(p, N_BASE, dt, nsteps, params=params, repeats=repeats, closure_schedule=sched)
            row["closure" if k == 0 else "closure_" + sched] = {
                "err": rel_l2(r.R00, ref.R00), "ms": r.ms, "e2e_ms": r.e2e_ms,
                "h2d_bytes": r.h2d_bytes, "d2h_bytes": r.d2h_bytes}
        cases.append(row)
    return summarize(cases, orders, compare)


def summarize(cases: List[Dict], orders: Sequence[int], compare: Optional[Sequence[int]] = None) -> Dict:
    """Mean error and time per method over the cases, and the error-matched
    speedup of the closure against the lowest plain order at least as
    accurate on average: among `compare` (default: all evaluated orders) and,
    as "strict", among all evaluated orders."""
    def mean(rows, key):
        vals = [r[key] for r in rows if key in r]
        return float(np.mean(vals)) if vals else float("nan")

    plain = {N: {k: mean([c["plain"][N] for c in cases], k) for k in ("err", "ms", "e2e_ms")} for N in orders}
    cl = {k: mean([c["closure"] for c in cases], k) for k in ("err", "ms", "e2e_ms")}

    def matched(candidates, key="ms"):
        N = next((N for N in sorted(candidates) if plain[N]["err"] <= cl["err"]), None)
        return N, (plain[N][key] / cl[key]) if N is not None else None

    cmp = sorted(compare) if compare is not None else sorted(orders)
    match, speedup = matched(cmp)
    strict_N, strict = matched(orders)
    e2e = matched(cmp, "e2e_ms")[1]
    out = {"cases": cases, "plain": plain, "closure": cl, "compare_orders": cmp, "matched_N": match,
           "error_matched_speedup": speedup, "strict_matched_N": strict_N, "strict_error_matched_speedup": strict,
           "e2e_error_matched_speedup": e2e if e2e is None or math.isfinite(e2e) else None,
           "gain_vs_p7": plain[N_BASE]["err"] / cl["err"] if N_BASE in plain and cl["err"] > 0 else None}
    return out


@dataclass
class FallbackRun:
    state: List[np.ndarray]       # components of order <= 7 at the final time, [ny, nx] each
    fell_back: bool               # True if the closed run failed its health check
    good_steps: int               # closed-run steps that passed the check
    fallback_N: int
    detail: str = ""


def run_with_fallback(problem: inputs.Problem, params: np.ndarray, dt: float, nsteps: int,
                      fallback_N: int = 15, every: int = 16, growth: float = 1.05,
                      closure_schedule: str = "merged") -> FallbackRun:
    """P_7 with the learned closure, watched by the library's health check
    (FP64 reduction every `every` steps: NaN/Inf, or L2 growth beyond
    `growth` times what the sources can add).  If a span fails, the closed
    state of the last span that passed seeds plain P_{fallback_N} (its
    moments up to order 8, the higher orders zero) and plain P_N runs the
    rest of the steps; the result then comes from plain P_N."""
    q7 = inputs.Problem(**{**problem.__dict__, "N": N_BASE})
    s = capi.Stepper.from_problem(q7, dt=dt, schedule=closure_schedule, closure="mlp8")
    try:
        s.set_closure(params)
        s.set_health_check(every, growth)
        try:
            s.step(nsteps)
            return FallbackRun(state=[s.moments(j) for j in range(36)], fell_back=False, good_steps=nsteps,
                               fallback_N=fallback_N)
        except capi.StarmapError as e:
            if e.code not in (capi.E_GROWTH, capi.E_NONFINITE):
                raise
            detail = str(e)
        good, _, _ = s.health()
        seed = [s.moments(j) for j in range(s.ncomp)]        # 45 components of the closed P_8 system
        t_good = s.time
    finally:
        s.close()
    qN = inputs.Problem(**{**problem.__dict__, "N": fallback_N})
    f = capi.Stepper.from_problem(qN, dt=dt, schedule="merged")
    try:
        f.clear()
        for j, u in enumerate(seed):       # the first 45 components of P_N are those of P_8
            f.set_moment(j, u)
        f.set_time(t_good)
        f.step(nsteps - good)
        state = [f.moments(j) for j in range(36)]
    finally:
        f.close()
    return FallbackRun(state=state, fell_back=True, good_steps=good, fallback_N=fallback_N, detail=detail)
