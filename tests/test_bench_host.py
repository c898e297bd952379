"""Host logic of bench.py: the multi-rank aggregation (world size 2, gloo on
CPU) and the reference arm's JSON line (the FP64 oracle on the host)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    units, ms = bench.aggregate(1000.0 * (rank + 1), 10.0 + 5.0 * rank, world)
    results[rank] = (units, ms)
    dist.destroy_process_group()


def test_aggregate_sums_units_and_takes_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            units, ms = results[r]
            assert units == 3000.0
            assert ms == 15.0


def test_reference_arm_prints_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    # every host core runs the oracle at once; the single-core figure is beside it
    assert 1 <= line["cpu_baseline"]["cores"] <= (os.cpu_count() or 1)
    assert line["cpu_baseline"]["single_core"] > 0


def test_closure_summary_matches_lowest_accurate_order():
    """The error-matched speedup takes the lowest plain order at least as
    accurate as the closure, among the comparison set and among all orders."""
    sys.path.insert(0, ROOT)
    from paper_1211_2205_gb300 import closure
    errs = {7: 0.29, 9: 0.15, 11: 0.072, 13: 0.035, 15: 0.018}
    ms = {7: 13.7, 9: 17.4, 11: 22.6, 13: 27.9, 15: 33.6}
    case = {"plain": {N: {"err": errs[N], "ms": ms[N]} for N in errs}, "closure": {"err": 0.055, "ms": 29.8}}
    out = closure.summarize([case, case], list(errs), compare=(7, 11, 15))
    assert out["matched_N"] == 15 and out["strict_matched_N"] == 13
    assert out["error_matched_speedup"] == pytest.approx(33.6 / 29.8)
    assert out["strict_error_matched_speedup"] == pytest.approx(27.9 / 29.8)
    assert out["gain_vs_p7"] == pytest.approx(0.29 / 0.055)
    worse = {"plain": case["plain"], "closure": {"err": 0.5, "ms": 1.0}}
    out = closure.summarize([worse], list(errs))
    assert out["matched_N"] == 7 and out["compare_orders"] == sorted(errs)
    # the end-to-end ratio takes the same matched order, on the host-clock times
    timed = {"plain": {N: {"err": errs[N], "ms": ms[N], "e2e_ms": 2 * ms[N]} for N in errs},
             "closure": {"err": 0.055, "ms": 29.8, "e2e_ms": 40.0}}
    out = closure.summarize([timed], list(errs), compare=(7, 11, 15))
    assert out["e2e_error_matched_speedup"] == pytest.approx(2 * 33.6 / 40.0)
    none = {"plain": case["plain"], "closure": {"err": 0.001, "ms": 1.0}}
    out = closure.summarize([none], list(errs))
    assert out["matched_N"] is None and out["error_matched_speedup"] is None


def test_algorithmic_bytes_are_three_values_per_update_per_step():
    """The roofline's numerator: a pass reads every input of the other
    parity once and reads and writes every output once, so the two passes
    of a merged step move 3 values per moment-cell update (12 B in FP32);
    at P_39 on 1024^2 the odd pass moves 5.20 GB."""
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    import bench
    from paper_1211_2205_gb300 import capi
    N, n = 39, 1024
    grid = capi.host_matrices(capi.PN2D, N)[2]

    class Fake:
        ncomp = len(grid)

        def moment_info(self, j):
            return {"grid": int(grid[j]), "nx": n, "ny": n}

    odd = bench.algorithmic_pass_bytes(Fake(), 1, 4)
    even = bench.algorithmic_pass_bytes(Fake(), 0, 4)
    assert odd == (2 * 420 + 400) * n * n * 4
    assert odd == pytest.approx(5.20e9, rel=2e-3)
    assert odd + even == 3 * 820 * n * n * 4
