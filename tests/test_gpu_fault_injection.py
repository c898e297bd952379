"""Host-side fault injection, with no GPU fault: each device allocation the
library makes fails in turn as if the device were out of memory.  The
failing call must return an error status (E_NOMEM or E_CUDA), nothing may
crash or leak device memory, and the process must still compute the right
answer afterwards.  Also: a handle destroyed with work still queued."""
import numpy as np
import pytest

from helpers import assert_parity, oracle_run
from paper_1211_2205_gb300 import capi, closure, inputs
from test_gpu_parity import _random_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _tiled():
    p = _random_problem(5, (70, 45), ("periodic", "extrapolation"), "fp32", 11, 3)
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    try:
        s.set_health_check(2, 1.05)
        s.step(4)
        s.advance_to(s.time + 0.5 * s.dt)
        return [s.output(j) for j in range(s.ncomp)]
    finally:
        s.close()


def _gather():
    p = _random_problem(3, (33, 31), ("extrapolation", "periodic"), "fp64", 12, 3)
    s = capi.Stepper.from_problem(p, kernel="gather")
    try:
        s.step(3)
        return [s.moments(j) for j in range(s.ncomp)] + [np.array(s.diagnostics())]
    finally:
        s.close()


def _closed():
    p = inputs.closure_medium(100, n=40, N=7)
    p = inputs.Problem(**{**p.__dict__, "nsteps": 2})
    s = capi.Stepper.from_problem(p, closure="mlp8", schedule="merged")
    try:
        s.set_closure(closure.init_params(1, scale_out=0.3))
        s.step(2)
        return [s.moments(j) for j in range(s.ncomp)]
    finally:
        s.close()


def _network():
    net = capi.Network(closure.init_params(2))
    try:
        X = torch.linspace(-1, 1, 256 * capi.MLP_INPUTS, device="cuda")
        T = torch.linspace(0, 1, 256 * capi.MLP_OUTPUTS, device="cuda")
        net.train_step(X, T, 256, 1e-3)
        net.sync()
        return [net.params.copy()]
    finally:
        net.close()


def _batch():
    probs = [inputs.batched_instance(k, nsteps=2) for k in (3, 8)]
    probs = [inputs.Problem(**{**q.__dict__, "n": (48, 48)}) for q in probs]
    b = capi.Batch.from_problems(probs, kernel="tiled_short")
    try:
        b.step(2)
        b.sync()
        return [inst.moments(0) for inst in b.instances]
    finally:
        b.close()


@pytest.mark.parametrize("work", [_tiled, _gather, _closed, _network, _batch])
def test_every_allocation_failure_is_reported_and_leaves_no_trace(work):
    want = work()                                   # a clean run, also warms every lazy allocation path
    base = _free_bytes()
    failures = 0
    for k in range(1, 200):
        assert capi.debug_fail_allocation(k) == capi.OK
        try:
            got = work()
        except capi.StarmapError as e:
            assert e.code in (capi.E_NOMEM, capi.E_CUDA), (k, e.code)
            failures += 1
            continue
        finally:
            capi.debug_fail_allocation(0)
        # the k-th allocation was beyond this work's last one: done
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        break
    else:
        pytest.fail("the work made more than 200 allocations")
    assert failures >= 2
    # nothing leaked (the library's handles are all destroyed again)
    assert abs(_free_bytes() - base) <= 64 << 20
    for a, b in zip(work(), want):
        assert np.array_equal(a, b)


def test_destroy_with_work_queued():
    p = _random_problem(7, (130, 90), ("periodic", "periodic"), "fp32", 21, 3)
    for _ in range(3):
        s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
        s.step(200)                                 # queued, not waited for
        s.close()
    s = capi.Stepper.from_problem(p, kernel="tiled", schedule="merged")
    s.step(p.nsteps)
    got = [s.moments(j) for j in range(s.ncomp)]
    _, ref = oracle_run(p, s)
    assert_parity(got, ref, 1e-5, "fp32")
    s.close()


def test_fail_allocation_argument():
    assert capi.debug_fail_allocation(-1) == capi.E_ARG
    assert capi.debug_fail_allocation(0) == capi.OK
