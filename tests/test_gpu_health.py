"""The periodic health check of the stepping and the learned closure's
fallback to plain P_N (failure detection on the host side: a deliberately
bad network makes the closed run diverge; nothing faults the GPU).

* A healthy run with the check on equals the same spans run without it,
  bit for bit, and reports every step as passed.
* A diverging closed run fails a span with E_GROWTH or E_NONFINITE; the
  state, time and step count go back to the last span that passed, which
  equals a fresh closed run of that many steps in the same spans.
* ``closure.run_with_fallback`` then finishes the run with plain P_N from
  that state, equal to the same continuation built by hand."""
import math

import numpy as np
import pytest

from paper_1211_2205_gb300 import capi, closure
from test_gpu_closure import _closure_problem, _params
from test_gpu_parity import _random_problem

pytestmark = pytest.mark.gpu


def _state(s, count=None):
    return [s.moments(j) for j in range(s.ncomp if count is None else count)]


@pytest.mark.parametrize("precision,kernel", [("fp64", "gather"), ("fp32", "tiled")])
def test_healthy_run_is_unchanged_by_the_check(precision, kernel):
    p = _random_problem(5, (41, 30), ("periodic", "extrapolation"), precision, 77, 12)
    a = capi.Stepper.from_problem(p, kernel=kernel, schedule="merged")
    a.set_health_check(4, 1.05)
    a.step(12)
    good, l2_good, l2_bad = a.health()
    assert good == 12 and a.steps_done == 12 and math.isnan(l2_bad)
    b = capi.Stepper.from_problem(p, kernel=kernel, schedule="merged")
    for _ in range(3):
        b.step(4)                       # the same spans without the check
    _, l2_b, bad = b.diagnostics()
    assert bad == 0 and l2_good == l2_b
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    assert a.time == b.time
    a.set_health_check(0)               # off again: plain stepping
    a.step(1)
    assert a.steps_done == 13


def _bad_params():
    """A network whose order-8 prediction is far too large: the closed run
    feeds energy into the order-7 rows every odd pass and diverges."""
    v = _params(61, scale_out=0.6)
    d = capi.params_to_dict(v)
    d["W3"] = d["W3"] * 400.0
    d["b3"] = d["b3"] + 20.0
    return capi.params_from_dict(d)


def test_diverging_closure_is_caught_and_rolled_back():
    p = _closure_problem(precision="fp32", n=(64, 48), nsteps=24)
    params = _bad_params()
    # without the check the run blows up
    w = capi.Stepper.from_problem(p, kernel="tiled", closure="mlp8", schedule="merged")
    w.set_closure(params)
    _, l2_0, _ = w.diagnostics()
    w.step(p.nsteps)
    _, l2_w, bad_w = w.diagnostics()
    assert bad_w > 0 or l2_w > 10 * l2_0
    w.close()
    s = capi.Stepper.from_problem(p, kernel="tiled", closure="mlp8", schedule="merged")
    s.set_closure(params)
    s.set_health_check(2, 1.05)
    with pytest.raises(capi.StarmapError) as e:
        s.step(p.nsteps)
    assert e.value.code in (capi.E_GROWTH, capi.E_NONFINITE)
    good, l2_good, l2_failed = s.health()
    assert good % 2 == 0 and good < p.nsteps
    assert s.steps_done == good and s.time == pytest.approx(good * s.dt, rel=1e-12)
    assert not (l2_failed <= 1.05 * l2_good)          # NaN or past the bound
    _, l2_now, bad_now = s.diagnostics()
    assert bad_now == 0 and l2_now == l2_good
    got = _state(s)
    ref = capi.Stepper.from_problem(p, kernel="tiled", closure="mlp8", schedule="merged")
    ref.set_closure(params)
    for _ in range(good // 2):
        ref.step(2)
    for x, y in zip(got, _state(ref)):
        assert np.array_equal(x, y)


def test_fallback_finishes_with_plain_pn():
    p = _closure_problem(precision="fp32", n=(64, 48), nsteps=24)
    params = _bad_params()
    dt = closure.common_dt(p, 39)
    r = closure.run_with_fallback(p, params, dt, p.nsteps, fallback_N=11, every=2)
    assert r.fell_back and r.good_steps < p.nsteps
    assert all(np.isfinite(u).all() for u in r.state)
    # the same continuation by hand: closed run to the last good span, its
    # 45 moments seed plain P_11, which runs the remaining steps
    c = capi.Stepper.from_problem(inputs_n(p, 7), dt=dt, closure="mlp8", schedule="merged")
    c.set_closure(params)
    for _ in range(r.good_steps // 2):
        c.step(2)
    seed = _state(c)
    f = capi.Stepper.from_problem(inputs_n(p, 11), dt=dt, schedule="merged")
    f.clear()
    for j, u in enumerate(seed):
        f.set_moment(j, u)
    f.set_time(c.time)
    f.step(p.nsteps - r.good_steps)
    for x, y in zip(r.state, _state(f, 36)):
        assert np.array_equal(x, y)
    # a healthy closure does not fall back
    ok = closure.run_with_fallback(p, _params(62, scale_out=0.3), dt, 6, fallback_N=11, every=2)
    assert not ok.fell_back and ok.good_steps == 6


def inputs_n(p, N):
    from paper_1211_2205_gb300 import inputs
    return inputs.Problem(**{**p.__dict__, "N": N})
