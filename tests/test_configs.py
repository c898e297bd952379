"""The run descriptions in configs/*.json: every file loads, names a
generator of the inputs module, and gives exactly the problems of a direct
call (the scalar fields equal, the material, source and initial fields
equal at sample points)."""
import glob
import os

import numpy as np
import pytest

from paper_1211_2205_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "configs", "*.json")))

DIRECT = {
    "gaussian_p5": lambda: [inputs.gaussian_p5()],
    "checkerboard_p13": lambda: [inputs.checkerboard_p13()],
    "random_p39": lambda: [inputs.random_p39()],
    "paper_p5": lambda: [inputs.checkerboard_p13(n=100, N=5, precision="fp64")],
    "batched_256": lambda: [inputs.batched_instance(k) for k in range(256)],
    "closure_p7": lambda: [inputs.closure_medium(s, n=512, N=7) for s in (100, 101, 102, 103)],
}


def _same(a: inputs.Problem, b: inputs.Problem):
    for f in ("name", "N", "ax", "n", "bc", "cn", "precision", "system", "sigma_sl_factor", "time_dependent",
              "nsteps", "t_final"):
        assert getattr(a, f) == getattr(b, f), f
    x0, x1, y0, y1 = a.ax
    X, Y = np.meshgrid(np.linspace(x0, x1, 13), np.linspace(y0, y1, 11))
    for fa, fb in ((a.sigma_a, b.sigma_a), (a.sigma_s0, b.sigma_s0)):
        assert np.array_equal(np.broadcast_to(fa(0.0, X, Y), X.shape), np.broadcast_to(fb(0.0, X, Y), X.shape))
    for la, lb in ((a.sources, b.sources), (a.ic, b.ic)):
        assert [j for j, _ in la] == [j for j, _ in lb]
        for (_, fa), (_, fb) in zip(la, lb):
            assert np.array_equal(np.broadcast_to(fa(0.0, X, Y), X.shape), np.broadcast_to(fb(0.0, X, Y), X.shape))


def test_every_config_is_covered():
    assert sorted(os.path.basename(f)[:-5] for f in FILES) == sorted(DIRECT)


@pytest.mark.parametrize("path", FILES, ids=lambda p: os.path.basename(p))
def test_config_gives_the_direct_problems(path):
    name = os.path.basename(path)[:-5]
    got, description = inputs.load_config(path)
    assert description
    want = DIRECT[name]()
    assert len(got) == len(want)
    for a, b in zip(got, want):
        _same(a, b)
    # by name as well as by path
    assert len(inputs.load_config(name)[0]) == len(want)
