"""What the trained closure gains (GPU, end to end at a small scale): train
the network on P_39 runs over random media with the library's own
kernels, then on a held-out medium the closed P_7 must be closer to P_39
(relative L2 error of R_0^0) than plain P_7 with the same dt and steps."""
import numpy as np
import pytest

from paper_1211_2205_gb300 import closure

pytestmark = pytest.mark.gpu


def test_trained_closure_beats_plain_p7_on_held_out_media():
    pytest.importorskip("torch")
    n, t_final = 128, 0.5
    data = closure.generate([0, 1, 2, 3], n=n, N_ref=39, snapshots=6, t_final=t_final)
    assert data.count > 10000
    tr = closure.train(data, steps=1500, batch=4096, lr0=2e-3, lr1=2e-5, seed=3)
    assert np.isfinite(tr.params).all()
    assert tr.losses[-1] < 0.25 * tr.losses[0]
    ev = closure.evaluate(tr.params, [100, 101], n=n, orders=(7, 11), t_final=t_final, repeats=1)
    for case in ev["cases"]:
        plain, closed = case["plain"][7]["err"], case["closure"]["err"]
        assert closed < 0.8 * plain, (case["seed"], plain, closed)
