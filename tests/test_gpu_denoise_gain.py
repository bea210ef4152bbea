"""What the trained denoiser gains over plain Monte Carlo: a small study (64^3 phantoms at
0.5 cm, 24 training cases) trains the network on engine-made pairs and, on held-out cases,
compares the error of denoised and plain doses at equal history counts against a
high-history reference."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_denoiser_beats_plain_mc_at_equal_histories(tmp_path):
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import denoiser
    rep = denoiser.run_study(n_train=24, n_eval=4, lows=(10**5, 10**6), n_high=10**7,
                             n_ref=(4 * 10**8, 6 * 10**7), steps=600, lr=1e-3, warmup=30, shape=(64, 64, 64),
                             voxel=(0.5, 0.5, 0.5), log=lambda m: None)
    print(json.dumps({k: v for k, v in rep.items() if k != "cases"}))
    assert rep["loss_last_100"] < rep["loss_first_100"]
    ratios = []
    for c in rep["cases"]:
        for row in c["curve"]:
            if 10**5 <= row["n"] <= 3.2 * 10**5:
                ratios.append(row["err_denoised"] / row["err_plain"])
        print(c["particle"], c["field_cm"], c["plain"], c["denoised"])
    # at the noise level of the training inputs the network must reduce the error on unseen
    # cases (a network this small and briefly trained has a bias floor of its own, so at
    # higher history counts its gain shrinks; the full-size study measures the time gain)
    assert max(ratios) < 1.0 and np.median(ratios) < 0.85, ratios
