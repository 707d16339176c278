"""The stored oracle gradient of the differentiation workload (tests/golden/gradient_channel_4x128_L512.json,
written by tests/golden/make_gradient_golden.py from the FP64 oracle alone): it is for the configuration the
package describes, with the seeded target, and its values are finite."""
import json
import os

import numpy as np

from paper_1504_06123_gb300 import configs, inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gradient_channel_4x128_L512.json")


def test_gradient_golden_file_is_the_oracle_workload():
    with open(GOLDEN) as f:
        gold = json.load(f)
    w = configs.gradient_channel()
    assert gold["theta"] == [w.G_inf, w.tau, w.gamma_c, w.g]
    np.testing.assert_array_equal(gold["theta_target"], inputs.perturbed(np.array(gold["theta"]), seed=w.seed))
    wl = gold["workload"]
    assert (wl["nx"], wl["ny"], wl["tau_lb"], wl["C"], wl["B"], wl["steps"]) == (w.nx, w.ny, w.tau_lb, w.C, w.B, w.steps)
    assert gold["h_relative"] == 1e-4
    assert len(gold["u_target"]) == w.nx * w.ny == len(gold["sigma_xy_target"])
    assert np.all(np.isfinite(gold["gradient"])) and gold["loss"] > 0
