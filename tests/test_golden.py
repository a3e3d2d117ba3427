"""The oracle reproduces its stored regression fixture (tests/golden)."""
import json
import os

import numpy as np

from tests.golden.make_golden import compute

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_oracle.json")


def test_oracle_matches_golden_fixture():
    want = json.load(open(HERE))
    got = compute()
    assert got["pixels"] == want["pixels"] and got["n_contrib"] == want["n_contrib"]
    for k in ("depth", "alpha", "unc", "nu_map", "median", "T_final", "color", "pose_grad"):
        np.testing.assert_allclose(np.array(got[k]), np.array(want[k]), rtol=1e-12, atol=1e-15, err_msg=k)
    np.testing.assert_allclose(got["loss"], want["loss"], rtol=1e-13)
