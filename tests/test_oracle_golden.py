"""Regression guard: the oracle reproduces the stored tiny-stream fixture."""
import json
import os

import numpy as np

from oracle.ttals_oracle import OnlineTTALS

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_golden_fixture():
    d = json.load(open(os.path.join(HERE, "golden", "oracle_tiny.json")))
    st = OnlineTTALS(d["dims"], d["ranks"], [np.array(c) for c in d["cores"]], np.array(d["g"]))
    for x, ref in zip(d["slices"], d["xhat"]):
        xh = st.step(np.array(x))
        assert np.abs(xh - np.array(ref)).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    assert np.abs(st.g - np.array(d["final_g"])).max() <= 1e-12
