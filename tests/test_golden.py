"""The oracle still reproduces its stored regression fixture (written by
tests/golden/make_golden.py, which calls only the oracle)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_reproduces_c1_fixture():
    with open(os.path.join(HERE, "golden", "c1_oracle_obs.json")) as fh:
        stored = json.load(fh)
    fresh = make_golden.c1_obs()
    for a, b in zip(stored["obs"], fresh["obs"]):
        for k, v in a.items():
            assert abs(v - b[k]) <= 1e-13 * max(1.0, abs(v)), k
