"""Oracle regression guard against tests/golden/oracle_values.json (CPU)."""
import json
import os

import numpy as np

from oracle import reweight
from paper_2510_05100_b300 import phase_space as ps

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_golden_values():
    with open(os.path.join(HERE, "golden", "oracle_values.json")) as f:
        gold = json.load(f)
    for proc, rec in gold.items():
        p = ps.make_events(proc, rec["nev"], rec["seed"])
        for pt, ref in zip(rec["points"], rec["me2"]):
            got = reweight.me2(proc, p, pt)
            assert np.allclose(got, ref, rtol=1e-13, atol=0), proc
