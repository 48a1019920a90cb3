"""Write oracle_values.json: oracle |M|^2 for a few seeded events (calls only oracle/)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import reweight  # noqa: E402
from paper_2510_05100_b300 import phase_space as ps  # noqa: E402

POINTS = {
    "ee_mumu": [ps.EE_ORIGINAL, ps.EE_NEW],
    "gg_ttx": [dict(mt=173.0, wt=0.0, alphas=0.118), dict(mt=171.0, wt=0.0, alphas=0.124)],
    "gg_ttxg": [dict(mt=173.0, wt=0.0, alphas=0.118), dict(mt=175.0, wt=0.0, alphas=0.112)],
    "gg_ttxgg": [dict(mt=173.0, wt=0.0, alphas=0.118), dict(mt=170.0, wt=1.0, alphas=0.126)],
}


def main():
    out = {}
    for proc, pts in POINTS.items():
        p = ps.make_events(proc, 3, 1234)
        out[proc] = {
            "seed": 1234, "nev": 3, "points": pts,
            "me2": [reweight.me2(proc, p, pt).tolist() for pt in pts],
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
