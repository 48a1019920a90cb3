"""Run a fixed reweighting case for profilers (ncu): python -m paper_2510_05100_b300.profile_case

  --proc gg_ttxg --mode fp64|mixed --nev N --launches L [--variant V]
  --surrogate-steps S          (surrogate training steps instead)
  --surrogate-infer fused|layered  (surrogate inference instead)

Generates the standard seeded events, then issues L rex_reweight launches to the
16-point (gg_ttxg, qq_ttx) / 8-point (gg_ttx) / 64-point (gg_ttxgg) grid and synchronises.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2510_05100_b300 import phase_space as ps  # noqa: E402
from paper_2510_05100_b300 import rex  # noqa: E402

GRIDS = {"gg_ttx": ps.grid_gg_ttx, "gg_ttxg": ps.grid_gg_ttxg, "gg_ttxgg": ps.grid_64,
         "qq_ttx": ps.grid_gg_ttxg, "qq_ttxg": ps.grid_gg_ttxg}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--proc", default="gg_ttxg")
    ap.add_argument("--mode", choices=["fp64", "mixed", "df64"], default="fp64")
    ap.add_argument("--nev", type=int, default=1 << 19)
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--variant", type=int, default=None, help="kernel thread-mapping variant (g g processes)")
    ap.add_argument("--surrogate-steps", type=int, default=0,
                    help="instead: train the surrogate for this many steps of 8192 samples")
    ap.add_argument("--surrogate-infer", choices=["fused", "layered"], default=None,
                    help="instead: surrogate inference of --nev events x 64 points, --launches times")
    a = ap.parse_args()
    if a.surrogate_infer:
        mom = torch.from_numpy(ps.make_events("gg_ttxg", a.nev, 3)).cuda()
        pts = ps.grid_64()
        s = rex.Surrogate(1)
        s.set_exact_alphas(0.118, 3)
        s.set_kernel(rex.SURROGATE_FUSED if a.surrogate_infer == "fused" else rex.SURROGATE_LAYERED)
        pred = torch.empty((a.nev, len(pts)), dtype=torch.float32, device="cuda")
        for _ in range(a.launches):
            s.reweight(mom, None, pts, pred=pred)
        torch.cuda.synchronize()
        print(f"surrogate {a.surrogate_infer} inference nev={a.nev} k={len(pts)} launches={a.launches} ok "
              f"pred[0,:3]={pred[0, :3].tolist()}")
        return
    if a.surrogate_steps:
        mom = torch.from_numpy(ps.make_events("gg_ttxg", a.nev, 3)).cuda()
        pts = ps.grid_gg_ttxg()
        ex = rex.Process("gg_ttxg", rex.FP64)
        ex.set_params(mt=173.0, wt=0.0, alphas=0.118)
        ratio = ex.reweight(mom, torch.ones(a.nev, dtype=torch.float64, device="cuda"), pts)
        s = rex.Surrogate(1)
        losses = s.train(mom, ratio, pts, steps=a.surrogate_steps, batch=8192)
        torch.cuda.synchronize()
        print(f"surrogate {a.surrogate_steps} steps ok, loss {losses[0]:.4g} -> {losses[-1]:.4g}")
        return
    mom = torch.from_numpy(ps.make_events(a.proc, a.nev, 3)).cuda()
    w = torch.ones(a.nev, dtype=torch.float64, device="cuda")
    pts = GRIDS[a.proc]()
    p = rex.Process(a.proc, {"fp64": rex.FP64, "mixed": rex.MIXED, "df64": rex.DF64}[a.mode])
    p.set_params(mt=173.0, wt=0.0, alphas=0.118)
    if a.variant is not None:
        p.variant = a.variant
    out = torch.empty((a.nev, len(pts)), dtype=torch.float64, device="cuda")
    for _ in range(a.launches):
        p.reweight(mom, w, pts, w_out=out)
    torch.cuda.synchronize()
    print(f"{a.proc} {a.mode} variant={p.variant} nev={a.nev} k={len(pts)} launches={a.launches} ok "
          f"w_out[0,:3]={out[0, :3].tolist()}")


if __name__ == "__main__":
    main()
