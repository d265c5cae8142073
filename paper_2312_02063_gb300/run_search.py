"""Run one hot-path call repeatedly on a synthetic Kepler-length star, in steady state (no
cache flush between calls), for profiling with external tools such as Nsight Compute.

  python -m paper_2312_02063_gb300.run_search --what box --n-periods 250000 --repeat 5
  python -m paper_2312_02063_gb300.run_search --what cnn --n-periods 250000 --repeat 5
  python -m paper_2312_02063_gb300.run_search --what cnn-score --n-profiles 16384 --repeat 5
  python -m paper_2312_02063_gb300.run_search --what fold --n-periods 32768 --layout 2 --warps 3

box: fold + box-SNR search (the default path, widths 1..108); cnn: fold + CNN search; cnn-score:
CNN scoring of device-generated profiles; fold: the fold alone (means and counts of every
period). --layout, --warps, --chunk and --tile set the fold's launch config (0: automatic).
Prints the mean CUDA-event time of the repeats after the first.
"""
from __future__ import annotations

import argparse
import math

import torch

from . import (SCORER_BOX, SCORER_CNN, Context, gpfc_fold, gpfc_score_cnn, gpfc_search,
               gpfc_synth_profiles)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["box", "cnn", "cnn-score", "fold"], default="box")
    ap.add_argument("--n-periods", type=int, default=250_000)
    ap.add_argument("--n-profiles", type=int, default=16_384)
    ap.add_argument("--repeat", type=int, default=5)
    ap.add_argument("--seed", type=int, default=20232204)
    for k in ("layout", "warps", "chunk", "tile"):
        ap.add_argument("--" + k, type=int, default=0)
    a = ap.parse_args()
    import lcsynth  # the synthetic-input generators
    from .train import init_weights
    ctx = Context(0)
    ctx.set_fold_config(warps=a.warps, layout=a.layout, chunk=a.chunk, tile=a.tile)
    dev = ctx.device
    w = init_weights(dev, 1)
    if a.what == "cnn-score":
        prof, counts, _, _, _ = gpfc_synth_profiles(ctx, 20233204, 0, a.n_profiles)
        out = torch.empty(a.n_profiles, dtype=torch.float32, device=dev)

        def call():
            gpfc_score_cnn(ctx, prof, w, counts, score=out)
    else:
        lc = lcsynth.light_curve_kepler(seed=a.seed)
        periods = lcsynth.freq_grid(a.n_periods)
        t = torch.from_numpy(lc.times).to(dev)
        f = torch.from_numpy(lc.flux).to(dev)
        p = torch.from_numpy(periods).to(dev)
        score = torch.empty(a.n_periods, dtype=torch.float32, device=dev)
        folded = torch.empty(a.n_periods, 256, dtype=torch.float32, device=dev)
        counts = torch.empty(a.n_periods, 256, dtype=torch.int32, device=dev)

        def call():
            if a.what == "fold":
                gpfc_fold(ctx, t, f, p, 256, lc.t0, folded=folded, counts=counts)
            elif a.what == "box":
                gpfc_search(ctx, t, f, p, 256, lc.t0, SCORER_BOX, 1, int(math.ceil(0.42 * 256)), 0.0, score)
            else:
                gpfc_search(ctx, t, f, p, 256, lc.t0, SCORER_CNN, score=score, weights=w)
    call()
    ctx.sync()
    ms = []
    for _ in range(max(1, a.repeat - 1)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(f"{a.what}: {sum(ms) / len(ms):.3f} ms per call (mean of {len(ms)}, steady state); "
          f"plan {ctx.last_fold_plan()}")
    ctx.close()


if __name__ == "__main__":
    main()
