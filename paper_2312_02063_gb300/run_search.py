"""Run one hot-path call repeatedly on a synthetic Kepler-length star, in steady state (no
cache flush between calls), for profiling with external tools such as Nsight Compute.

  python -m paper_2312_02063_gb300.run_search --what box --n-periods 250000 --repeat 5
  python -m paper_2312_02063_gb300.run_search --what cnn --n-periods 250000 --repeat 5
  python -m paper_2312_02063_gb300.run_search --what cnn-score --n-profiles 16384 --repeat 5
  python -m paper_2312_02063_gb300.run_search --what fold --n-periods 32768 --layout 2 --warps 3
  python -m paper_2312_02063_gb300.run_search --what probe

box: fold + box-SNR search (the default path, widths 1..108); cnn: fold + CNN search; cnn-score:
CNN scoring of device-generated profiles; fold: the fold alone (means and counts of every
period); probe: the shared-memory bin-update rates of every record kind (gpfc_probe_smem_rmw)
at full occupancy and at the fold's 256-bin footprints. --layout, --warps, --chunk and --tile set the fold's launch config (0: automatic).
Prints the mean CUDA-event time of the repeats after the first.
"""
from __future__ import annotations

import argparse
import math

import torch

from . import (SCORER_BOX, SCORER_CNN, Context, gpfc_fold, gpfc_probe_smem_rmw, gpfc_score_cnn, gpfc_search,
               gpfc_synth_profiles)


def probe_sweep():
    names = {(8, 0): "8 B packed, ld/st", (8, 1): "8 B two rows, 2 x red.u32", (6, 0): "6 B paired, ld/st",
             (6, 1): "6 B paired, red.f32 + red.u32", (4, 0): "4 B, ld/st", (4, 1): "4 B, red.u32"}
    print("record | op | bins x warps per SM | updates/clk/SM | G updates/s")
    for (word, op), name in names.items():
        for nbins, warps in ((32, 16), (256, 3), (256, 4)):
            if word * nbins * 32 * warps > 227 * 1024:
                continue
            ups, upc = gpfc_probe_smem_rmw(word, nbins, warps, 1, 20000, op=op)
            print(f"{name} | {nbins} x {warps} | {upc:.2f} | {ups / 1e9:.1f}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["box", "cnn", "cnn-score", "fold", "probe"], default="box")
    ap.add_argument("--n-periods", type=int, default=250_000)
    ap.add_argument("--n-profiles", type=int, default=16_384)
    ap.add_argument("--repeat", type=int, default=5)
    ap.add_argument("--seed", type=int, default=20232204)
    ap.add_argument("--n-samples", type=int, default=0, help="keep only the first N samples of the star (0: all)")
    for k in ("layout", "warps", "chunk", "tile", "streams"):
        ap.add_argument("--" + k, type=int, default=0)
    a = ap.parse_args()
    import lcsynth  # the synthetic-input generators
    from .train import init_weights
    if a.what == "probe":
        probe_sweep()
        return
    ctx = Context(0)
    ctx.set_fold_config(warps=a.warps, layout=a.layout, chunk=a.chunk, tile=a.tile, streams=a.streams)
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
        ns = a.n_samples if a.n_samples > 0 else lc.times.shape[0]
        t = torch.from_numpy(lc.times[:ns].copy()).to(dev)
        f = torch.from_numpy(lc.flux[:ns].copy()).to(dev)
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
