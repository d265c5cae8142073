"""Benchmark of the GPFC hot path on one GB300 (or N independent replicas).

A step is one full search of one Kepler-length light curve (65,536 cadences with ~4%
gapped, N ~ 62,900 samples) over 250,000 trial periods uniform in frequency in
[1, 5] c/d, 256 bins, box widths 1..108: quantise, fold, box-SNR score every period,
best period. The metric is sample*period folds per second (periods scored per second is
reported beside it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

`--impl reference` times the FP64 CPU oracle (the only reference this path has) on a
bounded sample of the same workload. For N > 1 (torchrun) every rank runs its own
replica (no data-path communication); value counts the work of all ranks.
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("sample·period folds/s and periods scored/s on 1 GB300, CNN vs box-SNR at fixed TPR/FPR")
UNIT = "sample·period folds/s"
NBINS = 256
N_PERIODS = 250_000  # default; --n-periods changes it (small cases for profiling)
W_MAX = int(math.ceil(0.42 * NBINS))  # 108: widths up to the longest injected duty cycle
SM_FOLD_UPDATES_PER_CLK = 16          # the pipe model: 128 B/clk / (4 B + 4 B of reductions)
# DRAM bytes (read + write) of the fold kernel's 18 launches of one 250,000-period search of
# the same light curve in steady state (no cache flush, one ncu pass), per period:
# profiles/dram_traffic_steady_state_kepler62835.md
SEARCH_DRAM_BYTES_PER_PERIOD = (0.403456e6 + 206.749696e6) / 250000
L2_FLUSH_BYTES = 256 << 20


def workload_name(n):
    return f"kepler-like light curve, {n} samples (65,536 cadences, 4% gaps), {N_PERIODS} periods, " \
           f"{NBINS} bins, fold + box-SNR (w 1..{W_MAX}) + best period"


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's); the value
    itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput: every rank processes its own replica of the workload."""
    return world * units_per_rank / (ms * 1e-3)


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 20 ms; started before the
    warm-up so that it is running when the timed region starts, it keeps only the samples
    whose nvidia-smi timestamps fall inside the region marked by begin() and end()."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.window = (None, None)

    def begin(self):
        self.window = (datetime.datetime.now(), None)

    def end(self):
        self.window = (self.window[0], datetime.datetime.now())

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                mhz, mhz_max = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            if t0 is not None and (ts < t0 or (t1 is not None and ts > t1)):
                continue  # outside the timed region
            sm.append(mhz)
            smax.append(mhz_max)
            for nm, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": 20}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def make_inputs():
    import lcsynth
    lc = lcsynth.light_curve_kepler()
    periods = lcsynth.freq_grid(N_PERIODS)
    return lc, periods


def cpu_oracle_rate(lc, periods, n_periods, seed=0):
    """Time the FP64 oracle (fold + box-SNR) on n_periods periods; returns (folds/s, seconds)."""
    import oracle
    idx = np.random.default_rng(seed).choice(len(periods), n_periods, replace=False)
    sub = np.ascontiguousarray(periods[np.sort(idx)])
    sigma = float(np.std(lc.flux.astype(np.float64)))
    t = time.perf_counter()
    _, cnt, sums = oracle.fold(lc.times, lc.flux, sub, NBINS, lc.t0)
    oracle.box_snr(sums, cnt, 1, W_MAX, sigma)
    dt = time.perf_counter() - t
    return lc.times.shape[0] * n_periods / dt, dt


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    lc, periods = make_inputs()
    n = lc.times.shape[0]
    per_step = 800
    for _ in range(args.warmup):
        cpu_oracle_rate(lc, periods, per_step // 4)
    rates, secs = [], []
    for s in range(args.steps):
        r, dt = cpu_oracle_rate(lc, periods, per_step, seed=s + 1)
        rates.append(r)
        secs.append(dt)
    value = n * per_step * len(secs) / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(n), "n_samples": n, "n_periods": N_PERIODS, "nbins": NBINS,
                   "w_max": W_MAX, "step_sample": f"{per_step} random periods of the {N_PERIODS}-period grid"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} periods per step, full light curve"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def timed(fn, flush, stream, reps=5):
    """Median CUDA-event time (ms) of fn() with an L2 flush before every repetition."""
    import torch
    fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return statistics.median(out)


def cnn_measurements(g, ctx, lc, periods, t_d, f_d, p_d, flush, stream, args):
    """Fold + CNN search on the same star, CNN and box scoring of 262,144 profiles, and the
    CNN vs box-SNR detection comparison at FPR = 1e-3 after a short training run."""
    import torch
    from paper_2312_02063_gb300 import train as tr
    peaks, src = measured_peaks()
    n = lc.times.shape[0]
    out = {}
    w = tr.init_weights(ctx.device, 1)
    score = torch.empty(len(periods), dtype=torch.float32, device=ctx.device)
    ms = timed(lambda: g.gpfc_search(ctx, t_d, f_d, p_d, NBINS, lc.t0, g.SCORER_CNN, score=score, weights=w),
               flush, stream)
    out["cnn_search"] = {"ms": ms, "periods_scored_per_s": len(periods) / (ms * 1e-3),
                         "folds_per_s": n * len(periods) / (ms * 1e-3),
                         "workload": "same star and grid as the main line, scorer = CNN"}
    npf = args.cnn_profiles
    prof, counts, _, _, _ = g.gpfc_synth_profiles(ctx, 20233204, 0, npf)
    sc = torch.empty(npf, dtype=torch.float32, device=ctx.device)
    ms = timed(lambda: g.gpfc_score_cnn(ctx, prof, w, counts, score=sc), flush, stream)
    flop = 3_056_128.0 * npf
    peak_tf = float(peaks.get("bf16_tflops", 1900.0))
    out["cnn_scoring"] = {"ms": ms, "profiles_per_s": npf / (ms * 1e-3), "tflops": flop / (ms * 1e-3) / 1e12,
                          "roofline": {"bound": "tensor", "achieved": flop / (ms * 1e-3) / 1e12, "peak": peak_tf,
                                       "unit": "TFLOP/s", "frac": flop / (ms * 1e-3) / 1e12 / peak_tf,
                                       "peak_basis": f"{src} bf16_tflops (burst)"},
                          "workload": f"{npf} folded 256-bin profiles (device-generated: half transits, half "
                                      "noise/sinusoid/eclipsing binary), FP32 in, BF16 tensor-core compute"}
    ms = timed(lambda: g.gpfc_score_box(ctx, prof, counts, 1, 32, 1.0, want_best=False), flush, stream)
    out["box_scoring"] = {"ms": ms, "profiles_per_s": npf / (ms * 1e-3),
                          "workload": f"same {npf} profiles, box widths 1..32"}
    if args.train_steps > 0:
        t_tr = time.perf_counter()
        wt, hist = tr.train(ctx, args.train_steps * 4096, batch=4096, lr=1e-3)
        t_tr = time.perf_counter() - t_tr
        res = tr.evaluate(ctx, wt, n_eval=args.eval_profiles, fpr=1e-3)
        out["detection"] = {"tpr_cnn": res["tpr_cnn"], "tpr_box": res["tpr_box"], "fpr": 1e-3,
                            "n_pos": res["n_pos"], "n_neg": res["n_neg"],
                            "train_profiles": args.train_steps * 4096, "train_s": t_tr, "final_loss": hist[-1][1],
                            "note": "training in the bench (Adam, lr 1e-3, batch 4096); the full training run is "
                                    "reported separately"}
        if args.star_count > 0:
            out["detection_star"] = star_detection(g, ctx, wt, args)
    if args.train_time_steps > 0:
        out["training"] = training_throughput(g, ctx, args, peaks, src)
    return out


def training_throughput(g, ctx, args, peaks, src):
    """Training steps of the C4 recipe (batch 4,096 profiles generated and folded on the GPU
    from 65,536-sample light curves, tensor-core forward and backward, Adam), timed with CUDA
    events after warm-up steps; the epoch time is the per-step time times 489 steps
    (2,000,000 profiles). Counted work per profile: forward 3,056,128 FLOP plus backward
    twice that (data generation not counted)."""
    import torch
    from paper_2312_02063_gb300 import train as tr
    t = tr.Trainer(ctx, batch=4096, lr=1e-3)
    for _ in range(3):
        t.step()
    ctx.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.train_time_steps):
        t.step()
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / args.train_time_steps
    # the same steps split: data generation alone, and forward + loss + backward + Adam on one
    # resident batch
    f, c, y, _, _ = g.gpfc_synth_profiles(ctx, tr.TRAIN_SEED, 0, 4096)
    a.record()
    for i in range(args.train_time_steps):
        g.gpfc_synth_profiles(ctx, tr.TRAIN_SEED, 4096 * (i + 1), 4096)
    b.record()
    b.synchronize()
    ms_gen = a.elapsed_time(b) / args.train_time_steps
    a.record()
    for _ in range(args.train_time_steps):
        logit, saved = g.gpfc_cnn_forward_train(ctx, f, t.params, c)
        _, dl = g.gpfc_bce_with_logits(ctx, logit, y)
        grads = g.gpfc_cnn_backward(ctx, dl, t.params, saved)
        for n in tr.CNN_PARAM_NAMES:
            g.gpfc_adam(ctx, t.params[n], grads[n], t.m[n], t.v[n], 10, 1e-3)
    b.record()
    b.synchronize()
    ms_model = a.elapsed_time(b) / args.train_time_steps
    flop = 3 * 3_056_128.0 * 4096
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
    tf = flop / (ms_model * 1e-3) / 1e12
    return {"ms_per_step": ms, "profiles_per_s": 4096 / (ms * 1e-3), "epoch_s_2M": ms * 1e-3 * (2_000_000 / 4096),
            "ms_data_generation": ms_gen, "ms_forward_backward_adam": ms_model, "model_tflops": tf,
            "roofline": {"bound": "tensor", "kernel": "forward + backward + Adam of one resident batch",
                         "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "peak_basis": f"{src} bf16_tflops_sustained"},
            "workload": "C4 training steps: 4,096 profiles per step generated and folded on the GPU from "
                        "65,536-sample light curves, BF16 tensor-core forward and backward, BCE, Adam",
                        "steps_timed": args.train_time_steps}


def star_detection(g, ctx, weights, args):
    """Star-level detection (Sec. 3.2, Figs. 10-13): labelled stars (half with one injected
    transit, half noise only) searched by gpfc_search_batched at several grid densities with
    each scorer; a star's score is its best period's score (CNN, box-SNR) or the SDE of its
    box-SNR periodogram (Eq. 3). ROC statistics come from gpfc_roc. The equal-accuracy entry
    compares the detectors' throughput at the smallest tested density where each reaches
    the same TPR at FPR 1e-3."""
    import torch
    import lcsynth
    from paper_2312_02063_gb300 import train as tr
    ds = lcsynth.detection_stars(args.star_count)
    S = len(ds.label)
    dev = ctx.device
    lc, t, f = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (ds.lc_offsets, ds.times, ds.flux))
    t0s = torch.zeros(S, dtype=torch.float64, device=dev)
    pos = torch.from_numpy(np.nonzero(ds.label == 1)[0]).to(dev)
    neg = torch.from_numpy(np.nonzero(ds.label == 0)[0]).to(dev)
    fprs = [1e-3, 1e-2, 1e-1]
    lens = np.diff(ds.lc_offsets)
    out = {"workload": f"{S} stars ({int(len(pos))} with one injected box, SNR 4-16 by Eq. 2; {int(len(neg))} noise "
                       f"only), {lens.min()}..{lens.max()} samples at 29.4 min with two 1-5 d gaps, white noise "
                       "1e-4..1e-3, periods 0.2-1 d; per-star frequency grids over [1, 5] c/d, 256 bins",
           "fprs": fprs, "rows": []}
    for P in args.star_densities:
        grid = torch.from_numpy(lcsynth.freq_grid(P)).to(dev)
        periods = grid.repeat(S)
        goff = torch.arange(S + 1, dtype=torch.int64, device=dev) * P
        score = torch.empty(S * P, dtype=torch.float32, device=dev)
        bi = torch.empty(S, dtype=torch.int64, device=dev)
        bs = torch.empty(S, dtype=torch.float32, device=dev)
        row = {"n_periods": P, "folds": float(np.sum(lens.astype(np.float64)) * P)}
        for name, scorer, kw in (("box", g.SCORER_BOX, {"w_max": tr.BOX_W_MAX}), ("cnn", g.SCORER_CNN, {"weights": weights})):
            def run():
                g.gpfc_search_batched(ctx, lc, t, f, goff, periods, NBINS, t0s, scorer, score=score, best_index=bi,
                                      best_score=bs, **kw)
            run()
            ctx.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run()
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b)
            row[name] = {"ms": ms, "stars_per_s": S / (ms * 1e-3), "folds_per_s": row["folds"] / (ms * 1e-3)}
            dets = {name + "_max": bs.clone()}
            sm, _ = g.peaks_to_numpy(*g.gpfc_peaks(ctx, score, periods, goff, max_peaks=0), 0)
            dets[name + "_sde"] = torch.from_numpy(np.ascontiguousarray(sm["sde"], np.float32)).to(dev)
            for dn, sc in dets.items():
                u2, thr, tp = g.gpfc_roc(ctx, sc[pos], sc[neg], fprs)
                ctx.sync()
                row[dn] = {"auc": int(u2.item()) / (2.0 * len(pos) * len(neg)),
                           "tpr": [int(v) / len(pos) for v in tp.cpu().numpy()]}
        out["rows"].append(row)
    # each scorer on one fold per star: injected stars at their true period, noise-only stars
    # at a seeded random period of the same range (profile quality without the look-elsewhere
    # of a periodogram)
    rnd = np.random.default_rng(1).uniform(0.2, 1.0, S)
    one = torch.from_numpy(np.where(ds.label == 1, ds.period, rnd)).to(dev)
    goff1 = torch.arange(S + 1, dtype=torch.int64, device=dev)
    s1 = torch.empty(S, dtype=torch.float32, device=dev)
    out["one_period"] = {}
    for name, scorer, kw in (("box", g.SCORER_BOX, {"w_max": tr.BOX_W_MAX}), ("cnn", g.SCORER_CNN, {"weights": weights})):
        g.gpfc_search_batched(ctx, lc, t, f, goff1, one, NBINS, t0s, scorer, score=s1, **kw)
        u2, thr, tp = g.gpfc_roc(ctx, s1[pos], s1[neg], fprs)
        ctx.sync()
        out["one_period"][name] = {"auc": int(u2.item()) / (2.0 * len(pos) * len(neg)),
                                   "tpr": [int(v) / len(pos) for v in tp.cpu().numpy()]}
    # equal accuracy: the better CNN detector against the better box detector at the densest grid
    last = out["rows"][-1]
    box = "box_sde" if last["box_sde"]["auc"] >= last["box_max"]["auc"] else "box_max"
    cnn = "cnn_sde" if last["cnn_sde"]["auc"] >= last["cnn_max"]["auc"] else "cnn_max"
    tpr = {d: [r[d]["tpr"][0] for r in out["rows"]] for d in (cnn, box)}
    target = min(max(tpr[cnn]), max(tpr[box]))
    eq = {"target_tpr_at_fpr_1e-3": target, "box_detector": box, "cnn_detector": cnn}
    for d, key in ((cnn, "cnn"), (box, "box")):
        k = next(i for i, v in enumerate(tpr[d]) if v >= target)
        r = out["rows"][k]
        eq[d] = {"n_periods": r["n_periods"], "stars_per_s": r[key]["stars_per_s"], "tpr": tpr[d][k]}
    eq["cnn_over_box_throughput"] = eq[cnn]["stars_per_s"] / eq[box]["stars_per_s"]
    out["equal_accuracy"] = eq
    return out


def batched_measurements(g, ctx, flush, stream, args):
    """Many-star search: stars of 8,192-70,000 samples with gaps, each with its own grid of
    20,000-250,000 periods, 256 bins, CNN (and box-SNR) scorer. The batched call (one
    graph-captured launch sequence, autotuned fold) against a loop of single-star calls."""
    import torch
    import lcsynth
    from paper_2312_02063_gb300 import train as tr
    sb = lcsynth.star_batch(n_stars=args.batch_stars)
    dev = ctx.device
    d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in
         (sb.lc_offsets, sb.times, sb.flux, sb.grid_offsets, sb.periods, sb.t0s)]
    S = args.batch_stars
    lens = np.diff(sb.lc_offsets)
    grids = np.diff(sb.grid_offsets)
    folds = float(np.sum(lens.astype(np.float64) * grids))
    npt = int(sb.grid_offsets[-1])
    w = tr.init_weights(dev, 1)
    score = torch.empty(npt, dtype=torch.float32, device=dev)
    bi = torch.empty(S, dtype=torch.int64, device=dev)
    bs = torch.empty(S, dtype=torch.float32, device=dev)
    out = {"workload": f"{S} stars, N {lens.min()}..{lens.max()} samples (sum {int(lens.sum())}), "
                       f"grids {grids.min()}..{grids.max()} periods (sum {npt}), 256 bins",
           "sample_period_folds": folds}
    for name, scorer, kw in (("cnn", g.SCORER_CNN, {"weights": w}), ("box", g.SCORER_BOX, {"w_max": W_MAX})):
        def run_batched():
            g.gpfc_search_batched(ctx, d[0], d[1], d[2], d[3], d[4], NBINS, d[5], scorer, score=score,
                                  best_index=bi, best_score=bs, **kw)
        per = [(int(sb.lc_offsets[s]), int(sb.lc_offsets[s + 1]), int(sb.grid_offsets[s]),
                int(sb.grid_offsets[s + 1])) for s in range(S)]
        bi1 = torch.empty(1, dtype=torch.int64, device=dev)
        bs1 = torch.empty(1, dtype=torch.float32, device=dev)

        def run_loop():
            for (a, b, c, e) in per:
                g.gpfc_search(ctx, d[1][a:b], d[2][a:b], d[4][c:e], NBINS, 0.0, scorer, score=score[c:e],
                              best_index=bi1, best_score=bs1, **kw)
        ms_b = timed(run_batched, flush, stream, reps=2)
        ms_l = timed(run_loop, flush, stream, reps=2)
        plan = ctx.last_fold_plan()
        out[name] = {"batched_ms": ms_b, "unbatched_ms": ms_l, "speedup": ms_l / ms_b,
                     "stars_per_s": S / (ms_b * 1e-3), "periods_per_s": npt / (ms_b * 1e-3),
                     "folds_per_s": folds / (ms_b * 1e-3),
                     "unbatched_stars_per_s": S / (ms_l * 1e-3), "unbatched_periods_per_s": npt / (ms_l * 1e-3)}
        # the plan of the batched call (the loop's last call may differ)
        run_batched()
        out[name]["fold_plan"] = ctx.last_fold_plan()
    ctx.sync()
    return out


def paper_fold_and_decision(g, ctx, lc, periods, t_d, f_d, p_d, score, flush, stream):
    """The paper's two-tier equal-count fold (4096 fine bins -> 256 bins of n/256 samples)
    on the same star and grid, and the per-star decision (SDE, peak rule, harmonics) over
    the box-SNR periodogram of the main step."""
    import torch
    n = lc.times.shape[0]
    out = torch.empty((len(periods), NBINS), dtype=torch.float32, device=ctx.device)
    ms = timed(lambda: g.gpfc_fold_equal_count(ctx, t_d, f_d, p_d, NBINS, 4096, lc.t0, out), flush, stream)
    res = {"two_tier_fold": {"ms": ms, "folds_per_s": n * len(periods) / (ms * 1e-3),
                             "workload": f"same star and grid, 4096 fine bins merged into {NBINS} equal-count bins"}}
    ms = timed(lambda: g.gpfc_peaks(ctx, score, p_d), flush, stream)
    sm, pk = g.peaks_to_numpy(*g.gpfc_peaks(ctx, score, p_d), 8)
    ctx.sync()
    bi = int(sm[0]["best_index"])
    res["decision"] = {"ms": ms, "sde": float(sm[0]["sde"]), "n_peaks": int(sm[0]["n_peaks"]),
                       "best_period_d": float(periods[bi]) if bi >= 0 else None,
                       "injected_period_d": float(lc.truth["period"]) if hasattr(lc, "truth") and
                       lc.truth and "period" in lc.truth else None,
                       "harmonics": [int(h) for h in pk[0]["harmonic"][: int(sm[0]["n_listed"])]],
                       "workload": "box-SNR periodogram of the main step: SDE, peaks above mean + 3 sd wider "
                                   "than 3 periods, harmonic flags"}
    return res


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2312_02063_gb300 as g

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = g.Context(local_rank)
    lc, periods = make_inputs()
    n = lc.times.shape[0]
    t_d = torch.from_numpy(lc.times).to(dev)
    f_d = torch.from_numpy(lc.flux).to(dev)
    p_d = torch.from_numpy(periods).to(dev)
    score = torch.empty(N_PERIODS, dtype=torch.float32, device=dev)
    bi = torch.empty(1, dtype=torch.int64, device=dev)
    bs = torch.empty(1, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the default path: from 256 bins the reduction fold (exact fixed-point sums, twelve
    # warps per SM) pipelined with the warp-per-profile box-SNR scorer on two side streams
    ctx.set_box_path(g.BOX_AUTO)

    def step():
        g.gpfc_search(ctx, t_d, f_d, p_d, NBINS, lc.t0, g.SCORER_BOX, 1, W_MAX, 0.0, score, bi, bs)

    clocks = ClockSampler(local_rank)
    clocks.start()  # running before the timed region begins
    for _ in range(max(3, args.warmup)):
        step()
    ctx.sync()
    ctx.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    fold_ms, fold_launches = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps, outside the events
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        kernel_ms.append(ctx.kernel_time_ms())
        fms, fl = ctx.fold_launch_times()
        fold_ms.append(fms)
        fold_launches.append(fl)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks.end()
    clk = clocks.stop()
    ctx.set_timing(False)
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist:
        total_ms = max_over_ranks(total_ms, dist, dev)
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = job_rate(world, n * N_PERIODS, ms_per_step)

    # end to end through host buffers: H2D of the step's inputs, the C-ABI call, D2H of
    # the periodogram and the best period
    th = torch.from_numpy(lc.times).pin_memory()
    fh = torch.from_numpy(lc.flux).pin_memory()
    ph = torch.from_numpy(periods).pin_memory()
    sh = torch.empty(N_PERIODS, dtype=torch.float32).pin_memory()
    bih = torch.empty(1, dtype=torch.int64).pin_memory()
    bsh = torch.empty(1, dtype=torch.float32).pin_memory()
    e2e_ms = []
    for k in range(args.steps + 2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        t_d.copy_(th, non_blocking=True)
        f_d.copy_(fh, non_blocking=True)
        p_d.copy_(ph, non_blocking=True)
        step()
        sh.copy_(score, non_blocking=True)
        bih.copy_(bi, non_blocking=True)
        bsh.copy_(bs, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= 2:
            e2e_ms.append(a.elapsed_time(b))
    ctx.sync()
    e2e_value = job_rate(world, n * N_PERIODS, max_over_ranks(statistics.mean(e2e_ms), dist, dev))
    h2d = th.numel() * 8 + fh.numel() * 4 + ph.numel() * 8
    d2h = sh.numel() * 4 + 8 + 4

    result = None
    if rank == 0:
        peaks, src = measured_peaks()
        smax = float(peaks.get("sm_max_mhz", 2070.0))
        sms = ctx.num_sms
        model_gups = sms * SM_FOLD_UPDATES_PER_CLK * smax * 1e6 / 1e9
        # the fold's binding pipe, measured here: lane-private shared-memory updates of the
        # fold's 8-byte bin record at full occupancy (16 warps x 32 bins per SM), as two
        # no-return reductions (the default fold's record) and as a 64-bit read-modify-write
        # (the FP32 layout's record), and both at the fold's own footprint (256 bins x 3
        # period groups per SM)
        probe = {}
        for key, cfg, op in (("red8_full", (8, 32, 16, 1), 1), ("red8_fold_footprint", (8, 256, 3, 1), 1),
                             ("rmw8_full", (8, 32, 16, 1), 0), ("rmw8_fold_footprint", (8, 256, 3, 1), 0)):
            ups, upc = g.gpfc_probe_smem_rmw(*cfg, iters=20000, op=op)
            probe[key] = {"gupdates_per_s": ups / 1e9, "updates_per_clk_sm": upc,
                          "config": f"{cfg[0]}-byte record, {'two 32-bit reductions' if op else 'load + store'}, "
                                    f"{cfg[1]} bins x {cfg[2]} warps per SM"}
        peak_gups = probe["red8_full"]["gupdates_per_s"]
        kmean = statistics.mean(kernel_ms)
        # the search kernel's own launch (fold + box-SNR): all n * N_PERIODS updates of a step
        # over its duration
        fold_step_ms = statistics.mean(fold_ms)
        launches = fold_launches[0]
        achieved = n * N_PERIODS / (fold_step_ms * 1e-3) / 1e9
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, dt = cpu_oracle_rate(lc, periods, args.cpu_periods)
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_periods} random periods of the grid, full light curve, "
                             f"fold + box-SNR, {dt:.1f} s"}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/f32", "data": "synthetic",
            "config": {"workload": workload_name(n), "n_samples": n, "n_periods": N_PERIODS,
                       "nbins": NBINS, "w_min": 1, "w_max": W_MAX,
                       "l2": "flushed between timed steps (256 MB write outside the events)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "periods_scored_per_s": world * N_PERIODS / (ms_per_step * 1e-3),
            "roofline": {"bound": "smem", "kernel": "fold_kernel (reduction layout, 3 period groups, 12 sample streams across them)",
                         "achieved": achieved,
                         "peak": peak_gups, "unit": "Gupdates/s", "frac": achieved / peak_gups,
                         "traffic": None if SEARCH_DRAM_BYTES_PER_PERIOD is None
                         else SEARCH_DRAM_BYTES_PER_PERIOD * N_PERIODS / launches,
                         "traffic_basis": "per fold launch: ncu dram__bytes_read+write of the fold launches of "
                                          "one 250,000-period search in steady state (no cache flush), scaled "
                                          "by periods and divided by the launches of a step",
                         "kernel_ms": fold_step_ms / launches, "launches_per_step": launches,
                         "search_ms": kmean,
                         "peak_basis": "measured in this run by gpfc_probe_smem_rmw: lane-private updates of "
                                       "the fold's 8-byte record (32-bit sum and count words) by two "
                                       "red.shared.add.u32, 16 warps x 32 bins per SM, "
                                       f"{probe['red8_full']['updates_per_clk_sm']:.2f} updates/clk/SM",
                         "peak_model": model_gups,
                         "peak_model_basis": f"{sms} SMs x {SM_FOLD_UPDATES_PER_CLK} updates/clk (128 B/clk over "
                                             f"8 B of reductions per update) x {smax:.0f} MHz ({src} sm_max_mhz)",
                         "probe": probe},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.mean(e2e_ms)},
            # per step: 4 prep kernels, each fold launch and its box-SNR launch, the argmax
            "gpu_launches": (5 + 2 * launches) * args.steps,
            "clocks": clk,
            "wall_s_timed": wall,
        }
        if not args.no_cnn:
            result.update(cnn_measurements(g, ctx, lc, periods, t_d, f_d, p_d, flush, stream, args))
        if not args.no_cnn:
            result.update(paper_fold_and_decision(g, ctx, lc, periods, t_d, f_d, p_d, score, flush, stream))
        if args.batch_stars > 0:
            result["batched"] = batched_measurements(g, ctx, flush, stream, args)
        print(json.dumps(result), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpfc", choices=["gpfc", "reference"])
    ap.add_argument("--cpu-periods", type=int, default=6000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-periods", type=int, default=N_PERIODS)
    ap.add_argument("--no-cnn", action="store_true", help="skip the CNN and detection measurements")
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--star-count", type=int, default=20000, help="labelled stars of the star-level comparison (0: skip)")
    ap.add_argument("--train-time-steps", type=int, default=50, help="timed training steps (0: skip)")
    ap.add_argument("--star-densities", type=int, nargs="+", default=[2000, 5000, 10000, 20000])
    ap.add_argument("--cnn-profiles", type=int, default=262_144)
    ap.add_argument("--eval-profiles", type=int, default=40_000)
    ap.add_argument("--batch-stars", type=int, default=64,
                    help="stars of the many-star search measurement (0: skip)")
    args = ap.parse_args()
    globals()["N_PERIODS"] = args.n_periods
    rank, world, local_rank = env_rank()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
