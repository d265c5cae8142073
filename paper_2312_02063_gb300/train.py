"""Training and evaluation of the CNN scorer on device-generated folded profiles.

Everything on the data path runs in libgpfc's kernels: light curves are generated and
folded on the GPU (gpfc_synth_profiles), the network's forward and backward passes,
the loss and the Adam updates are the library's own kernels. The detection comparison
ranks held-out profiles by the CNN score and by the box-SNR statistic (in units of each
light curve's flux standard deviation, as gpfc_search defines it) and reports the
true-positive rate at a fixed false-positive rate.

  python -m paper_2312_02063_gb300.train --profiles 2000000 --batch 4096 --out run.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import (CNN_PARAM_NAMES, CNN_PARAM_SHAPES, Context, gpfc_adam, gpfc_bce_with_logits, gpfc_cnn_backward,
               gpfc_cnn_forward_train, gpfc_score_box, gpfc_score_cnn, gpfc_synth_profiles, gpfc_synth_vectors)

TRAIN_SEED = 20234204
EVAL_SEED = 20234999
PAPER_SEED = 20236207      # the paper-recipe set: 2,000,000 vectors split 80/10/10 by index
PAPER_N = 2_000_000
BOX_W_MAX = 160   # widest transit of the training set: 3 h at P = 0.2 d is 0.625 of a cycle


def init_weights(device, seed: int = 1) -> dict:
    """He-uniform weights U(+-sqrt(6/fan_in)), zero biases, FP32 master copies."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    out = {}
    for n in CNN_PARAM_NAMES:
        shape = CNN_PARAM_SHAPES[n]
        if n.endswith(".b"):
            t = torch.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:]))
            lim = math.sqrt(6.0 / fan_in)
            t = (torch.rand(shape, generator=g) * 2 - 1) * lim
        out[n] = t.to(device=device, dtype=torch.float32).contiguous()
    return out


class Trainer:
    """Adam on BCE-with-logits over the device-generated training stream, with checkpoints.

    The state is the FP32 master weights, Adam's first and second moments, the number of
    Adam steps taken and the index of the next profile of the stream (profiles are
    generated by index, so the stream resumes exactly). Every kernel of a step is
    deterministic, so training N + M steps equals training N steps, saving, loading and
    training M steps, bit for bit.
    """

    def __init__(self, ctx: Context, batch: int = 4096, lr: float = 1e-3, seed: int = 1,
                 data_seed: int = TRAIN_SEED, weights: dict | None = None, recipe: str = "folded"):
        self.ctx = ctx
        self.batch = batch
        self.lr = lr
        self.data_seed = data_seed
        self.recipe = recipe  # "folded": light curves folded on the GPU; "paper": Sec. 2.7 vectors
        self.params = weights if weights is not None else init_weights(ctx.device, seed)
        self.m = {n: torch.zeros_like(p) for n, p in self.params.items()}
        self.v = {n: torch.zeros_like(p) for n, p in self.params.items()}
        self.steps = 0
        self.next_index = 0

    def step(self, nb: int | None = None):
        """One Adam step on the next nb (default: batch) profiles; returns the loss tensor."""
        nb = self.batch if nb is None else nb
        if self.recipe == "paper":
            f, y, _, _ = gpfc_synth_vectors(self.ctx, self.data_seed, self.next_index, nb)
            c = None
        else:
            f, c, y, _, _ = gpfc_synth_profiles(self.ctx, self.data_seed, self.next_index, nb)
        logit, saved = gpfc_cnn_forward_train(self.ctx, f, self.params, c)
        loss, dl = gpfc_bce_with_logits(self.ctx, logit, y)
        grads = gpfc_cnn_backward(self.ctx, dl, self.params, saved)
        self.steps += 1
        for n in CNN_PARAM_NAMES:
            gpfc_adam(self.ctx, self.params[n], grads[n], self.m[n], self.v[n], self.steps, self.lr)
        self.next_index += nb
        return loss

    def state_dict(self) -> dict:
        self.ctx.sync()
        return {"params": {n: t.detach().cpu().clone() for n, t in self.params.items()},
                "m": {n: t.detach().cpu().clone() for n, t in self.m.items()},
                "v": {n: t.detach().cpu().clone() for n, t in self.v.items()},
                "steps": self.steps, "next_index": self.next_index, "batch": self.batch, "lr": self.lr,
                "data_seed": self.data_seed, "recipe": self.recipe}

    def load_state_dict(self, sd: dict):
        dev = self.ctx.device
        self.params = {n: t.to(dev).contiguous() for n, t in sd["params"].items()}
        self.m = {n: t.to(dev).contiguous() for n, t in sd["m"].items()}
        self.v = {n: t.to(dev).contiguous() for n, t in sd["v"].items()}
        self.steps, self.next_index = int(sd["steps"]), int(sd["next_index"])
        self.batch, self.lr, self.data_seed = int(sd["batch"]), float(sd["lr"]), int(sd["data_seed"])
        self.recipe = sd.get("recipe", "folded")

    def save(self, path: str):
        torch.save(self.state_dict(), path)

    @classmethod
    def load(cls, ctx: Context, path: str) -> "Trainer":
        t = cls(ctx)
        t.load_state_dict(torch.load(path, map_location="cpu"))
        return t


def train(ctx: Context, n_profiles: int, batch: int = 4096, lr: float = 1e-3, seed: int = 1,
          data_seed: int = TRAIN_SEED, first: int = 0, weights: dict | None = None, log_every: int = 50,
          recipe: str = "folded"):
    """Adam on BCE-with-logits over n_profiles generated profiles (one pass, batch by batch).

    Returns (weights, history) where history lists (step, loss) every log_every steps.
    """
    tr = Trainer(ctx, batch, lr, seed, data_seed, weights, recipe)
    tr.next_index = first
    steps = (n_profiles + batch - 1) // batch
    hist = []
    for s in range(steps):
        loss = tr.step(min(batch, n_profiles - s * batch))
        if s % log_every == 0 or s == steps - 1:
            hist.append((s, float(loss.item())))
    ctx.sync()
    return tr.params, hist


def tpr_at_fpr(pos, neg, fpr):
    """TPR with the threshold at the (floor(fpr * n_neg) + 1)-th largest negative score."""
    neg = np.sort(np.asarray(neg, np.float64))[::-1]
    k = int(np.floor(fpr * len(neg)))
    thr = neg[k] if k < len(neg) else -np.inf
    return float(np.mean(np.asarray(pos, np.float64) > thr)), float(thr)


def evaluate(ctx: Context, weights: dict, n_eval: int = 200_000, seed: int = EVAL_SEED, fpr: float = 1e-3,
             chunk: int = 16384, w_max: int = BOX_W_MAX):
    """Held-out detection comparison: CNN score vs box-SNR at a fixed false-positive rate."""
    cnn, box, lab, kinds = [], [], [], []
    for j0 in range(0, n_eval, chunk):
        nb = min(chunk, n_eval - j0)
        f, c, y, _, sd = gpfc_synth_profiles(ctx, seed, j0, nb, want_std=True)
        s_cnn = gpfc_score_cnn(ctx, f, weights, c)
        s_box, _, _ = gpfc_score_box(ctx, f, c, 1, w_max, 1.0, want_best=False)
        cnn.append(s_cnn.cpu().numpy())
        box.append((s_box / sd).cpu().numpy())
        lab.append(y.cpu().numpy())
        j = np.arange(j0, j0 + nb)
        kinds.append(np.where(j % 2 == 0, 0, 1 + (j // 2) % 3))
    ctx.sync()
    cnn, box, lab, kinds = map(np.concatenate, (cnn, box, lab, kinds))
    pos, neg = lab > 0.5, lab < 0.5
    t_cnn, thr_cnn = tpr_at_fpr(cnn[pos], cnn[neg], fpr)
    t_box, thr_box = tpr_at_fpr(box[pos], box[neg], fpr)
    names = {1: "noise", 2: "sinusoid", 3: "eclipsing_binary"}
    fa = {names[k]: {"cnn": float(np.mean(cnn[kinds == k] > thr_cnn)), "box": float(np.mean(box[kinds == k] > thr_box))}
          for k in (1, 2, 3)}
    return {"fpr": fpr, "n_pos": int(pos.sum()), "n_neg": int(neg.sum()), "tpr_cnn": t_cnn, "tpr_box": t_box,
            "threshold_cnn": thr_cnn, "threshold_box": thr_box, "false_alarm_rate_by_kind": fa,
            "accuracy_cnn_at_0.5": float(np.mean((cnn > 0.5) == pos))}


def evaluate_paper(ctx: Context, weights: dict, first: int = int(0.9 * PAPER_N), n_eval: int = PAPER_N // 10,
                   seed: int = PAPER_SEED, fpr: float = 1e-3, chunk: int = 16384, w_max: int = 32):
    """Test split of the paper-recipe set: accuracy at a 0.5 threshold (the paper quotes
    94.0% for its own CNN, Sec. 2.7) and TPR at a fixed FPR for the CNN and for box-SNR (in
    units of each vector's noise)."""
    cnn, box, lab, alp = [], [], [], []
    for j0 in range(first, first + n_eval, chunk):
        nb = min(chunk, first + n_eval - j0)
        f, y, a, sb = gpfc_synth_vectors(ctx, seed, j0, nb)
        ones = torch.ones_like(f, dtype=torch.int32)
        s_cnn = gpfc_score_cnn(ctx, f, weights)
        s_box, _, _ = gpfc_score_box(ctx, f, ones, 1, w_max, 1.0, want_best=False)
        cnn.append(s_cnn.cpu().numpy())
        box.append((s_box / sb).cpu().numpy())
        lab.append(y.cpu().numpy())
        alp.append(a.cpu().numpy())
    ctx.sync()
    cnn, box, lab, alp = map(np.concatenate, (cnn, box, lab, alp))
    pos, neg = lab > 0.5, lab < 0.5
    t_cnn, thr_cnn = tpr_at_fpr(cnn[pos], cnn[neg], fpr)
    t_box, thr_box = tpr_at_fpr(box[pos], box[neg], fpr)
    return {"split": "test (last 10% of the 2M-vector set)", "n_pos": int(pos.sum()), "n_neg": int(neg.sum()),
            "accuracy_cnn_at_0.5": float(np.mean((cnn > 0.5) == pos)), "fpr": fpr, "tpr_cnn": t_cnn,
            "tpr_box": t_box, "threshold_cnn": thr_cnn, "threshold_box": thr_box}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profiles", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval", type=int, default=200_000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save", default=None, help="write the trained weights (torch.save of FP32 tensors)")
    ap.add_argument("--recipe", default="folded", choices=["folded", "paper"],
                    help="folded: light curves folded on the GPU (default); paper: the Sec. 2.7 vectors "
                         "(trains on the first 80%% of the 2M-vector set, tests on the last 10%%)")
    a = ap.parse_args()
    ctx = Context(0)
    t0 = time.time()
    w = None
    hist = []
    n_train = a.profiles if a.recipe == "folded" else min(a.profiles, int(0.8 * PAPER_N))
    data_seed = TRAIN_SEED if a.recipe == "folded" else PAPER_SEED
    for e in range(a.epochs):
        w, h = train(ctx, n_train, a.batch, a.lr, weights=w, data_seed=data_seed, recipe=a.recipe)
        hist += [(e, s, l) for s, l in h]
    t_train = time.time() - t0
    res = evaluate(ctx, w, a.eval) if a.recipe == "folded" else evaluate_paper(ctx, w)
    res["recipe"] = a.recipe
    res.update(train_profiles=n_train, epochs=a.epochs, batch=a.batch, lr=a.lr, train_seconds=t_train,
               loss_history=hist)
    print(json.dumps(res))
    if a.out:
        with open(a.out, "w") as fo:
            json.dump(res, fo, indent=1)
    if a.save:
        torch.save({n: t.cpu() for n, t in w.items()}, a.save)


if __name__ == "__main__":
    main()
