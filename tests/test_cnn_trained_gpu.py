"""GPU parity of the CNN scorer at trained weights (Sec. 2.5), against the FP64 oracle.

The other CNN parity tests use random-init weights, whose scores sit near 0.5. The
detection numbers come from trained networks, whose scores spread over (0, 1), so this
test trains the network for a few dozen Adam steps with the library's own training path
(train.train) and then scores 20,000 held-out profiles of the training recipe on the GPU
and in the oracle:

* every score within 2e-2 absolute of the oracle's;
* >= 99.9% agreement of the above/below decisions at 0.5 and at the threshold that gives
  a false-positive rate of 1e-3 on the oracle's scores of the negatives (the operating
  point of the detection comparison).

Both sides see the same parameters: weights rounded once to BF16 (what the tensor cores
take), biases in FP32 (what the kernels add).
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu

SCORE_ATOL = 2e-2
AGREE = 0.999
N_EVAL = 20_000
FPR = 1e-3


def oracle_scores(w, prof, counts):
    """oracle.cnn_score over chunks on all host cores (its C loop runs with the GIL released)."""
    workers = max(1, min(os.cpu_count() or 1, 32))
    parts = [ix for ix in np.array_split(np.arange(len(prof)), workers) if len(ix)]
    with cf.ThreadPoolExecutor(len(parts)) as ex:
        res = list(ex.map(lambda ix: oracle.cnn_score(w, prof[ix], counts[ix]), parts))
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])


@pytest.fixture(scope="module")
def trained():
    import paper_2312_02063_gb300 as g
    from paper_2312_02063_gb300 import train
    ctx = g.Context(0)
    w, hist = train.train(ctx, 96 * 4096, batch=4096, lr=1e-3, seed=3, log_every=95)
    wb = {n: (lcsynth.round_to_bf16(t.cpu().numpy()) if n.endswith(".w") else t.cpu().numpy().astype(np.float32))
          for n, t in w.items()}
    f, c, y, _, _ = g.gpfc_synth_profiles(ctx, train.EVAL_SEED, 0, N_EVAL)
    wd = {n: torch.from_numpy(v).to(ctx.device) for n, v in wb.items()}
    s = g.gpfc_score_cnn(ctx, f, wd, c)
    z = g.gpfc_cnn_logits(ctx, f, wd, c)
    ctx.sync()
    out = dict(w=wb, hist=hist, prof=f.cpu().numpy(), counts=c.cpu().numpy(), label=y.cpu().numpy(),
               s=s.cpu().numpy().astype(np.float64), z=z.cpu().numpy().astype(np.float64))
    out["zo"], out["so"] = oracle_scores(wb, out["prof"], out["counts"])
    ctx.close()
    return out


def test_training_moved_the_scores_off_one_half(trained):
    # the network is trained: the loss fell and the scores are spread, so the comparison
    # below covers saturated scores as well as the region around 0.5
    (_, l0), (_, l1) = trained["hist"][0], trained["hist"][-1]
    assert l1 < 0.9 * l0, trained["hist"]
    so = trained["so"]
    assert np.mean(np.abs(so - 0.5) > 0.4) > 0.1, np.percentile(so, [5, 25, 50, 75, 95])


def test_trained_scores_match_oracle(trained):
    s, so = trained["s"], trained["so"]
    err = np.abs(s - so)
    print(f"trained CNN: max |score - oracle| = {err.max():.3e}, mean {err.mean():.3e}, "
          f"max |logit - oracle| = {np.max(np.abs(trained['z'] - trained['zo'])):.3e}")
    assert err.max() <= SCORE_ATOL, err.max()


def test_trained_decisions_agree_at_half_and_at_fpr_1e3(trained):
    s, so, y = trained["s"], trained["so"], trained["label"]
    pos, neg = y > 0.5, y < 0.5
    assert neg.sum() >= 0.4 * N_EVAL and pos.sum() >= 0.4 * N_EVAL
    _, thr = oracle.tpr_at_fpr(so[pos], so[neg], FPR)
    for t in (0.5, thr):
        agree = float(np.mean((s > t) == (so > t)))
        print(f"threshold {t:.9f}: decision agreement {agree:.5f}")
        assert agree >= AGREE, (t, agree)
    # the GPU's own operating point detects what the oracle's does, to the same tolerance
    tpr_o, _ = oracle.tpr_at_fpr(so[pos], so[neg], FPR)
    tpr_g, _ = oracle.tpr_at_fpr(s[pos], s[neg], FPR)
    assert abs(tpr_g - tpr_o) <= 1e-2, (tpr_g, tpr_o)
