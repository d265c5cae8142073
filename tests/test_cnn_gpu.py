"""GPU parity of the CNN scorer (tcgen05 forward) against the FP64 oracle.

Tolerance: scores within 2e-2 absolute and >= 99.9% agreement of the above/below 0.5
decisions; the logits are also checked against a BF16-scale bound.
"""
import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu

SCORE_ATOL = 2e-2


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def dev_weights(ctx, w):
    return {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(ctx.device) for k, v in w.items()}


def scaled_weights(seed, fc2_scale):
    w = lcsynth.cnn_init(seed, bias_scale=0.05)
    w["fc2.w"] = lcsynth.round_to_bf16(w["fc2.w"] * fc2_scale)
    return w


def run(ctx, prof, w, counts=None):
    import paper_2312_02063_gb300 as g
    f = torch.from_numpy(prof).to(ctx.device)
    c = None if counts is None else torch.from_numpy(counts).to(ctx.device)
    wd = dev_weights(ctx, w)
    z = g.gpfc_cnn_logits(ctx, f, wd, c)
    s = g.gpfc_score_cnn(ctx, f, wd, c)
    ctx.sync()
    return z.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,seed,scale", [(4096, 1, 0.25), (1001, 2, 1.0), (3, 3, 0.25), (1, 4, 0.25)])
def test_cnn_scores_match_oracle(ctx, n, seed, scale):
    prof, _ = lcsynth.profiles_mixed(n, seed=seed)
    w = scaled_weights(seed, scale)
    z, s = run(ctx, prof, w)
    zo, so = oracle.cnn_score(w, prof)
    assert np.max(np.abs(s - so)) <= SCORE_ATOL, np.max(np.abs(s - so))
    flip = (s > 0.5) != (so > 0.5)
    if n >= 1000:
        assert np.mean(~flip) >= 0.999, np.mean(~flip)
    else:
        # one to three profiles: a flip is allowed only at a tie, within 1e-3 of 0.5
        assert np.all(np.abs(so[flip] - 0.5) < 1e-3), so[flip]
    np.testing.assert_allclose(1 / (1 + np.exp(-z)), s, atol=1e-6)
    assert np.max(np.abs(z - zo)) <= 0.05 * (1 + np.max(np.abs(zo)))


def test_cnn_empty_bins_by_counts_and_nan(ctx):
    prof, _ = lcsynth.profiles_mixed(300, seed=9)
    rng = np.random.default_rng(9)
    counts = rng.integers(0, 5, prof.shape).astype(np.int32)
    w = scaled_weights(9, 0.25)
    _, s = run(ctx, prof, w, counts)
    _, so = oracle.cnn_score(w, prof, counts)
    assert np.max(np.abs(s - so)) <= SCORE_ATOL
    pn = np.where(counts > 0, prof, np.nan).astype(np.float32)
    _, s2 = run(ctx, pn, w)
    assert np.max(np.abs(s2 - so)) <= SCORE_ATOL


def test_cnn_degenerate_profiles(ctx):
    w = scaled_weights(11, 0.25)
    prof = np.ones((4, 256), np.float32)
    prof[1] = np.nan            # every bin empty: input 0
    prof[2, ::2] = np.nan       # constant over the non-empty bins: input m
    prof[3] = 0.9993
    _, s = run(ctx, prof, w)
    _, so = oracle.cnn_score(w, prof)
    assert np.max(np.abs(s - so)) <= SCORE_ATOL


def test_search_with_cnn_scorer_matches_fold_then_score(ctx):
    # fused search (chunked fold -> CNN) equals the two-step path, and the oracle on samples
    import paper_2312_02063_gb300 as g
    lc = lcsynth.light_curve_kepler(seed=77, n_cad=20000)
    periods = lcsynth.freq_grid(45_000)  # more than one fold wave: several chunks
    w = scaled_weights(31, 0.25)
    wd = dev_weights(ctx, w)
    t = torch.from_numpy(lc.times).to(ctx.device)
    f = torch.from_numpy(lc.flux).to(ctx.device)
    p = torch.from_numpy(periods).to(ctx.device)
    sc, bi, bs = g.gpfc_search(ctx, t, f, p, 256, lc.t0, g.SCORER_CNN, weights=wd)
    fo, co = g.gpfc_fold(ctx, t, f, p, 256, lc.t0)
    s2 = g.gpfc_score_cnn(ctx, fo, wd, co)
    ctx.sync()
    sc, s2 = sc.cpu().numpy(), s2.cpu().numpy()
    assert np.array_equal(sc, s2)
    assert int(bi.item()) == int(np.argmax(sc)) and float(bs.item()) == sc.max()
    idx = np.random.default_rng(0).choice(len(periods), 40, replace=False)
    mean_o, cnt_o, _ = oracle.fold(lc.times, lc.flux, periods[idx], 256, lc.t0)
    _, so = oracle.cnn_score(w, mean_o.astype(np.float32), cnt_o.astype(np.int32))
    assert np.max(np.abs(sc[idx] - so)) <= SCORE_ATOL


def test_cnn_full_size_batch_sampled(ctx):
    """The full inference batch (262,144 profiles of 256 bins, the scoring benchmark's
    size and launch path): 300 sampled profiles against the FP64 oracle, and the scores of
    a repeated call identical."""
    import paper_2312_02063_gb300 as g
    n = 262144
    prof, counts, _, _, _ = g.gpfc_synth_profiles(ctx, 20233204, 0, n)
    w = scaled_weights(11, 0.25)
    wd = dev_weights(ctx, w)
    s = g.gpfc_score_cnn(ctx, prof, wd, counts)
    s2 = g.gpfc_score_cnn(ctx, prof, wd, counts)
    ctx.sync()
    s, s2 = s.cpu().numpy(), s2.cpu().numpy()
    assert np.array_equal(s, s2)
    idx = np.unique(np.concatenate([np.random.default_rng(5).choice(n, 296, replace=False), [0, 1, n - 2, n - 1]]))
    pf = prof[torch.from_numpy(idx).to(ctx.device)].cpu().numpy()
    pc = counts[torch.from_numpy(idx).to(ctx.device)].cpu().numpy()
    _, so = oracle.cnn_score(w, pf, pc)
    assert np.max(np.abs(s[idx] - so)) <= SCORE_ATOL
    flip = (s[idx] > 0.5) != (so > 0.5)
    print(f"full batch: {flip.sum()} decision flips at 0.5 in {len(idx)} sampled profiles, oracle scores "
          f"{so[flip]}")
    # 300 samples resolve 99.9% agreement only as 'no flip': a flip is allowed only at a
    # tie, within 1e-3 of 0.5 (the agreement itself is measured on 20,000 profiles in
    # test_cnn_trained_gpu.py)
    assert np.all(np.abs(so[flip] - 0.5) < 1e-3), so[flip]
