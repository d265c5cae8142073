"""GPU parity of the CNN training path (backward, loss, Adam) against the FP64 oracle.

The oracle's FP64 gradient is itself pinned to central finite differences on the CPU
(tests/test_oracle_cnn.py). GPU gradients come from the tensor-core forward (BF16
weights, activations carried as two BF16 terms, FP32 accumulation) and a backward whose
contractions are BF16 tensor-core GEMMs with FP32 accumulation, so they are compared by
cosine similarity (>= 0.999) and relative L2 error per parameter tensor: at most
GRAD_REL = 2e-2 (the gradient tolerance of the scope table) and, as a regression bound,
at most GRAD_REGRESSION = 2e-3 per tensor (measured: <= 8.4e-4 for the conv and fc1
weights, below 1e-5 for fc2 and fc1's bias).
"""
import numpy as np
import pytest
import torch

import lcsynth
import oracle

pytestmark = pytest.mark.gpu

GRAD_COS = 0.999
GRAD_REL = 2e-2
GRAD_REGRESSION = 2e-3


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _dev(ctx, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device)


def test_gradients_match_fp64_oracle(ctx):
    import paper_2312_02063_gb300 as g
    B = 384
    prof, lab = lcsynth.profiles_mixed(B, seed=21)
    w = lcsynth.cnn_init(21, bias_scale=0.05)
    w["fc2.w"] = lcsynth.round_to_bf16(w["fc2.w"] * 0.25)
    wd = {k: _dev(ctx, v) for k, v in w.items()}
    y = lab.astype(np.float32)
    logit, saved = g.gpfc_cnn_forward_train(ctx, _dev(ctx, prof), wd)
    loss, dlogit = g.gpfc_bce_with_logits(ctx, logit, _dev(ctx, y))
    grads = g.gpfc_cnn_backward(ctx, dlogit, wd, saved)
    ctx.sync()
    x = oracle.cnn_normalise(prof)
    loss_o, grads_o, _ = oracle.cnn_loss_backward(w, x, y)
    assert abs(float(loss.item()) - loss_o) <= 2e-2 * max(1.0, abs(loss_o))
    stats = {}
    for n in oracle.CNN_NAMES:
        a = grads[n].cpu().numpy().astype(np.float64).ravel()
        b = grads_o[n].ravel()
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))
        rel = float(np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300))
        stats[n] = (round(cos, 7), float(f"{rel:.3g}"))
    print("gradient cosine / relative L2 vs FP64 oracle:", stats)
    for n, (cos, rel) in stats.items():
        assert cos >= GRAD_COS and rel <= GRAD_REL, (n, stats)
        assert rel <= GRAD_REGRESSION, (n, stats)


def test_autograd_function_matches_direct_calls(ctx):
    import paper_2312_02063_gb300 as g
    B = 130
    prof, lab = lcsynth.profiles_mixed(B, seed=22)
    w = lcsynth.cnn_init(22, bias_scale=0.05)
    params = [_dev(ctx, w[n]).requires_grad_(True) for n in g.CNN_PARAM_NAMES]
    f = _dev(ctx, prof)
    z = g.CNNFunction.apply(ctx, f, None, *params)
    yt = _dev(ctx, lab.astype(np.float32))
    loss = torch.nn.functional.binary_cross_entropy_with_logits(z, yt)
    loss.backward()
    wd = {n: p.detach() for n, p in zip(g.CNN_PARAM_NAMES, params)}
    logit, saved = g.gpfc_cnn_forward_train(ctx, f, wd)
    _, dlogit = g.gpfc_bce_with_logits(ctx, logit, yt)
    grads = g.gpfc_cnn_backward(ctx, dlogit, wd, saved)
    ctx.sync()
    for n, p in zip(g.CNN_PARAM_NAMES, params):
        np.testing.assert_allclose(p.grad.cpu().numpy(), grads[n].cpu().numpy(), rtol=1e-4, atol=1e-7)


def test_backward_is_deterministic(ctx):
    import paper_2312_02063_gb300 as g
    prof, lab = lcsynth.profiles_mixed(200, seed=23)
    wd = {k: _dev(ctx, v) for k, v in lcsynth.cnn_init(23).items()}
    out = []
    for _ in range(2):
        logit, saved = g.gpfc_cnn_forward_train(ctx, _dev(ctx, prof), wd)
        _, dl = g.gpfc_bce_with_logits(ctx, logit, _dev(ctx, lab.astype(np.float32)))
        out.append(g.gpfc_cnn_backward(ctx, dl, wd, saved))
    ctx.sync()
    for n in g.CNN_PARAM_NAMES:
        assert torch.equal(out[0][n], out[1][n]), n


def test_adam_matches_oracle(ctx):
    import paper_2312_02063_gb300 as g
    rng = np.random.default_rng(5)
    p0 = rng.normal(0, 1, 1000).astype(np.float32)
    p, m, v = _dev(ctx, p0.copy()), torch.zeros(1000, device=ctx.device), torch.zeros(1000, device=ctx.device)
    po, mo, vo = p0.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for t in range(1, 6):
        gr = rng.normal(0, 1, 1000).astype(np.float32)
        g.gpfc_adam(ctx, p, _dev(ctx, gr), m, v, t, lr=1e-2)
        po, mo, vo = oracle.adam_step(po, gr, mo, vo, t, lr=1e-2)
    ctx.sync()
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=1e-5, atol=1e-6)


def test_training_resumes_bit_for_bit_from_a_checkpoint(ctx, tmp_path):
    """N + M steps equal N steps, a save to disk, a load into a new trainer and M steps:
    weights, Adam moments and the data-stream position carry over exactly."""
    from paper_2312_02063_gb300.train import Trainer
    a = Trainer(ctx, batch=256, lr=2e-3, seed=4)
    for _ in range(5):
        a.step()
    b = Trainer(ctx, batch=256, lr=2e-3, seed=4)
    for _ in range(3):
        b.step()
    path = str(tmp_path / "ckpt.pt")
    b.save(path)
    c = Trainer.load(ctx, path)
    for _ in range(2):
        c.step()
    sa, sc = a.state_dict(), c.state_dict()
    assert sa["steps"] == sc["steps"] == 5 and sa["next_index"] == sc["next_index"] == 5 * 256
    for part in ("params", "m", "v"):
        for n in sa[part]:
            assert torch.equal(sa[part][n], sc[part][n]), (part, n)
