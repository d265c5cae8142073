"""The allocation-free best-period entry point gives the same answer as gpfc_best_period.

gpfc_best_period_noalloc serves callers that cannot allocate memory where they call it
(they cannot create a context either, since that allocates). It keeps its scratch in a
static device array, so this test checks two calls in a row (the second must not see the
first one's scratch) against the context-based entry point. It lives in a file of its own
that pytest collects last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_best_period_matches_context_entry_point_twice():
    import paper_2312_02063_gb300 as g
    ctx = g.Context(0)
    dev = ctx.device
    rng = np.random.default_rng(2024)
    a = rng.normal(0, 1, 250_001).astype(np.float32)
    a[[17, 123_456]] = 9.5          # tie: the smaller index wins
    b = rng.normal(0, 1, 3_001).astype(np.float32)
    b[2_999] = 4.0                  # smaller maximum than a's: a stale key would win
    b[5] = np.nan
    out_i = torch.empty(1, dtype=torch.int64, device=dev)
    out_s = torch.empty(1, dtype=torch.float32, device=dev)
    for arr in (a, b):
        s = torch.from_numpy(arr).to(dev)
        ref_i, ref_s = g.gpfc_best_period(ctx, s)
        g.gpfc_best_period_noalloc(s, out_i, out_s)
        torch.cuda.synchronize()
        ctx.sync()
        assert int(out_i.item()) == int(ref_i.item())
        assert float(out_s.item()) == float(ref_s.item())
        assert int(out_i.item()) == int(np.nanargmax(arr))
    ctx.close()


def test_noalloc_with_one_output_given():
    """Either output may be NULL: index only, then score only, each equal to the context
    entry point's answer."""
    import paper_2312_02063_gb300 as g
    ctx = g.Context(0)
    dev = ctx.device
    lib = g.load_library()
    rng = np.random.default_rng(7)
    a = torch.from_numpy(rng.normal(0, 1, 100_003).astype(np.float32)).to(dev)
    ref_i, ref_s = g.gpfc_best_period(ctx, a)
    ctx.sync()
    out_i = torch.full((1,), -7, dtype=torch.int64, device=dev)
    out_s = torch.full((1,), -7.0, dtype=torch.float32, device=dev)
    stream = g._vp(torch.cuda.current_stream(dev).cuda_stream)
    assert lib.gpfc_best_period_noalloc(g._ptr(a), a.numel(), g._ptr(out_i), None, stream) == 0
    torch.cuda.synchronize()
    assert int(out_i.item()) == int(ref_i.item()) and float(out_s.item()) == -7.0
    assert lib.gpfc_best_period_noalloc(g._ptr(a), a.numel(), None, g._ptr(out_s), stream) == 0
    torch.cuda.synchronize()
    assert float(out_s.item()) == float(ref_s.item())
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_limit():
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    bi = torch.empty(1, dtype=torch.int64, device="cuda")
    rc = lib.gpfc_best_period_noalloc(g._ptr(dummy), 2 ** 31, g._ptr(bi), None, None)
    assert rc == -1
    rc = lib.gpfc_best_period_noalloc(g._ptr(dummy), 0, g._ptr(bi), None, None)
    assert rc == -1
