"""GPU parity on a loud star (Sec. 2.3 step 3): a full-length light curve with white noise
of 1e-2, red noise of 2e-3 and a 1%-deep transit. The centred sums swing far more than on
the quiet Kepler-like star (the worst cancellation for FP32 partial sums), and the flux
range makes the fixed-point unit of the default 256-bin fold coarser than the float32
flux grid, so its rounding is real. Counts bit-exact, means within 1e-6 relative,
box-SNR within 1e-5 relative plus the fixed-point allowance of tolerances.py, through
gpfc_fold and through every box-search path at 256 bins.
"""
import numpy as np
import pytest
import torch

import lcsynth
import oracle
from tolerances import box_atol, fixed_point_unit

pytestmark = pytest.mark.gpu

MEAN_RTOL = 1e-6
BOX_RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_2312_02063_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _dev(ctx, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device)


@pytest.fixture(scope="module")
def loud_star():
    lc = lcsynth.light_curve_kepler(seed=990011, sigma_white=1e-2, ar_sigma=2e-3, depth_ppm=(10000.0, 10000.0),
                                    dur_h=(2.0, 3.0))
    grid = lcsynth.freq_grid(250_000)
    rng = np.random.default_rng(12)
    k_true = int(np.argmin(np.abs(grid - lc.truth["period"])))
    idx = np.unique(np.concatenate([rng.choice(len(grid), 3000, replace=False),
                                    np.arange(max(0, k_true - 40), min(len(grid), k_true + 40))]))
    periods = grid[idx]
    mean_o, cnt_o, sum_o = oracle.fold(lc.times, lc.flux, periods, 256, lc.t0)
    sigma = float(np.std(lc.flux.astype(np.float64)))
    sc_o, s_o, w_o = oracle.box_snr(sum_o, cnt_o, 1, 108, sigma)
    return lc, periods, mean_o, cnt_o, sc_o, sigma


def test_loud_star_fold_matches_oracle(ctx, loud_star):
    import paper_2312_02063_gb300 as g
    lc, periods, mean_o, cnt_o, _, _ = loud_star
    fo, co = g.gpfc_fold(ctx, _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods), 256, lc.t0)
    ctx.sync()
    np.testing.assert_array_equal(co.cpu().numpy(), cnt_o)
    fo = fo.cpu().numpy().astype(np.float64)
    nz = cnt_o > 0
    rel = np.abs(fo[nz] - mean_o[nz]) / np.abs(mean_o[nz])
    print(f"loud star: max relative mean error {rel.max():.3e}")
    assert rel.max() <= MEAN_RTOL


@pytest.mark.parametrize("path", ["fused", "warp", "epilogue"])
def test_loud_star_box_snr_matches_oracle(ctx, loud_star, path):
    import paper_2312_02063_gb300 as g
    lc, periods, _, _, sc_o, sigma = loud_star
    ctx.set_box_path({"fused": g.BOX_FUSED, "warp": g.BOX_WARP, "epilogue": g.BOX_EPILOGUE}[path])
    try:
        sc, bi, _ = g.gpfc_search(ctx, _dev(ctx, lc.times), _dev(ctx, lc.flux), _dev(ctx, periods), 256, lc.t0,
                                  g.SCORER_BOX, 1, 108, sigma)
        ctx.sync()
    finally:
        ctx.set_box_path(g.BOX_AUTO)
    sc = sc.cpu().numpy().astype(np.float64)
    err = np.abs(sc - sc_o)
    tol = BOX_RTOL * np.maximum(np.abs(sc_o), 1.0) + box_atol(fixed_point_unit(lc.flux), sigma)
    print(f"loud star, {path} box search: max box-SNR error {err.max():.3e}, "
          f"largest fraction of its tolerance {np.max(err / tol):.3f}")
    assert np.all(err <= tol)
    assert int(bi.item()) == oracle.argmax(sc.astype(np.float32))
