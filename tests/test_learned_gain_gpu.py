"""What the trained CNN gains over the box-SNR detector alone.

Trains the scorer on the GPU (the library's own forward/backward/Adam kernels) on
device-generated folded profiles, then compares the true-positive rate at a false-
positive rate of 1e-3 on held-out profiles: the CNN must beat the box statistic, whose
false alarms come from eclipsing-binary-like double boxes and sinusoids.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_trained_cnn_beats_box_snr_at_fixed_fpr():
    import paper_2312_02063_gb300 as g
    from paper_2312_02063_gb300 import train as tr
    ctx = g.Context(0)
    w, hist = tr.train(ctx, 60 * 4096, batch=4096, lr=2e-3)
    assert hist[-1][1] < hist[0][1]
    res = tr.evaluate(ctx, w, n_eval=40_000, fpr=1e-3)
    print("detection at FPR 1e-3:", res)
    assert res["tpr_cnn"] > res["tpr_box"]
    ctx.close()
