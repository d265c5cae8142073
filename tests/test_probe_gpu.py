"""The shared-memory read-modify-write probe (the fold roofline's denominator) runs and
gives rates inside what one SM's shared-memory pipe can deliver: at most 32 lanes' words
per clock for 4-byte words and 16 for 8-byte words (128 bytes a clock, each word read
and written)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("word,nbins,warps,limit", [(8, 32, 16, 8.5), (4, 32, 16, 17.0), (8, 256, 3, 8.5)])
def test_probe_rates_are_physical(word, nbins, warps, limit):
    import paper_2312_02063_gb300 as g
    ups, upc = g.gpfc_probe_smem_rmw(word, nbins, warps, 1, 2000)
    print(f"{word}-byte words, {nbins} bins, {warps} warps: {upc:.2f} updates/clk/SM, {ups:.3e} updates/s")
    assert 0.5 < upc <= limit
    assert ups > 0
