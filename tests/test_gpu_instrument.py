"""FluxBinner with uncertainties (Sec. 4.5) and the SNR instrument model (Sec. 7) through the
C ABI against the FP64 oracle's statement of them."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07759_gb300 import transit
    return transit


@pytest.fixture(scope="module")
def ctx(T):
    return T.TransitContext(0)


def test_bin_spectra_with_uncertainties(T, ctx):
    """Three native spectra with per-wavenumber uncertainties, binned to 50 bins: fluxes and
    propagated uncertainties equal the oracle's to FP64 rounding, from a full-length input and
    from one that starts at the bins' first native index."""
    import torch
    tb = S.make_tables(1, 1, 4, 4, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    centre, width = S.bins_logspaced()
    bins = T.Bins(ctx, tables, centre, width)
    rng = np.random.default_rng(21)
    flux = 0.0105 + 1e-4 * rng.standard_normal((3, tb.n_wn))
    sig = 3e-5 * (1.0 + rng.random((3, tb.n_wn)))
    rf, rs = O.bin_with_uncertainty(tb.wn_grid, centre, width, flux, sig)
    f, s = T.bin_spectra(ctx, bins, torch.tensor(flux, device="cuda"),
                         torch.tensor(sig, device="cuda"))
    torch.cuda.synchronize()
    assert np.allclose(f.cpu().numpy(), rf, rtol=1e-13, atol=0)
    assert np.allclose(s.cpu().numpy(), rs, rtol=1e-13, atol=0)
    i0, i1 = bins.native_range
    w = O.bin_weights(tb.wn_grid, centre, width)
    nz = np.nonzero(w.sum(axis=0))[0]
    assert i0 <= nz[0] and nz[-1] < i1               # the library's range holds every weight
    f2, s2 = T.bin_spectra(ctx, bins, torch.tensor(flux[:, i0:i1].copy(), device="cuda"),
                           torch.tensor(sig[:, i0:i1].copy(), device="cuda"), base=i0)
    torch.cuda.synchronize()
    assert np.array_equal(f2.cpu().numpy(), f.cpu().numpy())
    assert np.array_equal(s2.cpu().numpy(), s.cpu().numpy())


def test_snr_instrument_matches_oracle(T, ctx):
    """Noise = largest binned depth / SNR / sqrt(n_obs) per spectrum; the observation adds it
    times the supplied standard-normal draws."""
    import torch
    rng = np.random.default_rng(22)
    binned = 0.0105 + 2e-4 * rng.random((5, 50))
    z = rng.standard_normal((5, 50))
    for snr, n in ((50.0, 1), (300.0, 7)):
        ro, rsig = O.snr_instrument(binned, snr, n, z)
        o, sg = T.snr_instrument(ctx, torch.tensor(binned, device="cuda"), snr, n,
                                 torch.tensor(z, device="cuda"))
        torch.cuda.synchronize()
        assert np.allclose(o.cpu().numpy(), ro, rtol=1e-14, atol=0)
        assert np.allclose(sg.cpu().numpy(), rsig, rtol=1e-14, atol=0)


def test_instrument_arguments_are_checked(T, ctx):
    import torch
    b = torch.zeros(2, 10, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TransitError):
        T.snr_instrument(ctx, b, 0.0, 1, b)
    with pytest.raises(T.TransitError):
        T.snr_instrument(ctx, b, 10.0, 0, b)
