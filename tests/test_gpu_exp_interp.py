"""Exponential temperature interpolation of the cross-sections (Sec. 5, sigma = a e^{-b/T}
through the two bracketing temperatures) on the GPU against the FP64 oracle's scheme.

Bar: 0.1 ppm = 1e-7 absolute transit depth for the FP32 path, 1 ppm for mixed precision.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
TOL = 1e-7
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07759_gb300 import transit
    return transit


@pytest.fixture(scope="module")
def ctx(T):
    return T.TransitContext(0)


def exp_tables(tb):
    return dataclasses.replace(tb, interp_mode=S.INTERP_EXP)


def single(T, ctx, tb, atm, bins=None, precision=None, storage=None):
    import torch
    tables = T.XsecTables(ctx, tb, storage=storage or T.TR_STORE_FP32)
    b = T.Bins(ctx, tables, *bins) if bins is not None else None
    a = T.Atmosphere(ctx, tables, atm)
    kw = {} if precision is None else {"precision": precision}
    dn, db = T.forward_transit(ctx, tables, a, b, **kw)
    ctx.sync_status()
    torch.cuda.synchronize()
    return dn.cpu().numpy(), (db.cpu().numpy() if db is not None else None)


def test_exp_scheme_full_model_matches_oracle(T, ctx):
    """5 absorbers on 22 x 27 tables, CIA, Rayleigh, grey cloud, 4-node temperature profile,
    20,003 native wavenumbers plus 50 bins: the exponential scheme within 0.1 ppm of the
    oracle's, and far closer to it than to the linear scheme."""
    tb = exp_tables(S.make_tables(2, 5, 22, 27, 20003, with_cia=True))
    atm = S.config2_atmosphere()
    bins = S.bins_logspaced()
    dn, db = single(T, ctx, tb, atm, bins)
    rn, rb, _ = O.forward(tb, atm, bins)
    assert np.abs(dn - rn).max() <= TOL
    assert np.abs(db - rb).max() <= TOL
    rl, _, _ = O.forward(dataclasses.replace(tb, interp_mode=S.INTERP_LINEAR), atm, bins)
    # the GPU result is the exponential scheme's, not the linear one's (the two schemes differ
    # by a few 1e-7 on these smooth synthetic tables)
    err_exp = np.abs(dn - rn).max()
    assert np.abs(dn - rl).max() > 10 * max(err_exp, 1e-9)


def test_exp_scheme_zero_values_fall_back_to_linear(T, ctx):
    """Cross-sections that are zero at some grid temperatures (the logarithm does not exist):
    those pairs take the linear value, as in the oracle."""
    tb = exp_tables(S.make_tables(3, 2, 13, 15, 1500, with_cia=False))
    rng = np.random.default_rng(4)
    mask = rng.random(tb.sigma.shape) < 0.15
    tb.sigma[mask] = 0.0
    atm = S.config1_atmosphere()
    atm.tnode_t = np.array([1234.5])
    dn, _ = single(T, ctx, tb, atm)
    rn, _, _ = O.forward(tb, atm)
    assert np.abs(dn - rn).max() <= TOL


def test_exp_scheme_batch_uneven_layers(T, ctx):
    """A batch with uneven layer counts and an invalid atmosphere, binned region only."""
    import torch
    tb = exp_tables(S.make_tables(1, 2, 13, 15, 10000, with_cia=False))
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=150)
    B = 12
    th = S.draw_theta(71, B, spec_h)
    nl = S.draw_nlayers(72, B)
    th[3, 2] = -1.0                                  # negative temperature: rejected
    binned, status = T.forward_transit_batch(ctx, tables, spec, torch.tensor(th, device="cuda"),
                                             torch.tensor(nl, device="cuda"), bins)
    ctx.sync_status()
    ref, rst = O.forward_batch(tb, spec_h, th, nl, bins_h)
    st = status.cpu().numpy()
    assert np.array_equal(st, rst) and st[3] != 0
    assert np.abs(binned.cpu().numpy() - ref).max() <= TOL


def test_exp_scheme_mixed_precision(T, ctx):
    """FP16 log10 tables with the exponential scheme (the logarithms come straight from the
    table) and the tensor-core contraction: within 1 ppm of the oracle."""
    tb = exp_tables(S.make_tables(2, 5, 22, 27, 20003, with_cia=True))
    atm = S.config2_atmosphere()
    dn, _ = single(T, ctx, tb, atm, precision=T.TR_PREC_MIXED,
                   storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    rn, _, _ = O.forward(tb, atm)
    assert np.abs(dn - rn).max() <= TOL_MIXED


def test_exp_scheme_unsupported_paths_are_rejected(T, ctx):
    """The adjoint implements the linear scheme only: it refuses tables loaded with the
    exponential scheme (TR_ERR_UNSUPPORTED) instead of returning a wrong gradient."""
    import torch
    tb = exp_tables(S.make_tables(1, 2, 13, 15, 2000, with_cia=False))
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=60)
    th = torch.tensor(S.draw_theta(5, 2, spec_h), device="cuda")
    with pytest.raises(T.TransitError) as ei:
        T.adjoint_transit(ctx, tables, spec, th, None, bins,
                          gbin=torch.zeros(2, len(bins_h[0]), dtype=torch.float64, device="cuda"))
    assert ei.value.code == 6                        # TR_ERR_UNSUPPORTED
