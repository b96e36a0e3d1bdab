"""Mixed-precision path (FP16 log10 sigma tables, tau on tcgen05 tensor cores as BF16 hi+lo
split products): parity with the FP32 GPU path where the FP16 encoding is exact (isolates the
tensor-core contraction), and with the FP64 oracle within 1 ppm on synthetic tables."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-6          # 1 ppm absolute depth


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07759_gb300 import transit
    return transit


@pytest.fixture(scope="module")
def ctx(T):
    return T.TransitContext(0)


def both_paths(T, ctx, tb, atm, bins=None):
    import torch
    tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    b = T.Bins(ctx, tables, *bins) if bins is not None else None
    a = T.Atmosphere(ctx, tables, atm)
    d32, b32 = T.forward_transit(ctx, tables, a, b, precision=T.TR_PREC_FP32)
    d16, b16 = T.forward_transit(ctx, tables, a, b, precision=T.TR_PREC_MIXED)
    ctx.sync_status()
    torch.cuda.synchronize()
    cv = (lambda x: x.cpu().numpy() if x is not None else None)
    return cv(d32), cv(b32), cv(d16), cv(b16)


@pytest.mark.parametrize("n_layers", [37, 100])
def test_tensor_core_contraction_matches_fp32_path(T, ctx, n_layers):
    """Tables of exact powers of ten encode exactly in FP16 log form, so the mixed path
    differs from the FP32 path only by the BF16 hi+lo contraction (and FP32 decoding)."""
    tb = S.make_tables(21, 3, 6, 7, 640, with_cia=True, wn_min=3000.0, wn_max=9000.0)
    rng = np.random.default_rng(3)
    tb.sigma[:] = (10.0 ** rng.integers(-33, -25, size=tb.sigma.shape)).astype(np.float32)
    atm = S.config2_atmosphere(n_mol=3)
    atm.n_layers = n_layers
    d32, _, d16, _ = both_paths(T, ctx, tb, atm)
    assert np.all(np.isfinite(d16))
    assert np.abs(d16 - d32).max() <= 2e-8               # 0.02 ppm


def test_mixed_full_model_within_1ppm_of_oracle(T, ctx):
    """5 absorbers on 22 x 27 tables, CIA, Rayleigh, cloud, 20,003 native wavenumbers."""
    tb = S.make_tables(2, 5, 22, 27, 20003, with_cia=True)
    atm = S.config2_atmosphere()
    bins = S.bins_logspaced()
    _, _, d16, b16 = both_paths(T, ctx, tb, atm, bins)
    rn, rb, _ = O.forward(tb, atm, bins)
    err = np.abs(d16 - rn).max()
    assert err <= TOL_MIXED, err
    assert np.abs(b16 - rb).max() <= TOL_MIXED


def test_mixed_batch_matches_oracle(T, ctx):
    import torch
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=150)
    B = 12
    th = S.draw_theta(61, B, spec_h)
    nl = S.draw_nlayers(62, B)
    binned, status = T.forward_transit_batch(ctx, tables, spec, torch.tensor(th, device="cuda"),
                                             torch.tensor(nl, device="cuda"), bins,
                                             precision=T.TR_PREC_MIXED)
    ctx.sync_status()
    ref, rst = O.forward_batch(tb, spec_h, th, nl, bins_h)
    assert np.array_equal(status.cpu().numpy(), rst)
    assert np.abs(binned.cpu().numpy() - ref).max() <= TOL_MIXED


def test_mixed_batch_uneven_layers_persistent_contraction(T, ctx):
    """Up to 100 layers (the persistent tensor-core contraction), uneven layer counts and an
    invalid atmosphere: binned depths within 1 ppm of the oracle, zero for the invalid one."""
    import torch
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=100)
    B = 10
    th = S.draw_theta(63, B, spec_h)
    nl = np.array([100, 51, 77, 100, 64, 90, 99, 100, 58, 83], dtype=np.int32)
    th[4, 2] = -5.0                  # negative temperature: rejected
    binned, status = T.forward_transit_batch(ctx, tables, spec, torch.tensor(th, device="cuda"),
                                             torch.tensor(nl, device="cuda"), bins,
                                             precision=T.TR_PREC_MIXED)
    ctx.sync_status()
    ref, rst = O.forward_batch(tb, spec_h, th, nl, bins_h)
    st = status.cpu().numpy()
    assert np.array_equal(st, rst) and st[4] != 0
    got = binned.cpu().numpy()
    assert np.abs(got - ref).max() <= TOL_MIXED
    assert np.all(got[4] == 0.0)
