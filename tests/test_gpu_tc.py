"""Parity of the FP32 path's tensor-core contraction (3xTF32: each FP32 operand split exactly
into a TF32 hi part and the remainder, tau = K_hi DL_hi + K_hi DL_lo + K_lo DL_hi accumulated
in FP32) with the FP64 oracle, and its agreement with the FFMA contraction on the same
opacity, through the C ABI.

Bar: 0.1 ppm = 1e-7 absolute transit depth against the oracle (the FP32 path's bar); against
the FFMA contraction 0.01 ppm: the dropped lo x lo term and the TF32 rounding of the lo parts
are each below 2^-20 of a product, so the two contractions differ by about FP32 accumulation
error."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

TOL = 1e-7
TOL_FFMA = 1e-8
KIND_FFMA8, KIND_TC = 1, 3

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


def item_atm(spec_h, th, n_layers):
    """The oracle's single-atmosphere description of batch item theta."""
    m, nt = spec_h.n_mol, spec_h.n_tnodes
    return S.Atmosphere(n_layers=int(n_layers), p_max=spec_h.p_max, p_min=spec_h.p_min,
                        tnode_log10p=spec_h.tnode_log10p, tnode_t=th[m:m + nt],
                        log10_x=th[:m], fill_frac=spec_h.fill_frac, r_p=th[m + nt] * S.R_JUP,
                        m_p=spec_h.m_p, r_s=spec_h.r_s, p_cloud_top=10.0 ** th[m + nt + 1],
                        p_cloud_bot=spec_h.p_cloud_bot, kappa_cloud=spec_h.kappa_cloud,
                        gravity_mode=spec_h.gravity_mode, cloud_mode=spec_h.cloud_mode)


def run_batch(T, ctx, tables, spec, th_h, nl_h, bins, kind):
    """Native and binned spectra of the batch with the contraction pinned to `kind`."""
    import torch
    B = th_h.shape[0]
    T.pin_forward_config(ctx, tables, spec, B, bins, native=True, form="two-stage", per_sm=0,
                         contract_per_sm=kind)
    try:
        binned, status, native = T.forward_transit_batch(
            ctx, tables, spec, torch.tensor(th_h, device="cuda"),
            torch.tensor(nl_h, device="cuda"), bins, native=True)
        torch.cuda.synchronize()
    finally:
        T.pin_forward_config(ctx, tables, spec, B, bins, native=True, form=None)
    return native.cpu().numpy(), binned.cpu().numpy(), status.cpu().numpy()


def test_uneven_layers_ragged_grid(T, ctx):
    """Layer counts 1 .. 112 around every 8- and 16-layer slice edge (the MMA's K step and N
    step), 3 absorbers, CIA, Rayleigh, fractional cloud, a native grid of 5 x 128 + 77 points
    (several units and a ragged tail): against the oracle per native wavenumber and bin, and
    against the FFMA contraction."""
    tb = S.make_tables(41, 3, 8, 9, 5 * 128 + 77, with_cia=True)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced(12, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(3)
    spec = T.BatchSpec(spec_h, max_layers=112)
    nl = np.array([1, 7, 8, 9, 15, 16, 17, 31, 64, 100, 111, 112], dtype=np.int32)
    th = S.draw_theta(4242, len(nl), spec_h)
    nat_tc, bin_tc, st_tc = run_batch(T, ctx, tables, spec, th, nl, bins, KIND_TC)
    nat_ff, bin_ff, st_ff = run_batch(T, ctx, tables, spec, th, nl, bins, KIND_FFMA8)
    assert np.all(st_tc == 0) and np.all(st_ff == 0)
    for b in range(len(nl)):
        rn, rb, _ = O.forward(tb, item_atm(spec_h, th[b], nl[b]), bins_h)
        assert np.abs(nat_tc[b] - rn).max() <= TOL, b
        assert np.abs(bin_tc[b] - rb).max() <= TOL, b
    assert np.abs(nat_tc - nat_ff).max() <= TOL_FFMA
    assert np.abs(bin_tc - bin_ff).max() <= TOL_FFMA


def test_invalid_items_and_item_changes(T, ctx):
    """Items the model rejects (sum of mixing ratios above 1) between valid ones: zero depth
    where the oracle rejects, and the path-length tiles rebuilt at every item change (units of
    consecutive items share CTAs)."""
    tb = S.make_tables(43, 2, 6, 7, 300, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced(8, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=96)
    B = 40
    th = S.draw_theta(4343, B, spec_h)
    th[3, :2] = -0.1                                    # sum X > 1: rejected
    th[17, :2] = -0.05
    nl = S.draw_nlayers(4344, B, 20, 96)
    nat, binned, st = run_batch(T, ctx, tables, spec, th, nl, bins, KIND_TC)
    ref_b, ref_st = O.forward_batch(tb, spec_h, th, nl, bins_h)
    assert np.array_equal(st, ref_st)
    assert st[3] != 0 and st[17] != 0
    assert np.all(nat[st != 0] == 0.0)
    ok = st == 0
    assert np.abs(binned[ok] - ref_b[ok]).max() <= TOL


def test_default_contraction_is_tensor_core(T, ctx):
    """The autotuner offers the FP32 path one contraction per shape: the tensor-core kernel up
    to 112 layers (the graph runs it), the FFMA kernel beyond; pinning the tensor-core kernel
    for more layers is refused."""
    import torch
    tb = S.make_tables(45, 2, 6, 7, 700, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced(8, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2)
    th_h = S.draw_theta(4545, 3, spec_h)
    th = torch.tensor(th_h, device="cuda")
    g = T.ForwardGraph(ctx, tables, T.BatchSpec(spec_h, max_layers=100), th, None, bins,
                       autotune=True)
    # (the fused form, which has no separate contraction, may win on a shape this small)
    info = g.info()
    assert info["form"] == "fused" or info["contraction"] == "tc_3xtf32"
    g.launch()
    torch.cuda.synchronize()
    ref, _ = O.forward_batch(tb, spec_h, th_h, np.full(3, 100, np.int32), bins_h)
    assert np.abs(g.binned.cpu().numpy() - ref).max() <= TOL
    g150 = T.ForwardGraph(ctx, tables, T.BatchSpec(spec_h, max_layers=150), th, None, bins,
                          autotune=True)
    info = g150.info()
    assert info["form"] == "fused" or info["contraction"] in ("ffma8", "ffma11")
    with pytest.raises(T.TransitError) as e:
        T.pin_forward_config(ctx, tables, T.BatchSpec(spec_h, max_layers=150), 3, bins,
                             form="two-stage", contract_per_sm=KIND_TC)
    assert e.value.code == T.TR_ERR_UNSUPPORTED
