"""Guillot2010 temperature profile (Sec. 4.2) and two-layer gas profiles (Sec. 4.3) on the GPU
(through the C ABI) against the FP64 oracle: batches with uneven layer counts in both
precisions, single atmospheres, the CUDA-graph form, the emission model and the calls that
refuse them.

Bars: FP32 0.1 ppm absolute depth per native wavenumber and bin, mixed precision 1 ppm,
geometry 1e-12 relative.
"""
import concurrent.futures as cf
import dataclasses
import os

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


@pytest.fixture(scope="module")
def tables_h():
    return S.make_tables(8, 3, 13, 15, 4001, with_cia=True, wn_min=1000.0, wn_max=12000.0)


def pmap(fn, items):
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(items), os.cpu_count() or 1))) as ex:
        return list(ex.map(fn, items))


def spec_of(n_mol, t_profile, gas_mode):
    sp = S.batch_spec(n_mol)
    sp.t_profile, sp.gas_mode = t_profile, gas_mode
    return sp


def atm_of(spec, th, n_layers):
    """The oracle's single-atmosphere description of batch item theta (any layout)."""
    m, c = spec.n_mol, spec.n_chem
    kw = {}
    if spec.gas_mode == S.GAS_TWOLAYER:
        kw.update(gas_mode=S.GAS_TWOLAYER, log10_x_top=th[m:2 * m], log10_p_switch=th[2 * m:3 * m])
    if spec.t_profile == S.TPROF_GUILLOT:
        g = th[c:c + 5]
        kw.update(t_profile=S.TPROF_GUILLOT, t_int=spec.t_int,
                  guillot=np.array([g[0], 10 ** g[1], 10 ** g[2], 10 ** g[3], g[4]]))
        tn = np.array([1.0])
        tlp = np.array([6.0])
    else:
        tn = th[c:c + spec.n_tnodes]
        tlp = spec.tnode_log10p
    k = c + spec.n_tpar
    return S.Atmosphere(n_layers=int(n_layers), p_max=spec.p_max, p_min=spec.p_min,
                        tnode_log10p=tlp, tnode_t=tn, log10_x=th[:m], fill_frac=spec.fill_frac,
                        r_p=th[k] * S.R_JUP, m_p=spec.m_p, r_s=spec.r_s,
                        p_cloud_top=10.0 ** th[k + 1], p_cloud_bot=spec.p_cloud_bot,
                        kappa_cloud=spec.kappa_cloud, gravity_mode=spec.gravity_mode,
                        cloud_mode=spec.cloud_mode, **kw)


def oracle_native(tb, spec, th, nl):
    def one(b):
        try:
            return O.forward(tb, atm_of(spec, th[b], nl[b]))[0]
        except O.OracleError as e:
            return e.status
    return pmap(one, list(range(len(th))))


@pytest.mark.parametrize("t_profile,gas_mode,precision", [
    (S.TPROF_GUILLOT, S.GAS_CONSTANT, "fp32"),
    (S.TPROF_NPOINT, S.GAS_TWOLAYER, "fp32"),
    (S.TPROF_GUILLOT, S.GAS_TWOLAYER, "fp32"),
    (S.TPROF_GUILLOT, S.GAS_TWOLAYER, "mixed"),
])
def test_profile_batches_match_oracle(T, ctx, tables_h, t_profile, gas_mode, precision):
    """A batch with uneven layer counts (1-150) and rejected items: native spectra and bins of
    every item against the oracle, statuses equal to the oracle's rejections."""
    import torch
    tb = tables_h
    storage = T.TR_STORE_FP32 | (T.TR_STORE_FP16_LOG10 if precision == "mixed" else 0)
    tables = T.XsecTables(ctx, tb, storage=storage)
    bins_h = S.bins_logspaced(20, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = spec_of(3, t_profile, gas_mode)
    B = 12
    th = S.draw_theta(960 + 10 * t_profile + gas_mode, B, spec_h, lx_range=(-7.0, -2.0))
    nl = np.array([100, 37, 150, 64, 1, 90, 120, 55, 75, 140, 100, 2], dtype=np.int32)
    if gas_mode == S.GAS_TWOLAYER:
        # item 3: one gas switched up while another is not yet: a layer with sum X > 1
        th[3, :3] = np.log10([0.6, 0.01, 1e-5])
        th[3, 3:6] = np.log10([0.01, 0.6, 1e-5])
        th[3, 6:9] = [1.5, 4.5, 3.0]
    if t_profile == S.TPROF_GUILLOT:
        th[5, spec_h.n_chem + 4] = 1.3                  # alpha > 1: rejected
    spec = T.BatchSpec(spec_h, max_layers=150)
    prec = T.TR_PREC_FP32 if precision == "fp32" else T.TR_PREC_MIXED
    dev = lambda x: torch.tensor(x, device="cuda")
    binned, status, nat = T.forward_transit_batch(ctx, tables, spec, dev(th), dev(nl), bins,
                                                  precision=prec, native=True)
    torch.cuda.synchronize()
    binned, status, nat = binned.cpu().numpy(), status.cpu().numpy(), nat.cpu().numpy()
    refs = oracle_native(tb, spec_h, th, nl)
    bar = 1e-7 if precision == "fp32" else 1e-6
    worst = 0.0
    for b, r in enumerate(refs):
        if isinstance(r, int):
            assert status[b] == T.TR_ERR_INVALID_MODEL, b
            assert np.all(nat[b] == 0.0) and np.all(binned[b] == 0.0)
            continue
        assert status[b] == 0, b
        err = float(np.abs(nat[b] - r).max())
        worst = max(worst, err)
        assert err <= bar, (b, err)
        rb, _ = O.bin_with_uncertainty(tb.wn_grid, *bins_h, r)
        assert np.abs(binned[b] - rb).max() <= bar, b
    if gas_mode == S.GAS_TWOLAYER:
        assert status[3] == T.TR_ERR_INVALID_MODEL
    if t_profile == S.TPROF_GUILLOT:
        assert status[5] == T.TR_ERR_INVALID_MODEL
    print(f"profiles t={t_profile} gas={gas_mode} {precision}: max |D - oracle| {worst * 1e6:.5f} ppm")


def test_single_atmosphere_guillot_two_layer_and_geometry(T, ctx, tables_h):
    """tr_build_atmosphere with a Guillot profile and two-layer gases (one switch on a layer
    boundary, two inside layers): altitudes (per-layer mean molecular weight) to 1e-12 and
    the native spectrum to 0.1 ppm against the oracle; its emission spectrum to 0.1 ppm."""
    import torch
    tb = tables_h
    tables = T.XsecTables(ctx, tb)
    atm = S.Atmosphere(n_layers=100, p_max=1e6, p_min=1e-4, tnode_log10p=np.array([6.0]),
                       tnode_t=np.array([1.0]), log10_x=np.array([-3.0, -4.0, -2.5]),
                       fill_frac=np.array([0.83, 0.17]), r_p=1.2 * S.R_JUP, m_p=S.M_JUP,
                       r_s=S.R_SUN, p_cloud_top=3e2, kappa_cloud=1e-2,
                       cloud_mode=S.CLOUD_FRACTIONAL, t_profile=S.TPROF_GUILLOT,
                       guillot=np.array([1700.0, 1e-2, 3e-3, 8e-2, 0.4]), t_int=150.0,
                       gas_mode=S.GAS_TWOLAYER, log10_x_top=np.array([-6.0, -3.0, -5.0]),
                       log10_p_switch=np.array([3.0, 1.234, 4.567]))
    a = T.Atmosphere(ctx, tables, atm)
    z, _, _ = a.readback()
    ref = O.profile(tb, atm)
    assert np.allclose(z[1:], ref["z"][1:], rtol=1e-12, atol=0)
    nat, _ = T.forward_transit(ctx, tables, a)
    torch.cuda.synchronize()
    dn, _, _ = O.forward(tb, atm)
    assert np.abs(nat.cpu().numpy() - dn).max() <= 1e-7
    em, _ = T.forward_emission(ctx, tables, a, n_mu=4, t_star=5800.0)
    torch.cuda.synchronize()
    assert np.abs(em.cpu().numpy() - O.emission(tb, atm, n_mu=4, t_star=5800.0)).max() <= 1e-7


def test_two_layer_graph_capture_and_autotuner(T, ctx, tables_h):
    """The CUDA-graph form with the autotuner on two-layer gases (the fused kernel, which
    implements constant mixing ratios only, is left out of the search) replays to the
    oracle's spectra, following parameters written in place."""
    import torch
    tb = tables_h
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced(20, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = spec_of(3, S.TPROF_NPOINT, S.GAS_TWOLAYER)
    B = 6
    th = torch.tensor(S.draw_theta(971, B, spec_h, lx_range=(-7.0, -2.0)), device="cuda")
    nl = torch.tensor(S.draw_nlayers(972, B), device="cuda")
    spec = T.BatchSpec(spec_h, max_layers=150)
    g = T.ForwardGraph(ctx, tables, spec, th, nl, bins, autotune=True)
    assert g.info()["form"] == "two-stage"
    for seed in (973, 974):
        th.copy_(torch.tensor(S.draw_theta(seed, B, spec_h, lx_range=(-7.0, -2.0))))
        g.launch()
        torch.cuda.synchronize()
        ref, st = O.forward_batch(tb, spec_h, th.cpu().numpy(), nl.cpu().numpy(), bins_h)
        assert np.array_equal(g.status.cpu().numpy(), st)
        assert np.abs(g.binned.cpu().numpy() - ref).max() <= 1e-7


def test_calls_that_refuse_the_new_profiles(T, ctx, tables_h):
    """The adjoint implements the N-point profile and constant mixing ratios; the
    allocation-free call constant mixing ratios; two-layer gases need the linear T scheme."""
    import ctypes as C
    import torch
    tb = tables_h
    tables = T.XsecTables(ctx, tb)
    bins = T.Bins(ctx, tables, *S.bins_logspaced(20, 1.2, 1.6))
    for tp, gm in ((S.TPROF_GUILLOT, S.GAS_CONSTANT), (S.TPROF_NPOINT, S.GAS_TWOLAYER)):
        spec_h = spec_of(3, tp, gm)
        spec = T.BatchSpec(spec_h, max_layers=100)
        th = torch.tensor(S.draw_theta(5, 2, spec_h), device="cuda")
        with pytest.raises(T.TransitError) as e:
            T.adjoint_transit(ctx, tables, spec, th, None, bins,
                              gbin=torch.zeros(2, bins.n_bin, dtype=torch.float64, device="cuda"))
        assert e.value.code == T.TR_ERR_UNSUPPORTED
    spec_h = spec_of(3, S.TPROF_NPOINT, S.GAS_TWOLAYER)
    spec = T.BatchSpec(spec_h, max_layers=100)
    th = torch.tensor(S.draw_theta(6, 2, spec_h), device="cuda")
    out = torch.empty(2, bins.n_bin, dtype=torch.float64, device="cuda")
    st = torch.empty(2, dtype=torch.int32, device="cuda")
    rc = ctx.lib.tr_forward_transit_batch_noalloc(
        ctx.handle, tables.handle, C.byref(spec.desc), 2, C.c_void_p(th.data_ptr()), None,
        bins.handle, C.c_void_p(out.data_ptr()), C.c_void_p(st.data_ptr()), None)
    assert rc == T.TR_ERR_UNSUPPORTED
    tbe = dataclasses.replace(tb, interp_mode=S.INTERP_EXP)
    tables_e = T.XsecTables(ctx, tbe)
    bins_e = T.Bins(ctx, tables_e, *S.bins_logspaced(20, 1.2, 1.6))
    with pytest.raises(T.TransitError) as e:
        T.forward_transit_batch(ctx, tables_e, spec, th, None, bins_e)
    assert e.value.code == T.TR_ERR_UNSUPPORTED
