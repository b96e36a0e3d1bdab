"""Emission model of Sec. 4 on the GPU (through the C ABI) against the FP64 oracle's statement
of it (readings E1-E4) and against closed forms.

Bar: 0.1 ppm absolute on the planet-star flux ratio at every native wavenumber (FP32 path),
and 1e-5 relative where the closed form is a blackbody.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
ABS = 1e-7
H, C, KB = 6.62607015e-34, 299792458.0, 1.380649e-23


@pytest.fixture(scope="module")
def T():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07759_gb300 import transit
    return transit


@pytest.fixture(scope="module")
def ctx(T):
    return T.TransitContext(0)


def blackbody_ratio(wn, t_p, t_s, rr):
    """(R_p/R_s)^2 B(nu, T_p) / B(nu, T_s): the nu^3 factors cancel."""
    x = H * C * 100.0 * np.asarray(wn) / KB
    return rr * np.expm1(x / t_s) / np.expm1(x / t_p)


def test_isothermal_atmosphere_emits_its_blackbody(T, ctx):
    """Whatever the opacity, an isothermal atmosphere over a surface at the same temperature
    shows B(T): F_p/F_s = (R_p/R_s)^2 B(T)/B(T_star) (and so does the oracle)."""
    import torch
    tb = S.make_tables(1, 2, 13, 15, 3000, with_cia=False)
    atm = S.config1_atmosphere()
    tables = T.XsecTables(ctx, tb)
    a = T.Atmosphere(ctx, tables, atm)
    for n_mu in (1, 4, 16):
        nat, _ = T.forward_emission(ctx, tables, a, n_mu=n_mu, t_star=5800.0)
        torch.cuda.synchronize()
        got = nat.cpu().numpy()
        ref = blackbody_ratio(tb.wn_grid, 1500.0, 5800.0, (atm.r_p / atm.r_s) ** 2)
        assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-12), n_mu
        orc = O.emission(tb, atm, n_mu=n_mu, t_star=5800.0)
        assert np.abs(got - orc).max() <= ABS


def test_zero_opacity_shows_the_surface(T, ctx):
    """Without opacity the intensity is the surface's at every angle: T_s is the temperature
    profile at p_max (reading E3), here the first node of a four-node profile."""
    import torch
    tb = S.make_tables(1, 1, 4, 4, 500, with_cia=False, with_rayleigh=False)
    tb.sigma[:] = 0.0
    atm = S.config2_atmosphere(n_mol=1)
    atm.cloud_mode = S.CLOUD_NONE
    tables = T.XsecTables(ctx, tb)
    a = T.Atmosphere(ctx, tables, atm)
    nat, _ = T.forward_emission(ctx, tables, a, n_mu=4, t_star=6100.0)
    torch.cuda.synchronize()
    got = nat.cpu().numpy()
    ref = blackbody_ratio(tb.wn_grid, atm.tnode_t[0], 6100.0, (atm.r_p / atm.r_s) ** 2)
    assert np.all(np.abs(got - ref) <= 1e-5 * ref + 1e-12)
    assert np.abs(got - O.emission(tb, atm, n_mu=4, t_star=6100.0)).max() <= ABS


def test_full_size_emission_matches_oracle(T, ctx):
    """The full-size model (100 layers, 5 absorbers, CIA, Rayleigh, cloud deck, four-node
    profile, 22 x 27 x 200,000 tables) at every native wavenumber and binned."""
    import torch
    tb = S.make_tables(2, 5, 22, 27, 200000, with_cia=True)
    atm = S.config2_atmosphere()
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    a = T.Atmosphere(ctx, tables, atm)
    nat, binned = T.forward_emission(ctx, tables, a, bins=bins, n_mu=4, t_star=5800.0)
    torch.cuda.synchronize()
    got = nat.cpu().numpy()
    ref = O.emission(tb, atm, n_mu=4, t_star=5800.0)
    err = np.abs(got - ref).max()
    print(f"full-size emission: max |F - oracle| {err * 1e6:.5f} ppm "
          f"(flux ratio up to {ref.max() * 1e6:.1f} ppm)")
    assert err <= ABS
    rb, _ = O.bin_with_uncertainty(tb.wn_grid, *bins_h, ref)
    assert np.abs(binned.cpu().numpy() - rb).max() <= ABS


def test_emission_batch_uneven_layers_and_invalid_item(T, ctx):
    """A batch with uneven layer counts and one rejected model: native and binned flux ratios
    of every valid item against the oracle, zeros and status 2 for the rejected one."""
    import torch
    tb = S.make_tables(6, 3, 13, 15, 4001, with_cia=True, wn_min=1000.0, wn_max=12000.0)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced(20, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(3)
    B = 6
    th = S.draw_theta(91, B, spec_h, lx_range=(-7.0, -3.0), t_range=(700.0, 2400.0))
    th[4, :2] = [-0.1, -0.2]
    nl = np.array([100, 37, 150, 64, 90, 1], dtype=np.int32)
    spec = T.BatchSpec(spec_h, max_layers=150)
    dev = lambda x: torch.tensor(x, device="cuda")
    binned, status, nat = T.forward_emission_batch(ctx, tables, spec, dev(th), dev(nl), bins,
                                                   n_mu=4, t_star=5500.0, native=True)
    binned_only, status2, _ = T.forward_emission_batch(ctx, tables, spec, dev(th), dev(nl),
                                                       bins, n_mu=4, t_star=5500.0)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    assert st.tolist() == [0, 0, 0, 0, T.TR_ERR_INVALID_MODEL, 0]
    assert torch.equal(status, status2)
    nat, binned, binned_only = (x.cpu().numpy() for x in (nat, binned, binned_only))
    assert np.all(nat[4] == 0.0) and np.all(binned[4] == 0.0)
    m, nt = spec_h.n_mol, spec_h.n_tnodes

    def ref(b):
        atm = S.Atmosphere(n_layers=int(nl[b]), p_max=spec_h.p_max, p_min=spec_h.p_min,
                           tnode_log10p=spec_h.tnode_log10p, tnode_t=th[b, m:m + nt],
                           log10_x=th[b, :m], fill_frac=spec_h.fill_frac,
                           r_p=th[b, m + nt] * S.R_JUP, m_p=spec_h.m_p, r_s=spec_h.r_s,
                           p_cloud_top=10.0 ** th[b, m + nt + 1],
                           p_cloud_bot=spec_h.p_cloud_bot, kappa_cloud=spec_h.kappa_cloud,
                           gravity_mode=spec_h.gravity_mode, cloud_mode=spec_h.cloud_mode)
        return O.emission(tb, atm, n_mu=4, t_star=5500.0)
    valid = [0, 1, 2, 3, 5]
    with cf.ThreadPoolExecutor(max_workers=min(5, os.cpu_count() or 1)) as ex:
        refs = list(ex.map(ref, valid))
    for b, r in zip(valid, refs):
        assert np.abs(nat[b] - r).max() <= ABS, b
        rb, _ = O.bin_with_uncertainty(tb.wn_grid, *bins_h, r)
        assert np.abs(binned[b] - rb).max() <= ABS, b
        assert np.abs(binned_only[b] - rb).max() <= ABS, b


def test_mixed_precision_emission_within_1ppm(T, ctx):
    """FP16 log10 tables (opacity decoded from them) with the FP32 vertical pass: the flux
    ratio within 1 ppm of the oracle on a 20,003-wavenumber five-absorber model; the
    measured error is printed."""
    import torch
    tb = S.make_tables(2, 5, 22, 27, 20003, with_cia=True)
    atm = S.config2_atmosphere()
    tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    a = T.Atmosphere(ctx, tables, atm)
    nat, _ = T.forward_emission(ctx, tables, a, n_mu=4, t_star=5800.0,
                                precision=T.TR_PREC_MIXED)
    torch.cuda.synchronize()
    err = np.abs(nat.cpu().numpy() - O.emission(tb, atm, n_mu=4, t_star=5800.0)).max()
    print(f"mixed-precision emission: max |F - oracle| {err * 1e6:.4f} ppm")
    assert err <= 1e-6


def test_emission_rejects_bad_arguments(T, ctx):
    import ctypes as C
    tb = S.make_tables(1, 1, 4, 4, 100, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    a = T.Atmosphere(ctx, tables, S.config1_atmosphere().__class__(
        n_layers=10, p_max=1e5, p_min=1.0, tnode_log10p=np.array([5.0]),
        tnode_t=np.array([1000.0]), log10_x=np.array([-4.0]), fill_frac=np.array([0.83, 0.17]),
        r_p=S.R_JUP, m_p=S.M_JUP, r_s=S.R_SUN))
    import torch
    out = torch.empty(tb.n_wn, dtype=torch.float64, device="cuda")
    for n_mu, ts in ((0, 5800.0), (17, 5800.0), (4, 0.0), (4, -1.0)):
        rc = ctx.lib.tr_forward_emission(ctx.handle, tables.handle, a.handle, None, n_mu,
                                         C.c_double(ts), C.c_void_p(out.data_ptr()), None,
                                         T.TR_PREC_FP32, None)
        assert rc == T.TR_ERR_ARG if hasattr(T, "TR_ERR_ARG") else rc == 1
