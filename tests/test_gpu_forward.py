"""Parity of the CUDA forward path (through the C ABI) with the FP64 oracle.

Bar: 0.1 ppm = 1e-7 absolute transit depth for the FP32 path, per native wavenumber and per
bin, on the same seeded inputs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

TOL = 1e-7          # 0.1 ppm absolute depth

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


def run_single(T, ctx, tb, atm, bins=None, native=True, tables=None):
    import torch
    tables = tables or T.XsecTables(ctx, tb)
    b = T.Bins(ctx, tables, *bins) if bins is not None else None
    a = T.Atmosphere(ctx, tables, atm)
    dn, db = T.forward_transit(ctx, tables, a, b, native=native)
    torch.cuda.synchronize()
    return (dn.cpu().numpy() if dn is not None else None,
            db.cpu().numpy() if db is not None else None)


def test_config1_native_and_binned(T, ctx):
    """Plain model of 100 layers, 2 absorbers, 10,000 wavenumbers."""
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    atm = S.config1_atmosphere()
    bins = S.bins_logspaced()
    dn, db = run_single(T, ctx, tb, atm, bins)
    rn, rb, _ = O.forward(tb, atm, bins)
    assert np.abs(dn - rn).max() <= TOL
    assert np.abs(db - rb).max() <= TOL


@pytest.mark.parametrize("n_layers", [1, 2, 7, 33, 150])
def test_ragged_shapes_all_contributions(T, ctx, n_layers):
    """Odd wavenumber count (several tiles plus a ragged tail), 3 absorbers, CIA, Rayleigh,
    4-node profile, discrete cloud; layer counts from 1 to 150."""
    tb = S.make_tables(7, 3, 6, 9, 257 * 2 + 3, with_cia=True, wn_min=2000.0, wn_max=12000.0)
    atm = S.config2_atmosphere(n_mol=3)
    atm.n_layers = n_layers
    atm.p_cloud_top = 3e2
    dn, _ = run_single(T, ctx, tb, atm)
    rn, _, _ = O.forward(tb, atm)
    assert np.abs(dn - rn).max() <= TOL


def test_zero_opacity_gives_geometric_depth(T, ctx):
    tb = S.make_tables(1, 1, 4, 4, 300, with_cia=False, with_rayleigh=False)
    tb.sigma[:] = 0.0
    atm = S.config1_atmosphere()
    atm.log10_x = np.array([-4.0])
    dn, _ = run_single(T, ctx, tb, atm)
    assert np.abs(dn - (S.R_JUP / S.R_SUN) ** 2).max() <= 1e-15


def test_cloud_top_on_layer_boundary_and_fractional(T, ctx):
    tb = S.make_tables(3, 2, 8, 8, 640, with_cia=True)
    for mode in (S.CLOUD_DISCRETE, S.CLOUD_FRACTIONAL):
        atm = S.config2_atmosphere(n_mol=2)
        atm.cloud_mode = mode
        atm.n_layers = 50
        atm.p_cloud_top = 1e6 * (1e-10) ** (17 / 50)      # exactly boundary 17
        dn, _ = run_single(T, ctx, tb, atm)
        rn, _, _ = O.forward(tb, atm)
        assert np.abs(dn - rn).max() <= TOL


def test_paper_out_of_range_rule(T, ctx):
    """Tables that do not cover the atmosphere: the paper's rule zeroes sigma below the grid."""
    tb = S.make_tables(5, 2, 7, 7, 400, with_cia=True, p_lo=1e-1, p_hi=1e5, t_lo=1000.0,
                       t_hi=2000.0, oor_mode=S.OOR_PAPER_ZERO)
    atm = S.config2_atmosphere(n_mol=2)
    dn, _ = run_single(T, ctx, tb, atm)
    rn, _, _ = O.forward(tb, atm)
    assert np.abs(dn - rn).max() <= TOL
    tb.oor_mode = S.OOR_CLAMP
    dn, _ = run_single(T, ctx, tb, atm)
    rn, _, _ = O.forward(tb, atm)
    assert np.abs(dn - rn).max() <= TOL


def test_binned_only_output(T, ctx):
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    atm = S.config1_atmosphere()
    bins = S.bins_logspaced()
    _, db = run_single(T, ctx, tb, atm, bins, native=False)
    _, rb, _ = O.forward(tb, atm, bins)
    assert np.abs(db - rb).max() <= TOL


@pytest.mark.slow
def test_config2_full_size(T, ctx):
    """Full-size model: 100 layers, 5 absorbers, 22 x 27 x 200,000 FP32 tables, CIA, cloud,
    4-node profile; every native wavenumber and the 50 bins."""
    tb = S.make_tables(2, 5, 22, 27, 200000, with_cia=True)
    atm = S.config2_atmosphere()
    bins = S.bins_logspaced()
    dn, db = run_single(T, ctx, tb, atm, bins)
    rn, rb, _ = O.forward(tb, atm, bins)
    assert np.abs(dn - rn).max() <= TOL
    assert np.abs(db - rb).max() <= TOL


def test_batch_matches_oracle_with_invalid_items(T, ctx):
    import torch
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=150)
    B = 48
    th = S.draw_theta(3001, B, spec_h)
    nl = S.draw_nlayers(3002, B)
    th[5, :2] = [-0.1, -0.2]        # sum X > 1
    th[9, 2] = -10.0                # negative temperature
    nl[11] = 0                      # no layers
    binned, status = T.forward_transit_batch(ctx, tables, spec, torch.tensor(th, device="cuda"),
                                             torch.tensor(nl, device="cuda"), bins)
    torch.cuda.synchronize()
    ref, rst = O.forward_batch(tb, spec_h, th, nl, bins_h)
    st = status.cpu().numpy()
    assert np.array_equal(st, rst)
    assert st[5] == 2 and st[9] == 2 and st[11] == 2
    got = binned.cpu().numpy()
    assert np.abs(got - ref).max() <= TOL
    assert np.all(got[st != 0] == 0.0)


def test_batch_is_deterministic_and_workspace_equivalent(T, ctx):
    import torch
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins = T.Bins(ctx, tables, *S.bins_logspaced())
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=150)
    B = 64
    th = torch.tensor(S.draw_theta(11, B, spec_h), device="cuda")
    nl = torch.tensor(S.draw_nlayers(12, B), device="cuda")
    a, _ = T.forward_transit_batch(ctx, tables, spec, th, nl, bins)
    ws = torch.empty(T.batch_workspace_size(ctx, tables, spec, bins, B), dtype=torch.uint8,
                     device="cuda")
    b, _ = T.forward_transit_batch(ctx, tables, spec, th, nl, bins, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_invalid_single_model_is_rejected(T, ctx):
    tb = S.make_tables(1, 2, 5, 5, 100, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    atm = S.config1_atmosphere()
    atm.log10_x = np.array([-0.1, -0.2])
    with pytest.raises(T.TransitError) as e:
        T.Atmosphere(ctx, tables, atm)
    assert e.value.code == T.TR_ERR_INVALID_MODEL


def test_geometry_matches_oracle_profile(T, ctx):
    """Device geometry: altitudes (FP64) to 1e-12 relative; annulus weights to FP32 rounding of
    the oracle's FP64 values; path lengths (conjugate form in FP32 with double-float altitude
    differences) within 4e-7 relative.  A relative path-length error d moves the depth by at
    most d / e * sum_j A_j / R_s^2 (about 5e-4 d here), far below the 0.1 ppm depth bar."""
    from oracle import oracle as O2
    tb = S.make_tables(2, 3, 6, 6, 64, with_cia=True)
    tables = T.XsecTables(ctx, tb)
    for n_layers, grav in ((100, S.GRAV_ALTITUDE), (37, S.GRAV_CONST), (150, S.GRAV_ALTITUDE)):
        atm = S.config2_atmosphere(n_mol=3)
        atm.n_layers = n_layers
        atm.gravity_mode = grav
        a = T.Atmosphere(ctx, tables, atm)
        z, dl, aj = a.readback()
        ref = O2.profile(tb, atm)
        assert np.allclose(z[1:], ref["z"][1:], rtol=1e-12, atol=0)
        dref = ref["DL"].astype(np.float32)
        assert np.all(np.abs(dl - dref) <= 4e-7 * np.abs(dref))
        aref = (ref["A"] / atm.r_s ** 2).astype(np.float32)
        assert np.all(np.abs(aj - aref) <= 2.5e-7 * aref)


@pytest.mark.parametrize("n_layers", [7, 150])
def test_two_kernel_form_on_long_ragged_grid(T, ctx, n_layers):
    """Native grids of >= 16,384 wavenumbers go through the streaming opacity kernel and the
    separate contraction kernel; a ragged 20,003-point grid checks the tail."""
    tb = S.make_tables(9, 3, 8, 9, 20003, with_cia=True)
    atm = S.config2_atmosphere(n_mol=3)
    atm.n_layers = n_layers
    dn, _ = run_single(T, ctx, tb, atm)
    rn, _, _ = O.forward(tb, atm)
    assert np.abs(dn - rn).max() <= TOL


def test_batch_native_output(T, ctx):
    import torch
    tb = S.make_tables(9, 2, 8, 9, 20003, with_cia=True)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced(10, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(2, cloud_mode=S.CLOUD_DISCRETE)
    spec = T.BatchSpec(spec_h, max_layers=90)
    th = S.draw_theta(77, 3, spec_h)
    nl = np.array([90, 41, 64], dtype=np.int32)
    binned, status, native = T.forward_transit_batch(
        ctx, tables, spec, torch.tensor(th, device="cuda"), torch.tensor(nl, device="cuda"),
        bins, native=True)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for b in range(3):
        atm = S.Atmosphere(n_layers=int(nl[b]), p_max=spec_h.p_max, p_min=spec_h.p_min,
                           tnode_log10p=spec_h.tnode_log10p, tnode_t=th[b, 2:6],
                           log10_x=th[b, :2], fill_frac=spec_h.fill_frac,
                           r_p=th[b, 6] * S.R_JUP, m_p=spec_h.m_p, r_s=spec_h.r_s,
                           p_cloud_top=10 ** th[b, 7], kappa_cloud=spec_h.kappa_cloud,
                           cloud_mode=S.CLOUD_DISCRETE)
        rn, rb, _ = O.forward(tb, atm, bins_h)
        assert np.abs(native[b].cpu().numpy() - rn).max() <= TOL
        assert np.abs(binned[b].cpu().numpy() - rb).max() <= TOL


def test_bounded_wait_timeout_is_reported(T, ctx):
    """Failure detection without a GPU fault: a kernel whose barrier can never complete gives
    up after a bounded number of polls, and tr_sync_status reports TR_ERR_TIMEOUT once."""
    import ctypes as C
    import torch
    from paper_1912_07759_gb300 import _native as N
    ctx.sync_status()                                    # clean before
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert ctx.lib.tr_selftest_wait_timeout(ctx.handle, s) == 0
    assert ctx.lib.tr_sync_status(ctx.handle, s) == N.TR_ERR_TIMEOUT
    assert ctx.lib.tr_sync_status(ctx.handle, s) == 0    # cleared after being reported
