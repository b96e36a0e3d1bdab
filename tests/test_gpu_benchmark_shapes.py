"""Parity with the FP64 oracle at the shapes the benchmark times (through the C ABI).

* forward + chi^2 gradient of 1,024 atmospheres, 5 absorbers on 13 x 15 x 10,000 tables, 50
  bins over the 946 binned-region wavenumbers, with the workspace holding K for the whole
  batch: 16 atmospheres (first, last and 14 seeded ones) against the oracle's dual-number
  gradient at 1e-4, and the Jacobian of 4 of them column by column;
* forward + gradient over the 18,907 binned-region wavenumbers of the 200,000-wavenumber
  tables with a batch that outgrows the K buffer (so the backward recomputes K), FP32 at 1e-4
  and mixed precision at the bar the FP16 encoding allows;
* the mixed-precision forward of 8 atmospheres on the full 200,000-wavenumber tables,
  <= 1 ppm at every native wavenumber (and the FP32 path <= 0.1 ppm).

The oracle runs in a thread pool (its ctypes calls release the GIL).
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
REL = 1e-4


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
def full_tables():
    return S.make_tables(2, 5, 22, 27, 200000, with_cia=True)


def pmap(fn, items):
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(items), os.cpu_count() or 1))) as ex:
        return list(ex.map(fn, items))


def grad_close(g, ref, rel=REL):
    floor = 1e-3 * np.abs(ref).max()
    return np.abs(g - ref) <= rel * np.maximum(np.abs(ref), floor)


def atm_of(spec_h, th, n_layers=100):
    """The oracle's description of batch item theta = [log10 X | T nodes | R_p/R_J | log10 P_top]."""
    m, nt = spec_h.n_mol, spec_h.n_tnodes
    return S.Atmosphere(n_layers=n_layers, p_max=spec_h.p_max, p_min=spec_h.p_min,
                        tnode_log10p=spec_h.tnode_log10p, tnode_t=th[m:m + nt],
                        log10_x=th[:m], fill_frac=spec_h.fill_frac, r_p=th[m + nt] * S.R_JUP,
                        m_p=spec_h.m_p, r_s=spec_h.r_s, p_cloud_top=10.0 ** th[m + nt + 1],
                        p_cloud_bot=spec_h.p_cloud_bot, kappa_cloud=spec_h.kappa_cloud,
                        gravity_mode=spec_h.gravity_mode, cloud_mode=spec_h.cloud_mode)


def test_adjoint_workload_1024_atmospheres_matches_oracle(T, ctx):
    import torch
    tb = S.make_tables(4, 5, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    assert bins.native_range[1] - bins.native_range[0] == 946
    spec_h = S.batch_spec(5)
    B = 1024
    spec = T.BatchSpec(spec_h, max_layers=100)
    th = S.draw_theta(4001, B, spec_h)
    sig, z = S.obs_noise(4002, bins.n_bin)
    th_true = S.draw_theta(4000, 1, spec_h)[0]
    _, _, b_true, _ = O.chi2_grad(tb, spec_h, th_true, 100, bins_h, np.zeros(len(sig)), sig)
    obs = b_true + sig * z
    ws = torch.empty(T.batch_workspace_size(ctx, tables, spec, bins, B, with_adjoint=True),
                     dtype=torch.uint8, device="cuda")
    dev = lambda x: torch.tensor(x, device="cuda")
    chi2, grad, binned, status = T.adjoint_transit(ctx, tables, spec, dev(th), None, bins,
                                                   obs=dev(obs), sigma_obs=dev(sig),
                                                   workspace=ws)
    torch.cuda.synchronize()
    chi2, grad, binned = chi2.cpu().numpy(), grad.cpu().numpy(), binned.cpu().numpy()
    status = status.cpu().numpy()
    rng = np.random.default_rng(77)
    pick = [0, B - 1] + sorted(rng.choice(np.arange(1, B - 1), 14, replace=False).tolist())

    def ref(b):
        try:
            return O.chi2_grad(tb, spec_h, th[b], 100, bins_h, obs, sig)
        except O.OracleError as e:
            return e.status
    refs = pmap(ref, pick)
    n_valid = 0
    for b, res in zip(pick, refs):
        if isinstance(res, int):
            assert status[b] == res == T.TR_ERR_INVALID_MODEL
            continue
        n_valid += 1
        c_ref, g_ref, b_ref, _ = res
        assert status[b] == 0
        assert np.abs(binned[b] - b_ref).max() <= 1e-7, b
        # chi^2 moves by what the binned depths' own differences (<= 0.1 ppm) explain
        r, dr = (b_ref - obs) / sig, np.abs(binned[b] - b_ref) / sig
        assert abs(chi2[b] - c_ref) <= np.sum((2 * np.abs(r) + dr) * dr) + 1e-9 * c_ref, b
        assert grad_close(grad[b], g_ref).all(), (b, grad[b], g_ref)
    assert n_valid >= 12
    # the Jacobian of the same batch, column by column for four of the atmospheres
    _, _, _, _, jac = T.adjoint_transit(ctx, tables, spec, dev(th), None, bins, want_grad=False,
                                        want_jac=True, workspace=ws)
    torch.cuda.synchronize()
    jac = jac.cpu().numpy()
    for b, res in list(zip(pick, refs))[:4]:
        if isinstance(res, int):
            continue
        j_ref = res[3]
        floor = 1e-3 * np.abs(j_ref).max(axis=1, keepdims=True)   # per bin's gradient row
        assert (np.abs(jac[b] - j_ref) <= REL * np.maximum(np.abs(j_ref), floor)).all(), b


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_gradient_over_200k_grid_recomputes_k_and_matches_oracle(T, ctx, full_tables, precision):
    """Binned region of the 200,000-wavenumber grid (18,907 wavenumbers), 320 atmospheres:
    their K (320 x 100 x 18,907 FP32) outgrows the 2 GiB K buffer, so the backward pass
    recomputes it.  FP32: 1e-4 against the oracle.  Mixed precision: the FP16 log10 tables
    perturb the cross-sections themselves (steps up to 2^-9 dex), so the bar is 2e-3; the
    measured error is printed."""
    import torch
    tb = full_tables
    storage = T.TR_STORE_FP32 if precision == "fp32" else T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10
    tables = T.XsecTables(ctx, tb, storage=storage)
    bins_h = S.bins_logspaced()
    bins = T.Bins(ctx, tables, *bins_h)
    assert bins.native_range[1] - bins.native_range[0] == 18907
    spec_h = S.batch_spec(5)
    B = 320
    spec = T.BatchSpec(spec_h, max_layers=100)
    th = S.draw_theta(5000, B, spec_h)
    sig, z = S.obs_noise(5002, bins.n_bin)
    obs = 0.0105 + sig * z
    dev = lambda x: torch.tensor(x, device="cuda")
    prec = T.TR_PREC_FP32 if precision == "fp32" else T.TR_PREC_MIXED
    chi2, grad, binned, status = T.adjoint_transit(ctx, tables, spec, dev(th), None, bins,
                                                   obs=dev(obs), sigma_obs=dev(sig),
                                                   precision=prec)
    torch.cuda.synchronize()
    grad, binned, status = grad.cpu().numpy(), binned.cpu().numpy(), status.cpu().numpy()
    pick = [b for b in (0, 117, 250, B - 1, 1, 2, 3) if status[b] == 0][:4]
    assert len(pick) == 4
    refs = pmap(lambda b: O.chi2_grad(tb, spec_h, th[b], 100, bins_h, obs, sig), pick)
    worst = 0.0
    bar_d, bar_g = (1e-7, REL) if precision == "fp32" else (1e-6, 2e-3)
    for b, (c_ref, g_ref, b_ref, _) in zip(pick, refs):
        assert np.abs(binned[b] - b_ref).max() <= bar_d, b
        floor = 1e-3 * np.abs(g_ref).max()
        rel = np.abs(grad[b] - g_ref) / np.maximum(np.abs(g_ref), floor)
        worst = max(worst, float(rel.max()))
        assert (rel <= bar_g).all(), (b, grad[b], g_ref)
    print(f"{precision} gradient over 18,907 wavenumbers, K recomputed: max relative error "
          f"vs FP64 oracle {worst:.2e}")


def test_mixed_forward_full_tables_batch_within_1ppm(T, ctx, full_tables):
    """Eight atmospheres from the priors on the full 22 x 27 x 200,000 tables, native spectrum:
    mixed precision <= 1 ppm and FP32 <= 0.1 ppm at every native wavenumber."""
    import torch
    tb = full_tables
    tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    bins = T.Bins(ctx, tables, *S.bins_logspaced())
    spec_h = S.batch_spec(5)
    B = 8
    spec = T.BatchSpec(spec_h, max_layers=100)
    th = S.draw_theta(5000, B, spec_h)
    out = {}
    for name, prec in (("mixed", T.TR_PREC_MIXED), ("fp32", T.TR_PREC_FP32)):
        _, st, nat = T.forward_transit_batch(ctx, tables, spec, torch.tensor(th, device="cuda"),
                                             None, bins, precision=prec, native=True)
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == 0)
        out[name] = nat.cpu().numpy()
    refs = pmap(lambda b: O.forward(tb, atm_of(spec_h, th[b]))[0], list(range(B)))
    err = {k: max(float(np.abs(v[b] - refs[b]).max()) for b in range(B)) for k, v in out.items()}
    print(f"200,000-wavenumber batch of {B}: max |D - oracle| mixed {err['mixed'] * 1e6:.4f} ppm, "
          f"FP32 {err['fp32'] * 1e6:.5f} ppm")
    assert err["mixed"] <= 1e-6
    assert err["fp32"] <= 1e-7
