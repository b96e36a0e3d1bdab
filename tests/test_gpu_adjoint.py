"""Hand-written adjoint (through the C ABI) against the FP64 oracle's exact dual-number
gradient: chi^2 and its gradient with respect to theta, and vector-Jacobian products.

Bar: |g - g_ref| <= 1e-4 max(|g_ref|, 1e-3 max|g_ref|) per component (relative 1e-4 with a
floor for components near zero); binned depths to 0.1 ppm.
"""
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


def grad_close(g, ref):
    floor = 1e-3 * np.abs(ref).max()
    return np.abs(g - ref) <= REL * np.maximum(np.abs(ref), floor)


def setup(T, ctx, n_mol, with_cia, cloud, grav=S.GRAV_ALTITUDE, n_wn=3000, nb=12):
    tb = S.make_tables(40 + n_mol, n_mol, 13, 15, n_wn, with_cia=with_cia, wn_min=4000.0,
                       wn_max=12000.0)
    tables = T.XsecTables(ctx, tb)
    bins_h = S.bins_logspaced(nb, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    spec_h = S.batch_spec(n_mol, cloud_mode=cloud)
    spec_h.gravity_mode = grav
    return tb, tables, bins_h, bins, spec_h


@pytest.mark.parametrize("n_mol,with_cia,cloud,grav", [
    (5, False, S.CLOUD_FRACTIONAL, S.GRAV_ALTITUDE),
    (3, True, S.CLOUD_FRACTIONAL, S.GRAV_ALTITUDE),
    (2, True, S.CLOUD_DISCRETE, S.GRAV_CONST),
])
def test_chi2_gradient_matches_oracle(T, ctx, n_mol, with_cia, cloud, grav):
    import torch
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, n_mol, with_cia, cloud, grav)
    B = 5
    th = S.draw_theta(700 + n_mol, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    nl = np.array([100, 40, 77, 63, 90], dtype=np.int32)
    spec = T.BatchSpec(spec_h, max_layers=100)
    sig, z = S.obs_noise(17, len(bins_h[0]))
    _, _, b_true, _ = O.chi2_grad(tb, spec_h, th[0], 100, bins_h, np.zeros(len(sig)), sig)
    obs = b_true + sig * z
    chi2, grad, binned, status = T.adjoint_transit(
        ctx, tables, spec, torch.tensor(th, device="cuda"), torch.tensor(nl, device="cuda"),
        bins, obs=torch.tensor(obs, device="cuda"), sigma_obs=torch.tensor(sig, device="cuda"))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    chi2, grad, binned = chi2.cpu().numpy(), grad.cpu().numpy(), binned.cpu().numpy()
    for b in range(B):
        c_ref, g_ref, b_ref, _ = O.chi2_grad(tb, spec_h, th[b], int(nl[b]), bins_h, obs, sig)
        assert np.abs(binned[b] - b_ref).max() <= 1e-7
        assert abs(chi2[b] - c_ref) <= 1e-3 * max(1.0, c_ref) + 2 * np.abs(
            (binned[b] - b_ref) / sig ** 2 * 2 * (b_ref - obs)).sum()
        ok = grad_close(grad[b], g_ref)
        assert ok.all(), (b, grad[b], g_ref)


def test_vector_jacobian_product_matches_oracle(T, ctx):
    import torch
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 4, True, S.CLOUD_FRACTIONAL)
    B = 4
    th = S.draw_theta(811, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    nl = np.array([60, 100, 33, 81], dtype=np.int32)
    spec = T.BatchSpec(spec_h, max_layers=100)
    rng = np.random.default_rng(5)
    gbin = rng.normal(size=(B, len(bins_h[0])))
    _, grad, _, status = T.adjoint_transit(
        ctx, tables, spec, torch.tensor(th, device="cuda"), torch.tensor(nl, device="cuda"),
        bins, gbin=torch.tensor(gbin, device="cuda"))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    grad = grad.cpu().numpy()
    sig = np.ones(len(bins_h[0]))
    for b in range(B):
        _, _, _, jac = O.chi2_grad(tb, spec_h, th[b], int(nl[b]), bins_h, np.zeros_like(sig), sig)
        ref = gbin[b] @ jac
        assert grad_close(grad[b], ref).all(), (b, grad[b], ref)


def test_invalid_items_get_zero_gradient_and_infinite_chi2(T, ctx):
    import torch
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 2, False, S.CLOUD_FRACTIONAL)
    th = S.draw_theta(9, 3, spec_h, t_range=(900.0, 1900.0))
    th[1, :2] = [-0.1, -0.2]
    spec = T.BatchSpec(spec_h, max_layers=50)
    obs = torch.zeros(len(bins_h[0]), dtype=torch.float64, device="cuda")
    sig = torch.full_like(obs, 1e-4)
    chi2, grad, _, status = T.adjoint_transit(ctx, tables, spec, torch.tensor(th, device="cuda"),
                                              None, bins, obs=obs, sigma_obs=sig)
    torch.cuda.synchronize()
    assert status.cpu().numpy().tolist() == [0, 2, 0]
    assert np.isinf(chi2[1].item()) and torch.all(grad[1] == 0)
    assert np.isfinite(chi2[0].item()) and torch.any(grad[0] != 0)


def test_autograd_function_backward_is_the_adjoint(T, ctx):
    """TransitSpectrum's backward gives the oracle's vector-Jacobian product."""
    import torch
    from paper_1912_07759_gb300 import autograd as A
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 3, True, S.CLOUD_FRACTIONAL)
    B = 3
    th_np = S.draw_theta(901, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                         lpc_range=(2.5, 4.5))
    model = A.BatchModel(ctx, tables, bins, T.BatchSpec(spec_h, max_layers=70))
    theta = torch.tensor(th_np, device="cuda", requires_grad=True)
    binned, status = A.spectrum(theta, model)
    w = torch.linspace(-1.0, 1.0, binned.shape[1], dtype=torch.float64, device="cuda")
    (binned * w).sum().backward()
    torch.cuda.synchronize()
    g = theta.grad.cpu().numpy()
    sig = np.ones(len(bins_h[0]))
    for b in range(B):
        _, _, _, jac = O.chi2_grad(tb, spec_h, th_np[b], 70, bins_h, np.zeros_like(sig), sig)
        ref = w.cpu().numpy() @ jac
        assert grad_close(g[b], ref).all(), (b, g[b], ref)


def _mixed_setup(T, ctx, tb):
    tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    bins_h = S.bins_logspaced(12, 1.2, 1.6)
    bins = T.Bins(ctx, tables, *bins_h)
    return tables, bins_h, bins


def test_mixed_adjoint_on_fp16_exact_tables(T, ctx):
    """Tables of exact powers of ten are exact in the FP16 log10 encoding, so the mixed-precision
    adjoint (FP16 tables, forward through the tensor-core contraction) differs from the FP64
    oracle only by arithmetic: the same 1e-4 relative bar as the FP32 adjoint."""
    import torch
    tb = S.make_tables(44, 3, 13, 15, 3000, with_cia=True, wn_min=4000.0, wn_max=12000.0)
    rng = np.random.default_rng(11)
    tb.sigma[:] = (10.0 ** rng.integers(-30, -25, size=tb.sigma.shape)).astype(np.float32)
    tables, bins_h, bins = _mixed_setup(T, ctx, tb)
    spec_h = S.batch_spec(3, cloud_mode=S.CLOUD_FRACTIONAL)
    B = 4
    th = S.draw_theta(705, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    nl = np.array([100, 40, 77, 63], dtype=np.int32)
    spec = T.BatchSpec(spec_h, max_layers=100)
    sig, z = S.obs_noise(19, len(bins_h[0]))
    _, _, b_true, _ = O.chi2_grad(tb, spec_h, th[0], 100, bins_h, np.zeros(len(sig)), sig)
    obs = b_true + sig * z
    chi2, grad, binned, status = T.adjoint_transit(
        ctx, tables, spec, torch.tensor(th, device="cuda"), torch.tensor(nl, device="cuda"),
        bins, obs=torch.tensor(obs, device="cuda"), sigma_obs=torch.tensor(sig, device="cuda"),
        precision=T.TR_PREC_MIXED)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    grad, binned = grad.cpu().numpy(), binned.cpu().numpy()
    for b in range(B):
        _, g_ref, b_ref, _ = O.chi2_grad(tb, spec_h, th[b], int(nl[b]), bins_h, obs, sig)
        assert np.abs(binned[b] - b_ref).max() <= 1e-6
        assert grad_close(grad[b], g_ref).all(), (b, grad[b], g_ref)


def test_mixed_adjoint_error_on_realistic_tables(T, ctx):
    """On the seeded smooth-continuum + line tables the FP16 log10 encoding itself perturbs the
    cross-sections (steps of at most 2^-9 dex near the strong lines, coarser for weak values),
    so the mixed gradient is compared with the oracle's at the tolerance that quantisation
    allows: 1 ppm on the binned depths, 2e-3 relative (with the same floor) on the gradient;
    the measured errors are printed (3.8e-4 on the seeded tables)."""
    import torch
    tb = S.make_tables(45, 3, 13, 15, 3000, with_cia=True, wn_min=4000.0, wn_max=12000.0)
    tables, bins_h, bins = _mixed_setup(T, ctx, tb)
    spec_h = S.batch_spec(3, cloud_mode=S.CLOUD_FRACTIONAL)
    B = 3
    th = S.draw_theta(706, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    spec = T.BatchSpec(spec_h, max_layers=100)
    rng = np.random.default_rng(6)
    gbin = rng.normal(size=(B, len(bins_h[0])))
    _, grad, binned, status = T.adjoint_transit(
        ctx, tables, spec, torch.tensor(th, device="cuda"), None, bins,
        gbin=torch.tensor(gbin, device="cuda"), precision=T.TR_PREC_MIXED)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    grad, binned = grad.cpu().numpy(), binned.cpu().numpy()
    sig = np.ones(len(bins_h[0]))
    worst = 0.0
    for b in range(B):
        _, _, b_ref, jac = O.chi2_grad(tb, spec_h, th[b], 100, bins_h, np.zeros_like(sig), sig)
        ref = gbin[b] @ jac
        assert np.abs(binned[b] - b_ref).max() <= 1e-6
        floor = 1e-3 * np.abs(ref).max()
        rel = np.abs(grad[b] - ref) / np.maximum(np.abs(ref), floor)
        worst = max(worst, rel.max())
        assert (rel <= 2e-3).all(), (b, grad[b], ref)
    print(f"mixed-precision gradient: max relative error vs FP64 oracle {worst:.2e}")


def test_large_batch_gradient_matches_small_batch_and_oracle(T, ctx):
    """40 atmospheres with two layer counts: the vector-Jacobian products match the oracle and
    the same atmospheres computed in a batch of 4 (the batch size changes the launch shapes of
    the adjoint's partial sums and their reduction, not the result beyond FP32 rounding)."""
    import torch
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 3, True, S.CLOUD_FRACTIONAL)
    B = 40
    th = S.draw_theta(831, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    nl = np.full(B, 100, dtype=np.int32)
    nl[1::3] = 57
    spec = T.BatchSpec(spec_h, max_layers=100)
    rng = np.random.default_rng(6)
    gbin = rng.normal(size=(B, len(bins_h[0])))
    dev = lambda x: torch.tensor(x, device="cuda")
    _, grad, _, status = T.adjoint_transit(ctx, tables, spec, dev(th), dev(nl), bins,
                                           gbin=dev(gbin))
    _, grad4, _, _ = T.adjoint_transit(ctx, tables, spec, dev(th[:4]), dev(nl[:4]), bins,
                                       gbin=dev(gbin[:4]))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    grad, grad4 = grad.cpu().numpy(), grad4.cpu().numpy()
    floor = 1e-3 * np.abs(grad4).max(axis=1, keepdims=True)
    assert (np.abs(grad[:4] - grad4) <= 1e-5 * np.maximum(np.abs(grad4), floor)).all()
    sig = np.ones(len(bins_h[0]))
    for b in (0, 1, 38):
        _, _, _, jac = O.chi2_grad(tb, spec_h, th[b], int(nl[b]), bins_h, np.zeros_like(sig), sig)
        ref = gbin[b] @ jac
        assert grad_close(grad[b], ref).all(), (b, grad[b], ref)


def test_stored_and_recomputed_opacity_give_the_same_gradient(T, ctx):
    """The backward pass reads the forward's K back when the workspace holds the whole batch
    (the default) and recomputes it from the tables on request (as for batches that outgrow
    the K buffer).  The recomputation repeats the opacity kernel's arithmetic (the same sums
    in the same order), so the two gradients are bitwise equal, and both match the oracle."""
    import torch
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 4, True, S.CLOUD_FRACTIONAL)
    B = 3
    th = S.draw_theta(905, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    nl = np.array([100, 71, 38], dtype=np.int32)
    spec = T.BatchSpec(spec_h, max_layers=100)
    rng = np.random.default_rng(9)
    gbin = rng.normal(size=(B, len(bins_h[0])))
    dev = lambda x: torch.tensor(x, device="cuda")
    grads = []
    for rk in (-1, 1):
        _, g, _, st = T.adjoint_transit(ctx, tables, spec, dev(th), dev(nl), bins,
                                        gbin=dev(gbin), recompute_k=rk)
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == 0)
        grads.append(g.cpu().numpy())
    assert np.array_equal(grads[0], grads[1]), np.abs(grads[0] - grads[1]).max()
    sig = np.ones(len(bins_h[0]))
    for b in range(B):
        _, _, _, jac = O.chi2_grad(tb, spec_h, th[b], int(nl[b]), bins_h, np.zeros_like(sig), sig)
        ref = gbin[b] @ jac
        for g in grads:
            assert grad_close(g[b], ref).all(), (b, g[b], ref)


def jac_close(J, ref, rel=REL):
    """Every entry of J [n_bin][n_theta] at the gradient bar: row j is the gradient of binned
    depth j, so |J_jk - ref_jk| <= rel max(|ref_jk|, 1e-3 max_k |ref_jk|) (the floor taken over
    the row, as for a gradient vector)."""
    floor = 1e-3 * np.abs(ref).max(axis=1, keepdims=True)
    return np.abs(J - ref) <= rel * np.maximum(np.abs(ref), floor)


def test_jacobian_matches_oracle_column_by_column(T, ctx):
    """d_jac: dD_bin/dtheta of every item from one call, against the oracle's dual-number
    Jacobian, every column (parameter) of every bin's row at the gradient bar; an invalid item
    gets zeros; in the same call the vector-Jacobian product equals the upstream gradient
    times that Jacobian."""
    import torch
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 4, True, S.CLOUD_FRACTIONAL)
    B = 5
    th = S.draw_theta(851, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    th[3, :2] = [-0.1, -0.2]                       # sum X > 1: rejected
    nl = np.array([100, 47, 88, 60, 73], dtype=np.int32)
    spec = T.BatchSpec(spec_h, max_layers=100)
    rng = np.random.default_rng(12)
    gbin = rng.normal(size=(B, len(bins_h[0])))
    dev = lambda x: torch.tensor(x, device="cuda")
    _, grad, binned, status, jac = T.adjoint_transit(ctx, tables, spec, dev(th), dev(nl), bins,
                                                     gbin=dev(gbin), want_jac=True)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    assert st.tolist() == [0, 0, 0, T.TR_ERR_INVALID_MODEL, 0]
    grad, binned, jac = grad.cpu().numpy(), binned.cpu().numpy(), jac.cpu().numpy()
    assert np.all(jac[3] == 0.0) and np.all(grad[3] == 0.0)
    sig = np.ones(len(bins_h[0]))
    for b in (0, 1, 2, 4):
        _, _, b_ref, j_ref = O.chi2_grad(tb, spec_h, th[b], int(nl[b]), bins_h,
                                         np.zeros_like(sig), sig)
        assert np.abs(binned[b] - b_ref).max() <= 1e-7
        ok = jac_close(jac[b], j_ref)
        assert ok.all(), (b, np.argwhere(~ok)[:5], jac[b][~ok][:5], j_ref[~ok][:5])
        vjp = gbin[b] @ jac[b]
        floor = 1e-3 * np.abs(vjp).max()
        assert (np.abs(grad[b] - vjp) <= 1e-5 * np.maximum(np.abs(vjp), floor)).all()


def test_jacobian_only_and_recomputed_opacity(T, ctx):
    """The Jacobian alone (no gradient pointer), with K read back and with K recomputed,
    equals the Jacobian computed next to a chi^2 gradient."""
    import torch
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 3, False, S.CLOUD_FRACTIONAL)
    B = 3
    th = S.draw_theta(852, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    spec = T.BatchSpec(spec_h, max_layers=90)
    dev = lambda x: torch.tensor(x, device="cuda")
    sig, z = S.obs_noise(23, len(bins_h[0]))
    obs = dev(0.0103 + sig * z)
    jacs = []
    for kw in (dict(obs=obs, sigma_obs=dev(sig)), dict(want_grad=False, want_binned=False),
               dict(want_grad=False, recompute_k=1)):
        out = T.adjoint_transit(ctx, tables, spec, dev(th), None, bins, want_jac=True, **kw)
        torch.cuda.synchronize()
        jacs.append(out[4].cpu().numpy())
    for J in jacs[1:]:
        floor = 1e-3 * np.abs(jacs[0]).max(axis=2, keepdims=True)
        assert (np.abs(J - jacs[0]) <= 1e-5 * np.maximum(np.abs(jacs[0]), floor)).all()
    _, _, _, j_ref = O.chi2_grad(tb, spec_h, th[1], 90, bins_h, np.zeros(len(sig)), sig)
    assert jac_close(jacs[1][1], j_ref).all()


def test_fisher_matrix_from_library_jacobian(T, ctx):
    """fisher_matrix: J^T diag(1/sigma^2) J from the library's Jacobian equals the same
    product of the oracle's Jacobian (relative 2e-4 with a floor at 1e-3 of the largest
    entry)."""
    import torch
    from paper_1912_07759_gb300 import autograd as A
    tb, tables, bins_h, bins, spec_h = setup(T, ctx, 3, True, S.CLOUD_FRACTIONAL)
    B = 2
    th = S.draw_theta(853, B, spec_h, lx_range=(-6.0, -2.5), t_range=(900.0, 1900.0),
                      lpc_range=(2.5, 4.5))
    model = A.BatchModel(ctx, tables, bins, T.BatchSpec(spec_h, max_layers=80))
    sig, _ = S.obs_noise(24, len(bins_h[0]))
    F, status = A.fisher_matrix(torch.tensor(th, device="cuda"), model,
                                torch.tensor(sig, device="cuda"))
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    F = F.cpu().numpy()
    for b in range(B):
        _, _, _, j_ref = O.chi2_grad(tb, spec_h, th[b], 80, bins_h, np.zeros(len(sig)), sig)
        F_ref = j_ref.T @ (j_ref / sig[:, None] ** 2)
        floor = 1e-3 * np.abs(F_ref).max()
        assert (np.abs(F[b] - F_ref) <= 2e-4 * np.maximum(np.abs(F_ref), floor)).all()
        assert np.allclose(F[b], F[b].T, rtol=1e-12, atol=0)
