"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: numbers the paper prints
(tests/golden/paper_values.json), closed forms of an isothermal exponential atmosphere,
brute-force chord integration, invariants of the binning, and finite differences of the
oracle's own value for its dual-number gradient.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07759_gb300 import synthetic as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
KB, AMU, GN = 1.380649e-23, 1.66053906660e-27, 6.67430e-11
R_J, M_J, R_SUN = S.R_JUP, S.M_JUP, S.R_SUN


def const_tables(sigma=0.0, n_wn=3, n_mol=1, mass_abs=None, ray=None, cia=None, cia_pair=None,
                 t_grid=(300.0, 3000.0), p_grid=(1e-6, 1e8), oor=S.OOR_CLAMP):
    """Tiny tables with sigma constant over (P, T, wn)."""
    wn = np.linspace(5000.0, 5002.0, n_wn)
    p = np.array(p_grid, dtype=np.float64)
    t = np.array(t_grid, dtype=np.float64)
    sig = np.full((n_mol, len(p), len(t), n_wn), sigma, dtype=np.float32)
    species = tuple(S.ABSORBERS[:n_mol]) + ("H2", "He")
    mass = np.array([S.MASS_AMU[s] for s in species])
    if mass_abs is not None:
        mass[:n_mol] = mass_abs
    if cia is None:
        tc, pairs, ca = np.zeros(0), np.zeros((0, 2), np.int32), np.zeros((0, 0, n_wn))
    else:
        tc = t.copy()
        pairs = np.array(cia_pair, dtype=np.int32).reshape(-1, 2)
        ca = np.full((pairs.shape[0], len(tc), n_wn), cia, dtype=np.float64)
    rr = None
    if ray is not None:
        rr = np.zeros((len(species), n_wn))
        for s, v in ray.items():
            rr[species.index(s)] = v
    return S.Tables(p_grid=p, t_grid=t, wn_grid=wn, sigma=sig, species=species, mass_amu=mass,
                    t_grid_cia=tc, cia_pair=pairs, cia=ca, rayleigh=rr, oor_mode=oor)


def iso_atm(n_layers=100, T=1500.0, log10_x=(-4.0,), fill=(0.83, 0.17), grav=S.GRAV_CONST,
            p_max=1e6, p_min=1e-4, **kw):
    return S.Atmosphere(n_layers=n_layers, p_max=p_max, p_min=p_min,
                        tnode_log10p=np.array([6.0]), tnode_t=np.array([T]),
                        log10_x=np.array(log10_x, dtype=np.float64),
                        fill_frac=np.array(fill), r_p=R_J, m_p=M_J, r_s=R_SUN,
                        gravity_mode=grav, **kw)


def mu_of(tb, atm):
    x = 10.0 ** np.asarray(atm.log10_x)
    rem = 1.0 - x.sum()
    X = np.concatenate([x, np.asarray(atm.fill_frac) * rem])
    return float((X * tb.mass_amu).sum()), X


def scale_height(tb, atm):
    mu, _ = mu_of(tb, atm)
    g = GN * atm.m_p / atm.r_p ** 2
    return KB * atm.tnode_t[0] / (mu * AMU * g)


def z_eff_exponential(H, tau0):
    """Effective height of an exponential absorber: int_0^inf (1 - exp(-tau0 e^{-z/H})) dz
    = H (gamma + ln tau0 + E1(tau0))."""
    from scipy.special import exp1
    return H * (np.euler_gamma + np.log(tau0) + exp1(tau0))


# ------------------------------------------------------------------------------- paper values
def test_paper_masses_and_radius_are_the_ones_used():
    """The masses and R_J used by the synthetic workloads are the paper's (Sec. 8.1, 8.2)."""
    for k, v in GOLD["mass_amu"]["value"].items():
        if k in S.MASS_AMU:
            assert S.MASS_AMU[k] == v
    assert S.R_JUP == GOLD["R_J_m"]["value"]


def test_mu_fill_convention_matches_paper_derived_mu():
    """P7: He = 0.17 * H2 of the remainder gives the paper's derived mu of 2.29-2.31."""
    r = GOLD["he_h2_ratio"]["value"]
    tb = const_tables()
    atm = iso_atm(log10_x=(-6.0,), fill=(1.0 / (1.0 + r), r / (1.0 + r)))
    p = O.profile(tb, atm)
    lo, hi = GOLD["mu_derived"]["value"]
    assert lo <= p["mu"] <= hi
    assert abs(p["mu"] - 2.3045) < 2e-4
    # the literal reading (H2 = 0.17 He) would give a heavy atmosphere, outside the range
    atm2 = iso_atm(log10_x=(-6.0,), fill=(r / (1.0 + r), 1.0 / (1.0 + r)))
    assert O.profile(tb, atm2)["mu"] > 3.0


def test_config1_depth_is_plausible():
    """P10 (plausibility, not a pin): a config-1 model lands near the paper's library
    example depth of about 0.0106 (Sec. 3)."""
    tb = S.make_tables(1, 2, 13, 15, 2000, with_cia=False)
    dn, _, _ = O.forward(tb, S.config1_atmosphere())
    assert 0.0100 < np.median(dn) < 0.0115


# ---------------------------------------------------------------------------- closed forms
def test_zero_opacity_gives_geometric_depth():
    """P1: with no opacity at all the depth is (R_p / R_s)^2 at every wavenumber."""
    tb = const_tables(0.0)
    dn, _, _ = O.forward(tb, iso_atm(grav=S.GRAV_ALTITUDE))
    ref = (R_J / R_SUN) ** 2
    assert np.all(np.abs(dn - ref) <= 4e-16 * ref)          # a couple of ulps
    assert abs(ref - 0.010098271011134767) < 1e-17


def test_opaque_atmosphere_gives_top_radius():
    """P2: opaque everywhere -> depth = r_N^2 / R_s^2, with z_N = H ln(p_max/p_min) for an
    isothermal atmosphere in constant gravity."""
    tb = const_tables(0.0)
    atm = iso_atm(cloud_mode=S.CLOUD_DISCRETE, p_cloud_top=1e-9, kappa_cloud=1e3)
    dn, _, _ = O.forward(tb, atm)
    H = scale_height(tb, atm)
    zN = H * np.log(atm.p_max / atm.p_min)
    ref = (R_J + zN) ** 2 / R_SUN ** 2
    assert np.allclose(dn, ref, rtol=1e-12, atol=0)


def z_eff_curved(H, kappa0, r_p):
    """Exponential closed form with the chord length taken at the effective radius itself
    (one fixed-point step): tau0 = kappa0 sqrt(2 pi (R_p + z) H)."""
    z = z_eff_exponential(H, kappa0 * np.sqrt(2 * np.pi * r_p * H))
    return z_eff_exponential(H, kappa0 * np.sqrt(2 * np.pi * (r_p + z) * H))


def test_opaque_non_isothermal_top_radius():
    """a4 with a temperature gradient: for T linear in ln P between nodes at p_max and p_min
    and constant gravity, z_N = k (T_bot + T_top)/2 ln(p_max/p_min) / (mu m_u g) exactly (the
    layer sum is the midpoint rule of a linear integrand), and an opaque atmosphere shows it."""
    tb = const_tables(0.0)
    atm = iso_atm(n_layers=37, cloud_mode=S.CLOUD_DISCRETE, p_cloud_top=1e-9, kappa_cloud=1e3)
    atm.tnode_log10p = np.array([6.0, -4.0])
    atm.tnode_t = np.array([2400.0, 700.0])
    mu, _ = mu_of(tb, atm)
    g = GN * M_J / R_J ** 2
    zN = KB * 0.5 * (2400.0 + 700.0) * np.log(1e10) / (mu * AMU * g)
    p = O.profile(tb, atm)
    assert abs(p["z"][-1] / zN - 1.0) < 1e-12
    dn, _, _ = O.forward(tb, atm)
    assert np.allclose(dn, (R_J + zN) ** 2 / R_SUN ** 2, rtol=1e-12, atol=0)


@pytest.mark.parametrize("n_layers", [2000])
def test_scale_height_slope_and_level_absorber(n_layers):
    """P3: isothermal, constant g, constant sigma: dR_eff/d ln sigma = H, and the level
    matches the exponential-atmosphere closed form H (gamma + ln tau0 + E1(tau0)) with
    tau0 = sigma X n0 sqrt(2 pi r H)."""
    x, s0 = 1e-4, 2e-25
    atm = iso_atm(n_layers=n_layers, log10_x=(np.log10(x),))
    H = scale_height(const_tables(), atm)
    n0 = atm.p_max / (KB * atm.tnode_t[0])
    reff = []
    for sig in (s0, s0 * np.e):
        dn, _, _ = O.forward(const_tables(sig), atm)
        reff.append(R_SUN * np.sqrt(dn[0]))
    slope = reff[1] - reff[0]
    assert abs(slope / H - 1.0) < 0.01
    z_ref = z_eff_curved(H, s0 * x * n0, R_J)
    assert abs((reff[0] - R_J) - z_ref) < 0.01 * H


def test_cia_level_has_half_scale_height():
    """CIA opacity scales as rho^2 X_a X_b (eq. cia_opt_dpth): its scale height is H/2 and
    the level follows the exponential closed form with n0^2 and the pair's mixing ratios."""
    atm = iso_atm(n_layers=2000, log10_x=(-8.0,))
    tb0 = const_tables(0.0)
    H = scale_height(tb0, atm)
    _, X = mu_of(tb0, atm)
    n0 = atm.p_max / (KB * atm.tnode_t[0])
    c0 = 1e-52
    reff = []
    for c in (c0, c0 * np.e):
        tb = const_tables(0.0, cia=c, cia_pair=[[2, 2]])       # He-He
        dn, _, _ = O.forward(tb, atm)
        reff.append(R_SUN * np.sqrt(dn[0]))
    assert abs((reff[1] - reff[0]) / (H / 2) - 1.0) < 0.01
    z_ref = z_eff_curved(H / 2, c0 * X[2] * X[2] * n0 ** 2, R_J)
    assert abs((reff[0] - R_J) - z_ref) < 0.01 * H


def test_rayleigh_level_uses_its_species_fraction():
    """Rayleigh opacity is rho X_s sigma_R (weighted like an absorber by its own species)."""
    atm = iso_atm(n_layers=2000, log10_x=(-8.0,))
    tb = const_tables(0.0, ray={"He": 3e-29})
    H = scale_height(tb, atm)
    _, X = mu_of(tb, atm)
    n0 = atm.p_max / (KB * atm.tnode_t[0])
    dn, _, _ = O.forward(tb, atm)
    z_ref = z_eff_curved(H, 3e-29 * X[2] * n0, R_J)
    assert abs((R_SUN * np.sqrt(dn[0]) - R_J) - z_ref) < 0.01 * H


def test_hydrostatic_altitude_with_inverse_square_gravity():
    """a4 with g = G M / r^2 converges to the isothermal solution
    1/R_p - 1/r = k T ln(p0/p) / (mu m_u G M)."""
    tb = const_tables()
    atm = iso_atm(n_layers=3000, grav=S.GRAV_ALTITUDE)
    p = O.profile(tb, atm)
    mu, _ = mu_of(tb, atm)
    c = KB * 1500.0 / (mu * AMU * GN * M_J)
    r_top = 1.0 / (1.0 / R_J - c * np.log(atm.p_max / atm.p_min))
    assert abs(p["z"][-1] / (r_top - R_J) - 1.0) < 1e-4
    # constant gravity: exactly z_N = H ln(p0/pN)
    p2 = O.profile(tb, iso_atm(n_layers=100))
    H = scale_height(tb, iso_atm())
    assert abs(p2["z"][-1] / (H * np.log(1e10)) - 1.0) < 1e-13


def test_pressure_grid():
    """a1: N+1 log-uniform boundaries from p_max to p_min; P_l = p_l sqrt(p_{l+1}/p_l)."""
    p = O.profile(const_tables(), iso_atm(n_layers=7))
    pb = p["pb"]
    assert pb[0] == pytest.approx(1e6, rel=1e-15) and pb[-1] == pytest.approx(1e-4, rel=1e-13)
    r = pb[1:] / pb[:-1]
    assert np.allclose(r, r[0], rtol=1e-13)
    assert np.allclose(p["P"], np.sqrt(pb[1:] * pb[:-1]), rtol=1e-15)
    assert p["delta"] == pytest.approx(np.log(1e10) / 7, rel=1e-15)


def test_npoint_temperature_profile():
    """a2: the N-point profile is linear in log P between nodes and clamped beyond them."""
    tb = const_tables()
    atm = iso_atm(n_layers=50)
    atm.tnode_log10p = np.array([5.0, 1.0, -2.0])
    atm.tnode_t = np.array([2000.0, 1000.0, 1300.0])
    p = O.profile(tb, atm)
    x = np.log10(p["P"])
    ref = np.interp(x[::-1], atm.tnode_log10p[::-1], atm.tnode_t[::-1])[::-1]
    assert np.allclose(p["T"], ref, rtol=1e-13)


def test_path_lengths_match_brute_force_chords():
    """P4: DL[j, l] equals the length of ray j (impact parameter r_j) inside shell l,
    measured by marching along the chord."""
    tb = const_tables()
    atm = iso_atm(n_layers=6, p_max=1e5, p_min=1e2, grav=S.GRAV_ALTITUDE)
    p = O.profile(tb, atm)
    r = R_J + p["z"]
    N = 6
    h = 2.0                                        # metres
    for j in range(N):
        xmax = np.sqrt(r[-1] ** 2 - r[j] ** 2)
        x = (np.arange(int(np.ceil(xmax / h))) + 0.5) * h
        rad = np.sqrt(r[j] ** 2 + x ** 2)
        shell = np.searchsorted(r, rad, side="right") - 1
        ok = (shell >= 0) & (shell < N)
        length = 2.0 * h * np.bincount(shell[ok], minlength=N)
        for l in range(N):
            if l < j:
                assert p["DL"][j, l] == 0.0
            else:
                assert abs(p["DL"][j, l] - length[l]) <= 4 * h + 1e-6 * length[l]


def test_annulus_weights_telescope():
    """R10: the annulus weights sum to r_N^2 - R_p^2 exactly in exact arithmetic."""
    p = O.profile(const_tables(), iso_atm(grav=S.GRAV_ALTITUDE))
    r = R_J + p["z"]
    assert np.isclose(p["A"].sum(), r[-1] ** 2 - R_J ** 2, rtol=1e-12)


# -------------------------------------------------------------------------------- cloud deck
# Reading R7 of eq. clouds: an absorbing deck between P_top and P_bot (P_bot defaults to the
# bottom boundary p_max).  Fractional mode: layer l, spanning boundary pressures p_l (bottom)
# > p_{l+1} (top), is covered by the fraction of its ln P extent that lies inside the deck.
# With N = 10 layers from 1e6 to 1e-4 Pa every layer is one decade: layer l spans
# log10 p in [5 - l, 6 - l], so the fractions below are read off by hand.
def cloud_of(n_layers=10, top=None, bot=0.0, mode=S.CLOUD_FRACTIONAL):
    atm = iso_atm(n_layers=n_layers, cloud_mode=mode, p_cloud_top=top, p_cloud_bot=bot,
                  kappa_cloud=1e-7)
    return O.profile(const_tables(), atm)["cloud"]


@pytest.mark.parametrize("top,bot,ref", [
    # top inside layer 2 ([1e3, 1e4] Pa): layers 0, 1 whole, layer 2 from 10^3.3 to 10^4
    (10 ** 3.3, 0.0, [1, 1, 0.7, 0, 0, 0, 0, 0, 0, 0]),
    # top exactly on the boundary between layers 2 and 3
    (1e3, 0.0, [1, 1, 1, 0, 0, 0, 0, 0, 0, 0]),
    # top above the atmosphere: every layer; below the bottom: none
    (1e-6, 0.0, [1] * 10),
    (1e7, 0.0, [0] * 10),
    # bottom of the deck set inside layer 1 (10^4.6 Pa): layer 0 outside, layer 1 from 1e4 up
    # to 10^4.6
    (10 ** 3.3, 10 ** 4.6, [0, 0.6, 0.7, 0, 0, 0, 0, 0, 0, 0]),
    # top and bottom inside the same layer
    (10 ** 3.3, 10 ** 3.8, [0, 0, 0.5, 0, 0, 0, 0, 0, 0, 0]),
    # bottom set explicitly at p_max equals the default
    (10 ** 3.3, 1e6, [1, 1, 0.7, 0, 0, 0, 0, 0, 0, 0]),
])
def test_fractional_cloud_deck_hand_values(top, bot, ref):
    """R7 fractional deck: per-layer cover fractions against values computed by hand."""
    assert np.allclose(cloud_of(top=top, bot=bot), ref, rtol=0, atol=1e-12)


def test_fractional_cloud_deck_finer_layers():
    """With N = 100 (a tenth of a decade per layer) a top at 10^2.03 Pa covers layers 0-38
    whole (each spans pressures above 10^2.1 Pa), 0.7 of layer 39 ([10^2.0, 10^2.1] Pa) and
    nothing above: the fraction is divided by the layer's own ln P extent, not by a decade."""
    c = cloud_of(n_layers=100, top=10 ** 2.03)
    ref = np.zeros(100)
    ref[:39] = 1.0
    ref[39] = 0.7
    assert np.allclose(c, ref, rtol=0, atol=1e-11)


def test_fractional_cloud_deck_is_linear_in_log_top_pressure():
    """Sweeping log10 P_top across layer 2 ([3, 4]) moves only that layer's fraction, as
    4 - log10 P_top (linear, from 1 to 0), with the layers below fully and above not at all
    covered."""
    for x in np.linspace(3.0, 4.0, 11):
        c = cloud_of(top=10 ** x)
        assert abs(c[2] - (4.0 - x)) < 1e-12
        assert np.allclose(c[:2], 1.0, rtol=0, atol=1e-12) and np.all(c[3:] == 0.0)


def test_fractional_deck_reduces_to_discrete_on_boundaries():
    """With P_top on a layer boundary the fractional deck equals the paper's discrete deck
    (a layer is cloudy when its pressure lies in the deck); off a boundary the discrete deck
    takes the partly covered layer whole when its centre is inside."""
    for k in range(11):
        top = 10.0 ** (6 - k)
        d = cloud_of(top=top, mode=S.CLOUD_DISCRETE)
        f = cloud_of(top=top)
        assert np.allclose(d, f, rtol=0, atol=1e-12)
        assert np.allclose(d, [1.0 if l < k else 0.0 for l in range(10)])
    # layer 2's centre is 10^3.5 Pa: inside a deck from 10^3.3, outside one from 10^3.7
    assert np.allclose(cloud_of(top=10 ** 3.3, mode=S.CLOUD_DISCRETE), [1, 1, 1] + [0] * 7)
    assert np.allclose(cloud_of(top=10 ** 3.7, mode=S.CLOUD_DISCRETE), [1, 1] + [0] * 8)
    assert np.allclose(cloud_of(top=10 ** 3.3, bot=10 ** 4.6, mode=S.CLOUD_DISCRETE),
                       [0, 1, 1] + [0] * 7)


def test_fractional_cloud_opacity_enters_unweighted():
    """The deck adds kappa c_l to the opacity of layer l, not multiplied by density (R7): with
    no other opacity the depth equals the one built from the oracle's path lengths and
    annulus weights (pinned above) and the hand fractions."""
    kappa = 1e-7
    atm = iso_atm(n_layers=10, cloud_mode=S.CLOUD_FRACTIONAL, p_cloud_top=10 ** 3.3,
                  kappa_cloud=kappa)
    tb = const_tables(0.0)
    p = O.profile(tb, atm)
    c = np.array([1, 1, 0.7, 0, 0, 0, 0, 0, 0, 0], dtype=np.float64)
    tau = p["DL"] @ (kappa * c)
    ref = (R_J ** 2 + np.sum(p["A"] * -np.expm1(-tau))) / R_SUN ** 2
    dn, _, _ = O.forward(tb, atm)
    assert np.all(np.abs(dn - ref) <= 1e-14 * ref)
    assert tau[0] > 0.5                          # the deck is optically significant


# ------------------------------------------------------------------------------ interpolation
def bilinear_tables():
    p = np.array([1e2, 1e3, 1e4, 1e5])
    t = np.array([500.0, 800.0, 1500.0, 2000.0, 2600.0])
    wn = np.array([1000.0, 2000.0, 3000.0])
    a, b, c, d = 3.0, 2e-5, 1e-3, 7e-8
    P, T = np.meshgrid(p, t, indexing="ij")
    f = (a + b * P + c * T + d * P * T) * 1e-26       # bilinear in (P, T)
    sig = np.stack([f * k for k in (1.0, 2.0, 0.5)], axis=-1)[None].astype(np.float32)
    tb = S.Tables(p_grid=p, t_grid=t, wn_grid=wn, sigma=sig, species=("H2O", "H2", "He"),
                  mass_amu=np.array([18.0, 2.0, 4.0]), t_grid_cia=np.zeros(0),
                  cia_pair=np.zeros((0, 2), np.int32), cia=np.zeros((0, 0, 3)), rayleigh=None)
    return tb, (a, b, c, d)


def test_interpolation_reproduces_bilinear_functions():
    """a6 (Sec. 5, linear scheme): linear in T then linear in P reproduces any function that
    is bilinear in (P, T); a swapped axis or a log-space interpolation would not."""
    tb, (a, b, c, d) = bilinear_tables()
    sig = tb.sigma.astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(20):
        P = rng.uniform(1e2, 1e5)
        T = rng.uniform(500.0, 2600.0)
        ip = np.searchsorted(tb.p_grid, P) - 1
        it = np.searchsorted(tb.t_grid, T) - 1
        # exact bilinear value built from the four float32 corner values
        tp = (P - tb.p_grid[ip]) / (tb.p_grid[ip + 1] - tb.p_grid[ip])
        tt = (T - tb.t_grid[it]) / (tb.t_grid[it + 1] - tb.t_grid[it])
        corners = sig[0, ip:ip + 2, it:it + 2, :]
        ref = ((1 - tp) * (1 - tt) * corners[0, 0] + (1 - tp) * tt * corners[0, 1]
               + tp * (1 - tt) * corners[1, 0] + tp * tt * corners[1, 1])
        got = O.interp(tb, 0, P, T)
        assert np.allclose(got, ref, rtol=1e-13)
        f = (a + b * P + c * T + d * P * T) * 1e-26
        assert np.allclose(got, f * np.array([1.0, 2.0, 0.5]), rtol=1e-6)


def test_interpolation_out_of_range_rules():
    """R6: clamp mode holds the edge value; the paper rule returns zero below the grid minimum
    and the edge value above the maximum (Sec. 5)."""
    tb, _ = bilinear_tables()
    sig = tb.sigma.astype(np.float64)
    assert np.allclose(O.interp(tb, 0, 1e6, 3000.0), sig[0, -1, -1], rtol=1e-15)
    assert np.allclose(O.interp(tb, 0, 1.0, 100.0), sig[0, 0, 0], rtol=1e-15)
    tb.oor_mode = S.OOR_PAPER_ZERO
    assert np.all(O.interp(tb, 0, 1.0, 1000.0) == 0.0)
    assert np.all(O.interp(tb, 0, 5e3, 100.0) == 0.0)
    assert np.allclose(O.interp(tb, 0, 1e6, 3000.0), sig[0, -1, -1], rtol=1e-15)
    # exactly on a grid node either bracket gives the node value
    assert np.allclose(O.interp(tb, 0, 1e3, 1500.0), sig[0, 1, 2], rtol=1e-15)


def arrhenius_tables():
    """Cross-sections that follow sigma = a e^{-b/T} exactly in T (a, b per wavenumber, a
    linear factor in P), the family the exponential scheme of Sec. 5 is built for."""
    p = np.array([1e1, 1e3, 1e5])
    t = np.array([400.0, 900.0, 1500.0, 2600.0])
    wn = np.array([1000.0, 2000.0, 3000.0, 4000.0])
    a = np.array([3e-24, 8e-25, 1e-23, 5e-26])
    b = np.array([1500.0, 4000.0, 800.0, 9000.0])
    fp = np.array([1.0, 1.7, 3.1])
    sig = (fp[:, None, None] * a[None, None, :] * np.exp(-b[None, None, :] / t[None, :, None]))
    tb = S.Tables(p_grid=p, t_grid=t, wn_grid=wn, sigma=sig[None].astype(np.float32),
                  species=("H2O", "H2", "He"), mass_amu=np.array([18.0, 2.0, 4.0]),
                  t_grid_cia=np.zeros(0), cia_pair=np.zeros((0, 2), np.int32),
                  cia=np.zeros((0, 0, 4)), rayleigh=None, interp_mode=S.INTERP_EXP)
    return tb, a, b, fp


def test_exponential_scheme_reproduces_arrhenius_law():
    """Sec. 5 exponential scheme: between two grid temperatures sigma = a e^{-b/T} is
    reproduced up to the FP32 storage of the node values (the linear scheme misses it by
    per cents); P stays linear."""
    tb, a, b, fp = arrhenius_tables()
    rng = np.random.default_rng(7)
    lin = S.Tables(**{**tb.__dict__, "interp_mode": S.INTERP_LINEAR})
    worst_lin = 0.0
    for _ in range(25):
        P = 10.0 ** rng.uniform(1.0, 5.0)
        T = rng.uniform(400.0, 2600.0)
        ip = np.searchsorted(tb.p_grid, P) - 1
        tp = (P - tb.p_grid[ip]) / (tb.p_grid[ip + 1] - tb.p_grid[ip])
        f = fp[ip] + (fp[ip + 1] - fp[ip]) * tp
        ref = f * a * np.exp(-b / T)
        got = O.interp(tb, 0, P, T)
        assert np.allclose(got, ref, rtol=3e-7)
        worst_lin = max(worst_lin, float(np.max(np.abs(O.interp(lin, 0, P, T) / ref - 1))))
    assert worst_lin > 1e-2


def test_exponential_scheme_nodes_zero_values_and_node_temperature():
    """The exponential scheme returns the node values on the grid, falls back to the linear
    value where a bracketing value is zero (a reading: the logarithm does not exist there),
    and a forward model whose temperatures sit on grid nodes gives the same depths in both
    schemes."""
    tb, a, b, fp = arrhenius_tables()
    sig = tb.sigma.astype(np.float64)
    assert np.allclose(O.interp(tb, 0, 1e3, 1500.0), sig[0, 1, 2], rtol=1e-15)
    tb.sigma[0, :, 2, 1] = 0.0                       # wavenumber 1: zero at T = 1500 K
    lin = S.Tables(**{**tb.__dict__, "interp_mode": S.INTERP_LINEAR})
    got, ref = O.interp(tb, 0, 1e3, 1200.0), O.interp(lin, 0, 1e3, 1200.0)
    assert got[1] == ref[1] and got[0] != ref[0]
    tbm = S.make_tables(1, 2, 13, 15, 800, with_cia=True)
    atm = S.config1_atmosphere()
    atm.tnode_t = np.array([float(tbm.t_grid[7])])   # isothermal, on a grid temperature
    d_lin, _, _ = O.forward(tbm, atm)
    d_exp, _, _ = O.forward(S.Tables(**{**tbm.__dict__, "interp_mode": S.INTERP_EXP}), atm)
    assert np.allclose(d_exp, d_lin, rtol=0, atol=1e-15)


# ------------------------------------------------------------------------------------ binning
def test_bin_weights_interior_one_and_partition_of_unity():
    """P6: native bins inside a target bin get w = 1 (Sec. 4.5); summed over contiguous target
    bins the weights of fully covered native bins add to 1; a constant spectrum bins to the
    same constant."""
    wn = S.wn_grid_loguniform(10000)
    c, w = S.bins_logspaced()
    W = O.bin_weights(wn, c, w)
    lam = 1e4 / wn
    inside = (lam > c[0] - w[0] / 2 + 1e-3) & (lam < c[-1] + w[-1] / 2 - 1e-3)
    tot = W.sum(axis=0)
    assert np.allclose(tot[inside], 1.0, rtol=1e-12)
    assert (W == GOLD["interior_bin_weight"]["value"]).sum() > 800
    assert np.all((W >= 0) & (W <= 1.0 + 1e-12))
    tb = const_tables(0.0, n_wn=500)
    tb.wn_grid = S.wn_grid_loguniform(500, 6000.0, 9000.0)
    atm = iso_atm(n_layers=10)
    dn, db, _ = O.forward(tb, atm, S.bins_logspaced(5, 1.2, 1.6))
    assert np.allclose(db, dn[0], rtol=1e-15)


def test_binned_uncertainty_matches_monte_carlo():
    """Sec. 4.5 propagation of uncertainties: sigma_j of the binned spectrum equals the spread
    of the binned flux over many noise draws of the native spectrum (brute force), for bins
    that cut native bins (fractional weights) as well as whole ones."""
    wn = np.geomspace(5000.0, 9000.0, 120)
    centre = np.array([1.2, 1.31, 1.45, 1.8])
    width = np.array([0.05, 0.013, 0.2, 0.1])
    rng = np.random.default_rng(11)
    flux = 0.01 + 1e-4 * rng.standard_normal(len(wn))
    sig = 1e-5 * (1.0 + rng.random(len(wn)))
    f, s = O.bin_with_uncertainty(wn, centre, width, flux, sig)
    draws = flux + sig * rng.standard_normal((20000, len(wn)))
    fb, _ = O.bin_with_uncertainty(wn, centre, width, draws)
    assert np.allclose(fb.mean(axis=0), f, rtol=0, atol=5 * s.max() / np.sqrt(20000))
    assert np.allclose(fb.std(axis=0), s, rtol=0.03)
    # a bin made of whole native bins 40..49 (edges at wavenumber midpoints, a hair inside):
    # the standard error of a mean of 10 equal uncertainties
    edge_nu = 0.5 * (wn[39:50] + wn[40:51])
    lo, hi = 1e4 / edge_nu[-1], 1e4 / edge_nu[0]
    eps = 1e-9 * (hi - lo)
    c1, w1 = np.array([(lo + hi) / 2]), np.array([hi - lo - 2 * eps])
    assert np.isclose(O.bin_weights(wn, c1, w1).sum(), 10.0, rtol=1e-6)
    _, s1 = O.bin_with_uncertainty(wn, c1, w1, flux, np.full(len(wn), 2e-5))
    assert np.allclose(s1, 2e-5 / np.sqrt(10.0), rtol=1e-6)


def test_snr_instrument_noise_level():
    """Sec. 7 SNR model: the noise is the largest binned value over the SNR, reduced by the
    square root of the number of stacked observations; with zero draws the observation is the
    binned spectrum itself."""
    rng = np.random.default_rng(12)
    binned = 0.01 + 1e-4 * rng.random((3, 20))
    obs, sig = O.snr_instrument(binned, 200.0, 1, np.zeros((3, 20)))
    assert np.array_equal(obs, binned)
    assert np.allclose(sig, binned.max(axis=1, keepdims=True) / 200.0, rtol=1e-15)
    _, sig4 = O.snr_instrument(binned, 200.0, 4, np.zeros((3, 20)))
    assert np.allclose(sig4, sig / 2.0, rtol=1e-15)
    z = rng.standard_normal((3, 20))
    obs1, _ = O.snr_instrument(binned, 200.0, 1, z)
    assert np.allclose((obs1 - binned) / sig, z, rtol=1e-12)


def test_binned_region_matches_full_spectrum_binning():
    """The batch path computes only the binned region; binning the full native spectrum must
    give the same numbers."""
    tb = S.make_tables(1, 2, 13, 15, 3000, with_cia=False)
    spec = S.batch_spec(2, cloud_mode=S.CLOUD_FRACTIONAL)
    th = S.draw_theta(5, 3, spec)
    nl = np.array([40, 55, 61], dtype=np.int32)
    bins = S.bins_logspaced()
    got, st = O.forward_batch(tb, spec, th, nl, bins)
    assert np.all(st == 0)
    Wm = O.bin_weights(tb.wn_grid, *bins)
    for b in range(3):
        atm = S.Atmosphere(n_layers=int(nl[b]), p_max=spec.p_max, p_min=spec.p_min,
                           tnode_log10p=spec.tnode_log10p, tnode_t=th[b, 2:6],
                           log10_x=th[b, :2], fill_frac=spec.fill_frac,
                           r_p=th[b, 6] * R_J, m_p=spec.m_p, r_s=spec.r_s,
                           p_cloud_top=10 ** th[b, 7], kappa_cloud=spec.kappa_cloud,
                           cloud_mode=S.CLOUD_FRACTIONAL)
        dn, _, _ = O.forward(tb, atm)
        ref = (Wm @ dn) / Wm.sum(axis=1)
        assert np.allclose(got[b], ref, rtol=1e-13, atol=0)


# ------------------------------------------------------------------------------- monotonicity
def test_depth_increases_with_abundance_when_mass_matches_background():
    """P5: with the absorber as heavy as the background (mu fixed) more absorber can only
    raise the depth, at every wavenumber."""
    tb = S.make_tables(1, 1, 13, 15, 400, with_cia=False, with_rayleigh=False)
    mu_bg = 0.83 * 2.01588 + 0.17 * 4.002602
    tb.mass_amu[0] = mu_bg
    prev = None
    for lx in (-7.0, -6.0, -5.0, -4.0, -3.0):
        atm = S.config1_atmosphere()
        atm.log10_x = np.array([lx])
        dn, _, _ = O.forward(tb, atm)
        if prev is not None:
            assert np.all(dn >= prev)
        prev = dn


# ----------------------------------------------------------------------------------- tiny case
def test_two_layer_case_by_hand():
    """P8: N = 2, three wavenumbers, one molecule on a 2 x 2 table, written out by hand."""
    p = np.array([1e1, 1e6]); t = np.array([1000.0, 2000.0]); wn = np.array([1e3, 2e3, 3e3])
    sig = np.zeros((1, 2, 2, 3), np.float32)
    sig[0, 0, 0] = [1e-28, 2e-28, 3e-28]; sig[0, 0, 1] = [2e-28, 1e-28, 5e-28]
    sig[0, 1, 0] = [4e-28, 1e-29, 2e-28]; sig[0, 1, 1] = [8e-28, 6e-28, 1e-28]
    tb = S.Tables(p_grid=p, t_grid=t, wn_grid=wn, sigma=sig, species=("H2O", "H2", "He"),
                  mass_amu=np.array([18.01528, 2.01588, 4.002602]), t_grid_cia=np.zeros(0),
                  cia_pair=np.zeros((0, 2), np.int32), cia=np.zeros((0, 0, 3)), rayleigh=None)
    atm = S.Atmosphere(n_layers=2, p_max=1e5, p_min=1e3, tnode_log10p=np.array([6.0]),
                       tnode_t=np.array([1200.0]), log10_x=np.array([-3.0]),
                       fill_frac=np.array([0.9, 0.1]), r_p=R_J, m_p=M_J, r_s=R_SUN)
    dn, _, tau = O.forward(tb, atm, want_tau=True)
    # by hand
    pb = [1e5, 1e4, 1e3]
    P = [np.sqrt(1e5 * 1e4), np.sqrt(1e4 * 1e3)]
    d = np.log(10.0)
    X = 1e-3
    mu = X * 18.01528 + (1 - X) * (0.9 * 2.01588 + 0.1 * 4.002602)
    z0 = 0.0
    g0 = GN * M_J / R_J ** 2
    H0 = KB * 1200.0 / (mu * AMU * g0)
    z1 = H0 * d
    g1 = GN * M_J / (R_J + z1) ** 2
    H1 = KB * 1200.0 / (mu * AMU * g1)
    z2 = z1 + H1 * d
    r0, r1, r2 = R_J, R_J + z1, R_J + z2
    tt = 0.2
    s = sig.astype(np.float64)[0]
    K = []
    for l in range(2):
        tp = (P[l] - 1e1) / (1e6 - 1e1)
        a1 = s[0, 0] + (s[0, 1] - s[0, 0]) * tt
        a2 = s[1, 0] + (s[1, 1] - s[1, 0]) * tt
        K.append(P[l] / (KB * 1200.0) * X * (a1 + (a2 - a1) * tp))
    DL00 = 2 * np.sqrt(r1 ** 2 - r0 ** 2)
    DL01 = 2 * (np.sqrt(r2 ** 2 - r0 ** 2) - np.sqrt(r1 ** 2 - r0 ** 2))
    DL11 = 2 * np.sqrt(r2 ** 2 - r1 ** 2)
    tau0 = DL00 * K[0] + DL01 * K[1]
    tau1 = DL11 * K[1]
    D = (r0 ** 2 + (r1 ** 2 - r0 ** 2) * (1 - np.exp(-tau0))
         + (r2 ** 2 - r1 ** 2) * (1 - np.exp(-tau1))) / R_SUN ** 2
    assert np.allclose(tau[0], tau0, rtol=1e-9)
    assert np.allclose(tau[1], tau1, rtol=1e-9)
    assert np.allclose(dn, D, rtol=1e-11)


# ---------------------------------------------------------------------------------- gradients
def test_invalid_models_are_rejected():
    """Model rejection (Sec. 6): sum X > 1, T <= 0, non-monotone nodes, no layers."""
    tb = S.make_tables(1, 2, 13, 15, 300, with_cia=False)
    spec = S.batch_spec(2)
    th = S.draw_theta(3, 5, spec)
    th[0, :2] = [-0.1, -0.2]           # sum X > 1
    th[1, 3] = -500.0                  # negative temperature node
    th[2, :] = np.nan
    nl = np.array([60, 60, 60, 0, 60, 60], dtype=np.int32)
    th = np.vstack([th, th[4]])
    th[5, 2] = -10.0                   # negative node at the bottom boundary, layers stay > 0
    _, st = O.forward_batch(tb, spec, th, nl, S.bins_logspaced())
    assert list(st) == [2, 2, 2, 2, 0, 2]


def test_dual_gradient_matches_central_differences():
    """P9: the oracle's exact (dual-number) gradient of chi^2 equals central differences of
    the oracle's own chi^2, away from kinks."""
    tb = S.make_tables(4, 3, 13, 15, 1500, with_cia=True)
    spec = S.batch_spec(3)
    th = S.draw_theta(11, 1, spec, lx_range=(-6, -3), t_range=(900, 1900))[0]
    th[-1] = 3.3
    bins = S.bins_logspaced(10, 1.2, 1.6)
    sig, z = S.obs_noise(4, 10)
    _, _, b0, _ = O.chi2_grad(tb, spec, th, 40, bins, np.zeros(10), sig)
    obs = b0 + 3 * sig * z
    c, g, b, jac = O.chi2_grad(tb, spec, th, 40, bins, obs, sig)
    steps = np.full(th.shape, 1e-5)
    steps[3:7] = 1e-3                # temperatures in K
    for k in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[k] += steps[k]; tm[k] -= steps[k]
        cp = O.chi2_grad(tb, spec, tp, 40, bins, obs, sig)
        cm = O.chi2_grad(tb, spec, tm, 40, bins, obs, sig)
        fd = (cp[0] - cm[0]) / (2 * steps[k])
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * np.abs(g).max()), k
        fdj = (cp[2] - cm[2]) / (2 * steps[k])
        scale = np.abs(jac[:, k]).max()
        roundoff = 8e-18 / steps[k]          # a few ulps of a depth of 0.01, over 2h
        assert np.all(np.abs(fdj - jac[:, k]) <= 1e-6 * scale + roundoff), k


# ---- emission model of Sec. 4 (the oracle's statement of the next hot-path row) ----

def test_gauss_legendre_nodes_match_library():
    """The cos(theta) quadrature: n-point Gauss-Legendre on [0, 1] equals numpy's nodes and
    weights on [-1, 1] mapped to [0, 1], and integrates mu^k exactly up to k = 2n - 1."""
    for n in range(1, 11):
        x, w = O.gauss_legendre01(n)
        t, v = np.polynomial.legendre.leggauss(n)
        order = np.argsort(x)
        assert np.allclose(np.sort(x), (t + 1.0) / 2.0, rtol=0, atol=1e-14)
        assert np.allclose(w[order], v[np.argsort(t)] / 2.0, rtol=0, atol=1e-14)
        for k in range(2 * n):
            assert np.isclose((w * x ** k).sum(), 1.0 / (k + 1), rtol=1e-13)


def test_planck_integrates_to_stefan_boltzmann():
    """The source function: the integral of B over wavenumber is sigma_SB T^4 / pi (and B tends
    to the Rayleigh-Jeans form 2 c k T nu^2 at low wavenumber)."""
    sigma_sb, k_b, c = 5.670374419e-8, 1.380649e-23, 299792458.0   # CODATA 2018
    for T in (300.0, 1500.0, 3000.0):
        nu = np.linspace(1e-3, 60.0 * k_b * T / (6.62607015e-34 * c) / 100.0, 400001)   # 1/cm
        B = O.planck(nu, T)
        integral = np.trapezoid(B, nu * 100.0)
        assert np.isclose(integral, sigma_sb * T ** 4 / np.pi, rtol=1e-6)
        lo = np.array([1e-3])
        assert np.isclose(O.planck(lo, T)[0], 2.0 * c * k_b * T * (100.0 * lo[0]) ** 2,
                          rtol=1e-5)


def test_emission_isothermal_atmosphere_is_a_blackbody():
    """Whatever the opacity, an atmosphere and surface at one temperature emit B(T): the
    layers' terms and the surface term add up to it exactly (Sec. 4, emission model)."""
    tb = S.make_tables(5, 2, 13, 15, 600, with_cia=True)
    atm = S.config1_atmosphere()
    for n_mu in (1, 4, 9):
        r = O.emission(tb, atm, n_mu=n_mu, t_star=5800.0)
        T = float(atm.tnode_t[0])
        ref = O.planck(tb.wn_grid, T) / O.planck(tb.wn_grid, 5800.0) * (atm.r_p / atm.r_s) ** 2
        assert np.allclose(r, ref, rtol=1e-12, atol=0)


def test_emission_without_opacity_shows_the_surface():
    """Zero opacity: the flux ratio is B(T_s)/B(T_star) (R_p/R_s)^2 with T_s the profile's
    temperature at p_max (here the bottom node of a two-node profile)."""
    tb = const_tables(0.0, n_wn=5)
    atm = iso_atm(n_layers=40)
    atm.tnode_log10p = np.array([6.0, -4.0])
    atm.tnode_t = np.array([2100.0, 900.0])
    r = O.emission(tb, atm, n_mu=4, t_star=6000.0)
    ref = O.planck(tb.wn_grid, 2100.0) / O.planck(tb.wn_grid, 6000.0) * (atm.r_p / atm.r_s) ** 2
    assert np.allclose(r, ref, rtol=1e-13, atol=0)


def test_emission_angular_integral_converges_to_e3():
    """The angular part: with many Gauss-Legendre points, sum_i x_i w_i e^{-tau/x_i} becomes
    int_0^1 mu e^{-tau/mu} dmu = E_3(tau), so the flux equals the exponential-integral form of
    the same layered atmosphere (layer optical depths from the oracle's profile and a constant
    cross-section)."""
    special = pytest.importorskip("scipy.special")
    sigma = 2e-27
    tb = const_tables(sigma, n_wn=3)
    atm = iso_atm(n_layers=30, log10_x=(-3.0,))
    atm.tnode_log10p = np.array([6.0, 2.0, -4.0])
    atm.tnode_t = np.array([2000.0, 1300.0, 800.0])
    pf = O.profile(tb, atm)
    X0 = pf["X"][:, 0]                                   # the absorber in every layer
    dtau = pf["rho"] * X0 * sigma * np.diff(pf["z"])        # per layer, l = 0 at the bottom
    tau_below_top = np.concatenate([[0.0], np.cumsum(dtau[::-1])])   # boundary optical depths from the top
    T_layers = pf["T"][::-1]                                 # from the top down
    Ts = 2000.0
    for i, nu in enumerate(tb.wn_grid):
        flux = 0.0
        for l in range(len(T_layers)):
            b = O.planck(np.array([nu]), T_layers[l])[0]
            flux += b * (special.expn(3, tau_below_top[l]) - special.expn(3, tau_below_top[l + 1]))
        flux += O.planck(np.array([nu]), Ts)[0] * special.expn(3, tau_below_top[-1])
        ref = flux / (O.planck(np.array([nu]), 5800.0)[0] * 0.5) * (atm.r_p / atm.r_s) ** 2
        r = O.emission(tb, atm, n_mu=48, t_star=5800.0)[i]
        assert np.isclose(r, ref, rtol=1e-9), (i, r, ref)
    # and few points are a coarse but close approximation
    r4 = O.emission(tb, atm, n_mu=4, t_star=5800.0)
    r48 = O.emission(tb, atm, n_mu=48, t_star=5800.0)
    assert np.allclose(r4, r48, rtol=2e-2)


# ------------------------------------------------------------- Guillot2010 temperature profile
# Readings G1-G3 (Sec. 4.2 names the profile and its parameters T_irr, kappa_irr, kappa_v1,
# kappa_v2, alpha): Guillot (2010) radiative equilibrium with two visible channels,
#   T^4 = 3/4 T_int^4 (2/3 + tau) + 3/4 T_irr^4 [(1 - alpha) xi(g1) + alpha xi(g2)],
# tau = kappa_irr P / g_s, g_s = G M_p / R_p^2, g_i = kappa_v,i / kappa_irr.  The pins below
# test it through its limits and expansions, not by restating it.
def guillot_atm(tirr, k_ir, kv1, kv2, alpha, t_int=100.0, n_layers=60, p_max=1e7, p_min=1e-3):
    return S.Atmosphere(n_layers=n_layers, p_max=p_max, p_min=p_min,
                        tnode_log10p=np.array([6.0]), tnode_t=np.array([1.0]),
                        log10_x=np.array([-6.0]), fill_frac=np.array([0.83, 0.17]),
                        r_p=R_J, m_p=M_J, r_s=R_SUN, gravity_mode=S.GRAV_CONST,
                        t_profile=S.TPROF_GUILLOT,
                        guillot=np.array([tirr, k_ir, kv1, kv2, alpha], dtype=np.float64),
                        t_int=t_int)


def guillot_tau(atm, P):
    return atm.guillot[1] * P / (GN * atm.m_p / atm.r_p ** 2)


def test_expint_matches_library():
    """E_1 and E_2 of the oracle (power series / continued fraction) equal scipy's."""
    special = pytest.importorskip("scipy.special")
    x = np.concatenate([np.logspace(-10, 2.3, 200), [2.0, 2.0 + 1e-12, 1.0]])
    e1, e2 = O.expint(x)
    assert np.allclose(e1, special.exp1(x), rtol=1e-12, atol=0)
    assert np.allclose(e2, special.expn(2, x), rtol=1e-12, atol=1e-300)


def test_guillot_without_irradiation_is_the_eddington_profile():
    """T_irr = 0: T^4 = 3/4 T_int^4 (tau + 2/3), the grey Eddington atmosphere, in every layer
    (tau from the layer pressure and the surface gravity, G1)."""
    atm = guillot_atm(0.0, 0.02, 0.004, 0.05, 0.3, t_int=700.0)
    p = O.profile(const_tables(), atm)
    tau = guillot_tau(atm, p["P"])
    assert np.allclose(p["T"] ** 4, 0.75 * 700.0 ** 4 * (tau + 2.0 / 3.0), rtol=1e-12, atol=0)


def test_guillot_top_and_deep_limits():
    """tau -> 0: xi -> 2/3 + 2g/3 (E_2(0) = 1); tau -> infinity: xi -> 2/3 + 2/(3g), so
    T^4 - 3/4 T_int^4 (2/3 + tau) tends to 3/4 T_irr^4 [(1-a)(2/3 + 2/(3g1)) + a(2/3 + 2/(3g2))]."""
    k_ir, kv1, kv2, a, tirr, tint = 1e-2, 3e-3, 4e-2, 0.35, 1800.0, 150.0
    g1, g2 = kv1 / k_ir, kv2 / k_ir
    # top: tau ~ 1e-13 at the top layer
    top = guillot_atm(tirr, k_ir, kv1, kv2, a, t_int=tint, n_layers=20, p_max=1e-6, p_min=1e-8)
    p = O.profile(const_tables(), top)
    ref0 = tint ** 4 / 2 + 0.75 * tirr ** 4 * ((1 - a) * (2 / 3 + 2 * g1 / 3) + a * (2 / 3 + 2 * g2 / 3))
    assert abs(p["T"][-1] ** 4 / ref0 - 1.0) < 1e-9
    # deep: g tau > 100 in the bottom layers
    deep = guillot_atm(tirr, k_ir, kv1, kv2, a, t_int=tint, n_layers=20, p_max=1e12, p_min=1e11)
    p = O.profile(const_tables(), deep)
    tau = guillot_tau(deep, p["P"][0])
    assert min(g1, g2) * tau > 100
    irr = p["T"][0] ** 4 - 0.75 * tint ** 4 * (2 / 3 + tau)
    ref_inf = 0.75 * tirr ** 4 * ((1 - a) * (2 / 3 + 2 / (3 * g1)) + a * (2 / 3 + 2 / (3 * g2)))
    assert abs(irr / ref_inf - 1.0) < 1e-6


def test_guillot_small_tau_expansion():
    """Near the top, xi(g, tau) = 2/3 + 2g/3 + tau + (2 g^2 tau / 3)(ln(g tau) + gamma_E - 1)
    + O(tau^2 ln tau) (from E_2(x) = 1 + x (ln x + gamma_E - 1) + O(x^2)): the first-order
    coefficient checks every term of xi at once."""
    g = 2.5
    kw = dict(tirr=1500.0, k_ir=1e-2, kv1=2.5e-2, kv2=1.0)
    atm = guillot_atm(t_int=0.0, alpha=0.0, n_layers=8, p_max=1e-2, p_min=1e-4, **kw)
    p = O.profile(const_tables(), atm)
    xi = p["T"] ** 4 / (0.75 * 1500.0 ** 4)
    tau = guillot_tau(atm, p["P"])
    assert tau.max() < 1e-5
    first = (xi - (2 / 3 + 2 * g / 3)) / tau
    ref = 1.0 + (2 * g * g / 3) * (np.log(g * tau) + np.euler_gamma - 1.0)
    assert np.allclose(first, ref, rtol=2e-3, atol=0)


def test_guillot_large_tau_approach():
    """Deep in, xi(g, tau) - (2/3 + 2/(3g)) decays as e^{-g tau} [c1/tau + c2/tau^2 + c3/tau^3
    + c4/tau^4 + ...] with c1 = 2/3 - 2/g^2, c2 = 8/g^3 - 4/(3g), c3 = 4(g^2 - 10)/g^4,
    c4 = 16(15 - g^2)/g^5 (from the asymptotic series E_2(x) ~ e^{-x}/x sum_k (-1)^k (k+1)!/x^k;
    the terms of order tau e^{-g tau} cancel, which fixes the 1/2 of (g tau/2 - 1) against the
    tau^2/2 of the E_2 term).  The series is asymptotic: at g tau = 18-25 four terms are good
    to better than 1 %."""
    g = 0.4
    atm = guillot_atm(1500.0, 1e-2, 4e-3, 1.0, 0.0, t_int=0.0, n_layers=40, p_max=1.7e5,
                      p_min=1.1e5)
    p = O.profile(const_tables(), atm)
    xi = p["T"] ** 4 / (0.75 * 1500.0 ** 4)
    tau = guillot_tau(atm, p["P"])
    sel = (g * tau > 18) & (g * tau < 25)
    assert sel.sum() >= 5
    t = tau[sel]
    lhs = (xi[sel] - (2 / 3 + 2 / (3 * g))) * np.exp(g * t)
    c = [2 / 3 - 2 / g ** 2, 8 / g ** 3 - 4 / (3 * g), 4 * (g * g - 10) / g ** 4,
         16 * (15 - g * g) / g ** 5]
    rhs = sum(ci / t ** (i + 1) for i, ci in enumerate(c))
    assert np.allclose(lhs, rhs, rtol=1e-2, atol=0)


def test_guillot_channel_symmetry_and_superposition():
    """Swapping the two visible channels with alpha -> 1 - alpha leaves the profile unchanged;
    equal channels make alpha irrelevant; T^4 is the sum of its internal and irradiated
    parts."""
    tb = const_tables()
    base = O.profile(tb, guillot_atm(1600.0, 1e-2, 2e-3, 5e-2, 0.3))["T"]
    swap = O.profile(tb, guillot_atm(1600.0, 1e-2, 5e-2, 2e-3, 0.7))["T"]
    assert np.allclose(base, swap, rtol=1e-13, atol=0)
    e1 = O.profile(tb, guillot_atm(1600.0, 1e-2, 7e-3, 7e-3, 0.1))["T"]
    e2 = O.profile(tb, guillot_atm(1600.0, 1e-2, 7e-3, 7e-3, 0.9))["T"]
    assert np.allclose(e1, e2, rtol=1e-13, atol=0)
    both = O.profile(tb, guillot_atm(1600.0, 1e-2, 2e-3, 5e-2, 0.3, t_int=400.0))["T"] ** 4
    irr = O.profile(tb, guillot_atm(1600.0, 1e-2, 2e-3, 5e-2, 0.3, t_int=0.0))["T"] ** 4
    internal = O.profile(tb, guillot_atm(0.0, 1e-2, 2e-3, 5e-2, 0.3, t_int=400.0))["T"] ** 4
    assert np.allclose(both, irr + internal, rtol=1e-12, atol=0)


def test_guillot_invalid_parameters_are_rejected():
    tb = const_tables()
    for args in ((-10.0, 1e-2, 1e-3, 1e-3, 0.5), (1500.0, 1e-2, 1e-3, 1e-3, 1.2),
                 (1500.0, 1e-2, 1e-3, 1e-3, -0.1), (1500.0, 0.0, 1e-3, 1e-3, 0.5)):
        with pytest.raises(O.OracleError):
            O.profile(tb, guillot_atm(*args))


# ------------------------------------------------------------------ two-layer gas profile
# Readings L1-L2 (Sec. 4.3 names the profile with surface and top mixing ratios): X_surf below
# the switch pressure, X_top above it; a layer straddling the switch takes f X_surf +
# (1 - f) X_top with f the fraction of its ln P extent below the switch.  N = 10 layers from
# 1e6 to 1e-4 Pa: layer l spans log10 P in [5 - l, 6 - l].
def two_layer_atm(x_surf, x_top, lp_sw, n_layers=10, **kw):
    return iso_atm(n_layers=n_layers, log10_x=x_surf, gas_mode=S.GAS_TWOLAYER,
                   log10_x_top=np.array(x_top, dtype=np.float64),
                   log10_p_switch=np.array(lp_sw, dtype=np.float64), **kw)


def test_two_layer_hand_values_and_per_layer_mean_molecular_weight():
    """Switch at 10^3.3 Pa inside layer 2 ([1e3, 1e4] Pa): layers 0-1 carry X_surf, layer 2
    0.7 X_surf + 0.3 X_top, layers 3-9 X_top; fill gases take each layer's remainder; mu and
    the constant-gravity altitude steps k T Delta / (mu_l m_u g) follow layer by layer."""
    tb = const_tables(n_mol=2, mass_abs=[18.01528, 44.0095])
    xs, xt = np.array([1e-2, 3e-2]), np.array([1e-4, 2e-3])
    atm = two_layer_atm(np.log10(xs), np.log10(xt), [3.3, 3.3])
    p = O.profile(tb, atm)
    f = np.array([1, 1, 0.7, 0, 0, 0, 0, 0, 0, 0], dtype=np.float64)
    X = f[:, None] * xs[None, :] + (1 - f[:, None]) * xt[None, :]
    rem = 1.0 - X.sum(axis=1)
    Xall = np.concatenate([X, 0.83 * rem[:, None], 0.17 * rem[:, None]], axis=1)
    assert np.allclose(p["X"], Xall, rtol=1e-12, atol=0)
    mu = Xall @ tb.mass_amu
    assert np.allclose(p["mu_l"], mu, rtol=1e-12, atol=0)
    g = GN * M_J / R_J ** 2
    dz = KB * 1500.0 * np.log(10.0) / (mu * AMU * g)
    assert np.allclose(np.diff(p["z"]), dz, rtol=1e-12, atol=0)


def test_two_layer_switch_sweep_and_equal_layers():
    """Sweeping log10 P_sw across layer 2 moves only that layer's mixing ratio, linearly in
    log P_sw from X_top to X_surf; equal surface and top values give the constant profile's
    spectrum exactly."""
    tb = const_tables()
    for x in np.linspace(3.0, 4.0, 6):
        p = O.profile(tb, two_layer_atm([-3.0], [-5.0], [x]))
        f = 4.0 - x
        assert abs(p["X"][2, 0] - (f * 1e-3 + (1 - f) * 1e-5)) < 1e-15
        assert np.allclose(p["X"][:2, 0], 1e-3, rtol=1e-14) and np.allclose(p["X"][3:, 0], 1e-5, rtol=1e-14)
    tb2 = const_tables(2e-26, n_wn=3)
    d_two, _, _ = O.forward(tb2, two_layer_atm([-4.0], [-4.0], [2.7], n_layers=50))
    d_one, _, _ = O.forward(tb2, iso_atm(n_layers=50, log10_x=(-4.0,)))
    assert np.array_equal(d_two, d_one)


def test_two_layer_rejects_a_layer_above_unity():
    """A layer can exceed sum X = 1 although the surface and top sums do not (one gas already
    switched up, the other not yet): the model is rejected (Sec. 6)."""
    tb = const_tables(n_mol=2, mass_abs=[18.0, 16.0])
    atm = two_layer_atm(np.log10([0.6, 0.01]), np.log10([0.01, 0.6]), [1.5, 4.5])
    with pytest.raises(O.OracleError):
        O.profile(tb, atm)
    ok = two_layer_atm(np.log10([0.6, 0.01]), np.log10([0.01, 0.6]), [4.5, 1.5])
    assert O.profile(tb, ok)["X"][:, :2].sum(axis=1).max() <= 1.0
