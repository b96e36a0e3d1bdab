"""Seeded synthetic inputs for the transmission forward model.

This module only draws inputs: cross-section tables, CIA and Rayleigh arrays, atmosphere
parameters, prior draws and bin layouts.  It contains none of the forward model's arithmetic
(no pressure grid, no interpolation, no optical depth, no binning weights), so that both the
CUDA path and the FP64 oracle can be fed the same arrays without sharing any code.

The paper measures on ExoMol / HITRAN cross-sections and HD 209458 b data (Sec. 8),
none of which are available here.  Seeded synthetic tables with the paper's structure stand in
for them:

* log10 sigma [cm^2] = -22 + a smooth Gaussian-process continuum in ln(nu) (64 random Fourier
  features, length scale 0.05, amplitude 1 dex) + 0.5 dex * (T - 1500)/1500 * a second GP
  + 0.2 * log10(P / 1e4 Pa) + lognormal line spikes (2 % of the grid cells, heights
  LogNormal(0, 0.7) dex, Gaussian width 1.5 cells * (P/1e4)^0.25), clipped to [-33, -17];
  stored in SI (m^2, i.e. -4 dex) as float32 linear sigma.
* CIA: log10 sigma [cm^5] = -46 + GP (1 dex) + 0.3 dex * (T - 1500)/1500, stored in m^5
  (-10 dex) as float64 (values near 1e-56 m^5 are below the float32 range).
* Rayleigh: sigma_R = A_s * nu^4 with A_H2 = 7.5e-49 and A_He = 5.0e-50 m^2 cm^4 (a stated
  synthetic choice; the paper cites Cox & Allen without a formula); absorbers have none.

Replicated pseudo-molecules (Sec. 8.1, molecule-count benchmark) are drawn with different seeds
(seed = 1000 * config + species index).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# Physical scales used to state the synthetic workloads (paper: R_J from the caption of the
# retrieved-parameters table, Sec. 8.2; H2, He, H2O, CH4 masses from the mass table of
# Sec. 8.1; CO, CO2, NH3 are standard atomic weights).
R_JUP = 6.9911e7          # m
M_JUP = 1.8981246e27      # kg (IAU nominal GM_J / G)
R_SUN = 6.957e8           # m (IAU nominal)

ABSORBERS = ("H2O", "CH4", "CO", "CO2", "NH3")
MASS_AMU = {"H2O": 18.01528, "CH4": 16.04276, "CO": 28.0101, "CO2": 44.0095,
            "NH3": 17.03052, "H2": 2.01588, "He": 4.002602}
RAYLEIGH_A = {"H2": 7.5e-49, "He": 5.0e-50}   # m^2 cm^4

OOR_CLAMP = 0
OOR_PAPER_ZERO = 1
INTERP_LINEAR = 0          # temperature interpolation schemes of Sec. 5
INTERP_EXP = 1
GRAV_ALTITUDE = 0
GRAV_CONST = 1
CLOUD_NONE = 0
CLOUD_DISCRETE = 1
CLOUD_FRACTIONAL = 2
TPROF_NPOINT = 0           # temperature profiles of Sec. 4.2: N-point (isothermal with one node)
TPROF_GUILLOT = 1          # Guillot2010 radiative equilibrium
GAS_CONSTANT = 0           # vertical mixing profiles of Sec. 4.3
GAS_TWOLAYER = 1
T_INT_DEFAULT = 100.0      # K, internal temperature of the Guillot profile (a stated choice)


# --------------------------------------------------------------------------------------------
# tables
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Tables:
    """Cross-section, CIA and Rayleigh inputs on one shared native wavenumber grid."""
    p_grid: np.ndarray            # [n_p] Pa, ascending (float64)
    t_grid: np.ndarray            # [n_t] K, ascending (float64)
    wn_grid: np.ndarray           # [n_wn] cm^-1, ascending (float64)
    sigma: np.ndarray             # [n_mol][n_p][n_t][n_wn] m^2, float32, C-contiguous
    species: tuple                # absorbers then fill gases
    mass_amu: np.ndarray          # [n_species] float64
    t_grid_cia: np.ndarray        # [n_t_cia] K (float64)
    cia_pair: np.ndarray          # [n_cia][2] int32 species indices
    cia: np.ndarray               # [n_cia][n_t_cia][n_wn] m^5 float64
    rayleigh: Optional[np.ndarray]  # [n_species][n_wn] m^2 float64, or None
    oor_mode: int = OOR_CLAMP
    interp_mode: int = INTERP_LINEAR

    @property
    def n_mol(self) -> int:
        return self.sigma.shape[0]

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_wn(self) -> int:
        return self.wn_grid.shape[0]


def wn_grid_loguniform(n_wn: int, wn_min: float = 300.0, wn_max: float = 30000.0) -> np.ndarray:
    """Constant-resolution native grid (log-uniform in wavenumber)."""
    return np.exp(np.linspace(np.log(wn_min), np.log(wn_max), n_wn))


def _gp_rff(rng: np.random.Generator, x: np.ndarray, length: float, amp: float,
            n_feat: int = 64) -> np.ndarray:
    """A smooth random function of x: random Fourier features of an RBF Gaussian process."""
    w = rng.normal(0.0, 1.0 / length, size=n_feat)
    b = rng.uniform(0.0, 2.0 * np.pi, size=n_feat)
    a = rng.normal(0.0, 1.0, size=n_feat)
    out = np.zeros_like(x)
    for k in range(n_feat):
        out += a[k] * np.cos(w[k] * x + b[k])
    return amp * np.sqrt(2.0 / n_feat) * out


def log10_xsec_cm2(seed: int, p_grid: np.ndarray, t_grid: np.ndarray,
                   wn_grid: np.ndarray) -> np.ndarray:
    """Synthetic log10 sigma [cm^2] of one molecule, shape [n_p][n_t][n_wn] (float32)."""
    rng = np.random.default_rng(seed)
    lnu = np.log(wn_grid)
    n_wn = wn_grid.shape[0]
    cont = (-22.0 + _gp_rff(rng, lnu, 0.05, 1.0)).astype(np.float32)
    tshape = _gp_rff(rng, lnu, 0.05, 1.0).astype(np.float32)
    n_lines = max(1, int(round(0.02 * n_wn)))
    centres = rng.uniform(0.0, n_wn - 1.0, size=n_lines)        # in grid-cell units
    heights = rng.lognormal(0.0, 0.7, size=n_lines)
    out = np.empty((p_grid.shape[0], t_grid.shape[0], n_wn), dtype=np.float32)
    for ip, p in enumerate(p_grid):
        width = 1.5 * (p / 1e4) ** 0.25
        half = int(np.ceil(5.0 * width)) + 1
        lines = np.zeros(n_wn, dtype=np.float64)
        offs = np.arange(-half, half + 1)
        for off in offs:
            idx = np.rint(centres).astype(np.int64) + off
            ok = (idx >= 0) & (idx < n_wn)
            prof = heights[ok] * np.exp(-0.5 * ((idx[ok] - centres[ok]) / width) ** 2)
            np.add.at(lines, idx[ok], prof)
        base = cont + np.float32(0.2 * np.log10(p / 1e4)) + lines.astype(np.float32)
        for it, t in enumerate(t_grid):
            v = base + np.float32(0.5 * (t - 1500.0) / 1500.0) * tshape
            np.clip(v, -33.0, -17.0, out=v)
            out[ip, it] = v
    return out


def make_tables(config: int, n_mol: int, n_p: int, n_t: int, n_wn: int,
                with_cia: bool, with_rayleigh: bool = True,
                wn_min: float = 300.0, wn_max: float = 30000.0,
                p_lo: float = 1e-5, p_hi: float = 1e7, t_lo: float = 300.0,
                t_hi: float = 3000.0, oor_mode: int = OOR_CLAMP) -> Tables:
    """Seeded tables: pressure grid log-uniform in [p_lo, p_hi], temperature grid linear in
    [t_lo, t_hi], native wavenumbers log-uniform; absorbers H2O, CH4, CO, CO2, NH3 (first
    n_mol), fill gases H2 and He."""
    assert 1 <= n_mol <= len(ABSORBERS)
    p_grid = np.exp(np.linspace(np.log(p_lo), np.log(p_hi), n_p))
    t_grid = np.linspace(t_lo, t_hi, n_t)
    wn = wn_grid_loguniform(n_wn, wn_min, wn_max)
    sigma = np.empty((n_mol, n_p, n_t, n_wn), dtype=np.float32)
    for m in range(n_mol):
        lx = log10_xsec_cm2(1000 * config + m, p_grid, t_grid, wn)
        lx -= np.float32(4.0)                   # cm^2 -> m^2
        np.power(np.float32(10.0), lx, out=sigma[m])
    species = tuple(ABSORBERS[:n_mol]) + ("H2", "He")
    mass = np.array([MASS_AMU[s] for s in species], dtype=np.float64)
    if with_cia:
        t_cia = t_grid.copy()
        pairs = np.array([[n_mol, n_mol], [n_mol, n_mol + 1]], dtype=np.int32)
        cia = np.empty((2, t_cia.shape[0], n_wn), dtype=np.float64)
        lnu = np.log(wn)
        for q in range(2):
            rng = np.random.default_rng(1000 * config + 100 + q)
            base = -46.0 + _gp_rff(rng, lnu, 0.1, 1.0)
            for it, t in enumerate(t_cia):
                cia[q, it] = 10.0 ** (base + 0.3 * (t - 1500.0) / 1500.0 - 10.0)
    else:
        t_cia = np.zeros(0, dtype=np.float64)
        pairs = np.zeros((0, 2), dtype=np.int32)
        cia = np.zeros((0, 0, n_wn), dtype=np.float64)
    if with_rayleigh:
        ray = np.zeros((len(species), n_wn), dtype=np.float64)
        for s, name in enumerate(species):
            if name in RAYLEIGH_A:
                ray[s] = RAYLEIGH_A[name] * wn ** 4
    else:
        ray = None
    return Tables(p_grid=p_grid, t_grid=t_grid, wn_grid=wn, sigma=sigma, species=species,
                  mass_amu=mass, t_grid_cia=t_cia, cia_pair=pairs, cia=cia, rayleigh=ray,
                  oor_mode=oor_mode)


# --------------------------------------------------------------------------------------------
# atmospheres
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Atmosphere:
    """Parameters of one forward model (the quantities the paper's model is built from)."""
    n_layers: int
    p_max: float                 # Pa, bottom boundary (layer 0)
    p_min: float                 # Pa, top boundary
    tnode_log10p: np.ndarray     # [n_tnodes] log10 Pa, descending; one node = isothermal
    tnode_t: np.ndarray          # [n_tnodes] K
    log10_x: np.ndarray          # [n_mol] constant mixing ratios of the absorbers
    fill_frac: np.ndarray        # [n_fill] fractions of the remaining volume
    r_p: float                   # m
    m_p: float                   # kg
    r_s: float                   # m
    p_cloud_top: float = 0.0     # Pa; <= 0 means no cloud
    p_cloud_bot: float = 0.0     # Pa; <= 0 means the bottom boundary
    kappa_cloud: float = 0.0     # m^-1
    gravity_mode: int = GRAV_ALTITUDE
    cloud_mode: int = CLOUD_NONE
    t_profile: int = TPROF_NPOINT
    guillot: Optional[np.ndarray] = None      # [5] T_irr (K), kappa_irr, kappa_v1, kappa_v2
                                              # (m^2/kg), alpha
    t_int: float = T_INT_DEFAULT
    gas_mode: int = GAS_CONSTANT
    log10_x_top: Optional[np.ndarray] = None  # [n_mol] two-layer: above the switch
    log10_p_switch: Optional[np.ndarray] = None   # [n_mol] two-layer: switch (log10 Pa)


@dataclasses.dataclass
class BatchSpec:
    """Fixed per-batch quantities; per-item theta = [log10 X_m | T nodes | R_p/R_J | log10 P_top]."""
    n_mol: int
    tnode_log10p: np.ndarray
    fill_frac: np.ndarray
    p_max: float
    p_min: float
    m_p: float
    r_s: float
    p_cloud_bot: float
    kappa_cloud: float
    gravity_mode: int = GRAV_ALTITUDE
    cloud_mode: int = CLOUD_FRACTIONAL
    t_profile: int = TPROF_NPOINT
    gas_mode: int = GAS_CONSTANT
    t_int: float = T_INT_DEFAULT

    @property
    def n_tnodes(self) -> int:
        return int(self.tnode_log10p.shape[0])

    @property
    def n_chem(self) -> int:
        """theta entries of the chemistry: log10 X, or log10 X_surf, log10 X_top, log10 P_sw."""
        return 3 * self.n_mol if self.gas_mode == GAS_TWOLAYER else self.n_mol

    @property
    def n_tpar(self) -> int:
        """theta entries of the temperature profile: the nodes, or the five Guillot ones."""
        return 5 if self.t_profile == TPROF_GUILLOT else self.n_tnodes

    @property
    def n_theta(self) -> int:
        return self.n_chem + self.n_tpar + 2


def config1_atmosphere() -> Atmosphere:
    """Plain model: 100 layers 1e6 -> 1e-4 Pa, isothermal 1500 K, H2/He 0.83/0.17, two
    absorbers at 1e-4 and 1e-5, Jupiter around the Sun, no cloud."""
    return Atmosphere(n_layers=100, p_max=1e6, p_min=1e-4,
                      tnode_log10p=np.array([6.0]), tnode_t=np.array([1500.0]),
                      log10_x=np.array([-4.0, -5.0]), fill_frac=np.array([0.83, 0.17]),
                      r_p=R_JUP, m_p=M_JUP, r_s=R_SUN)


def tnodes_4(p_max: float = 1e6, p_min: float = 1e-4) -> np.ndarray:
    """Four temperature nodes log-uniform in pressure from p_max to p_min (log10 Pa)."""
    return np.linspace(np.log10(p_max), np.log10(p_min), 4)


def config2_atmosphere(n_mol: int = 5) -> Atmosphere:
    """Full-size model: 100 layers, absorbers log10 X ~ U[-8,-3] (seed 2000), 4-node profile
    (2200, 1700, 1200, 800) K, grey cloud top at 1e3 Pa (discrete deck)."""
    rng = np.random.default_rng(2000)
    lx = rng.uniform(-8.0, -3.0, size=n_mol)
    return Atmosphere(n_layers=100, p_max=1e6, p_min=1e-4,
                      tnode_log10p=tnodes_4(), tnode_t=np.array([2200.0, 1700.0, 1200.0, 800.0]),
                      log10_x=lx, fill_frac=np.array([0.83, 0.17]),
                      r_p=R_JUP, m_p=M_JUP, r_s=R_SUN,
                      p_cloud_top=1e3, p_cloud_bot=0.0, kappa_cloud=1e-2,
                      gravity_mode=GRAV_ALTITUDE, cloud_mode=CLOUD_DISCRETE)


def batch_spec(n_mol: int, cloud_mode: int = CLOUD_FRACTIONAL) -> BatchSpec:
    return BatchSpec(n_mol=n_mol, tnode_log10p=tnodes_4(), fill_frac=np.array([0.83, 0.17]),
                     p_max=1e6, p_min=1e-4, m_p=M_JUP, r_s=R_SUN, p_cloud_bot=0.0,
                     kappa_cloud=1e-2, gravity_mode=GRAV_ALTITUDE, cloud_mode=cloud_mode)


def draw_theta(seed: int, batch: int, spec: BatchSpec,
               lx_range=(-12.0, -1.0), t_range=(500.0, 2500.0), rp_range=(0.8, 1.5),
               lpc_range=(2.0, 6.0)) -> np.ndarray:
    """Uniform prior draws (Sec. 6 uniform priors; ranges widened from the HD 209458 b priors
    of Sec. 8.2): theta[B][n_theta]."""
    rng = np.random.default_rng(seed)
    m, nt = spec.n_mol, spec.n_tnodes
    th = np.empty((batch, spec.n_theta), dtype=np.float64)
    th[:, :m] = rng.uniform(*lx_range, size=(batch, m))
    c = spec.n_chem
    if spec.gas_mode == GAS_TWOLAYER:
        # top mixing ratios 0-3 dex below the surface ones; switch between 10 Pa and 1e5 Pa
        th[:, m:2 * m] = th[:, :m] - rng.uniform(0.0, 3.0, size=(batch, m))
        th[:, 2 * m:3 * m] = rng.uniform(1.0, 5.0, size=(batch, m))
    if spec.t_profile == TPROF_GUILLOT:
        # T_irr over the paper's default prior bounds of the Guillot profile (Sec. 5.1 example:
        # 1300-2500 K); log10 kappa_irr in [-3, -1], log10 kappa_v1, kappa_v2 in [-4, 0] (m^2/kg);
        # alpha in [0, 1]
        th[:, c] = rng.uniform(1300.0, 2500.0, size=batch)
        th[:, c + 1] = rng.uniform(-3.0, -1.0, size=batch)
        th[:, c + 2:c + 4] = rng.uniform(-4.0, 0.0, size=(batch, 2))
        th[:, c + 4] = rng.uniform(0.0, 1.0, size=batch)
    else:
        th[:, c:c + nt] = rng.uniform(*t_range, size=(batch, nt))
    k = c + spec.n_tpar
    th[:, k] = rng.uniform(*rp_range, size=batch)
    th[:, k + 1] = rng.uniform(*lpc_range, size=batch)
    return th


def draw_nlayers(seed: int, batch: int, lo: int = 50, hi: int = 150) -> np.ndarray:
    """Uneven layer counts, uniform on {lo..hi}."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=batch).astype(np.int32)


def bins_logspaced(n_bin: int = 50, lam_lo_um: float = 1.1, lam_hi_um: float = 1.7):
    """Target bins as (centre, width) in micron with log-uniform edges over [lo, hi]."""
    edges = np.exp(np.linspace(np.log(lam_lo_um), np.log(lam_hi_um), n_bin + 1))
    return 0.5 * (edges[1:] + edges[:-1]), edges[1:] - edges[:-1]


def obs_noise(seed: int, n_bin: int, lo_ppm: float = 30.0, hi_ppm: float = 100.0):
    """Per-bin Gaussian noise levels (uniform 30-100 ppm) and one standard-normal draw each."""
    rng = np.random.default_rng(seed)
    sig = rng.uniform(lo_ppm, hi_ppm, size=n_bin) * 1e-6
    return sig, rng.normal(0.0, 1.0, size=n_bin)
