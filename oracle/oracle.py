"""ctypes binding of the FP64 CPU oracle (transit_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``.  The product (the CUDA library and its Python binding) never
imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "transit_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")
R_JUP = 6.9911e7

ORC_OK, ORC_ERR_ARG, ORC_ERR_INVALID_MODEL = 0, 1, 2

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)


class OrcTables(C.Structure):
    _fields_ = [("n_mol", C.c_int), ("n_p", C.c_int), ("n_t", C.c_int), ("n_wn", C.c_int),
                ("p_grid", _dp), ("t_grid", _dp), ("wn_grid", _dp), ("sigma", _fp),
                ("n_cia", C.c_int), ("n_t_cia", C.c_int), ("t_grid_cia", _dp),
                ("cia_pair", _ip), ("cia", _dp), ("n_species", C.c_int), ("mass_amu", _dp),
                ("rayleigh", _dp), ("oor_mode", C.c_int), ("interp_mode", C.c_int)]


class OrcAtm(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("p_max", C.c_double), ("p_min", C.c_double),
                ("n_tnodes", C.c_int), ("tnode_log10p", _dp), ("tnode_t", _dp),
                ("log10_x", _dp), ("fill_frac", _dp), ("r_p", C.c_double),
                ("m_p", C.c_double), ("r_s", C.c_double), ("p_cloud_top", C.c_double),
                ("p_cloud_bot", C.c_double), ("kappa_cloud", C.c_double),
                ("gravity_mode", C.c_int), ("cloud_mode", C.c_int), ("t_profile", C.c_int),
                ("guillot", _dp), ("t_int", C.c_double), ("gas_mode", C.c_int),
                ("log10_x_top", _dp), ("log10_p_switch", _dp)]


class OrcBins(C.Structure):
    _fields_ = [("n_bin", C.c_int), ("lam_centre_um", _dp), ("lam_width_um", _dp)]


class OrcBatch(C.Structure):
    _fields_ = [("n_mol", C.c_int), ("n_tnodes", C.c_int), ("tnode_log10p", _dp),
                ("fill_frac", _dp), ("p_max", C.c_double), ("p_min", C.c_double),
                ("m_p", C.c_double), ("r_s", C.c_double), ("p_cloud_bot", C.c_double),
                ("kappa_cloud", C.c_double), ("gravity_mode", C.c_int),
                ("cloud_mode", C.c_int), ("t_profile", C.c_int), ("gas_mode", C.c_int),
                ("t_int", C.c_double)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle with g++ (-O2, no fast-math)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB_OVERRIDE loads another build of this oracle (used to plant mistakes
            # in a copy of it and check that the pin tests catch them)
            path = os.environ.get("ORACLE_LIB_OVERRIDE")
            if not path:
                path = build()
            L = C.CDLL(path)
            L.orc_profile.restype = C.c_int
            L.orc_interp.restype = C.c_int
            L.orc_bin_weights.restype = C.c_int
            L.orc_forward.restype = C.c_int
            L.orc_forward_batch.restype = C.c_int
            L.orc_chi2_grad.restype = C.c_int
            L.orc_planck.restype = C.c_int
            L.orc_gauss_legendre01.restype = C.c_int
            L.orc_emission.restype = C.c_int
            L.orc_expint.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else _dp()


class _Keep:
    """Holds the numpy arrays a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def d(self, a):
        if a is None:
            return _dp()
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.refs.append(a)
        return a.ctypes.data_as(_dp)

    def f(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        self.refs.append(a)
        return a.ctypes.data_as(_fp)

    def i(self, a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        self.refs.append(a)
        return a.ctypes.data_as(_ip)


def _tables(tb, keep: _Keep) -> OrcTables:
    n_mol, n_p, n_t, n_wn = tb.sigma.shape
    return OrcTables(n_mol, n_p, n_t, n_wn, keep.d(tb.p_grid), keep.d(tb.t_grid),
                     keep.d(tb.wn_grid), keep.f(tb.sigma), int(tb.cia_pair.shape[0]),
                     int(tb.t_grid_cia.shape[0]), keep.d(tb.t_grid_cia),
                     keep.i(tb.cia_pair.reshape(-1)), keep.d(tb.cia.reshape(-1)),
                     len(tb.species), keep.d(tb.mass_amu),
                     keep.d(tb.rayleigh) if tb.rayleigh is not None else _dp(),
                     int(tb.oor_mode), int(getattr(tb, "interp_mode", 0)))


def _atm(a, keep: _Keep) -> OrcAtm:
    t_profile = int(getattr(a, "t_profile", 0))
    gas_mode = int(getattr(a, "gas_mode", 0))
    return OrcAtm(int(a.n_layers), float(a.p_max), float(a.p_min), len(a.tnode_t),
                  keep.d(a.tnode_log10p), keep.d(a.tnode_t), keep.d(a.log10_x),
                  keep.d(a.fill_frac), float(a.r_p), float(a.m_p), float(a.r_s),
                  float(a.p_cloud_top), float(a.p_cloud_bot), float(a.kappa_cloud),
                  int(a.gravity_mode), int(a.cloud_mode), t_profile,
                  keep.d(a.guillot) if t_profile == 1 else _dp(),
                  float(getattr(a, "t_int", 0.0)), gas_mode,
                  keep.d(a.log10_x_top) if gas_mode == 1 else _dp(),
                  keep.d(a.log10_p_switch) if gas_mode == 1 else _dp())


def _bins(centre, width, keep: _Keep) -> OrcBins:
    return OrcBins(len(centre), keep.d(centre), keep.d(width))


def _batch(spec, keep: _Keep) -> OrcBatch:
    return OrcBatch(int(spec.n_mol), int(spec.n_tnodes), keep.d(spec.tnode_log10p),
                    keep.d(spec.fill_frac), float(spec.p_max), float(spec.p_min),
                    float(spec.m_p), float(spec.r_s), float(spec.p_cloud_bot),
                    float(spec.kappa_cloud), int(spec.gravity_mode), int(spec.cloud_mode),
                    int(getattr(spec, "t_profile", 0)), int(getattr(spec, "gas_mode", 0)),
                    float(getattr(spec, "t_int", 0.0)))


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status}")
        self.status = status


def profile(tb, atm) -> dict:
    """Layer profile of one model: pressure, temperature, chemistry (X [N][n_species], mu of
    layer 0 and mu_l [N]), geometry, path lengths."""
    keep = _Keep()
    N, S = atm.n_layers, len(tb.species)
    out = {k: np.zeros(n) for k, n in [("pb", N + 1), ("P", N), ("T", N), ("X", N * S),
                                        ("g", N), ("H", N), ("z", N + 1), ("rho", N),
                                        ("cloud", N), ("DL", N * N), ("A", N), ("scal", 2),
                                        ("mu_l", N)]}
    t, a = _tables(tb, keep), _atm(atm, keep)
    st = lib().orc_profile(C.byref(t), C.byref(a), *[_d(out[k]) for k in
                           ["pb", "P", "T", "X", "g", "H", "z", "rho", "cloud", "DL", "A", "scal",
                            "mu_l"]])
    if st != ORC_OK:
        raise OracleError(st)
    out["DL"] = out["DL"].reshape(N, N)
    out["X"] = out["X"].reshape(N, S)
    out["mu"], out["delta"] = out["scal"]
    return out


def interp(tb, m: int, P: float, T: float) -> np.ndarray:
    keep = _Keep()
    out = np.zeros(tb.n_wn)
    t = _tables(tb, keep)
    st = lib().orc_interp(C.byref(t), int(m), C.c_double(P), C.c_double(T), _d(out))
    if st != ORC_OK:
        raise OracleError(st)
    return out


def bin_weights(wn, centre, width) -> np.ndarray:
    keep = _Keep()
    wn = np.ascontiguousarray(wn, dtype=np.float64)
    out = np.zeros((len(centre), len(wn)))
    b = _bins(centre, width, keep)
    st = lib().orc_bin_weights(_d(wn), len(wn), C.byref(b), _d(out))
    if st != ORC_OK:
        raise OracleError(st)
    return out


def bin_with_uncertainty(wn, centre, width, flux, sigma=None):
    """FluxBinner of Sec. 4.5 with the oracle's weights w_ij: F_j = sum_i w_ij F_i / sum_i w_ij
    (eq. F_j) and sigma_j = sqrt(sum_i w_ij^2 sigma_i^2 / (sum_i w_ij)^2) (eq. sigma_j), written
    as the paper states them; flux and sigma are [..., n_wn]."""
    w = bin_weights(wn, centre, width)
    ws = w.sum(axis=1)
    f = np.einsum("ji,...i->...j", w, np.asarray(flux, dtype=np.float64)) / ws
    if sigma is None:
        return f, None
    s2 = np.einsum("ji,...i->...j", w * w, np.asarray(sigma, dtype=np.float64) ** 2)
    return f, np.sqrt(s2 / ws ** 2)


def snr_instrument(binned, snr: float, n_obs: int, z):
    """SNR instrument model of Sec. 7: N = S / SNR with S the largest value of each spectrum,
    N' = N / sqrt(n); observation = binned + N' z, uncertainty N' at every bin."""
    binned = np.asarray(binned, dtype=np.float64)
    S = binned.max(axis=-1, keepdims=True)
    noise = (S / snr) / np.sqrt(n_obs)
    return binned + noise * np.asarray(z, dtype=np.float64), np.broadcast_to(noise, binned.shape).copy()


def expint(x):
    """Exponential integrals (E_1(x), E_2(x)) of the oracle (x > 0)."""
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    e1, e2 = np.zeros(len(x)), np.zeros(len(x))
    st = lib().orc_expint(_d(x), len(x), _d(e1), _d(e2))
    if st != ORC_OK:
        raise OracleError(st)
    return e1, e2


def planck(nu_cm, T: float) -> np.ndarray:
    """Planck function per wavenumber, B(nu, T) = 2 h c^2 nu^3 / (e^{h c nu / (k T)} - 1) with nu
    in 1/m (input in 1/cm); W m^-2 sr^-1 per 1/m (the emission model's source, Sec. 4)."""
    nu = np.ascontiguousarray(nu_cm, dtype=np.float64)
    out = np.zeros(len(nu))
    st = lib().orc_planck(_d(nu), len(nu), C.c_double(T), _d(out))
    if st != ORC_OK:
        raise OracleError(st)
    return out


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1] (the emission model's quadrature in
    cos(theta), Sec. 4)."""
    x, w = np.zeros(n), np.zeros(n)
    st = lib().orc_gauss_legendre01(int(n), _d(x), _d(w))
    if st != ORC_OK:
        raise OracleError(st)
    return x, w


def emission(tb, atm, n_mu: int = 4, t_star: float = 5800.0) -> np.ndarray:
    """Emission model of Sec. 4: planet-star flux ratio F_p/F_s [n_wn] (readings E1-E4 of the
    C oracle: vertical optical depth per layer, source constant in a layer, surface
    temperature at p_max, the star's intensity through the same quadrature)."""
    keep = _Keep()
    out = np.zeros(tb.n_wn)
    t, a = _tables(tb, keep), _atm(atm, keep)
    st = lib().orc_emission(C.byref(t), C.byref(a), int(n_mu), C.c_double(t_star), _d(out))
    if st != ORC_OK:
        raise OracleError(st)
    return out


def forward(tb, atm, bins=None, want_tau: bool = False):
    """(depth_native[n_wn], depth_binned[n_bin] or None, tau[N][n_wn] or None)."""
    keep = _Keep()
    W = tb.n_wn
    dn = np.zeros(W)
    db = np.zeros(len(bins[0])) if bins is not None else None
    tau = np.zeros((atm.n_layers, W)) if want_tau else None
    t, a = _tables(tb, keep), _atm(atm, keep)
    bp = C.byref(_bins(bins[0], bins[1], keep)) if bins is not None else None
    st = lib().orc_forward(C.byref(t), C.byref(a), bp, _d(dn), _d(db), _d(tau))
    if st != ORC_OK:
        raise OracleError(st)
    return dn, db, tau


def forward_batch(tb, spec, theta, nlayers, bins, n_threads: int = 1):
    """Binned spectra [B][n_bin] and status [B] of a batch of parameter vectors."""
    keep = _Keep()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    nl = np.ascontiguousarray(nlayers, dtype=np.int32)
    B = theta.shape[0]
    out = np.zeros((B, len(bins[0])))
    status = np.zeros(B, dtype=np.int32)
    t, s, b = _tables(tb, keep), _batch(spec, keep), _bins(bins[0], bins[1], keep)
    st = lib().orc_forward_batch(C.byref(t), C.byref(s), B, _d(theta), nl.ctypes.data_as(_ip),
                                 C.byref(b), _d(out), status.ctypes.data_as(_ip),
                                 int(n_threads))
    if st != ORC_OK:
        raise OracleError(st)
    return out, status


def chi2_grad(tb, spec, theta, n_layers, bins, obs, sig_obs):
    """(chi2, grad[n_theta], binned[n_bin], jac[n_bin][n_theta]) with exact dual gradients."""
    keep = _Keep()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    nth = theta.shape[0]
    nb = len(bins[0])
    chi2 = np.zeros(1)
    grad = np.zeros(nth)
    binned = np.zeros(nb)
    jac = np.zeros((nb, nth))
    t, s, b = _tables(tb, keep), _batch(spec, keep), _bins(bins[0], bins[1], keep)
    st = lib().orc_chi2_grad(C.byref(t), C.byref(s), _d(theta), int(n_layers), C.byref(b),
                             keep.d(obs), keep.d(sig_obs), _d(chi2), _d(grad), _d(binned),
                             _d(jac))
    if st != ORC_OK:
        raise OracleError(st)
    return chi2[0], grad, binned, jac
