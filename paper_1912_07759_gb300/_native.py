"""ctypes binding of libtransit.so (argument marshalling only; mirrors include/transit.h).

There is no fallback: if the library is missing or no CUDA device is usable, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtransit.so")

TR_OK, TR_ERR_ARG, TR_ERR_INVALID_MODEL, TR_ERR_OOM = 0, 1, 2, 3
TR_ERR_CUDA, TR_ERR_TIMEOUT, TR_ERR_UNSUPPORTED = 4, 5, 6
TR_STORE_FP32, TR_STORE_FP16_LOG10 = 1, 2
TR_OOR_CLAMP, TR_OOR_PAPER_ZERO = 0, 1
TR_GRAV_ALTITUDE, TR_GRAV_CONST = 0, 1
TR_CLOUD_NONE, TR_CLOUD_DISCRETE, TR_CLOUD_FRACTIONAL = 0, 1, 2
TR_PREC_FP32, TR_PREC_MIXED = 0, 1
TR_TPROF_NPOINT, TR_TPROF_GUILLOT = 0, 1
TR_GAS_CONSTANT, TR_GAS_TWOLAYER = 0, 1
TR_MAX_MOL, TR_MAX_CIA, TR_MAX_SPECIES, TR_MAX_TNODES, TR_MAX_LAYERS = 8, 4, 12, 8, 180
TR_NOALLOC_SCRATCH_BYTES = 16 << 20
TR_MAX_BATCH = 65535

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


class TableDesc(C.Structure):
    _fields_ = [("n_mol", C.c_int), ("n_p", C.c_int), ("n_t", C.c_int), ("n_wn", C.c_int),
                ("p_grid", _dp), ("t_grid", _dp), ("wn_grid", _dp), ("sigma", _fp),
                ("n_cia", C.c_int), ("n_t_cia", C.c_int), ("t_grid_cia", _dp),
                ("cia_pair", _ip), ("cia", _dp), ("n_species", C.c_int), ("mass_amu", _dp),
                ("rayleigh", _dp), ("storage", C.c_int), ("oor_mode", C.c_int),
                ("interp_mode", C.c_int)]


class AtmDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("p_max", C.c_double), ("p_min", C.c_double),
                ("n_tnodes", C.c_int), ("tnode_log10p", _dp), ("tnode_t", _dp),
                ("log10_x", _dp), ("fill_frac", _dp), ("r_p", C.c_double),
                ("m_p", C.c_double), ("r_s", C.c_double), ("p_cloud_top", C.c_double),
                ("p_cloud_bot", C.c_double), ("kappa_cloud", C.c_double),
                ("gravity_mode", C.c_int), ("cloud_mode", C.c_int), ("t_profile", C.c_int),
                ("guillot", _dp), ("t_int", C.c_double), ("gas_mode", C.c_int),
                ("log10_x_top", _dp), ("log10_p_switch", _dp)]


class BatchDesc(C.Structure):
    _fields_ = [("n_tnodes", C.c_int), ("tnode_log10p", _dp), ("fill_frac", _dp),
                ("p_max", C.c_double), ("p_min", C.c_double), ("m_p", C.c_double),
                ("r_s", C.c_double), ("p_cloud_bot", C.c_double),
                ("kappa_cloud", C.c_double), ("gravity_mode", C.c_int),
                ("cloud_mode", C.c_int), ("max_layers", C.c_int), ("t_profile", C.c_int),
                ("gas_mode", C.c_int), ("t_int", C.c_double)]


_vp = C.c_void_p
_SIGS = {
    "tr_create": (C.c_int, [C.POINTER(_vp), C.c_int]),
    "tr_destroy": (None, [_vp]),
    "tr_last_error": (C.c_char_p, [_vp]),
    "tr_sync_status": (C.c_int, [_vp, _vp]),
    "tr_selftest_wait_timeout": (C.c_int, [_vp, _vp]),
    "tr_load_xsec_tables": (C.c_int, [_vp, C.POINTER(TableDesc), C.POINTER(_vp)]),
    "tr_free_tables": (None, [_vp]),
    "tr_tables_device_bytes": (C.c_size_t, [_vp]),
    "tr_build_atmosphere": (C.c_int, [_vp, _vp, C.POINTER(AtmDesc), C.POINTER(_vp), _vp]),
    "tr_free_atmosphere": (None, [_vp]),
    "tr_atm_readback": (C.c_int, [_vp, _vp, _dp, _fp, _fp]),
    "tr_make_bins": (C.c_int, [_vp, _vp, C.c_int, _dp, _dp, C.POINTER(_vp)]),
    "tr_free_bins": (None, [_vp]),
    "tr_bins_native_range": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "tr_bin_spectra": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, C.c_longlong, C.c_int, _vp, _vp,
                                 _vp]),
    "tr_snr_instrument": (C.c_int, [_vp, C.c_int, C.c_int, _vp, C.c_double, C.c_int, _vp, _vp,
                                    _vp, _vp]),
    "tr_forward_transit": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]),
    "tr_batch_workspace_size": (C.c_size_t, [_vp, C.POINTER(BatchDesc), _vp, C.c_int, C.c_int]),
    "tr_forward_transit_batch": (C.c_int, [_vp, _vp, C.POINTER(BatchDesc), C.c_int, _vp, _vp,
                                           _vp, _vp, _vp, _vp, C.c_int, _vp, C.c_size_t, _vp]),
    "tr_adjoint_transit": (C.c_int, [_vp, _vp, C.POINTER(BatchDesc), C.c_int, _vp, _vp, _vp,
                                     _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, C.c_int,
                                     _vp, C.c_size_t, _vp]),
    "tr_forward_emission": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_double, _vp, _vp,
                                      C.c_int, _vp]),
    "tr_forward_emission_batch": (C.c_int, [_vp, _vp, C.POINTER(BatchDesc), C.c_int, _vp, _vp,
                                            _vp, C.c_int, C.c_double, _vp, _vp, _vp, C.c_int,
                                            _vp, C.c_size_t, _vp]),
    "tr_forward_transit_batch_noalloc": (C.c_int, [_vp, _vp, C.POINTER(BatchDesc), C.c_int, _vp,
                                                   _vp, _vp, _vp, _vp, _vp]),
    "tr_capture_forward_batch": (C.c_int, [_vp, _vp, C.POINTER(BatchDesc), C.c_int, _vp, _vp,
                                           _vp, _vp, _vp, _vp, C.c_int, _vp, C.c_size_t,
                                           C.c_int, _vp, C.POINTER(_vp)]),
    "tr_graph_launch": (C.c_int, [_vp, _vp]),
    "tr_graph_info": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float),
                                C.POINTER(C.c_int)]),
    "tr_free_graph": (None, [_vp]),
    "tr_pin_forward_config": (C.c_int, [_vp, _vp, C.POINTER(BatchDesc), C.c_int, _vp, C.c_int,
                                        C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "tr_unpin_forward_config": (C.c_int, [_vp, _vp, C.POINTER(BatchDesc), C.c_int, _vp,
                                          C.c_int, C.c_int]),
    "tr_profile_enable": (C.c_int, [_vp, C.c_int]),
    "tr_profile_read": (C.c_int, [_vp, C.c_int, C.c_char_p, _dp, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int)]),
}

_lock = threading.Lock()
_lib = None


def exported_names():
    return list(_SIGS)


def load(path: str = LIB_PATH):
    """Load libtransit.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; "
                    "g.build()'` (needs nvcc); there is no CPU fallback")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class TransitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code
