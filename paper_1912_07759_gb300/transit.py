"""Python face of libtransit.so: handles and calls with the C-ABI's names.

Every step of the forward model and its adjoint runs in the library's CUDA kernels; this
module only converts arguments (numpy host arrays for tables and descriptors, torch CUDA
tensors for per-call device inputs and outputs) and checks status codes.  PyTorch supplies
device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import _native as N
from ._native import (TR_CLOUD_DISCRETE, TR_CLOUD_FRACTIONAL, TR_CLOUD_NONE,  # noqa: F401
                      TR_GRAV_ALTITUDE, TR_GRAV_CONST, TR_OOR_CLAMP, TR_OOR_PAPER_ZERO,
                      TR_PREC_FP32, TR_PREC_MIXED, TR_STORE_FP16_LOG10, TR_STORE_FP32,
                      TR_OK, TR_ERR_ARG, TR_ERR_INVALID_MODEL, TR_ERR_UNSUPPORTED,
                      TR_TPROF_NPOINT, TR_TPROF_GUILLOT, TR_GAS_CONSTANT, TR_GAS_TWOLAYER,
                      TransitError)

R_JUP = 6.9911e7


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor], dtype, name: str) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return C.c_void_p(t.data_ptr())


class _Host:
    """Keeps host numpy arrays alive while a ctypes struct points at them."""

    def __init__(self):
        self.keep = []

    def d(self, a):
        if a is None:
            return N._dp()
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.keep.append(a)
        return a.ctypes.data_as(N._dp)

    def f(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        self.keep.append(a)
        return a.ctypes.data_as(N._fp)

    def i(self, a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        self.keep.append(a)
        return a.ctypes.data_as(N._ip)


class TransitContext:
    """tr_create / tr_destroy."""

    def __init__(self, device: int = 0):
        self.lib = N.load()
        self.device = device
        h = C.c_void_p()
        rc = self.lib.tr_create(C.byref(h), device)
        if rc != N.TR_OK:
            raise TransitError(rc, f"tr_create failed on device {device}")
        self.handle = h

    def check(self, rc: int, what: str):
        if rc != N.TR_OK:
            msg = self.lib.tr_last_error(self.handle).decode()
            raise TransitError(rc, f"{what}: {msg}")

    def sync_status(self, stream=None):
        """tr_sync_status: synchronise the stream and raise on a recorded device timeout."""
        self.check(self.lib.tr_sync_status(self.handle, _stream_ptr(stream)), "tr_sync_status")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class XsecTables:
    """tr_load_xsec_tables: device-resident cross-section, CIA and Rayleigh tables."""

    def __init__(self, ctx: TransitContext, tb, storage: int = TR_STORE_FP32):
        self.ctx = ctx
        h = _Host()
        n_mol, n_p, n_t, n_wn = tb.sigma.shape
        n_cia = int(tb.cia_pair.shape[0])
        desc = N.TableDesc(n_mol, n_p, n_t, n_wn, h.d(tb.p_grid), h.d(tb.t_grid),
                           h.d(tb.wn_grid), h.f(tb.sigma), n_cia,
                           int(tb.t_grid_cia.shape[0]) if n_cia else 0,
                           h.d(tb.t_grid_cia) if n_cia else N._dp(),
                           h.i(tb.cia_pair.reshape(-1)) if n_cia else N._ip(),
                           h.d(tb.cia.reshape(-1)) if n_cia else N._dp(),
                           len(tb.species), h.d(tb.mass_amu),
                           h.d(tb.rayleigh) if tb.rayleigh is not None else N._dp(),
                           int(storage), int(tb.oor_mode), int(getattr(tb, "interp_mode", 0)))
        out = C.c_void_p()
        ctx.check(ctx.lib.tr_load_xsec_tables(ctx.handle, C.byref(desc), C.byref(out)),
                  "tr_load_xsec_tables")
        self.handle = out
        self.n_mol, self.n_wn, self.n_species = n_mol, n_wn, len(tb.species)

    @property
    def device_bytes(self) -> int:
        return int(self.ctx.lib.tr_tables_device_bytes(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.tr_free_tables(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Bins:
    """tr_make_bins: FluxBinner target bins (centres and widths in micron)."""

    def __init__(self, ctx: TransitContext, tables: XsecTables, centre_um, width_um):
        self.ctx = ctx
        h = _Host()
        out = C.c_void_p()
        self.n_bin = len(centre_um)
        ctx.check(ctx.lib.tr_make_bins(ctx.handle, tables.handle, self.n_bin, h.d(centre_um),
                                       h.d(width_um), C.byref(out)), "tr_make_bins")
        self.handle = out
        i0, i1 = C.c_int(), C.c_int()
        ctx.lib.tr_bins_native_range(out, C.byref(i0), C.byref(i1))
        self.native_range = (i0.value, i1.value)

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.tr_free_bins(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Atmosphere:
    """tr_build_atmosphere: one atmosphere's FP64 geometry, resident on the device."""

    def __init__(self, ctx: TransitContext, tables: XsecTables, atm, stream=None):
        self.ctx = ctx
        h = _Host()
        t_profile = int(getattr(atm, "t_profile", 0))
        gas_mode = int(getattr(atm, "gas_mode", 0))
        desc = N.AtmDesc(int(atm.n_layers), float(atm.p_max), float(atm.p_min),
                         len(atm.tnode_t), h.d(atm.tnode_log10p), h.d(atm.tnode_t),
                         h.d(atm.log10_x), h.d(atm.fill_frac), float(atm.r_p), float(atm.m_p),
                         float(atm.r_s), float(atm.p_cloud_top), float(atm.p_cloud_bot),
                         float(atm.kappa_cloud), int(atm.gravity_mode), int(atm.cloud_mode),
                         t_profile, h.d(atm.guillot) if t_profile else N._dp(),
                         float(getattr(atm, "t_int", 0.0)), gas_mode,
                         h.d(atm.log10_x_top) if gas_mode else N._dp(),
                         h.d(atm.log10_p_switch) if gas_mode else N._dp())
        out = C.c_void_p()
        ctx.check(ctx.lib.tr_build_atmosphere(ctx.handle, tables.handle, C.byref(desc),
                                              C.byref(out), _stream_ptr(stream)),
                  "tr_build_atmosphere")
        self.handle = out
        self.n_layers = int(atm.n_layers)

    def readback(self):
        """tr_atm_readback: (z[N+1] float64, DL[N][N] float32 ray-major, a[N] float32)."""
        n = self.n_layers
        z = np.zeros(n + 1)
        dl = np.zeros((n, n), dtype=np.float32)
        a = np.zeros(n, dtype=np.float32)
        self.ctx.check(self.ctx.lib.tr_atm_readback(
            self.ctx.handle, self.handle, z.ctypes.data_as(N._dp), dl.ctypes.data_as(N._fp),
            a.ctypes.data_as(N._fp)), "tr_atm_readback")
        return z, dl, a

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.tr_free_atmosphere(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forward_transit(ctx: TransitContext, tables: XsecTables, atm: Atmosphere,
                    bins: Optional[Bins] = None, native: bool = True,
                    precision: int = TR_PREC_FP32, out_native: Optional[torch.Tensor] = None,
                    out_binned: Optional[torch.Tensor] = None, stream=None):
    """tr_forward_transit: (depth_native[n_wn] or None, depth_binned[n_bin] or None)."""
    dev = torch.device("cuda", ctx.device)
    if native and out_native is None:
        out_native = torch.empty(tables.n_wn, dtype=torch.float64, device=dev)
    if bins is not None and out_binned is None:
        out_binned = torch.empty(bins.n_bin, dtype=torch.float64, device=dev)
    ctx.check(ctx.lib.tr_forward_transit(
        ctx.handle, tables.handle, atm.handle, bins.handle if bins is not None else None,
        _ptr(out_native if native else None, torch.float64, "out_native"),
        _ptr(out_binned, torch.float64, "out_binned"), int(precision), _stream_ptr(stream)),
        "tr_forward_transit")
    return (out_native if native else None), out_binned


def forward_emission(ctx: TransitContext, tables: XsecTables, atm: Atmosphere,
                     bins: Optional[Bins] = None, n_mu: int = 4, t_star: float = 5800.0,
                     native: bool = True, precision: int = TR_PREC_FP32, stream=None):
    """tr_forward_emission: planet-star flux ratio (native[n_wn] or None, binned[n_bin] or
    None) of the emission model of Sec. 4 with an n_mu-point Gauss-Legendre rule."""
    dev = torch.device("cuda", ctx.device)
    out_native = torch.empty(tables.n_wn, dtype=torch.float64, device=dev) if native else None
    out_binned = (torch.empty(bins.n_bin, dtype=torch.float64, device=dev)
                  if bins is not None else None)
    ctx.check(ctx.lib.tr_forward_emission(
        ctx.handle, tables.handle, atm.handle, bins.handle if bins is not None else None,
        int(n_mu), C.c_double(t_star), _ptr(out_native, torch.float64, "out_native"),
        _ptr(out_binned, torch.float64, "out_binned"), int(precision), _stream_ptr(stream)),
        "tr_forward_emission")
    return out_native, out_binned


class BatchSpec:
    """tr_batch_desc: quantities fixed for a whole batch."""

    def __init__(self, spec, max_layers: int):
        self._h = _Host()
        h = self._h
        self.desc = N.BatchDesc(int(spec.n_tnodes), h.d(spec.tnode_log10p), h.d(spec.fill_frac),
                                float(spec.p_max), float(spec.p_min), float(spec.m_p),
                                float(spec.r_s), float(spec.p_cloud_bot),
                                float(spec.kappa_cloud), int(spec.gravity_mode),
                                int(spec.cloud_mode), int(max_layers),
                                int(getattr(spec, "t_profile", 0)),
                                int(getattr(spec, "gas_mode", 0)),
                                float(getattr(spec, "t_int", 0.0)))
        self.n_mol = int(spec.n_mol)
        self.n_theta = int(spec.n_theta)
        self.max_layers = int(max_layers)


def batch_workspace_size(ctx: TransitContext, tables: XsecTables, spec: BatchSpec,
                         bins: Optional[Bins], B: int, with_adjoint: bool = False) -> int:
    """tr_batch_workspace_size (bins=None: native-resolution output)."""
    return int(ctx.lib.tr_batch_workspace_size(tables.handle, C.byref(spec.desc),
                                               bins.handle if bins is not None else None,
                                               int(B), int(with_adjoint)))


def forward_transit_batch(ctx: TransitContext, tables: XsecTables, spec: BatchSpec,
                          theta: torch.Tensor, nlayers: Optional[torch.Tensor],
                          bins: Optional[Bins], precision: int = TR_PREC_FP32,
                          workspace: Optional[torch.Tensor] = None, native: bool = False,
                          out_native: Optional[torch.Tensor] = None,
                          out_binned: Optional[torch.Tensor] = None,
                          out_status: Optional[torch.Tensor] = None, stream=None):
    """tr_forward_transit_batch: (binned[B][n_bin] float64 or None, status[B] int32) and, with
    native=True, also native[B][n_wn]: returns (binned, status, native)."""
    B = int(theta.shape[0])
    dev = theta.device
    if bins is not None and out_binned is None:
        out_binned = torch.empty(B, bins.n_bin, dtype=torch.float64, device=dev)
    if native and out_native is None:
        out_native = torch.empty(B, tables.n_wn, dtype=torch.float64, device=dev)
    if out_status is None:
        out_status = torch.empty(B, dtype=torch.int32, device=dev)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ctx.check(ctx.lib.tr_forward_transit_batch(
        ctx.handle, tables.handle, C.byref(spec.desc), B,
        _ptr(theta, torch.float64, "theta"), _ptr(nlayers, torch.int32, "nlayers"),
        bins.handle if bins is not None else None,
        _ptr(out_native if native else None, torch.float64, "out_native"),
        _ptr(out_binned, torch.float64, "out_binned"),
        _ptr(out_status, torch.int32, "out_status"), int(precision),
        C.c_void_p(workspace.data_ptr()) if workspace is not None else C.c_void_p(0),
        C.c_size_t(ws_bytes), _stream_ptr(stream)), "tr_forward_transit_batch")
    if native:
        return out_binned, out_status, out_native
    return out_binned, out_status


def forward_emission_batch(ctx: TransitContext, tables: XsecTables, spec: "BatchSpec",
                           theta: torch.Tensor, nlayers: Optional[torch.Tensor],
                           bins: Optional[Bins], n_mu: int = 4, t_star: float = 5800.0,
                           native: bool = False, precision: int = TR_PREC_FP32,
                           workspace: Optional[torch.Tensor] = None, stream=None):
    """tr_forward_emission_batch: (binned[B][n_bin] or None, status[B], native[B][n_wn] or
    None) flux ratios of the emission model for a batch of parameter vectors."""
    B = int(theta.shape[0])
    dev = theta.device
    out_binned = (torch.empty(B, bins.n_bin, dtype=torch.float64, device=dev)
                  if bins is not None else None)
    out_native = torch.empty(B, tables.n_wn, dtype=torch.float64, device=dev) if native else None
    status = torch.empty(B, dtype=torch.int32, device=dev)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ctx.check(ctx.lib.tr_forward_emission_batch(
        ctx.handle, tables.handle, C.byref(spec.desc), B, _ptr(theta, torch.float64, "theta"),
        _ptr(nlayers, torch.int32, "nlayers"), bins.handle if bins is not None else None,
        int(n_mu), C.c_double(t_star), _ptr(out_native, torch.float64, "out_native"),
        _ptr(out_binned, torch.float64, "out_binned"), _ptr(status, torch.int32, "status"),
        int(precision),
        C.c_void_p(workspace.data_ptr()) if workspace is not None else C.c_void_p(0),
        C.c_size_t(ws_bytes), _stream_ptr(stream)), "tr_forward_emission_batch")
    return out_binned, status, out_native


class ForwardGraph:
    """tr_capture_forward_batch: the batched forward captured once as a CUDA graph (after an
    optional autotuning pass over the forward's configurations), replayed by launch().  The
    graph keeps the tensors given here: write new parameters into `theta` (and `nlayers`) in
    place between launches; outputs land in `binned`, `status` (and `native`)."""

    def __init__(self, ctx: TransitContext, tables: XsecTables, spec: BatchSpec,
                 theta: torch.Tensor, nlayers: Optional[torch.Tensor], bins: Optional[Bins],
                 precision: int = TR_PREC_FP32, workspace: Optional[torch.Tensor] = None,
                 native: bool = False, autotune: bool = True, stream=None):
        B = int(theta.shape[0])
        dev = theta.device
        self.ctx = ctx
        self._keep = (tables, spec, bins, theta, nlayers, workspace)
        self.theta, self.nlayers = theta, nlayers
        self.binned = (torch.empty(B, bins.n_bin, dtype=torch.float64, device=dev)
                       if bins is not None else None)
        self.native = (torch.empty(B, tables.n_wn, dtype=torch.float64, device=dev)
                       if native else None)
        self.status = torch.empty(B, dtype=torch.int32, device=dev)
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        h = C.c_void_p()
        ctx.check(ctx.lib.tr_capture_forward_batch(
            ctx.handle, tables.handle, C.byref(spec.desc), B,
            _ptr(theta, torch.float64, "theta"), _ptr(nlayers, torch.int32, "nlayers"),
            bins.handle if bins is not None else None,
            _ptr(self.native, torch.float64, "native"), _ptr(self.binned, torch.float64, "binned"),
            _ptr(self.status, torch.int32, "status"), int(precision),
            C.c_void_p(workspace.data_ptr()) if workspace is not None else C.c_void_p(0),
            C.c_size_t(ws_bytes), int(bool(autotune)), _stream_ptr(stream), C.byref(h)),
            "tr_capture_forward_batch")
        self.handle = h

    def launch(self, stream=None):
        self.ctx.check(self.ctx.lib.tr_graph_launch(self.handle, _stream_ptr(stream)),
                       "tr_graph_launch")

    def info(self) -> dict:
        form, per_sm, stages, cps, n = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ms = C.c_float()
        self.ctx.check(self.ctx.lib.tr_graph_info(self.handle, C.byref(form), C.byref(per_sm),
                                                  C.byref(stages), C.byref(cps), C.byref(ms),
                                                  C.byref(n)), "tr_graph_info")
        return {"form": "fused" if form.value == 1 else "two-stage",
                "opacity_ctas_per_sm": per_sm.value, "fused_stages_cap": stages.value,
                "contraction": {0: "auto", 1: "ffma8", 2: "ffma11", 3: "tc_3xtf32"}.get(
                    cps.value, str(cps.value)),
                "tuned_ms": ms.value,
                "candidates": n.value}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.ctx.lib.tr_free_graph(h)
            self.handle = None


def pin_forward_config(ctx: TransitContext, tables: XsecTables, spec: BatchSpec, B: int,
                       bins: Optional[Bins], native: bool = False, precision: int = TR_PREC_FP32,
                       form: Optional[str] = "two-stage", per_sm: int = 0, stages: int = 0,
                       contract_per_sm: int = 0):
    """tr_pin_forward_config / tr_unpin_forward_config (form=None): the configuration batch
    calls of this shape use ('two-stage' with per_sm opacity CTAs per SM, or 'fused')."""
    bh = bins.handle if bins is not None else None
    if form is None:
        ctx.check(ctx.lib.tr_unpin_forward_config(ctx.handle, tables.handle, C.byref(spec.desc),
                                                  B, bh, int(native), int(precision)),
                  "tr_unpin_forward_config")
        return
    f = {"two-stage": 0, "fused": 1}[form]
    ctx.check(ctx.lib.tr_pin_forward_config(ctx.handle, tables.handle, C.byref(spec.desc), B, bh,
                                            int(native), int(precision), f, int(per_sm),
                                            int(stages), int(contract_per_sm)),
              "tr_pin_forward_config")


def bin_spectra(ctx: TransitContext, bins: Bins, native: torch.Tensor,
                native_sigma: Optional[torch.Tensor] = None, base: int = 0, stream=None):
    """tr_bin_spectra: FluxBinner (Sec. 4.5) of native spectra native[B][n] (float64, CUDA;
    native index i at column i - base) with optional uncertainties: (binned[B][n_bin],
    binned_sigma[B][n_bin] or None)."""
    if native.dim() == 1:
        native = native[None]
    if native_sigma is not None and native_sigma.dim() == 1:
        native_sigma = native_sigma[None]
    B, n = int(native.shape[0]), int(native.shape[1])
    binned = torch.empty(B, bins.n_bin, dtype=torch.float64, device=native.device)
    bsig = torch.empty_like(binned) if native_sigma is not None else None
    ctx.check(ctx.lib.tr_bin_spectra(
        ctx.handle, bins.handle, B, _ptr(native, torch.float64, "native"),
        _ptr(native_sigma, torch.float64, "native_sigma"), C.c_longlong(n), int(base),
        _ptr(binned, torch.float64, "binned"), _ptr(bsig, torch.float64, "binned_sigma"),
        _stream_ptr(stream)), "tr_bin_spectra")
    return binned, bsig


def snr_instrument(ctx: TransitContext, binned: torch.Tensor, snr: float, n_obs: int,
                   z: torch.Tensor, stream=None):
    """tr_snr_instrument (Sec. 7): (observation[B][n_bin], sigma[B][n_bin]) from binned
    spectra and standard-normal draws z of the same shape."""
    if binned.dim() == 1:
        binned, z = binned[None], z[None]
    B, n_bin = int(binned.shape[0]), int(binned.shape[1])
    obs = torch.empty_like(binned)
    sig = torch.empty_like(binned)
    ctx.check(ctx.lib.tr_snr_instrument(
        ctx.handle, B, n_bin, _ptr(binned, torch.float64, "binned"), C.c_double(snr),
        int(n_obs), _ptr(z, torch.float64, "z"), _ptr(obs, torch.float64, "obs"),
        _ptr(sig, torch.float64, "sigma"), _stream_ptr(stream)), "tr_snr_instrument")
    return obs, sig


def profile_enable(ctx: TransitContext, on: bool = True):
    """tr_profile_enable: start (clearing totals) or stop per-kernel event timing."""
    ctx.check(ctx.lib.tr_profile_enable(ctx.handle, int(on)), "tr_profile_enable")


def profile_read(ctx: TransitContext, max_kernels: int = 16) -> dict:
    """tr_profile_read: {kernel name: (total device ms, launches)}."""
    names = C.create_string_buffer(48 * max_kernels)
    ms = (C.c_double * max_kernels)()
    cnt = (C.c_int64 * max_kernels)()
    n = C.c_int()
    ctx.check(ctx.lib.tr_profile_read(ctx.handle, max_kernels, names, ms, cnt, C.byref(n)),
              "tr_profile_read")
    out = {}
    for k in range(min(n.value, max_kernels)):
        name = names.raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[name] = (ms[k], int(cnt[k]))
    return out


def adjoint_transit(ctx: TransitContext, tables: XsecTables, spec: BatchSpec,
                    theta: torch.Tensor, nlayers: Optional[torch.Tensor], bins: Bins,
                    obs: Optional[torch.Tensor] = None, sigma_obs: Optional[torch.Tensor] = None,
                    gbin: Optional[torch.Tensor] = None, precision: int = TR_PREC_FP32,
                    workspace: Optional[torch.Tensor] = None, want_binned: bool = True,
                    recompute_k: int = -1, want_grad: bool = True, want_jac: bool = False,
                    stream=None):
    """tr_adjoint_transit: (chi2[B] or None, grad[B][n_theta] or None, binned[B][n_bin] or
    None, status[B]), and with want_jac=True also jac[B][n_bin][n_theta] (the Jacobian of the
    binned spectrum) as a fifth value.  With gbin the gradient is the vector-Jacobian product
    gbin . dD_bin/dtheta, else the chi^2 gradient (obs, sigma_obs needed); want_grad=False
    (with want_jac=True) computes only the Jacobian.  recompute_k: 1 recomputes the opacity in
    the backward pass; -1 (or 0) reuses the forward's when the workspace's K buffer holds the
    whole batch."""
    B = int(theta.shape[0])
    dev = theta.device
    if not want_grad and not want_jac:
        raise ValueError("nothing to compute: want_grad and want_jac are both False")
    chi2 = (torch.empty(B, dtype=torch.float64, device=dev)
            if (gbin is None and want_grad) else None)
    grad = torch.empty(B, spec.n_theta, dtype=torch.float64, device=dev) if want_grad else None
    jac = (torch.empty(B, bins.n_bin, spec.n_theta, dtype=torch.float64, device=dev)
           if want_jac else None)
    binned = torch.empty(B, bins.n_bin, dtype=torch.float64, device=dev) if want_binned else None
    status = torch.empty(B, dtype=torch.int32, device=dev)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ctx.check(ctx.lib.tr_adjoint_transit(
        ctx.handle, tables.handle, C.byref(spec.desc), B,
        _ptr(theta, torch.float64, "theta"), _ptr(nlayers, torch.int32, "nlayers"),
        bins.handle, _ptr(obs, torch.float64, "obs"), _ptr(sigma_obs, torch.float64, "sigma_obs"),
        _ptr(gbin, torch.float64, "gbin"), _ptr(chi2, torch.float64, "chi2"),
        _ptr(grad, torch.float64, "grad"), _ptr(jac, torch.float64, "jac"),
        _ptr(binned, torch.float64, "binned"),
        _ptr(status, torch.int32, "status"), int(precision), int(recompute_k),
        C.c_void_p(workspace.data_ptr()) if workspace is not None else C.c_void_p(0),
        C.c_size_t(ws_bytes), _stream_ptr(stream)), "tr_adjoint_transit")
    if want_jac:
        return chi2, grad, binned, status, jac
    return chi2, grad, binned, status
