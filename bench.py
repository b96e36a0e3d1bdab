#!/usr/bin/env python
"""Benchmark of the transmission forward model on GB300.

Workload (one step): the full-size single forward model -- 100 layers, 5 absorbers, FP32
cross-section tables 22 P x 27 T x 200,000 wavenumbers, CIA H2-H2 and H2-He, Rayleigh,
4-node temperature profile, grey cloud top at 1e3 Pa -- computed at native resolution and
binned to 50 bins over 1.1-1.7 micron: one replay of the forward captured as a CUDA graph
(tr_capture_forward_batch / tr_graph_launch, B = 1): FP64 geometry kernels, TMA-staged
opacity kernel, FP32 contraction + depth kernel, binning kernel.

Prints one JSON line.  `value` is device-timed spectra/s with inputs resident in HBM and the
L2 flushed before every timed step; `e2e` is the same through the C ABI with the parameter
vector copied from pinned host memory into a graph's input and the native + binned
spectrum copied back every step (two graphs alternate so that one step's read-back overlaps
the next step's compute).  Per-kernel times (and the rooflines) come from plain batch
calls of the same configuration.  `--impl reference` times the FP64 CPU oracle on the host
cores instead, on bounded wavenumber slices of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transit spectra/s and fwd+grad/s (100 layers×200k wn) vs plain GPU at stated ppm"
UNIT = "spectra/s"
WORKLOAD = ("full-size single forward model: 100 layers, 5 absorbers, FP32 tables "
            "22 P x 27 T x 200,000 wn, CIA H2-H2 + H2-He, Rayleigh, 4-node T profile, "
            "cloud top 1e3 Pa; native spectrum + 50 bins (1.1-1.7 um)")
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="budget of the CPU-oracle baseline leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (run the default configuration), e.g. under ncu")
    ap.add_argument("--ncu-case", choices=["single", "single_ffma", "mixed", "adjoint", "emission"],
                    default=None,
                    help="run a small case twice for an ncu capture and exit (no timing): the "
                         "full-size FP32 single forward in the tuned configuration, a mixed "
                         "forward of 8 atmospheres on 22 x 27 x 100,000 tables, forward + "
                         "gradient of 256 atmospheres, or the full-size emission spectrum")
    ap.add_argument("--batch-steps", type=int, default=20,
                    help="timed steps of the batched forward and forward+gradient workloads "
                         "(0 skips them)")
    return ap.parse_args()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ------------------------------------------------------------------------------ workload
def workload():
    from paper_1912_07759_gb300 import synthetic as S
    tb = S.make_tables(2, 5, 22, 27, 200000, with_cia=True)
    atm = S.config2_atmosphere()
    spec = S.BatchSpec(n_mol=5, tnode_log10p=atm.tnode_log10p, fill_frac=atm.fill_frac,
                       p_max=atm.p_max, p_min=atm.p_min, m_p=atm.m_p, r_s=atm.r_s,
                       p_cloud_bot=0.0, kappa_cloud=atm.kappa_cloud,
                       gravity_mode=atm.gravity_mode, cloud_mode=atm.cloud_mode)
    theta = np.concatenate([atm.log10_x, atm.tnode_t, [atm.r_p / S.R_JUP],
                            [np.log10(atm.p_cloud_top)]])[None, :]
    return S, tb, atm, spec, theta


def oracle_pool_map(fn, items):
    """Map fn over items on all host cores (threads: the oracle's ctypes calls release the
    GIL); returns (results, wall seconds, threads used)."""
    import concurrent.futures as cf
    n = max(1, min(len(items), os.cpu_count() or 1))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        res = list(ex.map(fn, items))
    return res, time.perf_counter() - t0, n


def check_subset(B: int, n: int = 64, seed: int = 64):
    """The seeded subset of batch items compared with the oracle: the first, the last and
    n - 2 others drawn without replacement."""
    rng = np.random.default_rng(seed)
    mid = rng.choice(np.arange(1, B - 1), n - 2, replace=False)
    return [0] + sorted(int(i) for i in mid) + [B - 1]


def atm_of_theta(S, spec_h, th, n_layers: int = 100):
    """The oracle's single-atmosphere description of batch item theta."""
    m, nt = spec_h.n_mol, spec_h.n_tnodes
    return S.Atmosphere(n_layers=int(n_layers), p_max=spec_h.p_max, p_min=spec_h.p_min,
                        tnode_log10p=spec_h.tnode_log10p, tnode_t=th[m:m + nt],
                        log10_x=th[:m], fill_frac=spec_h.fill_frac, r_p=th[m + nt] * S.R_JUP,
                        m_p=spec_h.m_p, r_s=spec_h.r_s, p_cloud_top=10.0 ** th[m + nt + 1],
                        p_cloud_bot=spec_h.p_cloud_bot, kappa_cloud=spec_h.kappa_cloud,
                        gravity_mode=spec_h.gravity_mode, cloud_mode=spec_h.cloud_mode)


def grad_rel_err(g, ref):
    """Largest |g - ref| / max(|ref|, 1e-3 max|ref|) (the gradient bar's measure)."""
    floor = 1e-3 * np.abs(ref).max()
    return float((np.abs(g - ref) / np.maximum(np.abs(ref), max(floor, 1e-300))).max())


def workload_config(world: int) -> dict:
    """The workload both arms measure (the same dict on the native and the reference line)."""
    return {"workload": WORKLOAD, "batch_per_gpu": 1, "layers": 100, "wavenumbers": 200000,
            "absorbers": 5, "bins": 50, "parallelism": f"replicas x{world}",
            "l2": "flushed (256 MiB write) before every timed GPU step"}


def time_steps(step, stream, steps: int, flush=None):
    """Sum of per-step CUDA-event times (ms) over `steps`, L2 flushed before each step."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        if flush is not None:
            flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return float(sum(a.elapsed_time(b) for a, b in ev))


def batched_workloads(T, ctx, dev, flush, steps: int, warmup: int):
    """Batched forward (4096 atmospheres drawn from the priors, 50-150 layers, 2 absorbers on
    13 x 15 x 10,000 tables, 50 bins) and forward + chi^2 gradient (1024 atmospheres, 100
    layers, 5 absorbers on 13 x 15 x 10,000 tables, 11 parameters, synthetic 30-100 ppm
    observation), both FP32 with FP64 geometry."""
    import torch
    from paper_1912_07759_gb300 import synthetic as S
    cuda = torch.device("cuda", dev)
    stream = torch.cuda.current_stream(cuda)
    out = {}
    # batched forward
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins = T.Bins(ctx, tables, *S.bins_logspaced())
    spec_h = S.batch_spec(2)
    B = 4096
    spec = T.BatchSpec(spec_h, max_layers=150)
    th = torch.tensor(S.draw_theta(3000, B, spec_h), device=cuda)
    nl = torch.tensor(S.draw_nlayers(3001, B), device=cuda)
    ws = torch.empty(T.batch_workspace_size(ctx, tables, spec, bins, B), dtype=torch.uint8, device=cuda)
    ob = torch.empty(B, bins.n_bin, dtype=torch.float64, device=cuda)
    st = torch.empty(B, dtype=torch.int32, device=cuda)

    # one persistent-kernel forward per step, captured once as a CUDA graph after the
    # autotuner has timed the forward's configurations on these inputs
    graph = T.ForwardGraph(ctx, tables, spec, th, nl, bins, workspace=ws, autotune=True)

    def fwd():
        graph.launch(stream)
    for _ in range(warmup):
        fwd()
    ms = time_steps(fwd, stream, steps, flush)
    # per-kernel times from plain batch calls of the same shape (they run the tuned choice)
    T.profile_enable(ctx, True)
    for _ in range(3):
        T.forward_transit_batch(ctx, tables, spec, th, nl, bins, workspace=ws, out_binned=ob,
                                out_status=st)
    torch.cuda.synchronize()
    prof = T.profile_read(ctx)
    T.profile_enable(ctx, False)
    # the FP64 oracle on the seeded 64-item subset: parity of the binned spectra, and the
    # oracle's own rate over all host cores (OpenMP across atmospheres)
    from oracle import oracle as O
    pick = check_subset(B)
    th_h, nl_h = th.cpu().numpy(), nl.cpu().numpy()
    ob_h, st_h = ob.cpu().numpy(), st.cpu().numpy()
    n_thr = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref, ref_st = O.forward_batch(tb, spec_h, th_h[pick], nl_h[pick], S.bins_logspaced(),
                                  n_threads=n_thr)
    t_orc = time.perf_counter() - t0
    ok = [i for i, b in enumerate(pick) if ref_st[i] == 0]
    err_ppm = float(np.abs(ob_h[pick][ok] - ref[ok]).max()) * 1e6 if ok else None
    status_match = bool(np.all((st_h[pick] == 0) == (ref_st == 0)))
    out["batched_forward"] = {
        "value": round(B * steps / (ms / 1e3), 1), "unit": UNIT, "ms_per_step": round(ms / steps, 4),
        "max_abs_err_vs_fp64_oracle_ppm": round(err_ppm, 5) if err_ppm is not None else None,
        "oracle_items_checked": len(pick), "oracle_status_match": status_match,
        "cpu_baseline": {"value": round(len(pick) / t_orc, 2), "unit": UNIT, "cores": n_thr,
                         "kind": "oracle",
                         "sample": f"FP64 oracle batch call (OpenMP across atmospheres) on the "
                                   f"{len(pick)} checked atmospheres of this workload, "
                                   f"{t_orc:.2f} s"},
        "workload": "4096 atmospheres from the priors, 50-150 layers, 2 absorbers, 13 x 15 x "
                    "10,000 FP32 tables, 50 bins (binned region only); one CUDA-graph launch "
                    "per step",
        "graph": graph.info(),
        "kernels_per_step": {k: {"launches": n / 3, "ms": round(v / 3, 4)}
                             for k, (v, n) in prof.items()}}
    del graph
    del ws
    # forward + gradient
    tb5 = S.make_tables(4, 5, 13, 15, 10000, with_cia=False)
    tables5 = T.XsecTables(ctx, tb5)
    bins5 = T.Bins(ctx, tables5, *S.bins_logspaced())
    spec5_h = S.batch_spec(5)
    B = 1024
    spec5 = T.BatchSpec(spec5_h, max_layers=100)
    th5 = torch.tensor(S.draw_theta(4001, B, spec5_h), device=cuda)
    sig, z = S.obs_noise(4002, bins5.n_bin)
    obs0, _ = T.forward_transit_batch(ctx, tables5, spec5,
                                      torch.tensor(S.draw_theta(4000, 1, spec5_h), device=cuda),
                                      None, bins5)
    obs = (obs0[0] + torch.tensor(sig * z, device=cuda)).contiguous()
    sig_t = torch.tensor(sig, device=cuda)
    ws5 = torch.empty(T.batch_workspace_size(ctx, tables5, spec5, bins5, B, with_adjoint=True),
                      dtype=torch.uint8, device=cuda)

    last = {}

    def fg():
        last["r"] = T.adjoint_transit(ctx, tables5, spec5, th5, None, bins5, obs=obs,
                                      sigma_obs=sig_t, workspace=ws5)
    for _ in range(warmup):
        fg()
    steps_g = max(3, steps // 2)
    T.profile_enable(ctx, True)
    ms = time_steps(fg, stream, steps_g, flush)
    prof = T.profile_read(ctx)
    T.profile_enable(ctx, False)
    chi2_d, grad_d, binned_d, st_d = (x.cpu().numpy() for x in last["r"])
    pick = check_subset(B, seed=65)
    th5_h, obs_h = th5.cpu().numpy(), obs.cpu().numpy()
    bins5_h = S.bins_logspaced()

    def orc(b):
        try:
            return O.chi2_grad(tb5, spec5_h, th5_h[b], 100, bins5_h, obs_h, sig)
        except O.OracleError as e:
            return e.status
    refs, t_orc, n_thr = oracle_pool_map(orc, pick)
    e_bin, e_grad, n_ok = 0.0, 0.0, 0
    for b, r in zip(pick, refs):
        if isinstance(r, int):
            continue
        n_ok += 1
        e_bin = max(e_bin, float(np.abs(binned_d[b] - r[2]).max()))
        e_grad = max(e_grad, grad_rel_err(grad_d[b], r[1]))
    out["fwd_grad"] = {
        "value": round(B * steps_g / (ms / 1e3), 1), "unit": "forward+gradient/s",
        "ms_per_step": round(ms / steps_g, 4),
        "max_abs_err_binned_vs_fp64_oracle_ppm": round(e_bin * 1e6, 5),
        "max_rel_err_grad_vs_fp64_oracle": e_grad,
        "oracle_items_checked": len(pick), "oracle_items_valid": n_ok,
        "cpu_baseline": {"value": round(len(pick) / t_orc, 2), "unit": "forward+gradient/s",
                         "cores": n_thr, "kind": "oracle",
                         "sample": f"FP64 oracle chi^2 + dual-number gradient of the {len(pick)} "
                                   f"checked atmospheres, one per host thread, {t_orc:.2f} s"},
        "workload": "1024 atmospheres, 100 layers, 5 absorbers, 13 x 15 x 10,000 FP32 tables, "
                    "chi^2 against a 50-bin observation, gradient w.r.t. 11 parameters",
        "kernels": {k: {"launches": n, "total_ms": round(v, 3)} for k, (v, n) in prof.items()}}
    # the Jacobian dD_bin/dtheta [1024][50][11] of the same batch from one call (one forward,
    # then a backward pass per bin over that bin's wavenumbers), and its error against the
    # oracle's dual-number Jacobian on the first eight checked atmospheres
    lastj = {}

    def jac_step():
        lastj["r"] = T.adjoint_transit(ctx, tables5, spec5, th5, None, bins5, want_grad=False,
                                       want_binned=False, want_jac=True, workspace=ws5)
    for _ in range(2):
        jac_step()
    steps_j = max(3, steps // 4)
    T.profile_enable(ctx, True)
    ms = time_steps(jac_step, stream, steps_j, flush)
    prof = T.profile_read(ctx)
    T.profile_enable(ctx, False)
    jac = lastj["r"][4].cpu().numpy()
    e_jac = 0.0
    for b, r in list(zip(pick, refs))[:8]:
        if isinstance(r, int):
            continue
        floor = 1e-3 * np.abs(r[3]).max(axis=1, keepdims=True)
        e_jac = max(e_jac, float((np.abs(jac[b] - r[3]) / np.maximum(np.abs(r[3]), floor)).max()))
    out["jacobian"] = {
        "value": round(B * steps_j / (ms / 1e3), 1), "unit": "Jacobians/s (50 bins x 11 parameters)",
        "ms_per_step": round(ms / steps_j, 4),
        "max_rel_err_vs_fp64_oracle": e_jac,
        "workload": "the forward + gradient batch above: 1024 atmospheres, d_jac[1024][50][11] "
                    "from one tr_adjoint_transit call",
        "kernels": {k: {"launches": n, "total_ms": round(v, 3)} for k, (v, n) in prof.items()}}
    return out


def emission_bench(T, ctx, tables, tb, bins, atm, dev, flush, steps: int):
    """Emission model of Sec. 4 on the full-size model (100 layers, 5 absorbers, CIA,
    Rayleigh, cloud, four-node profile, 200,000 wavenumbers, 4-point Gauss-Legendre): spectra/s
    of single-atmosphere calls (tr_forward_emission, native + 50 bins), per-kernel times, the
    vertical pass's rooflines (K read against HBM; its transcendental functions against the
    SFU), and the largest difference from the FP64 oracle over the native spectrum."""
    import torch
    from oracle import oracle as O
    cuda = torch.device("cuda", dev)
    stream = torch.cuda.current_stream(cuda)
    a = T.Atmosphere(ctx, tables, atm)
    n_mu = 4

    def step():
        T.forward_emission(ctx, tables, a, bins=bins, n_mu=n_mu, t_star=5800.0)
    for _ in range(5):
        step()
    T.profile_enable(ctx, True)
    ms = time_steps(step, stream, steps, flush)
    prof = T.profile_read(ctx)
    T.profile_enable(ctx, False)
    nat, _ = T.forward_emission(ctx, tables, a, bins=bins, n_mu=n_mu, t_star=5800.0)
    torch.cuda.synchronize()
    ref = O.emission(tb, atm, n_mu=n_mu, t_star=5800.0)
    err = float(np.abs(nat.cpu().numpy() - ref).max())
    kus = {k: v * 1e3 / n for k, (v, n) in prof.items()}
    N, W = atm.n_layers, tb.n_wn
    e_us = kus.get("k_emission")
    peaks = measured_peaks()
    roof = None
    if e_us:
        by = N * W * 4 + W * 8                      # K read, FP64 output
        gbs = by / (e_us * 1e-6) / 1e9
        sfu_ops = N * W * (n_mu + 2)                # n_mu exponentials, e^x - 1 and 1/x per layer
        props = torch.cuda.get_device_properties(dev)
        sfu_peak = props.multi_processor_count * 16 * 2.07e9
        roof = {"hbm": {"achieved_gbs": round(gbs, 1),
                        "frac": round(gbs / peaks["hbm_gbs"], 4) if peaks else None},
                "sfu": {"ops": sfu_ops, "achieved_per_s": sfu_ops / (e_us * 1e-6),
                        "peak_per_s": sfu_peak,
                        "frac": round(sfu_ops / (e_us * 1e-6) / sfu_peak, 4),
                        "peak_source": "derived: SMs x 16 SFU results per clock x 2070 MHz"}}
    return {"value": round(steps / (ms / 1e3), 1), "unit": "emission spectra/s",
            "ms_per_step": round(ms / steps, 4),
            "kernels_us": {k: round(v, 2) for k, v in kus.items()},
            "k_emission_roofline": roof,
            "max_abs_err_vs_fp64_oracle_ppm": round(err * 1e6, 5),
            "workload": "full-size model, emission (Sec. 4): planet-star flux ratio at 200,000 "
                        "wavenumbers + 50 bins, 4-point Gauss-Legendre, T_star 5800 K"}


def mixed_at_scale(T, ctx, tables, tb, bins, dev, flush, steps: int, warmup: int):
    """1024 atmospheres from the priors, 100 layers, 5 absorbers, 22 x 27 x 200,000 tables,
    full native spectrum: the mixed path (FP16 log10 sigma, BF16 hi+lo tensor-core tau) and
    the plain FP32 path on the same inputs, their throughput and their largest difference."""
    import torch
    from paper_1912_07759_gb300 import synthetic as S
    cuda = torch.device("cuda", dev)
    stream = torch.cuda.current_stream(cuda)
    spec_h = S.batch_spec(5)
    B = 1024
    spec = T.BatchSpec(spec_h, max_layers=100)
    th = torch.tensor(S.draw_theta(5000, B, spec_h), device=cuda)
    nat = torch.empty(B, tb.n_wn, dtype=torch.float64, device=cuda)
    ob = torch.empty(B, bins.n_bin, dtype=torch.float64, device=cuda)
    st = torch.empty(B, dtype=torch.int32, device=cuda)
    ws = torch.empty(T.batch_workspace_size(ctx, tables, spec, None, B), dtype=torch.uint8,
                     device=cuda)
    res, outs = {}, {}
    pick = check_subset(B, seed=66)
    pick_t = torch.tensor(pick, device=cuda)
    for name, prec in (("mixed", T.TR_PREC_MIXED), ("fp32", T.TR_PREC_FP32)):
        def step():
            T.forward_transit_batch(ctx, tables, spec, th, None, bins, precision=prec,
                                    workspace=ws, native=True, out_native=nat, out_binned=ob,
                                    out_status=st)
        for _ in range(warmup):
            step()
        T.profile_enable(ctx, True)
        ms = time_steps(step, stream, steps, flush)
        prof = T.profile_read(ctx)
        T.profile_enable(ctx, False)
        ctx.sync_status()
        outs[name] = nat.index_select(0, pick_t).cpu().numpy()
        res[name] = {"value": round(B * steps / (ms / 1e3), 1), "unit": UNIT,
                     "ms_per_step": round(ms / steps, 3),
                     "kernels": {k: {"launches": n, "total_ms": round(v, 3)}
                                 for k, (v, n) in prof.items()}}
    diff = float(np.abs(outs["mixed"] - outs["fp32"]).max())
    # error of each path against the FP64 oracle over the whole native spectrum of the seeded
    # 64-item subset (the oracle runs one atmosphere per host thread; its rate is this
    # workload's CPU baseline)
    from oracle import oracle as O
    th_h = th.cpu().numpy()
    refs, t_fwd, n_thr = oracle_pool_map(
        lambda b: O.forward(tb, atm_of_theta(S, spec_h, th_h[b]))[0], pick)
    err = {name: [float(np.abs(outs[name][i] - refs[i]).max()) for i in range(len(pick))]
           for name in outs}
    del outs, refs
    del ws
    # forward + chi^2 gradient of the binned spectrum, both precisions
    sig, zn = S.obs_noise(5002, bins.n_bin)
    obs = torch.tensor(0.0105 + sig * zn, device=cuda)      # a flat synthetic observation
    sig_t = torch.tensor(sig, device=cuda)
    wsg = torch.empty(T.batch_workspace_size(ctx, tables, spec, bins, B, with_adjoint=True),
                      dtype=torch.uint8, device=cuda)
    grads, fg = {}, {}
    gpick = check_subset(B, seed=67)
    for name, prec in (("mixed", T.TR_PREC_MIXED), ("fp32", T.TR_PREC_FP32)):
        last = {}

        def gstep():
            last["r"] = T.adjoint_transit(ctx, tables, spec, th, None, bins, obs=obs,
                                          sigma_obs=sig_t, precision=prec, workspace=wsg)
        for _ in range(warmup):
            gstep()
        T.profile_enable(ctx, True)
        ms = time_steps(gstep, stream, steps, flush)
        prof = T.profile_read(ctx)
        T.profile_enable(ctx, False)
        grads[name] = (last["r"][1].cpu().numpy()[gpick], last["r"][3].cpu().numpy()[gpick])
        fg[name] = {"value": round(B * steps / (ms / 1e3), 1), "unit": "forward+gradient/s",
                    "ms_per_step": round(ms / steps, 3),
                    "kernels": {k: {"launches": n, "total_ms": round(v, 3)}
                                for k, (v, n) in prof.items()}}
    del wsg
    gm, gf = grads["mixed"][0], grads["fp32"][0]
    floor = 1e-3 * np.abs(gf).max(axis=1, keepdims=True)
    grel = float((np.abs(gm - gf) / np.maximum(np.abs(gf), floor)).max())
    # each precision's gradient against the oracle's dual-number gradient on the seeded
    # 64-item subset (one atmosphere per host thread)
    obs_h = obs.cpu().numpy()
    bins_h = S.bins_logspaced()
    def orc_grad(b):
        try:
            return O.chi2_grad(tb, spec_h, th_h[b], 100, bins_h, obs_h, sig)[1]
        except O.OracleError:
            return None                                  # a rejected model: no gradient
    grefs, t_grad, n_thr_g = oracle_pool_map(orc_grad, gpick)
    gerr = {}
    for name in grads:
        g, st = grads[name]
        gerr[name] = [grad_rel_err(g[i], grefs[i]) for i in range(len(gpick))
                      if st[i] == 0 and grefs[i] is not None]
    return {"workload": "1024 atmospheres from the priors, 100 layers, 5 absorbers, FP32 + FP16 "
                        "tables 22 x 27 x 200,000, full native spectrum + 50 bins; forward + "
                        "chi^2 gradient over the binned region",
            "mixed": res["mixed"], "fp32": res["fp32"],
            "speedup_mixed_over_fp32": round(res["mixed"]["value"] / res["fp32"]["value"], 3),
            "max_abs_diff_mixed_vs_fp32_ppm_checked": round(diff * 1e6, 4),
            "max_abs_err_vs_fp64_oracle_ppm": {k: round(max(v) * 1e6, 5) for k, v in err.items()},
            "err_vs_fp64_oracle_ppm_per_spectrum": {
                k: {"items": pick, "max_abs_ppm": [round(x * 1e6, 5) for x in v]}
                for k, v in err.items()},
            "oracle_items_checked": len(pick),
            "cpu_baseline": {"value": round(len(pick) / t_fwd, 3), "unit": UNIT,
                             "cores": n_thr, "kind": "oracle",
                             "sample": f"FP64 oracle forward models (whole native spectrum) of "
                                       f"the {len(pick)} checked atmospheres, one per host "
                                       f"thread, {t_fwd:.1f} s"},
            "fwd_grad_mixed": fg["mixed"], "fwd_grad_fp32": fg["fp32"],
            "fwd_grad_speedup_mixed_over_fp32": round(fg["mixed"]["value"] / fg["fp32"]["value"], 3),
            "grad_max_rel_diff_mixed_vs_fp32_checked": round(grel, 6),
            "grad_max_rel_err_vs_fp64_oracle": {k: max(v) for k, v in gerr.items()},
            "grad_rel_err_vs_fp64_oracle_per_result": {
                k: {"items": gpick, "max_rel": [float(f"{x:.3e}") for x in v]}
                for k, v in gerr.items()},
            "grad_oracle_items_checked": len(gpick),
            "grad_cpu_baseline": {"value": round(len(gpick) / t_grad, 3),
                                  "unit": "forward+gradient/s", "cores": n_thr_g,
                                  "kind": "oracle",
                                  "sample": f"FP64 oracle chi^2 + dual-number gradient over the "
                                            f"binned region of the {len(gpick)} checked "
                                            f"atmospheres, one per host thread, {t_grad:.1f} s"}}


def mixed_single(T, ctx, tables, tb, bins, atm, theta, spec, dev, flush, steps: int):
    """The headline workload (one full-size atmosphere, native spectrum + 50 bins) in both
    precisions as CUDA-graph replays: the mixed path (FP16 log10 tables read at half the
    bytes, tensor-core contraction) against the plain FP32 path, with each one's largest
    difference from the FP64 oracle over the native spectrum."""
    import torch
    from oracle import oracle as O
    cuda = torch.device("cuda", dev)
    stream = torch.cuda.current_stream(cuda)
    th = torch.tensor(theta, device=cuda)
    nl = torch.full((1,), atm.n_layers, dtype=torch.int32, device=cuda)
    ws = torch.empty(T.batch_workspace_size(ctx, tables, spec, None, 1), dtype=torch.uint8,
                     device=cuda)
    ref, _, _ = O.forward(tb, atm)
    out = {}
    # fp32: the FP32 path as it runs by default (3xTF32 tensor-core contraction); fp32_ffma:
    # the same path with the contraction pinned to the FFMA kernel (eight warps)
    for name, prec, kind in (("mixed", T.TR_PREC_MIXED, None), ("fp32", T.TR_PREC_FP32, None),
                             ("fp32_ffma", T.TR_PREC_FP32, 1)):
        if kind is not None:
            T.pin_forward_config(ctx, tables, spec, 1, bins, native=True, precision=prec,
                                 form="two-stage", per_sm=0, contract_per_sm=kind)
        g = T.ForwardGraph(ctx, tables, spec, th, nl, bins, precision=prec, workspace=ws,
                           native=True, autotune=True)
        if kind is not None:
            T.pin_forward_config(ctx, tables, spec, 1, bins, native=True, precision=prec,
                                 form=None)

        def step():
            g.launch(stream)
        for _ in range(5):
            step()
        ms = time_steps(step, stream, steps, flush)
        torch.cuda.synchronize()
        err = float(np.abs(g.native[0].cpu().numpy() - ref).max())
        out[name] = {"value": round(steps / (ms / 1e3), 1), "unit": UNIT,
                     "ms_per_step": round(ms / steps, 4),
                     "max_abs_err_vs_fp64_oracle_ppm": round(err * 1e6, 5)}
        del g
    out["speedup_mixed_over_fp32"] = round(out["mixed"]["value"] / out["fp32"]["value"], 3)
    out["speedup_tc_over_ffma_contraction"] = round(out["fp32"]["value"] / out["fp32_ffma"]["value"], 3)
    out["workload"] = ("full-size single forward (100 layers x 200,000 wn, 5 absorbers, CIA, "
                       "Rayleigh, cloud), native + 50 bins, one CUDA-graph replay per step, "
                       "L2 flushed before each")
    del ws
    return out


def exp_interp(T, ctx, tb, atm, theta, spec, dev, flush, steps: int):
    """The full-size single forward with the exponential temperature scheme of Sec. 5
    (sigma = a e^{-b/T} between the bracketing temperatures) on the same tables: spectra/s of
    plain batch calls, per-kernel times and the largest difference from the FP64 oracle's
    exponential scheme over the whole native spectrum."""
    import dataclasses
    import torch
    from oracle import oracle as O
    from paper_1912_07759_gb300 import synthetic as S
    cuda = torch.device("cuda", dev)
    stream = torch.cuda.current_stream(cuda)
    th = torch.tensor(theta, device=cuda)
    nl = torch.full((1,), atm.n_layers, dtype=torch.int32, device=cuda)
    tbe = dataclasses.replace(tb, interp_mode=S.INTERP_EXP)
    tables = T.XsecTables(ctx, tbe, storage=T.TR_STORE_FP32)
    bins = T.Bins(ctx, tables, *S.bins_logspaced())
    ws = torch.empty(T.batch_workspace_size(ctx, tables, spec, None, 1), dtype=torch.uint8,
                     device=cuda)
    nat = torch.empty(1, tb.n_wn, dtype=torch.float64, device=cuda)
    ob = torch.empty(1, bins.n_bin, dtype=torch.float64, device=cuda)
    st = torch.empty(1, dtype=torch.int32, device=cuda)

    def step():
        T.forward_transit_batch(ctx, tables, spec, th, nl, bins, workspace=ws, native=True,
                                out_native=nat, out_binned=ob, out_status=st)
    for _ in range(5):
        step()
    T.profile_enable(ctx, True)
    ms = time_steps(step, stream, steps, flush)
    prof = T.profile_read(ctx)
    T.profile_enable(ctx, False)
    ctx.sync_status()
    ref, _, _ = O.forward(tbe, atm)
    err = float(np.abs(nat[0].cpu().numpy() - ref).max())
    out = {"value": round(steps / (ms / 1e3), 1), "unit": UNIT, "ms_per_step": round(ms / steps, 4),
           "kernels_us": {k: round(v * 1e3 / n, 2) for k, (v, n) in prof.items()},
           "max_abs_err_vs_fp64_oracle_ppm": round(err * 1e6, 5),
           "workload": "full-size single forward (plain batch calls), exponential temperature "
                       "scheme of Sec. 5 on the same FP32 tables"}
    del tables, ws
    return out


def instrument_bench(T, ctx, bins, tb, dev, flush, steps: int):
    """FluxBinner with uncertainties (Sec. 4.5) then the SNR instrument model (Sec. 7) on 1,024
    seeded native spectra over the bins' native range of the 200,000-wavenumber grid: spectra/s,
    the binning kernels' read rate against the measured HBM bandwidth, and the largest relative
    difference from the oracle's statement of both on two of the spectra."""
    import torch
    from oracle import oracle as O
    from paper_1912_07759_gb300 import synthetic as S
    cuda = torch.device("cuda", dev)
    stream = torch.cuda.current_stream(cuda)
    B = 1024
    i0, i1 = bins.native_range
    n = i1 - i0
    g = torch.Generator(device=cuda)
    g.manual_seed(31)
    flux = 0.0105 + 1e-4 * torch.randn(B, n, dtype=torch.float64, device=cuda, generator=g)
    sig = 3e-5 * (1.0 + torch.rand(B, n, dtype=torch.float64, device=cuda, generator=g))
    z = torch.randn(B, bins.n_bin, dtype=torch.float64, device=cuda, generator=g)

    def step():
        f, s = T.bin_spectra(ctx, bins, flux, sig, base=i0)
        T.snr_instrument(ctx, f, 200.0, 4, z)
    for _ in range(3):
        step()
    T.profile_enable(ctx, True)
    ms = time_steps(step, stream, steps, flush)
    prof = T.profile_read(ctx)
    T.profile_enable(ctx, False)
    ctx.sync_status()
    # against the oracle (bins over the full grid; the spectra are zero outside the range)
    f2, s2 = T.bin_spectra(ctx, bins, flux[:2], sig[:2], base=i0)
    torch.cuda.synchronize()
    full_f = np.zeros((2, tb.n_wn))
    full_s = np.zeros((2, tb.n_wn))
    full_f[:, i0:i1] = flux[:2].cpu().numpy()
    full_s[:, i0:i1] = sig[:2].cpu().numpy()
    centre, width = S.bins_logspaced()
    rf, rs = O.bin_with_uncertainty(tb.wn_grid, centre, width, full_f, full_s)
    err = max(float(np.max(np.abs(f2.cpu().numpy() - rf) / np.abs(rf))),
              float(np.max(np.abs(s2.cpu().numpy() - rs) / np.abs(rs))))
    kus = {k: v * 1e3 / c for k, (v, c) in prof.items()}
    bin_us = kus.get("k_bin", 0.0) + kus.get("k_bin_sigma", 0.0)
    read = 2 * B * n * 8                               # flux and uncertainties, FP64
    peaks = measured_peaks()
    gbs = read / (bin_us * 1e-6) / 1e9 if bin_us > 0 else None
    return {"value": round(B * steps / (ms / 1e3), 1),
            "unit": "binned spectra with uncertainties + SNR observations /s",
            "ms_per_step": round(ms / steps, 4),
            "kernels_us": {k: round(v, 2) for k, v in kus.items()},
            "binning_read_gbs": round(gbs, 1) if gbs else None,
            "binning_frac_of_measured_hbm": (round(gbs / peaks["hbm_gbs"], 4)
                                             if gbs and peaks else None),
            "max_rel_err_vs_fp64_oracle": err,
            "workload": f"1,024 native spectra with uncertainties over {n} wavenumbers "
                        f"(the 50 bins' range of the 200,000-wavenumber grid), FP64"}


def algorithmic_bytes(tb, atm, kernel: str = "method") -> int:
    """Bytes the forward model must move at least once: every distinct (molecule, P row,
    T row) table row the layers' brackets touch, the CIA rows and the Rayleigh rows (brackets
    follow the interpolation rule: largest grid index <= x, clamped, at the layer pressures
    and temperatures of the workload) and the FP64 native output -- the method's bytes, the
    opacity kernel's roofline numerator.  kernel="design_opacity" adds the K write of the
    two-stage form (N layers x wavenumbers x 4 B); "k_contract*" gives the contraction's own
    traffic (K read, path lengths, FP64 output)."""
    N = atm.n_layers
    W = tb.n_wn
    if kernel.startswith("k_contract"):
        return int(N * W * 4 + N * N * 4 + W * 8)
    lnb = np.log(atm.p_max) + (np.log(atm.p_min) - np.log(atm.p_max)) * np.arange(N + 1) / N
    pb = np.exp(lnb)
    P = pb[:-1] * np.sqrt(pb[1:] / pb[:-1])
    x = np.log10(P)
    xs, ts = atm.tnode_log10p[::-1], atm.tnode_t[::-1]
    T = np.interp(x, xs, ts)

    def br(grid, v):
        v = np.clip(v, grid[0], grid[-1])
        return np.clip(np.searchsorted(grid, v, side="right") - 1, 0, len(grid) - 2)

    ip, it = br(tb.p_grid, P), br(tb.t_grid, T)
    rows = set()
    for a, b in zip(ip, it):
        rows.update({(a, b), (a, b + 1), (a + 1, b), (a + 1, b + 1)})
    n_mol = tb.sigma.shape[0]
    by = n_mol * len(rows) * W * 4
    if tb.cia_pair.shape[0]:
        itc = br(tb.t_grid_cia, T)
        by += tb.cia_pair.shape[0] * len(set(itc) | set(itc + 1)) * W * 4
    if tb.rayleigh is not None:
        by += len(tb.species) * W * 4
    by += W * 8
    if kernel == "design_opacity":
        by += N * W * 4
    return int(by)


CSRC = os.path.join(ROOT, "paper_1912_07759_gb300", "csrc")
KERNEL_SOURCES = {  # the files each kernel is built from (its ncu summary records their hash)
    "k_opacity_fp32": ["forward_fp32.cu", "opacity.h", "tma.h", "tr_internal.h"],
    "k_opacity_fp16": ["forward_fp32.cu", "opacity.h", "tma.h", "tr_internal.h"],
    "k_contract_fp32": ["forward_fp32.cu", "tma.h", "tr_internal.h"],
    "k_contract_tc": ["tc_fp32.cu", "umma.h", "tma.h", "tr_internal.h"],
    "k_contract_umma": ["mixed.cu", "umma.h", "tma.h", "tr_internal.h"],
    "k_forward_tma": ["fused.cu", "opacity.h", "tma.h", "tr_internal.h"],
    "k_profile": ["geometry.cu", "tr_internal.h"],
    "k_altitude": ["geometry.cu", "tr_internal.h"],
    "k_pathlen": ["geometry.cu", "tr_internal.h"],
    "k_dl_tf32": ["tc_fp32.cu", "tr_internal.h"],
    "k_bin": ["binning.cu", "tr_internal.h"],
}


def sources_sha256(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()


def roofline_of(kname, prof_entry, tb, atm, peaks, sm_mhz, n_sm, step_s=None):
    """Roofline of one kernel of the main workload.  The opacity (and fused) kernels against
    the measured HBM copy bandwidth: achieved = the method's bytes (table rows, CIA, Rayleigh,
    FP64 output; algorithmic_bytes) / mean launch time; the two-stage form's K write is
    reported beside it as design bytes, and the method's bytes over the whole step's time as
    step_frac.  The FP32 contraction against the FP32 FMA pipe (SMs x 128 lanes x 2 FLOP x
    the SM clock seen during the timed region; algorithmic FLOPs = 2 x n_wn x N(N+1)/2 per
    launch)."""
    k_ms, k_n = prof_entry
    per_launch_s = k_ms / 1e3 / k_n
    if kname == "k_contract_tc":
        # the tensor-core contraction streams K once from HBM: its bytes (K read, path lengths,
        # FP64 output) against the measured copy bandwidth; beside it the tensor pipe: the TF32
        # flops the 3xTF32 MMAs execute (three products per 8-layer slice over the rays the
        # slice reaches, rounded to the MMA's N step of 16) against the TF32 peak taken as the
        # measured BF16 burst figure x the nominal TF32/BF16 ratio (1.125 / 2.25 PFLOP/s)
        N, W = atm.n_layers, tb.n_wn
        by = algorithmic_bytes(tb, atm, kname)
        peak, peak_src = (peaks["hbm_gbs"], "measured") if peaks else (6800.0, "fallback")
        KP = (N + 15) // 16 * 16
        n_sum = sum(min(KP, (8 * ks + 8 + 15) // 16 * 16) for ks in range(KP // 8))
        units = (W + 127) // 128
        tflop = 3 * 2 * 128 * 8 * n_sum * units / 1e12
        tc_peak = (peaks["bf16_tflops"] if peaks else 1900.0) * 0.5
        achieved = by / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": ncu_traffic(kname, "config2"),
                "kernel": kname, "algorithmic_bytes": by,
                "kernel_us": round(per_launch_s * 1e6, 2), "peak_source": peak_src,
                "tensor": {"executed_tflop": round(tflop, 4),
                           "achieved_tflops": round(tflop / per_launch_s, 1),
                           "peak_tflops": round(tc_peak, 1),
                           "frac": round(tflop / per_launch_s / tc_peak, 4),
                           "peak_source": "measured BF16 burst x nominal TF32/BF16 ratio 0.5"},
                "method_flops": 2.0 * W * N * (N + 1) / 2}
    if kname == "k_contract_fp32":
        N = atm.n_layers
        flops = 2.0 * tb.n_wn * N * (N + 1) / 2
        peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
        achieved = flops / per_launch_s / 1e12
        return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": ncu_traffic(kname, "config2"),
                "kernel": kname, "algorithmic_flops": flops,
                "kernel_us": round(per_launch_s * 1e6, 2),
                "peak_source": "derived: FP32 FMA lanes x SM clock during the timed region"}
    alg = algorithmic_bytes(tb, atm)
    peak, peak_src = (peaks["hbm_gbs"], "measured") if peaks else (6800.0, "fallback")
    achieved = alg / per_launch_s / 1e9
    out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
           "frac": round(achieved / peak, 4), "traffic": ncu_traffic(kname, "config2"),
           "kernel": kname, "algorithmic_bytes": alg,
           "kernel_us": round(per_launch_s * 1e6, 2), "peak_source": peak_src}
    if kname.startswith("k_opacity"):
        design = algorithmic_bytes(tb, atm, "design_opacity")
        out["design_bytes"] = design
        out["design_frac"] = round(design / per_launch_s / 1e9 / peak, 4)
    if step_s:
        out["step_frac"] = round(alg / step_s / 1e9 / peak, 4)
    return out


def ncu_traffic(kernel: str, workload_tag: str):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, if it was taken on
    the kernel's sources as they are now (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}.{workload_tag}.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != sources_sha256(kernel):
            return None
        return float(kv["traffic_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.lines = []
        self.idx = device_index

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "100"]
            import torch
            try:
                bus = torch.cuda.get_device_properties(self.idx).pci_bus_id
                cmd += ["-i", str(bus)]
            except Exception:
                cmd += ["-i", str(self.idx)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ CPU oracle
def oracle_rate(tb, atm, seconds: float):
    """Spectra/s of the FP64 oracle (one thread) on consecutive wavenumber slices of the
    workload, scaled to whole spectra; returns (rate, sample description)."""
    from oracle import oracle as O
    from paper_1912_07759_gb300 import synthetic as S
    W = tb.n_wn
    ws = 2000
    t_used, wn_done, calls, i0 = 0.0, 0, 0, 0
    while t_used < seconds:
        sl = slice(i0, i0 + ws)
        sub = S.Tables(p_grid=tb.p_grid, t_grid=tb.t_grid, wn_grid=tb.wn_grid[sl],
                       sigma=np.ascontiguousarray(tb.sigma[..., sl]), species=tb.species,
                       mass_amu=tb.mass_amu, t_grid_cia=tb.t_grid_cia, cia_pair=tb.cia_pair,
                       cia=np.ascontiguousarray(tb.cia[..., sl]),
                       rayleigh=None if tb.rayleigh is None else np.ascontiguousarray(tb.rayleigh[:, sl]),
                       oor_mode=tb.oor_mode)
        t0 = time.perf_counter()
        O.forward(sub, atm)
        t_used += time.perf_counter() - t0
        wn_done += ws
        calls += 1
        i0 = (i0 + ws) % (W - ws)
    rate = (wn_done / W) / t_used
    return rate, (f"{calls} oracle calls on {ws}-wavenumber slices of the 200,000-wavenumber "
                  f"workload ({wn_done / W:.3f} spectra of work, {t_used:.1f} s, 1 thread)")


# ------------------------------------------------------------------------------ ranks
def max_over_ranks(dist, value: float, device=None) -> float:
    """The largest of the ranks' values (a job's time is its slowest rank's); the value itself
    without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, t_max_ms: float) -> float:
    """Whole-job throughput of `world` replicas that each processed `units_per_rank` units,
    timed by the slowest rank (units per second)."""
    return world * units_per_rank / (t_max_ms / 1e3)


# ------------------------------------------------------------------------------ arms
def dist_setup(n):
    import torch
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        lr = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(lr)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lr))
        return dist, dist.get_rank(), dist.get_world_size(), lr
    return None, 0, 1, 0


def run_native(args):
    import torch
    dist, rank, world, dev = dist_setup(args.gpus)
    from paper_1912_07759_gb300 import transit as T
    from paper_1912_07759_gb300 import build as Bld
    Bld.build()
    S, tb, atm, spec_h, theta = workload()
    ctx = T.TransitContext(dev)
    tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
    bins = T.Bins(ctx, tables, *S.bins_logspaced())
    spec = T.BatchSpec(spec_h, max_layers=atm.n_layers)
    cuda = torch.device("cuda", dev)
    th = torch.tensor(theta, device=cuda)
    nl = torch.full((1,), atm.n_layers, dtype=torch.int32, device=cuda)
    ws = torch.empty(T.batch_workspace_size(ctx, tables, spec, None, 1), dtype=torch.uint8,
                     device=cuda)
    native = torch.empty(1, tb.n_wn, dtype=torch.float64, device=cuda)
    binned = torch.empty(1, bins.n_bin, dtype=torch.float64, device=cuda)
    status = torch.empty(1, dtype=torch.int32, device=cuda)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=cuda)
    stream = torch.cuda.current_stream(cuda)

    # the forward as one CUDA graph (tr_capture_forward_batch): the autotuner first times the
    # forward's configurations on this workload and the graph runs the fastest; a sampler
    # replays it with new parameters written into `th`
    graph = T.ForwardGraph(ctx, tables, spec, th, nl, bins, workspace=ws, native=True,
                           autotune=not args.no_tune)
    tuned = graph.info() if not args.no_tune else None

    def step():
        graph.launch(stream)

    def step_plain():
        T.forward_transit_batch(ctx, tables, spec, th, nl, bins, workspace=ws, native=True,
                                out_native=native, out_binned=binned, out_status=status)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    assert int(graph.status.item()) == 0

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    step_ms = float(sum(a.elapsed_time(b) for a, b in ev))
    # per-kernel device times (CUDA events around each launch on its stream) from plain batch
    # calls of the same configuration; graph replays cannot bracket single kernels
    Kp = min(K, 1000)
    for _ in range(3):
        step_plain()
    torch.cuda.synchronize()
    T.profile_enable(ctx, True)
    for _ in range(Kp):
        flush.zero_()
        step_plain()
    torch.cuda.synchronize()
    prof = T.profile_read(ctx)
    T.profile_enable(ctx, False)
    assert int(status.item()) == 0
    t_max = max_over_ranks(dist, step_ms, cuda)
    if dist is not None:
        dist.barrier()
    value = job_rate(world, K, t_max)

    # end to end through the C ABI with host buffers: every step copies its parameter vector
    # from pinned host memory into a graph's input, replays the graph and copies the native
    # and binned spectrum back to pinned host memory.  Two graphs of the same forward (the
    # second shares the workspace; each has its own input and outputs) alternate, and each
    # step's read-back runs on a second stream while the next step computes
    Ke = min(K, 1000)
    th2 = torch.tensor(theta, device=cuda)
    graph2 = T.ForwardGraph(ctx, tables, spec, th2, nl, bins, workspace=ws, native=True,
                            autotune=not args.no_tune)
    gs, ths = (graph, graph2), (th, th2)
    copy_stream = torch.cuda.Stream(cuda)
    th_host = torch.tensor(theta).pin_memory()
    nat_host = [torch.empty(1, tb.n_wn, dtype=torch.float64).pin_memory() for _ in range(2)]
    bin_host = [torch.empty(1, bins.n_bin, dtype=torch.float64).pin_memory() for _ in range(2)]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_steps(n):
        for k in range(n):
            i = k & 1
            if k >= 2:
                stream.wait_event(copied[i])          # this graph's last read-back is done
            ths[i].copy_(th_host, non_blocking=True)
            gs[i].launch(stream)
            done[i].record(stream)
            copy_stream.wait_event(done[i])
            with torch.cuda.stream(copy_stream):
                nat_host[i].copy_(gs[i].native, non_blocking=True)
                bin_host[i].copy_(gs[i].binned, non_blocking=True)
            copied[i].record(copy_stream)
        stream.wait_stream(copy_stream)

    e2e_steps(4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_steps(Ke)
    e1.record(stream)
    torch.cuda.synchronize()
    assert np.array_equal(nat_host[0].numpy(), nat_host[1].numpy())
    e2e_ms = max_over_ranks(dist, e0.elapsed_time(e1), cuda)
    e2e_value = job_rate(world, Ke, e2e_ms)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    clk_mhz = (clk.summary() or {}).get("sm_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    rooflines = {k: roofline_of(k, prof[k], tb, atm, peaks, clk_mhz, n_sm,
                                step_s=t_max / K / 1e3) for k in prof
                 if k.startswith(("k_opacity", "k_contract_fp32", "k_contract_tc", "k_forward"))}
    kname = max(rooflines, key=lambda k: prof[k][0])   # the dominant kernel of the step
    roof = rooflines[kname]
    kernels = {k: {"launches": n, "total_ms": round(ms, 3), "share": round(ms / sum(v[0] for v in prof.values()), 4)}
               for k, (ms, n) in prof.items()}
    kernels_note = (f"per-kernel times from {Kp} plain batch calls of the graph's configuration "
                    "(CUDA events on the launching stream, L2 flushed before each call); "
                    "k_pathlen and k_dl_tf32 run on the forward's second stream beside "
                    "k_opacity, so their event span includes the wait for SM room and is "
                    "off the step's critical path")
    extra = {}
    if args.batch_steps > 0:
        extra = batched_workloads(T, ctx, dev, flush, args.batch_steps, 3)
        extra["mixed_at_scale"] = mixed_at_scale(T, ctx, tables, tb, bins, dev, flush, 2, 1)
        extra["mixed_single"] = mixed_single(T, ctx, tables, tb, bins, atm, theta, spec, dev,
                                             flush, min(args.steps, 500))
        extra["exp_interpolation"] = exp_interp(T, ctx, tb, atm, theta, spec, dev, flush,
                                                min(args.steps, 500))
        try:
            extra["emission"] = emission_bench(T, ctx, tables, tb, bins, atm, dev, flush,
                                               min(args.steps, 500))
        except Exception as e:                          # an auxiliary line: report, go on
            extra["emission"] = {"error": f"{type(e).__name__}: {e}"[:300]}
        try:
            extra["instrument"] = instrument_bench(T, ctx, bins, tb, dev, flush,
                                                   min(args.steps, 200))
        except Exception as e:                          # an auxiliary line: report, go on
            extra["instrument"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    cpu = None
    if world == 1:
        rate, sample = oracle_rate(tb, atm, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
               "kind": "oracle", "sample": sample}
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": round(t_max / K, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(world),
        "precision": "FP32 tables and arithmetic, FP64 geometry and depth sum",
        "roofline": roof, "rooflines": rooflines, "autotuned": tuned, "kernels": kernels,
        "kernels_note": kernels_note,
        "gpu_launches": int(round(sum(n for _, n in prof.values()) / Kp * K)),
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT,
                "h2d_bytes_per_step": int(th.numel() * 8),
                "d2h_bytes_per_step": int((native.numel() + binned.numel()) * 8),
                "steps": Ke,
                "loop": "two graphs alternating; each step's read-back on a second stream "
                        "overlaps the next step's compute (no L2 flush)"},
        "clocks": clocks,
    }
    out.update(extra)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    S, tb, atm, spec_h, theta = workload()
    from oracle import oracle as O
    O.build()
    K, Wm = args.steps, max(args.warmup, 3)
    # bounded sample per step: a slice of the native grid sized so K + W steps fit ~2 minutes
    W = tb.n_wn
    budget = 120.0 / (K + Wm)
    t0 = time.perf_counter()
    rate_probe, _ = oracle_rate(tb, atm, 2.0)
    per_wn = 1.0 / (rate_probe * W)
    ws = int(min(W // 4, max(64, budget / per_wn)))
    times = []
    i0 = 0
    for k in range(K + Wm):
        sl = slice(i0, i0 + ws)
        sub = S.Tables(p_grid=tb.p_grid, t_grid=tb.t_grid, wn_grid=tb.wn_grid[sl],
                       sigma=np.ascontiguousarray(tb.sigma[..., sl]), species=tb.species,
                       mass_amu=tb.mass_amu, t_grid_cia=tb.t_grid_cia, cia_pair=tb.cia_pair,
                       cia=np.ascontiguousarray(tb.cia[..., sl]),
                       rayleigh=np.ascontiguousarray(tb.rayleigh[:, sl]),
                       oor_mode=tb.oor_mode)
        t1 = time.perf_counter()
        O.forward(sub, atm)
        if k >= Wm:
            times.append(time.perf_counter() - t1)
        i0 = (i0 + ws) % (W - ws)
    total = sum(times)
    value = (K * ws / W) / total
    sample = (f"each step: FP64 oracle forward model on a {ws}-wavenumber slice of the "
              f"200,000-wavenumber workload (1 thread); value scaled to whole spectra")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": K, "warmup": Wm, "ms_per_step": 1e3 * total / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args.gpus),
           "cpu_baseline": {"kind": "oracle", "cores": 1, "host_cores": os.cpu_count(),
                            "sample": sample, "value": value, "unit": UNIT},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "wall_s": round(time.perf_counter() - t0, 1)}
    print(json.dumps(out), flush=True)


def ncu_case(name: str):
    """Small workloads for ncu captures (each kernel launched twice; capture the second)."""
    import torch
    from paper_1912_07759_gb300 import transit as T
    from paper_1912_07759_gb300 import build as Bld
    from paper_1912_07759_gb300 import synthetic as S
    Bld.build()
    ctx = T.TransitContext(0)
    cuda = torch.device("cuda", 0)
    if name == "emission":
        _, tb, atm, _, _ = workload()
        tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32)
        a = T.Atmosphere(ctx, tables, atm)
        for _ in range(2):
            nat, _ = T.forward_emission(ctx, tables, a, n_mu=4, t_star=5800.0)
        torch.cuda.synchronize()
        ctx.sync_status()
        assert bool(torch.isfinite(nat).all())
        print(f"ncu case {name}: ok", flush=True)
        return
    if name == "adjoint":
        tb = S.make_tables(4, 5, 13, 15, 10000, with_cia=False)
        tables = T.XsecTables(ctx, tb)
        bins = T.Bins(ctx, tables, *S.bins_logspaced())
        spec_h = S.batch_spec(5)
        spec = T.BatchSpec(spec_h, max_layers=100)
        th = torch.tensor(S.draw_theta(4001, 256, spec_h), device=cuda)
        sig, z = S.obs_noise(4002, bins.n_bin)
        obs = torch.tensor(0.0105 + sig * z, device=cuda)
        for _ in range(2):
            _, _, _, st = T.adjoint_transit(ctx, tables, spec, th, None, bins, obs=obs,
                                            sigma_obs=torch.tensor(sig, device=cuda))
    else:
        if name in ("single", "single_ffma"):
            _, tb, atm, spec_h, theta = workload()
            tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32)
            bins = T.Bins(ctx, tables, *S.bins_logspaced())
            spec = T.BatchSpec(spec_h, max_layers=atm.n_layers)
            th = torch.tensor(theta, device=cuda)
            B, prec = 1, T.TR_PREC_FP32
            # the configuration the autotuner picks for this workload (3xTF32 contraction), or
            # the FFMA contraction with eight warps (the form of more than 112 layers)
            T.pin_forward_config(ctx, tables, spec, 1, bins, native=True, form="two-stage",
                                 per_sm=0, contract_per_sm=3 if name == "single" else 1)
        else:
            tb = S.make_tables(2, 5, 22, 27, 100000, with_cia=True)
            tables = T.XsecTables(ctx, tb, storage=T.TR_STORE_FP32 | T.TR_STORE_FP16_LOG10)
            bins = T.Bins(ctx, tables, *S.bins_logspaced())
            spec_h = S.batch_spec(5)
            spec = T.BatchSpec(spec_h, max_layers=100)
            B, prec = 8, T.TR_PREC_MIXED
            th = torch.tensor(S.draw_theta(5000, B, spec_h), device=cuda)
        for _ in range(2):
            _, st, _ = T.forward_transit_batch(ctx, tables, spec, th, None, bins, precision=prec,
                                               native=True)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert int(st.abs().sum().item()) == 0
    print(f"ncu case {name}: ok", flush=True)


def main():
    args = parse()
    if args.ncu_case:
        ncu_case(args.ncu_case)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
