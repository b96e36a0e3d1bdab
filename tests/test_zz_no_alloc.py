"""tr_forward_transit_batch_noalloc: the batched forward model for callers that cannot
allocate device memory (for example a sampler's likelihood callback held to a fixed memory
budget, or a host that cannot own device buffers).  It must give the same binned spectra and
statuses as tr_forward_transit_batch, call after call, although every call reuses the same
built-in scratch array.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_1912_07759_gb300 import synthetic as S

TOL = 1e-7          # 0.1 ppm absolute depth, the bar of the other parity tests

pytestmark = pytest.mark.gpu


def test_noalloc_batch_matches_workspace_batch_on_consecutive_calls():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1912_07759_gb300 import transit as T
    from paper_1912_07759_gb300 import _native as N

    ctx = T.TransitContext(0)
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins = T.Bins(ctx, tables, *S.bins_logspaced())
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=150)
    B = 40
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = ctx.lib
    # B = 40 atmospheres of up to 150 layers fit the built-in scratch (the call would return
    # TR_ERR_ARG otherwise, which the assertion on rc below would report)
    for call, seed in enumerate((501, 502)):       # two calls in a row, different inputs
        th_np = S.draw_theta(seed, B, spec_h)
        nl_np = S.draw_nlayers(seed + 1, B)
        th_np[3, :2] = [-0.1, -0.2]                # one invalid item per call
        th = torch.tensor(th_np, device="cuda")
        nl = torch.tensor(nl_np, device="cuda")
        ref, ref_st = T.forward_transit_batch(ctx, tables, spec, th, nl, bins)
        out = torch.full((B, bins.n_bin), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((B,), -1, dtype=torch.int32, device="cuda")
        rc = lib.tr_forward_transit_batch_noalloc(
            ctx.handle, tables.handle, C.byref(spec.desc), B, C.c_void_p(th.data_ptr()),
            C.c_void_p(nl.data_ptr()), bins.handle, C.c_void_p(out.data_ptr()),
            C.c_void_p(st.data_ptr()), stream)
        assert rc == 0, lib.tr_last_error(ctx.handle).decode()
        torch.cuda.synchronize()
        assert torch.equal(st, ref_st), call
        assert int(st[3]) == T.TR_ERR_INVALID_MODEL
        diff = (out - ref).abs().max().item()
        assert diff <= TOL, (call, diff)


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1912_07759_gb300 import transit as T
    from paper_1912_07759_gb300 import _native as N

    ctx = T.TransitContext(0)
    tb = S.make_tables(1, 2, 13, 15, 10000, with_cia=False)
    tables = T.XsecTables(ctx, tb)
    bins = T.Bins(ctx, tables, *S.bins_logspaced())
    spec_h = S.batch_spec(2)
    spec = T.BatchSpec(spec_h, max_layers=150)
    B = 4096
    th = torch.tensor(S.draw_theta(1, B, spec_h), device="cuda")
    out = torch.empty(B, bins.n_bin, dtype=torch.float64, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    rc = ctx.lib.tr_forward_transit_batch_noalloc(
        ctx.handle, tables.handle, C.byref(spec.desc), B, C.c_void_p(th.data_ptr()), None,
        bins.handle, C.c_void_p(out.data_ptr()), C.c_void_p(st.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == N.TR_ERR_ARG
    assert b"scratch" in ctx.lib.tr_last_error(ctx.handle)
