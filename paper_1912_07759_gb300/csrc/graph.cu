// graph.cu -- the batched forward for sampler loops: tuned once, captured once in a CUDA graph,
// replayed with one launch per step.
//
// tr_capture_forward_batch
//   1. autotune (optional): every configuration of the forward's search space (ForwardChoice:
//      the two-stage form with 3, 2 or 1 opacity CTAs per SM and the ring depth that leaves,
//      times (FP32) the contraction as one CTA per SM with two K tiles or two CTAs per SM with
//      one, or the fused FP32 kernel) is run on the caller's own inputs -- one untimed run, then
//      kTuneReps runs timed with CUDA events on the caller's stream -- and the fastest median
//      wins; it is remembered on the context for this batch shape, so plain
//      tr_forward_transit_batch calls of the same shape use it too;
//   2. capture: the whole batched forward (geometry, opacity, contraction, binning) is issued
//      on a private stream in capture mode and instantiated as one executable graph.  The graph
//      keeps the buffers it was captured with: the caller updates d_theta / d_nlayers in place
//      between launches.
// tr_graph_launch replays it on any stream.
#include <algorithm>
#include <cstring>
#include <vector>
#include "tr_internal.h"

struct tr_graph {
  int device = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  tr::ForwardChoice choice{};
  float tuned_ms = 0.f;        // median time of the chosen configuration (0 when not tuned)
  int n_candidates = 0;        // configurations timed
};

using namespace tr;

namespace {

constexpr int kTuneReps = 5;

int graph_fail(tr_ctx* ctx, cudaError_t e, const char* what) {
  return set_error(ctx, TR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The search space for this batch (precision, K buffer always present in the workspace).
std::vector<ForwardChoice> candidates(const tr_tables* t, const tr_batch_desc* d, int B,
                                      int precision) {
  std::vector<ForwardChoice> c;
  const bool fp32 = precision == TR_PREC_FP32;
  // the FP32 contraction: the tensor-core kernel where the layer count fits it (one numerical
  // form per shape, so the choice never depends on timing noise), else the FFMA kernel with
  // eight or eleven warps; the mixed path has one tensor-core contraction
  std::vector<int> kinds;
  if (!fp32) kinds = {kContractAuto};
  else if (tc_contract_fits(d->max_layers)) kinds = {kContractTC};
  else kinds = {kContractFfma8, kContractFfma11};
  for (int per_sm : {0, 2, 1})
    for (int cps : kinds) c.push_back({kFormTwoStage, per_sm, 0, cps});
  if (fp32 && t->interp_mode == TR_INTERP_LINEAR && d->gas_mode == TR_GAS_CONSTANT &&
      fused_forward_fits(t->n_mol, t->n_cia, d->max_layers, B))
    c.push_back({kFormFused, 0, 0, 0});
  return c;
}

}  // namespace

extern "C" int tr_capture_forward_batch(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d,
                                        int B, const double* d_theta, const int32_t* d_nlayers,
                                        const tr_bins* bins, double* d_native, double* d_binned,
                                        int32_t* d_status, int precision, void* ws,
                                        size_t ws_bytes, int autotune, void* stream,
                                        tr_graph** out) {
  if (!out) return set_error(ctx, TR_ERR_ARG, "null output");
  *out = nullptr;
  int rc = check_forward_batch_args(ctx, t, d, B, d_theta, bins, d_native, d_binned);
  if (rc != TR_OK) return rc;
  if (B == 0) return set_error(ctx, TR_ERR_ARG, "empty batch");
  if (precision != TR_PREC_FP32 && precision != TR_PREC_MIXED)
    return set_error(ctx, TR_ERR_ARG, "unknown precision");
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool native = d_native != nullptr;
  // the workspace must exist before capture (no allocation may happen inside it)
  const size_t need = forward_batch_need(t, d, B, bins, native, precision);
  if (!ws) {
    rc = ensure_scratch(ctx, need);
    if (rc != TR_OK) return rc;
    ws = ctx->scratch;
    ws_bytes = ctx->scratch_bytes;
  } else if (ws_bytes < need) {
    return set_error(ctx, TR_ERR_OOM, "workspace smaller than tr_batch_workspace_size()");
  }
  const bool prof = ctx->prof_on;            // no kernel timers inside tuning or capture
  ctx->prof_on = false;
  auto restore = [&](int code) { ctx->prof_on = prof; return code; };

  tr_graph* g = new tr_graph();
  g->device = ctx->device;
  const std::string key = batch_shape_key(t, d, B, bins, native, precision);
  ForwardChoice best{kFormTwoStage, 0, 0, 0};
  const auto hit = ctx->tuned.find(key);
  if (hit != ctx->tuned.end()) {
    best = hit->second;
  } else if (autotune) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { delete g; return restore(graph_fail(ctx, e, "tuning events")); }
    float best_ms = 0.f;
    bool have = false;
    for (const ForwardChoice& c : candidates(t, d, B, precision)) {
      std::vector<float> ms;
      bool ok = true;
      for (int r = 0; r <= kTuneReps && ok; ++r) {
        cudaEventRecord(e0, s);
        ok = forward_batch_impl(ctx, t, d, B, d_theta, d_nlayers, bins, d_native, d_binned,
                                d_status, precision, ws, ws_bytes, s, &c) == TR_OK;
        cudaEventRecord(e1, s);
        if (!ok) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
        float m = 0.f;
        cudaEventElapsedTime(&m, e0, e1);
        if (r > 0) ms.push_back(m);                // the first run is untimed warm-up
      }
      if (!ok) { cudaGetLastError(); continue; }   // a configuration that does not launch here
      std::sort(ms.begin(), ms.end());
      const float med = ms[ms.size() / 2];
      ++g->n_candidates;
      if (!have || med < best_ms) { best = c; best_ms = med; have = true; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!have) { delete g; return restore(set_error(ctx, TR_ERR_CUDA, "no configuration ran")); }
    g->tuned_ms = best_ms;
    ctx->tuned[key] = best;
  }
  g->choice = best;

  // capture the forward on a private stream
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete g; return restore(graph_fail(ctx, e, "capture stream")); }
  e = cudaStreamSynchronize(s);              // tuning runs have finished with the buffers
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    delete g;
    return restore(graph_fail(ctx, e, "begin capture"));
  }
  rc = forward_batch_impl(ctx, t, d, B, d_theta, d_nlayers, bins, d_native, d_binned, d_status,
                          precision, ws, ws_bytes, cs, &best);
  e = cudaStreamEndCapture(cs, &g->graph);
  cudaStreamDestroy(cs);
  if (rc != TR_OK || e != cudaSuccess) {
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return restore(rc != TR_OK ? rc : graph_fail(ctx, e, "end capture"));
  }
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g->graph);
    delete g;
    return restore(graph_fail(ctx, e, "graph instantiation"));
  }
  *out = g;
  return restore(TR_OK);
}

extern "C" int tr_graph_launch(tr_graph* g, void* stream) {
  if (!g || !g->exec) return TR_ERR_ARG;
  cudaSetDevice(g->device);
  const cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TR_OK : TR_ERR_CUDA;
}

extern "C" int tr_graph_info(const tr_graph* g, int* form, int* per_sm, int* stages,
                             int* contract_per_sm, float* tuned_ms, int* n_candidates) {
  if (!g) return TR_ERR_ARG;
  if (contract_per_sm) *contract_per_sm = g->choice.contract_per_sm;
  if (form) *form = g->choice.form;
  if (per_sm) *per_sm = g->choice.per_sm;
  if (stages) *stages = g->choice.stages;
  if (tuned_ms) *tuned_ms = g->tuned_ms;
  if (n_candidates) *n_candidates = g->n_candidates;
  return TR_OK;
}

extern "C" void tr_free_graph(tr_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

extern "C" int tr_pin_forward_config(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d,
                                     int B, const tr_bins* bins, int native, int precision,
                                     int form, int per_sm, int stages, int contract_per_sm) {
  if (!ctx || !t || !d || B < 1) return set_error(ctx, TR_ERR_ARG, "bad arguments");
  if (!native && !bins) return set_error(ctx, TR_ERR_ARG, "binned shape needs bins");
  if (form != kFormTwoStage && form != kFormFused) return set_error(ctx, TR_ERR_ARG, "bad form");
  if (form == kFormFused && precision != TR_PREC_FP32)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "the fused form is FP32 only");
  if (per_sm < 0 || per_sm > 3 || stages < 0 || contract_per_sm < 0 || contract_per_sm > 3)
    return set_error(ctx, TR_ERR_ARG, "bad tunables");
  if (contract_per_sm == kContractTC && !tc_contract_fits(d->max_layers))
    return set_error(ctx, TR_ERR_UNSUPPORTED, "the tensor-core contraction takes up to 112 layers");
  const std::string key = batch_shape_key(t, d, B, bins, native != 0, precision);
  ctx->tuned[key] = ForwardChoice{form, per_sm, stages, contract_per_sm};
  return TR_OK;
}

extern "C" int tr_unpin_forward_config(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d,
                                       int B, const tr_bins* bins, int native, int precision) {
  if (!ctx || !t || !d || B < 1) return set_error(ctx, TR_ERR_ARG, "bad arguments");
  if (!native && !bins) return set_error(ctx, TR_ERR_ARG, "binned shape needs bins");
  ctx->tuned.erase(batch_shape_key(t, d, B, bins, native != 0, precision));
  return TR_OK;
}
