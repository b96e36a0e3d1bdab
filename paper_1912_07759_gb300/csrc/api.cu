// api.cu -- the extern "C" entry points of libtransit.so (declared in include/transit.h):
// argument checks, device memory of the handles, workspace carving and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>
#include "tr_internal.h"

using namespace tr;

namespace {

int fail(tr_ctx* ctx, int code, const char* fmt, const char* detail = "") {
  if (ctx) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), fmt, detail);
    ctx->err = buf;
  }
  return code;
}

int cuda_fail(tr_ctx* ctx, cudaError_t e, const char* what) {
  if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? TR_ERR_OOM : TR_ERR_CUDA;
}

bool ascending(const double* a, int n) {
  for (int i = 0; i + 1 < n; ++i)
    if (!(a[i] < a[i + 1])) return false;
  return true;
}

// Exponent e with 2^e near the largest |value|, so that value * 2^-e sits near 1.
int scale_exponent(const double* v, size_t n) {
  double mx = 0.0;
  for (size_t i = 0; i < n; ++i) mx = std::max(mx, std::fabs(v[i]));
  if (!(mx > 0.0) || !std::isfinite(mx)) return 0;
  int e = 0;
  std::frexp(mx, &e);
  return e;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct WsLayout {
  size_t layers, z, tl, zf, op, opx, dlt, dlp, aj, rayc, items, depth, end;
};

WsLayout ws_layout(int B, int max_layers, int n_in) {
  WsLayout w{};
  size_t off = 0;
  w.layers = off; off = align_up(off + (size_t)B * max_layers * sizeof(LayerDesc), 256);
  w.z = off;      off = align_up(off + (size_t)B * (max_layers + 1) * sizeof(double), 256);
  w.tl = off;     off = align_up(off + (size_t)B * max_layers * sizeof(double), 256);
  w.zf = off;     off = align_up(off + (size_t)B * (max_layers + 1) * sizeof(float4), 256);
  w.op = off;     off = align_up(off + (size_t)B * max_layers * 2 * sizeof(float4), 256);
  w.opx = off;    off = align_up(off + (size_t)B * kMaxZones * kOpxStride * sizeof(float), 256);
  w.dlt = off;    off = align_up(off + (size_t)B * max_layers * pad8(max_layers) * sizeof(float), 256);
  w.dlp = off;    off = align_up(off + (size_t)B * dlp_offset(max_layers) * sizeof(float), 256);
  w.aj = off;     off = align_up(off + (size_t)B * pad8(max_layers) * sizeof(float), 256);
  w.rayc = off;   off = align_up(off + (size_t)B * kMaxZones * TR_MAX_SPECIES * sizeof(float), 256);
  w.items = off;  off = align_up(off + (size_t)B * sizeof(ItemGeom), 256);
  w.depth = off;  off = align_up(off + (size_t)B * n_in * sizeof(double), 256);
  w.end = off;
  return w;
}

ItemBuffers carve(void* base, const WsLayout& w, int max_layers) {
  char* p = static_cast<char*>(base);
  ItemBuffers b;
  b.layers = reinterpret_cast<LayerDesc*>(p + w.layers);
  b.z = reinterpret_cast<double*>(p + w.z);
  b.tl = reinterpret_cast<double*>(p + w.tl);
  b.zf = reinterpret_cast<float4*>(p + w.zf);
  b.op = reinterpret_cast<float4*>(p + w.op);
  b.opx = reinterpret_cast<float*>(p + w.opx);
  b.dlt = reinterpret_cast<float*>(p + w.dlt);
  b.dlp = reinterpret_cast<float*>(p + w.dlp);
  b.aj = reinterpret_cast<float*>(p + w.aj);
  b.rayc = reinterpret_cast<float*>(p + w.rayc);
  b.items = reinterpret_cast<ItemGeom*>(p + w.items);
  b.npad = pad8(max_layers);
  b.zoned = 0;
  return b;
}

GeomParams geom_params(const tr_tables* t, int n_tnodes, const double* tnode_log10p,
                       const double* fill, double p_max, double p_min, double m_p, double r_s,
                       double p_cloud_bot, double kappa, int grav, int cloud, int max_layers,
                       int t_profile, int gas_mode, double t_int) {
  GeomParams g{};
  g.n_mol = t->n_mol; g.n_species = t->n_species; g.n_tnodes = n_tnodes;
  g.t_profile = t_profile; g.gas_mode = gas_mode; g.t_int = t_int;
  g.n_chem = gas_mode == TR_GAS_TWOLAYER ? 3 * t->n_mol : t->n_mol;
  g.n_tpar = t_profile == TR_TPROF_GUILLOT ? 5 : n_tnodes;
  g.gm_p = kG * m_p;
  g.n_p = t->n_p; g.n_t = t->n_t; g.n_cia = t->n_cia; g.n_t_cia = t->n_t_cia;
  g.gravity_mode = grav; g.cloud_mode = cloud; g.oor_mode = t->oor_mode;
  g.interp_mode = t->interp_mode;
  g.max_layers = max_layers; g.has_ray = t->has_ray;
  for (int q = 0; q < t->n_cia; ++q) {
    g.cia_a[q] = t->cia_a[q]; g.cia_b[q] = t->cia_b[q];
    g.cia_scale[q] = t->cia_scale[q];
  }
  for (int s = 0; s < t->n_species; ++s) {
    g.ray_scale[s] = t->ray_scale[s];
    g.mass[s] = t->mass[s];
  }
  for (int f = t->n_mol; f < t->n_species; ++f) g.fill[f] = fill[f - t->n_mol];
  for (int k = 0; k < n_tnodes; ++k) g.tnode_log10p[k] = tnode_log10p[k];
  g.p_max = p_max; g.p_min = p_min; g.m_p = m_p; g.r_s = r_s;
  g.p_cloud_bot = p_cloud_bot; g.kappa_cloud = kappa;
  g.ln_pmax = std::log(p_max);
  g.ln_pmin = std::log(p_min);
  g.inv_kb = 1.0 / kKB;
  g.inv_rs2 = 1.0 / (r_s * r_s);
  g.amu_g_mp = kAMU * kG * m_p;
  g.fill_mass = 0.0;
  for (int f = t->n_mol; f < t->n_species; ++f) g.fill_mass += g.fill[f] * g.mass[f];
  g.p_cbot = p_cloud_bot > 0.0 ? p_cloud_bot : p_max;
  g.ln_cbot = p_cloud_bot > 0.0 ? std::log(p_cloud_bot) : g.ln_pmax;
  for (int k = 0; k + 1 < n_tnodes; ++k)
    g.inv_dlog10p[k] = 1.0 / (tnode_log10p[k + 1] - tnode_log10p[k]);
  g.p_grid = t->d_p_grid; g.t_grid = t->d_t_grid; g.t_grid_cia = t->d_t_grid_cia;
  g.inv_dp = t->d_inv_dp; g.inv_dt = t->d_inv_dt; g.inv_dtc = t->d_inv_dtc;
  return g;
}

FwdParams fwd_params(const tr_tables* t, int max_layers, const ItemBuffers& buf, int wn_begin,
                     int wn_count, double* out, long long stride, int* dev_err) {
  FwdParams p{};
  p.dev_err = dev_err;
  p.sigma = t->d_sigma; p.n_mol = t->n_mol; p.n_p = t->n_p; p.n_t = t->n_t;
  p.wn_pad = t->wn_pad;
  p.cia = t->d_cia; p.n_cia = t->n_cia; p.n_t_cia = t->n_t_cia;
  p.ray = t->has_ray ? t->d_ray : nullptr; p.n_species = t->n_species;
  p.max_layers = max_layers; p.buf = buf;
  p.wn_begin = wn_begin; p.wn_count = wn_count;
  p.out = out; p.out_stride = stride;
  p.interp_mode = t->interp_mode;
  return p;
}

}  // namespace

size_t tr::forward_workspace_bytes(int B, int max_layers, int n_in) {
  return ws_layout(B, max_layers, n_in).end;
}

int tr::ensure_scratch(tr_ctx* ctx, size_t bytes) {
  if (ctx->scratch_bytes >= bytes) return TR_OK;
  if (ctx->scratch) cudaFree(ctx->scratch);
  ctx->scratch = nullptr; ctx->scratch_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->scratch, bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation");
  ctx->scratch_bytes = bytes;
  return TR_OK;
}

namespace {

int check_batch_desc(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d) {
  if (!d) return fail(ctx, TR_ERR_ARG, "null batch descriptor");
  if (d->t_profile != TR_TPROF_NPOINT && d->t_profile != TR_TPROF_GUILLOT)
    return fail(ctx, TR_ERR_ARG, "unknown temperature profile");
  if (d->gas_mode != TR_GAS_CONSTANT && d->gas_mode != TR_GAS_TWOLAYER)
    return fail(ctx, TR_ERR_ARG, "unknown gas profile");
  if (d->t_profile == TR_TPROF_GUILLOT && !(d->t_int >= 0.0 && std::isfinite(d->t_int)))
    return fail(ctx, TR_ERR_ARG, "bad internal temperature");
  if (d->n_tnodes < 1 || d->n_tnodes > TR_MAX_TNODES || !d->tnode_log10p)
    return fail(ctx, TR_ERR_ARG, "bad temperature nodes");
  for (int k = 0; k + 1 < d->n_tnodes; ++k)
    if (!(d->tnode_log10p[k] > d->tnode_log10p[k + 1]))
      return fail(ctx, TR_ERR_ARG, "temperature node pressures must be strictly descending");
  if (t->n_species > t->n_mol && !d->fill_frac) return fail(ctx, TR_ERR_ARG, "null fill_frac");
  if (!(d->p_max > d->p_min) || !(d->p_min > 0.0)) return fail(ctx, TR_ERR_ARG, "bad pressure range");
  if (!(d->m_p > 0.0) || !(d->r_s > 0.0)) return fail(ctx, TR_ERR_ARG, "bad planet mass or star radius");
  if (d->max_layers < 1 || d->max_layers > TR_MAX_LAYERS) return fail(ctx, TR_ERR_ARG, "bad max_layers");
  if (d->cloud_mode < 0 || d->cloud_mode > 2 || d->gravity_mode < 0 || d->gravity_mode > 1)
    return fail(ctx, TR_ERR_ARG, "bad cloud or gravity mode");
  return TR_OK;
}

}  // namespace

// Helpers for entry points defined in other translation units (they reuse the workspace
// layout and parameter packing above).
ItemBuffers tr::carve_forward_workspace(void* base, int B, int max_layers, int n_in,
                                        double** depth) {
  const WsLayout wl = ws_layout(B, max_layers, n_in);
  *depth = reinterpret_cast<double*>(static_cast<char*>(base) + wl.depth);
  return carve(base, wl, max_layers);
}

int tr::validate_batch_desc(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d) {
  return check_batch_desc(ctx, t, d);
}

GeomParams tr::batch_geom_params(const tr_tables* t, const tr_batch_desc* d) {
  return geom_params(t, d->n_tnodes, d->tnode_log10p, d->fill_frac, d->p_max, d->p_min, d->m_p,
                     d->r_s, d->p_cloud_bot, d->kappa_cloud, d->gravity_mode, d->cloud_mode,
                     d->max_layers, d->t_profile, d->gas_mode, d->t_int);
}

int tr::batch_n_theta(const tr_tables* t, const tr_batch_desc* d) {
  return (d->gas_mode == TR_GAS_TWOLAYER ? 3 * t->n_mol : t->n_mol) +
         (d->t_profile == TR_TPROF_GUILLOT ? 5 : d->n_tnodes) + 2;
}

FwdParams tr::forward_fp32_params(const tr_tables* t, int max_layers, const ItemBuffers& buf,
                                  int wn_begin, int wn_count, double* out, long long stride,
                                  int* dev_err) {
  return fwd_params(t, max_layers, buf, wn_begin, wn_count, out, stride, dev_err);
}

// ============================================================================ context
extern "C" int tr_create(tr_ctx** ctx, int device) {
  if (!ctx) return TR_ERR_ARG;
  *ctx = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) return TR_ERR_CUDA;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return TR_ERR_CUDA;
  tr_ctx* c = new tr_ctx();
  c->device = device;
  e = cudaMalloc(&c->dev_err, 256);
  if (e == cudaSuccess) e = cudaMemset(c->dev_err, 0, 256);

  if (e != cudaSuccess) { delete c; return TR_ERR_CUDA; }
  *ctx = c;
  return TR_OK;
}

extern "C" int tr_selftest_wait_timeout(tr_ctx* ctx, void* stream) {
  if (!ctx) return TR_ERR_ARG;
  cudaSetDevice(ctx->device);
  const cudaError_t e = launch_wait_selftest(ctx->dev_err, 1000, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "self-test launch");
}

extern "C" int tr_sync_status(tr_ctx* ctx, void* stream) {
  if (!ctx) return TR_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  int flags = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flags, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tr_sync_status");
  if (flags) {
    cudaMemset(ctx->dev_err, 0, sizeof(int));
    return fail(ctx, TR_ERR_TIMEOUT, "a bounded device wait expired; outputs of the affected calls are invalid");
  }
  return TR_OK;
}

extern "C" void tr_destroy(tr_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->dev_err) cudaFree(ctx->dev_err);
  for (auto& p : ctx->prof_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : ctx->prof_pool) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  delete ctx;
}

bool tr::fork_ready(tr_ctx* ctx, Fork* f) {
  if (!ctx->aux) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&a, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      if (a) cudaEventDestroy(a);
      if (st) cudaStreamDestroy(st);
      cudaGetLastError();
      return false;
    }
    ctx->aux = st; ctx->ev_fork = a; ctx->ev_join = b;
  }
  f->aux = ctx->aux;
  f->open = f->pending = false;
  return true;
}

cudaError_t tr::fork_start(tr_ctx* ctx, Fork* f, cudaStream_t s, bool detached) {
  if (!f || !f->pending) return cudaSuccess;
  f->pending = false;
  cudaStream_t ps = s;
  if (detached) {
    const cudaError_t e = cudaStreamWaitEvent(f->aux, ctx->ev_fork, 0);
    if (e != cudaSuccess) return e;
    f->open = true;
    ps = f->aux;
  }
  {
    KernelTimer kt(ctx, "k_altitude", ps);
    const cudaError_t e = launch_altitude(f->gp, f->B, f->buf, ps);
    if (e != cudaSuccess) return e;
  }
  KernelTimer kt(ctx, "k_pathlen", ps);
  return launch_pathlen(f->gp, f->B, f->buf, ps);
}

void tr::join_fork(tr_ctx* ctx, Fork* f, cudaStream_t s) {
  if (!f || !f->open) return;
  cudaEventRecord(ctx->ev_join, f->aux);
  cudaStreamWaitEvent(s, ctx->ev_join, 0);
  f->open = false;
}

// ============================================================================ kernel timing
tr::KernelTimer::KernelTimer(tr_ctx* ctx, const char* name, cudaStream_t s)
    : ctx_(ctx), name_(name), s_(s) {
  if (!ctx_ || !ctx_->prof_on) return;
  for (cudaEvent_t* e : {&a_, &b_}) {
    if (!ctx_->prof_pool.empty()) { *e = ctx_->prof_pool.back(); ctx_->prof_pool.pop_back(); }
    else if (cudaEventCreate(e) != cudaSuccess) { *e = nullptr; }
  }
  if (a_) cudaEventRecord(a_, s_);
}

tr::KernelTimer::~KernelTimer() {
  if (!a_ || !b_) {
    if (a_) ctx_->prof_pool.push_back(a_);
    if (b_) ctx_->prof_pool.push_back(b_);
    return;
  }
  cudaEventRecord(b_, s_);
  ctx_->prof_pending.push_back({name_, a_, b_});
}

extern "C" int tr_profile_enable(tr_ctx* ctx, int on) {
  if (!ctx) return TR_ERR_ARG;
  for (auto& p : ctx->prof_pending) {
    cudaEventSynchronize(p.b);
    ctx->prof_pool.push_back(p.a); ctx->prof_pool.push_back(p.b);
  }
  ctx->prof_pending.clear();
  ctx->prof_totals.clear();
  ctx->prof_on = on != 0;
  return TR_OK;
}

extern "C" int tr_profile_read(tr_ctx* ctx, int max_kernels, char* names, double* total_ms,
                               int64_t* launches, int* n_kernels) {
  if (!ctx || max_kernels < 0 || (max_kernels > 0 && (!names || !total_ms || !launches)))
    return TR_ERR_ARG;
  for (auto& p : ctx->prof_pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel timing");
    auto& tot = ctx->prof_totals[p.name];
    tot.first += ms; tot.second += 1;
    ctx->prof_pool.push_back(p.a); ctx->prof_pool.push_back(p.b);
  }
  ctx->prof_pending.clear();
  int k = 0;
  for (auto& kv : ctx->prof_totals) {
    if (k < max_kernels) {
      std::snprintf(names + 48 * k, 48, "%s", kv.first.c_str());
      total_ms[k] = kv.second.first;
      launches[k] = kv.second.second;
    }
    ++k;
  }
  if (n_kernels) *n_kernels = k;
  return TR_OK;
}

extern "C" const char* tr_last_error(const tr_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

// ============================================================================ tables
extern "C" void tr_free_tables(tr_tables* t) {
  if (!t) return;
  cudaSetDevice(t->device);
  cudaFree(t->d_sigma); cudaFree(t->d_cia); cudaFree(t->d_ray);
  cudaFree(t->d_p_grid); cudaFree(t->d_t_grid); cudaFree(t->d_t_grid_cia); cudaFree(t->d_wn);
  cudaFree(t->d_inv_dp); cudaFree(t->d_inv_dt); cudaFree(t->d_inv_dtc);
  cudaFree(t->d_logsig16);
  delete[] t->h_wn;
  delete t;
}

extern "C" size_t tr_tables_device_bytes(const tr_tables* t) { return t ? t->device_bytes : 0; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

bool tr::encode_2d_f32(CUtensorMap* m, const void* base, unsigned long long cols,
                       unsigned long long rows, unsigned long long row_stride_bytes,
                       unsigned box_cols, unsigned box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || !base) return false;
  const cuuint64_t gdim[2] = {cols, rows};
  const cuuint64_t gstride[1] = {row_stride_bytes};
  const cuuint32_t bdim[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), gdim, gstride, bdim,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a table [outer...][wn_pad] with the innermost box kOpacityTile wavenumbers;
// dims/box list the outer axes innermost first.  Out-of-range box elements read as zero.
static bool encode_table_map(CUtensorMap* m, const void* base, bool fp16, int wn_pad, int rank,
                             const int* dims, const int* box, int tile) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || !base) return false;
  const size_t es = fp16 ? 2 : 4;
  cuuint64_t gdim[5], gstride[4];
  cuuint32_t bdim[5], estr[5];
  gdim[0] = (cuuint64_t)wn_pad;
  bdim[0] = (cuuint32_t)tile;
  estr[0] = 1;
  cuuint64_t stride = (cuuint64_t)wn_pad * es;
  for (int i = 1; i < rank; ++i) {
    gdim[i] = (cuuint64_t)dims[i - 1];
    bdim[i] = (cuuint32_t)box[i - 1];
    estr[i] = 1;
    gstride[i - 1] = stride;
    stride *= (cuuint64_t)dims[i - 1];
  }
  const CUresult r = fn(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        (cuuint32_t)rank, const_cast<void*>(base), gdim, gstride, bdim, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The opacity kernels' tensor maps: sigma (FP32) and log10 sigma (FP16) as {wn, T, P, molecule}
// with box {tile, 2, 2, n_mol}; CIA as {wn, T_cia, pair} with box {tile, 2, n_cia}; tile =
// kOpacityTile for the two-stage kernel, kFusedTile for the fused one.
static bool encode_tables(tr_tables* t) {
  if (t->n_mol > 0) {
    const int dims[3] = {t->n_t, t->n_p, t->n_mol}, box[3] = {2, 2, t->n_mol};
    if (t->d_sigma &&
        (!encode_table_map(&t->tm_sig32, t->d_sigma, false, t->wn_pad, 4, dims, box, kOpacityTile) ||
         !encode_table_map(&t->tm_sig32_f, t->d_sigma, false, t->wn_pad, 4, dims, box, kFusedTile)))
      return false;
    if (t->d_logsig16 &&
        !encode_table_map(&t->tm_sig16, t->d_logsig16, true, t->wn_pad, 4, dims, box, kOpacityTile))
      return false;
  }
  if (t->n_cia > 0) {
    const int dims[2] = {t->n_t_cia, t->n_cia}, box[2] = {2, t->n_cia};
    if (!encode_table_map(&t->tm_cia, t->d_cia, false, t->wn_pad, 3, dims, box, kOpacityTile) ||
        !encode_table_map(&t->tm_cia_f, t->d_cia, false, t->wn_pad, 3, dims, box, kFusedTile))
      return false;
  }
  return true;
}

extern "C" int tr_load_xsec_tables(tr_ctx* ctx, const tr_table_desc* d, tr_tables** out) {
  if (!ctx || !d || !out) return fail(ctx, TR_ERR_ARG, "null argument");
  *out = nullptr;
  if (d->n_mol < 0 || d->n_mol > TR_MAX_MOL) return fail(ctx, TR_ERR_ARG, "n_mol out of range");
  if (d->n_p < 2 || d->n_t < 2 || d->n_wn < 2) return fail(ctx, TR_ERR_ARG, "table grids need >= 2 points");
  if ((long long)d->n_p * d->n_t > 16384 || d->n_t_cia > 1024)
    return fail(ctx, TR_ERR_ARG, "table grids larger than 16384 (P, T) cells or 1024 CIA temperatures");
  if (d->n_species < d->n_mol || d->n_species > TR_MAX_SPECIES) return fail(ctx, TR_ERR_ARG, "bad n_species");
  if (d->n_cia < 0 || d->n_cia > TR_MAX_CIA) return fail(ctx, TR_ERR_ARG, "n_cia out of range");
  if (d->n_cia > 0 && (d->n_t_cia < 2 || !d->t_grid_cia || !d->cia || !d->cia_pair))
    return fail(ctx, TR_ERR_ARG, "bad CIA tables");
  if (!d->p_grid || !d->t_grid || !d->wn_grid || !d->mass_amu || (d->n_mol > 0 && !d->sigma))
    return fail(ctx, TR_ERR_ARG, "null table array");
  if (!ascending(d->p_grid, d->n_p) || !ascending(d->t_grid, d->n_t) ||
      !ascending(d->wn_grid, d->n_wn) || (d->n_cia > 0 && !ascending(d->t_grid_cia, d->n_t_cia)))
    return fail(ctx, TR_ERR_ARG, "grids must be strictly ascending");
  if (!(d->p_grid[0] > 0.0) || !(d->t_grid[0] > 0.0)) return fail(ctx, TR_ERR_ARG, "grids must be positive");
  for (int q = 0; q < d->n_cia; ++q)
    for (int k = 0; k < 2; ++k)
      if (d->cia_pair[2 * q + k] < 0 || d->cia_pair[2 * q + k] >= d->n_species)
        return fail(ctx, TR_ERR_ARG, "CIA pair species index out of range");
  if (d->storage & ~(TR_STORE_FP32 | TR_STORE_FP16_LOG10) || d->storage == 0)
    return fail(ctx, TR_ERR_ARG, "bad storage mask");
  if (d->oor_mode != TR_OOR_CLAMP && d->oor_mode != TR_OOR_PAPER_ZERO)
    return fail(ctx, TR_ERR_ARG, "bad out-of-range mode");
  if (d->interp_mode != TR_INTERP_LINEAR && d->interp_mode != TR_INTERP_EXP)
    return fail(ctx, TR_ERR_ARG, "bad interpolation mode");
  cudaSetDevice(ctx->device);

  tr_tables* t = new tr_tables();
  t->device = ctx->device;
  t->n_mol = d->n_mol; t->n_p = d->n_p; t->n_t = d->n_t; t->n_wn = d->n_wn;
  t->wn_pad = (d->n_wn + 7) & ~7;
  t->n_cia = d->n_cia; t->n_t_cia = d->n_cia > 0 ? d->n_t_cia : 0;
  t->n_species = d->n_species; t->storage = d->storage; t->oor_mode = d->oor_mode;
  t->interp_mode = d->interp_mode;
  t->has_ray = d->rayleigh != nullptr;
  for (int s = 0; s < d->n_species; ++s) t->mass[s] = d->mass_amu[s];
  t->h_wn = new double[d->n_wn];
  std::memcpy(t->h_wn, d->wn_grid, sizeof(double) * d->n_wn);
  const size_t W = d->n_wn, WP = t->wn_pad;
  cudaError_t e = cudaSuccess;
  auto bail = [&](const char* what) {
    const int rc = cuda_fail(ctx, e, what);
    tr_free_tables(t);
    return rc;
  };

  // grids
  e = cudaMalloc(&t->d_p_grid, sizeof(double) * d->n_p); if (e) return bail("alloc p grid");
  e = cudaMalloc(&t->d_t_grid, sizeof(double) * d->n_t); if (e) return bail("alloc t grid");
  e = cudaMemcpy(t->d_p_grid, d->p_grid, sizeof(double) * d->n_p, cudaMemcpyHostToDevice); if (e) return bail("copy p grid");
  e = cudaMemcpy(t->d_t_grid, d->t_grid, sizeof(double) * d->n_t, cudaMemcpyHostToDevice); if (e) return bail("copy t grid");
  t->device_bytes += sizeof(double) * (d->n_p + d->n_t);
  e = cudaMalloc(&t->d_wn, sizeof(double) * d->n_wn); if (e) return bail("alloc wn grid");
  e = cudaMemcpy(t->d_wn, d->wn_grid, sizeof(double) * d->n_wn, cudaMemcpyHostToDevice); if (e) return bail("copy wn grid");
  t->device_bytes += sizeof(double) * d->n_wn;
  if (d->n_cia > 0) {
    e = cudaMalloc(&t->d_t_grid_cia, sizeof(double) * d->n_t_cia); if (e) return bail("alloc cia grid");
    e = cudaMemcpy(t->d_t_grid_cia, d->t_grid_cia, sizeof(double) * d->n_t_cia, cudaMemcpyHostToDevice);
    if (e) return bail("copy cia grid");
  }
  // inverse grid spacings: interpolation weights become multiplications on the device
  auto upload_inv = [&](const double* g, int n, double** dst) -> cudaError_t {
    std::vector<double> inv(std::max(n - 1, 1), 0.0);
    for (int i = 0; i + 1 < n; ++i) inv[i] = 1.0 / (g[i + 1] - g[i]);
    cudaError_t r = cudaMalloc(dst, sizeof(double) * inv.size());
    if (r == cudaSuccess) r = cudaMemcpy(*dst, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice);
    return r;
  };
  e = upload_inv(d->p_grid, d->n_p, &t->d_inv_dp); if (e) return bail("inverse P spacings");
  e = upload_inv(d->t_grid, d->n_t, &t->d_inv_dt); if (e) return bail("inverse T spacings");
  if (d->n_cia > 0) { e = upload_inv(d->t_grid_cia, d->n_t_cia, &t->d_inv_dtc); if (e) return bail("inverse CIA spacings"); }

  // sigma: rows of n_wn floats copied into rows of wn_pad floats (zero padding)
  const size_t rows = (size_t)d->n_mol * d->n_p * d->n_t;
  if (rows > 0) {                     // FP16 log tables are converted from this upload
    e = cudaMalloc(&t->d_sigma, sizeof(float) * rows * WP); if (e) return bail("alloc sigma");
    t->device_bytes += sizeof(float) * rows * WP;
    e = cudaMemset(t->d_sigma, 0, sizeof(float) * rows * WP); if (e) return bail("clear sigma");
    e = cudaMemcpy2D(t->d_sigma, WP * sizeof(float), d->sigma, W * sizeof(float),
                     W * sizeof(float), rows, cudaMemcpyHostToDevice);
    if (e) return bail("copy sigma");
  }
  // CIA and Rayleigh: double host arrays -> FP32 scaled by 2^-e per pair / species
  if (d->n_cia > 0) {
    const size_t per = (size_t)d->n_t_cia * W;
    std::vector<float> tmp((size_t)d->n_cia * d->n_t_cia * WP, 0.f);
    for (int q = 0; q < d->n_cia; ++q) {
      t->cia_a[q] = d->cia_pair[2 * q]; t->cia_b[q] = d->cia_pair[2 * q + 1];
      const double* src = d->cia + q * per;
      const int ex = scale_exponent(src, per);
      t->cia_scale[q] = std::ldexp(1.0, ex);
      for (int it = 0; it < d->n_t_cia; ++it)
        for (size_t i = 0; i < W; ++i)
          tmp[((size_t)q * d->n_t_cia + it) * WP + i] = (float)std::ldexp(src[(size_t)it * W + i], -ex);
    }
    e = cudaMalloc(&t->d_cia, sizeof(float) * tmp.size()); if (e) return bail("alloc cia");
    e = cudaMemcpy(t->d_cia, tmp.data(), sizeof(float) * tmp.size(), cudaMemcpyHostToDevice);
    if (e) return bail("copy cia");
    t->device_bytes += sizeof(float) * tmp.size();
  }
  if (t->has_ray) {
    std::vector<float> tmp((size_t)d->n_species * WP, 0.f);
    for (int s = 0; s < d->n_species; ++s) {
      const double* src = d->rayleigh + (size_t)s * W;
      const int ex = scale_exponent(src, W);
      t->ray_scale[s] = std::ldexp(1.0, ex);
      for (size_t i = 0; i < W; ++i) tmp[(size_t)s * WP + i] = (float)std::ldexp(src[i], -ex);
    }
    e = cudaMalloc(&t->d_ray, sizeof(float) * tmp.size()); if (e) return bail("alloc rayleigh");
    e = cudaMemcpy(t->d_ray, tmp.data(), sizeof(float) * tmp.size(), cudaMemcpyHostToDevice);
    if (e) return bail("copy rayleigh");
    t->device_bytes += sizeof(float) * tmp.size();
  }
  if (d->storage & TR_STORE_FP16_LOG10) {
    // offsets c_m: the stored values are log10 sigma - c_m with c_m three decades below the
    // 99.5th percentile of the molecule's log10 sigma (sampled), so the strong values that set
    // the spectrum sit at |x| < 4, where FP16 spacing is at most 2^-9 dex
    const size_t per = (size_t)d->n_p * d->n_t * W;
    for (int m = 0; m < d->n_mol; ++m) {
      std::vector<float> smp;
      const size_t step = std::max<size_t>(1, per / 200000);
      for (size_t i = 0; i < per; i += step) {
        const float v = d->sigma[(size_t)m * per + i];
        if (v > 0.f) smp.push_back(std::log10(v));
      }
      float c = 0.f;
      if (!smp.empty()) {
        const size_t k = (size_t)(0.995 * (smp.size() - 1));
        std::nth_element(smp.begin(), smp.begin() + k, smp.end());
        c = smp[k] - 3.f;
      }
      t->logsig_offset[m] = c;
    }
    const int rc = build_fp16_log_tables(ctx, t);
    if (rc != TR_OK) { tr_free_tables(t); return rc; }
  }
  if (!(d->storage & TR_STORE_FP32) && t->d_sigma) {
    cudaFree(t->d_sigma);
    t->d_sigma = nullptr;
    t->device_bytes -= sizeof(float) * rows * WP;
  }
  if (!encode_tables(t)) {
    tr_free_tables(t);
    return fail(ctx, TR_ERR_CUDA, "TMA tensor-map encoding of the tables failed");
  }
  *out = t;
  return TR_OK;
}

// ============================================================================ bins
extern "C" void tr_free_bins(tr_bins* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaFree(b->mem);
  delete b;
}

extern "C" int tr_bins_native_range(const tr_bins* b, int* i0, int* i1) {
  if (!b || !i0 || !i1) return TR_ERR_ARG;
  *i0 = b->dev.i0; *i1 = b->dev.i1;
  return TR_OK;
}

extern "C" int tr_bin_spectra(tr_ctx* ctx, const tr_bins* bins, int B, const double* d_native,
                              const double* d_native_sigma, long long stride, int base,
                              double* d_binned, double* d_binned_sigma, void* stream) {
  if (!ctx || !bins || !d_native || !d_binned || B < 0)
    return fail(ctx, TR_ERR_ARG, "null argument");
  if (d_native_sigma && !d_binned_sigma) return fail(ctx, TR_ERR_ARG, "no output for sigma");
  if (base < 0 || base > bins->dev.i0 || stride < (long long)(bins->dev.i1 - base))
    return fail(ctx, TR_ERR_ARG, "native range does not cover the bins");
  if (B == 0) return TR_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = run_bin(ctx, bins, B, d_native, stride, base, d_binned, s);
  if (rc != TR_OK || !d_native_sigma) return rc;
  KernelTimer kt(ctx, "k_bin_sigma", s);
  const cudaError_t e = launch_bin_sigma(bins->dev, B, d_native_sigma, stride, base,
                                         d_binned_sigma, s);
  return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "binned-uncertainty kernel");
}

extern "C" int tr_snr_instrument(tr_ctx* ctx, int B, int n_bin, const double* d_binned,
                                 double snr, int n_obs, const double* d_z, double* d_obs,
                                 double* d_sigma, void* stream) {
  if (!ctx || !d_binned || !d_z || !d_obs || !d_sigma || B < 0 || n_bin < 1)
    return fail(ctx, TR_ERR_ARG, "bad instrument arguments");
  if (!(snr > 0.0) || n_obs < 1) return fail(ctx, TR_ERR_ARG, "snr must be > 0, n_obs >= 1");
  if (B == 0) return TR_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  KernelTimer kt(ctx, "k_snr", s);
  const cudaError_t e = launch_snr(B, n_bin, d_binned, snr, n_obs, d_z, d_obs, d_sigma, s);
  return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "instrument kernel");
}

extern "C" int tr_make_bins(tr_ctx* ctx, const tr_tables* t, int n_bin, const double* lc,
                            const double* lw, tr_bins** out) {
  if (!ctx || !t || !lc || !lw || !out || n_bin < 1) return fail(ctx, TR_ERR_ARG, "bad bins arguments");
  *out = nullptr;
  const int W = t->n_wn;
  const double* wn = t->h_wn;
  std::vector<int> row_ptr(n_bin + 1, 0), col;
  std::vector<double> w, inv_wsum(n_bin, 0.0);
  std::vector<int> bin_lo, bin_hi;
  int lo = W, hi = 0;
  // FluxBinner (Sec. 4.5): native bin i covers the wavelengths between the midpoints of its
  // neighbouring wavenumbers; weight = overlap with target bin j / native width.
  std::vector<double> li_minus(W), li_plus(W);
  for (int i = 0; i < W; ++i) {
    const double nu_lo = i > 0 ? 0.5 * (wn[i - 1] + wn[i]) : wn[0] - 0.5 * (wn[1] - wn[0]);
    const double nu_hi = i < W - 1 ? 0.5 * (wn[i] + wn[i + 1]) : wn[W - 1] + 0.5 * (wn[W - 1] - wn[W - 2]);
    li_minus[i] = 1e4 / nu_hi;
    li_plus[i] = 1e4 / nu_lo;
  }
  for (int j = 0; j < n_bin; ++j) {
    if (!(lw[j] > 0.0)) return fail(ctx, TR_ERR_ARG, "bin widths must be positive");
    const double bm = lc[j] - 0.5 * lw[j], bp = lc[j] + 0.5 * lw[j];
    double sum = 0.0;
    // wavelength decreases with index: native bins overlapping [bm, bp] are contiguous
    for (int i = 0; i < W; ++i) {
      const double ov = std::min(bp, li_plus[i]) - std::max(bm, li_minus[i]);
      if (ov > 0.0) {
        const double wij = ov / (li_plus[i] - li_minus[i]);
        col.push_back(i); w.push_back(wij); sum += wij;
        lo = std::min(lo, i); hi = std::max(hi, i + 1);
      }
    }
    if (!(sum > 0.0)) return fail(ctx, TR_ERR_ARG, "a bin does not overlap the native grid");
    bin_lo.push_back(col[row_ptr[j]]);
    bin_hi.push_back(col.back() + 1);
    inv_wsum[j] = 1.0 / sum;
    row_ptr[j + 1] = (int)col.size();
  }
  cudaSetDevice(ctx->device);
  const size_t nnz = col.size();
  // transpose (per native wavenumber of the binned range) for the adjoint
  const int n_in = hi > lo ? hi - lo : 0;
  std::vector<int> t_ptr(n_in + 1, 0), t_bin(nnz);
  std::vector<double> t_w(nnz);
  for (size_t e = 0; e < nnz; ++e) t_ptr[col[e] - lo + 1]++;
  for (int k = 0; k < n_in; ++k) t_ptr[k + 1] += t_ptr[k];
  {
    std::vector<int> fill(t_ptr.begin(), t_ptr.end() - 1);
    for (int j = 0; j < n_bin; ++j)
      for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
        const int k = col[e] - lo;
        t_bin[fill[k]] = j;
        t_w[fill[k]] = w[e] * inv_wsum[j];
        fill[k]++;
      }
  }
  const size_t o_row = 0, o_col = align_up(sizeof(int) * (n_bin + 1), 256);
  const size_t o_w = align_up(o_col + sizeof(int) * nnz, 256);
  const size_t o_inv = align_up(o_w + sizeof(double) * nnz, 256);
  const size_t o_tptr = align_up(o_inv + sizeof(double) * n_bin, 256);
  const size_t o_tbin = align_up(o_tptr + sizeof(int) * (n_in + 1), 256);
  const size_t o_tw = align_up(o_tbin + sizeof(int) * nnz, 256);
  const size_t o_lo = align_up(o_tw + sizeof(double) * nnz, 256);
  const size_t total = align_up(o_lo + sizeof(int) * n_bin, 256);
  tr_bins* b = new tr_bins();
  b->device = ctx->device;
  cudaError_t e = cudaMalloc(&b->mem, total);
  if (e != cudaSuccess) { delete b; return cuda_fail(ctx, e, "alloc bins"); }
  char* m = static_cast<char*>(b->mem);
  e = cudaMemcpy(m + o_row, row_ptr.data(), sizeof(int) * (n_bin + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m + o_col, col.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m + o_w, w.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m + o_inv, inv_wsum.data(), sizeof(double) * n_bin, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m + o_tptr, t_ptr.data(), sizeof(int) * (n_in + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m + o_tbin, t_bin.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m + o_tw, t_w.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m + o_lo, bin_lo.data(), sizeof(int) * n_bin, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { tr_free_bins(b); return cuda_fail(ctx, e, "copy bins"); }
  b->dev.n_bin = n_bin; b->dev.i0 = lo; b->dev.i1 = hi;
  b->dev.row_ptr = reinterpret_cast<const int*>(m + o_row);
  b->dev.col = reinterpret_cast<const int*>(m + o_col);
  b->dev.w = reinterpret_cast<const double*>(m + o_w);
  b->dev.inv_wsum = reinterpret_cast<const double*>(m + o_inv);
  b->dev.t_ptr = reinterpret_cast<const int*>(m + o_tptr);
  b->dev.t_bin = reinterpret_cast<const int*>(m + o_tbin);
  b->dev.t_w = reinterpret_cast<const double*>(m + o_tw);
  b->dev.lo = reinterpret_cast<const int*>(m + o_lo);
  b->bin_lo = std::move(bin_lo);
  b->bin_hi = std::move(bin_hi);
  *out = b;
  return TR_OK;
}

// ============================================================================ one atmosphere
extern "C" void tr_free_atmosphere(tr_atm* a) {
  if (!a) return;
  cudaSetDevice(a->device);
  cudaFree(a->mem);
  delete a;
}

extern "C" int tr_build_atmosphere(tr_ctx* ctx, const tr_tables* t, const tr_atm_desc* d,
                                   tr_atm** out, void* stream) {
  if (!ctx || !t || !d || !out) return fail(ctx, TR_ERR_ARG, "null argument");
  *out = nullptr;
  if (d->n_layers < 1 || d->n_layers > TR_MAX_LAYERS) return fail(ctx, TR_ERR_INVALID_MODEL, "n_layers out of range");
  if (d->n_tnodes < 1 || d->n_tnodes > TR_MAX_TNODES || !d->tnode_log10p || !d->tnode_t)
    return fail(ctx, TR_ERR_ARG, "bad temperature nodes");
  if ((t->n_mol > 0 && !d->log10_x) || (t->n_species > t->n_mol && !d->fill_frac))
    return fail(ctx, TR_ERR_ARG, "null chemistry arrays");
  if (!(d->p_max > d->p_min) || !(d->p_min > 0.0)) return fail(ctx, TR_ERR_ARG, "bad pressure range");
  if (!(d->m_p > 0.0) || !(d->r_s > 0.0) || !(d->r_p > 0.0)) return fail(ctx, TR_ERR_INVALID_MODEL, "bad planet or star");
  if (d->t_profile != TR_TPROF_NPOINT && d->t_profile != TR_TPROF_GUILLOT)
    return fail(ctx, TR_ERR_ARG, "unknown temperature profile");
  if (d->gas_mode != TR_GAS_CONSTANT && d->gas_mode != TR_GAS_TWOLAYER)
    return fail(ctx, TR_ERR_ARG, "unknown gas profile");
  const bool guillot = d->t_profile == TR_TPROF_GUILLOT, two = d->gas_mode == TR_GAS_TWOLAYER;
  if (guillot && !d->guillot) return fail(ctx, TR_ERR_ARG, "null Guillot parameters");
  if (two && t->n_mol > 0 && (!d->log10_x_top || !d->log10_p_switch))
    return fail(ctx, TR_ERR_ARG, "null two-layer arrays");
  if (guillot)
    for (int k = 1; k < 4; ++k)
      if (!(d->guillot[k] > 0.0)) return fail(ctx, TR_ERR_INVALID_MODEL, "non-positive Guillot opacity");
  for (int k = 0; k + 1 < d->n_tnodes; ++k)
    if (!(d->tnode_log10p[k] > d->tnode_log10p[k + 1]))
      return fail(ctx, TR_ERR_INVALID_MODEL, "temperature node pressures must be strictly descending");
  // model rejection (Sec. 6), checked on the host so the call can report it synchronously
  double sumx = 0.0;
  for (int m = 0; m < t->n_mol; ++m) {
    if (!std::isfinite(d->log10_x[m])) return fail(ctx, TR_ERR_INVALID_MODEL, "non-finite mixing ratio");
    sumx += std::pow(10.0, d->log10_x[m]);
  }
  if (sumx > 1.0) return fail(ctx, TR_ERR_INVALID_MODEL, "mixing ratios sum above one");
  for (int k = 0; !guillot && k < d->n_tnodes; ++k)
    if (!(d->tnode_t[k] > 0.0) || !std::isfinite(d->tnode_t[k])) return fail(ctx, TR_ERR_INVALID_MODEL, "temperature <= 0");
  const int cloud = (d->cloud_mode != TR_CLOUD_NONE && d->p_cloud_top > 0.0) ? d->cloud_mode : TR_CLOUD_NONE;
  if (cloud < 0 || cloud > 2 || d->gravity_mode < 0 || d->gravity_mode > 1) return fail(ctx, TR_ERR_ARG, "bad mode");
  cudaSetDevice(ctx->device);

  const int NM = d->n_layers;
  const int n_chem = two ? 3 * t->n_mol : t->n_mol;
  const int n_tpar = guillot ? 5 : d->n_tnodes;
  const int n_theta = n_chem + n_tpar + 2;
  const WsLayout wl = ws_layout(1, NM, 0);
  const size_t theta_off = wl.end;
  const size_t total = theta_off + align_up(sizeof(double) * n_theta, 256);
  tr_atm* a = new tr_atm();
  a->device = ctx->device;
  a->n_layers = NM;
  cudaError_t e = cudaMalloc(&a->mem, total);
  if (e != cudaSuccess) { delete a; return cuda_fail(ctx, e, "alloc atmosphere"); }
  a->buf = carve(a->mem, wl, NM);
  a->buf.zoned = two ? 1 : 0;
  // the batch parameter layout (tr_forward_transit_batch) of this one atmosphere
  std::vector<double> th(n_theta);
  for (int m = 0; m < t->n_mol; ++m) th[m] = d->log10_x[m];
  if (two)
    for (int m = 0; m < t->n_mol; ++m) {
      th[t->n_mol + m] = d->log10_x_top[m];
      th[2 * t->n_mol + m] = d->log10_p_switch[m];
    }
  if (guillot) {
    th[n_chem] = d->guillot[0];
    for (int k = 1; k < 4; ++k) th[n_chem + k] = std::log10(d->guillot[k]);
    th[n_chem + 4] = d->guillot[4];
  } else {
    for (int k = 0; k < d->n_tnodes; ++k) th[n_chem + k] = d->tnode_t[k];
  }
  th[n_chem + n_tpar] = d->r_p / kRJup;
  th[n_chem + n_tpar + 1] = cloud != TR_CLOUD_NONE ? std::log10(d->p_cloud_top) : 0.0;
  double* d_theta = reinterpret_cast<double*>(static_cast<char*>(a->mem) + theta_off);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  e = cudaMemcpyAsync(d_theta, th.data(), sizeof(double) * n_theta, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { tr_free_atmosphere(a); return cuda_fail(ctx, e, "copy parameters"); }
  GeomParams gp = geom_params(t, d->n_tnodes, d->tnode_log10p, d->fill_frac, d->p_max, d->p_min,
                              d->m_p, d->r_s, d->p_cloud_bot, d->kappa_cloud, d->gravity_mode,
                              cloud, NM, d->t_profile, d->gas_mode, d->t_int);
  {
    KernelTimer kt(ctx, "k_geometry", s);
    e = launch_geometry(gp, 1, d_theta, n_theta, nullptr, nullptr, a->buf, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // th lives on this host stack frame
  if (e != cudaSuccess) { tr_free_atmosphere(a); return cuda_fail(ctx, e, "geometry kernel"); }
  a->rp2_rs2 = (d->r_p / d->r_s) * (d->r_p / d->r_s);
  *out = a;
  return TR_OK;
}

extern "C" int tr_atm_readback(tr_ctx* ctx, const tr_atm* a, double* z, float* dl, float* aj) {
  if (!ctx || !a) return fail(ctx, TR_ERR_ARG, "null argument");
  cudaSetDevice(ctx->device);
  const int N = a->n_layers;
  cudaError_t e = cudaSuccess;
  if (z) e = cudaMemcpy(z, a->buf.z, sizeof(double) * (N + 1), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && aj) e = cudaMemcpy(aj, a->buf.aj, sizeof(float) * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && dl) {
    const int npad = a->buf.npad;
    std::vector<float> dense((size_t)N * npad);
    e = cudaMemcpy(dense.data(), a->buf.dlt, sizeof(float) * dense.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      for (int j = 0; j < N; ++j)
        for (int l = 0; l < N; ++l)
          dl[(size_t)j * N + l] = l < j ? 0.f : dense[(size_t)l * npad + j];
    }
  }
  return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "readback");
}

int tr::set_error(tr_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int tr::run_forward(tr_ctx* ctx, const tr_tables* t, int max_layers, const ItemBuffers& buf,
                    int B, int wn_begin, int wn_count, double* out, long long stride,
                    int precision, cudaStream_t s, float* kbuf, void* dl16,
                    const ForwardChoice* choice, bool opacity_only, Fork* fork) {
  if (precision != TR_PREC_FP32 && precision != TR_PREC_MIXED)
    return fail(ctx, TR_ERR_ARG, "unknown precision");
  const bool mixed = precision == TR_PREC_MIXED;
  if (!mixed && !t->d_sigma && t->n_mol > 0)
    return fail(ctx, TR_ERR_UNSUPPORTED, "tables were loaded without FP32 storage");
  if (mixed && !t->d_logsig16 && t->n_mol > 0)
    return fail(ctx, TR_ERR_UNSUPPORTED, "tables were loaded without FP16 log10 storage");
  if (mixed && (!dl16 || !kbuf)) return fail(ctx, TR_ERR_ARG, "mixed precision needs its scratch");
  if (buf.zoned && t->interp_mode != TR_INTERP_LINEAR)
    return fail(ctx, TR_ERR_UNSUPPORTED, "two-layer gases need the linear temperature scheme");
  if (opacity_only && (!kbuf || forward_chunk_items(B, max_layers, wn_begin, wn_count) < B))
    return fail(ctx, TR_ERR_ARG, "the opacity stage alone needs a K buffer holding the batch");
  FwdParams p = fwd_params(t, max_layers, buf, wn_begin, wn_count, out, stride, ctx->dev_err);
  cudaError_t e = cudaSuccess;
  // the fused kernel implements the linear temperature scheme only
  // the fused kernel implements constant mixing ratios only (no chemistry zones)
  const bool fits = t->interp_mode == TR_INTERP_LINEAR && !buf.zoned &&
                    fused_forward_fits(t->n_mol, t->n_cia, max_layers, B);
  const bool two_stage_fp32 = kbuf && (!choice || choice->form == kFormTwoStage || !fits);
  if (!mixed && !two_stage_fp32) {                // the fused FP32 kernel (no K buffer)
    if (!fits) return fail(ctx, TR_ERR_UNSUPPORTED, "this model needs a K buffer (layer count, "
                                                  "temperature scheme or two-layer gases)");
    e = fork_start(ctx, fork, s, false);        // the fused kernel reads the path lengths
    if (e != cudaSuccess) return cuda_fail(ctx, e, "path-length kernel");
    KernelTimer kt(ctx, "k_forward_tma", s);
    e = launch_forward_fused(p, &t->tm_sig32_f, &t->tm_cia_f, B, choice ? choice->stages : 0,
                             nullptr, s);
    return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "forward kernel");
  }
  if (mixed) {
    p.logsig16 = t->d_logsig16;
    for (int m = 0; m < t->n_mol; ++m) p.logsig_off[m] = t->logsig_offset[m];
  }
  // the FP32 contraction: the tensor-core kernel where the layer count fits it and the
  // path-length tile scratch is there, else the FFMA kernel
  int kind = contract_kind(choice ? choice->contract_per_sm : kContractAuto, max_layers);
  if (kind == kContractTC && !dl16) kind = kContractFfma8;
  // the path-length tiles of the tensor-core contractions (after the path lengths)
  auto tiles_kernel = [&](cudaStream_t st) -> cudaError_t {
    if (opacity_only) return cudaSuccess;
    if (mixed) {
      KernelTimer kt(ctx, "k_dl_bf16", st);
      return launch_dl_bf16(buf, B, max_layers, dl16, st);
    }
    if (kind != kContractTC) return cudaSuccess;
    KernelTimer kt(ctx, "k_dl_tf32", st);
    return launch_dl_tf32(buf, B, max_layers, dl16, st);
  };
  // with a pending branch they follow the path lengths there, after the first opacity launch
  const bool branch = fork && fork->pending && !opacity_only;
  if (!branch) {
    e = fork_start(ctx, fork, s, false);
    if (e == cudaSuccess) e = tiles_kernel(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "path-length kernels");
  }
  // two stages per chunk of items: opacity -> K in kbuf -> contraction + depth
  const int chunk = forward_chunk_items(B, max_layers, wn_begin, wn_count);
  for (int b0 = 0; b0 < B && e == cudaSuccess; b0 += chunk) {
    const int bc = std::min(chunk, B - b0);
    p.b_off = b0;
    {
      KernelTimer kt(ctx, mixed ? "k_opacity_fp16" : "k_opacity_fp32", s);
      e = launch_opacity(p, mixed ? &t->tm_sig16 : &t->tm_sig32, &t->tm_cia, bc, kbuf,
                         choice ? choice->per_sm : 0, s);
    }
    if (e != cudaSuccess || opacity_only) break;
    if (branch && b0 == 0) {
      // the path lengths and their tiles beside the opacity kernel, then the join
      e = fork_start(ctx, fork, s, true);
      if (e == cudaSuccess) e = tiles_kernel(fork->aux);
      join_fork(ctx, fork, s);
      if (e != cudaSuccess) break;
    }
    KernelTimer kt(ctx, mixed ? "k_contract_umma" : kind == kContractTC ? "k_contract_tc"
                                                                        : "k_contract_fp32", s);
    e = mixed ? launch_contract_umma(p, bc, kbuf, dl16, s)
              : launch_contract_fp32(p, bc, kbuf, kind, dl16, s);
  }
  return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "forward kernels");
}

int tr::run_bin(tr_ctx* ctx, const tr_bins* bins, int B, const double* depth,
                   long long stride, int base, double* binned, cudaStream_t s) {
  KernelTimer kt(ctx, "k_bin", s);
  const cudaError_t e = launch_bin(bins->dev, B, depth, stride, base, binned, s);
  return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "bin kernel");
}

extern "C" int tr_forward_transit(tr_ctx* ctx, const tr_tables* t, const tr_atm* a,
                                  const tr_bins* bins, double* d_native, double* d_binned,
                                  int precision, void* stream) {
  if (!ctx || !t || !a) return fail(ctx, TR_ERR_ARG, "null argument");
  if (!d_native && !d_binned) return fail(ctx, TR_ERR_ARG, "no output requested");
  if (d_binned && !bins) return fail(ctx, TR_ERR_ARG, "binned output needs bins");
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // context scratch: [binned-region depths][K buffer][BF16 path-length tiles (mixed)]
  const int wb = d_native ? 0 : bins->dev.i0;
  const int wc = d_native ? t->n_wn : bins->dev.i1 - bins->dev.i0;
  const size_t off_k = align_up(sizeof(double) * (size_t)(d_native ? 0 : wc), 256);
  const size_t off_dl = off_k + align_up(forward_kbuf_bytes(1, a->n_layers, wb, wc), 256);
  const size_t dlb = dl_tile_bytes(1, a->n_layers, precision);
  const size_t total = off_dl + dlb;
  int rc = ensure_scratch(ctx, total);
  if (rc != TR_OK) return rc;
  char* sc = static_cast<char*>(ctx->scratch);
  float* kbuf = reinterpret_cast<float*>(sc + off_k);
  void* dl16 = dlb > 0 ? sc + off_dl : nullptr;
  if (d_native) {
    rc = run_forward(ctx, t, a->n_layers, a->buf, 1, 0, t->n_wn, d_native, t->n_wn, precision,
                     s, kbuf, dl16);
    if (rc != TR_OK || !d_binned) return rc;
    return run_bin(ctx, bins, 1, d_native, t->n_wn, 0, d_binned, s);
  }
  double* tmp = reinterpret_cast<double*>(sc);
  rc = run_forward(ctx, t, a->n_layers, a->buf, 1, wb, wc, tmp, wc, precision, s, kbuf, dl16);
  if (rc != TR_OK) return rc;
  return run_bin(ctx, bins, 1, tmp, wc, wb, d_binned, s);
}

// ============================================================================ batches
extern "C" size_t tr_batch_workspace_size(const tr_tables* t, const tr_batch_desc* d,
                                          const tr_bins* bins, int B, int with_adjoint) {
  if (!t || !d || B < 0 || d->max_layers < 1) return 0;
  const int n_in = bins ? bins->dev.i1 - bins->dev.i0 : 0;
  size_t bytes = forward_workspace_bytes(B, d->max_layers, n_in);
  const int wb = bins ? bins->dev.i0 : 0, wc = bins ? n_in : t->n_wn;
  bytes += align_up(forward_kbuf_bytes(B, d->max_layers, wb, wc), 256);
  // path-length tiles of whichever precision the tables serve that needs more
  bytes += align_up(std::max(t->d_logsig16 ? dl_tile_bytes(B, d->max_layers, TR_PREC_MIXED) : 0,
                             t->d_sigma ? dl_tile_bytes(B, d->max_layers, TR_PREC_FP32) : 0),
                    256);
  if (with_adjoint) bytes += adjoint_extra_bytes(t, d, bins, B);
  return bytes;
}

int tr::prepare_batch(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d, int n_in,
                      size_t need, int B, const double* d_theta, const int32_t* d_nlayers,
                      int32_t* d_status, void* ws, size_t ws_bytes, cudaStream_t s,
                      ItemBuffers* buf_out, double** depth_out, char** extra_out, Fork* fork) {
  int rc = check_batch_desc(ctx, t, d);
  if (rc != TR_OK) return rc;
  const WsLayout wl = ws_layout(B, d->max_layers, n_in);
  if (!ws) {
    rc = ensure_scratch(ctx, need);
    if (rc != TR_OK) return rc;
    ws = ctx->scratch;
  } else if (ws_bytes < need) {
    return fail(ctx, TR_ERR_OOM, "workspace smaller than tr_batch_workspace_size()");
  }
  *buf_out = carve(ws, wl, d->max_layers);
  buf_out->zoned = d->gas_mode == TR_GAS_TWOLAYER ? 1 : 0;
  *depth_out = reinterpret_cast<double*>(static_cast<char*>(ws) + wl.depth);
  if (extra_out) *extra_out = static_cast<char*>(ws) + wl.end;
  const GeomParams gp = batch_geom_params(t, d);
  const int n_theta = batch_n_theta(t, d);
  cudaError_t e;
  {
    KernelTimer kt(ctx, "k_profile", s);
    e = launch_profile(gp, B, d_theta, n_theta, d_nlayers, d_status, *buf_out, s);
  }
  if (e == cudaSuccess && fork) {
    // the path lengths go to the branch that run_forward opens beside the opacity kernel
    e = cudaEventRecord(ctx->ev_fork, s);
    if (e == cudaSuccess) {
      fork->pending = true;
      fork->gp = gp;
      fork->B = B;
      fork->buf = *buf_out;
    }
  } else if (e == cudaSuccess) {
    {
      KernelTimer kt(ctx, "k_altitude", s);
      e = launch_altitude(gp, B, *buf_out, s);
    }
    if (e == cudaSuccess) {
      KernelTimer kt(ctx, "k_pathlen", s);
      e = launch_pathlen(gp, B, *buf_out, s);
    }
  }
  return e == cudaSuccess ? TR_OK : cuda_fail(ctx, e, "geometry kernel");
}


size_t tr::dl_tile_bytes(int B, int max_layers, int precision) {
  if (precision == TR_PREC_MIXED) return mixed_dl_bytes(B, max_layers);
  return tc_dl_bytes(B, max_layers);
}

// Workspace bytes of a batched forward call (the same as tr_forward_transit_batch computes).
size_t tr::forward_batch_need(const tr_tables* t, const tr_batch_desc* d, int B,
                              const tr_bins* bins, bool native, int precision) {
  const int n_in = native ? 0 : bins->dev.i1 - bins->dev.i0;
  const int wb = native ? 0 : bins->dev.i0, wc = native ? t->n_wn : n_in;
  const size_t fwd = forward_workspace_bytes(B, d->max_layers, n_in);
  const size_t kb = align_up(forward_kbuf_bytes(B, d->max_layers, wb, wc), 256);
  return fwd + kb + align_up(dl_tile_bytes(B, d->max_layers, precision), 256);
}

// Key of a batch shape for the autotuner's results.
std::string tr::batch_shape_key(const tr_tables* t, const tr_batch_desc* d, int B,
                                const tr_bins* bins, bool native, int precision) {
  char k[160];
  std::snprintf(k, sizeof k, "%p/%d/%d/%d/%d/%d/%d", static_cast<const void*>(t), B,
                d->max_layers, precision, native ? -1 : bins->dev.i0,
                native ? t->n_wn : bins->dev.i1, native ? 1 : 0);
  return k;
}

int tr::forward_batch_impl(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d, int B,
                           const double* d_theta, const int32_t* d_nlayers, const tr_bins* bins,
                           double* d_native, double* d_binned, int32_t* d_status, int precision,
                           void* ws, size_t ws_bytes, cudaStream_t s,
                           const ForwardChoice* choice) {
  const int n_in = d_native ? 0 : bins->dev.i1 - bins->dev.i0;
  const int wb = d_native ? 0 : bins->dev.i0, wc = d_native ? t->n_wn : n_in;
  const size_t kb = align_up(forward_kbuf_bytes(B, d->max_layers, wb, wc), 256);
  const size_t need = forward_batch_need(t, d, B, bins, d_native != nullptr, precision);
  ItemBuffers buf; double* depth = nullptr; char* extra = nullptr;
  // the path-length kernels on a second branch beside the opacity kernel
  Fork fk;
  Fork* fork = fork_ready(ctx, &fk) ? &fk : nullptr;
  int rc = prepare_batch(ctx, t, d, n_in, need, B, d_theta, d_nlayers, d_status, ws, ws_bytes,
                         s, &buf, &depth, &extra, fork);
  if (rc != TR_OK) { join_fork(ctx, fork, s); return rc; }
  float* kbuf = reinterpret_cast<float*>(extra);
  void* dl16 = dl_tile_bytes(B, d->max_layers, precision) > 0 ? extra + kb : nullptr;
  if (d_native) {
    rc = run_forward(ctx, t, d->max_layers, buf, B, 0, t->n_wn, d_native, t->n_wn, precision, s,
                     kbuf, dl16, choice, false, fork);
    join_fork(ctx, fork, s);
    if (rc != TR_OK || !d_binned) return rc;
    return run_bin(ctx, bins, B, d_native, t->n_wn, 0, d_binned, s);
  }
  rc = run_forward(ctx, t, d->max_layers, buf, B, bins->dev.i0, n_in, depth, n_in, precision, s,
                   kbuf, dl16, choice, false, fork);
  join_fork(ctx, fork, s);
  if (rc != TR_OK) return rc;
  return run_bin(ctx, bins, B, depth, n_in, bins->dev.i0, d_binned, s);
}

int tr::check_forward_batch_args(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d, int B,
                                 const double* d_theta, const tr_bins* bins,
                                 const double* d_native, const double* d_binned) {
  if (!ctx || !t || !d_theta || B < 0) return fail(ctx, TR_ERR_ARG, "null argument");
  if (B > TR_MAX_BATCH) return fail(ctx, TR_ERR_ARG, "batch larger than TR_MAX_BATCH");
  if (!d_native && !d_binned) return fail(ctx, TR_ERR_ARG, "no output requested");
  if (d_binned && !bins) return fail(ctx, TR_ERR_ARG, "binned output needs bins");
  if (!d) return fail(ctx, TR_ERR_ARG, "null batch descriptor");
  return TR_OK;
}

extern "C" int tr_forward_transit_batch(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d,
                                        int B, const double* d_theta, const int32_t* d_nlayers,
                                        const tr_bins* bins, double* d_native, double* d_binned,
                                        int32_t* d_status, int precision, void* ws,
                                        size_t ws_bytes, void* stream) {
  int rc = check_forward_batch_args(ctx, t, d, B, d_theta, bins, d_native, d_binned);
  if (rc != TR_OK) return rc;
  if (B == 0) return TR_OK;
  cudaSetDevice(ctx->device);
  // a configuration the autotuner found for this shape on this context, if any
  const auto it = ctx->tuned.find(batch_shape_key(t, d, B, bins, d_native != nullptr, precision));
  const ForwardChoice* choice = it != ctx->tuned.end() ? &it->second : nullptr;
  return forward_batch_impl(ctx, t, d, B, d_theta, d_nlayers, bins, d_native, d_binned, d_status,
                            precision, ws, ws_bytes, static_cast<cudaStream_t>(stream), choice);
}
