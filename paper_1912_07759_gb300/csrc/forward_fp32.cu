// forward_fp32.cu -- FP32 forward model: opacity K[layer, wn] (Sec. 5 linear P/T
// interpolation, weighted by rho X and fused with Rayleigh, CIA and the grey cloud as in
// Sec. 8.1), slant optical depth tau[ray, wn] = sum_{l >= j} DL[j][l] K[l][wn] (Sec. 4,
// eqs. tot_opt_dpth, opt_dpth, cia_opt_dpth) and transit depth
// D = (R_p/R_s)^2 + sum_j a_j (1 - exp(-tau_j)) (Sec. 4, eqs. Delta_lambda, a_lambda).
//
// Two forms share the same device functions:
//  * fused (k_forward_fp32): one CTA = one atmosphere x 128 wavenumbers; K is built in shared
//    memory and never leaves it.  Used when no K buffer is available (the entry point that
//    allocates nothing).
//  * two-stage (k_opacity + k_contract_fp32), used whenever the caller's workspace (or the
//    context's scratch) holds a K buffer: items are processed in chunks whose K fits a 2 GiB
//    budget; k_opacity streams K (FP32) to HBM once, k_contract reads it back with the path
//    lengths and annulus weights (one bulk copy).  The mixed path shares k_opacity (FP16 log
//    tables) and contracts on the tensor cores (mixed.cu).
//
// The contraction: a warp owns 8-ray register tiles (j0..j0+7), a lane owns 4 wavenumbers;
// shells below j0 are skipped (the triangle); tiles are dealt to warps in snake order; the
// epilogue folds a_j (1 - e^-tau) per lane and the 8 warps' partial sums are added in FP64
// in a fixed order (deterministic), plus (R_p/R_s)^2 in FP64.
#include <algorithm>
#include <cuda_fp16.h>
#include "tma.h"
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kTW = 128;         // wavenumbers per CTA
constexpr int kThreads = 256;    // 8 warps
constexpr int kWarps = kThreads / 32;
constexpr int kRT = 8;           // rays per register tile

__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ void fma4(float4& k, float c, const float4& v) {
  k.x = fmaf(c, v.x, k.x); k.y = fmaf(c, v.y, k.y);
  k.z = fmaf(c, v.z, k.z); k.w = fmaf(c, v.w, k.w);
}

// Combined Rayleigh cross-section sum_s X_s sigma_R,s at 4 wavenumbers (scaled per species).
// Fully unrolled with predicated loads, so the loads of all species are in flight together.
__device__ __forceinline__ float4 rayleigh4(const FwdParams& p, int b, int w4) {
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!p.ray) return r;
  const float4* rc4 = reinterpret_cast<const float4*>(p.buf.rayc + (size_t)b * TR_MAX_SPECIES);
  static_assert(TR_MAX_SPECIES % 4 == 0, "species coefficients load as float4");
  float c[TR_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < TR_MAX_SPECIES / 4; ++k) {
    const float4 v = __ldg(rc4 + k);
    c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
  }
#pragma unroll
  for (int s = 0; s < TR_MAX_SPECIES; ++s)
    if (s < p.n_species && c[s] != 0.f) fma4(r, c[s], ldg4(p.ray + (size_t)s * p.wn_pad + w4));
  return r;
}

// K of one layer at 4 wavenumbers w4..w4+3 (w4 a multiple of 4 below wn_pad).
template <int MAXMOL>
__device__ __forceinline__ float4 opacity4(const FwdParams& p, const LayerDesc* __restrict__ d,
                                           const float4& ray, int w4) {
  const int ip = d->ip, it = d->it;
  const float rho = d->rho, kc = d->k_cloud;
  float4 k = make_float4(kc + rho * ray.x, kc + rho * ray.y, kc + rho * ray.z, kc + rho * ray.w);
  const size_t slab_t = (size_t)p.wn_pad;
  const size_t slab_p = (size_t)p.n_t * p.wn_pad;
  const float* base0 = p.sigma + ((size_t)ip * p.n_t + it) * p.wn_pad + w4;
#pragma unroll
  for (int m = 0; m < MAXMOL; ++m) {
    if (m < p.n_mol) {
      const float* base = base0 + (size_t)m * p.n_p * slab_p;
      const float4 s00 = ldg4(base), s01 = ldg4(base + slab_t);
      const float4 s10 = ldg4(base + slab_p), s11 = ldg4(base + slab_p + slab_t);
      const float4 c = *reinterpret_cast<const float4*>(d->cm[m]);
      fma4(k, c.x, s00); fma4(k, c.y, s01); fma4(k, c.z, s10); fma4(k, c.w, s11);
    }
  }
  for (int q = 0; q < p.n_cia; ++q) {
    const float* base = p.cia + ((size_t)q * p.n_t_cia + d->itc) * p.wn_pad + w4;
    const float4 c0 = ldg4(base), c1 = ldg4(base + p.wn_pad);
    fma4(k, d->cc[q][0], c0); fma4(k, d->cc[q][1], c1);
  }
  return k;
}

// Bulk copies of one atmosphere's path lengths (dense rows l = 0..N-1 of npad floats, zero
// for j > l) and annulus weights into shared memory; the caller has armed `bar` for the
// bytes returned by geometry_bytes().  Issued by one thread.
__device__ __forceinline__ uint32_t geometry_bytes(int N, int npad) {
  return (uint32_t)(sizeof(float) * ((size_t)N * npad + npad));
}
__device__ __forceinline__ void copy_geometry(const FwdParams& p, int b, int N, float* DLT,
                                              float* a_s, uint64_t* bar) {
  const int npad = p.buf.npad;
  bulk_g2s(DLT, p.buf.dlt + (size_t)b * p.max_layers * npad,
           (uint32_t)(sizeof(float) * (size_t)N * npad), bar);
  bulk_g2s(a_s, p.buf.aj + (size_t)b * npad, (uint32_t)(sizeof(float) * npad), bar);
}

// tau = DL K over 8-ray tiles, epilogue sum_j a_j (1 - e^-tau), FP64 cross-warp sum, output.
// DLT rows have npad floats (the row stride); ray tiles cover rays 0..ceil(N/8)*8-1.
__device__ __forceinline__ void contract_store(const FwdParams& p, int b, int N, int npad,
                                               const float* Kt, const float* DLT,
                                               const float* a_s, float* red, int w_first,
                                               double rp2_rs2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_rt = (N + kRT - 1) / kRT;
  float part[4] = {0.f, 0.f, 0.f, 0.f};
  for (int round = 0;; ++round) {
    // snake order: tiles 0..7 -> warps 0..7, 8..15 -> warps 7..0, ...
    const int pos = (round & 1) ? (kWarps - 1 - warp) : warp;
    const int tile = round * kWarps + pos;
    if (tile >= n_rt) break;
    const int j0 = tile * kRT;
    float acc[kRT][4];
#pragma unroll
    for (int r = 0; r < kRT; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
    for (int l = j0; l < N; ++l) {
      const float4 kv = *reinterpret_cast<const float4*>(Kt + (size_t)l * kTW + 4 * lane);
      const float4 d0 = *reinterpret_cast<const float4*>(DLT + (size_t)l * npad + j0);
      const float4 d1 = *reinterpret_cast<const float4*>(DLT + (size_t)l * npad + j0 + 4);
      const float dv[kRT] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
      for (int r = 0; r < kRT; ++r) {
        acc[r][0] = fmaf(dv[r], kv.x, acc[r][0]);
        acc[r][1] = fmaf(dv[r], kv.y, acc[r][1]);
        acc[r][2] = fmaf(dv[r], kv.z, acc[r][2]);
        acc[r][3] = fmaf(dv[r], kv.w, acc[r][3]);
      }
    }
    // 1 - e^-tau with the hardware exponential: its absolute error (a few 1e-7) times the
    // annulus weights (sum ~ 1e-3) stays below 1e-9 in depth, far inside 0.1 ppm
#pragma unroll
    for (int r = 0; r < kRT; ++r) {
      const float a = a_s[j0 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) part[c] = fmaf(a, 1.f - __expf(-acc[r][c]), part[c]);
    }
  }
  __syncthreads();                                        // all reads of Kt done
  *reinterpret_cast<float4*>(red + warp * kTW + 4 * lane) =
      make_float4(part[0], part[1], part[2], part[3]);
  __syncthreads();
  if (threadIdx.x < kTW) {
    const int w = w_first + threadIdx.x;
    if (w >= p.wn_begin && w < p.wn_begin + p.wn_count) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < kWarps; ++k) s += (double)red[k * kTW + threadIdx.x];
      p.out[(long long)b * p.out_stride + (w - p.wn_begin)] = rp2_rs2 + s;
    }
  }
}

__device__ __forceinline__ void zero_output(const FwdParams& p, int b, int w_first) {
  for (int i = threadIdx.x; i < kTW; i += kThreads) {
    const int w = w_first + i;
    if (w >= p.wn_begin && w < p.wn_begin + p.wn_count)
      p.out[(long long)b * p.out_stride + (w - p.wn_begin)] = 0.0;
  }
}

struct SmemPlan {
  int kt_rows, npad_max;
  __host__ __device__ SmemPlan(int max_layers)
      : kt_rows(max_layers > kWarps ? max_layers : kWarps), npad_max(pad8(max_layers)) {}
  __host__ __device__ size_t floats() const {
    return (size_t)kt_rows * kTW + (size_t)npad_max * npad_max + npad_max;
  }
};

// Arms the CTA's mbarrier (thread 0) and makes it visible before any copy is issued.
__device__ __forceinline__ void init_barrier(uint64_t* bar) {
  if (threadIdx.x == 0) { mbar_init(bar, 1); mbar_fence_init(); }
  __syncthreads();
}

template <int MAXMOL>
__global__ void __launch_bounds__(kThreads, 2)
k_forward_fp32(FwdParams p) {
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) uint64_t bar;
  const int b = blockIdx.y;
  const ItemGeom ig = p.buf.items[b];
  const int N = ig.n_layers;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w_first = (p.wn_begin & ~3) + blockIdx.x * kTW;   // 16-byte aligned start
  const SmemPlan sp(p.max_layers);
  float* Kt = smem;                                   // [kt_rows][kTW]
  float* DLT = Kt + (size_t)sp.kt_rows * kTW;         // [N][npad]
  float* a_s = DLT + (size_t)sp.npad_max * sp.npad_max;
  if (N == 0) { zero_output(p, b, w_first); return; }
  init_barrier(&bar);
  if (threadIdx.x == 0) {                             // path lengths stream in meanwhile
    mbar_arrive_expect_tx(&bar, geometry_bytes(N, sp.npad_max));
    copy_geometry(p, b, N, DLT, a_s, &bar);
  }
  // opacity of this tile: warp w builds layers w, w+8, ...
  const int w4 = w_first + 4 * lane;
  const bool in_row = w4 < p.wn_pad;
  const float4 ray = in_row ? rayleigh4(p, b, w4) : make_float4(0.f, 0.f, 0.f, 0.f);
  const LayerDesc* LD = p.buf.layers + (size_t)b * p.max_layers;
  for (int l = warp; l < N; l += kWarps) {
    const float4 k = in_row ? opacity4<MAXMOL>(p, LD + l, ray, w4)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(Kt + (size_t)l * kTW + 4 * lane) = k;
  }
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, p.dev_err, TR_DEVERR_TIMEOUT));
  if (!ok) { mbar_wait_bounded(&bar, 0, nullptr, 0); return; }   // copies may still land
  contract_store(p, b, N, sp.npad_max, Kt, DLT, a_s, Kt, w_first, ig.rp2_rs2);
}

// Streaming opacity (first stage of the two-stage form).  One CTA = one atmosphere x 64
// wavenumbers; warp w owns a run of consecutive layers [w G, (w+1) G), lane = 2 wavenumbers.
// Consecutive layers mostly share the same (P, T) bracket cell, so a warp keeps the four
// corner rows of every molecule (and the two CIA rows) of its current cell in registers and
// reloads them only when the cell changes: on the full-size model each warp makes about 4
// rounds of loads instead of 13.  With FP16 tables the rows are decoded (10^(h + c_m)) only
// on those reloads.  K is streamed to HBM once.  Instantiated per molecule / CIA capacity so
// that the cached rows stay in registers.
constexpr int kTO = 64;                          // wavenumbers per opacity CTA
constexpr float kLog2Of10 = 3.32192809488736234787f;

__device__ __forceinline__ float2 ldg2(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}
__device__ __forceinline__ void fma2(float2& k, float c, const float2& v) {
  k.x = fmaf(c, v.x, k.x); k.y = fmaf(c, v.y, k.y);
}
// 2^x by the hardware approximation (relative error ~2e-7, far below the FP16 storage step)
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// two FP16 log10 sigma values -> sigma = 10^(h + c) = 2^((h + c) log2 10)
__device__ __forceinline__ float2 ld_dec2(const __half* p, float c) {
  const float2 h = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
  return make_float2(ex2_fast((h.x + c) * kLog2Of10), ex2_fast((h.y + c) * kLog2Of10));
}

template <int MAXMOL, int MAXCIA, bool F16>
__global__ void __launch_bounds__(kThreads, 2)
k_opacity(FwdParams p, float* __restrict__ kbuf, long long kcols) {
  // items vary fastest across the grid, so the CTAs resident together work on the same
  // wavenumber tile and share its table rows through L2
  const int bc = blockIdx.x;                        // item within the chunk
  const int b = p.b_off + bc;
  const int N = p.buf.items[b].n_layers;
  if (N == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = (N + kWarps - 1) / kWarps;
  const int l_begin = warp * G, l_end = min(N, l_begin + G);
  const int col = blockIdx.y * kTO + 2 * lane;
  const int w2 = (p.wn_begin & ~3) + col;
  float* dst = kbuf + (size_t)bc * p.max_layers * kcols + col;
  const LayerDesc* LD = p.buf.layers + (size_t)b * p.max_layers;
  if (w2 >= p.wn_pad) {                              // beyond the table: columns never output
    for (int l = l_begin; l < l_end; ++l)
      __stcs(reinterpret_cast<float2*>(dst + (size_t)l * kcols), make_float2(0.f, 0.f));
    return;
  }
  float2 ray = make_float2(0.f, 0.f);
  if (p.ray) {
    const float* rc = p.buf.rayc + (size_t)b * TR_MAX_SPECIES;
    for (int s = 0; s < p.n_species; ++s) {
      const float c = rc[s];
      if (c != 0.f) fma2(ray, c, ldg2(p.ray + (size_t)s * p.wn_pad + w2));
    }
  }
  const size_t slab_t = (size_t)p.wn_pad, slab_p = (size_t)p.n_t * p.wn_pad;
  float2 v[MAXMOL][4];                               // corner rows of the current cell
  float2 cv[MAXCIA][2];                              // CIA rows of the current CIA bracket
  int cell = -1, ccell = -1;
  for (int l = l_begin; l < l_end; ++l) {
    const LayerDesc* d = LD + l;
    const int c = d->ip * p.n_t + d->it;
    if (c != cell) {                                 // uniform across the warp
      cell = c;
      const size_t off0 = (size_t)c * p.wn_pad + w2;
#pragma unroll
      for (int m = 0; m < MAXMOL; ++m) {
        if (m < p.n_mol) {
          const size_t om = off0 + (size_t)m * p.n_p * slab_p;
          if (F16) {
            const __half* bm = reinterpret_cast<const __half*>(p.logsig16) + om;
            const float cm = p.logsig_off[m];
            v[m][0] = ld_dec2(bm, cm); v[m][1] = ld_dec2(bm + slab_t, cm);
            v[m][2] = ld_dec2(bm + slab_p, cm); v[m][3] = ld_dec2(bm + slab_p + slab_t, cm);
          } else {
            const float* bm = p.sigma + om;
            v[m][0] = ldg2(bm); v[m][1] = ldg2(bm + slab_t);
            v[m][2] = ldg2(bm + slab_p); v[m][3] = ldg2(bm + slab_p + slab_t);
          }
        }
      }
    }
    if (p.n_cia > 0 && d->itc != ccell) {
      ccell = d->itc;
#pragma unroll
      for (int q = 0; q < MAXCIA; ++q) {
        if (q < p.n_cia) {
          const float* bq = p.cia + ((size_t)q * p.n_t_cia + ccell) * p.wn_pad + w2;
          cv[q][0] = ldg2(bq); cv[q][1] = ldg2(bq + p.wn_pad);
        }
      }
    }
    const float rho = d->rho, kc = d->k_cloud;
    float2 k = make_float2(fmaf(rho, ray.x, kc), fmaf(rho, ray.y, kc));
#pragma unroll
    for (int m = 0; m < MAXMOL; ++m) {
      if (m < p.n_mol) {
        const float4 cw = *reinterpret_cast<const float4*>(d->cm[m]);
        fma2(k, cw.x, v[m][0]); fma2(k, cw.y, v[m][1]); fma2(k, cw.z, v[m][2]); fma2(k, cw.w, v[m][3]);
      }
    }
#pragma unroll
    for (int q = 0; q < MAXCIA; ++q) {
      if (q < p.n_cia) { fma2(k, d->cc[q][0], cv[q][0]); fma2(k, d->cc[q][1], cv[q][1]); }
    }
    __stcs(reinterpret_cast<float2*>(dst + (size_t)l * kcols), k);
  }
}

template <int MAXMOL, int MAXCIA, bool F16>
cudaError_t launch_opacity_t(const FwdParams& p, int Bc, float* kbuf, long long kcols,
                             cudaStream_t s) {
  k_opacity<MAXMOL, MAXCIA, F16><<<dim3(Bc, (unsigned)(kcols / kTO)), kThreads, 0, s>>>(p, kbuf, kcols);
  return cudaGetLastError();
}

template <bool F16>
cudaError_t launch_opacity_p(const FwdParams& p, int Bc, float* kbuf, long long kcols,
                             cudaStream_t s) {
  static_assert(TR_MAX_MOL == 8 && TR_MAX_CIA == 4, "opacity instantiations cover the limits");
  if (p.n_cia <= 2) {
    if (p.n_mol <= 2) return launch_opacity_t<2, 2, F16>(p, Bc, kbuf, kcols, s);
    if (p.n_mol <= 5) return launch_opacity_t<5, 2, F16>(p, Bc, kbuf, kcols, s);
    return launch_opacity_t<8, 2, F16>(p, Bc, kbuf, kcols, s);
  }
  if (p.n_mol <= 2) return launch_opacity_t<2, 4, F16>(p, Bc, kbuf, kcols, s);
  if (p.n_mol <= 5) return launch_opacity_t<5, 4, F16>(p, Bc, kbuf, kcols, s);
  return launch_opacity_t<8, 4, F16>(p, Bc, kbuf, kcols, s);
}

// Contraction + depth reading K from kbuf: the path lengths and annulus weights arrive by one
// bulk copy on an mbarrier while the CTA's warps load the K tile with coalesced 16-byte
// loads (many small rows: plain loads beat per-row bulk copies here), then the contraction.
__global__ void __launch_bounds__(kThreads, 2)
k_contract_fp32(FwdParams p, const float* __restrict__ kbuf, long long kcols) {
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) uint64_t bar;
  const int b = p.b_off + blockIdx.y;
  const ItemGeom ig = p.buf.items[b];
  const int N = ig.n_layers;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w_first = (p.wn_begin & ~3) + blockIdx.x * kTW;
  const SmemPlan sp(p.max_layers);
  float* Kt = smem;
  float* DLT = Kt + (size_t)sp.kt_rows * kTW;
  float* a_s = DLT + (size_t)sp.npad_max * sp.npad_max;
  if (N == 0) { zero_output(p, b, w_first); return; }
  init_barrier(&bar);
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, geometry_bytes(N, sp.npad_max));
    copy_geometry(p, b, N, DLT, a_s, &bar);
  }
  const float* src = kbuf + (size_t)blockIdx.y * p.max_layers * kcols + (size_t)blockIdx.x * kTW + 4 * lane;
#pragma unroll 4
  for (int l = warp; l < N; l += kWarps)
    *reinterpret_cast<float4*>(Kt + (size_t)l * kTW + 4 * lane) =
        __ldcs(reinterpret_cast<const float4*>(src + (size_t)l * kcols));
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, p.dev_err, TR_DEVERR_TIMEOUT));
  if (!ok) { mbar_wait_bounded(&bar, 0, nullptr, 0); return; }   // copies may still land
  contract_store(p, b, N, sp.npad_max, Kt, DLT, a_s, Kt, w_first, ig.rp2_rs2);
}

int n_tiles_of(const FwdParams& p) {
  const int w_first = p.wn_begin & ~3;
  return (p.wn_begin + p.wn_count - w_first + kTW - 1) / kTW;
}

}  // namespace

constexpr size_t kKbufBudget = 2ull << 30;       // bytes of K per chunk of items

int forward_chunk_items(int B, int max_layers, int wn_begin, int wn_count) {
  const int w_first = wn_begin & ~3;
  const size_t cols = (size_t)((wn_begin + wn_count - w_first + kTW - 1) / kTW) * kTW;
  const size_t per = sizeof(float) * (size_t)max_layers * cols;
  const size_t n = std::max<size_t>(1, kKbufBudget / per);
  return (int)std::min<size_t>((size_t)std::max(B, 1), n);
}

size_t forward_kbuf_bytes(int B, int max_layers, int wn_begin, int wn_count) {
  const int w_first = wn_begin & ~3;
  const long long cols = (long long)((wn_begin + wn_count - w_first + kTW - 1) / kTW) * kTW;
  return sizeof(float) * (size_t)forward_chunk_items(B, max_layers, wn_begin, wn_count) *
         max_layers * cols;
}

cudaError_t launch_forward_fp32(const FwdParams& p, int B, cudaStream_t s) {
  if (B <= 0 || p.wn_count <= 0) return cudaSuccess;
  const size_t smem = sizeof(float) * SmemPlan(p.max_layers).floats();
  static_assert(TR_MAX_MOL == 8, "kernels instantiated for 8 molecules");
  auto kern = k_forward_fp32<TR_MAX_MOL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(n_tiles_of(p), B), kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_opacity(const FwdParams& p, int Bc, float* kbuf, cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  const long long kcols = (long long)n_tiles_of(p) * kTW;
  return p.logsig16 ? launch_opacity_p<true>(p, Bc, kbuf, kcols, s)
                    : launch_opacity_p<false>(p, Bc, kbuf, kcols, s);
}

cudaError_t launch_contract_fp32(const FwdParams& p, int Bc, const float* kbuf, cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  const int tiles = n_tiles_of(p);
  const size_t smem = sizeof(float) * SmemPlan(p.max_layers).floats();
  cudaError_t e = cudaFuncSetAttribute(k_contract_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_fp32<<<dim3(tiles, Bc), kThreads, smem, s>>>(p, kbuf, (long long)tiles * kTW);
  return cudaGetLastError();
}

}  // namespace tr
