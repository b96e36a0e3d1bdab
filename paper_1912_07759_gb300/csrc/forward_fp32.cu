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
//    budget; k_opacity stages the bracketing table rows in shared memory by TMA tensor-map
//    loads and streams K (FP32) to HBM once, k_contract reads it back with the path lengths
//    and annulus weights (one bulk copy).  The mixed path shares k_opacity (FP16 log tables)
//    and contracts on the tensor cores (mixed.cu).
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
  const int w_first = wn_first(p.wn_begin) + blockIdx.x * kTW;   // 16-byte aligned start
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

// ---- TMA-staged opacity (first stage of the two-stage form, both table precisions)
//
// Work unit = one item x kOT consecutive wavenumbers; a persistent grid of CTAs walks the units
// (items vary fastest, so CTAs running together share a wavenumber tile's table rows in L2).
// Within a unit the layers are walked in order as segments: maximal runs of consecutive
// layers with the same (P, T) cell and CIA temperature bracket.  A producer warp issues, per
// segment, one tiled TMA load of the four bracketing (P, T) rows of every molecule (box {kOT
// wn, 2 T, 2 P, n_mol}) and, when the CIA bracket changed, one of the two CIA rows of every
// pair (box {kOT wn, 2 T, n_cia}), into a ring of stages guarded by full / empty mbarriers;
// it runs up to `stages` segments ahead, across unit boundaries.  kOCW consumer warps (two
// wavenumbers per lane) take a segment's corner rows (decoding 10^(h + c_m) for FP16 tables),
// sum them over molecules with the item's mixing ratios (sum_m x_m sigma_m,c per corner c;
// likewise over CIA pairs), release the stage, and form K of each of the segment's layers from
// those sums: bilinear corner weights times rho, the CIA rows times rho^2, Rayleigh and cloud
// (Sec. 5 and Sec. 8.1) -- the mixing ratios are the same in every layer (Sec. 4.3), so the
// molecule sum is taken once per segment instead of once per layer.  K is streamed to HBM
// once.  Both roles read the layers' brackets and coefficients 32 layers per warp-wide load
// and find the segment starts with warp votes; the coefficients reach each layer by shuffles.
constexpr int kOT = kOpacityTile;                  // wavenumbers per unit
constexpr int kOCW = 4;                            // consumer warps
constexpr int kOThreads = 32 * (kOCW + 1);         // + one producer warp
constexpr int kOMaxStages = 8;
constexpr float kLog2Of10 = 3.32192809488736234787f;
static_assert(kOT == 64 * kOCW, "two wavenumbers per consumer lane");

struct OpacityPlan {                               // shared-memory ring of one CTA
  uint32_t mol_bytes, cia_bytes, stage_bytes;
  int stages;
  __host__ __device__ OpacityPlan(int n_mol, int n_cia, int elem_bytes, int n_stages) {
    mol_bytes = (uint32_t)(kOT * elem_bytes * 4 * n_mol);
    cia_bytes = (uint32_t)(kOT * 4 * 2 * n_cia);
    stage_bytes = (mol_bytes + cia_bytes + 127u) & ~127u;
    stages = n_stages;
  }
  __host__ __device__ uint32_t smem() const { return (uint32_t)stages * stage_bytes + 128u; }
};

// 2^x by the hardware approximation (relative error ~2e-7, far below the FP16 storage step)
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(bar)) : "memory");
}

// Segment starts among the 32 layers l0 .. l0+31 (lane i holds layer l0 + i's bracket header
// h = (ip, it, itc)): bit i of `start` is set when layer l0 + i begins a segment, of `mol`
// when its molecular cell differs from the layer before, of `cia` when its CIA bracket does.
// (cip, cit, citc) carry the header of layer l0 - 1 in and of the chunk's last layer out.
struct SegFlags { unsigned start, mol, cia; };
__device__ __forceinline__ SegFlags segment_flags(const int4& h, int l0, int N, int lane,
                                                  bool has_mol, bool has_cia, int& cip,
                                                  int& cit, int& citc) {
  int pip = __shfl_up_sync(0xffffffffu, h.x, 1);
  int pit = __shfl_up_sync(0xffffffffu, h.y, 1);
  int pitc = __shfl_up_sync(0xffffffffu, h.z, 1);
  if (lane == 0) { pip = cip; pit = cit; pitc = citc; }
  const int li = l0 + lane;
  const bool valid = li < N, first = li == 0;
  const bool mol = valid && has_mol && (first || h.x != pip || h.y != pit);
  const bool cia = valid && has_cia && (first || h.z != pitc);
  SegFlags f;
  f.start = __ballot_sync(0xffffffffu, valid && (mol || cia || first));
  f.mol = __ballot_sync(0xffffffffu, mol);
  f.cia = __ballot_sync(0xffffffffu, cia);
  const int last = min(31, N - 1 - l0);
  cip = __shfl_sync(0xffffffffu, h.x, last);
  cit = __shfl_sync(0xffffffffu, h.y, last);
  citc = __shfl_sync(0xffffffffu, h.z, last);
  return f;
}

template <int MAXMOL, int MAXCIA, bool F16>
__global__ void __launch_bounds__(kOThreads, 3)
k_opacity(FwdParams p, const __grid_constant__ CUtensorMap tm_sig,
          const __grid_constant__ CUtensorMap tm_cia, float* __restrict__ kbuf, long long kcols,
          int Bc, int n_tiles, int n_stages) {
  extern __shared__ unsigned char osm_raw[];
  __shared__ __align__(8) uint64_t full[kOMaxStages];
  __shared__ __align__(8) uint64_t empty[kOMaxStages];
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool has_mol = p.n_mol > 0, has_cia = p.n_cia > 0;
  const OpacityPlan plan(p.n_mol, p.n_cia, F16 ? 2 : 4, n_stages);
  const int S = plan.stages;
  unsigned char* ring = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(osm_raw) + 127) & ~(uintptr_t)127);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], kOCW); }
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const long long n_units = (long long)Bc * n_tiles;
  const int wbase = wn_first(p.wn_begin);

  if (warp == kOCW) {
    // ---------------- producer warp: the lanes read 32 layers' brackets at a time and find the
    // segment starts; lane 0 issues each segment's loads, in unit order
    int seg = 0;
    bool stop = false;
    for (long long u = blockIdx.x; u < n_units && !stop; u += gridDim.x) {
      const int bc = (int)(u % Bc), tile = (int)(u / Bc);
      const int b = p.b_off + bc;
      const int N = p.buf.items[b].n_layers;
      const int x0 = wbase + tile * kOT;
      const LayerDesc* L = p.buf.layers + (size_t)b * p.max_layers;
      int cip = -1, cit = -1, citc = -1;
      for (int l0 = 0; l0 < N && !stop; l0 += 32) {
        const int li = l0 + lane;
        const int4 h = li < N ? __ldg(reinterpret_cast<const int4*>(L + li)) : make_int4(-1, -1, -1, 0);
        const SegFlags f = segment_flags(h, l0, N, lane, has_mol, has_cia, cip, cit, citc);
        for (unsigned m = f.start; m != 0u; m &= m - 1u) {
          const int i = __ffs(m) - 1;
          const int ip = __shfl_sync(0xffffffffu, h.x, i);
          const int it = __shfl_sync(0xffffffffu, h.y, i);
          const int itc = __shfl_sync(0xffffffffu, h.z, i);
          const bool mol = (f.mol >> i) & 1u, cia = (f.cia >> i) & 1u;
          int ok = 1;
          if (lane == 0) {
            const int st = seg % S, k = seg / S;
            if (k > 0 && !mbar_wait_bounded(&empty[st], (k - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT))
              ok = 0;
            if (*(volatile int*)&abort_flag) ok = 0;
            if (ok) {
              unsigned char* sb = ring + st * plan.stage_bytes;
              mbar_arrive_expect_tx(&full[st],
                                    (mol ? plan.mol_bytes : 0u) + (cia ? plan.cia_bytes : 0u));
              if (mol) tma_load_4d(sb, &tm_sig, x0, it, ip, 0, &full[st]);
              if (cia) tma_load_3d(sb + plan.mol_bytes, &tm_cia, x0, itc, 0, &full[st]);
            } else {
              atomicExch(&abort_flag, 1);
            }
          }
          if (!__shfl_sync(0xffffffffu, ok, 0)) { stop = true; break; }
          ++seg;
        }
      }
    }
    // every copy this CTA issued has landed before the CTA may exit: wait for the last fill
    // of each stage (the consumers normally have already)
    if (lane == 0)
      for (int st = 0; st < S && st < seg; ++st) {
        const int last = ((seg - 1 - st) / S) * S + st;
        mbar_wait_bounded(&full[st], (last / S) & 1, nullptr, 0);
      }
    return;
  }

  // ---------------- consumers: warps 0..kOCW-1, two wavenumbers per lane
  const int c2 = 2 * (warp * 32 + lane);             // column offset within the unit
  int seg = 0;
  for (long long u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int bc = (int)(u % Bc), tile = (int)(u / Bc);
    const int b = p.b_off + bc;
    const int N = p.buf.items[b].n_layers;
    const int col = tile * kOT + c2;
    const int w = wbase + col;
    const bool store = col < kcols, in_row = w < p.wn_pad;
    const LayerDesc* L = p.buf.layers + (size_t)b * p.max_layers;
    const float4* op = p.buf.op + (size_t)b * p.max_layers * 2;
    float* dst = kbuf + (size_t)bc * p.max_layers * kcols + col;
    // Rayleigh cross-section sum_s X_s sigma_R,s (scaled per species)
    float ray0 = 0.f, ray1 = 0.f;
    if (p.ray && in_row) {
      const float* rc = p.buf.rayc + (size_t)b * TR_MAX_SPECIES;
      for (int s = 0; s < p.n_species; ++s) {
        const float c = __ldg(rc + s);
        if (c != 0.f) {
          const float2 r = __ldg(reinterpret_cast<const float2*>(p.ray + (size_t)s * p.wn_pad + w));
          ray0 = fmaf(c, r.x, ray0); ray1 = fmaf(c, r.y, ray1);
        }
      }
    }
    // per-item weights of the molecule and CIA-pair sums
    float xm[MAXMOL], yq[MAXCIA];
    const float* ox = p.buf.opx + (size_t)b * kOpxStride;
#pragma unroll
    for (int m = 0; m < MAXMOL; ++m) xm[m] = m < p.n_mol ? __ldg(ox + m) : 0.f;
#pragma unroll
    for (int q = 0; q < MAXCIA; ++q) yq[q] = q < p.n_cia ? __ldg(ox + TR_MAX_MOL + q) : 0.f;
    // cross-sections of the current segment summed over molecules, per bilinear corner
    // (sum_m x_m sigma_m,c), and over CIA pairs, per temperature row
    float us[4][2] = {}, uc[2][2] = {};
    int cip = -1, cit = -1, citc = -1;
    for (int l0 = 0; l0 < N; l0 += 32) {
      // lane i reads layer l0 + i's brackets and coefficients; they are broadcast per layer
      const int li = l0 + lane;
      int4 h = make_int4(-1, -1, -1, 0);
      float4 ha = make_float4(0.f, 0.f, 0.f, 0.f), hb = ha;
      if (li < N) {
        h = __ldg(reinterpret_cast<const int4*>(L + li));
        ha = __ldg(op + 2 * li);
        hb = __ldg(op + 2 * li + 1);
      }
      const SegFlags f = segment_flags(h, l0, N, lane, has_mol, has_cia, cip, cit, citc);
      const int n_here = min(32, N - l0);
      for (int i = 0; i < n_here; ++i) {
        if ((f.start >> i) & 1u) {                     // a new segment: take its stage
          const bool mol = (f.mol >> i) & 1u, cia = (f.cia >> i) & 1u;
          const int st = seg % S, k = seg / S;
          const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[st], k & 1, p.dev_err,
                                                                     TR_DEVERR_TIMEOUT) &&
                                                      !*(volatile int*)&abort_flag);
          if (!ok) { if (lane == 0) atomicExch(&abort_flag, 1); return; }
          const unsigned char* sb = ring + st * plan.stage_bytes;
          if (mol) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float s0 = 0.f, s1 = 0.f;
#pragma unroll
              for (int m = 0; m < MAXMOL; ++m) {
                if (m < p.n_mol) {
                  const int e = (m * 4 + c) * kOT + c2;   // box order: wn, T, P, molecule
                  float v0, v1;
                  if (F16) {
                    const float2 hv = __half22float2(*reinterpret_cast<const __half2*>(
                        reinterpret_cast<const __half*>(sb) + e));
                    const float off = p.logsig_off[m];
                    v0 = ex2_fast((hv.x + off) * kLog2Of10);
                    v1 = ex2_fast((hv.y + off) * kLog2Of10);
                  } else {
                    const float2 fv = *reinterpret_cast<const float2*>(
                        reinterpret_cast<const float*>(sb) + e);
                    v0 = fv.x; v1 = fv.y;
                  }
                  s0 = fmaf(xm[m], v0, s0); s1 = fmaf(xm[m], v1, s1);
                }
              }
              us[c][0] = s0; us[c][1] = s1;
            }
          }
          if (cia) {
            const float* cbuf = reinterpret_cast<const float*>(sb + plan.mol_bytes);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              float s0 = 0.f, s1 = 0.f;
#pragma unroll
              for (int q = 0; q < MAXCIA; ++q) {
                if (q < p.n_cia) {
                  const float2 fv = *reinterpret_cast<const float2*>(cbuf + (2 * q + t) * kOT + c2);
                  s0 = fmaf(yq[q], fv.x, s0); s1 = fmaf(yq[q], fv.y, s1);
                }
              }
              uc[t][0] = s0; uc[t][1] = s1;
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[st]);     // this warp is done with the stage
          ++seg;
        }
        // K = kappa_cloud + rho sigma_R + sum_c (rho x_max w_c) sum_m x_m sigma_m,c
        //       + sum_T (rho^2 y_max w_T) sum_q y_q sigma_q,T
        const float w0 = __shfl_sync(0xffffffffu, ha.x, i), w1 = __shfl_sync(0xffffffffu, ha.y, i);
        const float w2 = __shfl_sync(0xffffffffu, ha.z, i), w3 = __shfl_sync(0xffffffffu, ha.w, i);
        const float y0 = __shfl_sync(0xffffffffu, hb.x, i), y1 = __shfl_sync(0xffffffffu, hb.y, i);
        const float rho = __shfl_sync(0xffffffffu, hb.z, i), kc = __shfl_sync(0xffffffffu, hb.w, i);
        float k0 = fmaf(rho, ray0, kc), k1 = fmaf(rho, ray1, kc);
        k0 = fmaf(w0, us[0][0], k0); k1 = fmaf(w0, us[0][1], k1);
        k0 = fmaf(w1, us[1][0], k0); k1 = fmaf(w1, us[1][1], k1);
        k0 = fmaf(w2, us[2][0], k0); k1 = fmaf(w2, us[2][1], k1);
        k0 = fmaf(w3, us[3][0], k0); k1 = fmaf(w3, us[3][1], k1);
        k0 = fmaf(y0, uc[0][0], k0); k1 = fmaf(y0, uc[0][1], k1);
        k0 = fmaf(y1, uc[1][0], k0); k1 = fmaf(y1, uc[1][1], k1);
        if (store)
          __stcs(reinterpret_cast<float2*>(dst + (size_t)(l0 + i) * kcols),
                 in_row ? make_float2(k0, k1) : make_float2(0.f, 0.f));
      }
    }
  }
}

// Ring depth for `ctas` CTAs per SM: as many stages as fit the SM's shared memory, at most
// kOMaxStages, at least 2.
OpacityPlan opacity_plan(int n_mol, int n_cia, bool f16, int ctas) {
  constexpr uint32_t kSmemPerSm = 227u * 1024u;   // usable by the CTAs of one SM
  const OpacityPlan one(n_mol, n_cia, f16 ? 2 : 4, 1);
  const uint32_t sb = one.stage_bytes > 0 ? one.stage_bytes : 128u;
  const uint32_t per = kSmemPerSm / (uint32_t)ctas - 1024u - 256u;   // runtime reserve, statics
  int s = (int)((per - 128u) / sb);
  s = std::max(2, std::min(s, kOMaxStages));
  return OpacityPlan(n_mol, n_cia, f16 ? 2 : 4, s);
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int MAXMOL, int MAXCIA, bool F16>
cudaError_t launch_opacity_t(const FwdParams& p, const CUtensorMap& sig, const CUtensorMap& cia,
                             int Bc, float* kbuf, long long kcols, cudaStream_t s) {
  auto kern = k_opacity<MAXMOL, MAXCIA, F16>;
  // CTAs per SM: what the registers allow (at most 3), then the deepest ring that fits them
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOThreads, 0);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, std::min(per_sm, 3));
  OpacityPlan plan = opacity_plan(p.n_mol, p.n_cia, F16, per_sm);
  while (per_sm > 1 && plan.stages < 3) plan = opacity_plan(p.n_mol, p.n_cia, F16, --per_sm);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem());
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kOThreads, plan.smem());
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, std::min(per_sm, occ));
  const int n_tiles = (int)((kcols + kOT - 1) / kOT);
  const long long units = (long long)Bc * n_tiles;
  const int grid = (int)std::min<long long>(units, (long long)sm_count() * per_sm);
  kern<<<grid, kOThreads, plan.smem(), s>>>(p, sig, cia, kbuf, kcols, Bc, n_tiles, plan.stages);
  return cudaGetLastError();
}

template <bool F16>
cudaError_t launch_opacity_p(const FwdParams& p, const CUtensorMap& sig, const CUtensorMap& cia,
                             int Bc, float* kbuf, long long kcols, cudaStream_t s) {
  static_assert(TR_MAX_MOL == 8 && TR_MAX_CIA == 4, "opacity instantiations cover the limits");
  if (p.n_cia <= 2) {
    if (p.n_mol <= 2) return launch_opacity_t<2, 2, F16>(p, sig, cia, Bc, kbuf, kcols, s);
    if (p.n_mol <= 5) return launch_opacity_t<5, 2, F16>(p, sig, cia, Bc, kbuf, kcols, s);
    return launch_opacity_t<8, 2, F16>(p, sig, cia, Bc, kbuf, kcols, s);
  }
  if (p.n_mol <= 2) return launch_opacity_t<2, 4, F16>(p, sig, cia, Bc, kbuf, kcols, s);
  if (p.n_mol <= 5) return launch_opacity_t<5, 4, F16>(p, sig, cia, Bc, kbuf, kcols, s);
  return launch_opacity_t<8, 4, F16>(p, sig, cia, Bc, kbuf, kcols, s);
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
  const int w_first = wn_first(p.wn_begin) + blockIdx.x * kTW;
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
  const int w_first = wn_first(p.wn_begin);
  return (p.wn_begin + p.wn_count - w_first + kTW - 1) / kTW;
}

}  // namespace

constexpr size_t kKbufBudget = 2ull << 30;       // bytes of K per chunk of items

int forward_chunk_items(int B, int max_layers, int wn_begin, int wn_count) {
  const int w_first = wn_first(wn_begin);
  const size_t cols = (size_t)((wn_begin + wn_count - w_first + kTW - 1) / kTW) * kTW;
  const size_t per = sizeof(float) * (size_t)max_layers * cols;
  const size_t n = std::max<size_t>(1, kKbufBudget / per);
  return (int)std::min<size_t>((size_t)std::max(B, 1), n);
}

size_t forward_kbuf_bytes(int B, int max_layers, int wn_begin, int wn_count) {
  const int w_first = wn_first(wn_begin);
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

cudaError_t launch_opacity(const FwdParams& p, const CUtensorMap* tm_sig,
                           const CUtensorMap* tm_cia, int Bc, float* kbuf, cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  const long long kcols = (long long)n_tiles_of(p) * kTW;
  return p.logsig16 ? launch_opacity_p<true>(p, *tm_sig, *tm_cia, Bc, kbuf, kcols, s)
                    : launch_opacity_p<false>(p, *tm_sig, *tm_cia, Bc, kbuf, kcols, s);
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
