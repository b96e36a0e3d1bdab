// forward_fp32.cu -- the two-stage forward form: opacity K[layer, wn] (Sec. 5 linear P/T
// interpolation, weighted by rho X and fused with Rayleigh, CIA and the grey cloud as in
// Sec. 8.1) streamed to HBM by k_opacity, then the slant optical depth
// tau[ray, wn] = sum_{l >= j} DL[j][l] K[l][wn] (Sec. 4, eqs. tot_opt_dpth, opt_dpth,
// cia_opt_dpth) and transit depth D = (R_p/R_s)^2 + sum_j a_j (1 - exp(-tau_j)) (Sec. 4, eqs.
// Delta_lambda, a_lambda) by k_contract_fp32 (FP32) or k_contract_umma (mixed.cu, tensor
// cores).  Items are processed in chunks whose K fits a 2 GiB budget.  k_opacity stages the
// bracketing table rows in shared memory by TMA tensor-map loads (opacity.h); with FP16 log
// tables it decodes them on the fly.  This is the default form of both precisions when a K
// buffer is available; the fused kernel (fused.cu) serves callers without one.
//
// The FP32 contraction: a warp owns 8-ray register tiles (j0..j0+7), a lane owns 4
// wavenumbers; shells below j0 are skipped (the triangle); tiles are dealt to warps in snake
// order; the epilogue folds a_j (1 - e^-tau) per lane and the 8 warps' partial sums are added
// in FP64 in a fixed order (deterministic), plus (R_p/R_s)^2 in FP64.
#include <algorithm>
#include <cuda_fp16.h>
#include "opacity.h"
#include "tma.h"
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kTW = 128;         // wavenumbers per CTA
constexpr int kThreads = 256;    // 8 warps
constexpr int kWarps = kThreads / 32;
constexpr int kRT = 8;           // rays per register tile

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

// ---- TMA-staged opacity (first stage of the two-stage form, both table precisions)
//
// Work unit = one item x kOT consecutive wavenumbers; a persistent grid of CTAs walks the units
// (items vary fastest, so CTAs running together share a wavenumber tile's table rows in L2).
// A producer warp streams each unit's segments through the ring of table-row stages
// (opacity.h); kOCW consumer warps (two wavenumbers per lane) sum each segment's rows over
// molecules and CIA pairs and form K of every layer of the segment from those sums:
//   K = kappa_cloud + rho sigma_R + sum_c (rho x_max w_c) sum_m x_m sigma_m,c
//         + sum_T (rho^2 y_max w_T) sum_q y_q sigma_q,T
// with bilinear corner weights w_c and CIA temperature weights w_T (Sec. 5, Sec. 8.1).  K is
// streamed to HBM once.  Both roles read the layers' brackets and coefficients 32 layers per
// warp-wide load and find the segment starts with warp votes; the coefficients reach each
// layer by shuffles.
constexpr int kOT = kOpacityTile;                  // wavenumbers per unit
constexpr int kOCW = 4;                            // consumer warps
constexpr int kOThreads = 32 * (kOCW + 1);         // + one producer warp
static_assert(kOT == 64 * kOCW, "two wavenumbers per consumer lane");

template <int MAXMOL, int MAXCIA, bool F16>
__global__ void __launch_bounds__(kOThreads, 3)
k_opacity(FwdParams p, const __grid_constant__ CUtensorMap tm_sig,
          const __grid_constant__ CUtensorMap tm_cia, float* __restrict__ kbuf, long long kcols,
          int Bc, int n_tiles, int n_stages) {
  extern __shared__ unsigned char osm_raw[];
  __shared__ Ring rs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool has_mol = p.n_mol > 0, has_cia = p.n_cia > 0;
  const RingPlan plan(kOT, p.n_mol, p.n_cia, F16 ? 2 : 4, n_stages);
  unsigned char* ring = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(osm_raw) + 127) & ~(uintptr_t)127);
  if (threadIdx.x == 0) ring_init(rs, plan.stages, kOCW);
  __syncthreads();
  const long long n_units = (long long)Bc * n_tiles;
  const int wbase = wn_first(p.wn_begin);
  if (warp == kOCW) {
    ring_produce<kOT>(p, rs, plan, ring, &tm_sig, &tm_cia, Bc, n_units, lane, false);
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
    const float ray0 = in_row ? rayleigh1(p, b, w) : 0.f;
    const float ray1 = in_row ? rayleigh1(p, b, w + 1) : 0.f;
    float xm[MAXMOL], yq[MAXCIA];
    item_weights<MAXMOL, MAXCIA>(p, b, xm, yq);
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
          if (!ring_consume<kOT, 2, MAXMOL, MAXCIA, F16>(p, rs, plan, ring, seg,
                                                         (f.mol >> i) & 1u, (f.cia >> i) & 1u,
                                                         c2, xm, yq, us, uc, lane))
            return;
          ++seg;
        }
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

// Ring depth for `ctas` CTAs per SM of `fixed` bytes besides the ring each: as many stages as
// fit the SM's shared memory, at most kRingMaxStages, at least 2.
int ring_stages(uint32_t stage_bytes, int ctas, uint32_t fixed) {
  constexpr uint32_t kSmemPerSm = 227u * 1024u;   // usable by the CTAs of one SM
  const uint32_t sb = stage_bytes > 0 ? stage_bytes : 128u;
  const uint32_t per = kSmemPerSm / (uint32_t)ctas - 1024u - 512u;   // runtime reserve, statics
  const int s = per > fixed + 128u ? (int)((per - fixed - 128u) / sb) : 0;
  return std::max(2, std::min(s, kRingMaxStages));
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
                             int Bc, float* kbuf, long long kcols, int per_sm_cap,
                             cudaStream_t s) {
  auto kern = k_opacity<MAXMOL, MAXCIA, F16>;
  // CTAs per SM: what the registers allow (at most 3, or the caller's cap), then the deepest
  // ring that fits them
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOThreads, 0);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, std::min(per_sm, per_sm_cap > 0 ? std::min(per_sm_cap, 3) : 3));
  const RingPlan one(kOT, p.n_mol, p.n_cia, F16 ? 2 : 4, 1);
  int stages = ring_stages(one.stage_bytes, per_sm, 0);
  while (per_sm > 1 && stages < 3) stages = ring_stages(one.stage_bytes, --per_sm, 0);
  const RingPlan plan(kOT, p.n_mol, p.n_cia, F16 ? 2 : 4, stages);
  const uint32_t smem = plan.bytes() + 128u;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kOThreads, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, std::min(per_sm, occ));
  const int n_tiles = (int)((kcols + kOT - 1) / kOT);
  const long long units = (long long)Bc * n_tiles;
  const int grid = (int)std::min<long long>(units, (long long)sm_count() * per_sm);
  kern<<<grid, kOThreads, smem, s>>>(p, sig, cia, kbuf, kcols, Bc, n_tiles, stages);
  return cudaGetLastError();
}

template <bool F16>
cudaError_t launch_opacity_p(const FwdParams& p, const CUtensorMap& sig, const CUtensorMap& cia,
                             int Bc, float* kbuf, long long kcols, int cap, cudaStream_t s) {
  static_assert(TR_MAX_MOL == 8 && TR_MAX_CIA == 4, "opacity instantiations cover the limits");
  if (p.n_cia <= 2) {
    if (p.n_mol <= 2) return launch_opacity_t<2, 2, F16>(p, sig, cia, Bc, kbuf, kcols, cap, s);
    if (p.n_mol <= 5) return launch_opacity_t<5, 2, F16>(p, sig, cia, Bc, kbuf, kcols, cap, s);
    return launch_opacity_t<8, 2, F16>(p, sig, cia, Bc, kbuf, kcols, cap, s);
  }
  if (p.n_mol <= 2) return launch_opacity_t<2, 4, F16>(p, sig, cia, Bc, kbuf, kcols, cap, s);
  if (p.n_mol <= 5) return launch_opacity_t<5, 4, F16>(p, sig, cia, Bc, kbuf, kcols, cap, s);
  return launch_opacity_t<8, 4, F16>(p, sig, cia, Bc, kbuf, kcols, cap, s);
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

cudaError_t launch_opacity(const FwdParams& p, const CUtensorMap* tm_sig,
                           const CUtensorMap* tm_cia, int Bc, float* kbuf, int per_sm_cap,
                           cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  const long long kcols = (long long)n_tiles_of(p) * kTW;
  return p.logsig16
             ? launch_opacity_p<true>(p, *tm_sig, *tm_cia, Bc, kbuf, kcols, per_sm_cap, s)
             : launch_opacity_p<false>(p, *tm_sig, *tm_cia, Bc, kbuf, kcols, per_sm_cap, s);
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
