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
// wavenumbers; shells below j0 are skipped (the triangle); tiles go longest-first to the
// least-loaded warp; the epilogue folds a_j (1 - e^-tau) per lane and the 8 warps' partial sums
// are added in FP64 in a fixed order (deterministic), plus (R_p/R_s)^2 in FP64.
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

// tau = DL K over 8-ray tiles and the epilogue sum_j a_j (1 - e^-tau) into this lane's partial
// depths at its 4 wavenumbers.  DLP holds the packed path-length rows; ray tiles cover rays
// 0..ceil(N/8)*8-1 and are dealt longest-first to the least-loaded of the kWarps warps (a fixed
// schedule: the result does not depend on timing).  Rows go in unrolled blocks of 8.
__device__ __forceinline__ void contract_tiles(int N, const float* Kt, const float* DLP,
                                               const float* a_s, float (&part)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_rt = (N + kRT - 1) / kRT;
  int ld[kWarps];
#pragma unroll
  for (int k = 0; k < kWarps; ++k) ld[k] = 0;
  for (int t = 0; t < n_rt; ++t) {
    int wm = 0, lm = ld[0];
#pragma unroll
    for (int k = 1; k < kWarps; ++k) if (ld[k] < lm) { wm = k; lm = ld[k]; }
    const int len = N - t * kRT;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) ld[k] += k == wm ? len : 0;
    if (wm != warp) continue;
    const int j0 = t * kRT;
    float acc[kRT][4];
#pragma unroll
    for (int r = 0; r < kRT; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
    // rows in blocks of 8: in the packed layout rows l .. l+7 (l a multiple of 8) are
    // pad8(l+1) = l + 8 floats apart, so a block needs no address arithmetic per row
    const float* kp = Kt + (size_t)j0 * kTW + 4 * lane;
    const float* dp = DLP + dlp_offset(j0) + j0;
    int step = j0 + 8;
    int l = j0;
    for (; l + 8 <= N; l += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 kv = *reinterpret_cast<const float4*>(kp + u * kTW);
        const float4 d0 = *reinterpret_cast<const float4*>(dp + u * step);
        const float4 d1 = *reinterpret_cast<const float4*>(dp + u * step + 4);
        const float dv[kRT] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
        for (int r = 0; r < kRT; ++r) {
          acc[r][0] = fmaf(dv[r], kv.x, acc[r][0]);
          acc[r][1] = fmaf(dv[r], kv.y, acc[r][1]);
          acc[r][2] = fmaf(dv[r], kv.z, acc[r][2]);
          acc[r][3] = fmaf(dv[r], kv.w, acc[r][3]);
        }
      }
      kp += 8 * kTW;
      dp += 8 * step;
      step += 8;
    }
    for (int u = 0; l < N; ++l, ++u) {                 // the last rows (fewer than 8)
      const float4 kv = *reinterpret_cast<const float4*>(kp + u * kTW);
      const float4 d0 = *reinterpret_cast<const float4*>(dp + u * step);
      const float4 d1 = *reinterpret_cast<const float4*>(dp + u * step + 4);
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

// ---- FP32 contraction + depth, persistent (second stage of the two-stage form)
//
// Work unit = one item x kTW wavenumbers of K; the units are split into contiguous ranges, one
// per CTA (item-major, so consecutive units of a CTA mostly share the item and its path
// lengths).  A producer warp loads each unit's K tile [N][kTW] by 2-D TMA boxes of kCB rows
// into one of two tile buffers, plus the item's packed path lengths and annulus weights by bulk
// copy when the item changes (after the units of the previous item are done with them); the 8
// contraction warps work on the other buffer meanwhile: tau = DL K, 1 - e^-tau, the FP64
// depth sum (contract_tiles).
constexpr int kCB = 32;                          // K rows per TMA box
constexpr int kCThreads = kThreads + 32;         // + one producer warp

struct ContractLayout {                          // dynamic shared memory (128-byte aligned)
  uint32_t kt0, kt1, dl, aj, red, total;
  __host__ __device__ ContractLayout(int max_layers, int k_bufs) {
    const uint32_t rows = (uint32_t)((max_layers + kCB - 1) / kCB * kCB);
    const uint32_t ktb = rows * kTW * 4;
    kt0 = 0;
    kt1 = k_bufs > 1 ? ktb : 0;
    dl = kt1 + ktb;
    aj = dl + (((uint32_t)dlp_offset(max_layers) * 4 + 127u) & ~127u);
    red = aj + (((uint32_t)pad8(max_layers) * 4 + 127u) & ~127u);
    total = red + (uint32_t)(kWarps * kTW * 4) + 128u;
  }
};

__device__ __forceinline__ void contraction_warps_sync() {
  asm volatile("bar.sync 1, %0;" :: "r"(kThreads) : "memory");
}

template <int MINB>
__global__ void __launch_bounds__(kCThreads, MINB)
k_contract_fp32(FwdParams p, const __grid_constant__ CUtensorMap tm_k, long long kcols, int Bc,
                int n_tiles, int k_bufs) {
  extern __shared__ unsigned char csm_raw[];
  __shared__ __align__(8) uint64_t kfull[2], kempty[2];
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ContractLayout lay(p.max_layers, k_bufs);
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(csm_raw) + 127) & ~(uintptr_t)127);
  float* const K0 = reinterpret_cast<float*>(base + lay.kt0);
  float* const K1 = reinterpret_cast<float*>(base + lay.kt1);
  float* const DLP = reinterpret_cast<float*>(base + lay.dl);
  float* const a_s = reinterpret_cast<float*>(base + lay.aj);
  float* const red = reinterpret_cast<float*>(base + lay.red);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) { mbar_init(&kfull[i], 1); mbar_init(&kempty[i], kWarps); }
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const long long units = (long long)Bc * n_tiles;
  const long long per = (units + gridDim.x - 1) / gridDim.x;
  const long long u_begin = (long long)blockIdx.x * per;
  const long long u_end = u_begin + per < units ? u_begin + per : units;
  const int wbase = wn_first(p.wn_begin);

  if (warp == kWarps) {
    // ---------------- producer
    if (lane != 0) return;
    int k = 0, dl_item = -1;
    for (long long u = u_begin; u < u_end; ++u) {
      const int bc = (int)(u / n_tiles), tile = (int)(u % n_tiles);
      const int b = p.b_off + bc;
      const int N = p.buf.items[b].n_layers;
      if (N == 0) continue;
      const int kb = k_bufs > 1 ? (k & 1) : 0, use = k_bufs > 1 ? (k >> 1) : k;
      bool ok = use == 0 ||
                mbar_wait_bounded(&kempty[kb], (use - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
      const bool new_item = b != dl_item;
      if (ok && new_item && k > 0 && k_bufs > 1) {
        // the previous unit (other buffer) must be done with the path lengths too
        const int kp = k - 1;
        ok = mbar_wait_bounded(&kempty[kp & 1], (kp >> 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
      }
      if (!ok || *(volatile int*)&abort_flag) { atomicExch(&abort_flag, 1); break; }
      const int nbox = (N + kCB - 1) / kCB;
      uint32_t bytes = (uint32_t)nbox * kCB * kTW * 4;
      if (new_item) bytes += (uint32_t)(dlp_offset(N) * 4 + p.buf.npad * 4);
      mbar_arrive_expect_tx(&kfull[kb], bytes);
      float* Kt = kb ? K1 : K0;
      for (int i = 0; i < nbox; ++i)
        tma_load_2d(Kt + (size_t)i * kCB * kTW, &tm_k, tile * kTW, bc * p.max_layers + i * kCB,
                    &kfull[kb]);
      if (new_item) {
        bulk_g2s(DLP, p.buf.dlp + (size_t)b * dlp_offset(p.max_layers),
                 (uint32_t)(dlp_offset(N) * 4), &kfull[kb]);
        bulk_g2s(a_s, p.buf.aj + (size_t)b * p.buf.npad, (uint32_t)(p.buf.npad * 4), &kfull[kb]);
        dl_item = b;
      }
      ++k;
    }
    // every copy issued has landed before the CTA may exit
    for (int i = 0; i < 2 && i < k; ++i) {
      const int kb_last = k_bufs > 1 ? ((k - 1 - i) & 1) : 0;
      const int use_last = k_bufs > 1 ? ((k - 1 - i) >> 1) : (k - 1 - i);
      mbar_wait_bounded(&kfull[kb_last], use_last & 1, nullptr, 0);
    }
    return;
  }

  // ---------------- contraction warps
  int k = 0;
  bool failed = false;
  for (long long u = u_begin; u < u_end; ++u) {
    const int bc = (int)(u / n_tiles), tile = (int)(u % n_tiles);
    const int b = p.b_off + bc;
    const ItemGeom ig = p.buf.items[b];
    const int N = ig.n_layers;
    const int w_first = wbase + tile * kTW;
    if (N == 0) {
      if (threadIdx.x < kTW) {
        const int w = w_first + threadIdx.x;
        if (w >= p.wn_begin && w < p.wn_begin + p.wn_count)
          p.out[(long long)b * p.out_stride + (w - p.wn_begin)] = 0.0;
      }
      continue;
    }
    const int kb = k_bufs > 1 ? (k & 1) : 0, use = k_bufs > 1 ? (k >> 1) : k;
    ++k;
    if (!failed) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&kfull[kb], use & 1, p.dev_err,
                                                                TR_DEVERR_TIMEOUT));
      if (!ok) { failed = true; if (lane == 0) atomicExch(&abort_flag, 1); }
    }
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    if (!failed) {
      contract_tiles(N, kb ? K1 : K0, DLP, a_s, part);
      __syncwarp();
      if (lane == 0) mbar_arrive(&kempty[kb]);      // done with the tile and path lengths
    }
    *reinterpret_cast<float4*>(red + warp * kTW + 4 * lane) =
        make_float4(part[0], part[1], part[2], part[3]);
    contraction_warps_sync();
    if (*(volatile int*)&abort_flag) return;        // every contraction warp sees the same
    if (threadIdx.x < kTW) {
      const int w = w_first + threadIdx.x;
      if (w >= p.wn_begin && w < p.wn_begin + p.wn_count) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) s += (double)red[q * kTW + threadIdx.x];
        p.out[(long long)b * p.out_stride + (w - p.wn_begin)] = ig.rp2_rs2 + s;
      }
    }
    contraction_warps_sync();                       // red is free again
  }
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

template <int MINB>
cudaError_t launch_contract_t(const FwdParams& p, const CUtensorMap& tm, long long kcols, int Bc,
                              int tiles, int k_bufs, uint32_t smem, cudaStream_t s) {
  auto kern = k_contract_fp32<MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kCThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const long long units = (long long)Bc * tiles;
  const int grid = (int)std::min<long long>(units, (long long)sm_count() * std::min(occ, MINB));
  kern<<<grid, kCThreads, smem, s>>>(p, tm, kcols, Bc, tiles, k_bufs);
  return cudaGetLastError();
}

cudaError_t launch_contract_fp32(const FwdParams& p, int Bc, const float* kbuf, int per_sm,
                                 cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  const int tiles = n_tiles_of(p);
  const long long kcols = (long long)tiles * kTW;
  CUtensorMap tm{};
  if (!encode_2d_f32(&tm, kbuf, (unsigned long long)kcols,
                     (unsigned long long)Bc * p.max_layers, (unsigned long long)kcols * 4, kTW,
                     kCB))
    return cudaErrorInvalidValue;
  constexpr uint32_t kSmemSm = 227u * 1024u;
  if (per_sm == 2) {                  // two CTAs per SM, one K tile each, when they fit
    const uint32_t smem = ContractLayout(p.max_layers, 1).total;
    if (smem <= kSmemSm / 2 - 1024u) return launch_contract_t<2>(p, tm, kcols, Bc, tiles, 1, smem, s);
  }
  // one CTA per SM, two K tiles (loads of the next unit overlap the contraction) when they fit
  const int k_bufs = ContractLayout(p.max_layers, 2).total <= kSmemSm - 1024u ? 2 : 1;
  const uint32_t smem = ContractLayout(p.max_layers, k_bufs).total;
  if (smem > kSmemSm - 1024u) return cudaErrorInvalidConfiguration;
  return launch_contract_t<1>(p, tm, kcols, Bc, tiles, k_bufs, smem, s);
}

}  // namespace tr
