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
// The FP32 contraction: a warp takes one 16-ray register tile (j0..j0+15) of a unit at a time, a
// lane owns 4 wavenumbers; shells below j0 are skipped (the triangle); the tile's partial
// depth sum_j a_j (1 - e^-tau_j) is stored per tile, and the unit's depths are the tiles'
// partials added in tile order (deterministic) plus (R_p/R_s)^2 in FP64.
#include <algorithm>
#include <cuda_fp16.h>
#include <type_traits>
#include "opacity.h"
#include "tma.h"
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kTW = 128;         // wavenumbers per contraction unit (4 per lane)
constexpr int kRT = 16;          // rays per register tile

// tau = DL K for the 16 rays j0 .. j0+15 at this lane's 4 wavenumbers of the K tile Kt
// [rows][kTW], and the tile's partial depth sum_j a_j (1 - e^-tau_j) into part.  DLP holds the
// packed path-length rows (row l: rays 0 .. pad8(l+1)-1, zero for j > l), so rows l < j0 + 16
// contribute zero to the rays above l; rows go in unrolled blocks of 8.  Sixteen rays per
// K load halve the shared-memory reads per FMA against 8-ray tiles (the tile was bound by
// shared-memory wavefronts and issue together).
__device__ __forceinline__ void contract_tile(int N, int j0, const float* Kt, const float* DLP,
                                              const float* a_s, float (&part)[4]) {
  const int lane = threadIdx.x & 31;
  unsigned long long acc[kRT / 2][4];
#pragma unroll
  for (int r = 0; r < kRT / 2; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0ull;
  const float* kp = Kt + (size_t)j0 * kTW + 4 * lane;
  const float* dp = DLP + dlp_offset(j0) + j0;
  int step = j0 + 8;
  int l = j0;
  // acc[r][c]: rays (2r, 2r+1) of the tile at wavenumber c of the lane.  A row brings the K
  // values (duplicated into both halves) and the path lengths as pairs, as loaded; NQ float4
  // groups of rays (2 in the tile's first 8 rows, whose packed rows end at ray j0+7, else 4)
  auto row = [&](const float* kr, const float* dr, auto nq) {
    constexpr int NQ = decltype(nq)::value;
    const float4 kv = *reinterpret_cast<const float4*>(kr);
    const unsigned long long kc[4] = {pack_dup(kv.x), pack_dup(kv.y), pack_dup(kv.z), pack_dup(kv.w)};
#pragma unroll
    for (int g = 0; g < NQ; ++g) {
      const ulonglong2 d = *reinterpret_cast<const ulonglong2*>(dr + 4 * g);
#pragma unroll
      for (int c = 0; c < 4; ++c) { ffma2(acc[2 * g][c], d.x, kc[c]); ffma2(acc[2 * g + 1][c], d.y, kc[c]); }
    }
  };
  using Q2 = std::integral_constant<int, 2>;
  using Q4 = std::integral_constant<int, 4>;
  // in the packed layout rows l .. l+7 (l a multiple of 8) are pad8(l+1) = l + 8 floats
  // apart, so a block needs no address arithmetic per row; rows j0 .. j0+7 hold rays up to
  // j0+7 only
  if (l + 8 <= N) {
#pragma unroll
    for (int u = 0; u < 8; ++u) row(kp + u * kTW, dp + u * step, Q2{});
    kp += 8 * kTW; dp += 8 * step; step += 8; l += 8;
  } else {
    for (int u = 0; l < N; ++l, ++u) row(kp + u * kTW, dp + u * step, Q2{});
  }
  for (; l + 8 <= N; l += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) row(kp + u * kTW, dp + u * step, Q4{});
    kp += 8 * kTW;
    dp += 8 * step;
    step += 8;
  }
  for (int u = 0; l < N; ++l, ++u) row(kp + u * kTW, dp + u * step, Q4{});   // last rows (< 8)
  // 1 - e^-tau with the hardware exponential: its absolute error (a few 1e-7) times the
  // annulus weights (sum ~ 1e-3) stays below 1e-9 in depth, far inside 0.1 ppm; rays at or
  // beyond N add nothing
#pragma unroll
  for (int c = 0; c < 4; ++c) part[c] = 0.f;
#pragma unroll
  for (int r = 0; r < kRT / 2; ++r) {
    const int j = j0 + 2 * r;
    const float a0 = j < N ? a_s[j] : 0.f, a1 = j + 1 < N ? a_s[j + 1] : 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float t0, t1;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(t0), "=f"(t1) : "l"(acc[r][c]));
      part[c] = fmaf(a0, 1.f - __expf(-t0), part[c]);
      part[c] = fmaf(a1, 1.f - __expf(-t1), part[c]);
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

template <int MAXMOL, int MAXCIA, bool F16, bool EXPT>
__global__ void __launch_bounds__(kOThreads, (EXPT && MAXMOL > 5) ? 2 : 3)
k_opacity(FwdParams p, const __grid_constant__ CUtensorMap tm_sig,
          const __grid_constant__ CUtensorMap tm_cia, float* __restrict__ kbuf, long long kcols,
          int Bc, int n_tiles, int n_stages, int n_lb, int lb_size) {
  extern __shared__ unsigned char osm_raw[];
  __shared__ Ring rs;
  pdl_trigger();                                // the contraction may launch (it waits)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool has_mol = p.n_mol > 0, has_cia = p.n_cia > 0;
  const RingPlan plan(kOT, p.n_mol, p.n_cia, F16 ? 2 : 4, n_stages);
  unsigned char* ring = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(osm_raw) + 127) & ~(uintptr_t)127);
  if (threadIdx.x == 0) ring_init(rs, plan.stages, kOCW);
  __syncthreads();
  const long long n_units = (long long)Bc * n_lb * n_tiles;
  const int wbase = wn_first(p.wn_begin);
  if (warp == kOCW) {
    ring_produce<kOT>(p, rs, plan, ring, &tm_sig, &tm_cia, Bc, n_units, lane, false, n_lb,
                      lb_size);
    return;
  }
  // ---------------- consumers: warps 0..kOCW-1, two wavenumbers per lane.  They walk the same
  // chunks (32 layers of a unit) as the producer.  The global data of the chunk after the
  // current one -- its layers' brackets and coefficients and, at a unit start, the unit's
  // Rayleigh sums and sum weights -- is loaded one chunk ahead, so its latency overlaps the
  // current chunk's work.
  struct CChunk {
    long long u;
    OpUnit o;
    int l0;
    int4 h;
    float4 ha, hb;
    float2 ray;
    float xm[MAXMOL], yq[MAXCIA];
    int zone;                                     // chemistry zone of ray, xm and yq
  };
  const int c2 = 2 * (warp * 32 + lane);             // column offset within the unit
  auto first_from = [&](long long u, CChunk& c) -> bool {
    for (; u < n_units; u += gridDim.x) {
      const OpUnit o = op_unit(p, u, Bc, n_lb, lb_size);
      if (o.l_begin < o.l_end) { c.u = u; c.o = o; c.l0 = o.l_begin; return true; }
    }
    return false;
  };
  auto read = [&](CChunk& c, bool unit_start) {
    const int b = p.b_off + c.o.bc;
    const int li = c.l0 + lane;
    c.h = make_int4(-1, -1, -1, 0);
    c.ha = make_float4(0.f, 0.f, 0.f, 0.f);
    c.hb = c.ha;
    if (li < c.o.l_end) {
      const float4* op = p.buf.op + ((size_t)b * p.max_layers + li) * 2;
      c.h = __ldg(reinterpret_cast<const int4*>(p.buf.layers + (size_t)b * p.max_layers + li));
      c.ha = __ldg(op);
      c.hb = __ldg(op + 1);
    }
    if (unit_start) {
      // the weights of the zone of the unit's first layer (zone 0 with constant mixing ratios)
      // (the exponential scheme serves constant mixing ratios only: its register set is full)
      c.zone = (!EXPT && p.buf.zoned) ? __shfl_sync(0xffffffffu, c.h.w, 0) : 0;
      const int w = wbase + c.o.tile * kOT + c2;
      c.ray = w < p.wn_pad ? rayleigh2(p, b, c.zone, w) : make_float2(0.f, 0.f);
      item_weights<MAXMOL, MAXCIA>(p, b, c.zone, c.xm, c.yq);
    }
  };
  int seg = 0;
  int cip = -1, cit = -1, citc = -1, czone = -1;
  float us[4][2] = {}, uc[2][2] = {};
  // exponential T scheme: per molecule, P row and wavenumber log2 sigma at T_j and its step
  // to T_j+1 (or, for pairs marked in `lin`, the linear values)
  float lg[MAXMOL][2][2] = {}, dg[MAXMOL][2][2] = {};
  unsigned lin = 0u;
  bool anylin = false;
  CChunk cur, nxt;
  bool have = first_from(blockIdx.x, cur);
  if (have) read(cur, true);
  while (have) {
    bool have_next;
    if (cur.l0 + 32 < cur.o.l_end) {
      nxt = cur;
      nxt.l0 = cur.l0 + 32;
      read(nxt, false);
      have_next = true;
    } else {
      have_next = first_from(cur.u + gridDim.x, nxt);
      if (have_next) read(nxt, true);
    }
    const int N = cur.o.l_end, l0 = cur.l0;
    const int col = cur.o.tile * kOT + c2;
    const bool store = col < kcols, in_row = wbase + col < p.wn_pad;
    float* dst = kbuf + ((size_t)cur.o.bc * p.max_layers + l0) * kcols + col;
    if (l0 == cur.o.l_begin) cip = cit = citc = czone = -1;
    const SegFlags f = segment_flags<!EXPT>(cur.h, l0, cur.o.l_begin, N, lane, has_mol, has_cia,
                                            cip, cit, citc, czone);
    const float4 ha = cur.ha, hb = cur.hb;
    float ray0 = cur.ray.x, ray1 = cur.ray.y;
    const int n_here = min(32, N - l0);
    // K of one layer at this lane's two wavenumbers from the layer's coefficients, stored at dp
    auto one_layer = [&](float w0, float w1, float w2, float w3, float y0, float y1, float rho,
                         float kc, float* dp) {
      float k0 = fmaf(rho, ray0, kc), k1 = fmaf(rho, ray1, kc);
      if constexpr (EXPT) {
        // w0, w1: rho x_max (1 - t_P), rho x_max t_P; w2: exponential T weight u; w3: linear
        // T weight t.  At each P row 2^(lg + u dg) = 2^64 x_m s1^(1-u) s2^u.
        float m0 = 0.f, m1 = 0.f;
        if (!anylin) {
#pragma unroll
          for (int m = 0; m < MAXMOL; ++m) {
            if (m < p.n_mol) {
              const float g00 = ex2_fast(fmaf(w2, dg[m][0][0], lg[m][0][0]));
              const float g01 = ex2_fast(fmaf(w2, dg[m][0][1], lg[m][0][1]));
              const float g10 = ex2_fast(fmaf(w2, dg[m][1][0], lg[m][1][0]));
              const float g11 = ex2_fast(fmaf(w2, dg[m][1][1], lg[m][1][1]));
              m0 = fmaf(w0, g00, m0); m1 = fmaf(w0, g01, m1);
              m0 = fmaf(w1, g10, m0); m1 = fmaf(w1, g11, m1);
            }
          }
        } else {
#pragma unroll
          for (int m = 0; m < MAXMOL; ++m) {
            if (m < p.n_mol) {
              float g[2][2];
#pragma unroll
              for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                  const bool lb = (lin >> ((m * 2 + rr) * 2 + v)) & 1u;
                  const float e = fmaf(lb ? w3 : w2, dg[m][rr][v], lg[m][rr][v]);
                  g[rr][v] = lb ? e : ex2_fast(e);
                }
              m0 = fmaf(w0, g[0][0], m0); m1 = fmaf(w0, g[0][1], m1);
              m0 = fmaf(w1, g[1][0], m0); m1 = fmaf(w1, g[1][1], m1);
            }
          }
        }
        k0 = fmaf(m0, kExpScaleInv, k0); k1 = fmaf(m1, kExpScaleInv, k1);
      } else {
        k0 = fmaf(w0, us[0][0], k0); k1 = fmaf(w0, us[0][1], k1);
        k0 = fmaf(w1, us[1][0], k0); k1 = fmaf(w1, us[1][1], k1);
        k0 = fmaf(w2, us[2][0], k0); k1 = fmaf(w2, us[2][1], k1);
        k0 = fmaf(w3, us[3][0], k0); k1 = fmaf(w3, us[3][1], k1);
      }
      k0 = fmaf(y0, uc[0][0], k0); k1 = fmaf(y0, uc[0][1], k1);
      k0 = fmaf(y1, uc[1][0], k0); k1 = fmaf(y1, uc[1][1], k1);
      if (store)
        __stcs(reinterpret_cast<float2*>(dp), in_row ? make_float2(k0, k1) : make_float2(0.f, 0.f));
    };
    for (int i = 0; i < n_here;) {
      if ((f.start >> i) & 1u) {                       // a new segment: take its stage
        if (!EXPT && p.buf.zoned) {
          // two-layer gases: a segment in another chemistry zone takes that zone's weights
          const int zi = __shfl_sync(0xffffffffu, cur.h.w, i);
          if (zi != cur.zone) {
            const int b = p.b_off + cur.o.bc;
            const int w = wbase + col;
            cur.ray = in_row ? rayleigh2(p, b, zi, w) : make_float2(0.f, 0.f);
            item_weights<MAXMOL, MAXCIA>(p, b, zi, cur.xm, cur.yq);
            cur.zone = zi;
            ray0 = cur.ray.x; ray1 = cur.ray.y;
          }
        }
        bool ok;
        if constexpr (EXPT)
          ok = ring_consume_exp<kOT, MAXMOL, MAXCIA, F16>(p, rs, plan, ring, seg,
                                                          (f.mol >> i) & 1u, (f.cia >> i) & 1u,
                                                          c2, cur.xm, cur.yq, lg, dg, lin,
                                                          anylin, uc, lane);
        else
          ok = ring_consume<kOT, 2, MAXMOL, MAXCIA, F16>(p, rs, plan, ring, seg,
                                                         (f.mol >> i) & 1u, (f.cia >> i) & 1u,
                                                         c2, cur.xm, cur.yq, us, uc, lane);
        if (!ok) return;
        ++seg;
      }
      // two layers of one segment at a time (their shuffles and FMA chains interleave); the
      // exponential scheme keeps one layer per step (its register set would spill)
      const bool pair = !EXPT && i + 1 < n_here && !((f.start >> (i + 1)) & 1u);
      const float a0 = __shfl_sync(0xffffffffu, ha.x, i), a1 = __shfl_sync(0xffffffffu, ha.y, i);
      const float a2 = __shfl_sync(0xffffffffu, ha.z, i), a3 = __shfl_sync(0xffffffffu, ha.w, i);
      const float b0 = __shfl_sync(0xffffffffu, hb.x, i), b1 = __shfl_sync(0xffffffffu, hb.y, i);
      const float b2 = __shfl_sync(0xffffffffu, hb.z, i), b3 = __shfl_sync(0xffffffffu, hb.w, i);
      if (pair) {
        const int j = i + 1;
        const float e0 = __shfl_sync(0xffffffffu, ha.x, j), e1 = __shfl_sync(0xffffffffu, ha.y, j);
        const float e2 = __shfl_sync(0xffffffffu, ha.z, j), e3 = __shfl_sync(0xffffffffu, ha.w, j);
        const float f0 = __shfl_sync(0xffffffffu, hb.x, j), f1 = __shfl_sync(0xffffffffu, hb.y, j);
        const float f2 = __shfl_sync(0xffffffffu, hb.z, j), f3 = __shfl_sync(0xffffffffu, hb.w, j);
        one_layer(a0, a1, a2, a3, b0, b1, b2, b3, dst);
        one_layer(e0, e1, e2, e3, f0, f1, f2, f3, dst + kcols);
        dst += 2 * kcols;
        i += 2;
      } else {
        one_layer(a0, a1, a2, a3, b0, b1, b2, b3, dst);
        dst += kcols;
        i += 1;
      }
    }
    // the next chunk of the same unit continues with the zone weights this one ended with
    if (!EXPT && p.buf.zoned && have_next && nxt.u == cur.u) {
      nxt.ray = cur.ray;
      nxt.zone = cur.zone;
#pragma unroll
      for (int m = 0; m < MAXMOL; ++m) nxt.xm[m] = cur.xm[m];
#pragma unroll
      for (int q = 0; q < MAXCIA; ++q) nxt.yq[q] = cur.yq[q];
    }
    cur = nxt;
    have = have_next;
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

// Layer blocks per (item, wavenumber tile) unit of the opacity kernel: 1 unless there are
// fewer units than resident CTAs (a narrow wavenumber range of a few items), where splitting
// the layers (blocks of at least 8) gives the idle CTAs work.  Measured on the full-size
// single atmosphere (782 units, 456 CTAs), splitting to even out the last pass over the grid
// costs more in repeated segment loads and unit start-up than it saves.
int opacity_layer_blocks(long long units, long long slots, int max_layers) {
  if (units <= 0 || 2 * units > slots) return 1;
  const long long n = std::min<long long>(8, slots / units);
  return (int)std::max<long long>(1, std::min<long long>(n, max_layers / 8));
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

template <int MAXMOL, int MAXCIA, bool F16, bool EXPT = false>
cudaError_t launch_opacity_t(const FwdParams& p, const CUtensorMap& sig, const CUtensorMap& cia,
                             int Bc, float* kbuf, long long kcols, int per_sm_cap,
                             cudaStream_t s) {
  auto kern = k_opacity<MAXMOL, MAXCIA, F16, EXPT>;
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
  const long long units0 = (long long)Bc * n_tiles;
  const long long slots = (long long)sm_count() * per_sm;
  const int n_lb = opacity_layer_blocks(units0, slots, p.max_layers);
  const int lb_size = (p.max_layers + n_lb - 1) / n_lb;
  const long long units = units0 * n_lb;
  const int grid = (int)std::min<long long>(units, slots);
  kern<<<grid, kOThreads, smem, s>>>(p, sig, cia, kbuf, kcols, Bc, n_tiles, stages, n_lb,
                                     lb_size);
  return cudaGetLastError();
}

template <bool F16>
cudaError_t launch_opacity_p(const FwdParams& p, const CUtensorMap& sig, const CUtensorMap& cia,
                             int Bc, float* kbuf, long long kcols, int cap, cudaStream_t s) {
  static_assert(TR_MAX_MOL == 8 && TR_MAX_CIA == 4, "opacity instantiations cover the limits");
  if (p.interp_mode == TR_INTERP_EXP) {              // exponential T scheme (Sec. 5)
    if (p.n_mol <= 2) return launch_opacity_t<2, 4, F16, true>(p, sig, cia, Bc, kbuf, kcols, cap, s);
    if (p.n_mol <= 5) return launch_opacity_t<5, 4, F16, true>(p, sig, cia, Bc, kbuf, kcols, cap, s);
    return launch_opacity_t<8, 4, F16, true>(p, sig, cia, Bc, kbuf, kcols, cap, s);
  }
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
// into one of up to three tile slots, plus the item's packed path lengths and annulus weights by
// bulk copy when the item changes (after every earlier unit is done with them).  The W
// contraction warps take work items (unit, 16-ray tile) from a shared counter, a unit's longest
// tile first: tau = DL K for the tile's rays and its partial depth sum_j a_j (1 - e^-tau_j),
// stored per tile.  The warp that completes a unit's last tile adds the tiles' partials in
// tile order (a fixed order: the result does not depend on which warp took which tile),
// adds (R_p/R_s)^2 in FP64, writes the depths and hands the slot back to the producer.  No
// barrier over the CTA's warps: tiles of different lengths and units overlap freely.
constexpr int kCB = 8;                           // K rows per TMA box
constexpr int kMaxSlots = 3;                     // K-tile slots (units in flight per CTA)

struct ContractLayout {                          // dynamic shared memory (128-byte aligned)
  uint32_t ktb, slot, dl, aj, total;             // slot i: K tile at i*slot, partials at +ktb
  __host__ __device__ ContractLayout(int max_layers, int n_slots) {
    ktb = (uint32_t)pad8(max_layers) * kTW * 4;
    const uint32_t ptb = (uint32_t)((max_layers + kRT - 1) / kRT) * kTW * 4;
    slot = ktb + ptb;
    dl = (uint32_t)n_slots * slot;
    aj = dl + (((uint32_t)dlp_offset(max_layers) * 4 + 127u) & ~127u);
    total = aj + (((uint32_t)pad8(max_layers) * 4 + 127u) & ~127u) + 128u;
  }
};

// Bounded wait until *slot_unit == k (or the CTA aborts); false on a timeout or abort.
__device__ __forceinline__ bool wait_slot(const int* slot_unit, int k, const int* abort_flag,
                                          int* dev_err) {
  for (long long i = 0; i < kMaxPolls; ++i) {
    if (*(const volatile int*)slot_unit == k) return true;
    if (*(const volatile int*)abort_flag) return false;
    __nanosleep(64);
  }
  atomicOr(dev_err, TR_DEVERR_TIMEOUT);
  return false;
}

template <int W>
__global__ void __launch_bounds__(32 * (W + 1), 1)
k_contract_fp32(FwdParams p, const __grid_constant__ CUtensorMap tm_k, long long kcols, int Bc,
                int n_tiles, int n_slots) {
  extern __shared__ unsigned char csm_raw[];
  __shared__ __align__(8) uint64_t kfull[kMaxSlots], kempty[kMaxSlots];
  __shared__ int abort_flag, next_item, done[kMaxSlots], slot_unit[kMaxSlots];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ContractLayout lay(p.max_layers, n_slots);
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(csm_raw) + 127) & ~(uintptr_t)127);
  float* const DLP = reinterpret_cast<float*>(base + lay.dl);
  float* const a_s = reinterpret_cast<float*>(base + lay.aj);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kMaxSlots; ++i) {
      mbar_init(&kfull[i], 1); mbar_init(&kempty[i], 1);
      done[i] = 0;
      slot_unit[i] = i;                                 // units 0 .. S-1 go to slots 0 .. S-1
    }
    abort_flag = 0;
    next_item = 0;
    mbar_fence_init();
  }
  __syncthreads();
  // units of one chunk fit in 32 bits: the K buffer (2 GiB) bounds Bc x n_tiles x kTW x 4 B
  const int units = Bc * n_tiles;
  const int per = (units + (int)gridDim.x - 1) / (int)gridDim.x;
  const int u_begin = (int)blockIdx.x * per;
  const int u_end = u_begin + per < units ? u_begin + per : units;
  const int n_units = u_end > u_begin ? (int)(u_end - u_begin) : 0;
  const int rt_max = (p.max_layers + kRT - 1) / kRT;   // work items per unit
  const int wbase = wn_first(p.wn_begin);
  const int S = n_slots;

  if (warp == W) {
    // ---------------- producer
    if (lane != 0) return;
    int dl_item = -1;
    int k = 0;
    for (; k < n_units; ++k) {
      const int u = u_begin + k;
      const int bc = u / n_tiles, tile = u - bc * n_tiles;
      const int b = p.b_off + bc;
      const int N = p.buf.items[b].n_layers;
      const int sl = k % S, q = k / S;
      bool ok = q == 0 || mbar_wait_bounded(&kempty[sl], (q - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
      const bool new_item = N > 0 && b != dl_item;
      // the units in the other slots must be done with the path lengths too
      for (int d = 1; ok && new_item && d < S && d <= k; ++d) {
        const int kp = k - d;
        ok = mbar_wait_bounded(&kempty[kp % S], (kp / S) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
      }
      if (!ok || *(volatile int*)&abort_flag) { atomicExch(&abort_flag, 1); break; }
      if (N == 0) { mbar_arrive(&kfull[sl]); continue; }   // nothing to load
      const int nbox = (N + kCB - 1) / kCB;
      uint32_t bytes = (uint32_t)nbox * kCB * kTW * 4;
      if (new_item) bytes += (uint32_t)(dlp_offset(N) * 4 + p.buf.npad * 4);
      mbar_arrive_expect_tx(&kfull[sl], bytes);
      float* Kt = reinterpret_cast<float*>(base + sl * lay.slot);
      for (int i = 0; i < nbox; ++i)
        tma_load_2d(Kt + (size_t)i * kCB * kTW, &tm_k, tile * kTW, bc * p.max_layers + i * kCB,
                    &kfull[sl]);
      if (new_item) {
        bulk_g2s(DLP, p.buf.dlp + (size_t)b * dlp_offset(p.max_layers),
                 (uint32_t)(dlp_offset(N) * 4), &kfull[sl]);
        bulk_g2s(a_s, p.buf.aj + (size_t)b * p.buf.npad, (uint32_t)(p.buf.npad * 4), &kfull[sl]);
        dl_item = b;
      }
    }
    // every copy issued has landed before the CTA may exit
    for (int i = 0; i < S && i < k; ++i) {
      const int kl = k - 1 - i;
      mbar_wait_bounded(&kfull[kl % S], (kl / S) & 1, nullptr, 0);
    }
    return;
  }

  // ---------------- contraction warps
  const int n_items = n_units * rt_max;
  while (true) {
    int it = 0;
    if (lane == 0) it = atomicAdd(&next_item, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const int k = it / rt_max, t = it - k * rt_max;
    const int u = u_begin + k;
    const int bc = u / n_tiles, tile = u - bc * n_tiles;
    const int b = p.b_off + bc;
    const ItemGeom ig = p.buf.items[b];
    const int N = ig.n_layers;
    const int n_rt = (N + kRT - 1) / kRT;
    const int target = n_rt > 0 ? n_rt : 1;            // work items that count for the unit
    if (t >= target) continue;                          // beyond this item's rays
    const int sl = k % S, q = k / S;
    // the slot holds unit k - S until that unit's last tile hands it over; only then is
    // phase q the one kfull[sl] is in (a warp may take work of later units early)
    const bool ok = __all_sync(0xffffffffu, wait_slot(&slot_unit[sl], k, &abort_flag, p.dev_err) &&
                                                mbar_wait_bounded(&kfull[sl], q & 1, p.dev_err,
                                                                  TR_DEVERR_TIMEOUT) &&
                                                !*(volatile int*)&abort_flag);
    if (!ok) { if (lane == 0) atomicExch(&abort_flag, 1); return; }
    float* part = reinterpret_cast<float*>(base + sl * lay.slot + lay.ktb);
    if (N > 0) {
      float pt[4];
      contract_tile(N, t * kRT, reinterpret_cast<const float*>(base + sl * lay.slot), DLP, a_s, pt);
      *reinterpret_cast<float4*>(part + t * kTW + 4 * lane) = make_float4(pt[0], pt[1], pt[2], pt[3]);
    }
    __syncwarp();
    int prev = 0;
    if (lane == 0) {
      __threadfence_block();
      prev = atomicAdd(&done[sl], 1);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != target - 1) continue;
    // ---- last tile of the unit: depths = (R_p/R_s)^2 + sum over tiles in tile order
    __threadfence_block();
    const int w0 = wbase + tile * kTW + 4 * lane;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int w = w0 + c;
      if (w >= p.wn_begin && w < p.wn_begin + p.wn_count) {
        float s = 0.f;
        for (int i = 0; i < n_rt; ++i) s += part[i * kTW + 4 * lane + c];
        p.out[(long long)b * p.out_stride + (w - p.wn_begin)] = N > 0 ? ig.rp2_rs2 + (double)s : 0.0;
      }
    }
    __syncwarp();
    if (lane == 0) {
      done[sl] = 0;
      *(volatile int*)&slot_unit[sl] = k + S;           // the slot's next unit
      __threadfence_block();
      mbar_arrive(&kempty[sl]);                         // the slot is free again
    }
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

long long forward_kcols(int wn_begin, int wn_count) {
  const int w_first = wn_first(wn_begin);
  return (long long)((wn_begin + wn_count - w_first + kTW - 1) / kTW) * kTW;
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

template <int W>
cudaError_t launch_contract_t(const FwdParams& p, const CUtensorMap& tm, long long kcols, int Bc,
                              int tiles, int slots, uint32_t smem, cudaStream_t s) {
  auto kern = k_contract_fp32<W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (W + 1), smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const long long units = (long long)Bc * tiles;
  // the kernel counts units and (unit, ray tile) work items in 32 bits
  if (units * ((p.max_layers + kRT - 1) / kRT) > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(units, (long long)sm_count());
  kern<<<grid, 32 * (W + 1), smem, s>>>(p, tm, kcols, Bc, tiles, slots);
  return cudaGetLastError();
}

int contract_kind(int requested, int max_layers) {
  if (requested != kContractAuto) return requested;
  return tc_contract_fits(max_layers) ? kContractTC : kContractFfma8;
}

cudaError_t launch_contract_fp32(const FwdParams& p, int Bc, const float* kbuf, int kind,
                                 const void* dl_tiles, cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  kind = contract_kind(kind, p.max_layers);
  if (kind == kContractTC) return launch_contract_tc(p, Bc, kbuf, dl_tiles, s);
  const int tiles = n_tiles_of(p);
  const long long kcols = (long long)tiles * kTW;
  CUtensorMap tm{};
  if (!encode_2d_f32(&tm, kbuf, (unsigned long long)kcols,
                     (unsigned long long)Bc * p.max_layers, (unsigned long long)kcols * 4, kTW,
                     kCB))
    return cudaErrorInvalidValue;
  constexpr uint32_t kSmemMax = 227u * 1024u;
  // as many K-tile slots as fit, up to three (the next units' loads overlap the contraction)
  int slots = kMaxSlots;
  while (slots > 1 && ContractLayout(p.max_layers, slots).total > kSmemMax) --slots;
  const uint32_t smem = ContractLayout(p.max_layers, slots).total;
  if (smem > kSmemMax) return cudaErrorInvalidConfiguration;
  // eleven contraction warps (twelve plus the producer would be held to 128 registers and
  // spill; eleven keep 168), or eight
  if (kind == kContractFfma11) return launch_contract_t<11>(p, tm, kcols, Bc, tiles, slots, smem, s);
  return launch_contract_t<8>(p, tm, kcols, Bc, tiles, slots, smem, s);
}

}  // namespace tr
