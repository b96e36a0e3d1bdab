// adjoint.cu -- hand-written reverse-mode derivative of the batched forward model (the paper
// has no gradient path; this serves gradient-based samplers and Fisher matrices).
//
// Forward (recalled):  K_l(v) = sum_m w_ml sigma_m(P_l, T_l; v) + rho_l R(v)
//                              + sum_q c_ql sigma_q(T_l; v) + kappa c_l          (Sec. 4.4, 8.1)
//                      tau_j(v) = sum_{l>=j} DL[j][l] K_l(v)                     (Sec. 4)
//                      D(v) = (R_p/R_s)^2 + sum_j a_j (1 - e^{-tau_j(v)})        (Sec. 4)
//                      D_bin,k = sum_v w_kv D(v) / sum_v w_kv                    (Sec. 4.5)
// Backward, given G_bin = dL/dD_bin (chi^2: 2 (D_bin - obs) / sigma^2):
//   G_D(v)    = sum_k G_bin,k w_kv / sum w_k                    (k_gd)
//   G_tau_j   = G_D a_j e^{-tau_j};  G_a_j = sum_v G_D (1 - e^{-tau_j})
//   G_K_l(v)  = sum_{j<=l} DL[j][l] G_tau_j(v);  G_DL[j][l] = sum_v G_tau_j(v) K_l(v)
//   per layer: sum_v G_K sigma_m, sum_v G_K dsigma_m/dT, sum_v G_K sigma_R,s, CIA alike,
//              sum_v G_K                                          (k_adjoint_tile, FP32:
//              K is the forward's, read back from the workspace's K buffer when that holds
//              the whole batch, and recomputed from the tables when the batch outgrows it,
//              with the opacity kernel's per-cell sums and per-layer FMAs, so bit for bit; tau
//              is recomputed; with mixed precision the cross-sections come from the FP16
//              log10 tables, decoded on the fly, and the forward runs the mixed path)
//   then, per atmosphere (FP64 sums; the path-length terms in FP32 from double-float
//   altitudes): path lengths and annulus weights -> radii, the hydrostatic recursion,
//   densities, chemistry, temperature nodes, R_p and the cloud top (k_adjoint_item).  Tile partial sums are added in a fixed order: results are
//   deterministic.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cuda_fp16.h>
#include "tma.h"
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kAT = 64;           // wavenumbers per adjoint CTA (2 per lane)
constexpr int kAThreads = 256;
constexpr int kAWarps = kAThreads / 32;
constexpr int kRT = 8;            // rays (or layers) per register tile
constexpr int kItemThreads = 128;

// Float index of element (row, c) of the [rows][kAT] K and G_tau tiles: a row's 16-byte chunks
// are XOR-swizzled by row / 4, so the G_DL blocks' float4 reads of rows 4 apart (one per
// thread) fall in different banks; a lane's float2 stays inside one chunk.
__device__ __forceinline__ int tix(int row, int c) {
  return row * kAT + ((((c >> 2) ^ (row >> 2)) & (kAT / 4 - 1)) << 2) + (c & 3);
}

struct AdjParams {
  FwdParams f;                    // tables and item buffers; wn_begin / wn_count = binned range
  const double* inv_dt;           // [n_t - 1]
  const double* inv_dtc;          // [n_t_cia - 1]
  const float* gd;                // [B][n_in] dL/dD at the native wavenumbers of the range
  int n_in, tiles, n_feat;
  float* part_a;                  // [B][tiles][npad]
  float* part_dl;                 // [B][tiles][npad][npad]  (ray j, shell l), j <= l
  float* part_f;                  // [B][tiles][max_layers][n_feat]
  float* part_rp;                 // [B][tiles]  sum_v G_D
  const float* kstore;            // the forward's K of the whole batch, or NULL: recompute
  long long kcols;                // columns of a K row in kstore
  int tile0;                      // wavenumber tile of blockIdx.x == 0 (tiles = those launched)
  // Jacobian row: >= 0 takes dL/dD from the bins' weights of this one bin (the row of
  // dD_bin/dtheta), ignoring gd; -1 reads gd
  int jac_bin;
  const int* t_ptr; const int* t_bin; const double* t_w;   // the bins' transpose (BinsDev)
};

__device__ __forceinline__ float4 as_float4(int4 v) {
  return make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z),
                     __int_as_float(v.w));
}
// kLayer* flags of a layer descriptor from its third 16 bytes (k_cloud, cloud, pad_s + flags +
// pad_c, pad_f): the flags byte is byte 10 of the 16
__device__ __forceinline__ unsigned d_flags(int4 v) { return ((unsigned)v.z >> 16) & 0xffu; }
static_assert(offsetof(LayerDesc, flags) == 42 && offsetof(LayerDesc, tp) == 20,
              "layer descriptor offsets the header loads assume");

// Packed FP32 pairs beyond ffma2 (sm_100 and later): pack2(lo, hi) forms the pair, unpack2
// returns its halves; fma2, add2, sub2 and mul2 act on each half, rounded as the scalar
// operation would be.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

__device__ __forceinline__ float2 ldg2(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}

constexpr float kLog2Of10a = 3.32192809488736234787f;

// Two adjacent cross-sections of molecule m at element offset `off` of its table: the FP32
// table, or (F16) the FP16 log10 table decoded, sigma = 10^(h + c_m) by the hardware 2^x.
template <bool F16>
__device__ __forceinline__ float2 sig2(const FwdParams& p, int m, size_t off) {
  if constexpr (F16) {
    const __half2 h = __ldg(reinterpret_cast<const __half2*>(
        reinterpret_cast<const __half*>(p.logsig16) + off));
    const float2 f = __half22float2(h);
    const float c = p.logsig_off[m];
    float a, b;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"((f.x + c) * kLog2Of10a));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(b) : "f"((f.y + c) * kLog2Of10a));
    return make_float2(a, b);
  } else {
    return ldg2(p.sigma + off);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The layer-independent Rayleigh sum sum_s c_s sigma_R,s at wavenumbers w2, w2+1 (zone 0).
__device__ __forceinline__ float2 rayleigh_sum2(const FwdParams& p, int b, int w2) {
  float2 ray = make_float2(0.f, 0.f);
  if (p.ray) {
    const float* rc = p.buf.rayc + (size_t)b * kMaxZones * TR_MAX_SPECIES;   // zone 0
    for (int s = 0; s < p.n_species; ++s) {
      const float c = rc[s];
      if (c != 0.f) {
        const float2 v = ldg2(p.ray + (size_t)s * p.wn_pad + w2);
        ray.x = fmaf(c, v.x, ray.x); ray.y = fmaf(c, v.y, ray.y);
      }
    }
  }
  return ray;
}

// floats per feature row of a warp's reduction buffer: a multiple of 4 (rows read as float4)
// with rows 4 banks apart, so neither the lanes' column writes nor the 8-lane phases of the
// float4 row reads conflict
constexpr int kRedPitch = 36;

struct AdjSmem {
  int npad, kt_rows, n_feat;
  // the tile's Rayleigh rows (layer-independent) are staged once: TR_MAX_SPECIES x kAT floats
  __host__ __device__ AdjSmem(int max_layers, int nf)
      : npad(pad8(max_layers)), kt_rows(max_layers), n_feat(nf) {}
  // the warps' reduction buffers of the feature phase reuse the K tile's space (K is not
  // read after the G_DL phase) when they fit there, else follow the other buffers
  __host__ __device__ size_t red_floats() const { return (size_t)kAWarps * n_feat * kRedPitch; }
  __host__ __device__ bool red_in_kt() const { return red_floats() <= (size_t)kt_rows * kAT; }
  __host__ __device__ size_t floats() const {
    return (size_t)kt_rows * kAT + (size_t)npad * npad + npad + (size_t)npad * kAT + kAT +
           (size_t)TR_MAX_SPECIES * kAT + (red_in_kt() ? 0 : red_floats());
  }
};

// RECOMP: K recomputed from the tables (a.kstore is NULL) or read from the forward's buffer;
// instantiated separately, so each form's registers are allocated for its own K phase.
template <int MAXMOL, bool F16, bool RECOMP>
__global__ void __launch_bounds__(kAThreads, 2)
k_adjoint_tile(AdjParams a) {
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) uint64_t bar;
  const FwdParams& p = a.f;
  const int b = blockIdx.y, tile = blockIdx.x;        // tile: index among the launched tiles
  const int N = p.buf.items[b].n_layers;
  if (N == 0) return;                                   // the item kernel zeroes its gradient
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const AdjSmem sp(p.max_layers, a.n_feat);
  const int npad = sp.npad;
  float* Kt = smem;                                     // [max_layers][kAT]
  float* DLT = Kt + (size_t)sp.kt_rows * kAT;           // [npad][npad], rows l, columns j
  float* a_s = DLT + (size_t)npad * npad;               // [npad]
  float* Gt = a_s + npad;                               // [npad][kAT]  G_tau
  float* gd_s = Gt + (size_t)npad * kAT;                // [kAT]
  float* ray_s = gd_s + kAT;                            // [TR_MAX_SPECIES][kAT] Rayleigh rows
  // per warp: one layer's per-lane feature terms [n_feat][kRedPitch], summed over lanes by
  // columns (lane f adds feature f's 32 terms in lane order); in the K tile's space when
  // that holds them
  float* red = (sp.red_in_kt() ? Kt : ray_s + (size_t)TR_MAX_SPECIES * kAT) +
               (size_t)warp * a.n_feat * kRedPitch;
  const int w_first = wn_first(p.wn_begin) + (a.tile0 + tile) * kAT;

  if (threadIdx.x == 0) { mbar_init(&bar, 1); mbar_fence_init(); }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)(sizeof(float) * ((size_t)N * npad + npad));
    mbar_arrive_expect_tx(&bar, bytes);
    bulk_g2s(DLT, p.buf.dlt + (size_t)b * p.max_layers * npad,
             (uint32_t)(sizeof(float) * (size_t)N * npad), &bar);
    bulk_g2s(a_s, p.buf.aj + (size_t)b * npad, (uint32_t)(sizeof(float) * npad), &bar);
  }
  for (int i = N * npad + threadIdx.x; i < npad * npad; i += kAThreads) DLT[i] = 0.f;
  for (int i = threadIdx.x; i < kAT; i += kAThreads) {
    const int w = w_first + i;
    float g = 0.f;
    if (w >= p.wn_begin && w < p.wn_begin + a.n_in) {
      const int k = w - p.wn_begin;
      if (a.jac_bin < 0) {
        g = a.gd[(size_t)b * a.n_in + k];
      } else {                                          // dD_bin,jac_bin / dD at w
        for (int e = a.t_ptr[k]; e < a.t_ptr[k + 1]; ++e)
          if (a.t_bin[e] == a.jac_bin) g = (float)a.t_w[e];
      }
    }
    gd_s[i] = g;
  }
  if (p.ray) {                                          // the Rayleigh rows of this tile
    for (int i = threadIdx.x; i < p.n_species * kAT; i += kAThreads) {
      const int sp2 = i / kAT, c = i - sp2 * kAT, w = w_first + c;
      ray_s[i] = w < p.wn_pad ? __ldg(p.ray + (size_t)sp2 * p.wn_pad + w) : 0.f;
    }
  }
  // ---- K tile: the forward's, when its buffer holds the whole batch; else recomputed
  const int w2 = w_first + 2 * lane;
  const bool in_row = w2 < p.wn_pad;
  const LayerDesc* LD = p.buf.layers + (size_t)b * p.max_layers;
  if constexpr (!RECOMP) {
    const float* ks = a.kstore + (size_t)b * p.max_layers * a.kcols + (size_t)(a.tile0 + tile) * kAT + 2 * lane;
    for (int l = warp; l < N; l += kAWarps)
      *reinterpret_cast<float2*>(Kt + tix(l, 2 * lane)) =
          __ldg(reinterpret_cast<const float2*>(ks + (size_t)l * a.kcols));
  } else {
    // K recomputed with the opacity kernel's arithmetic, so that it equals the stored K bit
    // for bit: per (P, T) cell the molecule sums us_c = sum_m (x_m / x_max) sigma_m,c and per
    // CIA bracket the pair sums uc_t = sum_q (y_q / y_max) sigma_q,t, in species order; per
    // layer kc + rho sigma_R + sum_c w_c us_c + sum_t y_t uc_t with the layer's coefficients
    // (Sec. 5, Sec. 8.1).  Each warp takes a contiguous run of layers, reads their brackets
    // and coefficients 32 layers per warp-wide load, and gathers a cell's corner rows only
    // when the cell changes (consecutive layers share it).
    const float2 ray = in_row ? rayleigh_sum2(p, b, w2) : make_float2(0.f, 0.f);
    const float* ox = p.buf.opx + (size_t)b * kMaxZones * kOpxStride;     // zone 0 weights
    const float4* opb = p.buf.op + (size_t)b * p.max_layers * 2;
    const size_t slab_t = (size_t)p.wn_pad, slab_p = (size_t)p.n_t * p.wn_pad;
    const int wq = in_row ? w2 : 0;
    const int per = (N + kAWarps - 1) / kAWarps;
    const int lb = min(N, warp * per), le = min(N, lb + per);
    int c_ip = -1, c_it = -1, c_itc = -1;
    float us[4][2] = {}, uc[2][2] = {};
    for (int l0 = lb; l0 < le; l0 += 32) {
      const int li = l0 + lane;
      int4 h = make_int4(0, 0, 0, 0);
      float4 ha = make_float4(0.f, 0.f, 0.f, 0.f), hb = ha;
      if (li < le) {
        h = __ldg(reinterpret_cast<const int4*>(LD + li));      // ip, it, itc, zone
        ha = __ldg(opb + 2 * li);
        hb = __ldg(opb + 2 * li + 1);
      }
      const int n_here = min(32, le - l0);
      for (int i = 0; i < n_here; ++i) {
        const int ip = __shfl_sync(0xffffffffu, h.x, i), it = __shfl_sync(0xffffffffu, h.y, i);
        const int itc = __shfl_sync(0xffffffffu, h.z, i);
        if (ip != c_ip || it != c_it) {                  // a new cell (warp-uniform)
          const size_t o0 = ((size_t)ip * p.n_t + it) * p.wn_pad + wq;
#pragma unroll
          for (int c = 0; c < 4; ++c) us[c][0] = us[c][1] = 0.f;
#pragma unroll
          for (int m = 0; m < MAXMOL; ++m) {
            if (m < p.n_mol) {
              const float xm = __ldg(ox + m);
              const size_t om = o0 + (size_t)m * p.n_p * slab_p;
              const float2 v0 = sig2<F16>(p, m, om), v1 = sig2<F16>(p, m, om + slab_t),
                           v2 = sig2<F16>(p, m, om + slab_p),
                           v3 = sig2<F16>(p, m, om + slab_p + slab_t);
              us[0][0] = fmaf(xm, v0.x, us[0][0]); us[0][1] = fmaf(xm, v0.y, us[0][1]);
              us[1][0] = fmaf(xm, v1.x, us[1][0]); us[1][1] = fmaf(xm, v1.y, us[1][1]);
              us[2][0] = fmaf(xm, v2.x, us[2][0]); us[2][1] = fmaf(xm, v2.y, us[2][1]);
              us[3][0] = fmaf(xm, v3.x, us[3][0]); us[3][1] = fmaf(xm, v3.y, us[3][1]);
            }
          }
          c_ip = ip; c_it = it;
        }
        if (p.n_cia > 0 && itc != c_itc) {              // a new CIA bracket (warp-uniform)
          uc[0][0] = uc[0][1] = uc[1][0] = uc[1][1] = 0.f;
#pragma unroll
          for (int q = 0; q < TR_MAX_CIA; ++q) {
            if (q < p.n_cia) {
              const float yq = __ldg(ox + TR_MAX_MOL + q);
              const float* bq = p.cia + ((size_t)q * p.n_t_cia + itc) * p.wn_pad + wq;
              const float2 c0 = ldg2(bq), c1 = ldg2(bq + p.wn_pad);
              uc[0][0] = fmaf(yq, c0.x, uc[0][0]); uc[0][1] = fmaf(yq, c0.y, uc[0][1]);
              uc[1][0] = fmaf(yq, c1.x, uc[1][0]); uc[1][1] = fmaf(yq, c1.y, uc[1][1]);
            }
          }
          c_itc = itc;
        }
        const float w0 = __shfl_sync(0xffffffffu, ha.x, i), w1 = __shfl_sync(0xffffffffu, ha.y, i);
        const float wc2 = __shfl_sync(0xffffffffu, ha.z, i), w3 = __shfl_sync(0xffffffffu, ha.w, i);
        const float y0 = __shfl_sync(0xffffffffu, hb.x, i), y1 = __shfl_sync(0xffffffffu, hb.y, i);
        const float rho = __shfl_sync(0xffffffffu, hb.z, i), kc = __shfl_sync(0xffffffffu, hb.w, i);
        float k0 = fmaf(rho, ray.x, kc), k1 = fmaf(rho, ray.y, kc);
        k0 = fmaf(w0, us[0][0], k0); k1 = fmaf(w0, us[0][1], k1);
        k0 = fmaf(w1, us[1][0], k0); k1 = fmaf(w1, us[1][1], k1);
        k0 = fmaf(wc2, us[2][0], k0); k1 = fmaf(wc2, us[2][1], k1);
        k0 = fmaf(w3, us[3][0], k0); k1 = fmaf(w3, us[3][1], k1);
        k0 = fmaf(y0, uc[0][0], k0); k1 = fmaf(y0, uc[0][1], k1);
        k0 = fmaf(y1, uc[1][0], k0); k1 = fmaf(y1, uc[1][1], k1);
        *reinterpret_cast<float2*>(Kt + tix(l0 + i, 2 * lane)) =
            in_row ? make_float2(k0, k1) : make_float2(0.f, 0.f);
      }
    }
  }
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, p.dev_err, TR_DEVERR_TIMEOUT));
  if (!ok) { mbar_wait_bounded(&bar, 0, nullptr, 0); return; }

  const size_t item_tile = (size_t)b * a.tiles + tile;
  // ---- tau, G_tau = G_D a_j e^-tau, G_a_j = sum_v G_D (1 - e^-tau)
  const float2 g2 = *reinterpret_cast<const float2*>(gd_s + 2 * lane);
  const int n_rt = (N + kRT - 1) / kRT;
  for (int round = 0;; ++round) {
    const int pos = (round & 1) ? (kAWarps - 1 - warp) : warp;
    const int rt = round * kAWarps + pos;
    if (rt >= n_rt) break;
    const int j0 = rt * kRT;
    // packed FP32 pairs: rays (2r, 2r+1) at the lane's two wavenumbers
    unsigned long long acc2[kRT / 2][2];
#pragma unroll
    for (int r = 0; r < kRT / 2; ++r) acc2[r][0] = acc2[r][1] = 0ull;
    for (int l = j0; l < N; ++l) {
      const float2 kv = *reinterpret_cast<const float2*>(Kt + tix(l, 2 * lane));
      const ulonglong2 d0 = *reinterpret_cast<const ulonglong2*>(DLT + (size_t)l * npad + j0);
      const ulonglong2 d1 = *reinterpret_cast<const ulonglong2*>(DLT + (size_t)l * npad + j0 + 4);
      const unsigned long long dv[4] = {d0.x, d0.y, d1.x, d1.y};
      const unsigned long long k0 = pack_dup(kv.x), k1 = pack_dup(kv.y);
#pragma unroll
      for (int r = 0; r < kRT / 2; ++r) { ffma2(acc2[r][0], dv[r], k0); ffma2(acc2[r][1], dv[r], k1); }
    }
    float acc[kRT][2];
#pragma unroll
    for (int r = 0; r < kRT / 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c)
        asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[2 * r][c]), "=f"(acc[2 * r + 1][c]) : "l"(acc2[r][c]));
#pragma unroll
    for (int r = 0; r < kRT; ++r) {
      const int j = j0 + r;
      const float aj = a_s[j];
      const float e0 = __expf(-acc[r][0]), e1 = __expf(-acc[r][1]);
      *reinterpret_cast<float2*>(Gt + tix(j, 2 * lane)) = make_float2(g2.x * aj * e0, g2.y * aj * e1);
      const float ga = warp_sum(g2.x * (1.f - e0) + g2.y * (1.f - e1));
      if (lane == 0) a.part_a[item_tile * npad + j] = ga;
    }
  }
  for (int j = N + threadIdx.x; j < npad; j += kAThreads) {
    for (int c = 0; c < kAT; ++c) Gt[(size_t)j * kAT + c] = 0.f;
    a.part_a[item_tile * npad + j] = 0.f;
  }
  if (warp == 0) {
    const float s = warp_sum(g2.x + g2.y);
    if (lane == 0) a.part_rp[item_tile] = s;
  }
  __syncthreads();

  // ---- G_DL[j][l] = sum_v G_tau_j(v) K_l(v), j <= l, 4 x 4 blocks
  {
    const int nb = (N + 3) / 4;
    const int n_pairs = nb * (nb + 1) / 2;
    float* pdl = a.part_dl + item_tile * (size_t)npad * npad;
    for (int pi = threadIdx.x; pi < n_pairs; pi += kAThreads) {
      int lb = (int)((sqrtf(8.f * pi + 1.f) - 1.f) * 0.5f);
      while (lb * (lb + 1) / 2 > pi) --lb;
      while ((lb + 1) * (lb + 2) / 2 <= pi) ++lb;
      const int jb = pi - lb * (lb + 1) / 2;
      const int j0 = 4 * jb, l0 = 4 * lb;
      // packed FP32 pairs: acc2[x][y] holds the even- and odd-wavenumber halves of the sum
      unsigned long long acc2[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x) acc2[x][0] = acc2[x][1] = acc2[x][2] = acc2[x][3] = 0ull;
      for (int c = 0; c < kAT; c += 4) {
        ulonglong2 g[4], k[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          g[x] = *reinterpret_cast<const ulonglong2*>(Gt + tix(j0 + x, c));
          k[x] = (l0 + x < N) ? *reinterpret_cast<const ulonglong2*>(Kt + tix(l0 + x, c))
                              : make_ulonglong2(0ull, 0ull);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            ffma2(acc2[x][y], g[x].x, k[y].x);
            ffma2(acc2[x][y], g[x].y, k[y].y);
          }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int j = j0 + x, l = l0 + y;
          float e0, e1;
          asm("mov.b64 {%0, %1}, %2;" : "=f"(e0), "=f"(e1) : "l"(acc2[x][y]));
          if (j <= l && l < N) pdl[(size_t)j * npad + l] = e0 + e1;
        }
    }
  }

  // ---- G_K_l(v) = sum_{j<=l} DL[j][l] G_tau_j(v) over 8-layer tiles, then per-layer sums
  if (sp.red_in_kt()) __syncthreads();                 // every warp is done reading K
  const int n_lt = (N + kRT - 1) / kRT;
  const int nm = p.n_mol, ns = p.ray ? p.n_species : 0, nq = p.n_cia;
  const int f_dS = nm, f_R = 2 * nm, f_C = 2 * nm + p.n_species, f_dC = f_C + nq, f_K = f_dC + nq;
  // a tile's cost grows with its layer index (the contraction runs over j <= l), so the warps
  // take the tiles from the top down, in a snake over the warps: the largest tiles first, then
  // the smallest ones to the warps that took the smaller of the large ones
  for (int round = 0;; ++round) {
    const int pos = (round & 1) ? (kAWarps - 1 - warp) : warp;
    const int kt = round * kAWarps + pos;
    if (kt >= n_lt) break;
    const int lt = n_lt - 1 - kt;
    const int l0 = lt * kRT;
    // the tile's layer headers, lane r < kRT holding layer l0 + r's (brackets, weights, flags
    // and reciprocal T spacings), loaded before the contraction so that their latency
    // overlaps it; each layer below takes them by shuffle
    int4 hb = make_int4(0, 0, 0, 0);
    float4 hw = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned hfl = 0u;
    float hidt = 0.f, hidc = 0.f;
    if (lane < kRT && l0 + lane < N) {
      const int4* dd = reinterpret_cast<const int4*>(LD + l0 + lane);
      hb = __ldg(dd);                                    // ip, it, itc
      hw = as_float4(__ldg(dd + 1));               // rho, tp, tt, ttc
      hfl = d_flags(__ldg(dd + 2));
      hidt = (hfl & kLayerTClamp) ? 0.f : (float)a.inv_dt[hb.y];
      hidc = (nq > 0 && !(hfl & kLayerTcClamp)) ? (float)a.inv_dtc[hb.z] : 0.f;
    }
    float acc[kRT][2];
    const int jmax = min(N, l0 + kRT);
    if constexpr (MAXMOL <= 5) {
      // packed FP32 pairs over layers: acc2[r][c] holds layers (2r, 2r+1) at wavenumber c (with
      // eight absorbers the extra registers spill, so that form keeps scalar FMAs)
      unsigned long long acc2[kRT / 2][2];
#pragma unroll
      for (int r = 0; r < kRT / 2; ++r) acc2[r][0] = acc2[r][1] = 0ull;
      for (int j = 0; j < jmax; ++j) {
        const float2 g = *reinterpret_cast<const float2*>(Gt + tix(j, 2 * lane));
        const unsigned long long gx = pack_dup(g.x), gy = pack_dup(g.y);
#pragma unroll
        for (int r = 0; r < kRT / 2; ++r) {
          // zero for j > l and rows >= N
          const unsigned long long dl = pack2(DLT[(size_t)(l0 + 2 * r) * npad + j],
                                              DLT[(size_t)(l0 + 2 * r + 1) * npad + j]);
          ffma2(acc2[r][0], dl, gx);
          ffma2(acc2[r][1], dl, gy);
        }
      }
#pragma unroll
      for (int r = 0; r < kRT / 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float2 v = unpack2(acc2[r][c]);
          acc[2 * r][c] = v.x;
          acc[2 * r + 1][c] = v.y;
        }
    } else {
#pragma unroll
      for (int r = 0; r < kRT; ++r) acc[r][0] = acc[r][1] = 0.f;
      for (int j = 0; j < jmax; ++j) {
        const float2 g = *reinterpret_cast<const float2*>(Gt + tix(j, 2 * lane));
#pragma unroll
        for (int r = 0; r < kRT; ++r) {
          const float dl = DLT[(size_t)(l0 + r) * npad + j];   // zero for j > l and rows >= N
          acc[r][0] = fmaf(dl, g.x, acc[r][0]);
          acc[r][1] = fmaf(dl, g.y, acc[r][1]);
        }
      }
    }
    // the corner rows of the current (P, T) cell at this lane's two wavenumbers: consecutive
    // layers of one cell (a segment) share them, so they are gathered from L2 once per
    // segment, all together, instead of once per layer
    unsigned long long cs[MAXMOL][4];                  // (sigma(v), sigma(v + 1)) pairs
    int c_ip = -1, c_it = -1;
    for (int r = 0; r < kRT; ++r) {
      const int l = l0 + r;
      if (l >= N) break;
      float* pf = a.part_f + (item_tile * p.max_layers + l) * a.n_feat;
      const float gk0 = in_row ? acc[r][0] : 0.f, gk1 = in_row ? acc[r][1] : 0.f;
      const int d_ip = __shfl_sync(0xffffffffu, hb.x, r), d_it = __shfl_sync(0xffffffffu, hb.y, r);
      const int d_itc = __shfl_sync(0xffffffffu, hb.z, r);
      const float tp = __shfl_sync(0xffffffffu, hw.y, r), tt = __shfl_sync(0xffffffffu, hw.z, r);
      const float ttc = __shfl_sync(0xffffffffu, hw.w, r);
      const float idt = __shfl_sync(0xffffffffu, hidt, r);
      const float idc = __shfl_sync(0xffffffffu, hidc, r);
      const size_t slab_t = (size_t)p.wn_pad, slab_p = (size_t)p.n_t * p.wn_pad;
      const int wq = in_row ? w2 : 0;
      if (d_ip != c_ip || d_it != c_it) {               // a new cell (warp-uniform)
        const size_t o0 = ((size_t)d_ip * p.n_t + d_it) * p.wn_pad + wq;
#pragma unroll
        for (int m = 0; m < MAXMOL; ++m) {
          if (m < nm) {
            const size_t om = o0 + (size_t)m * p.n_p * slab_p;
            const float2 v0 = sig2<F16>(p, m, om), v1 = sig2<F16>(p, m, om + slab_t),
                         v2 = sig2<F16>(p, m, om + slab_p), v3 = sig2<F16>(p, m, om + slab_p + slab_t);
            cs[m][0] = pack2(v0.x, v0.y);
            cs[m][1] = pack2(v1.x, v1.y);
            cs[m][2] = pack2(v2.x, v2.y);
            cs[m][3] = pack2(v3.x, v3.y);
          }
        }
        c_ip = d_ip; c_it = d_it;
      }
      // this lane's terms of every feature of layer l (its two wavenumbers, as packed pairs)
      const unsigned long long tt2 = pack_dup(tt), tp2 = pack_dup(tp), up2 = pack_dup(1.f - tp);
      const unsigned long long idt2 = pack_dup(idt);
#pragma unroll
      for (int m = 0; m < MAXMOL; ++m) {
        if (m < nm) {
          // sigma(T) at both pressures, then sigma(P); d sigma / dT of the same bracket
          const unsigned long long d0 = sub2(cs[m][1], cs[m][0]), d1 = sub2(cs[m][3], cs[m][2]);
          const unsigned long long a1 = fma2(d0, tt2, cs[m][0]), a2 = fma2(d1, tt2, cs[m][2]);
          const float2 sg = unpack2(fma2(sub2(a2, a1), tp2, a1));
          const float2 dt = unpack2(mul2(fma2(d0, up2, mul2(d1, tp2)), idt2));
          red[m * kRedPitch + lane] = fmaf(gk0, sg.x, gk1 * sg.y);
          red[(f_dS + m) * kRedPitch + lane] = fmaf(gk0, dt.x, gk1 * dt.y);
        }
      }
      for (int s = 0; s < p.n_species; ++s) {
        float fr = 0.f;
        if (s < ns) {
          const float2 v = *reinterpret_cast<const float2*>(ray_s + s * kAT + 2 * lane);
          fr = gk0 * v.x + gk1 * v.y;
        }
        red[(f_R + s) * kRedPitch + lane] = fr;
      }
      if (nq > 0) {
        for (int q = 0; q < nq; ++q) {
          const float* bq = p.cia + ((size_t)q * p.n_t_cia + d_itc) * p.wn_pad + wq;
          const float2 c0 = ldg2(bq), c1 = ldg2(bq + p.wn_pad);
          const float sg0 = c0.x + (c1.x - c0.x) * ttc, sg1 = c0.y + (c1.y - c0.y) * ttc;
          red[(f_C + q) * kRedPitch + lane] = gk0 * sg0 + gk1 * sg1;
          red[(f_dC + q) * kRedPitch + lane] = gk0 * (c1.x - c0.x) * idc + gk1 * (c1.y - c0.y) * idc;
        }
      }
      red[f_K * kRedPitch + lane] = gk0 + gk1;
      __syncwarp();
      for (int f = lane; f < a.n_feat; f += 32) {       // feature f: its 32 terms in lane order
        const float4* row = reinterpret_cast<const float4*>(red + f * kRedPitch);
        // four chains (terms k = 0, 1, 2, 3 mod 4) as two packed pairs, fixed order
        unsigned long long s01 = 0ull, s23 = 0ull;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 v = row[k];
          s01 = add2(s01, pack2(v.x, v.y));
          s23 = add2(s23, pack2(v.z, v.w));
        }
        const float2 u = unpack2(s01), w = unpack2(s23);
        pf[f] = (u.x + u.y) + (w.x + w.y);
      }
      __syncwarp();                                     // red is free for the next layer
    }
  }
}

// dL/dD at native wavenumbers of the binned range, and chi^2 (chi^2 mode) per item.
__global__ void k_gd(BinsDev bd, int B, const double* __restrict__ binned,
                     const double* __restrict__ obs, const double* __restrict__ sig,
                     const double* __restrict__ gbin, const ItemGeom* __restrict__ items,
                     double* __restrict__ chi2, float* __restrict__ gd, int n_in) {
  __shared__ double gb[256];
  const int b = blockIdx.x;
  const bool valid = items[b].status == TR_OK;
  const double* Db = binned + (size_t)b * bd.n_bin;
  for (int k = threadIdx.x; k < bd.n_bin; k += blockDim.x) {
    double g = 0.0;
    if (valid) g = gbin ? gbin[(size_t)b * bd.n_bin + k] : 2.0 * (Db[k] - obs[k]) / (sig[k] * sig[k]);
    if (k < 256) gb[k] = g;
  }
  __syncthreads();
  if (threadIdx.x == 0 && chi2 && !gbin) {
    double c = 0.0;
    for (int k = 0; k < bd.n_bin; ++k) { const double r = (Db[k] - obs[k]) / sig[k]; c += r * r; }
    chi2[b] = valid ? c : INFINITY;
  }
  for (int i = threadIdx.x; i < n_in; i += blockDim.x) {
    double g = 0.0;
    for (int e = bd.t_ptr[i]; e < bd.t_ptr[i + 1]; ++e) g += gb[bd.t_bin[e]] * bd.t_w[e];
    gd[(size_t)b * n_in + i] = (float)g;
  }
}

// Sum of the wavenumber tiles' partial sums of one array [B][tiles][M] into its tile-0 slot,
// in tile order (deterministic), compensated (Kahan) so the FP32 sum of hundreds of tiles
// keeps about FP32 rounding; blockIdx.y picks the array.  Consecutive threads take
// consecutive elements, so every tile's row is read coalesced.  An array with tri > 0 is a
// [tri][tri] matrix of which only the entries (j, l) with l >= j are written and read (the
// G_DL partial sums): a warp whose 32 entries all lie below the diagonal skips them (a
// whole warp, so that the warps' long tile loops do not diverge; B tri^2 is a multiple of
// 64, so a warp's lanes leave the grid-stride loop together).
struct TileSumArgs {
  float* arr[4];
  long long m[4];
  int tri[4];
};
__global__ void k_adjoint_sum(TileSumArgs ts, int B, int tiles) {
  float* arr = ts.arr[blockIdx.y];
  const long long M = ts.m[blockIdx.y];
  const int tri = ts.tri[blockIdx.y];
  const long long n = (long long)B * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / M, m = i - b * M;
    if (tri > 0 && __all_sync(0xffffffffu, (int)m % tri < (int)m / tri)) continue;   // l < j
    float* row = arr + (size_t)b * tiles * M + m;
    float s = row[0], c = 0.f;
    for (int t = 1; t < tiles; ++t) {
      const float y = __fsub_rn(row[(size_t)t * M], c);
      const float u = __fadd_rn(s, y);
      c = __fsub_rn(__fsub_rn(u, s), y);
      s = u;
    }
    row[0] = s;
  }
}

struct ItemParams {
  GeomParams gp;
  const double* theta; int n_theta;
  ItemBuffers buf;
  const float* part_a; const float* part_dl; const float* part_f; const float* part_rp;
  int tiles, n_feat;              // partial sums are [B][tiles][...]
  int n_sum;                      // tiles to add (1 after k_adjoint_sum)
  double* grad;                   // item b's n_theta values at grad + b * grad_stride
  long long grad_stride;
};

// Fixed-order tree sum over the CTA's threads of NV doubles per thread (red: [NV][threads]);
// every thread gets the sums back in v.
template <int NV>
__device__ void block_sum_n(double (&v)[NV], double (*red)[kItemThreads]) {
#pragma unroll
  for (int i = 0; i < NV; ++i) red[i][threadIdx.x] = v[i];
  __syncthreads();
  for (int o = kItemThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
#pragma unroll
      for (int i = 0; i < NV; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + o];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = red[i][0];
  __syncthreads();
}

// (ah + al) - (bh + bl) to FP32 working precision (Knuth's TwoSum on the leading parts).
__device__ __forceinline__ float diff_df(float ah, float al, float bh, float bl) {
  const float s = __fsub_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
  return __fadd_rn(s, __fadd_rn(e, __fsub_rn(al, bl)));
}

// Dynamic shared memory of k_adjoint_item (bytes) for a maximum layer count.
__host__ __device__ inline size_t item_smem_bytes(int NM) {
  return sizeof(double) * (5 * (size_t)NM + 1)       // G_r, G_T, G_a, recursion factors, node weights
         + sizeof(float2) * ((size_t)NM + 1)         // z as double-float
         + sizeof(float) * ((size_t)NM + 1)          // r in FP32
         + sizeof(int) * (size_t)NM + 16;            // node segment per layer
}

// One CTA per atmosphere.  GB300 runs FP64 at a small fraction of its FP32 rate, so the
// O(N^2) path-length sensitivities are FP32 terms (from double-float altitudes, as the forward
// path lengths) accumulated in FP64; per-layer and per-item work is spread over the threads;
// the one serial chain left, the backward hydrostatic recursion, is one FP64 FMA per layer.
constexpr int kItemRed = TR_MAX_SPECIES + 1 + 2 + TR_MAX_TNODES;   // values of the CTA sums
__global__ void __launch_bounds__(kItemThreads)
k_adjoint_item(ItemParams ip) {
  extern __shared__ double dsm[];
  __shared__ double red[kItemRed][kItemThreads];
  __shared__ double s_X[TR_MAX_SPECIES], s_GX[TR_MAX_SPECIES];
  __shared__ double s_c[4];                            // cz, delta, mu, sum G_D
  const GeomParams& gp = ip.gp;
  const int b = blockIdx.x, t = threadIdx.x;
  const int nth = ip.n_theta;
  double* grad = ip.grad + (size_t)b * ip.grad_stride;
  const ItemGeom ig = ip.buf.items[b];
  if (ig.status != TR_OK || ig.n_layers == 0) {
    for (int k = t; k < nth; k += kItemThreads) grad[k] = 0.0;
    return;
  }
  const int N = ig.n_layers, NM = gp.max_layers, npad = ip.buf.npad;
  const double* th = ip.theta + (size_t)b * nth;
  const double* z = ip.buf.z + (size_t)b * (NM + 1);
  const double* T = ip.buf.tl + (size_t)b * NM;
  const LayerDesc* LD = ip.buf.layers + (size_t)b * NM;
  double* Gr = dsm;                 // [N + 1]
  double* GT = Gr + (NM + 1);       // [N]
  double* Ga = GT + NM;             // [N]
  double* fac = Ga + NM;            // [N] dr_{l+1} / dr_l of the recursion
  double* wn = fac + NM;            // [N] weight of node k_l + 1 in T_l
  float2* zs = reinterpret_cast<float2*>(wn + NM);          // [N + 1]
  float* rs = reinterpret_cast<float*>(zs + NM + 1);         // [N + 1]
  int* kn = reinterpret_cast<int*>(rs + NM + 1);             // [N] node segment of layer l
  const double rp = ig.r_p;
  const double inv_rs2 = gp.inv_rs2;
  const double ln10 = 2.302585092994046;
  const int nm = gp.n_mol, nq = gp.n_cia, ntn = gp.n_tnodes;

  // chemistry (as the profile kernel computes it), constants of the recursion
  if (t < nm) s_X[t] = exp10(th[t]);
  __syncthreads();
  if (t == 0) {
    double sumx = 0.0, mu = 0.0;
    for (int m = 0; m < nm; ++m) { sumx += s_X[m]; mu = fma(s_X[m], gp.mass[m], mu); }
    const double rem = 1.0 - sumx;
    for (int f = nm; f < gp.n_species; ++f) s_X[f] = gp.fill[f] * rem;
    mu = fma(rem, gp.fill_mass, mu);
    const double delta = (gp.ln_pmax - gp.ln_pmin) / N;
    s_c[0] = (kKB * delta) / (mu * gp.amu_g_mp);
    s_c[1] = delta;
    s_c[2] = mu;
    double grp = 0.0;
    for (int q = 0; q < ip.n_sum; ++q) grp += ip.part_rp[(size_t)b * ip.tiles + q];
    s_c[3] = grp;
  }
  // tile sums G_a; altitudes as double-float pairs and radii in FP32
  for (int j = t; j < N; j += kItemThreads) {
    double s = 0.0;
    for (int q = 0; q < ip.n_sum; ++q) s += ip.part_a[((size_t)b * ip.tiles + q) * npad + j];
    Ga[j] = s;
  }
  for (int k = t; k <= N; k += kItemThreads) {
    const double zk = z[k];
    const float h = (float)zk;
    zs[k] = make_float2(h, (float)(zk - (double)h));
    rs[k] = (float)(rp + zk);
  }
  __syncthreads();
  const double cz = s_c[0], delta = s_c[1], mu = s_c[2];

  // ---- radii from path lengths and annulus weights
  //      DL[j][l] = 2 (s(l+1,j) - s(l,j)), s(k,j) = sqrt(r_k^2 - r_j^2):
  //      ds(k,j)/dr_k = r_k / s,  ds(k,j)/dr_j = -r_j / s;  r_k^2 - r_j^2 = (z_k - z_j)(r_k + r_j)
  //      with z_k - z_j from the double-float altitudes; each term in FP32, sums in FP64
  auto gdl = [&](int j, int l) -> float {    // sum over tiles of G_DL[j][l] (0 outside j<=l<N)
    if (l < j || l >= N) return 0.f;
    float s = 0.f;
    for (int q = 0; q < ip.n_sum; ++q)
      s += ip.part_dl[(((size_t)b * ip.tiles + q) * npad + j) * npad + l];
    return s;
  };
  for (int k = t; k <= N; k += kItemThreads) {
    const float2 zk = zs[k];
    const float rk = rs[k];
    double g = 0.0;
    for (int j = 0; j < k; ++j) {                 // k as the outer radius of s(k, j)
      const float gs = 2.f * (gdl(j, k - 1) - gdl(j, k));
      if (gs != 0.f) {
        const float2 zj = zs[j];
        const float s2 = diff_df(zk.x, zk.y, zj.x, zj.y) * (rk + rs[j]);
        g += (double)(gs * rk * rsqrtf(s2));
      }
    }
    for (int kk = k + 1; kk <= N; ++kk) {         // k as the ray of s(kk, k)
      const float gs = 2.f * (gdl(k, kk - 1) - gdl(k, kk));
      if (gs != 0.f) {
        const float2 zu = zs[kk];
        const float s2 = diff_df(zu.x, zu.y, zk.x, zk.y) * (rs[kk] + rk);
        g -= (double)(gs * rk * rsqrtf(s2));
      }
    }
    // a_j = (r_{j+1}^2 - r_j^2) / R_s^2
    const double rkd = rp + z[k];
    if (k >= 1) g += Ga[k - 1] * 2.0 * rkd * inv_rs2;
    if (k < N) g -= Ga[k] * 2.0 * rkd * inv_rs2;
    Gr[k] = g;
  }

  // ---- per layer: opacity weights, densities, cloud; recursion factors; T-node weights
  const double dln = (gp.ln_pmin - gp.ln_pmax) / N;
  const int f_dS = nm, f_R = 2 * nm, f_C = 2 * nm + gp.n_species, f_dC = f_C + nq, f_K = f_dC + nq;
  double acc[kItemRed];
#pragma unroll
  for (int i = 0; i < kItemRed; ++i) acc[i] = 0.0;
  double* gx_loc = acc;                             // [TR_MAX_SPECIES]
  double& glp = acc[TR_MAX_SPECIES];
  for (int l = t; l < N; l += kItemThreads) {
    double F[2 * TR_MAX_MOL + TR_MAX_SPECIES + 2 * TR_MAX_CIA + 1];
    for (int f = 0; f < ip.n_feat; ++f) {
      double s = 0.0;
      for (int q = 0; q < ip.n_sum; ++q)
        s += ip.part_f[(((size_t)b * ip.tiles + q) * NM + l) * ip.n_feat + f];
      F[f] = s;
    }
    const LayerDesc& d = LD[l];
    const double lnp0 = fma((double)l, dln, gp.ln_pmax), lnp1 = fma((double)(l + 1), dln, gp.ln_pmax);
    const double lnp = 0.5 * (lnp0 + lnp1);
    const double P = exp(lnp);
    const double Tl = T[l];
    const double rho = (P * gp.inv_kb) / Tl;
    double gT = 0.0, grho = 0.0;
    if (!(d.flags & kLayerMolZero)) {
      for (int m = 0; m < nm; ++m) {
        grho += F[m] * s_X[m];
        gx_loc[m] += F[m] * rho;
        gT += rho * s_X[m] * F[f_dS + m];
      }
    }
    if (gp.has_ray) {
      for (int s = 0; s < gp.n_species; ++s) {
        const double R = F[f_R + s] * gp.ray_scale[s];
        grho += R * s_X[s];
        gx_loc[s] += R * rho;
      }
    }
    if (nq > 0 && !(d.flags & kLayerCiaZero)) {
      for (int q = 0; q < nq; ++q) {
        const double C = F[f_C + q] * gp.cia_scale[q], dC = F[f_dC + q] * gp.cia_scale[q];
        const double xa = s_X[gp.cia_a[q]], xb = s_X[gp.cia_b[q]];
        gT += rho * rho * xa * xb * dC;
        grho += C * 2.0 * rho * xa * xb;
        gx_loc[gp.cia_a[q]] += C * rho * rho * xb;
        gx_loc[gp.cia_b[q]] += C * rho * rho * xa;
      }
    }
    gT += grho * (-rho / Tl);
    if (gp.cloud_mode == TR_CLOUD_FRACTIONAL) {
      // c_l = clamp((min(ln p_l, ln P_bot) - max(ln P_top, ln p_{l+1})) / Delta, 0, 1)
      const double ln_top = th[nm + ntn + 1] * ln10;
      const double hi = fmin(lnp0, gp.ln_cbot);
      const double cf = (hi - fmax(ln_top, lnp1)) / delta;
      if (cf > 0.0 && cf < 1.0 && ln_top > lnp1) glp += gp.kappa_cloud * F[f_K] * (-ln10 / delta);
    }
    GT[l] = gT;
    // dr_{l+1}/dr_l: 1 + 2 cz T_l r_l (altitude-dependent gravity), 1 (constant)
    fac[l] = gp.gravity_mode == TR_GRAV_CONST ? 1.0 : fma(2.0 * cz * Tl, rp + z[l], 1.0);
    // temperature nodes: T_l linear in log10 P between nodes, clamped beyond them
    int kseg = 0;
    double f = 0.0;
    if (ntn > 1) {
      const double x = lnp * 0.43429448190325182765;
      if (x >= gp.tnode_log10p[0]) { kseg = 0; f = 0.0; }
      else if (x <= gp.tnode_log10p[ntn - 1]) { kseg = ntn - 2; f = 1.0; }
      else {
        while (!(gp.tnode_log10p[kseg] >= x && x >= gp.tnode_log10p[kseg + 1])) ++kseg;
        f = (x - gp.tnode_log10p[kseg]) * gp.inv_dlog10p[kseg];
      }
    }
    kn[l] = kseg;
    wn[l] = f;
  }
  __syncthreads();

  // ---- hydrostatic recursion, backwards (r_{l+1} = r_l + cz T_l r_l^2): one FMA per layer
  if (t == 0) {
    double g = Gr[N];
    for (int l = N - 1; l >= 0; --l) {
      g = fma(g, fac[l], Gr[l]);
      Gr[l] = g;
    }
  }
  __syncthreads();
  // per layer, with G_r of r_{l+1}: dT_l and dcz (and, for constant gravity, dR_p) terms;
  // then the CTA sums of the mixing-ratio, cloud, cz, R_p and node terms
  for (int l = t; l < N; l += kItemThreads) {
    const double g1 = Gr[l + 1];
    const double rl = gp.gravity_mode == TR_GRAV_CONST ? rp : rp + z[l];
    const double gT = GT[l] + g1 * cz * rl * rl;
    acc[TR_MAX_SPECIES + 1] += g1 * T[l] * rl * rl;                    // d/dcz
    if (gp.gravity_mode == TR_GRAV_CONST)
      acc[TR_MAX_SPECIES + 2] += g1 * 2.0 * cz * T[l] * rp;            // d/dR_p, direct
    double* gnode = acc + TR_MAX_SPECIES + 3;
    if (ntn == 1) {
      gnode[0] += gT;
    } else {
      gnode[kn[l]] += gT * (1.0 - wn[l]);
      gnode[kn[l] + 1] += gT * wn[l];
    }
  }
  block_sum_n<kItemRed>(acc, red);
  if (t == 0) {
    for (int s = 0; s < gp.n_species; ++s) s_GX[s] = acc[s];
    const double glp_sum = acc[TR_MAX_SPECIES], gcz = acc[TR_MAX_SPECIES + 1];
    const double grp_dir = acc[TR_MAX_SPECIES + 2];
    const double g_rp = Gr[0] + grp_dir + s_c[3] * 2.0 * rp * inv_rs2;
    const double gmu = gcz * (-cz / mu);
    // chemistry: X_m = 10^theta_m, fill gases f (1 - sum X), mu = sum X_s m_s
    double sum_fill = 0.0;
    for (int f = nm; f < gp.n_species; ++f) sum_fill += gp.fill[f] * (s_GX[f] + gmu * gp.mass[f]);
    for (int m = 0; m < nm; ++m) {
      const double gxm = s_GX[m] + gmu * gp.mass[m] - sum_fill;
      grad[m] = gxm * s_X[m] * ln10;
    }
    for (int k = 0; k < ntn; ++k) grad[nm + k] = acc[TR_MAX_SPECIES + 3 + k];
    grad[nm + ntn] = g_rp * kRJup;
    grad[nm + ntn + 1] = glp_sum;
  }
}

}  // namespace

size_t adjoint_extra_bytes(const tr_tables* t, const tr_batch_desc* d, const tr_bins* bins, int B) {
  if (!t || !d || !bins) return 0;
  const int n_in = bins->dev.i1 - bins->dev.i0;
  const int tiles = (bins->dev.i1 - wn_first(bins->dev.i0) + kAT - 1) / kAT;
  const int npad = pad8(d->max_layers);
  const int n_feat = 2 * t->n_mol + t->n_species + 2 * t->n_cia + 1;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t s = 0;
  s += al(sizeof(float) * (size_t)B * n_in);                               // gd
  s += al(sizeof(float) * (size_t)B * tiles * npad);                       // part_a
  s += al(sizeof(float) * (size_t)B * tiles * npad * npad);                // part_dl
  s += al(sizeof(float) * (size_t)B * tiles * d->max_layers * n_feat);     // part_f
  s += al(sizeof(float) * (size_t)B * tiles);                              // part_rp
  s += al(sizeof(double) * (size_t)B * bins->dev.n_bin);                   // binned scratch
  return s;
}

}  // namespace tr

using namespace tr;

extern "C" int tr_adjoint_transit(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d, int B,
                                  const double* d_theta, const int32_t* d_nlayers,
                                  const tr_bins* bins, const double* d_obs,
                                  const double* d_sigma_obs, const double* d_gbin,
                                  double* d_chi2, double* d_grad, double* d_jac, double* d_binned,
                                  int32_t* d_status, int precision, int recompute_k, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!ctx || !t || !d || !bins || !d_theta || B < 0)
    return set_error(ctx, TR_ERR_ARG, "null argument");
  if (!d_grad && !d_jac) return set_error(ctx, TR_ERR_ARG, "neither d_grad nor d_jac given");
  if (B > TR_MAX_BATCH) return set_error(ctx, TR_ERR_ARG, "batch larger than TR_MAX_BATCH");
  const bool chi2_mode = d_grad && !d_gbin;
  if (chi2_mode && (!d_obs || !d_sigma_obs || !d_chi2))
    return set_error(ctx, TR_ERR_ARG, "chi^2 mode needs obs, sigma_obs and chi2");
  if (precision != TR_PREC_FP32 && precision != TR_PREC_MIXED)
    return set_error(ctx, TR_ERR_ARG, "unknown precision");
  const bool mixed = precision == TR_PREC_MIXED;
  if (!mixed && !t->d_sigma && t->n_mol > 0)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "tables were loaded without FP32 storage");
  if (mixed && !t->d_logsig16 && t->n_mol > 0)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "tables were loaded without FP16 log10 storage");
  if (bins->dev.n_bin > 256) return set_error(ctx, TR_ERR_ARG, "the adjoint supports at most 256 bins");
  if (t->interp_mode != TR_INTERP_LINEAR)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "the adjoint implements the linear temperature scheme");
  if (d->t_profile != TR_TPROF_NPOINT || d->gas_mode != TR_GAS_CONSTANT)
    return set_error(ctx, TR_ERR_UNSUPPORTED,
                     "the adjoint implements the N-point temperature profile and constant "
                     "mixing ratios");
  if (B == 0) return TR_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_in = bins->dev.i1 - bins->dev.i0;
  const size_t fwd = forward_workspace_bytes(B, d->max_layers, n_in);
  auto al256 = [](size_t x) { return (x + 255) / 256 * 256; };
  // [forward item buffers + depths][K buffer][path-length tiles][adjoint buffers]
  const size_t kb = al256(forward_kbuf_bytes(B, d->max_layers, bins->dev.i0, n_in));
  const size_t db = al256(dl_tile_bytes(B, d->max_layers, precision));
  const size_t need = fwd + kb + db + adjoint_extra_bytes(t, d, bins, B);
  ItemBuffers buf; double* depth = nullptr; char* extra = nullptr;
  int rc = prepare_batch(ctx, t, d, n_in, need, B, d_theta, d_nlayers, d_status, ws, ws_bytes,
                         s, &buf, &depth, &extra);
  if (rc != TR_OK) return rc;
  float* kbuf = reinterpret_cast<float*>(extra);
  void* dl16 = db > 0 ? extra + kb : nullptr;
  extra += kb + db;
  const bool k_whole = forward_chunk_items(B, d->max_layers, bins->dev.i0, n_in) >= B;
  const bool use_kstore = k_whole && recompute_k != 1;
  // forward, in the two-stage form (the configuration tuned for this shape's forward, if
  // any), which leaves K in kbuf; when one chunk holds the whole batch the backward passes
  // read it back instead of recomputing it.  The binned spectrum is needed only for chi^2 or
  // when asked for: otherwise (vector-Jacobian products, Jacobian) only the opacity stage
  // runs, and not even that when the backward recomputes K.
  const bool need_binned = chi2_mode || d_binned;
  const auto it = ctx->tuned.find(batch_shape_key(t, d, B, bins, false, precision));
  ForwardChoice fc = it != ctx->tuned.end() ? it->second : ForwardChoice{kFormTwoStage, 0, 0, 0};
  fc.form = kFormTwoStage;
  if (need_binned || use_kstore) {
    rc = run_forward(ctx, t, d->max_layers, buf, B, bins->dev.i0, n_in, depth, n_in, precision,
                     s, kbuf, dl16, &fc, /*opacity_only=*/!need_binned);
    if (rc != TR_OK) return rc;
  }
  const int tiles = (bins->dev.i1 - wn_first(bins->dev.i0) + kAT - 1) / kAT;
  const int npad = pad8(d->max_layers);
  const int n_feat = 2 * t->n_mol + t->n_species + 2 * t->n_cia + 1;
  const int nth = t->n_mol + d->n_tnodes + 2;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  char* e = extra;
  float* gd = reinterpret_cast<float*>(e); e += al(sizeof(float) * (size_t)B * n_in);
  float* part_a = reinterpret_cast<float*>(e); e += al(sizeof(float) * (size_t)B * tiles * npad);
  float* part_dl = reinterpret_cast<float*>(e); e += al(sizeof(float) * (size_t)B * tiles * npad * npad);
  float* part_f = reinterpret_cast<float*>(e); e += al(sizeof(float) * (size_t)B * tiles * d->max_layers * n_feat);
  float* part_rp = reinterpret_cast<float*>(e); e += al(sizeof(float) * (size_t)B * tiles);
  double* binned = d_binned ? d_binned : reinterpret_cast<double*>(e);
  cudaError_t err = cudaSuccess;
  if (need_binned) {
    KernelTimer kt(ctx, "k_bin", s);
    err = launch_bin(bins->dev, B, depth, n_in, bins->dev.i0, binned, s);
  }
  if (err != cudaSuccess) return set_error(ctx, TR_ERR_CUDA, cudaGetErrorString(err));
  if (d_grad) {
    KernelTimer kt(ctx, "k_gd", s);
    k_gd<<<B, 256, 0, s>>>(bins->dev, B, binned, d_obs, d_sigma_obs, d_gbin, buf.items,
                           d_gbin ? nullptr : d_chi2, gd, n_in);
    err = cudaGetLastError();
  }
  if (err != cudaSuccess) return set_error(ctx, TR_ERR_CUDA, cudaGetErrorString(err));
  AdjParams ap{};
  ap.f.sigma = t->d_sigma; ap.f.n_mol = t->n_mol; ap.f.n_p = t->n_p; ap.f.n_t = t->n_t;
  ap.f.wn_pad = t->wn_pad; ap.f.cia = t->d_cia; ap.f.n_cia = t->n_cia; ap.f.n_t_cia = t->n_t_cia;
  ap.f.ray = t->has_ray ? t->d_ray : nullptr; ap.f.n_species = t->n_species;
  ap.f.max_layers = d->max_layers; ap.f.buf = buf; ap.f.wn_begin = bins->dev.i0;
  ap.f.wn_count = n_in; ap.f.dev_err = ctx->dev_err;
  if (mixed) {
    ap.f.logsig16 = t->d_logsig16;
    for (int m = 0; m < t->n_mol; ++m) ap.f.logsig_off[m] = t->logsig_offset[m];
  }
  ap.inv_dt = t->d_inv_dt; ap.inv_dtc = t->d_inv_dtc; ap.gd = gd; ap.n_in = n_in;
  ap.n_feat = n_feat; ap.part_a = part_a; ap.part_dl = part_dl;
  ap.part_f = part_f; ap.part_rp = part_rp;
  ap.kstore = use_kstore ? kbuf : nullptr;
  ap.kcols = forward_kcols(bins->dev.i0, n_in);
  ap.t_ptr = bins->dev.t_ptr; ap.t_bin = bins->dev.t_bin; ap.t_w = bins->dev.t_w;
  const size_t smem = sizeof(float) * AdjSmem(d->max_layers, n_feat).floats();
  static_assert(TR_MAX_MOL == 8, "adjoint instantiated for up to 5 or 8 molecules");
  void (*kern)(AdjParams);
  if (t->n_mol <= 5)
    kern = mixed ? (use_kstore ? k_adjoint_tile<5, true, false> : k_adjoint_tile<5, true, true>)
                 : (use_kstore ? k_adjoint_tile<5, false, false> : k_adjoint_tile<5, false, true>);
  else
    kern = mixed ? (use_kstore ? k_adjoint_tile<8, true, false> : k_adjoint_tile<8, true, true>)
                 : (use_kstore ? k_adjoint_tile<8, false, false> : k_adjoint_tile<8, false, true>);
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return set_error(ctx, TR_ERR_CUDA, std::string("adjoint tile kernel: ") + cudaGetErrorString(err));
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  ItemParams itp{};
  itp.gp = batch_geom_params(t, d); itp.theta = d_theta; itp.n_theta = nth; itp.buf = buf;
  itp.part_a = part_a; itp.part_dl = part_dl; itp.part_f = part_f; itp.part_rp = part_rp;
  itp.n_feat = n_feat;
  itp.n_sum = 1;                                            // tile 0 holds the sums
  const size_t smem_i = item_smem_bytes(d->max_layers);

  // One backward pass over wavenumber tiles [tile0, tile0 + nt): the tile kernel's partial
  // sums, their GPU-wide sum into tile 0, and the per-atmosphere kernel writing item b's
  // gradient at grad + b * stride.  jac_bin < 0 takes dL/dD from gd, else the weights of bin
  // jac_bin (one row of the Jacobian).
  auto backward = [&](int jac_bin, int tile0, int nt, double* grad, long long stride) -> int {
    ap.tile0 = tile0; ap.tiles = nt; ap.jac_bin = jac_bin;
    {
      KernelTimer kt(ctx, "k_adjoint_tile", s);
      kern<<<dim3(nt, B), kAThreads, smem, s>>>(ap);
      err = cudaGetLastError();
    }
    if (err != cudaSuccess) return set_error(ctx, TR_ERR_CUDA, std::string("adjoint tile kernel: ") + cudaGetErrorString(err));
    if (nt > 1) {
      // the tiles' partial sums into tile 0 by a GPU-wide pass, so the per-atmosphere kernel
      // reads one set of sums
      KernelTimer kt(ctx, "k_adjoint_sum", s);
      TileSumArgs ts{};
      ts.arr[0] = part_a;  ts.m[0] = npad;
      ts.arr[1] = part_dl; ts.m[1] = (long long)npad * npad; ts.tri[1] = npad;
      ts.arr[2] = part_f;  ts.m[2] = (long long)d->max_layers * n_feat;
      ts.arr[3] = part_rp; ts.m[3] = 1;
      const long long most = (long long)B * npad * npad;
      const int gx = (int)std::max<long long>(1, std::min<long long>((most + 255) / 256, 8LL * n_sm));
      k_adjoint_sum<<<dim3(gx, 4), 256, 0, s>>>(ts, B, nt);
      err = cudaGetLastError();
      if (err != cudaSuccess) return set_error(ctx, TR_ERR_CUDA, std::string("adjoint sum kernel: ") + cudaGetErrorString(err));
    }
    itp.tiles = nt; itp.grad = grad; itp.grad_stride = stride;
    {
      KernelTimer kt(ctx, "k_adjoint_item", s);
      k_adjoint_item<<<B, kItemThreads, smem_i, s>>>(itp);
      err = cudaGetLastError();
    }
    if (err != cudaSuccess) return set_error(ctx, TR_ERR_CUDA, std::string("adjoint item kernel: ") + cudaGetErrorString(err));
    return TR_OK;
  };
  if (d_grad) {
    rc = backward(-1, 0, tiles, d_grad, nth);
    if (rc != TR_OK) return rc;
  }
  if (d_jac) {
    // row k of dD_bin/dtheta: dL/dD is bin k's normalised weights, which vanish outside the
    // bin's native range, so the pass covers only the tiles of that range
    const int base = wn_first(bins->dev.i0);
    const int n_bin = bins->dev.n_bin;
    for (int k = 0; k < n_bin; ++k) {
      const int t0 = (bins->bin_lo[k] - base) / kAT;
      const int t1 = (bins->bin_hi[k] - 1 - base) / kAT + 1;
      rc = backward(k, t0, t1 - t0, d_jac + (size_t)k * nth, (long long)n_bin * nth);
      if (rc != TR_OK) return rc;
    }
  }
  return TR_OK;
}
