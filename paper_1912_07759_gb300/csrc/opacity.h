// opacity.h -- device pieces shared by the TMA-staged opacity kernels (the streaming two-stage
// kernel in forward_fp32.cu and the fused forward kernel in fused.cu):
//   * the shared-memory ring of table-row stages and its producer warp, which walks the work
//     units' layers as segments (maximal runs of layers with the same (P, T) cell and CIA
//     temperature bracket) and issues one tiled TMA load per segment for the molecules' four
//     bracketing (P, T) rows (box {TW wn, 2 T, 2 P, n_mol}) and one for the CIA pairs' two
//     rows (box {TW wn, 2 T, n_cia}) when the CIA bracket changed;
//   * the consumers' per-segment sums of the staged rows over molecules (weights x_m of the
//     item) and over CIA pairs (weights y_q), from which every layer's opacity is four corner
//     FMAs, two CIA FMAs, Rayleigh and cloud (Sec. 5 and Sec. 8.1: the mixing ratios are the
//     same in every layer, Sec. 4.3, so the molecule sum is taken once per segment).
// Work units are (item, layer block, wavenumber tile) triples, items varying fastest, then
// layer blocks; a persistent grid of CTAs takes units blockIdx.x, blockIdx.x + gridDim.x, ...
// Layer blocks split an item's layers into n_lb runs of lb_size layers: with few items (one
// full-size atmosphere has fewer wavenumber tiles than twice the resident CTAs) the finer
// units keep the last pass over the grid from running with a fraction of the CTAs idle.
#pragma once
#include <cuda_fp16.h>
#include "tma.h"
#include "tr_internal.h"

namespace tr {

constexpr float kLog2Of10 = 3.32192809488736234787f;
constexpr int kRingMaxStages = 8;

// 2^x by the hardware approximation (relative error ~2e-7, far below the FP16 storage step)
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2 x by the hardware approximation (absolute error a few 1e-7 for normal x > 0)
__device__ __forceinline__ float lg2_fast(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Byte sizes of one ring stage for a tile of TW wavenumbers.
struct RingPlan {
  uint32_t mol_bytes, cia_bytes, stage_bytes;
  int stages;
  __host__ __device__ RingPlan(int tw, int n_mol, int n_cia, int elem_bytes, int n_stages) {
    mol_bytes = (uint32_t)(tw * elem_bytes * 4 * n_mol);
    cia_bytes = (uint32_t)(tw * 4 * 2 * n_cia);
    stage_bytes = (mol_bytes + cia_bytes + 127u) & ~127u;
    stages = n_stages;
  }
  __host__ __device__ uint32_t bytes() const { return (uint32_t)stages * stage_bytes; }
};

// One work unit: item index within the chunk, wavenumber tile and layer range [l_begin,
// l_end) (empty when the item has no layers in its block).
struct OpUnit { int bc, tile, l_begin, l_end; };
__device__ __forceinline__ OpUnit op_unit(const FwdParams& p, long long u, int Bc, int n_lb,
                                          int lb_size) {
  OpUnit o;
  o.bc = (int)(u % Bc);
  const long long r = u / Bc;
  const int lb = (int)(r % n_lb);
  o.tile = (int)(r / n_lb);
  const int N = p.buf.items[p.b_off + o.bc].n_layers;
  o.l_begin = lb * lb_size;
  o.l_end = min(N, o.l_begin + lb_size);
  return o;
}

// Segment starts among the 32 layers l0 .. l0+31 of a unit's layer range [l_begin, l_end)
// (lane i holds layer l0 + i's bracket header h = (ip, it, itc, chemistry zone)): bit i of
// `start` is set when layer l0 + i begins a segment, of `mol` when its molecular cell or zone
// differs from the layer before, of `cia` when its CIA bracket or zone does (a new zone
// changes the molecule and pair weights of the sums).  (cip, cit, citc, czone) carry the
// header of layer l0 - 1 in (-1 at the range start: everything is loaded there) and of the
// chunk's last layer out.
// ZONES = false compiles the zone comparison out (callers that only see zone 0).
struct SegFlags { unsigned start, mol, cia; };
template <bool ZONES = true>
__device__ __forceinline__ SegFlags segment_flags(const int4& h, int l0, int l_begin, int l_end,
                                                  int lane, bool has_mol, bool has_cia,
                                                  int& cip, int& cit, int& citc, int& czone) {
  int pip = __shfl_up_sync(0xffffffffu, h.x, 1);
  int pit = __shfl_up_sync(0xffffffffu, h.y, 1);
  int pitc = __shfl_up_sync(0xffffffffu, h.z, 1);
  int pzone = ZONES ? __shfl_up_sync(0xffffffffu, h.w, 1) : 0;
  if (lane == 0) { pip = cip; pit = cit; pitc = citc; pzone = czone; }
  const int li = l0 + lane;
  const int N = l_end;
  const bool valid = li < N, first = li == l_begin;
  const bool zchg = ZONES && h.w != pzone;
  const bool mol = valid && has_mol && (first || h.x != pip || h.y != pit || zchg);
  const bool cia = valid && has_cia && (first || h.z != pitc || zchg);
  SegFlags f;
  f.start = __ballot_sync(0xffffffffu, valid && (mol || cia || first || zchg));
  f.mol = __ballot_sync(0xffffffffu, mol);
  f.cia = __ballot_sync(0xffffffffu, cia);
  const int last = min(31, N - 1 - l0);
  cip = __shfl_sync(0xffffffffu, h.x, last);
  cit = __shfl_sync(0xffffffffu, h.y, last);
  citc = __shfl_sync(0xffffffffu, h.z, last);
  if (ZONES) czone = __shfl_sync(0xffffffffu, h.w, last);
  return f;
}

// Ring state of one CTA: full[s] completes when stage s's loads have landed, empty[s] when
// all `n_consumers` consumer warps have released it.  abort_flag stops both roles after a
// bounded wait gave up.
struct Ring {
  uint64_t full[kRingMaxStages];
  uint64_t empty[kRingMaxStages];
  int abort_flag;
};

__device__ __forceinline__ void ring_init(Ring& r, int stages, int n_consumers) {
  for (int s = 0; s < stages; ++s) { mbar_init(&r.full[s], 1); mbar_init(&r.empty[s], n_consumers); }
  r.abort_flag = 0;
  mbar_fence_init();
}

// Producer warp (all 32 lanes call it): walks the CTA's units in order, 32 layers (a chunk)
// at a time; for every segment lane 0 waits for the stage to be free and issues its loads:
// only the rows that changed from the segment before, or, with whole_segments (segments
// consumed by different warps), all of them.  The headers of the chunk after the one being
// issued (in the same unit or the CTA's next one) are read one step ahead, so their latency
// overlaps the waits for free stages.  Returns after the last fill of every stage has landed
// (so no copy is in flight when the CTA exits).
template <int TW>
__device__ void ring_produce(const FwdParams& p, Ring& r, const RingPlan& plan,
                             unsigned char* ring, const CUtensorMap* tm_sig,
                             const CUtensorMap* tm_cia, int Bc, long long n_units, int lane,
                             bool whole_segments, int n_lb = 1, int lb_size = 1 << 30) {
  struct Chunk {
    long long u;
    OpUnit o;
    int l0, x0;
    int4 h;
    SegFlags f;
  };
  const int S = plan.stages;
  const bool has_mol = p.n_mol > 0, has_cia = p.n_cia > 0;
  const int wbase = wn_first(p.wn_begin);
  int cip = -1, cit = -1, citc = -1, czone = -1;   // header carried into the next chunk read
  // first chunk of the first unit with layers at or after unit u
  auto first_from = [&](long long u, Chunk& c) -> bool {
    for (; u < n_units; u += gridDim.x) {
      const OpUnit o = op_unit(p, u, Bc, n_lb, lb_size);
      if (o.l_begin < o.l_end) {
        c.u = u; c.o = o; c.l0 = o.l_begin; c.x0 = wbase + o.tile * TW;
        return true;
      }
    }
    return false;
  };
  // headers and segment flags of chunk c
  auto read = [&](Chunk& c) {
    const LayerDesc* L = p.buf.layers + (size_t)(p.b_off + c.o.bc) * p.max_layers;
    const int li = c.l0 + lane;
    c.h = li < c.o.l_end ? __ldg(reinterpret_cast<const int4*>(L + li)) : make_int4(-1, -1, -1, 0);
    if (c.l0 == c.o.l_begin) cip = cit = citc = czone = -1;
    c.f = segment_flags(c.h, c.l0, c.o.l_begin, c.o.l_end, lane, has_mol, has_cia, cip, cit,
                        citc, czone);
  };
  int seg = 0;
  bool stop = false;
  Chunk cur, nxt;
  bool have = first_from(blockIdx.x, cur);
  if (have) read(cur);
  while (have && !stop) {
    bool have_next;
    if (cur.l0 + 32 < cur.o.l_end) {
      nxt = cur;
      nxt.l0 = cur.l0 + 32;
      have_next = true;
    } else {
      have_next = first_from(cur.u + gridDim.x, nxt);
    }
    if (have_next) read(nxt);
    const SegFlags f = cur.f;
    for (unsigned m = f.start; m != 0u; m &= m - 1u) {
      const int i = __ffs(m) - 1;
      const int ip = __shfl_sync(0xffffffffu, cur.h.x, i);
      const int it = __shfl_sync(0xffffffffu, cur.h.y, i);
      const int itc = __shfl_sync(0xffffffffu, cur.h.z, i);
      const bool mol = whole_segments ? has_mol : ((f.mol >> i) & 1u);
      const bool cia = whole_segments ? has_cia : ((f.cia >> i) & 1u);
      int ok = 1;
      if (lane == 0) {
        const int st = seg % S, k = seg / S;
        if (k > 0 && !mbar_wait_bounded(&r.empty[st], (k - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT))
          ok = 0;
        if (*(volatile int*)&r.abort_flag) ok = 0;
        if (ok) {
          unsigned char* sb = ring + st * plan.stage_bytes;
          mbar_arrive_expect_tx(&r.full[st],
                                (mol ? plan.mol_bytes : 0u) + (cia ? plan.cia_bytes : 0u));
          if (mol) tma_load_4d(sb, tm_sig, cur.x0, it, ip, 0, &r.full[st]);
          if (cia) tma_load_3d(sb + plan.mol_bytes, tm_cia, cur.x0, itc, 0, &r.full[st]);
        } else {
          atomicExch(&r.abort_flag, 1);
        }
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) { stop = true; break; }
      ++seg;
    }
    cur = nxt;
    have = have_next;
  }
  if (lane == 0)
    for (int st = 0; st < S && st < seg; ++st) {
      const int last = ((seg - 1 - st) / S) * S + st;
      mbar_wait_bounded(&r.full[st], (last / S) & 1, nullptr, 0);
    }
}

// Consumer side of one segment start: waits for the stage (false: give up, the caller
// returns), forms the sums over molecules us[c][v] = sum_m x_m sigma_m,c at the VW
// wavenumbers col0 .. col0+VW-1 of the tile (corners c = (P_i,T_j) (P_i,T_j+1) (P_i+1,T_j)
// (P_i+1,T_j+1)) when `mol`, and over CIA pairs uc[t][v] = sum_q y_q sigma_q,t when `cia`,
// then releases the stage (one arrive per warp).
template <int TW, int VW, int MAXMOL, int MAXCIA, bool F16>
__device__ __forceinline__ bool ring_consume(const FwdParams& p, Ring& r, const RingPlan& plan,
                                             const unsigned char* ring, int seg, bool mol,
                                             bool cia, int col0, const float* xm,
                                             const float* yq, float (&us)[4][VW],
                                             float (&uc)[2][VW], int lane) {
  static_assert(VW == 1 || VW == 2, "one or two wavenumbers per lane");
  const int S = plan.stages;
  const int st = seg % S, k = seg / S;
  const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&r.full[st], k & 1, p.dev_err,
                                                             TR_DEVERR_TIMEOUT) &&
                                              !*(volatile int*)&r.abort_flag);
  if (!ok) { if (lane == 0) atomicExch(&r.abort_flag, 1); return false; }
  const unsigned char* sb = ring + st * plan.stage_bytes;
  if constexpr (VW == 2 && !F16) {
    // FP32 rows, two wavenumbers: the sums as packed pairs (fma.rn.f32x2, each half rounded as
    // fmaf in the same order: the same values as scalar FMAs with half the instructions)
    if (mol) {
      unsigned long long x2[MAXMOL];
#pragma unroll
      for (int m = 0; m < MAXMOL; ++m) x2[m] = pack_dup(xm[m]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        unsigned long long s2 = 0ull;
#pragma unroll
        for (int m = 0; m < MAXMOL; ++m)
          if (m < p.n_mol) {
            const int e = (m * 4 + c) * TW + col0;   // box order: wn, T, P, molecule
            ffma2(s2, x2[m], *reinterpret_cast<const unsigned long long*>(
                                 reinterpret_cast<const float*>(sb) + e));
          }
        const float2 sum = *reinterpret_cast<const float2*>(&s2);
        us[c][0] = sum.x;
        us[c][1] = sum.y;
      }
    }
    if (cia) {
      const float* cbuf = reinterpret_cast<const float*>(sb + plan.mol_bytes);
#pragma unroll
      for (int t2 = 0; t2 < 2; ++t2) {
        unsigned long long s2 = 0ull;
#pragma unroll
        for (int q = 0; q < MAXCIA; ++q)
          if (q < p.n_cia)
            ffma2(s2, pack_dup(yq[q]),
                  *reinterpret_cast<const unsigned long long*>(cbuf + (2 * q + t2) * TW + col0));
        const float2 sum = *reinterpret_cast<const float2*>(&s2);
        uc[t2][0] = sum.x;
        uc[t2][1] = sum.y;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&r.empty[st]);       // this warp is done with the stage
    return true;
  }
  if (mol) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float s[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) s[v] = 0.f;
#pragma unroll
      for (int m = 0; m < MAXMOL; ++m) {
        if (m < p.n_mol) {
          const int e = (m * 4 + c) * TW + col0;   // box order: wn, T, P, molecule
          float v[VW];
          if constexpr (F16) {
            const __half* hp = reinterpret_cast<const __half*>(sb) + e;
            const float off = p.logsig_off[m];
            if constexpr (VW == 2) {
              const float2 hv = __half22float2(*reinterpret_cast<const __half2*>(hp));
              v[0] = ex2_fast((hv.x + off) * kLog2Of10);
              v[1] = ex2_fast((hv.y + off) * kLog2Of10);
            } else {
              v[0] = ex2_fast((__half2float(*hp) + off) * kLog2Of10);
            }
          } else {
            const float* fp = reinterpret_cast<const float*>(sb) + e;
            if constexpr (VW == 2) {
              const float2 fv = *reinterpret_cast<const float2*>(fp);
              v[0] = fv.x; v[1] = fv.y;
            } else {
              v[0] = *fp;
            }
          }
#pragma unroll
          for (int q = 0; q < VW; ++q) s[q] = fmaf(xm[m], v[q], s[q]);
        }
      }
#pragma unroll
      for (int v = 0; v < VW; ++v) us[c][v] = s[v];
    }
  }
  if (cia) {
    const float* cbuf = reinterpret_cast<const float*>(sb + plan.mol_bytes);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      float s[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) s[v] = 0.f;
#pragma unroll
      for (int q = 0; q < MAXCIA; ++q) {
        if (q < p.n_cia) {
          const float* fp = cbuf + (2 * q + t) * TW + col0;
          if constexpr (VW == 2) {
            const float2 fv = *reinterpret_cast<const float2*>(fp);
            s[0] = fmaf(yq[q], fv.x, s[0]); s[1] = fmaf(yq[q], fv.y, s[1]);
          } else {
            s[0] = fmaf(yq[q], *fp, s[0]);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < VW; ++v) uc[t][v] = s[v];
    }
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&r.empty[st]);         // this warp is done with the stage
  return true;
}

// Consumer side of one segment start for the exponential temperature scheme (Sec. 5): the
// molecules' interpolation in T is not linear, so no sum over molecules can be taken per
// segment; instead, for every molecule m, P row r (P_i, P_i+1) and wavenumber v, the two
// bracketing values s1 (T_j) and s2 (T_j+1) become lg[m][r][v] = log2(x_m s1) + kExpScaleLog2
// and dg[m][r][v] = log2 s2 - log2 s1, and each layer takes 2^(lg + u dg) = 2^64 x_m
// s1^(1-u) s2^u with its exponential weight u.  The molecule weight x_m rides in the exponent,
// and the 2^64 scale keeps the products normal FP32 numbers (x_m s1 can lie below FP32's
// smallest normal); the layer sum is multiplied by 2^-64.  A pair with a value that is not a
// positive normal number keeps lg = 2^64 x_m s1, dg = 2^64 x_m (s2 - s1) and its bit in `lin`
// (the linear value lg + t dg is used, t the layer's linear weight); `anylin` tells whether
// any lane of the warp holds such a pair.  FP16 rows give log2 sigma directly
// (h + c_m) log2 10; -inf (sigma = 0) marks a pair linear.  CIA sums as in ring_consume.
constexpr float kExpScaleLog2 = 64.f;
constexpr float kExpScale = 18446744073709551616.f;          // 2^64
constexpr float kExpScaleInv = 5.42101086242752217004e-20f;  // 2^-64
template <int TW, int MAXMOL, int MAXCIA, bool F16>
__device__ __forceinline__ bool ring_consume_exp(const FwdParams& p, Ring& r,
                                                 const RingPlan& plan, const unsigned char* ring,
                                                 int seg, bool mol, bool cia, int col0,
                                                 const float* xm, const float* yq,
                                                 float (&lg)[MAXMOL][2][2],
                                                 float (&dg)[MAXMOL][2][2], unsigned& lin,
                                                 bool& anylin, float (&uc)[2][2], int lane) {
  const int S = plan.stages;
  const int st = seg % S, k = seg / S;
  const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&r.full[st], k & 1, p.dev_err,
                                                             TR_DEVERR_TIMEOUT) &&
                                              !*(volatile int*)&r.abort_flag);
  if (!ok) { if (lane == 0) atomicExch(&r.abort_flag, 1); return false; }
  const unsigned char* sb = ring + st * plan.stage_bytes;
  if (mol) {
    lin = 0u;
#pragma unroll
    for (int m = 0; m < MAXMOL; ++m) {
      if (m < p.n_mol) {
        const float lx = lg2_fast(xm[m]) + kExpScaleLog2;   // -inf for x_m = 0: terms vanish
        const float sx = xm[m] * kExpScale;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int e1 = (m * 4 + 2 * rr) * TW + col0, e2 = e1 + TW;   // T_j, T_j+1 rows
          float a[2], b[2];
          bool pos[2];
          if constexpr (F16) {
            const float2 h1 = __half22float2(*reinterpret_cast<const __half2*>(
                reinterpret_cast<const __half*>(sb) + e1));
            const float2 h2 = __half22float2(*reinterpret_cast<const __half2*>(
                reinterpret_cast<const __half*>(sb) + e2));
            const float off = p.logsig_off[m];
            a[0] = (h1.x + off) * kLog2Of10; a[1] = (h1.y + off) * kLog2Of10;
            b[0] = (h2.x + off) * kLog2Of10; b[1] = (h2.y + off) * kLog2Of10;
            pos[0] = isfinite(a[0]) && isfinite(b[0]);
            pos[1] = isfinite(a[1]) && isfinite(b[1]);
#pragma unroll
            for (int v = 0; v < 2; ++v)
              if (!pos[v]) { a[v] = ex2_fast(a[v]); b[v] = ex2_fast(b[v]); }   // sigma values
          } else {
            const float2 s1 = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(sb) + e1);
            const float2 s2 = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(sb) + e2);
            a[0] = s1.x; a[1] = s1.y; b[0] = s2.x; b[1] = s2.y;
            constexpr float kMinNormal = 1.17549435e-38f;
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              pos[v] = a[v] >= kMinNormal && b[v] >= kMinNormal;
              if (pos[v]) { a[v] = lg2_fast(a[v]); b[v] = lg2_fast(b[v]); }
            }
          }
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            lg[m][rr][v] = pos[v] ? a[v] + lx : sx * a[v];
            dg[m][rr][v] = pos[v] ? b[v] - a[v] : sx * (b[v] - a[v]);
            if (!pos[v]) lin |= 1u << ((m * 2 + rr) * 2 + v);
          }
        }
      }
    }
    anylin = __any_sync(0xffffffffu, lin != 0u);
  }
  if (cia) {
    const float* cbuf = reinterpret_cast<const float*>(sb + plan.mol_bytes);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int q = 0; q < MAXCIA; ++q) {
        if (q < p.n_cia) {
          const float2 fv = *reinterpret_cast<const float2*>(cbuf + (2 * q + t) * TW + col0);
          s0 = fmaf(yq[q], fv.x, s0); s1 = fmaf(yq[q], fv.y, s1);
        }
      }
      uc[t][0] = s0; uc[t][1] = s1;
    }
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&r.empty[st]);         // this warp is done with the stage
  return true;
}

// Weights of the molecule and CIA-pair sums of item b in chemistry zone `zone`.
template <int MAXMOL, int MAXCIA>
__device__ __forceinline__ void item_weights(const FwdParams& p, int b, int zone,
                                             float (&xm)[MAXMOL], float (&yq)[MAXCIA]) {
  const float* ox = p.buf.opx + ((size_t)b * kMaxZones + zone) * kOpxStride;
#pragma unroll
  for (int m = 0; m < MAXMOL; ++m) xm[m] = m < p.n_mol ? __ldg(ox + m) : 0.f;
#pragma unroll
  for (int q = 0; q < MAXCIA; ++q) yq[q] = q < p.n_cia ? __ldg(ox + TR_MAX_MOL + q) : 0.f;
}

// Rayleigh cross-section sum_s X_s sigma_R,s (scaled per species) at table columns w and
// w + 1 (w even): every species' coefficient and row pair are loaded together, then summed in
// species order.
__device__ __forceinline__ float2 rayleigh2(const FwdParams& p, int b, int zone, int w) {
  float2 r = make_float2(0.f, 0.f);
  if (!p.ray || w >= p.wn_pad) return r;
  const float* rc = p.buf.rayc + ((size_t)b * kMaxZones + zone) * TR_MAX_SPECIES;
  float c[TR_MAX_SPECIES];
  float2 v[TR_MAX_SPECIES];
#pragma unroll
  for (int s = 0; s < TR_MAX_SPECIES; ++s) {
    const bool on = s < p.n_species;
    c[s] = on ? __ldg(rc + s) : 0.f;
    v[s] = on ? __ldg(reinterpret_cast<const float2*>(p.ray + (size_t)s * p.wn_pad + w))
              : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int s = 0; s < TR_MAX_SPECIES; ++s) {
    r.x = fmaf(c[s], v[s].x, r.x);
    r.y = fmaf(c[s], v[s].y, r.y);
  }
  return r;
}

}  // namespace tr
