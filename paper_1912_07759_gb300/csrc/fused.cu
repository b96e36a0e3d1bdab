// fused.cu -- FP32 forward model in one persistent kernel: opacity K[layer, wn] (Sec. 5 linear
// P/T interpolation, weighted by rho X and fused with Rayleigh, CIA and the grey cloud as in
// Sec. 8.1), slant optical depth tau[ray, wn] = sum_{l >= j} DL[j][l] K[l][wn] (Sec. 4, eqs.
// tot_opt_dpth, opt_dpth, cia_opt_dpth) and transit depth
// D = (R_p/R_s)^2 + sum_j a_j (1 - exp(-tau_j)) (Sec. 4, eqs. Delta_lambda, a_lambda).
//
// Work unit = one item x kFT consecutive wavenumbers; a persistent grid of one CTA per SM walks
// the units (items fastest).  The CTA's warps specialise:
//   warp 0      producer: streams every unit's table-row segments through a ring of
//               shared-memory stages by TMA (opacity.h), running ahead across units;
//   warps 1-6   opacity: build each unit's K tile [N][kFT] in shared memory, two wavenumbers
//               per lane, in kFOG groups of kFGW warps, group g taking the segments s with
//               s % kFOG == g (per segment the rows are summed over molecules and CIA pairs;
//               per layer four corner FMAs, two CIA FMAs, Rayleigh and cloud), alternating
//               between two tiles;
//   warps 7-14  contraction: while the next tile is being built, tau = DL K over 8-ray register
//               tiles x 4 wavenumbers per lane (the triangle l >= j only; tiles dealt
//               longest-first to the least-loaded warp, a fixed schedule so results do not
//               depend on timing; the item's path lengths in shared memory), the epilogue
//               sum_j a_j (1 - e^-tau_j), then the warps' partial depths added in FP64 in a
//               fixed order.
// Tiles pass between the groups through full / empty mbarriers (the "full" one also covers the
// bulk copy of the item's packed path lengths and annulus weights into the tile's geometry
// buffer, made by warp 1 when the item changes); K never leaves the SM, so the
// memory-bound opacity and the FMA-bound contraction overlap.  After a bounded wait gives up,
// warps leave; the contraction warps leave together at their named barrier.
#include <algorithm>
#include "opacity.h"
#include "tma.h"
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kFT = kFusedTile;                    // wavenumbers per unit
constexpr int kFOG = 3;                            // opacity groups (segment s -> group s % kFOG)
constexpr int kFGW = 2;                            // warps per opacity group (two wn per lane)
constexpr int kFOW = kFOG * kFGW;                  // opacity warps
constexpr int kFCW = 8;                            // contraction warps
constexpr int kFThreads = 32 * (1 + kFOW + kFCW);  // + one producer warp (warp 0)
constexpr int kFRT = 8;                            // rays per register tile
static_assert(kFT == 64 * kFGW, "two wavenumbers per opacity lane");
static_assert(kFT == 4 * 32, "four wavenumbers per contraction lane");

__host__ __device__ inline uint32_t align128(uint32_t x) { return (x + 127u) & ~127u; }

// Dynamic shared memory of one CTA (byte offsets from a 128-byte aligned base): the ring,
// `k_bufs` K tiles (2: the opacity and contraction warps overlap; 1 when two do not fit),
// `dl_bufs` copies of an item's packed path lengths and annulus weights (2 only with two K
// tiles and more than one item), and the contraction warps' partial depths.
struct FusedLayout {
  uint32_t kt0, kt1, dl0, dl1, aj0, aj1, red, total;
  __host__ __device__ FusedLayout(uint32_t ring_bytes, int max_layers, int k_bufs, int dl_bufs) {
    const uint32_t ktb = align128((uint32_t)(max_layers * kFT * 4));
    const uint32_t dlb = align128((uint32_t)(dlp_offset(max_layers) * 4));
    const uint32_t ajb = align128((uint32_t)(pad8(max_layers) * 4));
    kt0 = align128(ring_bytes);
    kt1 = k_bufs > 1 ? kt0 + ktb : kt0;
    dl0 = kt1 + ktb;
    dl1 = dl_bufs > 1 ? dl0 + dlb : dl0;
    aj0 = dl1 + dlb;
    aj1 = dl_bufs > 1 ? aj0 + ajb : aj0;
    red = aj1 + ajb;
    total = red + (uint32_t)(kFCW * kFT * 4) + 128u;   // + base alignment slack
  }
};

__device__ __forceinline__ void contraction_sync() {
  asm volatile("bar.sync 1, %0;" :: "r"(kFCW * 32) : "memory");
}

template <int MAXMOL, int MAXCIA>
__global__ void __launch_bounds__(kFThreads, 1)
k_forward_tma(FwdParams p, const __grid_constant__ CUtensorMap tm_sig,
              const __grid_constant__ CUtensorMap tm_cia, int B, int n_tiles, int n_stages,
              int k_bufs, int dl_bufs) {
  extern __shared__ unsigned char fsm_raw[];
  __shared__ Ring rs;
  __shared__ __align__(8) uint64_t kfull[2];         // K tile written, geometry landed
  __shared__ __align__(8) uint64_t kempty[2];        // K tile read (kFCW arrivals)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool has_mol = p.n_mol > 0, has_cia = p.n_cia > 0;
  const RingPlan plan(kFT, p.n_mol, p.n_cia, 4, n_stages);
  const FusedLayout lay(plan.bytes(), p.max_layers, k_bufs, dl_bufs);
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(fsm_raw) + 127) & ~(uintptr_t)127);
  unsigned char* ring = base;
  if (threadIdx.x == 0) {
    ring_init(rs, plan.stages, kFGW);                // a stage is read by one group
    // kfull: kFOW warp arrivals + one arrival (with the geometry bytes, if any) by warp 1
    for (int i = 0; i < 2; ++i) { mbar_init(&kfull[i], kFOW + 1); mbar_init(&kempty[i], kFCW); }
    mbar_fence_init();
  }
  __syncthreads();
  const long long n_units = (long long)B * n_tiles;
  const int wbase = wn_first(p.wn_begin);
  if (warp == 0) {
    ring_produce<kFT>(p, rs, plan, ring, &tm_sig, &tm_cia, B, n_units, lane, true);
    return;
  }
  float* const K0 = reinterpret_cast<float*>(base + lay.kt0);
  float* const K1 = reinterpret_cast<float*>(base + lay.kt1);
  float* const D0 = reinterpret_cast<float*>(base + lay.dl0);
  float* const D1 = reinterpret_cast<float*>(base + lay.dl1);
  float* const A0 = reinterpret_cast<float*>(base + lay.aj0);
  float* const A1 = reinterpret_cast<float*>(base + lay.aj1);

  if (warp <= kFOW) {
    // ---------------- opacity warps: group g takes the segments s with s % kFOG == g; a lane
    // owns two wavenumbers; the K tile of every valid unit, alternating buffers
    const int ow = warp - 1;                         // 0 .. kFOW-1
    const int g = ow / kFGW;                         // opacity group
    const int c2 = 2 * (32 * (ow % kFGW) + lane);    // first of the lane's two columns
    int seg = 0, k_u = 0;
    int dl_item0 = -1, dl_item1 = -1;                // items held by the geometry buffers
    for (long long u = blockIdx.x; u < n_units; u += gridDim.x) {
      const int bc = (int)(u % B), tile = (int)(u / B);
      const int b = p.b_off + bc;
      const int N = p.buf.items[b].n_layers;
      if (N == 0) continue;
      const int kb = k_bufs > 1 ? (k_u & 1) : 0, use = k_bufs > 1 ? (k_u >> 1) : k_u;
      ++k_u;
      // wait until the contraction warps are done with this buffer's previous tile
      const bool ok = use == 0 || __all_sync(0xffffffffu, mbar_wait_bounded(
                                     &kempty[kb], (use - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT));
      if (!ok || *(volatile int*)&rs.abort_flag) { if (lane == 0) atomicExch(&rs.abort_flag, 1); return; }
      // warp 1: the item's packed path lengths and annulus weights into the tile's geometry
      // buffer unless it holds them already; one arrival on kfull either way
      const int gb = dl_bufs > 1 ? kb : 0;
      if (warp == 1 && lane == 0) {
        int& held = gb ? dl_item1 : dl_item0;
        if (held != b) {
          held = b;
          const uint32_t dl_bytes = (uint32_t)(dlp_offset(N) * 4);
          const uint32_t a_bytes = (uint32_t)(p.buf.npad * 4);
          mbar_arrive_expect_tx(&kfull[kb], dl_bytes + a_bytes);
          bulk_g2s(gb ? D1 : D0, p.buf.dlp + (size_t)b * dlp_offset(p.max_layers), dl_bytes, &kfull[kb]);
          bulk_g2s(gb ? A1 : A0, p.buf.aj + (size_t)b * p.buf.npad, a_bytes, &kfull[kb]);
        } else {
          mbar_arrive(&kfull[kb]);
        }
      }
      float* Kt = kb ? K1 : K0;
      const int w = wbase + tile * kFT + c2;
      const bool in_row = w < p.wn_pad;
      const LayerDesc* L = p.buf.layers + (size_t)b * p.max_layers;
      const float4* op = p.buf.op + (size_t)b * p.max_layers * 2;
      // constant mixing ratios only (run_forward keeps two-layer gases off this kernel):
      // chemistry zone 0
      const float2 ray = rayleigh2(p, b, 0, w);
      const float ray0 = ray.x, ray1 = ray.y;
      float xm[MAXMOL], yq[MAXCIA];
      item_weights<MAXMOL, MAXCIA>(p, b, 0, xm, yq);
      float us[4][2] = {}, uc[2][2] = {};
      int cip = -1, cit = -1, citc = -1, czone = -1;
      bool mine = false;                             // the current segment is this group's
      for (int l0 = 0; l0 < N; l0 += 32) {
        const int li = l0 + lane;
        int4 h = make_int4(-1, -1, -1, 0);
        float4 ha = make_float4(0.f, 0.f, 0.f, 0.f), hb = ha;
        if (li < N) {
          h = __ldg(reinterpret_cast<const int4*>(L + li));
          ha = __ldg(op + 2 * li);
          hb = __ldg(op + 2 * li + 1);
        }
        const SegFlags f = segment_flags<false>(h, l0, 0, N, lane, has_mol, has_cia, cip, cit,
                                                citc, czone);
        const int n_here = min(32, N - l0);
        for (int i = 0; i < n_here; ++i) {
          if ((f.start >> i) & 1u) {
            mine = seg % kFOG == g;
            // the molecular cell or CIA bracket may carry over from earlier segments, which
            // other groups took: reload both sums for every segment this group takes
            if (mine && !ring_consume<kFT, 2, MAXMOL, MAXCIA, false>(p, rs, plan, ring, seg,
                                                                      has_mol, has_cia, c2, xm,
                                                                      yq, us, uc, lane))
              return;
            ++seg;
          }
          if (!mine) continue;
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
          *reinterpret_cast<float2*>(Kt + (l0 + i) * kFT + c2) =
              in_row ? make_float2(k0, k1) : make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&kfull[kb]);        // this warp's rows are written
    }
    return;
  }

  // ---------------- contraction warps: tau = DL K, 1 - e^-tau, depth
  const int cw = warp - 1 - kFOW;                    // 0 .. kFCW-1
  const int tid = cw * 32 + lane;                    // 0 .. 32 kFCW - 1
  float* red = reinterpret_cast<float*>(base + lay.red);   // [kFCW][kFT]
  bool failed = false;
  int k_u = 0;
  for (long long u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int bc = (int)(u % B), tile = (int)(u / B);
    const int b = p.b_off + bc;
    const ItemGeom ig = p.buf.items[b];
    const int N = ig.n_layers;
    const int w_first = wbase + tile * kFT;
    double* out = p.out + (long long)b * p.out_stride;
    if (N == 0) {                                    // invalid item: zero depth
      if (tid < kFT) {
        const int w = w_first + tid;
        if (w >= p.wn_begin && w < p.wn_begin + p.wn_count) out[w - p.wn_begin] = 0.0;
      }
      continue;
    }
    const int kb = k_bufs > 1 ? (k_u & 1) : 0, use = k_bufs > 1 ? (k_u >> 1) : k_u;
    ++k_u;
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    if (!failed) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&kfull[kb], use & 1, p.dev_err,
                                                                TR_DEVERR_TIMEOUT));
      if (!ok) { failed = true; if (lane == 0) atomicExch(&rs.abort_flag, 1); }
    }
    if (!failed) {
      const float* Kt = kb ? K1 : K0;
      const int gb = dl_bufs > 1 ? kb : 0;
      const float* dl = gb ? D1 : D0;
      const float* aj = gb ? A1 : A0;
      // ray tiles longest-first to the least-loaded warp (fixed schedule)
      const int n_rt = (N + kFRT - 1) / kFRT;
      int ld[kFCW];
#pragma unroll
      for (int k = 0; k < kFCW; ++k) ld[k] = 0;
      for (int t = 0; t < n_rt; ++t) {
        int wm = 0, lm = ld[0];
#pragma unroll
        for (int k = 1; k < kFCW; ++k) if (ld[k] < lm) { wm = k; lm = ld[k]; }
        const int len = N - t * kFRT;
#pragma unroll
        for (int k = 0; k < kFCW; ++k) ld[k] += k == wm ? len : 0;
        if (wm != cw) continue;
        const int j0 = t * kFRT;
        float acc[kFRT][4];
#pragma unroll
        for (int r = 0; r < kFRT; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
        int off = dlp_offset(j0);
        float4 kv = *reinterpret_cast<const float4*>(Kt + j0 * kFT + 4 * lane);
        float4 d0 = *reinterpret_cast<const float4*>(dl + off + j0);
        float4 d1 = *reinterpret_cast<const float4*>(dl + off + j0 + 4);
        for (int l = j0; l < N; ++l) {
          // the next row's operands are loaded before this row's FMAs (one row ahead)
          off += pad8(l + 1);
          const int ln = min(l + 1, N - 1);
          const int offn = l + 1 < N ? off : off - pad8(l + 1);
          const float4 kn = *reinterpret_cast<const float4*>(Kt + ln * kFT + 4 * lane);
          const float4 e0 = *reinterpret_cast<const float4*>(dl + offn + j0);
          const float4 e1 = *reinterpret_cast<const float4*>(dl + offn + j0 + 4);
          const float dv[kFRT] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
          for (int r = 0; r < kFRT; ++r) {
            acc[r][0] = fmaf(dv[r], kv.x, acc[r][0]);
            acc[r][1] = fmaf(dv[r], kv.y, acc[r][1]);
            acc[r][2] = fmaf(dv[r], kv.z, acc[r][2]);
            acc[r][3] = fmaf(dv[r], kv.w, acc[r][3]);
          }
          kv = kn; d0 = e0; d1 = e1;
        }
        // 1 - e^-tau with the hardware exponential: its absolute error (a few 1e-7) times the
        // annulus weights (sum ~ 1e-3) stays below 1e-9 in depth, far inside 0.1 ppm
#pragma unroll
        for (int r = 0; r < kFRT; ++r) {
          const float a = aj[j0 + r];
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) part[c4] = fmaf(a, 1.f - __expf(-acc[r][c4]), part[c4]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&kempty[kb]);       // this warp is done reading the tile
    }
    *reinterpret_cast<float4*>(red + cw * kFT + 4 * lane) =
        make_float4(part[0], part[1], part[2], part[3]);
    contraction_sync();                              // all partial depths written
    if (*(volatile int*)&rs.abort_flag) return;      // every contraction warp sees the same
    // FP64 sum of the warps' partial depths in a fixed order
    if (tid < kFT) {
      const int w = w_first + tid;
      if (w >= p.wn_begin && w < p.wn_begin + p.wn_count) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kFCW; ++k) s += (double)red[k * kFT + tid];
        out[w - p.wn_begin] = ig.rp2_rs2 + s;
      }
    }
    contraction_sync();                              // red is free again
  }
}

// Ring depth for `ctas` CTAs per SM of `fixed` bytes besides the ring each: as many stages as
// fit the SM's shared memory, at most kRingMaxStages (0 when not even 2 fit).
int fused_ring_stages(uint32_t stage_bytes, int ctas, uint32_t fixed) {
  constexpr uint32_t kSmemPerSm = 227u * 1024u;   // usable by the CTAs of one SM
  const uint32_t sb = stage_bytes > 0 ? stage_bytes : 128u;
  const uint32_t per = kSmemPerSm / (uint32_t)ctas - 1024u - 512u;   // runtime reserve, statics
  const int s = per > fixed ? (int)((per - fixed) / sb) : 0;
  return s >= 2 ? std::min(s, kRingMaxStages) : 0;
}

int fused_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Wavenumber tiles of the computed native range.
int wn_first_tiles(const FwdParams& p) {
  const int w0 = wn_first(p.wn_begin);
  return (p.wn_begin + p.wn_count - w0 + kFT - 1) / kFT;
}

// Buffer counts of the fused kernel for these sizes (k_bufs 0: it does not fit) and the
// deepest ring that fits them.
struct FusedBuffers { int k_bufs, dl_bufs, stages; };
FusedBuffers fused_buffers(int n_mol, int n_cia, int max_layers, int B) {
  const RingPlan one(kFT, n_mol, n_cia, 4, 1);
  const int dl2 = B > 1 ? 2 : 1;
  int st = fused_ring_stages(one.stage_bytes, 1, FusedLayout(0, max_layers, 2, dl2).total);
  if (st >= 2) return {2, dl2, st};
  st = fused_ring_stages(one.stage_bytes, 1, FusedLayout(0, max_layers, 1, 1).total);
  if (st >= 2) return {1, 1, st};
  return {0, 0, 0};
}

template <int MAXMOL, int MAXCIA>
cudaError_t launch_fused_t(const FwdParams& p, const CUtensorMap& sig, const CUtensorMap& cia,
                           int B, int stages_cap, FusedChoice* used, cudaStream_t s) {
  auto kern = k_forward_tma<MAXMOL, MAXCIA>;
  const FusedBuffers fb = fused_buffers(p.n_mol, p.n_cia, p.max_layers, B);
  if (fb.k_bufs == 0) return cudaErrorInvalidConfiguration;
  const int stages = stages_cap > 0 ? std::min(fb.stages, std::max(2, stages_cap)) : fb.stages;
  const RingPlan plan(kFT, p.n_mol, p.n_cia, 4, stages);
  const uint32_t smem = FusedLayout(plan.bytes(), p.max_layers, fb.k_bufs, fb.dl_bufs).total;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = wn_first_tiles(p);
  const long long units = (long long)B * tiles;
  const int grid = (int)std::min<long long>(units, (long long)fused_sm_count());
  if (used) { used->k_bufs = fb.k_bufs; used->stages = stages; }
  kern<<<grid, kFThreads, smem, s>>>(p, sig, cia, B, tiles, stages, fb.k_bufs, fb.dl_bufs);
  return cudaGetLastError();
}

}  // namespace

bool fused_forward_fits(int n_mol, int n_cia, int max_layers, int B) {
  return fused_buffers(n_mol, n_cia, max_layers, B).k_bufs > 0;
}

cudaError_t launch_forward_fused(const FwdParams& p, const CUtensorMap* tm_sig,
                                 const CUtensorMap* tm_cia, int B, int stages_cap,
                                 FusedChoice* used, cudaStream_t s) {
  if (B <= 0 || p.wn_count <= 0) return cudaSuccess;
  static_assert(TR_MAX_MOL == 8 && TR_MAX_CIA == 4, "fused instantiations cover the limits");
  if (p.n_cia <= 2) {
    if (p.n_mol <= 2) return launch_fused_t<2, 2>(p, *tm_sig, *tm_cia, B, stages_cap, used, s);
    if (p.n_mol <= 5) return launch_fused_t<5, 2>(p, *tm_sig, *tm_cia, B, stages_cap, used, s);
    return launch_fused_t<8, 2>(p, *tm_sig, *tm_cia, B, stages_cap, used, s);
  }
  if (p.n_mol <= 2) return launch_fused_t<2, 4>(p, *tm_sig, *tm_cia, B, stages_cap, used, s);
  if (p.n_mol <= 5) return launch_fused_t<5, 4>(p, *tm_sig, *tm_cia, B, stages_cap, used, s);
  return launch_fused_t<8, 4>(p, *tm_sig, *tm_cia, B, stages_cap, used, s);
}

}  // namespace tr
