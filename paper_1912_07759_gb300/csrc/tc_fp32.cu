// tc_fp32.cu -- the FP32 path's slant optical depth tau[ray, wn] = sum_{l >= j} DL[j][l] K[l][wn]
// (Sec. 4, eqs. tot_opt_dpth, opt_dpth) on the 5th-generation tensor cores as three TF32
// products (3xTF32), and the transit depth D = (R_p/R_s)^2 + sum_j a_j (1 - e^-tau_j) (Sec. 4).
// Every FP32 operand x is split exactly into hi = x with its 13 low mantissa bits cleared (a
// TF32 value) and lo = x - hi, and tau = K_hi DL_hi + K_hi DL_lo + K_lo DL_hi is accumulated in
// FP32 in tensor memory.  The dropped K_lo DL_lo term and the TF32 rounding of the lo parts
// each stay below 2^-20 of a product, the size of FP32 accumulation error over the column.
//
// k_contract_tc: persistent, one CTA per SM over a contiguous range of (item, 128-wn) units.
// A unit's layers are taken as two halves (the top half first): each half is a job of its own
// for the splitters and the MMA, so the split of one half overlaps the MMAs of the one before.
// The kernel is instantiated per padded layer count, so the MMA issue and split loops are
// unrolled with constant operands: issued from a runtime loop, the MMAs went at about half the
// rate (the issuing thread, not the tensor pipe, set the pace).
// Warp roles, every hand-over through an mbarrier:
//   * warp 8 (producer): TMA loads of the unit's FP32 K tile [KP layers][128 wn] (boxes of 8
//     rows of the opacity kernel's K buffer) into one of two stages;
//   * warps 0-3 and 10-13 (splitters; thread = TMEM lane = one wavenumber of the unit, the two
//     warps of a lane quarter taking alternate 8-layer groups): when the item changes (once
//     every MMA of the previous unit is done), one thread bulk-copies the item's path-length
//     tiles DL_hi / DL_lo (rays x layers, K-major core matrices, built once per item by
//     k_dl_tf32) into shared memory; per half, each thread splits its wavenumber's K values of
//     the half's layers (zero at and beyond N) and stores K_hi and K_lo into one of two TMEM
//     half buffers (the MMA's A operand, column = layer);
//   * warp 9 (one thread): per half, for its 8-layer slices from the top down, three MMAs
//     D[128 x N_ks] (+)= A[128 x 8] B[N_ks x 8]^T, N_ks the rays the slice reaches (DL = 0 for
//     rays above a layer), into the unit's one of two TMEM accumulators; a commit frees the
//     half buffer, one after the bottom half hands the accumulator to the epilogue;
//   * warps 4-7 (epilogue): tau from TMEM -> sum_j a_j (1 - e^-tau_j) -> FP64 depth.
// All waits are bounded; on a timeout every role stops, in-flight copies and MMAs are waited
// for (bounded) and the TMEM is released before the CTA exits.
#include <algorithm>
#include "tma.h"
#include "tr_internal.h"
#include "umma.h"

namespace tr {
namespace {

constexpr int kTM = 128;                  // wavenumbers per unit = MMA M = TMEM lanes
constexpr int kTEpi0 = 4;                 // epilogue warps 4..7
constexpr int kTProd = 8;
constexpr int kTMma = 9;
constexpr int kTSplit1 = 10;              // splitters: warps 0..3 and 10..13
constexpr int kTSplitters = 8;
constexpr int kTThreads = 32 * (kTSplit1 + 4);
constexpr int kTMaxKP = 112;              // layers (padded to 16) the kernel takes
// TMEM columns: half buffer h at 128 h (K_hi at + 0, K_lo at + 64, KP / 2 columns each);
// accumulators at 256 and 384 (NP columns)
constexpr uint32_t kColHalf = 128, kColLo = 64, kColD0 = 256, kColD1 = 384, kTmemCols = 512;

__host__ __device__ inline int pad16i(int n) { return (n + 15) & ~15; }

struct TcLayout {
  uint32_t stage, dl, aj, total;
  __host__ __device__ TcLayout(int KP, int NP) {
    stage = (uint32_t)KP * kTM * 4;                       // FP32 K tile [KP][128]
    dl = 2 * stage;                                       // DL_hi, DL_lo [NP][KP] TF32
    aj = dl + 2u * (uint32_t)NP * KP * 4;
    total = aj + 2u * kTM * 4 + 128u;                     // + alignment slack
  }
};

// x with the 13 low mantissa bits cleared: exactly a TF32 value, whatever rounding the tensor
// core applies to its inputs
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// The path-length tiles of every item, the MMA's B operand: tiles[b][0] = DL_hi, [b][1] =
// DL_lo, each [NP rays][KP layers] in the K-major core-matrix layout (core matrix m = (j / 8) *
// (KP / 4) + l / 4 of 8 rays x 4 layers, 128 bytes, row j % 8, column l % 4), zero for j > l and
// outside the item's N layers.  Grid (core matrices / 4, B items): a warp writes one core
// matrix per store (lane = (ray, layer) of it, one value each) from four 32-byte row segments
// of the geometry kernel's layer-major DL.
__global__ void __launch_bounds__(128)
k_dl_tf32(ItemBuffers buf, int max_layers, int NP, int KP, float* __restrict__ tiles) {
  const int b = blockIdx.y;
  const int cm_k = KP / 4, n_cm = (NP / 8) * cm_k;
  const int m = 4 * blockIdx.x + (threadIdx.x >> 5);        // core matrix of this warp
  if (m >= n_cm) return;
  const int lane = threadIdx.x & 31, r = lane >> 2, c = lane & 3;
  const int j = 8 * (m / cm_k) + r, l = 4 * (m % cm_k) + c;
  const int N = buf.items[b].n_layers;
  const float* dlt = buf.dlt + (size_t)b * max_layers * buf.npad;
  const float x = (l < N && j <= l) ? __ldg(dlt + (size_t)l * buf.npad + j) : 0.f;
  const float h = tf32_hi(x);
  float* hi = tiles + (size_t)b * 2 * NP * KP;
  hi[(size_t)m * 32 + lane] = h;                            // row r, column c: 4 r + c = lane
  hi[(size_t)NP * KP + (size_t)m * 32 + lane] = x - h;
}

// Barrier over `threads` threads (named barrier `id`) that also returns whether any of them
// passed pred = true: the warps of one role take the same stop decision.
__device__ __forceinline__ bool tc_sync_or(int id, int threads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r) : "r"((uint32_t)pred), "r"(id), "r"(threads) : "memory");
  return r != 0;
}

// Instantiated per padded layer count KP (16 .. 112): the MMA issue loop and the split loop are
// unrolled with constant operands (a runtime loop issued the MMAs at about half the rate).
template <int KP>
__global__ void __launch_bounds__(kTThreads, 1)
k_contract_tc(FwdParams p, const __grid_constant__ CUtensorMap tm_k, int Bc, int n_tiles,
              const float* __restrict__ tiles) {
  constexpr int NP = KP;                    // rays (padded) = layers (padded)
  extern __shared__ __align__(128) uint8_t tsm_raw[];
  __shared__ __align__(8) uint64_t sfull[2], sempty[2], hfull[2], hfree[2], accfull[2],
      accempty[2], dlfull;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tsm_raw) + 127) &
                                             ~(uintptr_t)127);
  const TcLayout lay(KP, NP);
  uint8_t* B_hi = base + lay.dl;
  uint8_t* B_lo = B_hi + (size_t)NP * KP * 4;
  float* ep_aj = reinterpret_cast<float*>(base + lay.aj);      // [2][128], epilogue's copy
  const long long units = (long long)Bc * n_tiles;
  const long long per = (units + gridDim.x - 1) / gridDim.x;
  const long long u_begin = (long long)blockIdx.x * per;
  const long long u_end = u_begin + per < units ? u_begin + per : units;
  const int n_units = u_end > u_begin ? (int)(u_end - u_begin) : 0;
  const int wbase = wn_first(p.wn_begin);
  constexpr int HL = KP / 2;                // layers of a half (a multiple of 8)

  if (warp == 0) tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sfull[i], 1); mbar_init(&sempty[i], kTSplitters);
      mbar_init(&hfull[i], kTSplitters); mbar_init(&hfree[i], 1);
      mbar_init(&accfull[i], 1); mbar_init(&accempty[i], 4);
    }
    mbar_init(&dlfull, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  tcgen05_fence_before();
  __syncthreads();
  tcgen05_fence_after();
  const uint32_t tmem = tmem_base;
  // launched as a dependent of the opacity kernel: only the set-up above overlaps its tail
  pdl_wait();                                   // K and the path-length tiles are written

  if (warp == kTProd) {
    // ---------------- producer
    if (lane == 0) {
      int k = 0;
      for (; k < n_units; ++k) {
        const long long u = u_begin + k;
        const int bc = (int)(u / n_tiles), tile = (int)(u % n_tiles);
        const int s = k & 1, q = k >> 1;
        const bool ok = q == 0 ||
                        mbar_wait_bounded(&sempty[s], (q - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
        if (!ok || *(volatile int*)&abort_flag) { atomicExch(&abort_flag, 1); break; }
        uint8_t* st = base + s * lay.stage;
        mbar_arrive_expect_tx(&sfull[s], lay.stage);
        for (int i = 0; i < KP / 8; ++i)
          tma_load_2d(st + (size_t)i * 8 * kTM * 4, &tm_k, tile * kTM,
                      bc * p.max_layers + i * 8, &sfull[s]);
      }
      for (int i = 0; i < 2 && i < k; ++i) {      // every copy issued has landed
        const int kl = k - 1 - i;
        mbar_wait_bounded(&sfull[kl & 1], (kl >> 1) & 1, nullptr, 0);
      }
    }
  } else if (warp < kTEpi0 || warp >= kTSplit1) {
    // ---------------- splitters: thread v = wavenumber row v of the unit = TMEM lane v
    const int v = 32 * (warp & 3) + lane;          // 0 .. 127
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int g0 = warp >= kTSplit1 ? 1 : 0;      // the two warps of a lane quarter take
                                                   // alternate 8-layer groups
    const uint32_t tile_bytes = (uint32_t)NP * KP * 4;
    int dl_item = -1, dl_issued = 0;
    for (int k = 0; k < n_units; ++k) {
      const long long u = u_begin + k;
      const int b = p.b_off + (int)(u / n_tiles);
      const int N = __ldg(&p.buf.items[b].n_layers);
      const int s = k & 1;
      if (b != dl_item) {
        // the item's path-length tiles replace the old ones once every MMA of unit k-1 is done
        // (the commit of its bottom half, half job 2k - 1, completes after all of them; the
        // splitters have waited for the commit of half job 2k - 3 before splitting unit k-1,
        // so this barrier is at most one phase behind the one waited for)
        bool dok = k == 0 || mbar_wait_bounded(&hfree[1], (k - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
        dok = dok && !*(volatile int*)&abort_flag;
        if (tc_sync_or(1, 32 * kTSplitters, !dok)) { if (lane == 0) atomicExch(&abort_flag, 1); break; }
        // one thread starts the copy; the MMA thread waits for it (the split does not need it)
        if (tid == 0) {
          const float* src = tiles + (size_t)b * 2 * NP * KP;
          mbar_arrive_expect_tx(&dlfull, 2u * tile_bytes);
          bulk_g2s(B_hi, src, tile_bytes, &dlfull);
          bulk_g2s(B_lo, src + (size_t)NP * KP, tile_bytes, &dlfull);
        }
        ++dl_issued;
        dl_item = b;
      }
      // the unit's K tile has landed
      const bool ok = mbar_wait_bounded(&sfull[s], (k >> 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT) &&
                      !*(volatile int*)&abort_flag;
      if (tc_sync_or(1, 32 * kTSplitters, !ok)) { if (lane == 0) atomicExch(&abort_flag, 1); break; }
      const float* kf = reinterpret_cast<const float*>(base + s * lay.stage);
      bool stop = false;
      for (int hh = 1; hh >= 0; --hh) {
        // half job h = 2k + (1 - hh) (the top half first) into half buffer h & 1, once the MMAs
        // of half job h - 2 are done with it
        const int h = 2 * k + (1 - hh), hb = h & 1, hq = h >> 1;
        bool hok = hq == 0 || mbar_wait_bounded(&hfree[hb], (hq - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
        hok = hok && !*(volatile int*)&abort_flag;
        if (tc_sync_or(1, 32 * kTSplitters, !hok)) { if (lane == 0) atomicExch(&abort_flag, 1); stop = true; break; }
        tcgen05_fence_after();
        const uint32_t col = tmem + lane_base + kColHalf * hb;
#pragma unroll
        for (int gg = 0; gg < (HL / 8 + 1) / 2; ++gg) {
          const int g = 2 * gg + g0;
          if (g >= HL / 8) break;
          uint32_t hi[8], lo[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int l = hh * HL + 8 * g + i;
            const float x = l < N ? kf[l * kTM + v] : 0.f;
            const float hv = tf32_hi(x);
            hi[i] = __float_as_uint(hv);
            lo[i] = __float_as_uint(x - hv);
          }
          tmem_st8(col + 8 * g, hi);
          tmem_st8(col + kColLo + 8 * g, lo);
        }
        tmem_st_wait();
        tcgen05_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&hfull[hb]);     // this warp's rows of the half are written
      }
      if (stop) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(&sempty[s]);       // this warp's reads of the stage are done
    }
    // the last tile copy has landed before the CTA may exit (the MMA thread observes every copy
    // but the last one when the CTA stops early)
    if (tid == 0 && dl_issued > 0) mbar_wait_bounded(&dlfull, (dl_issued - 1) & 1, nullptr, 0);
  } else if (warp == kTMma) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t sbo = (uint32_t)(KP / 4) * 128;
      const uint32_t bh = smem_addr(B_hi), bl = smem_addr(B_lo);
      uint64_t* last = nullptr;                     // the last commit issued and its phase
      int last_par = 0, dl_item = -1, dl_copies = 0;
      bool stop = false;
      for (int k = 0; k < n_units && !stop; ++k) {
        const int a = k & 1, q = k >> 1;
        const int b = p.b_off + (int)((u_begin + k) / n_tiles);
        bool ok = q == 0 ||
                  mbar_wait_bounded(&accempty[a], (q - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
        // a new item's path-length tiles have landed (the splitters copy them at the item's
        // first unit, after every MMA of the previous unit is done)
        if (ok && b != dl_item) {
          ok = mbar_wait_bounded(&dlfull, dl_copies & 1, p.dev_err, TR_DEVERR_TIMEOUT);
          ++dl_copies;
          dl_item = b;
        }
        if (!ok) { atomicExch(&abort_flag, 1); break; }
        const uint32_t d = tmem + (a ? kColD1 : kColD0);
        bool first = true;
#pragma unroll
        for (int hh = 1; hh >= 0; --hh) {
          const int h = 2 * k + (1 - hh), hb = h & 1, hq = h >> 1;
          ok = mbar_wait_bounded(&hfull[hb], hq & 1, p.dev_err, TR_DEVERR_TIMEOUT) &&
               !*(volatile int*)&abort_flag;
          if (!ok) { atomicExch(&abort_flag, 1); stop = true; break; }
          tcgen05_fence_after();
          const uint32_t ah = tmem + kColHalf * hb, al = ah + kColLo;
#pragma unroll
          for (int i = HL / 8 - 1; i >= 0; --i) {
            const int ks = hh * (HL / 8) + i;        // the slice's 8 layers: 8 ks .. 8 ks + 7
            // the rays slice ks reaches: j <= 8 ks + 7, rounded up to the MMA's N step of 16
            const int n = min(NP, pad16i(8 * ks + 8));
            const uint32_t idesc = umma_idesc_tf32_f32(kTM, n);
            const uint32_t koff = (uint32_t)ks * 256;          // two core matrices along K
            const uint64_t dh = umma_smem_desc(bh + koff, 128, sbo);
            const uint64_t dlo = umma_smem_desc(bl + koff, 128, sbo);
            umma_tf32_ta(d, ah + 8 * i, dh, idesc, first ? 0u : 1u);
            umma_tf32_ta(d, ah + 8 * i, dlo, idesc, 1u);
            umma_tf32_ta(d, al + 8 * i, dh, idesc, 1u);
            first = false;
          }
          umma_commit(&hfree[hb]);                  // the half buffer is free
          last = &hfree[hb];
          last_par = hq & 1;
        }
        if (!stop) umma_commit(&accfull[a]);        // the accumulator is ready
      }
      // the MMAs issued are complete before the CTA may release the TMEM (the last commit
      // issued completes after all of them)
      if (last) mbar_wait_bounded(last, (uint32_t)last_par, nullptr, 0);
    }
  } else if (warp < kTProd) {
    // ---------------- epilogue: thread = TMEM lane = wavenumber row
    const int q4 = warp - kTEpi0;
    const int row = 32 * q4 + lane;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    for (int k = 0; k < n_units; ++k) {
      const long long u = u_begin + k;
      const int bc = (int)(u / n_tiles), tile = (int)(u % n_tiles);
      const int b = p.b_off + bc;
      const ItemGeom ig = p.buf.items[b];
      const int a = k & 1;
      float* aj = ep_aj + a * kTM;
      if (row < NP) aj[row] = row < p.buf.npad ? __ldg(p.buf.aj + (size_t)b * p.buf.npad + row) : 0.f;
      const bool ok = mbar_wait_bounded(&accfull[a], (k >> 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT) &&
                      !*(volatile int*)&abort_flag;
      // aj of this unit in place; all epilogue warps stop together on a failed wait
      if (tc_sync_or(2, 128, !ok)) { if (lane == 0) atomicExch(&abort_flag, 1); break; }
      tcgen05_fence_after();
      const uint32_t taddr = tmem + lane_base + (a ? kColD1 : kColD0);
      float part = 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float tau[16];
        tmem_ld16(taddr + (uint32_t)c0, tau);
#pragma unroll
        for (int i = 0; i < 16; ++i) part = fmaf(aj[c0 + i], 1.f - __expf(-tau[i]), part);
      }
      tcgen05_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[a]);     // this warp's TMEM lanes are read
      const int w = wbase + tile * kTM + row;
      if (w >= p.wn_begin && w < p.wn_begin + p.wn_count)
        p.out[(long long)b * p.out_stride + (w - p.wn_begin)] =
            ig.n_layers > 0 ? ig.rp2_rs2 + (double)part : 0.0;
    }
  }
  tcgen05_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

size_t tc_dl_bytes(int B, int max_layers) {
  if (!tc_contract_fits(max_layers)) return 0;
  const size_t P = (size_t)pad16i(max_layers);
  return sizeof(float) * 2 * (size_t)B * P * P;
}

cudaError_t launch_dl_tf32(const ItemBuffers& buf, int B, int max_layers, void* tiles,
                           cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  if (!tc_contract_fits(max_layers)) return cudaErrorInvalidValue;
  const int P = pad16i(max_layers);
  const int n_cm = (P / 8) * (P / 4);
  k_dl_tf32<<<dim3((n_cm + 3) / 4, B), 128, 0, s>>>(buf, max_layers, P, P,
                                                    static_cast<float*>(tiles));
  return cudaGetLastError();
}

bool tc_contract_fits(int max_layers) {
  const int KP = pad16i(max_layers);
  return max_layers >= 1 && KP <= kTMaxKP && TcLayout(KP, KP).total <= 227u * 1024u;
}

cudaError_t launch_contract_tc(const FwdParams& p, int Bc, const float* kbuf, const void* tiles,
                               cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  if (!tc_contract_fits(p.max_layers)) return cudaErrorInvalidValue;
  const int KP = pad16i(p.max_layers), NP = KP;
  const int w_first = wn_first(p.wn_begin);
  if (!tiles) return cudaErrorInvalidValue;
  const int tiles_w = (p.wn_begin + p.wn_count - w_first + kTM - 1) / kTM;
  const long long kcols = (long long)tiles_w * kTM;
  CUtensorMap tm{};
  if (!encode_2d_f32(&tm, kbuf, (unsigned long long)kcols, (unsigned long long)Bc * p.max_layers,
                     (unsigned long long)kcols * 4, kTM, 8))
    return cudaErrorInvalidValue;
  const uint32_t smem = TcLayout(KP, NP).total;
  void (*kern)(FwdParams, CUtensorMap, int, int, const float*) = nullptr;
  switch (KP) {
    case 16: kern = k_contract_tc<16>; break;
    case 32: kern = k_contract_tc<32>; break;
    case 48: kern = k_contract_tc<48>; break;
    case 64: kern = k_contract_tc<64>; break;
    case 80: kern = k_contract_tc<80>; break;
    case 96: kern = k_contract_tc<96>; break;
    case 112: kern = k_contract_tc<112>; break;
    default: return cudaErrorInvalidValue;
  }
  static_assert(kTMaxKP == 112, "one instantiation per padded layer count");
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const long long units = (long long)Bc * tiles_w;
  const int grid = (int)std::min<long long>(units, (long long)std::max(n_sm, 1));
  return launch_dependent(kern, dim3(grid), dim3(kTThreads), smem, s, p, tm, Bc, tiles_w,
                          static_cast<const float*>(tiles));
}

}  // namespace tr
