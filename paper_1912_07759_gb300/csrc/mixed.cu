// mixed.cu -- mixed-precision path: cross-sections stored as FP16 (log10 sigma - c_m) and
// decoded on the fly by the opacity kernel (forward_fp32.cu, 10^x, then linear P/T
// interpolation of sigma as in Sec. 5), and the slant optical depth tau = DL . K (Sec. 4) on
// the 5th-generation tensor cores (tcgen05) as three BF16 products hi*hi + hi*lo + lo*hi with
// FP32 accumulation in tensor memory.
//
// k_contract_umma: one CTA = one atmosphere x 128 wavenumbers (the MMA's M):
//   * warp 0 allocates the TMEM accumulator; thread 0 bulk-copies the atmosphere's DL as BF16
//     hi / lo tiles (prepared once per atmosphere by k_dl_bf16) and its annulus weights;
//   * all 8 warps load the K tile (FP32, written by the opacity kernel), split it into BF16
//     hi + lo and store both in the tensor cores' K-major no-swizzle layout;
//   * thread 0 issues 3 x KP/16 MMAs D[128 x NP] (+)= A[128 x 16] B[NP x 16]^T (A = K tile,
//     B = DL: rays x layers, zero below the diagonal) and commits them to an mbarrier;
//   * each thread reads its wavenumber's row of tau from TMEM (16 columns at a time), forms
//     sum_j a_j (1 - e^-tau_j); two warp groups split the columns; FP64 final sum.
// All waits are bounded; TMEM is always released before the CTA exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <algorithm>
#include <cmath>
#include <vector>
#include "tma.h"
#include "tr_internal.h"
#include "umma.h"

namespace tr {
namespace {

constexpr int kMT = 128;          // wavenumbers per CTA = MMA M = TMEM lanes
constexpr int kMThreads = 256;

__host__ __device__ inline int pad16(int n) { return (n + 15) & ~15; }

// ---------------------------------------------------------------------------- FP16 tables
__global__ void k_to_log16(const float* __restrict__ sigma, __half* __restrict__ out,
                           size_t per_mol, int n_mol, TrLogOffsets off) {
  const size_t n = per_mol * n_mol;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / per_mol);
    const float s = sigma[i];
    // log10 0 = -inf decodes back to exactly 0 (row padding, empty cells)
    out[i] = __float2half_rn(s > 0.f ? log10f(s) - off.c[m] : -INFINITY);
  }
}

// DL as the MMA's B operand: rays j (rows, NP) x layers l (K, KP), BF16 hi and lo in the
// K-major core-matrix layout; zero for l < j and outside N.
__global__ void k_dl_bf16(ItemBuffers buf, int max_layers, int NP, int KP,
                          __nv_bfloat16* __restrict__ out) {
  const int b = blockIdx.x;
  const int N = buf.items[b].n_layers;
  const float* dlt = buf.dlt + (size_t)b * max_layers * buf.npad;
  __nv_bfloat16* hi = out + (size_t)b * 2 * NP * KP;
  __nv_bfloat16* lo = hi + (size_t)NP * KP;
  for (int i = threadIdx.x; i < NP * KP; i += blockDim.x) {
    const int j = i / KP, l = i - j * KP;
    const float v = (j < N && l < N && j <= l) ? dlt[(size_t)l * buf.npad + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 r = __float2bfloat16_rn(v - __bfloat162float(h));
    const uint32_t o = umma_kmajor_offset(j, l, KP) / 2;
    hi[o] = h;
    lo[o] = r;
  }
}

struct UmmaParams {
  FwdParams f;                     // item buffers, range, output, chunk offset
  const float* kbuf;               // [chunk items][max_layers][kcols] FP32 K
  long long kcols;
  const __nv_bfloat16* dl16;       // [B][2][NP][KP]
  int NP, KP, tmem_cols;
};

__global__ void __launch_bounds__(kMThreads, 1)
k_contract_umma(UmmaParams mp) {
  extern __shared__ __align__(128) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ float red[kMT];
  const FwdParams& p = mp.f;
  const int b = p.b_off + blockIdx.y;
  const ItemGeom ig = p.buf.items[b];
  const int N = ig.n_layers;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int w_first = wn_first(p.wn_begin) + blockIdx.x * kMT;
  const int NP = mp.NP, KP = mp.KP;
  if (N == 0) {
    for (int i = tid; i < kMT; i += kMThreads) {
      const int w = w_first + i;
      if (w >= p.wn_begin && w < p.wn_begin + p.wn_count)
        p.out[(long long)b * p.out_stride + (w - p.wn_begin)] = 0.0;
    }
    return;
  }
  // shared memory: A hi, A lo [128 x KP], B hi, B lo [NP x KP] (bf16), a_j [NP] (float)
  const size_t a_bytes = (size_t)kMT * KP * 2, b_bytes = (size_t)NP * KP * 2;
  uint8_t* A_hi = sm;
  uint8_t* A_lo = A_hi + a_bytes;
  uint8_t* B_hi = A_lo + a_bytes;                      // B lo follows B hi (one bulk copy)
  float* a_s = reinterpret_cast<float*>(B_hi + 2 * b_bytes);

  if (warp == 0) tmem_alloc(&tmem_base, (uint32_t)mp.tmem_cols);
  if (tid == 0) {
    mbar_init(&bar_load, 1); mbar_init(&bar_mma, 1);
    mbar_fence_init();
  }
  tcgen05_fence_before();
  __syncthreads();
  tcgen05_fence_after();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t na = (uint32_t)(sizeof(float) * p.buf.npad);
    mbar_arrive_expect_tx(&bar_load, (uint32_t)(2 * b_bytes) + na);
    bulk_g2s(B_hi, mp.dl16 + (size_t)b * 2 * NP * KP, (uint32_t)(2 * b_bytes), &bar_load);
    bulk_g2s(a_s, p.buf.aj + (size_t)b * p.buf.npad, na, &bar_load);
  }
  for (int j = p.buf.npad + tid; j < NP; j += kMThreads) a_s[j] = 0.f;

  // ---- A tile: K rows l (FP32 from the opacity kernel) -> BF16 hi + lo; padding layers
  //      zero.  A thread packs 8 consecutive layers of one wavenumber (one 16-byte row of a
  //      core matrix) and stores it whole: consecutive threads fill consecutive rows, so the
  //      stores are free of bank conflicts.
  const float* src = mp.kbuf + (size_t)blockIdx.y * p.max_layers * mp.kcols + (size_t)blockIdx.x * kMT;
  for (int item = tid; item < kMT * (KP / 8); item += kMThreads) {
    const int v = item & (kMT - 1), lg = item / kMT;
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float x[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int l = lg * 8 + 2 * q + h;
        x[h] = (l < N) ? __ldcs(src + (size_t)l * mp.kcols + v) : 0.f;
      }
      const __nv_bfloat162 hi2 = __floats2bfloat162_rn(x[0], x[1]);
      const float2 hf = __bfloat1622float2(hi2);
      const __nv_bfloat162 lo2 = __floats2bfloat162_rn(x[0] - hf.x, x[1] - hf.y);
      hw[q] = *reinterpret_cast<const uint32_t*>(&hi2);
      lw[q] = *reinterpret_cast<const uint32_t*>(&lo2);
    }
    const uint32_t o = umma_kmajor_offset(v, lg * 8, KP);
    *reinterpret_cast<uint4*>(A_hi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(A_lo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
  fence_proxy_async_smem();
  bool ok = __syncthreads_and(mbar_wait_bounded(&bar_load, 0, p.dev_err, TR_DEVERR_TIMEOUT));
  if (ok && tid == 0) {
    // tau^T[128 x NP] = K^T[128 x KP] . DL^T[KP x NP] as hi*hi + hi*lo + lo*hi
    tcgen05_fence_after();
    const uint32_t idesc = umma_idesc_bf16_f32(kMT, NP);
    const uint32_t a_sbo = (uint32_t)(KP / 8) * 128, b_sbo = a_sbo;
    const uint32_t ah = smem_addr(A_hi), al = smem_addr(A_lo);
    const uint32_t bh = smem_addr(B_hi), bl = bh + (uint32_t)b_bytes;
    uint32_t acc = 0;
    for (int ks = 0; ks < KP / 16; ++ks) {
      const uint32_t koff = (uint32_t)ks * 256;          // two core matrices along K
      umma_bf16(tmem, umma_smem_desc(ah + koff, 128, a_sbo), umma_smem_desc(bh + koff, 128, b_sbo), idesc, acc);
      acc = 1;
      umma_bf16(tmem, umma_smem_desc(ah + koff, 128, a_sbo), umma_smem_desc(bl + koff, 128, b_sbo), idesc, 1);
      umma_bf16(tmem, umma_smem_desc(al + koff, 128, a_sbo), umma_smem_desc(bh + koff, 128, b_sbo), idesc, 1);
    }
    umma_commit(&bar_mma);
  }
  if (ok) ok = __syncthreads_and(mbar_wait_bounded(&bar_mma, 0, p.dev_err, TR_DEVERR_TIMEOUT));
  if (ok) {
    // ---- epilogue: thread (warp % 4, lane) owns wavenumber row 32 (warp % 4) + lane;
    //      warps 0-3 take the first half of the ray columns, warps 4-7 the rest
    tcgen05_fence_after();
    const int row = 32 * (warp & 3) + lane;
    const int half_cols = ((NP / 16 + 1) / 2) * 16;
    const int c_begin = warp < 4 ? 0 : half_cols, c_end = warp < 4 ? half_cols : NP;
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    float part = 0.f;
    for (int c0 = c_begin; c0 < c_end; c0 += 16) {
      float tau[16];
      tmem_ld16(taddr + (uint32_t)c0, tau);
#pragma unroll
      for (int i = 0; i < 16; ++i) part = fmaf(a_s[c0 + i], 1.f - __expf(-tau[i]), part);
    }
    if (warp >= 4) red[row] = part;
    __syncthreads();
    if (warp < 4) {
      const int w = w_first + row;
      if (w >= p.wn_begin && w < p.wn_begin + p.wn_count)
        p.out[(long long)b * p.out_stride + (w - p.wn_begin)] =
            ig.rp2_rs2 + ((double)part + (double)red[row]);
    }
  } else {
    // a wait ran out: let in-flight copies / MMAs land (bounded) before releasing memory
    mbar_wait_bounded(&bar_load, 0, nullptr, 0);
    mbar_wait_bounded(&bar_mma, 0, nullptr, 0);
  }
  tcgen05_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)mp.tmem_cols);
}

// ---------------------------------------------------------------------------- persistent form
//
// k_contract_umma_p: one persistent CTA per SM walks a contiguous range of (item, 128-wn)
// units.  Roles (warp-specialized, every hand-over through an mbarrier):
//   * warp kPProd: TMA loads of the unit's FP32 K tile [KP layers][128 wn] (2-D boxes of 8
//     rows) into one of two stages, plus the item's BF16 hi/lo path-length tiles (bulk copy)
//     when the item changes (after every earlier unit's MMAs are done with them);
//   * warps kPConv0 .. +7: split the stage's K into BF16 hi + lo in place, in the tensor cores'
//     K-major core-matrix layout (all reads of the stage, a barrier, then the writes);
//   * warp kPMma (one thread): for K slices ks = KP/16-1 down to 0 issues hi*hi, hi*lo and
//     lo*hi MMAs D[128 x N_ks] (+)= A[128 x 16] B[N_ks x 16]^T with N_ks = 16 (ks + 1): the
//     rays j > l of slice ks have DL = 0, so each slice touches only the rays it reaches; the
//     first (widest) slice initialises all columns.  Accumulators alternate between two TMEM
//     buffers; a commit frees the stage and one hands the accumulator to the epilogue;
//   * warps 0 .. 3 (TMEM lanes 0 .. 127 = the unit's wavenumbers): read tau from TMEM,
//     form sum_j a_j (1 - e^-tau_j) and write (R_p/R_s)^2 + the sum in FP64.
// All waits are bounded; on a timeout every role stops, in-flight copies and MMAs are waited
// for (bounded) and the TMEM is released before the CTA exits.
constexpr int kPEpi = 4;                   // epilogue warps 0..3
constexpr int kPConv0 = kPEpi;             // converter warps 4..11
constexpr int kPConvW = 8;
constexpr int kPProd = kPConv0 + kPConvW;  // 12
constexpr int kPMma = kPProd + 1;          // 13
constexpr int kPThreads = 32 * (kPMma + 1);
constexpr int kPMaxKP = 128;               // layers (padded to 16) the persistent form takes

struct UmmaPLayout {
  uint32_t stage, dl, aj, total;
  __host__ __device__ UmmaPLayout(int KP, int NP) {
    stage = (uint32_t)KP * kMT * 4;                       // FP32 K tile = BF16 hi + lo tile
    dl = 2 * stage;
    aj = dl + 2u * (uint32_t)NP * KP * 2;
    total = aj + 2u * kMT * 4 + 1024u;
  }
};

// Barrier over `threads` threads (named barrier `id`) that also returns whether any of them
// passed pred = true: the warps of one role take the same stop decision.
__device__ __forceinline__ bool named_sync_or(int id, int threads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r) : "r"((uint32_t)pred), "r"(id), "r"(threads) : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kPThreads, 1)
k_contract_umma_p(UmmaParams mp, const __grid_constant__ CUtensorMap tm_k, int Bc, int n_tiles) {
  extern __shared__ __align__(1024) uint8_t psm_raw[];
  __shared__ __align__(8) uint64_t sfull[2], sempty[2], aready[2], accfull[2], accempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const FwdParams& p = mp.f;
  const int KP = mp.KP, NP = mp.NP;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(psm_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const UmmaPLayout lay(KP, NP);
  uint8_t* B_hi = base + lay.dl;
  float* ep_aj = reinterpret_cast<float*>(base + lay.aj);      // [2][128], epilogue's copy
  const long long units = (long long)Bc * n_tiles;
  const long long per = (units + gridDim.x - 1) / gridDim.x;
  const long long u_begin = (long long)blockIdx.x * per;
  const long long u_end = u_begin + per < units ? u_begin + per : units;
  const int n_units = u_end > u_begin ? (int)(u_end - u_begin) : 0;
  const int wbase = wn_first(p.wn_begin);
  const uint32_t dl_bytes = 2u * (uint32_t)NP * KP * 2;

  if (warp == 0) tmem_alloc(&tmem_base, (uint32_t)(2 * mp.tmem_cols));
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sfull[i], 1); mbar_init(&sempty[i], 1); mbar_init(&aready[i], kPConvW);
      mbar_init(&accfull[i], 1); mbar_init(&accempty[i], kPEpi);
    }
    abort_flag = 0;
    mbar_fence_init();
  }
  tcgen05_fence_before();
  __syncthreads();
  tcgen05_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == kPProd) {
    // ---------------- producer
    if (lane == 0) {
      int dl_item = -1, k = 0;
      for (; k < n_units; ++k) {
        const long long u = u_begin + k;
        const int bc = (int)(u / n_tiles), tile = (int)(u % n_tiles);
        const int b = p.b_off + bc;
        const int s = k & 1, q = k >> 1;
        bool ok = q == 0 || mbar_wait_bounded(&sempty[s], (q - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
        const bool new_item = b != dl_item;
        if (ok && new_item && k > 0)            // unit k-1's MMAs are done with the old tiles
          ok = mbar_wait_bounded(&sempty[(k - 1) & 1], ((k - 1) >> 1) & 1, p.dev_err,
                                 TR_DEVERR_TIMEOUT);
        if (!ok || *(volatile int*)&abort_flag) { atomicExch(&abort_flag, 1); break; }
        uint8_t* st = base + s * lay.stage;
        mbar_arrive_expect_tx(&sfull[s], lay.stage + (new_item ? dl_bytes : 0u));
        for (int i = 0; i < KP / 8; ++i)
          tma_load_2d(st + (size_t)i * 8 * kMT * 4, &tm_k, tile * kMT,
                      bc * p.max_layers + i * 8, &sfull[s]);
        if (new_item) {
          bulk_g2s(B_hi, mp.dl16 + (size_t)b * 2 * NP * KP, dl_bytes, &sfull[s]);
          dl_item = b;
        }
      }
      for (int i = 0; i < 2 && i < k; ++i) {      // every copy issued has landed
        const int kl = k - 1 - i;
        mbar_wait_bounded(&sfull[kl & 1], (kl >> 1) & 1, nullptr, 0);
      }
    }
  } else if (warp >= kPConv0 && warp < kPConv0 + kPConvW) {
    // ---------------- converters: FP32 K -> BF16 hi + lo core matrices, in place
    const int ct = tid - 32 * kPConv0;              // 0 .. 255
    const int v = ct & (kMT - 1), half = ct >> 7;   // wavenumber row, layer-group parity
    const int ng = KP / 8;
    for (int k = 0; k < n_units; ++k) {
      const long long u = u_begin + k;
      const int b = p.b_off + (int)(u / n_tiles);
      const int N = __ldg(&p.buf.items[b].n_layers);
      const int s = k & 1;
      const bool ok = mbar_wait_bounded(&sfull[s], (k >> 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT) &&
                      !*(volatile int*)&abort_flag;
      uint8_t* st = base + s * lay.stage;
      const float* kf = reinterpret_cast<const float*>(st);
      float x[kPMaxKP / 2];
#pragma unroll
      for (int gi = 0; gi < kPMaxKP / 16; ++gi) {
        const int g = half + 2 * gi;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int l = 8 * g + i;
          x[8 * gi + i] = (g < ng && l < N) ? kf[l * kMT + v] : 0.f;
        }
      }
      // every read of the stage is done; all converter warps stop together on a failed wait
      if (named_sync_or(1, 32 * kPConvW, !ok)) { if (lane == 0) atomicExch(&abort_flag, 1); break; }
#pragma unroll
      for (int gi = 0; gi < kPMaxKP / 16; ++gi) {
        const int g = half + 2 * gi;
        if (g < ng) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float a0 = x[8 * gi + 2 * q], a1 = x[8 * gi + 2 * q + 1];
            const __nv_bfloat162 hi2 = __floats2bfloat162_rn(a0, a1);
            const float2 hf = __bfloat1622float2(hi2);
            const __nv_bfloat162 lo2 = __floats2bfloat162_rn(a0 - hf.x, a1 - hf.y);
            hw[q] = *reinterpret_cast<const uint32_t*>(&hi2);
            lw[q] = *reinterpret_cast<const uint32_t*>(&lo2);
          }
          const uint32_t o = umma_kmajor_offset(v, 8 * g, KP);
          *reinterpret_cast<uint4*>(st + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(st + (size_t)kMT * KP * 2 + o) =
              make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      }
      fence_proxy_async_smem();                     // visible to the tensor cores
      __syncwarp();
      if (lane == 0) mbar_arrive(&aready[s]);
    }
  } else if (warp == kPMma) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t sbo = (uint32_t)(KP / 8) * 128;
      const uint32_t bh = smem_addr(B_hi), bl = bh + (uint32_t)NP * KP * 2;
      int k = 0;
      for (; k < n_units; ++k) {
        const int s = k & 1, a = k & 1, q = k >> 1;
        bool ok = mbar_wait_bounded(&aready[s], q & 1, p.dev_err, TR_DEVERR_TIMEOUT);
        if (ok && q > 0)
          ok = mbar_wait_bounded(&accempty[a], (q - 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT);
        if (!ok || *(volatile int*)&abort_flag) { atomicExch(&abort_flag, 1); break; }
        tcgen05_fence_after();
        const uint32_t ah = smem_addr(base + s * lay.stage), al = ah + (uint32_t)kMT * KP * 2;
        const uint32_t d = tmem + (uint32_t)(a * mp.tmem_cols);
        bool first = true;
        for (int ks = KP / 16 - 1; ks >= 0; --ks) {
          const int n = min(NP, 16 * (ks + 1));
          const uint32_t idesc = umma_idesc_bf16_f32(kMT, n);
          const uint32_t koff = (uint32_t)ks * 256;
          umma_bf16(d, umma_smem_desc(ah + koff, 128, sbo), umma_smem_desc(bh + koff, 128, sbo),
                    idesc, first ? 0u : 1u);
          umma_bf16(d, umma_smem_desc(ah + koff, 128, sbo), umma_smem_desc(bl + koff, 128, sbo),
                    idesc, 1u);
          umma_bf16(d, umma_smem_desc(al + koff, 128, sbo), umma_smem_desc(bh + koff, 128, sbo),
                    idesc, 1u);
          first = false;
        }
        umma_commit(&sempty[s]);                    // the stage (A tiles, path lengths) is free
        umma_commit(&accfull[a]);                   // the accumulator is ready
      }
      // the MMAs issued are complete before the CTA may release the TMEM
      if (k > 0) mbar_wait_bounded(&accfull[(k - 1) & 1], ((k - 1) >> 1) & 1, nullptr, 0);
    }
  } else if (warp < kPEpi) {
    // ---------------- epilogue: thread = TMEM lane = wavenumber row
    const int row = 32 * warp + lane;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    for (int k = 0; k < n_units; ++k) {
      const long long u = u_begin + k;
      const int bc = (int)(u / n_tiles), tile = (int)(u % n_tiles);
      const int b = p.b_off + bc;
      const ItemGeom ig = p.buf.items[b];
      const int a = k & 1;
      float* aj = ep_aj + a * kMT;
      if (row < NP) aj[row] = row < p.buf.npad ? __ldg(p.buf.aj + (size_t)b * p.buf.npad + row) : 0.f;
      const bool ok = mbar_wait_bounded(&accfull[a], (k >> 1) & 1, p.dev_err, TR_DEVERR_TIMEOUT) &&
                      !*(volatile int*)&abort_flag;
      // aj of this unit in place; all epilogue warps stop together on a failed wait
      if (named_sync_or(2, 32 * kPEpi, !ok)) { if (lane == 0) atomicExch(&abort_flag, 1); break; }
      tcgen05_fence_after();
      const uint32_t taddr = tmem + lane_base + (uint32_t)(a * mp.tmem_cols);
      float part = 0.f;
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float tau[16];
        tmem_ld16(taddr + (uint32_t)c0, tau);
#pragma unroll
        for (int i = 0; i < 16; ++i) part = fmaf(aj[c0 + i], 1.f - __expf(-tau[i]), part);
      }
      tcgen05_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[a]);     // this warp's TMEM lanes are read
      const int w = wbase + tile * kMT + row;
      if (w >= p.wn_begin && w < p.wn_begin + p.wn_count)
        p.out[(long long)b * p.out_stride + (w - p.wn_begin)] =
            ig.n_layers > 0 ? ig.rp2_rs2 + (double)part : 0.0;
    }
  }
  tcgen05_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)(2 * mp.tmem_cols));
}

int tmem_cols_for(int NP) {
  int c = 32;
  while (c < NP) c <<= 1;
  return c;
}

}  // namespace

size_t mixed_dl_bytes(int B, int max_layers) {
  const int NP = pad16(max_layers), KP = pad16(max_layers);
  return sizeof(__nv_bfloat16) * 2 * (size_t)B * NP * KP;
}

int build_fp16_log_tables(tr_ctx* ctx, tr_tables* t) {
  if (t->n_mol == 0) return TR_OK;
  if (!t->d_sigma) return set_error(ctx, TR_ERR_ARG, "FP16 tables need the FP32 upload");
  const size_t per_mol = (size_t)t->n_p * t->n_t * t->wn_pad;
  __half* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(__half) * per_mol * t->n_mol);
  if (e != cudaSuccess) return set_error(ctx, TR_ERR_OOM, "alloc FP16 tables");
  TrLogOffsets off{};
  for (int m = 0; m < t->n_mol; ++m) off.c[m] = t->logsig_offset[m];
  k_to_log16<<<1024, 256>>>(t->d_sigma, out, per_mol, t->n_mol, off);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { cudaFree(out); return set_error(ctx, TR_ERR_CUDA, cudaGetErrorString(e)); }
  t->d_logsig16 = reinterpret_cast<uint16_t*>(out);
  t->device_bytes += sizeof(__half) * per_mol * t->n_mol;
  return TR_OK;
}

cudaError_t launch_dl_bf16(const ItemBuffers& buf, int B, int max_layers, void* dl16,
                           cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_dl_bf16<<<B, 256, 0, s>>>(buf, max_layers, pad16(max_layers), pad16(max_layers),
                             static_cast<__nv_bfloat16*>(dl16));
  return cudaGetLastError();
}

cudaError_t launch_contract_umma(const FwdParams& p, int Bc, const float* kbuf, const void* dl16,
                                 cudaStream_t s) {
  if (Bc <= 0 || p.wn_count <= 0) return cudaSuccess;
  const int NP = pad16(p.max_layers), KP = pad16(p.max_layers);
  if (NP > 256) return cudaErrorInvalidValue;
  UmmaParams mp{};
  mp.f = p;
  const int w_first = wn_first(p.wn_begin);
  const int tiles = (p.wn_begin + p.wn_count - w_first + kMT - 1) / kMT;
  mp.kbuf = kbuf;
  mp.kcols = (long long)tiles * kMT;
  mp.dl16 = static_cast<const __nv_bfloat16*>(dl16);
  mp.NP = NP; mp.KP = KP; mp.tmem_cols = tmem_cols_for(NP);
  if (KP <= kPMaxKP && UmmaPLayout(KP, NP).total <= 227u * 1024u) {
    // persistent warp-specialized form: one CTA per SM over a contiguous range of units
    CUtensorMap tm{};
    if (!encode_2d_f32(&tm, kbuf, (unsigned long long)mp.kcols,
                       (unsigned long long)Bc * p.max_layers, (unsigned long long)mp.kcols * 4,
                       kMT, 8))
      return cudaErrorInvalidValue;
    const uint32_t smem = UmmaPLayout(KP, NP).total;
    cudaError_t e = cudaFuncSetAttribute(k_contract_umma_p,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long units = (long long)Bc * tiles;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<long long>(units, (long long)std::max(n_sm, 1));
    k_contract_umma_p<<<grid, kPThreads, smem, s>>>(mp, tm, Bc, tiles);
    return cudaGetLastError();
  }
  const size_t smem = 2 * (size_t)kMT * KP * 2 + 2 * (size_t)NP * KP * 2 + sizeof(float) * NP;
  cudaError_t e = cudaFuncSetAttribute(k_contract_umma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_umma<<<dim3(tiles, Bc), kMThreads, smem, s>>>(mp);
  return cudaGetLastError();
}

}  // namespace tr
