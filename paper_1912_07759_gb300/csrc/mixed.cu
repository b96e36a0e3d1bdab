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
#include <cmath>
#include <vector>
#include "tma.h"
#include "tr_internal.h"
#include "umma.h"

namespace tr {
namespace {

constexpr int kMT = 128;          // wavenumbers per CTA = MMA M = TMEM lanes
constexpr int kMThreads = 256;
constexpr int kMWarps = kMThreads / 32;

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
  const size_t smem = 2 * (size_t)kMT * KP * 2 + 2 * (size_t)NP * KP * 2 + sizeof(float) * NP;
  cudaError_t e = cudaFuncSetAttribute(k_contract_umma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_contract_umma<<<dim3(tiles, Bc), kMThreads, smem, s>>>(mp);
  return cudaGetLastError();
}

}  // namespace tr
