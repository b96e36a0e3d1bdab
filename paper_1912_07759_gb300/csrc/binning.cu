// binning.cu -- FluxBinner (Sec. 4.5): binned_j = sum_i w_ij D_i / sum_i w_ij, one warp per
// (item, bin), FP64 accumulation and a fixed-order butterfly over the lanes (deterministic);
// binned uncertainties sigma_j = sqrt(sum_i w_ij^2 sigma_i^2) / sum_i w_ij alike; and the SNR
// instrument model of Sec. 7 (noise = largest binned value / SNR / sqrt(observations)).
#include "tma.h"
#include "tr_internal.h"

namespace tr {
namespace {

// A wait that can never complete: the barrier expects two arrivals and gets one.  The bounded
// wait gives up after `polls` polls and records TR_DEVERR_TIMEOUT (no copy is in flight).
__global__ void k_wait_selftest(int* err, long long polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    mbar_fence_init();
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(&bar)) : "memory");
    for (long long i = 0; i < polls; ++i)
      if (mbar_try_wait(&bar, 0)) return;
    atomicOr(err, TR_DEVERR_TIMEOUT);
  }
}

constexpr int kBinThreads = 128;
constexpr int kBinWarps = 8;                 // bins per CTA of the binning kernels (a warp each)

// Sum over the entries [e0, e1) of one bin of f(w_e, native value) by WPB warps (part `part`
// of them): lanes take consecutive entries (a bin's native indices are consecutive, from
// bd.lo[j], so the loads coalesce), four per lane and pass with all loads issued first, two
// FP64 chains per lane, then a fixed butterfly over the lanes.  f(0, 0) must be 0.
template <int WPB, class F>
__device__ __forceinline__ double warp_bin_sum(const BinsDev& bd, int j, const double* d,
                                               int base, int lane, int part, F f) {
  const int e0 = bd.row_ptr[j], e1 = bd.row_ptr[j + 1];
  const int i0 = bd.lo[j] - base;
  double s0 = 0.0, s1 = 0.0;
  for (int eb = e0 + 128 * part; eb < e1; eb += 128 * WPB) {
    double wv[4], dv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = eb + lane + 32 * k;
      const bool ok = e < e1;
      wv[k] = ok ? __ldg(bd.w + e) : 0.0;
      dv[k] = ok ? __ldg(d + i0 + (e - e0)) : 0.0;
    }
    s0 += f(wv[0], dv[0]);
    s1 += f(wv[1], dv[1]);
    s0 += f(wv[2], dv[2]);
    s1 += f(wv[3], dv[3]);
  }
  double s = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// WPB warps per (item, bin), 8 / WPB bins of one item per CTA; the WPB warp sums of a bin are
// added in warp order (deterministic).  MODE 0: binned_j = sum_i w_ij D_i / sum_i w_ij
// (eq. F_j of Sec. 4.5); MODE 1: sqrt(sum_i (w_ij sigma_i)^2) / sum_i w_ij (eq. sigma_j).
template <int WPB, int MODE>
__global__ void __launch_bounds__(32 * kBinWarps)
k_bin_t(BinsDev bd, int B, const double* __restrict__ vals, long long stride, int base,
        double* __restrict__ out) {
  __shared__ double part_s[kBinWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * (kBinWarps / WPB) + warp / WPB, b = blockIdx.y;
  double s = 0.0;
  if (j < bd.n_bin) {
    const double* d = vals + (long long)b * stride;
    if (MODE == 0)
      s = warp_bin_sum<WPB>(bd, j, d, base, lane, warp % WPB,
                            [](double w, double v) { return w * v; });
    else
      s = warp_bin_sum<WPB>(bd, j, d, base, lane, warp % WPB, [](double w, double v) {
        const double ws = w * v;
        return ws * ws;
      });
  }
  if (WPB > 1) {
    if (lane == 0) part_s[warp] = s;
    __syncthreads();
    if (warp % WPB != 0) return;
    for (int k = 1; k < WPB; ++k) s += part_s[warp + k];
  }
  if (lane == 0 && j < bd.n_bin)
    out[(long long)b * bd.n_bin + j] = (MODE == 0 ? s : sqrt(s)) * bd.inv_wsum[j];
}

// Warps per bin: several while the batch is too small to fill the GPU with one per bin.
template <int MODE>
cudaError_t launch_bin_mode(const BinsDev& bd, int B, const double* vals, long long stride,
                            int base, double* out, cudaStream_t s) {
  if ((long long)B * bd.n_bin < 2048) {
    k_bin_t<4, MODE><<<dim3((bd.n_bin + 1) / 2, B), 32 * kBinWarps, 0, s>>>(bd, B, vals, stride,
                                                                            base, out);
  } else {
    k_bin_t<1, MODE><<<dim3((bd.n_bin + kBinWarps - 1) / kBinWarps, B), 32 * kBinWarps, 0, s>>>(
        bd, B, vals, stride, base, out);
  }
  return cudaGetLastError();
}

// One CTA per spectrum: S = max_j binned_j (fixed-order tree), N' = S / snr / sqrt(n_obs),
// obs_j = binned_j + N' z_j, sigma_j = N'.
__global__ void __launch_bounds__(kBinThreads)
k_snr(int n_bin, const double* __restrict__ binned, double inv_snr_rootn,
      const double* __restrict__ z, double* __restrict__ obs, double* __restrict__ sigma) {
  __shared__ double red[kBinThreads];
  const int b = blockIdx.x;
  const double* x = binned + (long long)b * n_bin;
  double m = -INFINITY;
  for (int j = threadIdx.x; j < n_bin; j += kBinThreads) m = fmax(m, x[j]);
  red[threadIdx.x] = m;
  __syncthreads();
#pragma unroll
  for (int o = kBinThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const double noise = red[0] * inv_snr_rootn;
  for (int j = threadIdx.x; j < n_bin; j += kBinThreads) {
    const long long k = (long long)b * n_bin + j;
    obs[k] = fma(noise, z[k], x[j]);
    sigma[k] = noise;
  }
}

}  // namespace

cudaError_t launch_bin_sigma(const BinsDev& bd, int B, const double* sigma, long long stride,
                             int base, double* out, cudaStream_t s) {
  if (B <= 0 || bd.n_bin <= 0) return cudaSuccess;
  return launch_bin_mode<1>(bd, B, sigma, stride, base, out, s);
}

cudaError_t launch_snr(int B, int n_bin, const double* binned, double snr, int n_obs,
                       const double* z, double* obs, double* sigma, cudaStream_t s) {
  if (B <= 0 || n_bin <= 0) return cudaSuccess;
  k_snr<<<B, kBinThreads, 0, s>>>(n_bin, binned, 1.0 / (snr * sqrt((double)n_obs)), z, obs,
                                  sigma);
  return cudaGetLastError();
}

cudaError_t launch_bin(const BinsDev& bd, int B, const double* depth, long long depth_stride,
                       int depth_base, double* binned, cudaStream_t s) {
  if (B <= 0 || bd.n_bin <= 0) return cudaSuccess;
  return launch_bin_mode<0>(bd, B, depth, depth_stride, depth_base, binned, s);
}

cudaError_t launch_wait_selftest(int* err, long long polls, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err, polls);
  return cudaGetLastError();
}

}  // namespace tr
