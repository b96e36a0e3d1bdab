// binning.cu -- FluxBinner (Sec. 4.5): binned_j = sum_i w_ij D_i / sum_i w_ij, one CTA per
// (item, bin), FP64 accumulation and a fixed-order tree reduction (deterministic); binned
// uncertainties sigma_j = sqrt(sum_i w_ij^2 sigma_i^2) / sum_i w_ij alike; and the SNR
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

// One CTA per (item, bin): threads stride over the bin's native entries, FP64 partial sums,
// then a fixed-shape tree reduction in shared memory (deterministic).
__global__ void __launch_bounds__(kBinThreads)
k_bin(BinsDev bd, int B, const double* __restrict__ depth, long long stride, int base,
      double* __restrict__ binned) {
  __shared__ double red[kBinThreads];
  const int j = blockIdx.x, b = blockIdx.y;
  const double* d = depth + (long long)b * stride;
  double s = 0.0;
  for (int e = bd.row_ptr[j] + threadIdx.x; e < bd.row_ptr[j + 1]; e += kBinThreads)
    s += bd.w[e] * d[bd.col[e] - base];
  red[threadIdx.x] = s;
  __syncthreads();
#pragma unroll
  for (int o = kBinThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) binned[(long long)b * bd.n_bin + j] = red[0] * bd.inv_wsum[j];
}

// One CTA per (item, bin): sqrt(sum_i (w_ij sigma_i)^2) / sum_i w_ij, the same reduction.
__global__ void __launch_bounds__(kBinThreads)
k_bin_sigma(BinsDev bd, int B, const double* __restrict__ sigma, long long stride, int base,
            double* __restrict__ out) {
  __shared__ double red[kBinThreads];
  const int j = blockIdx.x, b = blockIdx.y;
  const double* d = sigma + (long long)b * stride;
  double s = 0.0;
  for (int e = bd.row_ptr[j] + threadIdx.x; e < bd.row_ptr[j + 1]; e += kBinThreads) {
    const double ws = bd.w[e] * d[bd.col[e] - base];
    s += ws * ws;
  }
  red[threadIdx.x] = s;
  __syncthreads();
#pragma unroll
  for (int o = kBinThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(long long)b * bd.n_bin + j] = sqrt(red[0]) * bd.inv_wsum[j];
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
  k_bin_sigma<<<dim3(bd.n_bin, B), kBinThreads, 0, s>>>(bd, B, sigma, stride, base, out);
  return cudaGetLastError();
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
  k_bin<<<dim3(bd.n_bin, B), kBinThreads, 0, s>>>(bd, B, depth, depth_stride, depth_base, binned);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* err, long long polls, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err, polls);
  return cudaGetLastError();
}

}  // namespace tr
