// binning.cu -- FluxBinner (Sec. 4.5): binned_j = sum_i w_ij D_i / sum_i w_ij, one warp per
// (item, bin), FP64 accumulation and a fixed-order warp reduction (deterministic).
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

__global__ void k_bin(BinsDev bd, int B, const double* __restrict__ depth, long long stride,
                      int base, double* __restrict__ binned) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= B * bd.n_bin) return;
  const int b = gw / bd.n_bin, j = gw - b * bd.n_bin;
  const double* d = depth + (long long)b * stride;
  double s = 0.0;
  for (int e = bd.row_ptr[j] + lane; e < bd.row_ptr[j + 1]; e += 32)
    s += bd.w[e] * d[bd.col[e] - base];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) binned[(long long)b * bd.n_bin + j] = s * bd.inv_wsum[j];
}

}  // namespace

cudaError_t launch_bin(const BinsDev& bd, int B, const double* depth, long long depth_stride,
                       int depth_base, double* binned, cudaStream_t s) {
  const long long warps = (long long)B * bd.n_bin;
  if (warps <= 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = (warps * 32 + threads - 1) / threads;
  k_bin<<<(unsigned)blocks, threads, 0, s>>>(bd, B, depth, depth_stride, depth_base, binned);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* err, long long polls, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err, polls);
  return cudaGetLastError();
}

}  // namespace tr
