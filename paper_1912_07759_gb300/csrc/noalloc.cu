// noalloc.cu -- tr_forward_transit_batch_noalloc: the batched FP32 forward model for callers
// that cannot allocate device memory.  Its scratch (per-item layer descriptors, path lengths,
// annulus weights and the binned-region depths) comes from one file-scope device array
// instead of cudaMalloc or a caller workspace.
#include <mutex>
#include "tr_internal.h"

namespace {

// The scratch array.  In host code `g_noalloc_scratch` is only a host-side stand-in for the
// symbol, not a device address: a kernel handed it would fault (or, where the GPU can reach
// host memory, silently touch the wrong memory).  Host code must use the address returned
// by cudaGetSymbolAddress for the current device, cached below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// One-time per-device set-up (the device must be current): device address of the array.
// The cached address assumes the device's primary context lives as long as the library: after
// a cudaDeviceReset the module is loaded again at another address (and every handle of the
// library is invalid too), so a process that resets a device must not call this entry point
// on it again.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[device] = p;
  }
  *out = g_dev_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" int tr_forward_transit_batch_noalloc(tr_ctx* ctx, const tr_tables* t,
                                                const tr_batch_desc* d, int B,
                                                const double* d_theta, const int32_t* d_nlayers,
                                                const tr_bins* bins, double* d_binned,
                                                int32_t* d_status, void* stream) {
  using namespace tr;
  if (!ctx || !t || !bins || !d_theta || !d_binned || B < 0)
    return set_error(ctx, TR_ERR_ARG, "null argument");
  // the geometry and binning kernels take B as a grid dimension
  if (B > TR_MAX_BATCH) return set_error(ctx, TR_ERR_ARG, "batch larger than TR_MAX_BATCH");
  if (B == 0) return TR_OK;
  int rc = validate_batch_desc(ctx, t, d);
  if (rc != TR_OK) return rc;
  if (!t->d_sigma && t->n_mol > 0)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "tables were loaded without FP32 storage");
  if (t->interp_mode != TR_INTERP_LINEAR)
    return set_error(ctx, TR_ERR_UNSUPPORTED,
                     "the allocation-free entry point implements the linear temperature scheme");
  if (d->gas_mode != TR_GAS_CONSTANT)
    return set_error(ctx, TR_ERR_UNSUPPORTED,
                     "the allocation-free entry point implements constant mixing ratios");
  const int n_in = bins->dev.i1 - bins->dev.i0;
  const size_t need = forward_workspace_bytes(B, d->max_layers, n_in);
  if (need > (size_t)TR_NOALLOC_SCRATCH_BYTES)
    return set_error(ctx, TR_ERR_ARG,
                     "batch needs " + std::to_string(need) + " bytes of scratch but the built-in "
                     "scratch holds " + std::to_string((size_t)TR_NOALLOC_SCRATCH_BYTES) +
                     " bytes: split the batch or use tr_forward_transit_batch");
  // the fused kernel stages each item's K tiles and path lengths in shared memory; refuse a
  // shape it cannot stage before anything is launched
  if (!fused_forward_fits(t->n_mol, t->n_cia, d->max_layers, B))
    return set_error(ctx, TR_ERR_UNSUPPORTED,
                     "the fused FP32 kernel cannot stage this many layers and species in shared "
                     "memory: use tr_forward_transit_batch");
  cudaError_t e = cudaSetDevice(ctx->device);
  void* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(ctx->device, &base);
  if (e != cudaSuccess)
    return set_error(ctx, TR_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* depth = nullptr;
  const ItemBuffers buf = carve_forward_workspace(base, B, d->max_layers, n_in, &depth);
  const int n_theta = batch_n_theta(t, d);
  e = launch_geometry(batch_geom_params(t, d), B, d_theta, n_theta, d_nlayers, d_status, buf, s);
  if (e == cudaSuccess)
    e = launch_forward_fused(forward_fp32_params(t, d->max_layers, buf, bins->dev.i0, n_in,
                                                 depth, n_in, ctx->dev_err),
                             &t->tm_sig32_f, &t->tm_cia_f, B, 0, nullptr, s);
  if (e == cudaSuccess) e = launch_bin(bins->dev, B, depth, n_in, bins->dev.i0, d_binned, s);
  if (e != cudaSuccess)
    return set_error(ctx, TR_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return TR_OK;
}
