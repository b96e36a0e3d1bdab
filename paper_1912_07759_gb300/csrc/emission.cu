// emission.cu -- the emission (eclipse) forward model of Sec. 4 on the GPU: the planet's
// intensity at the top of a plane-parallel atmosphere from the layers' Planck sources,
// integrated over the viewing angle by Gauss-Legendre quadrature, as a flux ratio to the star.
//
// The opacity K[layer, wn] is the transmission model's (the same two-stage opacity kernel
// writes it to the K buffer).  Readings of the paper's garbled intensity equation (it
// integrates in mu twice and drops the 1/mu of the slant path):
//   E1 layer l has vertical optical depth dtau_l = K_l (z_{l+1} - z_l);
//   E2 the source is B(T_l) throughout layer l, so its part of the formal solution is
//      B(T_l) (e^{-tau_top/mu} - e^{-tau_bot/mu});
//   E3 the surface emits B(T_s) with T_s the temperature profile at p_max;
//   E4 the star's intensity goes through the same quadrature, B(T_star) sum_k x_k w_k.
// The kernel walks the layers from the bottom up with the equivalent recursion
//   I <- B_l + (I - B_l) e^{-dtau_l / mu},  starting from I = B(T_s),
// whose value at the top is exactly the sum above (expand it layer by layer).  Per wavenumber
// the Planck functions of planet and star share the factor 2 h c^2 nu^3, which cancels in the
// ratio, so only b(T) = 1 / (e^{c_2 nu / T} - 1) is evaluated:
//   F_p / F_s = sum_k x_k w_k I(x_k) / (b(T_star) sum_k x_k w_k) * (R_p / R_s)^2.
#include <cmath>
#include <string>
#include <vector>
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kEmThreads = 256;
constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr int kEmMaxMu = 16;
// second radiation constant h c / k_B in cm K (wavenumbers are in 1/cm)
constexpr double kC2cmK = 6.62607015e-34 * 299792458.0 / 1.380649e-23 * 100.0;

struct EmParams {
  ItemBuffers buf;
  int max_layers;
  const float* kbuf;            // K of the chunk: kbuf[(c * max_layers + l) * kcols + x]
  long long kcols;
  const double* wn;             // [n_wn] native wavenumbers (1/cm)
  int wn_begin, wn_count, b_off;
  int n_mu;
  float mu_coef[kEmMaxMu];      // -log2(e) / x_k
  float xw[kEmMaxMu];           // x_k w_k / sum_j x_j w_j
  float c2_tstar;               // c_2 / T_star (cm)
  double* out;                  // item b's value at wavenumber wn_begin + i: out[b * stride + i]
  long long out_stride;
};

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// b(T) = 1 / (e^{c_2 nu / T} - 1) from x = c_2 nu / T.  For x < 1/2, where e^x - 1 would
// cancel, its Taylor series x (1 + x/2! + x^2/3! + ... + x^6/7!) (truncation below 2e-7
// relative); else the hardware 2^x (relative error of e^x - 1 below 1e-6 there).
__device__ __forceinline__ float planck_shape(float x) {
  if (x < 0.5f) {
    float q = fmaf(x, 1.f / 5040.f, 1.f / 720.f);
    q = fmaf(x, q, 1.f / 120.f);
    q = fmaf(x, q, 1.f / 24.f);
    q = fmaf(x, q, 1.f / 6.f);
    q = fmaf(x, q, 0.5f);
    q = fmaf(x, q, 1.f);
    return __fdividef(1.f, x * q);
  }
  return __fdividef(1.f, ex2f(x * 1.4426950408889634f) - 1.f);
}

// One thread per native wavenumber of the range, one CTA row per chunk item; MU: the largest
// n_mu the instance serves (its angle loop is unrolled to MU).
template <int MU>
__global__ void __launch_bounds__(kEmThreads) k_emission(EmParams p) {
  __shared__ float2 lay_s[TR_MAX_LAYERS];               // (dz_l, c_2 / T_l)
  const int c = blockIdx.y, b = p.b_off + c;
  const ItemGeom ig = p.buf.items[b];
  const int N = ig.n_layers;
  const double* z = p.buf.z + (size_t)b * (p.max_layers + 1);
  const double* tl = p.buf.tl + (size_t)b * p.max_layers;
  for (int l = threadIdx.x; l < N; l += kEmThreads)
    lay_s[l] = make_float2((float)(z[l + 1] - z[l]), (float)(kC2cmK / tl[l]));
  __syncthreads();
  const int i = blockIdx.x * kEmThreads + threadIdx.x;
  if (i >= p.wn_count) return;
  double* o = p.out + (size_t)b * p.out_stride + i;
  if (N == 0) { *o = 0.0; return; }
  const int w = p.wn_begin + i;
  const float nu = (float)__ldg(p.wn + w);
  const float* kr = p.kbuf + (size_t)c * p.max_layers * p.kcols + (w - wn_first(p.wn_begin));
  float I[MU];
  const float bs = planck_shape(nu * (float)(kC2cmK / ig.t_surf));   // surface, E3
#pragma unroll
  for (int k = 0; k < MU; ++k) I[k] = bs;
  // bottom (l = 0) to top, eight layers per step: their K values are loaded first so the
  // loads' latency overlaps instead of stalling every layer
  constexpr int kU = 8;
  auto layer = [&](float kval, int l) {
    const float2 ld = lay_s[l];
    const float dtau = kval * ld.x;
    const float bl = planck_shape(nu * ld.y);
#pragma unroll
    for (int k = 0; k < MU; ++k)
      if (k < p.n_mu) I[k] = fmaf(I[k] - bl, ex2f(dtau * p.mu_coef[k]), bl);
  };
  const long long kc = p.kcols;
  int l0 = 0;
  for (; l0 + kU <= N; l0 += kU, kr += kU * kc) {      // whole blocks, no per-layer guard
    float kv[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) kv[j] = __ldg(kr + j * kc);
#pragma unroll
    for (int j = 0; j < kU; ++j) layer(kv[j], l0 + j);
  }
  for (int j = 0; l0 + j < N; ++j) layer(__ldg(kr + j * kc), l0 + j);   // the last few
  float num = 0.f;
#pragma unroll
  for (int k = 0; k < MU; ++k)
    if (k < p.n_mu) num = fmaf(p.xw[k], I[k], num);
  const float bstar = planck_shape(nu * p.c2_tstar);
  *o = (bstar > 0.f) ? (double)num / (double)bstar * ig.rp2_rs2 : 0.0;
}

// n-point Gauss-Legendre rule on [0, 1]: the roots of the Legendre polynomial P_n, found by
// Newton's method from the asymptotic first guess cos(pi (k + 3/4) / (n + 1/2)), with P_n and
// P_{n-1} from Bonnet's recurrence (j + 1) P_{j+1} = (2j + 1) t P_j - j P_{j-1} and the
// derivative P_n' = n (P_{n-1} - t P_n) / (1 - t^2); weight 2 / ((1 - t^2) P_n'^2), then
// mapped from [-1, 1] to [0, 1] (nodes (1 + t)/2, weights halved).
void legendre_rule01(int n, std::vector<double>* x, std::vector<double>* w) {
  x->resize(n);
  w->resize(n);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    double t = std::cos(pi * (k + 0.75) / (n + 0.5));
    double pn = 0.0, pn1 = 0.0;
    for (int it = 0; it < 64; ++it) {
      double a = 1.0, bb = t;                           // P_0, P_1
      if (n == 1) { pn = t; pn1 = 1.0; }
      else {
        for (int j = 1; j < n; ++j) {
          const double c = ((2.0 * j + 1.0) * t * bb - j * a) / (j + 1.0);
          a = bb;
          bb = c;
        }
        pn = bb; pn1 = a;
      }
      const double d = n * (pn1 - t * pn) / (1.0 - t * t);
      const double step = pn / d;
      t -= step;
      if (std::fabs(step) <= 1e-15 * std::fabs(t) + 1e-300) break;
    }
    double a = 1.0, bb = t;
    if (n == 1) { pn = t; pn1 = 1.0; }
    else {
      for (int j = 1; j < n; ++j) {
        const double c = ((2.0 * j + 1.0) * t * bb - j * a) / (j + 1.0);
        a = bb;
        bb = c;
      }
      pn = bb; pn1 = a;
    }
    const double d = n * (pn1 - t * pn) / (1.0 - t * t);
    (*x)[k] = 0.5 * (1.0 + t);
    (*w)[k] = 1.0 / ((1.0 - t * t) * d * d);            // (2 / ((1 - t^2) d^2)) / 2
  }
}

int check_emission_args(tr_ctx* ctx, int n_mu, double t_star) {
  if (n_mu < 1 || n_mu > kEmMaxMu)
    return set_error(ctx, TR_ERR_ARG, "n_mu must be in 1.." + std::to_string(kEmMaxMu));
  if (!(t_star > 0.0) || !std::isfinite(t_star))
    return set_error(ctx, TR_ERR_ARG, "t_star must be positive");
  return TR_OK;
}

// Opacity (two-stage opacity kernel, chunk by chunk through kbuf) then the emission pass, for
// items [0, B) of `buf`, native range [wn_begin, wn_begin + wn_count).
int run_emission(tr_ctx* ctx, const tr_tables* t, int max_layers, const ItemBuffers& buf, int B,
                 int wn_begin, int wn_count, double* out, long long stride, int precision,
                 float* kbuf, int n_mu, double t_star, cudaStream_t s) {
  const bool mixed = precision == TR_PREC_MIXED;
  if (precision != TR_PREC_FP32 && !mixed) return set_error(ctx, TR_ERR_ARG, "unknown precision");
  if (!mixed && !t->d_sigma && t->n_mol > 0)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "tables were loaded without FP32 storage");
  if (mixed && !t->d_logsig16 && t->n_mol > 0)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "tables were loaded without FP16 log10 storage");
  if (buf.zoned && t->interp_mode != TR_INTERP_LINEAR)
    return set_error(ctx, TR_ERR_UNSUPPORTED, "two-layer gases need the linear temperature scheme");
  FwdParams fp = forward_fp32_params(t, max_layers, buf, wn_begin, wn_count, nullptr, 0,
                                     ctx->dev_err);
  if (mixed) {
    fp.logsig16 = t->d_logsig16;
    for (int m = 0; m < t->n_mol; ++m) fp.logsig_off[m] = t->logsig_offset[m];
  }
  EmParams ep{};
  ep.buf = buf; ep.max_layers = max_layers; ep.kbuf = kbuf;
  ep.kcols = forward_kcols(wn_begin, wn_count); ep.wn = t->d_wn;
  ep.wn_begin = wn_begin; ep.wn_count = wn_count; ep.n_mu = n_mu;
  std::vector<double> x, w;
  legendre_rule01(n_mu, &x, &w);
  double sxw = 0.0;
  for (int k = 0; k < n_mu; ++k) sxw += x[k] * w[k];
  for (int k = 0; k < n_mu; ++k) {
    ep.mu_coef[k] = (float)(-1.4426950408889634 / x[k]);
    ep.xw[k] = (float)(x[k] * w[k] / sxw);
  }
  ep.c2_tstar = (float)(kC2cmK / t_star);
  ep.out = out; ep.out_stride = stride;
  const int chunk = forward_chunk_items(B, max_layers, wn_begin, wn_count);
  cudaError_t e = cudaSuccess;
  for (int b0 = 0; b0 < B && e == cudaSuccess; b0 += chunk) {
    const int bc = std::min(chunk, B - b0);
    fp.b_off = b0;
    {
      KernelTimer kt(ctx, mixed ? "k_opacity_fp16" : "k_opacity_fp32", s);
      e = launch_opacity(fp, mixed ? &t->tm_sig16 : &t->tm_sig32, &t->tm_cia, bc, kbuf, 0, s);
    }
    if (e != cudaSuccess) break;
    ep.b_off = b0;
    KernelTimer kt(ctx, "k_emission", s);
    const dim3 grid((wn_count + kEmThreads - 1) / kEmThreads, bc);
    if (n_mu <= 4) k_emission<4><<<grid, kEmThreads, 0, s>>>(ep);
    else if (n_mu <= 8) k_emission<8><<<grid, kEmThreads, 0, s>>>(ep);
    else k_emission<kEmMaxMu><<<grid, kEmThreads, 0, s>>>(ep);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? TR_OK : set_error(ctx, TR_ERR_CUDA, std::string("emission kernels: ") + cudaGetErrorString(e));
}

}  // namespace
}  // namespace tr

using namespace tr;

extern "C" int tr_forward_emission(tr_ctx* ctx, const tr_tables* t, const tr_atm* a,
                                   const tr_bins* bins, int n_mu, double t_star,
                                   double* d_native, double* d_binned, int precision,
                                   void* stream) {
  if (!ctx || !t || !a) return set_error(ctx, TR_ERR_ARG, "null argument");
  if (!d_native && !d_binned) return set_error(ctx, TR_ERR_ARG, "no output requested");
  if (d_binned && !bins) return set_error(ctx, TR_ERR_ARG, "binned output needs bins");
  int rc = check_emission_args(ctx, n_mu, t_star);
  if (rc != TR_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // context scratch: [binned-region spectrum (binned output only)][K buffer]
  const int wb = d_native ? 0 : bins->dev.i0;
  const int wc = d_native ? t->n_wn : bins->dev.i1 - bins->dev.i0;
  const size_t off_k = al256(sizeof(double) * (size_t)(d_native ? 0 : wc));
  rc = ensure_scratch(ctx, off_k + forward_kbuf_bytes(1, a->n_layers, wb, wc));
  if (rc != TR_OK) return rc;
  char* sc = static_cast<char*>(ctx->scratch);
  float* kbuf = reinterpret_cast<float*>(sc + off_k);
  double* spec = d_native ? d_native : reinterpret_cast<double*>(sc);
  rc = run_emission(ctx, t, a->n_layers, a->buf, 1, wb, wc, spec, wc, precision, kbuf, n_mu,
                    t_star, s);
  if (rc != TR_OK || !d_binned) return rc;
  return run_bin(ctx, bins, 1, spec, wc, wb, d_binned, s);
}

extern "C" int tr_forward_emission_batch(tr_ctx* ctx, const tr_tables* t,
                                         const tr_batch_desc* d, int B, const double* d_theta,
                                         const int32_t* d_nlayers, const tr_bins* bins,
                                         int n_mu, double t_star, double* d_native,
                                         double* d_binned, int32_t* d_status, int precision,
                                         void* ws, size_t ws_bytes, void* stream) {
  int rc = check_forward_batch_args(ctx, t, d, B, d_theta, bins, d_native, d_binned);
  if (rc != TR_OK) return rc;
  rc = check_emission_args(ctx, n_mu, t_star);
  if (rc != TR_OK) return rc;
  if (B == 0) return TR_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the batched forward's workspace: [item buffers + binned-region spectra][K buffer][...]
  const int n_in = d_native ? 0 : bins->dev.i1 - bins->dev.i0;
  const size_t need = forward_batch_need(t, d, B, bins, d_native != nullptr, precision);
  ItemBuffers buf; double* depth = nullptr; char* extra = nullptr;
  rc = prepare_batch(ctx, t, d, n_in, need, B, d_theta, d_nlayers, d_status, ws, ws_bytes, s,
                     &buf, &depth, &extra);
  if (rc != TR_OK) return rc;
  float* kbuf = reinterpret_cast<float*>(extra);
  if (d_native) {
    rc = run_emission(ctx, t, d->max_layers, buf, B, 0, t->n_wn, d_native, t->n_wn, precision,
                      kbuf, n_mu, t_star, s);
    if (rc != TR_OK || !d_binned) return rc;
    return run_bin(ctx, bins, B, d_native, t->n_wn, 0, d_binned, s);
  }
  rc = run_emission(ctx, t, d->max_layers, buf, B, bins->dev.i0, n_in, depth, n_in, precision,
                    kbuf, n_mu, t_star, s);
  if (rc != TR_OK) return rc;
  return run_bin(ctx, bins, B, depth, n_in, bins->dev.i0, d_binned, s);
}
