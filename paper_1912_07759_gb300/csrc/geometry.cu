// geometry.cu -- FP64 atmosphere set-up on the device: pressure grid (Sec. 4.1), temperature
// profile (Sec. 4.2), free chemistry and mean molecular weight (Sec. 4.3), hydrostatic
// altitudes (Sec. 4, equation for z_l), number density, interpolation brackets and weights
// (Sec. 5, linear scheme and out-of-range rules), cloud deck (Sec. 4.4, eq. clouds), annulus
// weights and slant path lengths.
//
// Two kernels, so that the FP64 work (GB300 issues only a few FP64 operations per clock per
// SM) spreads over many SMs even for a single atmosphere:
//   k_profile   one CTA per atmosphere: threads work over layers; thread 0 runs the altitude
//               recursion, the only serial step; the CTA also builds the atmosphere's row
//               plan (the distinct table rows its layers touch);
//   k_pathlen   one warp per (atmosphere, 4 consecutive shells): lanes over rays, the square
//               root of the shell below carried in registers (one root per path length),
//               rows of the dense layer-major matrix written coalesced.
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kProfileThreads = 64;
constexpr int kPathWarps = 2;

// Largest i in [0, n-2] with grid[i] <= x (0 when x < grid[0]).
__device__ __forceinline__ int bracket(const double* __restrict__ grid, int n, double x) {
  if (!(grid[0] <= x)) return 0;
  int lo = 0, hi = n - 2;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (grid[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Linear-interpolation bracket and weight along one table axis; false when the paper's
// out-of-range rule gives zero (x below the grid minimum).  inv[i] = 1 / (grid[i+1] - grid[i]).
__device__ __forceinline__ bool axis(const double* __restrict__ grid,
                                     const double* __restrict__ inv, int n, double x, int oor,
                                     int* i, double* t) {
  if (oor == TR_OOR_PAPER_ZERO && x < grid[0]) { *i = 0; *t = 0.0; return false; }
  const double xc = fmin(fmax(x, grid[0]), grid[n - 1]);
  const int k = bracket(grid, n, xc);
  *i = k;
  *t = (xc - grid[k]) * inv[k];
  return true;
}

// sqrt(x) for x > 0 in FP64: single-precision reciprocal square root as the seed, then one
// Newton-Raphson (Heron) correction in FP64, s1 = s0 + y0 (x - s0^2) / 2 with s0 = x y0.  The
// seed's relative error e (~1e-7) leaves an error of order e^2 (~1e-14) after the step.
__device__ __forceinline__ double sqrt_newton(double x) {
  const double y0 = (double)rsqrtf((float)x);
  const double s0 = x * y0;
  const double r = fma(-s0, s0, x);
  return fma(0.5 * y0, r, s0);
}

struct ItemShared {
  double X[TR_MAX_SPECIES];
  double slope[TR_MAX_TNODES];   // dT / dlog10 P of each node segment
  double rp, mu, delta, lptop, cz, inv_kb;
  int N, status;
  int part[kProfileThreads];     // scan partial sums of the row plan
};

// Exclusive scan of the 0/1 marks in mark[0..n) into slots, by kProfileThreads threads
// (contiguous chunks, then a scan of the chunk sums).  Returns the total.
__device__ int scan_marks(const uint8_t* mark, uint16_t* slot, int n, int* part) {
  const int t = threadIdx.x;
  const int chunk = (n + kProfileThreads - 1) / kProfileThreads;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int c = 0;
  for (int i = lo; i < hi; ++i) c += mark[i];
  part[t] = c;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int k = 0; k < kProfileThreads; ++k) { const int v = part[k]; part[k] = acc; acc += v; }
  }
  __syncthreads();
  int base = part[t];
  for (int i = lo; i < hi; ++i) { slot[i] = (uint16_t)base; base += mark[i]; }
  __syncthreads();
  int total = 0;
  if (n > 0) total = slot[n - 1] + mark[n - 1];
  return total;
}

// One CTA per atmosphere: threads work over layers, thread 0 runs the altitude recursion.
__global__ void __launch_bounds__(kProfileThreads)
k_profile(GeomParams gp, int B, const double* __restrict__ theta, int n_theta,
          const int32_t* __restrict__ nlayers, int32_t* __restrict__ status_out,
          ItemBuffers buf) {
  extern __shared__ double sm[];
  __shared__ ItemShared w;
  const int b = blockIdx.x;
  if (b >= B) return;
  const int tid = threadIdx.x;
  const int NM = gp.max_layers;
  const int n_cells_all = gp.n_p * gp.n_t;
  double* P = sm;                                   // [NM]
  double* T = P + NM;                               // [NM]
  double* lnpb = T + NM;                            // [NM + 1] ln of boundary pressures
  double* r = lnpb + NM + 1;                        // [NM + 1] radii of the boundaries
  uint16_t* cslot_all = reinterpret_cast<uint16_t*>(r + NM + 1);   // [n_cells_all + n_t_cia]
  uint8_t* mark = reinterpret_cast<uint8_t*>(cslot_all + n_cells_all + gp.n_t_cia);
  double* z = buf.z + (size_t)b * (NM + 1);         // [NM + 1] altitudes (global: k_pathlen)
  const double* th = theta + (size_t)b * n_theta;

  // ---- chemistry (Sec. 4.3) and temperature-node slopes (Sec. 4.2)
  if (tid < gp.n_mol) w.X[tid] = exp10(th[tid]);
  if (tid + 1 < gp.n_tnodes) {
    const double* tn = th + gp.n_mol;
    w.slope[tid] = (tn[tid + 1] - tn[tid]) / (gp.tnode_log10p[tid + 1] - gp.tnode_log10p[tid]);
  }
  __syncthreads();
  // ---- validation (model rejection of Sec. 6)
  if (tid == 0) {
    int st = TR_OK;
    const int N = nlayers ? nlayers[b] : NM;
    if (N < 1 || N > NM) st = TR_ERR_INVALID_MODEL;
    for (int k = 0; k < n_theta; ++k)
      if (!isfinite(th[k])) st = TR_ERR_INVALID_MODEL;
    double mu = 0.0;
    if (st == TR_OK) {
      double sumx = 0.0;
      for (int m = 0; m < gp.n_mol; ++m) sumx += w.X[m];
      if (sumx > 1.0) st = TR_ERR_INVALID_MODEL;
      const double rem = 1.0 - sumx;
      for (int f = gp.n_mol; f < gp.n_species; ++f) w.X[f] = gp.fill[f] * rem;
      for (int s = 0; s < gp.n_species; ++s) mu += w.X[s] * gp.mass[s];
      if (!(mu > 0.0)) st = TR_ERR_INVALID_MODEL;
      for (int k = 0; k < gp.n_tnodes; ++k)
        if (!(th[gp.n_mol + k] > 0.0)) st = TR_ERR_INVALID_MODEL;
      w.rp = th[gp.n_mol + gp.n_tnodes] * kRJup;
      if (!(w.rp > 0.0)) st = TR_ERR_INVALID_MODEL;
      w.lptop = th[gp.n_mol + gp.n_tnodes + 1];
    }
    w.mu = mu;
    w.N = (st == TR_OK) ? N : 0;
    w.status = st;
    w.delta = (log(gp.p_max) - log(gp.p_min)) / (st == TR_OK ? N : 1);
    // z_{l+1} - z_l = H_l Delta = k_B T_l Delta / (mu m_u g_l), g_l = G M_p / r_l^2:
    // the step is cz T_l r_l^2 with cz = k_B Delta / (mu m_u G M_p)
    w.cz = (st == TR_OK) ? kKB * w.delta / (mu * kAMU * kG * gp.m_p) : 0.0;
    w.inv_kb = 1.0 / kKB;
    buf.items[b].status = st;
    buf.items[b].n_layers = w.N;
    buf.items[b].r_p = (st == TR_OK) ? w.rp : 0.0;
    buf.items[b].rp2_rs2 = (st == TR_OK) ? (w.rp * w.rp) / (gp.r_s * gp.r_s) : 0.0;
    if (status_out) status_out[b] = st;
  }
  __syncthreads();
  const int N = w.N;
  float* aj = buf.aj + (size_t)b * buf.npad;
  if (w.status != TR_OK) {
    for (int j = tid; j < buf.npad; j += kProfileThreads) aj[j] = 0.f;
    if (tid == 0) { buf.plans[b].n_cells = -1; buf.plans[b].n_cia = 0; }
    return;
  }

  // ---- pressure grid (Sec. 4.1) and temperature profile (Sec. 4.2), parallel over layers:
  //      P_l = p_l sqrt(p_{l+1}/p_l) = exp((ln p_l + ln p_{l+1}) / 2)
  const double lmax = log(gp.p_max), lmin = log(gp.p_min);
  for (int k = tid; k <= N; k += kProfileThreads) lnpb[k] = lmax + (lmin - lmax) * k / N;
  __syncthreads();
  const double inv_ln10 = 0.43429448190325182765;
  for (int l = tid; l < N; l += kProfileThreads) {
    const double lnp = 0.5 * (lnpb[l] + lnpb[l + 1]);
    P[l] = exp(lnp);
    const double* tn = th + gp.n_mol;
    double t;
    if (gp.n_tnodes == 1) {
      t = tn[0];
    } else {
      const double x = lnp * inv_ln10;
      const int nt = gp.n_tnodes;
      if (x >= gp.tnode_log10p[0]) t = tn[0];
      else if (x <= gp.tnode_log10p[nt - 1]) t = tn[nt - 1];
      else {
        int k = 0;
        while (!(gp.tnode_log10p[k] >= x && x >= gp.tnode_log10p[k + 1])) ++k;
        t = tn[k] + w.slope[k] * (x - gp.tnode_log10p[k]);
      }
    }
    T[l] = t;
  }
  for (int i = tid; i < n_cells_all + gp.n_t_cia; i += kProfileThreads) mark[i] = 0;
  __syncthreads();

  // ---- hydrostatic altitudes (Sec. 4), serial in l on thread 0, on the boundary radii:
  //      r_{l+1} = r_l + a_l r_l^2 with a_l = cz T_l (constant gravity: r_l^2 -> R_p^2).
  //      Meanwhile the other threads mark the table rows the layers touch.
  if (tid == 0) {
    const double rp = w.rp, cz = w.cz;
    double rl = rp;
    r[0] = rp;
    if (gp.gravity_mode == TR_GRAV_CONST) {
      const double k2 = cz * rp * rp;
      for (int l = 0; l < N; ++l) { rl = fma(k2, T[l], rl); r[l + 1] = rl; }
    } else {
      for (int l = 0; l < N; ++l) { rl = fma(cz * T[l] * rl, rl, rl); r[l + 1] = rl; }
    }
  }
  // per-layer brackets in the same pass (needed for the row plan)
  LayerDesc* L = buf.layers + (size_t)b * NM;
  for (int l = tid; l < N; l += kProfileThreads) {
    const int ip = bracket(gp.p_grid, gp.n_p, fmin(fmax(P[l], gp.p_grid[0]), gp.p_grid[gp.n_p - 1]));
    const int it = bracket(gp.t_grid, gp.n_t, fmin(fmax(T[l], gp.t_grid[0]), gp.t_grid[gp.n_t - 1]));
    const int c0 = ip * gp.n_t + it;
    mark[c0] = 1; mark[c0 + 1] = 1; mark[c0 + gp.n_t] = 1; mark[c0 + gp.n_t + 1] = 1;
    if (gp.n_cia > 0) {
      const int itc = bracket(gp.t_grid_cia, gp.n_t_cia,
                              fmin(fmax(T[l], gp.t_grid_cia[0]), gp.t_grid_cia[gp.n_t_cia - 1]));
      mark[n_cells_all + itc] = 1; mark[n_cells_all + itc + 1] = 1;
    }
  }
  __syncthreads();
  RowPlan& plan = buf.plans[b];
  const int n_cells = scan_marks(mark, cslot_all, n_cells_all, w.part);
  const int n_ccia = gp.n_cia > 0 ? scan_marks(mark + n_cells_all, cslot_all + n_cells_all,
                                               gp.n_t_cia, w.part) : 0;
  const bool plan_ok = n_cells <= kPlanMaxCells && n_ccia <= kPlanMaxCia;
  for (int i = tid; i < n_cells_all; i += kProfileThreads)
    if (mark[i] && plan_ok) plan.cell[cslot_all[i]] = (uint16_t)i;
  for (int i = tid; i < gp.n_t_cia; i += kProfileThreads)
    if (mark[n_cells_all + i] && plan_ok) plan.cia_row[cslot_all[n_cells_all + i]] = (uint16_t)i;
  if (tid == 0) { plan.n_cells = plan_ok ? n_cells : -1; plan.n_cia = plan_ok ? n_ccia : 0; }
  for (int k = tid; k <= N; k += kProfileThreads) z[k] = r[k] - w.rp;
  __syncthreads();

  // ---- per-layer descriptors: density, brackets, corner coefficients, cloud; annulus weights
  const double rp = w.rp;
  const double inv_rs2 = 1.0 / (gp.r_s * gp.r_s);
  for (int l = tid; l < N; l += kProfileThreads) {
    LayerDesc d;
    const double rho = P[l] * w.inv_kb / T[l];
    double tp = 0.0, tt = 0.0, ttc = 0.0;
    const bool okp = axis(gp.p_grid, gp.inv_dp, gp.n_p, P[l], gp.oor_mode, &d.ip, &tp);
    const bool okt = axis(gp.t_grid, gp.inv_dt, gp.n_t, T[l], gp.oor_mode, &d.it, &tt);
    const bool okm = okp && okt;
    // the brackets of axis() equal the clamped ones used for the row plan, also when the
    // paper's rule zeroes sigma (then the weights below are zero)
    const int c0 = d.ip * gp.n_t + d.it;
    d.slot[0] = (uint8_t)cslot_all[c0];
    d.slot[1] = (uint8_t)cslot_all[c0 + 1];
    d.slot[2] = (uint8_t)cslot_all[c0 + gp.n_t];
    d.slot[3] = (uint8_t)cslot_all[c0 + gp.n_t + 1];
    d.rho = (float)rho;
    d.tp = (float)tp;
    d.tt = (float)tt;
    // bilinear corner weights (P_i, T_j), (P_i, T_j+1), (P_i+1, T_j), (P_i+1, T_j+1) in FP32
    const float tpf = (float)tp, ttf = (float)tt;
    const float cw[4] = {(1.f - tpf) * (1.f - ttf), (1.f - tpf) * ttf, tpf * (1.f - ttf), tpf * ttf};
    for (int m = 0; m < TR_MAX_MOL; ++m) {
      const float wm = (m < gp.n_mol && okm) ? (float)(rho * w.X[m]) : 0.f;
      d.w_mol[m] = wm;
      for (int k = 0; k < 4; ++k) d.cm[m][k] = wm * cw[k];
    }
    bool okc = true;
    d.itc = 0;
    if (gp.n_cia > 0)
      okc = axis(gp.t_grid_cia, gp.inv_dtc, gp.n_t_cia, T[l], gp.oor_mode, &d.itc, &ttc);
    d.cslot[0] = gp.n_cia > 0 ? (uint8_t)cslot_all[n_cells_all + d.itc] : 0;
    d.cslot[1] = gp.n_cia > 0 ? (uint8_t)cslot_all[n_cells_all + d.itc + 1] : 0;
    d.flags = (uint8_t)((okm ? 0 : kLayerMolZero) |
                        ((T[l] <= gp.t_grid[0] || T[l] >= gp.t_grid[gp.n_t - 1]) ? kLayerTClamp : 0) |
                        (okc ? 0 : kLayerCiaZero) |
                        ((gp.n_cia > 0 && (T[l] <= gp.t_grid_cia[0] ||
                                           T[l] >= gp.t_grid_cia[gp.n_t_cia - 1])) ? kLayerTcClamp : 0));
    d.pad_c = 0;
    d.pad_f = 0.f;
    buf.tl[(size_t)b * NM + l] = T[l];
    d.ttc = (float)ttc;
    const double rho2 = rho * rho;
    for (int q = 0; q < TR_MAX_CIA; ++q) {
      const float wc = (q < gp.n_cia && okc)
          ? (float)(rho2 * (w.X[gp.cia_a[q]] * w.X[gp.cia_b[q]] * gp.cia_scale[q])) : 0.f;
      d.w_cia[q] = wc;
      d.cc[q][0] = wc * (1.f - d.ttc);
      d.cc[q][1] = wc * d.ttc;
    }
    double cf = 0.0;
    if (gp.cloud_mode == TR_CLOUD_DISCRETE) {
      const double p_top = exp10(w.lptop);
      const double p_bot = gp.p_cloud_bot > 0.0 ? gp.p_cloud_bot : gp.p_max;
      cf = (P[l] >= p_top && P[l] <= p_bot) ? 1.0 : 0.0;
    } else if (gp.cloud_mode == TR_CLOUD_FRACTIONAL) {
      const double ln_bot = gp.p_cloud_bot > 0.0 ? log(gp.p_cloud_bot) : lmax;
      const double ln_top = w.lptop * 2.302585092994046;   // ln 10
      const double hi = fmin(lnpb[l], ln_bot);
      const double lo = fmax(ln_top, lnpb[l + 1]);
      cf = fmin(fmax((hi - lo) / w.delta, 0.0), 1.0);
    }
    d.cloud = (float)cf;
    d.k_cloud = (float)(gp.kappa_cloud * cf);
    L[l] = d;
    // A_j / R_s^2 = (r_{j+1} - r_j)(r_{j+1} + r_j) / R_s^2
    aj[l] = (float)((z[l + 1] - z[l]) * (r[l + 1] + r[l]) * inv_rs2);
  }
  for (int j = N + tid; j < buf.npad; j += kProfileThreads) aj[j] = 0.f;
  if (tid < TR_MAX_SPECIES)
    buf.rayc[(size_t)b * TR_MAX_SPECIES + tid] =
        (gp.has_ray && tid < gp.n_species) ? (float)(w.X[tid] * gp.ray_scale[tid]) : 0.f;
  (void)rp;
}

// Slant path lengths (reading R1): DL[j][l] = 2 (s(l+1, j) - s(l, j)) for l >= j with
// s(k, j) = sqrt(r_k^2 - r_j^2), r_k^2 - r_j^2 = (z_k - z_j)(r_k + r_j).  Written dense and
// layer-major: row l holds rays j = 0..npad-1 (zero for j > l and j >= N).  A warp walks
// rows_per_warp consecutive rows with lanes over rays, carrying s(l, j) from the row below,
// so each path length costs one square root (plus one per ray at the first row); rows are
// written coalesced.
__global__ void __launch_bounds__(32 * kPathWarps)
k_pathlen(int max_layers, int rows_per_warp, ItemBuffers buf) {
  const int b = blockIdx.y;
  const int l0 = (blockIdx.x * kPathWarps + (threadIdx.x >> 5)) * rows_per_warp;
  const int lane = threadIdx.x & 31;
  const int N = buf.items[b].n_layers;
  if (l0 >= N) return;
  const double* z = buf.z + (size_t)b * (max_layers + 1);
  const double two_rp = 2.0 * buf.items[b].r_p;
  float* dl = buf.dlt + (size_t)b * max_layers * buf.npad;
  const int l1 = min(l0 + rows_per_warp, N);
  for (int j0 = 0; j0 < buf.npad; j0 += 32) {
    const int j = j0 + lane;
    const bool ray = j < N && j <= l1 - 1;
    const double zj = ray ? z[j] : 0.0;
    // s(l0, j) for rays below row l0 (s(j, j) = 0)
    double s_lo = 0.0;
    if (ray && j < l0) s_lo = sqrt_newton((z[l0] - zj) * (two_rp + z[l0] + zj));
    for (int l = l0; l < l1; ++l) {
      float v = 0.f;
      if (ray && j <= l) {
        const double zu = z[l + 1];
        const double s_hi = sqrt_newton((zu - zj) * (two_rp + zu + zj));
        v = (float)(2.0 * (s_hi - s_lo));
        s_lo = s_hi;
      }
      if (j < buf.npad) dl[(size_t)l * buf.npad + j] = v;
    }
  }
}

}  // namespace

cudaError_t launch_geometry(const GeomParams& gp, int B, const double* d_theta, int n_theta,
                            const int32_t* d_nlayers, int32_t* d_status, ItemBuffers buf,
                            cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const size_t cells = (size_t)gp.n_p * gp.n_t + gp.n_t_cia;
  const size_t smem = sizeof(double) * (4 * (size_t)gp.max_layers + 2) + cells * 3 + 16;
  k_profile<<<B, kProfileThreads, smem, s>>>(gp, B, d_theta, n_theta, d_nlayers, d_status, buf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // few atmospheres: one shell row per warp, spread over many SMs; many: 4 rows per warp
  const int rows_per_warp = B < 16 ? 1 : 4;
  const int rows_per_cta = kPathWarps * rows_per_warp;
  dim3 grid((gp.max_layers + rows_per_cta - 1) / rows_per_cta, B);
  k_pathlen<<<grid, 32 * kPathWarps, 0, s>>>(gp.max_layers, rows_per_warp, buf);
  return cudaGetLastError();
}

}  // namespace tr
