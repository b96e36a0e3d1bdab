// geometry.cu -- FP64 atmosphere set-up on the device: pressure grid (Sec. 4.1), temperature
// profile (Sec. 4.2), free chemistry and mean molecular weight (Sec. 4.3), hydrostatic
// altitudes (Sec. 4, equation for z_l), number density, interpolation brackets (Sec. 5,
// linear scheme and out-of-range rules), cloud deck (Sec. 4.4, eq. clouds), slant path lengths
// and annulus weights.  One CTA per atmosphere; the altitude recursion is the only serial
// step (one thread), everything else is parallel over layers or rays.
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kGeomThreads = 64;

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
// out-of-range rule gives zero (x below the grid minimum).
__device__ __forceinline__ bool axis(const double* __restrict__ grid, int n, double x, int oor,
                                     int* i, float* t) {
  if (oor == TR_OOR_PAPER_ZERO && x < grid[0]) { *i = 0; *t = 0.f; return false; }
  const double xc = fmin(fmax(x, grid[0]), grid[n - 1]);
  const int k = bracket(grid, n, xc);
  *i = k;
  *t = (float)((xc - grid[k]) / (grid[k + 1] - grid[k]));
  return true;
}

__global__ void __launch_bounds__(kGeomThreads)
k_geometry(GeomParams gp, int B, const double* __restrict__ theta, int n_theta,
           const int32_t* __restrict__ nlayers, int32_t* __restrict__ status_out,
           ItemBuffers buf) {
  extern __shared__ double sm[];
  const int b = blockIdx.x;
  if (b >= B) return;
  const int NM = gp.max_layers;
  double* z = sm;              // [NM + 1]
  double* P = z + NM + 1;      // [NM]
  double* T = P + NM;          // [NM]
  double* c = T + NM;          // [NM] altitude step coefficients
  double* lnpb = c + NM;       // [NM + 1] ln of boundary pressures
  __shared__ double s_X[TR_MAX_SPECIES];
  __shared__ double s_rp, s_mu, s_delta, s_lptop;
  __shared__ int s_N, s_status;

  const double* th = theta + (size_t)b * n_theta;
  const int tid = threadIdx.x;

  // ---- validation and chemistry (Sec. 4.3; model rejection of Sec. 6)
  if (tid == 0) {
    int st = TR_OK;
    const int N = nlayers ? nlayers[b] : NM;
    if (N < 1 || N > NM) st = TR_ERR_INVALID_MODEL;
    for (int k = 0; k < n_theta; ++k)
      if (!isfinite(th[k])) st = TR_ERR_INVALID_MODEL;
    double sumx = 0.0, mu = 0.0;
    if (st == TR_OK) {
      for (int m = 0; m < gp.n_mol; ++m) { s_X[m] = exp10(th[m]); sumx += s_X[m]; }
      if (sumx > 1.0) st = TR_ERR_INVALID_MODEL;
      const double rem = 1.0 - sumx;
      for (int f = gp.n_mol; f < gp.n_species; ++f) s_X[f] = gp.fill[f] * rem;
      for (int s = 0; s < gp.n_species; ++s) mu += s_X[s] * gp.mass[s];
      if (!(mu > 0.0)) st = TR_ERR_INVALID_MODEL;
      for (int k = 0; k < gp.n_tnodes; ++k)
        if (!(th[gp.n_mol + k] > 0.0)) st = TR_ERR_INVALID_MODEL;
      s_rp = th[gp.n_mol + gp.n_tnodes] * kRJup;
      if (!(s_rp > 0.0)) st = TR_ERR_INVALID_MODEL;
      s_lptop = th[gp.n_mol + gp.n_tnodes + 1];
    }
    s_mu = mu;
    s_N = (st == TR_OK) ? N : 0;
    s_status = st;
    s_delta = (log(gp.p_max) - log(gp.p_min)) / (st == TR_OK ? N : 1);
    buf.items[b].status = st;
    buf.items[b].n_layers = s_N;
    buf.items[b].rp2_rs2 = (st == TR_OK) ? (s_rp * s_rp) / (gp.r_s * gp.r_s) : 0.0;
    if (status_out) status_out[b] = st;
  }
  __syncthreads();
  const int N = s_N;
  float* aj = buf.aj + (size_t)b * NM;
  if (s_status != TR_OK) {
    for (int j = tid; j < NM; j += blockDim.x) aj[j] = 0.f;
    return;
  }

  // ---- pressure grid (Sec. 4.1) and temperature profile (Sec. 4.2), parallel over layers
  const double lmax = log(gp.p_max), lmin = log(gp.p_min);
  for (int k = tid; k <= N; k += blockDim.x) lnpb[k] = lmax + (lmin - lmax) * k / N;
  __syncthreads();
  for (int l = tid; l < N; l += blockDim.x) {
    const double pl = exp(lnpb[l]);
    const double pu = exp(lnpb[l + 1]);
    P[l] = pl * sqrt(pu / pl);
    const double* tn = th + gp.n_mol;
    double t;
    if (gp.n_tnodes == 1) {
      t = tn[0];
    } else {
      const double x = log10(P[l]);
      const int nt = gp.n_tnodes;
      if (x >= gp.tnode_log10p[0]) t = tn[0];
      else if (x <= gp.tnode_log10p[nt - 1]) t = tn[nt - 1];
      else {
        int k = 0;
        while (!(gp.tnode_log10p[k] >= x && x >= gp.tnode_log10p[k + 1])) ++k;
        const double f = (x - gp.tnode_log10p[k]) / (gp.tnode_log10p[k + 1] - gp.tnode_log10p[k]);
        t = tn[k] + (tn[k + 1] - tn[k]) * f;
      }
    }
    T[l] = t;
    // z_{l+1} - z_l = H_l Delta = k_B T_l Delta / (mu m_u g_l), g_l = G M_p / r_l^2
    c[l] = kKB * t * s_delta / (s_mu * kAMU * kG * gp.m_p);
  }
  __syncthreads();

  // ---- hydrostatic altitudes (Sec. 4): serial in l
  if (tid == 0) {
    const double rp = s_rp;
    double zl = 0.0;
    z[0] = 0.0;
    for (int l = 0; l < N; ++l) {
      const double r = (gp.gravity_mode == TR_GRAV_CONST) ? rp : rp + zl;
      zl = zl + c[l] * (r * r);
      z[l + 1] = zl;
    }
  }
  __syncthreads();

  // ---- per-layer descriptors: density, brackets, weights, cloud; annulus weights
  const double rp = s_rp;
  const double inv_rs2 = 1.0 / (gp.r_s * gp.r_s);
  LayerDesc* L = buf.layers + (size_t)b * NM;
  for (int l = tid; l < N; l += blockDim.x) {
    LayerDesc d;
    const double rho = P[l] / (kKB * T[l]);
    const bool okp = axis(gp.p_grid, gp.n_p, P[l], gp.oor_mode, &d.ip, &d.tp);
    const bool okt = axis(gp.t_grid, gp.n_t, T[l], gp.oor_mode, &d.it, &d.tt);
    d.zero_mol = (okp && okt) ? 0 : 1;
    d.rho = (float)rho;
    for (int m = 0; m < TR_MAX_MOL; ++m)
      d.w_mol[m] = (m < gp.n_mol && !d.zero_mol) ? (float)(rho * s_X[m]) : 0.f;
    bool okc = true;
    d.itc = 0; d.ttc = 0.f;
    if (gp.n_cia > 0) okc = axis(gp.t_grid_cia, gp.n_t_cia, T[l], gp.oor_mode, &d.itc, &d.ttc);
    d.zero_cia = okc ? 0.f : 1.f;
    for (int q = 0; q < TR_MAX_CIA; ++q)
      d.w_cia[q] = (q < gp.n_cia && okc)
          ? (float)(rho * rho * s_X[gp.cia_a[q]] * s_X[gp.cia_b[q]] * gp.cia_scale[q]) : 0.f;
    double cf = 0.0;
    if (gp.cloud_mode == TR_CLOUD_DISCRETE) {
      const double p_top = exp10(s_lptop);
      const double p_bot = gp.p_cloud_bot > 0.0 ? gp.p_cloud_bot : gp.p_max;
      cf = (P[l] >= p_top && P[l] <= p_bot) ? 1.0 : 0.0;
    } else if (gp.cloud_mode == TR_CLOUD_FRACTIONAL) {
      const double ln_bot = gp.p_cloud_bot > 0.0 ? log(gp.p_cloud_bot) : lmax;
      const double ln_top = s_lptop * 2.302585092994046;   // ln 10
      const double hi = fmin(lnpb[l], ln_bot);
      const double lo = fmax(ln_top, lnpb[l + 1]);
      cf = fmin(fmax((hi - lo) / s_delta, 0.0), 1.0);
    }
    d.k_cloud = (float)(gp.kappa_cloud * cf);
    d.pad0 = d.pad1 = 0.f;
    L[l] = d;
    aj[l] = (float)((z[l + 1] - z[l]) * (2.0 * rp + z[l] + z[l + 1]) * inv_rs2);
  }
  for (int j = N + tid; j < NM; j += blockDim.x) aj[j] = 0.f;
  if (tid < TR_MAX_SPECIES)
    buf.rayc[(size_t)b * TR_MAX_SPECIES + tid] =
        (gp.has_ray && tid < gp.n_species) ? (float)(s_X[tid] * gp.ray_scale[tid]) : 0.f;

  // ---- slant path lengths: DL[j][l] = 2 (s(l+1, j) - s(l, j)), s(k, j) = sqrt(r_k^2 - r_j^2)
  //      with r_k^2 - r_j^2 = (z_k - z_j)(r_k + r_j); rays are paired (t, N-1-t) so every
  //      thread walks about N shells.
  float* dl = buf.dlt + (size_t)b * buf.dlt_stride;
  const int half = (N + 1) / 2;
  for (int t = tid; t < half; t += blockDim.x) {
    for (int pass = 0; pass < 2; ++pass) {
      const int j = pass == 0 ? t : N - 1 - t;
      if (pass == 1 && j == t) break;
      const double zj = z[j];
      double s_lo = 0.0;
      for (int l = j; l < N; ++l) {
        const double s_hi = sqrt((z[l + 1] - zj) * (2.0 * rp + z[l + 1] + zj));
        dl[(size_t)l * (l + 1) / 2 + j] = (float)(2.0 * (s_hi - s_lo));
        s_lo = s_hi;
      }
    }
  }
}

}  // namespace

cudaError_t launch_geometry(const GeomParams& gp, int B, const double* d_theta, int n_theta,
                            const int32_t* d_nlayers, int32_t* d_status, ItemBuffers buf,
                            cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * (5 * (size_t)gp.max_layers + 2);
  k_geometry<<<B, kGeomThreads, smem, s>>>(gp, B, d_theta, n_theta, d_nlayers, d_status, buf);
  return cudaGetLastError();
}

}  // namespace tr
