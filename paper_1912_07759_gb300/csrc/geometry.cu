// geometry.cu -- FP64 atmosphere set-up on the device: pressure grid (Sec. 4.1), temperature
// profile (Sec. 4.2), free chemistry and mean molecular weight (Sec. 4.3), hydrostatic
// altitudes (Sec. 4, equation for z_l), number density, interpolation brackets and weights
// (Sec. 5, linear scheme and out-of-range rules), cloud deck (Sec. 4.4, eq. clouds), annulus
// weights and slant path lengths.
//
// Two kernels, so that the FP64 work (GB300 issues only a few FP64 operations per clock per
// SM) spreads over many SMs even for a single atmosphere:
//   k_profile   one CTA per atmosphere: threads work over layers; one thread runs the altitude
//               recursion, the only serial step, while the others write the layer
//               descriptors;
//   k_pathlen   one warp per (atmosphere, 1 or 4 consecutive shells): lanes over rays, the
//               root of the shell below carried in registers (one root per path length),
//               rows of the dense layer-major matrix written coalesced.  Path lengths are
//               taken in a conjugate form that needs FP64 only for the altitude differences,
//               which double-float arithmetic in FP32 supplies (k_profile writes the
//               double-float altitudes).
#include "tr_internal.h"

namespace tr {
namespace {

constexpr int kProfileThreads = 128;
constexpr int kPathWarps = 4;
constexpr int kStageGrid = 512;   // axis grids up to this many points in all are staged in smem

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
// The bracket equals the clamped one (x clamped to the grid) in every case.
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

// Out-of-line FP64 special functions and division: k_profile runs once per atmosphere on a
// cold instruction cache, where instruction fetch dominates its time; each routine's code then
// exists once instead of at every call site.  Results are those of the inline forms.
__device__ __noinline__ double exp_ol(double x) { return exp(x); }
__device__ __noinline__ double log_ol(double x) { return log(x); }
__device__ __noinline__ double exp10_ol(double x) { return exp10(x); }
__device__ __noinline__ double div_ol(double a, double b) { return a / b; }

struct ItemShared {
  double X[TR_MAX_SPECIES];
  double slope[TR_MAX_TNODES];   // dT / dlog10 P of each node segment
  double rp, mu, delta, lptop, cz, inv_kb, lmax, lmin, p_top, p_bot, ln_bot, ln_top;
  double xmax, ymax;             // largest absorber mixing ratio and CIA pair product
  int N, status;
};

// Dynamic shared memory of k_profile for a maximum layer count and table grid.
__host__ __device__ inline size_t profile_smem_bytes(int NM, int n_p, int n_t, int n_t_cia,
                                                     bool staged) {
  size_t b = sizeof(double) * (7 * (size_t)NM + 2);
  if (staged) b += sizeof(double) * 2 * ((size_t)n_p + n_t + n_t_cia);
  b += sizeof(int) * 3 * (size_t)NM + (size_t)NM;     // brackets, flags
  return b + 16;
}

// One CTA per atmosphere: threads work over layers.  The serial altitude recursion runs on one
// thread of warp 1 while the other warps write the layer descriptors.  Grids are read from
// shared memory when they are small (they nearly always are), and each layer's brackets are
// found once.
__global__ void __launch_bounds__(kProfileThreads)
k_profile(GeomParams gp, int B, const double* __restrict__ theta, int n_theta,
          const int32_t* __restrict__ nlayers, int32_t* __restrict__ status_out,
          ItemBuffers buf, int staged) {
  extern __shared__ double sm[];
  __shared__ ItemShared w;
  const int b = blockIdx.x;
  if (b >= B) return;
  const int tid = threadIdx.x;
  const int NM = gp.max_layers;
  double* P = sm;                                   // [NM]
  double* T = P + NM;                               // [NM]
  double* lnpb = T + NM;                            // [NM + 1] ln of boundary pressures
  double* r = lnpb + NM + 1;                        // [NM + 1] radii of the boundaries
  double* tp = r + NM + 1;                          // [NM] bracket weights along P, T, T_cia
  double* tt = tp + NM;
  double* ttc = tt + NM;
  double* gnext = ttc + NM;
  const double *pg = gp.p_grid, *ipg = gp.inv_dp, *tg = gp.t_grid, *itg = gp.inv_dt,
               *tcg = gp.t_grid_cia, *itcg = gp.inv_dtc;
  if (staged) {
    double* q = gnext;
    double* spg = q; q += gp.n_p;
    double* sipg = q; q += gp.n_p;
    double* stg = q; q += gp.n_t;
    double* sitg = q; q += gp.n_t;
    double* stcg = q; q += gp.n_t_cia;
    double* sitcg = q; q += gp.n_t_cia;
    for (int i = tid; i < gp.n_p; i += kProfileThreads) {
      spg[i] = gp.p_grid[i];
      sipg[i] = i + 1 < gp.n_p ? gp.inv_dp[i] : 0.0;
    }
    for (int i = tid; i < gp.n_t; i += kProfileThreads) {
      stg[i] = gp.t_grid[i];
      sitg[i] = i + 1 < gp.n_t ? gp.inv_dt[i] : 0.0;
    }
    for (int i = tid; i < gp.n_t_cia; i += kProfileThreads) {
      stcg[i] = gp.t_grid_cia[i];
      sitcg[i] = i + 1 < gp.n_t_cia ? gp.inv_dtc[i] : 0.0;
    }
    pg = spg; ipg = sipg; tg = stg; itg = sitg; tcg = stcg; itcg = sitcg;
    gnext = q;
  }
  int* ipl = reinterpret_cast<int*>(gnext);         // [NM] brackets
  int* itl = ipl + NM;
  int* itcl = itl + NM;
  uint8_t* okl = reinterpret_cast<uint8_t*>(itcl + NM);   // [NM] bit 0 P/T ok, bit 1 CIA ok
  double* z = buf.z + (size_t)b * (NM + 1);         // [NM + 1] altitudes (global: k_pathlen)
  const double* th = theta + (size_t)b * n_theta;

  // ---- chemistry (Sec. 4.3) and temperature-node slopes (Sec. 4.2)
  if (tid < gp.n_mol) w.X[tid] = exp10_ol(th[tid]);
  if (tid + 1 < gp.n_tnodes) {
    const double* tn = th + gp.n_mol;
    w.slope[tid] = div_ol(tn[tid + 1] - tn[tid], gp.tnode_log10p[tid + 1] - gp.tnode_log10p[tid]);
  }
  __syncthreads();
  // ---- validation (model rejection of Sec. 6) and per-item constants
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
    // scales of the molecule- and pair-summed cross-sections (no FP32 underflow of the sums)
    double xmax = 0.0, ymax = 0.0;
    for (int m = 0; m < gp.n_mol; ++m) xmax = fmax(xmax, w.X[m]);
    for (int q = 0; q < gp.n_cia; ++q)
      ymax = fmax(ymax, w.X[gp.cia_a[q]] * w.X[gp.cia_b[q]] * gp.cia_scale[q]);
    w.xmax = (st == TR_OK && xmax > 0.0) ? xmax : 1.0;
    w.ymax = (st == TR_OK && ymax > 0.0) ? ymax : 1.0;
    w.mu = mu;
    w.N = (st == TR_OK) ? N : 0;
    w.status = st;
    w.lmax = log_ol(gp.p_max);
    w.lmin = log_ol(gp.p_min);
    w.delta = div_ol(w.lmax - w.lmin, (double)(st == TR_OK ? N : 1));
    // z_{l+1} - z_l = H_l Delta = k_B T_l Delta / (mu m_u g_l), g_l = G M_p / r_l^2:
    // the step is cz T_l r_l^2 with cz = k_B Delta / (mu m_u G M_p)
    w.cz = (st == TR_OK) ? div_ol(kKB * w.delta, mu * kAMU * kG * gp.m_p) : 0.0;
    w.inv_kb = div_ol(1.0, kKB);
    if (gp.cloud_mode == TR_CLOUD_DISCRETE) {
      w.p_top = exp10_ol(w.lptop);
      w.p_bot = gp.p_cloud_bot > 0.0 ? gp.p_cloud_bot : gp.p_max;
    } else if (gp.cloud_mode == TR_CLOUD_FRACTIONAL) {
      w.ln_bot = gp.p_cloud_bot > 0.0 ? log_ol(gp.p_cloud_bot) : w.lmax;
      w.ln_top = w.lptop * 2.302585092994046;   // ln 10
    }
    buf.items[b].status = st;
    buf.items[b].n_layers = w.N;
    buf.items[b].r_p = (st == TR_OK) ? w.rp : 0.0;
    buf.items[b].rp2_rs2 = (st == TR_OK) ? div_ol(w.rp * w.rp, gp.r_s * gp.r_s) : 0.0;
    if (status_out) status_out[b] = st;
  }
  __syncthreads();
  const int N = w.N;
  float* aj = buf.aj + (size_t)b * buf.npad;
  if (w.status != TR_OK) {
    for (int j = tid; j < buf.npad; j += kProfileThreads) aj[j] = 0.f;
    return;
  }

  // ---- pressure grid (Sec. 4.1): ln p of the N + 1 boundaries, linear in ln p
  for (int k = tid; k <= N; k += kProfileThreads)
    lnpb[k] = w.lmax + div_ol((w.lmin - w.lmax) * k, (double)N);
  __syncthreads();
  // ---- layer pressure P_l = exp((ln p_l + ln p_{l+1}) / 2), temperature (Sec. 4.2) and the
  //      interpolation brackets (Sec. 5)
  const double inv_ln10 = 0.43429448190325182765;
  for (int l = tid; l < N; l += kProfileThreads) {
    const double lnp = 0.5 * (lnpb[l] + lnpb[l + 1]);
    const double p = exp_ol(lnp);
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
    P[l] = p;
    T[l] = t;
    int ip, it, itc = 0;
    double wp, wt, wtc = 0.0;
    const bool okp = axis(pg, ipg, gp.n_p, p, gp.oor_mode, &ip, &wp);
    const bool okt = axis(tg, itg, gp.n_t, t, gp.oor_mode, &it, &wt);
    bool okc = true;
    if (gp.n_cia > 0) okc = axis(tcg, itcg, gp.n_t_cia, t, gp.oor_mode, &itc, &wtc);
    ipl[l] = ip; itl[l] = it; itcl[l] = itc;
    tp[l] = wp; tt[l] = wt; ttc[l] = wtc;
    okl[l] = (uint8_t)((okp && okt ? 1 : 0) | (okc ? 2 : 0));
  }
  __syncthreads();

  // ---- warp 1, lane 0: hydrostatic altitudes (Sec. 4), serial in l, on the boundary radii:
  //      r_{l+1} = r_l + a_l r_l^2 with a_l = cz T_l (constant gravity: r_l^2 -> R_p^2);
  //      meanwhile warps 0, 2, 3 write the per-layer descriptors (they do not need the radii)
  const int warp = tid >> 5;
  if (warp == 1) {
    if (tid == 32) {
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
  } else {
  // ---- per-layer descriptors: density, corner coefficients, cloud
  LayerDesc* L = buf.layers + (size_t)b * NM;
  const int td = tid < 32 ? tid : tid - 32;
  for (int l = td; l < N; l += kProfileThreads - 32) {
    LayerDesc d;
    const double rho = div_ol(P[l] * w.inv_kb, T[l]);
    const bool okm = okl[l] & 1, okc = okl[l] & 2;
    d.ip = ipl[l];
    d.it = itl[l];
    d.itc = itcl[l];
    d.pad_h = 0;
    d.rho = (float)rho;
    d.tp = (float)tp[l];
    d.tt = (float)tt[l];
    // bilinear corner weights (P_i, T_j), (P_i, T_j+1), (P_i+1, T_j), (P_i+1, T_j+1) in FP32
    const float tpf = d.tp, ttf = d.tt;
    const float cw[4] = {(1.f - tpf) * (1.f - ttf), (1.f - tpf) * ttf, tpf * (1.f - ttf), tpf * ttf};
    for (int m = 0; m < TR_MAX_MOL; ++m) {
      const float wm = (m < gp.n_mol && okm) ? (float)(rho * w.X[m]) : 0.f;
      d.w_mol[m] = wm;
      for (int k = 0; k < 4; ++k) d.cm[m][k] = wm * cw[k];
    }
    d.pad_s = 0;
    const double Tl = T[l];
    d.flags = (uint8_t)((okm ? 0 : kLayerMolZero) |
                        ((Tl <= tg[0] || Tl >= tg[gp.n_t - 1]) ? kLayerTClamp : 0) |
                        (okc ? 0 : kLayerCiaZero) |
                        ((gp.n_cia > 0 && (Tl <= tcg[0] || Tl >= tcg[gp.n_t_cia - 1]))
                             ? kLayerTcClamp : 0));
    d.pad_c = 0;
    d.pad_f = 0.f;
    buf.tl[(size_t)b * NM + l] = Tl;
    d.ttc = (float)ttc[l];
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
      cf = (P[l] >= w.p_top && P[l] <= w.p_bot) ? 1.0 : 0.0;
    } else if (gp.cloud_mode == TR_CLOUD_FRACTIONAL) {
      const double hi = fmin(lnpb[l], w.ln_bot);
      const double lo = fmax(w.ln_top, lnpb[l + 1]);
      cf = fmin(fmax(div_ol(hi - lo, w.delta), 0.0), 1.0);
    }
    d.cloud = (float)cf;
    d.k_cloud = (float)(gp.kappa_cloud * cf);
    L[l] = d;
    // the same opacity for cross-sections pre-summed over molecules and CIA pairs
    const float wx = (okm && gp.n_mol > 0) ? (float)(rho * w.xmax) : 0.f;
    const float wy = (okc && gp.n_cia > 0) ? (float)(rho2 * w.ymax) : 0.f;
    float4* opl = buf.op + ((size_t)b * NM + l) * 2;
    if (gp.interp_mode == TR_INTERP_EXP) {
      // exponential scheme in T (Sec. 5): sigma(T) = s1^(1-u) s2^u with the weight
      // u = (1/T1 - 1/T) / (1/T1 - 1/T2) = t T2 / T (t the linear weight of the clamped T);
      // the opacity kernels take the P-row weights, u, and t for values that fall back to
      // the linear scheme
      const int it = itl[l];
      const double T1 = tg[it], T2 = tg[it + 1];
      const double Tc = T1 + tt[l] * (T2 - T1);
      const float u = (float)(tt[l] * T2 / Tc);
      opl[0] = make_float4(wx * (1.f - tpf), wx * tpf, u, ttf);
    } else {
      opl[0] = make_float4(wx * cw[0], wx * cw[1], wx * cw[2], wx * cw[3]);
    }
    opl[1] = make_float4(wy * (1.f - d.ttc), wy * d.ttc, d.rho, d.k_cloud);
  }
  }
  __syncthreads();
  // altitudes, and what the path-length kernel needs of them in FP32: z_k as double-float,
  // the row numerator 2 (r_{k+1}^2 - r_k^2) = 2 (z_{k+1} - z_k)(2 R_p + z_{k+1} + z_k) and
  // 2 R_p + z_k
  float4* zf = buf.zf + (size_t)b * (NM + 1);
  for (int k = tid; k <= N; k += kProfileThreads) {
    const double zk = r[k] - w.rp;
    z[k] = zk;
    const float hi = (float)zk;
    float num = 0.f;
    if (k < N) {
      const double zu = r[k + 1] - w.rp;
      num = (float)(2.0 * ((zu - zk) * (2.0 * w.rp + zu + zk)));
    }
    zf[k] = make_float4(hi, (float)(zk - (double)hi), num, (float)(2.0 * w.rp + zk));
  }

  // A_j / R_s^2 = (r_{j+1} - r_j)(r_{j+1} + r_j) / R_s^2 = (z_{j+1} - z_j)(r_{j+1} + r_j) / R_s^2
  const double inv_rs2 = div_ol(1.0, gp.r_s * gp.r_s);
  for (int l = tid; l < N; l += kProfileThreads)
    aj[l] = (float)(((r[l + 1] - w.rp) - (r[l] - w.rp)) * (r[l + 1] + r[l]) * inv_rs2);
  for (int j = N + tid; j < buf.npad; j += kProfileThreads) aj[j] = 0.f;
  if (tid < kOpxStride) {
    float x = 0.f;
    if (tid < gp.n_mol) x = (float)div_ol(w.X[tid], w.xmax);
    const int q = tid - TR_MAX_MOL;
    if (q >= 0 && q < gp.n_cia)
      x = (float)div_ol(w.X[gp.cia_a[q]] * w.X[gp.cia_b[q]] * gp.cia_scale[q], w.ymax);
    buf.opx[(size_t)b * kOpxStride + tid] = x;
  }
  if (tid < TR_MAX_SPECIES)
    buf.rayc[(size_t)b * TR_MAX_SPECIES + tid] =
        (gp.has_ray && tid < gp.n_species) ? (float)(w.X[tid] * gp.ray_scale[tid]) : 0.f;
}

// (ah + al) - (bh + bl) to FP32 working precision: the leading difference is taken exactly as
// s + e (Knuth's TwoSum), then the low parts are added in.
__device__ __forceinline__ float diff_df(float ah, float al, float bh, float bl) {
  const float s = __fsub_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
  return __fadd_rn(s, __fadd_rn(e, __fsub_rn(al, bl)));
}

// Slant path lengths (reading R1): DL[j][l] = 2 (s(l+1, j) - s(l, j)) for l >= j with
// s(k, j) = sqrt(r_k^2 - r_j^2) and r_k^2 - r_j^2 = (z_k - z_j)(2 R_p + z_k + z_j).  Written in
// the conjugate form
//   DL[j][l] = 2 (r_{l+1}^2 - r_l^2) / (s(l+1, j) + s(l, j)),
// a quotient of positive terms, so the difference of two near-equal roots never has to be
// formed.  The numerator comes from k_profile (one FP64 product per row); each root needs
// z_k - z_j to working precision, taken from the double-float altitudes, and the rest is FP32:
// the kernel issues no FP64 instruction (GB300 runs FP32 at many times its FP64 rate).
// Written dense and layer-major: row l holds rays j = 0..npad-1 (zero for j > l and j >= N);
// and packed: row l holds rays 0 .. pad8(l+1)-1 (zero for j > l).
// A warp walks rows_per_warp consecutive rows with lanes over rays, carrying s(l, j) from the
// row below; rows are written coalesced.
__global__ void __launch_bounds__(32 * kPathWarps)
k_pathlen(int max_layers, int rows_per_warp, ItemBuffers buf) {
  const int b = blockIdx.y;
  const int l0 = (blockIdx.x * kPathWarps + (threadIdx.x >> 5)) * rows_per_warp;
  const int lane = threadIdx.x & 31;
  const int N = buf.items[b].n_layers;
  if (l0 >= N) return;
  const float4* zf = buf.zf + (size_t)b * (max_layers + 1);
  float* dl = buf.dlt + (size_t)b * max_layers * buf.npad;
  float* dlp = buf.dlp + (size_t)b * dlp_offset(max_layers);
  const int l1 = min(l0 + rows_per_warp, N);
  const float4 f0 = zf[l0];
  for (int j0 = 0; j0 < buf.npad; j0 += 32) {
    const int j = j0 + lane;
    const bool ray = j < N && j <= l1 - 1;
    const float4 fj = ray ? zf[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    // s(l0, j) for rays below row l0 (s(j, j) = 0)
    float s_lo = 0.f;
    if (ray && j < l0) s_lo = sqrtf(diff_df(f0.x, f0.y, fj.x, fj.y) * (fj.w + f0.x));
    for (int l = l0; l < l1; ++l) {
      const float4 fu = zf[l + 1];
      const float num = zf[l].z;
      float v = 0.f;
      if (ray && j <= l) {
        const float s_hi = sqrtf(diff_df(fu.x, fu.y, fj.x, fj.y) * (fj.w + fu.x));
        const float den = s_hi + s_lo;
        v = den > 0.f ? num / den : 0.f;
        s_lo = s_hi;
      }
      if (j < buf.npad) dl[(size_t)l * buf.npad + j] = v;
      if (j < pad8(l + 1)) dlp[dlp_offset(l) + j] = v;
    }
  }
}

}  // namespace

cudaError_t launch_profile(const GeomParams& gp, int B, const double* d_theta, int n_theta,
                           const int32_t* d_nlayers, int32_t* d_status, ItemBuffers buf,
                           cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int staged = (gp.n_p + gp.n_t + gp.n_t_cia) <= kStageGrid;
  const size_t smem = profile_smem_bytes(gp.max_layers, gp.n_p, gp.n_t, gp.n_t_cia, staged);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_profile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_profile<<<B, kProfileThreads, smem, s>>>(gp, B, d_theta, n_theta, d_nlayers, d_status, buf,
                                             staged);
  return cudaGetLastError();
}

cudaError_t launch_pathlen(const GeomParams& gp, int B, ItemBuffers buf, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  // few atmospheres: one shell row per warp, spread over many SMs; many: 4 rows per warp
  const int rows_per_warp = B < 16 ? 1 : 4;
  const int rows_per_cta = kPathWarps * rows_per_warp;
  dim3 grid((gp.max_layers + rows_per_cta - 1) / rows_per_cta, B);
  k_pathlen<<<grid, 32 * kPathWarps, 0, s>>>(gp.max_layers, rows_per_warp, buf);
  return cudaGetLastError();
}

cudaError_t launch_geometry(const GeomParams& gp, int B, const double* d_theta, int n_theta,
                            const int32_t* d_nlayers, int32_t* d_status, ItemBuffers buf,
                            cudaStream_t s) {
  cudaError_t e = launch_profile(gp, B, d_theta, n_theta, d_nlayers, d_status, buf, s);
  if (e != cudaSuccess) return e;
  return launch_pathlen(gp, B, buf, s);
}

}  // namespace tr
