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

constexpr int kProfileThreads = 160;   // warp 0: item constants, then the altitude recursion
constexpr int kLayerThreads = kProfileThreads - 32;   // warps 1-4: layers
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

struct ItemShared {
  double X[TR_MAX_SPECIES];      // constant mixing ratios (surface values for two-layer gases)
  double Xtop[TR_MAX_MOL];       // two-layer gases: the absorbers above their switches
  int bad;                       // a layer rejected the model (T <= 0, sum X > 1)
  double Y[TR_MAX_CIA];          // CIA pair products X_a X_b 2^e_q
  float Xf[TR_MAX_MOL];          // absorber mixing ratios in FP32
  double rp, cz, xmax, ymax;
  float xmaxf;
  int N, status;
};

// Dynamic shared memory of k_profile for a maximum layer count and table grid: the staged
// grids (values and reciprocal spacings), then per layer the number density (FP64), the
// temperature (FP64 and as a double-float pair), the double-float altitudes, six FP32
// interpolation / cloud values, three brackets and two flag bytes.
__host__ __device__ inline size_t profile_smem_bytes(int NM, int n_p, int n_t, int n_t_cia,
                                                     bool staged, bool zoned) {
  size_t b = staged ? sizeof(double) * 2 * ((size_t)n_p + n_t + n_t_cia) : 0;
  // two-layer gases: every layer's absorber mixing ratios (FP64) and chemistry zone
  if (zoned) b += sizeof(double) * TR_MAX_MOL * (size_t)NM + sizeof(int) * (size_t)NM;
  b += sizeof(double) * 2 * (size_t)NM;                // rho, T
  b += sizeof(float2) * (2 * (size_t)NM + 1);          // T and z as double-float pairs
  b += sizeof(float) * 6 * (size_t)NM;                 // t_P, t_T, t_Tc, u, cloud, k_cloud
  b += sizeof(int) * 3 * (size_t)NM + 2 * (size_t)NM;  // brackets, flags
  return b + 16;
}

// E_2(x) for x > 0 (the Guillot profile): for x <= 1, e^{-x} - x E_1(x) with E_1 from its
// power series -gamma - ln x - sum_k (-x)^k / (k k!); for x > 1 the continued fraction of
// E_2 (Abramowitz & Stegun 5.1.22, n = 2, in its even form with partial numerators
// -k (k + 1) and denominators x + 2 + 2k) evaluated forwards by Lentz's method.
__device__ double expint2(double x) {
  if (x <= 1.0) {
    double term = 1.0, sum = 0.0;
    for (int k = 1; k <= 30; ++k) {
      term *= -x / k;
      sum += term / k;
    }
    const double e1 = -0.57721566490153286061 - log(x) - sum;
    return exp(-x) - x * e1;
  }
  const double tiny = 1e-300;
  double bk = x + 2.0, c = 1.0 / tiny, d = 1.0 / bk, h = d;
  for (int k = 1; k < 500; ++k) {
    const double ak = -(double)k * (k + 1);
    bk += 2.0;
    d = 1.0 / fma(ak, d, bk);
    c = bk + ak / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}

// Guillot (2010) profile with two visible channels at pressure P (Pa): T^4 from the
// parameters g = [T_irr, log10 kappa_irr, log10 kappa_v1, log10 kappa_v2, alpha] for surface
// gravity gs:
//   T^4 = 3/4 T_int^4 (2/3 + tau) + 3/4 T_irr^4 [(1 - alpha) xi(g1) + alpha xi(g2)],
//   xi(g) = 2/3 + 2/(3g) [1 + (g tau/2 - 1) e^{-g tau}] + 2g/3 (1 - tau^2/2) E_2(g tau),
//   tau = kappa_irr P / gs, g_i = kappa_v,i / kappa_irr.
__device__ double guillot_t4(const double* g, double t_int, double P, double gs) {
  const double k_ir = exp10(g[1]);
  const double tau = k_ir * P / gs;
  double xs[2];
  for (int c = 0; c < 2; ++c) {
    const double gm = exp10(g[2 + c]) / k_ir;
    const double gt = gm * tau;
    xs[c] = 2.0 / 3.0 + (2.0 / (3.0 * gm)) * (1.0 + (0.5 * gt - 1.0) * exp(-gt)) +
            (2.0 * gm / 3.0) * (1.0 - 0.5 * tau * tau) * expint2(gt);
  }
  const double ti2 = t_int * t_int, tr2 = g[0] * g[0];
  return 0.75 * ti2 * ti2 * (2.0 / 3.0 + tau) + 0.75 * tr2 * tr2 * ((1.0 - g[4]) * xs[0] + g[4] * xs[1]);
}

// Temperature at log10 pressure x of an item: its N-point profile (nodes tn) or Guillot.
template <bool GUILLOT>
__device__ double item_temperature(const GeomParams& gp, const double* tn, double x, double gs) {
  if (GUILLOT) return sqrt(sqrt(guillot_t4(tn, gp.t_int, exp10(x), gs)));
  if (gp.n_tnodes == 1) return tn[0];
  const int nt = gp.n_tnodes;
  if (x >= gp.tnode_log10p[0]) return tn[0];
  if (x <= gp.tnode_log10p[nt - 1]) return tn[nt - 1];
  int k = 0;
  while (!(gp.tnode_log10p[k] >= x && x >= gp.tnode_log10p[k + 1])) ++k;
  return tn[k] + (tn[k + 1] - tn[k]) * gp.inv_dlog10p[k] * (x - gp.tnode_log10p[k]);
}

// Error-free transformations of FP32 sums (Knuth's TwoSum; Dekker's fast form when |a| >= |b|).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ float2 split_df(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// One CTA per atmosphere, three phases between barriers:
//   1. warp 0 takes the item's constants (mixing ratios, mean molecular weight, radius,
//      validation), lanes in parallel and one short serial sum; meanwhile warps 1-4 take each
//      layer's pressure, temperature, brackets and weights, density and cloud, none of which
//      depends on the chemistry;
//   2. warp 0, lane 0 runs the altitude recursion (the only serial chain) in double-float
//      FP32 arithmetic, which GB300 issues far faster than FP64; meanwhile warps 1-4 write the
//      layer descriptors (which need the chemistry);
//   3. all threads write the altitudes, annulus weights and the path-length kernel's inputs.
template <bool ZONED, bool GUILLOT>
__global__ void __launch_bounds__(kProfileThreads)
k_profile(GeomParams gp, int B, const double* __restrict__ theta, int n_theta,
          const int32_t* __restrict__ nlayers, int32_t* __restrict__ status_out,
          ItemBuffers buf, int staged) {
  extern __shared__ double sm[];
  __shared__ ItemShared w;
  const int b = blockIdx.x;
  if (b >= B) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NM = gp.max_layers;
  const double *pg = gp.p_grid, *ipg = gp.inv_dp, *tg = gp.t_grid, *itg = gp.inv_dt,
               *tcg = gp.t_grid_cia, *itcg = gp.inv_dtc;
  double* q = sm;
  if (staged) {
    double* spg = q; q += gp.n_p;
    double* sipg = q; q += gp.n_p;
    double* stg = q; q += gp.n_t;
    double* sitg = q; q += gp.n_t;
    double* stcg = q; q += gp.n_t_cia;
    double* sitcg = q; q += gp.n_t_cia;
    for (int i = tid - 32; i >= 0 && i < gp.n_p; i += kLayerThreads) {
      spg[i] = gp.p_grid[i];
      sipg[i] = i + 1 < gp.n_p ? gp.inv_dp[i] : 0.0;
    }
    for (int i = tid - 32; i >= 0 && i < gp.n_t; i += kLayerThreads) {
      stg[i] = gp.t_grid[i];
      sitg[i] = i + 1 < gp.n_t ? gp.inv_dt[i] : 0.0;
    }
    for (int i = tid - 32; i >= 0 && i < gp.n_t_cia; i += kLayerThreads) {
      stcg[i] = gp.t_grid_cia[i];
      sitcg[i] = i + 1 < gp.n_t_cia ? gp.inv_dtc[i] : 0.0;
    }
    pg = spg; ipg = sipg; tg = stg; itg = sitg; tcg = stcg; itcg = sitcg;
  }
  constexpr bool zoned = ZONED;
  double* rho_s = q;                                  // [NM]
  double* T_s = rho_s + NM;                           // [NM]
  double* xl_s = T_s + NM;                            // [NM][TR_MAX_MOL] two-layer mixing ratios
  // [NM] T (two-layer gases: T / mu_l) as double-float, the altitude recursion's input
  float2* tdf = reinterpret_cast<float2*>(xl_s + (zoned ? (size_t)NM * TR_MAX_MOL : 0));
  float2* zdf = tdf + NM;                             // [NM + 1] altitudes as double-float
  float* tp_s = reinterpret_cast<float*>(zdf + NM + 1);
  float* tt_s = tp_s + NM;
  float* ttc_s = tt_s + NM;
  float* u_s = ttc_s + NM;                            // exponential T weight
  float* cl_s = u_s + NM;                             // cloud fraction
  float* kc_s = cl_s + NM;                            // cloud opacity
  int* ip_s = reinterpret_cast<int*>(kc_s + NM);
  int* it_s = ip_s + NM;
  int* itc_s = it_s + NM;
  int* zn_s = itc_s + NM;                                   // [NM] chemistry zone (two-layer)
  uint8_t* ok_s = reinterpret_cast<uint8_t*>(zn_s + (zoned ? NM : 0));   // bit 0 P/T in range, bit 1 CIA
  uint8_t* fl_s = ok_s + NM;                                // kLayer* flags
  const double* th = theta + (size_t)b * n_theta;
  const int n_in = nlayers ? nlayers[b] : NM;
  const int NL = (n_in >= 1 && n_in <= NM) ? n_in : 0;     // 0: invalid layer count

  if (warp == 0) {
    // ---- item constants: chemistry (Sec. 4.3) and the model rejection of Sec. 6
    bool bad = NL == 0;
    for (int k = lane; k < n_theta; k += 32) bad |= !isfinite(th[k]);
    if (GUILLOT) {                                     // T_irr >= 0, 0 <= alpha <= 1
      const double* gq = th + gp.n_chem;
      if (lane == 0) bad |= !(gq[0] >= 0.0) || !(gq[4] >= 0.0) || !(gq[4] <= 1.0);
    } else if (lane < gp.n_tnodes) {
      bad |= !(th[gp.n_chem + lane] > 0.0);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane < gp.n_mol) w.X[lane] = exp10(th[lane]);
    if (zoned && lane < gp.n_mol) w.Xtop[lane] = exp10(th[gp.n_mol + lane]);
    __syncwarp();
    double rem = 0.0;
    if (lane == 0) {
      int st = bad ? TR_ERR_INVALID_MODEL : TR_OK;
      double sumx = 0.0, mu = 0.0, xmax = 0.0;
      for (int m = 0; m < gp.n_mol; ++m) {
        const double x = w.X[m];
        sumx += x;
        mu = fma(x, gp.mass[m], mu);
        xmax = fmax(xmax, x);
      }
      if (!zoned && sumx > 1.0) st = TR_ERR_INVALID_MODEL;
      rem = 1.0 - sumx;
      mu = fma(rem, gp.fill_mass, mu);                // + sum_f (fill_f rem) m_f
      if (!zoned && !(mu > 0.0)) st = TR_ERR_INVALID_MODEL;
      if (zoned) {
        // two-layer gases: the layers check their own sums; the recursion takes T_l / mu_l
        // with a reference mu of 1, and the scale of the molecule sums bounds every layer
        mu = 1.0;
        for (int m = 0; m < gp.n_mol; ++m) xmax = fmax(xmax, w.Xtop[m]);
      }
      const double rp = th[gp.n_chem + gp.n_tpar] * kRJup;
      if (!(rp > 0.0)) st = TR_ERR_INVALID_MODEL;
      const double delta = (gp.ln_pmax - gp.ln_pmin) / (double)(NL > 0 ? NL : 1);
      // z_{l+1} - z_l = H_l Delta = k_B T_l Delta / (mu m_u g_l), g_l = G M_p / r_l^2: the step
      // is cz T_l r_l^2 with cz = k_B Delta / (mu m_u G M_p)
      w.cz = st == TR_OK ? (kKB * delta) / (mu * gp.amu_g_mp) : 0.0;
      w.rp = rp;
      w.xmax = (st == TR_OK && xmax > 0.0) ? xmax : 1.0;
      w.N = st == TR_OK ? NL : 0;
      w.status = st;
      buf.items[b].status = st;
      buf.items[b].n_layers = w.N;
      buf.items[b].r_p = st == TR_OK ? rp : 0.0;
      buf.items[b].rp2_rs2 = st == TR_OK ? rp * rp * gp.inv_rs2 : 0.0;
      // the temperature profile's value at p_max (the emission model's surface temperature)
      buf.items[b].t_surf =
          st == TR_OK ? item_temperature<GUILLOT>(gp, th + gp.n_chem, gp.ln_pmax * 0.43429448190325182765,
                                         gp.gm_p / (rp * rp))
                      : 0.0;
      if (status_out) status_out[b] = st;
    }
    rem = __shfl_sync(0xffffffffu, rem, 0);
    const int f = gp.n_mol + lane;                    // fill gases share the remainder
    if (f < gp.n_species) w.X[f] = gp.fill[f] * rem;
    __syncwarp();
    if (lane < gp.n_cia) {
      if (zoned) {
        // a bound of every layer's pair product: the larger of an absorber's two values, a
        // fill gas's whole fraction
        const int a = gp.cia_a[lane], c = gp.cia_b[lane];
        const double ba = a < gp.n_mol ? fmax(w.X[a], w.Xtop[a]) : gp.fill[a];
        const double bc = c < gp.n_mol ? fmax(w.X[c], w.Xtop[c]) : gp.fill[c];
        w.Y[lane] = ba * bc * gp.cia_scale[lane];
      } else {
        w.Y[lane] = w.X[gp.cia_a[lane]] * w.X[gp.cia_b[lane]] * gp.cia_scale[lane];
      }
    }
    if (lane < TR_MAX_MOL) w.Xf[lane] = lane < gp.n_mol ? (float)w.X[lane] : 0.f;
    __syncwarp();
    if (lane == 0) {
      // scale of the pair-summed CIA cross-sections (no FP32 underflow of the sums)
      double ymax = 0.0;
      for (int c = 0; c < gp.n_cia; ++c) ymax = fmax(ymax, w.Y[c]);
      w.ymax = (w.status == TR_OK && ymax > 0.0) ? ymax : 1.0;
      w.xmaxf = (float)w.xmax;
    }
  } else {
    if (tid == 32) w.bad = 0;
    asm volatile("bar.sync 1, %0;" :: "n"(kLayerThreads) : "memory");   // staged grids, w.bad
  }
  if (warp > 0 && NL > 0) {
    // ---- per layer: pressure grid (Sec. 4.1), temperature (Sec. 4.2), interpolation
    //      brackets and weights (Sec. 5), density and cloud (Sec. 4.4)
    const double* tn = th + gp.n_chem;
    const double lptop = th[gp.n_chem + gp.n_tpar + 1];
    const double rp_l = th[gp.n_chem + gp.n_tpar] * kRJup;
    const double gs = gp.gm_p / (rp_l * rp_l);        // surface gravity of the Guillot profile
    const double dln = (gp.ln_pmin - gp.ln_pmax) / (double)NL;    // ln p step (negative)
    const double inv_delta = (double)NL / (gp.ln_pmax - gp.ln_pmin);
    double p_top = 0.0, ln_top = 0.0;
    if (gp.cloud_mode == TR_CLOUD_DISCRETE) p_top = exp10(lptop);
    else if (gp.cloud_mode == TR_CLOUD_FRACTIONAL) ln_top = lptop * 2.302585092994046;   // ln 10
    const double inv_ln10 = 0.43429448190325182765;
    for (int l = tid - 32; l < NL; l += kLayerThreads) {
      // boundaries ln p_l, ln p_{l+1} linear in ln p; P_l = exp((ln p_l + ln p_{l+1}) / 2)
      const double lb0 = fma((double)l, dln, gp.ln_pmax);
      const double lb1 = fma((double)(l + 1), dln, gp.ln_pmax);
      const double lnp = 0.5 * (lb0 + lb1);
      const double p = exp(lnp);
      double t;
      if (GUILLOT) {
        const double t4 = guillot_t4(tn, gp.t_int, p, gs);
        const bool good = t4 > 0.0 && isfinite(t4);
        if (!good) atomicExch(&w.bad, 1);
        t = good ? sqrt(sqrt(t4)) : 1.0;
      } else if (gp.n_tnodes == 1) {
        t = tn[0];
      } else {
        const double x = lnp * inv_ln10;
        const int nt = gp.n_tnodes;
        if (x >= gp.tnode_log10p[0]) t = tn[0];
        else if (x <= gp.tnode_log10p[nt - 1]) t = tn[nt - 1];
        else {
          int k = 0;
          while (!(gp.tnode_log10p[k] >= x && x >= gp.tnode_log10p[k + 1])) ++k;
          const double slope = (tn[k + 1] - tn[k]) * gp.inv_dlog10p[k];
          t = tn[k] + slope * (x - gp.tnode_log10p[k]);
        }
      }
      int ip, it, itc = 0;
      double wp, wt, wtc = 0.0;
      const bool okp = axis(pg, ipg, gp.n_p, p, gp.oor_mode, &ip, &wp);
      const bool okt = axis(tg, itg, gp.n_t, t, gp.oor_mode, &it, &wt);
      bool okc = true;
      if (gp.n_cia > 0) okc = axis(tcg, itcg, gp.n_t_cia, t, gp.oor_mode, &itc, &wtc);
      const bool okm = okp && okt;
      ip_s[l] = ip; it_s[l] = it; itc_s[l] = itc;
      tp_s[l] = (float)wp; tt_s[l] = (float)wt; ttc_s[l] = (float)wtc;
      ok_s[l] = (uint8_t)((okm ? 1 : 0) | (okc ? 2 : 0));
      fl_s[l] = (uint8_t)((okm ? 0 : kLayerMolZero) |
                          ((t <= tg[0] || t >= tg[gp.n_t - 1]) ? kLayerTClamp : 0) |
                          (okc ? 0 : kLayerCiaZero) |
                          ((gp.n_cia > 0 && (t <= tcg[0] || t >= tcg[gp.n_t_cia - 1]))
                               ? kLayerTcClamp : 0));
      if (gp.interp_mode == TR_INTERP_EXP) {
        // exponential scheme in T (Sec. 5): sigma(T) = s1^(1-u) s2^u with the weight
        // u = (1/T1 - 1/T) / (1/T1 - 1/T2) = t T2 / T (t the linear weight of the clamped T)
        const double T1 = tg[it], T2 = tg[it + 1];
        const double Tc = T1 + wt * (T2 - T1);
        u_s[l] = (float)((wt * T2) / Tc);
      }
      rho_s[l] = (p * gp.inv_kb) / t;
      T_s[l] = t;
      if (zoned) {
        // two-layer gases: X_surf below the switch, X_top above, the ln P-weighted mean in the
        // layer that straddles it; the layer's mean molecular weight and chemistry zone (the sum
        // of the absorbers' states: 0 below, 1 straddling, 2 above)
        double sumx = 0.0, mu = 0.0;
        int zone = 0;
        for (int m = 0; m < gp.n_mol; ++m) {
          const double lsw = th[2 * gp.n_mol + m] * 2.302585092994046;
          double fb;
          if (lsw <= lb1) { fb = 1.0; }
          else if (lsw >= lb0) { fb = 0.0; zone += 2; }
          else { fb = (lb0 - lsw) * inv_delta; zone += 1; }
          const double x = fb * exp10(th[m]) + (1.0 - fb) * exp10(th[gp.n_mol + m]);
          xl_s[(size_t)l * TR_MAX_MOL + m] = x;
          sumx += x;
          mu = fma(x, gp.mass[m], mu);
        }
        mu = fma(1.0 - sumx, gp.fill_mass, mu);
        if (sumx > 1.0 || !(mu > 0.0)) atomicExch(&w.bad, 1);
        zn_s[l] = zone;
        tdf[l] = split_df(t / (mu > 0.0 ? mu : 1.0));
      } else {
        tdf[l] = split_df(t);
      }
      double cf = 0.0;
      if (gp.cloud_mode == TR_CLOUD_DISCRETE) {
        cf = (p >= p_top && p <= gp.p_cbot) ? 1.0 : 0.0;
      } else if (gp.cloud_mode == TR_CLOUD_FRACTIONAL) {
        const double hi = fmin(lb0, gp.ln_cbot);
        const double lo = fmax(ln_top, lb1);
        cf = fmin(fmax((hi - lo) * inv_delta, 0.0), 1.0);
      }
      cl_s[l] = (float)cf;
      kc_s[l] = (float)(gp.kappa_cloud * cf);
    }
  }
  __syncthreads();
  if (tid == 0 && w.bad && w.status == TR_OK) {       // a layer rejected the model (Sec. 6)
    w.status = TR_ERR_INVALID_MODEL;
    w.N = 0;
    buf.items[b].status = TR_ERR_INVALID_MODEL;
    buf.items[b].n_layers = 0;
    buf.items[b].r_p = 0.0;
    buf.items[b].rp2_rs2 = 0.0;
    buf.items[b].t_surf = 0.0;
    if (status_out) status_out[b] = TR_ERR_INVALID_MODEL;
  }
  __syncthreads();
  const int N = w.N;
  float* aj = buf.aj + (size_t)b * buf.npad;
  if (w.status != TR_OK) {
    for (int j = tid; j < buf.npad; j += kProfileThreads) aj[j] = 0.f;
    return;
  }

  if (warp == 0) {
    // the altitude recursion's inputs for k_altitude, left in the altitude rows it rewrites:
    // T_l (two-layer gases: T_l / mu_l) as a double-float pair in zf[l].xy and the step
    // coefficient c (constant gravity: cz R_p^2) in zf[0].zw
    float4* zf = buf.zf + (size_t)b * (NM + 1);
    const bool cg = gp.gravity_mode == TR_GRAV_CONST;
    const float2 c = split_df(cg ? w.cz * w.rp * w.rp : w.cz);
    for (int l = lane; l < N; l += 32) {
      const float2 tl = tdf[l];
      zf[l] = make_float4(tl.x, tl.y, l == 0 ? c.x : 0.f, l == 0 ? c.y : 0.f);
    }
  } else {
    const int lt = tid - 32;
    // ---- per-layer descriptors: density-weighted mixing ratios (FP32 products of the FP32
    //      density and mixing ratios), corner coefficients; CIA weights in FP64 (rho^2 X_a X_b
    //      2^e_q can lie outside FP32's range before the product)
    LayerDesc* L = buf.layers + (size_t)b * NM;
    for (int l = lt; l < N; l += kLayerThreads) {
      LayerDesc d;
      const double rho = rho_s[l];
      const float rhof = (float)rho;
      const bool okm = ok_s[l] & 1, okc = ok_s[l] & 2;
      d.ip = ip_s[l];
      d.it = it_s[l];
      d.itc = itc_s[l];
      d.zone = zoned ? zn_s[l] : 0;
      // this layer's mixing ratios of every species (two-layer gases) and CIA pair products
      double xs[ZONED ? TR_MAX_SPECIES : 1];
      double ypl[ZONED ? TR_MAX_CIA : 1];
      if constexpr (ZONED) {
        double sx = 0.0;
        for (int m = 0; m < gp.n_mol; ++m) { xs[m] = xl_s[(size_t)l * TR_MAX_MOL + m]; sx += xs[m]; }
        for (int f2 = gp.n_mol; f2 < gp.n_species; ++f2) xs[f2] = gp.fill[f2] * (1.0 - sx);
        for (int c = 0; c < gp.n_cia; ++c)
          ypl[c] = xs[gp.cia_a[c]] * xs[gp.cia_b[c]] * gp.cia_scale[c];
      }
      d.rho = rhof;
      d.tp = tp_s[l];
      d.tt = tt_s[l];
      // bilinear corner weights (P_i, T_j), (P_i, T_j+1), (P_i+1, T_j), (P_i+1, T_j+1) in FP32
      const float tpf = d.tp, ttf = d.tt;
      float cw[4];
      corner_weights(tpf, ttf, cw);
#pragma unroll
      for (int m = 0; m < TR_MAX_MOL; ++m) {
        float xm = w.Xf[m];
        if constexpr (ZONED) xm = m < gp.n_mol ? (float)xs[m] : 0.f;
        d.w_mol[m] = okm ? rhof * xm : 0.f;
      }
      d.pad_s = 0;
      d.flags = fl_s[l];
      d.pad_c = 0;
      d.pad_f = 0.f;
      d.ttc = ttc_s[l];
      const double rho2 = rho * rho;
#pragma unroll
      for (int c = 0; c < TR_MAX_CIA; ++c) {
        double yc = w.Y[c];
        if constexpr (ZONED) yc = ypl[c];
        d.w_cia[c] = (c < gp.n_cia && okc) ? (float)(rho2 * yc) : 0.f;
      }
      d.cloud = cl_s[l];
      d.k_cloud = kc_s[l];
      L[l] = d;
      buf.tl[(size_t)b * NM + l] = T_s[l];
      // the same opacity for cross-sections pre-summed over molecules and CIA pairs
      const float wx = (okm && gp.n_mol > 0) ? rhof * w.xmaxf : 0.f;
      const float wy = (okc && gp.n_cia > 0) ? (float)(rho2 * w.ymax) : 0.f;
      float4* opl = buf.op + ((size_t)b * NM + l) * 2;
      if (gp.interp_mode == TR_INTERP_EXP)
        // exponential scheme: the P-row weights, the exponential T weight u and the linear
        // T weight t for values that fall back to the linear scheme
        opl[0] = make_float4(wx * (1.f - tpf), wx * tpf, u_s[l], ttf);
      else
        opl[0] = make_float4(wx * cw[0], wx * cw[1], wx * cw[2], wx * cw[3]);
      opl[1] = make_float4(wy * (1.f - d.ttc), wy * d.ttc, d.rho, d.k_cloud);
      if constexpr (ZONED) if (l == 0 || zn_s[l - 1] != zn_s[l]) {
        // the first layer of a zone writes the zone's weights of the molecule and pair sums
        // and its Rayleigh coefficients
        float* ox = buf.opx + ((size_t)b * kMaxZones + d.zone) * kOpxStride;
        for (int k = 0; k < kOpxStride; ++k) {
          float x = 0.f;
          if (k < gp.n_mol) x = (float)(xs[k] / w.xmax);
          const int c = k - TR_MAX_MOL;
          if (c >= 0 && c < gp.n_cia) x = (float)(ypl[c] / w.ymax);
          ox[k] = x;
        }
        float* rz = buf.rayc + ((size_t)b * kMaxZones + d.zone) * TR_MAX_SPECIES;
        for (int sp = 0; sp < TR_MAX_SPECIES; ++sp)
          rz[sp] = (gp.has_ray && sp < gp.n_species) ? (float)(xs[sp] * gp.ray_scale[sp]) : 0.f;
      }
    }
    // per-item weights of the molecule- and pair-summed cross-sections, Rayleigh coefficients
    if (zoned) {
      // written by each zone's first layer above
    } else if (lt < kOpxStride) {
      float x = 0.f;
      if (lt < gp.n_mol) x = (float)(w.X[lt] / w.xmax);
      const int c = lt - TR_MAX_MOL;
      if (c >= 0 && c < gp.n_cia) x = (float)(w.Y[c] / w.ymax);
      buf.opx[(size_t)b * kMaxZones * kOpxStride + lt] = x;
    } else if (lt - kOpxStride < TR_MAX_SPECIES) {
      const int sp = lt - kOpxStride;
      buf.rayc[(size_t)b * kMaxZones * TR_MAX_SPECIES + sp] =
          (gp.has_ray && sp < gp.n_species) ? (float)(w.X[sp] * gp.ray_scale[sp]) : 0.f;
    }
  }
  for (int j = N + tid; j < buf.npad; j += kProfileThreads) aj[j] = 0.f;
}

// Hydrostatic altitudes (Sec. 4), one warp per atmosphere: z_{l+1} = z_l + cz T_l (R_p + z_l)^2
// (constant gravity: + cz R_p^2 T_l), serial in l, run by lane 0 in double-float arithmetic
// (each value an unevaluated FP32 sum hi + lo, products split exactly by FMA) from the inputs
// k_profile leaves in the item's altitude rows; then the warp writes the altitudes and what the
// path-length kernel needs of them in FP32: z_k as double-float, the row numerator
// 2 (r_{k+1}^2 - r_k^2) = 2 (z_{k+1} - z_k)(2 R_p + z_{k+1} + z_k) and 2 R_p + z_k, and the
// annulus weights A_j / R_s^2 = (z_{j+1} - z_j)(2 R_p + z_{j+1} + z_j) / R_s^2.  Only the
// contraction (annulus weights) and the path lengths read these, so the kernel runs beside
// the opacity kernel in the batched forward.
constexpr int kAltWarps = 4;
__global__ void __launch_bounds__(32 * kAltWarps)
k_altitude(int B, int max_layers, int const_gravity, double inv_rs2, ItemBuffers buf) {
  extern __shared__ float2 alt_sm[];                // per warp: T pairs, then altitude pairs
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * kAltWarps + warp;
  if (b >= B) return;
  const ItemGeom ig = buf.items[b];
  const int N = ig.n_layers;
  if (ig.status != TR_OK || N <= 0) return;        // k_profile zeroed its annulus weights
  float2* tdf = alt_sm + (size_t)warp * 2 * (max_layers + 1);
  float2* zdf = tdf + (max_layers + 1);
  float4* zf = buf.zf + (size_t)b * (max_layers + 1);
  for (int l = lane; l < N; l += 32) {
    const float4 v = zf[l];
    tdf[l] = make_float2(v.x, v.y);
  }
  const float4 v0 = zf[0];
  __syncwarp();
  if (lane == 0) {
    // the next layer's T (and step coefficient) is loaded before this layer's altitude is
    // stored, so the loads stay off the dependent chain
    const float2 rp = split_df(ig.r_p);
    const float2 c = make_float2(v0.z, v0.w);
    float zh = 0.f, zl = 0.f;
    zdf[0] = make_float2(0.f, 0.f);
    const bool cg = const_gravity != 0;
    auto coef = [&](int l, float& ah, float& al) {      // c T_l as a double-float pair
      const float2 tt = tdf[l < N ? l : N - 1];
      ah = c.x * tt.x;
      al = fmaf(c.x, tt.x, -ah) + (c.x * tt.y + c.y * tt.x);
    };
    float ah, al;
    coef(0, ah, al);
    for (int l = 0; l < N; ++l) {
      float nah, nal;
      coef(l + 1, nah, nal);
      float ih, il;
      if (cg) {                                       // step c T_l
        ih = ah; il = al;
      } else {                                        // step a (R_p + z_l)^2, a = cz T_l
        float sh, se;
        two_sum(rp.x, zh, sh, se);
        const float sl = se + (rp.y + zl);
        const float qh = sh * sh;
        const float ql = fmaf(sh, sh, -qh) + 2.f * sh * sl;
        ih = ah * qh;
        il = fmaf(ah, qh, -ih) + (ah * ql + al * qh);
      }
      float nh, ne;
      two_sum(zh, ih, nh, ne);
      fast_two_sum(nh, ne + (zl + il), zh, zl);
      zdf[l + 1] = make_float2(zh, zl);
      ah = nah; al = nal;
    }
  }
  __syncwarp();
  double* z = buf.z + (size_t)b * (max_layers + 1);
  float* aj = buf.aj + (size_t)b * buf.npad;
  const double rp2 = 2.0 * ig.r_p;
  for (int k = lane; k <= N; k += 32) {
    const float2 zk2 = zdf[k];
    const double zk = (double)zk2.x + (double)zk2.y;
    z[k] = zk;
    float num = 0.f;
    if (k < N) {
      const float2 zu2 = zdf[k + 1];
      const double zu = (double)zu2.x + (double)zu2.y;
      const double dr2 = (zu - zk) * (rp2 + zu + zk);
      num = (float)(2.0 * dr2);
      aj[k] = (float)(dr2 * inv_rs2);
    }
    zf[k] = make_float4(zk2.x, zk2.y, num, (float)(rp2 + zk));
  }
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
  const size_t smem = profile_smem_bytes(gp.max_layers, gp.n_p, gp.n_t, gp.n_t_cia, staged,
                                         gp.gas_mode == TR_GAS_TWOLAYER);
  // instantiated per mode, so the default (N-point, constant mixing ratios) carries none of
  // the other modes' code
  const bool zoned = gp.gas_mode == TR_GAS_TWOLAYER, guillot = gp.t_profile == TR_TPROF_GUILLOT;
  auto kern = zoned ? (guillot ? k_profile<true, true> : k_profile<true, false>)
                    : (guillot ? k_profile<false, true> : k_profile<false, false>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<B, kProfileThreads, smem, s>>>(gp, B, d_theta, n_theta, d_nlayers, d_status, buf,
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

cudaError_t launch_altitude(const GeomParams& gp, int B, ItemBuffers buf, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const size_t smem = sizeof(float2) * 2 * (size_t)(gp.max_layers + 1) * kAltWarps;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_altitude, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_altitude<<<(B + kAltWarps - 1) / kAltWarps, 32 * kAltWarps, smem, s>>>(
      B, gp.max_layers, gp.gravity_mode == TR_GRAV_CONST ? 1 : 0, gp.inv_rs2, buf);
  return cudaGetLastError();
}

cudaError_t launch_geometry(const GeomParams& gp, int B, const double* d_theta, int n_theta,
                            const int32_t* d_nlayers, int32_t* d_status, ItemBuffers buf,
                            cudaStream_t s) {
  cudaError_t e = launch_profile(gp, B, d_theta, n_theta, d_nlayers, d_status, buf, s);
  if (e == cudaSuccess) e = launch_altitude(gp, B, buf, s);
  if (e != cudaSuccess) return e;
  return launch_pathlen(gp, B, buf, s);
}

}  // namespace tr
