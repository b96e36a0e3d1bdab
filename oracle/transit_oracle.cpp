/*
 * transit_oracle.cpp -- plain, slow FP64 CPU oracle of the transmission forward model of
 * TauREx 3 (Al-Refaie et al., arXiv:1912.07759).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by the test suite, by the smoke check and by
 * the CPU-baseline leg of the benchmark; the product path (the CUDA library) never includes,
 * links or calls it, and it includes nothing from the product.
 *
 * It computes the discrete model step by step, in the order the paper states it:
 *   pressure grid (Sec. 4.1, eq. for P_l)  ->  temperature profile (Sec. 4.2, N-point profile)
 *   ->  free chemistry with fill gases and mean molecular weight (Sec. 4.3)
 *   ->  hydrostatic altitude grid (Sec. 4, equation for z_l, Delta z_l, H_l)
 *   ->  slant path lengths of each ray through each shell
 *   ->  linear-in-T (or the exponential scheme of Sec. 5, sigma = a e^{-b/T}) and linear-in-P
 *       interpolation of the cross-sections (Sec. 5, eqs. sigma(T), sigma(P), exp-interp)
 *       with the out-of-range rules of Sec. 5
 *   ->  weighting by mixing ratio and number density, CIA (eq. cia_opt_dpth), Rayleigh and the
 *       grey cloud deck (eq. clouds), all fused into one opacity K[layer, wn] (Sec. 8.1)
 *   ->  optical depth tau[ray, wn] = sum over shells of path length * K (eqs. tot_opt_dpth,
 *       opt_dpth) -> transit depth (eqs. for Delta_lambda and a_lambda)
 *   ->  FluxBinner weights and weighted mean (Sec. 4.5, eqs. w_ij, F_j) -> chi^2.
 * and, for the emission model of Sec. 4 (plane-parallel: the surface term plus the layers'
 * emission attenuated along cos(theta), integrated in cos(theta) by Gauss-Legendre), the
 * planet-star flux ratio from the same opacity K (readings E1-E4 at orc_emission).
 *
 * Readings where the paper is silent or garbled (each is also stated where it is used):
 *   R1 ray j has impact parameter r_j = R_p + z_j; shell l = [r_l, r_{l+1}) carries K_l.
 *   R2 g_l = G M_p / (R_p + z_l)^2 (or G M_p / R_p^2 in constant-gravity mode).
 *   R3 the altitude recursion is carried one step past the last layer, so z has N+1 entries
 *      and shell l has thickness z_{l+1} - z_l = H_l * Delta.
 *   R4 fill gases take explicit fractions of the remaining volume 1 - sum X_m.
 *   R5 sigma is interpolated linearly in P and in T (not log P, not log sigma); bracket i is
 *      the largest index with grid[i] <= x.  With the exponential scheme T is interpolated as
 *      a e^{-b/T} through the two bracketing values (P stays linear; CIA stays linear in T,
 *      the paper states the scheme for the absorbers' cross-sections); where one of the two
 *      values is not positive the linear value is used.
 *   R6 out-of-range: clamp to the grid edge (default), or the paper's rule (below the grid
 *      minimum -> zero, above the maximum -> the edge value).
 *   R7 grey cloud: opacity kappa [1/m] (not multiplied by rho) in layers with
 *      P_top <= P <= P_bot; discrete (layer centre inside the deck) or fractional (fraction of
 *      the layer's ln P extent inside the deck).
 *   R8 Rayleigh cross-sections are inputs per species, weighted like absorbers.
 *   R10 annulus weights A_j = r_{j+1}^2 - r_j^2.
 *   G1-G3 Guillot2010 temperature profile (Sec. 4.2 names it and its parameters T_irr,
 *      kappa_irr, kappa_v1, kappa_v2, alpha without stating it): Guillot (2010) radiative
 *      equilibrium with two visible channels (Line et al. 2013),
 *        T^4 = 3/4 T_int^4 (2/3 + tau) + 3/4 T_irr^4 [(1 - alpha) xi(g1) + alpha xi(g2)],
 *        xi(g) = 2/3 + 2/(3g) [1 + (g tau/2 - 1) e^{-g tau}] + 2g/3 (1 - tau^2/2) E_2(g tau),
 *      g_i = kappa_v,i / kappa_irr, tau = kappa_irr P / g_s with the surface gravity
 *      g_s = G M_p / R_p^2 (G1: the profile is a function of pressure, set before altitudes
 *      exist), T_int a fixed internal temperature (G2: not among the fitted parameters),
 *      opacities in m^2/kg (G3).
 *   L1-L2 two-layer gas profile (Sec. 4.3, named with surface and top mixing ratios): X_m is
 *      X_surf below the switch pressure P_sw,m and X_top above it (L1); a layer straddling
 *      the switch takes the ln P-average over the layer, f X_surf + (1 - f) X_top with f the
 *      fraction of its ln P extent below the switch (L2).  Fill gases share each layer's
 *      remainder, so mu, H and the densities of every species vary by layer.
 *
 * Gradients: every model step is templated on the scalar type.  Instantiated with a
 * forward-mode dual number it yields the exact derivatives of this same discrete function
 * with respect to the parameter vector theta (no finite differences).
 *
 * Build: g++ -O2 -std=c++17 -fPIC -shared [-fopenmp]  (no -ffast-math).
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// Physical constants (SI).  The paper works in SI (Sec. 3) but lists only molecular masses
// (mass table, Sec. 8.1) and R_J; the others are CODATA-2018 / IAU nominal values.
constexpr double G_NEWTON = 6.67430e-11;
constexpr double K_BOLTZ = 1.380649e-23;
constexpr double AMU = 1.66053906660e-27;
constexpr double R_JUPITER = 6.9911e7;   // retrieved-parameters table caption, Sec. 8.2
constexpr double H_PLANCK = 6.62607015e-34;
constexpr double C_LIGHT = 299792458.0;

// ------------------------------------------------------------------------------------------
// forward-mode dual number with a fixed maximum number of tangent directions
// ------------------------------------------------------------------------------------------
constexpr int NDIR = 16;

struct Dual {
  double v;
  double d[NDIR];
  Dual() : v(0.0) { std::memset(d, 0, sizeof(d)); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof(d)); }   // NOLINT: implicit constant
};

inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
inline Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int k = 0; k < NDIR; ++k) r.d[k] = -a.d[k];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  const double inv = 1.0 / (b.v * b.v);
  for (int k = 0; k < NDIR; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) * inv;
  return r;
}
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual sqrt(const Dual& a) {
  Dual r(std::sqrt(a.v));
  const double s = (r.v > 0.0) ? 0.5 / r.v : 0.0;
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] * s;
  return r;
}
inline Dual exp(const Dual& a) {
  Dual r(std::exp(a.v));
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] * r.v;
  return r;
}
inline Dual expm1(const Dual& a) {
  Dual r(std::expm1(a.v));
  const double e = std::exp(a.v);
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] * e;
  return r;
}
inline Dual log(const Dual& a) {
  Dual r(std::log(a.v));
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] / a.v;
  return r;
}

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::sqrt; using std::exp; using std::expm1; using std::log;

template <class S> S pow10s(const S& x) { return exp(x * std::log(10.0)); }

// Exponential integral E_1(x), x > 0: its power series -gamma - ln x + sum_k (-1)^(k+1) x^k /
// (k k!) for x <= 2, else the continued fraction of Abramowitz & Stegun 5.1.22 (n = 1),
//   E_1(x) = e^{-x} / (x + 1/(1 + 1/(x + 2/(1 + 2/(x + 3/(1 + ...)))))),
// evaluated from a deep fixed tail backwards.
double expint_e1(double x) {
  if (x <= 2.0) {
    double sum = 0.0, term = 1.0;
    for (int k = 1; k < 60; ++k) {
      term *= -x / k;                       // (-x)^k / k!
      sum -= term / k;                      // (-1)^(k+1) x^k / (k k!)
    }
    return -0.57721566490153286061 - std::log(x) + sum;
  }
  double t = 0.0;                           // tail of the fraction
  for (int k = 400; k >= 1; --k) {
    t = k / (1.0 + k / (x + t));            // k/(1 + k/(x + ...))
  }
  return std::exp(-x) / (x + t);
}
// E_2(x) = e^{-x} - x E_1(x) (A&S 5.1.14), E_2(0) = 1; d E_2 / dx = -E_1(x).
double expint_e2(double x) { return x > 0.0 ? std::exp(-x) - x * expint_e1(x) : 1.0; }
inline Dual expint_e2(const Dual& a) {
  Dual r(expint_e2(a.v));
  const double d = -expint_e1(a.v);
  for (int k = 0; k < NDIR; ++k) r.d[k] = a.d[k] * d;
  return r;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// C interface structs (ctypes mirrors them in oracle/oracle.py)
// ------------------------------------------------------------------------------------------
extern "C" {

typedef struct {
  int n_mol, n_p, n_t, n_wn;
  const double* p_grid;      // [n_p] Pa ascending
  const double* t_grid;      // [n_t] K ascending
  const double* wn_grid;     // [n_wn] cm^-1 ascending
  const float* sigma;        // [n_mol][n_p][n_t][n_wn] m^2
  int n_cia, n_t_cia;
  const double* t_grid_cia;  // [n_t_cia] K ascending
  const int* cia_pair;       // [n_cia][2] species indices
  const double* cia;         // [n_cia][n_t_cia][n_wn] m^5
  int n_species;             // absorbers first, then fill gases
  const double* mass_amu;    // [n_species]
  const double* rayleigh;    // [n_species][n_wn] m^2 or NULL
  int oor_mode;              // 0 clamp, 1 paper rule (below minimum -> 0)
  int interp_mode;           // 0 linear in T (default), 1 exponential in T (Sec. 5)
} orc_tables;

typedef struct {
  int n_layers;
  double p_max, p_min;             // Pa; boundary 0 is the bottom (p_max)
  int n_tnodes;
  const double* tnode_log10p;      // [n_tnodes] descending
  const double* tnode_t;           // [n_tnodes] K
  const double* log10_x;           // [n_mol]
  const double* fill_frac;         // [n_species - n_mol]
  double r_p, m_p, r_s;            // m, kg, m
  double p_cloud_top, p_cloud_bot, kappa_cloud;
  int gravity_mode;                // 0 altitude-dependent, 1 constant
  int cloud_mode;                  // 0 none, 1 discrete, 2 fractional
  int t_profile;                   // 0 N-point (nodes above), 1 Guillot2010
  const double* guillot;           // [5] T_irr (K), kappa_irr, kappa_v1, kappa_v2 (m^2/kg), alpha
  double t_int;                    // K, Guillot internal temperature
  int gas_mode;                    // 0 constant mixing ratios, 1 two-layer
  const double* log10_x_top;       // [n_mol] two-layer: mixing ratios above the switch
  const double* log10_p_switch;    // [n_mol] two-layer: switch pressures (log10 Pa)
} orc_atm;

typedef struct {
  int n_bin;
  const double* lam_centre_um;     // [n_bin]
  const double* lam_width_um;      // [n_bin]
} orc_bins;

typedef struct {
  int n_mol, n_tnodes;
  const double* tnode_log10p;
  const double* fill_frac;
  double p_max, p_min, m_p, r_s, p_cloud_bot, kappa_cloud;
  int gravity_mode, cloud_mode;
  int t_profile, gas_mode;         // as in orc_atm; they set the layout of theta
  double t_int;
} orc_batch;

}  // extern "C"

namespace {

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_INVALID_MODEL = 2 };

// Parameters of one model in the scalar type S (those that theta can change are S).
template <class S>
struct Params {
  int n_layers;
  double p_max, p_min;
  int n_tnodes;
  std::vector<double> tnode_log10p;
  std::vector<S> tnode_t;
  std::vector<S> log10_x;
  std::vector<double> fill_frac;
  S r_p;
  double m_p, r_s;
  int cloud_on;
  S log10_p_cloud_top;
  double p_cloud_bot, kappa_cloud;
  int gravity_mode, cloud_mode;
  int t_profile = 0;
  std::vector<S> guillot;          // T_irr, kappa_irr, kappa_v1, kappa_v2, alpha
  double t_int = 0.0;
  int gas_mode = 0;
  std::vector<S> log10_x_top, log10_p_switch;
};

// Everything the layer-by-layer set-up produces.
template <class S>
struct Profile {
  int N = 0;
  std::vector<double> pb;     // [N+1] boundary pressures, pb[0] = p_max (bottom)
  std::vector<double> P;      // [N] layer pressures
  double delta = 0.0;         // ln(pb[l] / pb[l+1])
  std::vector<S> T;           // [N]
  std::vector<S> X;           // [N][n_species] mixing ratios of every layer
  std::vector<S> mu;          // [N] mean molecular weight (amu)
  std::vector<S> g, H, rho;   // [N]
  std::vector<S> z;           // [N+1]
  std::vector<S> cloud;       // [N] cloud fraction of each layer
  std::vector<S> DL;          // [N*N] path length of ray j in shell l (row j)
  std::vector<S> A;           // [N] annulus weights r_{j+1}^2 - r_j^2
  S r_p;
};

// Largest index i in [0, n-2] with grid[i] <= x (0 when x is below grid[0]).  Plain scan.
int bracket(const double* grid, int n, double x) {
  int i = 0;
  for (int k = 0; k < n - 1; ++k)
    if (grid[k] <= x) i = k;
  return i;
}

// Linear interpolation set-up along one table axis, Sec. 5 (linear scheme) with the
// out-of-range rules of Sec. 5 (R6).  Returns false when the paper rule gives zero.
template <class S>
bool axis_weights(const double* grid, int n, const S& x, int oor_mode, int* i_out, S* t_out) {
  const double xv = val(x);
  if (oor_mode == 1 && xv < grid[0]) return false;          // both bounds below range -> 0
  S xc = x;
  if (xv <= grid[0]) xc = S(grid[0]);                       // clamp (constant: no derivative)
  if (xv >= grid[n - 1]) xc = S(grid[n - 1]);
  const int i = bracket(grid, n, val(xc));
  *i_out = i;
  *t_out = (xc - S(grid[i])) / S(grid[i + 1] - grid[i]);
  return true;
}

// Temperature interpolation of one cross-section between its values s1 at T1 and s2 at T2
// (tt = (T - T1) / (T2 - T1), T already clamped to the bracket).  Linear scheme (Sec. 5):
// s1 + (s2 - s1) tt.  Exponential scheme (Sec. 5, eq. exp-interp): sigma(T) = a e^{-b/T} with
// b = (1/T2 - 1/T1)^{-1} ln(s1/s2) and a = s1 e^{b/T1}, written out as the paper states it.
// Reading (the paper gives no rule): where s1 or s2 is not positive the logarithm does not
// exist and the linear value is used.
template <class S>
S interp_t(double s1, double s2, const S& tt, double T1, double T2, int mode) {
  if (mode != 1 || !(s1 > 0.0) || !(s2 > 0.0)) return S(s1) + (S(s2) - S(s1)) * tt;
  const double b = std::log(s1 / s2) / (1.0 / T2 - 1.0 / T1);
  const double a = s1 * std::exp(b / T1);
  const S T = S(T1) + tt * S(T2 - T1);
  return S(a) * exp(S(-b) / T);
}

// Guillot (2010) radiative-equilibrium profile with two visible channels (G1-G3): T^4 at
// pressure P for surface gravity gs.
template <class S>
S guillot_t4(const Params<S>& pr, double P, const S& gs) {
  const S tirr = pr.guillot[0], k_ir = pr.guillot[1], alpha = pr.guillot[4];
  const S tau = k_ir * S(P) / gs;
  auto xi = [&](const S& g) {
    const S gt = g * tau;
    return S(2.0 / 3.0) + S(2.0 / 3.0) / g * (S(1.0) + (gt * S(0.5) - S(1.0)) * exp(-gt)) +
           S(2.0 / 3.0) * g * (S(1.0) - tau * tau * S(0.5)) * expint_e2(gt);
  };
  const S g1 = pr.guillot[2] / k_ir, g2 = pr.guillot[3] / k_ir;
  const double tint4 = pr.t_int * pr.t_int * pr.t_int * pr.t_int;
  const S tirr4 = tirr * tirr * tirr * tirr;
  return S(0.75 * tint4) * (S(2.0 / 3.0) + tau) +
         S(0.75) * tirr4 * ((S(1.0) - alpha) * xi(g1) + alpha * xi(g2));
}

template <class S>
int build_profile(const orc_tables& tb, const Params<S>& pr, Profile<S>& out) {
  const int N = pr.n_layers;
  if (N < 1) return ORC_ERR_INVALID_MODEL;
  if (!(pr.p_max > pr.p_min) || !(pr.p_min > 0.0)) return ORC_ERR_INVALID_MODEL;
  out.N = N;

  // -- a1: N+1 boundaries log-uniform from p_max to p_min; layer pressure P_l = p_l sqrt(p_{l+1}/p_l)
  out.pb.resize(N + 1);
  const double lmax = std::log(pr.p_max), lmin = std::log(pr.p_min);
  for (int k = 0; k <= N; ++k) out.pb[k] = std::exp(lmax + (lmin - lmax) * k / N);
  out.P.resize(N);
  for (int l = 0; l < N; ++l) out.P[l] = out.pb[l] * std::sqrt(out.pb[l + 1] / out.pb[l]);
  out.delta = (lmax - lmin) / N;

  // -- a2: temperature.  One node: isothermal.  Several: linear in log P between nodes
  //    (N-point profile), clamped to the end nodes outside their range.
  out.T.assign(N, S(0.0));
  if (pr.t_profile == 1) {
    // Guillot2010 (G1-G3): the model is rejected for T_irr < 0, alpha outside [0, 1],
    // non-positive opacities or a non-positive T^4
    if (!(pr.m_p > 0.0) || !(val(pr.r_p) > 0.0)) return ORC_ERR_INVALID_MODEL;
    for (int k = 0; k < 5; ++k)
      if (!std::isfinite(val(pr.guillot[k]))) return ORC_ERR_INVALID_MODEL;
    if (!(val(pr.guillot[0]) >= 0.0) || !(val(pr.guillot[4]) >= 0.0) ||
        !(val(pr.guillot[4]) <= 1.0) || !(pr.t_int >= 0.0))
      return ORC_ERR_INVALID_MODEL;
    for (int k = 1; k < 4; ++k)
      if (!(val(pr.guillot[k]) > 0.0)) return ORC_ERR_INVALID_MODEL;
    const S gs = S(G_NEWTON * pr.m_p) / (pr.r_p * pr.r_p);
    for (int l = 0; l < N; ++l) {
      const S t4 = guillot_t4(pr, out.P[l], gs);
      if (!(val(t4) > 0.0) || !std::isfinite(val(t4))) return ORC_ERR_INVALID_MODEL;
      out.T[l] = sqrt(sqrt(t4));
    }
  }
  if (pr.t_profile != 1 && pr.n_tnodes < 1) return ORC_ERR_INVALID_MODEL;
  // a non-positive (or non-finite) node temperature is a non-physical model (Sec. 6, model
  // rejection), even where no layer centre falls close enough to the node to go negative
  for (int k = 0; pr.t_profile != 1 && k < pr.n_tnodes; ++k)
    if (!(val(pr.tnode_t[k]) > 0.0) || !std::isfinite(val(pr.tnode_t[k])))
      return ORC_ERR_INVALID_MODEL;
  for (int k = 0; pr.t_profile != 1 && k + 1 < pr.n_tnodes; ++k)
    if (!(pr.tnode_log10p[k] > pr.tnode_log10p[k + 1])) return ORC_ERR_INVALID_MODEL;
  for (int l = 0; pr.t_profile != 1 && l < N; ++l) {
    if (pr.n_tnodes == 1) { out.T[l] = pr.tnode_t[0]; continue; }
    const double x = std::log10(out.P[l]);
    const int nt = pr.n_tnodes;
    if (x >= pr.tnode_log10p[0]) { out.T[l] = pr.tnode_t[0]; continue; }
    if (x <= pr.tnode_log10p[nt - 1]) { out.T[l] = pr.tnode_t[nt - 1]; continue; }
    int k = 0;
    while (!(pr.tnode_log10p[k] >= x && x >= pr.tnode_log10p[k + 1])) ++k;
    const double f = (x - pr.tnode_log10p[k]) / (pr.tnode_log10p[k + 1] - pr.tnode_log10p[k]);
    out.T[l] = pr.tnode_t[k] + (pr.tnode_t[k + 1] - pr.tnode_t[k]) * S(f);
  }
  for (int l = 0; l < N; ++l)
    if (!(val(out.T[l]) > 0.0) || !std::isfinite(val(out.T[l]))) return ORC_ERR_INVALID_MODEL;

  // -- a3: mixing ratios of every layer -- constant, or two-layer (L1-L2); fill gases share
  //    each layer's remainder (R4); mean molecular weight of each layer
  const int n_fill = tb.n_species - tb.n_mol, ns = tb.n_species;
  out.X.assign((size_t)N * ns, S(0.0));
  out.mu.assign(N, S(0.0));
  std::vector<S> x_surf(tb.n_mol), x_top(tb.n_mol);
  for (int m = 0; m < tb.n_mol; ++m) {
    if (!std::isfinite(val(pr.log10_x[m]))) return ORC_ERR_INVALID_MODEL;
    x_surf[m] = pow10s(pr.log10_x[m]);
    if (pr.gas_mode == 1) {
      if (!std::isfinite(val(pr.log10_x_top[m])) || !std::isfinite(val(pr.log10_p_switch[m])))
        return ORC_ERR_INVALID_MODEL;
      x_top[m] = pow10s(pr.log10_x_top[m]);
    }
  }
  for (int l = 0; l < N; ++l) {
    S* Xl = &out.X[(size_t)l * ns];
    S sum_x(0.0);
    for (int m = 0; m < tb.n_mol; ++m) {
      if (pr.gas_mode == 1) {
        // fraction of [ln p_{l+1}, ln p_l] below the switch (pressures above P_sw)
        const S ln_sw = pr.log10_p_switch[m] * S(std::log(10.0));
        const double lo_layer = std::log(out.pb[l + 1]);
        const S lo = (val(ln_sw) > lo_layer) ? ln_sw : S(lo_layer);
        S f = (S(std::log(out.pb[l])) - lo) / S(out.delta);
        if (val(f) < 0.0) f = S(0.0);
        if (val(f) > 1.0) f = S(1.0);
        Xl[m] = f * x_surf[m] + (S(1.0) - f) * x_top[m];
      } else {
        Xl[m] = x_surf[m];
      }
      sum_x += Xl[m];
    }
    if (val(sum_x) > 1.0) return ORC_ERR_INVALID_MODEL;
    const S rem = S(1.0) - sum_x;
    for (int f = 0; f < n_fill; ++f) Xl[tb.n_mol + f] = S(pr.fill_frac[f]) * rem;
    for (int s2 = 0; s2 < ns; ++s2) out.mu[l] += Xl[s2] * S(tb.mass_amu[s2]);
    if (!(val(out.mu[l]) > 0.0)) return ORC_ERR_INVALID_MODEL;
  }

  // -- a4: hydrostatic altitudes (Sec. 4): z_0 = 0, z_{l+1} = z_l + H_l * Delta (R3),
  //    H_l = k_B T_l / (mu_l m_u g_l), g_l from R2; number density rho_l = P_l / (k_B T_l)
  if (!(val(pr.r_p) > 0.0) || !(pr.m_p > 0.0) || !(pr.r_s > 0.0)) return ORC_ERR_INVALID_MODEL;
  out.r_p = pr.r_p;
  out.g.assign(N, S(0.0)); out.H.assign(N, S(0.0)); out.rho.assign(N, S(0.0));
  out.z.assign(N + 1, S(0.0));
  for (int l = 0; l < N; ++l) {
    const S r = pr.r_p + out.z[l];
    if (pr.gravity_mode == 1) out.g[l] = S(G_NEWTON * pr.m_p) / (pr.r_p * pr.r_p);
    else out.g[l] = S(G_NEWTON * pr.m_p) / (r * r);
    out.H[l] = S(K_BOLTZ) * out.T[l] / (out.mu[l] * S(AMU) * out.g[l]);
    out.z[l + 1] = out.z[l] + out.H[l] * S(out.delta);
    out.rho[l] = S(out.P[l]) / (S(K_BOLTZ) * out.T[l]);
  }

  // -- grey cloud deck (eq. clouds, R7)
  out.cloud.assign(N, S(0.0));
  if (pr.cloud_on && pr.cloud_mode != 0) {
    const double p_bot = (pr.p_cloud_bot > 0.0) ? pr.p_cloud_bot : pr.p_max;
    for (int l = 0; l < N; ++l) {
      if (pr.cloud_mode == 1) {
        const double p_top = std::pow(10.0, val(pr.log10_p_cloud_top));
        out.cloud[l] = S((out.P[l] >= p_top && out.P[l] <= p_bot) ? 1.0 : 0.0);
      } else {
        // fraction of [ln p_{l+1}, ln p_l] lying inside [ln P_top, ln P_bot]
        const S ln_top = pr.log10_p_cloud_top * S(std::log(10.0));
        const double hi = std::min(std::log(out.pb[l]), std::log(p_bot));
        const double lo_layer = std::log(out.pb[l + 1]);
        S lo = (val(ln_top) > lo_layer) ? ln_top : S(lo_layer);
        S f = (S(hi) - lo) / S(out.delta);
        if (val(f) < 0.0) f = S(0.0);
        if (val(f) > 1.0) f = S(1.0);
        out.cloud[l] = f;
      }
    }
  }

  // -- a5: slant path length of ray j (impact parameter r_j) through shell l >= j (R1):
  //    DL[j][l] = 2 ( sqrt(r_{l+1}^2 - r_j^2) - sqrt(r_l^2 - r_j^2) ),  r_k = R_p + z_k.
  //    r_k^2 - r_j^2 is evaluated as (z_k - z_j)(r_k + r_j), the same quantity written
  //    without subtracting two large squares.
  out.DL.assign((size_t)N * N, S(0.0));
  for (int j = 0; j < N; ++j) {
    const S rj = pr.r_p + out.z[j];
    for (int l = j; l < N; ++l) {
      const S r_hi = pr.r_p + out.z[l + 1];
      const S r_lo = pr.r_p + out.z[l];
      const S s_hi = sqrt((out.z[l + 1] - out.z[j]) * (r_hi + rj));
      const S s_lo = (l == j) ? S(0.0) : sqrt((out.z[l] - out.z[j]) * (r_lo + rj));
      out.DL[(size_t)j * N + l] = S(2.0) * (s_hi - s_lo);
    }
  }
  // -- annulus weights (R10): A_j = r_{j+1}^2 - r_j^2 = (z_{j+1} - z_j)(r_{j+1} + r_j)
  out.A.assign(N, S(0.0));
  for (int j = 0; j < N; ++j)
    out.A[j] = (out.z[j + 1] - out.z[j]) * (S(2.0) * pr.r_p + out.z[j + 1] + out.z[j]);
  return ORC_OK;
}

// a6 + a7: opacity K[l][i] for the native indices i in [i0, i1).
template <class S>
void opacity(const orc_tables& tb, const Params<S>& pr, const Profile<S>& pf, int i0, int i1,
             std::vector<S>& K) {
  const int N = pf.N, W = i1 - i0;
  K.assign((size_t)N * W, S(0.0));
  for (int l = 0; l < N; ++l) {
    S* Kl = &K[(size_t)l * W];
    // molecular absorption: rho * X_m * sigma_m(P_l, T_l), sigma bilinear in (P, T)
    for (int m = 0; m < tb.n_mol; ++m) {
      int ip = 0, it = 0; S tp, tt;
      if (!axis_weights(tb.p_grid, tb.n_p, S(pf.P[l]), tb.oor_mode, &ip, &tp)) continue;
      if (!axis_weights(tb.t_grid, tb.n_t, pf.T[l], tb.oor_mode, &it, &tt)) continue;
      const S w = pf.rho[l] * pf.X[(size_t)l * tb.n_species + m];
      const size_t slab = (size_t)tb.n_t * tb.n_wn;
      const float* s00 = tb.sigma + ((size_t)m * tb.n_p + ip) * slab + (size_t)it * tb.n_wn;
      const float* s01 = s00 + tb.n_wn;           // T_{it+1}
      const float* s10 = s00 + slab;              // P_{ip+1}
      const float* s11 = s10 + tb.n_wn;
      const double T1 = tb.t_grid[it], T2 = tb.t_grid[it + 1];
      for (int i = i0; i < i1; ++i) {
        // sigma(T) at both bracketing pressures, then sigma(P) between them
        const S at_p1 = interp_t(s00[i], s01[i], tt, T1, T2, tb.interp_mode);
        const S at_p2 = interp_t(s10[i], s11[i], tt, T1, T2, tb.interp_mode);
        const S sig = at_p1 + (at_p2 - at_p1) * tp;
        Kl[i - i0] += w * sig;
      }
    }
    // Rayleigh scattering: rho * X_s * sigma_R,s
    if (tb.rayleigh) {
      for (int s = 0; s < tb.n_species; ++s) {
        const S w = pf.rho[l] * pf.X[(size_t)l * tb.n_species + s];
        const double* sr = tb.rayleigh + (size_t)s * tb.n_wn;
        for (int i = i0; i < i1; ++i) Kl[i - i0] += w * S(sr[i]);
      }
    }
    // collision-induced absorption: rho^2 * X_a * X_b * sigma_cia(T_l)
    for (int q = 0; q < tb.n_cia; ++q) {
      int it = 0; S tt;
      if (!axis_weights(tb.t_grid_cia, tb.n_t_cia, pf.T[l], tb.oor_mode, &it, &tt)) continue;
      const S* Xl = &pf.X[(size_t)l * tb.n_species];
      const S w = pf.rho[l] * pf.rho[l] * Xl[tb.cia_pair[2 * q]] * Xl[tb.cia_pair[2 * q + 1]];
      const double* c0 = tb.cia + ((size_t)q * tb.n_t_cia + it) * tb.n_wn;
      const double* c1 = c0 + tb.n_wn;
      for (int i = i0; i < i1; ++i) Kl[i - i0] += w * (S(c0[i]) + (S(c1[i]) - S(c0[i])) * tt);
    }
    // grey cloud: kappa * cloud fraction
    if (val(pf.cloud[l]) != 0.0) {
      const S kc = S(pr.kappa_cloud) * pf.cloud[l];
      for (int i = i0; i < i1; ++i) Kl[i - i0] += kc;
    }
  }
}

// a8 + a9: tau[j][i] = sum_{l>=j} DL[j][l] K[l][i];  D_i = (R_p^2 + sum_j A_j (1 - e^-tau)) / R_s^2
template <class S>
void depth(const Profile<S>& pf, double r_s, const std::vector<S>& K, int W,
           std::vector<S>& D, double* tau_out) {
  const int N = pf.N;
  D.assign(W, S(0.0));
  std::vector<S> tau(W);
  std::vector<S> acc(W, S(0.0));
  for (int j = 0; j < N; ++j) {
    for (int i = 0; i < W; ++i) tau[i] = S(0.0);
    for (int l = j; l < N; ++l) {
      const S dl = pf.DL[(size_t)j * N + l];
      const S* Kl = &K[(size_t)l * W];
      for (int i = 0; i < W; ++i) tau[i] += dl * Kl[i];
    }
    if (tau_out)
      for (int i = 0; i < W; ++i) tau_out[(size_t)j * W + i] = val(tau[i]);
    for (int i = 0; i < W; ++i) acc[i] += pf.A[j] * (-expm1(-tau[i]));
  }
  const S rs2 = S(r_s * r_s);
  for (int i = 0; i < W; ++i) D[i] = (pf.r_p * pf.r_p + acc[i]) / rs2;
}

// FluxBinner weights (Sec. 4.5): native bin i spans the wavelengths between the midpoints of
// its neighbouring wavenumbers (one-sided at the grid ends); w_ij = overlap / width_i.
void bin_weights(const double* wn, int W, const orc_bins& bins, std::vector<double>& w) {
  w.assign((size_t)bins.n_bin * W, 0.0);
  for (int i = 0; i < W; ++i) {
    const double nu_lo = (i > 0) ? 0.5 * (wn[i - 1] + wn[i]) : wn[0] - 0.5 * (wn[1] - wn[0]);
    const double nu_hi = (i < W - 1) ? 0.5 * (wn[i] + wn[i + 1])
                                     : wn[W - 1] + 0.5 * (wn[W - 1] - wn[W - 2]);
    const double li_minus = 1e4 / nu_hi, li_plus = 1e4 / nu_lo;
    const double dli = li_plus - li_minus;
    for (int j = 0; j < bins.n_bin; ++j) {
      const double lj_minus = bins.lam_centre_um[j] - 0.5 * bins.lam_width_um[j];
      const double lj_plus = bins.lam_centre_um[j] + 0.5 * bins.lam_width_um[j];
      const double ov = std::min(lj_plus, li_plus) - std::max(lj_minus, li_minus);
      if (ov > 0.0) w[(size_t)j * W + i] = ov / dli;
    }
  }
}

// Native index range [i0, i1) that carries any bin weight (binning restricts the spectrum
// to the binned region, Sec. 4.5); the full range when bins is NULL.
void bin_range(const std::vector<double>& w, int n_bin, int W, int* i0, int* i1) {
  int lo = W, hi = 0;
  for (int j = 0; j < n_bin; ++j)
    for (int i = 0; i < W; ++i)
      if (w[(size_t)j * W + i] > 0.0) { lo = std::min(lo, i); hi = std::max(hi, i + 1); }
  if (lo >= hi) { lo = 0; hi = 0; }
  *i0 = lo; *i1 = hi;
}

template <class S>
void bin_spectrum(const std::vector<double>& w, int n_bin, int W, int i0,
                  const std::vector<S>& D, std::vector<S>& out) {
  out.assign(n_bin, S(0.0));
  for (int j = 0; j < n_bin; ++j) {
    S num(0.0); double den = 0.0;
    for (int i = 0; i < (int)D.size(); ++i) {
      const double wij = w[(size_t)j * W + i0 + i];
      if (wij == 0.0) continue;
      num += S(wij) * D[i];
      den += wij;
    }
    out[j] = (den > 0.0) ? num / S(den) : S(0.0);
  }
}

template <class S>
Params<S> params_from_atm(const orc_tables& tb, const orc_atm& a) {
  Params<S> p;
  p.n_layers = a.n_layers; p.p_max = a.p_max; p.p_min = a.p_min;
  p.n_tnodes = a.n_tnodes;
  p.tnode_log10p.assign(a.tnode_log10p, a.tnode_log10p + a.n_tnodes);
  p.tnode_t.clear();
  for (int k = 0; k < a.n_tnodes; ++k) p.tnode_t.push_back(S(a.tnode_t[k]));
  p.log10_x.clear();
  for (int m = 0; m < tb.n_mol; ++m) p.log10_x.push_back(S(a.log10_x[m]));
  p.fill_frac.assign(a.fill_frac, a.fill_frac + (tb.n_species - tb.n_mol));
  p.r_p = S(a.r_p); p.m_p = a.m_p; p.r_s = a.r_s;
  p.cloud_on = (a.cloud_mode != 0 && a.p_cloud_top > 0.0);
  p.log10_p_cloud_top = S(p.cloud_on ? std::log10(a.p_cloud_top) : 0.0);
  p.p_cloud_bot = a.p_cloud_bot; p.kappa_cloud = a.kappa_cloud;
  p.gravity_mode = a.gravity_mode; p.cloud_mode = a.cloud_mode;
  p.t_profile = a.t_profile; p.t_int = a.t_int; p.gas_mode = a.gas_mode;
  if (a.t_profile == 1)
    for (int k = 0; k < 5; ++k) p.guillot.push_back(S(a.guillot[k]));
  if (a.gas_mode == 1)
    for (int m = 0; m < tb.n_mol; ++m) {
      p.log10_x_top.push_back(S(a.log10_x_top[m]));
      p.log10_p_switch.push_back(S(a.log10_p_switch[m]));
    }
  return p;
}

// Length of theta for a batch: chemistry (n_mol log10 X, or for two-layer gases n_mol each of
// log10 X_surf, log10 X_top, log10 P_switch) | temperature (n_tnodes nodes, or the five
// Guillot parameters) | R_p / R_J | log10 P_cloud_top.
int theta_len(const orc_batch& b) {
  return (b.gas_mode == 1 ? 3 * b.n_mol : b.n_mol) + (b.t_profile == 1 ? 5 : b.n_tnodes) + 2;
}

// theta = [chemistry | temperature | R_p / R_J | log10 P_cloud_top (Pa)]; chemistry is
// log10 X_m (n_mol), or [log10 X_surf | log10 X_top | log10 P_switch] (3 n_mol) for two-layer
// gases; temperature is the T nodes (n_tnodes), or [T_irr (K) | log10 kappa_irr |
// log10 kappa_v1 | log10 kappa_v2 (m^2/kg) | alpha] for the Guillot2010 profile
template <class S>
Params<S> params_from_theta(const orc_tables& tb, const orc_batch& b, const S* th, int n_layers) {
  Params<S> p;
  p.n_layers = n_layers; p.p_max = b.p_max; p.p_min = b.p_min;
  p.n_tnodes = b.n_tnodes;
  p.tnode_log10p.assign(b.tnode_log10p, b.tnode_log10p + b.n_tnodes);
  const int nm = b.n_mol;
  const int n_chem = b.gas_mode == 1 ? 3 * nm : nm;
  const int n_t = b.t_profile == 1 ? 5 : b.n_tnodes;
  p.log10_x.assign(th, th + nm);
  p.gas_mode = b.gas_mode;
  if (b.gas_mode == 1) {
    p.log10_x_top.assign(th + nm, th + 2 * nm);
    p.log10_p_switch.assign(th + 2 * nm, th + 3 * nm);
  }
  p.t_profile = b.t_profile;
  p.t_int = b.t_int;
  if (b.t_profile == 1) {
    const S* g = th + n_chem;
    p.guillot = {g[0], pow10s(g[1]), pow10s(g[2]), pow10s(g[3]), g[4]};
  } else {
    p.tnode_t.assign(th + n_chem, th + n_chem + b.n_tnodes);
  }
  p.fill_frac.assign(b.fill_frac, b.fill_frac + (tb.n_species - tb.n_mol));
  p.r_p = th[n_chem + n_t] * S(R_JUPITER);
  p.m_p = b.m_p; p.r_s = b.r_s;
  p.cloud_on = (b.cloud_mode != 0);
  p.log10_p_cloud_top = th[n_chem + n_t + 1];
  p.p_cloud_bot = b.p_cloud_bot; p.kappa_cloud = b.kappa_cloud;
  p.gravity_mode = b.gravity_mode; p.cloud_mode = b.cloud_mode;
  return p;
}

// Planck function per wavenumber (Sec. 4, emission model: B of the layer temperatures):
// B(nu, T) = 2 h c^2 nu^3 / (e^{h c nu / (k_B T)} - 1), nu in 1/m (nu_cm in 1/cm), SI units
// W m^-2 sr^-1 per 1/m.
double planck(double nu_cm, double T) {
  const double nu = 100.0 * nu_cm;
  return 2.0 * H_PLANCK * C_LIGHT * C_LIGHT * nu * nu * nu /
         std::expm1(H_PLANCK * C_LIGHT * nu / (K_BOLTZ * T));
}

// n-point Gauss-Legendre nodes and weights on [0, 1]: the roots t of the Legendre polynomial
// P_n by Newton's method from cos(pi (i + 3/4) / (n + 1/2)), with P_n from the three-term
// recurrence k P_k = (2k - 1) t P_{k-1} - (k - 1) P_{k-2} and P_n'(t) = n (t P_n - P_{n-1}) /
// (t^2 - 1); weight 2 / ((1 - t^2) P_n'(t)^2); then x = (t + 1)/2, w -> w/2.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double t = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = (n == 1) ? 1.0 : n * (t * p1 - p0) / (t * t - 1.0);
      const double step = p1 / dp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      const double pk = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    dp = (n == 1) ? 1.0 : n * (t * p1 - p0) / (t * t - 1.0);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 0.5 * 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Temperature of the profile at log10 p (the N-point rule of Sec. 4.2, clamped at the ends;
// or the Guillot2010 profile).
double t_at(const Params<double>& pr, double x) {
  if (pr.t_profile == 1) {
    const double gs = G_NEWTON * pr.m_p / (pr.r_p * pr.r_p);
    return std::sqrt(std::sqrt(guillot_t4(pr, std::pow(10.0, x), gs)));
  }
  const int nt = pr.n_tnodes;
  if (nt == 1 || x >= pr.tnode_log10p[0]) return pr.tnode_t[0];
  if (x <= pr.tnode_log10p[nt - 1]) return pr.tnode_t[nt - 1];
  int k = 0;
  while (!(pr.tnode_log10p[k] >= x && x >= pr.tnode_log10p[k + 1])) ++k;
  const double f = (x - pr.tnode_log10p[k]) / (pr.tnode_log10p[k + 1] - pr.tnode_log10p[k]);
  return pr.tnode_t[k] + (pr.tnode_t[k + 1] - pr.tnode_t[k]) * f;
}

bool tables_ok(const orc_tables* tb) {
  if (!tb || tb->n_mol < 0 || tb->n_p < 2 || tb->n_t < 2 || tb->n_wn < 2) return false;
  if (tb->n_species < tb->n_mol) return false;
  if (tb->n_cia > 0 && tb->n_t_cia < 2) return false;
  return true;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// exported entry points (ctypes)
// ------------------------------------------------------------------------------------------
extern "C" {

// Layer-by-layer profile of one model (a1-a5 plus cloud fractions and annulus weights).
// Arrays: pb[N+1], P[N], T[N], X[n_species], g[N], H[N], z[N+1], rho[N], cloud[N], DL[N*N], A[N].
// scal[0] = mu (amu), scal[1] = Delta.
// X: [N][n_species] mixing ratios of every layer; scal[0] = mu of layer 0; mu_l: [N] or NULL.
int orc_profile(const orc_tables* tb, const orc_atm* atm, double* pb, double* P, double* T,
                double* X, double* g, double* H, double* z, double* rho, double* cloud,
                double* DL, double* A, double* scal, double* mu_l) {
  if (!tables_ok(tb) || !atm) return ORC_ERR_ARG;
  Params<double> pr = params_from_atm<double>(*tb, *atm);
  Profile<double> pf;
  const int st = build_profile(*tb, pr, pf);
  if (st != ORC_OK) return st;
  const int N = pf.N;
  std::copy(pf.pb.begin(), pf.pb.end(), pb);
  std::copy(pf.P.begin(), pf.P.end(), P);
  std::copy(pf.T.begin(), pf.T.end(), T);
  std::copy(pf.X.begin(), pf.X.end(), X);
  std::copy(pf.g.begin(), pf.g.end(), g);
  std::copy(pf.H.begin(), pf.H.end(), H);
  std::copy(pf.z.begin(), pf.z.end(), z);
  std::copy(pf.rho.begin(), pf.rho.end(), rho);
  std::copy(pf.cloud.begin(), pf.cloud.end(), cloud);
  std::copy(pf.DL.begin(), pf.DL.end(), DL);
  std::copy(pf.A.begin(), pf.A.end(), A);
  scal[0] = pf.mu[0]; scal[1] = pf.delta;
  if (mu_l) std::copy(pf.mu.begin(), pf.mu.end(), mu_l);
  (void)N;
  return ORC_OK;
}

// Interpolated cross-section of molecule m at (P, T) on the whole native grid (a6 alone).
int orc_interp(const orc_tables* tb, int m, double P, double T, double* out) {
  if (!tables_ok(tb) || m < 0 || m >= tb->n_mol) return ORC_ERR_ARG;
  int ip = 0, it = 0; double tp = 0.0, tt = 0.0;
  if (!axis_weights(tb->p_grid, tb->n_p, P, tb->oor_mode, &ip, &tp) ||
      !axis_weights(tb->t_grid, tb->n_t, T, tb->oor_mode, &it, &tt)) {
    for (int i = 0; i < tb->n_wn; ++i) out[i] = 0.0;
    return ORC_OK;
  }
  const size_t slab = (size_t)tb->n_t * tb->n_wn;
  const float* s00 = tb->sigma + ((size_t)m * tb->n_p + ip) * slab + (size_t)it * tb->n_wn;
  const float* s01 = s00 + tb->n_wn;
  const float* s10 = s00 + slab;
  const float* s11 = s10 + tb->n_wn;
  const double T1 = tb->t_grid[it], T2 = tb->t_grid[it + 1];
  for (int i = 0; i < tb->n_wn; ++i) {
    const double a1 = interp_t(s00[i], s01[i], tt, T1, T2, tb->interp_mode);
    const double a2 = interp_t(s10[i], s11[i], tt, T1, T2, tb->interp_mode);
    out[i] = a1 + (a2 - a1) * tp;
  }
  return ORC_OK;
}

// Exponential integrals E_1(x) and E_2(x) at n points x > 0 (E_2 of the Guillot profile).
int orc_expint(const double* x, int n, double* e1, double* e2) {
  if (!x || n < 0 || !e1 || !e2) return ORC_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!(x[i] > 0.0)) return ORC_ERR_ARG;
    e1[i] = expint_e1(x[i]);
    e2[i] = expint_e2(x[i]);
  }
  return ORC_OK;
}

// Planck function at n wavenumbers (1/cm) and one temperature (K): out[n].
int orc_planck(const double* nu_cm, int n, double T, double* out) {
  if (!nu_cm || n < 0 || !out || !(T > 0.0)) return ORC_ERR_ARG;
  for (int i = 0; i < n; ++i) out[i] = planck(nu_cm[i], T);
  return ORC_OK;
}

// Gauss-Legendre nodes x[n] and weights w[n] on [0, 1].
int orc_gauss_legendre01(int n, double* x_out, double* w_out) {
  if (n < 1 || !x_out || !w_out) return ORC_ERR_ARG;
  std::vector<double> x, w;
  gauss_legendre01(n, x, w);
  std::copy(x.begin(), x.end(), x_out);
  std::copy(w.begin(), w.end(), w_out);
  return ORC_OK;
}

// Emission model of Sec. 4 (plane-parallel atmosphere, intensity at the top integrated over
// the viewing angle): fp_fs[n_wn] = I / I_s (R_p / R_s)^2, with
//   I(mu) = B(T_s) e^{-tau_s / mu} + sum_l B(T_l) (e^{-tau_l,top / mu} - e^{-tau_l,bottom / mu}),
//   I = sum_i I(x_i) x_i w_i  (n_mu-point Gauss-Legendre on [0, 1]),
// from the same opacity K as the transmission model.  Readings (the paper's equation is
// garbled: it integrates in mu twice and drops the 1/mu of the slant path):
//   E1 layer l's vertical optical depth is K_l (z_{l+1} - z_l); tau is counted from the top
//      (layer N-1) down to the surface (boundary 0), tau_s the total;
//   E2 the source is B(T_l) throughout layer l, so the layer's part of the formal solution
//      int B e^{-tau/mu} dtau/mu is B(T_l) (e^{-tau_top/mu} - e^{-tau_bot/mu});
//   E3 T_s is the profile's temperature at p_max (the paper's "temperature at maximum
//      atmospheric pressure");
//   E4 I_s is the same quadrature of the star's isotropic intensity, B(T_star) sum_i x_i w_i.
int orc_emission(const orc_tables* tb, const orc_atm* atm, int n_mu, double t_star,
                 double* fp_fs) {
  if (!tables_ok(tb) || !atm || n_mu < 1 || !(t_star > 0.0) || !fp_fs) return ORC_ERR_ARG;
  Params<double> pr = params_from_atm<double>(*tb, *atm);
  Profile<double> pf;
  const int st = build_profile(*tb, pr, pf);
  if (st != ORC_OK) return st;
  const int W = tb->n_wn, N = pf.N;
  std::vector<double> K;
  opacity(*tb, pr, pf, 0, W, K);
  std::vector<double> x, w;
  gauss_legendre01(n_mu, x, w);
  double xw = 0.0;
  for (int k = 0; k < n_mu; ++k) xw += x[k] * w[k];
  const double t_s = t_at(pr, std::log10(pr.p_max));
  const double rr = (pr.r_p / pr.r_s) * (pr.r_p / pr.r_s);
  std::vector<double> I(n_mu);
  for (int i = 0; i < W; ++i) {
    const double nu = tb->wn_grid[i];
    for (int k = 0; k < n_mu; ++k) I[k] = 0.0;
    double tau_top = 0.0;
    for (int l = N - 1; l >= 0; --l) {              // from the top layer down
      const double tau_bot = tau_top + K[(size_t)l * W + i] * (pf.z[l + 1] - pf.z[l]);
      const double b = planck(nu, pf.T[l]);
      for (int k = 0; k < n_mu; ++k)
        I[k] += b * (std::exp(-tau_top / x[k]) - std::exp(-tau_bot / x[k]));
      tau_top = tau_bot;
    }
    const double bs = planck(nu, t_s);
    double flux = 0.0;
    for (int k = 0; k < n_mu; ++k) flux += (I[k] + bs * std::exp(-tau_top / x[k])) * x[k] * w[k];
    fp_fs[i] = flux / (planck(nu, t_star) * xw) * rr;
  }
  return ORC_OK;
}

// Dense FluxBinner weights w[n_bin][n_wn].
int orc_bin_weights(const double* wn, int W, const orc_bins* bins, double* w_out) {
  if (!wn || W < 2 || !bins || bins->n_bin < 1) return ORC_ERR_ARG;
  std::vector<double> w;
  bin_weights(wn, W, *bins, w);
  std::copy(w.begin(), w.end(), w_out);
  return ORC_OK;
}

// One forward model: native depth[n_wn] (optional), binned depth[n_bin] (optional, needs
// bins), optical depth tau[N][n_wn] (optional).  Native outputs cover the full grid.
int orc_forward(const orc_tables* tb, const orc_atm* atm, const orc_bins* bins,
                double* depth_native, double* depth_binned, double* tau) {
  if (!tables_ok(tb) || !atm) return ORC_ERR_ARG;
  Params<double> pr = params_from_atm<double>(*tb, *atm);
  Profile<double> pf;
  const int st = build_profile(*tb, pr, pf);
  if (st != ORC_OK) return st;
  const int W = tb->n_wn;
  std::vector<double> K, D;
  opacity(*tb, pr, pf, 0, W, K);
  depth(pf, pr.r_s, K, W, D, tau);
  if (depth_native) std::copy(D.begin(), D.end(), depth_native);
  if (depth_binned && bins) {
    std::vector<double> w, Db;
    bin_weights(tb->wn_grid, W, *bins, w);
    bin_spectrum(w, bins->n_bin, W, 0, D, Db);
    std::copy(Db.begin(), Db.end(), depth_binned);
  }
  return ORC_OK;
}

// Batch of binned forward models, theta[B][n_theta]; computes only the binned region.
// status[b] = 0 or ORC_ERR_INVALID_MODEL (binned row then all zero).  n_threads > 1 uses
// OpenMP across models (timing only; each model is computed the same way).
int orc_forward_batch(const orc_tables* tb, const orc_batch* bt, int B, const double* theta,
                      const int* nlayers, const orc_bins* bins, double* binned, int* status,
                      int n_threads) {
  if (!tables_ok(tb) || !bt || !bins || B < 0 || bt->n_mol != tb->n_mol) return ORC_ERR_ARG;
  const int W = tb->n_wn, nth = theta_len(*bt);
  std::vector<double> w;
  bin_weights(tb->wn_grid, W, *bins, w);
  int i0 = 0, i1 = 0;
  bin_range(w, bins->n_bin, W, &i0, &i1);
#ifdef _OPENMP
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int b = 0; b < B; ++b) {
    Params<double> pr = params_from_theta<double>(*tb, *bt, theta + (size_t)b * nth, nlayers[b]);
    Profile<double> pf;
    const int st = build_profile(*tb, pr, pf);
    status[b] = st;
    double* out = binned + (size_t)b * bins->n_bin;
    if (st != ORC_OK) { for (int j = 0; j < bins->n_bin; ++j) out[j] = 0.0; continue; }
    std::vector<double> K, D, Db;
    opacity(*tb, pr, pf, i0, i1, K);
    depth(pf, pr.r_s, K, i1 - i0, D, nullptr);
    bin_spectrum(w, bins->n_bin, W, i0, D, Db);
    std::copy(Db.begin(), Db.end(), out);
  }
  return ORC_OK;
}

// chi^2 = sum_j ((D_bin_j - obs_j) / sigma_j)^2 of one model and its exact gradient with
// respect to theta (dual numbers).  Outputs: chi2, grad[n_theta], binned[n_bin],
// jac[n_bin][n_theta] (optional).
int orc_chi2_grad(const orc_tables* tb, const orc_batch* bt, const double* theta, int n_layers,
                  const orc_bins* bins, const double* obs, const double* sig_obs,
                  double* chi2, double* grad, double* binned, double* jac) {
  if (!tables_ok(tb) || !bt || !bins || bt->n_mol != tb->n_mol) return ORC_ERR_ARG;
  const int nth = theta_len(*bt);
  if (nth > NDIR) return ORC_ERR_ARG;
  const int W = tb->n_wn;
  std::vector<Dual> th(nth);
  for (int k = 0; k < nth; ++k) { th[k] = Dual(theta[k]); th[k].d[k] = 1.0; }
  Params<Dual> pr = params_from_theta<Dual>(*tb, *bt, th.data(), n_layers);
  Profile<Dual> pf;
  const int st = build_profile(*tb, pr, pf);
  if (st != ORC_OK) return st;
  std::vector<double> w;
  bin_weights(tb->wn_grid, W, *bins, w);
  int i0 = 0, i1 = 0;
  bin_range(w, bins->n_bin, W, &i0, &i1);
  std::vector<Dual> K, D, Db;
  opacity(*tb, pr, pf, i0, i1, K);
  depth(pf, pr.r_s, K, i1 - i0, D, nullptr);
  bin_spectrum(w, bins->n_bin, W, i0, D, Db);
  Dual c(0.0);
  for (int j = 0; j < bins->n_bin; ++j) {
    const Dual r = (Db[j] - Dual(obs[j])) / Dual(sig_obs[j]);
    c += r * r;
  }
  *chi2 = c.v;
  for (int k = 0; k < nth; ++k) grad[k] = c.d[k];
  for (int j = 0; j < bins->n_bin; ++j) {
    if (binned) binned[j] = Db[j].v;
    if (jac) for (int k = 0; k < nth; ++k) jac[(size_t)j * nth + k] = Db[j].d[k];
  }
  return ORC_OK;
}

}  // extern "C"
