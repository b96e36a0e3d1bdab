/*
 * transit.h -- C ABI of the GB300 transmission forward model (TauREx 3, arXiv:1912.07759).
 *
 * The library computes, on one GPU, the 1-D transmission spectrum of an exoplanet atmosphere:
 * cross-section interpolation from (P, T, wavenumber) tables, weighting by mixing ratio and
 * number density with CIA, Rayleigh and grey-cloud opacity fused into one opacity K[layer, wn]
 * (Sec. 4.4 and Sec. 8.1), the slant optical depth tau = DL . K (Sec. 4, eqs. tot_opt_dpth,
 * opt_dpth, cia_opt_dpth) and the transit depth (Sec. 4, eqs. for Delta_lambda, a_lambda),
 * native and binned (Sec. 4.5).  Batched forward models and a hand-written adjoint for
 * chi^2 gradients are additions of this library; the paper has no GPU or gradient path.
 *
 * Conventions common to every call
 *  - Units are SI (Sec. 3) except wavenumbers (cm^-1) and bin wavelengths (micron).
 *  - Every call returns an int status (TR_OK or a TR_ERR_* code); tr_last_error() gives a
 *    message.  Batch calls also write a per-item status and return TR_OK when the launch
 *    itself succeeded.
 *  - Pointers named d_* are device pointers owned by the caller (for example PyTorch tensors),
 *    contiguous, of the stated type.  All other pointers are host pointers, borrowed for the
 *    duration of the call.
 *  - Handles (tr_ctx, tr_tables, tr_atm, tr_bins) own their device memory and are released
 *    with the matching tr_free_* / tr_destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *    that take a stream are asynchronous on it and never synchronise the device, except
 *    where stated.  A context is not thread-safe; use one per host thread.
 *  - There is no CPU fallback: without a usable CUDA device every call fails.
 */
#ifndef TRANSIT_H_
#define TRANSIT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
  TR_OK = 0,
  TR_ERR_ARG = 1,            /* null pointer, bad size, unsorted grid, unsupported shape */
  TR_ERR_INVALID_MODEL = 2,  /* sum X > 1, T <= 0, non-monotone T nodes, N < 1, non-finite
                                parameters: the model rejection of Sec. 6 */
  TR_ERR_OOM = 3,            /* device allocation failed or workspace too small */
  TR_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  TR_ERR_TIMEOUT = 5,        /* a bounded device wait expired */
  TR_ERR_UNSUPPORTED = 6     /* option not available (e.g. precision without its tables) */
};

/* table storage (bit mask) */
enum { TR_STORE_FP32 = 1, TR_STORE_FP16_LOG10 = 2 };
/* out-of-range rule of Sec. 5: clamp to the grid edge, or the paper's rule (below the grid
   minimum -> zero cross-section, above the maximum -> edge value) */
enum { TR_OOR_CLAMP = 0, TR_OOR_PAPER_ZERO = 1 };
/* temperature interpolation of the absorbers' cross-sections (Sec. 5): linear (the default),
   or the exponential scheme sigma(T) = a e^{-b/T} through the two bracketing temperatures
   (b = (1/T2 - 1/T1)^{-1} ln(sigma(T1)/sigma(T2)), a = sigma(T1) e^{b/T1}; where a bracketing
   value is not positive the linear value is used).  Pressure and CIA stay linear.  The
   exponential scheme is supported by the forward calls (two-stage kernels, both precisions);
   the adjoint and the allocation-free entry point return TR_ERR_UNSUPPORTED for it. */
enum { TR_INTERP_LINEAR = 0, TR_INTERP_EXP = 1 };
/* gravity: g_l = G M_p / (R_p + z_l)^2, or constant G M_p / R_p^2 */
enum { TR_GRAV_ALTITUDE = 0, TR_GRAV_CONST = 1 };
/* grey cloud deck (Sec. 4.4, eq. clouds): none; discrete (a layer is cloudy when its
   pressure lies in [P_top, P_bot]); fractional (the fraction of the layer's ln P extent
   inside the deck, which makes the depth differentiable in P_top) */
enum { TR_CLOUD_NONE = 0, TR_CLOUD_DISCRETE = 1, TR_CLOUD_FRACTIONAL = 2 };
/* temperature profile (Sec. 4.2): N-point (isothermal with one node), or Guillot2010
   radiative equilibrium with two visible channels,
     T^4 = 3/4 T_int^4 (2/3 + tau) + 3/4 T_irr^4 [(1 - alpha) xi(g1) + alpha xi(g2)],
     xi(g) = 2/3 + 2/(3g) [1 + (g tau/2 - 1) e^{-g tau}] + 2g/3 (1 - tau^2/2) E_2(g tau),
   g_i = kappa_v,i / kappa_irr, tau = kappa_irr P / g_s, g_s = G M_p / R_p^2 (opacities in
   m^2/kg; the paper names the profile and its parameters without stating it) */
enum { TR_TPROF_NPOINT = 0, TR_TPROF_GUILLOT = 1 };
/* vertical mixing profile of the absorbers (Sec. 4.3): constant, or two-layer: X_surf below
   the switch pressure P_sw and X_top above it, a layer straddling the switch taking
   f X_surf + (1 - f) X_top with f the fraction of its ln P extent below the switch; fill gases
   share each layer's remainder, so the mean molecular weight varies by layer */
enum { TR_GAS_CONSTANT = 0, TR_GAS_TWOLAYER = 1 };
/* arithmetic of the forward path: FP32 tables and FP32 opacity, the tau contraction on tensor
   cores as three TF32 products of exact hi + lo splits (3xTF32, FP32 accumulation, errors below
   2^-20 of a product; up to 112 layers, FP32 FMAs beyond); or FP16 log10 sigma tables with the
   tau contraction on tensor cores as BF16 hi+lo split products */
enum { TR_PREC_FP32 = 0, TR_PREC_MIXED = 1 };

/* compile-time limits of the library */
enum { TR_MAX_MOL = 8, TR_MAX_CIA = 4, TR_MAX_SPECIES = 12, TR_MAX_TNODES = 8,
       TR_MAX_LAYERS = 180, TR_MAX_BATCH = 65535 };   /* the FP32 kernel stages K and DL for all layers in shared memory */

typedef struct tr_ctx tr_ctx;
typedef struct tr_tables tr_tables;
typedef struct tr_atm tr_atm;
typedef struct tr_bins tr_bins;

/* Create a context on CUDA device `device` (made current on the calling thread). */
int tr_create(tr_ctx** ctx, int device);
/* Destroy a context and its internal scratch memory. */
void tr_destroy(tr_ctx* ctx);
/* Message of the last failed call on this context (never NULL). */
const char* tr_last_error(const tr_ctx* ctx);
/* Synchronise `stream` and report device-side failures of earlier calls on this context:
   every wait inside the library's kernels is bounded; a wait that runs out records an error
   word instead of hanging, and this call returns TR_ERR_TIMEOUT once for it (then clears
   it).  The outputs of the affected calls are invalid. */
int tr_sync_status(tr_ctx* ctx, void* stream);
/* Failure-detection self-test: launches a kernel whose only wait can never complete (a
   barrier that expects an arrival nobody makes); its bounded wait gives up after 1000 polls
   and records the timeout, which the next tr_sync_status() must report as TR_ERR_TIMEOUT.
   Nothing faults or hangs. */
int tr_selftest_wait_timeout(tr_ctx* ctx, void* stream);

/*
 * Cross-section tables (Sec. 5: temperature-pressure-wavenumber grids with linear P and T
 * interpolation; Sec. 5.2: the opacity cache).  All molecules, CIA pairs and Rayleigh arrays
 * share one native wavenumber grid (Sec. 5: the native grid of the forward model).
 *   p_grid [n_p] Pa, t_grid [n_t] K, wn_grid [n_wn] cm^-1: strictly ascending, n >= 2.
 *   sigma [n_mol][n_p][n_t][n_wn] float, linear cross-section in m^2 (normal FP32 values).
 *   cia [n_cia][n_t_cia][n_wn] double, m^5, on t_grid_cia [n_t_cia]; cia_pair[n_cia][2]
 *     species indices (the pair's mixing ratios weight it, eq. cia_opt_dpth).
 *   rayleigh [n_species][n_wn] double, m^2, or NULL (weighted like absorbers).
 *   species: indices 0..n_mol-1 are the absorbers (in sigma order), n_mol..n_species-1 are
 *     fill gases; mass_amu [n_species] their masses (Sec. 4.3, mean molecular weight).
 *   storage: TR_STORE_FP32 and/or TR_STORE_FP16_LOG10 (the latter is needed by
 *     TR_PREC_MIXED; it stores fp16(log10 sigma - c_m) with one offset c_m per molecule).
 * The host arrays are copied; the handle owns the device copy.  Synchronous.
 */
typedef struct {
  int n_mol, n_p, n_t, n_wn;
  const double* p_grid;
  const double* t_grid;
  const double* wn_grid;
  const float* sigma;
  int n_cia, n_t_cia;
  const double* t_grid_cia;
  const int32_t* cia_pair;
  const double* cia;
  int n_species;
  const double* mass_amu;
  const double* rayleigh;
  int storage;
  int oor_mode;
  int interp_mode;             /* TR_INTERP_LINEAR or TR_INTERP_EXP */
} tr_table_desc;

int tr_load_xsec_tables(tr_ctx* ctx, const tr_table_desc* desc, tr_tables** out);
void tr_free_tables(tr_tables* tables);
/* Bytes of device memory the handle holds. */
size_t tr_tables_device_bytes(const tr_tables* tables);

/*
 * One atmosphere (Sec. 4: SimpleForwardModel set-up).  Builds, on the device in FP64, the
 * pressure grid (Sec. 4.1: n_layers+1 log-uniform boundaries from p_max at the bottom to
 * p_min; layer pressure P_l = p_l sqrt(p_{l+1}/p_l)), the temperature profile (Sec. 4.2:
 * isothermal when n_tnodes == 1, else linear in log P between nodes, clamped beyond them),
 * constant mixing ratios with fill gases taking fractions fill_frac of 1 - sum X (Sec. 4.3),
 * the hydrostatic altitudes (Sec. 4: z_0 = 0, z_{l+1} = z_l + H_l ln(p_l/p_{l+1}),
 * H_l = k_B T_l / (mu m_u g_l)), the slant path lengths of each ray through each shell and
 * the interpolation brackets of each layer.
 *   tnode_log10p [n_tnodes] strictly descending, tnode_t [n_tnodes] K (N-point profile).
 *   t_profile TR_TPROF_GUILLOT: guillot [5] = T_irr (K), kappa_irr, kappa_v1, kappa_v2
 *     (m^2/kg), alpha in [0, 1]; t_int the internal temperature (K); the nodes are ignored.
 *   log10_x [n_mol] (the surface values with TR_GAS_TWOLAYER); fill_frac [n_species - n_mol].
 *   gas_mode TR_GAS_TWOLAYER: log10_x_top [n_mol], log10_p_switch [n_mol] (log10 Pa).
 *   p_cloud_top <= 0 or cloud_mode == TR_CLOUD_NONE: no cloud; p_cloud_bot <= 0: p_max;
 *   kappa_cloud: cloud opacity in 1/m.
 * Returns TR_ERR_INVALID_MODEL for a rejected model.  Enqueued on `stream`; the handle may
 * be used by later calls on the same stream.
 */
typedef struct {
  int n_layers;
  double p_max, p_min;
  int n_tnodes;
  const double* tnode_log10p;
  const double* tnode_t;
  const double* log10_x;
  const double* fill_frac;
  double r_p, m_p, r_s;
  double p_cloud_top, p_cloud_bot, kappa_cloud;
  int gravity_mode;
  int cloud_mode;
  int t_profile;                /* TR_TPROF_* */
  const double* guillot;        /* [5] with TR_TPROF_GUILLOT, else NULL */
  double t_int;                 /* K, Guillot internal temperature */
  int gas_mode;                 /* TR_GAS_* */
  const double* log10_x_top;    /* [n_mol] with TR_GAS_TWOLAYER, else NULL */
  const double* log10_p_switch; /* [n_mol] with TR_GAS_TWOLAYER, else NULL */
} tr_atm_desc;

int tr_build_atmosphere(tr_ctx* ctx, const tr_tables* tables, const tr_atm_desc* desc,
                        tr_atm** out, void* stream);
void tr_free_atmosphere(tr_atm* atm);

/*
 * Geometry of an atmosphere handle copied to host arrays (inspection and tests): z
 * [n_layers+1] boundary altitudes (m, FP64); dl [n_layers][n_layers] path length of ray j
 * through shell l in row j (zero for l < j, FP32); a [n_layers] annulus weights
 * (r_{j+1}^2 - r_j^2) / R_s^2 (FP32).  Any output may be NULL.  Synchronous.
 */
int tr_atm_readback(tr_ctx* ctx, const tr_atm* atm, double* z, float* dl, float* a);

/*
 * Target bins for the FluxBinner of Sec. 4.5: bin j spans lam_centre_um[j] -+ width/2
 * (micron); native bin i spans the wavelengths between the midpoints of its neighbouring
 * wavenumbers (one-sided at the grid ends); w_ij = overlap / native width (eq. w_ij) and the
 * binned value is sum_i w_ij F_i / sum_i w_ij (eq. F_j).  Bins must overlap the native grid.
 * Synchronous; the handle owns the device copy of the weights.
 */
int tr_make_bins(tr_ctx* ctx, const tr_tables* tables, int n_bin, const double* lam_centre_um,
                 const double* lam_width_um, tr_bins** out);
void tr_free_bins(tr_bins* bins);
/* Native index range [*i0, *i1) that carries bin weight. */
int tr_bins_native_range(const tr_bins* bins, int* i0, int* i1);

/*
 * FluxBinner of Sec. 4.5 on B native spectra with uncertainties (eqs. F_j and sigma_j):
 *   d_binned[b][j]       = sum_i w_ij F_i / sum_i w_ij,
 *   d_binned_sigma[b][j] = sqrt(sum_i w_ij^2 sigma_i^2) / sum_i w_ij,
 * with the weights of `bins`.  Native spectrum b is d_native[b * stride + (i - base)] for
 * native index i (double; the range [base, base + ...) must cover the bins' native range);
 * d_native_sigma likewise (double) or NULL (then d_binned_sigma is not written and may be
 * NULL).  Outputs [B][n_bin] double, caller-owned.  Enqueued on `stream`.
 */
int tr_bin_spectra(tr_ctx* ctx, const tr_bins* bins, int B, const double* d_native,
                   const double* d_native_sigma, long long stride, int base, double* d_binned,
                   double* d_binned_sigma, void* stream);

/*
 * SNR instrument model of Sec. 7: for each spectrum b of B binned spectra
 * d_binned[b][n_bin], the noise is N = S / snr with S the largest value of the spectrum,
 * divided by sqrt(n_obs) for n_obs stacked observations (N' = N / sqrt(n_obs)); writes the
 * symmetric uncertainty d_sigma[b][j] = N' and the noisy observation
 * d_obs[b][j] = d_binned[b][j] + N' d_z[b][j] with standard-normal draws d_z[B][n_bin]
 * supplied by the caller (double).  snr > 0, n_obs >= 1; all arrays device, caller-owned.
 * Enqueued on `stream`.
 */
int tr_snr_instrument(tr_ctx* ctx, int B, int n_bin, const double* d_binned, double snr,
                      int n_obs, const double* d_z, double* d_obs, double* d_sigma,
                      void* stream);

/*
 * Transit depth of one atmosphere (Sec. 4, eqs. for Delta_lambda and a_lambda):
 *   D(wn) = (R_p^2 + sum_j A_j (1 - exp(-tau_j(wn)))) / R_s^2,
 *   tau_j(wn) = sum_{l >= j} DL[j][l] K_l(wn),  A_j = r_{j+1}^2 - r_j^2,
 * with K_l the fused opacity of layer l.
 *   d_depth_native [n_wn] double or NULL; d_depth_binned [n_bin] double or NULL (needs bins).
 *   precision: TR_PREC_FP32 or TR_PREC_MIXED.
 * Enqueued on `stream`.
 */
int tr_forward_transit(tr_ctx* ctx, const tr_tables* tables, const tr_atm* atm,
                       const tr_bins* bins, double* d_depth_native, double* d_depth_binned,
                       int precision, void* stream);

/*
 * Batch of independent atmospheres (the models a sampler evaluates; Sec. 6).  Per item b the
 * parameter vector d_theta[b][n_theta] is
 *   [ chemistry | temperature | R_p in R_J | log10 P_cloud_top (Pa) ]
 * chemistry: log10 X_m (n_mol) with TR_GAS_CONSTANT; with TR_GAS_TWOLAYER log10 X_surf (n_mol),
 *   log10 X_top (n_mol), log10 P_switch in Pa (n_mol);
 * temperature: the nodes in K (n_tnodes) with TR_TPROF_NPOINT; with TR_TPROF_GUILLOT T_irr (K),
 *   log10 kappa_irr, log10 kappa_v1, log10 kappa_v2 (m^2/kg), alpha;
 * so n_theta = n_mol + n_tnodes + 2 in the default modes, R_J = 6.9911e7 m (Sec. 8.2).
 * Everything else is fixed per batch in tr_batch_desc.  d_nlayers[b] (int32) is the layer count of item b,
 * 1 <= d_nlayers[b] <= max_layers (NULL: all max_layers).  Only the binned region of the
 * native grid is computed (Sec. 4.5: binning restricts the spectrum to its region).
 */
typedef struct {
  int n_tnodes;
  const double* tnode_log10p;   /* [n_tnodes] descending */
  const double* fill_frac;      /* [n_species - n_mol] */
  double p_max, p_min, m_p, r_s, p_cloud_bot, kappa_cloud;
  int gravity_mode, cloud_mode;
  int max_layers;               /* upper bound of d_nlayers; sizes the workspace */
  int t_profile;                /* TR_TPROF_* (0: N-point, the nodes above) */
  int gas_mode;                 /* TR_GAS_* (0: constant) */
  double t_int;                 /* K, internal temperature of the Guillot profile */
} tr_batch_desc;

/* Device workspace in bytes needed by a batch call of B items (forward or adjoint); with
   bins == NULL the size for native-resolution output (the whole grid) is returned. */
size_t tr_batch_workspace_size(const tr_tables* tables, const tr_batch_desc* desc,
                               const tr_bins* bins, int B, int with_adjoint);

/*
 * Batched forward model.  Outputs d_binned[B][n_bin] (double; needs bins), optionally
 * d_native[B][n_wn] (double, the full native spectrum of every item; NULL to compute only
 * the binned region), and d_status[B] (int32: TR_OK or TR_ERR_INVALID_MODEL; an invalid
 * item's outputs are zero).  At least one of d_native, d_binned must be given.
 *   d_workspace: caller-owned device memory of workspace_bytes >=
 *     tr_batch_workspace_size(..., with_adjoint=0) (computed with bins == NULL when
 *     d_native is given), or NULL to let the context allocate (the context then grows its
 *     own scratch, which synchronises the device).
 * Enqueued on `stream`.
 */
int tr_forward_transit_batch(tr_ctx* ctx, const tr_tables* tables, const tr_batch_desc* desc,
                             int B, const double* d_theta, const int32_t* d_nlayers,
                             const tr_bins* bins, double* d_native, double* d_binned,
                             int32_t* d_status, int precision, void* d_workspace,
                             size_t workspace_bytes, void* stream);

/*
 * Emission (eclipse) spectrum of Sec. 4: the planet-star flux ratio F_p/F_s per native
 * wavenumber of a plane-parallel atmosphere, from the same opacity K[layer, wn] as the
 * transmission model (cross-sections, CIA, Rayleigh and the grey cloud of Sec. 4.4, Sec. 5):
 *   I(mu) = B(T_s) e^{-tau_s/mu} + sum_l B(T_l) (e^{-tau_l,top/mu} - e^{-tau_l,bottom/mu}),
 *   F_p/F_s = sum_k x_k w_k I(x_k) / (B(T_star) sum_k x_k w_k) (R_p/R_s)^2,
 * with layer l's vertical optical depth K_l (z_{l+1} - z_l), tau counted from the top, T_s the
 * temperature profile at p_max, B the Planck function and (x_k, w_k) the n_mu-point
 * Gauss-Legendre rule on [0, 1] (the paper's quadrature over the viewing angle; it uses 4
 * points).  The paper's printed intensity is garbled (it integrates in mu twice and drops the
 * 1/mu of the slant path); the formula above is the formal solution it describes.
 *   n_mu: 1..16; t_star: stellar temperature in K (> 0).
 *   d_native [n_wn] double or NULL; d_binned [n_bin] double or NULL (the FluxBinner of
 *   Sec. 4.5 over the flux ratio; needs bins).  precision: TR_PREC_FP32 or TR_PREC_MIXED (the
 *   latter reads the FP16 log10 tables; the vertical pass is FP32 either way).
 * Enqueued on `stream`.
 */
int tr_forward_emission(tr_ctx* ctx, const tr_tables* tables, const tr_atm* atm,
                        const tr_bins* bins, int n_mu, double t_star, double* d_native,
                        double* d_binned, int precision, void* stream);
/*
 * Batched emission spectra: the items, theta layout, layer counts, per-item status and
 * workspace of tr_forward_transit_batch (the same workspace size serves), with the outputs
 * of tr_forward_emission per item: d_native [B][n_wn] and/or d_binned [B][n_bin] (double).
 * With d_native NULL only the binned region of the native grid is computed.  An invalid
 * item's outputs are zero.  Enqueued on `stream`.
 */
int tr_forward_emission_batch(tr_ctx* ctx, const tr_tables* tables, const tr_batch_desc* desc,
                              int B, const double* d_theta, const int32_t* d_nlayers,
                              const tr_bins* bins, int n_mu, double t_star, double* d_native,
                              double* d_binned, int32_t* d_status, int precision,
                              void* d_workspace, size_t workspace_bytes, void* stream);

/*
 * The batched forward of a sampler loop as one CUDA graph (the paper has no counterpart; its
 * retrievals evaluate the forward model once per live point, Sec. 6, and this packages that
 * repeated call).  Same arguments and outputs as tr_forward_transit_batch, plus:
 *   autotune: non-zero to time every configuration of the forward (two-stage form with 3, 2
 *     or 1 opacity CTAs per SM; for FP32 also the fused kernel) on these inputs first -- one
 *     warm-up and five timed runs each on `stream` -- and keep the fastest.  The choice is
 *     remembered on the context for this batch shape (tables, B, max_layers, precision,
 *     output range), so later captures and tr_forward_transit_batch calls of the same shape
 *     use it.  0: a configuration remembered earlier, else the defaults.
 *   d_workspace: as for tr_forward_transit_batch; with NULL the context's scratch is grown
 *     before capture and the graph keeps using it (do not free or regrow the context's
 *     scratch while the graph is in use: batch calls needing more scratch regrow it).
 * The tuning runs write the outputs.  The capture records the whole forward (geometry,
 * opacity, contraction, binning) on a private stream; *out owns the instantiated graph.  The
 * graph reads d_theta / d_nlayers and writes the outputs at the addresses given here: update
 * the inputs in place between launches.  Errors: the batch call's, TR_ERR_CUDA when capture
 * or instantiation fails.
 */
typedef struct tr_graph tr_graph;
int tr_capture_forward_batch(tr_ctx* ctx, const tr_tables* tables, const tr_batch_desc* desc,
                             int B, const double* d_theta, const int32_t* d_nlayers,
                             const tr_bins* bins, double* d_native, double* d_binned,
                             int32_t* d_status, int precision, void* d_workspace,
                             size_t workspace_bytes, int autotune, void* stream, tr_graph** out);
/* One replay of the captured forward, enqueued on `stream`. */
int tr_graph_launch(tr_graph* graph, void* stream);
/* The configuration the graph runs: form (0 two-stage, 1 fused), opacity CTAs per SM of the
   two-stage form (0 = as many as fit), fused ring-depth cap (0 = deepest), FP32 contraction
   (3: the 3xTF32 tensor-core kernel, which takes up to 112 layers; 1, 2: the FFMA kernel, one
   CTA per SM with eight or eleven contraction warps; 0: 3 where the layer count fits it, else
   1), the tuned median time in ms (0 when not tuned here) and how many configurations were
   timed.  Any pointer may be NULL. */
int tr_graph_info(const tr_graph* graph, int* form, int* per_sm, int* stages,
                  int* contract_per_sm, float* tuned_ms, int* n_candidates);
void tr_free_graph(tr_graph* graph);
/* Set (pin) or forget the forward configuration the context uses for one batch shape (the
   autotuner's result, or a caller's choice): form 0 two-stage (per_sm opacity CTAs per SM,
   0..3, 0 = as many as fit; contract_per_sm the FP32 contraction, 0..3 as in tr_graph_info;
   3 on more than 112 layers is TR_ERR_UNSUPPORTED) or 1 fused FP32 kernel (stages: ring-depth cap, 0 = deepest).
   native: 1 for native-resolution output, 0 for the binned region of `bins`. */
int tr_pin_forward_config(tr_ctx* ctx, const tr_tables* tables, const tr_batch_desc* desc,
                          int B, const tr_bins* bins, int native, int precision, int form,
                          int per_sm, int stages, int contract_per_sm);
int tr_unpin_forward_config(tr_ctx* ctx, const tr_tables* tables, const tr_batch_desc* desc,
                            int B, const tr_bins* bins, int native, int precision);

/*
 * Batched forward model plus hand-written adjoint (reverse-mode derivative of the same
 * discrete model; the paper has no gradient path: this serves gradient-based samplers and
 * Fisher matrices).  The backward passes reuse the forward's opacity K from the workspace
 * when its K buffer (2 GiB) holds the whole batch and recompute K from the tables when the
 * batch outgrows it.  Outputs, each written when its pointer is not NULL (at least one of
 * d_grad, d_jac):
 *   d_grad[B][n_theta], in one of two modes:
 *     d_gbin != NULL: vector-Jacobian product.  d_gbin[B][n_bin] is an upstream gradient
 *       dL/dD_bin; d_grad[b][k] = sum_j d_gbin[b][j] dD_bin_j/dtheta_k.  d_obs, d_sigma_obs
 *       and d_chi2 are ignored (may be NULL).
 *     d_gbin == NULL: chi^2 mode.  chi^2_b = sum_j ((D_bin_j - obs_j) / sig_j)^2 with
 *       d_obs [n_bin], d_sigma_obs [n_bin] (double, shared by all items); writes d_chi2[B]
 *       and its gradient in d_grad.
 *   d_jac[B][n_bin][n_theta]: the Jacobian dD_bin_j/dtheta_k of every item (double), one
 *     backward pass per bin over the wavenumber tiles of that bin's native range, after the
 *     one forward.  With d_grad == NULL only the Jacobian is computed (d_gbin, d_obs,
 *     d_sigma_obs, d_chi2 are then ignored).
 *   d_binned[B][n_bin] (double) and d_status[B] (int32).
 * Invalid items get zero gradients and Jacobians (and chi^2 = +inf in chi^2 mode).  When
 * neither chi^2 nor d_binned is asked for, the forward runs only its geometry and opacity
 * stages (the backward passes need K, not the spectrum).
 *   recompute_k: 1 recomputes K in the backward pass; 0 or -1 (automatic) reuse the forward's
 *     K when the workspace's K buffer holds the whole batch (recomputing it otherwise).  The
 *     recomputation repeats the forward's arithmetic (the same sums in the same order), so
 *     the choice changes the time, not the results (the GPU tests check bitwise equal
 *     gradients with FP32 tables).
 *   d_workspace: >= tr_batch_workspace_size(..., with_adjoint=1) bytes, or NULL.
 * At most 256 bins; tables with the exponential temperature scheme are refused
 * (TR_ERR_UNSUPPORTED).  Enqueued on `stream`.
 */
int tr_adjoint_transit(tr_ctx* ctx, const tr_tables* tables, const tr_batch_desc* desc, int B,
                       const double* d_theta, const int32_t* d_nlayers, const tr_bins* bins,
                       const double* d_obs, const double* d_sigma_obs, const double* d_gbin,
                       double* d_chi2, double* d_grad, double* d_jac, double* d_binned,
                       int32_t* d_status, int precision, int recompute_k, void* d_workspace,
                       size_t workspace_bytes, void* stream);

/*
 * Batched forward model that allocates nothing (the paper has no counterpart; this is a
 * service to callers that cannot allocate device memory themselves).  Some callers cannot
 * call cudaMalloc or hand the library a workspace: a likelihood callback run by a sampler
 * under a fixed device-memory budget, code that must not trigger the device-wide
 * synchronisation an allocation implies while other streams are busy, or a foreign-language
 * host with no way to own device buffers.  This entry point computes the same binned spectra
 * as tr_forward_transit_batch (FP32 path, binned output only) but takes its scratch from one
 * array of TR_NOALLOC_SCRATCH_BYTES (16 MiB) that lives in the library's device memory.
 *   - The array occupies 16 MiB on every device where the library's module holding it is
 *     loaded, until the process exits.  It is shared by all calls on that device and keeps
 *     the last call's contents; nothing in it needs to start at zero (every word a call reads
 *     was written earlier in the same call).  Calls that overlap on the GPU (other streams,
 *     other host threads, other contexts) race on it: serialise them.
 *   - The first call on a device looks up the array's device address (a one-time set-up per
 *     device, with that device current); make that first call before any stream capture.  The
 *     address is kept for the life of the process: do not call this entry point on a device
 *     after cudaDeviceReset (which invalidates every handle of the library as well).
 *   - The scratch a batch needs is the forward's per-item buffers (layer descriptors,
 *     altitudes, path lengths, annulus weights) and its binned-region depths: the part of
 *     tr_batch_workspace_size(tables, desc, bins, B, 0) that comes before the K buffer,
 *     which this path does not use.  It grows as B x (max_layers^2 + n_in): about 90 KB per
 *     item of 100 layers over the 945 binned wavenumbers of a 10,000-wavenumber grid, so
 *     about 185 such items fit.  A batch that needs more is rejected with TR_ERR_ARG (the
 *     message of tr_last_error gives both sizes); split it into smaller batches.  B above
 *     TR_MAX_BATCH is rejected with TR_ERR_ARG, and a shape whose K tiles and path lengths
 *     the fused FP32 kernel cannot stage in shared memory with TR_ERR_UNSUPPORTED, before
 *     anything is launched.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.  Tables and bins are
 *     inputs prepared earlier; d_theta, d_nlayers, d_binned, d_status are as in
 *     tr_forward_transit_batch.  Kernel timing (tr_profile_*) does not record its launches.
 */
enum { TR_NOALLOC_SCRATCH_BYTES = 16 << 20 };
int tr_forward_transit_batch_noalloc(tr_ctx* ctx, const tr_tables* tables,
                                     const tr_batch_desc* desc, int B, const double* d_theta,
                                     const int32_t* d_nlayers, const tr_bins* bins,
                                     double* d_binned, int32_t* d_status, void* stream);

/*
 * Kernel timing (the library's tracing hook; the paper times whole forward models with
 * timeit, Sec. 8.1).  While enabled, every kernel a context launches is bracketed by CUDA
 * events on the stream it is launched on.  tr_profile_read() waits for those events and
 * returns, per kernel name, the summed device time in ms and the launch count.
 *   tr_profile_enable(ctx, 1) clears the totals and starts recording; 0 stops.
 *   names: max_kernels entries of 48 chars each (NUL-terminated); *n_kernels receives the
 *   number of distinct kernels (may exceed max_kernels; only max_kernels are written).
 */
int tr_profile_enable(tr_ctx* ctx, int on);
int tr_profile_read(tr_ctx* ctx, int max_kernels, char* names, double* total_ms,
                    int64_t* launches, int* n_kernels);

#ifdef __cplusplus
}
#endif
#endif /* TRANSIT_H_ */
