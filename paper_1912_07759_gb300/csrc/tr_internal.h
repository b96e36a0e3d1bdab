// tr_internal.h -- internal types shared by the translation units of libtransit.so.
//
// Device data layout (all on one GPU):
//   tables    sigma32 [n_mol][n_p][n_t][wn_pad] float (linear m^2; rows padded with zeros to a
//             multiple of 8 values so every row of the FP32 and FP16 tables starts 16-byte
//             aligned, as TMA tensor maps require)
//             logsig16 [n_mol][n_p][n_t][wn_pad] half, log10 sigma - c_m (mixed precision)
//             cia32   [n_cia][n_t_cia][wn_pad] float, pair q scaled by 2^-e_q (exact power of
//             two; the weight carries 2^e_q) because m^5 values sit below the FP32 range
//             ray32   [n_species][wn_pad] float, species s scaled by 2^-e_s likewise
//   per item  LayerDesc[n_layers]   brackets, weights and cloud opacity of each layer
//             z    [max_layers + 1] FP64 altitudes of the layer boundaries
//             dlt  [max_layers][npad] dense layer-major path lengths: row l (shell) holds
//                  DL[j][l] for rays j = 0..npad-1 (zero for j > l and j >= N), the layout
//                  the contraction keeps in shared memory (one bulk copy per atmosphere)
//             aj   [npad] float annulus weights (r_{j+1}^2 - r_j^2) / R_s^2, zero beyond N
//   npad = max_layers rounded up to a multiple of 8 (the contraction's ray tile)
//             rayc [TR_MAX_SPECIES] float Rayleigh mixing coefficients X_s 2^e_s
//             ItemGeom  (R_p/R_s)^2 in FP64, layer count, status
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>            // CUtensorMap (type only; the encoder comes through the runtime)
#include <cuda_runtime.h>
#include <map>
#include <string>
#include <vector>
#include "../../include/transit.h"

namespace tr {

// SI constants.  CODATA-2018 G, k_B, m_u; R_J as the paper states it (Sec. 8.2).
constexpr double kG = 6.67430e-11;
constexpr double kKB = 1.380649e-23;
constexpr double kAMU = 1.66053906660e-27;
constexpr double kRJup = 6.9911e7;

struct LayerDesc {
  int ip, it, itc;             // P and T brackets (molecules), T bracket (CIA)
  int zone;                    // chemistry zone (0 with constant mixing ratios)
  float rho, tp, tt, ttc;      // number density; interpolation weights in P, T, T (CIA)
  float k_cloud, cloud;        // cloud opacity [1/m] and cloud fraction
  uint16_t pad_s;
  uint8_t flags, pad_c;        // kLayer* bits
  float pad_f;
  float w_mol[TR_MAX_MOL];     // rho X_m (0 when the paper's out-of-range rule zeroes sigma)
  float w_cia[TR_MAX_CIA];     // rho^2 X_a X_b 2^e_q
};
static_assert(sizeof(LayerDesc) == 96, "LayerDesc layout");
// The bilinear corner weights (P_i,T_j) (P_i,T_j+1) (P_i+1,T_j) (P_i+1,T_j+1) of a layer's
// interpolation weights tp, tt (FP32; every kernel that forms them uses this expression).
__host__ __device__ inline void corner_weights(float tp, float tt, float (&cw)[4]) {
  cw[0] = (1.f - tp) * (1.f - tt);
  cw[1] = (1.f - tp) * tt;
  cw[2] = tp * (1.f - tt);
  cw[3] = tp * tt;
}
enum : uint8_t {
  kLayerMolZero = 1,   // the paper's out-of-range rule zeroes the molecular cross-sections
  kLayerTClamp = 2,    // T at or beyond the molecular T grid edge (no T derivative)
  kLayerCiaZero = 4,   // CIA zeroed by the out-of-range rule
  kLayerTcClamp = 8    // T at or beyond the CIA T grid edge
};

struct ItemGeom {
  double rp2_rs2;   // (R_p / R_s)^2
  double r_p;       // m
  double t_surf;    // K: the temperature profile at p_max (the emission model's surface)
  int n_layers;     // 0 when the item is invalid
  int status;
};

// Everything the FP64 geometry kernel needs besides the per-item parameters.
struct GeomParams {
  int n_mol, n_species, n_tnodes, n_p, n_t, n_cia, n_t_cia;
  int gravity_mode, cloud_mode, oor_mode, max_layers, has_ray;
  int interp_mode;                        // TR_INTERP_*
  int t_profile, gas_mode;                // TR_TPROF_*, TR_GAS_*
  int n_chem, n_tpar;                     // theta entries of the chemistry and the T profile
  double t_int, gm_p;                     // Guillot internal temperature (K); G M_p
  int cia_a[TR_MAX_CIA], cia_b[TR_MAX_CIA];
  double cia_scale[TR_MAX_CIA];           // 2^e_q, carried by the CIA weight
  double ray_scale[TR_MAX_SPECIES];       // 2^e_s
  double mass[TR_MAX_SPECIES];
  double fill[TR_MAX_SPECIES];
  double tnode_log10p[TR_MAX_TNODES];
  double p_max, p_min, m_p, r_s, p_cloud_bot, kappa_cloud;
  // batch constants taken on the host: ln p_max, ln p_min, 1 / k_B, 1 / R_s^2,
  // m_u G M_p, sum_f fill_f m_f, the cloud deck's bottom pressure and its ln, and the
  // reciprocal node spacings of the temperature profile
  double ln_pmax, ln_pmin, inv_kb, inv_rs2, amu_g_mp, fill_mass, p_cbot, ln_cbot;
  double inv_dlog10p[TR_MAX_TNODES];      // 1 / (log10 p_{k+1} - log10 p_k) of the T nodes
  const double* p_grid;      // device [n_p]
  const double* t_grid;      // device [n_t]
  const double* t_grid_cia;  // device [n_t_cia]
  const double* inv_dp;      // device [n_p - 1] 1 / (p[i+1] - p[i])
  const double* inv_dt;      // device [n_t - 1]
  const double* inv_dtc;     // device [n_t_cia - 1]
};

// Per-call batch buffers (views into a workspace or a handle's own memory).
struct ItemBuffers {
  LayerDesc* layers;   // [B][max_layers]
  double* z;           // [B][max_layers + 1] altitudes
  double* tl;          // [B][max_layers] layer temperatures (FP64, for the adjoint)
  float* dlp;          // [B][dlp_offset(max_layers)] the same path lengths packed by rows:
                       //   row l at dlp_offset(l) holds rays 0 .. pad8(l+1)-1
  float4* zf;          // [B][max_layers + 1] per boundary k: z_k as double-float (hi, lo),
                       //   2 (r_{k+1}^2 - r_k^2) (0 at k = N) and 2 R_p + z_k, in FP32
  float4* op;          // [B][max_layers][2] opacity coefficients of layer l for cross-sections
                       //   pre-summed over molecules (see opx): [0] = corner weights
                       //   rho x_max w_c (c = (P_i,T_j) (P_i,T_j+1) (P_i+1,T_j) (P_i+1,T_j+1)),
                       //   0 under the out-of-range zero rule (with the exponential T scheme:
                       //   rho x_max (1 - t_P), rho x_max t_P, the exponential T weight u and
                       //   the linear T weight t); [1] = (CIA weights
                       //   rho^2 y_max (1 - t), rho^2 y_max t; rho; cloud opacity)
  float* opx;          // [B][kMaxZones][kOpxStride] x_m / x_max (m < TR_MAX_MOL), then
                       //   y_q / y_max with y_q = X_a X_b 2^e_q (q < TR_MAX_CIA): the weights of
                       //   the sums in each chemistry zone (zone 0 only for constant mixing
                       //   ratios; LayerDesc::zone names a layer's)
  float* dlt;          // [B][max_layers][npad] path lengths, layer-major dense
  float* aj;           // [B][npad]
  float* rayc;         // [B][kMaxZones][TR_MAX_SPECIES] X_s 2^e_s per chemistry zone
  ItemGeom* items;     // [B]
  int npad;            // max_layers rounded up to a multiple of 8
  int zoned;           // 1 when mixing ratios vary with height (two-layer gases): layers
                       //   carry a zone index and the opacity sums change with it
};

__host__ __device__ inline int pad8(int n) { return (n + 7) & ~7; }

// Programmatic dependent launch.  A kernel launched by launch_dependent may start while the
// kernel before it in the stream is still running (once every CTA of that kernel has called
// pdl_trigger, or exited); it must call pdl_wait before it reads anything earlier work wrote
// (pdl_wait returns once the kernels it depends on have completed and their writes are
// visible, and at once for a kernel launched normally).  Only the launch and the set-up
// before pdl_wait overlap the predecessor.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Packed FP32 pairs (fma.rn.f32x2, sm_100 and later): one instruction performs two FP32 FMAs,
// each rounded as fmaf, so results equal those of scalar FMAs in the same order while the
// issue slots per FMA halve.  pack_dup puts x in both halves of a pair.
__device__ __forceinline__ unsigned long long pack_dup(float x) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void ffma2(unsigned long long& acc, unsigned long long a,
                                      unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
#endif
constexpr int kOpxStride = 16;   // floats of per-item opacity weights (TR_MAX_MOL + TR_MAX_CIA, padded)
// Chemistry zones of a two-layer atmosphere: runs of layers with the same mixing ratios.  Each
// absorber is below, straddling or above its switch (0, 1, 2), monotone with height; the sum
// of the states names the zone (the same sum on two layers means the same states).
constexpr int kMaxZones = 2 * TR_MAX_MOL + 1;
static_assert(TR_MAX_MOL + TR_MAX_CIA <= kOpxStride, "per-item opacity weights fit their stride");

// Launchers (stream-ordered; return cudaGetLastError()).
// k_profile (per-atmosphere set-up: everything the opacity kernels read), k_altitude (the
// hydrostatic altitudes and annulus weights, from the inputs k_profile leaves in the altitude
// rows) and k_pathlen (path lengths); launch_geometry runs the three in order.
cudaError_t launch_profile(const GeomParams& gp, int B, const double* d_theta, int n_theta,
                           const int32_t* d_nlayers, int32_t* d_status, ItemBuffers buf,
                           cudaStream_t s);
cudaError_t launch_altitude(const GeomParams& gp, int B, ItemBuffers buf, cudaStream_t s);
cudaError_t launch_pathlen(const GeomParams& gp, int B, ItemBuffers buf, cudaStream_t s);
cudaError_t launch_geometry(const GeomParams& gp, int B, const double* d_theta, int n_theta,
                            const int32_t* d_nlayers, int32_t* d_status, ItemBuffers buf,
                            cudaStream_t s);

// First table column of a computed native range [wn_begin, ...): the range start rounded down
// to a multiple of 8 values (16 bytes of FP16), the alignment TMA tile loads need.  Column
// tiles of every forward and adjoint kernel start here.
__host__ __device__ inline int wn_first(int wn_begin) { return wn_begin & ~7; }

// Wavenumbers per CTA of the TMA-staged opacity kernel (one per thread): the inner box size of
// the tables' tensor maps.
constexpr int kOpacityTile = 256;
// Wavenumbers per work unit of the fused forward kernel (the inner box of its tensor maps).
constexpr int kFusedTile = 128;

// Offset of row l in the packed path-length layout (row l holds rays 0 .. pad8(l+1)-1):
// sum_{k<l} pad8(k+1) = 8 (q+1)(4q + r) with l = 8q + r.
__host__ __device__ inline int dlp_offset(int l) {
  const int q = l >> 3, r = l & 7;
  return 8 * (q + 1) * (4 * q + r);
}

struct FwdParams {
  const float* sigma; int n_mol, n_p, n_t, wn_pad;
  const float* cia; int n_cia, n_t_cia;
  const float* ray; int n_species;
  int max_layers;
  ItemBuffers buf;
  int wn_begin, wn_count;     // computed native range
  double* out; long long out_stride;   // out[b * out_stride + (wn - wn_begin)]
  int* dev_err;               // device error word (TR_DEVERR_* bits), set on a bounded-wait timeout
  int b_off;                  // first item of a chunked launch (grid item index + b_off)
  const void* logsig16;       // FP16 log10 sigma tables (mixed opacity), or NULL
  float logsig_off[TR_MAX_MOL];
  int interp_mode;            // TR_INTERP_* of the tables
};
enum { TR_DEVERR_TIMEOUT = 1 };
// Two-stage form: streaming opacity kernel writing K for a chunk of items to kbuf, then the
// contraction + depth kernel.  kbuf holds forward_kbuf_bytes(...) bytes: the K of
// forward_chunk_items(...) items, processed chunk by chunk.
size_t forward_kbuf_bytes(int B, int max_layers, int wn_begin, int wn_count);
// Columns of a K row in the buffer: the range [wn_first(wn_begin), wn_begin + wn_count) rounded
// up to the contraction's 128-wavenumber tiles; K of chunk item c, layer l, column x is at
// kbuf[(c * max_layers + l) * kcols + x].
long long forward_kcols(int wn_begin, int wn_count);
int forward_chunk_items(int B, int max_layers, int wn_begin, int wn_count);
// Opacity of items [p.b_off, p.b_off + Bc): FP32 tables, or the FP16 log tables when
// p.logsig16 is set (decoded on the fly).  tm_sig / tm_cia: tensor maps of the table in use
// and of the CIA table (boxes {kOpacityTile, 2, 2, n_mol} and {kOpacityTile, 2, n_cia}).
// per_sm_cap: at most this many CTAs per SM (0: up to 3, as registers allow); the ring of
// each takes the shared memory the others leave.
cudaError_t launch_opacity(const FwdParams& p, const CUtensorMap* tm_sig,
                           const CUtensorMap* tm_cia, int Bc, float* kbuf, int per_sm_cap,
                           cudaStream_t s);
// The FP32 path's contraction + depth for items [p.b_off, p.b_off + Bc) reading K.  `kind`:
// kContractTC the 3xTF32 tensor-core kernel (tc_fp32.cu; layer counts up to 112),
// kContractFfma8 / kContractFfma11 the FFMA kernel with eight or eleven contraction warps (one
// persistent CTA per SM, up to three K-tile slots), kContractAuto the tensor-core kernel when
// the layer count fits it, else the FFMA kernel with eight warps.
enum { kContractAuto = 0, kContractFfma8 = 1, kContractFfma11 = 2, kContractTC = 3 };
int contract_kind(int requested, int max_layers);     // the kind kContractAuto resolves to
// tiles: the path-length tiles of every item of the batch (tc_dl_bytes, written by
// launch_dl_tf32), needed by kContractTC
cudaError_t launch_contract_fp32(const FwdParams& p, int Bc, const float* kbuf, int kind,
                                 const void* tiles, cudaStream_t s);
bool tc_contract_fits(int max_layers);
size_t tc_dl_bytes(int B, int max_layers);            // TF32 hi/lo path-length tiles of B items
cudaError_t launch_dl_tf32(const ItemBuffers& buf, int B, int max_layers, void* tiles,
                           cudaStream_t s);
cudaError_t launch_contract_tc(const FwdParams& p, int Bc, const float* kbuf, const void* tiles,
                               cudaStream_t s);
// Fused FP32 forward (fused.cu): TMA-staged opacity into double-buffered shared-memory K
// tiles, contraction and depth in one persistent warp-specialized kernel (one CTA per SM);
// needs no K buffer.  stages_cap: ring depth limit (0 = the deepest ring that fits); `used`
// (may be NULL) receives the configuration launched.  fused_forward_fits: whether the kernel's
// shared memory holds at least one K tile, one copy of the path lengths and a ring of at least
// 2 stages for these table, layer and batch sizes.
struct FusedChoice { int k_bufs, stages; };
bool fused_forward_fits(int n_mol, int n_cia, int max_layers, int B);
cudaError_t launch_forward_fused(const FwdParams& p, const CUtensorMap* tm_sig,
                                 const CUtensorMap* tm_cia, int B, int stages_cap,
                                 FusedChoice* used, cudaStream_t s);

struct BinsDev {
  int n_bin, i0, i1;          // native range [i0, i1) with weight
  const int* row_ptr;         // [n_bin + 1] into col/w
  const int* col;             // native index
  const double* w;            // weight w_ij
  const double* inv_wsum;     // [n_bin] 1 / sum_i w_ij
  // transpose for the adjoint: native i0 + k has entries t_ptr[k] .. t_ptr[k+1] of
  // (t_bin, t_w = w_ij / sum_i w_ij)
  const int* t_ptr;           // [i1 - i0 + 1]
  const int* t_bin;
  const double* t_w;
  const int* lo;              // [n_bin] native index of each bin's first entry (consecutive)
};
// A kernel whose only wait can never complete; it must give up and set the error word.
cudaError_t launch_wait_selftest(int* err, long long polls, cudaStream_t s);
// binned[b][j] = inv_wsum[j] * sum w_ij depth[b][col - base]
cudaError_t launch_bin(const BinsDev& bd, int B, const double* depth, long long depth_stride,
                       int depth_base, double* binned, cudaStream_t s);
// out[b][j] = inv_wsum[j] * sqrt(sum (w_ij sigma[b][col - base])^2)
cudaError_t launch_bin_sigma(const BinsDev& bd, int B, const double* sigma, long long stride,
                             int base, double* out, cudaStream_t s);
// SNR instrument model: noise = max_j binned[b][j] / snr / sqrt(n_obs); obs = binned + noise z
cudaError_t launch_snr(int B, int n_bin, const double* binned, double snr, int n_obs,
                       const double* z, double* obs, double* sigma, cudaStream_t s);

}  // namespace tr

struct tr_ctx;
struct tr_tables;
struct tr_bins;

struct TrLogOffsets { float c[TR_MAX_MOL]; };   // per-molecule offsets c_m of the FP16 tables

namespace tr {
// mixed.cu: FP16 log10 sigma tables and the mixed-precision forward path
int build_fp16_log_tables(tr_ctx* ctx, tr_tables* t);
size_t mixed_dl_bytes(int B, int max_layers);   // BF16 hi/lo path-length tiles of B items
// Path-length tile scratch of a two-stage forward of B items in `precision` (the mixed path's
// BF16 tiles, or the FP32 path's TF32 tiles when its tensor-core contraction applies).
size_t dl_tile_bytes(int B, int max_layers, int precision);
// BF16 hi/lo path-length tiles of all B items into dl16 (mixed_dl_bytes).
cudaError_t launch_dl_bf16(const ItemBuffers& buf, int B, int max_layers, void* dl16, cudaStream_t s);
// Contraction on tcgen05 tensor cores + depth for items [p.b_off, p.b_off + Bc) reading K.
cudaError_t launch_contract_umma(const FwdParams& p, int Bc, const float* kbuf, const void* dl16,
                                 cudaStream_t s);
// adjoint.cu: extra workspace of the adjoint
size_t adjoint_extra_bytes(const tr_tables* t, const tr_batch_desc* d, const tr_bins* bins, int B);
// The batched forward's second branch: the path-length kernels (which only the contraction
// reads) run on the context's auxiliary stream beside the opacity kernel.  prepare_batch
// records the fork event after the profile kernel and leaves the path-length kernel pending;
// run_forward issues it (and the path-length tile kernel) on the auxiliary stream, which
// waits for the fork event, right after the first opacity launch, and joins before the first
// kernel that reads path lengths (an event on the auxiliary stream that the caller's stream
// waits for).  A form without an opacity kernel runs the pending kernel on the caller's
// stream.  join_fork closes a branch still open, so every call leaves the caller's stream
// joined (a captured graph has no dangling branch).
struct Fork {
  cudaStream_t aux = nullptr;
  bool open = false, pending = false;
  GeomParams gp{};
  int B = 0;
  ItemBuffers buf{};
};
// Creates the auxiliary stream and its events on first use; false when that fails (the
// forward then runs on the caller's stream alone).
bool fork_ready(tr_ctx* ctx, Fork* f);
// Issues the pending path-length kernel: on the branch (detached) or on s.
cudaError_t fork_start(tr_ctx* ctx, Fork* f, cudaStream_t s, bool detached);
void join_fork(tr_ctx* ctx, Fork* f, cudaStream_t s);
// api.cu: geometry of a batch into a workspace (shared by the forward and adjoint calls)
// n_in: wavenumbers of the per-item depth scratch (0 when depths go to a caller buffer);
// fork (may be NULL): run the path-length kernel on fork->aux after the profile kernel
int prepare_batch(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d, int n_in,
                  size_t need_bytes, int B, const double* d_theta, const int32_t* d_nlayers,
                  int32_t* d_status, void* ws, size_t ws_bytes, cudaStream_t s,
                  ItemBuffers* buf_out, double** depth_out, char** extra_out,
                  Fork* fork = nullptr);
// size of the forward part of a batch workspace (item buffers + depth scratch)
size_t forward_workspace_bytes(int B, int max_layers, int n_in);
int set_error(tr_ctx* ctx, int code, const std::string& msg);
// kbuf: buffer of forward_kbuf_bytes() for the two-stage form (items processed in chunks);
// mixed precision needs it, the fused FP32 kernel does not.
// dl16: scratch of dl_tile_bytes() (path-length tiles of the tensor-core contractions); the
// FP32 path falls back to its FFMA contraction without it.
// How run_forward computes a forward (the autotuner's search space): for FP32 the two-stage
// kernels (the default when kbuf is given; also used when the fused kernel's shared memory
// does not fit) or the fused kernel (without kbuf, or when `choice` asks for it); mixed
// precision always takes the two-stage form (tensor-core contraction).  per_sm: CTAs per SM of
// the two-stage opacity kernel (0 = as many as fit, up to 3); stages: ring depth cap of the
// fused kernel (0 = the deepest that fits); contract_per_sm: the FP32 two-stage contraction
// (launch_contract_fp32's kind).
enum { kFormTwoStage = 0, kFormFused = 1 };
struct ForwardChoice { int form, per_sm, stages, contract_per_sm; };
int run_forward(tr_ctx* ctx, const tr_tables* t, int max_layers, const ItemBuffers& buf, int B,
                int wn_begin, int wn_count, double* out, long long stride, int precision,
                cudaStream_t s, float* kbuf = nullptr, void* dl16 = nullptr,
                const ForwardChoice* choice = nullptr, bool opacity_only = false,
                Fork* fork = nullptr);

// Batched forward (tr_forward_transit_batch) with an explicit configuration (NULL: defaults),
// its argument checks, workspace size and the autotuner's key of its shape.
int forward_batch_impl(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d, int B,
                       const double* d_theta, const int32_t* d_nlayers, const tr_bins* bins,
                       double* d_native, double* d_binned, int32_t* d_status, int precision,
                       void* ws, size_t ws_bytes, cudaStream_t s, const ForwardChoice* choice);
int check_forward_batch_args(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d, int B,
                             const double* d_theta, const tr_bins* bins, const double* d_native,
                             const double* d_binned);
size_t forward_batch_need(const tr_tables* t, const tr_batch_desc* d, int B, const tr_bins* bins,
                          bool native, int precision);
std::string batch_shape_key(const tr_tables* t, const tr_batch_desc* d, int B,
                            const tr_bins* bins, bool native, int precision);
int run_bin(tr_ctx* ctx, const tr_bins* bins, int B, const double* depth, long long stride,
            int base, double* binned, cudaStream_t s);
int ensure_scratch(tr_ctx* ctx, size_t bytes);


// 2-D FP32 tensor map (rows of `cols` floats, `row_stride_bytes` apart) with box
// {box_cols, box_rows}; out-of-range box elements read as zero.  False when encoding fails.
bool encode_2d_f32(CUtensorMap* m, const void* base, unsigned long long cols,
                   unsigned long long rows, unsigned long long row_stride_bytes,
                   unsigned box_cols, unsigned box_rows);

// api.cu helpers shared with other translation units
ItemBuffers carve_forward_workspace(void* base, int B, int max_layers, int n_in, double** depth);
int validate_batch_desc(tr_ctx* ctx, const tr_tables* t, const tr_batch_desc* d);
GeomParams batch_geom_params(const tr_tables* t, const tr_batch_desc* d);
// Length of a batch item's parameter vector (chemistry | temperature | R_p | log10 P_top).
int batch_n_theta(const tr_tables* t, const tr_batch_desc* d);
FwdParams forward_fp32_params(const tr_tables* t, int max_layers, const ItemBuffers& buf,
                              int wn_begin, int wn_count, double* out, long long stride,
                              int* dev_err);

// Brackets one kernel launch with CUDA events on its stream while the context's kernel
// timing is enabled (tr_profile_enable); a no-op otherwise.
class KernelTimer {
 public:
  KernelTimer(tr_ctx* ctx, const char* name, cudaStream_t s);
  ~KernelTimer();
 private:
  tr_ctx* ctx_;
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};
}  // namespace tr

// ------------------------------------------------------------------------------ handles
struct tr_ctx {
  int device = 0;
  std::string err;
  int* dev_err = nullptr;     // device error word written by kernels on a bounded-wait timeout
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  // kernel timing
  struct Pending { const char* name; cudaEvent_t a, b; };
  bool prof_on = false;
  std::vector<Pending> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  std::map<std::string, std::pair<double, long long>> prof_totals;
  // autotuner results: batch shape -> fastest forward configuration found on this context
  std::map<std::string, tr::ForwardChoice> tuned;
  // the batched forward's auxiliary stream (highest priority) and its fork / join events
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

struct tr_tables {
  int device = 0;
  int n_mol = 0, n_p = 0, n_t = 0, n_wn = 0, wn_pad = 0;
  int n_cia = 0, n_t_cia = 0, n_species = 0, storage = 0, oor_mode = 0;
  int interp_mode = 0;                     // TR_INTERP_*
  int has_ray = 0;
  int cia_a[TR_MAX_CIA] = {}, cia_b[TR_MAX_CIA] = {};
  double cia_scale[TR_MAX_CIA] = {};
  double ray_scale[TR_MAX_SPECIES] = {};
  double mass[TR_MAX_SPECIES] = {};
  double* h_wn = nullptr;                  // host copy of the native grid
  double* d_wn = nullptr;                  // device copy of the native grid
  float* d_sigma = nullptr;
  float* d_cia = nullptr;
  float* d_ray = nullptr;
  double* d_p_grid = nullptr;
  double* d_t_grid = nullptr;
  double* d_t_grid_cia = nullptr;
  double* d_inv_dp = nullptr;              // 1 / grid spacings (P, T, CIA T)
  double* d_inv_dt = nullptr;
  double* d_inv_dtc = nullptr;
  uint16_t* d_logsig16 = nullptr;          // fp16 bits of log10 sigma - c_m
  float logsig_offset[TR_MAX_MOL] = {};    // c_m
  // TMA tensor maps (encoded at load): FP32 sigma, FP16 log10 sigma and CIA with inner box
  // kOpacityTile wavenumbers (two-stage opacity), FP32 sigma and CIA with inner box
  // kFusedTile (fused forward)
  CUtensorMap tm_sig32{};
  CUtensorMap tm_sig16{};
  CUtensorMap tm_cia{};
  CUtensorMap tm_sig32_f{};
  CUtensorMap tm_cia_f{};
  size_t device_bytes = 0;
};

struct tr_atm {
  int device = 0;
  int n_layers = 0;
  void* mem = nullptr;      // one allocation holding the item buffers
  tr::ItemBuffers buf{};
  double rp2_rs2 = 0.0;
};

struct tr_bins {
  int device = 0;
  tr::BinsDev dev{};
  void* mem = nullptr;
  std::vector<int> bin_lo, bin_hi;   // native range [bin_lo[j], bin_hi[j]) of bin j (host)
};
