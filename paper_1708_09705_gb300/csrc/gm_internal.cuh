// Internal declarations of libgmead (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gmead.h"

namespace gm {

// ---------------------------------------------------------------- constants
constexpr int kGH = 64;          // Gauss-Hermite nodes of the tilted rule
constexpr int kMaxNodes = 128;   // Gauss-Legendre nodes per sightline (max)
constexpr int kMaxSightlinePoints = 1024;  // points of one sightline (joint predictive, sampler)
constexpr int kMaxPicBlock = 8192;         // stars of one sub-catalogue (dense PIC blocks)
constexpr int kMaxPicInducing = 4096;      // inducing points of the PIC posterior

// Device status flags (OR-ed by kernels, read by the host after a call).
enum : unsigned {
  kFlagNonFinite = 1u,
  kFlagNotSPD = 2u,
  kFlagTimeout = 4u,
  kFlagProbeOverflow = 8u,
  kFlagBadIndex = 16u,
  kFlagHitLimit = 32u,   // a sampler step used up its wall hits
};

// Log-spaced cubic table of g(x), x = r^2 / L0^2.  Segment k >= 0 covers
// [x_lo(k), x_lo(k+1)) with x_lo(k) = 2^(emin + k / 2^m) * (1 + (k mod 2^m)/2^m),
// i.e. 2^m equal sub-intervals per octave; the segment of x is read from the
// exponent and leading mantissa bits of x.  Index n_real holds zeros (g beyond
// 2^emax is below 1e-19 and dropped).  Arguments below 2^emin are clamped
// (the error there is < 1e-10 of g(0)).
struct TableGeom {
  int m;        // log2(segments per octave)
  int emin;     // first octave exponent
  int emax;     // end octave exponent (exclusive)
  __host__ __device__ int n_real() const { return (emax - emin) << m; }
  __host__ __device__ int n_pts() const { return 3 * n_real() + 1; }
};
constexpr TableGeom kTabF32{4, -100, 11};
constexpr TableGeom kTabF64{7, -100, 11};

// ---------------------------------------------------------------- context
struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Workspace;  // solver scratch, see gm_solve.cu
struct Deflation;  // deflation vectors of the variance panels, see gm_deflate.cu
struct PicState;   // factors of the last PIC posterior, see gm_pic.cu
struct PackState;  // packed multi-field panels, see gm_fields.cu

// Per-field cell grid and hyperparameters.  A context holds one field per
// independent problem (sky field / sub-catalogue); stars of different fields
// are never neighbours, so K is block diagonal by field.
struct FieldGrid {
  double ox, oy, oz, inv_cell;  // grid origin, 1 / cell edge (edge >= cutoff)
  double cut2, inv_cut, inv_L0;  // cutoff^2, 1 / cutoff, 1 / outer scale
  int gx, gy, gz, pad;           // cells per axis
  int64_t cell_off;              // id of the field's first cell
};

// Four doubles, 32-byte aligned (one FP64 table segment).
struct alignas(32) D4 {
  double x, y, z, w;
};

}  // namespace gm

struct gm_ctx {
  gm_config cfg{};
  int64_t n = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  gm_allocator alloc{};
  bool has_alloc = false;
  std::string last_error;
  gm_stats stats{};
  int64_t launches = 0;   // kernels launched during the current API call

  // owned device allocations (freed at destroy)
  std::vector<gm::Buffer> owned;

  // ---- stars, internal (spatially sorted) order
  int64_t* perm = nullptr;     // internal -> caller index
  int64_t* iperm = nullptr;    // caller -> internal index (made on first use)
  double* s = nullptr;         // distance
  double* ux = nullptr;        // unit vector components
  double* uy = nullptr;
  double* uz = nullptr;
  double* obs = nullptr;
  double* obs_sigma = nullptr;

  // ---- fields and their cell grids (cell edge >= the field's cutoff)
  int32_t n_fields = 1;
  std::vector<int64_t> h_fptr;    // internal row offset of each field (n_fields + 1)
  std::vector<gm::FieldGrid> h_fgrid;
  int64_t* fptr = nullptr;        // device copy of h_fptr
  gm::FieldGrid* fgrid = nullptr; // device copy of h_fgrid
  int32_t* field_of = nullptr;    // field of each internal star
  int64_t n_cells = 0;
  int32_t* cell_start = nullptr;  // n_cells + 1

  // ---- covariance, CSR over internal order
  bool built = false;
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  void* val = nullptr;         // double (FP64) or float (FP32)
  gm::Buffer col_buf, val_buf;
  int64_t* diag_pos = nullptr;
  // row-block tiles of K (FP32 mode): 32-row blocks that never straddle a
  // field (block b = rows blk_row0[b] .. blk_row0[b+1]-1), union columns, values
  gm::Buffer t_bptr, t_ucol, t_val;
  int64_t t_nblk = 0;
  std::vector<int64_t> h_boff;     // first block of each field (n_fields + 1)
  int64_t* boff = nullptr;         // device copy
  int64_t* blk_row0 = nullptr;     // device, t_nblk + 1
  int64_t t_union = 0;
  // 128-row tiles of K for the tensor-core panel product (single-field FP32):
  // K-step prefix per block, padded union columns, BF16 operand images
  int64_t tc_nblk = 0, tc_nks = 0;
  gm::Buffer tc_kbase, tc_upad, tc_img;
  gm::Buffer tc_planes;             // BF16 planes of the panel PD (async tile product)
  std::vector<int64_t> h_tc_boff;   // first tile block of each field (n_fields + 1)
  gm::Buffer tc_brow0, tc_boffd;    // first row of each block (+ end); device h_tc_boff
  gm::Buffer tc_trow, tc_tpos;      // tile order: row at tile position p, position of row i
  bool tc_order = false;            // tc_trow / tc_tpos in use (else position = row)
  int tc_pf = 0;                    // tuned variant of the tile product (0: untuned) for
                                    // panels wider than one column group (and packed panels)
  int tc_pf_narrow = 0;             // ... for panels of one column group (<= 256 columns)
  double* kdiag = nullptr;
  double* prior_m = nullptr;

  // ---- quadrature tables
  double* gl_zeta = nullptr;   // Q nodes on [0,1]
  double* gl_w = nullptr;      // Q weights (sum 1)
  double* gh_x = nullptr;      // Gauss-Hermite nodes
  double* gh_wx = nullptr;     // weights * exp(x^2)
  double* phi_pts = nullptr;   // phi at table points (hyperparameter-free)
  void* gtab = nullptr;        // cubic coefficients of g (float4 / double4)
  double gtab_sigma2 = -1;
  int gtab_form = -1;

  // ---- covariance surrogate (FP32 parameters, BF16 operand images)
  float* mlp_params = nullptr;
  unsigned char* mlp_img = nullptr;
  unsigned char* mlp_bimg = nullptr;  // transposed weight images of the backward pass
  bool mlp_trained = false;   // parameters set (by training or by the caller)

  // ---- EP state
  double* tau = nullptr;
  double* nu = nullptr;
  double* mu = nullptr;        // posterior mean for (tau, nu) when post_valid
  double* var = nullptr;
  double* alpha = nullptr;     // mu = m + K alpha
  bool post_valid = false;
  int64_t warm_R = 0;          // panel width of saved variance solutions (0 = none)
  int warm_probe = 0;          // those solutions are per colour class (1) or per star (0)

  // ---- probed variances: colour class of each internal star, classes per field
  int32_t* probe_colour = nullptr;
  std::vector<int32_t> h_probe_ncol;
  double probe_factor_done = 0;  // probe_factor the colouring was made for

  // ---- mean function of the density (exponential disc + bump of Sect. 5),
  // set by gm_set_mean_fn / gm_learn_mean; off: constant mean density rho_bar
  bool mean_fn_on = false;
  double mean_theta[5] = {0, 0, 0, 0, 0};  // L, H, rho0, s_bump, A_bump
  double mean_rsun = 0, mean_w = 0;
  gm::Buffer mf_J, mf_gl, mf_part;        // Jacobian, 64-node rule, partials

  // ---- status flags and pinned readback
  unsigned* d_flags = nullptr;
  void* h_pinned = nullptr;    // 64 KB pinned host scratch

  gm::Workspace* ws = nullptr;
  gm::Deflation* defl = nullptr;
  gm::PicState* pic = nullptr;
  gm::PackState* pack = nullptr;

  // ---- optional per-kernel timing (CUDA events on the context stream, or
  // on prof_stream while a private stream is in use)
  bool prof_on = false;
  cudaStream_t prof_stream = nullptr;
  const char* prof_pending = nullptr;
  struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  struct ProfAcc {
    const char* name;
    int64_t launches;
    double ms;
  };
  std::vector<ProfAcc> prof_acc;
};

namespace gm {

// Running sum for per-element dot-product partials.  FP32 panels use a
// compensated (Kahan) FP32 sum: GB300's FP64 pipe is a small fraction of its
// FP32 rate, so one FP64 add per panel element bounded the element-wise
// passes; the compensation keeps the total within a few FP32 ulps whatever
// the number of terms.  FP64 panels keep a plain FP64 sum.
template <typename TV>
struct PartialSum {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct PartialSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace gm

namespace gm {

// ---------------------------------------------------------------- helpers
gm_status set_error(gm_ctx* c, gm_status st, const std::string& msg);
gm_status cuda_fail(gm_ctx* c, cudaError_t e, const char* what);

void* dev_alloc(gm_ctx* c, size_t bytes);            // owned until destroy
void dev_free_now(gm_ctx* c, void* p, size_t bytes);
bool ensure(gm_ctx* c, Buffer& b, size_t bytes);      // grow-only scratch

// Device buffer of one call, released (stream-ordered) when the scope ends,
// error returns included.
struct ScopedDev {
  gm_ctx* c;
  void* p;
  size_t bytes;
  ScopedDev(gm_ctx* ctx, size_t n) : c(ctx), p(dev_alloc(ctx, n)), bytes(n) {}
  ~ScopedDev() {
    if (p) dev_free_now(c, p, bytes);
  }
  struct Adopt {};
  ScopedDev(gm_ctx* ctx, void* ptr, size_t n, Adopt) : c(ctx), p(ptr), bytes(n) {}
  ScopedDev(const ScopedDev&) = delete;
  ScopedDev& operator=(const ScopedDev&) = delete;
};

#define GM_CUDA_CHECK(ctx, expr)                                   \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return ::gm::cuda_fail((ctx), _e, #expr); \
  } while (0)

// Timing hooks: GM_PROF(ctx, "name") before a launch records a start event
// when profiling is on; GM_LAUNCH_CHECK records the matching stop event.
void prof_begin(gm_ctx* c, const char* name);
void prof_end(gm_ctx* c);
void prof_collect(gm_ctx* c);  // after a stream sync: fold records into totals

#define GM_PROF(ctx, name) \
  do {                      \
    if ((ctx)->prof_on) ::gm::prof_begin((ctx), (name)); \
  } while (0)

#define GM_LAUNCH_CHECK(ctx)                                      \
  do {                                                            \
    (ctx)->launches++;                                            \
    if ((ctx)->prof_pending) ::gm::prof_end(ctx);                 \
    cudaError_t _e = cudaGetLastError();                          \
    if (_e != cudaSuccess) return ::gm::cuda_fail((ctx), _e, "kernel launch"); \
  } while (0)

inline int sm_count(gm_ctx* c) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, c->device);
  return v > 0 ? v : 1;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- host rules
// Gauss-Legendre on [-1,1] and Gauss-Hermite (weight exp(-x^2)) by Newton
// iteration on the three-term recurrences (gm_rules.cpp).
void gauss_legendre(int n, double* x, double* w);
void gauss_hermite(int n, double* x, double* w_times_expx2);

// ---------------------------------------------------------------- stages
// field_id: field of each caller star (device, int32) or null (one field).
gm_status geometry_init(gm_ctx* c, const double* l, const double* b,
                        const double* s, const double* obs, const double* sig,
                        const int32_t* field_id, const double* field_L0,
                        const double* field_cut);
// Ascending bitonic sort of n_pad (a power of two >= 1024) 64-bit keys.
gm_status sort_u64(gm_ctx* c, unsigned long long* keys, int64_t n_pad);
// Exclusive scan of n counts: out[0..n], out[n] = total.
gm_status scan_i64(gm_ctx* c, const int64_t* in, int64_t* out, int64_t n);
gm_status unit_vectors(gm_ctx* c, int64_t n, const double* l, const double* b, double* ux,
                       double* uy, double* uz);
// Rows = the given positions (internal stars or queries), columns = stars.
// Counts neighbours within the cutoff of each row, scans to row_ptr (n_rows+1)
// and fills sorted column indices.  `self` marks rows that are the stars
// themselves (diag_pos is then filled).
// row_field: field of each row (null: field 0).
gm_status neighbour_csr(gm_ctx* c, int64_t n_rows, const double* rs,
                        const double* rux, const double* ruy, const double* ruz,
                        const int32_t* row_field, bool self, int64_t* row_ptr,
                        Buffer& col_buf, int64_t* nnz_out, int64_t* diag_pos);
gm_status phi_points_init(gm_ctx* c);
gm_status gtab_update(gm_ctx* c);
// Pair quadrature for CSR entries; symmetric mode computes j >= i and
// mirrors.  Writes values (double or float per precision) and, in symmetric
// mode, K_ii and the prior mean.
gm_status pair_quadrature(gm_ctx* c, int64_t n_rows, const double* rs,
                          const double* rux, const double* ruy, const double* ruz,
                          const int32_t* row_field, const int64_t* row_ptr,
                          const int32_t* col, int64_t nnz, void* val, bool symmetric);
// Quadrature for an explicit pair list (distances, chord): K untapered, FP64 out.
gm_status pairlist_quadrature(gm_ctx* c, int64_t n, const double* si, const double* sj,
                              const double* chord, double* out);
// Copies each lower-triangle entry from its transpose (rows sorted).
gm_status mirror_csr(gm_ctx* c, int64_t n, const int64_t* row_ptr, const int32_t* col, int64_t nnz,
                     void* val);
// Covariance values from the surrogate with quadrature fallback (gm_mlp.cu).
gm_status surrogate_values(gm_ctx* c);
// Diagonal-only quadrature (query self-covariance) into kss (FP64).
gm_status self_quadrature(gm_ctx* c, int64_t n_rows, const double* rs, double* kss);

// Colour classes for probed variances when cfg.probe_factor > 0 (gm_probe.cu).
gm_status probe_colouring(gm_ctx* c);

// 128-row tiles and the tensor-core panel product (gm_tc.cu).
bool tc_wanted(gm_ctx* c);
gm_status tc_tiles_build(gm_ctx* c);
// planes_ready: c->tc_planes already hold the BF16 pieces of PD (written by
// deflate_update_tc) for the asynchronous variant, which then skips its split.
gm_status panel_spmm_tc(gm_ctx* c, int64_t n, int R, const float* dv, const float* P,
                        const float* PD, float* Q, double* part_pq, bool planes_ready = false);
// the tile product's variant for a single panel of R columns (0: not yet tuned)
int tc_variant(gm_ctx* c, int R);
// Packed multi-field panels (no partials); tune = choose the prefetch depth
// (on the context stream, outside any graph capture) instead of launching.
gm_status panel_spmm_tc_packed(gm_ctx* c, int64_t n_items, const int2* items,
                               const int64_t* blk_base, const int32_t* blk_width, const float* dv,
                               const float* P, const float* PD, float* Q, int64_t pd_elems,
                               cudaStream_t st, bool tune);

// Q = B P for an n x R FP32 panel with PD = d o P given (the variance panels'
// product); part: max(tile blocks, ceil(n / 8)) x R doubles of scratch.
gm_status panel_apply_B_f32(gm_ctx* c, int R, const float* dv, const float* P, const float* PD,
                            float* Q, double* part);

// Spectral deflation of the FP32 variance-panel preconditioner (gm_deflate.cu).
gm_status deflate_prepare(gm_ctx* c, const float* dv, const float* minv);
bool deflate_ready(gm_ctx* c);
// C = Y^T R for the panel residuals; corr_row[c] = sum_j w_j C_jc^2
gm_status deflate_rhs(gm_ctx* c, int R, const float* Rr, double* corr_row);
// P = M^-1 R + Yw C + beta P on active columns (all, beta 0 when null), PD = d o P
gm_status deflate_update(gm_ctx* c, int R, int nbx, const float* minv, const float* dv,
                         const double* beta, const int* active, const float* Rr, float* P,
                         float* PD);
// Single right-hand side (posterior-mean CG): c = Y^T r, rz_slot[0] +=
// sum_j w_j c_j^2; then p = M^-1 r + Yw c + beta p, pd = d o p.
gm_status deflate1_rhs(gm_ctx* c, const float* r, double* rz_slot);
gm_status deflate1_update(gm_ctx* c, const float* minv, const float* dv, const double* part,
                          int G, int prev, int next, const float* r, float* p, float* pd);
void deflate_free(gm_ctx* c);
// Tensor-core form of the deflated panel CG step (FP32 panels with tensor-core
// tiles; GM_DEFLATE_TC=0 keeps the CUDA-core kernels above).
bool deflate_tc(gm_ctx* c);
// row chunks of deflate_step_tc for a panel of R columns (its partial rows)
int deflate_tc_chunks(gm_ctx* c, int R);
// alpha non-null: X += alpha P, Rr -= alpha Q and the per-chunk partial sums
// of r^T M^-1 r / r^T r (part_rz / part_rr, nch rows of R); alpha null: Rr
// only.  Then C = Y^T Rr for deflate_update_tc and corr8 (8 rows of R) with
// sum over rows = sum_j w_j C_jc^2.
gm_status deflate_step_tc(gm_ctx* c, int R, int nch, const double* alpha, const float* minv,
                          float* X, float* Rr, const float* P, const float* Q, double* part_rz,
                          double* part_rr, double* corr8);
// P = M^-1 Rr + Yw C + beta P on active columns (all, beta 0 when null); PD =
// d o P in FP32, or (planes) its three BF16 pieces in c->tc_planes.
gm_status deflate_update_tc(gm_ctx* c, int R, const float* minv, const float* dv,
                            const double* beta, const int* active, const float* Rr, float* P,
                            float* PD, bool planes);
// kernels of the tensor-core form (gm_deflate_tc.cu)
size_t dtc_yimg_bytes(int64_t n);
size_t dtc_rowimg_bytes(int64_t n);
size_t dtc_cimg_bytes(int R);
gm_status dtc_images(gm_ctx* c, int64_t n, const float* Y, const float* Yw, void* yimg,
                     void* ywimg);
int dtc_chunks(gm_ctx* c, int64_t n, int R);
gm_status dtc_step(gm_ctx* c, int64_t n, int R, int nch, const void* yimg, const double* alpha,
                   const float* minv, float* X, float* Rr, const float* P, const float* Q,
                   double* part_rz, double* part_rr, float* Cp, const float* w, void* cimg,
                   double* corr8);
gm_status dtc_update(gm_ctx* c, int64_t n, int R, const void* ywimg, const void* cimg,
                     const float* minv, const float* dv, const double* beta, const int* active,
                     const float* Rr, float* P, float* PD, uint16_t* planes);

// Row-block tiles of K for the FP32 variance panels (gm_tiles.cu).
gm_status tiles_build(gm_ctx* c);
gm_status panel_spmm_tiled(gm_ctx* c, int64_t n, int R, int nbx, const float* dv, const float* P,
                           const float* PD, float* Q, double* part_pq);

// Posterior of the current sites: mu, var, alpha (gm_solve.cu).
gm_status refresh_posterior(gm_ctx* c);
// posterior mean only (alpha and mu) for the current sites and prior mean
gm_status posterior_mean_only(gm_ctx* c);
// device status flags -> status (and cleared)
gm_status read_flags(gm_ctx* c);
// prior mean from the mean function at n points: m = ln E[A] - kss/2;
// J (5 columns of n, may be null) = dm / d ln theta  (gm_learn.cu)
gm_status mean_fn_apply(gm_ctx* c, int64_t n, const double* s, const double* ux,
                        const double* uy, const double* uz, const double* kss, double* m,
                        double* J);
// Variances k_rr - v_r^T B^-1 v_r for rows of an arbitrary CSR over stars
// (v_r = S^1/2 k_r); used for the stars themselves and for queries.  With
// pair_cross, the cross terms v_b^T B^-1 v_a of consecutive rows: pairs
// (2p, 2p + 1) when cross_group = 2, else all pairs a < b within groups of
// cross_group rows (a power of two up to 32, dividing the panel width).
gm_status panel_variances(gm_ctx* c, int64_t n_rows, const int64_t* row_ptr,
                          const int32_t* col, const void* val, const double* kdiag_rows,
                          double* var_out, int64_t* iters_out, double* resid_out,
                          double* pair_cross = nullptr, int cross_group = 2);
gm_status csr_dot_alpha(gm_ctx* c, int64_t n_rows, const int64_t* row_ptr,
                        const int32_t* col, const void* val, const double* alpha,
                        const double* base, double* out);

// EP site update over all stars (gm_site.cu).
gm_status site_update(gm_ctx* c, double* max_delta, int64_t* skipped);

void workspace_free(gm_ctx* c);

// PITC / PIC posterior of u at R inducing points (gm_pic.cu): us, ux, uy, uz
// the inducing distances and unit vectors (device), h_block_int the block of
// each internal star (host).  The factors, the posterior mean (R) and
// covariance (R x R) stay in the context (pic_mean, pic_cov) for
// pic_predict.  FP64 single-field contexts with the covariance built.
// Synchronises.
gm_status pic_posterior(gm_ctx* c, int R, const double* us, const double* ux, const double* uy,
                        const double* uz, const int32_t* h_block_int, int nb);
bool pic_ready(gm_ctx* c);
int pic_blocks(gm_ctx* c);
int pic_inducing(gm_ctx* c);
const double* pic_mean(gm_ctx* c);
const double* pic_cov(gm_ctx* c);
void pic_free(gm_ctx* c);
// PIC predictive mean and variance at nq queries (device arrays): geometry,
// block of each query, prior variance kss and mean ms, the queries' CSR over
// the stars (tapered FP64 values).  Synchronises.
gm_status pic_predict(gm_ctx* c, int64_t nq, const double* qs, const double* qx,
                      const double* qy, const double* qz, const int32_t* qblk, const double* kss,
                      const double* ms, const int64_t* qptr, const int32_t* qcol,
                      const double* qval, double* mean, double* var);

// Exact-HMC samples of each sightline's predictive truncated to a
// non-decreasing sequence (gm_sightline.cu).  Device arrays in the caller
// layout of gm_monotone_sample; flags: a device word for kFlagNonFinite,
// kFlagNotSPD and kFlagHitLimit.  Synchronises the stream.
gm_status monotone_sample(gm_ctx* c, int64_t nsl, int m, const double* mean, const double* cov,
                          const double* mom, int n_burn, int n_samples, double* out,
                          int64_t* hits, unsigned* flags);

// Packed per-field variance panels for multi-field contexts (gm_fields.cu).
gm_status panels_fields(gm_ctx* c, const float* dv, const float* minv, const double* d64,
                        double* var_out, int64_t* iters_out, double* resid_out);
void pack_free(gm_ctx* c);
void pack_invalidate(gm_ctx* c);

}  // namespace gm
