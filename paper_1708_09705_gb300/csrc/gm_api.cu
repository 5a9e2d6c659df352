// C ABI of libgmead (declared in include/gmead.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

gm_status set_error(gm_ctx* c, gm_status st, const std::string& msg) {
  if (c) c->last_error = std::string(gm_status_str(st)) + ": " + msg;
  return st;
}

gm_status cuda_fail(gm_ctx* c, cudaError_t e, const char* what) {
  if (c) c->last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GM_E_NOMEM : GM_E_CUDA;
}

void* dev_alloc(gm_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->has_alloc) {
    p = c->alloc.alloc(bytes, (void*)c->stream, c->alloc.user);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->owned.push_back(Buffer{p, bytes});
  return p;
}

static void raw_free(gm_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (c->has_alloc)
    c->alloc.free(p, bytes, (void*)c->stream, c->alloc.user);
  else
    cudaFreeAsync(p, c->stream);
}

void dev_free_now(gm_ctx* c, void* p, size_t bytes) {
  for (size_t k = 0; k < c->owned.size(); ++k) {
    if (c->owned[k].p == p) {
      c->owned.erase(c->owned.begin() + k);
      break;
    }
  }
  raw_free(c, p, bytes);
}

bool ensure(gm_ctx* c, Buffer& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return true;
  if (b.p) dev_free_now(c, b.p, b.bytes);
  b.p = dev_alloc(c, bytes);
  b.bytes = b.p ? bytes : 0;
  return b.p != nullptr;
}

// ---------------------------------------------------------------- timing
static cudaEvent_t prof_event(gm_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void prof_begin(gm_ctx* c, const char* name) {
  if (c->prof_pending) prof_end(c);  // two launches before one check
  cudaEvent_t a = prof_event(c), b = prof_event(c);
  if (!a || !b) return;
  cudaEventRecord(a, c->prof_stream ? c->prof_stream : c->stream);
  c->prof_recs.push_back({name, a, b});
  c->prof_pending = name;
}

void prof_end(gm_ctx* c) {
  if (!c->prof_recs.empty())
    cudaEventRecord(c->prof_recs.back().b, c->prof_stream ? c->prof_stream : c->stream);
  c->prof_pending = nullptr;
}

void prof_collect(gm_ctx* c) {
  if (c->prof_recs.empty()) return;
  cudaEventSynchronize(c->prof_recs.back().b);
  for (auto& r : c->prof_recs) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0;
    }
    bool found = false;
    for (auto& acc : c->prof_acc)
      if (std::strcmp(acc.name, r.name) == 0) {
        acc.launches++;
        acc.ms += ms;
        found = true;
        break;
      }
    if (!found) c->prof_acc.push_back({r.name, 1, (double)ms});
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_recs.clear();
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copies n doubles from a host or device pointer into device memory.
static gm_status copy_in(gm_ctx* c, double* dst, const void* src, size_t bytes) {
  cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(dst, src, bytes, k, c->stream));
  return GM_OK;
}

// Copies device data out to a host or device pointer and waits.
static gm_status copy_out(gm_ctx* c, void* dst, const void* src, size_t bytes) {
  cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(dst, src, bytes, k, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  return GM_OK;
}

gm_status read_flags(gm_ctx* c) {
  unsigned* h = (unsigned*)c->h_pinned;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                   c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  unsigned f = *h;
  if (f) GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream));
  if (f & kFlagNonFinite) return set_error(c, GM_E_NONFINITE, "non-finite value in a kernel");
  if (f & kFlagNotSPD)
    return set_error(c, GM_E_NOT_SPD, "CG found p^T B p <= 0: covariance not positive definite");
  if (f & kFlagTimeout) return set_error(c, GM_E_TIMEOUT, "bounded device wait expired");
  return GM_OK;
}

// element-wise kernels for the API layer
__global__ void k_scatter_ext(int64_t n, const int64_t* __restrict__ perm,
                              const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[perm[k]] = src[k];
}
__global__ void k_invert_perm(int64_t n, const int64_t* __restrict__ perm,
                              int64_t* __restrict__ iperm) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    iperm[perm[k]] = k;
}

// Stored K_ij for caller index pairs: binary search of the internal column
// of j in the internal row of i (columns are sorted); 0 when not stored.
template <typename TA>
__global__ void k_entries(int64_t nq, int64_t n, const int64_t* __restrict__ qi,
                          const int64_t* __restrict__ qj, const int64_t* __restrict__ iperm,
                          const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                          const TA* __restrict__ val, double* __restrict__ out,
                          unsigned* __restrict__ flags) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = qi[q], b = qj[q];
    if (a < 0 || a >= n || b < 0 || b >= n) {
      out[q] = NAN;
      atomicOr(flags, kFlagBadIndex);
      continue;
    }
    const int64_t r = iperm[a];
    const int32_t cj = (int32_t)iperm[b];
    int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
    double v = 0.0;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      const int32_t cm = col[mid];
      if (cm == cj) {
        v = (double)val[mid];
        break;
      }
      if (cm < cj) lo = mid + 1; else hi = mid;
    }
    out[q] = v;
  }
}

__global__ void k_scatter_i32(int64_t n, const int64_t* __restrict__ perm,
                              const int32_t* __restrict__ src, int32_t* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[perm[k]] = src[k];
}

__global__ void k_gather_ext(int64_t n, const int64_t* __restrict__ perm,
                             const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[perm[k]];
}

__global__ void k_check_inputs(int64_t n, const double* __restrict__ s,
                               const double* __restrict__ obs, const double* __restrict__ sig,
                               const double* __restrict__ l, const double* __restrict__ b,
                               unsigned* __restrict__ bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    bool ok = isfinite(s[k]) && s[k] > 0 && isfinite(obs[k]) && isfinite(sig[k]) && sig[k] > 0 &&
              isfinite(l[k]) && isfinite(b[k]);
    if (!ok) atomicOr(bad, 1u);
  }
}

__global__ void k_check_sites(int64_t n, const double* __restrict__ tau,
                              const double* __restrict__ nu, unsigned* __restrict__ bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    if (!(isfinite(tau[k]) && tau[k] >= 0 && isfinite(nu[k]))) atomicOr(bad, 1u);
}

template <typename T>
__global__ void k_to_double(int64_t n, const T* __restrict__ src, double* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = (double)src[k];
}

__global__ void k_query_mean(int64_t n, double log_rho_bar, int form, double sigma2,
                             const double* __restrict__ s, const double* __restrict__ kss,
                             double* __restrict__ m) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    m[k] = log_rho_bar + log(s[k]) - (form == GM_FORM_LOGNORMAL ? 0.5 * kss[k] : 0.5 * sigma2);
}

static int eb(gm_ctx* c, int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * sm_count(c)));
}

static gm_status validate(const gm_config* f) {
  if (!(f->sigma2 > 0) || !(f->outer_scale_pc > 0) || !(f->rho_bar > 0) || !(f->cutoff_pc > 0))
    return GM_E_INVAL;
  if (!std::isfinite(f->sigma2) || !std::isfinite(f->outer_scale_pc) ||
      !std::isfinite(f->rho_bar) || !std::isfinite(f->cutoff_pc))
    return GM_E_INVAL;
  if (f->n_nodes < 2 || f->n_nodes > kMaxNodes) return GM_E_INVAL;
  if (f->form != GM_FORM_LOGNORMAL && f->form != GM_FORM_LINEAR) return GM_E_INVAL;
  if (f->taper != GM_TAPER_WENDLAND && f->taper != GM_TAPER_HARD) return GM_E_INVAL;
  if (f->precision != GM_PREC_FP64 && f->precision != GM_PREC_FP32) return GM_E_INVAL;
  if (f->likelihood != GM_LIK_GAUSS_IN_A && f->likelihood != GM_LIK_GAUSS_IN_LNA)
    return GM_E_INVAL;
  if (!(f->damping > 0 && f->damping <= 1)) return GM_E_INVAL;
  if (!(f->vc_floor >= 0) || !(f->cg_tol > 0) || f->cg_max_iter <= 0) return GM_E_INVAL;
  if (f->rhs_panel < 0 || (f->warm_start != 0 && f->warm_start != 1)) return GM_E_INVAL;
  if (f->cov_source != GM_COV_QUADRATURE && f->cov_source != GM_COV_SURROGATE) return GM_E_INVAL;
  if (f->quad_rule != GM_QUAD_GL && f->quad_rule != GM_QUAD_BAND) return GM_E_INVAL;
  if (f->tc_products != 0 && f->tc_products != 3 && f->tc_products != 6) return GM_E_INVAL;
  if (!(f->surrogate_gate > 0)) return GM_E_INVAL;
  if (!(f->probe_factor >= 0) || !std::isfinite(f->probe_factor)) return GM_E_INVAL;
  if (f->deflate != 0 && f->deflate != 64) return GM_E_INVAL;
  return GM_OK;
}

}  // namespace gm

using namespace gm;

extern "C" {

void gm_config_default(gm_config* f) {
  if (!f) return;
  std::memset(f, 0, sizeof(*f));
  f->sigma2 = 1.0;
  f->outer_scale_pc = 20.0;
  f->rho_bar = 1e-3;
  f->cutoff_pc = 60.0;
  f->n_nodes = 32;
  f->form = GM_FORM_LOGNORMAL;
  f->taper = GM_TAPER_WENDLAND;
  f->precision = GM_PREC_FP64;
  f->likelihood = GM_LIK_GAUSS_IN_A;
  f->cg_max_iter = 2000;
  f->damping = 1.0;
  f->vc_floor = 1e-8;
  f->cg_tol = 1e-10;
  f->rhs_panel = 0;
  f->warm_start = 1;
  f->cov_source = GM_COV_QUADRATURE;
  f->surrogate_gate = 1e-4;
  f->quad_rule = GM_QUAD_BAND;  // the converged rule; workloads name their own
  f->tc_products = 6;
}

const char* gm_status_str(gm_status s) {
  switch (s) {
    case GM_OK: return "GM_OK";
    case GM_E_INVAL: return "GM_E_INVAL";
    case GM_E_NOMEM: return "GM_E_NOMEM";
    case GM_E_CUDA: return "GM_E_CUDA";
    case GM_E_NOT_SPD: return "GM_E_NOT_SPD";
    case GM_E_NOCONV: return "GM_E_NOCONV";
    case GM_E_NONFINITE: return "GM_E_NONFINITE";
    case GM_E_TIMEOUT: return "GM_E_TIMEOUT";
    case GM_E_STATE: return "GM_E_STATE";
  }
  return "GM_E_UNKNOWN";
}

const char* gm_last_error(gm_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

void* gm_stream(gm_ctx* c) { return c ? (void*)c->stream : nullptr; }

gm_status gm_ep_init_fields(gm_ctx** out, const gm_config* cfg, int64_t n, const double* l,
                            const double* b, const double* s, const double* obs,
                            const double* obs_sigma, int32_t n_fields, const int32_t* field_id,
                            const double* field_L0, const double* field_cutoff, void* stream,
                            const gm_allocator* alloc) {
  if (!out || !cfg) return GM_E_INVAL;
  *out = nullptr;
  if (n < 1 || n >= (1ll << 31) || !l || !b || !s || !obs || !obs_sigma) return GM_E_INVAL;
  if (validate(cfg) != GM_OK) return GM_E_INVAL;
  if (n_fields < 1 || n_fields > (1 << 20) || (n_fields > 1 && !field_id)) return GM_E_INVAL;
  // several fields: FP32 panels and the quadrature source only
  if (n_fields > 1 && (cfg->precision != GM_PREC_FP32 || cfg->cov_source != GM_COV_QUADRATURE))
    return GM_E_INVAL;
  for (int32_t f = 0; field_L0 && f < n_fields; ++f)
    if (!(field_L0[f] > 0) || !std::isfinite(field_L0[f])) return GM_E_INVAL;
  for (int32_t f = 0; field_cutoff && f < n_fields; ++f)
    if (!(field_cutoff[f] > 0) || !std::isfinite(field_cutoff[f])) return GM_E_INVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return GM_E_INVAL;
  gm_ctx* c = new (std::nothrow) gm_ctx();
  if (!c) return GM_E_NOMEM;
  c->cfg = *cfg;
  c->n = n;
  c->n_fields = n_fields;
  c->stream = (cudaStream_t)stream;
  if (alloc) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  c->stats.n_stars = n;
  gm_status st = GM_OK;
  auto fail = [&](gm_status e) {
    *out = c;  // keep the context so that the caller can read gm_last_error
    return e;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(cuda_fail(c, cudaGetLastError(), "cudaGetDevice"));
  if (cudaMallocHost(&c->h_pinned, 1 << 16) != cudaSuccess)
    return fail(cuda_fail(c, cudaGetLastError(), "cudaMallocHost"));
  const size_t nb = (size_t)n * sizeof(double);
  c->perm = (int64_t*)dev_alloc(c, (size_t)n * sizeof(int64_t));
  for (double** p : {&c->s, &c->ux, &c->uy, &c->uz, &c->obs, &c->obs_sigma, &c->tau, &c->nu,
                     &c->mu, &c->var, &c->alpha, &c->kdiag, &c->prior_m})
    *p = (double*)dev_alloc(c, nb);
  c->row_ptr = (int64_t*)dev_alloc(c, (size_t)(n + 1) * sizeof(int64_t));
  c->diag_pos = (int64_t*)dev_alloc(c, (size_t)n * sizeof(int64_t));
  c->d_flags = (unsigned*)dev_alloc(c, 16);
  c->gl_zeta = (double*)dev_alloc(c, kMaxNodes * sizeof(double));
  c->gl_w = (double*)dev_alloc(c, kMaxNodes * sizeof(double));
  c->gh_x = (double*)dev_alloc(c, kGH * sizeof(double));
  c->gh_wx = (double*)dev_alloc(c, kGH * sizeof(double));
  for (void* p : {(void*)c->perm, (void*)c->s, (void*)c->tau, (void*)c->prior_m, (void*)c->row_ptr,
                  (void*)c->diag_pos, (void*)c->d_flags, (void*)c->gl_zeta, (void*)c->gh_wx,
                  (void*)c->ux, (void*)c->uy, (void*)c->uz, (void*)c->obs, (void*)c->obs_sigma,
                  (void*)c->nu, (void*)c->mu, (void*)c->var, (void*)c->alpha, (void*)c->kdiag,
                  (void*)c->gl_w, (void*)c->gh_x})
    if (!p) return fail(set_error(c, GM_E_NOMEM, "context arrays"));
  if (cudaMemsetAsync(c->d_flags, 0, 16, c->stream) != cudaSuccess)
    return fail(cuda_fail(c, cudaGetLastError(), "memset"));
  // quadrature rules
  {
    std::vector<double> x(c->cfg.n_nodes), w(c->cfg.n_nodes), z(c->cfg.n_nodes), v(c->cfg.n_nodes);
    gauss_legendre(c->cfg.n_nodes, x.data(), w.data());
    for (int q = 0; q < c->cfg.n_nodes; ++q) {
      z[q] = 0.5 * (1.0 + x[q]);
      v[q] = 0.5 * w[q];
    }
    std::vector<double> hx(kGH), hw(kGH);
    gauss_hermite(kGH, hx.data(), hw.data());
    double* hp = (double*)c->h_pinned;
    std::memcpy(hp, z.data(), z.size() * sizeof(double));
    std::memcpy(hp + 128, v.data(), v.size() * sizeof(double));
    std::memcpy(hp + 256, hx.data(), kGH * sizeof(double));
    std::memcpy(hp + 384, hw.data(), kGH * sizeof(double));
    cudaMemcpyAsync(c->gl_zeta, hp, z.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->gl_w, hp + 128, v.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->gh_x, hp + 256, kGH * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->gh_wx, hp + 384, kGH * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
      return fail(cuda_fail(c, cudaGetLastError(), "rule upload"));
  }
  // inputs (caller order) -> device scratch
  double* in[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  const double* src[5] = {l, b, s, obs, obs_sigma};
  for (int k = 0; k < 5; ++k) {
    in[k] = (double*)dev_alloc(c, nb);
    if (!in[k]) return fail(set_error(c, GM_E_NOMEM, "input staging"));
    st = copy_in(c, in[k], src[k], nb);
    if (st != GM_OK) return fail(st);
  }
  GM_PROF(c, "k_check_inputs");
  k_check_inputs<<<eb(c, n), 256, 0, c->stream>>>(n, in[2], in[3], in[4], in[0], in[1], c->d_flags);
  {
    unsigned* h = (unsigned*)c->h_pinned;
    cudaMemcpyAsync(h, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
      return fail(cuda_fail(c, cudaGetLastError(), "input check"));
    if (*h) return fail(set_error(c, GM_E_INVAL, "non-finite input, s <= 0 or obs_sigma <= 0"));
  }
  int32_t* fid = nullptr;
  if (n_fields > 1) {
    fid = (int32_t*)dev_alloc(c, (size_t)n * sizeof(int32_t));
    if (!fid) return fail(set_error(c, GM_E_NOMEM, "field ids"));
    cudaMemcpyKind k = is_device_ptr(field_id) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(fid, field_id, (size_t)n * sizeof(int32_t), k, c->stream) != cudaSuccess)
      return fail(cuda_fail(c, cudaGetLastError(), "field ids"));
  }
  st = geometry_init(c, in[0], in[1], in[2], in[3], in[4], fid, field_L0, field_cutoff);
  if (st != GM_OK) return fail(st);
  if (fid) dev_free_now(c, fid, (size_t)n * sizeof(int32_t));
  for (int k = 4; k >= 0; --k) dev_free_now(c, in[k], nb);
  st = phi_points_init(c);
  if (st != GM_OK) return fail(st);
  cudaMemsetAsync(c->tau, 0, nb, c->stream);
  cudaMemsetAsync(c->nu, 0, nb, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(cuda_fail(c, cudaGetLastError(), "init"));
  *out = c;
  return GM_OK;
}

gm_status gm_ep_init(gm_ctx** out, const gm_config* cfg, int64_t n, const double* l,
                     const double* b, const double* s, const double* obs,
                     const double* obs_sigma, void* stream, const gm_allocator* alloc) {
  return gm_ep_init_fields(out, cfg, n, l, b, s, obs, obs_sigma, 1, nullptr, nullptr, nullptr,
                           stream, alloc);
}

gm_status gm_build_cov(gm_ctx* c, int64_t* nnz_out) {
  if (!c) return GM_E_INVAL;
  c->launches = 0;
  pic_free(c);  // factors of a PIC posterior over the previous K
  gm_status st = neighbour_csr(c, c->n, c->s, c->ux, c->uy, c->uz, c->field_of, true, c->row_ptr,
                               c->col_buf, &c->nnz, c->diag_pos);
  if (st != GM_OK) return st;
  c->col = (int32_t*)c->col_buf.p;
  const size_t vs = c->cfg.precision == GM_PREC_FP32 ? sizeof(float) : sizeof(double);
  if (!ensure(c, c->val_buf, std::max<int64_t>(c->nnz, 1) * vs))
    return set_error(c, GM_E_NOMEM, "CSR values");
  c->val = c->val_buf.p;
  if (c->cfg.cov_source == GM_COV_SURROGATE) {
    st = surrogate_values(c);
  } else {
    st = pair_quadrature(c, c->n, c->s, c->ux, c->uy, c->uz, c->field_of, c->row_ptr, c->col, c->nnz,
                         c->val, true);
  }
  if (st != GM_OK) return st;
  if (c->mean_fn_on) {  // the prior mean from the mean function of the density
    st = mean_fn_apply(c, c->n, c->s, c->ux, c->uy, c->uz, c->kdiag, c->prior_m, nullptr);
    if (st != GM_OK) return st;
  }
  c->t_nblk = 0;
  c->tc_nblk = 0;
  c->warm_R = 0;
  pack_invalidate(c);
  st = tc_wanted(c) ? tc_tiles_build(c) : tiles_build(c);
  if (st != GM_OK) return st;
  st = probe_colouring(c);
  if (st != GM_OK) return st;
  st = read_flags(c);
  if (st != GM_OK) return st;
  prof_collect(c);
  c->built = true;
  c->post_valid = false;
  c->stats.nnz = c->nnz;
  c->stats.n_pairs = (c->nnz + c->n) / 2;
  c->stats.kernel_launches = c->launches;
  if (nnz_out) *nnz_out = c->nnz;
  return GM_OK;
}

gm_status gm_ep_sweep(gm_ctx* c, int32_t n_sweeps, double tol, int32_t* sweeps_done,
                      double* max_delta) {
  if (!c || n_sweeps < 0) return GM_E_INVAL;
  if (!c->built) return set_error(c, GM_E_STATE, "gm_build_cov must precede gm_ep_sweep");
  c->launches = 0;
  int done = 0;
  double delta = 0;
  for (; done < n_sweeps;) {
    gm_status st = GM_OK;
    if (!c->post_valid) {
      st = refresh_posterior(c);
      if (st == GM_OK) st = read_flags(c);
      if (st != GM_OK) return st;
    }
    int64_t skipped = 0;
    st = site_update(c, &delta, &skipped);
    if (st == GM_OK) st = read_flags(c);
    if (st != GM_OK) return st;
    prof_collect(c);
    c->post_valid = false;
    c->stats.sites_skipped = skipped;
    c->stats.last_max_delta = delta;
    ++done;
    if (tol > 0 && delta < tol) break;
  }
  c->stats.kernel_launches = c->launches;
  if (sweeps_done) *sweeps_done = done;
  if (max_delta) *max_delta = delta;
  return GM_OK;
}

static gm_status ensure_posterior(gm_ctx* c) {
  if (!c->built) return set_error(c, GM_E_STATE, "gm_build_cov must come first");
  if (c->post_valid) return GM_OK;
  gm_status st = refresh_posterior(c);
  if (st == GM_OK) st = read_flags(c);
  return st;
}

gm_status gm_get_posterior(gm_ctx* c, double* mean_out, double* var_out) {
  if (!c) return GM_E_INVAL;
  c->launches = 0;
  gm_status st = ensure_posterior(c);
  if (st != GM_OK) return st;
  double* tmp = (double*)dev_alloc(c, 2 * c->n * sizeof(double));
  if (!tmp) return set_error(c, GM_E_NOMEM, "posterior staging");
  GM_PROF(c, "k_scatter_ext");
  k_scatter_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->mu, tmp);
  GM_PROF(c, "k_scatter_ext");
  k_scatter_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->var, tmp + c->n);
  GM_LAUNCH_CHECK(c);
  if (mean_out && (st = copy_out(c, mean_out, tmp, c->n * sizeof(double))) != GM_OK) return st;
  if (var_out && (st = copy_out(c, var_out, tmp + c->n, c->n * sizeof(double))) != GM_OK) return st;
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  dev_free_now(c, tmp, 2 * c->n * sizeof(double));
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}

gm_status gm_get_prior(gm_ctx* c, double* mean_out, double* kdiag_out) {
  if (!c) return GM_E_INVAL;
  if (!c->built) return set_error(c, GM_E_STATE, "gm_build_cov must come first");
  double* tmp = (double*)dev_alloc(c, 2 * c->n * sizeof(double));
  if (!tmp) return set_error(c, GM_E_NOMEM, "prior staging");
  GM_PROF(c, "k_scatter_ext");
  k_scatter_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->prior_m, tmp);
  GM_PROF(c, "k_scatter_ext");
  k_scatter_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->kdiag, tmp + c->n);
  GM_LAUNCH_CHECK(c);
  gm_status st;
  if (mean_out && (st = copy_out(c, mean_out, tmp, c->n * sizeof(double))) != GM_OK) return st;
  if (kdiag_out && (st = copy_out(c, kdiag_out, tmp + c->n, c->n * sizeof(double))) != GM_OK) return st;
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  dev_free_now(c, tmp, 2 * c->n * sizeof(double));
  return GM_OK;
}

gm_status gm_get_sites(gm_ctx* c, double* tau_out, double* nu_out) {
  if (!c) return GM_E_INVAL;
  double* tmp = (double*)dev_alloc(c, 2 * c->n * sizeof(double));
  if (!tmp) return set_error(c, GM_E_NOMEM, "site staging");
  GM_PROF(c, "k_scatter_ext");
  k_scatter_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->tau, tmp);
  GM_PROF(c, "k_scatter_ext");
  k_scatter_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->nu, tmp + c->n);
  GM_LAUNCH_CHECK(c);
  gm_status st;
  if (tau_out && (st = copy_out(c, tau_out, tmp, c->n * sizeof(double))) != GM_OK) return st;
  if (nu_out && (st = copy_out(c, nu_out, tmp + c->n, c->n * sizeof(double))) != GM_OK) return st;
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  dev_free_now(c, tmp, 2 * c->n * sizeof(double));
  return GM_OK;
}

gm_status gm_set_sites(gm_ctx* c, const double* tau, const double* nu) {
  if (!c || !tau || !nu) return GM_E_INVAL;
  const size_t nb = c->n * sizeof(double);
  double* tmp = (double*)dev_alloc(c, 2 * nb);
  if (!tmp) return set_error(c, GM_E_NOMEM, "site staging");
  gm_status st = copy_in(c, tmp, tau, nb);
  if (st == GM_OK) st = copy_in(c, tmp + c->n, nu, nb);
  if (st != GM_OK) return st;
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags + 1, 0, sizeof(unsigned), c->stream));
  GM_PROF(c, "k_check_sites");
  k_check_sites<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, tmp, tmp + c->n, c->d_flags + 1);
  GM_LAUNCH_CHECK(c);
  unsigned* h = (unsigned*)c->h_pinned;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  if (*h) {
    dev_free_now(c, tmp, 2 * nb);
    return set_error(c, GM_E_INVAL, "sites must be finite with tau >= 0");
  }
  GM_PROF(c, "k_gather_ext");
  k_gather_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, tmp, c->tau);
  GM_PROF(c, "k_gather_ext");
  k_gather_ext<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, tmp + c->n, c->nu);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  dev_free_now(c, tmp, 2 * nb);
  c->post_valid = false;
  c->warm_R = 0;
  return GM_OK;
}

gm_status gm_get_perm(gm_ctx* c, int64_t* perm_out) {
  if (!c || !perm_out) return GM_E_INVAL;
  return copy_out(c, perm_out, c->perm, c->n * sizeof(int64_t));
}

gm_status gm_get_csr(gm_ctx* c, int64_t* row_ptr_out, int32_t* col_out, double* val_out) {
  if (!c) return GM_E_INVAL;
  if (!c->built) return set_error(c, GM_E_STATE, "gm_build_cov must come first");
  gm_status st;
  if (row_ptr_out && (st = copy_out(c, row_ptr_out, c->row_ptr, (c->n + 1) * sizeof(int64_t))) != GM_OK)
    return st;
  if (col_out && (st = copy_out(c, col_out, c->col, c->nnz * sizeof(int32_t))) != GM_OK) return st;
  if (val_out) {
    double* tmp = (double*)dev_alloc(c, std::max<int64_t>(c->nnz, 1) * sizeof(double));
    if (!tmp) return set_error(c, GM_E_NOMEM, "CSR staging");
    GM_PROF(c, "k_to_double");
    if (c->cfg.precision == GM_PREC_FP32)
      k_to_double<float><<<eb(c, c->nnz), 256, 0, c->stream>>>(c->nnz, (const float*)c->val, tmp);
    else
      k_to_double<double><<<eb(c, c->nnz), 256, 0, c->stream>>>(c->nnz, (const double*)c->val, tmp);
    GM_LAUNCH_CHECK(c);
    st = copy_out(c, val_out, tmp, c->nnz * sizeof(double));
    dev_free_now(c, tmp, std::max<int64_t>(c->nnz, 1) * sizeof(double));
    if (st != GM_OK) return st;
  }
  return GM_OK;
}

gm_status gm_get_entries(gm_ctx* c, int64_t nq, const int64_t* i, const int64_t* j,
                         double* out) {
  if (!c || nq < 0 || (nq > 0 && (!i || !j || !out))) return GM_E_INVAL;
  if (!c->built) return set_error(c, GM_E_STATE, "gm_build_cov must come first");
  if (nq == 0) return GM_OK;
  c->launches = 0;
  if (!c->iperm) {
    c->iperm = (int64_t*)dev_alloc(c, c->n * sizeof(int64_t));
    if (!c->iperm) return set_error(c, GM_E_NOMEM, "inverse permutation");
    GM_PROF(c, "k_invert_perm");
    k_invert_perm<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->iperm);
    GM_LAUNCH_CHECK(c);
  }
  const size_t ib = nq * sizeof(int64_t);
  unsigned char* tmp = (unsigned char*)dev_alloc(c, 2 * ib + nq * sizeof(double));
  if (!tmp) return set_error(c, GM_E_NOMEM, "entry staging");
  int64_t* di = (int64_t*)tmp;
  int64_t* dj = (int64_t*)(tmp + ib);
  double* dout = (double*)(tmp + 2 * ib);
  gm_status st;
  if ((st = copy_in(c, (double*)di, i, ib)) != GM_OK || (st = copy_in(c, (double*)dj, j, ib)) != GM_OK)
    return st;
  GM_PROF(c, "k_entries");
  if (c->cfg.precision == GM_PREC_FP32)
    k_entries<float><<<eb(c, nq), 256, 0, c->stream>>>(nq, c->n, di, dj, c->iperm, c->row_ptr,
                                                       c->col, (const float*)c->val, dout,
                                                       c->d_flags);
  else
    k_entries<double><<<eb(c, nq), 256, 0, c->stream>>>(nq, c->n, di, dj, c->iperm, c->row_ptr,
                                                        c->col, (const double*)c->val, dout,
                                                        c->d_flags);
  GM_LAUNCH_CHECK(c);
  if ((st = copy_out(c, out, dout, nq * sizeof(double))) != GM_OK) return st;
  unsigned* h = (unsigned*)c->h_pinned;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                   c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  dev_free_now(c, tmp, 2 * ib + nq * sizeof(double));
  if (*h & kFlagBadIndex) {
    GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream));
    return set_error(c, GM_E_INVAL, "star index out of range");
  }
  return GM_OK;
}

gm_status gm_get_probe_colours(gm_ctx* c, int32_t* colour_out) {
  if (!c || !colour_out) return GM_E_INVAL;
  if (!c->built || !c->probe_colour || c->probe_factor_done <= 0)
    return set_error(c, GM_E_STATE, "no probing colouring (probe_factor 0 or no gm_build_cov)");
  c->launches = 0;
  int32_t* tmp = (int32_t*)dev_alloc(c, c->n * sizeof(int32_t));
  if (!tmp) return set_error(c, GM_E_NOMEM, "colour staging");
  GM_PROF(c, "k_scatter_i32");
  k_scatter_i32<<<eb(c, c->n), 256, 0, c->stream>>>(c->n, c->perm, c->probe_colour, tmp);
  GM_LAUNCH_CHECK(c);
  gm_status st = copy_out(c, colour_out, tmp, c->n * sizeof(int32_t));
  if (st != GM_OK) return st;
  dev_free_now(c, tmp, c->n * sizeof(int32_t));
  return GM_OK;
}

gm_status gm_get_stats(gm_ctx* c, gm_stats* out) {
  if (!c || !out) return GM_E_INVAL;
  *out = c->stats;
  out->tile_variant = c->tc_nblk > 0 ? c->tc_pf : 0;
  return GM_OK;
}

// Predictive means and variances at nq device-resident points (ql, qb, qs);
// with pair_cross, rows (2p, 2p + 1) are pairs and pair_cross[p] receives
// v_{2p+1}^T B^-1 v_{2p} (cross_group = 2), or rows come in groups of
// cross_group and pair_cross receives every pair a < b of each group.
static gm_status predict_points(gm_ctx* c, int64_t nq, const double* ql, const double* qb,
                                const double* qs, double* mean, double* var,
                                double* pair_cross, int cross_group = 2) {
  const size_t nb = nq * sizeof(double);
  // query work arrays: ux, uy, uz, kss, mq (released on every return)
  ScopedDev bq(c, 5 * nb), bqp(c, (nq + 1) * sizeof(int64_t));
  double* q = (double*)bq.p;
  int64_t* qptr = (int64_t*)bqp.p;
  if (!q || !qptr) return set_error(c, GM_E_NOMEM, "query arrays");
  double *ux = q, *uy = q + nq, *uz = q + 2 * nq, *kss = q + 3 * nq, *mq = q + 4 * nq;
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags + 1, 0, sizeof(unsigned), c->stream));
  GM_PROF(c, "k_check_inputs");
  k_check_inputs<<<eb(c, nq), 256, 0, c->stream>>>(nq, qs, qs, qs, ql, qb, c->d_flags + 1);
  GM_LAUNCH_CHECK(c);
  {
    unsigned* h = (unsigned*)c->h_pinned;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (*h) return set_error(c, GM_E_INVAL, "query distances must be finite and > 0");
  }
  gm_status st = unit_vectors(c, nq, ql, qb, ux, uy, uz);
  if (st != GM_OK) return st;
  Buffer qcol;
  int64_t qnnz = 0;
  st = neighbour_csr(c, nq, qs, ux, uy, uz, nullptr, false, qptr, qcol, &qnnz, nullptr);
  if (st != GM_OK) return st;
  ScopedDev bqc(c, qcol.p, qcol.bytes, ScopedDev::Adopt{});
  const size_t vs = c->cfg.precision == GM_PREC_FP32 ? sizeof(float) : sizeof(double);
  ScopedDev bqv(c, std::max<int64_t>(qnnz, 1) * vs);
  void* qval = bqv.p;
  if (!qval) return set_error(c, GM_E_NOMEM, "query values");
  st = pair_quadrature(c, nq, qs, ux, uy, uz, nullptr, qptr, (const int32_t*)qcol.p, qnnz, qval,
                       false);
  if (st == GM_OK) st = self_quadrature(c, nq, qs, kss);
  if (st != GM_OK) return st;
  // prior mean at the queries
  // m_q = ln(rho_bar s_q) - k_qq/2 (lognormal) or - sigma2/2 (linear)
  if (c->mean_fn_on) {
    st = mean_fn_apply(c, nq, qs, ux, uy, uz, kss, mq, nullptr);
    if (st != GM_OK) return st;
  } else {
    GM_PROF(c, "k_query_mean");
    k_query_mean<<<eb(c, nq), 256, 0, c->stream>>>(nq, std::log(c->cfg.rho_bar), c->cfg.form,
                                                   c->cfg.sigma2, qs, kss, mq);
    GM_LAUNCH_CHECK(c);
  }
  st = csr_dot_alpha(c, nq, qptr, (const int32_t*)qcol.p, qval, c->alpha, mq, mean);
  if (st != GM_OK) return st;
  int64_t it = 0;
  double res = 0;
  c->warm_R = 0;  // the query panels overwrite the saved star solutions
  st = panel_variances(c, nq, qptr, (const int32_t*)qcol.p, qval, kss, var, &it, &res,
                       pair_cross, cross_group);
  if (st == GM_OK) st = read_flags(c);
  if (st != GM_OK) return st;
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  return GM_OK;
}

gm_status gm_predict(gm_ctx* c, int64_t nq, const double* l, const double* b, const double* s,
                     double* mean_out, double* var_out) {
  if (!c || nq < 0 || (nq > 0 && (!l || !b || !s || !mean_out || !var_out))) return GM_E_INVAL;
  if (c->n_fields > 1)
    return set_error(c, GM_E_STATE, "prediction needs a single-field context");
  if (nq == 0) return GM_OK;
  c->launches = 0;
  gm_status st = ensure_posterior(c);
  if (st != GM_OK) return st;
  const size_t nb = nq * sizeof(double);
  ScopedDev buf(c, 5 * nb);  // l, b, s, mean, var
  double* q = (double*)buf.p;
  if (!q) return set_error(c, GM_E_NOMEM, "query arrays");
  double *ql = q, *qb = q + nq, *qs = q + 2 * nq, *mean = q + 3 * nq, *var = q + 4 * nq;
  if ((st = copy_in(c, ql, l, nb)) != GM_OK || (st = copy_in(c, qb, b, nb)) != GM_OK ||
      (st = copy_in(c, qs, s, nb)) != GM_OK)
    return st;
  st = predict_points(c, nq, ql, qb, qs, mean, var, nullptr);
  if (st != GM_OK) return st;
  if ((st = copy_out(c, mean_out, mean, nb)) != GM_OK) return st;
  if ((st = copy_out(c, var_out, var, nb)) != GM_OK) return st;
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}

// Pair points: (l, b, s) at row 2q, (l, b, s + ds) at row 2q + 1; and the
// pair's own quadrature inputs (s, s + ds, chord 0).
__global__ void k_pair_points(int64_t nq, double ds, const double* __restrict__ l,
                              const double* __restrict__ b, const double* __restrict__ s,
                              double* __restrict__ l2, double* __restrict__ b2,
                              double* __restrict__ s2, double* __restrict__ si,
                              double* __restrict__ sj, double* __restrict__ ch) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    l2[2 * q] = l2[2 * q + 1] = l[q];
    b2[2 * q] = b2[2 * q + 1] = b[q];
    s2[2 * q] = s[q];
    s2[2 * q + 1] = s[q] + ds;
    si[q] = s[q];
    sj[q] = s[q] + ds;
    ch[q] = 0.0;
  }
}

// E[exp(c^T a) 1{d^T a > 0}] for a ~ N(mu, S), 2-vectors (completing the square)
__device__ __forceinline__ double trunc_exp(double m1, double m2, double s11, double s22,
                                            double s12, double c1, double c2) {
  const double mx = c1 * m1 + c2 * m2;
  const double vx = c1 * c1 * s11 + 2.0 * c1 * c2 * s12 + c2 * c2 * s22;
  const double md = m2 - m1;
  const double vd = s11 + s22 - 2.0 * s12;
  const double cxd = (c1 - c2) * s12 + c2 * s22 - c1 * s11;  // Cov(c^T a, a2 - a1)
  return exp(mx + 0.5 * vx) * normcdf((md + cxd) / sqrt(vd));
}

// Joint 2 x 2 posterior of each pair and the pseudo-density moments of
// (A2 - A1) / ds given A2 > A1 (Sect. 5): mean_out[2q..], cov_out[3q..]
// (var near, var far, cov), dens_out[2q..] (mean, variance).
__global__ void k_pair_density(int64_t nq, double ds, double inv_cut, int taper,
                               const double* __restrict__ mean, const double* __restrict__ var,
                               const double* __restrict__ cross, const double* __restrict__ k12u,
                               double* __restrict__ cov_out, double* __restrict__ dens_out,
                               unsigned* __restrict__ flags) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double h = ds * inv_cut;
    double w = h <= 1.0 ? 1.0 : 0.0;
    if (taper == GM_TAPER_WENDLAND) {
      const double u = 1.0 - h;
      w = h < 1.0 ? u * u * u * u * (4.0 * h + 1.0) : 0.0;
    }
    const double m1 = mean[2 * q], m2 = mean[2 * q + 1];
    const double s11 = var[2 * q], s22 = var[2 * q + 1];
    const double s12 = w * k12u[q] - cross[q];
    cov_out[3 * q] = s11;
    cov_out[3 * q + 1] = s22;
    cov_out[3 * q + 2] = s12;
    const double vd = s11 + s22 - 2.0 * s12;
    double dm = NAN, dv = NAN;
    if (vd > 0) {
      const double pd = normcdf((m2 - m1) / sqrt(vd));
      const double e1 = trunc_exp(m1, m2, s11, s22, s12, 1.0, 0.0);
      const double e2 = trunc_exp(m1, m2, s11, s22, s12, 0.0, 1.0);
      const double e11 = trunc_exp(m1, m2, s11, s22, s12, 2.0, 0.0);
      const double e22 = trunc_exp(m1, m2, s11, s22, s12, 0.0, 2.0);
      const double e12 = trunc_exp(m1, m2, s11, s22, s12, 1.0, 1.0);
      const double mo1 = (e2 - e1) / pd, mo2 = (e22 - 2.0 * e12 + e11) / pd;
      dm = mo1 / ds;
      dv = (mo2 - mo1 * mo1) / (ds * ds);
    }
    if (!isfinite(dm) || !isfinite(dv)) atomicOr(flags, kFlagNonFinite);
    dens_out[2 * q] = dm;
    dens_out[2 * q + 1] = dv;
  }
}

gm_status gm_predict_pairs(gm_ctx* c, int64_t nq, const double* l, const double* b,
                           const double* s, double ds, double* mean_out, double* cov_out,
                           double* dens_out) {
  if (!c || nq < 0 || !(ds > 0) || !std::isfinite(ds) ||
      (nq > 0 && (!l || !b || !s || !mean_out || !cov_out || !dens_out)))
    return GM_E_INVAL;
  if (c->n_fields > 1)
    return set_error(c, GM_E_STATE, "prediction needs a single-field context");
  if (nq == 0) return GM_OK;
  c->launches = 0;
  gm_status st = ensure_posterior(c);
  if (st != GM_OK) return st;
  const size_t nb = nq * sizeof(double);
  // l, b, s (nq); l2, b2, s2, mean, var (2 nq); si, sj, ch, k12, cross (nq);
  // cov (3 nq), dens (2 nq)
  ScopedDev buf(c, 23 * nb);
  double* q = (double*)buf.p;
  if (!q) return set_error(c, GM_E_NOMEM, "pair arrays");
  double *ql = q, *qb = q + nq, *qs = q + 2 * nq, *l2 = q + 3 * nq, *b2 = q + 5 * nq,
         *s2 = q + 7 * nq, *mean = q + 9 * nq, *var = q + 11 * nq, *si = q + 13 * nq,
         *sj = q + 14 * nq, *ch = q + 15 * nq, *k12 = q + 16 * nq, *cross = q + 17 * nq,
         *cov = q + 18 * nq, *dens = q + 21 * nq;
  if ((st = copy_in(c, ql, l, nb)) != GM_OK || (st = copy_in(c, qb, b, nb)) != GM_OK ||
      (st = copy_in(c, qs, s, nb)) != GM_OK)
    return st;
  GM_PROF(c, "k_pair_points");
  k_pair_points<<<eb(c, nq), 256, 0, c->stream>>>(nq, ds, ql, qb, qs, l2, b2, s2, si, sj, ch);
  GM_LAUNCH_CHECK(c);
  st = predict_points(c, 2 * nq, l2, b2, s2, mean, var, cross);
  if (st == GM_OK) st = pairlist_quadrature(c, nq, si, sj, ch, k12);
  if (st != GM_OK) return st;
  GM_PROF(c, "k_pair_density");
  k_pair_density<<<eb(c, nq), 256, 0, c->stream>>>(nq, ds, 1.0 / c->cfg.cutoff_pc, c->cfg.taper,
                                                   mean, var, cross, k12, cov, dens, c->d_flags);
  GM_LAUNCH_CHECK(c);
  if ((st = read_flags(c)) != GM_OK) return st;
  if ((st = copy_out(c, mean_out, mean, 2 * nb)) != GM_OK) return st;
  if ((st = copy_out(c, cov_out, cov, 3 * nb)) != GM_OK) return st;
  if ((st = copy_out(c, dens_out, dens, 2 * nb)) != GM_OK) return st;
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}

// Index of the pair (a, c), a < c, among the m (m - 1) / 2 pairs of one
// sightline in row-major order.
__host__ __device__ inline int64_t sl_pair_index(int m, int a, int c) {
  return (int64_t)a * m - (int64_t)a * (a + 1) / 2 + (c - a - 1);
}

// Pair points of every sightline: pair p = (q, a, c) has rows 2p (point a)
// and 2p + 1 (point c) and quadrature inputs (s_a, s_c, chord 0).  Flags a
// sightline whose distances do not increase.
__global__ void k_sl_pairs(int64_t nsl, int m, const double* __restrict__ l,
                           const double* __restrict__ b, const double* __restrict__ s,
                           double* __restrict__ l2, double* __restrict__ b2,
                           double* __restrict__ s2, double* __restrict__ si,
                           double* __restrict__ sj, double* __restrict__ ch,
                           unsigned* __restrict__ bad) {
  const int64_t npq = (int64_t)m * (m - 1) / 2;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nsl * npq;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = p / npq;
    int64_t k = p - q * npq;
    int a = 0;
    while (k >= m - 1 - a) {
      k -= m - 1 - a;
      ++a;
    }
    const int c = a + 1 + (int)k;
    const double sa = s[q * m + a], sc = s[q * m + c];
    if (!(sc > sa)) atomicOr(bad, 1u);
    l2[2 * p] = l2[2 * p + 1] = l[q];
    b2[2 * p] = b2[2 * p + 1] = b[q];
    s2[2 * p] = sa;
    s2[2 * p + 1] = sc;
    si[p] = sa;
    sj[p] = sc;
    ch[p] = 0.0;
  }
}

// Joint predictive of each sightline from its pairs: entry (a, c) of the
// covariance is W(|s_c - s_a| / cutoff) k(s_a, s_c) - v_c^T B^-1 v_a, the
// diagonal and the means come from a pair holding the point.
__global__ void k_sl_assemble(int64_t nsl, int m, double inv_cut, int taper,
                              const double* __restrict__ s, const double* __restrict__ mean2,
                              const double* __restrict__ var2, const double* __restrict__ cross,
                              const double* __restrict__ k12u, double* __restrict__ mean_out,
                              double* __restrict__ cov_out) {
  const int64_t npq = (int64_t)m * (m - 1) / 2;
  const int64_t mm = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nsl * mm;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / mm;
    const int r = (int)(e - q * mm);
    const int a = r / m, c = r - a * m;
    if (a == c) {
      const bool near = a < m - 1;
      const int64_t p = q * npq + (near ? sl_pair_index(m, a, a + 1) : sl_pair_index(m, m - 2, m - 1));
      const int64_t row = near ? 2 * p : 2 * p + 1;
      cov_out[e] = var2[row];
      mean_out[q * m + a] = mean2[row];
    } else {
      const int lo = a < c ? a : c, hi = a < c ? c : a;
      const int64_t p = q * npq + sl_pair_index(m, lo, hi);
      const double h = (s[q * m + hi] - s[q * m + lo]) * inv_cut;
      double w = h <= 1.0 ? 1.0 : 0.0;
      if (taper == GM_TAPER_WENDLAND) {
        const double u = 1.0 - h;
        w = h < 1.0 ? u * u * u * u * (4.0 * h + 1.0) : 0.0;
      }
      cov_out[e] = w * k12u[p] - cross[p];
    }
  }
}

// Grouped sightline inputs: point rows q m + a (direction of sightline q)
// and the quadrature inputs (s_a, s_c, chord 0) of every pair a < c.
__global__ void k_sl_group_inputs(int64_t nsl, int m, const double* __restrict__ l,
                                  const double* __restrict__ b, const double* __restrict__ s,
                                  double* __restrict__ l2, double* __restrict__ b2,
                                  double* __restrict__ si, double* __restrict__ sj,
                                  double* __restrict__ ch, unsigned* __restrict__ bad) {
  const int64_t np = nsl * m;
  const int64_t npq = (int64_t)m * (m - 1) / 2;
  const int64_t total = np > nsl * npq ? np : nsl * npq;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < np) {
      l2[e] = l[e / m];
      b2[e] = b[e / m];
    }
    if (e < nsl * npq) {
      const int64_t q = e / npq;
      int64_t k = e - q * npq;
      int a = 0;
      while (k >= m - 1 - a) {
        k -= m - 1 - a;
        ++a;
      }
      const int c = a + 1 + (int)k;
      const double sa = s[q * m + a], sc = s[q * m + c];
      if (!(sc > sa)) atomicOr(bad, 1u);
      si[e] = sa;
      sj[e] = sc;
      ch[e] = 0.0;
    }
  }
}

// Joint predictive of each sightline from its point rows (means, variances)
// and the grouped cross terms: entry (a, c) = W(|s_c - s_a| / cutoff)
// k(s_a, s_c) - v_c^T B^-1 v_a.
__global__ void k_sl_assemble_group(int64_t nsl, int m, double inv_cut, int taper,
                                    const double* __restrict__ s,
                                    const double* __restrict__ mp,
                                    const double* __restrict__ vp,
                                    const double* __restrict__ cross,
                                    const double* __restrict__ k12u,
                                    double* __restrict__ mean_out,
                                    double* __restrict__ cov_out) {
  const int64_t npq = (int64_t)m * (m - 1) / 2;
  const int64_t mm = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nsl * mm;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / mm;
    const int r = (int)(e - q * mm);
    const int a = r / m, c = r - a * m;
    if (a == c) {
      cov_out[e] = vp[q * m + a];
      mean_out[q * m + a] = mp[q * m + a];
    } else {
      const int lo = a < c ? a : c, hi = a < c ? c : a;
      const int64_t p = q * npq + sl_pair_index(m, lo, hi);
      const double h = (s[q * m + hi] - s[q * m + lo]) * inv_cut;
      double w = h <= 1.0 ? 1.0 : 0.0;
      if (taper == GM_TAPER_WENDLAND) {
        const double u = 1.0 - h;
        w = h < 1.0 ? u * u * u * u * (4.0 * h + 1.0) : 0.0;
      }
      cov_out[e] = w * k12u[p] - cross[p];
    }
  }
}

gm_status gm_predict_sightlines(gm_ctx* c, int64_t nsl, int32_t m, const double* l,
                                const double* b, const double* s, double* mean_out,
                                double* cov_out) {
  if (!c || nsl < 0 || m < 1 || m > kMaxSightlinePoints ||
      (nsl > 0 && (!l || !b || !s || !mean_out || !cov_out)))
    return GM_E_INVAL;
  if (c->n_fields > 1)
    return set_error(c, GM_E_STATE, "prediction needs a single-field context");
  if (nsl == 0) return GM_OK;
  c->launches = 0;
  gm_status st = ensure_posterior(c);
  if (st != GM_OK) return st;
  const int64_t np = nsl * m;  // points
  const int64_t mm = (int64_t)m * m;
  if (m == 1) {  // no pairs: the single-point predictive
    ScopedDev buf(c, 5 * np * sizeof(double));
    double* q = (double*)buf.p;
    if (!q) return set_error(c, GM_E_NOMEM, "sightline arrays");
    if ((st = copy_in(c, q, l, np * sizeof(double))) != GM_OK ||
        (st = copy_in(c, q + np, b, np * sizeof(double))) != GM_OK ||
        (st = copy_in(c, q + 2 * np, s, np * sizeof(double))) != GM_OK)
      return st;
    st = predict_points(c, np, q, q + np, q + 2 * np, q + 3 * np, q + 4 * np, nullptr);
    if (st != GM_OK) return st;
    if ((st = copy_out(c, mean_out, q + 3 * np, np * sizeof(double))) != GM_OK) return st;
    if ((st = copy_out(c, cov_out, q + 4 * np, np * sizeof(double))) != GM_OK) return st;
    c->stats.kernel_launches = c->launches;
    return GM_OK;
  }
  const int64_t npr = nsl * ((int64_t)m * (m - 1) / 2);  // pairs
  if (m == 4 || m == 8 || m == 16 || m == 32) {
    // a sightline's m points are m consecutive query columns of one panel
    // group (m divides the panel width): every cross term comes from the m
    // solves, no pair columns
    // l, b (nsl); s, mean, l2, b2, mp, vp (np); cov (nsl m^2); si, sj, ch, k12, cross (npr)
    const size_t ndg = 2 * nsl + 6 * np + nsl * mm + 5 * npr;
    ScopedDev bufg(c, ndg * sizeof(double));
    double* g = (double*)bufg.p;
    if (!g) return set_error(c, GM_E_NOMEM, "sightline arrays");
    double *gl = g, *gb = gl + nsl, *gs = gb + nsl, *gmean = gs + np, *l2 = gmean + np,
           *b2 = l2 + np, *mp = b2 + np, *vp = mp + np, *gcov = vp + np, *si = gcov + nsl * mm,
           *sj = si + npr, *ch = sj + npr, *k12 = ch + npr, *cross = k12 + npr;
    if ((st = copy_in(c, gl, l, nsl * sizeof(double))) != GM_OK ||
        (st = copy_in(c, gb, b, nsl * sizeof(double))) != GM_OK ||
        (st = copy_in(c, gs, s, np * sizeof(double))) != GM_OK)
      return st;
    GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags + 2, 0, sizeof(unsigned), c->stream));
    GM_PROF(c, "k_sl_group_inputs");
    k_sl_group_inputs<<<eb(c, std::max(np, npr)), 256, 0, c->stream>>>(
        nsl, m, gl, gb, gs, l2, b2, si, sj, ch, c->d_flags + 2);
    GM_LAUNCH_CHECK(c);
    {
      unsigned* h = (unsigned*)c->h_pinned;
      GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags + 2, sizeof(unsigned),
                                       cudaMemcpyDeviceToHost, c->stream));
      GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
      if (*h) return set_error(c, GM_E_INVAL, "sightline distances must increase");
    }
    st = predict_points(c, np, l2, b2, gs, mp, vp, cross, m);
    if (st == GM_OK) st = pairlist_quadrature(c, npr, si, sj, ch, k12);
    if (st != GM_OK) return st;
    GM_PROF(c, "k_sl_assemble_group");
    k_sl_assemble_group<<<eb(c, nsl * mm), 256, 0, c->stream>>>(
        nsl, m, 1.0 / c->cfg.cutoff_pc, c->cfg.taper, gs, mp, vp, cross, k12, gmean, gcov);
    GM_LAUNCH_CHECK(c);
    if ((st = read_flags(c)) != GM_OK) return st;
    if ((st = copy_out(c, mean_out, gmean, np * sizeof(double))) != GM_OK) return st;
    if ((st = copy_out(c, cov_out, gcov, nsl * mm * sizeof(double))) != GM_OK) return st;
    c->stats.kernel_launches = c->launches;
    return GM_OK;
  }
  // l, b (nsl); s, mean (np); cov (nsl m^2); l2, b2, s2, mean2, var2 (2 npr);
  // si, sj, ch, k12, cross (npr)
  const size_t nd = 2 * nsl + 2 * np + nsl * mm + 15 * npr;
  ScopedDev buf(c, nd * sizeof(double));
  double* q = (double*)buf.p;
  if (!q) return set_error(c, GM_E_NOMEM, "sightline pair arrays");
  double *ql = q, *qb = ql + nsl, *qs = qb + nsl, *mean = qs + np, *cov = mean + np,
         *l2 = cov + nsl * mm, *b2 = l2 + 2 * npr, *s2 = b2 + 2 * npr, *mean2 = s2 + 2 * npr,
         *var2 = mean2 + 2 * npr, *si = var2 + 2 * npr, *sj = si + npr, *ch = sj + npr,
         *k12 = ch + npr, *cross = k12 + npr;
  if ((st = copy_in(c, ql, l, nsl * sizeof(double))) != GM_OK ||
      (st = copy_in(c, qb, b, nsl * sizeof(double))) != GM_OK ||
      (st = copy_in(c, qs, s, np * sizeof(double))) != GM_OK)
    return st;
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags + 2, 0, sizeof(unsigned), c->stream));
  GM_PROF(c, "k_sl_pairs");
  k_sl_pairs<<<eb(c, npr), 256, 0, c->stream>>>(nsl, m, ql, qb, qs, l2, b2, s2, si, sj, ch,
                                                c->d_flags + 2);
  GM_LAUNCH_CHECK(c);
  {
    unsigned* h = (unsigned*)c->h_pinned;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags + 2, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                     c->stream));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (*h) return set_error(c, GM_E_INVAL, "sightline distances must increase");
  }
  st = predict_points(c, 2 * npr, l2, b2, s2, mean2, var2, cross);
  if (st == GM_OK) st = pairlist_quadrature(c, npr, si, sj, ch, k12);
  if (st != GM_OK) return st;
  GM_PROF(c, "k_sl_assemble");
  k_sl_assemble<<<eb(c, nsl * mm), 256, 0, c->stream>>>(nsl, m, 1.0 / c->cfg.cutoff_pc,
                                                        c->cfg.taper, qs, mean2, var2, cross,
                                                        k12, mean, cov);
  GM_LAUNCH_CHECK(c);
  if ((st = read_flags(c)) != GM_OK) return st;
  if ((st = copy_out(c, mean_out, mean, np * sizeof(double))) != GM_OK) return st;
  if ((st = copy_out(c, cov_out, cov, nsl * mm * sizeof(double))) != GM_OK) return st;
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}

gm_status gm_monotone_sample(gm_ctx* c, int64_t nsl, int32_t m, const double* mean,
                             const double* cov, const double* momenta, int32_t n_burn,
                             int32_t n_samples, double* samples_out, int64_t* hits_out) {
  if (!c || nsl < 0 || m < 1 || m > kMaxSightlinePoints || n_burn < 0 || n_samples < 0 ||
      (nsl > 0 && (!mean || !cov || !momenta || (n_samples > 0 && !samples_out))))
    return GM_E_INVAL;
  if (nsl == 0 || (int64_t)n_burn + n_samples == 0) return GM_OK;
  c->launches = 0;
  const int64_t T = (int64_t)n_burn + n_samples;
  const int64_t mm = (int64_t)m * m;
  // mean (nsl m), cov (nsl m^2), momenta (nsl T m), samples (nsl n_samples m), hits (nsl)
  const size_t nd = nsl * (m + mm + T * m + (int64_t)n_samples * m + 1);
  ScopedDev buf(c, nd * sizeof(double));
  double* q = (double*)buf.p;
  if (!q) return set_error(c, GM_E_NOMEM, "sampler arrays");
  double *dm = q, *dc = dm + nsl * m, *dp = dc + nsl * mm, *dout = dp + nsl * T * m;
  int64_t* dh = (int64_t*)(dout + nsl * (int64_t)n_samples * m);
  gm_status st;
  if ((st = copy_in(c, dm, mean, nsl * m * sizeof(double))) != GM_OK ||
      (st = copy_in(c, dc, cov, nsl * mm * sizeof(double))) != GM_OK ||
      (st = copy_in(c, dp, momenta, nsl * T * m * sizeof(double))) != GM_OK)
    return st;
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags + 2, 0, sizeof(unsigned), c->stream));
  st = monotone_sample(c, nsl, m, dm, dc, dp, n_burn, n_samples, dout, dh, c->d_flags + 2);
  if (st != GM_OK) return st;
  unsigned* h = (unsigned*)c->h_pinned;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags + 2, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                   c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  const unsigned f = *h;
  if (f & kFlagNonFinite) return set_error(c, GM_E_NONFINITE, "non-finite mean or covariance");
  if (n_samples > 0 &&
      (st = copy_out(c, samples_out, dout, nsl * (int64_t)n_samples * m * sizeof(double))) != GM_OK)
    return st;
  if (hits_out && (st = copy_out(c, hits_out, dh, nsl * sizeof(int64_t))) != GM_OK) return st;
  c->stats.kernel_launches = c->launches;
  if (f & kFlagNotSPD)
    return set_error(c, GM_E_NOT_SPD, "a sightline covariance is not positive definite");
  if (f & kFlagHitLimit)
    return set_error(c, GM_E_NOCONV, "a sampler step reached the wall-hit limit");
  return GM_OK;
}

gm_status gm_pic_posterior(gm_ctx* c, int32_t n_blocks, const int32_t* block_of, int64_t R,
                           const double* l, const double* b, const double* s,
                           double* mean_out, double* cov_out) {
  if (!c || n_blocks < 1 || !block_of || R < 1 || R > kMaxPicInducing || !l || !b || !s ||
      !mean_out || !cov_out)
    return GM_E_INVAL;
  if (!c->built) return set_error(c, GM_E_STATE, "gm_build_cov must come first");
  if (c->n_fields > 1 || c->cfg.precision != GM_PREC_FP64 ||
      c->cfg.likelihood != GM_LIK_GAUSS_IN_LNA)
    return set_error(c, GM_E_STATE,
                     "the PIC posterior needs a single-field FP64 context with the Gaussian "
                     "likelihood in ln A");
  c->launches = 0;
  const int64_t n = c->n;
  // block of each internal star (host)
  std::vector<int32_t> blk(n);
  std::vector<int64_t> perm(n);
  if (is_device_ptr(block_of)) {
    GM_CUDA_CHECK(c, cudaMemcpy(blk.data(), block_of, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(blk.data(), block_of, n * sizeof(int32_t));
  }
  GM_CUDA_CHECK(c, cudaMemcpyAsync(perm.data(), c->perm, n * sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, c->stream));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  std::vector<int32_t> blk_int(n);
  for (int64_t k = 0; k < n; ++k) {
    const int32_t v = blk[perm[k]];
    if (v < 0 || v >= n_blocks) return set_error(c, GM_E_INVAL, "block id out of range");
    blk_int[k] = v;
  }
  const size_t nb_ = R * sizeof(double);
  // l, b, s, ux, uy, uz (R)
  ScopedDev buf(c, 6 * nb_);
  if (!buf.p) return set_error(c, GM_E_NOMEM, "inducing arrays");
  double *ql = (double*)buf.p, *qb = ql + R, *qs = qb + R, *ux = qs + R, *uy = ux + R,
         *uz = uy + R;
  gm_status st;
  if ((st = copy_in(c, ql, l, nb_)) != GM_OK || (st = copy_in(c, qb, b, nb_)) != GM_OK ||
      (st = copy_in(c, qs, s, nb_)) != GM_OK)
    return st;
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags + 1, 0, sizeof(unsigned), c->stream));
  GM_PROF(c, "k_check_inputs");
  k_check_inputs<<<eb(c, R), 256, 0, c->stream>>>(R, qs, qs, qs, ql, qb, c->d_flags + 1);
  GM_LAUNCH_CHECK(c);
  {
    unsigned* h = (unsigned*)c->h_pinned;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                     c->stream));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (*h) return set_error(c, GM_E_INVAL, "inducing distances must be finite and > 0");
  }
  if ((st = unit_vectors(c, R, ql, qb, ux, uy, uz)) != GM_OK) return st;
  if ((st = pic_posterior(c, (int)R, qs, ux, uy, uz, blk_int.data(), n_blocks)) != GM_OK) {
    pic_free(c);
    return st;
  }
  {
    unsigned* h = (unsigned*)c->h_pinned;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                     c->stream));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    const unsigned f = *h;
    if (f) GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), c->stream));
    if (f & (kFlagNonFinite | kFlagNotSPD)) pic_free(c);
    if (f & kFlagNonFinite) return set_error(c, GM_E_NONFINITE, "non-finite covariance value");
    if (f & kFlagNotSPD)
      return set_error(c, GM_E_NOT_SPD,
                       "K_uu, a sub-catalogue's conditional covariance or the posterior "
                       "precision of u has no Cholesky factor");
  }
  if ((st = copy_out(c, mean_out, pic_mean(c), nb_)) != GM_OK) return st;
  if ((st = copy_out(c, cov_out, pic_cov(c), R * nb_)) != GM_OK) return st;
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}

gm_status gm_pic_predict(gm_ctx* c, int64_t nq, const int32_t* q_block, const double* l,
                         const double* b, const double* s, double* mean_out, double* var_out) {
  if (!c || nq < 0 || (nq > 0 && (!q_block || !l || !b || !s || !mean_out || !var_out)))
    return GM_E_INVAL;
  if (!pic_ready(c)) return set_error(c, GM_E_STATE, "gm_pic_posterior must come first");
  if (nq == 0) return GM_OK;
  c->launches = 0;
  const int nb = pic_blocks(c);
  std::vector<int32_t> qb_h(nq);
  if (is_device_ptr(q_block)) {
    GM_CUDA_CHECK(c, cudaMemcpy(qb_h.data(), q_block, nq * sizeof(int32_t), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(qb_h.data(), q_block, nq * sizeof(int32_t));
  }
  for (int64_t q = 0; q < nq; ++q)
    if (qb_h[q] < 0 || qb_h[q] >= nb) return set_error(c, GM_E_INVAL, "query block out of range");
  const size_t nb_ = nq * sizeof(double);
  // l, b, s, ux, uy, uz, kss, ms, mean, var (nq)
  ScopedDev buf(c, 10 * nb_);
  ScopedDev bqb(c, nq * sizeof(int32_t));
  ScopedDev bqp(c, (nq + 1) * sizeof(int64_t));
  if (!buf.p || !bqb.p || !bqp.p) return set_error(c, GM_E_NOMEM, "PIC query arrays");
  double *ql = (double*)buf.p, *qb = ql + nq, *qs = qb + nq, *ux = qs + nq, *uy = ux + nq,
         *uz = uy + nq, *kss = uz + nq, *ms = kss + nq, *mean = ms + nq, *var = mean + nq;
  int32_t* qblk = (int32_t*)bqb.p;
  int64_t* qptr = (int64_t*)bqp.p;
  gm_status st;
  if ((st = copy_in(c, ql, l, nb_)) != GM_OK || (st = copy_in(c, qb, b, nb_)) != GM_OK ||
      (st = copy_in(c, qs, s, nb_)) != GM_OK)
    return st;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(qblk, qb_h.data(), nq * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   c->stream));
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags + 1, 0, sizeof(unsigned), c->stream));
  GM_PROF(c, "k_check_inputs");
  k_check_inputs<<<eb(c, nq), 256, 0, c->stream>>>(nq, qs, qs, qs, ql, qb, c->d_flags + 1);
  GM_LAUNCH_CHECK(c);
  {
    unsigned* h = (unsigned*)c->h_pinned;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(h, c->d_flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                     c->stream));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (*h) return set_error(c, GM_E_INVAL, "query distances must be finite and > 0");
  }
  if ((st = unit_vectors(c, nq, ql, qb, ux, uy, uz)) != GM_OK) return st;
  if ((st = self_quadrature(c, nq, qs, kss)) != GM_OK) return st;
  if (c->mean_fn_on) {
    if ((st = mean_fn_apply(c, nq, qs, ux, uy, uz, kss, ms, nullptr)) != GM_OK) return st;
  } else {
    GM_PROF(c, "k_query_mean");
    k_query_mean<<<eb(c, nq), 256, 0, c->stream>>>(nq, std::log(c->cfg.rho_bar), c->cfg.form,
                                                   c->cfg.sigma2, qs, kss, ms);
    GM_LAUNCH_CHECK(c);
  }
  Buffer qcol;
  int64_t qnnz = 0;
  st = neighbour_csr(c, nq, qs, ux, uy, uz, nullptr, false, qptr, qcol, &qnnz, nullptr);
  if (st != GM_OK) return st;
  ScopedDev bqc(c, qcol.p, qcol.bytes, ScopedDev::Adopt{});
  ScopedDev bqv(c, (size_t)std::max<int64_t>(qnnz, 1) * sizeof(double));
  if (!bqv.p) return set_error(c, GM_E_NOMEM, "PIC query values");
  st = pair_quadrature(c, nq, qs, ux, uy, uz, nullptr, qptr, (const int32_t*)qcol.p, qnnz, bqv.p,
                       false);
  if (st == GM_OK)
    st = pic_predict(c, nq, qs, ux, uy, uz, qblk, kss, ms, qptr, (const int32_t*)qcol.p,
                     (const double*)bqv.p, mean, var);
  if (st == GM_OK) st = read_flags(c);
  if (st != GM_OK) return st;
  if ((st = copy_out(c, mean_out, mean, nb_)) != GM_OK) return st;
  if ((st = copy_out(c, var_out, var, nb_)) != GM_OK) return st;
  c->stats.kernel_launches = c->launches;
  return GM_OK;
}

gm_status gm_profile(gm_ctx* c, int32_t enable) {
  if (!c) return GM_E_INVAL;
  prof_collect(c);
  c->prof_on = enable != 0;
  if (enable == 0) c->prof_acc.clear();
  return GM_OK;
}

int32_t gm_kernel_time_count(gm_ctx* c) {
  if (!c) return 0;
  prof_collect(c);
  return (int32_t)c->prof_acc.size();
}

gm_status gm_kernel_time(gm_ctx* c, int32_t k, const char** name, int64_t* launches,
                         double* total_ms) {
  if (!c || k < 0 || k >= (int32_t)c->prof_acc.size()) return GM_E_INVAL;
  if (name) *name = c->prof_acc[k].name;
  if (launches) *launches = c->prof_acc[k].launches;
  if (total_ms) *total_ms = c->prof_acc[k].ms;
  return GM_OK;
}

void gm_destroy(gm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  prof_collect(c);
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  c->prof_pool.clear();
  workspace_free(c);
  deflate_free(c);
  pic_free(c);
  for (auto& b : c->owned) {
    if (c->has_alloc)
      c->alloc.free(b.p, b.bytes, (void*)c->stream, c->alloc.user);
    else
      cudaFreeAsync(b.p, c->stream);
  }
  c->owned.clear();
  cudaStreamSynchronize(c->stream);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  delete c;
}

}  // extern "C"

