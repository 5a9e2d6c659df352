// EP site update, one thread per star, FP64 (App. A.2).
//
// For star i with posterior marginal N(mu_i, Sigma_ii) and site (tau_i, nu_i):
//   cavity (eq. cavity):  tau_c = 1/Sigma_ii - tau_i, nu_c = mu_i/Sigma_ii - nu_i,
//     with the cavity variance floored (Sect. 5); tau_c <= 0 skips the star;
//   tilted (eq. tilted):  N(a; mu_c, v_c) * L_i(a), L_i the star's likelihood;
//   moment matching (eq. KL1'): mean mh and variance vh of the tilted give
//     tau_new = 1/vh - tau_c, nu_new = mh/vh - nu_c;
//   damped replacement; an update with tau_new < 0 is skipped.
// Gaussian-in-ln-A likelihood: the tilted is Gaussian (closed form).
// Gaussian-in-A likelihood: mode and curvature of the tilted log-density by
// safeguarded Newton ascent, then a 64-node Gauss-Hermite rule centred at the
// mode and scaled by the curvature.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "gm_internal.cuh"

namespace gm {

struct SiteParams {
  double damping;
  double vc_floor;
  int lik;
};

__device__ __forceinline__ double log_tilted(double a, double mc, double vc, double obs,
                                             double s2) {
  double ea = exp(a);
  double u = a - mc, w = obs - ea;
  return -0.5 * u * u / vc - 0.5 * w * w / s2;
}

__device__ void tilted_gauss_in_a(double mc, double vc, double obs, double s2,
                                  const double* __restrict__ ghx, const double* __restrict__ ghw,
                                  double* mh, double* vh) {
  double a;
  if (obs > 0) {
    double aL = log(obs), vL = s2 / (obs * obs);
    a = (mc / vc + aL / vL) / (1.0 / vc + 1.0 / vL);
  } else {
    a = mc;
  }
  for (int it = 0; it < 100; ++it) {
    double ea = exp(a);
    double gr = -(a - mc) / vc + (obs - ea) * ea / s2;
    double H = -1.0 / vc + (obs * ea - 2.0 * ea * ea) / s2;
    double step = H < 0 ? -gr / H : gr * vc;
    step = fmax(-1.0, fmin(1.0, step));
    double h0 = log_tilted(a, mc, vc, obs, s2);
    int k = 0;
    while (log_tilted(a + step, mc, vc, obs, s2) < h0 && k < 60) {
      step *= 0.5;
      ++k;
    }
    a += step;
    if (fabs(step) <= 1e-14 * (1.0 + fabs(a))) break;
  }
  double ea = exp(a);
  double H = -1.0 / vc + (obs * ea - 2.0 * ea * ea) / s2;
  double sh = H < 0 ? 1.0 / sqrt(-H) : sqrt(vc);
  double h0 = log_tilted(a, mc, vc, obs, s2);
  const double sc = 1.4142135623730951 * sh;
  // moments about the mode, then shifted
  double S0 = 0, S1 = 0, S2 = 0;
  for (int k = 0; k < kGH; ++k) {
    double y = sc * ghx[k];
    double wk = ghw[k] * exp(log_tilted(a + y, mc, vc, obs, s2) - h0);
    S0 += wk;
    S1 += wk * y;
    S2 += wk * y * y;
  }
  double m1 = S1 / S0;
  *mh = a + m1;
  *vh = S2 / S0 - m1 * m1;
}

__global__ void k_site_update(int64_t n, SiteParams P, const double* __restrict__ mu,
                              const double* __restrict__ var, const double* __restrict__ obs,
                              const double* __restrict__ sig, double* __restrict__ tau,
                              double* __restrict__ nu, const double* __restrict__ gh_x,
                              const double* __restrict__ gh_w, double* __restrict__ part_delta,
                              unsigned long long* __restrict__ skipped,
                              unsigned* __restrict__ flags) {
  __shared__ double ghx[kGH], ghw[kGH];
  __shared__ double sh[32];
  for (int k = threadIdx.x; k < kGH; k += blockDim.x) {
    ghx[k] = gh_x[k];
    ghw[k] = gh_w[k];
  }
  __syncthreads();
  double dmax = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double t0 = tau[i], n0 = nu[i];
    const double S = var[i], m = mu[i];
    double tc = 1.0 / S - t0;
    double ncv = m / S - n0;
    bool skip = !(tc > 0) || !isfinite(tc) || !isfinite(ncv);
    double t_new = t0, n_new = n0;
    if (!skip) {
      const double mc = ncv / tc;
      const double vc = fmax(1.0 / tc, P.vc_floor);
      tc = 1.0 / vc;
      ncv = mc / vc;
      const double s2 = sig[i] * sig[i];
      double mh, vh;
      if (P.lik == GM_LIK_GAUSS_IN_LNA) {
        vh = 1.0 / (1.0 / vc + 1.0 / s2);
        mh = vh * (mc / vc + obs[i] / s2);
      } else {
        tilted_gauss_in_a(mc, vc, obs[i], s2, ghx, ghw, &mh, &vh);
      }
      t_new = 1.0 / vh - tc;
      n_new = mh / vh - ncv;
      if (!(t_new >= 0) || !isfinite(n_new) || !isfinite(t_new)) skip = true;
    }
    if (skip) {
      atomicAdd(skipped, 1ull);
      continue;
    }
    const double tn = (1.0 - P.damping) * t0 + P.damping * t_new;
    const double nn = (1.0 - P.damping) * n0 + P.damping * n_new;
    tau[i] = tn;
    nu[i] = nn;
    double dt = fabs(tn - t0) / (1.0 + fabs(t0));
    double dn = fabs(nn - n0) / (1.0 + fabs(n0));
    dmax = fmax(dmax, fmax(dt, dn));
  }
  // block max (fixed order)
  for (int off = 16; off > 0; off >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, sh[w]);
    if (!isfinite(v)) atomicOr(flags, kFlagNonFinite);
    part_delta[blockIdx.x] = v;
  }
}

gm_status site_update(gm_ctx* c, double* max_delta, int64_t* skipped) {
  const int64_t n = c->n;
  cudaStream_t st = c->stream;
  const int G = (int)std::min<int64_t>(ceil_div(n, 128), 4 * sm_count(c));
  double* part = (double*)dev_alloc(c, (G + 1) * sizeof(double) + sizeof(unsigned long long));
  if (!part) return set_error(c, GM_E_NOMEM, "site partials");
  unsigned long long* cnt = (unsigned long long*)(part + G);
  GM_CUDA_CHECK(c, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  SiteParams P{c->cfg.damping, c->cfg.vc_floor, c->cfg.likelihood};
  GM_PROF(c, "k_site_update");
  k_site_update<<<G, 128, 0, st>>>(n, P, c->mu, c->var, c->obs, c->obs_sigma, c->tau, c->nu,
                                   c->gh_x, c->gh_wx, part, cnt, c->d_flags);
  GM_LAUNCH_CHECK(c);
  double* hp = (double*)c->h_pinned;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hp, part, (G + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  double m = 0;
  for (int k = 0; k < G; ++k) m = std::fmax(m, hp[k]);
  unsigned long long sk;
  std::memcpy(&sk, hp + G, sizeof(sk));
  *max_delta = m;
  *skipped = (int64_t)sk;
  dev_free_now(c, part, (G + 1) * sizeof(double) + sizeof(unsigned long long));
  return GM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free site update (gm_site_update_noalloc).
//
// Some callers cannot allocate device memory while they run: a host
// framework that owns every device allocation through its own pool, code
// running inside a memory-capped or pre-reserved budget, or a service loop
// that must not call cudaMalloc/cudaFree on its latency path.  For them the
// EP site update runs on caller-owned arrays, with its scratch (Gauss-Hermite
// table, per-block maxima, skip counter, flags) in the file-scope array
// below.  It is sized for one block per 128 stars up to kNaMaxBlocks blocks,
// so n <= kNaMaxStars.  Every GPU that loads the library holds the array
// until the process exits.  All calls share it: concurrent calls on the GPU
// race with one another and must be serialised by the caller.
// ---------------------------------------------------------------------------
constexpr int kNaMaxBlocks = 8192;
constexpr int64_t kNaMaxStars = 128ll * kNaMaxBlocks;  // 1,048,576
constexpr int kNaSlots = 2 * kGH + kNaMaxBlocks + 4;   // doubles
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_na_scratch[kNaSlots];

// Scratch layout (doubles): [0, kGH) nodes, [kGH, 2 kGH) weights * exp(x^2),
// [2 kGH, 2 kGH + kNaMaxBlocks) per-block maxima, then the skip counter
// (as an unsigned 64-bit word), the flags word and the reduced maximum.
// Per device, the scratch address at which the rule was last uploaded.  The
// address is resolved again on every call, so a module reloaded after a
// device reset (new address) gets its rule uploaded again instead of a stale
// pointer being used.
static double* g_na_ptr[kNaMaxDevices] = {nullptr};

__global__ void k_na_reduce_max(int nb, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[32];
  double v = 0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) v = fmax(v, part[k]);
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    *out = m;
  }
}

// Device memory of the current device `dev`, or managed memory.  Memory of
// another GPU is refused: without peer access the kernel could not read it.
static bool na_device_ptr(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Resolves the device address of the scratch array on the current device
// (the host-side name is only a stand-in) on every call, and uploads the
// Gauss-Hermite rule when that address has not seen it yet (first call on a
// device, or a module reloaded after a device reset).  The upload is a
// synchronous copy followed by a device synchronisation, so the rule is on
// the device before any kernel on any stream (a non-blocking one included)
// can read it; that first call therefore must not run inside a stream
// capture.  Serialised by a mutex.
static gm_status na_setup(int dev, double** out) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  double* p = nullptr;
  if (cudaGetSymbolAddress((void**)&p, g_na_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return GM_E_CUDA;
  }
  if (g_na_ptr[dev] != p) {
    double rule[2 * kGH];
    gauss_hermite(kGH, rule, rule + kGH);
    if (cudaMemcpy(p, rule, sizeof(rule), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      return GM_E_CUDA;
    }
    g_na_ptr[dev] = p;
  }
  *out = p;
  return GM_OK;
}

}  // namespace gm

extern "C" gm_status gm_site_update_noalloc(int64_t n, const double* mu, const double* var,
                                            const double* obs, const double* obs_sigma,
                                            double* tau, double* nu, int32_t likelihood,
                                            double damping, double vc_floor, void* stream,
                                            double* max_delta_out, int64_t* skipped_out) {
  using namespace gm;
  if (n < 1 || n > kNaMaxStars) return GM_E_INVAL;
  if (!mu || !var || !obs || !obs_sigma || !tau || !nu) return GM_E_INVAL;
  if (likelihood != GM_LIK_GAUSS_IN_A && likelihood != GM_LIK_GAUSS_IN_LNA) return GM_E_INVAL;
  if (!(damping > 0 && damping <= 1) || !(vc_floor >= 0)) return GM_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    return GM_E_CUDA;
  }
  for (const void* p : {(const void*)mu, (const void*)var, (const void*)obs,
                        (const void*)obs_sigma, (const void*)tau, (const void*)nu})
    if (!na_device_ptr(p, dev)) return GM_E_INVAL;
  double* base = nullptr;
  gm_status st = na_setup(dev, &base);
  if (st != GM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* gh_x = base;
  double* gh_w = base + kGH;
  double* part = base + 2 * kGH;
  unsigned long long* skipped = (unsigned long long*)(part + kNaMaxBlocks);
  unsigned* flags = (unsigned*)(part + kNaMaxBlocks + 1);
  double* maxd = part + kNaMaxBlocks + 2;
  // the counter and the flags keep the previous call's values: clear them
  if (cudaMemsetAsync(skipped, 0, 2 * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return GM_E_CUDA;
  }
  const int G = (int)ceil_div(n, 128);
  SiteParams P{damping, vc_floor, likelihood};
  k_site_update<<<G, 128, 0, s>>>(n, P, mu, var, obs, obs_sigma, tau, nu, gh_x, gh_w, part,
                                   skipped, flags);
  k_na_reduce_max<<<1, 1024, 0, s>>>(G, part, maxd);
  if (cudaGetLastError() != cudaSuccess) return GM_E_CUDA;
  unsigned long long h[3];
  if (cudaMemcpyAsync(h, skipped, 3 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GM_E_CUDA;
  }
  unsigned fl = (unsigned)(h[1] & 0xffffffffull);
  double md;
  std::memcpy(&md, &h[2], sizeof(md));
  if (max_delta_out) *max_delta_out = md;
  if (skipped_out) *skipped_out = (int64_t)h[0];
  return (fl & kFlagNonFinite) ? GM_E_NONFINITE : GM_OK;
}
