// Sightline sampler of the dA/ds >= 0 conditioning (Sect. 5): exact HMC for
// each sightline's truncated Gaussian predictive, one thread per sightline.
// The per-sightline arithmetic is in gm_hmc.cuh.
#include <algorithm>

#include "gm_hmc.cuh"
#include "gm_internal.cuh"

namespace gm {

// Caller layout (sightline-major) -> sightline-fastest scratch:
// mu_t[i * nsl + q] = mean[q * m + i], S_t[e * nsl + q] = cov[q * m * m + e].
__global__ void k_sl_stage(int64_t nsl, int m, const double* __restrict__ mean,
                           const double* __restrict__ cov, double* __restrict__ mu_t,
                           double* __restrict__ S_t, unsigned* __restrict__ flags) {
  const int64_t per = (int64_t)m + (int64_t)m * m;
  const int64_t total = per * nsl;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = k / nsl, q = k - e * nsl;
    double v;
    if (e < m) {
      v = mean[q * m + e];
      mu_t[e * nsl + q] = v;
    } else {
      v = cov[q * (int64_t)m * m + (e - m)];
      S_t[(e - m) * nsl + q] = v;
    }
    if (!isfinite(v)) atomicOr(flags, kFlagNonFinite);
  }
}

__global__ void __launch_bounds__(128)
    k_monotone_hmc(int64_t nsl, int m, int n_burn, int n_samples,
                   const double* __restrict__ mu_t, const double* __restrict__ S_t,
                   double* __restrict__ L_t, double* __restrict__ y_t, double* __restrict__ w_t,
                   const double* __restrict__ mom, double* __restrict__ out,
                   int64_t* __restrict__ hits, unsigned* __restrict__ flags) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nsl) return;
  const int64_t T = (int64_t)n_burn + n_samples;
  int64_t h = 0;
  const unsigned s = gmhmc::sample_sightline(mu_t + q, S_t + q, L_t + q, y_t + q, w_t + q, nsl,
                                             mom + q * T * m, out + q * (int64_t)n_samples * m,
                                             m, n_burn, n_samples, &h);
  hits[q] = h;
  if (s & gmhmc::kNotPD) atomicOr(flags, kFlagNotSPD);
  if (s & gmhmc::kHitLimit) atomicOr(flags, kFlagHitLimit);
}

gm_status monotone_sample(gm_ctx* c, int64_t nsl, int m, const double* mean, const double* cov,
                          const double* mom, int n_burn, int n_samples, double* out,
                          int64_t* hits, unsigned* flags) {
  const int64_t mm = (int64_t)m * m;
  // scratch: mu_t (m), S_t (m^2), L_t (m^2), y_t (m), w_t (m) per sightline
  const size_t bytes = (size_t)nsl * (3 * m + 2 * mm) * sizeof(double);
  ScopedDev buf(c, bytes);
  double* ws = (double*)buf.p;
  if (!ws) return set_error(c, GM_E_NOMEM, "sampler scratch");
  double *mu_t = ws, *S_t = mu_t + nsl * m, *L_t = S_t + nsl * mm, *y_t = L_t + nsl * mm,
         *w_t = y_t + nsl * m;
  const int64_t per = m + mm;
  const int sb = (int)std::max<int64_t>(
      1, std::min<int64_t>(ceil_div(per * nsl, 256), 8 * sm_count(c)));
  GM_PROF(c, "k_sl_stage");
  k_sl_stage<<<sb, 256, 0, c->stream>>>(nsl, m, mean, cov, mu_t, S_t, flags);
  GM_LAUNCH_CHECK(c);
  {
    unsigned* h = (unsigned*)c->h_pinned;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                     c->stream));
    GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (*h & kFlagNonFinite) return GM_OK;  // the caller reads the flag and reports it
  }
  GM_PROF(c, "k_monotone_hmc");
  k_monotone_hmc<<<(unsigned)ceil_div(nsl, 128), 128, 0, c->stream>>>(
      nsl, m, n_burn, n_samples, mu_t, S_t, L_t, y_t, w_t, mom, out, hits, flags);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  return GM_OK;
}

}  // namespace gm
