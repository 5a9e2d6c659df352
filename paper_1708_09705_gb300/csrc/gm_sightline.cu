// Sightline sampler of the dA/ds >= 0 conditioning (Sect. 5): exact HMC for
// each sightline's truncated Gaussian predictive, one thread per sightline.
// The per-sightline arithmetic is in gm_hmc.cuh.
#include <algorithm>
#include <cstdlib>

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

// One warp per sightline (m <= 32), two warps per block; the warp's state,
// S and L live in shared memory (gmhmc::WarpState), the phases of a step are
// separated by warp barriers.  Same chain as k_monotone_hmc.
__global__ void __launch_bounds__(64)
    k_monotone_hmc_warp(int64_t nsl, int m, int n_burn, int n_samples,
                        const double* __restrict__ mu_t, const double* __restrict__ S_t,
                        const double* __restrict__ mom, double* __restrict__ out,
                        int64_t* __restrict__ hits, unsigned* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t q = blockIdx.x * 2 + wib;
  if (q >= nsl) return;  // the whole warp
  const size_t per = sizeof(gmhmc::WarpState) + 2 * (size_t)m * m * sizeof(double);
  gmhmc::WarpState& W = *reinterpret_cast<gmhmc::WarpState*>(sm + wib * per);
  if (lane == 0) {
    W.S = reinterpret_cast<double*>(sm + wib * per + sizeof(gmhmc::WarpState));
    W.L = W.S + m * m;
  }
  __syncwarp();
  gmhmc::w_stage(W, lane, m, mu_t + q, S_t + q, nsl);
  __syncwarp();
  if (lane == 0) gmhmc::w_setup(W, m);
  __syncwarp();
  const int64_t T = (int64_t)n_burn + n_samples;
  double* o = out + q * (int64_t)n_samples * m;
  if (W.status) {
    for (int64_t k = lane; k < (int64_t)n_samples * m; k += 32) o[k] = NAN;
    if (lane == 0) {
      hits[q] = 0;
      atomicOr(flags, kFlagNotSPD);
    }
    return;
  }
  unsigned status = 0;
  for (int64_t it = 0; it < T; ++it) {
    gmhmc::w_momentum(W, lane, m, mom + (q * T + it) * m);
    __syncwarp();
    gmhmc::w_velocity(W, lane, m);
    if (lane == 0) W.t_left = gmhmc::kHalfPi;
    __syncwarp();
    int n = 0;
    for (; n < gmhmc::kMaxWallHits; ++n) {
      gmhmc::w_hit(W, lane, m);
      __syncwarp();
      double tb;
      const int j = gmhmc::w_best(W, m, &tb);
      if (j < 0) {
        gmhmc::w_rotate(W, lane, m, W.t_left);
        __syncwarp();
        break;
      }
      gmhmc::w_rotate(W, lane, m, tb);
      __syncwarp();
      if (lane == 0) gmhmc::w_reflect_factor(W, m, j);
      __syncwarp();
      gmhmc::w_reflect(W, lane, m, j);
      __syncwarp();
      if (lane == 0) {
        W.t_left -= tb;
        W.nhits++;
      }
      __syncwarp();
    }
    if (n == gmhmc::kMaxWallHits) status |= gmhmc::kHitLimit;
    if (it >= n_burn && lane < m) o[(it - n_burn) * m + lane] = W.mu[lane] + W.y[lane];
    __syncwarp();
  }
  if (lane == 0) {
    hits[q] = W.nhits;
    if (status & gmhmc::kHitLimit) atomicOr(flags, kFlagHitLimit);
  }
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
  // GM_HMC_WARP=1 selects one warp per sightline (m <= 32); the default is
  // one thread per sightline
  const char* e = std::getenv("GM_HMC_WARP");
  if (m <= gmhmc::kWarpMax && e && e[0] == '1') {
    const size_t per = sizeof(gmhmc::WarpState) + 2 * (size_t)m * m * sizeof(double);
    GM_PROF(c, "k_monotone_hmc_warp");
    k_monotone_hmc_warp<<<(unsigned)ceil_div(nsl, 2), 64, 2 * per, c->stream>>>(
        nsl, m, n_burn, n_samples, mu_t, S_t, mom, out, hits, flags);
    GM_LAUNCH_CHECK(c);
  } else {
    GM_PROF(c, "k_monotone_hmc");
    k_monotone_hmc<<<(unsigned)ceil_div(nsl, 128), 128, 0, c->stream>>>(
        nsl, m, n_burn, n_samples, mu_t, S_t, L_t, y_t, w_t, mom, out, hits, flags);
    GM_LAUNCH_CHECK(c);
  }
  GM_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
  return GM_OK;
}

}  // namespace gm
