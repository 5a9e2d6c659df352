// Colour classes for probed posterior variances.
//
// The EP cavities need the marginal variances of the posterior (App. A.2,
// eq. cavity); exactly, each star costs one solve with B = I + S^1/2 K S^1/2.
// Probing (Tang & Saad 2012, "A probing method for computing the diagonal of
// a matrix inverse") lets all stars of one colour class share a solve: the
// class's right-hand sides are summed and each member reads its own variance
// from the common solution.  The error is the sum of the cross terms between
// members, which decays with their separation because B^-1 does; members of a
// class here are at least D = probe_factor x cutoff apart.
//
// Colouring: greedy (each star takes the smallest colour not held by an
// already coloured star closer than D) in a fixed order that runs in
// parallel.  Stars are bucketed in a grid of cells of edge >= D per field; a
// cell's class is the parity of its three cell coordinates.  Two distinct
// cells of one class are a whole cell apart, so their stars never conflict:
// the eight classes are coloured one after another, every cell of a class by
// its own thread block, the stars of a cell in index order.  The result is
// the sequential greedy colouring in the order (class, cell, star) and does
// not depend on the launch shape.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

constexpr int kMaxColours = 1 << 17;
constexpr int kColWords = kMaxColours / 32;  // 16 KB bitmap per block

__device__ __forceinline__ void probe_cell(const FieldGrid& g, double x, double y, double z,
                                           int* cx, int* cy, int* cz) {
  const int a = (int)floor((x - g.ox) * g.inv_cell);
  const int b = (int)floor((y - g.oy) * g.inv_cell);
  const int c = (int)floor((z - g.oz) * g.inv_cell);
  *cx = min(max(a, 0), g.gx - 1);
  *cy = min(max(b, 0), g.gy - 1);
  *cz = min(max(c, 0), g.gz - 1);
}

// Squared 3-D distance by the chord form (s_i - s_j)^2 + s_i s_j |u_i - u_j|^2.
__device__ __forceinline__ double probe_d2(double si, double xi, double yi, double zi, double sj,
                                           double xj, double yj, double zj) {
  const double dx = xi - xj, dy = yi - yj, dz = zi - zj, ds = si - sj;
  return fma(ds, ds, si * sj * fma(dx, dx, fma(dy, dy, dz * dz)));
}

__global__ void k_probe_keys(int64_t n, int64_t n_pad, const FieldGrid* __restrict__ cg,
                             const int32_t* __restrict__ field_of, const double* __restrict__ s,
                             const double* __restrict__ ux, const double* __restrict__ uy,
                             const double* __restrict__ uz, unsigned long long* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      const FieldGrid g = cg[field_of[i]];
      int cx, cy, cz;
      probe_cell(g, s[i] * ux[i], s[i] * uy[i], s[i] * uz[i], &cx, &cy, &cz);
      const unsigned long long id =
          (unsigned long long)g.cell_off + ((unsigned long long)cx * g.gy + cy) * g.gz + cz;
      keys[i] = (id << 32) | (unsigned long long)i;
    } else {
      keys[i] = ~0ull;
    }
  }
}

// ord[k] = star of sorted position k; cstart[c] = first position of cell c.
__global__ void k_probe_order(int64_t n, int64_t n_cells, const unsigned long long* __restrict__ keys,
                              int32_t* __restrict__ ord, int32_t* __restrict__ cstart) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < n) ord[k] = (int32_t)(keys[k] & 0xffffffffull);
    const int64_t prev = k == 0 ? -1 : (int64_t)(keys[k - 1] >> 32);
    const int64_t cur = k == n ? n_cells : (int64_t)(keys[k] >> 32);
    for (int64_t c = prev + 1; c <= cur; ++c) cstart[c] = (int32_t)k;
  }
}

// One class: block per listed cell (field, cx, cy, cz); the cell's stars in
// order, each scanning the 27 surrounding cells for coloured stars closer
// than D and taking the smallest free colour.
__global__ void __launch_bounds__(256) k_probe_greedy(
    int64_t n_list, const int4* __restrict__ list, const FieldGrid* __restrict__ cg,
    const int32_t* __restrict__ cstart, const int32_t* __restrict__ ord,
    const double* __restrict__ s, const double* __restrict__ ux, const double* __restrict__ uy,
    const double* __restrict__ uz, int32_t* __restrict__ colour, int* __restrict__ max_colour,
    unsigned* __restrict__ flags) {
  __shared__ unsigned bm[kColWords];
  __shared__ int sh_best, sh_nw;
  const int t = threadIdx.x;
  for (int64_t it = blockIdx.x; it < n_list; it += gridDim.x) {
    const int4 q = list[it];
    const FieldGrid g = cg[q.x];
    const int64_t id = g.cell_off + ((int64_t)q.y * g.gy + q.z) * g.gz + q.w;
    const int32_t k0 = cstart[id], k1 = cstart[id + 1];
    for (int32_t k = k0; k < k1; ++k) {
      const int32_t i = ord[k];
      if (t == 0) {
        sh_best = INT_MAX;
        sh_nw = min(kColWords, (__ldcg(max_colour) >> 5) + 2);
      }
      __syncthreads();
      const int nw = sh_nw;
      for (int w = t; w < nw; w += blockDim.x) bm[w] = 0u;
      __syncthreads();
      const double si = s[i], xi = ux[i], yi = uy[i], zi = uz[i];
      for (int dx = -1; dx <= 1; ++dx) {
        const int ax = q.y + dx;
        if (ax < 0 || ax >= g.gx) continue;
        for (int dy = -1; dy <= 1; ++dy) {
          const int ay = q.z + dy;
          if (ay < 0 || ay >= g.gy) continue;
          const int z0 = max(q.w - 1, 0), z1 = min(q.w + 1, g.gz - 1);
          const int64_t c0 = g.cell_off + ((int64_t)ax * g.gy + ay) * g.gz + z0;
          const int64_t c1 = g.cell_off + ((int64_t)ax * g.gy + ay) * g.gz + z1 + 1;
          for (int32_t p = cstart[c0] + t; p < cstart[c1]; p += blockDim.x) {
            const int32_t j = ord[p];
            const int32_t cj = __ldcg(colour + j);
            if (cj >= 0 && probe_d2(si, xi, yi, zi, s[j], ux[j], uy[j], uz[j]) < g.cut2)
              atomicOr(&bm[cj >> 5], 1u << (cj & 31));
          }
        }
      }
      __syncthreads();
      for (int w = t; w < nw; w += blockDim.x) {
        const unsigned fr = ~bm[w];
        if (fr) atomicMin(&sh_best, w * 32 + __ffs(fr) - 1);
      }
      __syncthreads();
      if (t == 0) {
        int b = sh_best;
        if (b >= kMaxColours) {
          atomicOr(flags, kFlagProbeOverflow);
          b = 0;
        }
        colour[i] = b;
        atomicMax(max_colour, b);
      }
      __syncthreads();
    }
  }
}

// Colours per field: ncol[f] = 1 + largest colour over the field's rows.
__global__ void k_probe_field_ncol(const int64_t* __restrict__ fptr, const int32_t* __restrict__ colour,
                                   int32_t* __restrict__ ncol) {
  __shared__ int sh;
  const int f = blockIdx.x;
  if (threadIdx.x == 0) sh = -1;
  __syncthreads();
  int m = -1;
  for (int64_t i = fptr[f] + threadIdx.x; i < fptr[f + 1]; i += blockDim.x) m = max(m, colour[i]);
  atomicMax(&sh, m);
  __syncthreads();
  if (threadIdx.x == 0) ncol[f] = sh + 1;
}

gm_status probe_colouring(gm_ctx* c) {
  const double fac = c->cfg.probe_factor;
  if (!(fac > 0)) return GM_OK;
  if (c->probe_colour && c->probe_factor_done == fac) return GM_OK;
  const int64_t n = c->n;
  const int nf = c->n_fields;
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  // colour grids: same origin as the neighbour grid, cell edge >= D (a hair
  // above, so that rounding cannot put stars closer than D two cells apart)
  std::vector<FieldGrid> cg(nf);
  int64_t off = 0;
  for (int f = 0; f < nf; ++f) {
    const FieldGrid& g = c->h_fgrid[f];
    const double cut = std::sqrt(g.cut2);
    const double D = fac * cut;
    const double ext[3] = {g.gx / g.inv_cell, g.gy / g.inv_cell, g.gz / g.inv_cell};
    double cell = D * (1.0 + 1e-6);
    int dims[3] = {1, 1, 1};
    for (int k = 0; k < 64; ++k) {
      int64_t tot = 1;
      for (int d = 0; d < 3; ++d) {
        dims[d] = (int)std::min<double>(std::floor(ext[d] / cell) + 1.0, 1 << 24);
        tot *= dims[d];
      }
      if (tot <= (1ll << 24)) break;
      cell *= 1.26;
    }
    FieldGrid q = g;
    q.inv_cell = 1.0 / cell;
    q.cut2 = D * D;
    q.gx = dims[0];
    q.gy = dims[1];
    q.gz = dims[2];
    q.cell_off = off;
    off += (int64_t)dims[0] * dims[1] * dims[2];
    cg[f] = q;
  }
  if (off >= (1ll << 31)) return set_error(c, GM_E_INVAL, "probing grid too large");
  const int64_t n_cells = off;
  int64_t n_pad = 1024;
  while (n_pad < n) n_pad <<= 1;
  const size_t kb_bytes = n_pad * sizeof(unsigned long long);
  FieldGrid* dcg = (FieldGrid*)dev_alloc(c, nf * sizeof(FieldGrid));
  unsigned long long* keys = (unsigned long long*)dev_alloc(c, kb_bytes);
  int32_t* ord = (int32_t*)dev_alloc(c, n * sizeof(int32_t));
  int32_t* cstart = (int32_t*)dev_alloc(c, (n_cells + 1) * sizeof(int32_t));
  int32_t* ncol = (int32_t*)dev_alloc(c, nf * sizeof(int32_t));
  int* maxc = (int*)dev_alloc(c, sizeof(int));
  if (!c->probe_colour) c->probe_colour = (int32_t*)dev_alloc(c, n * sizeof(int32_t));
  if (!dcg || !keys || !ord || !cstart || !ncol || !maxc || !c->probe_colour)
    return set_error(c, GM_E_NOMEM, "probing colouring");
  GM_CUDA_CHECK(c, cudaMemcpyAsync(dcg, cg.data(), nf * sizeof(FieldGrid), cudaMemcpyHostToDevice, st));
  const int kb = (int)std::min<int64_t>(ceil_div(n_pad, 256), 16 * sms);
  GM_PROF(c, "k_probe_keys");
  k_probe_keys<<<kb, 256, 0, st>>>(n, n_pad, dcg, c->field_of, c->s, c->ux, c->uy, c->uz, keys);
  GM_LAUNCH_CHECK(c);
  {
    gm_status s = sort_u64(c, keys, n_pad);
    if (s != GM_OK) return s;
  }
  GM_PROF(c, "k_probe_order");
  k_probe_order<<<(int)std::min<int64_t>(ceil_div(n + 1, 256), 8 * sms), 256, 0, st>>>(
      n, n_cells, keys, ord, cstart);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaMemsetAsync(c->probe_colour, 0xff, n * sizeof(int32_t), st));
  GM_CUDA_CHECK(c, cudaMemsetAsync(maxc, 0, sizeof(int), st));
  // occupied cells of each class
  std::vector<int32_t> hcs(n_cells + 1);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hcs.data(), cstart, (n_cells + 1) * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  std::vector<int4> lists[8];
  for (int f = 0; f < nf; ++f) {
    const FieldGrid& q = cg[f];
    for (int x = 0; x < q.gx; ++x)
      for (int y = 0; y < q.gy; ++y)
        for (int z = 0; z < q.gz; ++z) {
          const int64_t id = q.cell_off + ((int64_t)x * q.gy + y) * q.gz + z;
          if (hcs[id + 1] > hcs[id]) lists[(x & 1) * 4 + (y & 1) * 2 + (z & 1)].push_back(make_int4(f, x, y, z));
        }
  }
  size_t lmax = 1;
  for (auto& l : lists) lmax = std::max(lmax, l.size());
  int4* dlist = (int4*)dev_alloc(c, lmax * sizeof(int4));
  if (!dlist) return set_error(c, GM_E_NOMEM, "probing cell lists");
  for (int k = 0; k < 8; ++k) {
    if (lists[k].empty()) continue;
    GM_CUDA_CHECK(c, cudaMemcpyAsync(dlist, lists[k].data(), lists[k].size() * sizeof(int4),
                                     cudaMemcpyHostToDevice, st));
    const int gb = (int)std::min<int64_t>((int64_t)lists[k].size(), 64 * sms);
    GM_PROF(c, "k_probe_greedy");
    k_probe_greedy<<<gb, 256, 0, st>>>((int64_t)lists[k].size(), dlist, dcg, cstart, ord, c->s,
                                        c->ux, c->uy, c->uz, c->probe_colour, maxc, c->d_flags);
    GM_LAUNCH_CHECK(c);
    // the list buffer is reused by the next class
    GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  }
  GM_PROF(c, "k_probe_field_ncol");
  k_probe_field_ncol<<<nf, 256, 0, st>>>(c->fptr, c->probe_colour, ncol);
  GM_LAUNCH_CHECK(c);
  c->h_probe_ncol.assign(nf, 0);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(c->h_probe_ncol.data(), ncol, nf * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, st));
  unsigned hf = 0;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(&hf, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  dev_free_now(c, dlist, lmax * sizeof(int4));
  dev_free_now(c, maxc, sizeof(int));
  dev_free_now(c, ncol, nf * sizeof(int32_t));
  dev_free_now(c, cstart, (n_cells + 1) * sizeof(int32_t));
  dev_free_now(c, ord, n * sizeof(int32_t));
  dev_free_now(c, keys, kb_bytes);
  dev_free_now(c, dcg, nf * sizeof(FieldGrid));
  if (hf & kFlagProbeOverflow) {
    GM_CUDA_CHECK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), st));
    c->probe_factor_done = 0;
    return set_error(c, GM_E_INVAL, "probing needs more than 131072 colours per field; "
                                    "lower probe_factor or use exact variances");
  }
  int64_t tot = 0;
  for (int f = 0; f < nf; ++f) tot += c->h_probe_ncol[f];
  c->stats.probe_colours = tot;
  c->probe_factor_done = fac;
  return GM_OK;
}

}  // namespace gm
