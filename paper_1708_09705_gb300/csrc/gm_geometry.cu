// Geometry, spatial ordering and the neighbour CSR (the sparsity pattern of
// the covariance: pairs whose 3-D separation is within the cutoff).
//
// Stars are renumbered by a stable sort on the id of the grid cell that
// holds them (cell edge >= cutoff), so that each cell owns a contiguous range
// of internal indices and a row's neighbours, visited cell by cell in
// increasing cell id, come out in increasing column order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

// ------------------------------------------------------------ unit vectors
__global__ void k_unit_vectors(int64_t n, const double* __restrict__ l,
                               const double* __restrict__ b, double* __restrict__ ux,
                               double* __restrict__ uy, double* __restrict__ uz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double sl, cl, sb, cb;
    sincos(l[i], &sl, &cl);
    sincos(b[i], &sb, &cb);
    ux[i] = cb * cl;
    uy[i] = cb * sl;
    uz[i] = sb;
  }
}

// Bounding box of each field's star positions: one block per field, fixed
// reduction order.  out[f*8 + 0..5] = min xyz, max xyz; out[f*8 + 6] = count.
__global__ void k_field_bbox(int64_t n, const int32_t* __restrict__ fid,
                             const double* __restrict__ s, const double* __restrict__ ux,
                             const double* __restrict__ uy, const double* __restrict__ uz,
                             double* __restrict__ out) {
  __shared__ double sh[7][256];
  const int f = blockIdx.x;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double cnt = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    if (fid && fid[i] != f) continue;
    double p[3] = {s[i] * ux[i], s[i] * uy[i], s[i] * uz[i]};
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], p[d]);
      hi[d] = fmax(hi[d], p[d]);
    }
    cnt += 1;
  }
  for (int d = 0; d < 3; ++d) {
    sh[d][threadIdx.x] = lo[d];
    sh[d + 3][threadIdx.x] = hi[d];
  }
  sh[6][threadIdx.x] = cnt;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      for (int d = 0; d < 3; ++d) {
        sh[d][threadIdx.x] = fmin(sh[d][threadIdx.x], sh[d][threadIdx.x + w]);
        sh[d + 3][threadIdx.x] = fmax(sh[d + 3][threadIdx.x], sh[d + 3][threadIdx.x + w]);
      }
      sh[6][threadIdx.x] += sh[6][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 7) out[(int64_t)f * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__device__ __forceinline__ void cell_coords(const FieldGrid& g, double x, double y, double z,
                                            int* cx, int* cy, int* cz) {
  int a = (int)floor((x - g.ox) * g.inv_cell);
  int b = (int)floor((y - g.oy) * g.inv_cell);
  int c = (int)floor((z - g.oz) * g.inv_cell);
  *cx = min(max(a, 0), g.gx - 1);
  *cy = min(max(b, 0), g.gy - 1);
  *cz = min(max(c, 0), g.gz - 1);
}

__global__ void k_cell_keys(int64_t n, int64_t n_pad, const FieldGrid* __restrict__ fg,
                            const int32_t* __restrict__ fid, const double* __restrict__ s,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            const double* __restrict__ uz, unsigned long long* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      const FieldGrid g = fg[fid ? fid[i] : 0];
      int cx, cy, cz;
      cell_coords(g, s[i] * ux[i], s[i] * uy[i], s[i] * uz[i], &cx, &cy, &cz);
      unsigned long long id =
          (unsigned long long)g.cell_off + ((unsigned long long)cx * g.gy + cy) * g.gz + cz;
      keys[i] = (id << 32) | (unsigned long long)i;
    } else {
      keys[i] = ~0ull;
    }
  }
}

// Bitonic sort, global compare-exchange pass for stride j >= 1024.
__global__ void k_bitonic_global(unsigned long long* a, int64_t n_pad, int64_t k, int64_t j) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = i ^ j;
    if (p > i) {
      bool asc = (i & k) == 0;
      unsigned long long x = a[i], y = a[p];
      if ((x > y) == asc) {
        a[i] = y;
        a[p] = x;
      }
    }
  }
}

// Bitonic sort, all strides j < 1024 of phase k inside one 1024-element tile.
__global__ void k_bitonic_shared(unsigned long long* a, int64_t n_pad, int64_t k, int64_t j0) {
  __shared__ unsigned long long t[1024];
  int64_t base = (int64_t)blockIdx.x * 1024;
  for (int q = threadIdx.x; q < 1024; q += blockDim.x) t[q] = a[base + q];
  __syncthreads();
  for (int64_t j = j0; j > 0; j >>= 1) {
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
      int p = q ^ (int)j;
      if (p > q) {
        bool asc = ((base + q) & k) == 0;
        unsigned long long x = t[q], y = t[p];
        if ((x > y) == asc) {
          t[q] = y;
          t[p] = x;
        }
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < 1024; q += blockDim.x) a[base + q] = t[q];
}

// Apply the sorted order: internal star k <- caller star (key & 0xffffffff).
__global__ void k_apply_perm(int64_t n, const unsigned long long* __restrict__ keys,
                             const double* __restrict__ s_in, const double* __restrict__ ux_in,
                             const double* __restrict__ uy_in, const double* __restrict__ uz_in,
                             const double* __restrict__ obs_in, const double* __restrict__ sig_in,
                             int64_t* __restrict__ perm, double* __restrict__ s,
                             double* __restrict__ ux, double* __restrict__ uy,
                             double* __restrict__ uz, double* __restrict__ obs,
                             double* __restrict__ sig, int32_t* __restrict__ cell_of,
                             const int32_t* __restrict__ fid, int32_t* __restrict__ field_of) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long key = keys[k];
    int64_t i = (int64_t)(key & 0xffffffffull);
    perm[k] = i;
    s[k] = s_in[i];
    ux[k] = ux_in[i];
    uy[k] = uy_in[i];
    uz[k] = uz_in[i];
    obs[k] = obs_in[i];
    sig[k] = sig_in[i];
    cell_of[k] = (int32_t)(key >> 32);
    field_of[k] = fid ? fid[i] : 0;
  }
}

// cell_start[c] = first internal index whose cell id >= c.
__global__ void k_cell_start(int64_t n, int64_t n_cells, const int32_t* __restrict__ cell_of,
                             int32_t* __restrict__ cell_start) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t prev = k == 0 ? -1 : cell_of[k - 1];
    int64_t cur = k == n ? n_cells : cell_of[k];
    for (int64_t c = prev + 1; c <= cur; ++c) cell_start[c] = (int32_t)k;
  }
}

// ------------------------------------------------------------ neighbours
// d^2 between a row point (s_r, u_r) and star j, in FP64 by the chord form
// (s_r - s_j)^2 + s_r s_j |u_r - u_j|^2, which is the squared 3-D distance.
__device__ __forceinline__ double dist2(double sr, double xr, double yr, double zr, double sj,
                                        double xj, double yj, double zj) {
  double dx = xr - xj, dy = yr - yj, dz = zr - zj;
  double ds = sr - sj;
  return fma(ds, ds, sr * sj * fma(dx, dx, fma(dy, dy, dz * dz)));
}

template <bool kFill>
__global__ void k_neighbours(int64_t n_rows, const FieldGrid* __restrict__ fg,
                             const int32_t* __restrict__ row_field, const double* __restrict__ rs,
                             const double* __restrict__ rux, const double* __restrict__ ruy,
                             const double* __restrict__ ruz, const double* __restrict__ s,
                             const double* __restrict__ ux, const double* __restrict__ uy,
                             const double* __restrict__ uz, const int32_t* __restrict__ cell_start,
                             int64_t* __restrict__ count_or_ptr, int32_t* __restrict__ col,
                             int64_t* __restrict__ diag_pos, bool self) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n_rows; r += nwarps) {
    const double sr = rs[r], xr = rux[r], yr = ruy[r], zr = ruz[r];
    const FieldGrid g = fg[row_field ? row_field[r] : 0];
    const double cut2 = g.cut2;
    int cx, cy, cz;
    cell_coords(g, sr * xr, sr * yr, sr * zr, &cx, &cy, &cz);
    int64_t pos = kFill ? count_or_ptr[r] : 0;
    int64_t cnt = 0;
    for (int dx = -1; dx <= 1; ++dx) {
      int ax = cx + dx;
      if (ax < 0 || ax >= g.gx) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        int ay = cy + dy;
        if (ay < 0 || ay >= g.gy) continue;
        // the three z-neighbours are consecutive cells: one contiguous range
        int z0 = max(cz - 1, 0), z1 = min(cz + 1, g.gz - 1);
        int64_t c0 = g.cell_off + ((int64_t)ax * g.gy + ay) * g.gz + z0;
        int64_t c1 = g.cell_off + ((int64_t)ax * g.gy + ay) * g.gz + z1 + 1;
        int32_t j0 = cell_start[c0], j1 = cell_start[c1];
        for (int32_t jb = j0; jb < j1; jb += 32) {
          int32_t j = jb + lane;
          bool in = false;
          if (j < j1) in = dist2(sr, xr, yr, zr, s[j], ux[j], uy[j], uz[j]) <= cut2;
          unsigned m = __ballot_sync(0xffffffffu, in);
          if (kFill) {
            if (in) {
              int64_t p = pos + cnt + __popc(m & ((1u << lane) - 1u));
              col[p] = j;
              if (self && j == r) diag_pos[r] = p;
            }
          }
          cnt += __popc(m);
        }
      }
    }
    if (!kFill && lane == 0) count_or_ptr[r] = cnt;
  }
}

// ------------------------------------------------------------ scan (int64)
// Exclusive scan of n counts into out[0..n] in three passes over 1024-element
// tiles (tile scan, scan of tile sums by one block, offset add).
__device__ __forceinline__ int64_t block_excl_scan_1024(int64_t v, int64_t* sh, int64_t* total) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t add = t >= off ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  int64_t incl = sh[t];
  *total = sh[1023];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(int64_t n, const int64_t* __restrict__ in,
                                                     int64_t* __restrict__ out,
                                                     int64_t* __restrict__ tile_sums) {
  __shared__ int64_t sh[1024];
  int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  int64_t tot;
  int64_t ex = block_excl_scan_1024(v, sh, &tot);
  if (i < n) out[i] = ex;
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t n_tiles, int64_t* __restrict__ sums,
                                                    int64_t* __restrict__ grand) {
  __shared__ int64_t sh[1024];
  int64_t carry = 0;
  for (int64_t b = 0; b < n_tiles; b += 1024) {
    int64_t i = b + threadIdx.x;
    int64_t v = i < n_tiles ? sums[i] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan_1024(v, sh, &tot);
    if (i < n_tiles) sums[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int64_t n, int64_t* __restrict__ out, const int64_t* __restrict__ sums,
                           const int64_t* __restrict__ grand) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i == n)
      out[n] = *grand;
    else
      out[i] += sums[i / 1024];
  }
}

// ------------------------------------------------------------ host side
gm_status sort_u64(gm_ctx* c, unsigned long long* keys, int64_t n_pad) {
  cudaStream_t st = c->stream;
  const int kb = (int)std::min<int64_t>(ceil_div(n_pad, 256), 16 * sm_count(c));
  for (int64_t k = 2; k <= n_pad; k <<= 1) {
    int64_t j = k >> 1;
    for (; j >= 1024; j >>= 1) {
      GM_PROF(c, "k_bitonic_global");
      k_bitonic_global<<<kb, 256, 0, st>>>(keys, n_pad, k, j);
      GM_LAUNCH_CHECK(c);
    }
    GM_PROF(c, "k_bitonic_shared");
    k_bitonic_shared<<<(unsigned)(n_pad / 1024), 512, 0, st>>>(keys, n_pad, k, j);
    GM_LAUNCH_CHECK(c);
  }
  return GM_OK;
}

gm_status scan_i64(gm_ctx* c, const int64_t* in, int64_t* out, int64_t n) {
  cudaStream_t st = c->stream;
  const int64_t n_tiles = ceil_div(n + 1, 1024);
  int64_t* sums = (int64_t*)dev_alloc(c, (n_tiles + 1) * sizeof(int64_t));
  if (!sums) return set_error(c, GM_E_NOMEM, "scan partials");
  GM_PROF(c, "k_scan_tiles");
  k_scan_tiles<<<(unsigned)ceil_div(n, 1024), 1024, 0, st>>>(n, in, out, sums);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_scan_sums");
  k_scan_sums<<<1, 1024, 0, st>>>(ceil_div(n, 1024), sums, sums + n_tiles);
  GM_LAUNCH_CHECK(c);
  const int ab = (int)std::min<int64_t>(ceil_div(n + 1, 256), 8 * sm_count(c));
  GM_PROF(c, "k_scan_add");
  k_scan_add<<<ab, 256, 0, st>>>(n, out, sums, sums + n_tiles);
  GM_LAUNCH_CHECK(c);
  dev_free_now(c, sums, (n_tiles + 1) * sizeof(int64_t));
  return GM_OK;
}

gm_status geometry_init(gm_ctx* c, const double* l, const double* b, const double* s,
                        const double* obs, const double* sig, const int32_t* fid,
                        const double* field_L0, const double* field_cut) {
  const int64_t n = c->n;
  const int nf = c->n_fields;
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 8 * sms);
  // caller-order scratch
  double* ux_in = (double*)dev_alloc(c, n * sizeof(double));
  double* uy_in = (double*)dev_alloc(c, n * sizeof(double));
  double* uz_in = (double*)dev_alloc(c, n * sizeof(double));
  double* bbox = (double*)dev_alloc(c, (size_t)nf * 8 * sizeof(double));
  if (!ux_in || !uy_in || !uz_in || !bbox) return set_error(c, GM_E_NOMEM, "geometry scratch");
  GM_PROF(c, "k_unit_vectors");
  k_unit_vectors<<<blocks, 256, 0, st>>>(n, l, b, ux_in, uy_in, uz_in);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_field_bbox");
  k_field_bbox<<<nf, 256, 0, st>>>(n, fid, s, ux_in, uy_in, uz_in, bbox);
  GM_LAUNCH_CHECK(c);
  std::vector<double> hb((size_t)nf * 8);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hb.data(), bbox, hb.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  // per-field grid: cell edge >= cutoff, at most 2^24 cells per field
  c->h_fgrid.assign(nf, FieldGrid{});
  c->h_fptr.assign(nf + 1, 0);
  int64_t off = 0;
  for (int f = 0; f < nf; ++f) {
    const double* B = hb.data() + (size_t)f * 8;
    const double L0 = field_L0 ? field_L0[f] : c->cfg.outer_scale_pc;
    const double cut = field_cut ? field_cut[f] : c->cfg.cutoff_pc;
    FieldGrid& g = c->h_fgrid[f];
    const int64_t cnt = (int64_t)B[6];
    double lo[3] = {B[0], B[1], B[2]}, hi[3] = {B[3], B[4], B[5]};
    if (cnt == 0)
      for (int d = 0; d < 3; ++d) lo[d] = hi[d] = 0.0;
    double cell = cut;
    int dims[3] = {1, 1, 1};
    for (int it = 0; it < 64; ++it) {
      int64_t tot = 1;
      for (int d = 0; d < 3; ++d) {
        dims[d] = (int)std::min<double>(std::floor((hi[d] - lo[d]) / cell) + 1.0, 1 << 24);
        tot *= dims[d];
      }
      if (tot <= (1ll << 24)) break;
      cell *= 1.26;
    }
    g.ox = lo[0];
    g.oy = lo[1];
    g.oz = lo[2];
    g.inv_cell = 1.0 / cell;
    g.cut2 = cut * cut;
    g.inv_cut = 1.0 / cut;
    g.inv_L0 = 1.0 / L0;
    g.gx = dims[0];
    g.gy = dims[1];
    g.gz = dims[2];
    g.cell_off = off;
    off += (int64_t)dims[0] * dims[1] * dims[2];
    c->h_fptr[f + 1] = c->h_fptr[f] + cnt;
  }
  if (off >= (1ll << 31) || c->h_fptr[nf] != n)
    return set_error(c, GM_E_INVAL, "field ids out of range or too many grid cells");
  c->n_cells = off;
  c->fgrid = (FieldGrid*)dev_alloc(c, (size_t)nf * sizeof(FieldGrid));
  c->fptr = (int64_t*)dev_alloc(c, (size_t)(nf + 1) * sizeof(int64_t));
  c->field_of = (int32_t*)dev_alloc(c, n * sizeof(int32_t));
  if (!c->fgrid || !c->fptr || !c->field_of) return set_error(c, GM_E_NOMEM, "field tables");
  GM_CUDA_CHECK(c, cudaMemcpyAsync(c->fgrid, c->h_fgrid.data(), nf * sizeof(FieldGrid),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(c->fptr, c->h_fptr.data(), (nf + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  const int64_t n_cells = c->n_cells;

  int64_t n_pad = 1024;
  while (n_pad < n) n_pad <<= 1;
  unsigned long long* keys = (unsigned long long*)dev_alloc(c, n_pad * sizeof(unsigned long long));
  int32_t* cell_of = (int32_t*)dev_alloc(c, n * sizeof(int32_t));
  c->cell_start = (int32_t*)dev_alloc(c, (n_cells + 1) * sizeof(int32_t));
  if (!keys || !cell_of || !c->cell_start) return set_error(c, GM_E_NOMEM, "cell grid");
  const int kb = (int)std::min<int64_t>(ceil_div(n_pad, 256), 16 * sms);
  GM_PROF(c, "k_cell_keys");
  k_cell_keys<<<kb, 256, 0, st>>>(n, n_pad, c->fgrid, fid, s, ux_in, uy_in, uz_in, keys);
  GM_LAUNCH_CHECK(c);
  {
    gm_status sst = sort_u64(c, keys, n_pad);
    if (sst != GM_OK) return sst;
  }
  GM_PROF(c, "k_apply_perm");
  k_apply_perm<<<blocks, 256, 0, st>>>(n, keys, s, ux_in, uy_in, uz_in, obs, sig, c->perm, c->s,
                                       c->ux, c->uy, c->uz, c->obs, c->obs_sigma, cell_of, fid,
                                       c->field_of);
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_cell_start");
  k_cell_start<<<blocks, 256, 0, st>>>(n, n_cells, cell_of, c->cell_start);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  dev_free_now(c, keys, n_pad * sizeof(unsigned long long));
  dev_free_now(c, cell_of, n * sizeof(int32_t));
  dev_free_now(c, bbox, (size_t)nf * 8 * sizeof(double));
  dev_free_now(c, uz_in, n * sizeof(double));
  dev_free_now(c, uy_in, n * sizeof(double));
  dev_free_now(c, ux_in, n * sizeof(double));
  return GM_OK;
}

gm_status unit_vectors(gm_ctx* c, int64_t n, const double* l, const double* b, double* ux,
                       double* uy, double* uz) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * sm_count(c)));
  GM_PROF(c, "k_unit_vectors");
  k_unit_vectors<<<blocks, 256, 0, c->stream>>>(n, l, b, ux, uy, uz);
  GM_LAUNCH_CHECK(c);
  return GM_OK;
}

gm_status neighbour_csr(gm_ctx* c, int64_t n_rows, const double* rs, const double* rux,
                        const double* ruy, const double* ruz, const int32_t* row_field, bool self,
                        int64_t* row_ptr, Buffer& col_buf, int64_t* nnz_out, int64_t* diag_pos) {
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  int64_t* counts = (int64_t*)dev_alloc(c, (n_rows + 1) * sizeof(int64_t));
  if (!counts) return set_error(c, GM_E_NOMEM, "neighbour counts");
  const int wb = (int)std::min<int64_t>(ceil_div(n_rows * 32, 256), 32 * sms);
  GM_PROF(c, "k_neighbours");
  k_neighbours<false><<<wb, 256, 0, st>>>(n_rows, c->fgrid, row_field, rs, rux, ruy, ruz, c->s, c->ux, c->uy,
                                          c->uz, c->cell_start, counts, nullptr, nullptr, self);
  GM_LAUNCH_CHECK(c);
  {
    gm_status sst = scan_i64(c, counts, row_ptr, n_rows);
    if (sst != GM_OK) return sst;
  }
  int64_t nnz = 0;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(&nnz, row_ptr + n_rows, sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  if (nnz >= (1ll << 40)) return set_error(c, GM_E_NOMEM, "neighbour count overflow");
  if (!ensure(c, col_buf, std::max<int64_t>(nnz, 1) * sizeof(int32_t)))
    return set_error(c, GM_E_NOMEM, "CSR column indices");
  GM_PROF(c, "k_neighbours");
  k_neighbours<true><<<wb, 256, 0, st>>>(n_rows, c->fgrid, row_field, rs, rux, ruy, ruz, c->s, c->ux, c->uy,
                                         c->uz, c->cell_start, row_ptr, (int32_t*)col_buf.p,
                                         diag_pos, self);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  dev_free_now(c, counts, (n_rows + 1) * sizeof(int64_t));
  *nnz_out = nnz;
  return GM_OK;
}

}  // namespace gm
