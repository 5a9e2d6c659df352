// Marginal variances for many independent fields at once.
//
// A context with several fields (independent sky fields / sub-catalogues,
// whose stars are never neighbours) has a block-diagonal K.  Each field f
// solves its own N_f right-hand sides against its own N_f rows, so its
// panels are N_f x W_f (W_f = N_f rounded up to 32) and all fields' panels
// are packed into one array (with probed variances a field's columns are
// its colour classes instead of its stars, W_f = classes rounded up to 32).
// Every CG step runs as one launch over all fields: the tiled panel product
// over (row block, column-chunk group)
// items, element-wise updates over (field, column chunk, row segment)
// items with per-column partial sums, and a per-column reduction that keeps
// each column's CG scalars.  The sequence of one iteration is captured as a
// CUDA graph (eight iterations per graph launch).  The panel product runs on
// the tensor cores over field-aligned 128-row tiles (prefetch depth tuned on
// first use) or, with GM_SPMM=simt, on the CUDA cores over 32-row tiles
// (block shape tuned on first use).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

constexpr int kSeg = 256;  // rows per element-wise work item
constexpr int kTileF = 32;

struct PackField {
  int64_t row0, nrows, W, P, Wptr, S, PO;
};

struct PackState {
  bool valid = false;
  int64_t total_elems = 0, total_cols = 0, total_parts = 0;
  std::vector<PackField> h_pf;
  PackField* pf = nullptr;
  int64_t* wptr = nullptr;       // n_fields + 1 column offsets
  int4* eitems = nullptr;        // (f, chunk, segment, -)
  int64_t n_eitems = 0;
  int2* sitems = nullptr;        // (block, chunk group)
  int64_t n_sitems4 = 0, n_sitems8 = 0;
  int2* sitems4 = nullptr;
  int32_t* blk_field = nullptr;
  Buffer X, R, Pp, PD, Q, pa, pb, scal, active;
  int wpb = 0;                   // tuned warps per block of the panel product (4 or 8)
  // tensor-core product: (tile block, column group) items, per-block panel base and width
  int2* tc_items = nullptr;
  int64_t n_tc_items = 0;
  int64_t* tc_base = nullptr;
  int32_t* tc_width = nullptr;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

static PackState& PS(gm_ctx* c) {
  if (!c->pack) c->pack = new PackState();
  return *c->pack;
}

void pack_free(gm_ctx* c) {
  if (!c->pack) return;
  if (c->pack->gstream) cudaStreamDestroy(c->pack->gstream);
  if (c->pack->ev0) cudaEventDestroy(c->pack->ev0);
  if (c->pack->ev1) cudaEventDestroy(c->pack->ev1);
  delete c->pack;
  c->pack = nullptr;
}

void pack_invalidate(gm_ctx* c) {
  if (c->pack) c->pack->valid = false;
}

// ---------------------------------------------------------------- kernels
// Right-hand sides: column c of field f solves for star row0_f + c with
// e_c (site-dominated star) or d o k_c, as in the single-panel solver.
__global__ void k_pk_rhs(int64_t n, const int32_t* __restrict__ field_of,
                         const PackField* __restrict__ pf, const int64_t* __restrict__ row_ptr,
                         const int32_t* __restrict__ col, const float* __restrict__ val,
                         const float* __restrict__ dv, const double* __restrict__ tau,
                         const double* __restrict__ kd, float* __restrict__ Rr) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nw) {
    const PackField F = pf[field_of[r]];
    const int64_t cc = r - F.row0;
    if (tau[r] * kd[r] >= 1.0) {
      if (lane == 0) Rr[F.P + cc * F.W + cc] = 1.f;
      continue;
    }
    for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
      const int32_t j = col[e];
      Rr[F.P + (j - F.row0) * F.W + cc] = dv[j] * val[e];
    }
  }
}

// Probed right-hand sides: column k of field f sums the right-hand sides of
// the field's stars of colour class k; thread per row j (fixed summation
// order), as in the single-panel solver.
__global__ void k_pk_rhs_probe(int64_t n, const int32_t* __restrict__ field_of,
                               const PackField* __restrict__ pf, const int64_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, const float* __restrict__ val,
                               const float* __restrict__ dv, const double* __restrict__ tau,
                               const double* __restrict__ kd, const int32_t* __restrict__ pcol,
                               float* __restrict__ Rr) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const PackField F = pf[field_of[j]];
    float* row = Rr + F.P + (j - F.row0) * F.W;
    const float dj = dv[j];
    for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
      const int32_t r = col[e];
      if (tau[r] * kd[r] >= 1.0) continue;
      row[pcol[r]] += dj * val[e];
    }
    if (tau[j] * kd[j] >= 1.0) row[pcol[j]] += 1.f;
  }
}

enum { kPkInit = 0, kPkPQ = 1, kPkUpd1 = 2, kPkUpd2 = 3 };

// Element-wise pass over (field, column chunk, row segment) items; one warp
// per item, lane = column.  Partials pa/pb at PO_f + s W_f + c.
template <int MODE>
__global__ void k_pk_elem(int64_t n_items, const int4* __restrict__ items,
                          const PackField* __restrict__ pf, const float* __restrict__ minv,
                          const float* __restrict__ dv, const double* __restrict__ scal,
                          int64_t tcols, const int* __restrict__ active, float* __restrict__ X,
                          float* __restrict__ Rr, float* __restrict__ P, float* __restrict__ PD,
                          const float* __restrict__ Q, double* __restrict__ pa,
                          double* __restrict__ pb) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < n_items; it += nw) {
    const int4 w = items[it];
    const PackField F = pf[w.x];
    const int64_t c = (int64_t)w.y * 32 + lane;
    const int64_t gid = F.Wptr + c;
    const int64_t i0 = (int64_t)w.z * kSeg, i1 = min(i0 + kSeg, F.nrows);
    PartialSum<float> s1, s2;
    if (MODE == kPkUpd2 && !active[gid]) continue;
    const float alpha = MODE == kPkUpd1 ? (float)scal[gid] : 0.f;
    const float beta = MODE == kPkUpd2 ? (float)scal[tcols + gid] : 0.f;
    for (int64_t i = i0; i < i1; ++i) {
      const int64_t k = F.P + i * F.W + c;
      const int64_t r = F.row0 + i;
      if (MODE == kPkInit) {
        const float ri = Rr[k], zi = minv[r] * ri;
        X[k] = 0.f;
        P[k] = zi;
        PD[k] = dv[r] * zi;
        s1.add(ri * zi);
        s2.add(ri * ri);
      } else if (MODE == kPkPQ) {
        s1.add(P[k] * Q[k]);
      } else if (MODE == kPkUpd1) {
        X[k] += alpha * P[k];
        const float ri = Rr[k] - alpha * Q[k];
        Rr[k] = ri;
        s1.add(ri * (minv[r] * ri));
        s2.add(ri * ri);
      } else {
        const float pi = minv[r] * Rr[k] + beta * P[k];
        P[k] = pi;
        PD[k] = dv[r] * pi;
      }
    }
    if (MODE != kPkUpd2) {
      const int64_t po = F.PO + (int64_t)w.z * F.W + c;
      pa[po] = s1.value();
      if (MODE != kPkPQ) pb[po] = s2.value();
    }
  }
}

// Per-column sums of the partials of its field's segments, and the CG
// scalars (scal layout: alpha, beta, rz_prev, rz_new, bb, rr; each tcols).
__global__ void k_pk_reduce(int mode, int64_t tcols, int n_fields, const int64_t* __restrict__ wptr,
                            const PackField* __restrict__ pf, double tol2,
                            const double* __restrict__ pa, const double* __restrict__ pb,
                            double* __restrict__ scal, int* __restrict__ active,
                            int* __restrict__ n_active, unsigned* __restrict__ flags) {
  for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < tcols;
       gid += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_fields;  // field: wptr[lo] <= gid < wptr[lo+1]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (wptr[mid] <= gid) lo = mid; else hi = mid;
    }
    const PackField F = pf[lo];
    const int64_t c = gid - F.Wptr;
    double a = 0, b = 0;
    for (int64_t s = 0; s < F.S; ++s) {
      a += pa[F.PO + s * F.W + c];
      if (pb) b += pb[F.PO + s * F.W + c];
    }
    double* alpha = scal;
    double* beta = scal + tcols;
    double* rzp = scal + 2 * tcols;
    double* bb = scal + 4 * tcols;
    double* rr = scal + 5 * tcols;
    if (mode == 0) {
      rzp[gid] = a;
      bb[gid] = b;
      rr[gid] = b;
      const int act = (c < F.nrows) && (b > 0);
      active[gid] = act;
      if (act) atomicAdd(n_active, 1);
    } else if (mode == 1) {
      double al = 0;
      if (active[gid]) {
        if (a > 0 && rzp[gid] > 0) al = rzp[gid] / a;
        else if (rzp[gid] > 0) {
          atomicOr(flags, kFlagNotSPD);
          active[gid] = 0;
        }
      }
      alpha[gid] = al;
    } else {
      rr[gid] = b;
      double be = 0;
      if (active[gid]) {
        if (!isfinite(a) || !isfinite(b)) {
          atomicOr(flags, kFlagNonFinite);
          active[gid] = 0;
        } else if (b <= tol2 * bb[gid]) {
          active[gid] = 0;
        } else {
          be = rzp[gid] > 0 ? a / rzp[gid] : 0.0;
          atomicAdd(n_active, 1);
        }
      }
      beta[gid] = be;
      rzp[gid] = a;
    }
  }
}

// Q = P + d o (K PD) for all fields: item = (row block b, group of WPB
// column chunks of b's field).  Same register-blocked inner product as the
// single-panel kernel.
template <int WPB>
__global__ void __launch_bounds__(WPB * 32) k_pk_spmm(
    int64_t n_items, const int2* __restrict__ items, const int32_t* __restrict__ blk_field,
    const PackField* __restrict__ pf, const int64_t* __restrict__ blk_row0,
    const int64_t* __restrict__ bptr, const int32_t* __restrict__ ucol,
    const float* __restrict__ tval, const float* __restrict__ dv, const float* __restrict__ P,
    const float* __restrict__ PD, float* __restrict__ Q) {
  __shared__ float4 sA[kTileF * kTileF / 4];
  __shared__ float4 sB[WPB][kTileF * kTileF / 4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int rg = lane >> 2, cg = lane & 3;
  float* sBw = reinterpret_cast<float*>(sB[wib]);
  for (int64_t itm = blockIdx.x; itm < n_items; itm += gridDim.x) {
    const int2 w = items[itm];
    const int64_t b = w.x;
    const PackField F = pf[blk_field[b]];
    const int64_t c0 = ((int64_t)w.y * WPB + wib) * 32;
    const bool live = c0 < F.W;
    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
    const int64_t u0 = bptr[b], u1 = bptr[b + 1];
    for (int64_t ub = u0; ub < u1; ub += 32) {
      const int cnt = (u1 - ub) < 32 ? (int)(u1 - ub) : 32;
      __syncthreads();
      for (int t = threadIdx.x; t < kTileF * kTileF / 4; t += WPB * 32) {
        const int k = t >> 3, q = t & 7;
        sA[t] = k < cnt ? __ldg(reinterpret_cast<const float4*>(tval + (ub + k) * kTileF) + q)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const int jl = lane < cnt ? ucol[ub + lane] : 0;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const int64_t j = __shfl_sync(0xffffffffu, jl, k);
        sBw[k * 32 + lane] =
            (live && k < cnt) ? PD[F.P + (j - F.row0) * F.W + c0 + lane] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        const float4 a = sA[k * 8 + rg];
        const float4 b0 = sB[wib][k * 8 + 2 * cg];
        const float4 b1 = sB[wib][k * 8 + 2 * cg + 1];
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
      }
    }
    if (live) {
      const int64_t r0b = blk_row0[b], r1b = blk_row0[b + 1];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t i = r0b + 4 * rg + r;
        if (i < r1b) {
          const float di = dv[i];
          const int64_t k0 = F.P + (i - F.row0) * F.W + c0 + 8 * cg;
          const float4 p0 = *reinterpret_cast<const float4*>(P + k0);
          const float4 p1 = *reinterpret_cast<const float4*>(P + k0 + 4);
          const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
          float qv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) qv[q] = pv[q] + di * acc[r][q];
          *reinterpret_cast<float4*>(Q + k0) = make_float4(qv[0], qv[1], qv[2], qv[3]);
          *reinterpret_cast<float4*>(Q + k0 + 4) = make_float4(qv[4], qv[5], qv[6], qv[7]);
        }
      }
    }
  }
}

__global__ void k_pk_final(int64_t n, const int32_t* __restrict__ field_of,
                           const PackField* __restrict__ pf, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, const float* __restrict__ val,
                           const double* __restrict__ d64, const float* __restrict__ X,
                           const double* __restrict__ kd, const double* __restrict__ tau,
                           const int32_t* __restrict__ pcol, double* __restrict__ var_out,
                           unsigned* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nw) {
    const PackField F = pf[field_of[r]];
    // the star's column: its own, or its colour class's when probing
    const int64_t cc = pcol ? (int64_t)pcol[r] : r - F.row0;
    double v;
    if (tau[r] * kd[r] >= 1.0) {
      v = (1.0 - (double)X[F.P + (r - F.row0) * F.W + cc]) / tau[r];
    } else {
      double acc = 0;
      for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) {
        const int32_t j = col[e];
        acc += d64[j] * (double)val[e] * (double)X[F.P + (j - F.row0) * F.W + cc];
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      v = kd[r] - acc;
    }
    if (lane == 0) {
      if (!isfinite(v)) atomicOr(flags, kFlagNonFinite);
      var_out[r] = v;
    }
  }
}

// ---------------------------------------------------------------- host
static gm_status pack_setup(gm_ctx* c) {
  PackState& S = PS(c);
  if (S.valid) return GM_OK;
  const int nf = c->n_fields;
  S.h_pf.assign(nf, PackField{});
  std::vector<int64_t> wptr(nf + 1, 0);
  std::vector<int4> eit;
  int64_t P = 0, Wp = 0, PO = 0;
  const bool probe = c->probe_colour && c->probe_factor_done > 0;
  for (int f = 0; f < nf; ++f) {
    PackField& F = S.h_pf[f];
    F.row0 = c->h_fptr[f];
    F.nrows = c->h_fptr[f + 1] - F.row0;
    const int64_t cols = probe ? (int64_t)c->h_probe_ncol[f] : F.nrows;
    F.W = ceil_div(std::max<int64_t>(cols, 1), 32) * 32;
    F.P = P;
    F.Wptr = Wp;
    F.S = std::max<int64_t>(1, ceil_div(F.nrows, kSeg));
    F.PO = PO;
    P += F.nrows * F.W;
    Wp += F.W;
    PO += F.S * F.W;
    wptr[f + 1] = Wp;
    for (int64_t k = 0; k < F.W / 32; ++k)
      for (int64_t s = 0; s < F.S; ++s) eit.push_back(make_int4(f, (int)k, (int)s, 0));
  }
  S.total_elems = P;
  S.total_cols = Wp;
  S.total_parts = PO;
  S.n_eitems = (int64_t)eit.size();
  std::vector<int2> it8, it4;
  std::vector<int32_t> bf(c->t_nblk);
  // CUDA-core 32-row tiles exist only when the tensor-core tiles were not
  // built (their block table h_boff is empty otherwise)
  for (int f = 0; c->t_nblk > 0 && f < nf; ++f) {
    const int64_t chunks = S.h_pf[f].W / 32;
    for (int64_t b = c->h_boff[f]; b < c->h_boff[f + 1]; ++b) {
      bf[b] = f;
      for (int64_t g = 0; g < ceil_div(chunks, 8); ++g) it8.push_back(make_int2((int)b, (int)g));
      for (int64_t g = 0; g < ceil_div(chunks, 4); ++g) it4.push_back(make_int2((int)b, (int)g));
    }
  }
  S.n_sitems8 = (int64_t)it8.size();
  S.n_sitems4 = (int64_t)it4.size();
  // tensor-core tiles (field-aligned 128-row blocks): items and panel geometry
  std::vector<int2> itc;
  std::vector<int64_t> tbase(std::max<int64_t>(c->tc_nblk, 1), 0);
  std::vector<int32_t> twidth(std::max<int64_t>(c->tc_nblk, 1), 0);
  if (c->tc_nblk > 0) {
    for (int f = 0; f < nf; ++f) {
      const PackField& F = S.h_pf[f];
      for (int64_t b = c->h_tc_boff[f]; b < c->h_tc_boff[f + 1]; ++b) {
        tbase[b] = F.P - F.row0 * F.W;
        twidth[b] = (int32_t)F.W;
        for (int64_t g = 0; g < ceil_div(F.W, 256); ++g) itc.push_back(make_int2((int)b, (int)g));
      }
    }
  }
  S.n_tc_items = (int64_t)itc.size();
  cudaStream_t st = c->stream;
  S.pf = (PackField*)dev_alloc(c, nf * sizeof(PackField));
  S.wptr = (int64_t*)dev_alloc(c, (nf + 1) * sizeof(int64_t));
  S.eitems = (int4*)dev_alloc(c, std::max<int64_t>(1, S.n_eitems) * sizeof(int4));
  S.sitems = (int2*)dev_alloc(c, std::max<int64_t>(1, S.n_sitems8) * sizeof(int2));
  S.sitems4 = (int2*)dev_alloc(c, std::max<int64_t>(1, S.n_sitems4) * sizeof(int2));
  S.blk_field = (int32_t*)dev_alloc(c, std::max<int64_t>(1, c->t_nblk) * sizeof(int32_t));
  S.tc_items = (int2*)dev_alloc(c, std::max<int64_t>(1, S.n_tc_items) * sizeof(int2));
  S.tc_base = (int64_t*)dev_alloc(c, tbase.size() * sizeof(int64_t));
  S.tc_width = (int32_t*)dev_alloc(c, twidth.size() * sizeof(int32_t));
  if (!S.pf || !S.wptr || !S.eitems || !S.sitems || !S.sitems4 || !S.blk_field || !S.tc_items ||
      !S.tc_base || !S.tc_width)
    return set_error(c, GM_E_NOMEM, "field pack tables");
  if (S.n_tc_items > 0)
    GM_CUDA_CHECK(c, cudaMemcpyAsync(S.tc_items, itc.data(), S.n_tc_items * sizeof(int2),
                                     cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.tc_base, tbase.data(), tbase.size() * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.tc_width, twidth.data(), twidth.size() * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.pf, S.h_pf.data(), nf * sizeof(PackField), cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.wptr, wptr.data(), (nf + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.eitems, eit.data(), S.n_eitems * sizeof(int4), cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.sitems, it8.data(), S.n_sitems8 * sizeof(int2), cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.sitems4, it4.data(), S.n_sitems4 * sizeof(int2), cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaMemcpyAsync(S.blk_field, bf.data(), c->t_nblk * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  const size_t eb = (size_t)S.total_elems * sizeof(float);
  bool ok = ensure(c, S.X, eb) && ensure(c, S.R, eb) && ensure(c, S.Pp, eb) && ensure(c, S.PD, eb) &&
            ensure(c, S.Q, eb) && ensure(c, S.pa, (size_t)S.total_parts * sizeof(double)) &&
            ensure(c, S.pb, (size_t)S.total_parts * sizeof(double)) &&
            ensure(c, S.scal, 6 * (size_t)S.total_cols * sizeof(double)) &&
            ensure(c, S.active, (size_t)(S.total_cols + 32) * sizeof(int));
  if (!ok) return set_error(c, GM_E_NOMEM, "field panels");
  if (!S.gstream) {
    GM_CUDA_CHECK(c, cudaStreamCreateWithFlags(&S.gstream, cudaStreamNonBlocking));
    GM_CUDA_CHECK(c, cudaEventCreateWithFlags(&S.ev0, cudaEventDisableTiming));
    GM_CUDA_CHECK(c, cudaEventCreateWithFlags(&S.ev1, cudaEventDisableTiming));
  }
  S.valid = true;
  return GM_OK;
}

static void launch_spmm(gm_ctx* c, PackState& S, int wpb, cudaStream_t st, const float* dv) {
  if (S.n_tc_items > 0) {
    panel_spmm_tc_packed(c, S.n_tc_items, S.tc_items, S.tc_base, S.tc_width, dv,
                         (const float*)S.Pp.p, (const float*)S.PD.p, (float*)S.Q.p,
                         (int64_t)(S.PD.bytes / sizeof(float)), st, false);
    return;
  }
  const int sms = sm_count(c);
  if (wpb == 4) {
    const int g = (int)std::min<int64_t>(S.n_sitems4, 8 * sms);
    k_pk_spmm<4><<<g, 128, 0, st>>>(S.n_sitems4, S.sitems4, S.blk_field, S.pf, c->blk_row0,
                                    (const int64_t*)c->t_bptr.p, (const int32_t*)c->t_ucol.p,
                                    (const float*)c->t_val.p, dv, (const float*)S.Pp.p,
                                    (const float*)S.PD.p, (float*)S.Q.p);
  } else {
    const int g = (int)std::min<int64_t>(S.n_sitems8, 4 * sms);
    k_pk_spmm<8><<<g, 256, 0, st>>>(S.n_sitems8, S.sitems, S.blk_field, S.pf, c->blk_row0,
                                    (const int64_t*)c->t_bptr.p, (const int32_t*)c->t_ucol.p,
                                    (const float*)c->t_val.p, dv, (const float*)S.Pp.p,
                                    (const float*)S.PD.p, (float*)S.Q.p);
  }
}

// Times both block shapes of the panel product once and keeps the faster;
// the choice can be pinned with GM_PANEL_WARPS=4|8.
static gm_status autotune(gm_ctx* c, PackState& S, const float* dv) {
  if (S.n_tc_items > 0)
    return panel_spmm_tc_packed(c, S.n_tc_items, S.tc_items, S.tc_base, S.tc_width, dv,
                                (const float*)S.Pp.p, (const float*)S.PD.p, (float*)S.Q.p,
                                (int64_t)(S.PD.bytes / sizeof(float)), c->stream, true);
  if (S.wpb) return GM_OK;
  if (const char* env = std::getenv("GM_PANEL_WARPS")) {
    const int w = std::atoi(env);
    if (w == 4 || w == 8) {
      S.wpb = w;
      return GM_OK;
    }
  }
  cudaEvent_t a, b;
  GM_CUDA_CHECK(c, cudaEventCreate(&a));
  GM_CUDA_CHECK(c, cudaEventCreate(&b));
  float best = 1e30f;
  for (int w : {8, 4}) {
    float t = 0;
    for (int rep = 0; rep < 2; ++rep) {  // second launch timed
      GM_CUDA_CHECK(c, cudaEventRecord(a, c->stream));
      launch_spmm(c, S, w, c->stream, dv);
      GM_CUDA_CHECK(c, cudaEventRecord(b, c->stream));
      GM_CUDA_CHECK(c, cudaEventSynchronize(b));
      GM_CUDA_CHECK(c, cudaEventElapsedTime(&t, a, b));
    }
    c->launches += 2;
    if (t < best) {
      best = t;
      S.wpb = w;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return GM_OK;
}

gm_status panels_fields(gm_ctx* c, const float* dv, const float* minv, const double* d64,
                        double* var_out, int64_t* iters_out, double* resid_out) {
  gm_status s = pack_setup(c);
  if (s != GM_OK) return s;
  PackState& S = PS(c);
  const int64_t n = c->n, tc = S.total_cols;
  cudaStream_t st = c->stream;
  const int sms = sm_count(c);
  float *X = (float*)S.X.p, *Rr = (float*)S.R.p, *P = (float*)S.Pp.p, *PD = (float*)S.PD.p,
        *Q = (float*)S.Q.p;
  double *pa = (double*)S.pa.p, *pb = (double*)S.pb.p, *scal = (double*)S.scal.p;
  int* active = (int*)S.active.p;
  int* n_active = active + tc;
  const double tol = std::max(c->cfg.cg_tol, 1e-5);
  const double tol2 = tol * tol;
  const int wb = (int)std::min<int64_t>(ceil_div(n * 32, 256), 16 * sms);
  const int ib = (int)std::min<int64_t>(ceil_div(S.n_eitems * 32, 256), 16 * sms);
  const int rb = (int)std::min<int64_t>(ceil_div(tc, 256), 8 * sms);
  const int nf = c->n_fields;
  const bool probe = c->probe_colour && c->probe_factor_done > 0;
  GM_CUDA_CHECK(c, cudaMemsetAsync(Rr, 0, (size_t)S.total_elems * sizeof(float), st));
  if (probe) {
    GM_PROF(c, "k_pk_rhs_probe");
    k_pk_rhs_probe<<<(int)std::min<int64_t>(ceil_div(n, 256), 16 * sms), 256, 0, st>>>(
        n, c->field_of, S.pf, c->row_ptr, c->col, (const float*)c->val, dv, c->tau, c->kdiag,
        c->probe_colour, Rr);
  } else {
    GM_PROF(c, "k_pk_rhs");
    k_pk_rhs<<<wb, 256, 0, st>>>(n, c->field_of, S.pf, c->row_ptr, c->col, (const float*)c->val,
                                 dv, c->tau, c->kdiag, Rr);
  }
  GM_LAUNCH_CHECK(c);
  GM_PROF(c, "k_pk_elem_init");
  k_pk_elem<kPkInit><<<ib, 256, 0, st>>>(S.n_eitems, S.eitems, S.pf, minv, dv, scal, tc, active,
                                         X, Rr, P, PD, Q, pa, pb);
  GM_LAUNCH_CHECK(c);
  GM_CUDA_CHECK(c, cudaMemsetAsync(n_active, 0, sizeof(int), st));
  GM_PROF(c, "k_pk_reduce");
  k_pk_reduce<<<rb, 256, 0, st>>>(0, tc, nf, S.wptr, S.pf, tol2, pa, pb, scal, active, n_active,
                                  c->d_flags);
  GM_LAUNCH_CHECK(c);
  int* hn = (int*)c->h_pinned;
  GM_CUDA_CHECK(c, cudaMemcpyAsync(hn, n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  int64_t iters = 0;
  if (*hn > 0) {
    s = autotune(c, S, dv);
    if (s != GM_OK) return s;
    // one CUDA graph = 8 CG iterations on the private stream
    const int chunk = 8;
    GM_CUDA_CHECK(c, cudaEventRecord(S.ev0, st));
    GM_CUDA_CHECK(c, cudaStreamWaitEvent(S.gstream, S.ev0, 0));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GM_CUDA_CHECK(c, cudaStreamBeginCapture(S.gstream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < chunk; ++k) {
      launch_spmm(c, S, S.wpb, S.gstream, dv);
      k_pk_elem<kPkPQ><<<ib, 256, 0, S.gstream>>>(S.n_eitems, S.eitems, S.pf, minv, dv, scal, tc,
                                                  active, X, Rr, P, PD, Q, pa, pb);
      k_pk_reduce<<<rb, 256, 0, S.gstream>>>(1, tc, nf, S.wptr, S.pf, tol2, pa, nullptr, scal,
                                             active, n_active, c->d_flags);
      k_pk_elem<kPkUpd1><<<ib, 256, 0, S.gstream>>>(S.n_eitems, S.eitems, S.pf, minv, dv, scal, tc,
                                                    active, X, Rr, P, PD, Q, pa, pb);
      cudaMemsetAsync(n_active, 0, sizeof(int), S.gstream);
      k_pk_reduce<<<rb, 256, 0, S.gstream>>>(2, tc, nf, S.wptr, S.pf, tol2, pa, pb, scal, active,
                                             n_active, c->d_flags);
      k_pk_elem<kPkUpd2><<<ib, 256, 0, S.gstream>>>(S.n_eitems, S.eitems, S.pf, minv, dv, scal, tc,
                                                    active, X, Rr, P, PD, Q, pa, pb);
    }
    cudaError_t ce = cudaStreamEndCapture(S.gstream, &graph);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "graph capture");
    GM_CUDA_CHECK(c, cudaGraphInstantiate(&exec, graph, 0));
    const int max_it = c->cfg.cg_max_iter;
    for (int done = 0; done < max_it; done += chunk) {
      c->prof_stream = S.gstream;
      GM_PROF(c, "graph_cg8");
      GM_CUDA_CHECK(c, cudaGraphLaunch(exec, S.gstream));
      c->launches += 6 * chunk - 1;
      GM_LAUNCH_CHECK(c);
      c->prof_stream = nullptr;
      iters += chunk;
      GM_CUDA_CHECK(c, cudaMemcpyAsync(hn, n_active, sizeof(int), cudaMemcpyDeviceToHost, S.gstream));
      GM_CUDA_CHECK(c, cudaStreamSynchronize(S.gstream));
      if (*hn == 0) break;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    GM_CUDA_CHECK(c, cudaEventRecord(S.ev1, S.gstream));
    GM_CUDA_CHECK(c, cudaStreamWaitEvent(st, S.ev1, 0));
  }
  GM_PROF(c, "k_pk_final");
  k_pk_final<<<wb, 256, 0, st>>>(n, c->field_of, S.pf, c->row_ptr, c->col, (const float*)c->val,
                                 d64, X, c->kdiag, c->tau, probe ? c->probe_colour : nullptr,
                                 var_out, c->d_flags);
  GM_LAUNCH_CHECK(c);
  std::vector<double> h(2 * tc);
  GM_CUDA_CHECK(c, cudaMemcpyAsync(h.data(), scal + 4 * tc, 2 * tc * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
  GM_CUDA_CHECK(c, cudaStreamSynchronize(st));
  double worst = 0;
  for (int64_t k = 0; k < tc; ++k)
    if (h[k] > 0) worst = std::max(worst, std::sqrt(h[tc + k] / h[k]));
  *iters_out = iters;
  *resid_out = worst;
  return GM_OK;
}

}  // namespace gm
