// H^2 matrix-vector products (the representation of Sect. 4 applied with
// the standard H^2 recursion):
//
//   gather        x in original order -> xp in cluster order, [n][R]
//   forward leaf  x-hat_tau = V_tau^T x|tau-hat                  (leaves)
//   forward up    x-hat_tau = sum_children E_c^T x-hat_c          (per level)
//   coupling      y-hat_tau = sum_sigma S_{tau sigma} x-hat_sigma (all levels)
//   backward      y-hat_c  += E_c y-hat_parent                    (per level)
//   leaf output   y|tau-hat = V_tau y-hat_tau + sum N_{tau sigma} x|sigma-hat,
//                 scattered straight to the original order.
//
// The transposed product uses the same data: S_{tau sigma}^T grouped by the
// column cluster and N^T grouped by the column leaf.
//
// Layouts: vectors in cluster order are row-major [rows][R]; V_tau is
// |tau-hat| x r row-major, E_c is r_c x r_parent row-major, S and N blocks
// row-major.  Storage type TM (double / float / bfloat16), arithmetic and
// vector type TV (double / float).

#include <cuda_bf16.h>

#include <algorithm>

#include "internal.hpp"

namespace gca {

namespace {

__device__ __forceinline__ double ld(const double* p) { return *p; }
__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <typename TV>
__global__ void k_gather(int n, int R, const int* __restrict__ perm, const TV* __restrict__ x,
                         int64_t ldx, TV* __restrict__ xp) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * R) return;
  const int i = (int)(idx / R), c = (int)(idx % R);
  xp[idx] = x[perm[i] + c * ldx];
}

template <typename TM, typename TV>
__global__ void k_forward_leaf(const int* __restrict__ leaves, const int* __restrict__ begin,
                               const int* __restrict__ end, const int64_t* __restrict__ voff,
                               const int64_t* __restrict__ xoff, const int* __restrict__ rank,
                               const TM* __restrict__ V, const TV* __restrict__ xp,
                               TV* __restrict__ xh, int R) {
  const int c = leaves[blockIdx.x];
  const int r = rank[c], b = begin[c], nr = end[c] - b;
  const TM* Vc = V + voff[c];
  for (int idx = threadIdx.x; idx < r * R; idx += blockDim.x) {
    const int a = idx / R, cc = idx % R;
    TV s = 0;
    for (int i = 0; i < nr; ++i) s += (TV)ld(Vc + (int64_t)i * r + a) * xp[(int64_t)(b + i) * R + cc];
    xh[(xoff[c] + a) * R + cc] = s;
  }
}

template <typename TM, typename TV>
__global__ void k_forward_up(const int* __restrict__ list, const int* __restrict__ child0,
                             const int* __restrict__ child1, const int64_t* __restrict__ eoff,
                             const int64_t* __restrict__ xoff, const int* __restrict__ rank,
                             const TM* __restrict__ E, TV* __restrict__ xh, int R) {
  const int c = list[blockIdx.x];
  const int r = rank[c];
  for (int idx = threadIdx.x; idx < r * R; idx += blockDim.x) {
    const int a = idx / R, cc = idx % R;
    TV s = 0;
    for (int h = 0; h < 2; ++h) {
      const int ch = h ? child1[c] : child0[c];
      const int rc = rank[ch];
      const TM* Ec = E + eoff[ch];
      const TV* xc = xh + xoff[ch] * R;
      for (int b = 0; b < rc; ++b) s += (TV)ld(Ec + (int64_t)b * r + a) * xc[(int64_t)b * R + cc];
    }
    xh[(xoff[c] + a) * R + cc] = s;
  }
}

// one CTA per row cluster (or column cluster when transposed)
template <typename TM, typename TV, bool TRANS>
__global__ void k_couple(const int* __restrict__ list, const int* __restrict__ ptr,
                         const int* __restrict__ blk, const int* __restrict__ far_t,
                         const int* __restrict__ far_s, const int64_t* __restrict__ soff,
                         const int64_t* __restrict__ xoff, const int* __restrict__ rank,
                         const TM* __restrict__ S, const TV* __restrict__ xh,
                         TV* __restrict__ yh, int R) {
  const int c = list[blockIdx.x];
  const int r = rank[c];
  for (int idx = threadIdx.x; idx < r * R; idx += blockDim.x) {
    const int a = idx / R, cc = idx % R;
    TV s = 0;
    for (int e = ptr[c]; e < ptr[c + 1]; ++e) {
      const int b = blk[e];
      const TM* Sb = S + soff[b];
      if (!TRANS) {
        const int o = far_s[b], ro = rank[o];
        const TV* xo = xh + xoff[o] * R;
        for (int j = 0; j < ro; ++j) s += (TV)ld(Sb + (int64_t)a * ro + j) * xo[(int64_t)j * R + cc];
      } else {
        const int o = far_t[b], ro = rank[o];
        const TV* xo = xh + xoff[o] * R;
        for (int j = 0; j < ro; ++j) s += (TV)ld(Sb + (int64_t)j * r + a) * xo[(int64_t)j * R + cc];
      }
    }
    yh[(xoff[c] + a) * R + cc] = s;
  }
}

template <typename TM, typename TV>
__global__ void k_backward_down(const int* __restrict__ list, const int* __restrict__ parent,
                                const int64_t* __restrict__ eoff, const int64_t* __restrict__ xoff,
                                const int* __restrict__ rank, const TM* __restrict__ E,
                                TV* __restrict__ yh, int R) {
  const int c = list[blockIdx.x];
  const int r = rank[c], p = parent[c], rp = rank[p];
  const TM* Ec = E + eoff[c];
  const TV* yp = yh + xoff[p] * R;
  for (int idx = threadIdx.x; idx < r * R; idx += blockDim.x) {
    const int a = idx / R, cc = idx % R;
    TV s = yh[(xoff[c] + a) * R + cc];
    for (int b = 0; b < rp; ++b) s += (TV)ld(Ec + (int64_t)a * rp + b) * yp[(int64_t)b * R + cc];
    yh[(xoff[c] + a) * R + cc] = s;
  }
}

template <typename TM, typename TN, typename TV, bool TRANS>
__global__ void k_leaf_out(const int* __restrict__ leaves, const int* __restrict__ begin,
                           const int* __restrict__ end, const int64_t* __restrict__ voff,
                           const int64_t* __restrict__ xoff, const int* __restrict__ rank,
                           const TM* __restrict__ V, const TV* __restrict__ yh,
                           const int* __restrict__ nptr, const int* __restrict__ nblk,
                           const int* __restrict__ near_t, const int* __restrict__ near_s,
                           const int64_t* __restrict__ noff, const TN* __restrict__ N,
                           const TV* __restrict__ xp, const int* __restrict__ perm,
                           TV* __restrict__ y, int64_t ldy, int R) {
  const int c = leaves[blockIdx.x];
  const int r = rank[c], b = begin[c], nr = end[c] - b;
  const TM* Vc = V + voff[c];
  for (int idx = threadIdx.x; idx < nr * R; idx += blockDim.x) {
    const int i = idx / R, cc = idx % R;
    TV s = 0;
    for (int a = 0; a < r; ++a) s += (TV)ld(Vc + (int64_t)i * r + a) * yh[(xoff[c] + a) * R + cc];
    for (int e = nptr[c]; e < nptr[c + 1]; ++e) {
      const int blkid = nblk[e];
      const TN* Nb = N + noff[blkid];
      const int o = TRANS ? near_t[blkid] : near_s[blkid];
      const int bo = begin[o], no = end[o] - bo;
      if (!TRANS) {
        for (int j = 0; j < no; ++j) s += (TV)ld(Nb + (int64_t)i * no + j) * xp[(int64_t)(bo + j) * R + cc];
      } else {
        for (int j = 0; j < no; ++j) s += (TV)ld(Nb + (int64_t)j * nr + i) * xp[(int64_t)(bo + j) * R + cc];
      }
    }
    y[perm[b + i] + cc * ldy] = s;
  }
}

template <typename TM, typename TN, typename TV>
int run(const gca_h2* h, const TM* V, const TM* E, const TM* S, const TN* N, bool trans, int R,
        const TV* x, int64_t ldx, TV* y, int64_t ldy, cudaStream_t st) {
  const int n = h->n;
  GCA_TRY(h->w_xp.reserve(sizeof(TV) * (size_t)n * R));
  GCA_TRY(h->w_xh.reserve(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum, 1) * R));
  GCA_TRY(h->w_yh.reserve(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum, 1) * R));
  TV* xp = h->w_xp.as<TV>();
  TV* xh = h->w_xh.as<TV>();
  TV* yh = h->w_yh.as<TV>();
  const int T = 256;
  k_gather<TV><<<(unsigned)(((int64_t)n * R + T - 1) / T), T, 0, st>>>(n, R, h->d_perm.as<int>(), x,
                                                                     ldx, xp);
  const int nleaf = (int)h->leaves.size();
  const bool has_bases = h->rank_sum > 0;
  if (has_bases) {
    k_forward_leaf<TM, TV><<<nleaf, T, 0, st>>>(h->d_leaves.as<int>(), h->d_begin.as<int>(),
                                               h->d_end.as<int>(), h->d_voff.as<int64_t>(),
                                               h->d_xoff.as<int64_t>(), h->d_rank.as<int>(), V, xp,
                                               xh, R);
    for (int L = h->depth - 1; L >= 1; --L)
      if (h->n_up_level[L] > 0)
        k_forward_up<TM, TV><<<h->n_up_level[L], T, 0, st>>>(
            h->d_up_level[L].as<int>(), h->d_child0.as<int>(), h->d_child1.as<int>(),
            h->d_eoff.as<int64_t>(), h->d_xoff.as<int64_t>(), h->d_rank.as<int>(), E, xh, R);
    GCA_TRY_CUDA(cudaMemsetAsync(yh, 0, sizeof(TV) * (size_t)h->rank_sum * R, st));
    if (!trans && h->n_far_rows > 0)
      k_couple<TM, TV, false><<<h->n_far_rows, T, 0, st>>>(
          h->d_far_rows.as<int>(), h->d_far_row_ptr.as<int>(), h->d_far_row_blk.as<int>(),
          h->d_far_t.as<int>(), h->d_far_s.as<int>(), h->d_soff.as<int64_t>(), h->d_xoff.as<int64_t>(),
          h->d_rank.as<int>(), S, xh, yh, R);
    if (trans && h->n_far_cols > 0)
      k_couple<TM, TV, true><<<h->n_far_cols, T, 0, st>>>(
          h->d_far_cols.as<int>(), h->d_far_col_ptr.as<int>(), h->d_far_col_blk.as<int>(),
          h->d_far_t.as<int>(), h->d_far_s.as<int>(), h->d_soff.as<int64_t>(), h->d_xoff.as<int64_t>(),
          h->d_rank.as<int>(), S, xh, yh, R);
    for (int L = 2; L <= h->depth; ++L)
      if (h->n_down_level[L] > 0)
        k_backward_down<TM, TV><<<h->n_down_level[L], T, 0, st>>>(
            h->d_down_level[L].as<int>(), h->d_parent.as<int>(), h->d_eoff.as<int64_t>(),
            h->d_xoff.as<int64_t>(), h->d_rank.as<int>(), E, yh, R);
  }
  if (!trans)
    k_leaf_out<TM, TN, TV, false><<<nleaf, T, 0, st>>>(
        h->d_leaves.as<int>(), h->d_begin.as<int>(), h->d_end.as<int>(), h->d_voff.as<int64_t>(),
        h->d_xoff.as<int64_t>(), h->d_rank.as<int>(), V, yh, h->d_near_row_ptr.as<int>(),
        h->d_near_row_blk.as<int>(), h->d_near_t.as<int>(), h->d_near_s.as<int>(),
        h->d_noff.as<int64_t>(), N, xp, h->d_perm.as<int>(), y, ldy, R);
  else
    k_leaf_out<TM, TN, TV, true><<<nleaf, T, 0, st>>>(
        h->d_leaves.as<int>(), h->d_begin.as<int>(), h->d_end.as<int>(), h->d_voff.as<int64_t>(),
        h->d_xoff.as<int64_t>(), h->d_rank.as<int>(), V, yh, h->d_near_col_ptr.as<int>(),
        h->d_near_col_blk.as<int>(), h->d_near_t.as<int>(), h->d_near_s.as<int>(),
        h->d_noff.as<int64_t>(), N, xp, h->d_perm.as<int>(), y, ldy, R);
  GCA_TRY_CUDA(cudaGetLastError());
  return GCA_OK;
}

}  // namespace

// Index structures of the products (called at the end of gca_build).
int finish_plan(gca_h2* h, cudaStream_t st) {
  const int nc = h->nc;
  h->far_row = index_blocks(nc, h->far_t);
  h->far_col = index_blocks(nc, h->far_s);
  h->near_row = index_blocks(nc, h->near_t);
  h->near_col = index_blocks(nc, h->near_s);
  GCA_TRY(upload(h->d_far_row_ptr, h->far_row.ptr, st));
  GCA_TRY(upload(h->d_far_row_blk, h->far_row.blk, st));
  GCA_TRY(upload(h->d_far_col_ptr, h->far_col.ptr, st));
  GCA_TRY(upload(h->d_far_col_blk, h->far_col.blk, st));
  GCA_TRY(upload(h->d_near_row_ptr, h->near_row.ptr, st));
  GCA_TRY(upload(h->d_near_row_blk, h->near_row.blk, st));
  GCA_TRY(upload(h->d_near_col_ptr, h->near_col.ptr, st));
  GCA_TRY(upload(h->d_near_col_blk, h->near_col.blk, st));
  std::vector<int> rows, cols;
  for (int c = 0; c < nc; ++c) {
    if (h->far_row.ptr[c + 1] > h->far_row.ptr[c]) rows.push_back(c);
    if (h->far_col.ptr[c + 1] > h->far_col.ptr[c]) cols.push_back(c);
  }
  h->n_far_rows = (int)rows.size();
  h->n_far_cols = (int)cols.size();
  GCA_TRY(upload(h->d_far_rows, rows, st));
  GCA_TRY(upload(h->d_far_cols, cols, st));
  GCA_TRY(upload(h->d_leaves, h->leaves, st));
  GCA_TRY(upload(h->d_voff, h->voff, st));
  GCA_TRY(upload(h->d_eoff, h->eoff, st));
  GCA_TRY(upload(h->d_xoff, h->xoff, st));
  GCA_TRY(upload(h->d_parent, h->parent, st));
  GCA_TRY(upload(h->d_child0, h->child0, st));
  GCA_TRY(upload(h->d_child1, h->child1, st));
  h->d_up_level = std::vector<DevMem>(h->depth + 1);
  h->d_down_level = std::vector<DevMem>(h->depth + 1);
  h->n_up_level.assign(h->depth + 1, 0);
  h->n_down_level.assign(h->depth + 1, 0);
  for (int L = 1; L <= h->depth; ++L) {
    std::vector<int> up, down;
    for (int c : h->by_level[L]) {
      if (h->child0[c] >= 0) up.push_back(c);
      if (L >= 2) down.push_back(c);
    }
    h->n_up_level[L] = (int)up.size();
    h->n_down_level[L] = (int)down.size();
    GCA_TRY(upload(h->d_up_level[L], up, st));
    GCA_TRY(upload(h->d_down_level[L], down, st));
  }
  return GCA_OK;
}

int matvec(const gca_h2* h, gca_prec prec, bool trans, int32_t nrhs, const void* x, int64_t ldx,
           void* y, int64_t ldy, cudaStream_t st) {
  if (!h || !x || !y || nrhs < 1 || nrhs > 4096 || ldx < h->n || ldy < h->n) {
    set_error("h2_matvec: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  switch (prec) {
    case GCA_F64:
      return run<double, double, double>(h, h->V64.as<double>(), h->E64.as<double>(), h->S64.as<double>(),
                                         h->N64.as<double>(), trans, nrhs, (const double*)x, ldx,
                                         (double*)y, ldy, st);
    case GCA_F32:
      return run<float, float, float>(h, h->V32.as<float>(), h->E32.as<float>(), h->S32.as<float>(),
                                      h->N32.as<float>(), trans, nrhs, (const float*)x, ldx,
                                      (float*)y, ldy, st);
    case GCA_BF16:
      return run<__nv_bfloat16, float, float>(h, h->V16.as<__nv_bfloat16>(), h->E16.as<__nv_bfloat16>(),
                                              h->S16.as<__nv_bfloat16>(), h->N32.as<float>(), trans,
                                              nrhs, (const float*)x, ldx, (float*)y, ldy, st);
  }
  set_error("h2_matvec: unknown precision");
  return GCA_ERR_INVALID_ARG;
}

}  // namespace gca
