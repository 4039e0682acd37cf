// gca_h2_import: a handle from a host copy of an H^2 representation (Sect. 4)
// computed elsewhere, in the layout gca_h2_export writes.  The products then
// run on it exactly as on a handle from gca_build; the construction is not
// involved, which isolates the products in parity runs.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "internal.hpp"

namespace gca {

namespace {

int bad(const std::string& msg) {
  set_error("gca_h2_import: " + msg);
  return GCA_ERR_INVALID_ARG;
}

bool finite_all(const double* p, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

int import_h2(const gca_tree* tree, int32_t nt, int32_t nfar, int32_t nnear, const gca_host_dump* d,
              uint32_t flags, cudaStream_t st, gca_h2** out) {
  const auto t0 = std::chrono::steady_clock::now();
  if (nt < 1 || nfar < 0 || nnear < 0 || !d || !d->rank || !d->V || !d->E || (nfar > 0 && (!d->far || !d->S)) ||
      (nnear > 0 && (!d->near || !d->N)))
    return bad("null pointer or negative size");
  if ((flags & ~(uint32_t)(GCA_DROP_F64 | GCA_DROP_F32 | GCA_DROP_BF16 | GCA_DROP_EXPORT)) != 0)
    return bad("unknown flags");
  const gca_mesh shape{0, nt, nullptr, nullptr};
  GCA_TRY(validate_tree(&shape, tree, GCA_MAX_LEAF));
  auto h = std::make_unique<gca_h2>();
  h->params = gca_params{};
  h->params.flags = flags;
  h->n = nt;
  h->nc = tree->nclusters;
  const int nc = h->nc;
  h->perm.assign(tree->perm, tree->perm + nt);
  h->begin.assign(tree->begin, tree->begin + nc);
  h->end.assign(tree->end, tree->end + nc);
  h->child0.assign(tree->child0, tree->child0 + nc);
  h->child1.assign(tree->child1, tree->child1 + nc);
  h->level.assign(tree->level, tree->level + nc);
  h->parent.assign(nc, -1);
  for (int c = 0; c < nc; ++c)
    if (h->child0[c] >= 0) h->parent[h->child0[c]] = h->parent[h->child1[c]] = c;
  h->depth = *std::max_element(h->level.begin(), h->level.end());
  h->by_level.assign(h->depth + 1, {});
  for (int c = 0; c < nc; ++c) {
    h->by_level[h->level[c]].push_back(c);
    if (h->child0[c] < 0) {
      h->leaves.push_back(c);
      h->max_leaf = std::max(h->max_leaf, h->end[c] - h->begin[c]);
    }
  }
  // ranks: the root has no basis; a leaf basis has at most |tau-hat| columns,
  // a parent's at most the sum of its children's ranks (its rows, Sect. 4)
  h->rank.assign(d->rank, d->rank + nc);
  if (h->rank[0] != 0) return bad("the root must have rank 0");
  for (int c = 1; c < nc; ++c) {
    const int r = h->rank[c];
    const int cap = h->child0[c] < 0 ? h->end[c] - h->begin[c] : h->rank[h->child0[c]] + h->rank[h->child1[c]];
    if (r < 0 || r > cap || r > 0xffff) return bad("rank of cluster " + std::to_string(c) + " out of range");
  }
  h->xoff.assign(nc + 1, 0);
  for (int c = 0; c < nc; ++c) h->xoff[c + 1] = h->xoff[c] + h->rank[c];
  h->rank_sum = h->xoff[nc];
  h->max_rank = *std::max_element(h->rank.begin(), h->rank.end());
  h->poff.assign(nc, -1);
  h->piv.assign(std::max<int64_t>(h->rank_sum, 1), 0);
  if (h->rank_sum > 0 && !d->pivots) return bad("pivots are NULL");
  for (int c = 0; c < nc; ++c) {
    h->poff[c] = h->xoff[c];
    for (int t = 0; t < h->rank[c]; ++t) {
      const int p = d->pivots[h->xoff[c] + t];
      if (p < 0 || p >= nt) return bad("pivot out of range");
      h->piv[h->xoff[c] + t] = p;
    }
  }
  // block lists
  h->far_t.resize(nfar);
  h->far_s.resize(nfar);
  for (int b = 0; b < nfar; ++b) {
    const int t = d->far[2 * b], s = d->far[2 * b + 1];
    if (t < 1 || t >= nc || s < 1 || s >= nc) return bad("coupling block " + std::to_string(b) + " names a bad cluster");
    h->far_t[b] = t;
    h->far_s[b] = s;
  }
  h->near_t.resize(nnear);
  h->near_s.resize(nnear);
  for (int b = 0; b < nnear; ++b) {
    const int t = d->near[2 * b], s = d->near[2 * b + 1];
    if (t < 0 || t >= nc || s < 0 || s >= nc || h->child0[t] >= 0 || h->child0[s] >= 0)
      return bad("near-field block " + std::to_string(b) + " is not a pair of leaves");
    h->near_t[b] = t;
    h->near_s[b] = s;
  }
  // coefficient offsets, in the order of gca_host_dump
  h->voff.assign(nc, -1);
  h->eoff.assign(nc, -1);
  for (int c = 1; c < nc; ++c)
    if (h->child0[c] < 0) {
      h->voff[c] = h->v_entries;
      h->v_entries += (int64_t)(h->end[c] - h->begin[c]) * h->rank[c];
    }
  for (int c = 1; c < nc; ++c)
    if (h->parent[c] > 0) {
      h->eoff[c] = h->e_entries;
      h->e_entries += (int64_t)h->rank[c] * h->rank[h->parent[c]];
    }
  h->soff.assign(nfar + 1, 0);
  for (int b = 0; b < nfar; ++b)
    h->soff[b + 1] = h->soff[b] + (int64_t)h->rank[h->far_t[b]] * h->rank[h->far_s[b]];
  h->s_entries = h->soff[nfar];
  h->noff.assign(nnear + 1, 0);
  for (int b = 0; b < nnear; ++b) {
    const int t = h->near_t[b], s = h->near_s[b];
    h->noff[b + 1] = h->noff[b] + (int64_t)(h->end[t] - h->begin[t]) * (h->end[s] - h->begin[s]);
  }
  h->n_entries = h->noff[nnear];
  if (!finite_all(d->V, h->v_entries) || !finite_all(d->E, h->e_entries) ||
      (nfar > 0 && !finite_all(d->S, h->s_entries)) || (nnear > 0 && !finite_all(d->N, h->n_entries))) {
    set_error("gca_h2_import: non-finite coefficient");
    return GCA_ERR_NUMERIC;
  }
  // device copies: the tree, the row-major coefficients, the panels and the plan
  GCA_TRY_CUDA(cudaGetDevice(&h->device));
  h->device += test_hooks().device_skew;
  GCA_TRY(upload(h->d_perm, h->perm, st));
  GCA_TRY(upload(h->d_begin, h->begin, st));
  GCA_TRY(upload(h->d_end, h->end, st));
  GCA_TRY(upload(h->d_rank, h->rank, st));
  struct Item {
    DevMem* dst;
    const double* src;
    int64_t n;
  };
  const Item items[4] = {{&h->V64, d->V, h->v_entries}, {&h->E64, d->E, h->e_entries},
                         {&h->S64, d->S, h->s_entries}, {&h->N64, d->N, h->n_entries}};
  for (const Item& it : items) {
    GCA_TRY(it.dst->alloc(sizeof(double) * (size_t)std::max<int64_t>(it.n, 1)));
    if (it.n > 0)
      GCA_TRY_CUDA(cudaMemcpyAsync(it.dst->p, it.src, sizeof(double) * it.n, cudaMemcpyHostToDevice, st));
  }
  layout_panels(h.get());
  GCA_TRY(alloc_panels(h.get()));
  GCA_TRY(make_panels_sync(h.get(), st));
  PlanHandle plan = plan_new();
  GCA_TRY(finish_plan(h.get(), plan.get(), st));
  GCA_TRY_CUDA(cudaStreamSynchronize(st));
  // as gca_build: the float64 panels serve gca_h2_export when they exist
  if ((flags & GCA_DROP_EXPORT) || !(flags & GCA_DROP_F64)) {
    h->V64.release();
    h->E64.release();
    h->S64.release();
    h->N64.release();
  }
  h->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = h.release();
  return GCA_OK;
}

}  // namespace gca
