// Host side of the library: mesh and tree validation, the cluster-tree
// helper gca_tree_build, admissibility and the block tree (Sect. 2).
//
// Floating-point decisions (which side of the midpoint a centroid falls on,
// whether a block is admissible) are taken with plain IEEE operations in a
// fixed order and without contraction into fused multiply-adds, so that the
// same mesh always yields the same tree and block structure.

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "internal.hpp"

namespace gca {

int validate_mesh(const gca_mesh* mesh) {
  if (!mesh || mesh->nt <= 0 || mesh->nv < 3 || !mesh->vertices || !mesh->triangles) {
    set_error("mesh: null pointer or empty");
    return GCA_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < 3LL * mesh->nv; ++i)
    if (!std::isfinite(mesh->vertices[i])) {
      set_error("mesh: non-finite vertex coordinate");
      return GCA_ERR_NUMERIC;
    }
  for (int32_t t = 0; t < mesh->nt; ++t) {
    const int32_t* tri = mesh->triangles + 3LL * t;
    for (int a = 0; a < 3; ++a)
      if (tri[a] < 0 || tri[a] >= mesh->nv) {
        set_error("mesh: vertex id out of range in triangle " + std::to_string(t));
        return GCA_ERR_INVALID_ARG;
      }
    if (tri[0] == tri[1] || tri[1] == tri[2] || tri[0] == tri[2]) {
      set_error("mesh: repeated vertex id in triangle " + std::to_string(t));
      return GCA_ERR_INVALID_ARG;
    }
    const double* a = mesh->vertices + 3LL * tri[0];
    const double* b = mesh->vertices + 3LL * tri[1];
    const double* c = mesh->vertices + 3LL * tri[2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    if (!(cx * cx + cy * cy + cz * cz > 0.0)) {
      set_error("mesh: degenerate triangle " + std::to_string(t));
      return GCA_ERR_INVALID_ARG;
    }
  }
  return GCA_OK;
}

int validate_tree(const gca_mesh* mesh, const gca_tree* tr, int32_t max_leaf) {
  if (!tr || tr->nclusters < 1 || !tr->perm || !tr->begin || !tr->end || !tr->child0 ||
      !tr->child1 || !tr->level) {
    set_error("tree: null pointer or empty");
    return GCA_ERR_INVALID_ARG;
  }
  const int n = mesh->nt, nc = tr->nclusters;
  if (nc > 2 * n - 1) {
    set_error("tree: more clusters than a binary tree over n triangles can have");
    return GCA_ERR_INVALID_ARG;
  }
  std::vector<char> seen(n, 0);
  for (int i = 0; i < n; ++i) {
    int p = tr->perm[i];
    if (p < 0 || p >= n || seen[p]) {
      set_error("tree: perm is not a permutation");
      return GCA_ERR_INVALID_ARG;
    }
    seen[p] = 1;
  }
  if (tr->begin[0] != 0 || tr->end[0] != n || tr->level[0] != 0) {
    set_error("tree: cluster 0 must be the root [0, n) at level 0");
    return GCA_ERR_INVALID_ARG;
  }
  std::vector<int> parent(nc, -1);
  for (int c = 0; c < nc; ++c) {
    int b = tr->begin[c], e = tr->end[c], c0 = tr->child0[c], c1 = tr->child1[c];
    if (b < 0 || e > n || b >= e) {
      set_error("tree: bad range of cluster " + std::to_string(c));
      return GCA_ERR_INVALID_ARG;
    }
    if ((c0 < 0) != (c1 < 0)) {
      set_error("tree: cluster " + std::to_string(c) + " has exactly one child");
      return GCA_ERR_INVALID_ARG;
    }
    if (c0 < 0) {
      if (e - b > max_leaf) {
        set_error("tree: leaf " + std::to_string(c) + " larger than GCA_MAX_LEAF");
        return GCA_ERR_UNSUPPORTED;
      }
      continue;
    }
    if (c0 >= nc || c1 >= nc || c0 == 0 || c1 == 0 || c0 == c1) {
      set_error("tree: bad child ids of cluster " + std::to_string(c));
      return GCA_ERR_INVALID_ARG;
    }
    if (parent[c0] >= 0 || parent[c1] >= 0) {
      set_error("tree: a cluster has two parents");
      return GCA_ERR_INVALID_ARG;
    }
    parent[c0] = c;
    parent[c1] = c;
    if (tr->begin[c0] != b || tr->end[c1] != e || tr->end[c0] != tr->begin[c1]) {
      set_error("tree: children of cluster " + std::to_string(c) + " do not split its range");
      return GCA_ERR_INVALID_ARG;
    }
    if (tr->level[c0] != tr->level[c] + 1 || tr->level[c1] != tr->level[c] + 1) {
      set_error("tree: level of a child is not its parent's plus one");
      return GCA_ERR_INVALID_ARG;
    }
  }
  for (int c = 1; c < nc; ++c)
    if (parent[c] < 0) {
      set_error("tree: cluster " + std::to_string(c) + " is not reachable from the root");
      return GCA_ERR_INVALID_ARG;
    }
  return GCA_OK;
}

void box_diameters(const std::vector<double>& box, std::vector<double>& diam) {
  const size_t nc = box.size() / 6;
  diam.resize(nc);
  for (size_t c = 0; c < nc; ++c) {
    double dx = box[6 * c + 3] - box[6 * c + 0];
    double dy = box[6 * c + 4] - box[6 * c + 1];
    double dz = box[6 * c + 5] - box[6 * c + 2];
    double s = dx * dx;
    s = s + dy * dy;
    s = s + dz * dz;
    diam[c] = std::sqrt(s);
  }
}

static double box_distance(const double* a, const double* b) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    double g1 = b[d] - a[3 + d];  // lo_sigma - hi_tau
    double g2 = a[d] - b[3 + d];  // lo_tau - hi_sigma
    double g = std::max(0.0, std::max(g1, g2));
    double t = g * g;
    s = (d == 0) ? t : s + t;
  }
  return std::sqrt(s);
}

void block_tree(const std::vector<int>& child0, const std::vector<int>& child1,
                const std::vector<double>& box, const std::vector<double>& diam, double eta,
                std::vector<int>& far_t, std::vector<int>& far_s, std::vector<int>& near_t,
                std::vector<int>& near_s) {
  std::vector<std::pair<int, int>> far, near, stack{{0, 0}};
  const double two_eta = 2.0 * eta;
  while (!stack.empty()) {
    auto [t, s] = stack.back();
    stack.pop_back();
    double dist = box_distance(&box[6 * t], &box[6 * s]);
    if (std::max(diam[t], diam[s]) <= two_eta * dist) {
      far.emplace_back(t, s);
      continue;
    }
    bool lt = child0[t] < 0, ls = child0[s] < 0;
    if (lt && ls) {
      near.emplace_back(t, s);
    } else if (lt) {
      stack.emplace_back(t, child1[s]);
      stack.emplace_back(t, child0[s]);
    } else if (ls) {
      stack.emplace_back(child1[t], s);
      stack.emplace_back(child0[t], s);
    } else {
      for (int ct : {child1[t], child0[t]})
        for (int cs : {child1[s], child0[s]}) stack.emplace_back(ct, cs);
    }
  }
  std::sort(far.begin(), far.end());
  std::sort(near.begin(), near.end());
  far_t.clear(); far_s.clear(); near_t.clear(); near_s.clear();
  for (auto& p : far) { far_t.push_back(p.first); far_s.push_back(p.second); }
  for (auto& p : near) { near_t.push_back(p.first); near_s.push_back(p.second); }
}

BlockIndex index_blocks(int nclusters, const std::vector<int>& key) {
  BlockIndex ix;
  ix.ptr.assign(nclusters + 1, 0);
  for (int c : key) ix.ptr[c + 1]++;
  for (int c = 0; c < nclusters; ++c) ix.ptr[c + 1] += ix.ptr[c];
  ix.blk.resize(key.size());
  std::vector<int> fill(ix.ptr.begin(), ix.ptr.end() - 1);
  for (size_t b = 0; b < key.size(); ++b) ix.blk[fill[key[b]]++] = static_cast<int>(b);
  return ix;
}

}  // namespace gca

namespace {

// The bisection of gca_tree_build on n points (x, y, z per index).
int bisect(int n, const std::vector<double>& cent, int32_t leaf_size, int32_t max_clusters,
           int32_t* perm, int32_t* begin, int32_t* end, int32_t* child0, int32_t* child1,
           int32_t* level, int32_t* nclusters, const char* who) {
  using namespace gca;
  std::vector<int> p(n);
  std::iota(p.begin(), p.end(), 0);
  std::vector<int> B{0}, E{n}, C0{-1}, C1{-1}, L{0};
  std::vector<int> tmp;
  for (size_t head = 0; head < B.size(); ++head) {
    const int c = static_cast<int>(head);
    const int b = B[c], e = E[c];
    if (e - b <= leaf_size) continue;
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) lo[d] = hi[d] = cent[3 * (size_t)p[b] + d];
    for (int i = b + 1; i < e; ++i)
      for (int d = 0; d < 3; ++d) {
        double x = cent[3 * (size_t)p[i] + d];
        lo[d] = std::min(lo[d], x);
        hi[d] = std::max(hi[d], x);
      }
    int axis = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
    const double mid = 0.5 * (lo[axis] + hi[axis]);
    tmp.clear();
    int nlow = 0;
    for (int i = b; i < e; ++i)
      if (cent[3 * (size_t)p[i] + axis] < mid) { tmp.push_back(p[i]); ++nlow; }
    if (nlow == 0 || nlow == e - b) {
      tmp.assign(p.begin() + b, p.begin() + e);
      std::stable_sort(tmp.begin(), tmp.end(), [&](int u, int v) {
        return cent[3 * (size_t)u + axis] < cent[3 * (size_t)v + axis];
      });
      nlow = (e - b) / 2;
    } else {
      for (int i = b; i < e; ++i)
        if (!(cent[3 * (size_t)p[i] + axis] < mid)) tmp.push_back(p[i]);
    }
    std::copy(tmp.begin(), tmp.end(), p.begin() + b);
    if ((int)B.size() + 2 > max_clusters) {
      set_error(std::string(who) + ": max_clusters too small");
      return GCA_ERR_INVALID_ARG;
    }
    for (auto [cb, ce] : {std::pair<int, int>{b, b + nlow}, std::pair<int, int>{b + nlow, e}}) {
      B.push_back(cb); E.push_back(ce); C0.push_back(-1); C1.push_back(-1); L.push_back(L[c] + 1);
    }
    C0[c] = (int)B.size() - 2;
    C1[c] = (int)B.size() - 1;
  }
  std::copy(p.begin(), p.end(), perm);
  std::copy(B.begin(), B.end(), begin);
  std::copy(E.begin(), E.end(), end);
  std::copy(C0.begin(), C0.end(), child0);
  std::copy(C1.begin(), C1.end(), child1);
  std::copy(L.begin(), L.end(), level);
  *nclusters = (int32_t)B.size();
  return GCA_OK;
}

}  // namespace

extern "C" int gca_tree_build(const gca_mesh* mesh, int32_t leaf_size, int32_t max_clusters,
                              int32_t* perm, int32_t* begin, int32_t* end, int32_t* child0,
                              int32_t* child1, int32_t* level, int32_t* nclusters) {
  using namespace gca;
  int st = validate_mesh(mesh);
  if (st != GCA_OK) return st;
  if (leaf_size < 1 || !perm || !begin || !end || !child0 || !child1 || !level || !nclusters) {
    set_error("gca_tree_build: bad arguments");
    return GCA_ERR_INVALID_ARG;
  }
  const int n = mesh->nt;
  std::vector<double> cent(3 * (size_t)n);
  for (int t = 0; t < n; ++t) {
    const int32_t* tri = mesh->triangles + 3LL * t;
    for (int d = 0; d < 3; ++d) {
      double s = mesh->vertices[3LL * tri[0] + d] + mesh->vertices[3LL * tri[1] + d];
      s = s + mesh->vertices[3LL * tri[2] + d];
      cent[3 * (size_t)t + d] = s / 3.0;
    }
  }
  return bisect(n, cent, leaf_size, max_clusters, perm, begin, end, child0, child1, level, nclusters,
                "gca_tree_build");
}

extern "C" int gca_tree_build_points(int32_t n, const double* points, int32_t leaf_size, int32_t max_clusters,
                                     int32_t* perm, int32_t* begin, int32_t* end, int32_t* child0,
                                     int32_t* child1, int32_t* level, int32_t* nclusters) {
  using namespace gca;
  if (n < 1 || !points || leaf_size < 1 || !perm || !begin || !end || !child0 || !child1 || !level ||
      !nclusters) {
    set_error("gca_tree_build_points: bad arguments");
    return GCA_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < 3LL * n; ++i)
    if (!std::isfinite(points[i])) {
      set_error("gca_tree_build_points: non-finite coordinate");
      return GCA_ERR_NUMERIC;
    }
  std::vector<double> cent(points, points + 3LL * n);
  return bisect(n, cent, leaf_size, max_clusters, perm, begin, end, child0, child1, level, nclusters,
                "gca_tree_build_points");
}
