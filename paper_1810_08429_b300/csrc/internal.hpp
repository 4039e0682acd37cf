// Internal definitions of the GCA-H^2 library: the handle, device buffers,
// status plumbing and constants shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "gca.h"

namespace gca {

// Last error text of the calling thread (returned by gca_last_error()).
void set_error(const std::string& msg);

#define GCA_TRY_CUDA(expr)                                                      \
  do {                                                                          \
    cudaError_t e__ = (expr);                                                   \
    if (e__ != cudaSuccess) {                                                   \
      ::gca::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));    \
      return e__ == cudaErrorMemoryAllocation ? GCA_ERR_OOM : GCA_ERR_CUDA;     \
    }                                                                           \
  } while (0)

#define GCA_TRY(expr)            \
  do {                           \
    int s__ = (expr);            \
    if (s__ != GCA_OK) return s__; \
  } while (0)

// Owning device allocation (cudaMalloc / cudaFree).
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  int alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error(std::string("cudaMalloc(") + std::to_string(nbytes) + "): " + cudaGetErrorString(e));
      return GCA_ERR_OOM;
    }
    bytes = nbytes;
    return GCA_OK;
  }
  // grow-only reallocation without preserving contents
  int reserve(size_t nbytes) {
    if (nbytes <= bytes && p) return GCA_OK;
    return alloc(nbytes);
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

template <typename T>
int upload(DevMem& m, const std::vector<T>& v, cudaStream_t s) {
  GCA_TRY(m.alloc(v.size() * sizeof(T)));
  if (!v.empty())
    GCA_TRY_CUDA(cudaMemcpyAsync(m.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return GCA_OK;
}

// Host-side tree helpers (tree.cpp)
int validate_mesh(const gca_mesh* mesh);
int validate_tree(const gca_mesh* mesh, const gca_tree* tree, int32_t max_leaf);
void box_diameters(const std::vector<double>& box, std::vector<double>& diam);
void block_tree(const std::vector<int>& child0, const std::vector<int>& child1,
                const std::vector<double>& box, const std::vector<double>& diam, double eta,
                std::vector<int>& far_t, std::vector<int>& far_s, std::vector<int>& near_t,
                std::vector<int>& near_s);

// Entry points of the translation units.
int build(const gca_mesh* mesh, const gca_tree* tree, const gca_params* prm, cudaStream_t st,
          gca_h2** out);
int finish_plan(gca_h2* h, cudaStream_t st);
int matvec(const gca_h2* h, gca_prec prec, bool trans, int32_t nrhs, const void* x, int64_t ldx,
           void* y, int64_t ldy, cudaStream_t st);

// Compressed sparse index of blocks by one of their two clusters.
struct BlockIndex {
  std::vector<int> ptr;   // [nclusters + 1]
  std::vector<int> blk;   // block ids
};
BlockIndex index_blocks(int nclusters, const std::vector<int>& key);

}  // namespace gca

// The handle.  Host copies of the tree and of every offset table, device
// copies of the mesh, tree and all stored coefficients.
struct gca_h2 {
  int n = 0, nv = 0, nc = 0, depth = 0, m = 0, k = 0;
  gca_params params{};
  double build_seconds = 0.0;

  // tree (host)
  std::vector<int> perm, begin, end, child0, child1, level, parent;
  std::vector<int> rank;               // r_tau, 0 for the root
  std::vector<int64_t> xoff;           // offset of x-hat_tau (prefix sum of rank)
  int64_t rank_sum = 0;
  int max_rank = 0;
  std::vector<int> piv;                // tilde-tau, triangle ids, cluster c at poff[c]
  std::vector<int64_t> poff;
  std::vector<int> leaves;             // leaf ids
  std::vector<std::vector<int>> by_level;  // clusters of each level

  // blocks (host): sorted by row cluster then column cluster
  std::vector<int> far_t, far_s, near_t, near_s;
  std::vector<int64_t> soff, noff;     // coefficient offsets per block
  std::vector<int64_t> voff;           // per cluster (leaves), -1 otherwise
  std::vector<int64_t> eoff;           // per cluster with a non-root parent, -1 otherwise
  int64_t v_entries = 0, e_entries = 0, s_entries = 0, n_entries = 0;
  int64_t n_singular[4] = {0, 0, 0, 0};
  gca::BlockIndex far_row, far_col, near_row, near_col;

  // device: geometry and tree
  gca::DevMem d_vert, d_tri, d_perm, d_begin, d_end, d_rank, d_xoff;
  // device: coefficients, three precisions
  gca::DevMem V64, E64, S64, N64, V32, E32, S32, N32, V16, E16, S16;
  // device: product plans
  gca::DevMem d_leaves, d_voff, d_eoff, d_parent, d_child0, d_child1;
  gca::DevMem d_far_t, d_far_s, d_soff, d_near_t, d_near_s, d_noff;
  gca::DevMem d_far_row_ptr, d_far_row_blk, d_far_col_ptr, d_far_col_blk;
  gca::DevMem d_near_row_ptr, d_near_row_blk, d_near_col_ptr, d_near_col_blk;
  std::vector<gca::DevMem*> level_lists_owner;
  std::vector<gca::DevMem> d_up_level;    // per level: non-leaf clusters (forward/up)
  std::vector<int> n_up_level;
  std::vector<gca::DevMem> d_down_level;  // per level: clusters whose parent is at this level - 1
  std::vector<int> n_down_level;
  gca::DevMem d_far_rows;                 // clusters with >= 1 far block as row
  gca::DevMem d_far_cols;                 // clusters with >= 1 far block as column
  int n_far_rows = 0, n_far_cols = 0;
  int max_leaf = 0;

  // device: product work buffers (grown on demand)
  mutable gca::DevMem w_xp, w_xh, w_yh;
};
