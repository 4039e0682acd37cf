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

struct gca_h2_batch;

namespace gca {

// Stored blocks in panel layout: leaf bases, transfers, couplings, near field,
// each also transposed; the column bases and transfers of an operator whose
// columns have bases of their own (the double layer).
enum PanelKind { kV = 0, kVt, kE, kEt, kS, kSt, kN, kNt, kW, kWt, kF, kFt, kPanelKinds };

// Last error text of the calling thread (returned by gca_last_error()).
void set_error(const std::string& msg);
std::string last_error();

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

// Test hooks (gca_test_hook, api.cu): settings that make failure paths
// reachable without a GPU fault.  `alloc_should_fail` counts device
// allocations and reports true for the one chosen by "fail_alloc".
struct TestHooks {
  long long wait_cycles;  // bound of every device-side wait of the products
  int stall_chain;        // product dependency waits need one more completion than any plan gives
  int device_skew;        // handles record (current device + skew) as their device
};
TestHooks test_hooks();
bool alloc_should_fail();
constexpr long long kDefaultWaitCycles = 1LL << 31;  // about a second at 2 GHz

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
    cudaError_t e = alloc_should_fail() ? cudaErrorMemoryAllocation : cudaMalloc(&p, nbytes);
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

// Finer phase names requested (gca_profile_enable(2)): the build splits its
// per-level phases by level and launch shape (profile.cu).
bool profile_detail();

// Event pair around a phase when profiling is enabled (profile.cu).
class PhaseScope {
 public:
  PhaseScope(const char* name, cudaStream_t s);
  PhaseScope(const std::string& name, cudaStream_t s) : PhaseScope(name.c_str(), s) {}
  ~PhaseScope();
  // kernel launches inside the phase (default 1)
  void launches(int k) { launches_ = k; }
  PhaseScope(const PhaseScope&) = delete;
  PhaseScope& operator=(const PhaseScope&) = delete;

 private:
  std::string name_;
  cudaStream_t s_;
  void* a_ = nullptr;
  void* b_ = nullptr;
  bool active_ = false;
  int launches_ = 1;
};

// Entry points of the translation units.
// op 0: the single-layer matrix G; op 1: the double-layer matrix K; op 2: the
// collocation matrix C of the single layer; op 3: G by single-level GCA; op 4:
// G by Green quadrature; op 5: G in the nodal (piecewise linear) basis;
// op 6: the nodal basis on curved triangles (midpoints: [nt][3][3])
int build(const gca_mesh* mesh, const gca_tree* tree, const gca_params* prm, cudaStream_t st,
          gca_h2** out, int op = 0, const double* midpoints = nullptr);
// gca_build_batch (build.cu): `count` single-layer meshes whose cross
// approximations share one launch per tree level
int build_group(int count, const gca_mesh* meshes, const gca_tree* trees, const gca_params* prm, cudaStream_t st,
                gca_h2** out);
// gca_support_union (build.cu)
int support_union(const gca_mesh* mesh, int nlists, const int32_t* list_ptr, const int32_t* lists,
                  int32_t* rows, int64_t cap, int32_t* counts, cudaStream_t st);
// Product plan (matvec.cu): plan_direction runs the host planning of one
// direction (it needs the ranks, block lists and panel offsets; the build
// calls it while its kernels run); finish_plan plans what is left and
// uploads the plan with the inverse permutation.
struct PlanJob;
struct PlanJobDelete {
  void operator()(PlanJob* j) const;
};
using PlanHandle = std::unique_ptr<PlanJob, PlanJobDelete>;
PlanHandle plan_new();
void plan_direction(const gca_h2* h, int dir, PlanJob* job);
int finish_plan(gca_h2* h, PlanJob* job, cudaStream_t st);
// Panel layout (build.cu): element offsets of every block, the device
// arrays, the number of panel jobs, then the panels themselves.
void layout_panels(gca_h2* h);
int alloc_panels(gca_h2* h);
int64_t panel_jobs(const gca_h2* h);
struct PanelJob;
int make_panels(gca_h2* h, DevMem& jobs_buf, std::vector<PanelJob>& host_jobs, cudaStream_t st);
int make_panels_sync(gca_h2* h, cudaStream_t st);
// gca_h2_export of panel kind q (kV, kE, kS, kN, kW, kF) from the float64
// panels into a host array of n doubles, in the export layout (build.cu)
int export_from_panels(const gca_h2* h, int q, double* host, int64_t n);
// gca_h2_import (import.cpp)
int import_h2(const gca_tree* tree, int32_t nt, int32_t nfar, int32_t nnear, const gca_host_dump* d,
              uint32_t flags, cudaStream_t st, gca_h2** out);
int product_status(const gca_h2* h, int* out);
// GCA_OK when `device` is the current device, else INVALID_ARG with a message
// naming both ordinals (the handle's memory would be another device's).
int check_device(int device, const char* what);
int prepare_batch(gca_h2_batch* b, cudaStream_t st);
int matvec_noalloc(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx, void* y,
                   int64_t ldy, cudaStream_t st);
int matvec_batch(const gca_h2_batch* b, gca_prec prec, bool trans, const int32_t* nrhs,
                 const void* const* x, const int64_t* ldx, void* const* y, const int64_t* ldy,
                 cudaStream_t st);
// autotuner of the products' tile width (matvec.cu)
int tune_batch(const gca_h2_batch* b, gca_prec prec, bool trans, const int32_t* nrhs, const void* const* x,
               const int64_t* ldx, void* const* y, const int64_t* ldy, cudaStream_t st, int* rc_out);
int tune_save(const char* path);
int tune_load(const char* path);
int tune_get(const char* device, gca_prec prec, bool trans, int32_t nrhs, int64_t rows, int* rc);
void tune_clear();
int matvec(const gca_h2* h, gca_prec prec, bool trans, int32_t nrhs, const void* x, int64_t ldx,
           void* y, int64_t ldy, cudaStream_t st);

// Device workspace of the products of a handle or a batch: the scratch
// vectors (zeroed per product) and, per precision and direction, the slot
// descriptors and merged claim orders together with the host bytes they were
// built from, so that repeated products in any order upload nothing.
struct DescCache {
  DevMem mem;
  std::vector<unsigned char> key;
};
struct ProductCache {
  DevMem ws;
  DescCache desc[6];  // (float64, float32, bfloat16) x (product, transposed product)
  // merged claim orders of a batch for one right-hand-side chunk per mesh,
  // per direction: chain claims, then free claims
  DevMem maps1[2];
  int64_t maps1_chain[2] = {0, 0};
  int64_t maps1_free[2] = {0, 0};
};

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

  // device: geometry and tree
  gca::DevMem d_vert, d_tri, d_perm, d_begin, d_end, d_rank;
  gca::DevMem d_iperm;  // inverse of perm: position in cluster order of each triangle
  // device: block lists (build kernels)
  gca::DevMem d_far_t, d_far_s, d_soff, d_near_t, d_near_s, d_noff;
  // device: coefficients, row-major float64 (as exported)
  gca::DevMem V64, E64, S64, N64;
  // device: coefficients in panel layout (panel.cuh) for the products, in
  // both orientations, three precisions (near field: float64 / float32)
  gca::DevMem P64[gca::kPanelKinds], P32[gca::kPanelKinds], P16[gca::kPanelKinds];
  std::vector<int64_t> panel_off[gca::kPanelKinds];  // per block, elements (all precisions)
  int64_t psize[gca::kPanelKinds] = {0};
  // persistent product, per direction: group records of up to 8 segment
  // descriptors each, the chain groups in claim order followed by the free
  // (near-field) groups, and the simulated start time of every chain group
  // (used to interleave the claim orders of the meshes of a batch)
  gca::DevMem d_segs[2];
  int64_t n_chain[2] = {0, 0};  // chain groups per direction
  int64_t n_free[2] = {0, 0};   // free groups per direction
  std::vector<float> chain_t[2];
  float makespan[2] = {0.f, 0.f};
  int max_leaf = 0;

  // device: product workspace (grown on demand): x-hat, y-hat, dependency
  // counters and the work-claim counter, zeroed by one memset per product
  mutable gca::ProductCache pc;
  mutable gca::DevMem d_status;  // sticky error bits of the products
  int max_rows = 0;              // largest block dimension (bounds the staged X)
  int device = -1;               // ordinal of the device that holds the handle's memory

  // The operator: 0 the single layer (one basis per cluster serves rows and
  // columns), 1 the double layer, 2 the collocated single layer.  For op 1 and
  // 2 the columns have bases W, transfers F and pivots tilde-sigma' of their
  // own (the double layer's; the Galerkin single layer's under the
  // collocation rows) and the couplings are r_tau x r'_sigma.  Ops 5 and 6
  // (the nodal basis on flat and on curved triangles) are one-sided like
  // op 0 with the vertices as indices.
  int op = 0;
  // Built symmetric operator (the single layer G in either basis, and its
  // single-level GCA): one basis per cluster and every block (tau, sigma)
  // has its mirror (sigma, tau).  The couplings of a mirrored pair are
  // evaluated once (S_{sigma tau} = S_{tau sigma}^T exactly), so the
  // transposed product runs the product's own plan and S panels; only the
  // near field, whose mirrored blocks are integrated separately (singular
  // rules are not symmetric in the two triangles), gets a second panel
  // array: at the offset of block b, N_{mirror(b)}^T, so that the plan's
  // near-field segments read the transposed entries.  No S^T panels and no
  // transposed plan are kept.  Imported handles keep both orientations.
  bool mirrored = false;
  std::vector<int> near_mirror;  // mirrored: index of each near block's mirror
  // the plan direction that serves a product of direction `dir`
  int served_dir(int dir) const { return mirrored ? 0 : dir; }
  std::vector<int> rank2;              // r'_sigma (op 1)
  std::vector<int64_t> xoff2;
  int64_t rank_sum2 = 0;
  int max_rank2 = 0;
  std::vector<int> piv2;
  std::vector<int64_t> poff2, voff2, eoff2;
  int64_t w_entries = 0, f_entries = 0;
  gca::DevMem W64, F64;                // row-major float64, as exported

  // the bases a product direction (0: G x, 1: G^T x) transforms its input
  // with and returns its output through
  // op 3: single-level GCA (a basis V_tau for every cluster of a block, on
  // all of its triangles, no transfers); op 4: Green quadrature (A_tau per
  // cluster, the factors B_{tau sigma}^* as the blocks' couplings)
  bool two_sided() const { return op == 1 || op == 2; }
  bool single_level() const { return op == 3 || op == 4; }
  bool in_cols(int dir) const { return two_sided() && dir == 0; }
  bool out_cols(int dir) const { return two_sided() && dir == 1; }
  const std::vector<int>& rank_in(int dir) const { return in_cols(dir) ? rank2 : rank; }
  const std::vector<int>& rank_out(int dir) const { return out_cols(dir) ? rank2 : rank; }
  const std::vector<int64_t>& xoff_in(int dir) const { return in_cols(dir) ? xoff2 : xoff; }
  const std::vector<int64_t>& xoff_out(int dir) const { return out_cols(dir) ? xoff2 : xoff; }
  int64_t rank_sum_in(int dir) const { return in_cols(dir) ? rank_sum2 : rank_sum; }
  int64_t rank_sum_out(int dir) const { return out_cols(dir) ? rank_sum2 : rank_sum; }
};

// A batch of handles applied in one persistent launch.
struct gca_h2_batch {
  std::vector<gca_h2*> h;          // owned
  mutable gca::ProductCache pc;    // shared product workspace
  mutable gca::DevMem d_status;
  int device = -1;                 // ordinal of the device that holds the batch
  ~gca_h2_batch() {
    for (auto* p : h) delete p;
  }
};
