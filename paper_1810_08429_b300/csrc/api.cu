// Extern "C" entry points declared in gca.h: argument checks and dispatch
// to the build / product translation units, statistics, export and error
// text.

#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>
#include <memory>
#include <algorithm>
#include <vector>

#include "internal.hpp"

namespace gca {
namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_wait_cycles{kDefaultWaitCycles};
std::atomic<int> g_stall_chain{0};
std::atomic<int> g_device_skew{0};
std::atomic<long long> g_fail_alloc{0};  // allocations left before the injected failure (0: off)
}  // namespace
void set_error(const std::string& msg) { g_last_error = msg; }
std::string last_error() { return g_last_error; }

TestHooks test_hooks() {
  return TestHooks{g_wait_cycles.load(), g_stall_chain.load(), g_device_skew.load()};
}

bool alloc_should_fail() {
  long long left = g_fail_alloc.load();
  while (left > 0) {
    if (g_fail_alloc.compare_exchange_weak(left, left - 1)) return left == 1;
  }
  return false;
}

int check_device(int device, const char* what) {
  int cur = -1;
  GCA_TRY_CUDA(cudaGetDevice(&cur));
  if (cur != device) {
    set_error(std::string(what) + ": built on device " + std::to_string(device) + ", but device " +
              std::to_string(cur) + " is current (make the handle's device current first)");
    return GCA_ERR_INVALID_ARG;
  }
  return GCA_OK;
}
}  // namespace gca

extern "C" {

const char* gca_last_error(void) { return gca::g_last_error.c_str(); }

int gca_build(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params, void* stream,
              gca_h2** out) {
  if (!out) {
    gca::set_error("gca_build: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::build(mesh, tree, params, static_cast<cudaStream_t>(stream), out);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_build_double_layer(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params, void* stream,
                           gca_h2** out) {
  if (!out) {
    gca::set_error("gca_build_double_layer: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::build(mesh, tree, params, static_cast<cudaStream_t>(stream), out, 1);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build_double_layer: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_build_p1(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params, void* stream,
                 gca_h2** out) {
  if (!out) {
    gca::set_error("gca_build_p1: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::build(mesh, tree, params, static_cast<cudaStream_t>(stream), out, 5);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build_p1: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_build_p1_curved(const gca_mesh* mesh, const double* midpoints, const gca_tree* tree,
                        const gca_params* params, void* stream, gca_h2** out) {
  if (!out) {
    gca::set_error("gca_build_p1_curved: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::build(mesh, tree, params, static_cast<cudaStream_t>(stream), out, 6, midpoints);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build_p1_curved: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_support_union(const gca_mesh* mesh, int32_t nlists, const int32_t* list_ptr, const int32_t* lists,
                      int32_t* rows, int64_t cap, int32_t* counts, void* stream) {
  try {
    return gca::support_union(mesh, nlists, list_ptr, lists, rows, cap, counts, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_support_union: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_build_collocation(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params, void* stream,
                          gca_h2** out) {
  if (!out) {
    gca::set_error("gca_build_collocation: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::build(mesh, tree, params, static_cast<cudaStream_t>(stream), out, 2);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build_collocation: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_build_single_level(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params, void* stream,
                           gca_h2** out) {
  if (!out) {
    gca::set_error("gca_build_single_level: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::build(mesh, tree, params, static_cast<cudaStream_t>(stream), out, 3);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build_single_level: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_build_green_quadrature(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params, void* stream,
                               gca_h2** out) {
  if (!out) {
    gca::set_error("gca_build_green_quadrature: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::build(mesh, tree, params, static_cast<cudaStream_t>(stream), out, 4);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build_green_quadrature: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_h2_column_stats(const gca_h2* h, gca_column_stats* o) {
  if (!h || !o) {
    gca::set_error("gca_h2_column_stats: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  std::memset(o, 0, sizeof(*o));
  o->op = h->op;
  if (h->two_sided()) {
    o->max_rank = h->max_rank2;
    o->rank_sum = h->rank_sum2;
    o->w_entries = h->w_entries;
    o->f_entries = h->f_entries;
  } else {
    o->max_rank = h->max_rank;
    o->rank_sum = h->rank_sum;
    o->w_entries = h->v_entries;
    o->f_entries = h->e_entries;
  }
  return GCA_OK;
}

int gca_h2_export_columns(const gca_h2* h, gca_host_dump* o) {
  if (!h || !o) {
    gca::set_error("gca_h2_export_columns: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  if (!h->two_sided()) {
    // one basis serves rows and columns
    gca_host_dump d{o->rank, o->pivots, nullptr, nullptr, o->V, o->E, nullptr, nullptr};
    return gca_h2_export(h, &d);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    gca::set_error("gca_h2_export_columns: device error before export");
    return GCA_ERR_CUDA;
  }
  if (o->far || o->near || o->S || o->N) {
    gca::set_error("gca_h2_export_columns: far, near, S and N belong to gca_h2_export");
    return GCA_ERR_INVALID_ARG;
  }
  if (o->rank) std::memcpy(o->rank, h->rank2.data(), sizeof(int) * h->nc);
  if (o->pivots) {
    int64_t at = 0;
    for (int c = 0; c < h->nc; ++c)
      for (int t = 0; t < h->rank2[c]; ++t) o->pivots[at++] = h->piv2[h->poff2[c] + t];
  }
  if ((h->params.flags & GCA_DROP_EXPORT) && (o->V || o->E)) {
    gca::set_error("gca_h2_export_columns: the handle was built with GCA_DROP_EXPORT");
    return GCA_ERR_UNSUPPORTED;
  }
  struct Item { double* dst; const gca::DevMem* src; int64_t n; int kind; };
  const Item items[2] = {{o->V, &h->W64, h->w_entries, gca::kW}, {o->E, &h->F64, h->f_entries, gca::kF}};
  for (const auto& it : items)
    if (it.dst && it.n > 0) {
      if (!it.src->p) {
        const int st = gca::export_from_panels(h, it.kind, it.dst, it.n);
        if (st != GCA_OK) return st;
        continue;
      }
      cudaError_t e = cudaMemcpy(it.dst, it.src->p, sizeof(double) * it.n, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        gca::set_error(std::string("gca_h2_export_columns: ") + cudaGetErrorString(e));
        return GCA_ERR_CUDA;
      }
    }
  return GCA_OK;
}

int h2_matvec(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx, void* y,
              int64_t ldy, void* stream) {
  return gca::matvec(h, prec, false, nrhs, x, ldx, y, ldy, static_cast<cudaStream_t>(stream));
}

int h2_matvec_transpose(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx,
                        void* y, int64_t ldy, void* stream) {
  return gca::matvec(h, prec, true, nrhs, x, ldx, y, ldy, static_cast<cudaStream_t>(stream));
}

int h2_matvec_noalloc(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx,
                      void* y, int64_t ldy, void* stream) {
  return gca::matvec_noalloc(h, prec, nrhs, x, ldx, y, ldy, static_cast<cudaStream_t>(stream));
}

int gca_h2_import(const gca_tree* tree, int32_t nt, int32_t nfar, int32_t nnear, const gca_host_dump* dump,
                  uint32_t flags, void* stream, gca_h2** out) {
  if (!out) {
    gca::set_error("gca_h2_import: out is NULL");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    return gca::import_h2(tree, nt, nfar, nnear, dump, flags, static_cast<cudaStream_t>(stream), out);
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_h2_import: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_h2_stats(const gca_h2* h, gca_stats* o) {
  if (!h || !o) {
    gca::set_error("gca_h2_stats: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  std::memset(o, 0, sizeof(*o));
  o->n = h->n;
  o->nclusters = h->nc;
  o->depth = h->depth;
  o->k = h->k;
  o->nfar = (int32_t)h->far_t.size();
  o->nnear = (int32_t)h->near_t.size();
  o->max_rank = h->max_rank;
  o->rank_sum = h->rank_sum;
  o->v_entries = h->v_entries;
  o->e_entries = h->e_entries;
  o->s_entries = h->s_entries;
  o->n_entries = h->n_entries;
  for (int c = 0; c < 4; ++c) o->n_singular[c] = h->n_singular[c];
  o->build_seconds = h->build_seconds;
  return GCA_OK;
}

int gca_h2_export(const gca_h2* h, gca_host_dump* o) {
  if (!h || !o) {
    gca::set_error("gca_h2_export: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    gca::set_error("gca_h2_export: device error before export");
    return GCA_ERR_CUDA;
  }
  if (o->rank) std::memcpy(o->rank, h->rank.data(), sizeof(int) * h->nc);
  if (o->pivots) {
    int64_t at = 0;
    for (int c = 0; c < h->nc; ++c)
      for (int t = 0; t < h->rank[c]; ++t)
        o->pivots[at++] = h->op == 4 ? -1 : h->piv[h->poff[c] + t];  // Green quadrature: no pivots
  }
  if (o->far)
    for (size_t b = 0; b < h->far_t.size(); ++b) {
      o->far[2 * b] = h->far_t[b];
      o->far[2 * b + 1] = h->far_s[b];
    }
  if (o->near)
    for (size_t b = 0; b < h->near_t.size(); ++b) {
      o->near[2 * b] = h->near_t[b];
      o->near[2 * b + 1] = h->near_s[b];
    }
  if ((h->params.flags & GCA_DROP_EXPORT) && (o->V || o->E || o->S || o->N)) {
    gca::set_error("gca_h2_export: the handle was built with GCA_DROP_EXPORT");
    return GCA_ERR_UNSUPPORTED;
  }
  // the row-major copy where the handle keeps one, else the float64 panels
  struct Item { double* dst; const gca::DevMem* src; int64_t n; int kind; };
  const Item items[4] = {{o->V, &h->V64, h->v_entries, gca::kV}, {o->E, &h->E64, h->e_entries, gca::kE},
                         {o->S, &h->S64, h->s_entries, gca::kS}, {o->N, &h->N64, h->n_entries, gca::kN}};
  for (const auto& it : items)
    if (it.dst && it.n > 0) {
      if (!it.src->p) {
        const int st = gca::export_from_panels(h, it.kind, it.dst, it.n);
        if (st != GCA_OK) return st;
        continue;
      }
      cudaError_t e = cudaMemcpy(it.dst, it.src->p, sizeof(double) * it.n, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        gca::set_error(std::string("gca_h2_export: ") + cudaGetErrorString(e));
        return GCA_ERR_CUDA;
      }
    }
  return GCA_OK;
}

int gca_h2_status(const gca_h2* h, int32_t* status) {
  if (!h || !status) {
    gca::set_error("gca_h2_status: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  int v = 0;
  int st = gca::product_status(h, &v);
  if (st != GCA_OK) return st;
  *status = v;
  return GCA_OK;
}

namespace {
// the first error recorded in a product status word
int status_error(int bits, const char* what) {
  if (bits & 1) {
    gca::set_error(std::string(what) + ": a bounded device-side wait of a product expired");
    return GCA_ERR_TIMEOUT;
  }
  if (bits & 2) {
    gca::set_error(std::string(what) + ": a product kernel met a malformed work record");
    return GCA_ERR_INVALID_ARG;
  }
  return GCA_OK;
}

int sync_status(const gca::DevMem& st, void* stream, int* bits) {
  GCA_TRY_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  GCA_TRY_CUDA(cudaMemcpy(bits, st.p, sizeof(int), cudaMemcpyDeviceToHost));
  return GCA_OK;
}
}  // namespace

int gca_h2_check(const gca_h2* h, void* stream) {
  if (!h) {
    gca::set_error("gca_h2_check: NULL handle");
    return GCA_ERR_INVALID_ARG;
  }
  GCA_TRY(gca::check_device(h->device, "gca_h2_check"));
  int bits = 0;
  GCA_TRY(sync_status(h->d_status, stream, &bits));
  return status_error(bits, "gca_h2_check");
}

int gca_h2_clear_status(const gca_h2* h) {
  if (!h) {
    gca::set_error("gca_h2_clear_status: NULL handle");
    return GCA_ERR_INVALID_ARG;
  }
  GCA_TRY(gca::check_device(h->device, "gca_h2_clear_status"));
  GCA_TRY_CUDA(cudaDeviceSynchronize());
  GCA_TRY_CUDA(cudaMemset(h->d_status.p, 0, sizeof(int)));
  return GCA_OK;
}

int gca_test_hook(const char* name, int64_t value) {
  if (!name) {
    gca::set_error("gca_test_hook: NULL name");
    return GCA_ERR_INVALID_ARG;
  }
  const std::string n(name);
  if (n == "wait_cycles") {
    gca::g_wait_cycles = value > 0 ? (long long)value : gca::kDefaultWaitCycles;
  } else if (n == "stall_chain") {
    gca::g_stall_chain = value != 0 ? 1 : 0;
  } else if (n == "fail_alloc") {
    gca::g_fail_alloc = value > 0 ? (long long)value : 0;
  } else if (n == "device_skew") {
    gca::g_device_skew = (int)value;
  } else {
    gca::set_error("gca_test_hook: unknown hook " + n);
    return GCA_ERR_INVALID_ARG;
  }
  return GCA_OK;
}

void gca_free(gca_h2* h) { delete h; }

int gca_build_batch(int32_t count, const gca_mesh* meshes, const gca_tree* trees,
                    const gca_params* params, void* stream, gca_h2_batch** out) {
  if (!out || count < 1 || !meshes || !trees) {
    gca::set_error("gca_build_batch: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    auto b = std::make_unique<gca_h2_batch>();
    // groups of up to 8 meshes share their cross approximation launches (the
    // temporaries of a group's constructions are alive together)
    constexpr int32_t kGroup = 8;
    for (int32_t i0 = 0; i0 < count; i0 += kGroup) {
      const int32_t g = std::min(kGroup, count - i0);
      std::vector<gca_h2*> hs(g, nullptr);
      int st = gca::build_group(g, meshes + i0, trees + i0, params, static_cast<cudaStream_t>(stream), hs.data());
      for (gca_h2* h : hs)
        if (h) b->h.push_back(h);  // owned by the batch from here on, freed with it on error
      if (st != GCA_OK) {
        gca::set_error("gca_build_batch: meshes " + std::to_string(i0) + ".." + std::to_string(i0 + g - 1) +
                       ": " + gca_last_error());
        return st;
      }
    }
    b->device = b->h[0]->device;
    int st = b->d_status.alloc(sizeof(int));
    if (st != GCA_OK) return st;
    if (cudaMemset(b->d_status.p, 0, sizeof(int)) != cudaSuccess) {
      gca::set_error("gca_build_batch: cudaMemset failed");
      return GCA_ERR_CUDA;
    }
    st = gca::prepare_batch(b.get(), static_cast<cudaStream_t>(stream));
    if (st != GCA_OK) return st;
    *out = b.release();
    return GCA_OK;
  } catch (const std::bad_alloc&) {
    gca::set_error("gca_build_batch: host allocation failed");
    return GCA_ERR_OOM;
  }
}

int gca_batch_size(const gca_h2_batch* b, int32_t* count) {
  if (!b || !count) {
    gca::set_error("gca_batch_size: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  *count = (int32_t)b->h.size();
  return GCA_OK;
}

int gca_batch_handle(const gca_h2_batch* b, int32_t i, const gca_h2** h) {
  if (!b || !h || i < 0 || i >= (int32_t)b->h.size()) {
    gca::set_error("gca_batch_handle: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  *h = b->h[i];
  return GCA_OK;
}

int h2_matvec_batch(const gca_h2_batch* b, gca_prec prec, const int32_t* nrhs, const void* const* x,
                    const int64_t* ldx, void* const* y, const int64_t* ldy, void* stream) {
  return gca::matvec_batch(b, prec, false, nrhs, x, ldx, y, ldy, static_cast<cudaStream_t>(stream));
}

int h2_matvec_transpose_batch(const gca_h2_batch* b, gca_prec prec, const int32_t* nrhs,
                              const void* const* x, const int64_t* ldx, void* const* y,
                              const int64_t* ldy, void* stream) {
  return gca::matvec_batch(b, prec, true, nrhs, x, ldx, y, ldy, static_cast<cudaStream_t>(stream));
}

int gca_batch_status(const gca_h2_batch* b, int32_t* status) {
  if (!b || !status) {
    gca::set_error("gca_batch_status: NULL argument");
    return GCA_ERR_INVALID_ARG;
  }
  int v = 0;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&v, b->d_status.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    gca::set_error("gca_batch_status: CUDA error");
    return GCA_ERR_CUDA;
  }
  *status = v;
  return GCA_OK;
}

int gca_batch_check(const gca_h2_batch* b, void* stream) {
  if (!b) {
    gca::set_error("gca_batch_check: NULL batch");
    return GCA_ERR_INVALID_ARG;
  }
  GCA_TRY(gca::check_device(b->device, "gca_batch_check"));
  int bits = 0;
  GCA_TRY(sync_status(b->d_status, stream, &bits));
  return status_error(bits, "gca_batch_check");
}

int gca_batch_clear_status(const gca_h2_batch* b) {
  if (!b) {
    gca::set_error("gca_batch_clear_status: NULL batch");
    return GCA_ERR_INVALID_ARG;
  }
  GCA_TRY(gca::check_device(b->device, "gca_batch_clear_status"));
  GCA_TRY_CUDA(cudaDeviceSynchronize());
  GCA_TRY_CUDA(cudaMemset(b->d_status.p, 0, sizeof(int)));
  return GCA_OK;
}

void gca_free_batch(gca_h2_batch* b) { delete b; }

int gca_tune_batch(const gca_h2_batch* b, gca_prec prec, int32_t transpose, const int32_t* nrhs,
                   const void* const* x, const int64_t* ldx, void* const* y, const int64_t* ldy, void* stream,
                   int32_t* width) {
  int w = 0;
  const int st = gca::tune_batch(b, prec, transpose != 0, nrhs, x, ldx, y, ldy,
                                 static_cast<cudaStream_t>(stream), &w);
  if (st == GCA_OK && width) *width = w;
  return st;
}

int gca_tune_save(const char* path) { return gca::tune_save(path); }

int gca_tune_load(const char* path) { return gca::tune_load(path); }

int gca_tune_get(const char* device, gca_prec prec, int32_t transpose, int32_t nrhs, int64_t rows,
                 int32_t* width) {
  int w = 0;
  const int st = gca::tune_get(device, prec, transpose != 0, nrhs, rows, &w);
  if (st == GCA_OK && width) *width = w;
  return st;
}

void gca_tune_clear(void) { gca::tune_clear(); }

const char* gca_strerror(int status) {
  switch (status) {
    case GCA_OK: return "ok";
    case GCA_ERR_INVALID_ARG: return "invalid argument";
    case GCA_ERR_CUDA: return "CUDA runtime error";
    case GCA_ERR_OOM: return "out of memory";
    case GCA_ERR_NUMERIC: return "non-finite value";
    case GCA_ERR_TIMEOUT: return "device wait timed out";
    case GCA_ERR_UNSUPPORTED: return "unsupported size or option";
    case GCA_ERR_IO: return "file error or not a checkpoint";
    default: return "unknown status";
  }
}

}  // extern "C"
