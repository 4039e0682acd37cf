// H^2 matrix-vector products in one persistent launch.
//
// The product with the representation of Sect. 4 is the standard H^2
// recursion: forward transform x-hat_tau = V_tau^* x (leaves) and
// x-hat_tau = sum_c E_c^* x-hat_c (up the tree), coupling
// y-hat_tau = sum_sigma S_{tau sigma} x-hat_sigma, backward transform
// y-hat_c += E_c y-hat_parent (down the tree), and at the leaves
// y = V_tau y-hat_tau + sum_sigma N_{tau sigma} x|sigma-hat.  The transposed
// product swaps S, N for S^T, N^T.
//
// Every stage is a small dense product with a stored block in panel layout
// (panel.cuh).  The whole recursion is cut into warp work items of 32
// output rows x one block, listed in a dependency-respecting order:
//
//   forward (leaves, then level by level up) -> coupling -> near field
//   -> backward (level by level down) -> leaf bases
//
// and executed by one persistent kernel whose warps claim items with an
// atomic counter.  An item waits (bounded spin, acquire) until the vector it
// reads is complete, i.e. until a per-cluster counter has seen every item
// that contributes to it, then stages that vector in shared memory, streams
// its block from HBM and adds its 32 x RC results with atomics; items that
// complete a vector other items read bump that vector's counter (release).
// Items are claimed in list order and only wait for earlier items, so the
// earliest unfinished item always has its inputs and the launch cannot
// deadlock however many warps are resident.  A wait that exceeds its bound
// sets a timeout bit in the handle's status word and goes on (no hang).
//
// x is gathered into cluster order first and y scattered back to the
// caller's order last; x-hat, y-hat, y (cluster order) and the counters are
// zeroed by one memset per product.

#include <cuda_bf16.h>

#include <algorithm>
#include <string>

#include "internal.hpp"
#include "panel.cuh"

namespace gca {

namespace {

constexpr int kBatch = 2;            // items claimed per atomic
constexpr int kSpinLimit = 1 << 20;  // bounded wait: well under a second with the back-off below
constexpr int kStatusTimeout = 1;

// One warp work item (host builds them, device executes them).
struct MvItem {
  int64_t a_off;  // element offset of the block in its panel array
  int64_t x_row;  // first row of the input vector block
  int64_t o_row;  // output row of lane 0
  int m;          // rows of the stored block (panel stride)
  int k;          // columns of the stored block = rows of the input block
  int a0;         // first block row handled by this item
  int kind;       // panel kind | (input << 4) | (output << 8)
  int wait_idx;   // counter that must reach wait_cnt * nchunk first (-1: none)
  int wait_cnt;
  int sig_idx;    // counter bumped after the outputs are added (-1: none)
  int pad;
};

enum { kInXh = 0, kInYh = 1, kInX = 2 };
enum { kOutXh = 0, kOutYh = 1, kOutY = 2 };

template <typename T, typename TV>
struct MvArgs {
  const void* A[kPanelKinds];  // panel arrays (near-field kinds hold TN)
  const MvItem* items;
  int64_t n_items;
  int nchunk;
  int R;
  const TV* x;                 // caller's x, original order, column-major
  int64_t ldx;
  TV* y;                       // caller's y, original order, column-major (zeroed)
  int64_t ldy;
  const int* perm;
  const TV* xp;                // x in cluster order [n][R]
  TV* yp;                      // y in cluster order [n][R] (zeroed)
  TV* xh;                      // [rank_sum][R]
  TV* yh;
  int* counters;               // [2 nc]
  unsigned long long* next;    // work-claim counter
  int* status;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// 16-byte copy that reads src_bytes (0 or 16) and zero-fills the rest
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Ring of the per-warp block stream: kStages stages of kStagePanels panels,
// each panel 32 rows x 16 bytes.
constexpr int kStagePanels = 8;
constexpr int kStages = 4;
constexpr int kRingBytes = kStages * kStagePanels * 32 * 16;

// acc[c] += sum_k A[a0 + lane, k] Xs[k, c] over the 32-row slice of a panel
// block, streamed through the warp's shared-memory ring with cp.async.
template <typename T, typename TA, int RC>
__device__ __forceinline__ void stream_block(const T* __restrict__ A, int M, int a0, int kp,
                                             const TA* __restrict__ Xs, unsigned char* ring,
                                             int lane, TA (&acc)[RC]) {
  constexpr int P = Panel<T>::P;
  const int np = kp / P;
  const int nst = (np + kStagePanels - 1) / kStagePanels;
  const bool valid = a0 + lane < M;
  const uint4* src = reinterpret_cast<const uint4*>(A) + a0 + lane;
  auto issue = [&](int s) {
    if (s < nst) {
      unsigned char* slot = ring + (s % kStages) * (kStagePanels * 512) + lane * 16;
#pragma unroll
      for (int g = 0; g < kStagePanels; ++g) {
        const int p = s * kStagePanels + g;
        if (p < np)
          cp_async16_zfill(slot + g * 512, valid ? src + (int64_t)p * M : reinterpret_cast<const uint4*>(A),
                           valid ? 16 : 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) issue(s);
  for (int s = 0; s < nst; ++s) {
    issue(s + kStages - 1);
    cp_async_wait_group<kStages - 1>();
    __syncwarp();
    const unsigned char* slot = ring + (s % kStages) * (kStagePanels * 512) + lane * 16;
#pragma unroll
    for (int g = 0; g < kStagePanels; ++g) {
      const int p = s * kStagePanels + g;
      if (p >= np) break;
      TA v[P];
      unpack(*reinterpret_cast<const uint4*>(slot + g * 512), v);
#pragma unroll
      for (int kk = 0; kk < P; ++kk) {
        const TA* xr = Xs + (p * P + kk) * RC;
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[c] = fma(v[kk], xr[c], acc[c]);
      }
    }
    __syncwarp();
  }
}

// add RC consecutive values of one output row (16-byte vector atomics when
// the row segment is 16-byte aligned: R and c0 multiples of 4)
template <int RC>
__device__ __forceinline__ void add_row(float* p, const float (&v)[RC], int valid_cols, bool aligned) {
  if (RC % 4 == 0 && valid_cols == RC && aligned) {
#pragma unroll
    for (int c = 0; c < RC; c += 4)
      atomicAdd(reinterpret_cast<float4*>(p + c), make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]));
  } else {
#pragma unroll
    for (int c = 0; c < RC; ++c)
      if (c < valid_cols) atomicAdd(p + c, v[c]);
  }
}
template <int RC>
__device__ __forceinline__ void add_row(double* p, const double (&v)[RC], int valid_cols, bool) {
#pragma unroll
  for (int c = 0; c < RC; ++c)
    if (c < valid_cols) atomicAdd(p + c, v[c]);
}

template <typename TV>
__global__ void k_gather(int n, int R, const int* __restrict__ perm, const TV* __restrict__ x,
                         int64_t ldx, TV* __restrict__ xp) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * R) return;
  const int i = (int)(idx / R), c = (int)(idx % R);
  xp[idx] = x[perm[i] + c * ldx];
}

template <typename TV>
__global__ void k_scatter(int n, int R, const int* __restrict__ perm, const TV* __restrict__ yp,
                          TV* __restrict__ y, int64_t ldy) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * R) return;
  const int c = (int)(idx / n), i = (int)(idx % n);
  y[perm[i] + c * ldy] = yp[(int64_t)i * R + c];
}

template <typename T, typename TN, typename TA, typename TV, int RC>
__global__ void __launch_bounds__(32) k_h2_persistent(MvArgs<T, TV> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* ring = smem_raw;
  TA* Xs = reinterpret_cast<TA*>(smem_raw + kRingBytes);
  const int lane = threadIdx.x;
  const int64_t total = g.n_items * g.nchunk;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(g.next, (unsigned long long)kBatch);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base >= total) break;
    const int64_t stop = min((int64_t)base + kBatch, total);
    for (int64_t w = (int64_t)base; w < stop; ++w) {
      const MvItem it = g.items[w / g.nchunk];
      const int c0 = (int)(w % g.nchunk) * RC;
      const int ain = it.kind & 15, xin = (it.kind >> 4) & 15, out = (it.kind >> 8) & 15;

      // wait until the input vector block is complete
      if (it.wait_idx >= 0) {
        const int need = it.wait_cnt * g.nchunk;
        int spins = 0;
        while (ld_acquire(g.counters + it.wait_idx) < need) {
          if (++spins > kSpinLimit) {
            if (lane == 0) atomicOr(g.status, kStatusTimeout);
            break;
          }
          __nanosleep(128);
        }
      }

      // stage the input rows (zero beyond k up to pad8(k)) for RHS c0 .. c0+RC
      const int kp = pad8(it.k);
      {
        const TV* X = (xin == kInXh ? g.xh : (xin == kInYh ? g.yh : g.xp)) + it.x_row * g.R + c0;
        constexpr int V = 16 / (int)sizeof(TA);  // values per 16-byte copy
        if (RC % V == 0 && g.R % V == 0 && c0 + RC <= g.R) {
          for (int i = lane; i < it.k * (RC / V); i += 32) {
            const int r = i / (RC / V), c = (i % (RC / V)) * V;
            cp_async16(Xs + r * RC + c, X + (int64_t)r * g.R + c);
          }
          cp_async_commit();
          for (int i = it.k * RC + lane; i < kp * RC; i += 32) Xs[i] = (TA)0;
        } else {
          for (int i = lane; i < kp * RC; i += 32) {
            const int r = i / RC, c = i % RC;
            Xs[i] = (r < it.k && c0 + c < g.R) ? (TA)__ldcg(X + (int64_t)r * g.R + c) : (TA)0;
          }
        }
      }
      __syncwarp();

      // 32 rows of the block times the staged vector block (the vector's
      // cp.async group completes with the block's first stage)
      const bool valid = it.a0 + lane < it.m;
      TA acc[RC];
#pragma unroll
      for (int c = 0; c < RC; ++c) acc[c] = (TA)0;
      if (ain == kN || ain == kNt)
        stream_block<TN, TA, RC>(static_cast<const TN*>(g.A[ain]) + it.a_off, it.m, it.a0, kp, Xs,
                                 ring, lane, acc);
      else
        stream_block<T, TA, RC>(static_cast<const T*>(g.A[ain]) + it.a_off, it.m, it.a0, kp, Xs, ring,
                                lane, acc);

      if (valid) {
        TV* orow = (out == kOutXh ? g.xh : (out == kOutYh ? g.yh : g.yp)) + (it.o_row + lane) * g.R + c0;
        add_row<RC>(orow, acc, min(RC, g.R - c0), (g.R % 4) == 0 && (c0 % 4) == 0);
      }
      if (it.sig_idx >= 0) {
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(g.counters + it.sig_idx, 1);
      }
      __syncwarp();
    }
  }
}

}  // namespace

// Work items of one direction (0: product, 1: transposed product).
int build_items(gca_h2* h, int dir, cudaStream_t st) {
  const int nc = h->nc;
  const bool trans = dir == 1;
  std::vector<MvItem> items;
  std::vector<int> cx(nc, 0), cy(nc, 0);  // contributions to x-hat_c, y-hat_c
  auto chunks = [&](int kind, int in, int out, int64_t a_off, int m, int k, int64_t x_row,
                    int64_t o_row0, int wait_idx, int wait_cnt, int sig_idx, int* sig_cnt) {
    for (int a0 = 0; a0 < m; a0 += 32) {
      MvItem it{};
      it.a_off = a_off;
      it.x_row = x_row;
      it.o_row = o_row0 + a0;
      it.m = m;
      it.k = k;
      it.a0 = a0;
      it.kind = kind | (in << 4) | (out << 8);
      it.wait_idx = wait_cnt > 0 ? wait_idx : -1;
      it.wait_cnt = wait_cnt;
      it.sig_idx = sig_idx;
      items.push_back(it);
      if (sig_cnt) ++*sig_cnt;
    }
  };
  const auto& O = h->panel_off;
  // forward transform: leaves
  for (int c : h->leaves)
    if (c > 0 && h->rank[c] > 0)
      chunks(kVt, kInX, kOutXh, O[kVt][c], h->rank[c], h->end[c] - h->begin[c], h->begin[c],
             h->xoff[c], -1, 0, c, &cx[c]);
  // forward transform: up the tree, deepest level first
  for (int L = h->depth - 1; L >= 1; --L)
    for (int p : h->by_level[L]) {
      if (h->child0[p] < 0) continue;
      for (int ch : {h->child0[p], h->child1[p]})
        chunks(kEt, kInXh, kOutXh, O[kEt][ch], h->rank[p], h->rank[ch], h->xoff[ch], h->xoff[p], ch,
               cx[ch], p, &cx[p]);
    }
  // coupling, blocks whose input cluster is deepest first
  const int nfar = (int)h->far_t.size();
  std::vector<int> order(nfar);
  for (int b = 0; b < nfar; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
    const int iu = trans ? h->far_t[u] : h->far_s[u], iv = trans ? h->far_t[v] : h->far_s[v];
    return h->level[iu] > h->level[iv];
  });
  for (int b : order) {
    const int t = h->far_t[b], s = h->far_s[b];
    const int own = trans ? s : t, in = trans ? t : s;
    chunks(trans ? kSt : kS, kInXh, kOutYh, O[trans ? kSt : kS][b], h->rank[own], h->rank[in],
           h->xoff[in], h->xoff[own], in, cx[in], nc + own, &cy[own]);
  }
  // near field (no dependencies)
  for (int b = 0; b < (int)h->near_t.size(); ++b) {
    const int t = h->near_t[b], s = h->near_s[b];
    const int own = trans ? s : t, in = trans ? t : s;
    chunks(trans ? kNt : kN, kInX, kOutY, O[trans ? kNt : kN][b], h->end[own] - h->begin[own],
           h->end[in] - h->begin[in], h->begin[in], h->begin[own], -1, 0, -1, nullptr);
  }
  // backward transform, level by level down (y-hat of the parent must be final)
  for (int L = 2; L <= h->depth; ++L)
    for (int c : h->by_level[L]) {
      const int p = h->parent[c];
      if (cy[p] == 0 || h->rank[c] == 0) continue;  // y-hat_p = 0
      chunks(kE, kInYh, kOutYh, O[kE][c], h->rank[c], h->rank[p], h->xoff[p], h->xoff[c], nc + p,
             cy[p], nc + c, &cy[c]);
    }
  // leaf bases
  for (int c : h->leaves)
    if (c > 0 && h->rank[c] > 0 && cy[c] > 0)
      chunks(kV, kInYh, kOutY, O[kV][c], h->end[c] - h->begin[c], h->rank[c], h->xoff[c],
             h->begin[c], nc + c, cy[c], -1, nullptr);
  h->n_items[dir] = (int64_t)items.size();
  GCA_TRY(upload(h->d_items[dir], items, st));
  return GCA_OK;
}

int finish_plan(gca_h2* h, cudaStream_t st) {
  h->max_rows = std::max(h->max_rank, h->max_leaf);
  GCA_TRY(build_items(h, 0, st));
  GCA_TRY(build_items(h, 1, st));
  GCA_TRY(h->d_status.alloc(sizeof(int)));
  GCA_TRY_CUDA(cudaMemsetAsync(h->d_status.p, 0, sizeof(int), st));
  return GCA_OK;
}

namespace {

template <typename T, typename TN, typename TA, typename TV, int RC>
int run_rc(const gca_h2* h, const DevMem* P, const DevMem* PN, bool trans, int R, const TV* x,
           int64_t ldx, TV* y, int64_t ldy, cudaStream_t st) {
  const char* pn = sizeof(T) == 8 ? ".f64" : (sizeof(T) == 4 ? ".f32" : ".bf16");
  PhaseScope ps(std::string("mv_persistent") + pn + (trans ? ".T" : ""), st);
  ps.launches(4);
  const int dir = trans ? 1 : 0;
  const int nchunk = (R + RC - 1) / RC;
  // workspace: x-hat | y-hat | y (cluster order) | counters | claim counter | x (cluster order)
  auto up256 = [](size_t b) { return (b + 255) & ~(size_t)255; };  // keeps every region aligned
  const size_t vec_bytes = up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum, 1) * R);
  const size_t n_bytes = up256(sizeof(TV) * (size_t)h->n * R);
  const size_t cnt_bytes = up256(sizeof(int) * 2 * (size_t)h->nc);
  const size_t zeroed = 2 * vec_bytes + n_bytes + cnt_bytes + 256;
  GCA_TRY(h->w_ws.reserve(zeroed + n_bytes));
  unsigned char* base = h->w_ws.as<unsigned char>();
  MvArgs<T, TV> g{};
  for (int q = 0; q < kPanelKinds; ++q) g.A[q] = (q == kN || q == kNt) ? PN[q].p : P[q].p;
  g.items = h->d_items[dir].as<MvItem>();
  g.n_items = h->n_items[dir];
  g.nchunk = nchunk;
  g.R = R;
  g.x = x;
  g.ldx = ldx;
  g.y = y;
  g.ldy = ldy;
  g.perm = h->d_perm.as<int>();
  g.xh = reinterpret_cast<TV*>(base);
  g.yh = reinterpret_cast<TV*>(base + vec_bytes);
  g.yp = reinterpret_cast<TV*>(base + 2 * vec_bytes);
  g.counters = reinterpret_cast<int*>(base + 2 * vec_bytes + n_bytes);
  g.next = reinterpret_cast<unsigned long long*>(base + 2 * vec_bytes + n_bytes + cnt_bytes);
  TV* xp = reinterpret_cast<TV*>(base + zeroed);
  g.xp = xp;
  g.status = h->d_status.as<int>();
  GCA_TRY_CUDA(cudaMemsetAsync(base, 0, zeroed, st));
  const int nt = 256;
  const unsigned nb = (unsigned)(((int64_t)h->n * R + nt - 1) / nt);
  k_gather<TV><<<nb, nt, 0, st>>>(h->n, R, h->d_perm.as<int>(), x, ldx, xp);
  const size_t smem = kRingBytes + sizeof(TA) * (size_t)pad8(h->max_rows) * RC;
  auto kern = k_h2_persistent<T, TN, TA, TV, RC>;
  if (smem > 48 * 1024)
    GCA_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  GCA_TRY_CUDA(cudaGetDevice(&dev));
  GCA_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GCA_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem));
  const int64_t want = (g.n_items * nchunk + kBatch - 1) / kBatch;
  const int64_t cap = (int64_t)sms * std::max(per_sm, 1);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(want, cap));
  if (g.n_items > 0) kern<<<grid, 32, smem, st>>>(g);
  k_scatter<TV><<<nb, nt, 0, st>>>(h->n, R, h->d_perm.as<int>(), g.yp, y, ldy);
  GCA_TRY_CUDA(cudaGetLastError());
  return GCA_OK;
}

template <typename T, typename TN, typename TA, typename TV>
int run(const gca_h2* h, const DevMem* P, const DevMem* PN, bool trans, int R, const TV* x,
        int64_t ldx, TV* y, int64_t ldy, cudaStream_t st) {
  if (R >= 16) return run_rc<T, TN, TA, TV, 16>(h, P, PN, trans, R, x, ldx, y, ldy, st);
  if (R > 4) return run_rc<T, TN, TA, TV, 8>(h, P, PN, trans, R, x, ldx, y, ldy, st);
  if (R > 2) return run_rc<T, TN, TA, TV, 4>(h, P, PN, trans, R, x, ldx, y, ldy, st);
  if (R > 1) return run_rc<T, TN, TA, TV, 2>(h, P, PN, trans, R, x, ldx, y, ldy, st);
  return run_rc<T, TN, TA, TV, 1>(h, P, PN, trans, R, x, ldx, y, ldy, st);
}

}  // namespace

int matvec(const gca_h2* h, gca_prec prec, bool trans, int32_t nrhs, const void* x, int64_t ldx,
           void* y, int64_t ldy, cudaStream_t st) {
  if (!h || !x || !y || nrhs < 1 || nrhs > 4096 || ldx < h->n || ldy < h->n) {
    set_error("h2_matvec: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  switch (prec) {
    case GCA_F64:
      return run<double, double, double, double>(h, h->P64, h->P64, trans, nrhs, (const double*)x,
                                                 ldx, (double*)y, ldy, st);
    case GCA_F32:
      return run<float, float, float, float>(h, h->P32, h->P32, trans, nrhs, (const float*)x, ldx,
                                             (float*)y, ldy, st);
    case GCA_BF16:
      return run<__nv_bfloat16, float, float, float>(h, h->P16, h->P32, trans, nrhs,
                                                     (const float*)x, ldx, (float*)y, ldy, st);
  }
  set_error("h2_matvec: unknown precision");
  return GCA_ERR_INVALID_ARG;
}

int product_status(const gca_h2* h, int* out) {
  int v = 0;
  GCA_TRY_CUDA(cudaDeviceSynchronize());
  GCA_TRY_CUDA(cudaMemcpy(&v, h->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
  *out = v;
  return GCA_OK;
}

}  // namespace gca
