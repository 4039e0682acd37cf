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
#include <mutex>
#include <queue>
#include <cstring>
#include <string>

#include "internal.hpp"
#include "panel.cuh"

namespace gca {

namespace {

constexpr int kSpinLimit = 1 << 20;  // bounded wait: well under a second with the back-off below
constexpr int kStatusTimeout = 1;

// One warp work item (host builds them, device executes them).
struct MvItem {
  int64_t a_off;  // element offset of the block in its panel array
  int64_t x_row;  // first row of the input vector block
  int64_t o_row;  // output row of lane 0
  int m;          // rows of the stored block (panel stride)
  int k;          // columns of this item's column chunk (<= kChunk)
  int a0;         // first block row handled by this item
  int k0;         // first block column of the chunk
  int kind;       // panel kind | (input << 4) | (output << 8)
  int wait_idx;   // counter that must reach wait_cnt * nchunk first (-1: none)
  int wait_cnt;
  int sig_idx;    // counter bumped after the outputs are added (-1: none)
  int flush;      // last segment of its group: add the accumulated rows to the output
};

enum { kInXh = 0, kInYh = 1, kInX = 2 };
enum { kOutXh = 0, kOutYh = 1, kOutY = 2 };

// Everything one mesh (slot) of a launch needs; a launch runs the work of
// any number of slots, each slot's work list in dependency order, slot after
// slot in claim order.
template <typename TV>
struct SlotArgs {
  const void* A[kPanelKinds];  // panel arrays (near-field kinds hold the near storage type)
  const MvItem* items;
  const int2* groups;          // chain list: [begin, end) segment ranges claimed as a unit
  const int2* free_groups;     // free list (no dependencies)
  int64_t work_begin;          // first chain claim index of this slot
  int64_t n_work;              // chain groups * nchunk
  int64_t free_begin;          // first free claim index of this slot
  int64_t n_free;              // free groups * nchunk
  int nchunk;
  int R;
  int n;
  int pad;
  const TV* x;                 // caller's x, original order, column-major
  int64_t ldx;
  TV* y;                       // caller's y, original order, column-major
  int64_t ldy;
  const int* perm;
  const TV* xp;                // x in cluster order [n][R]
  TV* yp;                      // y in cluster order [n][R] (zeroed)
  TV* xh;                      // [rank_sum][R]
  TV* yh;
  int* counters;               // [2 nc]
};

struct LaunchArgs {
  const void* slots;           // SlotArgs<TV>[nslots]
  int nslots;
  int64_t total;               // chain claims over all slots
  int64_t total_free;          // free claims over all slots
  unsigned long long* next;    // chain claim counter
  unsigned long long* next_free;  // free claim counter
  int* status;
  int* abort_flag;             // raised by any timed-out wait; every wait gives up
};

template <typename TV>
__device__ __forceinline__ int find_slot(const SlotArgs<TV>* sl, int nslots, int64_t w) {
  int lo = 0, hi = nslots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sl[mid].work_begin <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename TV>
__device__ __forceinline__ int find_free_slot(const SlotArgs<TV>* sl, int nslots, int64_t w) {
  int lo = 0, hi = nslots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sl[mid].free_begin <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------- pipeline
//
// Every warp of the persistent launch works on its own: it claims a group
// (claim-ahead), streams the group's block panels into its private ring of
// shared-memory stages with 1-D bulk copies (TMA) completing on per-stage
// mbarriers, waits for the segment's input vector block (bounded spin on the
// dependency counter), stages it, and accumulates in registers.  A segment =
// kItemRows rows x kChunk columns of one stored block; the stages of the
// group's segments form one stream, so the next segment's panels are in
// flight while the current one is computed.  A warp stalled on a dependency
// stalls nobody else.
constexpr int kWarps = 4;                                   // independent warps per CTA
constexpr int kThreads = 32 * kWarps;
constexpr int kItemRows = 64;                               // rows per segment (one warp tile)
constexpr int kChunk = 64;                                  // columns per segment
constexpr int kStagePanels = 4;
constexpr int kStageBytes = kStagePanels * kItemRows * 16;  // 4 KB: one contiguous copy
constexpr int kStages = 3;
constexpr int kMbarLimit = 1 << 20;
constexpr int kMaxGroupSegs = 8;  // segments of a group

// shared memory of one warp: ring, input block, mbarriers (kStages + 1)
template <typename TA, int RC>
__host__ __device__ constexpr size_t warp_smem() {
  return ((size_t)kStages * kStageBytes + sizeof(TA) * (size_t)kChunk * RC + (kStages + 1) * 8 + 127) /
         128 * 128;
}
template <typename TA, int RC>
__host__ __device__ constexpr size_t cta_smem() {
  return kWarps * warp_smem<TA, RC>();
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, unsigned tx) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(b)),
               "r"(tx)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of parity `parity`; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag,
                                          int* status) {
  for (int i = 0; i < kMbarLimit; ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if ((i & 63) == 63 && *abort_flag) return false;
  }
  atomicOr(status, kStatusTimeout);
  *abort_flag = 1;
  return false;
}
// Bounded wait used only while draining copies before exit (ignores the
// abort flag, so that no copy is still landing when the warp retires).
__device__ __forceinline__ void mbar_drain(uint64_t* b, unsigned parity) {
  for (int i = 0; i < kMbarLimit; ++i)
    if (mbar_try_wait(b, parity)) return;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// orders this thread's generic-proxy shared-memory accesses before later
// bulk copies (async proxy) into the same buffers
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// orders global-memory writes seen through an acquire before later bulk
// copies (async proxy) that read them
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Fire-and-forget reductions into global memory (no return value, so the
// issuing warp does not wait for the L2 round trip).
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// add N consecutive values of one output row (16-byte vector reductions
// when the segment is 16-byte aligned)
template <int N>
__device__ __forceinline__ void add_row(float* p, const float* v, int valid_cols, bool aligned) {
  if (N % 4 == 0 && valid_cols >= N && aligned) {
#pragma unroll
    for (int c = 0; c < N; c += 4) red_add4(p + c, v[c], v[c + 1], v[c + 2], v[c + 3]);
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c)
      if (c < valid_cols) red_add(p + c, v[c]);
  }
}
template <int N>
__device__ __forceinline__ void add_row(double* p, const double* v, int valid_cols, bool) {
#pragma unroll
  for (int c = 0; c < N; ++c)
    if (c < valid_cols) red_add(p + c, v[c]);
}

// x (original order) -> x in cluster order, all slots of a launch
// (blockIdx.y = slot)
template <typename TV>
__global__ void k_gather(const SlotArgs<TV>* __restrict__ slots) {
  const SlotArgs<TV>& sa = slots[blockIdx.y];
  const int64_t tot = (int64_t)sa.n * sa.R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / sa.R), c = (int)(idx % sa.R);
    const_cast<TV*>(sa.xp)[idx] = sa.x[sa.perm[i] + c * sa.ldx];
  }
}

// y in cluster order -> caller's y (original order)
template <typename TV>
__global__ void k_scatter(const SlotArgs<TV>* __restrict__ slots) {
  const SlotArgs<TV>& sa = slots[blockIdx.y];
  const int64_t tot = (int64_t)sa.n * sa.R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / sa.n), i = (int)(idx % sa.n);
    sa.y[sa.perm[i] + c * sa.ldy] = sa.yp[(int64_t)i * sa.R + c];
  }
}

// Register tile of a warp: 64 rows x RC right-hand sides.  CPL = min(RC, 8)
// columns per lane, NCG = RC / CPL column groups, RG = 32 / NCG row groups,
// RPL = 64 / RG rows per lane; lane (rg, cg) owns rows rg + RG * i (i < RPL)
// and columns cg * CPL + [0, CPL).  Rows of one load instruction are
// consecutive (conflict-free 16-byte shared loads).
template <int RC>
struct Tile {
  static constexpr int CPL = RC < 8 ? RC : 8;
  static constexpr int NCG = RC / CPL;
  static constexpr int RG = 32 / NCG;
  static constexpr int RPL = 64 / RG;
};

// One ring stage: npst panels (P columns each, `pst` bytes apart) of the
// lane's rows.
template <typename T, typename TA, int RC>
__device__ __forceinline__ void consume_stage(const unsigned char* stage, int pst, int npst, int p0,
                                              const TA* __restrict__ Xs, int rg, int cg,
                                              TA (&acc)[Tile<RC>::RPL][Tile<RC>::CPL]) {
  using Tl = Tile<RC>;
  constexpr int P = Panel<T>::P;
  // the stage's sum (at most kStagePanels * P terms) is formed on its own
  // and then added: two-level summation keeps the rounding error of the
  // long sums over a group's segments near that of a few short chains
  TA part[Tl::RPL][Tl::CPL];
#pragma unroll
  for (int i = 0; i < Tl::RPL; ++i)
#pragma unroll
    for (int c = 0; c < Tl::CPL; ++c) part[i][c] = (TA)0;
#pragma unroll
  for (int g = 0; g < kStagePanels; ++g) {
    if (g >= npst) break;
    TA v[Tl::RPL][P];
#pragma unroll
    for (int i = 0; i < Tl::RPL; ++i)
      unpack(*reinterpret_cast<const uint4*>(stage + g * pst + (rg + Tl::RG * i) * 16), v[i]);
#pragma unroll
    for (int kk = 0; kk < P; ++kk) {
      const TA* xr = Xs + ((p0 + g) * P + kk) * RC + cg * Tl::CPL;
      TA x[Tl::CPL];
#pragma unroll
      for (int c = 0; c < Tl::CPL; ++c) x[c] = xr[c];
#pragma unroll
      for (int i = 0; i < Tl::RPL; ++i)
#pragma unroll
        for (int c = 0; c < Tl::CPL; ++c) part[i][c] = fma(v[i][kk], x[c], part[i][c]);
    }
  }
#pragma unroll
  for (int i = 0; i < Tl::RPL; ++i)
#pragma unroll
    for (int c = 0; c < Tl::CPL; ++c) acc[i][c] += part[i][c];
}

// A segment (one tile of a stored block) as the issuing side sees it.
struct SegSrc {
  const unsigned char* A;  // the tile
  int rows;                // rows of the tile: panels are rows * 16 bytes apart
  int np;                  // panels of the tile
};

template <typename T, typename TN, typename TV>
__device__ __forceinline__ SegSrc seg_src(const SlotArgs<TV>& sa, const MvItem& it) {
  const int ain = it.kind & 15;
  const bool is_near = ain == kN || ain == kNt;
  const int P = is_near ? Panel<TN>::P : Panel<T>::P;
  const int esz = is_near ? (int)sizeof(TN) : (int)sizeof(T);
  SegSrc s;
  s.A = static_cast<const unsigned char*>(sa.A[ain]) + it.a_off * esz;
  s.rows = min(kItemRows, it.m - it.a0);
  s.np = pad8(it.k) / P;
  return s;
}

// Per-warp state of the stage ring (shared memory of the warp).
template <typename TA, int RC>
struct WarpRing {
  unsigned char* ring;
  TA* Xs;
  uint64_t* full;
  uint64_t* xbar;
  uint32_t fill, use, xuse;  // stages issued / consumed, input blocks copied
};

// Every segment of group [grp.x, grp.y) has its input block complete.
template <typename TV>
__device__ __forceinline__ bool group_ready(const SlotArgs<TV>& sa, int2 grp, int lane) {
  bool ok = true;
  for (int s = grp.x + lane; s < grp.y; s += 32) {
    const MvItem& it = sa.items[s];
    if (it.wait_idx >= 0 && ld_acquire(sa.counters + it.wait_idx) < it.wait_cnt * sa.nchunk) ok = false;
  }
  return __all_sync(0xffffffffu, ok);
}

// One claimed unit: the segments of one group for right-hand sides
// [c0, c0 + RC).  Returns false when a wait timed out or the launch aborted.
template <typename T, typename TN, typename TA, typename TV, int RC>
__device__ bool run_group(const SlotArgs<TV>& sa, int2 grp, int c0, WarpRing<TA, RC>& w,
                          TA (&acc)[Tile<RC>::RPL][Tile<RC>::CPL], const LaunchArgs& L, int lane) {
  using Tl = Tile<RC>;
  volatile int* abort_flag = L.abort_flag;
  const int rg = lane % Tl::RG, cg = lane / Tl::RG;
  // issuing cursor: segment `is`, its stage `ist`; stages of consecutive
  // segments form one stream through the ring
  int is = grp.x, ist = 0;
  SegSrc src = seg_src<T, TN, TV>(sa, sa.items[is]);
  auto issue = [&]() {
    if (is >= grp.y || w.fill - w.use >= (uint32_t)kStages) return;
    const int s = (int)(w.fill % kStages);
    if (lane == 0) {
      const int p0 = ist * kStagePanels;
      const int npst = min(kStagePanels, src.np - p0);
      const unsigned bytes = (unsigned)(npst * src.rows * 16);  // contiguous panels of the tile
      mbar_arrive_tx(w.full + s, bytes);
      bulk_g2s(w.ring + s * kStageBytes, src.A + (int64_t)p0 * src.rows * 16, bytes, w.full + s);
    }
    ++w.fill;
    if (++ist * kStagePanels >= src.np) {
      ist = 0;
      if (++is < grp.y) src = seg_src<T, TN, TV>(sa, sa.items[is]);
    }
  };
  for (int q = 0; q < kStages; ++q) issue();

  for (int us = grp.x; us < grp.y; ++us) {
    const MvItem it = sa.items[us];
    const int xin = (it.kind >> 4) & 15, out = (it.kind >> 8) & 15;
    const int rows = min(kItemRows, it.m - it.a0);
    const int ain = it.kind & 15;
    const bool is_near = ain == kN || ain == kNt;
    const int np = pad8(it.k) / (is_near ? Panel<TN>::P : Panel<T>::P);
    const int kp = pad8(it.k);
    // input vector block complete?
    if (it.wait_idx >= 0) {
      const int need = it.wait_cnt * sa.nchunk;
      int timeout = 0;
      if (lane == 0) {
        int spins = 0;
        while (ld_acquire(sa.counters + it.wait_idx) < need) {
          if (++spins > kSpinLimit) {
            atomicOr(L.status, kStatusTimeout);
            *abort_flag = 1;
            timeout = 1;
            break;
          }
          if (*abort_flag) {
            timeout = 1;
            break;
          }
          __nanosleep(32);
        }
      }
      if (__shfl_sync(0xffffffffu, timeout, 0)) return false;
    }
    // stage the input rows k0 .. k0 + kp (zero beyond the block's columns);
    // every lane is done reading the previous block (__syncwarp)
    const TV* X = (xin == kInXh ? sa.xh : (xin == kInYh ? sa.yh : sa.xp)) + it.x_row * sa.R + c0;
    const bool bulk = RC == sa.R && (RC * sizeof(TV)) % 16 == 0 && sizeof(TA) == sizeof(TV);
    fence_proxy_async();
    if (it.wait_idx >= 0) fence_proxy_async_global();  // the block was written by other warps
    __syncwarp();
    if (bulk) {
      for (int i = it.k * RC + lane; i < kp * RC; i += 32) w.Xs[i] = (TA)0;
      if (lane == 0) {
        const unsigned bytes = (unsigned)(it.k * RC * sizeof(TV));
        mbar_arrive_tx(w.xbar, bytes);
        bulk_g2s(w.Xs, X, bytes, w.xbar);
      }
      ++w.xuse;
      if (!mbar_wait(w.xbar, (w.xuse - 1) & 1, abort_flag, L.status)) return false;
    } else {
      for (int i = lane; i < kp * RC; i += 32) {
        const int r = i / RC, c = i % RC;
        w.Xs[i] = (r < it.k && c0 + c < sa.R) ? (TA)__ldcg(X + (int64_t)r * sa.R + c) : (TA)0;
      }
    }
    __syncwarp();
    for (int p0 = 0; p0 < np; p0 += kStagePanels) {
      const int s = (int)(w.use % kStages);
      if (!mbar_wait(w.full + s, (w.use / kStages) & 1, abort_flag, L.status)) return false;
      const unsigned char* stg = w.ring + s * kStageBytes;
      const int npst = min(kStagePanels, np - p0);
      if (is_near)
        consume_stage<TN, TA, RC>(stg, rows * 16, npst, p0, w.Xs, rg, cg, acc);
      else
        consume_stage<T, TA, RC>(stg, rows * 16, npst, p0, w.Xs, rg, cg, acc);
      ++w.use;
      fence_proxy_async();
      __syncwarp();
      issue();  // refill the freed stage (possibly with the next segment's panels)
    }
    if (!it.flush) continue;
    TV* obase = out == kOutXh ? sa.xh : (out == kOutYh ? sa.yh : sa.yp);
    const int R = sa.R;
    const int col0 = c0 + cg * Tl::CPL;
    const int vc = min(Tl::CPL, R - col0);
    const bool aligned = (R % 4) == 0 && (col0 % 4) == 0;
#pragma unroll
    for (int i = 0; i < Tl::RPL; ++i) {
      const int r = rg + Tl::RG * i;
      if (r < rows && vc > 0) add_row<Tl::CPL>(obase + (it.o_row + r) * R + col0, acc[i], vc, aligned);
    }
#pragma unroll
    for (int i = 0; i < Tl::RPL; ++i)
#pragma unroll
      for (int c = 0; c < Tl::CPL; ++c) acc[i][c] = (TA)0;
    if (it.sig_idx >= 0) {
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(sa.counters + it.sig_idx, 1);
    }
  }
  return true;
}

// Claim the next unit of a list; -1 once the list is exhausted.
__device__ __forceinline__ int64_t claim(unsigned long long* next, int64_t total, int lane) {
  unsigned long long v = 0;
  if (lane == 0) v = atomicAdd(next, 1ull);
  v = __shfl_sync(0xffffffffu, v, 0);
  return (int64_t)v < total ? (int64_t)v : -1;
}

// Persistent product over all slots of a launch.  Two work lists: the
// dependency chain (forward and backward transforms, couplings), claimed in
// a dependency order, and the free list (near field), which waits for
// nothing.  A warp whose chain group is not ready yet does free work
// meanwhile, and blocks on the chain only when the free list is exhausted.
template <typename T, typename TN, typename TA, typename TV, int RC>
__global__ void __launch_bounds__(kThreads) k_h2_persistent(LaunchArgs L) {
  using Tl = Tile<RC>;
  const SlotArgs<TV>* slots = static_cast<const SlotArgs<TV>*>(L.slots);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr size_t kRingBytes = (size_t)kStages * kStageBytes;
  constexpr size_t kXBytes = sizeof(TA) * (size_t)kChunk * RC;
  WarpRing<TA, RC> w;
  w.ring = smem_raw + warp * warp_smem<TA, RC>();
  w.Xs = reinterpret_cast<TA*>(w.ring + kRingBytes);
  w.full = reinterpret_cast<uint64_t*>(w.ring + kRingBytes + kXBytes);
  w.xbar = w.full + kStages;
  w.fill = w.use = w.xuse = 0;
  if (lane == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(w.full + i, 1);
    mbar_init(w.xbar, 1);
    fence_mbar_init();
  }
  __syncwarp();

  TA acc[Tl::RPL][Tl::CPL];
#pragma unroll
  for (int i = 0; i < Tl::RPL; ++i)
#pragma unroll
    for (int c = 0; c < Tl::CPL; ++c) acc[i][c] = (TA)0;

  bool ok = true;
  int64_t cu = claim(L.next, L.total, lane);
  bool free_left = true;
  while (ok) {
    if (cu >= 0) {
      const SlotArgs<TV>& sa = slots[find_slot(slots, L.nslots, cu)];
      const int64_t lw = cu - sa.work_begin;
      const int2 grp = sa.groups[lw / sa.nchunk];
      if (free_left && !group_ready(sa, grp, lane)) {
        const int64_t fu = claim(L.next_free, L.total_free, lane);
        if (fu >= 0) {
          const SlotArgs<TV>& sf = slots[find_free_slot(slots, L.nslots, fu)];
          const int64_t lf = fu - sf.free_begin;
          ok = run_group<T, TN, TA, TV, RC>(sf, sf.free_groups[lf / sf.nchunk], (int)(lf % sf.nchunk) * RC, w,
                                            acc, L, lane);
          continue;
        }
        free_left = false;
      }
      ok = run_group<T, TN, TA, TV, RC>(sa, grp, (int)(lw % sa.nchunk) * RC, w, acc, L, lane);
      cu = claim(L.next, L.total, lane);
      continue;
    }
    if (!free_left) break;
    const int64_t fu = claim(L.next_free, L.total_free, lane);
    if (fu < 0) break;
    const SlotArgs<TV>& sf = slots[find_free_slot(slots, L.nslots, fu)];
    const int64_t lf = fu - sf.free_begin;
    ok = run_group<T, TN, TA, TV, RC>(sf, sf.free_groups[lf / sf.nchunk], (int)(lf % sf.nchunk) * RC, w, acc,
                                      L, lane);
  }
  // drain: every issued copy has landed before the warp exits
  if (lane == 0) {
    for (uint32_t u = w.use; u < w.fill; ++u) mbar_drain(w.full + (u % kStages), (u / kStages) & 1);
    if (w.xuse > 0) mbar_drain(w.xbar, (w.xuse - 1) & 1);
  }
  __syncwarp();
}

}  // namespace

// Claim order of the groups.  The emission order below is a valid
// dependency order but makes CTAs claim groups long before their inputs
// exist.  This list scheduler simulates the launch: kWorkers warps, a group
// costs a fixed latency plus its bytes at a CTA's share of HBM bandwidth, a
// group is ready once every counter it waits for has seen all of its
// contributions, and among ready groups the one with the longest remaining
// dependency path (upward rank) starts first.  Groups are then claimed in
// simulated start order, which is again a dependency order (a group starts
// only after everything it waits for has finished), so the launch stays
// deadlock free.
void schedule_groups(const std::vector<MvItem>& items, std::vector<int2>& groups, int ncounters) {
  const int ng = (int)groups.size();
  if (ng < 2) return;
  constexpr double kWorkers = 148 * 16, kLatency = 2.0e-6, kBandwidth = 6.0e12;  // s, B/s
  std::vector<double> cost(ng);
  std::vector<int> sig(ng, -1);
  std::vector<std::vector<std::pair<int, int>>> waits(ng);
  std::vector<std::vector<int>> waiters(ncounters);
  std::vector<int> total(ncounters, 0);
  for (int gi = 0; gi < ng; ++gi) {
    double bytes = 0;
    for (int sgi = groups[gi].x; sgi < groups[gi].y; ++sgi) {
      const MvItem& it = items[sgi];
      bytes += 16.0 * std::min(kItemRows, it.m - it.a0) * (pad8(it.k) / 4);  // float panels
      if (it.wait_idx >= 0) waits[gi].push_back({it.wait_idx, it.wait_cnt});
    }
    cost[gi] = kLatency + bytes / (kBandwidth / kWorkers);
    sig[gi] = items[groups[gi].y - 1].sig_idx;
    if (sig[gi] >= 0) total[sig[gi]]++;
    std::sort(waits[gi].begin(), waits[gi].end());
    waits[gi].erase(std::unique(waits[gi].begin(), waits[gi].end()), waits[gi].end());
    for (auto& w : waits[gi]) waiters[w.first].push_back(gi);
  }
  // upward rank: emission order is topological, so one reverse sweep suffices
  std::vector<double> rank(ng, 0.0), cmax(ncounters, 0.0);
  for (int gi = ng - 1; gi >= 0; --gi) {
    rank[gi] = cost[gi] + (sig[gi] >= 0 ? cmax[sig[gi]] : 0.0);
    for (auto& w : waits[gi]) cmax[w.first] = std::max(cmax[w.first], rank[gi]);
  }
  std::vector<int> pending(ng), done(ncounters, 0);
  using Ready = std::pair<double, int>;  // (rank, group)
  std::priority_queue<Ready> ready;
  for (int gi = 0; gi < ng; ++gi) {
    pending[gi] = (int)waits[gi].size();
    if (pending[gi] == 0) ready.push({rank[gi], gi});
  }
  using Run = std::pair<double, int>;  // (finish, group), earliest first
  std::priority_queue<Run, std::vector<Run>, std::greater<Run>> running;
  std::vector<int> order;
  order.reserve(ng);
  double t = 0.0;
  int free_workers = (int)kWorkers;
  while ((int)order.size() < ng) {
    while (free_workers > 0 && !ready.empty()) {
      const int gi = ready.top().second;
      ready.pop();
      order.push_back(gi);
      running.push({t + cost[gi], gi});
      --free_workers;
    }
    if (running.empty()) break;  // cannot happen for a dependency-ordered list
    const Run r = running.top();
    running.pop();
    t = r.first;
    ++free_workers;
    const int c = sig[r.second];
    if (c >= 0 && ++done[c] == total[c])
      for (int gw : waiters[c]) {
        // a group waits for the counter to reach its full count
        if (--pending[gw] == 0) ready.push({rank[gw], gw});
      }
  }
  if ((int)order.size() != ng) return;  // keep the emission order
  std::vector<int2> out(ng);
  for (int i = 0; i < ng; ++i) out[i] = groups[order[i]];
  groups.swap(out);
}

// Work items of one direction (0: product, 1: transposed product).
// Segments = (block, 128-row slice, 64-column chunk); groups = runs of
// segments with the same output rows claimed and accumulated together.
int build_items(gca_h2* h, int dir, cudaStream_t st) {
  const int nc = h->nc;
  const bool trans = dir == 1;
  std::vector<MvItem> items;
  std::vector<int2> groups, free_groups;
  std::vector<int2>* target = &groups;  // list the groups being emitted go to
  std::vector<int> cx(nc, 0), cy(nc, 0);  // contributions (groups) to x-hat_c, y-hat_c
  struct Blk {
    int kind;
    int64_t a_off;
    int m, k;
    int64_t x_row;
    int wait_idx, wait_cnt;
  };
  // one group per slice of rows [a0, a0 + 128) over a list of blocks sharing output rows
  auto emit = [&](const std::vector<Blk>& blks, int in, int out, int64_t o_row0, int m, int sig_idx,
                  int* sig_cnt, int max_segs) {
    for (int a0 = 0; a0 < m; a0 += kItemRows) {
      int start = (int)items.size();
      int segs = 0;
      auto close = [&]() {
        if ((int)items.size() == start) return;
        items.back().flush = 1;
        items.back().sig_idx = sig_idx;
        target->push_back(make_int2(start, (int)items.size()));
        if (sig_cnt) ++*sig_cnt;
        start = (int)items.size();
        segs = 0;
      };
      for (const Blk& b : blks)
        for (int k0 = 0; k0 < b.k; k0 += kChunk) {
          if (segs == max_segs) close();
          MvItem it{};
          // the tile (a0, k0) of the block (tiled panel layout, panel.cuh)
          it.a_off = b.a_off + (int64_t)a0 * pad8(b.k) + (int64_t)std::min(kItemRows, m - a0) * k0;
          it.x_row = b.x_row + k0;
          it.o_row = o_row0 + a0;
          it.m = m;
          it.k = std::min(kChunk, b.k - k0);
          it.a0 = a0;
          it.k0 = k0;
          it.kind = b.kind | (in << 4) | (out << 8);
          it.wait_idx = b.wait_cnt > 0 ? b.wait_idx : -1;
          it.wait_cnt = b.wait_cnt;
          it.sig_idx = -1;
          it.flush = 0;
          items.push_back(it);
          ++segs;
        }
      close();
    }
  };
  const auto& O = h->panel_off;
  const int kCoupleSegs = 4, kNearSegs = 8;
  // forward transform: leaves
  for (int c : h->leaves)
    if (c > 0 && h->rank[c] > 0)
      emit({{kVt, O[kVt][c], h->rank[c], h->end[c] - h->begin[c], h->begin[c], -1, 0}}, kInX, kOutXh,
           h->xoff[c], h->rank[c], c, &cx[c], 1);
  // forward transform: up the tree, deepest level first (one segment per group:
  // the chain is latency bound, so its work is spread over many CTAs)
  for (int L = h->depth - 1; L >= 1; --L)
    for (int p : h->by_level[L]) {
      if (h->child0[p] < 0) continue;
      for (int ch : {h->child0[p], h->child1[p]})
        emit({{kEt, O[kEt][ch], h->rank[p], h->rank[ch], h->xoff[ch], ch, cx[ch]}}, kInXh, kOutXh,
             h->xoff[p], h->rank[p], p, &cx[p], 1);
    }
  // coupling: per output cluster, its blocks (deepest input first) in groups
  // of a few segments; clusters deepest first, since their inputs are ready
  // first.  The near field has no dependencies and is placed after the
  // couplings of the two deepest levels, as work for the CTAs while the
  // forward transform climbs the tree.
  std::vector<std::vector<int>> far_by_own(nc);
  for (int b = 0; b < (int)h->far_t.size(); ++b)
    far_by_own[trans ? h->far_s[b] : h->far_t[b]].push_back(b);
  std::vector<int> owners;
  for (int c = 0; c < nc; ++c)
    if (!far_by_own[c].empty()) owners.push_back(c);
  std::stable_sort(owners.begin(), owners.end(), [&](int u, int v) { return h->level[u] > h->level[v]; });
  auto emit_couple = [&](int own) {
    auto& bl = far_by_own[own];
    std::stable_sort(bl.begin(), bl.end(), [&](int u, int v) {
      const int iu = trans ? h->far_t[u] : h->far_s[u], iv = trans ? h->far_t[v] : h->far_s[v];
      return h->level[iu] > h->level[iv];
    });
    std::vector<Blk> blks;
    for (int b : bl) {
      const int in = trans ? h->far_t[b] : h->far_s[b];
      blks.push_back({trans ? kSt : kS, O[trans ? kSt : kS][b], h->rank[own], h->rank[in], h->xoff[in], in,
                      cx[in]});
    }
    emit(blks, kInXh, kOutYh, h->xoff[own], h->rank[own], nc + own, &cy[own], kCoupleSegs);
  };
  size_t oi = 0;
  for (; oi < owners.size() && h->level[owners[oi]] >= h->depth - 1; ++oi) emit_couple(owners[oi]);
  {
    // the near field waits for nothing: its own list, which warps work on
    // while their chain groups wait for inputs
    target = &free_groups;
    std::vector<std::vector<int>> by_own(nc);
    for (int b = 0; b < (int)h->near_t.size(); ++b) by_own[trans ? h->near_s[b] : h->near_t[b]].push_back(b);
    for (int own = 0; own < nc; ++own) {
      if (by_own[own].empty()) continue;
      std::vector<Blk> blks;
      for (int b : by_own[own]) {
        const int in = trans ? h->near_t[b] : h->near_s[b];
        blks.push_back({trans ? kNt : kN, O[trans ? kNt : kN][b], h->end[own] - h->begin[own],
                        h->end[in] - h->begin[in], h->begin[in], -1, 0});
      }
      emit(blks, kInX, kOutY, h->begin[own], h->end[own] - h->begin[own], -1, nullptr, kNearSegs);
    }
    target = &groups;
  }
  for (; oi < owners.size(); ++oi) emit_couple(owners[oi]);
  // backward transform, level by level down (y-hat of the parent must be final)
  for (int L = 2; L <= h->depth; ++L)
    for (int c : h->by_level[L]) {
      const int p = h->parent[c];
      if (cy[p] == 0 || h->rank[c] == 0) continue;  // y-hat_p = 0
      emit({{kE, O[kE][c], h->rank[c], h->rank[p], h->xoff[p], nc + p, cy[p]}}, kInYh, kOutYh,
           h->xoff[c], h->rank[c], nc + c, &cy[c], 1);
    }
  // leaf bases
  for (int c : h->leaves)
    if (c > 0 && h->rank[c] > 0 && cy[c] > 0)
      emit({{kV, O[kV][c], h->end[c] - h->begin[c], h->rank[c], h->xoff[c], nc + c, cy[c]}}, kInYh,
           kOutY, h->begin[c], h->end[c] - h->begin[c], -1, nullptr, 1);
  for (const int2& g : groups)
    if (g.y - g.x > kMaxGroupSegs) {
      set_error("internal: work group longer than the per-warp descriptor cache");
      return GCA_ERR_UNSUPPORTED;
    }
  for (const int2& g : free_groups)
    if (g.y - g.x > kMaxGroupSegs) {
      set_error("internal: work group longer than the per-warp descriptor cache");
      return GCA_ERR_UNSUPPORTED;
    }
  schedule_groups(items, groups, 2 * nc);
  h->n_items[dir] = (int64_t)groups.size();
  h->n_free[dir] = (int64_t)free_groups.size();
  groups.insert(groups.end(), free_groups.begin(), free_groups.end());
  GCA_TRY(upload(h->d_items[dir], items, st));
  GCA_TRY(upload(h->d_groups[dir], groups, st));
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

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }  // keeps every region aligned

// One persistent launch over `count` handles (slots).  Workspace layout:
// [claim counter, abort flag | per slot: x-hat, y-hat, y (cluster order),
// counters] zeroed by one memset, then per slot x (cluster order), then the
// slot descriptors.
template <typename T, typename TN, typename TA, typename TV, int RC>
int launch_rc(const gca_h2* const* hs, int count, int dir, const int32_t* nrhs, const void* const* x,
              const int64_t* ldx, void* const* y, const int64_t* ldy, DevMem& ws,
              std::vector<unsigned char>& ws_cache, int* status, cudaStream_t st) {
  const char* pn = sizeof(T) == 8 ? ".f64" : (sizeof(T) == 4 ? ".f32" : ".bf16");
  PhaseScope ps(std::string("mv_persistent") + pn + (dir ? ".T" : ""), st);
  ps.launches(4);
  std::vector<SlotArgs<TV>> sl(count);
  size_t off = 256;  // claim counter + abort flag
  std::vector<size_t> o_xh(count), o_yh(count), o_yp(count), o_cnt(count), o_xp(count);
  for (int i = 0; i < count; ++i) {
    const gca_h2* h = hs[i];
    const int R = nrhs[i];
    o_xh[i] = off;
    off += up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum, 1) * R);
    o_yh[i] = off;
    off += up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum, 1) * R);
    o_yp[i] = off;
    off += up256(sizeof(TV) * (size_t)h->n * R);
    o_cnt[i] = off;
    off += up256(sizeof(int) * 2 * (size_t)h->nc);
  }
  const size_t zeroed = off;
  for (int i = 0; i < count; ++i) {
    o_xp[i] = off;
    off += up256(sizeof(TV) * (size_t)hs[i]->n * nrhs[i]);
  }
  const size_t o_slots = off;
  off += up256(sizeof(SlotArgs<TV>) * count);
  if (off > ws.bytes) ws_cache.clear();
  GCA_TRY(ws.reserve(off));
  unsigned char* base = ws.as<unsigned char>();
  int64_t work = 0, free_work = 0;
  int max_n = 0;
  for (int i = 0; i < count; ++i) {
    const gca_h2* h = hs[i];
    SlotArgs<TV>& a = sl[i];
    const DevMem* P = sizeof(T) == 8 ? h->P64 : (sizeof(T) == 4 ? h->P32 : h->P16);
    const DevMem* PN = sizeof(TN) == 8 ? h->P64 : h->P32;
    for (int q = 0; q < kPanelKinds; ++q) a.A[q] = (q == kN || q == kNt) ? PN[q].p : P[q].p;
    a.items = h->d_items[dir].as<MvItem>();
    a.groups = h->d_groups[dir].as<int2>();
    a.free_groups = a.groups + h->n_items[dir];
    a.R = nrhs[i];
    a.nchunk = (a.R + RC - 1) / RC;
    a.n_work = h->n_items[dir] * a.nchunk;
    a.work_begin = work;
    work += a.n_work;
    a.n_free = h->n_free[dir] * a.nchunk;
    a.free_begin = free_work;
    free_work += a.n_free;
    a.n = h->n;
    a.x = static_cast<const TV*>(x[i]);
    a.ldx = ldx[i];
    a.y = static_cast<TV*>(y[i]);
    a.ldy = ldy[i];
    a.perm = h->d_perm.as<int>();
    a.xh = reinterpret_cast<TV*>(base + o_xh[i]);
    a.yh = reinterpret_cast<TV*>(base + o_yh[i]);
    a.yp = reinterpret_cast<TV*>(base + o_yp[i]);
    a.counters = reinterpret_cast<int*>(base + o_cnt[i]);
    a.xp = reinterpret_cast<TV*>(base + o_xp[i]);
    max_n = std::max(max_n, h->n * a.R);
  }
  LaunchArgs L;
  L.slots = base + o_slots;
  L.nslots = count;
  L.total = work;
  L.total_free = free_work;
  L.next = reinterpret_cast<unsigned long long*>(base);
  L.next_free = reinterpret_cast<unsigned long long*>(base + 8);
  L.abort_flag = reinterpret_cast<int*>(base + 16);
  L.status = status;
  // the descriptors change only with the arguments: upload when they differ
  // from what the workspace already holds
  const size_t sbytes = sizeof(SlotArgs<TV>) * count;
  if (ws_cache.size() != sbytes + sizeof(void*) ||
      std::memcmp(ws_cache.data(), sl.data(), sbytes) != 0 ||
      std::memcmp(ws_cache.data() + sbytes, &base, sizeof(void*)) != 0) {
    GCA_TRY_CUDA(cudaMemcpyAsync(base + o_slots, sl.data(), sbytes, cudaMemcpyHostToDevice, st));
    GCA_TRY_CUDA(cudaStreamSynchronize(st));  // sl is a stack vector
    ws_cache.assign(reinterpret_cast<const unsigned char*>(sl.data()),
                    reinterpret_cast<const unsigned char*>(sl.data()) + sbytes);
    ws_cache.insert(ws_cache.end(), reinterpret_cast<const unsigned char*>(&base),
                    reinterpret_cast<const unsigned char*>(&base) + sizeof(void*));
  }
  GCA_TRY_CUDA(cudaMemsetAsync(base, 0, zeroed, st));
  const auto* d_slots = reinterpret_cast<const SlotArgs<TV>*>(base + o_slots);
  const unsigned gx = (unsigned)std::min<int64_t>(1024, (max_n + 255) / 256);
  k_gather<TV><<<dim3(std::max(1u, gx), count), 256, 0, st>>>(d_slots);
  if (work + free_work > 0) {
    const size_t smem = cta_smem<TA, RC>();
    auto kern = k_h2_persistent<T, TN, TA, TV, RC>;
    // resident CTAs on the device, found once per device (later launches
    // make no attribute or occupancy calls, so they can be graph captured)
    static std::mutex mu;
    static int64_t cap_by_dev[64] = {};
    int dev = 0;
    GCA_TRY_CUDA(cudaGetDevice(&dev));
    int64_t cap = 0;
    {
      std::lock_guard<std::mutex> lk(mu);
      cap = dev >= 0 && dev < 64 ? cap_by_dev[dev] : 0;
    }
    if (cap == 0) {
      if (smem > 48 * 1024)
        GCA_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int sms = 0, per_sm = 0;
      GCA_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      GCA_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
      cap = (int64_t)sms * std::max(per_sm, 1);
      std::lock_guard<std::mutex> lk(mu);
      if (dev >= 0 && dev < 64) cap_by_dev[dev] = cap;
    }
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + free_work + kWarps - 1) / kWarps, cap));
    kern<<<grid, kThreads, smem, st>>>(L);
  }
  k_scatter<TV><<<dim3(std::max(1u, gx), count), 256, 0, st>>>(d_slots);
  GCA_TRY_CUDA(cudaGetLastError());
  return GCA_OK;
}

template <typename T, typename TN, typename TA, typename TV>
int launch(const gca_h2* const* hs, int count, int dir, const int32_t* nrhs, const void* const* x,
           const int64_t* ldx, void* const* y, const int64_t* ldy, DevMem& ws,
           std::vector<unsigned char>& wc, int* status, cudaStream_t st) {
  int R = 1;
  for (int i = 0; i < count; ++i) R = std::max(R, (int)nrhs[i]);
  if (R >= 16) return launch_rc<T, TN, TA, TV, 16>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc, status, st);
  if (R > 4) return launch_rc<T, TN, TA, TV, 8>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc, status, st);
  if (R > 2) return launch_rc<T, TN, TA, TV, 4>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc, status, st);
  if (R > 1) return launch_rc<T, TN, TA, TV, 2>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc, status, st);
  return launch_rc<T, TN, TA, TV, 1>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc, status, st);
}

// the handle kept the panels of this precision (gca_params.flags)
bool has_precision(const gca_h2* h, gca_prec prec) {
  const uint32_t fl = h->params.flags;
  switch (prec) {
    case GCA_F64: return !(fl & GCA_DROP_F64);
    case GCA_F32: return !(fl & GCA_DROP_F32);
    case GCA_BF16: return !(fl & GCA_DROP_BF16);
  }
  return false;
}

int launch_any(const gca_h2* const* hs, int count, gca_prec prec, bool trans, const int32_t* nrhs,
               const void* const* x, const int64_t* ldx, void* const* y, const int64_t* ldy, DevMem& ws,
               std::vector<unsigned char>& wc, int* status, cudaStream_t st) {
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !x[i] || !y[i] || nrhs[i] < 1 || nrhs[i] > 4096 || ldx[i] < hs[i]->n ||
        ldy[i] < hs[i]->n) {
      set_error("h2_matvec: invalid arguments (handle " + std::to_string(i) + ")");
      return GCA_ERR_INVALID_ARG;
    }
    if (!has_precision(hs[i], prec)) {
      set_error("h2_matvec: handle " + std::to_string(i) + " was built without this precision");
      return GCA_ERR_UNSUPPORTED;
    }
  }
  const int dir = trans ? 1 : 0;
  switch (prec) {
    case GCA_F64:
      return launch<double, double, double, double>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc, status, st);
    case GCA_F32:
      return launch<float, float, float, float>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc, status, st);
    case GCA_BF16:
      return launch<__nv_bfloat16, float, float, float>(hs, count, dir, nrhs, x, ldx, y, ldy, ws, wc,
                                                        status, st);
  }
  set_error("h2_matvec: unknown precision");
  return GCA_ERR_INVALID_ARG;
}

}  // namespace

int matvec(const gca_h2* h, gca_prec prec, bool trans, int32_t nrhs, const void* x, int64_t ldx,
           void* y, int64_t ldy, cudaStream_t st) {
  if (!h) {
    set_error("h2_matvec: NULL handle");
    return GCA_ERR_INVALID_ARG;
  }
  const gca_h2* hs[1] = {h};
  const void* xs[1] = {x};
  void* ys[1] = {y};
  return launch_any(hs, 1, prec, trans, &nrhs, xs, &ldx, ys, &ldy, h->w_ws, h->w_cache,
                    h->d_status.as<int>(), st);
}

int matvec_batch(const gca_h2_batch* b, gca_prec prec, bool trans, const int32_t* nrhs,
                 const void* const* x, const int64_t* ldx, void* const* y, const int64_t* ldy,
                 cudaStream_t st) {
  if (!b || b->h.empty() || !nrhs || !x || !ldx || !y || !ldy) {
    set_error("h2_matvec_batch: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  std::vector<const gca_h2*> hs(b->h.begin(), b->h.end());
  return launch_any(hs.data(), (int)hs.size(), prec, trans, nrhs, x, ldx, y, ldy, b->ws, b->w_cache,
                    b->d_status.as<int>(), st);
}

// ------------------------------------------------------- no-alloc product
//
// Some callers cannot allocate device memory while they run a product: code
// that executes inside a region where cudaMalloc is forbidden or would
// synchronise at the wrong moment (for instance between kernels of a
// latency-critical loop, or inside host callbacks), and programs that manage
// every byte of device memory themselves.  h2_matvec_noalloc serves them: it
// runs the same persistent product as h2_matvec, but its workspace (x-hat,
// y-hat, the cluster-order copies of x and y, the dependency counters and the
// slot descriptor) lives in the file-scope array below instead of memory the
// handle allocates.  Every GPU that loads this library holds the array until
// the process exits.  Only the array's device address, found once per device
// with cudaGetSymbolAddress, is ever handed to a kernel: in host code the name
// g_noalloc_scratch is just a host-side stand-in.

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// device address of the scratch array on the current device (looked up on the
// first call per device, with that device current)
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  GCA_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("h2_matvec_noalloc: device ordinal out of range");
    return GCA_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("h2_matvec_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return GCA_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return GCA_OK;
}

template <typename TV>
__global__ void k_put_slot(SlotArgs<TV> a, SlotArgs<TV>* dst) { *dst = a; }

// h2_matvec's launch for one handle with the workspace carved out of `base`
// (capacity `cap` bytes); nothing is allocated.
template <typename T, typename TN, typename TA, typename TV, int RC>
int launch_noalloc_rc(const gca_h2* h, int R, const void* x, int64_t ldx, void* y, int64_t ldy,
                      unsigned char* base, size_t cap, cudaStream_t st) {
  const size_t b_xh = up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum, 1) * R);
  const size_t b_yp = up256(sizeof(TV) * (size_t)h->n * R);
  const size_t b_cnt = up256(sizeof(int) * 2 * (size_t)h->nc);
  const size_t o_xh = 256, o_yh = o_xh + b_xh, o_yp = o_yh + b_xh, o_cnt = o_yp + b_yp;
  const size_t zeroed = o_cnt + b_cnt;
  const size_t o_xp = zeroed, o_slot = o_xp + b_yp;
  const size_t need = o_slot + up256(sizeof(SlotArgs<TV>));
  if (need > cap) {
    set_error("h2_matvec_noalloc: this product needs " + std::to_string(need) +
              " bytes of workspace, more than the " + std::to_string(cap) +
              "-byte scratch array (fewer right-hand sides or h2_matvec)");
    return GCA_ERR_UNSUPPORTED;
  }
  SlotArgs<TV> a{};
  const DevMem* P = sizeof(T) == 8 ? h->P64 : (sizeof(T) == 4 ? h->P32 : h->P16);
  const DevMem* PN = sizeof(TN) == 8 ? h->P64 : h->P32;
  for (int q = 0; q < kPanelKinds; ++q) a.A[q] = (q == kN || q == kNt) ? PN[q].p : P[q].p;
  a.items = h->d_items[0].as<MvItem>();
  a.groups = h->d_groups[0].as<int2>();
  a.free_groups = a.groups + h->n_items[0];
  a.R = R;
  a.nchunk = (R + RC - 1) / RC;
  a.n_work = h->n_items[0] * a.nchunk;
  a.work_begin = 0;
  a.n_free = h->n_free[0] * a.nchunk;
  a.free_begin = 0;
  a.n = h->n;
  a.x = static_cast<const TV*>(x);
  a.ldx = ldx;
  a.y = static_cast<TV*>(y);
  a.ldy = ldy;
  a.perm = h->d_perm.as<int>();
  a.xh = reinterpret_cast<TV*>(base + o_xh);
  a.yh = reinterpret_cast<TV*>(base + o_yh);
  a.yp = reinterpret_cast<TV*>(base + o_yp);
  a.counters = reinterpret_cast<int*>(base + o_cnt);
  a.xp = reinterpret_cast<TV*>(base + o_xp);
  LaunchArgs L;
  L.slots = base + o_slot;
  L.nslots = 1;
  L.total = a.n_work;
  L.total_free = a.n_free;
  L.next = reinterpret_cast<unsigned long long*>(base);
  L.next_free = reinterpret_cast<unsigned long long*>(base + 8);
  L.abort_flag = reinterpret_cast<int*>(base + 16);
  L.status = h->d_status.as<int>();
  // the array keeps the previous call's contents: the claim counter, abort
  // flag, x-hat, y-hat, y and the counters must start at zero
  GCA_TRY_CUDA(cudaMemsetAsync(base, 0, zeroed, st));
  // the descriptor travels as a kernel argument: no host buffer to keep alive
  auto* d_slots = reinterpret_cast<SlotArgs<TV>*>(base + o_slot);
  k_put_slot<TV><<<1, 1, 0, st>>>(a, d_slots);
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, ((int64_t)h->n * R + 255) / 256));
  k_gather<TV><<<dim3(gx, 1), 256, 0, st>>>(d_slots);
  if (a.n_work + a.n_free > 0) {
    const size_t smem = cta_smem<TA, RC>();
    auto kern = k_h2_persistent<T, TN, TA, TV, RC>;
    if (smem > 48 * 1024)
      GCA_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    GCA_TRY_CUDA(cudaGetDevice(&dev));
    GCA_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GCA_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    const int64_t capc = (int64_t)sms * std::max(per_sm, 1);
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.n_work + a.n_free + kWarps - 1) / kWarps, capc));
    kern<<<grid, kThreads, smem, st>>>(L);
  }
  k_scatter<TV><<<dim3(gx, 1), 256, 0, st>>>(d_slots);
  GCA_TRY_CUDA(cudaGetLastError());
  return GCA_OK;
}

template <typename T, typename TN, typename TA, typename TV>
int launch_noalloc(const gca_h2* h, int R, const void* x, int64_t ldx, void* y, int64_t ldy,
                   unsigned char* base, size_t cap, cudaStream_t st) {
  if (R >= 16) return launch_noalloc_rc<T, TN, TA, TV, 16>(h, R, x, ldx, y, ldy, base, cap, st);
  if (R > 4) return launch_noalloc_rc<T, TN, TA, TV, 8>(h, R, x, ldx, y, ldy, base, cap, st);
  if (R > 2) return launch_noalloc_rc<T, TN, TA, TV, 4>(h, R, x, ldx, y, ldy, base, cap, st);
  if (R > 1) return launch_noalloc_rc<T, TN, TA, TV, 2>(h, R, x, ldx, y, ldy, base, cap, st);
  return launch_noalloc_rc<T, TN, TA, TV, 1>(h, R, x, ldx, y, ldy, base, cap, st);
}

}  // namespace

int matvec_noalloc(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx, void* y,
                   int64_t ldy, cudaStream_t st) {
  if (!h || !x || !y || nrhs < 1 || nrhs > 4096 || ldx < h->n || ldy < h->n) {
    set_error("h2_matvec_noalloc: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  if (!has_precision(h, prec)) {
    set_error("h2_matvec_noalloc: the handle was built without this precision");
    return GCA_ERR_UNSUPPORTED;
  }
  unsigned char* base = nullptr;
  GCA_TRY(noalloc_scratch(&base));
  switch (prec) {
    case GCA_F64:
      return launch_noalloc<double, double, double, double>(h, nrhs, x, ldx, y, ldy, base,
                                                            kNoAllocScratchBytes, st);
    case GCA_F32:
      return launch_noalloc<float, float, float, float>(h, nrhs, x, ldx, y, ldy, base,
                                                        kNoAllocScratchBytes, st);
    case GCA_BF16:
      return launch_noalloc<__nv_bfloat16, float, float, float>(h, nrhs, x, ldx, y, ldy, base,
                                                                kNoAllocScratchBytes, st);
  }
  set_error("h2_matvec_noalloc: unknown precision");
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
