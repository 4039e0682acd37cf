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
// (panel.cuh).  The recursion is cut into segments (one tile of a block:
// up to 64 output rows x 64 input rows) and segments sharing output rows
// into groups of at most 8, the unit a warp claims.  Two lists:
//
//   chain: leaf forward -> upward transfers -> couplings -> downward
//          transfers -> leaf bases, in a dependency order fixed by a list
//          scheduler on the host;
//   free:  the near field, which depends on nothing.
//
// One persistent kernel runs both lists; its warps work independently.  A
// group waits (bounded spin, acquire) until every vector it reads is
// complete, i.e. until a per-cluster counter has seen every group that adds
// to it; a warp whose chain group is not ready runs a free group meanwhile.
// Groups are claimed in list order and only wait for earlier groups, so the
// earliest unfinished group always has its inputs and the launch cannot
// deadlock however many warps are resident.  A wait that exceeds its bound
// sets a timeout bit in the handle's status word and the launch winds down
// (no hang).
//
// Per warp, everything that can be fetched ahead is: the next group's claim
// (an atomic issued when the current group starts) and its descriptors (one
// bulk copy into shared memory), the block tiles (a ring of bulk copies on
// mbarriers that runs across the segments of a group) and each segment's
// input vector block (two buffers, the next segment's block in flight while
// the current one is used).
//
// x is gathered into cluster order first and y scattered back to the
// caller's order last; x-hat, y-hat, y (cluster order) and the counters are
// zeroed by one memset per product.

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <cstdio>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <type_traits>

#include "internal.hpp"
#include "panel.cuh"

namespace gca {

namespace {

constexpr int kStatusTimeout = 1;
constexpr int kStatusBadPlan = 2;

// Work item of the host-side plan (one segment).
struct MvItem {
  int64_t a_off;  // element offset of the tile in its panel array
  int64_t x_row;  // first row of the input vector block
  int64_t o_row;  // output row of the tile's first row
  int m;          // rows of the stored block
  int k;          // columns of this tile (<= kChunk)
  int a0;         // first block row of the tile
  int k0;         // first block column of the tile
  int kind;       // panel kind | (input << 4) | (output << 8)
  int wait_idx;   // counter that must reach wait_cnt * nchunk first (-1: none)
  int wait_cnt;
  int sig_idx;    // counter bumped after the outputs are added (-1: none)
  int flush;      // last segment of its group: add the accumulated rows to the output
};

// Device descriptor of a segment: 32 bytes, 8 per group record.
struct MvSeg {
  uint32_t a8;       // tile offset in units of 8 elements of its panel array
  int32_t x_row;     // first row of the input vector block
  int32_t o_row;     // output row of the tile's first row
  uint32_t rk;       // tile rows | columns << 16
  uint32_t flags;    // panel kind | input << 8 | output << 16 | last << 24
  int32_t wait_idx;  // -1: none
  int32_t wait_cnt;
  int32_t sig_idx;   // -1: none
};
static_assert(sizeof(MvSeg) == 32, "segment descriptor must be 32 bytes");

constexpr int kMaxGroupSegs = 8;                            // segments of a group
constexpr int kRecordBytes = kMaxGroupSegs * (int)sizeof(MvSeg);  // one group record

enum { kInXh = 0, kInYh = 1, kInX = 2 };
enum { kOutXh = 0, kOutYh = 1, kOutY = 2 };

// Everything one mesh (slot) of a launch needs.
template <typename TV>
struct SlotArgs {
  const void* A[kPanelKinds];  // panel arrays (near-field kinds hold the near storage type)
  const MvSeg* segs;           // group records: chain groups, then free groups
  int64_t n_chain;             // chain groups
  int64_t n_free;              // free groups
  int nchunk;                  // right-hand-side chunks of RC columns
  int R;
  int n;
  int rc;                      // RC: columns of a chunk
  int rs_in;                   // rows of x-hat (the input side's bases)
  int rs_out;                  // rows of y-hat (the output side's bases)
  const TV* x;                 // caller's x, original order, column-major
  int64_t ldx;
  TV* y;                       // caller's y, original order, column-major
  int64_t ldy;
  const int* perm;
  const int* iperm;            // inverse of perm
  // the vectors of the recursion, chunk-major: column c of row i at
  // ((c / RC) * rows + i) * RC + c % RC, so that the rows of one chunk are
  // contiguous (one bulk copy per input block, whatever R)
  const TV* xp;                // x in cluster order [nchunk][n][RC]
  TV* yp;                      // y in cluster order [nchunk][n][RC] (zeroed)
  TV* xh;                      // [nchunk][rs_in][RC]
  TV* yh;
  int* counters;               // [2 nc]
};

// The slot descriptors of a launch over at most kInlineSlots meshes travel
// as a kernel parameter (nothing to upload); larger launches read a device
// copy.
constexpr int kInlineSlots = 8;
template <typename TV>
struct SlotPack {
  SlotArgs<TV> s[kInlineSlots];
};

struct LaunchArgs {
  const void* slots;           // SlotArgs<TV>[nslots] in device memory (nslots > kInlineSlots)
  int nslots;
  const int2* chain_map;       // claim -> (slot, claim within the slot); null: one slot
  const int2* free_map;
  int map_rep;                 // > 1: the maps hold one entry per group, and claim c is
                               // chunk c % map_rep of entry c / map_rep (every slot has
                               // map_rep chunks)
  int64_t total;               // chain claims over all slots
  int64_t total_free;          // free claims over all slots
  unsigned long long* next;    // chain claim counter
  unsigned long long* next_free;  // free claim counter
  int* status;
  int* abort_flag;             // raised by any timed-out wait; every wait gives up
  const void* zeros;           // kZeroBytes of zeros (pads input blocks)
  long long wait_cycles;       // bound of every wait, SM clock cycles
  int wait_extra;              // added to every dependency count (0; 1 only in failure-path tests)
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------- pipeline
//
// A CTA holds kPairs pairs of warps.  In each pair a consumer warp only
// computes: it waits on mbarriers for the group its producer hands it, for
// each segment's input vector block and for each ring stage of block panels,
// multiplies, and adds its results to the output.  The producer warp does
// everything that waits on memory: it claims groups (one ahead), copies
// their descriptor records, waits for the counters of chain inputs, and
// issues the bulk copies (TMA, 1-D) of the panels and input blocks into the
// consumer's buffers, running ahead of the consumer by the ring's depth.
constexpr int kPairs = 4;                                   // producer/consumer pairs per CTA
// register split between the warpgroups (float products, two CTAs per SM):
// launched with kLaunchRegs a thread, producers give up what consumers take
constexpr int kLaunchRegs = 128, kProducerRegs = 80, kConsumerRegs = 176;
static_assert(kProducerRegs + kConsumerRegs == 2 * kLaunchRegs, "register split must balance");
template <typename TA>
constexpr bool kSplitRegs = sizeof(TA) == 4;
constexpr int kThreads = 64 * kPairs;                       // consumers: warps 0..3, producers: 4..7
constexpr int kItemRows = 64;                               // rows per segment (one warp tile)
constexpr int kChunk = 64;                                  // columns per segment
constexpr int kStagePanels = 8;
constexpr int kStageBytes = kStagePanels * kItemRows * 16;  // 8 KB: one contiguous copy
// ring stages of a pair: two at wide tiles (shared memory for two CTAs per
// SM), three for the float-staged products at up to 4 right-hand sides per
// tile, whose input blocks are small (more bytes in flight per pair where
// each stage's compute is short)
template <typename TA, int RC>
constexpr int kStagesOf = (RC <= 4 && sizeof(TA) <= 4) ? 3 : 2;
constexpr int kDescSlots = 4;                               // records: chain 0, 1; free 2, 3
constexpr size_t kZeroBytes = (size_t)kChunk * 16 * 8;      // a full input block of doubles
// a waiting warp sleeps until the phase completes or this many ns pass
constexpr unsigned kSuspendNs = 20000;

// Shared memory of one pair: ring, two input blocks, four descriptor
// records, the two-entry group queue, mbarriers.
template <typename TA, int RC>
struct PairSmem {
  static constexpr size_t kXSlot = sizeof(TA) * (size_t)kChunk * RC;
  static constexpr size_t kRing = 0;
  static constexpr int kStages = kStagesOf<TA, RC>;
  static constexpr size_t kX = (size_t)kStages * kStageBytes;
  static constexpr size_t kDesc = kX + 2 * kXSlot;
  static constexpr size_t kQueue = kDesc + (size_t)kDescSlots * kRecordBytes;
  static constexpr size_t kBar = kQueue + 2 * sizeof(int4);
  // full/empty per stage, xfull/xempty per block, ufull/uempty per queue
  // entry, dland/dfree per record
  static constexpr int kBars = 2 * kStages + 4 + 4 + 2 * kDescSlots;
  static constexpr size_t kBytes = (kBar + 8 * kBars + 127) / 128 * 128;
};
template <typename TA, int RC>
__host__ __device__ constexpr size_t cta_smem() {
  return kPairs * PairSmem<TA, RC>::kBytes;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, unsigned tx) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(b)),
               "r"(tx)
               : "memory");
}
// potentially blocking test: the warp is suspended until the phase
// completes or kSuspendNs pass, so waiting warps take no issue slots from
// the computing ones
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// non-blocking: has the phase of parity `parity` completed?
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of parity `parity`; false on timeout or abort.
// Between polls the warp sleeps (doubling up to kMaxSleep ns), so that a
// waiting warp takes almost no issue slots from the computing warps of its
// SM sub-partition; the abort flag and the deadline are checked every 16th
// poll.
template <unsigned kMaxSleep = 128>
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag,
                                          int* status, long long wait_cycles) {
  if (mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  unsigned ns = 16;
  for (unsigned it = 1;; ++it) {
    __nanosleep(ns);
    ns = ns < kMaxSleep ? 2 * ns : kMaxSleep;
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 15) == 0) {
      if (*abort_flag) return false;
      if (clock64() - t0 > wait_cycles) break;
    }
  }
  atomicOr(status, kStatusTimeout);
  *abort_flag = 1;
  return false;
}
// Bounded wait used only while draining copies before exit (ignores the
// abort flag, so that no copy is still landing when the warp retires).
__device__ __forceinline__ void mbar_drain(uint64_t* b, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity)) {
    __nanosleep(256);
    if (clock64() - t0 > kDefaultWaitCycles) return;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// orders global-memory writes seen through an acquire before later bulk
// copies (async proxy) that read them
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// claim counter increment whose result is read later (the warp runs on
// until the value is used)
__device__ __forceinline__ unsigned long long atom_add_u64(unsigned long long* p) {
  unsigned long long v;
  asm volatile("atom.relaxed.gpu.global.add.u64 %0, [%1], 1;" : "=l"(v) : "l"(p) : "memory");
  return v;
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
// counter increment with release semantics at GPU scope: writes that happen
// before it (this thread's, and other lanes' ordered by a warp barrier) are
// visible to a thread that reads the new value with an acquire
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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
// (blockIdx.y = slot).  The caller's x is read in its own order (coalesced,
// 16 bytes a thread where the columns allow it: x may be page-locked host
// memory read over the bus, where fewer, wider requests matter) and written
// to its cluster-order position.
template <typename TV>
__global__ void k_gather(const SlotArgs<TV>* __restrict__ dslots, const __grid_constant__ SlotPack<TV> pack,
                         int inline_slots) {
  const SlotArgs<TV>& sa = inline_slots ? pack.s[blockIdx.y] : dslots[blockIdx.y];
  constexpr int V = 16 / (int)sizeof(TV);
  TV* xp = const_cast<TV*>(sa.xp);
  if (sa.n % V == 0 && sa.ldx % V == 0 && (reinterpret_cast<uintptr_t>(sa.x) & 15) == 0) {
    const int nv = sa.n / V;
    const int64_t tot = (int64_t)nv * sa.R;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
      const int c = (int)(idx / nv), j = (int)(idx % nv) * V;
      const uint4 u = *reinterpret_cast<const uint4*>(sa.x + j + (int64_t)c * sa.ldx);
      TV v[V];
      memcpy(v, &u, 16);
#pragma unroll
      for (int e = 0; e < V; ++e) xp[((int64_t)(c / sa.rc) * sa.n + sa.iperm[j + e]) * sa.rc + c % sa.rc] = v[e];
    }
    return;
  }
  const int64_t tot = (int64_t)sa.n * sa.R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / sa.n), j = (int)(idx % sa.n);
    xp[((int64_t)(c / sa.rc) * sa.n + sa.iperm[j]) * sa.rc + c % sa.rc] = sa.x[j + c * sa.ldx];
  }
}

// y in cluster order -> caller's y (original order), written in the
// caller's order (coalesced, 16 bytes a thread where the columns allow it,
// also into page-locked host memory)
template <typename TV>
__global__ void k_scatter(const SlotArgs<TV>* __restrict__ dslots, const __grid_constant__ SlotPack<TV> pack,
                          int inline_slots) {
  const SlotArgs<TV>& sa = inline_slots ? pack.s[blockIdx.y] : dslots[blockIdx.y];
  constexpr int V = 16 / (int)sizeof(TV);
  if (sa.n % V == 0 && sa.ldy % V == 0 && (reinterpret_cast<uintptr_t>(sa.y) & 15) == 0) {
    const int nv = sa.n / V;
    const int64_t tot = (int64_t)nv * sa.R;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
      const int c = (int)(idx / nv), j = (int)(idx % nv) * V;
      TV v[V];
#pragma unroll
      for (int e = 0; e < V; ++e) v[e] = sa.yp[((int64_t)(c / sa.rc) * sa.n + sa.iperm[j + e]) * sa.rc + c % sa.rc];
      uint4 u;
      memcpy(&u, v, 16);
      *reinterpret_cast<uint4*>(sa.y + j + (int64_t)c * sa.ldy) = u;
    }
    return;
  }
  const int64_t tot = (int64_t)sa.n * sa.R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / sa.n), j = (int)(idx % sa.n);
    sa.y[j + c * sa.ldy] = sa.yp[((int64_t)(c / sa.rc) * sa.n + sa.iperm[j]) * sa.rc + c % sa.rc];
  }
}

// Register tile of a consumer: 64 rows x RC right-hand sides.  CPL =
// min(RC, 8) columns per lane, NCG = RC / CPL column groups, RG = 32 / NCG
// row groups, RPL = 64 / RG rows per lane; lane (rg, cg) owns rows
// rg + RG * i (i < RPL) and columns cg * CPL + [0, CPL).  Rows of one load
// instruction are consecutive (conflict-free 16-byte shared loads).
template <int RC>
struct Tile {
  static constexpr int CPL = RC < 8 ? RC : 8;
  static constexpr int NCG = RC / CPL;
  static constexpr int RG = 32 / NCG;
  static constexpr int RPL = 64 / RG;
};

// 16-byte load from a shared-memory address (an explicit shared-space load:
// the buffers reach the inner loop through a struct, and a generic load
// would go through the address-space check of the load/store unit).  The
// memory clobber keeps it after the mbarrier wait that makes the data valid.
__device__ __forceinline__ uint4 lds128(unsigned addr) {
  uint4 u;
  asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(u.x), "=r"(u.y), "=r"(u.z), "=r"(u.w) : "r"(addr)
      : "memory");
  return u;
}

// CPL consecutive values of a staged input row: 16-byte shared loads where
// the row segment is 16-byte aligned (CPL * sizeof(TA) a multiple of 16;
// every buffer and row start is)
template <typename TA, int CPL>
__device__ __forceinline__ void load_row(const TA* __restrict__ p, TA (&x)[CPL]) {
  if constexpr ((CPL * sizeof(TA)) % 16 == 0) {
    constexpr int V = 16 / (int)sizeof(TA);
    const unsigned a = smem_u32(p);
#pragma unroll
    for (int c = 0; c < CPL; c += V) {
      const uint4 u = lds128(a + c * (unsigned)sizeof(TA));
      if constexpr (sizeof(TA) == 4) {
        x[c] = __uint_as_float(u.x);
        x[c + 1] = __uint_as_float(u.y);
        x[c + 2] = __uint_as_float(u.z);
        x[c + 3] = __uint_as_float(u.w);
      } else {
        x[c] = __hiloint2double((int)u.y, (int)u.x);
        x[c + 1] = __hiloint2double((int)u.w, (int)u.z);
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < CPL; ++c) x[c] = p[c];
  }
}

// One panel (P columns) of the lane's rows in the first NI row groups times
// the staged input rows.  In float the products run as packed pairs
// (fma.rn.f32x2: two adjacent right-hand sides of a row per instruction,
// each rounded as a scalar fma), which halves the FMA instructions of the
// issue-bound inner loop.
template <typename T, typename TA, int RC, int NI>
__device__ __forceinline__ void panel_fma(const unsigned char* panel, const TA* __restrict__ xr, int rg, int cg,
                                          TA (&part)[Tile<RC>::RPL][Tile<RC>::CPL]) {
  using Tl = Tile<RC>;
  constexpr int P = Panel<T>::P;
  TA v[NI][P];
  const unsigned pa = smem_u32(panel) + rg * 16;
#pragma unroll
  for (int i = 0; i < NI; ++i) unpack(lds128(pa + Tl::RG * i * 16), v[i]);
#pragma unroll
  for (int kk = 0; kk < P; ++kk) {
    TA x[Tl::CPL];
    load_row<TA, Tl::CPL>(xr + kk * RC + cg * Tl::CPL, x);
    if constexpr (std::is_same<TA, float>::value && Tl::CPL % 2 == 0) {
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const float2 vv = make_float2(v[i][kk], v[i][kk]);
#pragma unroll
        for (int c = 0; c < Tl::CPL; c += 2) {
          const float2 p = __ffma2_rn(vv, make_float2(x[c], x[c + 1]), make_float2(part[i][c], part[i][c + 1]));
          part[i][c] = p.x;
          part[i][c + 1] = p.y;
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int c = 0; c < Tl::CPL; ++c) part[i][c] = fma(v[i][kk], x[c], part[i][c]);
    }
  }
}

// One ring stage: npst panels (`pst` bytes apart) of the lane's rows in the
// first NI row groups (the groups beyond the tile's rows are skipped: the
// condition is the same for every lane).  The stage's sum (at most
// kStagePanels * P terms) is formed on its own and then added: two-level
// summation keeps the rounding error of the long sums over a group's
// segments near that of a few short chains.
template <typename T, typename TA, int RC, int NI>
__device__ __forceinline__ void consume_rows(const unsigned char* stage, int pst, int npst, int p0,
                                             const TA* __restrict__ Xs, int rg, int cg,
                                             TA (&acc)[Tile<RC>::RPL][Tile<RC>::CPL]) {
  using Tl = Tile<RC>;
  constexpr int P = Panel<T>::P;
  TA part[Tl::RPL][Tl::CPL];
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int c = 0; c < Tl::CPL; ++c) part[i][c] = (TA)0;
#pragma unroll 1
  for (int g = 0; g < npst; ++g) panel_fma<T, TA, RC, NI>(stage + g * pst, Xs + (p0 + g) * P * RC, rg, cg, part);
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int c = 0; c < Tl::CPL; ++c) acc[i][c] += part[i][c];
}

template <typename T, typename TA, int RC, bool kSkipRows = true>
__device__ __forceinline__ void consume_stage(const unsigned char* stage, int rows, int npst, int p0,
                                              const TA* __restrict__ Xs, int rg, int cg,
                                              TA (&acc)[Tile<RC>::RPL][Tile<RC>::CPL]) {
  using Tl = Tile<RC>;
  const int pst = rows * 16;
  const int ni = (rows + Tl::RG - 1) / Tl::RG;  // row groups holding rows of the tile
  if constexpr (!kSkipRows) {
    consume_rows<T, TA, RC, Tl::RPL>(stage, pst, npst, p0, Xs, rg, cg, acc);
  } else if constexpr (Tl::RPL == 4) {
    if (ni >= 4)
      consume_rows<T, TA, RC, 4>(stage, pst, npst, p0, Xs, rg, cg, acc);
    else if (ni == 3)
      consume_rows<T, TA, RC, 3>(stage, pst, npst, p0, Xs, rg, cg, acc);
    else if (ni == 2)
      consume_rows<T, TA, RC, 2>(stage, pst, npst, p0, Xs, rg, cg, acc);
    else
      consume_rows<T, TA, RC, 1>(stage, pst, npst, p0, Xs, rg, cg, acc);
  } else {
    static_assert(Tl::RPL == 2, "row groups per lane");
    if (ni >= 2)
      consume_rows<T, TA, RC, 2>(stage, pst, npst, p0, Xs, rg, cg, acc);
    else
      consume_rows<T, TA, RC, 1>(stage, pst, npst, p0, Xs, rg, cg, acc);
  }
}

// ------------------------------------------- bfloat16 blocks on tensor cores
//
// In the bfloat16 product the stored V, E and S panels are bfloat16 and the
// products run on the tensor cores (mma.sync m16n8k16, bfloat16 operands,
// float accumulation).  The panel layout already is the operand layout of
// ldmatrix: a panel row is one 16-byte row of an 8 x 8 matrix, two
// consecutive panels are the two k halves of a 16 x 16 A fragment.  The
// staged float input rows are split into bfloat16 hi + lo parts (x = hi + lo
// to 16 bits), so that the input is not rounded to 8 bits; each k step is
// two products.  Warp tile: 64 rows (four m16 tiles) x RC columns (RC / 8
// n8 tiles); lane (g, t) = (lane / 4, lane % 4) holds rows g, g + 8 and
// columns 2t, 2t + 1 of each m16 x n8 accumulator.
template <typename T, int RC>
constexpr bool kTensorCore = std::is_same<T, __nv_bfloat16>::value && (RC == 8 || RC == 16);

__device__ __forceinline__ void ldmatrix_x4(unsigned addr, unsigned (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// two floats as bfloat16 (round to nearest), the first in the low half
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  unsigned r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// x = hi + lo with hi, lo bfloat16 pairs
__device__ __forceinline__ void split_bf16(float x0, float x1, unsigned& hi, unsigned& lo) {
  hi = pack_bf16(x0, x1);
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
  lo = pack_bf16(x0 - h0, x1 - h1);
}

// One ring stage of bfloat16 panels (npst of them, `rows` rows each) on the
// tensor cores.  p0: the stage's first panel within the segment.
template <int RC>
__device__ __forceinline__ void mma_stage(const unsigned char* stage, int rows, int npst, int p0,
                                          const float* __restrict__ Xs, int lane, float (&accm)[4][RC / 8][4]) {
  constexpr int NT = RC / 8;
  const int g = lane >> 2, t = lane & 3;
  const int q = lane >> 3, r8 = lane & 7;
  const int pst = rows * 16;
  const int mtiles = (rows + 15) >> 4;
  const unsigned sbase = smem_u32(stage);
  for (int pp = 0; pp < npst; pp += 2) {
    const bool two = pp + 1 < npst;  // a last single panel is the lower k half only
    const int kb = (p0 + pp) * 8;    // first input row of the k step
    unsigned bh[NT][2], bl[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const float* xc = Xs + (kb + 2 * t) * RC + 8 * nt + g;
      split_bf16(xc[0], xc[RC], bh[nt][0], bl[nt][0]);
      split_bf16(xc[8 * RC], xc[9 * RC], bh[nt][1], bl[nt][1]);
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      if (mt >= mtiles) break;
      unsigned a[4];
      const int row = 16 * mt + r8 + 8 * (q & 1);
      const int panel = pp + (two ? (q >> 1) : 0);
      ldmatrix_x4(sbase + panel * pst + row * 16, a);
      if (!two) a[2] = a[3] = 0u;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        mma_bf16(accm[mt][nt], a, bh[nt][0], bh[nt][1]);
        mma_bf16(accm[mt][nt], a, bl[nt][0], bl[nt][1]);
      }
    }
  }
}

__device__ __forceinline__ void red_add2(float* p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// Shared-memory regions and mbarriers of one pair.
template <typename TA, int RC>
struct Pair {
  static constexpr int kStages = kStagesOf<TA, RC>;
  unsigned char* ring;
  TA* xb;
  MvSeg* rec;
  int4* queue;  // {slot (-1: no more groups), first right-hand side, record, 0}
  uint64_t* bar;
  __device__ uint64_t* full(int s) const { return bar + s; }
  __device__ uint64_t* empty(int s) const { return bar + kStages + s; }
  __device__ uint64_t* xfull(int j) const { return bar + 2 * kStages + j; }
  __device__ uint64_t* xempty(int j) const { return bar + 2 * kStages + 2 + j; }
  __device__ uint64_t* ufull(int q) const { return bar + 2 * kStages + 4 + q; }
  __device__ uint64_t* uempty(int q) const { return bar + 2 * kStages + 6 + q; }
  __device__ uint64_t* dland(int d) const { return bar + 2 * kStages + 8 + d; }
  __device__ uint64_t* dfree(int d) const { return bar + 2 * kStages + 8 + kDescSlots + d; }
  __device__ TA* xslot(int j) const { return xb + (size_t)j * kChunk * RC; }
};

// A group held by a producer: its slot, the right-hand-side chunk and the
// descriptor record it was copied to.
struct Unit {
  int slot;    // -1: none
  int c0;      // first right-hand side
  int dslot;   // descriptor record of the pair
};

// The segments of a group: lane j < nseg holds the descriptor of segment j;
// `notready` marks segments whose input vector block is not complete yet,
// `haswait` those that depend on other groups.
struct Probe {
  MvSeg d;
  int nseg;
  unsigned notready;
  unsigned haswait;
};

__device__ __forceinline__ MvSeg read_seg(const MvSeg* rec, int lane) {
  MvSeg d{};
  if (lane < kMaxGroupSegs) {
    const uint4* q = reinterpret_cast<const uint4*>(rec + lane);
    const uint4 a = q[0], b = q[1];
    d.a8 = a.x;
    d.x_row = (int)a.y;
    d.o_row = (int)a.z;
    d.rk = a.w;
    d.flags = b.x;
    d.wait_idx = (int)b.y;
    d.wait_cnt = (int)b.z;
    d.sig_idx = (int)b.w;
  }
  return d;
}

__device__ __forceinline__ int count_segs(const MvSeg& d, int lane) {
  const unsigned lastmask = __ballot_sync(0xffffffffu, lane < kMaxGroupSegs && ((d.flags >> 24) & 1));
  return lastmask ? __ffs(lastmask) : 0;
}

template <typename T, typename TN, typename TV>
__device__ __forceinline__ void seg_geom(const SlotArgs<TV>& sa, uint32_t a8, uint32_t rk, uint32_t flags,
                                         const unsigned char*& A, int& rows, int& np) {
  const int ain = flags & 0xff;
  const bool is_near = ain == kN || ain == kNt;
  const int P = is_near ? Panel<TN>::P : Panel<T>::P;
  const int esz = is_near ? (int)sizeof(TN) : (int)sizeof(T);
  A = static_cast<const unsigned char*>(sa.A[ain]) + (int64_t)a8 * 8 * esz;
  rows = (int)(rk & 0xffff);
  np = pad8((int)(rk >> 16)) / P;
}

template <typename TV, int RC>
__device__ __forceinline__ bool bulk_inputs(const SlotArgs<TV>& sa) {
  return (RC * sizeof(TV)) % 16 == 0;
}

// ------------------------------------------------------------- producer
template <typename T, typename TN, typename TA, typename TV, int RC>
__device__ void producer_loop(const LaunchArgs& L, const SlotArgs<TV>* slots, const Pair<TA, RC>& P, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int kStages = kStagesOf<TA, RC>;
  volatile int* abort_flag = L.abort_flag;
  uint32_t fill = 0, xfill = 0, uhand = 0;
  uint32_t dland_par = 0, dland_pend = 0, dfree_par = 0, dused = 0;
  bool ok = true;
  // Counter signals.  A group that completes a vector bumps the vector's
  // counter once its consumer has added its rows to the output.  The
  // consumer reduces, passes a warp barrier and arrives on the group's queue
  // entry (uempty, a release at CTA scope); the producer observes that
  // arrival and increments the counter with a release reduction at GPU
  // scope, which is cumulative over the consumer's reductions.  The consumer
  // never waits for its reductions to be performed; the producer does, in
  // time it would otherwise spend waiting.
  uint32_t usig = 0;                             // handed groups whose signal is done
  int* sig_q0 = nullptr;                         // counter of the group in queue entry 0
  int* sig_q1 = nullptr;                         // ... entry 1
  auto sig_one = [&](bool block) -> bool {       // retire the oldest handed group
    if (usig == uhand) return false;
    const int q = (int)(usig & 1);
    const unsigned par = (usig >> 1) & 1;
    if (block) {
      if (!mbar_wait<512>(P.uempty(q), par, abort_flag, L.status, L.wait_cycles)) {
        ok = false;
        return false;
      }
    } else if (!mbar_test(P.uempty(q), par)) {
      return false;
    }
    int* c = q ? sig_q1 : sig_q0;
    if (c && lane == 0) red_release_add(c, 1);
    __syncwarp();
    ++usig;
    return true;
  };
  auto sig_poll = [&]() {
    while (sig_one(false)) {
    }
  };
  // bounded wait that keeps delivering counter signals meanwhile
  auto wait = [&](uint64_t* b, unsigned par) -> bool {
    if (mbar_try_wait(b, par)) return true;
    const long long t0 = clock64();
    unsigned ns = 16;
    for (unsigned it = 1;; ++it) {
      sig_poll();
      if (!ok) return false;
      __nanosleep(ns);
      ns = ns < 512 ? 2 * ns : 512;
      if (mbar_try_wait(b, par)) return true;
      if ((it & 15) == 0) {
        if (*abort_flag) return false;
        if (clock64() - t0 > L.wait_cycles) {
          atomicOr(L.status, kStatusTimeout);
          *abort_flag = 1;
          return false;
        }
      }
    }
  };

  // copy the record of claim c of a list into record d (after the consumer
  // has released d's previous record)
  auto fetch = [&](int64_t c, bool chain, int d) -> Unit {
    Unit u{-1, 0, d};
    if (c < 0 || !ok) return u;
    if ((dused >> d) & 1) {
      if (!wait(P.dfree(d), (dfree_par >> d) & 1)) {
        ok = false;
        return u;
      }
      dfree_par ^= 1u << d;
    }
    int s = 0;
    int64_t loc = c;
    const int2* map = chain ? L.chain_map : L.free_map;
    if (map) {
      const int rep = L.map_rep;
      const int2 m = map[rep > 1 ? c / rep : c];
      s = m.x;
      loc = rep > 1 ? (int64_t)m.y * rep + c % rep : m.y;
    }
    const SlotArgs<TV>& sa = slots[s];
    const int64_t g = loc / sa.nchunk + (chain ? 0 : sa.n_chain);
    u.slot = s;
    u.c0 = (int)(loc % sa.nchunk) * RC;
    if (lane == 0) {
      mbar_arrive_tx(P.dland(d), kRecordBytes);
      bulk_g2s(P.rec + d * kMaxGroupSegs, sa.segs + g * kMaxGroupSegs, kRecordBytes, P.dland(d));
    }
    dland_pend |= 1u << d;
    dused |= 1u << d;
    return u;
  };
  auto land = [&](int d) -> bool {
    if (!((dland_pend >> d) & 1)) return true;
    if (!wait(P.dland(d), (dland_par >> d) & 1)) return false;
    dland_par ^= 1u << d;
    dland_pend &= ~(1u << d);
    return true;
  };
  auto probe = [&](const SlotArgs<TV>& sa, int d, Probe& pr) -> bool {
    pr.d = read_seg(P.rec + d * kMaxGroupSegs, lane);
    pr.nseg = count_segs(pr.d, lane);
    const bool w = lane < pr.nseg && pr.d.wait_idx >= 0;
    bool nr = false;
    if (w) nr = ld_acquire(sa.counters + pr.d.wait_idx) < pr.d.wait_cnt * sa.nchunk + L.wait_extra;
    pr.notready = __ballot_sync(FULL, nr);
    pr.haswait = __ballot_sync(FULL, w);
    __syncwarp();
    return pr.nseg > 0;
  };
  auto claim_now = [&](unsigned long long* ctr, int64_t total) -> int64_t {
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1ull);
    v = __shfl_sync(FULL, v, 0);
    return (int64_t)v < total ? (int64_t)v : -1;
  };
  // hand group (slot, c0, record d) to the consumer; `sig`: the counter it
  // bumps when done (null: none)
  auto hand = [&](int slot, int c0, int d, int* sig) -> bool {
    const int q = (int)(uhand & 1);
    if (uhand >= 2 && !wait(P.uempty(q), ((uhand >> 1) - 1) & 1)) return false;
    // the group that used this entry is done: its signal goes out first
    while (usig + 2 <= uhand)
      if (!sig_one(true)) return false;
    if (q)
      sig_q1 = sig;
    else
      sig_q0 = sig;
    if (lane == 0) {
      P.queue[q] = make_int4(slot, c0, d, 0);
      mbar_arrive(P.ufull(q));
    }
    __syncwarp();
    ++uhand;
    return true;
  };

  Unit cu = fetch(claim_now(L.next, L.total), true, 0);
  Unit fu = fetch(claim_now(L.next_free, L.total_free), false, 2);
  while (ok) {
    Unit u;
    bool chain;
    Probe pr;
    if (cu.slot >= 0) {
      if (!(ok = land(cu.dslot))) break;
      if (!probe(slots[cu.slot], cu.dslot, pr)) {
        atomicOr(L.status, kStatusBadPlan);
        *abort_flag = 1;
        ok = false;
        break;
      }
      chain = !(pr.notready && fu.slot >= 0);
      if (!chain) {
        // the chain group waits for inputs: hand the held free group first
        if (!(ok = land(fu.dslot))) break;
        if (!probe(slots[fu.slot], fu.dslot, pr)) {
          atomicOr(L.status, kStatusBadPlan);
          *abort_flag = 1;
          ok = false;
          break;
        }
      }
      u = chain ? cu : fu;
    } else if (fu.slot >= 0) {
      if (!(ok = land(fu.dslot))) break;
      if (!probe(slots[fu.slot], fu.dslot, pr)) {
        atomicOr(L.status, kStatusBadPlan);
        *abort_flag = 1;
        ok = false;
        break;
      }
      chain = false;
      u = fu;
    } else {
      break;
    }
    const SlotArgs<TV>& sa = slots[u.slot];
    {
      const int sig = __shfl_sync(FULL, pr.d.sig_idx, pr.nseg - 1);
      if (!(ok = hand(u.slot, u.c0, u.dslot, sig >= 0 ? sa.counters + sig : nullptr))) break;
    }
    // claim the successor on the same list; its record is fetched once the
    // first data of this group is on its way
    unsigned long long* ctr = chain ? L.next : L.next_free;
    const int64_t total = chain ? L.total : L.total_free;
    unsigned long long token = 0;
    if (lane == 0) token = atom_add_u64(ctr);
    bool fetched = false;
    Unit next{-1, 0, u.dslot ^ 1};
    auto fetch_next = [&]() {
      if (fetched) return;
      fetched = true;
      const int64_t c = (int64_t)__shfl_sync(FULL, token, 0);
      next = fetch(c < total ? c : -1, chain, u.dslot ^ 1);
    };
    const bool bulk = bulk_inputs<TV, RC>(sa);
    const MvSeg& d = pr.d;
    for (int s = 0; s < pr.nseg && ok; ++s) {
      const uint32_t fl = __shfl_sync(FULL, d.flags, s);
      const uint32_t rk = __shfl_sync(FULL, d.rk, s);
      const unsigned char* A;
      int rows, np;
      seg_geom<T, TN, TV>(sa, __shfl_sync(FULL, d.a8, s), rk, fl, A, rows, np);
      int p0 = 0;  // panels of this segment issued so far
      auto issue_stage = [&]() {
        const int st = (int)(fill % kStages);
        if (lane == 0) {
          const int npst = min(kStagePanels, np - p0);
          const unsigned bytes = (unsigned)(npst * rows * 16);  // contiguous panels of the tile
          mbar_arrive_tx(P.full(st), bytes);
          bulk_g2s(P.ring + st * kStageBytes, A + (int64_t)p0 * rows * 16, bytes, P.full(st));
        }
        ++fill;
        p0 += kStagePanels;
      };
      auto stage_free_now = [&]() {
        return fill < (uint32_t)kStages ||
               mbar_test(P.empty((int)(fill % kStages)), ((fill / kStages) - 1) & 1);
      };
      if ((pr.notready >> s) & 1) {
        // the block's panels do not depend on the input: put what fits in
        // flight, then wait for the input vector block to be complete
        while (p0 < np && stage_free_now()) issue_stage();
        const int widx = __shfl_sync(FULL, d.wait_idx, s);
        const int need = __shfl_sync(FULL, d.wait_cnt, s) * sa.nchunk + L.wait_extra;
        bool timeout = false;
        {
          const long long t0 = clock64();
          unsigned ns = 32;
          for (unsigned spins = 1;; ++spins) {
            int v = 0;
            if (lane == 0) v = ld_acquire(sa.counters + widx);  // lane 0 issues the copy below
            if (__shfl_sync(FULL, v, 0) >= need) break;
            sig_poll();
            if (!ok) {
              timeout = true;
              break;
            }
            if ((spins & 7) == 0) {
              if (*abort_flag) {
                timeout = true;
                break;
              }
              if (clock64() - t0 > L.wait_cycles) {
                atomicOr(L.status, kStatusTimeout);
                *abort_flag = 1;
                timeout = true;
                break;
              }
            }
            __nanosleep(ns);
            ns = ns < 256 ? 2 * ns : 256;
          }
        }
        if (timeout) {
          ok = false;
          break;
        }
      }
      // the segment's input vector block
      {
        const int j = (int)(xfill & 1);
        if (xfill >= 2 && !wait(P.xempty(j), ((xfill >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        const int xin = (fl >> 8) & 0xff;
        const int k = (int)(rk >> 16);
        const int xrow = __shfl_sync(FULL, d.x_row, s);
        // rows [xrow, xrow + k) of chunk c0 / RC of the input vector
        const TV* X = (xin == kInXh ? sa.xh : (xin == kInYh ? sa.yh : sa.xp)) +
                      ((int64_t)(u.c0 / RC) * (xin == kInX ? sa.n : (xin == kInXh ? sa.rs_in : sa.rs_out)) +
                       xrow) * RC;
        // rows past the block's columns meet zero panel columns (and, on the
        // tensor cores, the zeroed upper half of a last single panel): they
        // are copied in as zeros, so the buffer only ever gets bulk copies
        const int ain = fl & 0xff;
        const int kz = (kTensorCore<T, RC> && ain != kN && ain != kNt) ? (k + 15) & ~15 : pad8(k);
        if (bulk) {
          if (lane == 0) {
            if ((pr.haswait >> s) & 1) fence_proxy_async_global();  // written by other warps
            const unsigned bytes = (unsigned)(k * RC * sizeof(TV));
            const unsigned zb = (unsigned)((kz - k) * RC * sizeof(TV));
            mbar_arrive_tx(P.xfull(j), bytes + zb);
            bulk_g2s(P.xslot(j), X, bytes, P.xfull(j));
            if (zb) bulk_g2s(P.xslot(j) + (size_t)k * RC, L.zeros, zb, P.xfull(j));
          }
        } else {
          TA* Xs = P.xslot(j);
          const int c0 = u.c0;
          const int kp = kz;
          for (int i = lane; i < kp * RC; i += 32) {
            const int r = i / RC, c = i % RC;
            Xs[i] = (r < k && c0 + c < sa.R) ? (TA)__ldcg(X + (int64_t)r * RC + c) : (TA)0;
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(P.xfull(j));
        }
        ++xfill;
      }
      // the rest of the segment's panels
      while (p0 < np) {
        if (fill >= (uint32_t)kStages &&
            !wait(P.empty((int)(fill % kStages)), ((fill / kStages) - 1) & 1)) {
          ok = false;
          break;
        }
        issue_stage();
        sig_poll();
        if (s == 0) fetch_next();
      }
      if (!ok) break;
    }
    fetch_next();
    if (chain)
      cu = next;
    else
      fu = next;
  }
  // the last signals, then: no more groups
  while (ok && usig < uhand)
    if (!sig_one(true)) break;
  if (ok) ok = hand(-1, 0, 0, nullptr);
  // drain: every issued copy has landed before the warp exits
  if (lane == 0) {
    for (uint32_t f = fill > (uint32_t)kStages ? fill - kStages : 0; f < fill; ++f)
      mbar_drain(P.full((int)(f % kStages)), (f / kStages) & 1);
    for (uint32_t f = xfill > 2u ? xfill - 2 : 0; f < xfill; ++f) mbar_drain(P.xfull((int)(f & 1)), (f >> 1) & 1);
    for (int dd = 0; dd < kDescSlots; ++dd)
      if ((dland_pend >> dd) & 1) mbar_drain(P.dland(dd), (dland_par >> dd) & 1);
  }
  __syncwarp();
}

// ------------------------------------------------------------- consumer
template <typename T, typename TN, typename TA, typename TV, int RC>
__device__ void consumer_loop(const LaunchArgs& L, const SlotArgs<TV>* slots, const Pair<TA, RC>& P, int lane) {
  constexpr int kStages = kStagesOf<TA, RC>;
  using Tl = Tile<RC>;
  constexpr unsigned FULL = 0xffffffffu;
  volatile int* abort_flag = L.abort_flag;
  const int rg = lane % Tl::RG, cg = lane / Tl::RG;
  uint32_t use = 0, xuse = 0, ucnt = 0;
  TA acc[Tl::RPL][Tl::CPL];
#pragma unroll
  for (int i = 0; i < Tl::RPL; ++i)
#pragma unroll
    for (int c = 0; c < Tl::CPL; ++c) acc[i][c] = (TA)0;
  constexpr bool kTC = kTensorCore<T, RC>;
  constexpr int NT = RC >= 8 ? RC / 8 : 1;
  float accm[4][NT][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) accm[i][nt][e] = 0.f;
  while (true) {
    const int q = (int)(ucnt & 1);
    if (!mbar_wait(P.ufull(q), (ucnt >> 1) & 1, abort_flag, L.status, L.wait_cycles)) return;
    const int4 msg = P.queue[q];
    ++ucnt;
    if (msg.x < 0) return;
    const SlotArgs<TV>& sa = slots[msg.x];
    const int c0 = msg.y;
    const MvSeg d = read_seg(P.rec + msg.z * kMaxGroupSegs, lane);
    const int nseg = count_segs(d, lane);
    __syncwarp();
    if (lane == 0) mbar_arrive(P.dfree(msg.z));  // the record may be reused
    const bool bulk = bulk_inputs<TV, RC>(sa);
    // bfloat16 far-field groups run on the tensor cores (all segments of a
    // group are of one kind)
    bool tc = false;
    if constexpr (kTC) {
      const int ain0 = __shfl_sync(FULL, d.flags, 0) & 0xff;
      tc = ain0 != kN && ain0 != kNt;
    }
    for (int s = 0; s < nseg; ++s) {
      const uint32_t fl = __shfl_sync(FULL, d.flags, s);
      const uint32_t rk = __shfl_sync(FULL, d.rk, s);
      const int rows = (int)(rk & 0xffff);
      const int k = (int)(rk >> 16);
      const int kp = pad8(k);
      const int ain = fl & 0xff;
      const bool is_near = ain == kN || ain == kNt;
      const int np = kp / (is_near ? Panel<TN>::P : Panel<T>::P);
      const int j = (int)(xuse & 1);
      if (!mbar_wait(P.xfull(j), (xuse >> 1) & 1, abort_flag, L.status, L.wait_cycles)) return;
      const TA* Xs = P.xslot(j);  // padded with zero rows by the producer
      for (int p0 = 0; p0 < np; p0 += kStagePanels) {
        const int st = (int)(use % kStages);
        if (!mbar_wait(P.full(st), (use / kStages) & 1, abort_flag, L.status, L.wait_cycles)) return;
        const unsigned char* stg = P.ring + st * kStageBytes;
        const int npst = min(kStagePanels, np - p0);
        if constexpr (sizeof(T) == sizeof(TN)) {
          consume_stage<T, TA, RC>(stg, rows, npst, p0, Xs, rg, cg, acc);
        } else if constexpr (kTC) {
          if (tc)
            mma_stage<RC>(stg, rows, npst, p0, reinterpret_cast<const float*>(Xs), lane, accm);
          else  // the near field: leaf rows, one variant (keeps the kernel's code small)
            consume_stage<TN, TA, RC, false>(stg, rows, npst, p0, Xs, rg, cg, acc);
        } else {
          if (is_near)
            consume_stage<TN, TA, RC>(stg, rows, npst, p0, Xs, rg, cg, acc);
          else
            consume_stage<T, TA, RC>(stg, rows, npst, p0, Xs, rg, cg, acc);
        }
        ++use;
        __syncwarp();  // every lane's reads of the stage have returned
        if (lane == 0) mbar_arrive(P.empty(st));
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(P.xempty(j));
      ++xuse;
      if (!((fl >> 24) & 1)) continue;
      // last segment: add the accumulated rows to the output
      const int out = (fl >> 16) & 0xff;
      TV* obase = out == kOutXh ? sa.xh : (out == kOutYh ? sa.yh : sa.yp);
      const int o_row = __shfl_sync(FULL, d.o_row, s);
      // rows of this chunk of the output (chunk-major, RC columns a row; the
      // columns past R are padding that nothing reads)
      TV* const ochunk =
          obase + (int64_t)(c0 / RC) * (out == kOutY ? sa.n : (out == kOutXh ? sa.rs_in : sa.rs_out)) * RC;
      if constexpr (kTC) {
        if (tc) {
          // accumulator fragments: rows 16 mt + g (+ 8), columns 8 nt + 2t (+ 1)
          const int g = lane >> 2, t = lane & 3;
#pragma unroll
          for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int r = 16 * mt + g + 8 * h;
                float* o = reinterpret_cast<float*>(ochunk) + ((int64_t)o_row + r) * RC + 8 * nt + 2 * t;
                if (r < rows) red_add2(o, accm[mt][nt][2 * h], accm[mt][nt][2 * h + 1]);
                accm[mt][nt][2 * h] = accm[mt][nt][2 * h + 1] = 0.f;
              }
            }
          continue;
        }
      }
      const int col0 = cg * Tl::CPL;
      const bool aligned = (Tl::CPL * sizeof(TV)) % 16 == 0;
#pragma unroll
      for (int i = 0; i < Tl::RPL; ++i) {
        const int r = rg + Tl::RG * i;
        if (r < rows) add_row<Tl::CPL>(ochunk + ((int64_t)o_row + r) * RC + col0, acc[i], Tl::CPL, aligned);
      }
#pragma unroll
      for (int i = 0; i < Tl::RPL; ++i)
#pragma unroll
        for (int c = 0; c < Tl::CPL; ++c) acc[i][c] = (TA)0;
    }
    // every lane's output reductions come before this arrival: the producer
    // signals the group's counter once it sees it
    __syncwarp();
    if (lane == 0) mbar_arrive(P.uempty(q));
  }
}

// Persistent product over all slots of a launch.  Two lists: the dependency
// chain (forward and backward transforms, couplings), claimed in a
// dependency order, and the free list (near field), which waits for
// nothing.  A producer holds at most one chain group and one free group; it
// hands its consumer the chain group when that is ready (or the free list is
// used up) and the free group otherwise, and claims the successor on the
// same list while it streams a group.
// (float: two CTAs per SM within 128 registers a thread; double: one CTA,
// whose buffers fill the shared memory and whose accumulators need more)
template <typename T, typename TN, typename TA, typename TV, int RC>
__global__ void __launch_bounds__(kThreads, sizeof(TA) == 8 ? 1 : 2)
    k_h2_persistent(const __grid_constant__ LaunchArgs L, const __grid_constant__ SlotPack<TV> pack) {
  using PS = PairSmem<TA, RC>;
  const SlotArgs<TV>* slots = L.slots ? static_cast<const SlotArgs<TV>*>(L.slots) : pack.s;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pair = warp % kPairs;
  unsigned char* base = smem_raw + pair * PS::kBytes;
  Pair<TA, RC> P;
  P.ring = base + PS::kRing;
  P.xb = reinterpret_cast<TA*>(base + PS::kX);
  P.rec = reinterpret_cast<MvSeg*>(base + PS::kDesc);
  P.queue = reinterpret_cast<int4*>(base + PS::kQueue);
  P.bar = reinterpret_cast<uint64_t*>(base + PS::kBar);
  if (warp < kPairs && lane == 0) {
    for (int i = 0; i < PS::kBars; ++i) mbar_init(P.bar + i, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if constexpr (kSplitRegs<TA>) {
    // the producers need few registers, the consumers' tiles many: move
    // registers from the producer warpgroup to the consumer warpgroup
    // (kProducerRegs + kConsumerRegs = 2 * kLaunchRegs, checked on the host
    // against the launch's register count)
    if (warp >= kPairs) {
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
      producer_loop<T, TN, TA, TV, RC>(L, slots, P, lane);
    } else {
      asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kConsumerRegs));
      consumer_loop<T, TN, TA, TV, RC>(L, slots, P, lane);
    }
  } else {
    if (warp >= kPairs)
      producer_loop<T, TN, TA, TV, RC>(L, slots, P, lane);
    else
      consumer_loop<T, TN, TA, TV, RC>(L, slots, P, lane);
  }
}

}  // namespace

// Claim order of the groups.  The emission order below is a valid
// dependency order but makes warps claim groups long before their inputs
// exist.  This list scheduler simulates the launch: kWorkers warps, a group
// costs a fixed latency (its record, its inputs' signal path and the copy
// latency; with the 2 us of a bare copy the simulated chain ran ahead of the
// real one, and warps claimed chain groups long before their inputs were
// complete) plus its bytes at a warp's share of HBM bandwidth, a
// group is ready once every counter it waits for has seen all of its
// contributions, and among ready groups the one with the longest remaining
// dependency path (upward rank) starts first.  Groups are then claimed in
// simulated start order, which is again a dependency order (a group starts
// only after everything it waits for has finished), so the launch stays
// deadlock free.  The simulated start times are returned in `start` (claim
// order) and the simulated end of the last group in `makespan`.
void schedule_groups(const std::vector<MvItem>& items, std::vector<int2>& groups, int ncounters,
                     std::vector<float>& start, float& makespan) {
  const int ng = (int)groups.size();
  start.assign(ng, 0.f);
  makespan = 0.f;
  if (ng < 1) return;
  constexpr double kWorkers = 148 * 8, kLatency = 10.0e-6, kBandwidth = 6.0e12;  // s, B/s
  std::vector<double> cost(ng);
  std::vector<int> sig(ng, -1);
  // the distinct counters each group waits for (wptr/wcnt, compressed by
  // group) and the groups waiting for each counter (cptr/cgrp, by counter)
  std::vector<int> wptr(ng + 1, 0), wctr;
  wctr.reserve(ng);
  std::vector<int> total(ncounters, 0), nwait(ncounters + 1, 0);
  for (int gi = 0; gi < ng; ++gi) {
    double bytes = 0;
    int w[kMaxGroupSegs], nw = 0;
    for (int sgi = groups[gi].x; sgi < groups[gi].y; ++sgi) {
      const MvItem& it = items[sgi];
      bytes += 16.0 * std::min(kItemRows, it.m - it.a0) * (pad8(it.k) / 4);  // float panels
      if (it.wait_idx >= 0 && nw < kMaxGroupSegs) w[nw++] = it.wait_idx;
    }
    std::sort(w, w + nw);
    nw = (int)(std::unique(w, w + nw) - w);
    for (int j = 0; j < nw; ++j) {
      wctr.push_back(w[j]);
      ++nwait[w[j] + 1];
    }
    wptr[gi + 1] = (int)wctr.size();
    cost[gi] = kLatency + bytes / (kBandwidth / kWorkers);
    sig[gi] = items[groups[gi].y - 1].sig_idx;
    if (sig[gi] >= 0) total[sig[gi]]++;
  }
  for (int c = 0; c < ncounters; ++c) nwait[c + 1] += nwait[c];
  std::vector<int> cgrp(wctr.size()), cfill(nwait.begin(), nwait.end() - 1);
  for (int gi = 0; gi < ng; ++gi)
    for (int j = wptr[gi]; j < wptr[gi + 1]; ++j) cgrp[cfill[wctr[j]]++] = gi;
  // upward rank: emission order is topological, so one reverse sweep suffices
  std::vector<double> rank(ng, 0.0), cmax(ncounters, 0.0);
  for (int gi = ng - 1; gi >= 0; --gi) {
    rank[gi] = cost[gi] + (sig[gi] >= 0 ? cmax[sig[gi]] : 0.0);
    for (int j = wptr[gi]; j < wptr[gi + 1]; ++j) cmax[wctr[j]] = std::max(cmax[wctr[j]], rank[gi]);
  }
  std::vector<int> pending(ng), done(ncounters, 0);
  using Ready = std::pair<double, int>;  // (rank, group)
  std::vector<Ready> ready_store;
  ready_store.reserve(ng);
  std::priority_queue<Ready> ready(std::less<Ready>(), std::move(ready_store));
  for (int gi = 0; gi < ng; ++gi) {
    pending[gi] = wptr[gi + 1] - wptr[gi];
    if (pending[gi] == 0) ready.push({rank[gi], gi});
  }
  using Run = std::pair<double, int>;  // (finish, group), earliest first
  std::priority_queue<Run, std::vector<Run>, std::greater<Run>> running;
  std::vector<int> order;
  std::vector<float> t_order;
  order.reserve(ng);
  t_order.reserve(ng);
  double t = 0.0;
  int free_workers = (int)kWorkers;
  while ((int)order.size() < ng) {
    while (free_workers > 0 && !ready.empty()) {
      const int gi = ready.top().second;
      ready.pop();
      order.push_back(gi);
      t_order.push_back((float)t);
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
      for (int j = nwait[c]; j < nwait[c + 1]; ++j) {
        // a group waits for the counter to reach its full count
        const int gw = cgrp[j];
        if (--pending[gw] == 0) ready.push({rank[gw], gw});
      }
  }
  if ((int)order.size() != ng) {  // keep the emission order
    for (int i = 0; i < ng; ++i) start[i] = (float)i / ng;
    makespan = 1.f;
    return;
  }
  while (!running.empty()) {
    t = running.top().first;
    running.pop();
  }
  std::vector<int2> out(ng);
  for (int i = 0; i < ng; ++i) out[i] = groups[order[i]];
  groups.swap(out);
  start.swap(t_order);
  makespan = (float)t;
}

namespace {

// host descriptor of a plan item
int to_seg(const MvItem& it, MvSeg& s) {
  if (it.a_off % 8 != 0 || it.a_off / 8 > 0xffffffffLL || it.x_row > INT32_MAX || it.o_row > INT32_MAX) {
    set_error("internal: product plan offsets exceed the descriptor range");
    return GCA_ERR_UNSUPPORTED;
  }
  s.a8 = (uint32_t)(it.a_off / 8);
  s.x_row = (int32_t)it.x_row;
  s.o_row = (int32_t)it.o_row;
  s.rk = (uint32_t)std::min(kItemRows, it.m - it.a0) | ((uint32_t)it.k << 16);
  s.flags = (uint32_t)(it.kind & 15) | ((uint32_t)((it.kind >> 4) & 15) << 8) |
            ((uint32_t)((it.kind >> 8) & 15) << 16) | ((uint32_t)(it.flush ? 1 : 0) << 24);
  s.wait_idx = it.wait_idx;
  s.wait_cnt = it.wait_cnt;
  s.sig_idx = it.sig_idx;
  return GCA_OK;
}

}  // namespace

// Work items of one direction (0: product, 1: transposed product).
// Segments = (block, 64-row slice, 64-column chunk); groups = runs of
// segments with the same output rows claimed and accumulated together.
// Host part of the product plan of one direction (pure host code: it runs
// while the device computes the coefficients).
struct DirPlan {
  std::vector<MvSeg> segs;  // group records in claim order: chain, then free
  int64_t n_chain = 0, n_free = 0;
  std::vector<float> chain_t;
  float makespan = 0.f;
  int status = GCA_OK;
  std::string error;
};

int plan_dir(const gca_h2* h, int dir, DirPlan& P) {
  const int nc = h->nc;
  const bool trans = dir == 1;
  std::vector<MvItem> items;
  std::vector<int2> groups, free_groups;
  std::vector<int2>* target = &groups;  // list the groups being emitted go to
  std::vector<int> cx(nc, 0), cy(nc, 0);  // contributions (groups) to x-hat_c, y-hat_c
  {
    const size_t nblk = h->far_t.size() + h->near_t.size();
    items.reserve(2 * nblk + 4 * (size_t)nc);
    groups.reserve(nblk / 2 + 4 * (size_t)nc);
  }
  struct Blk {
    int kind;
    int64_t a_off;
    int m, k;
    int64_t x_row;
    int wait_idx, wait_cnt;
  };
  // one group per slice of rows [a0, a0 + 64) over a list of blocks sharing
  // output rows; a segment covers `piece` columns of one tile (a multiple of
  // 8 dividing kChunk: column kc of a tile starts at element kc * rows in
  // every precision, so a piece is one contiguous run of panels)
  auto emit = [&](const std::vector<Blk>& blks, int in, int out, int64_t o_row0, int m, int sig_idx,
                  int* sig_cnt, int max_segs, int piece) {
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
        for (int k0 = 0; k0 < b.k; k0 += piece) {
          if (segs == max_segs) close();
          MvItem it{};
          // columns [k0, k0 + piece) of row slice a0 of the block (tiled
          // panel layout, panel.cuh)
          it.a_off = b.a_off + (int64_t)a0 * pad8(b.k) + (int64_t)std::min(kItemRows, m - a0) * k0;
          it.x_row = b.x_row + k0;
          it.o_row = o_row0 + a0;
          it.m = m;
          it.k = std::min(piece, b.k - k0);
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
  const int kCoupleSegs = 8, kNearSegs = 8;
  // input side (forward transform) and output side (backward transform) of
  // this direction: the cluster bases V, E, or the column bases W, F of an
  // operator that has them
  const auto& rin = h->rank_in(dir);
  const auto& rout = h->rank_out(dir);
  const auto& xin = h->xoff_in(dir);
  const auto& xout = h->xoff_out(dir);
  const int kLeafIn = h->in_cols(dir) ? kWt : kVt, kUpIn = h->in_cols(dir) ? kFt : kEt;
  const int kDownOut = h->out_cols(dir) ? kF : kE, kLeafOut = h->out_cols(dir) ? kW : kV;
  // segments of the transforms (the critical path of the product): one tile
  // each, every tile of a transfer block in a group of its own, so that each
  // step of the tree recursion is spread over many warps
  const int kChainPiece = kChunk;
  // Single-level bases (op 3) and Green quadrature (op 4) have a basis for
  // every cluster of a block and no transfers; Green quadrature's couplings
  // B^* read x itself in the product and write y itself in the transposed one.
  const bool single = h->single_level();
  const bool gq = h->op == 4;
  // forward transform: leaves (every cluster with a basis when single)
  for (int c = 1; c < nc; ++c)
    if ((h->child0[c] < 0 || single) && rin[c] > 0 && !(gq && !trans))
      emit({{kLeafIn, O[kLeafIn][c], rin[c], h->end[c] - h->begin[c], h->begin[c], -1, 0}}, kInX, kOutXh,
           xin[c], rin[c], c, &cx[c], 1, kChainPiece);
  // forward transform: up the tree, deepest level first (one segment per group:
  // the chain is latency bound, so its work is spread over many warps)
  for (int L = h->depth - 1; L >= 1 && !single; --L)
    for (int p : h->by_level[L]) {
      if (h->child0[p] < 0) continue;
      for (int ch : {h->child0[p], h->child1[p]})
        emit({{kUpIn, O[kUpIn][ch], rin[p], rin[ch], xin[ch], ch, cx[ch]}}, kInXh, kOutXh, xin[p], rin[p], p,
             &cx[p], 1, kChainPiece);
    }
  // coupling: per output cluster, its blocks (deepest input first) in groups
  // of a few segments; clusters deepest first, since their inputs are ready
  // first.  The near field has no dependencies and goes to the free list.
  std::vector<std::vector<int>> far_by_own(nc);
  for (int b = 0; b < (int)h->far_t.size(); ++b)
    far_by_own[trans ? h->far_s[b] : h->far_t[b]].push_back(b);
  std::vector<int> owners;
  for (int c = 0; c < nc; ++c)
    if (!far_by_own[c].empty()) owners.push_back(c);
  std::stable_sort(owners.begin(), owners.end(), [&](int u, int v) { return h->level[u] > h->level[v]; });
  for (int own : owners) {
    auto& bl = far_by_own[own];
    std::stable_sort(bl.begin(), bl.end(), [&](int u, int v) {
      const int iu = trans ? h->far_t[u] : h->far_s[u], iv = trans ? h->far_t[v] : h->far_s[v];
      return h->level[iu] > h->level[iv];
    });
    std::vector<Blk> blks;
    if (gq && !trans) {
      // y-hat_tau += B_{tau sigma}^* x|sigma-hat
      for (int b : bl) {
        const int in = h->far_s[b];
        blks.push_back({kS, O[kS][b], rout[own], h->end[in] - h->begin[in], h->begin[in], -1, 0});
      }
      emit(blks, kInX, kOutYh, xout[own], rout[own], nc + own, &cy[own], kCoupleSegs, kChunk);
    } else if (gq) {
      // y|sigma-hat += B_{tau sigma} x-hat_tau, x-hat_tau = A_tau^* x|tau-hat
      for (int b : bl) {
        const int in = h->far_t[b];
        blks.push_back({kSt, O[kSt][b], h->end[own] - h->begin[own], rin[in], xin[in], in, cx[in]});
      }
      emit(blks, kInXh, kOutY, h->begin[own], h->end[own] - h->begin[own], -1, nullptr, kCoupleSegs, kChunk);
    } else {
      for (int b : bl) {
        const int in = trans ? h->far_t[b] : h->far_s[b];
        blks.push_back({trans ? kSt : kS, O[trans ? kSt : kS][b], rout[own], rin[in], xin[in], in, cx[in]});
      }
      emit(blks, kInXh, kOutYh, xout[own], rout[own], nc + own, &cy[own], kCoupleSegs, kChunk);
    }
  }
  {
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
      emit(blks, kInX, kOutY, h->begin[own], h->end[own] - h->begin[own], -1, nullptr, kNearSegs, kChunk);
    }
    target = &groups;
  }
  // backward transform, level by level down (y-hat of the parent must be final)
  for (int L = 2; L <= h->depth && !single; ++L)
    for (int c : h->by_level[L]) {
      const int p = h->parent[c];
      if (cy[p] == 0 || rout[c] == 0) continue;  // y-hat_p = 0
      emit({{kDownOut, O[kDownOut][c], rout[c], rout[p], xout[p], nc + p, cy[p]}}, kInYh, kOutYh, xout[c],
           rout[c], nc + c, &cy[c], 1, kChainPiece);
    }
  // leaf bases (every cluster with a basis when single)
  for (int c = 1; c < nc; ++c)
    if ((h->child0[c] < 0 || single) && rout[c] > 0 && cy[c] > 0)
      emit({{kLeafOut, O[kLeafOut][c], h->end[c] - h->begin[c], rout[c], xout[c], nc + c, cy[c]}}, kInYh,
           kOutY, h->begin[c], h->end[c] - h->begin[c], -1, nullptr, 1, kChainPiece);
  for (const auto* gl : {&groups, &free_groups})
    for (const int2& g : *gl)
      if (g.y - g.x > kMaxGroupSegs) {
        set_error("internal: work group longer than a group record");
        return GCA_ERR_UNSUPPORTED;
      }
  schedule_groups(items, groups, 2 * nc, P.chain_t, P.makespan);
  P.n_chain = (int64_t)groups.size();
  P.n_free = (int64_t)free_groups.size();
  // group records in claim order: chain groups, then free groups
  P.segs.assign((groups.size() + free_groups.size()) * kMaxGroupSegs, MvSeg{});
  size_t gi = 0;
  for (const auto* gl : {&groups, &free_groups})
    for (const int2& g : *gl) {
      for (int j = g.x; j < g.y; ++j) GCA_TRY(to_seg(items[j], P.segs[gi * kMaxGroupSegs + (j - g.x)]));
      ++gi;
    }
  return GCA_OK;
}

// The plans of both directions, each computed on the calling thread.  (On
// worker threads the planning ran several times slower than here, so the
// build instead plans while its kernels are queued on the device.)
struct PlanJob {
  DirPlan p[2];
  bool done[2] = {false, false};
};

void PlanJobDelete::operator()(PlanJob* j) const { delete j; }

PlanHandle plan_new() { return PlanHandle(new PlanJob); }

void plan_direction(const gca_h2* h, int dir, PlanJob* job) {
  DirPlan& P = job->p[dir];
  P.status = plan_dir(h, dir, P);
  if (P.status != GCA_OK) P.error = last_error();
  job->done[dir] = true;
}

int finish_plan(gca_h2* h, PlanJob* job, cudaStream_t st) {
  h->max_rows = std::max(std::max(h->max_rank, h->max_rank2), h->max_leaf);
  {
    std::vector<int> iperm(h->n);
    for (int i = 0; i < h->n; ++i) iperm[h->perm[i]] = i;
    GCA_TRY(upload(h->d_iperm, iperm, st));
  }
  for (int dir = 0; dir < 2; ++dir) {
    if (h->served_dir(dir) != dir) continue;  // mirrored: no transposed plan
    if (!job->done[dir]) plan_direction(h, dir, job);
    DirPlan& P = job->p[dir];
    if (P.status != GCA_OK) {
      set_error(P.error);
      return P.status;
    }
    h->n_chain[dir] = P.n_chain;
    h->n_free[dir] = P.n_free;
    h->chain_t[dir].swap(P.chain_t);
    h->makespan[dir] = P.makespan;
    GCA_TRY(upload(h->d_segs[dir], P.segs, st));
  }
  GCA_TRY(h->d_status.alloc(sizeof(int)));
  GCA_TRY_CUDA(cudaMemsetAsync(h->d_status.p, 0, sizeof(int), st));
  return GCA_OK;
}

namespace {

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }  // keeps every region aligned

// Claim orders of a batch: every slot's list in its own order, the slots
// interleaved by scheduled start time (chain) or by relative position
// (free), so that all meshes progress together.
void merge_claims(const gca_h2* const* hs, int count, int dir, const std::vector<int>& nchunk,
                  std::vector<int2>& chain_map, std::vector<int2>& free_map) {
  using Key = std::pair<float, int>;  // (time, slot)
  chain_map.clear();
  free_map.clear();
  {
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> q;
    std::vector<int64_t> pos(count, 0);
    for (int s = 0; s < count; ++s)
      if (hs[s]->n_chain[dir] > 0) q.push({hs[s]->chain_t[dir][0], s});
    while (!q.empty()) {
      const int s = q.top().second;
      q.pop();
      const int64_t g = pos[s]++;
      for (int c = 0; c < nchunk[s]; ++c) chain_map.push_back(make_int2(s, (int)(g * nchunk[s] + c)));
      if (pos[s] < hs[s]->n_chain[dir]) q.push({hs[s]->chain_t[dir][pos[s]], s});
    }
  }
  {
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> q;
    std::vector<int64_t> pos(count, 0);
    auto key = [&](int s) { return (float)((pos[s] + 0.5) / (double)hs[s]->n_free[dir]); };
    for (int s = 0; s < count; ++s)
      if (hs[s]->n_free[dir] > 0) q.push({key(s), s});
    while (!q.empty()) {
      const int s = q.top().second;
      q.pop();
      const int64_t g = pos[s]++;
      for (int c = 0; c < nchunk[s]; ++c) free_map.push_back(make_int2(s, (int)(g * nchunk[s] + c)));
      if (pos[s] < hs[s]->n_free[dir]) q.push({key(s), s});
    }
  }
}

template <typename T, typename TN, typename TV>
void fill_slot(SlotArgs<TV>& a, const gca_h2* h, int dir, int R, int RC, const void* x, int64_t ldx,
               void* y, int64_t ldy, bool trans = false) {
  const DevMem* P = sizeof(T) == 8 ? h->P64 : (sizeof(T) == 4 ? h->P32 : h->P16);
  const DevMem* PN = sizeof(TN) == 8 ? h->P64 : h->P32;
  for (int q = 0; q < kPanelKinds; ++q) a.A[q] = (q == kN || q == kNt) ? PN[q].p : P[q].p;
  // a mirrored handle's transposed product: the product's plan, whose
  // near-field segments then read N_{mirror(b)}^T at block b's offset
  if (trans && h->mirrored) a.A[kN] = PN[kNt].p;
  a.segs = h->d_segs[dir].as<MvSeg>();
  a.n_chain = h->n_chain[dir];
  a.n_free = h->n_free[dir];
  a.R = R;
  a.nchunk = (R + RC - 1) / RC;
  a.n = h->n;
  a.rc = RC;
  a.rs_in = (int)h->rank_sum_in(dir);
  a.rs_out = (int)h->rank_sum_out(dir);
  a.x = static_cast<const TV*>(x);
  a.ldx = ldx;
  a.y = static_cast<TV*>(y);
  a.ldy = ldy;
  a.perm = h->d_perm.as<int>();
  a.iperm = h->d_iperm.as<int>();
}

// Launches the persistent kernel with as many CTAs as fit on the device (found once per device and kernel, so that later launches
// make no attribute or occupancy calls and can be graph captured).
template <typename T, typename TN, typename TA, typename TV, int RC>
int launch_persistent(const LaunchArgs& L, const SlotPack<TV>& pack, int64_t units, cudaStream_t st) {
  const size_t smem = cta_smem<TA, RC>();
  auto kern = k_h2_persistent<T, TN, TA, TV, RC>;
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
    if constexpr (kSplitRegs<TA>) {
      // setmaxnreg moves registers inside the CTA's launch allocation: the
      // split only balances if every thread was launched with kLaunchRegs
      cudaFuncAttributes fa{};
      GCA_TRY_CUDA(cudaFuncGetAttributes(&fa, kern));
      if (fa.numRegs != kLaunchRegs) {
        set_error("internal: product kernel compiled with " + std::to_string(fa.numRegs) +
                  " registers a thread, the register split needs " + std::to_string(kLaunchRegs));
        return GCA_ERR_UNSUPPORTED;
      }
    }
    int sms = 0, per_sm = 0;
    GCA_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GCA_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    cap = (int64_t)sms * std::max(per_sm, 1);
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64) cap_by_dev[dev] = cap;
  }
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((units + kPairs - 1) / kPairs, cap));
  kern<<<grid, kThreads, smem, st>>>(L, pack);
  return GCA_OK;
}

// One persistent launch over `count` handles (slots).  Workspace layout:
// [claim counters, abort flag, zeros | per slot: x-hat, y-hat, y (cluster
// order), counters] zeroed by one memset, then per slot x (cluster order).
// Up to kInlineSlots slot descriptors travel as a kernel parameter; the
// merged claim orders of a batch come precomputed from gca_build_batch when
// every mesh takes one right-hand-side chunk.  Other launches keep their
// descriptors (and claim orders) in the device cache of the precision and
// direction, uploaded when the arguments change.
template <typename T, typename TN, typename TA, typename TV, int RC>
int launch_rc(const gca_h2* const* hs, int count, int dir, bool trans, const int32_t* nrhs, const void* const* x,
              const int64_t* ldx, void* const* y, const int64_t* ldy, ProductCache& pc, int* status,
              cudaStream_t st) {
  const char* pn = sizeof(T) == 8 ? ".f64" : (sizeof(T) == 4 ? ".f32" : ".bf16");
  PhaseScope ps(std::string("mv_persistent") + pn + (trans ? ".T" : ""), st);
  ps.launches(3);
  DevMem& ws = pc.ws;
  std::vector<SlotArgs<TV>> sl(count);
  size_t off = 256 + kZeroBytes;  // claim counters + abort flag, zeros
  std::vector<size_t> o_xh(count), o_yh(count), o_yp(count), o_cnt(count), o_xp(count);
  for (int i = 0; i < count; ++i) {
    const gca_h2* h = hs[i];
    const int R = (nrhs[i] + RC - 1) / RC * RC;  // chunk-major vectors: whole chunks
    o_xh[i] = off;
    off += up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum_in(dir), 1) * R);
    o_yh[i] = off;
    off += up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum_out(dir), 1) * R);
    o_yp[i] = off;
    off += up256(sizeof(TV) * (size_t)h->n * R);
    o_cnt[i] = off;
    off += up256(sizeof(int) * 2 * (size_t)h->nc);
  }
  const size_t zeroed = off;
  for (int i = 0; i < count; ++i) {
    o_xp[i] = off;
    off += up256(sizeof(TV) * (size_t)hs[i]->n * ((nrhs[i] + RC - 1) / RC * RC));
  }
  std::vector<int> nchunk(count);
  int64_t work = 0, free_work = 0;
  int max_n = 0;
  for (int i = 0; i < count; ++i) {
    nchunk[i] = (nrhs[i] + RC - 1) / RC;
    work += hs[i]->n_chain[dir] * nchunk[i];
    free_work += hs[i]->n_free[dir] * nchunk[i];
    max_n = std::max(max_n, hs[i]->n * nrhs[i]);
  }
  GCA_TRY(ws.reserve(off));
  unsigned char* base = ws.as<unsigned char>();
  for (int i = 0; i < count; ++i) {
    SlotArgs<TV>& a = sl[i];
    fill_slot<T, TN, TV>(a, hs[i], dir, nrhs[i], RC, x[i], ldx[i], y[i], ldy[i], trans);
    a.xh = reinterpret_cast<TV*>(base + o_xh[i]);
    a.yh = reinterpret_cast<TV*>(base + o_yh[i]);
    a.yp = reinterpret_cast<TV*>(base + o_yp[i]);
    a.counters = reinterpret_cast<int*>(base + o_cnt[i]);
    a.xp = reinterpret_cast<TV*>(base + o_xp[i]);
  }
  const bool inline_slots = count <= kInlineSlots;
  // the batch's one-chunk claim orders serve every product whose meshes all
  // take the same number of chunks: each group's claim is repeated per chunk
  bool same_chunks = true;
  for (int i = 1; i < count; ++i) same_chunks = same_chunks && nchunk[i] == nchunk[0];
  const int rep = count > 0 ? nchunk[0] : 1;
  const bool pre_maps = count > 1 && same_chunks && pc.maps1[dir].p && pc.maps1_chain[dir] * rep == work &&
                        pc.maps1_free[dir] * rep == free_work;
  const bool dev_maps = count > 1 && !pre_maps;
  SlotPack<TV> pack;
  std::memset(&pack, 0, sizeof(pack));
  LaunchArgs L;
  L.slots = nullptr;
  L.chain_map = nullptr;
  L.free_map = nullptr;
  L.map_rep = 1;
  if (inline_slots)
    for (int i = 0; i < count; ++i) pack.s[i] = sl[i];
  if (pre_maps) {
    L.chain_map = pc.maps1[dir].as<int2>();
    L.free_map = L.chain_map + work / rep;
    L.map_rep = rep;
  }
  const SlotArgs<TV>* d_slots = nullptr;
  if (!inline_slots || dev_maps) {
    DescCache& dc = pc.desc[(sizeof(T) == 8 ? 0 : (sizeof(T) == 4 ? 1 : 2)) * 2 + (trans ? 1 : 0)];
    size_t doff = up256(sizeof(SlotArgs<TV>) * count);
    const size_t o_cmap = doff;
    if (dev_maps) doff += up256(sizeof(int2) * (size_t)std::max<int64_t>(work, 1));
    const size_t o_fmap = doff;
    if (dev_maps) doff += up256(sizeof(int2) * (size_t)std::max<int64_t>(free_work, 1));
    if (doff > dc.mem.bytes) dc.key.clear();
    GCA_TRY(dc.mem.reserve(doff));
    unsigned char* dbase = dc.mem.as<unsigned char>();
    // the descriptors (and claim orders) change only with the arguments:
    // upload when they differ from what the cache already holds (the
    // descriptors contain the workspace and the caller's vector addresses)
    const size_t sbytes = sizeof(SlotArgs<TV>) * count;
    std::vector<unsigned char> key(sbytes + 1);
    std::memcpy(key.data(), sl.data(), sbytes);
    key[sbytes] = dev_maps ? 1 : 0;
    if (dc.key != key) {
      GCA_TRY_CUDA(cudaMemcpyAsync(dbase, sl.data(), sbytes, cudaMemcpyHostToDevice, st));
      std::vector<int2> cmap, fmap;
      if (dev_maps) {
        merge_claims(hs, count, dir, nchunk, cmap, fmap);
        if ((int64_t)cmap.size() != work || (int64_t)fmap.size() != free_work) {
          set_error("internal: merged claim order has the wrong length");
          return GCA_ERR_UNSUPPORTED;
        }
        if (work > 0)
          GCA_TRY_CUDA(cudaMemcpyAsync(dbase + o_cmap, cmap.data(), sizeof(int2) * work, cudaMemcpyHostToDevice, st));
        if (free_work > 0)
          GCA_TRY_CUDA(
              cudaMemcpyAsync(dbase + o_fmap, fmap.data(), sizeof(int2) * free_work, cudaMemcpyHostToDevice, st));
      }
      GCA_TRY_CUDA(cudaStreamSynchronize(st));  // sl, cmap, fmap are host vectors of this frame
      dc.key.swap(key);
    }
    d_slots = reinterpret_cast<const SlotArgs<TV>*>(dbase);
    if (!inline_slots) L.slots = dbase;
    if (dev_maps) {
      L.chain_map = reinterpret_cast<const int2*>(dbase + o_cmap);
      L.free_map = reinterpret_cast<const int2*>(dbase + o_fmap);
    }
  }
  L.nslots = count;
  L.total = work;
  L.total_free = free_work;
  L.next = reinterpret_cast<unsigned long long*>(base);
  L.next_free = reinterpret_cast<unsigned long long*>(base + 8);
  L.abort_flag = reinterpret_cast<int*>(base + 16);
  L.zeros = base + 256;
  L.status = status;
  {
    const TestHooks th = test_hooks();
    L.wait_cycles = th.wait_cycles;
    L.wait_extra = th.stall_chain;
  }
  GCA_TRY_CUDA(cudaMemsetAsync(base, 0, zeroed, st));
  const unsigned gx = (unsigned)std::min<int64_t>(1024, (max_n + 255) / 256);
  k_gather<TV><<<dim3(std::max(1u, gx), count), 256, 0, st>>>(d_slots, pack, inline_slots ? 1 : 0);
  if (work + free_work > 0) GCA_TRY((launch_persistent<T, TN, TA, TV, RC>(L, pack, work + free_work, st)));
  k_scatter<TV><<<dim3(std::max(1u, gx), count), 256, 0, st>>>(d_slots, pack, inline_slots ? 1 : 0);
  GCA_TRY_CUDA(cudaGetLastError());
  return GCA_OK;
}

// ------------------------------------------------------------- autotuner
//
// The tile width RC (right-hand sides of a warp tile; a product runs in
// chunks of RC columns) is a per-launch choice among the compiled widths 1,
// 2, 4, 8 and 16.  By default the smallest width at or above the largest R
// (16 from R = 16 on; at most 4 in float64, below).  gca_tune_batch times the
// widths from a quarter to four times the default on a real product and
// records the fastest per (device name, precision, direction, largest R,
// log2 of the total rows); later products with that key use it.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
thread_local int g_force_rc = 0;  // width forced while tuning (0: none)

// the float64 product is bound by the FP64 pipe, not by streaming the
// blocks: narrow tiles (more chunks, each block streamed once per chunk) run
// it faster (the autotuner measured width 4 about 8% faster than 16 at
// R = 16, 32 and 64 on the 20480-triangle pair)
int default_width(int R, int prec) {
  const int w = R >= 16 ? 16 : (R > 4 ? 8 : (R > 2 ? 4 : (R > 1 ? 2 : 1)));
  return prec == GCA_F64 ? std::min(w, 4) : w;
}

std::string device_name() {
  int dev = 0;
  cudaDeviceProp pr{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string nm(pr.name);
  for (char& c : nm)
    if (c == '|' || c == ' ' || c == '\n') c = '_';
  return nm;
}

std::string tune_key(const std::string& dev, int prec, int dir, int R, int64_t rows) {
  int lg = 0;
  while (lg < 62 && (int64_t(1) << (lg + 1)) <= rows) ++lg;
  return dev + "|" + std::to_string(prec) + "|" + std::to_string(dir) + "|" + std::to_string(R) + "|" +
         std::to_string(lg);
}

int tuned_width(int prec, int dir, int R, int64_t rows) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune.empty()) return 0;
  const auto it = g_tune.find(tune_key(device_name(), prec, dir, R, rows));
  return it == g_tune.end() ? 0 : it->second;
}

template <typename T, typename TN, typename TA, typename TV>
int launch(const gca_h2* const* hs, int count, int dir, bool trans, const int32_t* nrhs, const void* const* x,
           const int64_t* ldx, void* const* y, const int64_t* ldy, ProductCache& pc, int* status,
           cudaStream_t st) {
  int R = 1;
  int64_t rows = 0;
  for (int i = 0; i < count; ++i) {
    R = std::max(R, (int)nrhs[i]);
    rows += hs[i]->n;
  }
  constexpr int prec = sizeof(T) == 8 ? GCA_F64 : (sizeof(T) == 4 ? GCA_F32 : GCA_BF16);
  int rc = g_force_rc;
  // the tuner's key holds the caller's direction (a mirrored handle's
  // transposed product runs plan 0 but keeps its own tuned width)
  if (rc == 0) rc = tuned_width(prec, trans ? 1 : 0, R, rows);
  if (rc == 0) rc = default_width(R, prec);
  switch (rc) {
    case 16: return launch_rc<T, TN, TA, TV, 16>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc, status, st);
    case 8: return launch_rc<T, TN, TA, TV, 8>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc, status, st);
    case 4: return launch_rc<T, TN, TA, TV, 4>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc, status, st);
    case 2: return launch_rc<T, TN, TA, TV, 2>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc, status, st);
    default: return launch_rc<T, TN, TA, TV, 1>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc, status, st);
  }
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

// The address under which a kernel reads or writes a caller's x or y:
// device memory of the current device as it is, page-locked host memory
// mapped into the device's address space by its device alias; anything else
// (pageable host memory, another device's memory) is refused rather than
// handed to a kernel.
int resolve_io(const void* p, const void** dev_p, const char* what, int i) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    a.type = cudaMemoryTypeUnregistered;
  }
  int dev = 0;
  GCA_TRY_CUDA(cudaGetDevice(&dev));
  if ((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev) {
    *dev_p = p;
    return GCA_OK;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *dev_p = a.devicePointer;
    return GCA_OK;
  }
  set_error(std::string("h2_matvec: ") + what + " of product " + std::to_string(i) +
            " is neither memory of the current device nor mapped page-locked host memory");
  return GCA_ERR_INVALID_ARG;
}

int launch_any(const gca_h2* const* hs, int count, gca_prec prec, bool trans, const int32_t* nrhs,
               const void* const* x_in, const int64_t* ldx, void* const* y_in, const int64_t* ldy,
               ProductCache& pc, int* status, cudaStream_t st) {
  std::vector<const void*> xs(count);
  std::vector<void*> ys(count);
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) {
      set_error("h2_matvec: NULL handle " + std::to_string(i));
      return GCA_ERR_INVALID_ARG;
    }
    GCA_TRY(check_device(hs[i]->device, "h2_matvec"));
    if (!x_in[i] || !y_in[i]) {
      set_error("h2_matvec: invalid arguments (handle " + std::to_string(i) + ")");
      return GCA_ERR_INVALID_ARG;
    }
    const void* yd = nullptr;
    GCA_TRY(resolve_io(x_in[i], &xs[i], "x", i));
    GCA_TRY(resolve_io(y_in[i], &yd, "y", i));
    ys[i] = const_cast<void*>(yd);
  }
  const void* const* x = xs.data();
  void* const* y = ys.data();
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
  // plan direction: a mirrored (symmetric) handle serves G^T x with the
  // plan of G x (and its transposed near-field panels)
  const int dir = hs[0]->served_dir(trans ? 1 : 0);
  for (int i = 1; i < count; ++i)
    if (hs[i]->served_dir(trans ? 1 : 0) != dir) {
      set_error("h2_matvec: a launch mixes symmetric and non-symmetric handles");
      return GCA_ERR_UNSUPPORTED;
    }
  switch (prec) {
    case GCA_F64:
      return launch<double, double, double, double>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc, status, st);
    case GCA_F32:
      return launch<float, float, float, float>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc, status, st);
    case GCA_BF16:
      return launch<__nv_bfloat16, float, float, float>(hs, count, dir, trans, nrhs, x, ldx, y, ldy, pc,
                                                        status, st);
  }
  set_error("h2_matvec: unknown precision");
  return GCA_ERR_INVALID_ARG;
}

}  // namespace

// Claim orders of a batch for one right-hand-side chunk per mesh (R <= 16),
// merged and uploaded once when the batch is built.
int prepare_batch(gca_h2_batch* b, cudaStream_t st) {
  const int count = (int)b->h.size();
  if (count < 2) return GCA_OK;
  std::vector<const gca_h2*> hs(b->h.begin(), b->h.end());
  std::vector<int> nchunk(count, 1);
  for (int dir = 0; dir < 2; ++dir) {
    if (hs[0]->served_dir(dir) != dir) continue;  // mirrored: the transposed product runs plan 0
    std::vector<int2> cmap, fmap;
    merge_claims(hs.data(), count, dir, nchunk, cmap, fmap);
    cmap.insert(cmap.end(), fmap.begin(), fmap.end());
    b->pc.maps1_chain[dir] = (int64_t)cmap.size() - (int64_t)fmap.size();
    b->pc.maps1_free[dir] = (int64_t)fmap.size();
    if (cmap.empty()) cmap.push_back(make_int2(0, 0));
    GCA_TRY(upload(b->pc.maps1[dir], cmap, st));
  }
  GCA_TRY_CUDA(cudaStreamSynchronize(st));  // the host vectors go out of scope
  return GCA_OK;
}

namespace {

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
  return launch_any(hs, 1, prec, trans, &nrhs, xs, &ldx, ys, &ldy, h->pc, h->d_status.as<int>(), st);
}

int matvec_batch(const gca_h2_batch* b, gca_prec prec, bool trans, const int32_t* nrhs,
                 const void* const* x, const int64_t* ldx, void* const* y, const int64_t* ldy,
                 cudaStream_t st) {
  if (!b || b->h.empty() || !nrhs || !x || !ldx || !y || !ldy) {
    set_error("h2_matvec_batch: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  std::vector<const gca_h2*> hs(b->h.begin(), b->h.end());
  return launch_any(hs.data(), (int)hs.size(), prec, trans, nrhs, x, ldx, y, ldy, b->pc,
                    b->d_status.as<int>(), st);
}

int tune_batch(const gca_h2_batch* b, gca_prec prec, bool trans, const int32_t* nrhs, const void* const* x,
               const int64_t* ldx, void* const* y, const int64_t* ldy, cudaStream_t st, int* rc_out) {
  if (!b || b->h.empty() || !nrhs || !x || !ldx || !y || !ldy || !rc_out) {
    set_error("gca_tune_batch: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  int R = 1;
  int64_t rows = 0;
  for (size_t i = 0; i < b->h.size(); ++i) {
    R = std::max(R, (int)nrhs[i]);
    rows += b->h[i]->n;
  }
  const int d = default_width(R, (int)prec);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GCA_TRY_CUDA(cudaEventCreate(&e0));
  GCA_TRY_CUDA(cudaEventCreate(&e1));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  int best = 0;
  float best_ms = 0.f;
  for (int rc : {16, 8, 4, 2, 1}) {
    if (rc > 4 * d || 4 * rc < d) continue;  // from a quarter to four times the default
    g_force_rc = rc;
    int s = GCA_OK;
    for (int w = 0; w < 2 && s == GCA_OK; ++w) s = matvec_batch(b, prec, trans, nrhs, x, ldx, y, ldy, st);
    std::vector<float> ms;
    for (int r = 0; r < 5 && s == GCA_OK; ++r) {
      cudaEventRecord(e0, st);
      s = matvec_batch(b, prec, trans, nrhs, x, ldx, y, ldy, st);
      cudaEventRecord(e1, st);
      float t = 0.f;
      if (s == GCA_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)) {
        set_error("gca_tune_batch: timing failed");
        s = GCA_ERR_CUDA;
      }
      ms.push_back(t);
    }
    g_force_rc = 0;
    if (s != GCA_OK) return s;
    std::sort(ms.begin(), ms.end());
    const float med = ms[ms.size() / 2];
    if (best == 0 || med < best_ms) {
      best = rc;
      best_ms = med;
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(device_name(), (int)prec, trans ? 1 : 0, R, rows)] = best;
  }
  *rc_out = best;
  return GCA_OK;
}

int tune_save(const char* path) {
  if (!path) {
    set_error("gca_tune_save: NULL path");
    return GCA_ERR_INVALID_ARG;
  }
  std::FILE* f = std::fopen(path, "w");
  if (!f) {
    set_error(std::string("gca_tune_save: cannot open ") + path);
    return GCA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : g_tune) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
  const bool ok = std::fclose(f) == 0;
  if (!ok) {
    set_error(std::string("gca_tune_save: write failed: ") + path);
    return GCA_ERR_INVALID_ARG;
  }
  return GCA_OK;
}

int tune_load(const char* path) {
  if (!path) {
    set_error("gca_tune_load: NULL path");
    return GCA_ERR_INVALID_ARG;
  }
  std::FILE* f = std::fopen(path, "r");
  if (!f) {
    set_error(std::string("gca_tune_load: cannot open ") + path);
    return GCA_ERR_INVALID_ARG;
  }
  std::map<std::string, int> add;
  char key[512];
  int rc = 0;
  int st = GCA_OK;
  for (;;) {
    const int got = std::fscanf(f, "%511s %d", key, &rc);
    if (got == EOF) break;
    if (got != 2 || (rc != 1 && rc != 2 && rc != 4 && rc != 8 && rc != 16)) {
      set_error(std::string("gca_tune_load: malformed line in ") + path);
      st = GCA_ERR_INVALID_ARG;
      break;
    }
    add[key] = rc;
  }
  std::fclose(f);
  if (st != GCA_OK) return st;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : add) g_tune[kv.first] = kv.second;
  return GCA_OK;
}

int tune_get(const char* device, gca_prec prec, bool trans, int32_t nrhs, int64_t rows, int* rc) {
  if (!device || !rc || nrhs < 1 || rows < 1) {
    set_error("gca_tune_get: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const auto it = g_tune.find(tune_key(device, (int)prec, trans ? 1 : 0, nrhs, rows));
  *rc = it == g_tune.end() ? 0 : it->second;
  return GCA_OK;
}

void tune_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
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

// h2_matvec's launch for one handle with the workspace carved out of `base`
// (capacity `cap` bytes); nothing is allocated.
template <typename T, typename TN, typename TA, typename TV, int RC>
int launch_noalloc_rc(const gca_h2* h, int R, const void* x, int64_t ldx, void* y, int64_t ldy,
                      unsigned char* base, size_t cap, cudaStream_t st) {
  const int Rp = (R + RC - 1) / RC * RC;  // chunk-major vectors: whole chunks
  const size_t b_xh = up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum_in(0), 1) * Rp);
  const size_t b_yh = up256(sizeof(TV) * (size_t)std::max<int64_t>(h->rank_sum_out(0), 1) * Rp);
  const size_t b_yp = up256(sizeof(TV) * (size_t)h->n * Rp);
  const size_t b_cnt = up256(sizeof(int) * 2 * (size_t)h->nc);
  const size_t o_xh = 256 + kZeroBytes, o_yh = o_xh + b_xh, o_yp = o_yh + b_yh, o_cnt = o_yp + b_yp;
  const size_t zeroed = o_cnt + b_cnt;
  const size_t o_xp = zeroed;
  const size_t need = o_xp + b_yp;
  if (need > cap) {
    set_error("h2_matvec_noalloc: this product needs " + std::to_string(need) +
              " bytes of workspace, more than the " + std::to_string(cap) +
              "-byte scratch array (fewer right-hand sides or h2_matvec)");
    return GCA_ERR_UNSUPPORTED;
  }
  const char* pn = sizeof(T) == 8 ? ".f64" : (sizeof(T) == 4 ? ".f32" : ".bf16");
  PhaseScope ps(std::string("mv_persistent_noalloc") + pn, st);
  ps.launches(3);
  SlotArgs<TV> a{};
  fill_slot<T, TN, TV>(a, h, 0, R, RC, x, ldx, y, ldy);
  a.xh = reinterpret_cast<TV*>(base + o_xh);
  a.yh = reinterpret_cast<TV*>(base + o_yh);
  a.yp = reinterpret_cast<TV*>(base + o_yp);
  a.counters = reinterpret_cast<int*>(base + o_cnt);
  a.xp = reinterpret_cast<TV*>(base + o_xp);
  LaunchArgs L;
  L.slots = nullptr;  // the descriptor travels inline as a kernel parameter
  L.nslots = 1;
  L.map_rep = 1;
  L.chain_map = nullptr;
  L.free_map = nullptr;
  L.total = a.n_chain * a.nchunk;
  L.total_free = a.n_free * a.nchunk;
  L.next = reinterpret_cast<unsigned long long*>(base);
  L.next_free = reinterpret_cast<unsigned long long*>(base + 8);
  L.abort_flag = reinterpret_cast<int*>(base + 16);
  L.zeros = base + 256;
  L.status = h->d_status.as<int>();
  {
    const TestHooks th = test_hooks();
    L.wait_cycles = th.wait_cycles;
    L.wait_extra = th.stall_chain;
  }
  // the array keeps the previous call's contents: the claim counters, abort
  // flag, x-hat, y-hat, y and the counters must start at zero
  GCA_TRY_CUDA(cudaMemsetAsync(base, 0, zeroed, st));
  // the descriptor travels as a kernel parameter: nothing to copy or keep alive
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, ((int64_t)h->n * R + 255) / 256));
  SlotPack<TV> pack;
  std::memset(&pack, 0, sizeof(pack));
  pack.s[0] = a;
  k_gather<TV><<<dim3(gx, 1), 256, 0, st>>>(nullptr, pack, 1);
  if (L.total + L.total_free > 0)
    GCA_TRY((launch_persistent<T, TN, TA, TV, RC>(L, pack, L.total + L.total_free, st)));
  k_scatter<TV><<<dim3(gx, 1), 256, 0, st>>>(nullptr, pack, 1);
  GCA_TRY_CUDA(cudaGetLastError());
  return GCA_OK;
}

template <typename T, typename TN, typename TA, typename TV>
int launch_noalloc(const gca_h2* h, int R, const void* x, int64_t ldx, void* y, int64_t ldy,
                   unsigned char* base, size_t cap, cudaStream_t st) {
  constexpr int prec = sizeof(T) == 8 ? GCA_F64 : (sizeof(T) == 4 ? GCA_F32 : GCA_BF16);
  switch (default_width(R, prec)) {
    case 16: return launch_noalloc_rc<T, TN, TA, TV, 16>(h, R, x, ldx, y, ldy, base, cap, st);
    case 8: return launch_noalloc_rc<T, TN, TA, TV, 8>(h, R, x, ldx, y, ldy, base, cap, st);
    case 4: return launch_noalloc_rc<T, TN, TA, TV, 4>(h, R, x, ldx, y, ldy, base, cap, st);
    case 2: return launch_noalloc_rc<T, TN, TA, TV, 2>(h, R, x, ldx, y, ldy, base, cap, st);
    default: return launch_noalloc_rc<T, TN, TA, TV, 1>(h, R, x, ldx, y, ldy, base, cap, st);
  }
}

}  // namespace

int matvec_noalloc(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx, void* y,
                   int64_t ldy, cudaStream_t st) {
  if (!h || !x || !y || nrhs < 1 || nrhs > 4096 || ldx < h->n || ldy < h->n) {
    set_error("h2_matvec_noalloc: invalid arguments");
    return GCA_ERR_INVALID_ARG;
  }
  GCA_TRY(check_device(h->device, "h2_matvec_noalloc"));
  if (!has_precision(h, prec)) {
    set_error("h2_matvec_noalloc: the handle was built without this precision");
    return GCA_ERR_UNSUPPORTED;
  }
  const void* xd = nullptr;
  const void* yd = nullptr;
  GCA_TRY(resolve_io(x, &xd, "x", 0));
  GCA_TRY(resolve_io(y, &yd, "y", 0));
  x = xd;
  y = const_cast<void*>(yd);
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
