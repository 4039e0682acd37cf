// GCA-H^2 construction on the GPU (Sect. 2 - Sect. 4, Sect. 8).
//
// Pipeline of gca_build (all arithmetic in float64 on the device):
//   1. k_tri_geom       7-point rule nodes and weights of every triangle
//   2. k_cluster_boxes  bounding box of each cluster's vertices
//      host             diameters, admissibility, block tree (tree.cpp)
//   3. k_box_quad       Gauss rule on the faces of omega_tau (Eq. (2))
//   4. k_aca            per tree level, deepest first, one CTA (small
//                       matrices) or one thread-block cluster of 8/16 CTAs
//                       (large ones) per cluster: the Green quadrature matrix
//                       A_tau (leaves: all triangles; parents: the children's
//                       pivot rows) is formed in shared memory, cross-
//                       approximated with complete pivoting (Sect. 3), and
//                       V^ = U L^{-1} is written.  The host reads the level's
//                       ranks back to size the next level.
//   5. k_pack           leaf bases V_tau and transfer matrices E_tau
//                       (Sect. 4) in float64 / float32 / bfloat16
//   6. k_couple_entries S_{tau sigma} = G|tilde-tau x tilde-sigma (7 x 7
//                       point rule: pivots of admissible blocks never touch)
//   7. k_near_entries   G|tau-hat x sigma-hat for inadmissible leaf pairs;
//                       disjoint pairs directly, touching pairs appended to
//                       one list per Sauter-Schwab case (Sect. 8), which
//      k_singular<case> then integrate with one warp per entry.
//   8. reduced-precision copies of S and N.

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <numeric>

#include "internal.hpp"
#include "panel.cuh"
#include "rules.hpp"

namespace gca {

namespace {

constexpr double kInv4Pi = 0.07957747154594767;  // 1 / (4 pi)

// a point and a weight, 32-byte aligned for single vector loads
struct __align__(32) P4 {
  double x, y, z, w;
};
// threads of a cross approximation CTA: 512 for jobs on clusters of 2 or 4
// CTAs (about 60-150 rows per CTA: more warps in flight hide the update's
// latency), 256 otherwise (a few rows per warp on 8 or 16 CTAs, where the
// per-pivot barriers and reductions over more warps cost more than they hide)
constexpr int kAcaThreads = 256;
constexpr int kAcaThreadsWide = 512;
inline bool aca_wide(int C) { return C == 2 || C == 4; }
constexpr int kStatusNumeric = 1;
constexpr int kStatusOverflow = 2;

// ------------------------------------------------------------------ geometry

__global__ void k_tri_geom(int nt, const double* __restrict__ vert, const int* __restrict__ tri,
                           Rules rules, P4* __restrict__ tq, double* __restrict__ area2,
                           double* __restrict__ nrm) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
  double a[3], b[3], c[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = vert[3 * ia + d];
    b[d] = vert[3 * ib + d];
    c[d] = vert[3 * ic + d];
  }
  double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double cx = u[1] * v[2] - u[2] * v[1];
  double cy = u[2] * v[0] - u[0] * v[2];
  double cz = u[0] * v[1] - u[1] * v[0];
  const double a2 = sqrt(cx * cx + cy * cy + cz * cz);
  area2[t] = a2;  // |(b - a) x (c - a)|, the Jacobian of the parametrisations of T
  if (nrm) {      // outer unit normal (the orientation of the stored vertex order)
    nrm[3 * t] = cx / a2;
    nrm[3 * t + 1] = cy / a2;
    nrm[3 * t + 2] = cz / a2;
  }
  double area = 0.5 * a2;
  for (int q = 0; q < 7; ++q) {
    double l0 = rules.bary[q][0], l1 = rules.bary[q][1], l2 = rules.bary[q][2];
    tq[7 * t + q] = P4{l0 * a[0] + l1 * b[0] + l2 * c[0], l0 * a[1] + l1 * b[1] + l2 * c[1],
                       l0 * a[2] + l1 * b[2] + l2 * c[2], rules.w7[q] * area};
  }
}

// A quadrature node as float pairs (value = hi + lo) for the coupling
// entries.  The coordinates are taken relative to an origin o and the high
// parts lie on a grid of step g = 2^(E - 22), where every |x - o| < 2^E: the
// high parts are integers times g below 2^22 g, so the difference of two of
// them is exact in float; the low parts hold the rest (|lo| <= g / 2, stored
// to 2^-24 of that).  The weight is split the same way (hi = nearest float).
struct __align__(16) SplitNode {
  float4 hi;  // x, y, z, w
  float4 lo;
};

__global__ void k_split_nodes(int64_t count, const P4* __restrict__ tq, double ox, double oy, double oz,
                              double g, SplitNode* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const P4 p = tq[i];
  const double inv_g = 1.0 / g;  // g is a power of two: exact
  auto split = [&](double u, float& hi, float& lo) {
    const double h = rint(u * inv_g) * g;  // on the grid, exact in float
    hi = (float)h;
    lo = (float)(u - h);  // u - h is exact in double
  };
  SplitNode n;
  split(p.x - ox, n.hi.x, n.lo.x);
  split(p.y - oy, n.hi.y, n.lo.y);
  split(p.z - oz, n.hi.z, n.lo.z);
  n.hi.w = (float)p.w;
  n.lo.w = (float)(p.w - (double)n.hi.w);
  out[i] = n;
}

// one warp per cluster: min / max over the vertices of its triangles
__global__ void k_cluster_boxes(int nc, const int* __restrict__ begin, const int* __restrict__ end,
                                const int* __restrict__ perm, const int* __restrict__ tri,
                                const double* __restrict__ vert, double* __restrict__ box) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nc) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = begin[warp] + lane; i < end[warp]; i += 32) {
    const int t = perm[i];
    for (int a = 0; a < 3; ++a) {
      const int v = tri[3 * t + a];
      for (int d = 0; d < 3; ++d) {
        double x = vert[3 * v + d];
        lo[d] = fmin(lo[d], x);
        hi[d] = fmax(hi[d], x);
      }
    }
  }
  for (int off = 16; off; off >>= 1)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
      hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
    }
  if (lane == 0)
    for (int d = 0; d < 3; ++d) {
      box[6 * warp + d] = lo[d];
      box[6 * warp + 3 + d] = hi[d];
    }
}

// Gauss rule on the six faces of omega = box widened by margin * diam.
// Point nu = face * m^2 + a * m + b; faces -x, +x, -y, +y, -z, +z; on each
// face the lower remaining axis carries the index a.  Output (x, y, z,
// sqrt(w)) per point; the outward normal is implied by the face.
__global__ void k_box_quad(int nc, Rules rules, const double* __restrict__ box,
                           const double* __restrict__ diam, double margin,
                           P4* __restrict__ zq) {
  const int m = rules.m, k = 6 * m * m;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nc * k) return;
  const int c = idx / k, nu = idx % k;
  const int face = nu / (m * m), a = (nu / m) % m, b = nu % m;
  const int d = face >> 1, side = face & 1;
  const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
  const double delta = margin * diam[c];
  double lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    lo[e] = box[6 * c + e] - delta;
    hi[e] = box[6 * c + 3 + e] + delta;
  }
  const double mid1 = 0.5 * (lo[d1] + hi[d1]), half1 = 0.5 * (hi[d1] - lo[d1]);
  const double mid2 = 0.5 * (lo[d2] + hi[d2]), half2 = 0.5 * (hi[d2] - lo[d2]);
  double z[3];
  z[d] = side ? hi[d] : lo[d];
  z[d1] = mid1 + half1 * rules.box_t[a];
  z[d2] = mid2 + half2 * rules.box_t[b];
  const double w = rules.box_w[a] * rules.box_w[b] * half1 * half2;
  zq[idx] = P4{z[0], z[1], z[2], sqrt(w)};
}

// ------------------------------------------------------ Green matrix + ACA

struct AcaJob {
  int c;          // cluster
  int rows;       // rows of A^
  int leaf;       // rows are the cluster's triangles (1) or the children's pivots (0)
  int rmax;       // min(rows, 2k)
  int tbegin;     // leaf: first position in perm
  int r0;         // non-leaf: rank of child0 (its pivots come first)
  int mesh;       // entry of the launch's mesh table
  int kind;       // 0: Green matrix A_tau of the single layer; 1: column matrix of the double
                  // layer; 2: rows of the collocation matrix (values at the centroids);
                  // 3: rows of the nodal basis (Sect. 5)
  int64_t piv0;   // non-leaf: pivot pool offsets of the children
  int64_t piv1;
  int64_t vh_off; // V^ (rows x r, row-major) in the mesh's V^ pool
  int64_t p_off;  // this cluster's pivots in the mesh's pivot pool
  double diam;    // d_tau
};

// Per-mesh arrays of an ACA launch (one launch may serve several meshes).
struct AcaMesh {
  const int* perm;
  const P4* tq;
  const P4* zq;
  int* piv_pool;
  double* vh_pool;
  int* rank_out;
  const double* nrm;  // outer unit normals per triangle (column matrices of the double layer)
  const int* sup_ptr;   // nodal basis: support of vertex v = sup_item[sup_ptr[v] .. sup_ptr[v + 1])
  const int* sup_item;  // (triangle << 2) | corner of the vertex
  double bary[7][3];    // barycentric coordinates of the 7-point rule's nodes
  int* status;          // the mesh's sticky error bits (NaN in a Green matrix)
};

// Cross approximation of one job on a thread-block cluster of C CTAs (C = 1
// for small jobs).  CTA q owns the rows [q rpc, (q + 1) rpc) of A^ with all
// 2k columns (nu: g-column, nu + k: dg-column), row-major in shared memory,
// and the same rows of the interpolation matrix V^.  One step of the cross
// approximation with complete pivoting (Sect. 3):
//   1. the rank-one update R <- R - u v^T of the residual and the update of
//      V^ below, over the rows and columns not yet eliminated;
//   2. the CTA's largest |R| (IEEE bit patterns: an integer max is exact for
//      non-negative doubles) and, among its entries within the tie window of
//      that maximum, the smallest column-major index (column, then row);
//   3. the CTA posts maximum, candidate and the candidate's residual row and
//      V^ row into a double-buffered slot of its shared memory; one cluster
//      barrier;
//   4. every CTA reads all posts through distributed shared memory: the
//      cluster maximum (stopping rule), the tie threshold and the winning
//      candidate, whose posted rows give the pivot row v and w = V^[i*, :].
//      The entries of a CTA within the cluster's tie window are a subset of
//      those within its own, so its posted candidate is its answer whenever
//      the candidate itself lies in the cluster's window; otherwise (a near
//      tie straddling two CTAs' windows) one more round rescans at the
//      cluster's threshold;
//   5. u = R[:, j*] / p for the CTA's rows still in play; the pivot row and
//      column leave the active region (swapped to its end, with the maps
//      from storage positions to row and column indices of A^).
// The pivot row and column of the residual are zero after their step (up to
// rounding in an implementation that keeps updating them), so they never
// hold a later pivot: the update skips them, which roughly halves its
// float64 work.  V^ = A^[:, Q] A^[P, Q]^{-1} = U L^{-1} is kept up to date
// instead of being solved at the end: with pivot row i* and u = R[:, j*] / p,
//   V^ <- [V^ - u V^[i*, :], u],
// since the new unit lower triangular factor's inverse adds the row
// -U[i*, :] L^{-1} = -V^[i*, :]; so V^[P, :] = I exactly, and a pivot row's
// V^ row is final when it leaves the active region.
constexpr int kAcaPosts = 3;   // two alternating posts per step, one for rescans
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

struct AcaPost {
  unsigned long long maxbits;  // the CTA's largest |R|
  unsigned long long candbits; // |R| of its candidate
  int key;                     // candidate's column-major index j * rows + i in A^ (INT_MAX: none)
  int tri;                     // candidate row's triangle id
  double pval;                 // candidate's signed value
  int cslot;                   // candidate's column storage position (the same in every CTA)
  int rslot;                   // candidate's row storage position in the posting CTA
  int bad;                     // the candidate could not be certified (rescan)
  int pad;
};
constexpr int kAcaMaxCluster = 16;

// candidate rows posted by a CTA (residual row, then V^ row); the headers go
// to every CTA of the cluster
__host__ __device__ constexpr size_t aca_post_doubles(int k2, int rmax_cap) {
  return (size_t)k2 + (size_t)rmax_cap;
}

// Summary of a set of residual entries for complete pivoting with a tie
// window: its largest |R| (bits m), and the smallest key k among its entries
// with |R| >= m (1 - tie), with that entry's |R| (bits v).  For any threshold
// T >= m (1 - tie) the set's entries at or above T are a subset of those at
// its own window, so k is their smallest key whenever v >= T; otherwise the
// summary cannot answer (bad) and the entries are scanned again.  Merging two
// summaries applies this to both sides at the merged window.
struct Cand {
  unsigned long long m, k, v;
  int bad;
};
__device__ __forceinline__ unsigned long long tie_bits(unsigned long long m, double keep) {
  return m > kInfBits ? m : (unsigned long long)__double_as_longlong(__longlong_as_double((long long)m) * keep);
}
__device__ __forceinline__ Cand cand_merge(const Cand& a, const Cand& b, double keep) {
  Cand o;
  o.m = a.m > b.m ? a.m : b.m;
  o.k = ~0ull;
  o.v = 0;
  o.bad = 0;
  const unsigned long long thr = tie_bits(o.m, keep);
  if (a.m >= thr) {
    if (a.bad || a.v < thr) o.bad = 1;
    else if (a.k < o.k) { o.k = a.k; o.v = a.v; }
  }
  if (b.m >= thr) {
    if (b.bad || b.v < thr) o.bad = 1;
    else if (b.k < o.k) { o.k = b.k; o.v = b.v; }
  }
  return o;
}
__device__ __forceinline__ Cand cand_shfl(const Cand& a, int off) {
  Cand o;
  o.m = __shfl_xor_sync(0xffffffffu, a.m, off);
  o.k = __shfl_xor_sync(0xffffffffu, a.k, off);
  o.v = __shfl_xor_sync(0xffffffffu, a.v, off);
  o.bad = __shfl_xor_sync(0xffffffffu, a.bad, off);
  return o;
}

// shared memory of one CTA: residual rows, posts, u, v, w, the rows'
// triangles and indices, the columns' indices and the pivots' triangles
// (V^ of the rows lives in a global scratch array of the launch)
__host__ __device__ constexpr size_t aca_smem_bytes(int rpc_cap, int k2, int rmax_cap) {
  return sizeof(double) * ((size_t)rpc_cap * k2 +
                           kAcaPosts * aca_post_doubles(k2, rmax_cap) + rpc_cap + k2 + rmax_cap) +
         sizeof(int) * (2 * (size_t)rpc_cap + k2 + rmax_cap);
}


__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  for (int off = 16; off; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o < v ? o : v;
  }
  return v;
}
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & kAbsMask;
}

// LC: columns of a lane in the row updates (2k <= 32 LC)
template <int LC, int NT>
__global__ void __launch_bounds__(NT)
k_aca(const AcaJob* __restrict__ jobs, const AcaMesh* __restrict__ meshes, int k, int rpc_cap, int rmax_cap,
      double tol, double tie, double* __restrict__ wbuf) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const AcaJob job = jobs[blockIdx.x / C];
  const AcaMesh M = meshes[job.mesh];
  const int rows = job.rows, k2 = 2 * k;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wid = tid >> 5, nwarps = nth >> 5;
  const int rpc = (rows + C - 1) / C;
  const int row0 = q * rpc;
  const int nr = max(0, min(rpc, rows - row0));  // rows of this CTA

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);            // nr x k2, row-major (storage order)
  // V^ of the CTA's rows (nr x rmax, row-major) in global memory: shared
  // memory holds the residual rows only, so that two CTAs fit on an SM
  double* W = wbuf + (size_t)blockIdx.x * rpc_cap * rmax_cap;
  double* posts = S + (size_t)rpc_cap * k2;                   // kAcaPosts x post
  double* s_u = posts + kAcaPosts * aca_post_doubles(k2, rmax_cap);  // rpc_cap
  double* s_v = s_u + rpc_cap;                                // k2
  double* s_w = s_v + k2;                                     // rmax_cap
  int* s_tri = reinterpret_cast<int*>(s_w + rmax_cap);         // rpc_cap: triangle of each stored row
  int* s_rid = s_tri + rpc_cap;                               // rpc_cap: row of A^ of each stored row
  int* s_cid = s_rid + rpc_cap;                               // k2: column of A^ of each stored column
  int* s_ptri = s_cid + k2;                                   // rmax_cap: pivots' triangles
  __shared__ unsigned long long s_red[32];
  __shared__ unsigned long long s_bcast;
  __shared__ Cand s_cand[32];
  __shared__ AcaPost s_hdr[kAcaPosts][kAcaMaxCluster];  // every CTA's header, pushed by its owner
  const size_t post_stride = aca_post_doubles(k2, rmax_cap);
  auto post_row = [&](double* base, int b) { return base + b * post_stride; };
  const double keep = 1.0 - tie;

  for (int i = tid; i < nr; i += nth) {
    const int g = row0 + i;
    s_tri[i] = job.leaf ? M.perm[job.tbegin + g]
                        : (g < job.r0 ? M.piv_pool[job.piv0 + g] : M.piv_pool[job.piv1 + (g - job.r0)]);
    s_rid[i] = g;
  }
  for (int c = tid; c < k2; c += nth) s_cid[c] = c;
  __syncthreads();

  // own rows of A^ (Sect. 2): columns nu (g) and nu + k (dg) for every box point
  const P4* z = M.zq + (int64_t)job.c * k;
  const int m2 = k / 6;
  for (int idx = tid; idx < nr * k; idx += nth) {
    const int i = idx / k, nu = idx - i * k;
    const P4 zz = z[nu];
    const int face = nu / m2, d = face >> 1;
    const double sgn = (face & 1) ? 1.0 : -1.0;
    const P4* xq = M.tq + 7 * (int64_t)s_tri[i];
    double gs = 0.0, ds = 0.0;
    if (job.kind == 0) {
      // a_{i nu} = sqrt(w) int g(x, z) phi_i, a_{i nu+k} = -d sqrt(w) int dg/dn_z(x, z) phi_i
#pragma unroll
      for (int qq = 0; qq < 7; ++qq) {
        const P4 x = xq[qq];
        const double dx = x.x - zz.x, dy = x.y - zz.y, dz = x.z - zz.z;
        const double ir = rsqrt(dx * dx + dy * dy + dz * dz);
        const double dn = sgn * (d == 0 ? dx : (d == 1 ? dy : dz));
        gs += x.w * ir;
        ds += x.w * dn * ir * ir * ir;
      }
    } else if (job.kind == 3) {
      // nodal rows (Sect. 5): the 7-point rule on every triangle of the
      // vertex's support, each node weighted by the barycentric coordinate of
      // the vertex's corner
      const int v = s_tri[i];
      for (int e = M.sup_ptr[v]; e < M.sup_ptr[v + 1]; ++e) {
        const int it = M.sup_item[e], cn = it & 3;
        const P4* xt = M.tq + 7 * (int64_t)(it >> 2);
#pragma unroll
        for (int qq = 0; qq < 7; ++qq) {
          const P4 x = xt[qq];
          const double wl = x.w * M.bary[qq][cn];
          const double dx = x.x - zz.x, dy = x.y - zz.y, dz = x.z - zz.z;
          const double ir = rsqrt(dx * dx + dy * dy + dz * dz);
          const double dn = sgn * (d == 0 ? dx : (d == 1 ? dy : dz));
          gs += wl * ir;
          ds += wl * dn * ir * ir * ir;
        }
      }
    } else if (job.kind == 2) {
      // collocation rows: a_{i nu} = sqrt(w) g(x_i, z), a_{i nu+k} = -d sqrt(w)
      // dg/dn_z(x_i, z) at the centroid x_i (the 7-point rule's centre)
      const P4 x = xq[0];
      const double dx = x.x - zz.x, dy = x.y - zz.y, dz = x.z - zz.z;
      const double ir = rsqrt(dx * dx + dy * dy + dz * dz);
      const double dn = sgn * (d == 0 ? dx : (d == 1 ? dy : dz));
      gs = ir;
      ds = dn * ir * ir * ir;
    } else {
      // the double layer's column matrix: a'_{j nu} = sqrt(w) int dg/dn_y(y, z) phi_j,
      // a'_{j nu+k} = -d sqrt(w) int d2g/dn_y dn_z(y, z) phi_j, with e = z - y,
      // dg/dn_y = <n_y, e> / (4 pi r^3), d2g = (<n_y, n_z> / r^3 - 3 <n_y, e> <n_z, e> / r^5) / (4 pi)
      const double* ny = M.nrm + 3 * (int64_t)s_tri[i];
      const double n0 = ny[0], n1 = ny[1], n2 = ny[2];
      const double nn = sgn * (d == 0 ? n0 : (d == 1 ? n1 : n2));
#pragma unroll
      for (int qq = 0; qq < 7; ++qq) {
        const P4 y = xq[qq];
        const double ex = zz.x - y.x, ey = zz.y - y.y, ez = zz.z - y.z;
        const double ir = rsqrt(ex * ex + ey * ey + ez * ez);
        const double ir3 = ir * ir * ir;
        const double nye = n0 * ex + n1 * ey + n2 * ez;
        const double nze = sgn * (d == 0 ? ex : (d == 1 ? ey : ez));
        gs += y.w * nye * ir3;
        ds += y.w * (nn - 3.0 * nye * nze * ir * ir) * ir3;
      }
    }
    S[(int64_t)i * k2 + nu] = zz.w * gs * kInv4Pi;
    S[(int64_t)i * k2 + k + nu] = -job.diam * zz.w * ds * kInv4Pi;
  }
  __syncthreads();

  // block-wide reductions (every thread gets the result)
  auto block_min = [&](unsigned long long v) {
    v = warp_min_u64(v);
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (wid == 0) {
      unsigned long long m = lane < nwarps ? s_red[lane] : ~0ull;
      m = warp_min_u64(m);
      if (lane == 0) s_bcast = m;
    }
    __syncthreads();
    return s_bcast;
  };
  auto block_cand = [&](Cand c) {
    for (int off = 16; off; off >>= 1) c = cand_merge(c, cand_shfl(c, off), keep);
    if (lane == 0) s_cand[wid] = c;
    __syncthreads();
    Cand o = s_cand[0];
    for (int w = 1; w < nwarps; ++w) o = cand_merge(o, s_cand[w], keep);
    __syncthreads();
    return o;
  };
  // smallest (key << 32 | storage position) over the active entries with
  // |R| >= thr; one warp per row, the lanes over the columns
  int na = nr, nca = k2;
  auto find_key = [&](unsigned long long thr) {
    unsigned long long best = ~0ull;
    int cid[LC];
#pragma unroll
    for (int m = 0; m < LC; ++m) cid[m] = lane + 32 * m < nca ? s_cid[lane + 32 * m] : 0;
    for (int i = wid; i < na; i += nwarps) {
      const double* Sr = S + (int64_t)i * k2;
      const int rid = s_rid[i];
#pragma unroll
      for (int m = 0; m < LC; ++m) {
        const int c = lane + 32 * m;
        if (c < nca && abs_bits(Sr[c]) >= thr) {
          const unsigned long long kk =
              ((unsigned long long)(cid[m] * rows + rid) << 32) | (unsigned)(i * k2 + c);
          best = kk < best ? kk : best;
        }
      }
    }
    return block_min(best);
  };
  // post the CTA's summary into slot b: the candidate's residual and V^ rows
  // stay in this CTA; the header goes to every CTA of the cluster
  auto post = [&](int b, const Cand& cd, int r) {
    double* prow = post_row(posts, b);
    const bool has = cd.k != ~0ull && !cd.bad;
    const int pos = has ? (int)(cd.k & 0xffffffffu) : 0;
    const int i = pos / k2, c = pos - (pos / k2) * k2;
    if (has) {
      for (int cc = tid; cc < nca; cc += nth) prow[cc] = S[(int64_t)i * k2 + cc];
      for (int cc = tid; cc < r; cc += nth) prow[k2 + cc] = W[(int64_t)i * rmax_cap + cc];
    }
    if (tid < C) {
      AcaPost h;
      h.maxbits = cd.m;
      h.bad = cd.bad;
      h.pad = 0;
      if (has) {
        const double pv = S[(int64_t)i * k2 + c];
        h.candbits = abs_bits(pv);
        h.key = (int)(cd.k >> 32);
        h.pval = pv;
        h.tri = s_tri[i];
        h.cslot = c;
        h.rslot = i;
      } else {
        h.candbits = 0;
        h.key = INT_MAX;
        h.pval = 0.0;
        h.tri = -1;
        h.cslot = -1;
        h.rslot = -1;
      }
      *cluster.map_shared_rank(&s_hdr[b][q], tid) = h;
    }
  };

  int r = 0;
  double first = 0.0;
  int jslot = -1, islot = -1;  // storage positions of the last pivot's column and (owner) row
  bool own = false;            // this CTA holds the last pivot row
  for (;;) {
    Cand cd{0, ~0ull, 0, 0};        // this lane's running summary
    unsigned long long wthr = 0;    // its window threshold
    if (r > 0) {
      const int t = r - 1;
      // the pivot column leaves the active region: swap it with the last
      // active column (every CTA; the same positions everywhere)
      const int cl = nca - 1;
      if (jslot != cl) {
        for (int i = tid; i < na; i += nth) {
          double* Sr = S + (int64_t)i * k2;
          const double a = Sr[jslot];
          Sr[jslot] = Sr[cl];
          Sr[cl] = a;
        }
        if (tid == 0) {
          const double a = s_v[jslot];
          s_v[jslot] = s_v[cl];
          s_v[cl] = a;
          const int b = s_cid[jslot];
          s_cid[jslot] = s_cid[cl];
          s_cid[cl] = b;
        }
      }
      __syncthreads();
      nca = cl;
      if (own) {
        // the pivot row leaves too: swap with the last active row; its V^ row
        // becomes the unit vector e_t
        const int rl = na - 1;
        if (islot != rl) {
          double* A = S + (int64_t)islot * k2;
          double* B = S + (int64_t)rl * k2;
          for (int c = tid; c < nca; c += nth) {
            const double a = A[c];
            A[c] = B[c];
            B[c] = a;
          }
          double* WA = W + (int64_t)islot * rmax_cap;
          double* WB = W + (int64_t)rl * rmax_cap;
          for (int c = tid; c < t; c += nth) WA[c] = WB[c];
          if (tid == 0) {
            s_u[islot] = s_u[rl];
            const int a = s_tri[islot];
            s_tri[islot] = s_tri[rl];
            s_tri[rl] = a;
            const int b = s_rid[islot];
            s_rid[islot] = s_rid[rl];
            s_rid[rl] = b;
          }
        }
        __syncthreads();
        double* WB = W + (int64_t)rl * rmax_cap;
        for (int c = tid; c < job.rmax; c += nth) WB[c] = c == t ? 1.0 : 0.0;
        na = rl;
      }
      // V^ and residual of the active rows, one warp per row: lane columns
      // lane + 32 m of w and v in registers
      double wr[LC], vr[LC];
#pragma unroll
      for (int m = 0; m < LC; ++m) {
        const int c = lane + 32 * m;
        wr[m] = c < t ? s_w[c] : 0.0;
        vr[m] = c < nca ? s_v[c] : 0.0;
      }
      const bool last = r == job.rmax;
      int cid[LC];
#pragma unroll
      for (int m = 0; m < LC; ++m) cid[m] = lane + 32 * m < nca ? s_cid[lane + 32 * m] : 0;
      for (int i = wid; i < na; i += nwarps) {
        const double ui = s_u[i];
        double* Wr = W + (int64_t)i * rmax_cap;
#pragma unroll
        for (int m = 0; m < LC; ++m) {
          const int c = lane + 32 * m;
          if (c < t) Wr[c] = fma(-ui, wr[m], Wr[c]);
        }
        if (lane == 0) Wr[t] = ui;
        if (last) continue;
        double* Sr = S + (int64_t)i * k2;
        const unsigned long long rk = (unsigned long long)s_rid[i];
#pragma unroll
        for (int m = 0; m < LC; ++m) {
          const int c = lane + 32 * m;
          if (c < nca) {
            const double val = fma(-ui, vr[m], Sr[c]);
            Sr[c] = val;
            // running summary of this lane's entries (a new maximum resets
            // the window; a rise within the window keeps a certified key)
            const unsigned long long b = abs_bits(val);
            const unsigned long long key =
                ((unsigned long long)cid[m] * rows + rk) << 32 | (unsigned)(i * k2 + c);
            if (b > cd.m) {
              const unsigned long long thr = tie_bits(b, keep);
              if (cd.m >= thr && (cd.bad || cd.v < thr)) cd.bad = 1;
              if (cd.m < thr || cd.bad) {
                cd.k = key;
                cd.v = b;
              } else if (key < cd.k) {
                cd.k = key;
                cd.v = b;
              }
              cd.m = b;
              wthr = thr;
            } else if (b >= wthr && key < cd.k) {
              cd.k = key;
              cd.v = b;
            }
          }
        }
      }
      if (last) break;
    } else {
      for (int i = wid; i < na; i += nwarps)
        for (int c = lane; c < nca; c += 32) {
          const unsigned long long b = abs_bits(S[(int64_t)i * k2 + c]);
          const unsigned long long key = ((unsigned long long)c * rows + s_rid[i]) << 32 | (unsigned)(i * k2 + c);
          if (b > cd.m) {
            const unsigned long long thr = tie_bits(b, keep);
            if (cd.m >= thr && (cd.bad || cd.v < thr)) cd.bad = 1;
            if (cd.m < thr || cd.bad) {
              cd.k = key;
              cd.v = b;
            } else if (key < cd.k) {
              cd.k = key;
              cd.v = b;
            }
            cd.m = b;
            wthr = thr;
          } else if (b >= wthr && key < cd.k) {
            cd.k = key;
            cd.v = b;
          }
        }
    }
    Cand cc = block_cand(cd);
    if (cc.bad && cc.m <= kInfBits) {
      // a near tie the running summaries could not certify: scan again
      const unsigned long long kp = find_key(tie_bits(cc.m, keep));
      cc.k = kp;
      cc.v = kp == ~0ull ? 0 : abs_bits(S[kp & 0xffffffffu]);
      cc.bad = 0;
    }
    const int slot = r & 1;
    post(slot, cc, r);
    __syncthreads();
    cluster.sync();
    // every warp takes the same decision from the same headers (lane p holds
    // CTA p's)
    Cand g{0, ~0ull, 0, 0};
    if (lane < C) {
      const AcaPost& h = s_hdr[slot][lane];
      g.m = h.maxbits;
      g.k = h.key == INT_MAX ? ~0ull : (unsigned long long)h.key;
      g.v = h.candbits;
      g.bad = h.bad;
    }
    for (int off = 16; off; off >>= 1) g = cand_merge(g, cand_shfl(g, off), keep);
    const unsigned long long gmax = g.m;
    if (gmax > kInfBits) {
      if (tid == 0 && q == 0) atomicOr(M.status, kStatusNumeric);
      break;
    }
    const double big = __longlong_as_double((long long)gmax);
    if (r == 0) first = big;
    if (big == 0.0 || (r > 0 && big <= tol * first)) break;
    int pslot = slot;
    unsigned long long kk = g.k;
    if (g.bad) {
      // a CTA's own window held a candidate outside the cluster's window:
      // every CTA posts its smallest key at the cluster's threshold
      const unsigned long long thr = tie_bits(gmax, keep);
      Cand c2{cc.m, ~0ull, 0, 0};
      if (cc.m >= thr) {
        c2.k = find_key(thr);
        c2.v = c2.k == ~0ull ? 0 : abs_bits(S[c2.k & 0xffffffffu]);
      }
      post(2, c2, r);
      __syncthreads();
      cluster.sync();
      unsigned long long k2s = ~0ull;
      if (lane < C && s_hdr[2][lane].key != INT_MAX) k2s = (unsigned long long)s_hdr[2][lane].key;
      kk = warp_min_u64(k2s);
      pslot = 2;
    }
    const int owner = __ffs(__ballot_sync(0xffffffffu, lane < C && s_hdr[pslot][lane].key == (int)kk)) - 1;
    // the pivot row v, w = V^[i*, :] and p from the winner's post; u for the
    // CTA's active rows
    const AcaPost* wh = &s_hdr[pslot][owner];
    const double* wrow = post_row(cluster.map_shared_rank(posts, owner), pslot);
    const double p = wh->pval;
    jslot = wh->cslot;
    own = owner == q;
    islot = own ? wh->rslot : -1;
    for (int c = tid; c < nca; c += nth) s_v[c] = wrow[c];
    for (int c = tid; c < r; c += nth) s_w[c] = wrow[k2 + c];
    for (int i = tid; i < na; i += nth) s_u[i] = S[(int64_t)i * k2 + jslot] / p;
    if (tid == 0) s_ptri[r] = wh->tri;
    ++r;
    __syncthreads();
  }
  cluster.sync();  // no CTA still reads a peer's posts
  // V^ (rows x r, row-major by row of A^) and the pivots' triangles in
  // selection order
  double* Vh = M.vh_pool + job.vh_off;
  for (int i = wid; i < nr; i += nwarps) {
    const double* Wr = W + (int64_t)i * rmax_cap;
    double* out = Vh + (int64_t)s_rid[i] * r;
    for (int c = lane; c < r; c += 32) out[c] = Wr[c];
  }
  if (q == 0) {
    for (int t = tid; t < r; t += nth) M.piv_pool[job.p_off + t] = s_ptri[t];
    if (tid == 0) M.rank_out[job.c] = r;
  }
}

// --------------------------------------------------------------- packing

struct Segment {
  int64_t src;
  int64_t dst;
  int64_t len;
};

__global__ void k_pack(const Segment* __restrict__ seg, const double* __restrict__ src,
                       double* __restrict__ d64) {
  const Segment s = seg[blockIdx.x];
  for (int64_t i = threadIdx.x; i < s.len; i += blockDim.x) d64[s.dst + i] = src[s.src + i];
}

}  // namespace

// Row-major float64 blocks -> panel layout (panel.cuh) in float64, float32
// and (optionally) bfloat16; one CTA per block.  With `trans` the panel
// holds the transposed block (m x k panel of a k x m row-major source).
struct PanelJob {
  int64_t src;
  int64_t dst;
  int m;
  int k;
  int trans;
  int pad;
};

// Tiled panel layout of one M x K block (K_pad = pad8(K)): row slices of
// kTileRows rows, each slice split into column chunks of kTileCols columns,
// every (slice, chunk) tile stored contiguously as column panels of P
// entries per row.  Tile (a0, k0) with ms = min(kTileRows, M - a0) rows
// starts at element a0 * K_pad + ms * k0; inside it entry (a, kk) sits at
// (kk / P) * ms * P + a * P + kk % P.  A product segment is one tile, so it
// moves with one contiguous copy.
constexpr int kTileRows = 64, kTileCols = 64;

// Element d of the panel layout of an m x kp block, split into the parts
// that do not depend on the panel width P: its tile's first row and column,
// the tile's row count ms and the offset f inside the tile.  Block-local
// indices stay below 2^31, so 32-bit division suffices.
struct TilePos {
  int row0, col0, ms, f;
};

__device__ __forceinline__ TilePos tile_pos(int m, int kp, int d) {
  const int slice = kTileRows * kp;
  const int i = d / slice;
  const int e = d - i * slice;
  const int ms = min(kTileRows, m - i * kTileRows);
  const int tile = ms * kTileCols;
  const int j = e / tile;
  return TilePos{i * kTileRows, j * kTileCols, ms, e - j * tile};
}

// (row, column) of the entry at offset f of a tile with ms rows and panels of
// P = 2^lgp entries per row
__device__ __forceinline__ void tile_entry(const TilePos& t, int lgp, int& row, int& col) {
  const int mp = t.ms << lgp;
  const int p = t.f / mp, g = t.f - p * mp;
  row = t.row0 + (g >> lgp);
  col = t.col0 + (p << lgp) + (g & ((1 << lgp) - 1));
}

__global__ void k_to_panel(const PanelJob* __restrict__ jobs, const double* __restrict__ src,
                           double* __restrict__ d64, float* __restrict__ d32,
                           __nv_bfloat16* __restrict__ d16) {
  const PanelJob j = jobs[blockIdx.x];
  const int kp = pad8(j.k);
  const int total = j.m * kp;
  auto at = [&](int a, int kk) -> double {
    if (kk >= j.k) return 0.0;
    return j.trans ? src[j.src + (int64_t)kk * j.m + a] : src[j.src + (int64_t)a * j.k + kk];
  };
  for (int d = threadIdx.x; d < total; d += blockDim.x) {
    const TilePos t = tile_pos(j.m, kp, d);
    int a, kk;
    if (d64) {
      tile_entry(t, 1, a, kk);
      d64[j.dst + d] = at(a, kk);
    }
    if (d32) {
      tile_entry(t, 2, a, kk);
      d32[j.dst + d] = (float)at(a, kk);
    }
    if (d16) {
      tile_entry(t, 3, a, kk);
      d16[j.dst + d] = __double2bfloat16(at(a, kk));
    }
  }
}

// Row-major float64 blocks back from the float64 panels (the inverse of
// k_to_panel on an untransposed kind, panels of P = 2): one CTA per block.
__global__ void k_from_panel(const PanelJob* __restrict__ jobs, const double* __restrict__ p64,
                             double* __restrict__ dst) {
  const PanelJob j = jobs[blockIdx.x];
  const int kp = pad8(j.k);
  const int total = j.m * kp;
  for (int d = threadIdx.x; d < total; d += blockDim.x) {
    const TilePos t = tile_pos(j.m, kp, d);
    int a, kk;
    tile_entry(t, 1, a, kk);
    if (kk < j.k) dst[j.dst + (int64_t)a * j.k + kk] = p64[j.src + d];
  }
}

// Does every block (t[b], s[b]) of a list have its mirror (s[b], t[b]) in
// the list?  If so, mir[b] = index of the mirror.
bool blocks_mirrored(const std::vector<int>& t, const std::vector<int>& s, std::vector<int>& mir) {
  const size_t n = t.size();
  std::vector<std::pair<std::pair<int, int>, int>> a(n);
  for (size_t i = 0; i < n; ++i) a[i] = {{t[i], s[i]}, (int)i};
  std::sort(a.begin(), a.end());
  mir.assign(n, -1);
  for (size_t i = 0; i < n; ++i) {
    const std::pair<int, int> want{s[i], t[i]};
    auto it = std::lower_bound(a.begin(), a.end(), std::make_pair(want, INT_MIN));
    if (it == a.end() || it->first != want) return false;
    mir[i] = it->second;
  }
  return true;
}

// Every stored block in panel form: f(kind, index, rows, columns, transposed)
// for V, V^T, E, E^T, S, S^T, N, N^T (index PanelKind), in storage order.
// A mirrored handle stores no S^T; its N^T array holds, at block b's
// offset, N_{mirror(b)}^T (the shape of N_b), read by the product's own plan
// in the transposed product.
template <typename F>
void for_each_panel(const gca_h2* h, F&& f) {
  const int nc = h->nc;
  const int nfar = (int)h->far_t.size(), nnear = (int)h->near_t.size();
  const bool single = h->single_level();  // bases of every cluster, no transfers
  for (int c = 1; c < nc; ++c) {
    if (h->child0[c] < 0 || single) {
      const int nr = h->end[c] - h->begin[c], r = h->rank[c];
      f(kV, c, nr, r, 0);
      f(kVt, c, r, nr, 1);
    }
    if (h->parent[c] > 0 && !single) {
      const int r = h->rank[c], rp = h->rank[h->parent[c]];
      f(kE, c, r, rp, 0);
      f(kEt, c, rp, r, 1);
    }
  }
  for (int b = 0; b < nfar; ++b) {
    const int rt = h->rank[h->far_t[b]];
    // r'_sigma (column bases), r_sigma, or |sigma-hat| (Green quadrature: B^*)
    const int rs = h->two_sided() ? h->rank2[h->far_s[b]]
                   : h->op == 4   ? h->end[h->far_s[b]] - h->begin[h->far_s[b]]
                                  : h->rank[h->far_s[b]];
    f(kS, b, rt, rs, 0);
    if (!h->mirrored) f(kSt, b, rs, rt, 1);
  }
  for (int b = 0; b < nnear; ++b) {
    const int t = h->near_t[b], s = h->near_s[b];
    const int mt = h->end[t] - h->begin[t], ms = h->end[s] - h->begin[s];
    f(kN, b, mt, ms, 0);
    if (h->mirrored)
      f(kNt, b, mt, ms, 1);
    else
      f(kNt, b, ms, mt, 1);
  }
  if (!h->two_sided()) return;
  // column bases W and transfers F (their own ranks r')
  for (int c = 1; c < nc; ++c) {
    if (h->child0[c] < 0) {
      const int nr = h->end[c] - h->begin[c], r = h->rank2[c];
      f(kW, c, nr, r, 0);
      f(kWt, c, r, nr, 1);
    }
    if (h->parent[c] > 0) {
      const int r = h->rank2[c], rp = h->rank2[h->parent[c]];
      f(kF, c, r, rp, 0);
      f(kFt, c, rp, r, 1);
    }
  }
}

// Element offsets of every block in its panel array (the same for all
// precisions) and the array sizes; needs only the ranks and block lists.
void layout_panels(gca_h2* h) {
  const int nc = h->nc;
  const int nfar = (int)h->far_t.size(), nnear = (int)h->near_t.size();
  const int count[kPanelKinds] = {nc, nc, nc, nc, nfar, nfar, nnear, nnear, nc, nc, nc, nc};
  for (int q = 0; q < kPanelKinds; ++q) {
    h->panel_off[q].assign(count[q], -1);
    h->psize[q] = 0;
  }
  for_each_panel(h, [&](int kind, int idx, int m, int k, int) {
    h->panel_off[kind][idx] = h->psize[kind];
    h->psize[kind] += (int64_t)m * pad8(k);
  });
}

// Which precisions of panel kind q a handle keeps (the float32 near field
// also serves the bfloat16 products).
void panel_precisions(const gca_h2* h, int q, bool& k64, bool& k32, bool& k16) {
  const uint32_t fl = h->params.flags;
  const bool near = q == kN || q == kNt;
  k64 = !(fl & GCA_DROP_F64);
  k32 = !(fl & GCA_DROP_F32) || (near && !(fl & GCA_DROP_BF16));
  k16 = !near && !(fl & GCA_DROP_BF16);
}

// Device arrays of the panels at the sizes of layout_panels.
int alloc_panels(gca_h2* h) {
  for (int q = 0; q < kPanelKinds; ++q) {
    bool k64, k32, k16;
    panel_precisions(h, q, k64, k32, k16);
    if (k64) GCA_TRY(h->P64[q].alloc(sizeof(double) * h->psize[q]));
    if (k32) GCA_TRY(h->P32[q].alloc(sizeof(float) * h->psize[q]));
    if (k16) GCA_TRY(h->P16[q].alloc(sizeof(__nv_bfloat16) * h->psize[q]));
  }
  return GCA_OK;
}

// Number of panel jobs of make_panels (the size of its job buffer).
int64_t panel_jobs(const gca_h2* h) {
  int64_t n = 0;
  for_each_panel(h, [&](int, int, int, int, int) { ++n; });
  return n;
}

// Panels of all stored blocks from the row-major float64 coefficients, at the
// offsets of layout_panels, into the arrays of alloc_panels.  `jobs_buf`
// holds at least panel_jobs(h) jobs; `host_jobs` receives their host copy
// and must outlive the next synchronisation of the stream (the launches are
// asynchronous).
int make_panels(gca_h2* h, DevMem& jobs_buf, std::vector<PanelJob>& host_jobs, cudaStream_t st) {
  int64_t first[kPanelKinds + 1] = {0};
  host_jobs.clear();
  for (int q = 0; q < kPanelKinds; ++q) {
    for_each_panel(h, [&](int kind, int idx, int m, int k, int trans) {
      if (kind != q) return;
      const int64_t src = (kind == kV || kind == kVt)   ? h->voff[idx]
                          : (kind == kE || kind == kEt) ? h->eoff[idx]
                          : (kind == kS || kind == kSt) ? h->soff[idx]
                          : kind == kN                  ? h->noff[idx]
                          : kind == kNt ? h->noff[h->mirrored ? h->near_mirror[idx] : idx]
                          : (kind == kW || kind == kWt) ? h->voff2[idx]
                                                        : h->eoff2[idx];
      host_jobs.push_back({src, h->panel_off[kind][idx], m, k, trans, 0});
    });
    first[q + 1] = (int64_t)host_jobs.size();
  }
  if (host_jobs.size() * sizeof(PanelJob) > jobs_buf.bytes) {
    set_error("internal: panel job buffer too small");
    return GCA_ERR_UNSUPPORTED;
  }
  if (host_jobs.empty()) return GCA_OK;
  GCA_TRY_CUDA(cudaMemcpyAsync(jobs_buf.p, host_jobs.data(), sizeof(PanelJob) * host_jobs.size(),
                               cudaMemcpyHostToDevice, st));
  const DevMem* srcs[kPanelKinds] = {&h->V64, &h->V64, &h->E64, &h->E64, &h->S64, &h->S64,
                                     &h->N64, &h->N64, &h->W64, &h->W64, &h->F64, &h->F64};
  for (int q = 0; q < kPanelKinds; ++q) {
    bool k64, k32, k16;
    panel_precisions(h, q, k64, k32, k16);
    const int64_t cnt = first[q + 1] - first[q];
    if (cnt == 0 || !(k64 || k32 || k16)) continue;
    k_to_panel<<<(unsigned)cnt, 256, 0, st>>>(
        jobs_buf.as<PanelJob>() + first[q], srcs[q]->as<double>(), k64 ? h->P64[q].as<double>() : nullptr,
        k32 ? h->P32[q].as<float>() : nullptr, k16 ? h->P16[q].as<__nv_bfloat16>() : nullptr);
    GCA_TRY_CUDA(cudaGetLastError());
  }
  return GCA_OK;
}

// The row-major float64 coefficients of panel kind q (kV, kE, kS, kN, kW or
// kF) in the export layout, rebuilt from the float64 panels into the host
// array `host` of n doubles.  Synchronous; allocates a device buffer of n
// doubles for the call.
int export_from_panels(const gca_h2* h, int q, double* host, int64_t n) {
  if (n <= 0) return GCA_OK;
  if (!h->P64[q].p) {
    set_error("gca_h2_export: no float64 panels and no row-major copy (GCA_DROP_F64)");
    return GCA_ERR_UNSUPPORTED;
  }
  std::vector<PanelJob> jobs;
  for_each_panel(h, [&](int kind, int idx, int m, int k, int) {
    if (kind != q || (int64_t)m * k == 0) return;
    const int64_t off = q == kV ? h->voff[idx]
                        : q == kE ? h->eoff[idx]
                        : q == kS ? h->soff[idx]
                        : q == kN ? h->noff[idx]
                        : q == kW ? h->voff2[idx]
                                  : h->eoff2[idx];
    jobs.push_back(PanelJob{h->panel_off[q][idx], off, m, k, 0, 0});
  });
  DevMem d_jobs, d_out;
  GCA_TRY(upload(d_jobs, jobs, 0));
  GCA_TRY(d_out.alloc(sizeof(double) * (size_t)n));
  if (!jobs.empty()) {
    k_from_panel<<<(unsigned)jobs.size(), 256>>>(d_jobs.as<PanelJob>(), h->P64[q].as<double>(), d_out.as<double>());
    GCA_TRY_CUDA(cudaGetLastError());
  }
  GCA_TRY_CUDA(cudaMemcpy(host, d_out.p, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
  return GCA_OK;
}

// Panels of every stored block, synchronously (the imported handles, which
// have no entry kernels to overlap with).
int make_panels_sync(gca_h2* h, cudaStream_t st) {
  DevMem jobs;
  GCA_TRY(jobs.alloc(sizeof(PanelJob) * (size_t)std::max<int64_t>(panel_jobs(h), 1)));
  std::vector<PanelJob> host_jobs;
  GCA_TRY(make_panels(h, jobs, host_jobs, st));
  GCA_TRY_CUDA(cudaStreamSynchronize(st));
  return GCA_OK;
}

namespace {

// ------------------------------------------------------ regular entries

// 7 x 7 rule: sum_p sum_q w_p w_q / (4 pi |x_p - y_q|)
__device__ __forceinline__ double regular_entry(const P4* __restrict__ xq,
                                                const P4* __restrict__ yq) {
  double s = 0.0;
#pragma unroll
  for (int p = 0; p < 7; ++p) {
    const P4 x = xq[p];
    double sp = 0.0;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const P4 y = yq[q];
      const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
      sp += y.w * rsqrt(dx * dx + dy * dy + dz * dz);
    }
    s += x.w * sp;
  }
  return s * kInv4Pi;
}

// Float-pair arithmetic (a value is hi + lo with |lo| <= ulp(hi)), after
// Dekker's and Knuth's error-free transformations: the rounded sum or product
// and its exact rounding error.  The _rn intrinsics are never contracted
// into fused operations, which would break the transformations.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// One entry by the 7 x 7 rule of regular_entry, evaluated on the FP32 pipe
// in float-pair arithmetic.  Per node pair: d = (x_hi - y_hi) + (x_lo - y_lo)
// with an exact high part; r^2 = |d|^2 as a float pair; 1/r from rsqrtf
// refined by one Newton step whose residual 1 - y0^2 r^2 is formed exactly
// to first order; the weighted terms are summed as float pairs and rounded
// to double once per entry.  A term's relative error is about
// 2^(E - 45) / |d| (2^E bounds |x - o|, d = x - y; it comes from the
// rounding of the nodes' low parts): 1e-13 and below for the admissible
// pairs of the coupling blocks, whose nodes lie at least a fraction of a
// cluster diameter apart.  min_r2 returns the smallest |d|^2 (high part)
// met, so that callers with close pairs can fall back to float64.
__device__ __forceinline__ double regular_entry_split(const SplitNode* __restrict__ xq,
                                                      const SplitNode* __restrict__ yq, float& min_r2) {
  float sh = 0.f, sl = 0.f;
  float mr = 3.0e38f;
#pragma unroll 1
  for (int p = 0; p < 7; ++p) {
    const SplitNode x = xq[p];
    float ih = 0.f, il = 0.f;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const SplitNode y = yq[q];
      const float dh0 = __fsub_rn(x.hi.x, y.hi.x), dl0 = __fsub_rn(x.lo.x, y.lo.x);
      const float dh1 = __fsub_rn(x.hi.y, y.hi.y), dl1 = __fsub_rn(x.lo.y, y.lo.y);
      const float dh2 = __fsub_rn(x.hi.z, y.hi.z), dl2 = __fsub_rn(x.lo.z, y.lo.z);
      // |d|^2 = sum dh^2 + (2 dh + dl) dl; the dl^2 part matters: it is
      // (g / |d|)^2 relative, 1e-10 at a few hundred grid steps
      const float p0 = __fmul_rn(dh0, dh0), p1 = __fmul_rn(dh1, dh1), p2 = __fmul_rn(dh2, dh2);
      float low = __fmaf_rn(dh0, dh0, -p0);
      low = __fadd_rn(low, __fmaf_rn(dh1, dh1, -p1));
      low = __fadd_rn(low, __fmaf_rn(dh2, dh2, -p2));
      low = __fmaf_rn(__fadd_rn(__fadd_rn(dh0, dh0), dl0), dl0, low);
      low = __fmaf_rn(__fadd_rn(__fadd_rn(dh1, dh1), dl1), dl1, low);
      low = __fmaf_rn(__fadd_rn(__fadd_rn(dh2, dh2), dl2), dl2, low);
      float s01, e01, rh, e2;
      two_sum(p0, p1, s01, e01);
      two_sum(s01, p2, rh, e2);
      const float rl = __fadd_rn(low, __fadd_rn(e01, e2));
      mr = fminf(mr, rh);
      // 1/r = y0 (1 + rho / 2), rho = 1 - y0^2 r^2 (|rho| ~ 2^-22: y0 must
      // start from rh + rl, since the cross terms put r^2 - rh at 2 g / |d|)
      const float y0 = rsqrtf(__fadd_rn(rh, rl));
      const float u = __fmul_rn(y0, y0), uu = __fmaf_rn(y0, y0, -u);
      const float m = __fmul_rn(u, rh), me = __fmaf_rn(u, rh, -m);
      const float rho = __fmaf_rn(-uu, rh, __fmaf_rn(-u, rl, __fsub_rn(__fsub_rn(1.f, m), me)));
      const float dy = __fmul_rn(__fmul_rn(0.5f, y0), rho);
      // term w_q / r as a float pair, added to the inner sum
      const float th = __fmul_rn(y.hi.w, y0);
      const float tl = __fadd_rn(__fmaf_rn(y.hi.w, y0, -th), __fmaf_rn(y.hi.w, dy, __fmul_rn(y.lo.w, y0)));
      float ns, ne;
      two_sum(ih, th, ns, ne);
      ih = ns;
      il = __fadd_rn(il, __fadd_rn(ne, tl));
    }
    // outer sum += w_p * inner
    const float th = __fmul_rn(x.hi.w, ih);
    const float tl = __fadd_rn(__fmaf_rn(x.hi.w, ih, -th), __fmaf_rn(x.hi.w, il, __fmul_rn(x.lo.w, ih)));
    float ns, ne;
    two_sum(sh, th, ns, ne);
    sh = ns;
    sl = __fadd_rn(sl, __fadd_rn(ne, tl));
  }
  min_r2 = mr;
  return ((double)sh + (double)sl) * kInv4Pi;
}

// One CTA per pair of mirrored admissible blocks (tau, sigma) and
// (sigma, tau): G is symmetric (Eq. 1 with g(x, y) = g(y, x) and the same
// rule on both triangles), so S_{sigma tau} = S_{tau sigma}^T and every
// entry is computed once and stored twice.  pairs[i] = (b, m): block b and
// its mirror m (-1: b is computed alone).  The column pivots' nodes are
// staged in shared memory.  S is row-major r_tau x r_sigma per block.
// F64: the same entries by the float64 rule of regular_entry (GCA_F64_ENTRIES).
template <bool F64>
__global__ void k_couple_entries(const int2* __restrict__ pairs, const int* __restrict__ far_t,
                                 const int* __restrict__ far_s, const int64_t* __restrict__ soff,
                                 const int* __restrict__ rank, const int64_t* __restrict__ poff,
                                 const int* __restrict__ piv, const SplitNode* __restrict__ tn,
                                 const P4* __restrict__ tq, double* __restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SplitNode* ys = reinterpret_cast<SplitNode*>(smem_raw);
  P4* yq = reinterpret_cast<P4*>(smem_raw);  // F64: the same bytes (sizeof(P4) == sizeof(SplitNode))
  const int2 bm = pairs[blockIdx.x];
  const int b = bm.x;
  const int t = far_t[b], s = far_s[b];
  const int rt = rank[t], rs = rank[s];
  const int* pt = piv + poff[t];
  const int* ps = piv + poff[s];
  for (int i = threadIdx.x; i < rs * 7; i += blockDim.x) {
    if (F64)
      yq[i] = tq[7 * (int64_t)ps[i / 7] + i % 7];
    else
      ys[i] = tn[7 * (int64_t)ps[i / 7] + i % 7];
  }
  __syncthreads();
  double* out = S + soff[b];
  double* mir = bm.y >= 0 ? S + soff[bm.y] : nullptr;
  for (int idx = threadIdx.x; idx < rt * rs; idx += blockDim.x) {
    const int a = idx / rs, c = idx % rs;
    double v;
    if (F64) {
      v = regular_entry(tq + 7 * (int64_t)pt[a], yq + 7 * c);
    } else {
      float mr;
      v = regular_entry_split(tn + 7 * (int64_t)pt[a], ys + 7 * c, mr);
    }
    out[idx] = v;
    if (mir) mir[(int64_t)c * rt + a] = v;
  }
}
static_assert(sizeof(P4) == sizeof(SplitNode), "k_couple_entries stages either kind of node in the same bytes");

struct SingularItem {
  int64_t pos;  // position in N
  int ti;
  int tj;
};

// One CTA per near block: disjoint pairs by the 7 x 7 rule, touching pairs
// appended to the list of their case (1 common vertex, 2 common edge,
// 3 identical).  A disjoint pair is evaluated in float-pair arithmetic and
// again in float64 when two of its nodes are closer than sqrt(near_r2) =
// 2^(E - 8) (so that the float-pair error stays below about 2^-37).
template <bool F64>
__global__ void k_near_entries(const int* __restrict__ near_t, const int* __restrict__ near_s,
                               const int64_t* __restrict__ noff, const int* __restrict__ begin,
                               const int* __restrict__ end, const int* __restrict__ perm,
                               const int* __restrict__ tri, const P4* __restrict__ tq,
                               const SplitNode* __restrict__ tn, float near_r2,
                               double* __restrict__ N, SingularItem* __restrict__ lists,
                               int64_t cap, unsigned long long* __restrict__ counts,
                               int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int t = near_t[b], s = near_s[b];
  const int bt = begin[t], nt = end[t] - bt, bs = begin[s], ns = end[s] - bs;
  P4* ys = reinterpret_cast<P4*>(smem_raw);
  SplitNode* yn = reinterpret_cast<SplitNode*>(smem_raw + sizeof(P4) * 7 * (size_t)ns);
  for (int i = threadIdx.x; i < ns * 7; i += blockDim.x) {
    const int64_t src = 7 * (int64_t)perm[bs + i / 7] + i % 7;
    ys[i] = tq[src];
    yn[i] = tn[src];
  }
  __syncthreads();
  const int64_t base = noff[b];
  for (int idx = threadIdx.x; idx < nt * ns; idx += blockDim.x) {
    const int i = idx / ns, j = idx % ns;
    const int ti = perm[bt + i], tj = perm[bs + j];
    int shared = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int va = tri[3 * ti + a];
      shared += (va == tri[3 * tj]) + (va == tri[3 * tj + 1]) + (va == tri[3 * tj + 2]);
    }
    if (shared == 0) {
      double v;
      if (F64) {
        v = regular_entry(tq + 7 * (int64_t)ti, ys + 7 * j);
      } else {
        float mr;
        v = regular_entry_split(tn + 7 * (int64_t)ti, yn + 7 * j, mr);
        if (mr < near_r2) v = regular_entry(tq + 7 * (int64_t)ti, ys + 7 * j);
      }
      N[base + idx] = v;
    } else {
      const unsigned long long slot = atomicAdd(&counts[shared], 1ull);
      if (slot < (unsigned long long)cap) {
        lists[(shared - 1) * cap + slot] = SingularItem{base + idx, ti, tj};
      } else {
        atomicOr(status, kStatusOverflow);
      }
    }
  }
}

// ------------------------------------------------- Sauter-Schwab (Sect. 8)
//
// Both triangles are parametrised over {0 <= u2 <= u1 <= 1} by
// x(u) = P0 + u1 (P1 - P0) + u2 (P2 - P1) with the shared vertex (or the
// first shared edge vertex) at P0 = Q0.  The substitutions map [0,1]^4 onto
// T x T in 6 (identical), 5 (common edge) or 2 (common vertex) pieces; on
// each piece u = xi * u^(eta), v = xi * v^(eta), so x - y = xi h(eta) and,
// with the Jacobian xi^3 w^(eta), the integrand is xi^2 w^(eta) / |h(eta)|.
// The xi-integral is therefore exactly 1/3 and only eta is sampled (q^3
// Gauss points per piece).

template <int CASE, typename R>
R sauter_piece(int piece, R e1, R e2, R e3, R& u1, R& u2, R& v1, R& v2) {
  if (CASE == 3) {
    const double w = e1 * e1 * e2;
    switch (piece) {
      case 0: u1 = 1.0; u2 = 1.0 - e1 + e1 * e2; v1 = 1.0 - e1 * e2 * e3; v2 = 1.0 - e1; break;
      case 1: v1 = 1.0; v2 = 1.0 - e1 + e1 * e2; u1 = 1.0 - e1 * e2 * e3; u2 = 1.0 - e1; break;
      case 2: u1 = 1.0; u2 = e1 * (1.0 - e2 + e2 * e3); v1 = 1.0 - e1 * e2; v2 = e1 * (1.0 - e2); break;
      case 3: v1 = 1.0; v2 = e1 * (1.0 - e2 + e2 * e3); u1 = 1.0 - e1 * e2; u2 = e1 * (1.0 - e2); break;
      case 4: u1 = 1.0 - e1 * e2 * e3; u2 = e1 * (1.0 - e2 * e3); v1 = 1.0; v2 = e1 * (1.0 - e2); break;
      default: v1 = 1.0 - e1 * e2 * e3; v2 = e1 * (1.0 - e2 * e3); u1 = 1.0; u2 = e1 * (1.0 - e2); break;
    }
    return w;
  } else if (CASE == 2) {
    switch (piece) {
      case 0: u1 = 1.0; u2 = e1 * e3; v1 = 1.0 - e1 * e2; v2 = e1 * (1.0 - e2); return e1 * e1;
      case 1: u1 = 1.0; u2 = e1; v1 = 1.0 - e1 * e2 * e3; v2 = e1 * e2 * (1.0 - e3); break;
      case 2: u1 = 1.0 - e1 * e2; u2 = e1 * (1.0 - e2); v1 = 1.0; v2 = e1 * e2 * e3; break;
      case 3: u1 = 1.0 - e1 * e2 * e3; u2 = e1 * e2 * (1.0 - e3); v1 = 1.0; v2 = e1; break;
      default: u1 = 1.0 - e1 * e2 * e3; u2 = e1 * (1.0 - e2 * e3); v1 = 1.0; v2 = e1 * e2; break;
    }
    return e1 * e1 * e2;
  } else {
    if (piece == 0) {
      u1 = 1.0; u2 = e1; v1 = e2; v2 = e2 * e3;
    } else {
      v1 = 1.0; v2 = e1; u1 = e2; u2 = e2 * e3;
    }
    return e2;
  }
}

// One sample point of a Sauter-Schwab piece: h(eta) = sum_k c_k V_k over the
// edge vectors V_k of the pair (case 1: e1, e2, f1, f2; case 2: e1, e2, f2
// with c_0 = u1 - v1, since f1 = e1; case 3: e1, e2 with c = (u1 - v1,
// u2 - v2)) and the weight W = w_a w_b w_c w^(eta), all as float pairs.
// The table is computed on the host in long double, so the differences of
// the identical-vertex cases are formed before any rounding.
struct __align__(16) SSEntry {
  float4 ch, cl;  // coefficients, high and low parts
  float wh, wl;   // weight
  float pad[2];
};

template <int CASE>
void sauter_table(const Rules& rules, std::vector<SSEntry>& out) {
  const int q = rules.q, q3 = q * q * q;
  constexpr int pieces = CASE == 3 ? 6 : (CASE == 2 ? 5 : 2);
  auto split = [](long double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (long double)hi);
  };
  for (int s = 0; s < pieces * q3; ++s) {
    const int piece = s / q3, r = s % q3;
    const int a = r / (q * q), b = (r / q) % q, c = r % q;
    long double u1, u2, v1, v2;
    const long double wj = sauter_piece<CASE, long double>(piece, rules.ss_t[a], rules.ss_t[b], rules.ss_t[c],
                                                           u1, u2, v1, v2);
    long double cf[4] = {0, 0, 0, 0};
    if (CASE == 1) {
      cf[0] = u1; cf[1] = u2; cf[2] = -v1; cf[3] = -v2;
    } else if (CASE == 2) {
      cf[0] = u1 - v1; cf[1] = u2; cf[2] = -v2;
    } else {
      cf[0] = u1 - v1; cf[1] = u2 - v2;
    }
    SSEntry e{};
    split(cf[0], e.ch.x, e.cl.x);
    split(cf[1], e.ch.y, e.cl.y);
    split(cf[2], e.ch.z, e.cl.z);
    split(cf[3], e.ch.w, e.cl.w);
    split((long double)rules.ss_w[a] * rules.ss_w[b] * rules.ss_w[c] * wj, e.wh, e.wl);
    out.push_back(e);
  }
}

// c * (vh + vl) with c = ch + cl, added to the float pair (sh, sl)
__device__ __forceinline__ void fp_mul_add(float ch, float cl, float vh, float vl, float& sh, float& sl) {
  const float th = __fmul_rn(ch, vh);
  const float tl = __fmaf_rn(ch, vl, __fmaf_rn(cl, vh, __fmaf_rn(ch, vh, -th)));
  float ns, ne;
  two_sum(sh, th, ns, ne);
  sh = ns;
  sl = __fadd_rn(sl, __fadd_rn(ne, tl));
}

// s + (th + tl) for float pairs s = (sh, sl)
__device__ __forceinline__ void pair_acc(float& sh, float& sl, float th, float tl) {
  float ns, ne;
  two_sum(sh, th, ns, ne);
  sh = ns;
  sl = __fadd_rn(sl, __fadd_rn(ne, tl));
}

// (ah + al)(bh + bl) as a float pair to first order
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float& th, float& tl) {
  th = __fmul_rn(ah, bh);
  tl = __fadd_rn(__fmaf_rn(ah, bh, -th), __fmaf_rn(ah, bl, __fmul_rn(al, bh)));
}

// one warp per touching pair; the eta samples in float-pair arithmetic (the
// regular rule's error-free sums, |h|^2 as a float pair and one Newton step
// from rsqrtf), the pair's sum and its Jacobians (2 |T|) in float64
template <int CASE>
__global__ void k_singular(const SingularItem* __restrict__ items,
                           const unsigned long long* __restrict__ counts, int64_t cap,
                           const int* __restrict__ tri, const double* __restrict__ vert,
                           const double* __restrict__ area2, const SSEntry* __restrict__ table, int nsamples,
                           double* __restrict__ N) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t count = min((long long)counts[CASE], (long long)cap);
  if (w >= count) return;
  const SingularItem it = items[w];
  int ti[3], tj[3];
  for (int a = 0; a < 3; ++a) {
    ti[a] = tri[3 * it.ti + a];
    tj[a] = tri[3 * it.tj + a];
  }
  int P[3], Q[3];
  if (CASE == 3) {
    for (int a = 0; a < 3; ++a) P[a] = Q[a] = ti[a];
  } else if (CASE == 2) {
    // shared ids in the order they occur in triangle i, then the others
    int sh[2], ns = 0, oi = -1, oj = -1;
    for (int a = 0; a < 3; ++a) {
      const bool in_j = ti[a] == tj[0] || ti[a] == tj[1] || ti[a] == tj[2];
      if (in_j) sh[ns++] = ti[a]; else oi = ti[a];
    }
    for (int a = 0; a < 3; ++a)
      if (tj[a] != sh[0] && tj[a] != sh[1]) oj = tj[a];
    P[0] = Q[0] = sh[0];
    P[1] = Q[1] = sh[1];
    P[2] = oi;
    Q[2] = oj;
  } else {
    int pi = 0, pj = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (ti[a] == tj[b]) { pi = a; pj = b; }
    for (int a = 0; a < 3; ++a) {
      P[a] = ti[(pi + a) % 3];
      Q[a] = tj[(pj + a) % 3];
    }
  }
  // The edge vectors of h as float pairs (case 1: e1, e2, f1, f2; case 2: e1,
  // e2, f2, since f1 = e1; case 3: e1, e2), e1 = P1 - P0, e2 = P2 - P1,
  // f1 = Q1 - Q0, f2 = Q2 - Q1.  Lane 3k + d forms component d of vector k in
  // float64 and splits it; the others receive it by shuffles.
  constexpr int NT = CASE == 3 ? 2 : (CASE == 2 ? 3 : 4);
  float my_h = 0.f, my_l = 0.f;
  if (lane < 3 * NT) {
    const int k = lane / 3, d = lane - 3 * k;
    const bool useq = (CASE == 1 && k >= 2) || (CASE == 2 && k == 2);
    const bool second = !(k == 0 || (CASE == 1 && k == 2));  // edge (1, 2) instead of (0, 1)
    const int i0 = useq ? (second ? Q[1] : Q[0]) : (second ? P[1] : P[0]);
    const int i1 = useq ? (second ? Q[2] : Q[1]) : (second ? P[2] : P[1]);
    const double x = vert[3 * i1 + d] - vert[3 * i0 + d];
    my_h = (float)x;
    my_l = (float)(x - (double)my_h);
  }
  float vh[NT][3], vl[NT][3];
#pragma unroll
  for (int k = 0; k < NT; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      vh[k][d] = __shfl_sync(0xffffffffu, my_h, 3 * k + d);
      vl[k][d] = __shfl_sync(0xffffffffu, my_l, 3 * k + d);
    }
  float ah = 0.f, al = 0.f;
  for (int s = lane; s < nsamples; s += 32) {
    const SSEntry e = table[s];
    const float ch[4] = {e.ch.x, e.ch.y, e.ch.z, e.ch.w}, cl[4] = {e.cl.x, e.cl.y, e.cl.z, e.cl.w};
    float hh[3], hl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      hh[d] = 0.f;
      hl[d] = 0.f;
#pragma unroll
      for (int k = 0; k < NT; ++k) fp_mul_add(ch[k], cl[k], vh[k][d], vl[k][d], hh[d], hl[d]);
    }
    // |h|^2 as a float pair
    const float p0 = __fmul_rn(hh[0], hh[0]), p1 = __fmul_rn(hh[1], hh[1]), p2 = __fmul_rn(hh[2], hh[2]);
    float low = __fmaf_rn(hh[0], hh[0], -p0);
    low = __fadd_rn(low, __fmaf_rn(hh[1], hh[1], -p1));
    low = __fadd_rn(low, __fmaf_rn(hh[2], hh[2], -p2));
    low = __fmaf_rn(__fadd_rn(__fadd_rn(hh[0], hh[0]), hl[0]), hl[0], low);
    low = __fmaf_rn(__fadd_rn(__fadd_rn(hh[1], hh[1]), hl[1]), hl[1], low);
    low = __fmaf_rn(__fadd_rn(__fadd_rn(hh[2], hh[2]), hl[2]), hl[2], low);
    float s01, e01, rh, e2;
    two_sum(p0, p1, s01, e01);
    two_sum(s01, p2, rh, e2);
    const float rl = __fadd_rn(low, __fadd_rn(e01, e2));
    // 1/|h| = y0 (1 + rho / 2), rho = 1 - y0^2 |h|^2
    const float y0 = rsqrtf(__fadd_rn(rh, rl));
    const float u = __fmul_rn(y0, y0), uu = __fmaf_rn(y0, y0, -u);
    const float m = __fmul_rn(u, rh), me = __fmaf_rn(u, rh, -m);
    const float rho = __fmaf_rn(-uu, rh, __fmaf_rn(-u, rl, __fsub_rn(__fsub_rn(1.f, m), me)));
    const float dy = __fmul_rn(__fmul_rn(0.5f, y0), rho);
    // acc += W / |h|
    const float th = __fmul_rn(e.wh, y0);
    const float tl = __fadd_rn(__fmaf_rn(e.wh, y0, -th), __fmaf_rn(e.wh, dy, __fmul_rn(e.wl, y0)));
    float ns, ne;
    two_sum(ah, th, ns, ne);
    ah = ns;
    al = __fadd_rn(al, __fadd_rn(ne, tl));
  }
  double acc = (double)ah + (double)al;
  for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  // Jacobians |e1 x e2| and |f1 x f2|: twice the triangles' areas
  if (lane == 0) N[it.pos] = acc * area2[it.ti] * area2[it.tj] * (kInv4Pi / 3.0);
}

// ------------------------------------------------ double-layer entries
//
// k_ij = int_{T_i} int_{T_j} dg/dn_y(x, y) dy dx with dg/dn_y(x, y) =
// <n_j, x - y> / (4 pi |x - y|^3), n_j the outer unit normal of T_j (the
// kernel of the integral equation of Sect. 1), in float64: the 7 x 7 rule for
// disjoint pairs, 0 for identical (flat) triangles, the Sauter-Schwab
// substitutions for a common edge or vertex.

__device__ __forceinline__ double dl_regular_entry(const P4* __restrict__ xq, const P4* __restrict__ yq,
                                                   double n0, double n1, double n2) {
  double s = 0.0;
#pragma unroll 1
  for (int p = 0; p < 7; ++p) {
    const P4 x = xq[p];
    double sp = 0.0;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const P4 y = yq[q];
      const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
      const double ir = rsqrt(dx * dx + dy * dy + dz * dz);
      sp += y.w * (n0 * dx + n1 * dy + n2 * dz) * ir * ir * ir;
    }
    s += x.w * sp;
  }
  return s * kInv4Pi;
}

// The double layer's 7 x 7 rule in float-pair arithmetic on the FP32 pipe
// (the recipe of regular_entry_split): per node pair d = x - y with exact
// high differences, |d|^2 and 1/|d| as float pairs, <n_y, d> with the
// normal split into float pairs (nh + nl), the term w_q <n_y, d> / |d|^3
// summed as float pairs and rounded to float64 once.  min_r2 returns the
// smallest |d|^2 (high part) met, for the near field's float64 fallback.
__device__ __forceinline__ double dl_entry_split(const SplitNode* __restrict__ xq, const SplitNode* __restrict__ yq,
                                                 const float* nh, const float* nl, float& min_r2) {
  float sh = 0.f, sl = 0.f;
  float mr = 3.0e38f;
#pragma unroll 1
  for (int p = 0; p < 7; ++p) {
    const SplitNode x = xq[p];
    float ih = 0.f, il = 0.f;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const SplitNode y = yq[q];
      const float dh0 = __fsub_rn(x.hi.x, y.hi.x), dl0 = __fsub_rn(x.lo.x, y.lo.x);
      const float dh1 = __fsub_rn(x.hi.y, y.hi.y), dl1 = __fsub_rn(x.lo.y, y.lo.y);
      const float dh2 = __fsub_rn(x.hi.z, y.hi.z), dl2 = __fsub_rn(x.lo.z, y.lo.z);
      const float p0 = __fmul_rn(dh0, dh0), p1 = __fmul_rn(dh1, dh1), p2 = __fmul_rn(dh2, dh2);
      float low = __fmaf_rn(dh0, dh0, -p0);
      low = __fadd_rn(low, __fmaf_rn(dh1, dh1, -p1));
      low = __fadd_rn(low, __fmaf_rn(dh2, dh2, -p2));
      low = __fmaf_rn(__fadd_rn(__fadd_rn(dh0, dh0), dl0), dl0, low);
      low = __fmaf_rn(__fadd_rn(__fadd_rn(dh1, dh1), dl1), dl1, low);
      low = __fmaf_rn(__fadd_rn(__fadd_rn(dh2, dh2), dl2), dl2, low);
      float s01, e01, rh, e2;
      two_sum(p0, p1, s01, e01);
      two_sum(s01, p2, rh, e2);
      const float rl = __fadd_rn(low, __fadd_rn(e01, e2));
      mr = fminf(mr, rh);
      const float y0 = rsqrtf(__fadd_rn(rh, rl));
      const float u = __fmul_rn(y0, y0), uu = __fmaf_rn(y0, y0, -u);
      const float m = __fmul_rn(u, rh), me = __fmaf_rn(u, rh, -m);
      const float rho = __fmaf_rn(-uu, rh, __fmaf_rn(-u, rl, __fsub_rn(__fsub_rn(1.f, m), me)));
      const float dy = __fmul_rn(__fmul_rn(0.5f, y0), rho);
      // <n_y, d>
      float ndh = 0.f, ndl = 0.f;
      fp_mul_add(nh[0], nl[0], dh0, dl0, ndh, ndl);
      fp_mul_add(nh[1], nl[1], dh1, dl1, ndh, ndl);
      fp_mul_add(nh[2], nl[2], dh2, dl2, ndh, ndl);
      // w_q <n_y, d> / |d|^3
      float ah, al, bh, bl;
      pair_mul(y0, dy, y0, dy, ah, al);
      pair_mul(ah, al, y0, dy, bh, bl);
      pair_mul(ndh, ndl, bh, bl, ah, al);
      pair_mul(y.hi.w, y.lo.w, ah, al, bh, bl);
      pair_acc(ih, il, bh, bl);
    }
    float th, tl;
    pair_mul(x.hi.w, x.lo.w, ih, il, th, tl);
    pair_acc(sh, sl, th, tl);
  }
  min_r2 = mr;
  return ((double)sh + (double)sl) * kInv4Pi;
}

// One CTA per coupling block (tau, sigma): K|tilde-tau x tilde-sigma', the
// row pivots of tau against the column pivots of sigma (r_tau x r'_sigma,
// row-major), in float-pair arithmetic (admissible pairs lie a fraction of
// a cluster diameter apart).  K is not symmetric, so every block is
// computed.
__global__ void k_dl_couple(const int* __restrict__ far_t, const int* __restrict__ far_s,
                            const int64_t* __restrict__ soff, const int* __restrict__ rank,
                            const int* __restrict__ rank2, const int64_t* __restrict__ poff,
                            const int64_t* __restrict__ poff2, const int* __restrict__ piv,
                            const int* __restrict__ piv2, const SplitNode* __restrict__ tn,
                            const double* __restrict__ nrm, double* __restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int t = far_t[b], s = far_s[b];
  const int rt = rank[t], rs = rank2[s];
  SplitNode* ys = reinterpret_cast<SplitNode*>(smem_raw);
  float* yn = reinterpret_cast<float*>(ys + 7 * (size_t)rs);  // per column: 3 high, then 3 low parts
  const int* pt = piv + poff[t];
  const int* ps = piv2 + poff2[s];
  for (int i = threadIdx.x; i < rs * 7; i += blockDim.x) ys[i] = tn[7 * (int64_t)ps[i / 7] + i % 7];
  for (int i = threadIdx.x; i < rs * 3; i += blockDim.x) {
    const double n = nrm[3 * (int64_t)ps[i / 3] + i % 3];
    const float h = (float)n;
    yn[6 * (i / 3) + i % 3] = h;
    yn[6 * (i / 3) + 3 + i % 3] = (float)(n - (double)h);
  }
  __syncthreads();
  double* out = S + soff[b];
  for (int idx = threadIdx.x; idx < rt * rs; idx += blockDim.x) {
    const int a = idx / rs, c = idx - (idx / rs) * rs;
    float mr;
    out[idx] = dl_entry_split(tn + 7 * (int64_t)pt[a], ys + 7 * c, yn + 6 * c, yn + 6 * c + 3, mr);
  }
}

// One CTA per near block of the double layer: disjoint pairs by the 7 x 7
// rule, identical triangles 0, pairs with a common edge or vertex appended to
// the list of their case (1 vertex, 2 edge).
__global__ void k_dl_near_entries(const int* __restrict__ near_t, const int* __restrict__ near_s,
                                  const int64_t* __restrict__ noff, const int* __restrict__ begin,
                                  const int* __restrict__ end, const int* __restrict__ perm,
                                  const int* __restrict__ tri, const P4* __restrict__ tq,
                                  const SplitNode* __restrict__ tn, float near_r2,
                                  const double* __restrict__ nrm, double* __restrict__ N,
                                  SingularItem* __restrict__ lists, int64_t cap,
                                  unsigned long long* __restrict__ counts, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int t = near_t[b], s = near_s[b];
  const int bt = begin[t], nt = end[t] - bt, bs = begin[s], ns = end[s] - bs;
  P4* ys = reinterpret_cast<P4*>(smem_raw);
  SplitNode* yt = reinterpret_cast<SplitNode*>(ys + 7 * (size_t)ns);
  double* yn = reinterpret_cast<double*>(yt + 7 * (size_t)ns);
  float* yf = reinterpret_cast<float*>(yn + 3 * (size_t)ns);  // per column: 3 high, then 3 low parts
  for (int i = threadIdx.x; i < ns * 7; i += blockDim.x) {
    const int64_t src = 7 * (int64_t)perm[bs + i / 7] + i % 7;
    ys[i] = tq[src];
    yt[i] = tn[src];
  }
  for (int i = threadIdx.x; i < ns * 3; i += blockDim.x) {
    const double n = nrm[3 * (int64_t)perm[bs + i / 3] + i % 3];
    const float h = (float)n;
    yn[i] = n;
    yf[6 * (i / 3) + i % 3] = h;
    yf[6 * (i / 3) + 3 + i % 3] = (float)(n - (double)h);
  }
  __syncthreads();
  const int64_t base = noff[b];
  for (int idx = threadIdx.x; idx < nt * ns; idx += blockDim.x) {
    const int i = idx / ns, j = idx - (idx / ns) * ns;
    const int ti = perm[bt + i], tj = perm[bs + j];
    int shared = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int va = tri[3 * ti + a];
      shared += (va == tri[3 * tj]) + (va == tri[3 * tj + 1]) + (va == tri[3 * tj + 2]);
    }
    if (shared == 0) {
      // float pairs, or float64 for nodes closer than sqrt(near_r2)
      float mr;
      double v = dl_entry_split(tn + 7 * (int64_t)ti, yt + 7 * j, yf + 6 * j, yf + 6 * j + 3, mr);
      if (mr < near_r2) v = dl_regular_entry(tq + 7 * (int64_t)ti, ys + 7 * j, yn[3 * j], yn[3 * j + 1], yn[3 * j + 2]);
      N[base + idx] = v;
    } else if (shared == 3) {
      N[base + idx] = 0.0;  // x - y lies in the plane of T_j
      atomicAdd(&counts[3], 1ull);
    } else {
      const unsigned long long slot = atomicAdd(&counts[shared], 1ull);
      if (slot < (unsigned long long)cap) {
        lists[(shared - 1) * cap + slot] = SingularItem{base + idx, ti, tj};
      } else {
        atomicOr(status, kStatusOverflow);
      }
    }
  }
}

// A Sauter-Schwab sample of the double layer in float64: the coefficients of
// h(eta) = (x - y) / xi in the edge vectors (as in SSEntry) and the weight
// (Gauss weights times the piece's Jacobian without xi^3).
struct __align__(16) SSEntry64 {
  double c[4];
  double w;
  double pad;
};

template <int CASE>
void sauter_table64(const Rules& rules, std::vector<SSEntry64>& out) {
  const int q = rules.q, q3 = q * q * q;
  constexpr int pieces = CASE == 3 ? 6 : (CASE == 2 ? 5 : 2);
  for (int s = 0; s < pieces * q3; ++s) {
    const int piece = s / q3, r = s % q3;
    const int a = r / (q * q), b = (r / q) % q, c = r % q;
    long double u1, u2, v1, v2;
    const long double wj = sauter_piece<CASE, long double>(piece, rules.ss_t[a], rules.ss_t[b], rules.ss_t[c],
                                                           u1, u2, v1, v2);
    SSEntry64 e{};
    if (CASE == 1) {
      e.c[0] = (double)u1; e.c[1] = (double)u2; e.c[2] = (double)-v1; e.c[3] = (double)-v2;
    } else if (CASE == 2) {
      e.c[0] = (double)(u1 - v1); e.c[1] = (double)u2; e.c[2] = (double)-v2; e.c[3] = 0.0;
    } else {
      e.c[0] = (double)(u1 - v1); e.c[1] = (double)(u2 - v2); e.c[2] = 0.0; e.c[3] = 0.0;
    }
    e.w = (double)((long double)rules.ss_w[a] * rules.ss_w[b] * rules.ss_w[c] * wj);
    out.push_back(e);
  }
}

// The single layer's touching pairs in float64 (GCA_F64_ENTRIES): one warp
// per pair, the vertex orders and edge vectors of k_singular, 1 / |h| summed
// over the eta samples of a float64 table (the xi-integral exactly 1/3).
template <int CASE>
__global__ void k_singular64(const SingularItem* __restrict__ items, const unsigned long long* __restrict__ counts,
                             int64_t cap, const int* __restrict__ tri, const double* __restrict__ vert,
                             const double* __restrict__ area2, const SSEntry64* __restrict__ table, int nsamples,
                             double* __restrict__ N) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t count = min((long long)counts[CASE], (long long)cap);
  if (w >= count) return;
  const SingularItem it = items[w];
  int ti[3], tj[3];
  for (int a = 0; a < 3; ++a) {
    ti[a] = tri[3 * it.ti + a];
    tj[a] = tri[3 * it.tj + a];
  }
  int P[3], Q[3];
  if (CASE == 3) {
    for (int a = 0; a < 3; ++a) P[a] = Q[a] = ti[a];
  } else if (CASE == 2) {
    int sh[2], ns = 0, oi = -1, oj = -1;
    for (int a = 0; a < 3; ++a) {
      const bool in_j = ti[a] == tj[0] || ti[a] == tj[1] || ti[a] == tj[2];
      if (in_j) sh[ns++] = ti[a]; else oi = ti[a];
    }
    for (int a = 0; a < 3; ++a)
      if (tj[a] != sh[0] && tj[a] != sh[1]) oj = tj[a];
    P[0] = Q[0] = sh[0];
    P[1] = Q[1] = sh[1];
    P[2] = oi;
    Q[2] = oj;
  } else {
    int pi = 0, pj = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (ti[a] == tj[b]) { pi = a; pj = b; }
    for (int a = 0; a < 3; ++a) {
      P[a] = ti[(pi + a) % 3];
      Q[a] = tj[(pj + a) % 3];
    }
  }
  double V[4][3];
  for (int d = 0; d < 3; ++d) {
    V[0][d] = vert[3 * P[1] + d] - vert[3 * P[0] + d];
    V[1][d] = vert[3 * P[2] + d] - vert[3 * P[1] + d];
    V[2][d] = CASE == 1 ? vert[3 * Q[1] + d] - vert[3 * Q[0] + d]
                        : (CASE == 2 ? vert[3 * Q[2] + d] - vert[3 * Q[1] + d] : 0.0);
    V[3][d] = CASE == 1 ? vert[3 * Q[2] + d] - vert[3 * Q[1] + d] : 0.0;
  }
  double acc = 0.0;
  for (int s = lane; s < nsamples; s += 32) {
    const SSEntry64 e = table[s];
    double h[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) h[d] = e.c[0] * V[0][d] + e.c[1] * V[1][d] + e.c[2] * V[2][d] + e.c[3] * V[3][d];
    acc += e.w * rsqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
  }
  for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) N[it.pos] = acc * area2[it.ti] * area2[it.tj] * (kInv4Pi / 3.0);
}

// one warp per pair with a common vertex (CASE 1) or edge (CASE 2): on each
// piece x - y = xi h(eta), the kernel times the Jacobian xi^3 is
// xi <n_j, h> / |h|^3, so the xi-integral is exactly 1/2 and eta is sampled
template <int CASE>
__global__ void k_dl_singular(const SingularItem* __restrict__ items,
                              const unsigned long long* __restrict__ counts, int64_t cap,
                              const int* __restrict__ tri, const double* __restrict__ vert,
                              const double* __restrict__ area2, const double* __restrict__ nrm,
                              const SSEntry64* __restrict__ table, int nsamples, double* __restrict__ N) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t count = min((long long)counts[CASE], (long long)cap);
  if (w >= count) return;
  const SingularItem it = items[w];
  int ti[3], tj[3];
  for (int a = 0; a < 3; ++a) {
    ti[a] = tri[3 * it.ti + a];
    tj[a] = tri[3 * it.tj + a];
  }
  int P[3], Q[3];
  if (CASE == 2) {
    int sh[2], ns = 0, oi = -1, oj = -1;
    for (int a = 0; a < 3; ++a) {
      const bool in_j = ti[a] == tj[0] || ti[a] == tj[1] || ti[a] == tj[2];
      if (in_j) sh[ns++] = ti[a]; else oi = ti[a];
    }
    for (int a = 0; a < 3; ++a)
      if (tj[a] != sh[0] && tj[a] != sh[1]) oj = tj[a];
    P[0] = Q[0] = sh[0];
    P[1] = Q[1] = sh[1];
    P[2] = oi;
    Q[2] = oj;
  } else {
    int pi = 0, pj = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (ti[a] == tj[b]) { pi = a; pj = b; }
    for (int a = 0; a < 3; ++a) {
      P[a] = ti[(pi + a) % 3];
      Q[a] = tj[(pj + a) % 3];
    }
  }
  // edge vectors: case 1 e1, e2, f1, f2; case 2 e1, e2, f2 (f1 = e1)
  double V[4][3];
  for (int d = 0; d < 3; ++d) {
    V[0][d] = vert[3 * P[1] + d] - vert[3 * P[0] + d];
    V[1][d] = vert[3 * P[2] + d] - vert[3 * P[1] + d];
    if (CASE == 1) {
      V[2][d] = vert[3 * Q[1] + d] - vert[3 * Q[0] + d];
      V[3][d] = vert[3 * Q[2] + d] - vert[3 * Q[1] + d];
    } else {
      V[2][d] = vert[3 * Q[2] + d] - vert[3 * Q[1] + d];
      V[3][d] = 0.0;
    }
  }
  const double n0 = nrm[3 * (int64_t)it.tj], n1 = nrm[3 * (int64_t)it.tj + 1], n2 = nrm[3 * (int64_t)it.tj + 2];
  double acc = 0.0;
  for (int s = lane; s < nsamples; s += 32) {
    const SSEntry64 e = table[s];
    double h[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) h[d] = e.c[0] * V[0][d] + e.c[1] * V[1][d] + e.c[2] * V[2][d] + e.c[3] * V[3][d];
    const double ir = rsqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    acc += e.w * (n0 * h[0] + n1 * h[1] + n2 * h[2]) * ir * ir * ir;
  }
  for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) N[it.pos] = acc * area2[it.ti] * area2[it.tj] * (kInv4Pi / 2.0);
}

// ----------------------------------------------- Green quadrature factors
//
// The pure Green quadrature of Sect. 2: G|tau-hat x sigma-hat ~ A_tau B^*,
//   a_{i nu}   =        sqrt(w) int g(x, z_nu) phi_i,   a_{i nu+k} = -d_tau sqrt(w) int dg/dn_z(x, z_nu) phi_i,
//   b_{j nu}   =        sqrt(w) int dg/dn_z(z_nu, y) phi_j,  b_{j nu+k} = sqrt(w) / d_tau int g(z_nu, y) phi_j,
// with the box rule z_nu, n_nu, w_nu of omega_tau (Eq. (2)); float64.

struct GqJob {
  int c;          // the cluster whose box carries the rule
  int s;          // the cluster whose triangles are integrated
  int64_t off;    // output offset
};

// A_tau of every listed cluster (row-major |tau-hat| x 2k), one CTA each
__global__ void k_gq_rows(const GqJob* __restrict__ jobs, int k, const int* __restrict__ begin,
                          const int* __restrict__ end, const int* __restrict__ perm, const P4* __restrict__ tq,
                          const P4* __restrict__ zq, const double* __restrict__ diam, double* __restrict__ out) {
  const GqJob jb = jobs[blockIdx.x];
  const int c = jb.c, b0 = begin[c], nr = end[c] - b0, m2 = k / 6;
  const P4* z = zq + (int64_t)c * k;
  double* A = out + jb.off;
  for (int idx = threadIdx.x; idx < nr * k; idx += blockDim.x) {
    const int i = idx / k, nu = idx - i * k;
    const P4 zz = z[nu];
    const int face = nu / m2, d = face >> 1;
    const double sgn = (face & 1) ? 1.0 : -1.0;
    const P4* xq = tq + 7 * (int64_t)perm[b0 + i];
    double gs = 0.0, ds = 0.0;
#pragma unroll
    for (int qq = 0; qq < 7; ++qq) {
      const P4 x = xq[qq];
      const double dx = x.x - zz.x, dy = x.y - zz.y, dz = x.z - zz.z;
      const double ir = rsqrt(dx * dx + dy * dy + dz * dz);
      const double dn = sgn * (d == 0 ? dx : (d == 1 ? dy : dz));
      gs += x.w * ir;
      ds += x.w * dn * ir * ir * ir;
    }
    A[(int64_t)i * 2 * k + nu] = zz.w * gs * kInv4Pi;
    A[(int64_t)i * 2 * k + k + nu] = -diam[c] * zz.w * ds * kInv4Pi;
  }
}

// B_{tau sigma}^* of every coupling block (row-major 2k x |sigma-hat|), one CTA each
__global__ void k_gq_factors(const GqJob* __restrict__ jobs, int k, const int* __restrict__ begin,
                             const int* __restrict__ end, const int* __restrict__ perm, const P4* __restrict__ tq,
                             const P4* __restrict__ zq, const double* __restrict__ diam, double* __restrict__ out) {
  const GqJob jb = jobs[blockIdx.x];
  const int c = jb.c, s = jb.s, b0 = begin[s], ns = end[s] - b0, m2 = k / 6;
  const P4* z = zq + (int64_t)c * k;
  const double inv_d = 1.0 / diam[c];
  double* B = out + jb.off;
  for (int idx = threadIdx.x; idx < ns * k; idx += blockDim.x) {
    const int j = idx / k, nu = idx - j * k;
    const P4 zz = z[nu];
    const int face = nu / m2, d = face >> 1;
    const double sgn = (face & 1) ? 1.0 : -1.0;
    const P4* yq = tq + 7 * (int64_t)perm[b0 + j];
    double dn_s = 0.0, g_s = 0.0;
#pragma unroll
    for (int qq = 0; qq < 7; ++qq) {
      const P4 y = yq[qq];
      const double ex = y.x - zz.x, ey = y.y - zz.y, ez = y.z - zz.z;
      const double ir = rsqrt(ex * ex + ey * ey + ez * ez);
      const double dn = sgn * (d == 0 ? ex : (d == 1 ? ey : ez));
      dn_s += y.w * dn * ir * ir * ir;
      g_s += y.w * ir;
    }
    B[(int64_t)nu * ns + j] = zz.w * dn_s * kInv4Pi;
    B[(int64_t)(k + nu) * ns + j] = zz.w * inv_d * g_s * kInv4Pi;
  }
}

// ------------------------------------------------- collocation entries
//
// c_ij = int_{T_j} g(x_i, y) dy at the centroid x_i of T_i (the collocation
// variant of Sect. 6 for the piecewise constant basis), in float64: the
// 7-point rule on T_j for j != i; for j = i the Duffy transformation around
// x_i: T_i splits into (x_i, P_k, P_k+1), on which y = x_i + s ((1 - t) P_k +
// t P_k+1 - x_i) makes the integrand J_k / |(1 - t) P_k + t P_k+1 - x_i|
// independent of s; t takes the rule `duffy` (nodes and weights on [0, 1]).

__device__ __forceinline__ double col_regular_entry(const P4& x, const P4* __restrict__ yq) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const P4 y = yq[q];
    const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
    s += y.w * rsqrt(dx * dx + dy * dy + dz * dz);
  }
  return s * kInv4Pi;
}

__device__ double col_duffy_entry(const P4& x, const double* __restrict__ vert, const int* __restrict__ tri, int t,
                                  const double2* __restrict__ duffy, int nd) {
  double P[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) P[a][d] = vert[3 * tri[3 * t + a] + d];
  const double xc[3] = {x.x, x.y, x.z};
  double total = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double* A = P[k];
    const double* B = P[(k + 1) % 3];
    const double a0 = A[0] - xc[0], a1 = A[1] - xc[1], a2 = A[2] - xc[2];
    const double b0 = B[0] - xc[0], b1 = B[1] - xc[1], b2 = B[2] - xc[2];
    const double c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
    const double jac = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    double sk = 0.0;
    for (int q = 0; q < nd; ++q) {
      const double tq = duffy[q].x;
      const double e0 = a0 + tq * (b0 - a0), e1 = a1 + tq * (b1 - a1), e2 = a2 + tq * (b2 - a2);
      sk += duffy[q].y * rsqrt(e0 * e0 + e1 * e1 + e2 * e2);
    }
    total += jac * sk;
  }
  return total * kInv4Pi;
}

// One CTA per coupling block: C|tilde-tau x tilde-sigma', the centroids of the
// row pivots against the 7-point rules of the column pivots.
__global__ void k_col_couple(const int* __restrict__ far_t, const int* __restrict__ far_s,
                             const int64_t* __restrict__ soff, const int* __restrict__ rank,
                             const int* __restrict__ rank2, const int64_t* __restrict__ poff,
                             const int64_t* __restrict__ poff2, const int* __restrict__ piv,
                             const int* __restrict__ piv2, const P4* __restrict__ tq, double* __restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int t = far_t[b], s = far_s[b];
  const int rt = rank[t], rs = rank2[s];
  P4* ys = reinterpret_cast<P4*>(smem_raw);
  const int* pt = piv + poff[t];
  const int* ps = piv2 + poff2[s];
  for (int i = threadIdx.x; i < rs * 7; i += blockDim.x) ys[i] = tq[7 * (int64_t)ps[i / 7] + i % 7];
  __syncthreads();
  double* out = S + soff[b];
  for (int idx = threadIdx.x; idx < rt * rs; idx += blockDim.x) {
    const int a = idx / rs, c = idx - (idx / rs) * rs;
    out[idx] = col_regular_entry(tq[7 * (int64_t)pt[a]], ys + 7 * c);
  }
}

// One CTA per near block of the collocation matrix.
__global__ void k_col_near_entries(const int* __restrict__ near_t, const int* __restrict__ near_s,
                                   const int64_t* __restrict__ noff, const int* __restrict__ begin,
                                   const int* __restrict__ end, const int* __restrict__ perm,
                                   const int* __restrict__ tri, const double* __restrict__ vert,
                                   const P4* __restrict__ tq, const double2* __restrict__ duffy, int nd,
                                   double* __restrict__ N, unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int t = near_t[b], s = near_s[b];
  const int bt = begin[t], nt = end[t] - bt, bs = begin[s], ns = end[s] - bs;
  P4* ys = reinterpret_cast<P4*>(smem_raw);
  for (int i = threadIdx.x; i < ns * 7; i += blockDim.x) ys[i] = tq[7 * (int64_t)perm[bs + i / 7] + i % 7];
  __syncthreads();
  const int64_t base = noff[b];
  for (int idx = threadIdx.x; idx < nt * ns; idx += blockDim.x) {
    const int i = idx / ns, j = idx - (idx / ns) * ns;
    const int ti = perm[bt + i], tj = perm[bs + j];
    const P4 x = tq[7 * (int64_t)ti];
    if (ti == tj) {
      N[base + idx] = col_duffy_entry(x, vert, tri, ti, duffy, nd);
      atomicAdd(&counts[3], 1ull);
    } else {
      N[base + idx] = col_regular_entry(x, ys + 7 * j);
    }
  }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

#include "p1.cuh"

int check_status(DevMem& st, cudaStream_t s, const char* where) {
  int h = 0;
  GCA_TRY_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GCA_TRY_CUDA(cudaStreamSynchronize(s));
  if (h & kStatusNumeric) {
    set_error(std::string(where) + ": NaN in the Green quadrature matrix");
    return GCA_ERR_NUMERIC;
  }
  if (h & kStatusOverflow) {
    set_error(std::string(where) + ": singular-pair list overflow (mesh not conforming?)");
    return GCA_ERR_INVALID_ARG;
  }
  return GCA_OK;
}

// Launches of k_aca for one level: jobs grouped by cluster size C (CTAs per
// job).  A job takes the smallest C whose rows fit in shared memory; levels
// with few jobs spread them over more CTAs (up to 16), so that the level
// keeps the SMs busy and each CTA's share of the FP64 rank-one updates stays
// small, as long as every CTA keeps at least kMinRowsPerCta rows.
class AcaLauncher {
 public:
  AcaLauncher() = default;
  AcaLauncher(const AcaLauncher&) = delete;
  AcaLauncher& operator=(const AcaLauncher&) = delete;
  ~AcaLauncher() {
    for (int i = 0; i < 5; ++i) {
      if (side_[i]) cudaStreamDestroy(side_[i]);
      if (join_[i]) cudaEventDestroy(join_[i]);
    }
    if (fork_) cudaEventDestroy(fork_);
  }
  int init(int k) {
    k_ = k;
    int dev = 0;
    GCA_TRY_CUDA(cudaGetDevice(&dev));
    int optin = 0;
    GCA_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    GCA_TRY_CUDA(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev));
    kern_[0] = 2 * k <= 128 ? k_aca<4, kAcaThreads>
                            : (2 * k <= 192 ? k_aca<6, kAcaThreads> : k_aca<14, kAcaThreads>);
    kern_[1] = 2 * k <= 128 ? k_aca<4, kAcaThreadsWide>
                            : (2 * k <= 192 ? k_aca<6, kAcaThreadsWide> : k_aca<14, kAcaThreadsWide>);
    budget_ = (size_t)optin;
    for (auto* kern : kern_) {
      cudaFuncAttributes fa{};
      GCA_TRY_CUDA(cudaFuncGetAttributes(&fa, kern));
      budget_ = std::min(budget_, (size_t)optin - fa.sharedSizeBytes);
    }
    for (auto* kern : kern_) {
      GCA_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget_));
      GCA_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    return GCA_OK;
  }
  // room for the V^ scratch of a level of the given rows (the clusters of a
  // level cover at most `rows` rows, each job at most 2k columns, plus the
  // rounding of every job up to its group's largest), so that the levels do
  // not reallocate it (a reallocation frees device memory and so waits for
  // every stream); launch() grows it where this bound falls short
  int reserve_scratch(size_t rows, size_t jobs) {
    return wbuf_.reserve(sizeof(double) * (rows + (size_t)GCA_MAX_LEAF * jobs) * 2 * (size_t)k_);
  }
  size_t smem(int rows, int C) const {
    const int rpc = (rows + C - 1) / C;
    return aca_smem_bytes(rpc, 2 * k_, std::min(rows, 2 * k_));
  }
  int launch(const std::vector<AcaJob>& jobs, DevMem& d_jobs, const AcaMesh* d_mesh, int level, double tol,
             double tie, cudaStream_t st) {
    constexpr int kMinRowsPerCta = 16;
    int spread = 1;
    while (spread < 16 && (int64_t)jobs.size() * spread < sms_) spread *= 2;
    std::vector<AcaJob> by_c[5];
    for (const auto& j : jobs) {
      int g = 0;
      while (g < 5 && smem(j.rows, 1 << g) > budget_) ++g;
      if (g == 5) {
        set_error("gca_build: cross approximation matrix too large for the cluster kernel");
        return GCA_ERR_UNSUPPORTED;
      }
      while (g < 4 && (1 << g) < spread && (j.rows >> (g + 1)) >= kMinRowsPerCta) ++g;
      by_c[g].push_back(j);
    }
    GCA_TRY(d_jobs.reserve(sizeof(AcaJob) * jobs.size()));
    std::vector<AcaJob> host;  // grouped copy, uploaded at once
    for (int g = 0; g < 5; ++g) host.insert(host.end(), by_c[g].begin(), by_c[g].end());
    GCA_TRY_CUDA(cudaMemcpyAsync(d_jobs.p, host.data(), sizeof(AcaJob) * host.size(), cudaMemcpyHostToDevice, st));
    // the groups of one level are independent: each runs on a side stream
    // forked from and joined back into `st`
    int ngroups = 0;
    for (int g = 0; g < 5; ++g) ngroups += !by_c[g].empty();
    // The side streams have the device's highest priority, so that the
    // level's CTAs take the SMs ahead of the near field's (which runs on a
    // lowest-priority stream beside the levels and fills the SMs they leave
    // idle); every level runs on them.
    const bool fork = true;
    if (fork) {
      int least = 0, greatest = 0;
      GCA_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      for (int i = 0; i < 5; ++i)
        if (!side_[i]) {
          GCA_TRY_CUDA(cudaStreamCreateWithPriority(&side_[i], cudaStreamNonBlocking, greatest));
          GCA_TRY_CUDA(cudaEventCreateWithFlags(&join_[i], cudaEventDisableTiming));
        }
      if (!fork_) GCA_TRY_CUDA(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
      GCA_TRY_CUDA(cudaEventRecord(fork_, st));
    }
    // V^ scratch of every CTA of the level: rpc_cap x rmax_cap per CTA, the
    // groups one after the other (they run concurrently)
    size_t wtotal = 0;
    size_t woff[5] = {0, 0, 0, 0, 0};
    for (int g = 0; g < 5; ++g) {
      if (by_c[g].empty()) continue;
      const int C = 1 << g;
      int rows_cap = 1;
      for (const auto& j : by_c[g]) rows_cap = std::max(rows_cap, j.rows);
      woff[g] = wtotal;
      wtotal += by_c[g].size() * C * (size_t)((rows_cap + C - 1) / C) * std::min(rows_cap, 2 * k_);
    }
    GCA_TRY(wbuf_.reserve(sizeof(double) * std::max<size_t>(wtotal, 1)));
    std::unique_ptr<PhaseScope> level_scope;
    if (!profile_detail()) {
      level_scope = std::make_unique<PhaseScope>("green_aca", st);
      level_scope->launches(ngroups);
    }
    size_t at = 0;
    for (int g = 0; g < 5; ++g) {
      if (by_c[g].empty()) continue;
      const int C = 1 << g;
      cudaStream_t gs = st;
      if (fork) {
        gs = side_[g];
        GCA_TRY_CUDA(cudaStreamWaitEvent(gs, fork_, 0));
      }
      int rows_cap = 1;
      for (const auto& j : by_c[g]) rows_cap = std::max(rows_cap, j.rows);
      const int rpc_cap = (rows_cap + C - 1) / C;
      const int rmax_cap = std::min(rows_cap, 2 * k_);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(by_c[g].size() * C));
      const int wide = aca_wide(C) ? 1 : 0;
      cfg.blockDim = dim3(wide ? kAcaThreadsWide : kAcaThreads);
      cfg.dynamicSmemBytes = smem(rows_cap, C);
      cfg.stream = gs;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      {
        std::unique_ptr<PhaseScope> ps;
        if (profile_detail())
          ps = std::make_unique<PhaseScope>("green_aca.L" + std::to_string(level) + ".c" + std::to_string(C), gs);
        GCA_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern_[wide], (const AcaJob*)(d_jobs.as<AcaJob>() + at), d_mesh, k_,
                                        rpc_cap, rmax_cap, tol, tie, wbuf_.as<double>() + woff[g]));
      }
      if (fork) {
        GCA_TRY_CUDA(cudaEventRecord(join_[g], gs));
        GCA_TRY_CUDA(cudaStreamWaitEvent(st, join_[g], 0));
      }
      at += by_c[g].size();
    }
    level_scope.reset();
    // `host` must outlive the copy: the caller synchronises before the next level
    GCA_TRY_CUDA(cudaStreamSynchronize(st));
    return GCA_OK;
  }

 private:
  int k_ = 0;
  int sms_ = 148;
  cudaStream_t side_[5] = {};
  cudaEvent_t join_[5] = {};
  cudaEvent_t fork_ = nullptr;
  size_t budget_ = 0;
  void (*kern_[2])(const AcaJob*, const AcaMesh*, int, int, int, double, double, double*) = {nullptr, nullptr};
  DevMem wbuf_;  // V^ scratch of the launches (grow-only)
};

}  // namespace

// Supports of the nodal basis functions (Sect. 5): for vertex v the
// triangles containing it in ascending order, item[ptr[v] .. ptr[v + 1]) =
// (triangle << 2) | corner.  Every vertex must belong to a triangle.
int node_supports(const gca_mesh* mesh, std::vector<int>& ptr, std::vector<int>& item, const char* who) {
  const int nv = mesh->nv, nt = mesh->nt;
  if (nt >= (1 << 29)) {
    set_error(std::string(who) + ": too many triangles for the support encoding");
    return GCA_ERR_UNSUPPORTED;
  }
  ptr.assign(nv + 1, 0);
  for (int64_t e = 0; e < 3LL * nt; ++e) ptr[mesh->triangles[e] + 1]++;
  for (int v = 0; v < nv; ++v) {
    if (ptr[v + 1] == 0) {
      set_error(std::string(who) + ": vertex " + std::to_string(v) + " belongs to no triangle");
      return GCA_ERR_INVALID_ARG;
    }
    ptr[v + 1] += ptr[v];
  }
  item.resize(3 * (size_t)nt);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int t = 0; t < nt; ++t)
    for (int c = 0; c < 3; ++c) item[fill[mesh->triangles[3 * (size_t)t + c]]++] = (t << 2) | c;
  return GCA_OK;
}

// One construction (see the header of this file) in stages, so that a batch
// can run the cross approximations of several meshes level by level in
// common launches: prepare() (geometry, block tree, box rules), rows() (the
// row bases: one BasisPass, or the Green quadrature matrices), finish() (the
// column bases of two-sided operators, entries, panels, product plan).
struct BasisOut {
  std::vector<int>* rank;
  std::vector<int64_t>* poff;
  std::vector<int64_t>* voff;
  std::vector<int64_t>* eoff;
  int64_t* v_entries;
  int64_t* e_entries;
  DevMem* V64;
  DevMem* E64;
};
class Builder;

// One side's nested bases (Sect. 3, Sect. 4), level by level from the
// deepest (kind 0: the cluster bases V, E of the rows from A_tau; 1: the
// double layer's column bases W, F from its column matrix; 2: the
// collocation rows; 3: the nodal rows): ranks, pivots in the pool d_piv
// (offsets poff), and the row-major float64 leaf bases and transfer
// matrices.  begin() sizes the pools, jobs(L) appends level L's cross
// approximations (job.mesh: the caller's index of this mesh in the launch's
// mesh table, whose entry is `am`), after() reads the level's ranks back
// once its launch is done, end() packs V and E.
struct BasisPass {
  BasisPass(Builder& b_, int kind_, const BasisOut& o_, DevMem& piv, DevMem& rank, int64_t& used)
      : b(b_), kind(kind_), o(o_), d_piv(piv), d_rank(rank), piv_used(used) {}
  int begin();
  int jobs(int L, int mesh_index, std::vector<AcaJob>& out);
  int after();
  int end();
  Builder& b;
  int kind;
  BasisOut o;
  DevMem& d_piv;
  DevMem& d_rank;
  int64_t& piv_used;
  std::vector<int64_t> vh_off;
  std::vector<int> rows_of;
  int64_t piv_cap = 0, vh_cap = 0, vh_used = 0;
  DevMem d_vh;
  AcaMesh am{};
};

class Builder {
 public:
  Builder(const gca_mesh* mesh_, const gca_tree* tree_, const gca_params* prm_, cudaStream_t st_, int op_,
          const double* midpoints_ = nullptr)
      : mesh(mesh_), tree(tree_), prm(prm_), st(st_), op(op_), midpoints(midpoints_) {}
  ~Builder() {
    if (near_st_) {
      cudaStreamSynchronize(near_st_);
      cudaStreamDestroy(near_st_);
    }
    if (near_ready_) cudaEventDestroy(near_ready_);
    if (near_done_) cudaEventDestroy(near_done_);
  }
  Builder(const Builder&) = delete;
  Builder& operator=(const Builder&) = delete;
  int prepare();
  int near_field();
  int rows();
  int finish(gca_h2** out);
  // the barycentric coordinates of the 7-point rule as float pairs
  BarySplit bary_split() const {
    BarySplit bs{};
    for (int i = 0; i < 7; ++i)
      for (int a = 0; a < 3; ++a) {
        bs.h[i][a] = (float)rules.bary[i][a];
        bs.l[i][a] = (float)(rules.bary[i][a] - (double)bs.h[i][a]);
      }
    return bs;
  }
  // the pass of the row bases (the single layer's, op 0, 1, 3; the
  // collocation rows, op 2; the nodal rows, op 5)
  std::unique_ptr<BasisPass> rows_pass() {
    return std::make_unique<BasisPass>(*this, op == 2 ? 2 : (p1 ? 3 : 0),
                                       BasisOut{&h->rank, &h->poff, &h->voff, &h->eoff, &h->v_entries,
                                                &h->e_entries, &h->V64, &h->E64},
                                       d_piv, d_rank, piv_used);
  }
  // passes on this mesh (the rows, and the columns of a two-sided
  // operator, which do not depend on each other): one launch per level
  // holds the jobs of all of them (job.mesh selects the pass's table entry);
  // `fork_near` launches the near field once the passes' pools are allocated
  // (an allocation can wait for all work on the device, the side stream's
  // included)
  int run_passes(std::initializer_list<BasisPass*> passes, bool fork_near) {
    std::vector<AcaMesh> table;
    for (BasisPass* p : passes) {
      GCA_TRY(p->begin());
      table.push_back(p->am);
    }
    DevMem d_mesh, d_jobs;
    // room for every level's jobs at once: a reallocation between levels
    // would free device memory and so wait for the near-field stream
    GCA_TRY(d_jobs.reserve(sizeof(AcaJob) * (size_t)nc * passes.size()));
    GCA_TRY(aca.reserve_scratch((size_t)n * passes.size(), (size_t)nc * passes.size()));
    GCA_TRY(upload(d_mesh, table, st));
    if (fork_near) GCA_TRY(near_field());
    std::vector<AcaJob> js;
    for (int L = h->depth; L >= 1; --L) {
      js.clear();
      int i = 0;
      for (BasisPass* p : passes) GCA_TRY(p->jobs(L, i++, js));
      if (js.empty()) continue;
      GCA_TRY(aca.launch(js, d_jobs, d_mesh.as<AcaMesh>(), L, prm->aca_tol, tie, st));
      for (BasisPass* p : passes) GCA_TRY(p->after());
    }
    for (BasisPass* p : passes) GCA_TRY(p->end());
    return GCA_OK;
  }

  const gca_mesh* mesh;
  const gca_tree* tree;
  const gca_params* prm;
  cudaStream_t st;
  int op;
  const double* midpoints;  // op 6: [nt][3][3] surface points over the edges
  std::chrono::steady_clock::time_point t0;
  bool p1 = false, single = false, curved = false;
  DevMem d_mid;
  std::vector<int> sup_ptr, sup_item;
  std::unique_ptr<gca_h2> h;
  int n = 0, nc = 0, k = 0, ntri = 0;
  double margin = 0.0;
  Rules rules{};
  std::vector<double> vert;
  std::vector<int> tri;
  DevMem d_tq, d_area2, d_box, d_diam, d_zq, d_status, d_nrm, d_sup_ptr, d_sup_item, d_tn;
  std::vector<double> box, diam;
  float near_r2 = 0.f;
  std::vector<char> needed;
  AcaLauncher aca;
  double tie = std::ldexp(1.0, -40);
  DevMem d_piv, d_rank, d_piv2, d_rank2;
  int64_t piv_used = 0, piv2_used = 0;
  // the near field (near_field()): touching-pair lists and their bound, the
  // counts by case, its status word, the sample table, the nodal basis's
  // near unions and blocks, and the side stream it runs on
  std::vector<int64_t> valence;
  int64_t cap = 0;
  bool f64_entries = false;
  DevMem d_items, d_counts, d_status_near, d_tab, d_nujobs, d_nucount, d_nurows, d_p1near;
  cudaStream_t near_st_ = nullptr;
  cudaEvent_t near_ready_ = nullptr, near_done_ = nullptr;
};

int Builder::prepare() {
  t0 = std::chrono::steady_clock::now();
  GCA_TRY(validate_mesh(mesh));
  // op 5 (nodal basis, Sect. 5): the indices are the vertices
  p1 = op == 5 || op == 6;
  curved = op == 6;
  gca_mesh shape = *mesh;
  if (p1) shape.nt = mesh->nv;
  GCA_TRY(validate_tree(&shape, tree, GCA_MAX_LEAF));
  if (!prm || !(prm->eta > 0.0) || prm->box_gauss_m < 1 || prm->box_gauss_m > GCA_MAX_BOX_M ||
      !(prm->aca_tol >= 0.0) || prm->tri_rule != 7 || prm->sauter_q < 1 ||
      prm->sauter_q > GCA_MAX_SAUTER_Q ||
      (prm->flags & ~(uint32_t)(GCA_DROP_F64 | GCA_DROP_F32 | GCA_DROP_BF16 | GCA_DROP_EXPORT | GCA_F64_ENTRIES)) !=
          0) {
    set_error("gca_build: invalid parameters");
    return GCA_ERR_INVALID_ARG;
  }
  // supports of the nodal basis functions: the triangles at each vertex in
  // ascending order, as (triangle << 2) | corner
  if (p1) GCA_TRY(node_supports(mesh, sup_ptr, sup_item, curved ? "gca_build_p1_curved" : "gca_build_p1"));
  if (curved) {
    if (!midpoints) {
      set_error("gca_build_p1_curved: midpoints is NULL");
      return GCA_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < 9LL * mesh->nt; ++i)
      if (!std::isfinite(midpoints[i])) {
        set_error("gca_build_p1_curved: non-finite edge point");
        return GCA_ERR_NUMERIC;
      }
  }
  h = std::make_unique<gca_h2>();
  GCA_TRY_CUDA(cudaGetDevice(&h->device));
  h->device += test_hooks().device_skew;
  h->op = op;
  h->params = *prm;
  h->n = p1 ? mesh->nv : mesh->nt;
  h->nv = mesh->nv;
  h->nc = tree->nclusters;
  h->m = prm->box_gauss_m;
  h->k = 6 * h->m * h->m;
  n = h->n;
  nc = h->nc;
  k = h->k;
  ntri = mesh->nt;
  margin = prm->omega_margin < 0.0 ? 1.0 / (4.0 * prm->eta) : prm->omega_margin;
  rules = make_rules(h->m, prm->sauter_q);

  h->perm.assign(tree->perm, tree->perm + n);
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

  // geometry upload
  vert.assign(mesh->vertices, mesh->vertices + 3LL * mesh->nv);
  tri.assign(mesh->triangles, mesh->triangles + 3LL * ntri);
  GCA_TRY(upload(h->d_vert, vert, st));
  GCA_TRY(upload(h->d_tri, tri, st));
  GCA_TRY(upload(h->d_perm, h->perm, st));
  GCA_TRY(upload(h->d_begin, h->begin, st));
  GCA_TRY(upload(h->d_end, h->end, st));
  GCA_TRY(d_tq.alloc(sizeof(P4) * 7 * (size_t)ntri));
  if (op == 1) GCA_TRY(d_nrm.alloc(sizeof(double) * 3 * (size_t)ntri));
  GCA_TRY(d_area2.alloc(sizeof(double) * (size_t)ntri));
  if (p1) {
    GCA_TRY(upload(d_sup_ptr, sup_ptr, st));
    GCA_TRY(upload(d_sup_item, sup_item, st));
  }
  if (curved) {
    std::vector<double> mids(midpoints, midpoints + 9LL * ntri);
    GCA_TRY(upload(d_mid, mids, st));
    GCA_TRY_CUDA(cudaStreamSynchronize(st));  // mids is a local
  }
  GCA_TRY(d_box.alloc(sizeof(double) * 6 * (size_t)nc));
  GCA_TRY(d_status.alloc(sizeof(int)));
  GCA_TRY_CUDA(cudaMemsetAsync(d_status.p, 0, sizeof(int), st));
  {
    PhaseScope ps__("tri_geom", st);
    if (curved)
      k_tri_geom_curved<<<blocks_for(ntri, 128), 128, 0, st>>>(ntri, h->d_vert.as<double>(), h->d_tri.as<int>(),
                                                               d_mid.as<double>(), rules, d_tq.as<P4>(),
                                                               d_area2.as<double>());
    else
      k_tri_geom<<<blocks_for(ntri, 128), 128, 0, st>>>(ntri, h->d_vert.as<double>(), h->d_tri.as<int>(), rules,
                                                    d_tq.as<P4>(), d_area2.as<double>(),
                                                    op == 1 ? d_nrm.as<double>() : nullptr);
  }
  {
    PhaseScope ps__("cluster_boxes", st);
    if (curved)
      k_p1c_boxes<<<blocks_for(32LL * nc, 128), 128, 0, st>>>(
          nc, h->d_begin.as<int>(), h->d_end.as<int>(), h->d_perm.as<int>(), d_sup_ptr.as<int>(),
          d_sup_item.as<int>(), h->d_tri.as<int>(), h->d_vert.as<double>(), d_mid.as<double>(),
          d_box.as<double>());
    else if (p1)
      k_p1_boxes<<<blocks_for(32LL * nc, 128), 128, 0, st>>>(
          nc, h->d_begin.as<int>(), h->d_end.as<int>(), h->d_perm.as<int>(), d_sup_ptr.as<int>(),
          d_sup_item.as<int>(), h->d_tri.as<int>(), h->d_vert.as<double>(), d_box.as<double>());
    else
      k_cluster_boxes<<<blocks_for(32LL * nc, 128), 128, 0, st>>>(
          nc, h->d_begin.as<int>(), h->d_end.as<int>(), h->d_perm.as<int>(), h->d_tri.as<int>(),
          h->d_vert.as<double>(), d_box.as<double>());
  }
  GCA_TRY_CUDA(cudaGetLastError());
  box.assign(6 * (size_t)nc, 0.0);
  GCA_TRY_CUDA(cudaMemcpyAsync(box.data(), d_box.p, box.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  GCA_TRY_CUDA(cudaStreamSynchronize(st));
  box_diameters(box, diam);
  // split nodes of the coupling entries: origin at the root box's centre,
  // grid step 2^(E - 22) with 2^E above the box's largest half width
  near_r2 = 0.f;  // float-pair entries of the near field need |d| >= 2^(E - 8)
  {
    double half = 0.0, o[3];
    for (int d = 0; d < 3; ++d) {
      o[d] = 0.5 * (box[d] + box[3 + d]);
      half = std::max(half, 0.5 * (box[3 + d] - box[d]));
    }
    int E = 0;
    std::frexp(std::max(half, 1e-300), &E);  // half < 2^E
    if (E < -40 || E > 40) {
      // |d|^2 and the grid must stay inside float's exponent range
      set_error("gca_build: mesh half width outside [2^-41, 2^40]; rescale the coordinates");
      return GCA_ERR_UNSUPPORTED;
    }
    const double g = std::ldexp(1.0, E - 22);
    near_r2 = (float)std::ldexp(1.0, 2 * (E - 8));
    GCA_TRY(d_tn.alloc(sizeof(SplitNode) * 7 * (size_t)ntri));
    PhaseScope ps__("split_nodes", st);
    k_split_nodes<<<blocks_for(7LL * ntri, 256), 256, 0, st>>>(7LL * ntri, d_tq.as<P4>(), o[0], o[1], o[2], g,
                                                               d_tn.as<SplitNode>());
  }
  block_tree(h->child0, h->child1, box, diam, prm->eta, h->far_t, h->far_s, h->near_t, h->near_s);
  GCA_TRY(upload(d_diam, diam, st));
  // the symmetric operators (G of Eq. 1 in either basis, its single-level
  // GCA) on a block tree whose blocks all come with their mirrors
  {
    std::vector<int> far_mirror;
    h->mirrored = (op == 0 || op == 3 || p1) && blocks_mirrored(h->far_t, h->far_s, far_mirror) &&
                  blocks_mirrored(h->near_t, h->near_s, h->near_mirror);
    if (!h->mirrored) h->near_mirror.clear();
  }

  // box quadrature
  GCA_TRY(d_zq.alloc(sizeof(P4) * (size_t)nc * k));
  {
    PhaseScope ps__("box_quad", st);
    k_box_quad<<<blocks_for((int64_t)nc * k, 128), 128, 0, st>>>(nc, rules, d_box.as<double>(),
                                                                 d_diam.as<double>(), margin,
                                                                 d_zq.as<P4>());
  }
  GCA_TRY_CUDA(cudaGetLastError());

  // A cluster basis enters the matrix only through the admissible blocks of
  // the cluster and, by nestedness, of its ancestors (Sect. 4); the bases of
  // the other clusters are not built (rank 0).
  needed.assign(nc, 0);
  for (size_t b = 0; b < h->far_t.size(); ++b) needed[h->far_t[b]] = needed[h->far_s[b]] = 1;
  // single-level bases (op 3) and Green quadrature (op 4) serve only the
  // clusters of the blocks themselves; nested bases also their descendants
  single = op == 3 || op == 4;
  for (int L = 0; L < h->depth && !single; ++L)
    for (int c : h->by_level[L])
      if (needed[c] && h->child0[c] >= 0) needed[h->child0[c]] = needed[h->child1[c]] = 1;

  // Nested bases, level by level from the deepest (kind 0: the cluster bases
  // V, E of the rows from A_tau; kind 1: the double layer's column bases W, F
  // from its column matrix): ranks, pivots in the pool d_piv (offsets poff),
  // and the row-major float64 leaf bases and transfer matrices.
  GCA_TRY(aca.init(k));
  return GCA_OK;
}

int BasisPass::begin() {
    const int nc = b.nc, k = b.k;
    gca_h2* h = b.h.get();
    std::vector<int>& rank = *o.rank;
    std::vector<int64_t>& poff = *o.poff;
    rank.assign(nc, 0);
    poff.assign(nc, -1);
    vh_off.assign(nc, -1);
    rows_of.assign(nc, 0);
    piv_cap = 0;
    vh_cap = 0;
    for (int c = 1; c < nc; ++c) {
      // upper bounds, refined per level below
      piv_cap += std::min<int64_t>(h->end[c] - h->begin[c], 2 * k);
    }
    cudaStream_t st = b.st;
    GCA_TRY(d_piv.alloc(sizeof(int) * (size_t)std::max<int64_t>(piv_cap, 1)));
    GCA_TRY(d_rank.alloc(sizeof(int) * (size_t)nc));
    GCA_TRY_CUDA(cudaMemsetAsync(d_rank.p, 0, sizeof(int) * nc, st));
    // V^ pool: rows <= min(|tau-hat|, 4k) for every cluster bounds its size
    vh_used = 0;
    piv_used = 0;
    for (int c = 1; c < nc; ++c) {
      int64_t rows = (h->child0[c] < 0 || b.single) ? (h->end[c] - h->begin[c])
                                                  : std::min<int64_t>(h->end[c] - h->begin[c], 4 * k);
      vh_cap += rows * std::min<int64_t>(rows, 2 * k);
    }
    GCA_TRY(d_vh.alloc(sizeof(double) * (size_t)std::max<int64_t>(vh_cap, 1)));
    am = AcaMesh{h->d_perm.as<int>(), b.d_tq.as<P4>(), b.d_zq.as<P4>(), d_piv.as<int>(), d_vh.as<double>(),
                 d_rank.as<int>(), b.d_nrm.as<double>(), b.d_sup_ptr.as<int>(), b.d_sup_item.as<int>(), {},
                 b.d_status.as<int>()};
    std::memcpy(am.bary, b.rules.bary, sizeof(am.bary));
    return GCA_OK;
}

int BasisPass::jobs(int L, int mesh_index, std::vector<AcaJob>& out) {
      const int k = b.k;
      gca_h2* h = b.h.get();
      std::vector<int>& rank = *o.rank;
      std::vector<int64_t>& poff = *o.poff;
      if (L > h->depth) return GCA_OK;
      for (int c : h->by_level[L]) {
        if (!b.needed[c]) continue;
        AcaJob j{};
        j.c = c;
        j.kind = kind;
        j.leaf = h->child0[c] < 0 || b.single;  // single-level: A_tau on all of tau's triangles
        if (j.leaf) {
          j.rows = h->end[c] - h->begin[c];
          j.tbegin = h->begin[c];
        } else {
          const int c0 = h->child0[c], c1 = h->child1[c];
          j.r0 = rank[c0];
          j.rows = j.r0 + rank[c1];
          j.piv0 = poff[c0];
          j.piv1 = poff[c1];
        }
        j.rmax = std::min(j.rows, 2 * k);
        j.mesh = mesh_index;
        j.diam = b.diam[c];
        j.p_off = piv_used;
        poff[c] = piv_used;
        piv_used += j.rmax;
        j.vh_off = vh_used;
        vh_off[c] = vh_used;
        vh_used += (int64_t)j.rows * j.rmax;
        rows_of[c] = j.rows;
        out.push_back(j);
      }
      if (piv_used > piv_cap || vh_used > vh_cap) {
        set_error("gca_build: internal pool bound exceeded");
        return GCA_ERR_INVALID_ARG;
      }
      return GCA_OK;
}

int BasisPass::after() {
    GCA_TRY(check_status(b.d_status, b.st, "cross approximation"));
    GCA_TRY_CUDA(cudaMemcpyAsync(o.rank->data(), d_rank.p, sizeof(int) * b.nc, cudaMemcpyDeviceToHost, b.st));
    GCA_TRY_CUDA(cudaStreamSynchronize(b.st));
    return GCA_OK;
}

int BasisPass::end() {
    const int nc = b.nc;
    const bool single = b.single;
    gca_h2* h = b.h.get();
    cudaStream_t st = b.st;
    std::vector<int>& rank = *o.rank;
    // row-major leaf bases and transfer matrices from the V^ pool
    o.voff->assign(nc, -1);
    o.eoff->assign(nc, -1);
    *o.v_entries = 0;
    *o.e_entries = 0;
    for (int c = 1; c < nc; ++c)
      if (h->child0[c] < 0 || single) {
        (*o.voff)[c] = *o.v_entries;
        *o.v_entries += (int64_t)(h->end[c] - h->begin[c]) * rank[c];
      }
    for (int c = 1; c < nc; ++c)
      if (h->parent[c] > 0 && !single) {
        (*o.eoff)[c] = *o.e_entries;
        *o.e_entries += (int64_t)rank[c] * rank[h->parent[c]];
      }
    std::vector<Segment> vseg, eseg;
    for (int c = 1; c < nc; ++c) {
      const int r = rank[c];
      if (r == 0) continue;  // unused basis
      if (h->child0[c] < 0 || single) {
        vseg.push_back({vh_off[c], (*o.voff)[c], (int64_t)rows_of[c] * r});
      } else {
        const int c0 = h->child0[c], c1 = h->child1[c];
        eseg.push_back({vh_off[c], (*o.eoff)[c0], (int64_t)rank[c0] * r});
        eseg.push_back({vh_off[c] + (int64_t)rank[c0] * r, (*o.eoff)[c1], (int64_t)rank[c1] * r});
      }
    }
    GCA_TRY(o.V64->alloc(sizeof(double) * *o.v_entries));
    GCA_TRY(o.E64->alloc(sizeof(double) * *o.e_entries));
    DevMem d_seg;
    for (auto* sv : {&vseg, &eseg}) {
      if (sv->empty()) continue;
      GCA_TRY(d_seg.reserve(sizeof(Segment) * sv->size()));
      GCA_TRY_CUDA(cudaMemcpyAsync(d_seg.p, sv->data(), sizeof(Segment) * sv->size(),
                                   cudaMemcpyHostToDevice, st));
      const bool isv = sv == &vseg;
      {
        PhaseScope ps__("pack", st);
        k_pack<<<(unsigned)sv->size(), 256, 0, st>>>(d_seg.as<Segment>(), d_vh.as<double>(),
                                                     isv ? o.V64->as<double>() : o.E64->as<double>());
      }
      GCA_TRY_CUDA(cudaGetLastError());
      GCA_TRY_CUDA(cudaStreamSynchronize(st));  // d_seg is reused
    }
    return GCA_OK;
}

int Builder::rows() {
  // rows: the Galerkin single layer's bases (op 0, 1; single level for op 3),
  // the collocation rows (op 2), or the Green quadrature matrices A_tau of
  // the clusters of the blocks (op 4: "rank" 2k, no pivots)
  if (op == 4) {
    GCA_TRY(near_field());
    h->rank.assign(nc, 0);
    h->voff.assign(nc, -1);
    h->eoff.assign(nc, -1);
    h->v_entries = 0;
    std::vector<GqJob> gj;
    for (int c = 1; c < nc; ++c)
      if (needed[c]) {
        h->rank[c] = 2 * k;
        h->voff[c] = h->v_entries;
        gj.push_back({c, c, h->v_entries});
        h->v_entries += (int64_t)(h->end[c] - h->begin[c]) * 2 * k;
      }
    GCA_TRY(h->V64.alloc(sizeof(double) * (size_t)std::max<int64_t>(h->v_entries, 1)));
    GCA_TRY(h->E64.alloc(sizeof(double)));
    DevMem d_gj;
    GCA_TRY(upload(d_gj, gj, st));
    if (!gj.empty()) {
      PhaseScope ps__("gq_rows", st);
      k_gq_rows<<<(unsigned)gj.size(), 256, 0, st>>>(d_gj.as<GqJob>(), k, h->d_begin.as<int>(), h->d_end.as<int>(),
                                                    h->d_perm.as<int>(), d_tq.as<P4>(), d_zq.as<P4>(),
                                                    d_diam.as<double>(), h->V64.as<double>());
      GCA_TRY_CUDA(cudaGetLastError());
    }
    h->poff.assign(nc, 0);
    GCA_TRY(d_piv.alloc(sizeof(int)));
    GCA_TRY_CUDA(cudaStreamSynchronize(st));  // gj is a local
  } else if (h->two_sided()) {
    // columns: the double layer's own bases (op 1) or the Galerkin single
    // layer's (op 2), in the same launches as the rows
    auto rp = rows_pass();
    BasisPass cp(*this, op == 1 ? 1 : 0,
                 BasisOut{&h->rank2, &h->poff2, &h->voff2, &h->eoff2, &h->w_entries, &h->f_entries, &h->W64,
                          &h->F64},
                 d_piv2, d_rank2, piv2_used);
    GCA_TRY(run_passes({rp.get(), &cp}, true));
  } else {
    GCA_TRY(run_passes({rows_pass().get()}, true));
  }
  return GCA_OK;
}

// The near field (Sect. 8) needs the block tree and the quadrature nodes but
// no basis.  Its entry and Sauter-Schwab kernels run on a side stream forked
// from the build stream after the geometry, beside the cross approximation,
// and finish() joins them back before the panels.  The touching-pair kernels
// are launched for the bound `cap` of their lists (warps beyond the count
// found on the device return at once), so no host read-back sits between
// the entry kernels and them.
int Builder::near_field() {
  const int nnear = (int)h->near_t.size();
  h->noff.assign(nnear + 1, 0);
  for (int b = 0; b < nnear; ++b) {
    const int t = h->near_t[b], s = h->near_s[b];
    h->noff[b + 1] = h->noff[b] + (int64_t)(h->end[t] - h->begin[t]) * (h->end[s] - h->begin[s]);
  }
  h->n_entries = h->noff[nnear];
  GCA_TRY(upload(h->d_near_t, h->near_t, st));
  GCA_TRY(upload(h->d_near_s, h->near_s, st));
  GCA_TRY(upload(h->d_noff, h->noff, st));
  GCA_TRY(h->N64.alloc(sizeof(double) * h->n_entries));
  // bound on touching ordered pairs: sum over vertices of (triangles at v)^2
  valence.assign(mesh->nv, 0);
  for (int64_t t = 0; t < 3LL * ntri; ++t) valence[tri[t]]++;
  cap = 0;
  for (auto v : valence) cap += v * v;
  // the nodal basis: a touching pair occurs in the unions of at most three
  // row and three column leaves
  if (p1) cap *= 9;
  GCA_TRY(d_items.alloc((p1 ? sizeof(P1Item) : sizeof(SingularItem) * 3) * (size_t)std::max<int64_t>(cap, 1)));
  GCA_TRY(d_counts.alloc(sizeof(unsigned long long) * 5));
  GCA_TRY(d_status_near.alloc(sizeof(int)));
  f64_entries = (prm->flags & GCA_F64_ENTRIES) && (op == 0 || op == 3 || op == 4);
  // sample tables: the single layer's (float pairs, or float64 with
  // GCA_F64_ENTRIES), the double layer's (float64, vertex and edge), the
  // nodal basis's (float pairs with the barycentric slopes; curved: float64
  // with xi sampled); the collocation's Duffy rule (4q Gauss points on [0, 1])
  std::vector<SSEntry> ss;
  std::vector<SSEntry64> ss64;
  std::vector<SSEntryP1> ssp1;
  std::vector<SSEntryCurvedSplit> ssc;
  std::vector<double2> duffy;
  int ss_off[4] = {0, 0, 0, 0}, ss64_off[4] = {0, 0, 0, 0};
  int3 t_off{0, 0, 0}, t_cnt{0, 0, 0};
  if (p1 && curved) {
    sauter_table_curved_split<1>(rules, ssc);
    t_cnt.x = (int)ssc.size();
    sauter_table_curved_split<2>(rules, ssc);
    t_off.y = t_cnt.x;
    t_cnt.y = (int)ssc.size() - t_off.y;
    sauter_table_curved_split<3>(rules, ssc);
    t_off.z = t_off.y + t_cnt.y;
    t_cnt.z = (int)ssc.size() - t_off.z;
    GCA_TRY(upload(d_tab, ssc, st));
  } else if (p1) {
    sauter_table_p1<1>(rules, ssp1);
    t_cnt.x = (int)ssp1.size();
    sauter_table_p1<2>(rules, ssp1);
    t_off.y = t_cnt.x;
    t_cnt.y = (int)ssp1.size() - t_off.y;
    sauter_table_p1<3>(rules, ssp1);
    t_off.z = t_off.y + t_cnt.y;
    t_cnt.z = (int)ssp1.size() - t_off.z;
    GCA_TRY(upload(d_tab, ssp1, st));
  } else if (op == 1 || f64_entries) {
    sauter_table64<1>(rules, ss64);
    ss64_off[1] = (int)ss64.size();
    sauter_table64<2>(rules, ss64);
    ss64_off[2] = (int)ss64.size();
    if (f64_entries) sauter_table64<3>(rules, ss64);
    ss64_off[3] = (int)ss64.size();
    GCA_TRY(upload(d_tab, ss64, st));
  } else if (op == 2) {
    const int nd = 4 * prm->sauter_q;
    std::vector<double> xt(nd), wt(nd);
    gauss_legendre(nd, xt.data(), wt.data());
    for (int i = 0; i < nd; ++i) duffy.push_back(make_double2(0.5 * (xt[i] + 1.0), 0.5 * wt[i]));
    GCA_TRY(upload(d_tab, duffy, st));
  } else {
    sauter_table<1>(rules, ss);
    ss_off[1] = (int)ss.size();
    sauter_table<2>(rules, ss);
    ss_off[2] = (int)ss.size();
    sauter_table<3>(rules, ss);
    ss_off[3] = (int)ss.size();
    GCA_TRY(upload(d_tab, ss, st));
  }
  // the nodal basis: the support unions of the near-field leaves and the
  // near blocks, mirrored pairs together
  std::vector<UnionJob> ujobs;
  std::vector<P1Block> p1near;
  int pcap = 1, max_len = 1;
  if (p1) {
    std::vector<int> uleaf(nc, -1);
    int64_t rows_total = 0, max_m = 1;
    for (int b = 0; b < nnear; ++b)
      for (int c : {h->near_t[b], h->near_s[b]})
        if (uleaf[c] < 0) {
          int64_t m = 0;
          for (int i = h->begin[c]; i < h->end[c]; ++i) m += valence[h->perm[i]];
          ujobs.push_back(UnionJob{h->d_perm.as<int>() + h->begin[c], h->end[c] - h->begin[c], 0, rows_total});
          uleaf[c] = (int)ujobs.size() - 1;
          rows_total += m;
          max_m = std::max(max_m, m);
          max_len = std::max(max_len, h->end[c] - h->begin[c]);
        }
    while (pcap < max_m) pcap <<= 1;
    if (pcap > kUnionMax) {
      set_error("gca_build_p1: a support union has more than 16384 entries");
      return GCA_ERR_UNSUPPORTED;
    }
    for (int b = 0; b < nnear; ++b) {
      const int t = h->near_t[b], s = h->near_s[b];
      int m = -1;
      if (t != s) {
        int lo = 0, hi = nnear;
        while (lo < hi) {
          const int mid = (lo + hi) / 2;
          if (h->near_t[mid] < s || (h->near_t[mid] == s && h->near_s[mid] < t)) lo = mid + 1; else hi = mid;
        }
        if (lo < nnear && h->near_t[lo] == s && h->near_s[lo] == t) m = lo;
      }
      if (t > s && m >= 0) continue;  // computed with its mirror
      const int nt_ = h->end[t] - h->begin[t], ns_ = h->end[s] - h->begin[s];
      p1near.push_back(P1Block{h->noff[b], m >= 0 ? h->noff[m] : -1, ns_, nt_, uleaf[t], uleaf[s]});
    }
    GCA_TRY(upload(d_nujobs, ujobs, st));
    GCA_TRY(d_nucount.alloc(sizeof(int) * std::max<size_t>(ujobs.size(), 1)));
    GCA_TRY(d_nurows.alloc(sizeof(int4) * (size_t)std::max<int64_t>(rows_total, 1)));
    GCA_TRY(upload(d_p1near, p1near, st));
  }
  // fork: the side stream waits for everything enqueued so far on the build
  // stream (geometry, split nodes, the uploads above)
  {
    int least = 0, greatest = 0;
    GCA_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    GCA_TRY_CUDA(cudaStreamCreateWithPriority(&near_st_, cudaStreamNonBlocking, least));
  }
  GCA_TRY_CUDA(cudaEventCreateWithFlags(&near_ready_, cudaEventDisableTiming));
  GCA_TRY_CUDA(cudaEventCreateWithFlags(&near_done_, cudaEventDisableTiming));
  GCA_TRY_CUDA(cudaEventRecord(near_ready_, st));
  cudaStream_t ns = near_st_;
  GCA_TRY_CUDA(cudaStreamWaitEvent(ns, near_ready_, 0));
  GCA_TRY_CUDA(cudaMemsetAsync(d_counts.p, 0, sizeof(unsigned long long) * 5, ns));
  GCA_TRY_CUDA(cudaMemsetAsync(d_status_near.p, 0, sizeof(int), ns));
  const int* tri_d = h->d_tri.as<int>();
  const double* vert_d = h->d_vert.as<double>();
  const double* a2 = d_area2.as<double>();
  double* N64 = h->N64.as<double>();
  unsigned long long* cnt = d_counts.as<unsigned long long>();
  int* nstat = d_status_near.as<int>();
  const unsigned sing_blocks = blocks_for(32LL * std::max<int64_t>(cap, 1), 256);
  if (nnear == 0) {
    // nothing to integrate
  } else if (p1) {
    GCA_TRY_CUDA(cudaMemsetAsync(N64, 0, sizeof(double) * h->n_entries, ns));
    if (!ujobs.empty()) {
      const size_t smem = sizeof(unsigned long long) * (size_t)pcap + sizeof(int) * (size_t)(max_len + 1);
      GCA_TRY_CUDA(cudaFuncSetAttribute(k_support_union, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      PhaseScope ps__("p1_union", ns);
      k_support_union<<<(unsigned)ujobs.size(), 256, smem, ns>>>(d_nujobs.as<UnionJob>(), d_sup_ptr.as<int>(),
                                                                d_sup_item.as<int>(), pcap, d_nurows.as<int4>(),
                                                                d_nucount.as<int>(), nstat);
      GCA_TRY_CUDA(cudaGetLastError());
    }
    if (!p1near.empty()) {
      PhaseScope ps__("p1_near_entries", ns);
      k_p1_entries<true><<<(unsigned)p1near.size(), 256, 0, ns>>>(
          d_p1near.as<P1Block>(), d_nujobs.as<UnionJob>(), d_nucount.as<int>(), d_nurows.as<int4>(), tri_d,
          d_tq.as<P4>(), d_tn.as<SplitNode>(), rules, bary_split(), near_r2, N64, d_items.as<P1Item>(), cap, cnt,
          nstat);
      GCA_TRY_CUDA(cudaGetLastError());
    }
    PhaseScope ps__("p1_singular", ns);
    if (curved)
      k_p1c_singular_split<<<sing_blocks, 256, 0, ns>>>(d_items.as<P1Item>(), cnt, cap, tri_d, vert_d,
                                                         d_mid.as<double>(), d_tab.as<SSEntryCurvedSplit>(), t_off,
                                                         t_cnt, N64);
    else
      k_p1_singular<<<sing_blocks, 256, 0, ns>>>(d_items.as<P1Item>(), cnt, cap, tri_d, vert_d, a2,
                                                  d_tab.as<SSEntryP1>(), t_off, t_cnt, N64);
    GCA_TRY_CUDA(cudaGetLastError());
  } else if (op == 2) {
    const size_t smem = sizeof(P4) * 7 * (size_t)h->max_leaf;
    GCA_TRY_CUDA(cudaFuncSetAttribute(k_col_near_entries, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhaseScope ps__("col_near_entries", ns);
    // the collocation's diagonal entries are integrated in place
    k_col_near_entries<<<nnear, 256, smem, ns>>>(
        h->d_near_t.as<int>(), h->d_near_s.as<int>(), h->d_noff.as<int64_t>(), h->d_begin.as<int>(),
        h->d_end.as<int>(), h->d_perm.as<int>(), tri_d, vert_d, d_tq.as<P4>(), d_tab.as<double2>(),
        (int)duffy.size(), N64, cnt);
    GCA_TRY_CUDA(cudaGetLastError());
  } else {
    const SingularItem* items = d_items.as<SingularItem>();
    if (op == 1) {
      const size_t smem =
          ((sizeof(P4) + sizeof(SplitNode)) * 7 + sizeof(double) * 3 + sizeof(float) * 6) * (size_t)h->max_leaf;
      GCA_TRY_CUDA(cudaFuncSetAttribute(k_dl_near_entries, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      PhaseScope ps__("dl_near_entries", ns);
      k_dl_near_entries<<<nnear, 256, smem, ns>>>(
          h->d_near_t.as<int>(), h->d_near_s.as<int>(), h->d_noff.as<int64_t>(), h->d_begin.as<int>(),
          h->d_end.as<int>(), h->d_perm.as<int>(), tri_d, d_tq.as<P4>(), d_tn.as<SplitNode>(), near_r2,
          d_nrm.as<double>(), N64, d_items.as<SingularItem>(), cap, cnt, nstat);
      GCA_TRY_CUDA(cudaGetLastError());
    } else {
      const size_t smem = (sizeof(P4) + sizeof(SplitNode)) * 7 * (size_t)h->max_leaf;
      auto kern = f64_entries ? k_near_entries<true> : k_near_entries<false>;
      GCA_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      PhaseScope ps__("near_entries", ns);
      kern<<<nnear, 256, smem, ns>>>(h->d_near_t.as<int>(), h->d_near_s.as<int>(), h->d_noff.as<int64_t>(),
                                     h->d_begin.as<int>(), h->d_end.as<int>(), h->d_perm.as<int>(), tri_d,
                                     d_tq.as<P4>(), d_tn.as<SplitNode>(), near_r2, N64, d_items.as<SingularItem>(),
                                     cap, cnt, nstat);
      GCA_TRY_CUDA(cudaGetLastError());
    }
    PhaseScope ps_sing("singular", ns);
    ps_sing.launches(op == 1 ? 2 : 3);
    if (op == 1) {
      const SSEntry64* tab64 = d_tab.as<SSEntry64>();
      k_dl_singular<1><<<sing_blocks, 256, 0, ns>>>(items, cnt, cap, tri_d, vert_d, a2, d_nrm.as<double>(), tab64,
                                                     ss64_off[1], N64);
      k_dl_singular<2><<<sing_blocks, 256, 0, ns>>>(items + cap, cnt, cap, tri_d, vert_d, a2, d_nrm.as<double>(),
                                                     tab64 + ss64_off[1], ss64_off[2] - ss64_off[1], N64);
    } else if (f64_entries) {
      const SSEntry64* tab64 = d_tab.as<SSEntry64>();
      k_singular64<1><<<sing_blocks, 256, 0, ns>>>(items, cnt, cap, tri_d, vert_d, a2, tab64, ss64_off[1], N64);
      k_singular64<2><<<sing_blocks, 256, 0, ns>>>(items + cap, cnt, cap, tri_d, vert_d, a2, tab64 + ss64_off[1],
                                                    ss64_off[2] - ss64_off[1], N64);
      k_singular64<3><<<sing_blocks, 256, 0, ns>>>(items + 2 * cap, cnt, cap, tri_d, vert_d, a2, tab64 + ss64_off[2],
                                                    ss64_off[3] - ss64_off[2], N64);
    } else {
      const SSEntry* tab = d_tab.as<SSEntry>();
      k_singular<1><<<sing_blocks, 256, 0, ns>>>(items, cnt, cap, tri_d, vert_d, a2, tab, ss_off[1], N64);
      k_singular<2><<<sing_blocks, 256, 0, ns>>>(items + cap, cnt, cap, tri_d, vert_d, a2, tab + ss_off[1],
                                                  ss_off[2] - ss_off[1], N64);
      k_singular<3><<<sing_blocks, 256, 0, ns>>>(items + 2 * cap, cnt, cap, tri_d, vert_d, a2, tab + ss_off[2],
                                                  ss_off[3] - ss_off[2], N64);
    }
    GCA_TRY_CUDA(cudaGetLastError());
  }
  GCA_TRY_CUDA(cudaEventRecord(near_done_, ns));
  // the host tables above are pageable and were copied when upload returned
  return GCA_OK;
}

int Builder::finish(gca_h2** out) {
  h->xoff.assign(nc + 1, 0);
  for (int c = 0; c < nc; ++c) h->xoff[c + 1] = h->xoff[c] + h->rank[c];
  h->rank_sum = h->xoff[nc];
  h->max_rank = *std::max_element(h->rank.begin(), h->rank.end());
  if (h->two_sided()) {
    // the column bases were built with the rows (rows())
    h->xoff2.assign(nc + 1, 0);
    for (int c = 0; c < nc; ++c) h->xoff2[c + 1] = h->xoff2[c] + h->rank2[c];
    h->rank_sum2 = h->xoff2[nc];
    h->max_rank2 = *std::max_element(h->rank2.begin(), h->rank2.end());
  }

  // Offsets of the coupling and near-field coefficients, the panel layout and
  // every device buffer of the rest of the build are set up first, so that
  // the host has nothing to do but the product plan while the device
  // computes the entries.
  const int nfar = (int)h->far_t.size(), nnear = (int)h->near_t.size();
  h->piv.resize(std::max<int64_t>(piv_used, 1));
  if (piv_used > 0)
    GCA_TRY_CUDA(cudaMemcpyAsync(h->piv.data(), d_piv.p, sizeof(int) * piv_used, cudaMemcpyDeviceToHost, st));
  GCA_TRY(upload(h->d_rank, h->rank, st));
  DevMem d_poff, d_poff2, d_rank2v;
  GCA_TRY(upload(d_poff, h->poff, st));
  if (h->two_sided()) {
    h->piv2.resize(std::max<int64_t>(piv2_used, 1));
    GCA_TRY_CUDA(cudaMemcpyAsync(h->piv2.data(), d_piv2.p, sizeof(int) * piv2_used, cudaMemcpyDeviceToHost, st));
    GCA_TRY(upload(d_poff2, h->poff2, st));
    GCA_TRY(upload(d_rank2v, h->rank2, st));
  }
  // coupling blocks: r_tau x r_sigma (single layer) or r_tau x r'_sigma (double layer)
  const std::vector<int>& rcol = h->two_sided() ? h->rank2 : h->rank;
  h->soff.assign(nfar + 1, 0);
  for (int b = 0; b < nfar; ++b)
    h->soff[b + 1] = h->soff[b] + (int64_t)h->rank[h->far_t[b]] *
                                      (op == 4 ? h->end[h->far_s[b]] - h->begin[h->far_s[b]] : rcol[h->far_s[b]]);
  h->s_entries = h->soff[nfar];
  GCA_TRY(upload(h->d_far_t, h->far_t, st));
  GCA_TRY(upload(h->d_far_s, h->far_s, st));
  GCA_TRY(upload(h->d_soff, h->soff, st));
  GCA_TRY(h->S64.alloc(sizeof(double) * h->s_entries));
  // mirrored pairs of coupling blocks: the block list is sorted by (row,
  // column) cluster, and the block tree is symmetric (the admissibility
  // condition and the splitting rule do not depend on the order of tau and
  // sigma); a block whose mirror is missing is computed alone
  std::vector<int2> pairs;
  pairs.reserve(nfar / 2 + 1);
  for (int b = 0; b < nfar && (op == 0 || op == 3 || p1); ++b) {
    const int t = h->far_t[b], s = h->far_s[b];
    int m = -1;
    {
      int lo = 0, hi = nfar;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (h->far_t[mid] < s || (h->far_t[mid] == s && h->far_s[mid] < t)) lo = mid + 1; else hi = mid;
      }
      if (lo < nfar && h->far_t[lo] == s && h->far_s[lo] == t) m = lo;
    }
    if (m < 0)
      pairs.push_back(make_int2(b, -1));
    else if (t < s)
      pairs.push_back(make_int2(b, m));
  }
  DevMem d_pairs;
  GCA_TRY(upload(d_pairs, pairs, st));
  DevMem d_counts_far;  // the nodal basis's couplings: count of regular pairs
  if (p1) {
    GCA_TRY_CUDA(cudaMemsetAsync(h->S64.p, 0, sizeof(double) * h->s_entries, st));
    GCA_TRY(d_counts_far.alloc(sizeof(unsigned long long) * 5));
    GCA_TRY_CUDA(cudaMemsetAsync(d_counts_far.p, 0, sizeof(unsigned long long) * 5, st));
  }
  layout_panels(h.get());
  GCA_TRY(alloc_panels(h.get()));
  DevMem d_pjobs;
  GCA_TRY(d_pjobs.alloc(sizeof(PanelJob) * (size_t)panel_jobs(h.get())));
  GCA_TRY_CUDA(cudaStreamSynchronize(st));  // the host copy of the pivots

  // coupling matrices
  // nodal basis (Sect. 5): support unions of the pivot lists of the
  // clusters in admissible blocks, then the pair-by-pair assembly of the
  // couplings (mirrored blocks together; the near field runs in near_field())
  std::vector<UnionJob> ujobs;
  std::vector<P1Block> p1far;
  DevMem d_ujobs, d_ucount, d_urows, d_p1far;
  if (p1) {
    std::vector<int> upiv(nc, -1);
    int64_t rows_total = 0;
    int64_t max_m = 1;
    int max_len = 1;
    auto add_union = [&](const int* dlist, const int* hlist, int len) {
      int64_t m = 0;
      for (int a = 0; a < len; ++a) m += valence[hlist[a]];
      ujobs.push_back(UnionJob{dlist, len, 0, rows_total});
      rows_total += m;
      max_m = std::max(max_m, m);
      max_len = std::max(max_len, len);
      return (int)ujobs.size() - 1;
    };
    for (int b = 0; b < nfar; ++b)
      for (int c : {h->far_t[b], h->far_s[b]})
        if (upiv[c] < 0)
          upiv[c] = add_union(d_piv.as<int>() + h->poff[c], h->piv.data() + h->poff[c], h->rank[c]);
    int pcap = 1;
    while (pcap < max_m) pcap <<= 1;
    if (pcap > kUnionMax) {
      set_error("gca_build_p1: a support union has more than 16384 entries");
      return GCA_ERR_UNSUPPORTED;
    }
    for (const int2& pr : pairs) {
      const int b = pr.x, m = pr.y, t = h->far_t[b], s = h->far_s[b];
      p1far.push_back(P1Block{h->soff[b], m >= 0 ? h->soff[m] : -1, h->rank[s], h->rank[t], upiv[t], upiv[s]});
    }
    GCA_TRY(upload(d_ujobs, ujobs, st));
    GCA_TRY(d_ucount.alloc(sizeof(int) * std::max<size_t>(ujobs.size(), 1)));
    GCA_TRY(d_urows.alloc(sizeof(int4) * (size_t)std::max<int64_t>(rows_total, 1)));
    GCA_TRY(upload(d_p1far, p1far, st));
    if (!ujobs.empty()) {
      const size_t smem = sizeof(unsigned long long) * (size_t)pcap + sizeof(int) * (size_t)(max_len + 1);
      GCA_TRY_CUDA(cudaFuncSetAttribute(k_support_union, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      PhaseScope ps__("p1_union", st);
      k_support_union<<<(unsigned)ujobs.size(), 256, smem, st>>>(d_ujobs.as<UnionJob>(), d_sup_ptr.as<int>(),
                                                                d_sup_item.as<int>(), pcap, d_urows.as<int4>(),
                                                                d_ucount.as<int>(), d_status.as<int>());
      GCA_TRY_CUDA(cudaGetLastError());
    }
    if (!p1far.empty()) {
      PhaseScope ps__("p1_couple_entries", st);
      k_p1_entries<false><<<(unsigned)p1far.size(), 256, 0, st>>>(
          d_p1far.as<P1Block>(), d_ujobs.as<UnionJob>(), d_ucount.as<int>(), d_urows.as<int4>(),
          h->d_tri.as<int>(), d_tq.as<P4>(), d_tn.as<SplitNode>(), rules, bary_split(), near_r2,
          h->S64.as<double>(), nullptr, 0, d_counts_far.as<unsigned long long>(), d_status.as<int>());
      GCA_TRY_CUDA(cudaGetLastError());
    }
  } else if (nfar > 0 && op == 4) {
    std::vector<GqJob> gj;
    for (int b = 0; b < nfar; ++b) gj.push_back({h->far_t[b], h->far_s[b], h->soff[b]});
    DevMem d_gj;
    GCA_TRY(upload(d_gj, gj, st));
    {
      PhaseScope ps__("gq_factors", st);
      k_gq_factors<<<(unsigned)nfar, 256, 0, st>>>(d_gj.as<GqJob>(), k, h->d_begin.as<int>(), h->d_end.as<int>(),
                                                  h->d_perm.as<int>(), d_tq.as<P4>(), d_zq.as<P4>(),
                                                  d_diam.as<double>(), h->S64.as<double>());
    }
    GCA_TRY_CUDA(cudaGetLastError());
    GCA_TRY_CUDA(cudaStreamSynchronize(st));  // gj is a local
  } else if (nfar > 0 && op == 2) {
    const size_t smem = sizeof(P4) * 7 * (size_t)std::max(h->max_rank2, 1);
    GCA_TRY_CUDA(cudaFuncSetAttribute(k_col_couple, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
      PhaseScope ps__("col_couple_entries", st);
      k_col_couple<<<(unsigned)nfar, 256, smem, st>>>(
          h->d_far_t.as<int>(), h->d_far_s.as<int>(), h->d_soff.as<int64_t>(), h->d_rank.as<int>(),
          d_rank2v.as<int>(), d_poff.as<int64_t>(), d_poff2.as<int64_t>(), d_piv.as<int>(), d_piv2.as<int>(),
          d_tq.as<P4>(), h->S64.as<double>());
    }
    GCA_TRY_CUDA(cudaGetLastError());
  } else if (nfar > 0 && op == 1) {
    const size_t smem = (sizeof(SplitNode) * 7 + sizeof(float) * 6) * (size_t)std::max(h->max_rank2, 1);
    GCA_TRY_CUDA(cudaFuncSetAttribute(k_dl_couple, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
      PhaseScope ps__("dl_couple_entries", st);
      k_dl_couple<<<(unsigned)nfar, 256, smem, st>>>(
          h->d_far_t.as<int>(), h->d_far_s.as<int>(), h->d_soff.as<int64_t>(), h->d_rank.as<int>(),
          d_rank2v.as<int>(), d_poff.as<int64_t>(), d_poff2.as<int64_t>(), d_piv.as<int>(), d_piv2.as<int>(),
          d_tn.as<SplitNode>(), d_nrm.as<double>(), h->S64.as<double>());
    }
    GCA_TRY_CUDA(cudaGetLastError());
  } else if (nfar > 0) {
    const size_t smem = sizeof(SplitNode) * 7 * (size_t)std::max(h->max_rank, 1);
    auto kern = f64_entries ? k_couple_entries<true> : k_couple_entries<false>;
    GCA_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
      PhaseScope ps__("couple_entries", st);
      kern<<<(unsigned)pairs.size(), 256, smem, st>>>(
          d_pairs.as<int2>(), h->d_far_t.as<int>(), h->d_far_s.as<int>(), h->d_soff.as<int64_t>(),
          h->d_rank.as<int>(), d_poff.as<int64_t>(), d_piv.as<int>(), d_tn.as<SplitNode>(), d_tq.as<P4>(),
          h->S64.as<double>());
    }
    GCA_TRY_CUDA(cudaGetLastError());
  }

  // the product plan needs only the ranks, the block lists and the panel
  // offsets: the host computes one direction while the coupling and
  // near-field kernels run, the other while the singular and panel kernels run
  PlanHandle plan = plan_new();
  plan_direction(h.get(), 0, plan.get());
  // the near field: joined back into the build stream; its sticky status and
  // the counts of its pairs by case
  if (near_st_) {
    GCA_TRY_CUDA(cudaStreamWaitEvent(st, near_done_, 0));
    GCA_TRY(check_status(d_status_near, st, "near field"));
    unsigned long long counts[5];
    GCA_TRY_CUDA(cudaMemcpyAsync(counts, d_counts.p, sizeof(counts), cudaMemcpyDeviceToHost, st));
    GCA_TRY_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c <= 3; ++c) h->n_singular[c] = (int64_t)counts[c];
    if (!p1) h->n_singular[0] = h->n_entries - (h->n_singular[1] + h->n_singular[2] + h->n_singular[3]);
  }

  // panel layout for the products, three precisions
  std::vector<PanelJob> panel_host_jobs;  // kept until the synchronisation below
  {
    PhaseScope ps_conv("to_panel", st);
    ps_conv.launches(kPanelKinds);
    GCA_TRY(make_panels(h.get(), d_pjobs, panel_host_jobs, st));
  }
  if (!h->mirrored) plan_direction(h.get(), 1, plan.get());

  GCA_TRY(finish_plan(h.get(), plan.get(), st));
  GCA_TRY_CUDA(cudaStreamSynchronize(st));
  // the float64 panels hold the exported coefficients too (gca_h2_export
  // rebuilds the row-major layout from them), so the row-major copies stay
  // only where there are no float64 panels
  if ((prm->flags & GCA_DROP_EXPORT) || !(prm->flags & GCA_DROP_F64)) {
    h->V64.release();
    h->E64.release();
    h->S64.release();
    h->N64.release();
    h->W64.release();
    h->F64.release();
  }
  h->build_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = h.release();
  return GCA_OK;
}


// The whole construction of one mesh.
int build(const gca_mesh* mesh, const gca_tree* tree, const gca_params* prm, cudaStream_t st,
          gca_h2** out, int op, const double* midpoints) {
  Builder b(mesh, tree, prm, st, op, midpoints);
  GCA_TRY(b.prepare());
  GCA_TRY(b.rows());
  return b.finish(out);
}

// The single layer of several meshes (gca_build_batch) in groups: the
// cross approximations of a group's meshes share one launch per tree level
// (job.mesh selects the mesh), so the coarse levels, which hold few
// clusters per mesh, fill more of the device.  Each mesh is otherwise built
// as by build().
int build_group(int count, const gca_mesh* meshes, const gca_tree* trees, const gca_params* prm, cudaStream_t st,
                gca_h2** out) {
  std::vector<std::unique_ptr<Builder>> bs;
  for (int i = 0; i < count; ++i) {
    bs.push_back(std::make_unique<Builder>(meshes + i, trees + i, prm, st, 0));
    GCA_TRY(bs.back()->prepare());
  }
  std::vector<std::unique_ptr<BasisPass>> passes;
  int depth = 0;
  for (auto& b : bs) {
    passes.push_back(b->rows_pass());
    GCA_TRY(passes.back()->begin());
    depth = std::max(depth, b->h->depth);
  }
  std::vector<AcaMesh> table;
  for (auto& p : passes) table.push_back(p->am);
  DevMem d_table, d_jobs;
  GCA_TRY(upload(d_table, table, st));
  size_t all_clusters = 0, all_rows = 0;
  for (auto& b : bs) {
    all_clusters += (size_t)b->nc;
    all_rows += (size_t)b->n;
  }
  GCA_TRY(bs[0]->aca.reserve_scratch(all_rows, all_clusters));
  GCA_TRY(d_jobs.reserve(sizeof(AcaJob) * all_clusters));  // no reallocation between levels
  // the near fields, once every allocation before the levels is made
  for (auto& b : bs) GCA_TRY(b->near_field());
  std::vector<AcaJob> js;
  for (int L = depth; L >= 1; --L) {
    js.clear();
    for (int i = 0; i < count; ++i) GCA_TRY(passes[i]->jobs(L, i, js));
    if (js.empty()) continue;
    GCA_TRY(bs[0]->aca.launch(js, d_jobs, d_table.as<AcaMesh>(), L, prm->aca_tol, bs[0]->tie, st));
    for (auto& p : passes) GCA_TRY(p->after());
  }
  for (auto& p : passes) GCA_TRY(p->end());
  for (int i = 0; i < count; ++i) GCA_TRY(bs[i]->finish(out + i));
  return GCA_OK;
}

// gca_support_union: the lists' unions on the device, copied back compacted.
int support_union(const gca_mesh* mesh, int nlists, const int32_t* list_ptr, const int32_t* lists,
                  int32_t* rows, int64_t cap, int32_t* counts, cudaStream_t st) {
  GCA_TRY(validate_mesh(mesh));
  if (nlists < 0 || (nlists > 0 && (!list_ptr || !lists || !rows || !counts)) || cap < 0) {
    set_error("gca_support_union: bad arguments");
    return GCA_ERR_INVALID_ARG;
  }
  if (nlists == 0) return GCA_OK;
  std::vector<int> sup_ptr, sup_item;
  GCA_TRY(node_supports(mesh, sup_ptr, sup_item, "gca_support_union"));
  if (list_ptr[0] != 0) {
    set_error("gca_support_union: list_ptr[0] must be 0");
    return GCA_ERR_INVALID_ARG;
  }
  const int64_t total = list_ptr[nlists];
  std::vector<char> seen(mesh->nv, 0);
  std::vector<int64_t> bound(nlists + 1, 0);
  int64_t max_m = 1;
  int max_len = 1;
  for (int l = 0; l < nlists; ++l) {
    if (list_ptr[l + 1] < list_ptr[l]) {
      set_error("gca_support_union: list_ptr not ascending");
      return GCA_ERR_INVALID_ARG;
    }
    int64_t m = 0;
    for (int64_t a = list_ptr[l]; a < list_ptr[l + 1]; ++a) {
      const int v = lists[a];
      if (v < 0 || v >= mesh->nv || seen[v]) {
        set_error("gca_support_union: vertex id out of range or repeated in list " + std::to_string(l));
        return GCA_ERR_INVALID_ARG;
      }
      seen[v] = 1;
      m += sup_ptr[v + 1] - sup_ptr[v];
    }
    for (int64_t a = list_ptr[l]; a < list_ptr[l + 1]; ++a) seen[lists[a]] = 0;
    bound[l + 1] = bound[l] + m;
    max_m = std::max(max_m, m);
    max_len = std::max<int>(max_len, (int)(list_ptr[l + 1] - list_ptr[l]));
  }
  if (bound[nlists] > cap) {
    set_error("gca_support_union: cap below the support entries of the lists");
    return GCA_ERR_INVALID_ARG;
  }
  int pcap = 1;
  while (pcap < max_m) pcap <<= 1;
  if (pcap > kUnionMax) {
    set_error("gca_support_union: a list has more than 16384 support entries");
    return GCA_ERR_UNSUPPORTED;
  }
  DevMem d_ptr, d_item, d_lists, d_jobs, d_rows, d_counts, d_status;
  GCA_TRY(upload(d_ptr, sup_ptr, st));
  GCA_TRY(upload(d_item, sup_item, st));
  std::vector<int> hl(lists, lists + total);
  GCA_TRY(upload(d_lists, hl, st));
  std::vector<UnionJob> jobs(nlists);
  for (int l = 0; l < nlists; ++l)
    jobs[l] = UnionJob{d_lists.as<int>() + list_ptr[l], (int)(list_ptr[l + 1] - list_ptr[l]), 0, bound[l]};
  GCA_TRY(upload(d_jobs, jobs, st));
  GCA_TRY(d_rows.alloc(sizeof(int4) * (size_t)std::max<int64_t>(bound[nlists], 1)));
  GCA_TRY(d_counts.alloc(sizeof(int) * (size_t)nlists));
  GCA_TRY(d_status.alloc(sizeof(int)));
  GCA_TRY_CUDA(cudaMemsetAsync(d_status.p, 0, sizeof(int), st));
  const size_t smem = sizeof(unsigned long long) * (size_t)pcap + sizeof(int) * (size_t)(max_len + 1);
  GCA_TRY_CUDA(cudaFuncSetAttribute(k_support_union, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_support_union<<<(unsigned)nlists, 256, smem, st>>>(d_jobs.as<UnionJob>(), d_ptr.as<int>(), d_item.as<int>(),
                                                       pcap, d_rows.as<int4>(), d_counts.as<int>(),
                                                       d_status.as<int>());
  GCA_TRY_CUDA(cudaGetLastError());
  std::vector<int4> hrows((size_t)std::max<int64_t>(bound[nlists], 1));
  std::vector<int> hc(nlists);
  int hs = 0;
  GCA_TRY_CUDA(cudaMemcpyAsync(hrows.data(), d_rows.p, sizeof(int4) * hrows.size(), cudaMemcpyDeviceToHost, st));
  GCA_TRY_CUDA(cudaMemcpyAsync(hc.data(), d_counts.p, sizeof(int) * nlists, cudaMemcpyDeviceToHost, st));
  GCA_TRY_CUDA(cudaMemcpyAsync(&hs, d_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  GCA_TRY_CUDA(cudaStreamSynchronize(st));
  if (hs) {
    set_error("gca_support_union: internal capacity exceeded");
    return GCA_ERR_INVALID_ARG;
  }
  int64_t at = 0;
  for (int l = 0; l < nlists; ++l) {
    counts[l] = hc[l];
    for (int r = 0; r < hc[l]; ++r, ++at) {
      const int4 v = hrows[bound[l] + r];
      rows[4 * at] = v.x;
      rows[4 * at + 1] = v.y;
      rows[4 * at + 2] = v.z;
      rows[4 * at + 3] = v.w;
    }
  }
  return GCA_OK;
}

}  // namespace gca
