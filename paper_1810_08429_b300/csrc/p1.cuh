// Continuous piecewise linear (nodal) basis functions, Sect. 5: kernels of
// gca_build_p1 and gca_support_union.  Included by build.cu inside its
// anonymous namespace (P4, Rules, kInv4Pi and sauter_piece come from there).
//
// The basis function phi_i of vertex i is linear on every triangle of its
// support T_i (the fan around i), so every integral over T_i is a sum over
// triangles t with the barycentric coordinate lambda_c of i's corner c in t
// as weight.  A support entry packs (t << 2) | c.
//
//   k_p1_boxes      bounding box of the supports of a cluster's vertices
//   k_aca kind 3    Green matrix rows: the 7-point rule on every t in T_i,
//                   each node weighted by lambda_c (in build.cu)
//   k_support_union the union of the supports of an index list (Sect. 5),
//                   one row (t, l0, l1, l2) per triangle: the entries
//                   (t, c, position) of all supports are sorted by (t, c) in
//                   shared memory and the entries of one triangle combined
//   k_p1_entries    one CTA per block: every triangle pair of the two unions
//                   gives a 3 x 3 matrix M_ab = int_t lambda_a int_s g
//                   lambda_b, added to the entries (l_a, l_b) of the block
//                   (and to the mirrored block); disjoint pairs by the 7 x 7
//                   rule in float-pair arithmetic on the FP32 pipe (float64
//                   for close pairs), touching pairs handed to
//   k_p1_singular   Sauter-Schwab with barycentric weights in float-pair
//                   arithmetic, one warp per ordered pair (a mirrored
//                   block's pair is integrated in its own order, as the rule
//                   is not symmetric in rounding and quadrature error)
#pragma once

constexpr int kUnionMax = 16384;  // support entries of one list (shared-memory sort)

// one warp per cluster: min / max over the vertices of the triangles in the
// supports of the cluster's vertices
__global__ void k_p1_boxes(int nc, const int* __restrict__ begin, const int* __restrict__ end,
                           const int* __restrict__ perm, const int* __restrict__ sup_ptr,
                           const int* __restrict__ sup_item, const int* __restrict__ tri,
                           const double* __restrict__ vert, double* __restrict__ box) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nc) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = begin[warp] + lane; i < end[warp]; i += 32) {
    const int v = perm[i];
    for (int e = sup_ptr[v]; e < sup_ptr[v + 1]; ++e) {
      const int t = sup_item[e] >> 2;
      for (int a = 0; a < 3; ++a) {
        const int w = tri[3 * t + a];
        for (int d = 0; d < 3; ++d) {
          const double x = vert[3 * w + d];
          lo[d] = fmin(lo[d], x);
          hi[d] = fmax(hi[d], x);
        }
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

// One support union: the list's vertex ids, its length and the first row of
// its output in the row pool (room for the sum of the list's support sizes).
struct UnionJob {
  const int* list;
  int len;
  int pad;
  int64_t out;
};

// One CTA per list.  Shared memory: `pcap` 64-bit keys (a power of two at
// least the list's support entries) and len + 1 offsets.  Key of an entry:
// triangle (bits 32..63), corner (30..31), position in the list (0..29).
// After the bitonic sort the entries of a triangle are adjacent (at most
// three, one per corner); the first of them writes the row.
__global__ void __launch_bounds__(256)
k_support_union(const UnionJob* __restrict__ jobs, const int* __restrict__ sup_ptr,
                const int* __restrict__ sup_item, int pcap, int4* __restrict__ rows, int* __restrict__ counts,
                int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_raw);
  const UnionJob job = jobs[blockIdx.x];
  int* off = reinterpret_cast<int*>(key + pcap);  // len + 1
  __shared__ int s_part[256];
  __shared__ int s_total;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int a = tid; a < job.len; a += nth) {
    const int v = job.list[a];
    off[a + 1] = sup_ptr[v + 1] - sup_ptr[v];
  }
  __syncthreads();
  if (tid == 0) {
    off[0] = 0;
    for (int a = 0; a < job.len; ++a) off[a + 1] += off[a];
  }
  __syncthreads();
  const int m = off[job.len];
  if (m > pcap) {  // the host sizes pcap from the same counts; never taken
    if (tid == 0) {
      atomicOr(status, 2);
      counts[blockIdx.x] = 0;
    }
    return;
  }
  int P = 1;
  while (P < m) P <<= 1;
  for (int a = tid; a < job.len; a += nth) {
    const int v = job.list[a];
    const int e0 = sup_ptr[v];
    for (int e = e0; e < sup_ptr[v + 1]; ++e) {
      const int it = sup_item[e];
      key[off[a] + (e - e0)] = ((unsigned long long)(unsigned)(it >> 2) << 32) |
                               ((unsigned long long)(it & 3) << 30) | (unsigned long long)a;
    }
  }
  for (int i = m + tid; i < P; i += nth) key[i] = ~0ull;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += nth) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = key[i], y = key[l];
          if ((x > y) == ((i & k) == 0)) {
            key[i] = y;
            key[l] = x;
          }
        }
      }
      __syncthreads();
    }
  // rows: one per run of equal triangles; a chunk of the sorted entries per
  // thread, the heads counted, scanned over the threads, then written
  const int chunk = (m + nth - 1) / nth;
  const int c0 = min(m, tid * chunk), c1 = min(m, c0 + chunk);
  auto head = [&](int i) { return i == 0 || (key[i] >> 32) != (key[i - 1] >> 32); };
  int cnt = 0;
  for (int i = c0; i < c1; ++i) cnt += head(i);
  s_part[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < nth; ++t) {
      const int c = s_part[t];
      s_part[t] = acc;
      acc += c;
    }
    s_total = acc;
  }
  __syncthreads();
  int r = s_part[tid];
  for (int i = c0; i < c1; ++i) {
    if (!head(i)) continue;
    const unsigned t = (unsigned)(key[i] >> 32);
    int loc[3] = {-1, -1, -1};
    for (int j = i; j < m && (unsigned)(key[j] >> 32) == t; ++j)
      loc[(key[j] >> 30) & 3] = (int)(key[j] & 0x3fffffffu);
    rows[job.out + r] = make_int4((int)t, loc[0], loc[1], loc[2]);
    ++r;
  }
  if (tid == 0) counts[blockIdx.x] = s_total;
}

// A block of the nodal matrix: the rows' and the columns' support unions
// (indices into the union jobs), the block's first entry and row stride, and
// the mirrored block (G is symmetric: base2 < 0 when there is none).
struct P1Block {
  int64_t base;
  int64_t base2;
  int ld;
  int ld2;
  int ut;
  int us;
};

// A touching triangle pair of one block for k_p1_singular.
struct P1Item {
  int64_t base;
  int64_t base2;
  int ld;
  int ld2;
  int ti;
  int tj;
  int lr[3];  // positions of ti's corners in the row list (-1: none)
  int lc[3];  // positions of tj's corners in the column list
  int cs;     // shared vertices: 1 vertex, 2 edge, 3 identical
  int pad;
};

__device__ __forceinline__ void p1_scatter(double* __restrict__ out, int64_t base, int ld, int64_t base2, int ld2,
                                           const int lr[3], const int lc[3], const double M[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (lr[a] < 0) continue;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (lc[b] < 0) continue;
      atomicAdd(out + base + (int64_t)lr[a] * ld + lc[b], M[a][b]);
      if (base2 >= 0) atomicAdd(out + base2 + (int64_t)lc[b] * ld2 + lr[a], M[a][b]);
    }
  }
}

// 3 x 3 matrix of a disjoint pair in float64 (7 x 7 rule): the kernel
// values contracted with the barycentric weights of both nodes as they are
// formed, c_a(y_j) = sum_i w_i lambda_a(x_i) / |x_i - y_j| and
// M_ab += c_a w_j lambda_b(y_j).  Used for pairs whose nodes come closer
// than the float-pair arithmetic below resolves.
__device__ __noinline__ void p1_pair64(const P4* __restrict__ xq, const P4* __restrict__ yq, const Rules& rules,
                                       double (*M)[3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) M[a][b] = 0.0;
  for (int j = 0; j < 7; ++j) {
    const P4 y = yq[j];
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const P4 x = xq[i];
      const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
      const double t = x.w * rsqrt(dx * dx + dy * dy + dz * dz);
      c0 += t * rules.bary[i][0];
      c1 += t * rules.bary[i][1];
      c2 += t * rules.bary[i][2];
    }
    const double wy = y.w * kInv4Pi;
    for (int b = 0; b < 3; ++b) {
      const double wb = wy * rules.bary[j][b];
      M[0][b] += c0 * wb;
      M[1][b] += c1 * wb;
      M[2][b] += c2 * wb;
    }
  }
}

// The barycentric coordinates of the 7-point rule's nodes as float pairs.
struct BarySplit {
  float h[7][3];
  float l[7][3];
};

// Node weights of one triangle times the barycentric coordinates, as float
// pairs: W_ia = w_i lambda_a(x_i) = (w_h + w_l)(b_h + b_l) to first order.
__device__ __forceinline__ void p1_weights(const SplitNode* __restrict__ nd, const BarySplit& bs, float (*wh)[3],
                                           float (*wl)[3]) {
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const float w = nd[i].hi.w, wlo = nd[i].lo.w;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float h = __fmul_rn(w, bs.h[i][a]);
      wh[i][a] = h;
      wl[i][a] = __fadd_rn(__fmaf_rn(w, bs.h[i][a], -h), __fmaf_rn(w, bs.l[i][a], __fmul_rn(wlo, bs.h[i][a])));
    }
  }
}

// 1 / |x - y| of two split nodes as a float pair y0 + dy (the recipe of
// regular_entry_split: exact high differences, |d|^2 as a float pair,
// rsqrtf refined by one Newton step); r2 receives the high part of |d|^2.
__device__ __forceinline__ void inv_dist_split(float xh0, float xh1, float xh2, float xl0, float xl1, float xl2,
                                               const float4& yh, const float4& yl, float& y0, float& dy,
                                               float& r2) {
  const float dh0 = __fsub_rn(xh0, yh.x), dl0 = __fsub_rn(xl0, yl.x);
  const float dh1 = __fsub_rn(xh1, yh.y), dl1 = __fsub_rn(xl1, yl.y);
  const float dh2 = __fsub_rn(xh2, yh.z), dl2 = __fsub_rn(xl2, yl.z);
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
  r2 = rh;
  y0 = rsqrtf(__fadd_rn(rh, rl));
  const float u = __fmul_rn(y0, y0), uu = __fmaf_rn(y0, y0, -u);
  const float m = __fmul_rn(u, rh), me = __fmaf_rn(u, rh, -m);
  const float rho = __fmaf_rn(-uu, rh, __fmaf_rn(-u, rl, __fsub_rn(__fsub_rn(1.f, m), me)));
  dy = __fmul_rn(__fmul_rn(0.5f, y0), rho);
}

constexpr int kP1Chunk = 64;  // column triangles staged in shared memory at a time

// One CTA per block.  Columns are staged in chunks (split nodes and weights
// W'_jb in shared memory); a work item is a row triangle p with a residue g
// of the chunk's columns modulo G (G groups when the rows are fewer than the
// threads) and keeps p's split nodes and weights W_ia in registers.  A pair's
// 3 x 3 matrix is formed on the FP32 pipe in float-pair arithmetic (about
// 48 significant bits, as the single layer's coupling entries):
//   c_a(y_j) = sum_i W_ia / |x_i - y_j|,  M_ab += c_a W'_jb,
// and rounded to float64 once.  NEAR blocks test every pair for shared
// vertices first and append touching pairs to the singular list; a disjoint
// pair with nodes closer than sqrt(near_r2) is computed again in float64.
// The output is zero on entry (atomic sums).
template <bool NEAR>
__global__ void __launch_bounds__(256, NEAR ? 1 : 2)
k_p1_entries(const P1Block* __restrict__ blocks, const UnionJob* __restrict__ ujobs,
             const int* __restrict__ ucount, const int4* __restrict__ urows, const int* __restrict__ tri,
             const P4* __restrict__ tq, const SplitNode* __restrict__ tn, Rules rules, BarySplit bs,
             float near_r2, double* __restrict__ out, P1Item* __restrict__ items, int64_t cap,
             unsigned long long* __restrict__ counts, int* __restrict__ status) {
  __shared__ float4 ysh[kP1Chunk * 7];
  __shared__ float4 ysl[kP1Chunk * 7];
  __shared__ float2 ysw[kP1Chunk * 21];  // W'_jb (hi, lo), j-major
  __shared__ int4 cr[kP1Chunk];
  __shared__ int cv[kP1Chunk * 3];
  const P1Block B = blocks[blockIdx.x];
  const int4* R = urows + ujobs[B.ut].out;
  const int4* C = urows + ujobs[B.us].out;
  const int nr = ucount[B.ut], ncol = ucount[B.us];
  const int tid = threadIdx.x, nth = blockDim.x;
  int G = 1;
  while (G < 32 && nr * G * 2 <= nth) G *= 2;
  unsigned long long regular = 0;
  for (int q0 = 0; q0 < ncol; q0 += kP1Chunk) {
    const int cn = min(kP1Chunk, ncol - q0);
    __syncthreads();
    for (int i = tid; i < cn * 7; i += nth) {
      const SplitNode nd = tn[7 * (int64_t)C[q0 + i / 7].x + i % 7];
      ysh[i] = nd.hi;
      ysl[i] = nd.lo;
    }
    for (int i = tid; i < cn; i += nth) {
      const int4 c = C[q0 + i];
      cr[i] = c;
      if (NEAR)
        for (int a = 0; a < 3; ++a) cv[3 * i + a] = tri[3 * c.x + a];
      float wh[7][3], wl[7][3];
      p1_weights(tn + 7 * (int64_t)c.x, bs, wh, wl);
      for (int j = 0; j < 7; ++j)
        for (int b = 0; b < 3; ++b) ysw[21 * i + 3 * j + b] = make_float2(wh[j][b], wl[j][b]);
    }
    __syncthreads();
    for (int w = tid; w < nr * G; w += nth) {
      const int p = w / G, g = w - (w / G) * G;
      const int4 rp = R[p];
      const int lr[3] = {rp.y, rp.z, rp.w};
      const SplitNode* xn = tn + 7 * (int64_t)rp.x;
      float xh[7][3], xl[7][3], Wh[7][3], Wl[7][3];
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        const SplitNode nd = xn[i];
        xh[i][0] = nd.hi.x; xh[i][1] = nd.hi.y; xh[i][2] = nd.hi.z;
        xl[i][0] = nd.lo.x; xl[i][1] = nd.lo.y; xl[i][2] = nd.lo.z;
      }
      p1_weights(xn, bs, Wh, Wl);
      int tv[3] = {0, 0, 0};
      if (NEAR)
        for (int a = 0; a < 3; ++a) tv[a] = tri[3 * rp.x + a];
      for (int q = g; q < cn; q += G) {
        const int4 cq = cr[q];
        const int lc[3] = {cq.y, cq.z, cq.w};
        if (NEAR) {
          int sh = 0;
#pragma unroll
          for (int a = 0; a < 3; ++a)
            sh += (tv[a] == cv[3 * q]) + (tv[a] == cv[3 * q + 1]) + (tv[a] == cv[3 * q + 2]);
          if (sh) {
            // The Sauter-Schwab rule depends on the order of the pair (the
            // vertex orders follow the first triangle), so the mirrored
            // block's pair (s, t) is integrated as a pair of its own.
            const int nit = B.base2 >= 0 ? 2 : 1;
            const unsigned long long slot = atomicAdd(&counts[4], (unsigned long long)nit);
            atomicAdd(&counts[sh], (unsigned long long)nit);
            if (slot + nit <= (unsigned long long)cap) {
              for (int m = 0; m < nit; ++m) {
                P1Item it;
                it.base = m ? B.base2 : B.base;
                it.base2 = -1;
                it.ld = m ? B.ld2 : B.ld;
                it.ld2 = 0;
                it.ti = m ? cq.x : rp.x;
                it.tj = m ? rp.x : cq.x;
                for (int a = 0; a < 3; ++a) {
                  it.lr[a] = m ? lc[a] : lr[a];
                  it.lc[a] = m ? lr[a] : lc[a];
                }
                it.cs = sh;
                it.pad = 0;
                items[slot + m] = it;
              }
            } else {
              atomicOr(status, 2);
            }
            continue;
          }
        }
        float Mh[3][3], Ml[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) Mh[a][b] = Ml[a][b] = 0.f;
        float mr = 3.0e38f;
#pragma unroll 1
        for (int j = 0; j < 7; ++j) {
          const float4 yh = ysh[7 * q + j], yl = ysl[7 * q + j];
          float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
#pragma unroll
          for (int i = 0; i < 7; ++i) {
            float y0, dy, r2;
            inv_dist_split(xh[i][0], xh[i][1], xh[i][2], xl[i][0], xl[i][1], xl[i][2], yh, yl, y0, dy, r2);
            mr = fminf(mr, r2);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              float th, tl;
              pair_mul(Wh[i][a], Wl[i][a], y0, dy, th, tl);
              pair_acc(ch[a], cl[a], th, tl);
            }
          }
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const float2 wy = ysw[21 * q + 3 * j + b];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              float th, tl;
              pair_mul(ch[a], cl[a], wy.x, wy.y, th, tl);
              pair_acc(Mh[a][b], Ml[a][b], th, tl);
            }
          }
        }
        double M[3][3];
        if (NEAR && mr < near_r2) {
          p1_pair64(tq + 7 * (int64_t)rp.x, tq + 7 * (int64_t)cq.x, rules, M);
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) M[a][b] = ((double)Mh[a][b] + (double)Ml[a][b]) * kInv4Pi;
        }
        p1_scatter(out, B.base, B.ld, B.base2, B.ld2, lr, lc, M);
        ++regular;
      }
    }
  }
  for (int o = 16; o; o >>= 1) regular += __shfl_xor_sync(0xffffffffu, regular, o);
  if ((tid & 31) == 0 && regular) atomicAdd(&counts[0], regular);
}

// A Sauter-Schwab sample of the nodal basis as float pairs (computed on the
// host in long double): the coefficients of h(eta) = (x - y) / xi in the
// edge vectors (as SSEntry), the weight (Gauss weights times the piece's
// Jacobian without xi^3), and the slopes of the barycentric coordinates of
// both points in the ordered vertices, u = xi u^, v = xi v^:
// beta = (-u^1, u^1 - u^2, u^2) (beta_2 = -beta_0 - beta_1), beta' likewise.
struct __align__(16) SSEntryP1 {
  float4 ch, cl;  // h coefficients, high and low parts
  float4 ba;      // beta_0 (hi, lo), beta_1 (hi, lo)
  float4 bb;      // beta'_0 (hi, lo), beta'_1 (hi, lo)
  float wh, wl;   // weight
  float pad[2];
};

template <int CASE>
void sauter_table_p1(const Rules& rules, std::vector<SSEntryP1>& out) {
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
    SSEntryP1 e{};
    split(cf[0], e.ch.x, e.cl.x);
    split(cf[1], e.ch.y, e.cl.y);
    split(cf[2], e.ch.z, e.cl.z);
    split(cf[3], e.ch.w, e.cl.w);
    split(-u1, e.ba.x, e.ba.y);
    split(u1 - u2, e.ba.z, e.ba.w);
    split(-v1, e.bb.x, e.bb.y);
    split(v1 - v2, e.bb.z, e.bb.w);
    split((long double)rules.ss_w[a] * rules.ss_w[b] * rules.ss_w[c] * wj, e.wh, e.wl);
    out.push_back(e);
  }
}

// One warp per touching pair.  On each piece x - y = xi h(eta) and the
// barycentric coordinates of both points (in the ordered vertices) are
// alpha + xi beta with alpha = (1, 0, 0), so with f = w / |h| the
// xi-integral of xi^2 (alpha_a + xi beta_a)(alpha_b + xi beta'_b) is exact:
//   M_ab = sum f [alpha_a alpha_b / 3 + (alpha_a beta'_b + beta_a alpha_b) / 4 + beta_a beta'_b / 5].
// The samples run in float-pair arithmetic on the FP32 pipe (the single
// layer's Sauter-Schwab recipe: h from split edge vectors, |h|^2 as a float
// pair, one Newton step from rsqrtf) and accumulate the sums of f, f beta_a,
// f beta'_b and f beta_a beta'_b for a, b < 2 as float pairs; the third
// components follow from beta_2 = -beta_0 - beta_1, in float64.
__global__ void __launch_bounds__(256)
k_p1_singular(const P1Item* __restrict__ items, const unsigned long long* __restrict__ counts, int64_t cap,
              const int* __restrict__ tri, const double* __restrict__ vert, const double* __restrict__ area2,
              const SSEntryP1* __restrict__ table, int3 toff, int3 tcnt, double* __restrict__ out) {
  const int64_t wi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t count = min((long long)counts[4], (long long)cap);
  if (wi >= count) return;
  const P1Item it = items[wi];
  int ti[3], tj[3];
  for (int a = 0; a < 3; ++a) {
    ti[a] = tri[3 * it.ti + a];
    tj[a] = tri[3 * it.tj + a];
  }
  // vertex orders of the rules (identical: stored; edge: shared ids in the
  // order of ti, then the others; vertex: the shared id first, then
  // cyclically) and the stored corner of each ordered vertex
  int P[3], Q[3], ci[3], cj[3];
  const int cs = it.cs;
  if (cs == 3) {
    for (int a = 0; a < 3; ++a) {
      P[a] = Q[a] = ti[a];
      ci[a] = a;
      for (int b = 0; b < 3; ++b)
        if (tj[b] == ti[a]) cj[a] = b;
    }
  } else if (cs == 2) {
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
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        if (ti[b] == P[a]) ci[a] = b;
        if (tj[b] == Q[a]) cj[a] = b;
      }
  } else {
    int pi = 0, pj = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (ti[a] == tj[b]) { pi = a; pj = b; }
    for (int a = 0; a < 3; ++a) {
      ci[a] = (pi + a) % 3;
      cj[a] = (pj + a) % 3;
      P[a] = ti[ci[a]];
      Q[a] = tj[cj[a]];
    }
  }
  // edge vectors as float pairs (case 1: e1, e2, f1, f2; case 2: e1, e2, f2;
  // case 3: e1, e2): lane 3k + d forms component d of vector k in float64
  // and splits it, the others receive it by shuffles
  const int nt = cs == 3 ? 2 : (cs == 2 ? 3 : 4);
  float my_h = 0.f, my_l = 0.f;
  if (lane < 3 * nt) {
    const int k = lane / 3, d = lane - 3 * k;
    const bool useq = (cs == 1 && k >= 2) || (cs == 2 && k == 2);
    const bool second = !(k == 0 || (cs == 1 && k == 2));  // edge (1, 2) instead of (0, 1)
    const int i0 = useq ? (second ? Q[1] : Q[0]) : (second ? P[1] : P[0]);
    const int i1 = useq ? (second ? Q[2] : Q[1]) : (second ? P[2] : P[1]);
    const double x = vert[3 * i1 + d] - vert[3 * i0 + d];
    my_h = (float)x;
    my_l = (float)(x - (double)my_h);
  }
  float vh[4][3], vl[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      vh[k][d] = __shfl_sync(0xffffffffu, my_h, 3 * k + d);  // lanes >= 3 nt hold zeros
      vl[k][d] = __shfl_sync(0xffffffffu, my_l, 3 * k + d);
    }
  const int t0 = cs == 1 ? toff.x : (cs == 2 ? toff.y : toff.z);
  const int tn = cs == 1 ? tcnt.x : (cs == 2 ? tcnt.y : tcnt.z);
  // float-pair sums: 0 f, 1-2 f beta_a, 3-4 f beta'_b, 5-8 f beta_a beta'_b
  float sh[9], sl[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) sh[i] = sl[i] = 0.f;
  for (int s = lane; s < tn; s += 32) {
    const SSEntryP1 e = table[t0 + s];
    const float ch[4] = {e.ch.x, e.ch.y, e.ch.z, e.ch.w}, cl[4] = {e.cl.x, e.cl.y, e.cl.z, e.cl.w};
    float hh[3], hl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      hh[d] = 0.f;
      hl[d] = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < nt) fp_mul_add(ch[k], cl[k], vh[k][d], vl[k][d], hh[d], hl[d]);
    }
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
    const float y0 = rsqrtf(__fadd_rn(rh, rl));
    const float u = __fmul_rn(y0, y0), uu = __fmaf_rn(y0, y0, -u);
    const float m = __fmul_rn(u, rh), me = __fmaf_rn(u, rh, -m);
    const float rho = __fmaf_rn(-uu, rh, __fmaf_rn(-u, rl, __fsub_rn(__fsub_rn(1.f, m), me)));
    const float dy = __fmul_rn(__fmul_rn(0.5f, y0), rho);
    float fh, fl;  // f = w / |h|
    pair_mul(e.wh, e.wl, y0, dy, fh, fl);
    pair_acc(sh[0], sl[0], fh, fl);
    float gh[2], gl[2];  // f beta_a
    pair_mul(fh, fl, e.ba.x, e.ba.y, gh[0], gl[0]);
    pair_mul(fh, fl, e.ba.z, e.ba.w, gh[1], gl[1]);
    pair_acc(sh[1], sl[1], gh[0], gl[0]);
    pair_acc(sh[2], sl[2], gh[1], gl[1]);
    const float bh[2] = {e.bb.x, e.bb.z}, bl[2] = {e.bb.y, e.bb.w};
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      float th, tl;
      pair_mul(fh, fl, bh[b], bl[b], th, tl);
      pair_acc(sh[3 + b], sl[3 + b], th, tl);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        pair_mul(gh[a], gl[a], bh[b], bl[b], th, tl);
        pair_acc(sh[5 + 2 * a + b], sl[5 + 2 * a + b], th, tl);
      }
    }
  }
  double S[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double v = (double)sh[i] + (double)sl[i];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    S[i] = v;
  }
  if (lane != 0) return;
  const double s0 = S[0];
  const double sa[3] = {S[1], S[2], -(S[1] + S[2])};
  const double sb[3] = {S[3], S[4], -(S[3] + S[4])};
  double sab[3][3];
  sab[0][0] = S[5];
  sab[0][1] = S[6];
  sab[1][0] = S[7];
  sab[1][1] = S[8];
  for (int a = 0; a < 2; ++a) sab[a][2] = -(sab[a][0] + sab[a][1]);
  for (int b = 0; b < 3; ++b) sab[2][b] = -(sab[0][b] + sab[1][b]);
  const double jac = area2[it.ti] * area2[it.tj] * kInv4Pi;
  double M[3][3];  // stored corners
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double v = sab[a][b] / 5.0;
      if (a == 0) v += sb[b] / 4.0;
      if (b == 0) v += sa[a] / 4.0;
      if (a == 0 && b == 0) v += s0 / 3.0;
      M[ci[a]][cj[b]] = v * jac;
    }
  p1_scatter(out, it.base, it.ld, it.base2, it.ld2, it.lr, it.lc, M);
}

// ----------------------------------------------- curved triangles (Sect. 6)
//
// A curved triangle is the quadratic map Phi of the reference triangle
// through its vertices X0, X1, X2 and the surface points M01, M12, M20 over
// its edges (the midpoints array: [nt][3][3], edges (0, 1), (1, 2), (2, 0)):
//   Phi(lambda) = sum_a lambda_a (2 lambda_a - 1) X_a + 4 (lambda_0 lambda_1 M01
//                 + lambda_1 lambda_2 M12 + lambda_2 lambda_0 M20),
// with the Gramian gamma = |d1 Phi x d2 Phi| for x^ = (lambda_1, lambda_2).
// The mapped nodal basis keeps the barycentric weights of the flat case.

// Phi and gamma at lambda for six nodes X[6][3] (vertices, then edge points)
__device__ __forceinline__ void curved_eval(const double (*X)[3], double l0, double l1, double l2, double* x,
                                            double& gamma) {
  const double N[6] = {l0 * (2.0 * l0 - 1.0), l1 * (2.0 * l1 - 1.0), l2 * (2.0 * l2 - 1.0),
                       4.0 * l0 * l1,        4.0 * l1 * l2,        4.0 * l2 * l0};
  // d/dx^_1 = d/dlambda_1 - d/dlambda_0, d/dx^_2 = d/dlambda_2 - d/dlambda_0
  const double d1[6] = {-(4.0 * l0 - 1.0), 4.0 * l1 - 1.0, 0.0, 4.0 * (l0 - l1), 4.0 * l2, -4.0 * l2};
  const double d2[6] = {-(4.0 * l0 - 1.0), 0.0, 4.0 * l2 - 1.0, -4.0 * l1, 4.0 * l1, 4.0 * (l0 - l2)};
  double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      s += N[k] * X[k][d];
      t1[d] += d1[k] * X[k][d];
      t2[d] += d2[k] * X[k][d];
    }
    x[d] = s;
  }
  const double n0 = t1[1] * t2[2] - t1[2] * t2[1];
  const double n1 = t1[2] * t2[0] - t1[0] * t2[2];
  const double n2 = t1[0] * t2[1] - t1[1] * t2[0];
  gamma = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
}

// The 7-point rule on curved triangles: nodes Phi(lambda_q), weights
// w_q gamma(lambda_q) / 2 (the flat case: w_q |T|); area2 receives twice the
// rule's area of the triangle.
__global__ void k_tri_geom_curved(int nt, const double* __restrict__ vert, const int* __restrict__ tri,
                                  const double* __restrict__ mid, Rules rules, P4* __restrict__ tq,
                                  double* __restrict__ area2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double X[6][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      X[a][d] = vert[3 * tri[3 * t + a] + d];
      X[3 + a][d] = mid[9 * (int64_t)t + 3 * a + d];
    }
  double area = 0.0;
  for (int q = 0; q < 7; ++q) {
    double x[3], g;
    curved_eval(X, rules.bary[q][0], rules.bary[q][1], rules.bary[q][2], x, g);
    const double w = rules.w7[q] * g * 0.5;
    tq[7 * t + q] = P4{x[0], x[1], x[2], w};
    area += w;
  }
  area2[t] = 2.0 * area;
}

// one warp per cluster: min / max over the six nodes of the curved triangles
// in the supports of the cluster's vertices
__global__ void k_p1c_boxes(int nc, const int* __restrict__ begin, const int* __restrict__ end,
                            const int* __restrict__ perm, const int* __restrict__ sup_ptr,
                            const int* __restrict__ sup_item, const int* __restrict__ tri,
                            const double* __restrict__ vert, const double* __restrict__ mid,
                            double* __restrict__ box) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nc) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = begin[warp] + lane; i < end[warp]; i += 32) {
    const int v = perm[i];
    for (int e = sup_ptr[v]; e < sup_ptr[v + 1]; ++e) {
      const int t = sup_item[e] >> 2;
      for (int a = 0; a < 6; ++a)
        for (int d = 0; d < 3; ++d) {
          const double x = a < 3 ? vert[3 * tri[3 * t + a] + d] : mid[9 * (int64_t)t + 3 * (a - 3) + d];
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

// ------------------------------- curved pairs in float-pair arithmetic
//
// A sample of the curved Sauter-Schwab rule as float pairs (hi, lo),
// computed on the host in long double: the map is not affine, so xi is
// sampled like eta (u = xi u^(eta), v = xi v^(eta)); the monomials (u1, u2,
// u1^2, u1 u2, u2^2) of both points, the first two barycentric coordinates
// of both (the third follows from their sum being one), and the weight (the
// Gauss weights of all four variables times xi^3 and the piece's
// eta-Jacobian).
struct __align__(16) SSEntryCurvedSplit {
  float mu[5][2];
  float mv[5][2];
  float lu[2][2];
  float lv[2][2];
  float w[2];
};

template <int CASE>
void sauter_table_curved_split(const Rules& rules, std::vector<SSEntryCurvedSplit>& out) {
  const int q = rules.q, q3 = q * q * q;
  constexpr int pieces = CASE == 3 ? 6 : (CASE == 2 ? 5 : 2);
  auto split = [](long double x, float* hl) {
    hl[0] = (float)x;
    hl[1] = (float)(x - (long double)hl[0]);
  };
  for (int s = 0; s < pieces * q3; ++s) {
    const int piece = s / q3, r = s % q3;
    const int a = r / (q * q), b = (r / q) % q, c = r % q;
    long double u1, u2, v1, v2;
    const long double wj = sauter_piece<CASE, long double>(piece, rules.ss_t[a], rules.ss_t[b], rules.ss_t[c],
                                                           u1, u2, v1, v2);
    for (int x = 0; x < q; ++x) {
      const long double xi = rules.ss_t[x];
      const long double U1 = xi * u1, U2 = xi * u2, V1 = xi * v1, V2 = xi * v2;
      SSEntryCurvedSplit e{};
      const long double mu[5] = {U1, U2, U1 * U1, U1 * U2, U2 * U2};
      const long double mv[5] = {V1, V2, V1 * V1, V1 * V2, V2 * V2};
      for (int k = 0; k < 5; ++k) {
        split(mu[k], e.mu[k]);
        split(mv[k], e.mv[k]);
      }
      split(1.0L - U1, e.lu[0]);
      split(U1 - U2, e.lu[1]);
      split(1.0L - V1, e.lv[0]);
      split(V1 - V2, e.lv[1]);
      split((long double)rules.ss_w[x] * rules.ss_w[a] * rules.ss_w[b] * rules.ss_w[c] * xi * xi * xi * wj, e.w);
      out.push_back(e);
    }
  }
}

// a - b for float pairs, to first order
__device__ __forceinline__ void pair_sub(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float e;
  two_sum(ah, -bh, sh, e);
  sl = __fadd_rn(e, __fsub_rn(al, bl));
}

// sqrt of a float pair a > 0: y = sqrtf(a_h), then one Newton step on the
// exact residual a - y^2
__device__ __forceinline__ void pair_sqrt(float ah, float al, float& sh, float& sl) {
  const float y = sqrtf(ah);
  const float p = __fmul_rn(y, y), pe = __fmaf_rn(y, y, -p);
  const float res = __fadd_rn(__fsub_rn(__fsub_rn(ah, p), pe), al);
  sh = y;
  sl = __fdiv_rn(res, __fmul_rn(2.f, y));
}

// One warp per ordered touching pair of curved triangles in float-pair
// arithmetic on the FP32 pipe: the vertex orders of the flat rules (the
// stored edge points follow their edges); the maps in the reference
// coordinates u (lambda = (1 - u1, u1 - u2, u2)),
//   Phi(u) = X0 + B1 u1 + B2 u2 + C11 u1^2 + C12 u1 u2 + C22 u2^2,
//   B1 = 4 M01 - 3 X0 - X1,         B2 = X1 - X2 - 4 M01 + 4 M20,
//   C11 = 2 X0 + 2 X1 - 4 M01,      C12 = 4 (M01 + M12 - M20 - X1),
//   C22 = 2 X1 + 2 X2 - 4 M12,
// have |d Phi/du1 x d Phi/du2| as Gramian (x^ = (u1 - u2, u2) has Jacobian
// 1), and both start at the shared vertex.  The monomial coefficients are
// formed in float64 per pair and split into float
// pairs; per sample x - y (the shared vertex cancelling), the tangents, the
// normals, the Gramians (a float-pair square root), 1 / |x - y| (rsqrtf and
// one Newton step) and f = w gamma_t gamma_s / |x - y| are float pairs, and
// the sums of f, f lambda_a(u), f lambda_b(v) and f lambda_a(u) lambda_b(v)
// for a, b < 2 are kept as float pairs (the third coordinates follow from
// lambda_0 + lambda_1 + lambda_2 = 1, in float64).
__global__ void __launch_bounds__(256, 2)
k_p1c_singular_split(const P1Item* __restrict__ items, const unsigned long long* __restrict__ counts,
                     int64_t cap, const int* __restrict__ tri, const double* __restrict__ vert,
                     const double* __restrict__ mid, const SSEntryCurvedSplit* __restrict__ table, int3 toff,
                     int3 tcnt, double* __restrict__ out) {
  const int64_t wi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t count = min((long long)counts[4], (long long)cap);
  if (wi >= count) return;
  const P1Item it = items[wi];
  int ti[3], tj[3];
  for (int a = 0; a < 3; ++a) {
    ti[a] = tri[3 * it.ti + a];
    tj[a] = tri[3 * it.tj + a];
  }
  int ci[3], cj[3];
  const int cs = it.cs;
  if (cs == 3) {
    for (int a = 0; a < 3; ++a) {
      ci[a] = a;
      for (int b = 0; b < 3; ++b)
        if (tj[b] == ti[a]) cj[a] = b;
    }
  } else if (cs == 2) {
    int sh[2], ns = 0, oi = -1, oj = -1;
    for (int a = 0; a < 3; ++a) {
      const bool in_j = ti[a] == tj[0] || ti[a] == tj[1] || ti[a] == tj[2];
      if (in_j) sh[ns++] = ti[a]; else oi = ti[a];
    }
    for (int a = 0; a < 3; ++a)
      if (tj[a] != sh[0] && tj[a] != sh[1]) oj = tj[a];
    const int P[3] = {sh[0], sh[1], oi}, Q[3] = {sh[0], sh[1], oj};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        if (ti[b] == P[a]) ci[a] = b;
        if (tj[b] == Q[a]) cj[a] = b;
      }
  } else {
    int pi = 0, pj = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (ti[a] == tj[b]) { pi = a; pj = b; }
    for (int a = 0; a < 3; ++a) {
      ci[a] = (pi + a) % 3;
      cj[a] = (pj + a) % 3;
    }
  }
  auto slot = [](int a, int b) { return a + b == 1 ? 0 : (a + b == 3 ? 1 : 2); };
  double XP[6][3], XQ[6][3];
  for (int a = 0; a < 3; ++a) {
    const int e = slot(ci[a], ci[(a + 1) % 3]), f = slot(cj[a], cj[(a + 1) % 3]);
    for (int d = 0; d < 3; ++d) {
      XP[a][d] = vert[3 * ti[ci[a]] + d];
      XQ[a][d] = vert[3 * tj[cj[a]] + d];
      XP[3 + a][d] = mid[9 * (int64_t)it.ti + 3 * e + d];
      XQ[3 + a][d] = mid[9 * (int64_t)it.tj + 3 * f + d];
    }
  }
  // monomial coefficients split into float pairs
  float kp[5][3][2], kq[5][3][2];
  for (int d = 0; d < 3; ++d) {
    const double cp[5] = {4.0 * XP[3][d] - 3.0 * XP[0][d] - XP[1][d],
                          XP[1][d] - XP[2][d] - 4.0 * XP[3][d] + 4.0 * XP[5][d],
                          2.0 * XP[0][d] + 2.0 * XP[1][d] - 4.0 * XP[3][d],
                          4.0 * (XP[3][d] + XP[4][d] - XP[5][d] - XP[1][d]),
                          2.0 * XP[1][d] + 2.0 * XP[2][d] - 4.0 * XP[4][d]};
    const double cq[5] = {4.0 * XQ[3][d] - 3.0 * XQ[0][d] - XQ[1][d],
                          XQ[1][d] - XQ[2][d] - 4.0 * XQ[3][d] + 4.0 * XQ[5][d],
                          2.0 * XQ[0][d] + 2.0 * XQ[1][d] - 4.0 * XQ[3][d],
                          4.0 * (XQ[3][d] + XQ[4][d] - XQ[5][d] - XQ[1][d]),
                          2.0 * XQ[1][d] + 2.0 * XQ[2][d] - 4.0 * XQ[4][d]};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      kp[k][d][0] = (float)cp[k];
      kp[k][d][1] = (float)(cp[k] - (double)kp[k][d][0]);
      kq[k][d][0] = (float)cq[k];
      kq[k][d][1] = (float)(cq[k] - (double)kq[k][d][0]);
    }
  }
  // Gramian |d Phi/du1 x d Phi/du2| at the monomials m = (u1, u2, ...)
  auto gram = [](const float (*K)[3][2], const float (*m)[2], float& gh, float& gl) {
    float t1[3][2], t2[3][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // t1 = K0 + 2 K2 u1 + K3 u2, t2 = K1 + K3 u1 + 2 K4 u2 (doubling is exact)
      t1[d][0] = K[0][d][0];
      t1[d][1] = K[0][d][1];
      fp_mul_add(2.f * K[2][d][0], 2.f * K[2][d][1], m[0][0], m[0][1], t1[d][0], t1[d][1]);
      fp_mul_add(K[3][d][0], K[3][d][1], m[1][0], m[1][1], t1[d][0], t1[d][1]);
      t2[d][0] = K[1][d][0];
      t2[d][1] = K[1][d][1];
      fp_mul_add(K[3][d][0], K[3][d][1], m[0][0], m[0][1], t2[d][0], t2[d][1]);
      fp_mul_add(2.f * K[4][d][0], 2.f * K[4][d][1], m[1][0], m[1][1], t2[d][0], t2[d][1]);
    }
    float n2h = 0.f, n2l = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int e = (d + 1) % 3, f = (d + 2) % 3;
      float ah, al, bh, bl, nh, nl;
      pair_mul(t1[e][0], t1[e][1], t2[f][0], t2[f][1], ah, al);
      pair_mul(t1[f][0], t1[f][1], t2[e][0], t2[e][1], bh, bl);
      pair_sub(ah, al, bh, bl, nh, nl);
      fp_mul_add(nh, nl, nh, nl, n2h, n2l);
    }
    pair_sqrt(n2h, n2l, gh, gl);
  };
  const int t0 = cs == 1 ? toff.x : (cs == 2 ? toff.y : toff.z);
  const int tn = cs == 1 ? tcnt.x : (cs == 2 ? tcnt.y : tcnt.z);
  // float-pair sums: 0 f, 1-2 f lambda_a(u), 3-4 f lambda_b(v), 5-8 f lambda_a(u) lambda_b(v)
  float sh[9], sl[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) sh[i] = sl[i] = 0.f;
  for (int s = lane; s < tn; s += 32) {
    const SSEntryCurvedSplit e = table[t0 + s];
    float r2h = 0.f, r2l = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float dh = 0.f, dl = 0.f;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        fp_mul_add(kp[k][d][0], kp[k][d][1], e.mu[k][0], e.mu[k][1], dh, dl);
        fp_mul_add(-kq[k][d][0], -kq[k][d][1], e.mv[k][0], e.mv[k][1], dh, dl);
      }
      fp_mul_add(dh, dl, dh, dl, r2h, r2l);
    }
    // 1 / |x - y|: rsqrtf and one Newton step on the exact residual
    const float y0 = rsqrtf(__fadd_rn(r2h, r2l));
    const float u = __fmul_rn(y0, y0), uu = __fmaf_rn(y0, y0, -u);
    const float mm = __fmul_rn(u, r2h), me = __fmaf_rn(u, r2h, -mm);
    const float rho = __fmaf_rn(-uu, r2h, __fmaf_rn(-u, r2l, __fsub_rn(__fsub_rn(1.f, mm), me)));
    const float dy = __fmul_rn(__fmul_rn(0.5f, y0), rho);
    float gth, gtl, gsh, gsl;
    gram(kp, e.mu, gth, gtl);
    gram(kq, e.mv, gsh, gsl);
    float fh, fl;
    pair_mul(e.w[0], e.w[1], y0, dy, fh, fl);
    pair_mul(fh, fl, gth, gtl, fh, fl);
    pair_mul(fh, fl, gsh, gsl, fh, fl);
    pair_acc(sh[0], sl[0], fh, fl);
    float gh[2], gl[2];  // f lambda_a(u)
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      pair_mul(fh, fl, e.lu[a][0], e.lu[a][1], gh[a], gl[a]);
      pair_acc(sh[1 + a], sl[1 + a], gh[a], gl[a]);
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      float th, tl;
      pair_mul(fh, fl, e.lv[b][0], e.lv[b][1], th, tl);
      pair_acc(sh[3 + b], sl[3 + b], th, tl);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        pair_mul(gh[a], gl[a], e.lv[b][0], e.lv[b][1], th, tl);
        pair_acc(sh[5 + 2 * a + b], sl[5 + 2 * a + b], th, tl);
      }
    }
  }
  double S[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double v = (double)sh[i] + (double)sl[i];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    S[i] = v;
  }
  if (lane != 0) return;
  // sums with lambda_2 = 1 - lambda_0 - lambda_1 on either side
  double acc[3][3];
  const double su[3] = {S[1], S[2], S[0] - S[1] - S[2]};
  const double sv[3] = {S[3], S[4], S[0] - S[3] - S[4]};
  acc[0][0] = S[5];
  acc[0][1] = S[6];
  acc[1][0] = S[7];
  acc[1][1] = S[8];
  for (int a = 0; a < 2; ++a) acc[a][2] = su[a] - acc[a][0] - acc[a][1];
  for (int b = 0; b < 3; ++b) acc[2][b] = sv[b] - acc[0][b] - acc[1][b];
  double M[3][3];  // stored corners
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) M[ci[a]][cj[b]] = acc[a][b] * kInv4Pi;
  p1_scatter(out, it.base, it.ld, it.base2, it.ld2, it.lr, it.lc, M);
}
