/*
 * gca.h -- C-ABI of the B300 GCA-H^2 library.
 *
 * Green cross approximation (GCA) H^2-matrix compression of the Galerkin
 * single-layer Laplace matrix (Boerm & Christophersen, "GCA-H^2 matrix
 * compression for electrostatic simulations"), built and applied on one GPU.
 *
 *   g(x, y) = 1 / (4 pi |x - y|)                                  (Sect. 1)
 *   g_ij    = int phi_i(x) int g(x, y) phi_j(y) dy dx             (Eq. (1))
 *
 * with piecewise constant phi_i = indicator of triangle i.  The library
 * builds the H^2 representation
 *
 *   G|tau x sigma ~ V_tau S_{tau sigma} V_sigma^*      admissible blocks,
 *   G|tau x sigma   exactly                            inadmissible leaves,
 *
 * with nested bases V_tau = [V_1 E_1; V_2 E_2] obtained by cross
 * approximation of Green quadrature matrices (Sect. 2 - Sect. 4), and
 * applies it (and its transpose) to blocks of vectors.
 *
 * Conventions shared by every entry point:
 *   - Return value: 0 (GCA_OK) on success, a negative gca_status otherwise;
 *     gca_strerror() gives a one-line text.  On error, outputs are left
 *     unspecified and no handle is returned.
 *   - Host pointers (meshes, trees, parameter structs, export buffers) are
 *     owned by the caller and only read/written during the call.
 *   - The products' x and y are owned by the caller: memory of the current
 *     device, or page-locked host memory mapped into the device's address
 *     space (cudaHostAlloc, cudaMallocHost, or cudaHostRegister with
 *     cudaHostRegisterMapped), which the product reads and writes in place
 *     over the bus -- the transfer then happens inside the product's own
 *     kernels.  Any other pointer (pageable host memory, another device's
 *     memory) is refused with GCA_ERR_INVALID_ARG.
 *   - Handles own all of their device memory until gca_free().  A handle
 *     (or batch) lives on the device that was current when it was built or
 *     imported; every call that launches work on it checks that this device
 *     is current and otherwise fails with GCA_ERR_INVALID_ARG, naming both
 *     ordinals, before anything is launched.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Products are stream ordered and do not synchronise.
 *     gca_build synchronises the stream (it sizes its outputs from ranks
 *     found on the device).
 *   - Every index is 0-based; triangles are referred to by their position
 *     in the caller's triangle array ("original order").
 */
#ifndef GCA_H
#define GCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GCA_OK = 0,
  GCA_ERR_INVALID_ARG = -1, /* bad mesh, tree, parameter or size          */
  GCA_ERR_CUDA = -2,        /* a CUDA runtime call failed                 */
  GCA_ERR_OOM = -3,         /* device or host allocation failed           */
  GCA_ERR_NUMERIC = -4,     /* NaN/Inf in the input or in an intermediate */
  GCA_ERR_TIMEOUT = -5,     /* a bounded device-side wait expired         */
  GCA_ERR_UNSUPPORTED = -6, /* valid request outside the built limits     */
  GCA_ERR_IO = -7           /* a file could not be read or written, or is
                               not a complete checkpoint                  */
} gca_status;

/* Surface mesh (Sect. 2): nv vertices, nt flat triangles.  vertices is
 * [nv][3] float64 row-major, triangles [nt][3] int32 row-major with vertex
 * ids in [0, nv).  The mesh must be conforming (neighbouring triangles
 * share vertex ids): the singular quadrature picks its rule by counting
 * shared ids (Sect. 8).  Degenerate (zero-area) triangles are rejected. */
typedef struct {
  int32_t nv;
  int32_t nt;
  const double* vertices;
  const int32_t* triangles;
} gca_mesh;

/* Cluster tree (Sect. 2): clusters are index sets tau-hat of triangles,
 * stored as ranges [begin, end) of `perm`, which lists triangle ids in
 * cluster order.  Cluster 0 is the root ([0, nt), level 0).  A cluster is
 * a leaf iff child0 == child1 == -1; otherwise child0 covers
 * [begin, m) and child1 [m, end) for some begin < m < end, and
 * level[child] = level[parent] + 1.  All arrays are host int32 of length
 * nclusters (perm: nt). */
typedef struct {
  int32_t nclusters;
  const int32_t* perm;
  const int32_t* begin;
  const int32_t* end;
  const int32_t* child0;
  const int32_t* child1;
  const int32_t* level;
} gca_tree;

/* Parameters of the construction.
 *   leaf_size    only used by gca_tree_build; gca_build accepts any valid
 *                tree whose leaves hold at most GCA_MAX_LEAF triangles.
 *   eta          admissibility max(diam tau, diam sigma) <= 2 eta dist
 *                (Sect. 2), eta > 0.
 *   box_gauss_m  m: Gauss-Legendre points per direction on each face of
 *                the box omega; k = 6 m^2 quadrature points (Eq. (2)).
 *                1 <= m <= GCA_MAX_BOX_M.
 *   aca_tol      relative stopping tolerance of the cross approximation
 *                (Sect. 3): stop before a pivot <= aca_tol * |first pivot|.
 *   tri_rule     triangle rule for regular integrals; only 7 (the
 *                degree-5 seven-point rule) is implemented.
 *   sauter_q     Gauss order per variable of the Sauter-Schwab rules for
 *                touching pairs (Sect. 8), 1 <= q <= GCA_MAX_SAUTER_Q.
 *   omega_margin omega = box(tau) widened by omega_margin * diam(tau) on
 *                each side; a value < 0 selects 1 / (4 eta).
 *   flags        what the handle keeps after the build, a bit set of
 *                GCA_DROP_* (0 keeps everything).  Dropping the copies a
 *                caller never uses cuts the handle's device memory (for
 *                many meshes in one batch); a product in a dropped
 *                precision, or an export of dropped coefficients, then
 *                fails with GCA_ERR_UNSUPPORTED. */
typedef struct {
  int32_t leaf_size;
  double eta;
  int32_t box_gauss_m;
  double aca_tol;
  int32_t tri_rule;
  int32_t sauter_q;
  double omega_margin;
  uint32_t flags;
} gca_params;

enum {
  GCA_DROP_F64 = 1,    /* no float64 panels: GCA_F64 products rejected      */
  GCA_DROP_F32 = 2,    /* no float32 V, E, S panels: GCA_F32 products
                          rejected (the float32 near field stays while
                          GCA_BF16 products are kept)                      */
  GCA_DROP_BF16 = 4,   /* no bfloat16 panels: GCA_BF16 products rejected    */
  GCA_DROP_EXPORT = 8, /* gca_h2_export of V, E, S, N is rejected (a handle
                          keeps no row-major float64 copy of them unless it
                          has no float64 panels, GCA_DROP_F64: export
                          rebuilds them from the float64 panels)           */
  GCA_F64_ENTRIES = 16 /* single layer (gca_build, gca_build_batch,
                          gca_build_single_level, gca_build_green_quadrature):
                          coupling and near-field entries and the
                          Sauter-Schwab samples in float64 arithmetic
                          instead of float-pair arithmetic on the FP32 pipe
                          (the paper's precision for the near-singular
                          quadrature; slower on this GPU's FP64 pipe)      */
};

enum {
  GCA_MAX_LEAF = 128,
  GCA_MAX_BOX_M = 6,
  GCA_MAX_SAUTER_Q = 16
};

/* Arithmetic of a product.  GCA_F64: everything in float64, x and y are
 * float64.  GCA_F32: bases, transfers, couplings and near field in
 * float32, float32 x and y.  GCA_BF16: bases, transfers and couplings in
 * bfloat16 with float32 accumulation, near field float32; x, y float32. */
typedef enum { GCA_F64 = 0, GCA_F32 = 1, GCA_BF16 = 2 } gca_prec;

typedef struct gca_h2 gca_h2;             /* opaque handle */
typedef struct gca_h2_batch gca_h2_batch; /* opaque batch of handles */

/* Sizes and counters of a built handle. */
typedef struct {
  int32_t n;            /* triangles                                      */
  int32_t nclusters;
  int32_t depth;        /* deepest level                                  */
  int32_t k;            /* quadrature points per box, 6 m^2               */
  int32_t nfar;         /* admissible (coupling) blocks                   */
  int32_t nnear;        /* inadmissible leaf (near-field) blocks          */
  int32_t max_rank;
  int32_t reserved;
  int64_t rank_sum;     /* sum of r_tau over all clusters (root: 0)       */
  int64_t v_entries;    /* coefficients of the leaf bases V_tau           */
  int64_t e_entries;    /* coefficients of the transfer matrices E_tau    */
  int64_t s_entries;    /* coefficients of the coupling matrices S        */
  int64_t n_entries;    /* coefficients of the near-field blocks          */
  int64_t n_singular[4];/* near entries by shared vertices: 0,1,2,3       */
  double build_seconds; /* wall time of gca_build (host clock)            */
} gca_stats;

/* Host copy of a built handle, for inspection and tests.  The caller
 * allocates every array with the sizes from gca_h2_stats:
 *   rank   [nclusters]     r_tau (0 for the root)
 *   pivots [rank_sum]      tilde-tau as triangle ids in selection order,
 *                          clusters in increasing id
 *   far    [2*nfar]        (tau, sigma) pairs, sorted by tau then sigma
 *   near   [2*nnear]       (tau, sigma) pairs, sorted by tau then sigma
 *   V      [v_entries]     for each leaf in increasing id: |tau-hat| x r
 *                          row-major, rows in cluster (perm) order
 *   E      [e_entries]     for each cluster whose parent is not the root,
 *                          in increasing id: r_child x r_parent row-major
 *   S      [s_entries]     for each far block in the order of `far`:
 *                          r_tau x r_sigma row-major
 *   N      [n_entries]     for each near block in the order of `near`:
 *                          |tau-hat| x |sigma-hat| row-major, cluster order
 * Any pointer may be NULL to skip that array. */
typedef struct {
  int32_t* rank;
  int32_t* pivots;
  int32_t* far;
  int32_t* near;
  double* V;
  double* E;
  double* S;
  double* N;
} gca_host_dump;

/* Cluster tree by recursive bisection (helper; the tree stays an input of
 * gca_build).  The bounding box of the triangle centroids (a+b+c)/3 is
 * split at its midpoint across its longest axis (ties: lowest axis);
 * centroids below the midpoint go to child0, keeping their order.  If a
 * side would be empty, the set is sorted stably by that coordinate and
 * halved (child0 gets the lower floor(size/2)).  Sets of at most
 * leaf_size triangles are leaves; clusters are numbered breadth first.
 * Output arrays are caller-allocated host int32: perm [nt], the others
 * [max_clusters] (2*nt - 1 always suffices).  *nclusters receives the
 * count.  Errors: INVALID_ARG (bad mesh, leaf_size < 1, too small
 * max_clusters). */
int gca_tree_build(const gca_mesh* mesh, int32_t leaf_size, int32_t max_clusters,
                   int32_t* perm, int32_t* begin, int32_t* end, int32_t* child0,
                   int32_t* child1, int32_t* level, int32_t* nclusters);

/* The same bisection on n given points (x, y, z per index, host, [n][3]),
 * e.g. the vertices of a mesh for the nodal basis of gca_build_p1.
 * Outputs and errors as gca_tree_build (NUMERIC for a non-finite
 * coordinate). */
int gca_tree_build_points(int32_t n, const double* points, int32_t leaf_size, int32_t max_clusters,
                          int32_t* perm, int32_t* begin, int32_t* end, int32_t* child0,
                          int32_t* child1, int32_t* level, int32_t* nclusters);

/* Build the GCA-H^2 representation of G on the current device (Sect. 2 -
 * Sect. 4, Sect. 8): cluster boxes, box quadrature, Green quadrature
 * matrices, complete-pivoting cross approximation level by level from the
 * leaves (leaf bases V_tau, transfer matrices E_tau, pivot sets tilde-tau),
 * coupling matrices S = G|tilde-tau x tilde-sigma and near-field blocks
 * G|tau-hat x sigma-hat, plus float32 / bfloat16 copies for the reduced
 * precision products.  The coefficients are stored in float64.  The Green
 * matrices and the cross approximation are computed in float64; the 7 x 7
 * and Sauter-Schwab quadratures of S and N in float-pair arithmetic (about
 * 48 significant bits, 1e-13 relative or better; near-field pairs with
 * nodes closer than 2^-8 of the mesh's half width fall back to float64).
 * Cluster bases that no admissible block uses, directly or through an
 * ancestor, are not built (rank 0).  mesh/tree/params are copied; *out
 * receives a new handle.  Synchronises `stream`.  Errors: INVALID_ARG,
 * OOM, CUDA, NUMERIC; UNSUPPORTED when the mesh's half width lies outside
 * [2^-41, 2^40] (float exponent range of the float-pair quadrature). */
int gca_build(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params,
              void* stream, gca_h2** out);

/* The double-layer operator of the integral equation of Sect. 1: the
 * Galerkin matrix K with k_ij = int_{T_i} int_{T_j} dg/dn_y(x, y) dy dx,
 * dg/dn_y(x, y) = <n_y, x - y> / (4 pi |x - y|^3), n_y the outer unit normal
 * of the flat triangle holding y (from its vertex order), and its GCA-H^2
 * approximation K|tau x sigma ~ V_tau K|tilde-tau x tilde-sigma' W_sigma^*.
 *   - rows: x -> dg/dn_y(x, y) is harmonic near tau, so Green's formula in x
 *     (Sect. 2) gives the single layer's factors: V_tau, E_tau and
 *     tilde-tau are those of gca_build;
 *   - columns: applying <n_y, grad_y> to Green's formula for y -> g(x, y)
 *     gives the column Green matrix
 *       a'_{j nu}    =          sqrt(w_nu) int dg/dn_y(y, z_nu) phi_j(y) dy,
 *       a'_{j nu+k}  = -d_sigma sqrt(w_nu) int d2g/dn_y dn_z(y, z_nu) phi_j(y) dy,
 *     d2g/dn_y dn_z(y, z) = (<n_y, n_z> / r^3 - 3 <n_y, e><n_z, e> / r^5) / (4 pi),
 *     e = z - y; its cross approximation (Sect. 3), nested as in Sect. 4,
 *     gives tilde-sigma', the column bases W and transfer matrices F;
 *   - entries: the 7 x 7 rule for disjoint pairs in float-pair arithmetic
 *     (about 48 significant bits; near-field pairs with nodes closer than
 *     2^-8 of the mesh's half width in float64), 0 for identical flat
 *     triangles, Sauter-Schwab in float64 for a common edge or vertex
 *     (Sect. 8).
 * The handle works with h2_matvec (K x), h2_matvec_transpose (K^T x, a
 * genuinely different product), h2_matvec_noalloc, gca_h2_stats (S: the
 * r_tau x r'_sigma couplings, N: the near field), gca_h2_export (row bases,
 * couplings, near field) and gca_h2_export_columns.  Arguments, errors and
 * synchronisation as gca_build. */
int gca_build_double_layer(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params,
                           void* stream, gca_h2** out);

/* The collocation variant of the single layer (Sect. 6): a single integral
 * per entry instead of the double integral of Eq. (1),
 *   c_ij = int_{T_j} g(x_i, y) dy,
 * with the centroid x_i of triangle i as collocation point (the
 * piecewise-constant counterpart of the paper's vertices), and its GCA-H^2
 * approximation C|tau x sigma ~ V_tau C|tilde-tau x tilde-sigma' W_sigma^*:
 *   - rows: x -> g(x, y) is harmonic near tau, so Green's formula evaluated
 *     at the collocation points gives a_{i nu} = sqrt(w_nu) g(x_i, z_nu),
 *     a_{i nu+k} = -d_tau sqrt(w_nu) dg/dn_z(x_i, z_nu), cross-approximated
 *     and nested into the row bases V, E;
 *   - columns: the y-factors are the Galerkin ones, so the column bases W, F
 *     are those of gca_build;
 *   - entries in float64: the 7-point rule on T_j for j != i; for j = i a
 *     Duffy transformation around x_i (three sub-triangles, the radial
 *     integral exact, 4 sauter_q Gauss points along each edge).
 * The handle works like a gca_build_double_layer handle (two-sided bases,
 * h2_matvec for C x, h2_matvec_transpose for C^T x, gca_h2_export_columns);
 * n_singular[3] of its stats counts the Duffy entries.  Arguments, errors
 * and synchronisation as gca_build. */
int gca_build_collocation(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params,
                          void* stream, gca_h2** out);

/* The two approximations of the single-layer matrix that GCA-H^2 improves
 * on, for the error-versus-storage comparison of the paper (Sect. 2 - 4):
 *   - gca_build_single_level: single-level GCA (Sect. 3),
 *     G|tau x sigma ~ V_tau G|tilde-tau x tilde-sigma V_sigma^*, with V_tau
 *     from the cross approximation of A_tau on all of tau's triangles for
 *     every cluster of an admissible block, and no transfer matrices.
 *     Export: V holds |tau-hat| x r_tau for every cluster 1..nclusters-1 in
 *     increasing id (not only the leaves); E is empty.  The cross
 *     approximation of a cluster's whole A_tau must fit the cluster kernel's
 *     shared memory (GCA_ERR_UNSUPPORTED otherwise: about 1000 triangles at
 *     m = 4, 1800 at m = 3).
 *   - gca_build_green_quadrature: pure Green quadrature (Sect. 2, Eq. (2)),
 *     G|tau x sigma ~ A_tau B_{tau sigma}^*, A_tau the Green quadrature
 *     matrix of tau (|tau-hat| x 2k) and B_{tau sigma} the factor of sigma on
 *     tau's box.  Export: rank = 2k for the clusters of the blocks (-1 as
 *     pivots: there are none), V = A_tau for those clusters in increasing id,
 *     S = B_{tau sigma}^* (2k x |sigma-hat| row-major) per block.
 * Both: float64 Green and coupling matrices, the near field as gca_build,
 * products (and transposes) with h2_matvec; arguments and errors as
 * gca_build. */
int gca_build_single_level(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params,
                           void* stream, gca_h2** out);
int gca_build_green_quadrature(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params,
                               void* stream, gca_h2** out);

/* The single-layer matrix in the continuous piecewise linear (nodal) basis
 * of Sect. 5: phi_i is linear on every triangle, 1 in vertex i and 0 in
 * the other vertices, so its support T_i is the fan of triangles around i
 * and
 *   g_ij = sum_{t in T_i} sum_{s in T_j} int_t phi_i(x) int_s g(x, y) phi_j(y) dy dx.
 * Indices are the mesh's VERTICES: the tree is a tree over vertex ids
 * (e.g. gca_tree_build_points on the vertex positions), n = nv, and the
 * products take x and y of nv rows in the caller's vertex order.  Every
 * vertex must belong to a triangle (INVALID_ARG otherwise).
 *   - cluster boxes: bounding boxes of all triangles in the supports of the
 *     cluster's basis functions (Sect. 2: the box must contain the
 *     supports);
 *   - Green matrices: a_{i nu} = sqrt(w_nu) int g(x, z_nu) phi_i(x) dx and
 *     a_{i nu+k} = -d_tau sqrt(w_nu) int dg/dn_z(x, z_nu) phi_i(x) dx, the
 *     7-point rule on every triangle of T_i weighted by the barycentric
 *     coordinate of vertex i; cross approximation and nesting as gca_build;
 *   - entries (couplings G|tilde-tau x tilde-sigma, near field
 *     G|tau-hat x sigma-hat) assembled triangle pair by triangle pair over
 *     the support unions of the two index lists (the mergesort of Sect. 5,
 *     gca_support_union): every pair's 3 x 3 matrix
 *     M_ab = int_t lambda_a int_s g lambda_b (barycentric lambda) is
 *     computed once and added to the entries of the corners in the lists;
 *     disjoint pairs by the 7 x 7 rule, touching pairs by Sauter-Schwab
 *     (order sauter_q) with the barycentric weights of both sample points,
 *     all in float64.
 * The matrix is symmetric; the handle works like a gca_build handle
 * (h2_matvec, h2_matvec_transpose, h2_matvec_noalloc, stats, export with
 * vertex ids as pivots and vertex order in V and N).  n_singular of the
 * stats counts touching triangle pairs by case (index 1 vertex, 2 edge,
 * 3 identical; index 0 the disjoint pairs).  Arguments, errors and
 * synchronisation as gca_build. */
int gca_build_p1(const gca_mesh* mesh, const gca_tree* tree, const gca_params* params,
                 void* stream, gca_h2** out);

/* The nodal basis of gca_build_p1 on curved triangles (Sect. 6): every
 * triangle t is the quadratic map Phi_t of the reference triangle through
 * its vertices and the surface points over its edges,
 *   Phi_t(lambda) = sum_a lambda_a (2 lambda_a - 1) X_a
 *                   + 4 (lambda_0 lambda_1 M01 + lambda_1 lambda_2 M12 + lambda_2 lambda_0 M20),
 * the basis functions are mapped nodal ones (phi_i o Phi_t = lambda_c),
 * and integrals over t carry the Gramian |d1 Phi_t x d2 Phi_t|.
 *   midpoints  host [nt][3][3], caller-owned, read during the call: for
 *              triangle t the points M01, M12, M20 over its edges (0, 1),
 *              (1, 2), (2, 0) (e.g. the edge midpoints projected onto the
 *              surface; the flat midpoints give gca_build_p1's matrix).
 * Cluster boxes hold all six nodes of every support triangle; the 7-point
 * rule takes nodes Phi(lambda_q) with weights w_q |Phi|'(lambda_q) / 2;
 * touching pairs use the Sauter-Schwab maps with all four variables sampled
 * (q^4 samples per piece, float64; the map is not affine).  Otherwise as
 * gca_build_p1.  Errors additionally: INVALID_ARG (midpoints NULL),
 * NUMERIC (a non-finite edge point). */
int gca_build_p1_curved(const gca_mesh* mesh, const double* midpoints, const gca_tree* tree,
                        const gca_params* params, void* stream, gca_h2** out);

/* The support unions of Sect. 5 on the device, for inspection and tests:
 * for each of nlists lists of vertex ids (host CSR: list l is
 * lists[list_ptr[l] .. list_ptr[l + 1]), no repeated id within a list) the
 * union of the supports T_i of its vertices, one row per triangle in
 * ascending triangle id: (triangle, l0, l1, l2) with l_c the position in
 * the list of the triangle's corner c, or -1 when that corner is not in
 * the list.  Each vertex contributes its support as a list sorted by
 * triangle; the lists are merged (a bitonic sort of the entries in shared
 * memory, one CTA per list) and the rows of one triangle combined.
 * Output (host): rows [cap][4] packed list after list, counts [nlists] the
 * rows of each list.  cap must be at least sum over the lists of
 * sum_{i in list} |T_i| (the rows before merging).  Errors: INVALID_ARG
 * (bad mesh, ids out of range, cap too small), UNSUPPORTED (a list with
 * more than 16384 support entries), CUDA.  Synchronises `stream`. */
int gca_support_union(const gca_mesh* mesh, int32_t nlists, const int32_t* list_ptr, const int32_t* lists,
                      int32_t* rows, int64_t cap, int32_t* counts, void* stream);

/* Sizes of the column side of a handle: op 0 (single layer: the row bases
 * serve the columns, the values repeat those of gca_h2_stats), op 1
 * (double layer) or op 2 (collocation); max_rank and rank_sum of r'_sigma,
 * coefficients of the column bases W and transfers F. */
typedef struct {
  int32_t op;
  int32_t max_rank;
  int64_t rank_sum;
  int64_t w_entries;
  int64_t f_entries;
} gca_column_stats;
int gca_h2_column_stats(const gca_h2* h, gca_column_stats* out);

/* Host copy of the column side in the layout of gca_host_dump: rank
 * [nclusters] (r'_sigma), pivots [rank_sum] (tilde-sigma'), V the column
 * bases W (leaves, |sigma-hat| x r' row-major), E the transfers F
 * (r'_child x r'_parent row-major); far, near, S and N must be NULL.  On a
 * single-layer handle it returns the row bases.  Errors: INVALID_ARG,
 * UNSUPPORTED (GCA_DROP_EXPORT), CUDA. */
int gca_h2_export_columns(const gca_h2* h, gca_host_dump* out);

/* y = G_H2 x for nrhs right-hand sides, G_H2 the representation of Sect. 4:
 * y|tau-hat = sum over admissible (tau, sigma) of V_tau S_{tau sigma}
 * V_sigma^* x|sigma-hat plus sum over inadmissible leaf pairs of
 * N_{tau sigma} x|sigma-hat, evaluated by the H^2 recursion (forward
 * transform x-hat_sigma = V_sigma^* x up the tree through the transfer
 * matrices E, coupling, backward transform down the tree, near field).
 * x: column-major n x nrhs with
 * leading dimension ldx >= n, rows in original triangle order; y: same layout
 * with ldy >= n, overwritten (device or mapped page-locked host memory, see
 * the conventions above).  Element type float64
 * for GCA_F64, float32 otherwise.  x and y must not overlap.  The handle
 * keeps internal work buffers: calls on the same handle must be ordered on
 * one stream.  1 <= nrhs <= 4096.  Errors: INVALID_ARG, CUDA, OOM. */
int h2_matvec(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx,
              void* y, int64_t ldy, void* stream);

/* y = G_H2 x without allocating any device memory (the paper has no
 * counterpart; this is a service to callers).  For callers that cannot call
 * cudaMalloc while they run a product -- code between kernels of a
 * latency-critical loop or in host callbacks, where an allocation would
 * synchronise or is not allowed, and programs that hand out all device memory
 * themselves.  Same arguments, conventions and result as h2_matvec (up to the
 * order of floating-point accumulation); the workspace comes from one
 * 32 MiB array in the library's device data instead of the handle:
 *   - every GPU that loads the library holds that array until the process
 *     exits;
 *   - the first call on a device looks up the array's address on that device
 *     (make that first call before any stream capture);
 *   - all calls share the array: calls that overlap on the GPU (other streams,
 *     other threads, other handles) race and give wrong results; order them;
 *   - a product whose workspace exceeds the array is rejected with
 *     GCA_ERR_UNSUPPORTED and a message giving the bytes it would need (the
 *     20480-triangle workload fits with 16 float32 right-hand sides);
 *   - the address looked up on the first call is kept for the life of the
 *     process: resetting the device (cudaDeviceReset) between calls is not
 *     supported, since the library's device data is reloaded elsewhere;
 *   - with tracing on its time is recorded as "mv_persistent_noalloc.<prec>".
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
int h2_matvec_noalloc(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x, int64_t ldx,
                      void* y, int64_t ldy, void* stream);

/* y = G_H2^T x, same conventions as h2_matvec: the representation of
 * Sect. 4 transposed, y|sigma-hat = sum V_sigma S_{tau sigma}^* V_tau^* x|tau-hat
 * plus sum N_{tau sigma}^* x|tau-hat.  A handle of a symmetric operator
 * (gca_build, gca_build_batch, gca_build_single_level, gca_build_p1,
 * gca_build_p1_curved: G of Eq. (1), whose coupling blocks come in mirrored
 * pairs S_{sigma tau} = S_{tau sigma}^T, evaluated once) keeps no transposed
 * couplings and no transposed plan: this runs h2_matvec's plan with the
 * mirrored near-field blocks transposed (their singular rules are not
 * symmetric in the two triangles, so they are kept).  Handles from
 * gca_h2_import and gca_h2_load keep both orientations. */
int h2_matvec_transpose(const gca_h2* h, gca_prec prec, int32_t nrhs, const void* x,
                        int64_t ldx, void* y, int64_t ldy, void* stream);

/* Tracing (process wide, for one thread).  While enabled, every phase of
 * gca_build and of the products records a pair of CUDA events on its stream.
 * gca_profile_read synchronises those events, writes the accumulated GPU
 * time and launch count per phase name (at most cap entries; *count gets
 * the number of phases) and clears the accumulators.  Phase names: build
 * phases ("green_aca", "couple_entries", ...) and product phases
 * "mv_<stage>.<f64|f32|bf16>[.T]".  on = 2 splits the per-level build
 * phases by tree level L and thread-block cluster size C
 * ("green_aca.L<L>.c<C>"); on = 0 stops recording. */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
} gca_phase;
int gca_profile_enable(int on);
int gca_profile_read(gca_phase* out, int32_t cap, int32_t* count);

/* Arithmetic throughput probe (not part of the method): chains of fused
 * multiply-adds on every SM; FLOP/s in float64 (scalar FMA) and float32
 * (packed pairs, fma.rn.f32x2: the instruction the float kernels issue), 2
 * per FMA.  Used as the denominator of the ALU roofline of the build
 * kernels. */
int gca_peak_probe(double* fp64_flops, double* fp32_flops);

/* Batches: independent GCA-H^2 matrices (one per mesh) built with the same
 * parameters and applied together in one persistent launch, which lets the
 * dependency chains of the meshes' tree recursions overlap each other's
 * streaming work.  gca_build_batch builds every mesh like gca_build (count
 * >= 1, meshes[i] with trees[i]); the batch owns the handles (read them with
 * gca_batch_handle, never free them individually).  The batched products take
 * per-mesh nrhs, x, ldx, y, ldy arrays (host arrays of length count; x, y
 * with the conventions of h2_matvec).  Calls on one batch must
 * be ordered on one stream.  Errors: as gca_build / h2_matvec. */
int gca_build_batch(int32_t count, const gca_mesh* meshes, const gca_tree* trees,
                    const gca_params* params, void* stream, gca_h2_batch** out);
int gca_batch_size(const gca_h2_batch* b, int32_t* count);
int gca_batch_handle(const gca_h2_batch* b, int32_t i, const gca_h2** h);
int h2_matvec_batch(const gca_h2_batch* b, gca_prec prec, const int32_t* nrhs, const void* const* x,
                    const int64_t* ldx, void* const* y, const int64_t* ldy, void* stream);
int h2_matvec_transpose_batch(const gca_h2_batch* b, gca_prec prec, const int32_t* nrhs,
                              const void* const* x, const int64_t* ldx, void* const* y,
                              const int64_t* ldy, void* stream);
/* Sticky error bits of the batched products (see gca_h2_status). */
int gca_batch_status(const gca_h2_batch* b, int32_t* status);
void gca_free_batch(gca_h2_batch* b);

/* Autotuner of the products' tile width (not part of the method; a service
 * to callers).  A product runs its right-hand sides in chunks of W columns,
 * one warp tile per chunk, with W one of 1, 2, 4, 8, 16; by default W is the
 * smallest of them at or above the largest nrhs (16 from 16 on), and at most 4
 * in float64 (whose products are FP64-bound; narrow tiles measured faster).
 * gca_tune_batch times the widths from a quarter to four times the default on the given
 * batched product (arguments as h2_matvec_batch / h2_matvec_transpose_batch;
 * the product is run in place and y is overwritten), records the fastest in
 * a process-wide table under the key (device name, precision, direction,
 * largest nrhs, floor(log2(total rows))) and returns it in *width (may be
 * NULL).  Later products (single or batched) whose key is in the table use
 * that width; h2_matvec_noalloc always uses the default.  Synchronises the
 * stream.  Errors: as h2_matvec_batch.
 * gca_tune_save writes the table to a text file, one "key width" line per
 * entry (key = device|precision|transpose|nrhs|log2rows, spaces in the device
 * name written as '_'); gca_tune_load merges such a file into the table
 * (INVALID_ARG on a malformed line, leaving the table unchanged);
 * gca_tune_get reads the width recorded for a key (0: none); gca_tune_clear
 * empties the table. */
int gca_tune_batch(const gca_h2_batch* b, gca_prec prec, int32_t transpose, const int32_t* nrhs,
                   const void* const* x, const int64_t* ldx, void* const* y, const int64_t* ldy,
                   void* stream, int32_t* width);
int gca_tune_save(const char* path);
int gca_tune_load(const char* path);
int gca_tune_get(const char* device, gca_prec prec, int32_t transpose, int32_t nrhs, int64_t rows,
                 int32_t* width);
void gca_tune_clear(void);

/* Sticky error bits of the products run on this handle so far (0: none;
 * 1: a bounded device-side wait of the persistent product kernel expired;
 * 2: the kernel met a malformed work record).  With any bit set the results
 * of that product are unreliable.  Synchronises the device. */
int gca_h2_status(const gca_h2* h, int32_t* status);

/* Synchronise `stream`, then turn the status bits of the products run on
 * this handle (batch) so far into a return code: GCA_ERR_TIMEOUT when a
 * bounded device-side wait expired (bit 1), GCA_ERR_INVALID_ARG when a
 * product met a malformed work record (bit 2), GCA_OK when neither.  The
 * bits stay set until gca_h2_clear_status (gca_batch_clear_status), which
 * synchronises the device and clears them; a product after the clear runs
 * normally (the expired product's results are unreliable, nothing else). */
int gca_h2_check(const gca_h2* h, void* stream);
int gca_h2_clear_status(const gca_h2* h);
int gca_batch_check(const gca_h2_batch* b, void* stream);
int gca_batch_clear_status(const gca_h2_batch* b);

/* Handle from a host copy of an H^2 representation (Sect. 4) computed
 * elsewhere, e.g. by another implementation of the construction, so that
 * the products (h2_matvec, h2_matvec_transpose, h2_matvec_noalloc) run on
 * it with the construction bypassed.  `tree` is the cluster tree over nt
 * triangles (as for gca_build); `dump` holds the representation in the
 * layout gca_h2_export writes, with nfar coupling and nnear near-field
 * blocks (pairs in any order; every array but `pivots` is required, and
 * `pivots` only when some rank is positive).  Requirements: rank 0 for the
 * root, 0 <= r_tau <= |tau-hat| at leaves and <= r_tau1 + r_tau2 above;
 * coupling blocks between non-root clusters; near-field blocks between
 * leaves; finite coefficients.  `flags` selects the kept copies as in
 * gca_params.flags; the stats' k and n_singular are 0.  The arrays are
 * copied; synchronises `stream`.  Errors: INVALID_ARG (inconsistent input),
 * NUMERIC (non-finite coefficient), OOM, CUDA. */
int gca_h2_import(const gca_tree* tree, int32_t nt, int32_t nfar, int32_t nnear, const gca_host_dump* dump,
                  uint32_t flags, void* stream, gca_h2** out);

/* Checkpoint of a handle (the paper has no counterpart; a service so that
 * a program can skip the construction): gca_h2_save writes the cluster tree
 * and the representation of Sect. 4 as gca_h2_export gives it (ranks,
 * pivots, block lists, V, E, S, N in float64) with the construction's
 * parameters and counts to the file `path`, and gca_h2_load rebuilds a
 * device handle from such a file through gca_h2_import, whose products
 * equal those of the saved handle (the float32 and bfloat16 copies are
 * rounded again from the float64 coefficients, to the same values).
 *
 * gca_h2_save: handles of gca_build, gca_build_batch, gca_h2_import,
 * gca_build_p1 and gca_build_p1_curved (one basis serving rows and
 * columns); the two-sided and single-level handles give UNSUPPORTED, as
 * does a handle built with GCA_DROP_EXPORT.  The file is written under
 * `path` + ".tmp" and renamed to `path`, replacing it; on failure nothing
 * is left under either name.  It is read back on a host of the same byte
 * order.  Synchronises the device.  Errors: INVALID_ARG (NULL handle, empty
 * path), UNSUPPORTED, OOM, IO, CUDA.
 *
 * gca_h2_load: `flags` selects the kept precisions as in gca_params.flags;
 * the other parameters and the stats' k and n_singular are those of the
 * saved handle.  A loaded nodal-basis handle multiplies like the saved one
 * (its indices are the vertices).  The file's magic, sizes, length and
 * checksum are checked before anything is allocated on the device.  The
 * handle is created on the current device; synchronises `stream`.  Errors:
 * INVALID_ARG (NULL out, empty path, a file whose representation the import
 * rejects), IO (missing, unreadable, truncated or corrupted file), NUMERIC,
 * OOM, CUDA. */
int gca_h2_save(const gca_h2* h, const char* path);
int gca_h2_load(const char* path, uint32_t flags, void* stream, gca_h2** out);

int gca_h2_stats(const gca_h2* h, gca_stats* out);
/* Host copy of a handle in the layout of gca_host_dump.  V, E, S and N are
 * rebuilt from the float64 panels (a handle keeps no second, row-major copy
 * of them unless it was built with GCA_DROP_F64); this allocates a device
 * buffer of the largest requested array for the call.  Synchronises the
 * device.  Errors: UNSUPPORTED (GCA_DROP_EXPORT), OOM, CUDA. */
int gca_h2_export(const gca_h2* h, gca_host_dump* out);
void gca_free(gca_h2* h);
const char* gca_strerror(int status);
/* Text of the last error raised on the calling thread (empty if none); valid
 * until the thread's next failing call. */
const char* gca_last_error(void);

/* Test hooks (not part of the method): process-wide settings that let tests
 * reach the failure paths without faulting a GPU.  `name`:
 *   "wait_cycles"  bound of every device-side wait of the product kernels,
 *                  in SM clock cycles (default 2^31, about a second);
 *                  value <= 0 restores the default.
 *   "stall_chain"  value != 0: every dependency wait of later products
 *                  needs one completion more than the plan provides (a
 *                  count that nothing reaches), so the first producer that
 *                  waits for an input runs out of its bounded wait, sets
 *                  status bit 1 and the launch winds down; 0: off.
 *   "fail_alloc"   value n > 0: the n-th device allocation of the library
 *                  from now on fails as if the device were out of memory
 *                  (the call then returns GCA_ERR_OOM and frees what it
 *                  allocated); 0: off.
 *   "device_skew"  handles and batches built or imported from now on record
 *                  (current device + value) as their device, so that the
 *                  wrong-device check can be exercised on one GPU; 0: off.
 * Errors: INVALID_ARG for an unknown name. */
int gca_test_hook(const char* name, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* GCA_H */
