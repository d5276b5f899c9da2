/*
 * fem.h -- C ABI of libfem: loop-free reassembly of finite element mass,
 * conductivity and Newton tangent matrices on one GB300 GPU (sm_103a).
 *
 * Method: Voet, "On the fast assemblage of finite element matrices with
 * application to nonlinear heat transfer problems".  All element matrices of
 * one kind come out of one tall, skinny product V = X Q (Section 4,
 * Algorithm 2): Q depends only on the reference element and the quadrature
 * rule, the geometric factors b_e = |det B_e| and A_e = (B_e^T B_e)^-1 only on
 * the mesh, and the coefficient evaluations S only on the unknown u (Section
 * 5, summary of dependencies).  The element matrices are then summed into a
 * global CSR matrix (the last step of Algorithm 2).
 *
 * Conventions used by every call:
 *  - Status: every function returns FEM_OK (0) or a negative FEM_E* code; a
 *    message for the last failure on the calling thread is available from
 *    fem_last_error().
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Calls that take a stream enqueue their GPU work on it
 *    and return without synchronising unless stated otherwise.
 *  - Memory: pointers named `d_*` must be device pointers of the current
 *    device.  Library-owned device memory comes from the allocator set with
 *    fem_set_allocator() (default: cudaMallocAsync/cudaFreeAsync on the
 *    call's stream).
 *  - Matrices: rows are test functions, columns trial functions,
 *    M_ij = int m phi_j phi_i and K_ij = int k(u) grad phi_j . grad phi_i
 *    (Section 2, definitions of M and of the conductivity matrix C).  The
 *    pattern (CSR, int32, columns ascending, explicit zeros kept) is the union
 *    over elements of all local (i, j) pairs (Section 3, step 2) and is shared
 *    by M, K and T.
 *  - Limits: n_elems * n_p^2 < 2^31 and nnz < 2^31.
 */
#ifndef FEM_H
#define FEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    FEM_OK = 0,
    FEM_EINVAL = -1,      /* bad argument, shape or index */
    FEM_ENOMEM = -2,      /* allocation failed (allocator returned NULL) */
    FEM_EDEGENERATE = -3, /* an element has |det B_e| <= 1e-14 ||B_e||^d */
    FEM_ECUDA = -4,       /* a CUDA runtime call or kernel launch failed */
    FEM_EBUSY = -5,       /* admission refused (server memory budget / queue) */
    FEM_EAGAIN = -6,      /* poll: result not ready yet */
    FEM_ETIMEOUT = -7,    /* poll or device wait gave up after its limit */
    FEM_ESTATE = -8       /* call out of order (e.g. assemble before symbolic) */
};

/* ------------------------------------------------------------- precision */
enum {
    FEM_FP64 = 0,   /* geometry, coefficients, element product and CSR sum in FP64 (SIMT) */
    FEM_TF32X3 = 1, /* FP32 coefficients; V = X Q on tcgen05 tensor cores as three TF32
                       products (Xhi Qhi + Xhi Qlo + Xlo Qhi), FP32 accumulate in TMEM;
                       FP32 CSR sums */
    FEM_FP32 = 2,   /* FP32 everywhere on the SIMT pipes (no tensor cores); reference point */
    FEM_BF16X3 = 3, /* as FEM_TF32X3 with X and Q split into two BF16 parts and three
                       kind::f16 products (x0 q0 + x0 q1 + x1 q0): ~16 significant bits */
    FEM_BF16X6 = 4  /* three BF16 parts and the six products of total part order < 3
                       (x0 q0 + x0 q1 + x1 q0 + x0 q2 + x1 q1 + x2 q0): ~24 bits.  The BF16
                       modes run the single-mesh tile kernel; P3 tetrahedra (whose tile does
                       not fit) and batches return FEM_EINVAL */
};

/* -------------------------------------------------------- memory locations */
enum { FEM_MEM_HOST = 0, FEM_MEM_DEVICE = 1 };

/* ------------------------------------------------------ conductivity laws */
enum {
    FEM_K_POLY = 0,  /* k(u) = sum_{i<n} p[i] u^i, n <= 8 */
    FEM_K_SIN = 1,   /* k(u) = p[0] + p[1] sin(p[2] u) */
    FEM_K_PWLIN = 2  /* n = 2m: knots p[0..m-1] ascending, values p[m..2m-1]; linear
                        between knots, constant outside; the first branch is closed on
                        both ends, later branches open on the left (Section 6, Experiment 2, k(T)) */
};

/* k(u) and its derivative k'(u) are evaluated analytically from this closed
 * description (k' enters the tangent, Section 5.2). */
typedef struct {
    int kind;       /* FEM_K_* */
    int n;          /* number of parameters used */
    double p[16];
} fem_coeff;

/* --------------------------------------------------------------- meshes */
/* Mesh description.  Elements are affine simplices of degree `order`
 * (Section 3 step 3: x = a + B_e xhat, B_e = [x_1 - x_0, ..., x_d - x_0]).
 * Local node order in `conn` rows: the d+1 vertices; then edge nodes, edges
 * in lexicographic order of their vertex pairs (a<b), for order 3 the node
 * nearer vertex a first; then face nodes (order 3), faces in lexicographic
 * order of their vertex triples.  Higher-order nodes must sit at the affine
 * images of their reference positions. */
typedef struct {
    int dim;            /* 2 (triangles) or 3 (tetrahedra) */
    int order;          /* Lagrange degree 1..3; n_p = C(order+dim, dim) */
    int64_t n_nodes;    /* number of dofs (rows of the matrices) */
    int64_t n_elems;
    const double* coords; /* n_nodes x dim, row-major, FP64 */
    const int32_t* conn;  /* n_elems x n_p, row-major, values in [0, n_nodes) */
    int mem;            /* FEM_MEM_HOST or FEM_MEM_DEVICE for coords and conn */
    int qdeg;           /* quadrature degree: 0 = 2*order (the default and only supported rule:
                           triangles 3/6/12 points, tetrahedra 4/11/24 points) */
    double mass_coeff;  /* constant m of the mass matrix (Section 2, eq. diff_eq) */
} fem_mesh_desc;

typedef struct fem_mesh fem_mesh;

/* Creates a mesh handle: copies coords and conn to the device (the caller
 * keeps ownership of its buffers; host buffers are read before return),
 * checks every connectivity index (FEM_EINVAL) and computes the per-element
 * geometric factors b_e = |det B_e| and A_e = (B_e^T B_e)^-1 once (Section 3
 * step 3; Algorithm 2; Section 5: W and b depend only on the mesh):
 * an FP64 cache for FEM_FP64, and an FP32 cache computed in FP32 with an FP64
 * recomputation for elements whose condition estimate ||B||_F^d/|det B|
 * exceeds 1e3.  P1 meshes also keep each element's Gram matrix G A_e G^T
 * (G the constant reference gradients; n_sym FP64 values per element), the
 * part of K_e that does not change with u.  Returns FEM_EDEGENERATE if an
 * element is degenerate.  Synchronises `stream` before returning. */
int fem_mesh_create(const fem_mesh_desc* desc, void* stream, fem_mesh** out);
int fem_mesh_destroy(fem_mesh* mesh);

typedef struct {
    int dim, order, n_p, n_q;
    int64_t n_nodes, n_elems;
    int64_t nnz;          /* -1 before fem_symbolic */
    int64_t n_flagged;    /* elements recomputed in FP64 in the FP32 geometry cache */
    size_t device_bytes;  /* library-owned device memory held by the mesh */
} fem_mesh_info;
int fem_mesh_get_info(const fem_mesh* mesh, fem_mesh_info* out);

/* ------------------------------------------------------------- symbolic */
typedef struct {
    int64_t n;           /* rows = cols = n_nodes */
    int64_t nnz;
    const int32_t* d_row_ptr;   /* n+1, device, owned by the mesh */
    const int32_t* d_col_idx;   /* nnz, device, owned by the mesh */
} fem_csr_pattern;

/* Builds, once per mesh, the CSR pattern and the element entries of every
 * CSR slot by a device sort of the keys (conn[e][i], conn[e][j]) (Section 3
 * step 2; the index set of nonzero entries that Algorithm 2 sums into): a
 * counting sort by row, then a per-row sort by column, stable in the element
 * entry index c = (e n_p + i) n_p + j.  Keeps on the device: row_ptr, col_idx,
 * the segmented lists seg_ptr / contrib (contributing c of every slot,
 * ascending) and, per 32 consecutive contributions, a mask of slot starts
 * and the slot of the first (what the CSR sum reads).  The map slot[c] from
 * element entries to CSR slots is derived from these when first needed
 * (fem_get_slot_map, fem_boundary_facets).  Idempotent. */
int fem_symbolic(fem_mesh* mesh, void* stream, fem_csr_pattern* out);

/* Copies the pattern into caller-owned device buffers d_row_ptr (n+1) and
 * d_col_idx (nnz), enqueued on `stream`. */
int fem_copy_pattern(fem_mesh* mesh, int32_t* d_row_ptr, int32_t* d_col_idx, void* stream);

/* Copies the element-entry -> slot map (n_elems * n_p^2 int32, entry
 * c = (e n_p + i) n_p + j) to d_slot (device, caller-owned).  Reassembly
 * does not read the map; the mesh builds it on the first call that needs
 * it (this one or fem_boundary_facets), from the sorted entries, and keeps
 * it (n_elems * n_p^2 int32 of device memory). */
int fem_get_slot_map(fem_mesh* mesh, int32_t* d_slot, void* stream);

/* ------------------------------------------------------------- numeric */
/* Reassembly of the CSR values, reusing the pattern and the geometry
 * (Section 5: only S is recomputed at each Newton step).  For each matrix
 * the element matrices are formed as one product V = X Q (Algorithm 2,
 * formation; Section 4.1 mass: X = Lambda = S*(w b^T); Section 4.2 conductivity:
 * X = Lambda (.) W; tangent: the Section 5.2 conductivity tensor multiplied
 * by u in its second mode, T_ij = int k'(u_h) phi_j grad u_h . grad phi_i),
 * using the symmetry of M and K to keep only the n_p(n_p+1)/2 distinct rows of
 * Q (Section 7), then summed into the CSR values by a deterministic
 * segmented reduction: every slot adds its contributions in one fixed order
 * given by the mesh alone (the contributions sorted by slot, cut into
 * aligned groups of 64: adjacent pairs, then a tree over the group, groups
 * in ascending order), with no atomics, so results are bit-reproducible run
 * to run and identical across ranges, batches and launch shapes.
 *
 * u: n_nodes nodal values in FP64 for every precision (the FP32 paths split
 * each gathered value as u = hi + lo, two FP32 values, inside the element
 * kernel, so that the nodal differences that carry grad u_h in the tangent
 * keep FP32 relative accuracy).
 * values: nnz outputs, FP64 for FEM_FP64 and FP32 otherwise.
 * u and values may be device pointers or host pointers (pageable or
 * page-locked); host pointers are staged through library-owned device
 * buffers and the call then synchronises `stream` before returning.
 * Requires fem_symbolic (FEM_ESTATE otherwise). */
int fem_assemble_mass(fem_mesh* mesh, int prec, void* values, void* stream);
int fem_assemble_stiffness(fem_mesh* mesh, const fem_coeff* k, const void* u, int prec,
                           void* values, void* stream);
int fem_assemble_tangent(fem_mesh* mesh, const fem_coeff* k, const void* u, int prec,
                         void* values, void* stream);
/* All three in one pass (any of vM, vK, vT may be NULL to skip it). */
int fem_assemble_all(fem_mesh* mesh, const fem_coeff* k, const void* u, int prec,
                     void* vM, void* vK, void* vT, void* stream);

/* Anisotropic conductivity (Section 7: with a d x d conductivity c the
 * element conductivity matrix takes A_e = B_e^-1 c B_e^-T in place of
 * B_e^-1 B_e^-T).  Sets a constant tensor c for the mesh: the conductivity
 * becomes k(u) c, in K(u) and in the tangent T(u) (whose entries become
 * int k'(u_h) phi_j (c grad u_h) . grad phi_i), on every path (single mesh,
 * ranges, batches, served requests).  c: d x d row-major, symmetric and
 * positive definite (FEM_EINVAL otherwise; checked on the host), or NULL
 * for the identity (the isotropic default).  Recomputes the mesh's geometry
 * cache (and, for P1, the elements' Gram matrices, which include c) on
 * `stream` and waits for it; the pattern is kept; element matrices
 * formed earlier must be formed again before fem_sum_elements. */
int fem_mesh_set_conductivity(fem_mesh* mesh, const double* c, void* stream);

/* Per-quadrature-point geometry (Section 7: with isoparametric mappings the
 * Jacobian depends on the quadrature point, so each element carries n_q
 * determinants and d^2 n_q Jacobian entries; an anisotropic conductivity
 * may vary over the points, A_qe = B^-1 c_q B^-T; only X changes).
 * fem_mesh_set_isoparametric(on = 1) maps every element through all its
 * nodes, x(xhat) = sum_i x_i phi_i(xhat): the higher-order nodes may sit off
 * their affine positions (curved elements).  on = 0 restores the affine
 * map.  fem_mesh_set_conductivity_field sets a d x d conductivity tensor
 * per quadrature point of the mesh's rule (n_elems x n_q x d x d,
 * row-major per point, host or device, copied; symmetric positive definite,
 * not checked on the device), overriding the constant tensor; NULL clears
 * it.  Either call recomputes a per-point geometry cache (|det B_q| and A_q
 * per element and point) on `stream` and waits for it (FEM_EDEGENERATE if
 * some det B_q vanishes); the pattern is kept; element matrices formed
 * earlier must be formed again.  While a mesh is in per-point mode its
 * products run on the SIMT pipes: FEM_FP64 and FEM_FP32 (the tensor-core
 * precisions, batches and, for isoparametric meshes, the boundary terms
 * return FEM_EINVAL). */
int fem_mesh_set_isoparametric(fem_mesh* mesh, int on, void* stream);
int fem_mesh_set_conductivity_field(fem_mesh* mesh, const double* c_field, void* stream);

/* u-dependent mass and its Newton term (Section 2 with a coefficient
 * m = m(u_h) in the mass; Section 5, where the Jacobian of the implicit
 * Euler residual holds  M(u) + (mass tensor) o_2 (u - u^s);  Section 5.1,
 * the mass tensor  M_ijk = int m'(u_h) phi_i phi_j phi_k):
 *   d_vMu <- M(u)_ij = int m(u_h) phi_j phi_i,
 *   d_vMt <- sum_j M_ijk (u - u^s)_j = int m'(u_h) (u - u^s)_h phi_k phi_i,
 * both symmetric, on the mesh's CSR pattern, each the product of the mass
 * basis matrix Q_M with new X (w_q |det B_e| m(u_q), resp.
 * w_q |det B_e| m'(u_q) (u - u^s)_q), then the deterministic CSR sum.
 * m: a coefficient law as k (FEM_COEFF_*; m' from the same law); the mesh's
 * constant mass coefficient is not used.  prec: FEM_FP64 or FEM_FP32 (SIMT
 * element products) or FEM_TF32X3 (tcgen05 tile; P3 tetrahedra: FEM_EINVAL);
 * other precisions: FEM_EINVAL.  d_u, d_us: FP64 nodal
 * values; d_us may be NULL when d_vMt is.  All four pointers are device
 * pointers (FEM_EINVAL otherwise); outputs FP64 for FEM_FP64 and FP32
 * otherwise, nnz each, either may be NULL to skip it.  The call reuses the
 * mesh's element-matrix scratch: matrices formed earlier by
 * fem_form_elements must be formed again before fem_sum_elements
 * (FEM_ESTATE otherwise).  Requires fem_symbolic. */
int fem_assemble_mass_u(fem_mesh* mesh, const fem_coeff* m, const void* d_u, const void* d_us, int prec,
                        void* d_vMu, void* d_vMt, void* stream);

/* The two phases of fem_assemble_all, which the paper times separately
 * (Section 4.2: formation of the element matrices versus assemblage of the
 * global matrices, the two parts of Algorithm 2).
 * fem_form_elements forms V = X Q for the matrices selected by `which`
 * (FEM_MAT_M | FEM_MAT_K | FEM_MAT_T) into scratch buffers owned by the mesh
 * (one kernel launch); d_u is a
 * device pointer to FP64 nodal values (unused when which == FEM_MAT_M).
 * fem_sum_elements sums the formed V into the CSR values (one kernel
 * launch); d_v* are device pointers, NULL to skip, and must have been formed
 * by the last fem_form_elements with the same `prec` (FEM_ESTATE otherwise).
 * Requires fem_symbolic. */
enum { FEM_MAT_M = 1, FEM_MAT_K = 2, FEM_MAT_T = 4 };
int fem_form_elements(fem_mesh* mesh, const fem_coeff* k, const void* d_u, int prec, int which,
                      void* stream);
int fem_sum_elements(fem_mesh* mesh, int prec, void* d_vM, void* d_vK, void* d_vT, void* stream);

/* ------------------------------------------------------ chunked reassembly */
/* Formation and summation over ranges: a caller can form part of the mesh
 * and sum the slots that part completes, e.g. to start summing before all
 * elements are formed, to interleave other work, or to keep one range's
 * element matrices in the GPU's L2 cache while they are summed.  (On GB300
 * the one-shot schedule of fem_assemble_all measured faster for the whole
 * 2-million-element P2 mesh, so fem_assemble_all does not chunk.)
 *
 * fem_chunk_plan splits the mesh into n <= max_chunks consecutive element
 * ranges [e_bounds[c], e_bounds[c+1]) of about target_bytes of V each
 * (0 = the library default, 48 MB), and gives for each the slot range
 * [s_bounds[c], s_bounds[c+1]) of CSR slots whose contributing elements all
 * lie in ranges 0..c, i.e. the slots that can be summed once range c is
 * formed.  e_bounds and s_bounds must hold max_chunks + 1 entries.  The plan
 * depends only on the pattern; it is computed once per mesh (a device pass
 * over the slots that synchronises `stream`).  Requires fem_symbolic.
 *
 * fem_form_elements_range forms V for elements [e_begin, e_end) (e_begin a
 * multiple of 128) into the mesh's scratch, as fem_form_elements does for
 * all elements; a range with e_begin > 0 must follow one with e_begin == 0
 * of the same reassembly (same u, precision and matrices).
 * fem_sum_elements_range writes the CSR values of slots [s_begin, s_end)
 * (d_v* are the whole nnz arrays); every element contributing to those slots
 * must have been formed.  A plan's ranges, formed and summed in order, give
 * the same values bit for bit as fem_form_elements + fem_sum_elements. */
int fem_chunk_plan(fem_mesh* mesh, int prec, size_t target_bytes, int max_chunks, int* n_chunks,
                   int64_t* e_bounds, int64_t* s_bounds, void* stream);
int fem_form_elements_range(fem_mesh* mesh, const fem_coeff* k, const void* d_u, int prec, int which,
                            int64_t e_begin, int64_t e_end, void* stream);
int fem_sum_elements_range(fem_mesh* mesh, int prec, int64_t s_begin, int64_t s_end, void* d_vM, void* d_vK,
                           void* d_vT, void* stream);

/* Synchronises `stream` and reports whether any library kernel recorded a
 * device-side failure since the last call: FEM_ETIMEOUT if a tensor-core
 * kernel gave up waiting on its MMA completion barrier (each such wait is
 * bounded at about one second of SM clocks), FEM_OK otherwise.  Clears the
 * record. */
int fem_device_status(void* stream);

/* ---------------------------------------------------------------- batches */
/* Many meshes of uneven size and element type reassembled by one captured
 * CUDA graph of a few persistent kernels (Section 7: a mesh with several
 * element types is split into one mesh per type whose contributions are
 * merged, and the formation of all element matrices can run in parallel).
 * The element tiles of all meshes form one work list, grouped by element
 * type, walked by one persistent tensor-core kernel (FEM_TF32X3; the tiles
 * of P3 tetrahedra, whose Q does not fit in shared memory, by a second
 * persistent kernel that streams Q in quadrature-point chunks; FEM_FP64 /
 * FEM_FP32 batches go through one batched SIMT kernel); one batched kernel
 * forms the CSR sums of all meshes.  Results are bit-identical to the same
 * meshes reassembled one by one with the same precision. */
typedef struct {
    int prec;       /* FEM_TF32X3 (default if opts is NULL), FEM_FP32 or FEM_FP64 */
    int tune;       /* 1: on the first launch, time the CSR-sum block size and the SIMT grid
                       on the real inputs and keep the fastest (the graph is captured after) */
    int use_graph;  /* 1: replay one CUDA graph per launch (default when opts is NULL) */
    int reserved;
} fem_batch_opts;
typedef struct {
    int n_meshes;
    int kernels_per_launch;  /* launches in one reassembly of the whole batch */
    int tc_tiles;            /* 128-element tensor-core tiles in the work list */
    int simt_blocks;         /* 64-element SIMT blocks */
    int sum_chunks;          /* CSR-sum work items */
    int sum_block;           /* threads per block of the CSR sum (tuned) */
    int simt_grid;           /* blocks of the SIMT kernel (tuned) */
    int tuned;               /* 1 once the tuner has run */
    int graph;               /* 1 if launches replay a CUDA graph */
    double tuned_ms;         /* fastest measured reassembly during tuning */
} fem_batch_info;
typedef struct fem_batch fem_batch;

/* Every mesh must have run fem_symbolic.  Allocates the meshes' element
 * scratch for the batch precision, builds the work lists and (unless tuning
 * is requested) captures the graph.  Synchronises `stream`.  While a batch
 * launch is in flight, its meshes must not be used by other calls.  While
 * the graph is captured (here, or after tuning in the first launch), no
 * other thread may synchronise the whole device: CUDA refuses that during a
 * stream capture. */
int fem_batch_create(fem_mesh* const* meshes, int n, const fem_batch_opts* opts, void* stream, fem_batch** out);
/* One reassembly of every mesh i: k[i] (law), d_u[i] (FP64 device nodal
 * values, may be NULL if mesh i needs M only), outputs d_vM[i], d_vK[i],
 * d_vT[i] (device CSR values, FP64 for FEM_FP64 and FP32 otherwise, NULL to
 * skip; any of the three arrays may be NULL).  Enqueued on `stream`. */
int fem_batch_launch(fem_batch* b, const fem_coeff* k, const double* const* d_u, void* const* d_vM,
                     void* const* d_vK, void* const* d_vT, void* stream);
int fem_batch_get_info(const fem_batch* b, fem_batch_info* out);
int fem_batch_destroy(fem_batch* b);

/* ----------------------------------------------------------- serving */
/* A request server for assembly and reassembly (Introduction: repeated
 * reassembly inside nonlinear solvers is a bottleneck; Section 5: between
 * Newton steps only S changes, the pattern, W and b stay).  A mesh sent with
 * an ASSEMBLE request stays resident on the device (geometry caches, CSR
 * pattern, slot segments, element scratch) under a mesh id; REASSEMBLE
 * requests then carry only a coefficient law and new nodal values.
 *
 * One scheduler thread per server owns the device work.  Continuous
 * batching: a queued request starts as soon as an in-flight slot is free
 * (max_inflight) and the device-memory budget allows, without waiting for
 * other requests to finish; started requests are spread over n_streams CUDA
 * streams so that the work of different meshes overlaps on the device.
 * Requests start in arrival order, except that a request waits (and later
 * ones may pass it) while another request of its mesh is in flight, so the
 * requests of one mesh run one at a time in submission order.  If the oldest
 * startable request does not fit the budget, nothing behind it starts.
 *
 * Budget accounting (bytes): every resident mesh (estimated from its size at
 * submit, its real size once built) plus the outputs of every request not yet
 * released.  A request that alone exceeds the budget, or that finds the
 * queue full, is refused at submit with FEM_EBUSY.  An ASSEMBLE request builds
 * the mesh and its pattern on the scheduler thread (it synchronises its
 * stream there), then reassembles it.  Results are the same values as
 * fem_assemble_all with the same precision.
 *
 * Fused launches (fuse_min > 0; FEM_FP64, FEM_TF32X3 and FEM_FP32 servers):
 * when at least fuse_min REASSEMBLE requests of idle meshes are startable,
 * they start together as one launch of a batch (fem_batch_*) over all
 * resident meshes, the meshes without a request in it skipped, on a stream
 * of its own.  The batch is rebuilt (the scheduler waits for the device
 * then) when the set of resident meshes has changed since it was built.
 * Batched results carry the same bits as single-mesh calls, so fusing
 * changes no value.  Fewer startable requests start one by one as above. */
enum { FEM_REQ_ASSEMBLE = 1, FEM_REQ_REASSEMBLE = 2 };
typedef struct {
    int prec;             /* FEM_FP64, FEM_TF32X3 or FEM_FP32 for every request */
    int max_inflight;     /* requests started and not finished, >= 1 */
    int n_streams;        /* CUDA streams the requests are spread over, 1..64 */
    int max_queue;        /* pending requests before submit refuses (FEM_EBUSY) */
    size_t budget_bytes;  /* device bytes for resident meshes + unreleased outputs */
    int fuse_min;         /* fuse this many startable REASSEMBLE requests or more; 0: never */
    int reserved;
} fem_serve_opts;
typedef struct {
    int kind;                    /* FEM_REQ_ASSEMBLE or FEM_REQ_REASSEMBLE */
    int which;                   /* FEM_MAT_M | FEM_MAT_K | FEM_MAT_T, nonzero */
    uint64_t mesh_id;            /* REASSEMBLE: id from an earlier ASSEMBLE result */
    const fem_mesh_desc* desc;   /* ASSEMBLE: the mesh (host or device buffers, copied at submit) */
    const fem_coeff* k;          /* law of k(u) (needed for K or T) */
    const double* u;             /* host FP64 nodal values (needed for K or T; copied at submit) */
} fem_request;
typedef struct {
    int status;                  /* FEM_OK, or the request's error (message in fem_last_error) */
    int prec;                    /* precision the values were computed in */
    uint64_t mesh_id;            /* the mesh's id (new for ASSEMBLE) */
    int64_t n, nnz;
    const int32_t* d_row_ptr;    /* device CSR pattern, owned by the resident mesh */
    const int32_t* d_col_idx;
    void* d_vM;                  /* device CSR values (NULL if not requested); library-owned */
    void* d_vK;                  /* until fem_serve_release(ticket) */
    void* d_vT;
    double t_submit_us, t_start_us, t_done_us;  /* host clock, microseconds since server creation;
                                                   t_done is when the scheduler saw completion */
} fem_result;
typedef struct {
    int pending, inflight, resident_meshes;
    size_t bytes_in_use, peak_bytes;
    int64_t single_launches;    /* requests started one by one */
    int64_t fused_launches;     /* fused launches, and the requests they carried */
    int64_t fused_requests;
    int64_t batch_builds;       /* builds of the fused launches' batch */
    double host_start_us;       /* scheduler time spent enqueueing device work (incl. batch builds) */
} fem_serve_counters;
typedef struct fem_server fem_server;

/* Creates a server on the current device (starts its scheduler thread).
 * Raises the release threshold of the device's default memory pool (the
 * source of request outputs) to budget_bytes if it is lower, so that freed
 * outputs stay mapped for later requests; the setting belongs to this
 * process's context and ends with it. */
int fem_serve_create(const fem_serve_opts* opts, fem_server** out);
/* Copies the request's inputs and queues it; *ticket identifies it. */
int fem_serve_submit(fem_server* s, const fem_request* req, uint64_t* ticket);
/* Waits up to timeout_us for the request: FEM_OK with *out filled once it
 * finished (out->status is the request's own status), FEM_EAGAIN if
 * timeout_us <= 0 and it has not, FEM_ETIMEOUT if the wait ran out. */
int fem_serve_poll(fem_server* s, uint64_t ticket, int timeout_us, fem_result* out);
/* Completion order: waits up to timeout_us for a finished request that no
 * earlier call returned and that is not released, and stores its ticket
 * (then fem_serve_poll gives its result at once).  FEM_EAGAIN if
 * timeout_us <= 0 and none is ready, FEM_ETIMEOUT if the wait ran out.
 * Lets a client release results as they finish instead of in submission
 * order, where one slow mesh would hold every later result's memory. */
int fem_serve_next_done(fem_server* s, int timeout_us, uint64_t* ticket);
/* Frees a finished request's outputs (the caller's reads of them must have
 * completed) and forgets the ticket. */
int fem_serve_release(fem_server* s, uint64_t ticket);
/* Destroys a resident mesh (FEM_ESTATE while a request of it is in flight).
 * Queued requests of the mesh then fail; pattern pointers of earlier results
 * become invalid. */
int fem_serve_evict(fem_server* s, uint64_t mesh_id);
int fem_serve_stats(fem_server* s, fem_serve_counters* out);
/* Stops the scheduler (queued requests are dropped), waits for the device
 * work in flight and frees everything the server holds. */
int fem_serve_destroy(fem_server* s);

/* ------------------------------------------- boundary terms and Newton step */
/* The Newton quantities of one implicit Euler step (Section 5):
 *   F(u) = M (u - u^s) + dt K(u) u - dt f(u),
 *   dF/du = Mt + M + dt (K + T) - dt B,
 * where f holds the boundary load b_i = int_{dOmega_N} g_N(u_h) phi_i dS
 * (Section 2; no volume source) and B_ik = int_{dOmega_N} g_N'(u_h) phi_i
 * phi_k dS is its derivative (Section 5).  Experiment 2 (Section 6) uses
 * convection plus radiation on the whole boundary, g_N = h_c (T_a - u) +
 * h_r (T_a^4 - u^4): pass it as a FEM_K_POLY law (coefficients h_c T_a +
 * h_r T_a^4, -h_c, 0, 0, -h_r); g_N' comes from the same law.  All in FP64.
 *
 * Boundary facets are the element faces that belong to no other element;
 * face f of an element is the face opposite its local vertex f, and its
 * nodes are the element's local nodes off that vertex.  fem_boundary_facets
 * finds them once per mesh on the device (requires fem_symbolic;
 * synchronises `stream`) and lists them in ascending (element, face) order;
 * *n_facets receives their number.  Idempotent. */
int fem_boundary_facets(fem_mesh* mesh, void* stream, int64_t* n_facets);
/* Copies the facet list: d_elem[f], d_face[f] (device, caller-owned, either
 * may be NULL).  Requires fem_boundary_facets. */
int fem_get_boundary_facets(fem_mesh* mesh, int32_t* d_elem, int32_t* d_face, void* stream);
/* B(u) into d_vB (nnz FP64 CSR values on the mesh pattern: the boundary
 * pattern is part of the volume pattern) and the boundary load into d_b (n
 * FP64 values; 0 off the boundary); either may be NULL.  Each facet's
 * matrices are one product V = X Q on the facet (X[q] = w_q |J_f| g'(u_q),
 * the paper's mass-type product, Section 4.1), then each boundary row adds
 * its facets in ascending order (deterministic).  Quadrature on a facet:
 * Gauss-Legendre with p+1 points on edges, the degree-2p triangle rule on
 * faces.  d_mask: one byte per facet, nonzero where the facet belongs to
 * dOmega_N (NULL: the whole boundary).  d_u: FP64 nodal values.  Device
 * pointers only (FEM_EINVAL otherwise).  Requires fem_symbolic (the facets
 * are found on the first call, which synchronises `stream`). */
int fem_assemble_boundary(fem_mesh* mesh, const fem_coeff* g, const double* d_u, const uint8_t* d_mask,
                          double* d_vB, double* d_b, void* stream);
/* d_y = alpha A d_x + beta d_y with A the FP64 CSR values d_vals on the mesh
 * pattern (a row's terms added by ascending column).  Device pointers. */
int fem_csr_spmv(fem_mesh* mesh, const double* d_vals, double alpha, const double* d_x, double beta, double* d_y,
                 void* stream);
/* d_F = M (u - u^s) + dt K u - dt b (FP64, n values; d_b may be NULL for
 * b = 0; M may be M(u) from fem_assemble_mass_u) and, if d_norms is not
 * NULL, d_norms[0] = ||F||_2 and d_norms[1] = ||F||_inf computed on the
 * device in one fixed order (rows by ascending column; chunks of 256 rows,
 * then the chunks in ascending order), so the norms are reproducible bit for
 * bit.  Device pointers only. */
int fem_residual(fem_mesh* mesh, const double* d_vM, const double* d_vK, const double* d_b, const double* d_u,
                 const double* d_us, double dt, double* d_F, double* d_norms, void* stream);
/* d_vJ = Mt + M + dt (K + T) - dt B entry by entry on the mesh pattern (the
 * Jacobian of the implicit Euler residual, Section 5); d_vMt (the mass
 * tensor times u - u^s, from fem_assemble_mass_u), d_vT (the tangent) and
 * d_vB may be NULL for zero.  FP64 device pointers.  d_vJ may alias one of
 * the inputs. */
int fem_jacobian(fem_mesh* mesh, double dt, const double* d_vM, const double* d_vMt, const double* d_vK,
                 const double* d_vT, const double* d_vB, double* d_vJ, void* stream);

/* ----------------------------------------------------- solving the heat problem */
/* The paper solves the Newton systems of Section 5 with MATLAB's backslash
 * or with GMRES (Section 6, Experiment 2); the linear solver is not part of
 * its method.  These calls close the loop on the GPU in FP64.
 *
 * fem_bicgstab: A x = b for FP64 CSR values d_vA on the mesh pattern,
 * Jacobi-preconditioned BiCGStab starting from the given d_x, until
 * ||b - A x||_2 <= rtol ||b||_2 or maxit iterations; *iters and *relres
 * (may be NULL) receive the iterations and the final relative residual.
 * Every reduction runs in a fixed order, so a solve is bitwise repeatable.
 * Scratch (8 vectors of n) is owned by the mesh.  Synchronises `stream`
 * once per iteration (the convergence test reads one number). */
int fem_bicgstab(fem_mesh* mesh, const double* d_vA, const double* d_b, double* d_x, double rtol, int maxit,
                 int* iters, double* relres, void* stream);

/* One implicit Euler step of m du/dt - div(k(u) grad u) = 0 with the
 * boundary flux g(u) (the load of fem_assemble_boundary; Experiment 2:
 * convection + radiation), the mesh's constant mass coefficient m, and
 * time step dt: Newton's method on F(u) = M (u - u^s) + dt K(u) u - dt b(u)
 * with the Jacobian M + dt (K + T) - dt B, each linear system solved by
 * fem_bicgstab (relative tolerance krylov_rtol, at most max_krylov
 * iterations).  d_us: the previous state; d_u: the initial guess on entry,
 * the new state on return.  Stops when ||F||_2 <= newton_rtol ||F(u_0)||_2
 * or after max_newton Newton updates.  *rep (may be NULL) receives the
 * counts and residuals.  Matrices and vectors of the step are owned by the
 * mesh.  Synchronises `stream`. */
typedef struct {
    int newton_iters, krylov_iters, converged, pad;
    double residual0, residual, max_krylov_relres;
} fem_heat_report;
int fem_heat_step(fem_mesh* mesh, const fem_coeff* k, const fem_coeff* g, const uint8_t* d_mask, double dt,
                  const double* d_us, double* d_u, double newton_rtol, int max_newton, double krylov_rtol,
                  int max_krylov, fem_heat_report* rep, void* stream);

/* The conductivity law alone, in FP64 on the GPU: d_k[i] = k(u_i) and
 * d_dk[i] = k'(u_i) for i < n, with the very device code the FP64 element
 * kernels evaluate at the quadrature points (the S of Algorithm 2, whose
 * entries are k(u_h) at the nodes x_q, Section 4.2; k' enters the tangent,
 * Section 5.2).  The sine law uses a table-driven sin/cos accurate to about
 * one unit in the last place.  All pointers are device pointers (FEM_EINVAL
 * otherwise); d_k or d_dk may be NULL to skip it.  Enqueued on `stream`. */
int fem_law_eval(const fem_coeff* k, const double* d_u, int64_t n, double* d_k, double* d_dk, void* stream);
/* The same in FP32, with the device code of the FP32 and tensor-core
 * element kernels, at u_i rounded to FP32: polynomials by Horner, the sine
 * law by CUDA's sincosf, the piecewise-linear law as in FP64.  Same pointer
 * rules and errors as fem_law_eval. */
int fem_law_eval_fp32(const fem_coeff* k, const double* d_u, int64_t n, float* d_k, float* d_dk, void* stream);

/* ------------------------------------------------------ reference element */
/* The library's reference tables for (dim, order, qdeg): quadrature points
 * xq (nq x dim) and weights wq (nq, summing to 1/dim!), basis values phi
 * (nq x n_p) and reference gradients grad (nq x n_p x dim).  Any output may
 * be NULL; *nq receives the number of points.  Host only, no GPU needed. */
int fem_reference_tables(int dim, int order, int qdeg, double* xq, double* wq, double* phi,
                         double* grad, int* nq);

/* ---------------------------------------------------------- allocator */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} fem_allocator;
/* NULL restores the default.  Not thread-safe with concurrent calls. */
int fem_set_allocator(const fem_allocator* a);

/* ------------------------------------------------------------- errors */
/* Copies the last error message of the calling thread into buf (always
 * NUL-terminated); returns its full length. */
int fem_last_error(char* buf, size_t len);

/* Library version string. */
const char* fem_version(void);


/* -------------------------------------- FP64 reassembly without allocation */
/* The paper has no counterpart to this call.  It is fem_assemble_all for
 * FEM_FP64 with device pointers only, for callers that must not allocate
 * device memory while they run: for example a solver loop whose device memory
 * is budgeted up front by a framework that owns the whole pool, or a
 * latency-critical service loop in which a driver allocation (which can
 * synchronise the device) is not acceptable.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: the element matrices between the
 * element product and the CSR sum live in one fixed device array of
 * FEM_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits.
 *  - Limit: the selected matrices must fit the array, i.e. n_elems times
 *    8 bytes times n_p(n_p+1)/2 for each of M and K plus n_p^2 for T (each
 *    part rounded up to 256 bytes) <= FEM_NOALLOC_SCRATCH_BYTES; larger meshes
 *    get FEM_EINVAL with the sizes in the message.
 *  - Set-up: the first call on a device looks up the array's device address
 *    and uploads the reference tables.  With CUDA's default lazy module
 *    loading, that look-up is when the driver loads the array into the
 *    device's memory: the first call on each device therefore makes that one
 *    driver allocation and may synchronise the device.  Make the first call
 *    before any stream capture and outside latency-critical loops (a warm-up
 *    call); later calls allocate nothing.
 *  - Pointers: d_u (when K or T is requested) and every non-NULL output must
 *    be device (or managed) memory of the current device, and the mesh must
 *    have been created on the current device; FEM_EINVAL otherwise, before
 *    any work is enqueued.
 *  - Sharing: all calls use the same array and it keeps the last call's
 *    contents (every entry is rewritten before it is read, nothing needs
 *    clearing); calls whose GPU work overlaps race on it.
 * Requires fem_symbolic.  d_u: FP64 nodal values (unused for M only);
 * d_vM, d_vK, d_vT: caller-owned FP64 CSR values, NULL to skip. */
#define FEM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int fem_assemble_all_noalloc(fem_mesh* mesh, const fem_coeff* k, const double* d_u, double* d_vM,
                             double* d_vK, double* d_vT, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FEM_H */
