// fem_internal.h -- host-side internals shared by the libfem translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fem.h"
#include "fem_device.cuh"

namespace fem {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define FEM_CUDA_TRY(call)                                   \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return ::fem::cuda_fail(_e, #call); \
    } while (0)

// ------------------------------------------------------------- allocation
// Tracks one library-owned device buffer and the allocator that made it
// (a buffer is always returned to that allocator, even if the hook changed).
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    fem_allocator owner = {nullptr, nullptr, nullptr};
    template <typename T>
    T* as() const { return static_cast<T*>(ptr); }
};
int buf_alloc(DevBuf& b, size_t bytes, cudaStream_t s);   // FEM_OK / FEM_ENOMEM

// Launch tracing: with FEM_TRACE_LAUNCH set in the environment, every
// persistent kernel launch prints its shape to stderr.
void trace_launch(const char* kernel, long long grid, int block, size_t smem, int ctas_per_sm);

// CTAs of `fa` that fit on one SM with `smem` dynamic shared memory (the full
// unified array as shared memory), from the register and shared-memory
// budgets; persistent kernels size their grids with it.
int ctas_per_sm(const cudaFuncAttributes& fa, int threads, size_t smem, int dev);
void buf_free(DevBuf& b, cudaStream_t s);

}  // namespace fem

// The mesh handle (opaque to callers).
struct fem_mesh {
    int d = 0, p = 0, np = 0, nq = 0, type = 0, device = 0;
    int64_t n = 0, E = 0;
    double m = 1.0;
    fem::DevBuf coords, conn;           // FP64 n x d, int32 E x np
    fem::DevBuf geo64, geo32;           // SoA [NGEO][E]: b_e, A_e upper triangle
    // P1 simplices: the Gram matrix G A_e G^T of every element (n_sym FP64
    // values per element, symmetric storage; G = the constant reference
    // gradients), the u-independent part of K_e
    fem::DevBuf gram64;
    int64_t n_flagged = 0;
    // constant conductivity tensor c (SPD; identity by default), stored
    // 3 x 3 row-major whatever d (entry (a, b) at 3a + b): A_e = B_e^-1 c B_e^-T
    double cond[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    // per-quadrature-point geometry (Section 7): iso = map through all the
    // element's nodes; cfield = E x n_q x d x d conductivity tensors (FP64);
    // perq = either is set, the element kernels then read geoq64/geoq32
    // (SoA [1 + d(d+1)/2][E n_q], point (e, q) at e n_q + q)
    bool iso = false, perq = false;
    fem::DevBuf cfield, geoq64, geoq32;
    // symbolic
    bool have_pattern = false;
    int64_t nnz = -1;
    fem::DevBuf row_ptr, col_idx, seg_ptr, contrib, slot, inc_ptr, inc;
    bool have_slot = false;             // slot (element entry -> slot) built (slot_map_build)
    // per group of 32 consecutive contributions k: x = bit l set iff
    // contribution 32k+l is the first of its slot, y = slot of contribution 32k
    fem::DevBuf seg_head;               // uint2 per group
    int max_seg = 0;                    // longest segment (contributions of one slot)
    int sum_block = 256;                // threads per block of the CSR sum
    // chunk plan: fine element chunks and the slot prefix each one completes
    bool have_plan = false;
    std::vector<int64_t> plan_e, plan_s;
    // numeric scratch: element matrices V (per matrix) in the precision of the last call
    // M and K interleaved (element e, symmetric entry s: M at 2(e n_sym + s),
    // K at 2(e n_sym + s) + 1), T row-major n_p x n_p per element
    fem::DevBuf VMK, VT;
    int v_prec = -1, v_mask = 0;        // what VM/VK/VT currently hold
    // staging for host-pointer arguments; the copy stream and events that
    // move staged CSR values to the host range by range while later ranges
    // are still being summed (created on first use)
    fem::DevBuf u_stage, out_stage;
    // boundary facets (once per mesh): (element, face opposite local vertex)
    // pairs ascending, node -> facet incidences, facet products scratch;
    // partial sums of the residual norms
    bool have_boundary = false;
    int64_t n_bfacets = 0;
    fem::DevBuf bfacet, bnode_ptr, bnode_inc, bscratch, npart;
    // solver scratch: Krylov vectors and reduction partials; the Newton
    // step's matrices and vectors
    fem::DevBuf solve, newton;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[4] = {};
    size_t device_bytes() const;
};

namespace fem {

// ---------------------------------------------------------- kernel launches
int geometry_run(fem_mesh& m, cudaStream_t s);           // fills geo64, geo32, n_flagged
int geometry_q_run(fem_mesh& m, cudaStream_t s);         // fills geoq64, geoq32 (per-point mode)
int symbolic_run(fem_mesh& m, cudaStream_t s);           // fills pattern and segments
int slot_map_build(fem_mesh& m, cudaStream_t s);         // the element-entry -> slot map (once, on demand)
int scan_exclusive(const int* in, int64_t n, int* out, cudaStream_t s);   // n ints -> n+1 prefix sums
// boundary facets, node -> facet incidences (once; needs the pattern)
int boundary_setup(fem_mesh& m, cudaStream_t s);
// B (CSR values, zeroed first) and the boundary load b (n values), FP64;
// mask: one byte per facet (NULL: all facets)
int boundary_assemble(fem_mesh& m, const CoeffDev& g, const double* u, const unsigned char* mask, double* vB,
                      double* b, cudaStream_t s);
// CSR-level Newton quantities on the mesh pattern, FP64 (csr_ops.cu)
int csr_spmv(const fem_mesh& m, const double* vals, double alpha, const double* x, double beta, double* y,
             cudaStream_t s);
int csr_residual(fem_mesh& m, const double* vM, const double* vK, const double* b, const double* u, const double* us,
                 double dt, double* F, double* norms, cudaStream_t s);
int csr_jacobian(const fem_mesh& m, double dt, const double* vM, const double* vMt, const double* vK,
                 const double* vT, const double* vB, double* vJ, cudaStream_t s);
// Jacobi-preconditioned BiCGStab for A x = b on the mesh pattern (solve.cu)
int bicgstab(fem_mesh& m, const double* A, const double* b, double* x, double rtol, int maxit, int* iters,
             double* relres, cudaStream_t s);
// one implicit Euler step by Newton's method (solve.cu)
int heat_step(fem_mesh& m, const fem_coeff* k, const CoeffDev& g, const unsigned char* mask, double dt,
              const double* us, double* u, double newton_rtol, int max_newton, double krylov_rtol, int max_krylov,
              fem_heat_report* rep, cudaStream_t s);

// Element products V = X Q.  Any of VM, VK, VT may be null (matrix skipped).
int element_simt_fp64(const fem_mesh& m, const CoeffDev& k, const double* u, double* VM, double* VK, double* VT,
                      cudaStream_t s, int64_t e0 = 0, int64_t e1 = -1);
// The FP64 conductivity law alone: k(u_i), k'(u_i) for i < n (either output may be null).
int law_eval_fp64(const CoeffDev& k, const double* u, int64_t n, double* kv, double* dkv, cudaStream_t s);
int law_eval_fp32(const CoeffDev& k, const double* u, int64_t n, float* kv, float* dkv, cudaStream_t s);
// FP32 paths split each gathered FP64 nodal value as hi + lo (split_f64).
int element_simt_fp32(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                      cudaStream_t s, int64_t e0 = 0, int64_t e1 = -1);
// e0, e1: element range [e0, e1) (e1 = -1: to the end); V pointers are the
// whole-mesh arrays, rows e0.. are written.
int element_tc_tf32x3(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                      cudaStream_t s, int64_t e0 = 0, int64_t e1 = -1);
// The BF16 split-precision product (nparts 2: BF16x3, 3: BF16x6).
// u-dependent mass and mass-tensor term into the interleaved M/K storage
// (M(u) at even, the tensor term at odd positions); SIMT, FP64 or FP32.
int element_mass_u(const fem_mesh& m, const CoeffDev& mk, const double* u, const double* us, int fp64, void* VMK,
                   bool doMu, bool doMt, cudaStream_t s);
// the same products as element_mass_u on tcgen05 (TF32x3), P1-P3
// triangles and P1-P2 tetrahedra
int element_mass_u_tc(const fem_mesh& m, const CoeffDev& mk, const double* u, const double* us, float* VMK, bool doMu,
                      bool doMt, cudaStream_t s);
int element_tc_bf16(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                    int nparts, cudaStream_t s, int64_t e0 = 0, int64_t e1 = -1);

// The FP64 element kernel of P1 simplices (per-element geometry) stores
// factored element matrices (element_simt.cu): per element 4 values (M's
// diagonal and off-diagonal value, K's factor b s0 twice) at the start of
// the M/K scratch, K_e = b s0 times the element's Gram matrix in gram64,
// and T_e as its two factors (2 n_p values).
inline bool p1_factored(const fem_mesh& m) { return (m.type == 0 || m.type == 3) && !m.perq; }

// Segmented reduction of V into CSR values (outputs may be null).
// p1f: V holds the factored P1 element matrices (only where p1_factored);
// otherwise M/K pairs per symmetric entry and T's full entries.
// s0, s1: slot range [s0, s1) (s1 = -1: to the end); outputs are the
// whole CSR arrays.
int scatter_fp64(const fem_mesh& m, const double* VM, const double* VK, const double* VT, double* vM, double* vK,
                 double* vT, bool p1f, cudaStream_t s, int64_t s0 = 0, int64_t s1 = -1);
int scatter_fp32(const fem_mesh& m, const float* VM, const float* VK, const float* VT, float* vM, float* vK,
                 float* vT, cudaStream_t s, int64_t s0 = 0, int64_t s1 = -1);

// Fine chunk plan of a mesh (once): plan_e[j] = first element of fine chunk
// j, plan_s[j] = number of slots whose contributors all lie in chunks < j.
constexpr int PLAN_MAX_FINE = 64;
int chunk_plan_fine(fem_mesh& m, cudaStream_t s);

// Coefficient validation and device form, shared by the C entry points.
int validate_coeff(const fem_coeff* k);
CoeffDev coeff_to_device(const fem_coeff* k);

// ------------------------------------------------------------ batched launch
// Per-mesh parameters of a batched launch (a device-side table the batched
// kernels read; the host rewrites it before every launch).
struct BatchMesh {
    const int* conn;
    const float* geo32;
    const double* geo64;
    int64_t E, n, nnz;
    int np, type;
    const double* u;                     // FP64 nodal values
    CoeffDev k;
    double mass;
    void* VM; void* VK; void* VT;        // element-matrix scratch (FP32 or FP64): VM = the interleaved
                                         // M/K base, VK = VM + one value, VT
    const double* gram64;                // P1: Gram matrices of the elements (see fem_mesh)
    const int* seg_ptr;
    const int* contrib;
    const uint2* seg_head;               // per group of 32 contributions (see fem_mesh)
    int max_seg, pad2;
    void* vM; void* vK; void* vT;        // CSR outputs, NULL = skip
};
// One unit of work: `count` consecutive elements (or nodes, or pair groups of
// 64 contributions) of one mesh.
struct BatchItem {
    int mesh;
    int type;
    int64_t first;
    int count;
    int pad;
};
int tc_type_supported(int type);        // does the tensor-core tile of this element type fit?
int tc_type_smem(int type);             // dynamic shared memory of its tile
int tc_type_alloc(int type);            // TMEM columns of its tile (power of two)
int batch_tc_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int talloc, int smem, int grid,
                    cudaStream_t s);
// P3 tetrahedra: tensor-core product with Q streamed in quadrature-point chunks
int tc_chunked_supported(int type);
int batch_tc_chunked_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, cudaStream_t s);
template <typename T>
int batch_simt_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int max_type_smem, int grid,
                      cudaStream_t s);
int batch_simt_smem(int type, int fp64);
// the CSR sums of the items of meshes with n_p nodes per element (max_seg:
// the longest slot of those meshes)
template <typename T>
int batch_scatter_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int np, int max_seg,
                         cudaStream_t s);

// One-time per-device upload of the reference tables of each kernel module.
int tables_init_simt();
int tables_init_tc();
int tc_error_flag(int clear);   // device error word of the tensor-core kernels (1 = timeout)

}  // namespace fem
