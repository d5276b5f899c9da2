// capi.cu -- the extern "C" boundary of libfem (see include/fem.h).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "fem_internal.h"
#include "refelem.h"

namespace fem {

namespace {
thread_local std::string g_last_error;
fem_allocator g_alloc = {nullptr, nullptr, nullptr};
std::mutex g_alloc_mu;
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    cudaGetLastError();   // do not leave a non-sticky error for the next launch check
    return FEM_ECUDA;
}

int buf_alloc(DevBuf& b, size_t bytes, cudaStream_t s) {
    if (b.ptr && b.bytes >= bytes) return FEM_OK;
    buf_free(b, s);
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        b.owner = g_alloc;
    }
    if (bytes == 0) bytes = 16;
    if (b.owner.alloc) {
        b.ptr = b.owner.alloc(bytes, s, b.owner.ctx);
    } else if (cudaMallocAsync(&b.ptr, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
    }
    if (!b.ptr) return fail(FEM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    b.bytes = bytes;
    return FEM_OK;
}

void trace_launch(const char* kernel, long long grid, int block, size_t smem, int ctas) {
    static const bool on = std::getenv("FEM_TRACE_LAUNCH") != nullptr;
    if (on)
        std::fprintf(stderr, "[libfem] %s grid=%lld block=%d smem=%zu ctas_per_sm=%d\n", kernel, grid, block, smem,
                     ctas);
}

int ctas_per_sm(const cudaFuncAttributes& fa, int threads, size_t smem, int dev) {
    int per_sm_smem = 0, reserved = 0, regs = 0, max_threads = 0, max_blocks = 0;
    cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaDeviceGetAttribute(&max_blocks, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    const size_t per_block = smem + fa.sharedSizeBytes + (size_t)reserved;
    int n = max_blocks > 0 ? max_blocks : 16;
    if (per_block > 0) n = std::min<long long>(n, (long long)per_sm_smem / (long long)per_block);
    const int warps = (threads + 31) / 32;
    const int regs_per_warp = ((fa.numRegs > 0 ? fa.numRegs : 1) * 32 + 255) / 256 * 256;
    if (regs > 0) n = std::min(n, regs / (regs_per_warp * warps));
    if (max_threads > 0) n = std::min(n, max_threads / (warps * 32));
    return n;
}

void buf_free(DevBuf& b, cudaStream_t s) {
    if (b.ptr) {
        if (b.owner.free) b.owner.free(b.ptr, b.bytes, s, b.owner.ctx);
        else cudaFreeAsync(b.ptr, s);
    }
    b.ptr = nullptr;
    b.bytes = 0;
    b.owner = fem_allocator{nullptr, nullptr, nullptr};
}

int tc_error_flag(int clear);

namespace {

int type_of(int d, int p) { return (d - 2) * 3 + (p - 1); }
bool valid_prec(int prec) { return prec >= FEM_FP64 && prec <= FEM_BF16X6; }
int nlocal(int d, int p) { return d == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6; }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_coeff(const fem_coeff* k) {
    if (!k) return fail(FEM_EINVAL, "coefficient is NULL");
    if (k->kind == FEM_K_POLY) {
        if (k->n < 1 || k->n > 8) return fail(FEM_EINVAL, "polynomial law needs 1..8 coefficients");
    } else if (k->kind == FEM_K_SIN) {
        if (k->n != 3) return fail(FEM_EINVAL, "sine law needs 3 parameters");
    } else if (k->kind == FEM_K_PWLIN) {
        if (k->n < 4 || k->n > 16 || (k->n & 1)) return fail(FEM_EINVAL, "piecewise-linear law needs 2m parameters, m in 2..8");
        int m = k->n / 2;
        for (int i = 0; i + 1 < m; ++i)
            if (!(k->p[i] < k->p[i + 1])) return fail(FEM_EINVAL, "knots must be strictly ascending");
    } else {
        return fail(FEM_EINVAL, "unknown conductivity law");
    }
    for (int i = 0; i < k->n; ++i)
        if (!std::isfinite(k->p[i])) return fail(FEM_EINVAL, "non-finite coefficient parameter");
    return FEM_OK;
}

CoeffDev to_dev(const fem_coeff* k) {
    CoeffDev c;
    std::memset(&c, 0, sizeof(c));
    if (!k) return c;
    c.kind = k->kind;
    c.n = k->n;
    if (k->kind == FEM_K_PWLIN) {
        // device layout: knots in p[0..7], values in p[8..15]
        const int m = k->n / 2;
        for (int i = 0; i < m; ++i) {
            c.p[i] = k->p[i];
            c.p[8 + i] = k->p[m + i];
        }
    } else {
        for (int i = 0; i < k->n; ++i) c.p[i] = k->p[i];   // unused parameters stay zero
    }
    if (k->kind == FEM_K_POLY) {
        // Zero leading coefficients are dropped: the device Horner of the
        // remaining degree gives the same bits (the dropped steps only carry
        // exact zeros) and is specialised for short polynomials.
        while (c.n > 1 && c.p[c.n - 1] == 0.0) --c.n;
    }
    return c;
}

// Formation (Algorithm 2, up to the products V): V for the matrices in `mask` (bit 0 M,
// bit 1 K, bit 2 T) into the mesh's scratch buffers.
template <typename T>
int form_t(fem_mesh* m, const fem_coeff* k, const double* ud, int prec, int mask, cudaStream_t s, int64_t e0 = 0,
           int64_t e1 = -1) {
    const int64_t E = m->E;
    const int nsym = m->np * (m->np + 1) / 2, nt = m->np * m->np;
    int rc;
    T *VM = nullptr, *VK = nullptr, *VT = nullptr;
    if (mask & 3) {   // M and K share one interleaved array: M at even, K at odd positions
        if ((rc = buf_alloc(m->VMK, 2 * sizeof(T) * (size_t)E * nsym, s))) return rc;
        if (mask & 1) VM = m->VMK.as<T>();
        if (mask & 2) VK = m->VMK.as<T>() + 1;
    }
    if (mask & 4) {
        if ((rc = buf_alloc(m->VT, sizeof(T) * (size_t)E * nt, s))) return rc;
        VT = m->VT.as<T>();
    }
    CoeffDev kd = to_dev(k);
    if constexpr (sizeof(T) == 8) {
        rc = element_simt_fp64(*m, kd, ud, VM, VK, VT, s, e0, e1);
    } else {
        const double* us = (mask & 6) ? ud : nullptr;
        if (m->perq && prec != FEM_FP32)
            return fail(FEM_EINVAL, "per-point geometry (isoparametric or a conductivity field) runs FEM_FP64 and "
                                    "FEM_FP32 only");
        rc = prec == FEM_TF32X3   ? element_tc_tf32x3(*m, kd, us, VM, VK, VT, s, e0, e1)
             : prec == FEM_BF16X3 ? element_tc_bf16(*m, kd, us, VM, VK, VT, 2, s, e0, e1)
             : prec == FEM_BF16X6 ? element_tc_bf16(*m, kd, us, VM, VK, VT, 3, s, e0, e1)
                                  : element_simt_fp32(*m, kd, us, VM, VK, VT, s, e0, e1);
    }
    if (rc) return rc;
    m->v_prec = prec;
    m->v_mask = mask;
    return FEM_OK;
}

// Global assembly (the last step of Algorithm 2) of the formed V into CSR values.
// plain: the M/K scratch holds M/K pairs per symmetric entry whatever the
// element type (the u-dependent mass); otherwise it holds what the element
// kernels formed (factored for P1 simplices in FP64).
template <typename T>
int sum_t(fem_mesh* m, T* vM, T* vK, T* vT, cudaStream_t s, int64_t s0 = 0, int64_t s1 = -1, bool plain = false) {
    const T* VM = vM ? m->VMK.as<T>() : nullptr;
    const T* VK = vK ? m->VMK.as<T>() + 1 : nullptr;
    const T* VT = vT ? m->VT.as<T>() : nullptr;
    if constexpr (sizeof(T) == 8)
        return scatter_fp64(*m, VM, VK, VT, vM, vK, vT, !plain && p1_factored(*m), s, s0, s1);
    else return scatter_fp32(*m, VM, VK, VT, vM, vK, vT, s, s0, s1);
}

// Element bytes of V per element (all three matrices) in a precision.
size_t v_bytes_per_element(const fem_mesh& m, int prec) {
    const size_t nsym = (size_t)m.np * (m.np + 1) / 2, nt = (size_t)m.np * m.np;
    return (prec == FEM_FP64 ? 8 : 4) * (2 * nsym + nt);
}

// Chunks of the fine plan of about `target` bytes of V each (at most
// max_chunks): element bounds eb[0..n], slot bounds sb[0..n].
int plan_chunks(fem_mesh* m, int prec, size_t target, int max_chunks, cudaStream_t s, std::vector<int64_t>& eb,
                std::vector<int64_t>& sb) {
    int rc = chunk_plan_fine(*m, s);
    if (rc) return rc;
    const int nfine = (int)m->plan_e.size() - 1;
    eb.clear();
    sb.clear();
    if (nfine <= 0) {
        eb = {0, 0};
        sb = {0, m->nnz > 0 ? m->nnz : 0};
        return FEM_OK;
    }
    const int64_t ec = m->plan_e[1] - m->plan_e[0];
    const size_t per_fine = (size_t)ec * v_bytes_per_element(*m, prec);
    int g = (int)std::max<size_t>(1, target / std::max<size_t>(per_fine, 1));
    if (max_chunks < 1) max_chunks = 1;
    while ((nfine + g - 1) / g > max_chunks) ++g;
    for (int j = 0;; j += g) {
        const int jj = std::min(j, nfine);
        eb.push_back(m->plan_e[jj]);
        sb.push_back(m->plan_s[jj]);
        if (jj == nfine) break;
    }
    return FEM_OK;
}

// default chunk size: V of one chunk stays well inside the 129 MB L2
constexpr size_t CHUNK_TARGET_BYTES = size_t(48) << 20;

template <typename T>
int assemble_t(fem_mesh* m, const fem_coeff* k, const void* u, int prec, void* vM, void* vK, void* vT,
               cudaStream_t s) {
    const int64_t nnz = m->nnz;
    bool host_io = false;
    const double* ud = nullptr;
    int rc;
    if (vK || vT) {
        if (!u) return fail(FEM_EINVAL, "u is NULL");
        if (is_device_ptr(u)) {
            ud = static_cast<const double*>(u);
        } else {
            host_io = true;
            if ((rc = buf_alloc(m->u_stage, sizeof(double) * (size_t)m->n, s))) return rc;
            FEM_CUDA_TRY(cudaMemcpyAsync(m->u_stage.ptr, u, sizeof(double) * (size_t)m->n, cudaMemcpyHostToDevice, s));
            ud = m->u_stage.as<double>();
        }
    }
    // outputs: device memory as given; host memory through a device stage and
    // one copy per array.  (Letting the CSR sum store straight into
    // page-locked host memory measured 2.3x slower end to end on GB300: its
    // scattered 4-byte stores cross the CPU-GPU link in small pieces.)
    void* outs[3] = {vM, vK, vT};
    T* outd[3] = {nullptr, nullptr, nullptr};
    bool out_staged[3] = {false, false, false};
    int nstaged = 0;
    for (int i = 0; i < 3; ++i) {
        if (!outs[i]) continue;
        if (is_device_ptr(outs[i])) {
            outd[i] = static_cast<T*>(outs[i]);
        } else {
            out_staged[i] = true;
            ++nstaged;
        }
    }
    if (nstaged) {
        host_io = true;
        if ((rc = buf_alloc(m->out_stage, sizeof(T) * (size_t)nnz * 3, s))) return rc;
        for (int i = 0; i < 3; ++i)
            if (out_staged[i]) outd[i] = m->out_stage.as<T>() + (size_t)i * nnz;
    }
    int mask = (vM ? 1 : 0) | (vK ? 2 : 0) | (vT ? 4 : 0);
    if (nstaged) {
        // staged outputs: the element ranges of a chunk plan are formed and
        // their completed slots summed in turn, and each chunk's values are
        // copied to the host on a second stream while the next chunk is
        // formed, so the copies (bound by the CPU-GPU link) overlap both
        // phases.  A slot's value does not depend on the plan.
        const size_t nsym = (size_t)m->np * (m->np + 1) / 2, nt = (size_t)m->np * m->np;
        const size_t vbytes = sizeof(T) * (size_t)m->E * (2 * nsym + nt);
        std::vector<int64_t> eb, sb;
        constexpr int NCH = 8;
        if ((rc = plan_chunks(m, prec, std::max(vbytes / NCH, CHUNK_TARGET_BYTES), NCH, s, eb, sb))) return rc;
        if (eb.size() > 2) {
            if (!m->copy_stream) {
                FEM_CUDA_TRY(cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking));
                for (auto& ev : m->copy_ev) FEM_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            }
            const int n = (int)eb.size() - 1;
            for (int c = 0; c < n; ++c) {
                if ((rc = form_t<T>(m, k, ud, prec, mask, s, eb[c], eb[c + 1]))) return rc;
                const int64_t a = sb[c], b = sb[c + 1];
                if (b <= a) continue;
                if ((rc = sum_t<T>(m, outd[0], outd[1], outd[2], s, a, b))) return rc;
                // the copy stream waits for this chunk's sums (an event may be
                // recorded again once a wait on it has been enqueued)
                FEM_CUDA_TRY(cudaEventRecord(m->copy_ev[0], s));
                FEM_CUDA_TRY(cudaStreamWaitEvent(m->copy_stream, m->copy_ev[0], 0));
                for (int i = 0; i < 3; ++i)
                    if (out_staged[i])
                        FEM_CUDA_TRY(cudaMemcpyAsync(static_cast<T*>(outs[i]) + a, outd[i] + a, sizeof(T) * (size_t)(b - a),
                                                     cudaMemcpyDeviceToHost, m->copy_stream));
            }
            FEM_CUDA_TRY(cudaStreamSynchronize(m->copy_stream));
            FEM_CUDA_TRY(cudaStreamSynchronize(s));
            return FEM_OK;
        }
    }
    // One formation, then one sum.  (Chunking the two phases so that each
    // range's V is summed while in L2 -- fem_chunk_plan and the range calls
    // -- measured slower on GB300 for device outputs: the sum is bound by its
    // gather latency, not by where V lives, and every extra launch adds a
    // tail.)
    if ((rc = form_t<T>(m, k, ud, prec, mask, s))) return rc;
    if (!nstaged) {
        if ((rc = sum_t<T>(m, outd[0], outd[1], outd[2], s))) return rc;
    } else {
        // staged outputs: sum in NR slot ranges and copy each range to the
        // host on a second stream as soon as it is summed, so the copies
        // (bound by the CPU-GPU link) overlap the rest of the sum.  A slot's
        // value does not depend on the range that covers it.
        constexpr int NR = 4;
        if (!m->copy_stream) {
            FEM_CUDA_TRY(cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking));
            for (auto& ev : m->copy_ev) FEM_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        }
        for (int r = 0; r < NR; ++r) {
            const int64_t a = nnz * r / NR, b = nnz * (r + 1) / NR;
            if ((rc = sum_t<T>(m, outd[0], outd[1], outd[2], s, a, b))) return rc;
            FEM_CUDA_TRY(cudaEventRecord(m->copy_ev[r], s));
            FEM_CUDA_TRY(cudaStreamWaitEvent(m->copy_stream, m->copy_ev[r], 0));
            for (int i = 0; i < 3; ++i)
                if (out_staged[i] && b > a)
                    FEM_CUDA_TRY(cudaMemcpyAsync(static_cast<T*>(outs[i]) + a, outd[i] + a, sizeof(T) * (size_t)(b - a),
                                                 cudaMemcpyDeviceToHost, m->copy_stream));
        }
        FEM_CUDA_TRY(cudaStreamSynchronize(m->copy_stream));
    }
    if (host_io) FEM_CUDA_TRY(cudaStreamSynchronize(s));
    return FEM_OK;
}

}  // namespace

int validate_coeff(const fem_coeff* k) { return check_coeff(k); }
CoeffDev coeff_to_device(const fem_coeff* k) { return to_dev(k); }

}  // namespace fem

size_t fem_mesh::device_bytes() const {
    const fem::DevBuf* bufs[] = {&coords, &conn, &geo64, &geo32, &gram64, &row_ptr, &col_idx, &seg_ptr, &contrib, &slot,
                                 &seg_head, &inc_ptr, &inc, &VMK, &VT, &u_stage, &out_stage, &bfacet, &bnode_ptr,
                                 &bnode_inc, &bscratch, &npart, &cfield, &geoq64, &geoq32, &solve, &newton};
    size_t t = 0;
    for (auto* b : bufs) t += b->bytes;
    return t;
}

using namespace fem;

extern "C" {

int fem_last_error(char* buf, size_t len) {
    const std::string& e = g_last_error;
    if (buf && len) {
        size_t n = e.size() < len - 1 ? e.size() : len - 1;
        std::memcpy(buf, e.data(), n);
        buf[n] = 0;
    }
    return (int)e.size();
}

const char* fem_version(void) { return "libfem 0.1 (sm_103a, tcgen05 TF32x3)"; }

int fem_set_allocator(const fem_allocator* a) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (a && (!a->alloc || !a->free)) return fail(FEM_EINVAL, "allocator needs both alloc and free");
    g_alloc = a ? *a : fem_allocator{nullptr, nullptr, nullptr};
    return FEM_OK;
}

int fem_reference_tables(int dim, int order, int qdeg, double* xq, double* wq, double* phi, double* grad, int* nq) {
    if ((dim != 2 && dim != 3) || order < 1 || order > 3) return fail(FEM_EINVAL, "dim must be 2|3, order 1..3");
    if (qdeg != 0 && qdeg != 2 * order) return fail(FEM_EINVAL, "only the degree-2*order rule is provided");
    const RefElem* R = refelem_for_type(type_of(dim, order));
    if (!R) return fail(FEM_EINVAL, "reference tables failed");
    if (nq) *nq = R->nq;
    if (xq) std::memcpy(xq, R->xq.data(), sizeof(double) * R->xq.size());
    if (wq) std::memcpy(wq, R->wq.data(), sizeof(double) * R->wq.size());
    if (phi) std::memcpy(phi, R->phi.data(), sizeof(double) * R->phi.size());
    if (grad) std::memcpy(grad, R->grad.data(), sizeof(double) * R->grad.size());
    return FEM_OK;
}

int fem_mesh_create(const fem_mesh_desc* desc, void* stream, fem_mesh** out) {
    if (!desc || !out) return fail(FEM_EINVAL, "NULL argument");
    *out = nullptr;
    const int d = desc->dim, p = desc->order;
    if ((d != 2 && d != 3) || p < 1 || p > 3) return fail(FEM_EINVAL, "dim must be 2|3 and order 1..3");
    if (desc->qdeg != 0 && desc->qdeg != 2 * p) return fail(FEM_EINVAL, "only the degree-2*order rule is provided");
    if (desc->n_nodes <= 0 || desc->n_nodes >= (int64_t)INT32_MAX || desc->n_elems < 0)
        return fail(FEM_EINVAL, "bad node or element count");
    const int np = nlocal(d, p);
    if ((desc->n_elems * np * np) >= ((int64_t)1 << 31)) return fail(FEM_EINVAL, "n_elems * n_p^2 must be < 2^31");
    if (!desc->coords || (desc->n_elems > 0 && !desc->conn)) return fail(FEM_EINVAL, "coords/conn is NULL");
    if (!std::isfinite(desc->mass_coeff)) return fail(FEM_EINVAL, "mass coefficient not finite");
    if (!refelem_for_type(type_of(d, p))) return fail(FEM_EINVAL, "reference tables failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    fem_mesh* m = new fem_mesh;
    m->d = d;
    m->p = p;
    m->np = np;
    m->type = type_of(d, p);
    m->nq = type_nq(m->type);
    m->n = desc->n_nodes;
    m->E = desc->n_elems;
    m->m = desc->mass_coeff;
    cudaGetDevice(&m->device);
    int rc;
    if ((rc = buf_alloc(m->coords, sizeof(double) * (size_t)m->n * d, s)) ||
        (rc = buf_alloc(m->conn, sizeof(int) * (size_t)m->E * np, s))) {
        fem_mesh_destroy(m);
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(m->coords.ptr, desc->coords, sizeof(double) * (size_t)m->n * d, cudaMemcpyDefault, s);
    if (e == cudaSuccess && m->E > 0)
        e = cudaMemcpyAsync(m->conn.ptr, desc->conn, sizeof(int) * (size_t)m->E * np, cudaMemcpyDefault, s);
    if (e != cudaSuccess) {
        fem_mesh_destroy(m);
        return cuda_fail(e, "copy mesh to device");
    }
    if ((rc = geometry_run(*m, s))) {
        std::string msg = g_last_error;
        fem_mesh_destroy(m);
        set_error(msg);
        return rc;
    }
    *out = m;
    return FEM_OK;
}

int fem_mesh_destroy(fem_mesh* m) {
    if (!m) return FEM_OK;
    cudaDeviceSynchronize();
    fem::DevBuf* bufs[] = {&m->coords, &m->conn, &m->geo64, &m->geo32, &m->gram64, &m->row_ptr, &m->col_idx, &m->seg_ptr,
                           &m->contrib, &m->slot, &m->seg_head, &m->inc_ptr, &m->inc, &m->VMK, &m->VT, &m->u_stage,
                           &m->out_stage, &m->bfacet, &m->bnode_ptr, &m->bnode_inc, &m->bscratch, &m->npart, &m->cfield, &m->geoq64, &m->geoq32, &m->solve,
                           &m->newton};
    for (auto* b : bufs) buf_free(*b, nullptr);
    if (m->copy_stream) {
        for (auto ev : m->copy_ev)
            if (ev) cudaEventDestroy(ev);
        cudaStreamDestroy(m->copy_stream);
    }
    cudaDeviceSynchronize();
    delete m;
    return FEM_OK;
}

int fem_mesh_get_info(const fem_mesh* m, fem_mesh_info* out) {
    if (!m || !out) return fail(FEM_EINVAL, "NULL argument");
    out->dim = m->d;
    out->order = m->p;
    out->n_p = m->np;
    out->n_q = m->nq;
    out->n_nodes = m->n;
    out->n_elems = m->E;
    out->nnz = m->have_pattern ? m->nnz : -1;
    out->n_flagged = m->n_flagged;
    out->device_bytes = m->device_bytes();
    return FEM_OK;
}

int fem_symbolic(fem_mesh* m, void* stream, fem_csr_pattern* out) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!m->have_pattern) {
        int rc = symbolic_run(*m, s);
        if (rc) return rc;
    }
    if (out) {
        out->n = m->n;
        out->nnz = m->nnz;
        out->d_row_ptr = m->row_ptr.as<int32_t>();
        out->d_col_idx = m->col_idx.as<int32_t>();
    }
    return FEM_OK;
}

int fem_copy_pattern(fem_mesh* m, int32_t* d_row_ptr, int32_t* d_col_idx, void* stream) {
    if (!m || !d_row_ptr || !d_col_idx) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FEM_CUDA_TRY(cudaMemcpyAsync(d_row_ptr, m->row_ptr.ptr, sizeof(int32_t) * (size_t)(m->n + 1),
                                 cudaMemcpyDeviceToDevice, s));
    if (m->nnz > 0)
        FEM_CUDA_TRY(cudaMemcpyAsync(d_col_idx, m->col_idx.ptr, sizeof(int32_t) * (size_t)m->nnz,
                                     cudaMemcpyDeviceToDevice, s));
    return FEM_OK;
}

int fem_get_slot_map(fem_mesh* m, int32_t* d_slot, void* stream) {
    if (!m || !d_slot) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    int rc = slot_map_build(*m, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    FEM_CUDA_TRY(cudaMemcpyAsync(d_slot, m->slot.ptr, sizeof(int32_t) * (size_t)(m->E * m->np * m->np),
                                 cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    return FEM_OK;
}

int fem_assemble_all(fem_mesh* m, const fem_coeff* k, const void* u, int prec, void* vM, void* vK, void* vT,
                     void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    if (!valid_prec(prec)) return fail(FEM_EINVAL, "unknown precision");
    if (!vM && !vK && !vT) return FEM_OK;
    if ((vK || vT)) {
        int rc = check_coeff(k);
        if (rc) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == FEM_FP64) return assemble_t<double>(m, k, u, prec, vM, vK, vT, s);
    return assemble_t<float>(m, k, u, prec, vM, vK, vT, s);
}

int fem_mesh_set_conductivity(fem_mesh* m, const double* c, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    const int d = m->d;
    double cn[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (c) {
        double amax = 0.0;
        for (int i = 0; i < d * d; ++i) {
            if (!std::isfinite(c[i])) return fail(FEM_EINVAL, "non-finite conductivity tensor");
            amax = std::max(amax, std::fabs(c[i]));
        }
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                if (std::fabs(c[a * d + b] - c[b * d + a]) > 1e-12 * amax)
                    return fail(FEM_EINVAL, "conductivity tensor is not symmetric");
                cn[a * 3 + b] = c[a * d + b];
            }
        // positive definite: a Cholesky factorisation exists
        double L[3][3] = {};
        for (int j = 0; j < d; ++j) {
            double s = cn[j * 3 + j];
            for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
            if (!(s > 1e-14 * amax)) return fail(FEM_EINVAL, "conductivity tensor is not positive definite");
            L[j][j] = std::sqrt(s);
            for (int i = j + 1; i < d; ++i) {
                double t = cn[i * 3 + j];
                for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
                L[i][j] = t / L[j][j];
            }
        }
    }
    for (int i = 0; i < 9; ++i) m->cond[i] = cn[i];
    m->v_prec = -1;   // formed element matrices used the previous tensor
    m->v_mask = 0;
    int rc = geometry_run(*m, static_cast<cudaStream_t>(stream));
    if (rc || !m->perq) return rc;
    return geometry_q_run(*m, static_cast<cudaStream_t>(stream));
}

int fem_mesh_set_isoparametric(fem_mesh* m, int on, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    m->iso = on != 0;
    m->perq = m->iso || m->cfield.ptr != nullptr;
    m->v_prec = -1;
    m->v_mask = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!m->perq) {
        buf_free(m->geoq64, s);
        buf_free(m->geoq32, s);
        return FEM_OK;
    }
    return geometry_q_run(*m, s);
}

int fem_mesh_set_conductivity_field(fem_mesh* m, const double* c_field, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    m->v_prec = -1;
    m->v_mask = 0;
    if (!c_field) {
        buf_free(m->cfield, s);
        m->perq = m->iso;
        if (!m->perq) {
            buf_free(m->geoq64, s);
            buf_free(m->geoq32, s);
            return FEM_OK;
        }
        return geometry_q_run(*m, s);
    }
    const size_t n = (size_t)m->E * m->nq * m->d * m->d;
    int rc = buf_alloc(m->cfield, sizeof(double) * n + 8, s);
    if (rc) return rc;
    FEM_CUDA_TRY(cudaMemcpyAsync(m->cfield.ptr, c_field, sizeof(double) * n,
                                 is_device_ptr(c_field) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    m->perq = true;
    return geometry_q_run(*m, s);
}

int fem_assemble_mass_u(fem_mesh* m, const fem_coeff* mk, const void* d_u, const void* d_us, int prec, void* d_vMu,
                        void* d_vMt, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    if (prec != FEM_FP64 && prec != FEM_FP32 && prec != FEM_TF32X3)
        return fail(FEM_EINVAL, "the u-dependent mass runs FEM_FP64, FEM_FP32 or FEM_TF32X3");
    if (m->perq && prec == FEM_TF32X3)
        return fail(FEM_EINVAL, "per-point geometry runs the SIMT products (FEM_FP64, FEM_FP32) only");
    if (!d_vMu && !d_vMt) return FEM_OK;
    int rc = check_coeff(mk);
    if (rc) return rc;
    if (!d_u) return fail(FEM_EINVAL, "u is NULL");
    if (d_vMt && !d_us) return fail(FEM_EINVAL, "u^s is NULL");
    const void* ptrs[4] = {d_u, d_vMt ? d_us : nullptr, d_vMu, d_vMt};
    for (const void* p : ptrs)
        if (p && !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_assemble_mass_u takes device pointers only");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t esz = prec == FEM_FP64 ? 8 : 4, nsym = (size_t)m->np * (m->np + 1) / 2;
    if ((rc = buf_alloc(m->VMK, 2 * esz * (size_t)m->E * nsym, s))) return rc;
    m->v_prec = -1;   // the scratch no longer holds matrices of fem_form_elements
    m->v_mask = 0;
    rc = prec == FEM_TF32X3
             ? element_mass_u_tc(*m, to_dev(mk), static_cast<const double*>(d_u), static_cast<const double*>(d_us),
                                 m->VMK.as<float>(), d_vMu != nullptr, d_vMt != nullptr, s)
             : element_mass_u(*m, to_dev(mk), static_cast<const double*>(d_u), static_cast<const double*>(d_us),
                              prec == FEM_FP64, m->VMK.ptr, d_vMu != nullptr, d_vMt != nullptr, s);
    if (rc) return rc;
    // M(u) from the even, the tensor term from the odd positions
    if (prec == FEM_FP64)
        return sum_t<double>(m, static_cast<double*>(d_vMu), static_cast<double*>(d_vMt), nullptr, s, 0, -1, true);
    return sum_t<float>(m, static_cast<float*>(d_vMu), static_cast<float*>(d_vMt), nullptr, s);
}

int fem_boundary_facets(fem_mesh* m, void* stream, int64_t* n_facets) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    int rc = boundary_setup(*m, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    if (n_facets) *n_facets = m->n_bfacets;
    return FEM_OK;
}

int fem_get_boundary_facets(fem_mesh* m, int32_t* d_elem, int32_t* d_face, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_boundary) return fail(FEM_ESTATE, "fem_boundary_facets has not run");
    if (m->n_bfacets == 0) return FEM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t* dst[2] = {d_elem, d_face};
    for (int i = 0; i < 2; ++i) {
        if (!dst[i]) continue;
        if (!is_device_ptr(dst[i])) return fail(FEM_EINVAL, "fem_get_boundary_facets takes device pointers");
        FEM_CUDA_TRY(cudaMemcpy2DAsync(const_cast<int32_t*>(dst[i]), sizeof(int32_t), m->bfacet.as<int>() + i,
                                       2 * sizeof(int32_t), sizeof(int32_t), (size_t)m->n_bfacets,
                                       cudaMemcpyDeviceToDevice, s));
    }
    return FEM_OK;
}

int fem_assemble_boundary(fem_mesh* m, const fem_coeff* g, const double* d_u, const uint8_t* d_mask, double* d_vB,
                          double* d_b, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    if (m->iso) return fail(FEM_EINVAL, "boundary terms are formed on straight facets: not on isoparametric meshes");
    int rc = check_coeff(g);
    if (rc) return rc;
    if (!d_vB && !d_b) return FEM_OK;
    const void* ptrs[4] = {d_u, d_mask, d_vB, d_b};
    for (const void* p : ptrs)
        if (p && !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_assemble_boundary takes device pointers only");
    if (!d_u) return fail(FEM_EINVAL, "u is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = boundary_setup(*m, s))) return rc;
    return boundary_assemble(*m, to_dev(g), d_u, d_mask, d_vB, d_b, s);
}

int fem_csr_spmv(fem_mesh* m, const double* d_vals, double alpha, const double* d_x, double beta, double* d_y,
                 void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    const void* ptrs[3] = {d_vals, d_x, d_y};
    for (const void* p : ptrs)
        if (!p || !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_csr_spmv takes non-NULL device pointers");
    return csr_spmv(*m, d_vals, alpha, d_x, beta, d_y, static_cast<cudaStream_t>(stream));
}

int fem_residual(fem_mesh* m, const double* d_vM, const double* d_vK, const double* d_b, const double* d_u,
                 const double* d_us, double dt, double* d_F, double* d_norms, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    const void* need[5] = {d_vM, d_vK, d_u, d_us, d_F};
    for (const void* p : need)
        if (!p || !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_residual: M, K, u, u^s and F are device pointers");
    if ((d_b && !is_device_ptr(d_b)) || (d_norms && !is_device_ptr(d_norms)))
        return fail(FEM_EINVAL, "fem_residual takes device pointers only");
    if (!std::isfinite(dt)) return fail(FEM_EINVAL, "dt is not finite");
    return csr_residual(*m, d_vM, d_vK, d_b, d_u, d_us, dt, d_F, d_norms, static_cast<cudaStream_t>(stream));
}

int fem_jacobian(fem_mesh* m, double dt, const double* d_vM, const double* d_vMt, const double* d_vK,
                 const double* d_vT, const double* d_vB, double* d_vJ, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    const void* need[3] = {d_vM, d_vK, d_vJ};
    for (const void* p : need)
        if (!p || !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_jacobian: M, K and J are device pointers");
    const void* opt[3] = {d_vMt, d_vT, d_vB};
    for (const void* p : opt)
        if (p && !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_jacobian takes device pointers only");
    if (!std::isfinite(dt)) return fail(FEM_EINVAL, "dt is not finite");
    return csr_jacobian(*m, dt, d_vM, d_vMt, d_vK, d_vT, d_vB, d_vJ, static_cast<cudaStream_t>(stream));
}

int fem_bicgstab(fem_mesh* m, const double* d_vA, const double* d_b, double* d_x, double rtol, int maxit, int* iters,
                 double* relres, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    const void* need[3] = {d_vA, d_b, d_x};
    for (const void* p : need)
        if (!p || !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_bicgstab takes non-NULL device pointers");
    if (!(rtol > 0) || maxit < 0) return fail(FEM_EINVAL, "rtol must be positive and maxit non-negative");
    return bicgstab(*m, d_vA, d_b, d_x, rtol, maxit, iters, relres, static_cast<cudaStream_t>(stream));
}

int fem_heat_step(fem_mesh* m, const fem_coeff* k, const fem_coeff* g, const uint8_t* d_mask, double dt,
                  const double* d_us, double* d_u, double newton_rtol, int max_newton, double krylov_rtol,
                  int max_krylov, fem_heat_report* rep, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    if (m->iso) return fail(FEM_EINVAL, "boundary terms are formed on straight facets: not on isoparametric meshes");
    int rc = check_coeff(k);
    if (rc) return rc;
    if ((rc = check_coeff(g))) return rc;
    const void* need[2] = {d_us, d_u};
    for (const void* p : need)
        if (!p || !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_heat_step: u^s and u are device pointers");
    if (d_mask && !is_device_ptr(d_mask)) return fail(FEM_EINVAL, "fem_heat_step takes device pointers only");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(FEM_EINVAL, "dt must be positive");
    if (!(newton_rtol > 0) || !(krylov_rtol > 0) || max_newton < 0 || max_krylov < 0)
        return fail(FEM_EINVAL, "tolerances must be positive and iteration limits non-negative");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = boundary_setup(*m, s))) return rc;
    return heat_step(*m, k, to_dev(g), d_mask, dt, d_us, d_u, newton_rtol, max_newton, krylov_rtol, max_krylov, rep,
                     s);
}

int fem_law_eval(const fem_coeff* k, const double* d_u, int64_t n, double* d_k, double* d_dk, void* stream) {
    int rc = check_coeff(k);
    if (rc) return rc;
    if (n < 0) return fail(FEM_EINVAL, "negative count");
    if (n == 0 || (!d_k && !d_dk)) return FEM_OK;
    const void* ptrs[3] = {d_u, d_k, d_dk};
    for (const void* p : ptrs)
        if (p && !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_law_eval takes device pointers only");
    if (!d_u) return fail(FEM_EINVAL, "u is NULL");
    return law_eval_fp64(to_dev(k), d_u, n, d_k, d_dk, static_cast<cudaStream_t>(stream));
}

int fem_law_eval_fp32(const fem_coeff* k, const double* d_u, int64_t n, float* d_k, float* d_dk, void* stream) {
    int rc = check_coeff(k);
    if (rc) return rc;
    if (n < 0) return fail(FEM_EINVAL, "negative count");
    if (n == 0 || (!d_k && !d_dk)) return FEM_OK;
    const void* ptrs[3] = {d_u, d_k, d_dk};
    for (const void* p : ptrs)
        if (p && !is_device_ptr(p)) return fail(FEM_EINVAL, "fem_law_eval_fp32 takes device pointers only");
    if (!d_u) return fail(FEM_EINVAL, "u is NULL");
    return law_eval_fp32(to_dev(k), d_u, n, d_k, d_dk, static_cast<cudaStream_t>(stream));
}

int fem_form_elements(fem_mesh* m, const fem_coeff* k, const void* d_u, int prec, int which, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!valid_prec(prec)) return fail(FEM_EINVAL, "unknown precision");
    if (which <= 0 || which > 7) return fail(FEM_EINVAL, "which must be a nonzero mask of FEM_MAT_M|K|T");
    if (which & 6) {
        int rc = check_coeff(k);
        if (rc) return rc;
        if (!d_u) return fail(FEM_EINVAL, "u is NULL");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == FEM_FP64) return form_t<double>(m, k, static_cast<const double*>(d_u), prec, which, s);
    return form_t<float>(m, k, static_cast<const double*>(d_u), prec, which, s);
}

int fem_sum_elements(fem_mesh* m, int prec, void* d_vM, void* d_vK, void* d_vT, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    int mask = (d_vM ? 1 : 0) | (d_vK ? 2 : 0) | (d_vT ? 4 : 0);
    if (!mask) return FEM_OK;
    if (m->v_prec != prec || (m->v_mask & mask) != mask)
        return fail(FEM_ESTATE, "element matrices of this precision were not formed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == FEM_FP64)
        return sum_t<double>(m, static_cast<double*>(d_vM), static_cast<double*>(d_vK), static_cast<double*>(d_vT), s);
    return sum_t<float>(m, static_cast<float*>(d_vM), static_cast<float*>(d_vK), static_cast<float*>(d_vT), s);
}

int fem_chunk_plan(fem_mesh* m, int prec, size_t target_bytes, int max_chunks, int* n_chunks, int64_t* e_bounds,
                   int64_t* s_bounds, void* stream) {
    if (!m || !n_chunks || !e_bounds || !s_bounds) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    if (!valid_prec(prec)) return fail(FEM_EINVAL, "unknown precision");
    if (max_chunks < 1) return fail(FEM_EINVAL, "max_chunks must be >= 1");
    std::vector<int64_t> eb, sb;
    int rc = plan_chunks(m, prec, target_bytes ? target_bytes : CHUNK_TARGET_BYTES, max_chunks,
                         static_cast<cudaStream_t>(stream), eb, sb);
    if (rc) return rc;
    *n_chunks = (int)eb.size() - 1;
    for (size_t i = 0; i < eb.size(); ++i) {
        e_bounds[i] = eb[i];
        s_bounds[i] = sb[i];
    }
    return FEM_OK;
}

int fem_form_elements_range(fem_mesh* m, const fem_coeff* k, const void* d_u, int prec, int which, int64_t e_begin,
                            int64_t e_end, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!valid_prec(prec)) return fail(FEM_EINVAL, "unknown precision");
    if (which <= 0 || which > 7) return fail(FEM_EINVAL, "which must be a nonzero mask of FEM_MAT_M|K|T");
    if (e_begin < 0 || e_begin > e_end || e_end > m->E || (e_begin % 128 != 0 && e_begin != e_end))
        return fail(FEM_EINVAL, "element range must satisfy 0 <= begin <= end <= n_elems, begin % 128 == 0");
    if (which & 6) {
        int rc = check_coeff(k);
        if (rc) return rc;
        if (!d_u) return fail(FEM_EINVAL, "u is NULL");
    }
    if (e_begin > 0 && (m->v_prec != prec || m->v_mask != which))
        return fail(FEM_ESTATE, "later ranges must follow a range starting at 0 with the same precision and matrices");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == FEM_FP64)
        return form_t<double>(m, k, static_cast<const double*>(d_u), prec, which, s, e_begin, e_end);
    return form_t<float>(m, k, static_cast<const double*>(d_u), prec, which, s, e_begin, e_end);
}

int fem_sum_elements_range(fem_mesh* m, int prec, int64_t s_begin, int64_t s_end, void* d_vM, void* d_vK,
                           void* d_vT, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    if (s_begin < 0 || s_begin > s_end || s_end > m->nnz) return fail(FEM_EINVAL, "slot range out of bounds");
    int mask = (d_vM ? 1 : 0) | (d_vK ? 2 : 0) | (d_vT ? 4 : 0);
    if (!mask) return FEM_OK;
    if (m->v_prec != prec || (m->v_mask & mask) != mask)
        return fail(FEM_ESTATE, "element matrices of this precision were not formed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == FEM_FP64)
        return sum_t<double>(m, static_cast<double*>(d_vM), static_cast<double*>(d_vK), static_cast<double*>(d_vT), s,
                             s_begin, s_end);
    return sum_t<float>(m, static_cast<float*>(d_vM), static_cast<float*>(d_vK), static_cast<float*>(d_vT), s,
                        s_begin, s_end);
}

int fem_assemble_mass(fem_mesh* m, int prec, void* values, void* stream) {
    if (!values) return fail(FEM_EINVAL, "values is NULL");
    return fem_assemble_all(m, nullptr, nullptr, prec, values, nullptr, nullptr, stream);
}

int fem_assemble_stiffness(fem_mesh* m, const fem_coeff* k, const void* u, int prec, void* values, void* stream) {
    if (!values) return fail(FEM_EINVAL, "values is NULL");
    return fem_assemble_all(m, k, u, prec, nullptr, values, nullptr, stream);
}

int fem_assemble_tangent(fem_mesh* m, const fem_coeff* k, const void* u, int prec, void* values, void* stream) {
    if (!values) return fail(FEM_EINVAL, "values is NULL");
    return fem_assemble_all(m, k, u, prec, nullptr, nullptr, values, stream);
}

int fem_device_status(void* stream) {
    FEM_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int f = tc_error_flag(1);
    if (f < 0) return fail(FEM_ECUDA, "cannot read device status word");
    if (f == 2) return fail(FEM_ECUDA, "a tensor-core kernel was launched with a wrong configuration and did not run");
    if (f) return fail(FEM_ETIMEOUT, "a tensor-core kernel gave up waiting for its MMA completion");
    return FEM_OK;
}

}  // extern "C"
