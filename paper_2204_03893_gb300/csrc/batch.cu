// batch.cu -- batched reassembly of many meshes of uneven size and element
// type in one CUDA graph of a few persistent kernels.
//
// The paper splits a mesh with several element types into one mesh per type
// and merges the contributions before forming the sparse matrix (Section 7),
// and notes that the formation of all element matrices can be done in
// parallel (Section 7).  A batch generalises both: the element tiles of all
// meshes form one work list (grouped by element type) that one persistent
// tensor-core kernel walks, P3 tetrahedra (whose tile does not fit the
// tensor-core layout) and FP64/FP32 batches go through one batched SIMT
// kernel, and one batched CSR-sum kernel walks slot chunks of all meshes.
// Per-launch inputs (u, coefficient laws, output pointers) live in a
// device-side table that is rewritten from pinned host memory before each
// graph launch; the graph itself never changes.  An optional tuner times the
// launch shapes on the first launch (all candidates give identical bits:
// per-slot summation order is independent of the launch shape).
#include <algorithm>
#include <cstring>
#include <vector>

#include "fem_internal.h"

struct fem_batch {
    int n = 0, prec = 0, device = 0;
    bool use_graph = true, tune = false, tuned = false;
    std::vector<fem_mesh*> meshes;
    std::vector<fem::BatchMesh> host;      // static fields filled at creation
    fem::DevBuf d_meshes;
    fem::BatchMesh* pinned[2] = {nullptr, nullptr};
    cudaEvent_t staged[2] = {nullptr, nullptr};
    int cur = 0;
    fem::DevBuf d_tc, d_tc5, d_simt, d_scatter;
    int n_tc = 0, n_tc5 = 0, n_simt = 0, n_scatter = 0;
    int tc_grid = 0;
    // tensor-core tiles are grouped by element type; each type gets its own
    // launch (sized for that type's shared memory and TMEM) on its own branch
    struct TypeRange {
        int type, begin, count, talloc, smem;
    };
    std::vector<TypeRange> tc_ranges;
    static constexpr int NBRANCH = 6;
    cudaStream_t branch[NBRANCH] = {};
    cudaEvent_t fork = nullptr, join[NBRANCH] = {};
    int simt_smem = 0, simt_grid = 0;
    int scatter_block = 256;
    // CSR-sum items grouped by n_p: one launch per group
    struct SumRange {
        int np, begin, count, max_seg;
    };
    std::vector<SumRange> sum_ranges;
    double tuned_ms = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
};

namespace fem {
int validate_coeff(const fem_coeff* k);
CoeffDev coeff_to_device(const fem_coeff* k);

namespace {

int upload_items(DevBuf& buf, const std::vector<BatchItem>& items, cudaStream_t s) {
    int rc = buf_alloc(buf, sizeof(BatchItem) * (items.empty() ? 1 : items.size()), s);
    if (rc) return rc;
    if (!items.empty())
        FEM_CUDA_TRY(cudaMemcpyAsync(buf.ptr, items.data(), sizeof(BatchItem) * items.size(),
                                     cudaMemcpyHostToDevice, s));
    return FEM_OK;
}

// The kernels of one reassembly on stream s: the element products as
// parallel branches (one per tensor-core element type, plus the
// SIMT walker), joined before the chunked P3-tetrahedron kernel (which holds
// all TMEM columns of its SMs) and the CSR sum.
int enqueue(fem_batch* b, cudaStream_t s) {
    int rc;
    const BatchMesh* tab = b->d_meshes.as<BatchMesh>();
    auto sums = [&](auto zero) -> int {
        using T = decltype(zero);
        for (const auto& g : b->sum_ranges) {
            const int r = batch_scatter_launch<T>(b->d_scatter.as<BatchItem>() + g.begin, g.count, tab, g.np,
                                                  g.max_seg, s);
            if (r) return r;
        }
        return FEM_OK;
    };
    if (b->prec == FEM_FP64) {
        if ((rc = batch_simt_launch<double>(b->d_simt.as<BatchItem>(), b->n_simt, tab, b->simt_smem, b->simt_grid, s)))
            return rc;
        return sums(0.0);
    }
    int nb = 0;
    FEM_CUDA_TRY(cudaEventRecord(b->fork, s));
    auto next_branch = [&](cudaStream_t& out) -> int {
        if (nb >= fem_batch::NBRANCH) {
            out = s;
            return FEM_OK;
        }
        out = b->branch[nb];
        FEM_CUDA_TRY(cudaStreamWaitEvent(out, b->fork, 0));
        ++nb;
        return FEM_OK;
    };
    for (const auto& r : b->tc_ranges) {
        cudaStream_t bs;
        if ((rc = next_branch(bs))) return rc;
        if ((rc = batch_tc_launch(b->d_tc.as<BatchItem>() + r.begin, r.count, tab, r.talloc, r.smem, b->tc_grid, bs)))
            return rc;
    }
    if (b->n_simt) {
        cudaStream_t bs;
        if ((rc = next_branch(bs))) return rc;
        if ((rc = batch_simt_launch<float>(b->d_simt.as<BatchItem>(), b->n_simt, tab, b->simt_smem, b->simt_grid, bs)))
            return rc;
    }
    for (int k = 0; k < nb; ++k) {
        FEM_CUDA_TRY(cudaEventRecord(b->join[k], b->branch[k]));
        FEM_CUDA_TRY(cudaStreamWaitEvent(s, b->join[k], 0));
    }
    if (b->n_tc5 && (rc = batch_tc_chunked_launch(b->d_tc5.as<BatchItem>(), b->n_tc5, tab, s))) return rc;
    return sums(0.0f);
}

// One item per run of block/32 groups of contributions (a warp's task):
// pair groups of 64 for FP32 values, steps of 256 for FP64 (the FP64 sum adds
// eight contributions per lane).
int build_scatter_items(fem_batch* b, int block, cudaStream_t s) {
    std::vector<BatchItem> items;
    const int run = std::max(1, block / 32);
    const int64_t unit = b->prec == FEM_FP64 ? 256 : 64;
    b->sum_ranges.clear();
    for (int np : {3, 4, 6, 10, 20}) {   // grouped by n_p, meshes in batch order within a group
        fem_batch::SumRange g{np, (int)items.size(), 0, 0};
        for (int i = 0; i < b->n; ++i) {
            const fem_mesh* m = b->meshes[i];
            if (m->np != np) continue;
            g.max_seg = std::max(g.max_seg, m->max_seg);
            const int64_t ng = (m->E * m->np * m->np + unit - 1) / unit;
            for (int64_t f = 0; f < ng; f += run)
                items.push_back(BatchItem{i, m->type, f, (int)std::min<int64_t>(run, ng - f), 0});
        }
        g.count = (int)items.size() - g.begin;
        if (g.count > 0) b->sum_ranges.push_back(g);
    }
    b->n_scatter = (int)items.size();
    return upload_items(b->d_scatter, items, s);
}

int capture(fem_batch* b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    FEM_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(b, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b->graph = g;
    FEM_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    return FEM_OK;
}

// time a few launch shapes on the real inputs and keep the fastest
int autotune(fem_batch* b, cudaStream_t s) {
    int dev = b->device, nsm = 0;
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks[] = {128, 256, 512};
    const int simt_per_sm[] = {8, 16, 32};
    cudaEvent_t e0, e1;
    FEM_CUDA_TRY(cudaEventCreate(&e0));
    FEM_CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e300;
    int best_block = b->scatter_block, best_simt = b->simt_grid;
    int rc = FEM_OK;
    for (int bl : blocks) {
        if ((rc = build_scatter_items(b, bl, s))) break;
        b->scatter_block = bl;
        for (int sp : simt_per_sm) {
            b->simt_grid = nsm * sp;
            if ((rc = enqueue(b, s))) break;       // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r)
                if ((rc = enqueue(b, s))) break;
            cudaEventRecord(e1, s);
            if (rc) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / 3.0 < best) {
                best = ms / 3.0;
                best_block = bl;
                best_simt = b->simt_grid;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->simt_grid = best_simt;
    b->tuned_ms = best;
    if ((rc = build_scatter_items(b, best_block, s))) return rc;
    b->scatter_block = best_block;
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    return FEM_OK;
}

}  // namespace
}  // namespace fem

using namespace fem;

extern "C" {

int fem_batch_create(fem_mesh* const* meshes, int n, const fem_batch_opts* opts, void* stream, fem_batch** out) {
    if (!meshes || n <= 0 || !out) return fail(FEM_EINVAL, "need at least one mesh");
    *out = nullptr;
    const int prec = opts ? opts->prec : FEM_TF32X3;
    if (prec != FEM_FP64 && prec != FEM_TF32X3 && prec != FEM_FP32)
        return fail(FEM_EINVAL, "batched reassembly runs FEM_TF32X3, FEM_FP32 or FEM_FP64");
    for (int i = 0; i < n; ++i) {
        if (!meshes[i]) return fail(FEM_EINVAL, "NULL mesh in batch");
        if (!meshes[i]->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run on every mesh");
        if (meshes[i]->perq)
            return fail(FEM_EINVAL, "batches take meshes with per-element geometry (no isoparametric mapping or "
                                    "conductivity field)");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if ((rc = tables_init_tc()) || (rc = tables_init_simt())) return rc;
    fem_batch* b = new fem_batch;
    b->n = n;
    b->prec = prec;
    b->use_graph = opts ? opts->use_graph != 0 : true;
    b->tune = opts ? opts->tune != 0 : false;
    b->meshes.assign(meshes, meshes + n);
    cudaGetDevice(&b->device);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    const size_t esz = prec == FEM_FP64 ? 8 : 4;
    std::vector<BatchItem> tc, tc5, simt;
    b->host.resize(n);
    for (int i = 0; i < n; ++i) {
        fem_mesh* m = meshes[i];
        const size_t nsym = (size_t)m->np * (m->np + 1) / 2, nt = (size_t)m->np * m->np;
        if ((rc = buf_alloc(m->VMK, 2 * esz * (size_t)m->E * nsym, s)) ||
            (rc = buf_alloc(m->VT, esz * (size_t)m->E * nt, s))) {
            fem_batch_destroy(b);
            return rc;
        }
        m->v_prec = -1;   // scratch now belongs to the batch's precision
        BatchMesh& h = b->host[i];
        std::memset(&h, 0, sizeof(h));
        h.conn = m->conn.as<int>();
        h.geo32 = m->geo32.as<float>();
        h.geo64 = m->geo64.as<double>();
        h.gram64 = m->gram64.as<double>();
        h.E = m->E;
        h.n = m->n;
        h.nnz = m->nnz;
        h.np = m->np;
        h.type = m->type;
        h.mass = m->m;
        h.VM = m->VMK.ptr;
        h.VK = static_cast<unsigned char*>(m->VMK.ptr) + esz;   // K: the odd positions
        h.VT = m->VT.ptr;
        h.seg_ptr = m->seg_ptr.as<int>();
        h.contrib = m->contrib.as<int>();
        h.seg_head = m->seg_head.as<uint2>();
        h.max_seg = m->max_seg;
        const bool on_tc = prec == FEM_TF32X3 && tc_type_supported(m->type);
        const bool on_tc5 = prec == FEM_TF32X3 && !on_tc && tc_chunked_supported(m->type);
        if (on_tc5) {
            for (int64_t f = 0; f < m->E; f += 128) tc5.push_back(BatchItem{i, m->type, f, 128, 0});
        } else if (on_tc) {
            for (int64_t f = 0; f < m->E; f += 128) tc.push_back(BatchItem{i, m->type, f, 128, 0});
        } else {
            for (int64_t f = 0; f < m->E; f += 64) simt.push_back(BatchItem{i, m->type, f, 64, 0});
            b->simt_smem = std::max(b->simt_smem, batch_simt_smem(m->type, prec == FEM_FP64));
        }
    }
    // tensor-core tiles grouped by element type: one launch per type
    std::stable_sort(tc.begin(), tc.end(), [](const BatchItem& a, const BatchItem& c) { return a.type < c.type; });
    for (int i0 = 0; i0 < (int)tc.size();) {
        int i1 = i0;
        while (i1 < (int)tc.size() && tc[i1].type == tc[i0].type) ++i1;
        const int t = tc[i0].type;
        b->tc_ranges.push_back({t, i0, i1 - i0, tc_type_alloc(t), tc_type_smem(t)});
        i0 = i1;
    }
    b->n_tc = (int)tc.size();
    b->n_tc5 = (int)tc5.size();
    b->n_simt = (int)simt.size();
    b->tc_grid = nsm;
    b->simt_grid = nsm * 16;
    if (b->simt_smem == 0) b->simt_smem = 16;
    if ((rc = upload_items(b->d_tc, tc, s)) || (rc = upload_items(b->d_tc5, tc5, s)) ||
        (rc = upload_items(b->d_simt, simt, s)) ||
        (rc = build_scatter_items(b, b->scatter_block, s)) ||
        (rc = buf_alloc(b->d_meshes, sizeof(BatchMesh) * n, s))) {
        fem_batch_destroy(b);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMallocHost((void**)&b->pinned[k], sizeof(BatchMesh) * n);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int k = 0; k < fem_batch::NBRANCH && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        fem_batch_destroy(b);
        return cuda_fail(e, "batch set-up");
    }
    if (b->use_graph && !b->tune && (rc = capture(b))) {
        fem_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FEM_OK;
}

int fem_batch_launch(fem_batch* b, const fem_coeff* k, const double* const* d_u, void* const* d_vM,
                     void* const* d_vK, void* const* d_vT, void* stream) {
    if (!b) return fail(FEM_EINVAL, "NULL batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // per-launch table: static fields + this launch's u, laws and outputs
    BatchMesh* st = b->pinned[b->cur];
    FEM_CUDA_TRY(cudaEventSynchronize(b->staged[b->cur]));   // the previous copy out of this buffer is done
    const size_t esz = b->prec == FEM_FP64 ? 8 : 4;
    for (int i = 0; i < b->n; ++i) {
        // scratch pointers are taken from the mesh at every launch: a
        // single-mesh call in between may have reallocated them
        fem_mesh* m = b->meshes[i];
        const size_t nsym = (size_t)m->np * (m->np + 1) / 2, nt = (size_t)m->np * m->np;
        int rc0;
        if ((rc0 = buf_alloc(m->VMK, 2 * esz * (size_t)m->E * nsym, s)) ||
            (rc0 = buf_alloc(m->VT, esz * (size_t)m->E * nt, s)))
            return rc0;
        m->v_prec = -1;
        BatchMesh h = b->host[i];
        h.VM = m->VMK.ptr;
        h.VK = static_cast<unsigned char*>(m->VMK.ptr) + esz;   // K: the odd positions
        h.VT = m->VT.ptr;
        h.vM = d_vM ? d_vM[i] : nullptr;
        h.vK = d_vK ? d_vK[i] : nullptr;
        h.vT = d_vT ? d_vT[i] : nullptr;
        if (h.vK || h.vT) {
            if (!k) return fail(FEM_EINVAL, "coefficient laws are NULL");
            int rc = validate_coeff(&k[i]);
            if (rc) return rc;
            if (!d_u || !d_u[i]) return fail(FEM_EINVAL, "u is NULL for a mesh that needs it");
            h.u = d_u[i];
            h.k = coeff_to_device(&k[i]);
        } else {
            h.u = nullptr;
        }
        st[i] = h;
    }
    FEM_CUDA_TRY(cudaMemcpyAsync(b->d_meshes.ptr, st, sizeof(BatchMesh) * b->n, cudaMemcpyHostToDevice, s));
    FEM_CUDA_TRY(cudaEventRecord(b->staged[b->cur], s));
    b->cur ^= 1;
    int rc;
    if (b->tune && !b->tuned) {
        if ((rc = autotune(b, s))) return rc;
        b->tuned = true;
        if (b->use_graph && (rc = capture(b))) return rc;
    }
    if (b->use_graph && b->exec) {
        FEM_CUDA_TRY(cudaGraphLaunch(b->exec, s));
        return FEM_OK;
    }
    return enqueue(b, s);
}

int fem_batch_get_info(const fem_batch* b, fem_batch_info* out) {
    if (!b || !out) return fail(FEM_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_meshes = b->n;
    out->kernels_per_launch =
        (int)b->tc_ranges.size() + (b->n_tc5 ? 1 : 0) + (b->n_simt ? 1 : 0) + (int)b->sum_ranges.size();
    out->tc_tiles = b->n_tc + b->n_tc5;
    out->simt_blocks = b->n_simt;
    out->sum_chunks = b->n_scatter;
    out->sum_block = b->scatter_block;
    out->simt_grid = b->simt_grid;
    out->tuned = b->tuned ? 1 : 0;
    out->tuned_ms = b->tuned_ms;
    out->graph = b->exec != nullptr ? 1 : 0;
    return FEM_OK;
}

int fem_batch_destroy(fem_batch* b) {
    if (!b) return FEM_OK;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int k = 0; k < fem_batch::NBRANCH; ++k) {
        if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    for (int k = 0; k < 2; ++k) {
        if (b->pinned[k]) cudaFreeHost(b->pinned[k]);
        if (b->staged[k]) cudaEventDestroy(b->staged[k]);
    }
    DevBuf* bufs[] = {&b->d_meshes, &b->d_tc, &b->d_tc5, &b->d_simt, &b->d_scatter};
    for (auto* x : bufs) buf_free(*x, nullptr);
    cudaDeviceSynchronize();
    delete b;
    return FEM_OK;
}

}  // extern "C"
