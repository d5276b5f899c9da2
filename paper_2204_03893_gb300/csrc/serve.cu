// serve.cu -- a request server for assembly / reassembly with continuous
// batching.
//
// The paper's motivation is that repeated reassembly inside nonlinear
// solvers is a bottleneck (Introduction), and that only S (the coefficient
// evaluations) changes between Newton steps while Q, w, W and b stay fixed
// (Section 5).  A server keeps, per mesh, everything that does not change
// resident on the device (geometry, CSR pattern, slot segments, element
// scratch) and turns each request into one element-product launch and one
// CSR-sum launch.
//
// Threading: submit/poll/release run on caller threads; one scheduler thread
// owns all device work.  It admits queued requests in arrival order while a
// slot is free (max_inflight) and the device-memory budget allows (resident
// meshes + outputs of requests not yet released), skipping a request only to
// keep the requests of one mesh in order (a mesh's scratch is reused, so its
// requests never overlap).  Admitted requests are spread over several CUDA
// streams, so work of different meshes overlaps on the device; completion is
// detected with CUDA events.  A request that can never fit the budget is
// refused at submit (FEM_EBUSY).
//
// Fused launches: when at least fuse_min REASSEMBLE requests of idle meshes
// are startable, they start together as one launch of a batch over all
// resident meshes (the meshes without a request skipped), on a stream of
// their own, instead of one element launch and one CSR-sum launch each.  The
// batch is rebuilt when the set of resident meshes has changed; a mesh the
// batch still references is destroyed only after the batch is (the
// scheduler then waits for the device).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <set>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fem_internal.h"

namespace fem {
int validate_coeff(const fem_coeff* k);
CoeffDev coeff_to_device(const fem_coeff* k);
}  // namespace fem

namespace {

using fem::buf_alloc;
using fem::buf_free;
using fem::cuda_fail;
using fem::fail;
using fem::set_error;
using Clock = std::chrono::steady_clock;

enum State { PENDING = 0, RUNNING = 1, DONE = 2 };

struct Resident {
    fem_mesh* mesh = nullptr;
    fem::DevBuf u;            // FP64 nodal values of the current request
    int busy = 0;             // a request of this mesh is in flight
    bool evicted = false;     // fem_serve_evict was called; destroyed once idle
    size_t bytes = 0;         // device bytes accounted for the mesh
    // pending requests of the mesh: the oldest is in the server's ready set
    // while the mesh is idle, the others wait here in submission order
    bool in_ready = false;
    uint64_t ready_ticket = 0;
    std::deque<uint64_t> waiting;
};

struct Request {
    uint64_t ticket = 0;
    int kind = 0, which = 7, status = FEM_OK;
    uint64_t mesh_id = 0;
    fem_coeff k;
    std::vector<double> u;                 // host copy of the nodal values (pageable fallback)
    double* u_pin = nullptr;               // ... or in a pinned block of the server's pool
    size_t u_cls = 0, u_n = 0;
    const double* u_data() const { return u_pin ? u_pin : u.data(); }
    // ASSEMBLE: host copies of the mesh description
    fem_mesh_desc desc;
    std::vector<double> coords;
    std::vector<int32_t> conn;
    size_t est_bytes = 0;                  // admission estimate (outputs + mesh if new)
    size_t out_bytes = 0;
    fem::DevBuf out[3];
    cudaEvent_t done = nullptr;
    int stream = 0;
    State state = PENDING;
    std::string msg;                       // error message of a failed request
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t group = 0;                     // fused launch the request started in (0: alone)
};

// Pinned host blocks for the nodal values of queued requests, so that the
// scheduler's upload is an asynchronous DMA and the host copy happens on the
// submitting thread.  Blocks come in power-of-two size classes and are
// reused; past `cap` bytes held, requests keep a pageable copy instead.
struct PinnedPool {
    std::mutex mu;
    std::map<size_t, std::vector<void*>> free;
    size_t held = 0, cap = size_t(1) << 30;
    void* get(size_t bytes, size_t& cls) {
        cls = 4096;
        while (cls < bytes) cls <<= 1;
        std::lock_guard<std::mutex> lk(mu);
        auto it = free.find(cls);
        if (it != free.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            return p;
        }
        if (held + cls > cap) return nullptr;
        void* p = nullptr;
        if (cudaHostAlloc(&p, cls, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        held += cls;
        return p;
    }
    void put(void* p, size_t cls) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        free[cls].push_back(p);
    }
    void clear() {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& kv : free)
            for (void* p : kv.second) cudaFreeHost(p);
        free.clear();
        held = 0;
    }
};

}  // namespace

struct fem_server {
    fem_serve_opts opts;
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread th;
    uint64_t next_ticket = 1, next_mesh = 1;
    std::set<uint64_t> ready;                                    // startable tickets, arrival order
    size_t pending = 0;                                          // submitted, not started
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::map<uint64_t, Resident> meshes;
    std::vector<cudaStream_t> streams;
    std::vector<uint64_t> running;                               // tickets in flight
    int rr = 0, inflight = 0;
    size_t in_use = 0;                                           // accounted device bytes
    size_t peak = 0;
    PinnedPool pinned;
    // fused launches: a batch over the resident meshes (mesh id -> index)
    fem_batch* batch = nullptr;
    bool batch_stale = true, building = false, fuse_off = false;
    bool hold = false;   // a batch build waits for the device to drain: start nothing new
    // fused launches in flight (at most FUSED_MAX: the batch stages its
    // per-launch tables in two pinned buffers, and a third launch would make
    // the scheduler wait for the first)
    std::set<int64_t> groups;
    int64_t next_group = 1;
    std::deque<uint64_t> done_order;   // finished tickets not yet returned by fem_serve_next_done
    std::map<uint64_t, int> batch_index;
    int batch_n = 0;
    cudaStream_t bstream = nullptr;
    // evicted meshes the batch may still reference, destroyed with it
    std::vector<std::pair<fem_mesh*, fem::DevBuf>> graveyard;
    int64_t n_single = 0, n_fused = 0, n_fused_req = 0, n_builds = 0;
    double host_start_us = 0;
};

namespace {

constexpr int FUSED_MAX = 2;

bool fusing(const fem_server* S);

double now_us(const fem_server* s) {
    return std::chrono::duration<double, std::micro>(Clock::now() - s->t0).count();
}

size_t esz_of(int prec) { return prec == FEM_FP64 ? 8 : 4; }

size_t nlocal(int d, int p) { return d == 2 ? (size_t)(p + 1) * (p + 2) / 2 : (size_t)(p + 1) * (p + 2) * (p + 3) / 6; }

// upper bound of the device bytes a new mesh will hold (coords, conn, two
// geometry caches, pattern, segments, slot map, offsets, scratch, u)
size_t mesh_estimate(const fem_mesh_desc& d, int prec) {
    const size_t np = nlocal(d.dim, d.order), E = (size_t)d.n_elems, n = (size_t)d.n_nodes;
    const size_t m2 = E * np * np, ngeo = 1 + (size_t)d.dim * (d.dim + 1) / 2;
    size_t b = n * d.dim * 8 + E * np * 4 + ngeo * E * 12;
    b += (n + 1) * 4 * 5;                 // row_ptr, inc_ptr and three transient counters of the sort
    b += m2 * 4 * 4 + E * np * 4;         // col_idx and seg_ptr (nnz <= m2), contrib, slot, inc
    b += (m2 / 32 + 2) * 8;               // segment heads per group of 32 contributions
    b += esz_of(prec) * E * (np * (np + 1) + np * np) + n * 8;   // V scratch, u
    if (np == (size_t)d.dim + 1) b += E * np * (np + 1) / 2 * 8;   // P1: the elements' Gram matrices
    return b + 4096;                      // rounding of small buffers
}

// Precision a mesh is reassembled in (the server's, for every element type).
int mesh_prec(int prec, const fem_mesh*) { return prec; }

// Runs on the scheduler thread with the lock released.  For ASSEMBLE the new
// mesh is returned in *created (the caller publishes it under the lock).
int start_request(fem_server* S, Request& r, Resident* res, fem_mesh** created, cudaStream_t st) {
    int rc;
    fem_mesh* m = res->mesh;
    if (r.kind == FEM_REQ_ASSEMBLE) {
        fem_mesh_desc d = r.desc;
        d.coords = r.coords.data();
        d.conn = r.conn.data();
        d.mem = FEM_MEM_HOST;
        if ((rc = fem_mesh_create(&d, st, &m))) return rc;
        *created = m;
        if ((rc = fem_symbolic(m, st, nullptr))) return rc;
    }
    const int prec = mesh_prec(S->opts.prec, m);
    const size_t esz = esz_of(prec);
    for (int i = 0; i < 3; ++i)
        if (r.which & (1 << i))
            if ((rc = buf_alloc(r.out[i], esz * (size_t)(m->nnz > 0 ? m->nnz : 1), st))) return rc;
    const double* du = nullptr;
    if (r.which & 6) {
        if (r.u_n != (size_t)m->n) return fail(FEM_EINVAL, "u has the wrong length for this mesh");
        if ((rc = buf_alloc(res->u, sizeof(double) * (size_t)m->n, st))) return rc;
        cudaError_t e = cudaMemcpyAsync(res->u.ptr, r.u_data(), sizeof(double) * r.u_n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "upload u");
        du = res->u.as<double>();
    }
    if ((rc = fem_form_elements(m, &r.k, du, prec, r.which, st))) return rc;
    if ((rc = fem_sum_elements(m, prec, r.out[0].ptr, r.out[1].ptr, r.out[2].ptr, st))) return rc;
    cudaError_t e = cudaEventRecord(r.done, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    return FEM_OK;
}

// The request's inputs are no longer needed (its upload has completed or
// never started): the pinned block goes back to the pool.
void drop_inputs(fem_server* S, Request& r) {
    if (r.u_pin) S->pinned.put(r.u_pin, r.u_cls);
    r.u_pin = nullptr;
    std::vector<double>().swap(r.u);
}

void finish(fem_server* S, Request& r, int status, const std::string& msg) {
    drop_inputs(S, r);
    r.status = status;
    r.msg = msg;
    r.state = DONE;
    r.t_done = now_us(S);
    S->done_order.push_back(r.ticket);
}

// Puts a request of an idle mesh (or an ASSEMBLE) into the ready set, or
// queues it behind the mesh's pending requests.  Lock held.
void enqueue_request(fem_server* S, Request& r) {
    if (r.kind == FEM_REQ_REASSEMBLE) {
        Resident& res = S->meshes[r.mesh_id];
        if (res.busy || res.in_ready) {
            res.waiting.push_back(r.ticket);
            return;
        }
        res.in_ready = true;
        res.ready_ticket = r.ticket;
    }
    S->ready.insert(r.ticket);
}

// The mesh has no request in flight any more: its next pending request (if
// any) becomes startable.  Lock held.
void mesh_idle(fem_server* S, Resident& res) {
    res.busy = 0;
    if (!res.in_ready && !res.waiting.empty()) {
        const uint64_t t = res.waiting.front();
        res.waiting.pop_front();
        res.in_ready = true;
        res.ready_ticket = t;
        S->ready.insert(t);
    }
}

// Moves finished requests to DONE.  Lock held.
bool reap(fem_server* S) {
    bool progress = false;
    for (size_t i = 0; i < S->running.size();) {
        Request& r = *S->reqs[S->running[i]];
        cudaError_t q = cudaEventQuery(r.done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q == cudaSuccess) finish(S, r, FEM_OK, "");
        else finish(S, r, FEM_ECUDA, std::string("request failed on the device: ") + cudaGetErrorString(q));
        if (r.group) S->groups.erase(r.group);   // the group's events complete together
        --S->inflight;
        Resident& res = S->meshes[r.mesh_id];
        mesh_idle(S, res);
        // account the mesh at its real size once it exists
        const size_t real = res.mesh ? res.mesh->device_bytes() : 0;
        if (real && real != res.bytes) {
            S->in_use = S->in_use - res.bytes + real;
            res.bytes = real;
        }
        S->running[i] = S->running.back();
        S->running.pop_back();
        progress = true;
    }
    return progress;
}

// Admits the oldest startable request if it can start now (requests of a
// mesh that is busy are not startable; when the oldest startable request does
// not fit the budget, nothing behind it is admitted).  Starts it with the lock
// released.  Returns false if nothing could be admitted.
bool admit_one(fem_server* S, std::unique_lock<std::mutex>& lk) {
    if (S->hold || S->inflight >= S->opts.max_inflight || S->ready.empty()) return false;
    const uint64_t ticket = *S->ready.begin();
    Request& r = *S->reqs[ticket];
    // while fused launches fill their slots, reassembly requests wait for the
    // next one instead of starting alone beside them
    if (r.kind == FEM_REQ_REASSEMBLE && fusing(S) && (int)S->groups.size() >= FUSED_MAX) return false;
    Resident* res = nullptr;
    if (r.kind == FEM_REQ_REASSEMBLE) {
        auto m = S->meshes.find(r.mesh_id);
        if (m == S->meshes.end() || m->second.evicted) {
            S->ready.erase(S->ready.begin());
            --S->pending;
            finish(S, r, FEM_EINVAL, "mesh was evicted before the request started");
            return true;
        }
        res = &m->second;
    }
    if (S->in_use + r.est_bytes > S->opts.budget_bytes) return false;
    S->ready.erase(S->ready.begin());
    --S->pending;
    if (r.kind == FEM_REQ_ASSEMBLE) {
        r.mesh_id = S->next_mesh++;
        res = &S->meshes[r.mesh_id];
        res->bytes = r.est_bytes - r.out_bytes;
    } else {
        res->in_ready = false;
    }
    res->busy = 1;
    S->in_use += r.est_bytes;
    S->peak = std::max(S->peak, S->in_use);
    r.state = RUNNING;
    r.t_start = now_us(S);
    r.stream = S->rr;
    S->rr = (S->rr + 1) % (int)S->streams.size();
    ++S->inflight;
    cudaStream_t st = S->streams[r.stream];
    fem_mesh* created = nullptr;
    lk.unlock();
    const double t0 = now_us(S);
    int rc = start_request(S, r, res, &created, st);
    const double t1 = now_us(S);
    std::string msg;
    if (rc) {
        char buf[512];
        fem_last_error(buf, sizeof buf);
        msg = buf;
        cudaStreamSynchronize(st);    // nothing of the failed request stays in flight
        if (created && r.kind == FEM_REQ_ASSEMBLE) {
            fem_mesh_destroy(created);
            created = nullptr;
        }
    }
    lk.lock();
    S->host_start_us += t1 - t0;
    ++S->n_single;
    if (created) {
        res->mesh = created;
        S->batch_stale = true;   // the resident set changed
    }
    if (rc) {
        finish(S, r, rc, msg);
        --S->inflight;
        // the outputs stay accounted until release; a mesh that was not created is dropped
        S->in_use -= r.est_bytes - r.out_bytes;
        if (r.kind == FEM_REQ_ASSEMBLE) S->meshes.erase(r.mesh_id);
        else mesh_idle(S, *res);
    } else {
        S->running.push_back(r.ticket);
    }
    return true;
}

bool fusable_prec(int prec) { return prec == FEM_FP64 || prec == FEM_TF32X3 || prec == FEM_FP32; }

bool fusing(const fem_server* S) { return S->opts.fuse_min > 0 && !S->fuse_off && fusable_prec(S->opts.prec); }

// Enqueues one fused launch for the requests `rs` of the meshes `res` (lock
// released): outputs and u uploads on the batch stream, the batch launch with
// the other meshes skipped, then each request's completion event.
int start_fused(fem_server* S, fem_batch* b, int n, const std::map<uint64_t, int>& index,
                const std::vector<Request*>& rs, const std::vector<Resident*>& res) {
    cudaStream_t st = S->bstream;
    const size_t esz = esz_of(S->opts.prec);
    std::vector<fem_coeff> k((size_t)n);
    std::memset(k.data(), 0, sizeof(fem_coeff) * k.size());
    std::vector<const double*> du((size_t)n, nullptr);
    std::vector<void*> vM((size_t)n, nullptr), vK((size_t)n, nullptr), vT((size_t)n, nullptr);
    int rc;
    for (size_t j = 0; j < rs.size(); ++j) {
        Request& r = *rs[j];
        Resident& re = *res[j];
        fem_mesh* m = re.mesh;
        auto it = index.find(r.mesh_id);
        if (it == index.end()) return fail(FEM_ESTATE, "mesh is not in the fused batch");
        const int i = it->second;
        for (int c = 0; c < 3; ++c)
            if (r.which & (1 << c))
                if ((rc = buf_alloc(r.out[c], esz * (size_t)(m->nnz > 0 ? m->nnz : 1), st))) return rc;
        if (r.which & 6) {
            if (r.u_n != (size_t)m->n) return fail(FEM_EINVAL, "u has the wrong length for this mesh");
            if ((rc = buf_alloc(re.u, sizeof(double) * (size_t)m->n, st))) return rc;
            cudaError_t e = cudaMemcpyAsync(re.u.ptr, r.u_data(), sizeof(double) * r.u_n, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "upload u");
            du[i] = re.u.as<double>();
            k[i] = r.k;
        }
        vM[i] = r.out[0].ptr;
        vK[i] = r.out[1].ptr;
        vT[i] = r.out[2].ptr;
    }
    if ((rc = fem_batch_launch(b, k.data(), du.data(), vM.data(), vK.data(), vT.data(), st))) return rc;
    for (Request* r : rs) {
        cudaError_t e = cudaEventRecord(r->done, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    return FEM_OK;
}

// Destroys the batch and the evicted meshes it may reference (waits for the
// device).  Lock held on entry and exit, released meanwhile.
void bury(fem_server* S, std::unique_lock<std::mutex>& lk) {
    fem_batch* old = S->batch;
    S->batch = nullptr;
    S->batch_index.clear();
    S->batch_n = 0;
    S->batch_stale = true;
    std::vector<std::pair<fem_mesh*, fem::DevBuf>> dead;
    dead.swap(S->graveyard);
    S->building = true;
    lk.unlock();
    const double t0 = now_us(S);
    if (old) fem_batch_destroy(old);
    for (auto& d : dead) {
        buf_free(d.second, nullptr);
        fem_mesh_destroy(d.first);
    }
    const double t1 = now_us(S);
    lk.lock();
    S->building = false;
    S->host_start_us += t1 - t0;
}

// Starts the startable REASSEMBLE requests (oldest first, within the
// in-flight and budget limits) as one fused launch if there are at least
// fuse_min of them, (re)building the batch first if the resident set
// changed.  Returns false if nothing was done.  Lock held on entry and exit.
bool admit_fused(fem_server* S, std::unique_lock<std::mutex>& lk) {
    if (!fusing(S) || (int)S->groups.size() >= FUSED_MAX) return false;
    std::vector<uint64_t> cand;
    size_t bytes = 0;
    for (uint64_t t : S->ready) {
        if (S->inflight + (int)cand.size() >= S->opts.max_inflight) break;
        Request& r = *S->reqs[t];
        if (r.kind != FEM_REQ_REASSEMBLE) continue;
        auto m = S->meshes.find(r.mesh_id);
        if (m == S->meshes.end() || m->second.evicted || !m->second.mesh) continue;
        if (S->in_use + bytes + r.est_bytes > S->opts.budget_bytes) break;
        bytes += r.est_bytes;
        cand.push_back(t);
    }
    if ((int)cand.size() < S->opts.fuse_min) {
        S->hold = false;
        return false;
    }
    if (S->batch_stale || !S->batch) {
        // building allocates the meshes' element scratch where it is missing,
        // which must not happen under a kernel of another stream: let the
        // device drain first (nothing new starts meanwhile)
        if (S->inflight > 0) {
            S->hold = true;
            return false;
        }
        S->hold = false;
        bury(S, lk);
        std::vector<uint64_t> ids;
        std::vector<fem_mesh*> ms;
        for (auto& kv : S->meshes)
            if (kv.second.mesh && !kv.second.evicted) {
                ids.push_back(kv.first);
                ms.push_back(kv.second.mesh);
            }
        S->building = true;   // eviction now leaves these meshes to the scheduler
        lk.unlock();
        const double t0 = now_us(S);
        fem_batch_opts bo;
        std::memset(&bo, 0, sizeof bo);
        bo.prec = S->opts.prec;
        // no graph: capturing one would make device-wide synchronisation by
        // the caller's threads fail meanwhile; a fused launch enqueues its few
        // kernels directly
        bo.use_graph = 0;
        fem_batch* nb = nullptr;
        const int rc = fem_batch_create(ms.data(), (int)ms.size(), &bo, S->bstream, &nb);
        const double t1 = now_us(S);
        lk.lock();
        S->building = false;
        S->host_start_us += t1 - t0;
        ++S->n_builds;
        if (rc) {
            S->fuse_off = true;   // requests start one by one from now on
            return true;
        }
        S->batch = nb;
        S->batch_n = (int)ids.size();
        for (size_t i = 0; i < ids.size(); ++i) S->batch_index[ids[i]] = (int)i;
        S->batch_stale = false;
        return true;   // the ready set may have changed meanwhile: collect again
    }
    std::vector<Request*> rs;
    std::vector<Resident*> res;
    const double now = now_us(S);
    const int64_t group = S->next_group++;
    S->groups.insert(group);
    for (uint64_t t : cand) {
        Request& r = *S->reqs[t];
        Resident& re = S->meshes[r.mesh_id];
        S->ready.erase(t);
        --S->pending;
        re.in_ready = false;
        re.busy = 1;
        S->in_use += r.est_bytes;
        r.state = RUNNING;
        r.t_start = now;
        r.stream = -1;
        r.group = group;
        ++S->inflight;
        rs.push_back(&r);
        res.push_back(&re);
    }
    S->peak = std::max(S->peak, S->in_use);
    fem_batch* b = S->batch;
    const int n = S->batch_n;
    const std::map<uint64_t, int> index = S->batch_index;
    lk.unlock();
    const double t0 = now_us(S);
    int rc = start_fused(S, b, n, index, rs, res);
    std::string msg;
    if (rc) {
        char buf[512];
        fem_last_error(buf, sizeof buf);
        msg = buf;
        cudaStreamSynchronize(S->bstream);   // nothing of the failed launch stays in flight
    }
    const double t1 = now_us(S);
    lk.lock();
    S->host_start_us += t1 - t0;
    ++S->n_fused;
    S->n_fused_req += (int64_t)rs.size();
    if (rc) S->groups.erase(group);
    for (size_t j = 0; j < rs.size(); ++j) {
        if (rc) {
            finish(S, *rs[j], rc, msg);
            --S->inflight;
            mesh_idle(S, *res[j]);
        } else {
            S->running.push_back(rs[j]->ticket);
        }
    }
    return true;
}

void scheduler(fem_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progress = reap(S);
        if (!S->graveyard.empty()) {
            bury(S, lk);
            progress = true;
        }
        // a fused launch is tried before every single start, so that requests
        // that queued up while the scheduler was busy start together
        while (!S->stop) {
            if (admit_fused(S, lk) || admit_one(S, lk)) progress = true;
            else break;
        }
        if (progress) S->cv_done.notify_all();
        else S->cv_work.wait_for(lk, std::chrono::microseconds(S->inflight ? 10 : 1000));
    }
}

}  // namespace

using namespace fem;

extern "C" {

int fem_serve_create(const fem_serve_opts* opts, fem_server** out) {
    if (!opts || !out) return fail(FEM_EINVAL, "NULL argument");
    *out = nullptr;
    if (opts->prec < FEM_FP64 || opts->prec > FEM_BF16X6)
        return fail(FEM_EINVAL, "unknown precision");
    if (opts->max_inflight < 1 || opts->n_streams < 1 || opts->n_streams > 64 || opts->budget_bytes == 0)
        return fail(FEM_EINVAL, "need max_inflight >= 1, 1 <= n_streams <= 64 and a nonzero budget");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    fem_server* S = new fem_server;
    S->opts = *opts;
    S->device = dev;
    S->t0 = Clock::now();
    for (int i = 0; i < opts->n_streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto x : S->streams) cudaStreamDestroy(x);
            delete S;
            return cuda_fail(e, "cudaStreamCreate");
        }
        S->streams.push_back(st);
    }
    e = cudaStreamCreateWithFlags(&S->bstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (auto x : S->streams) cudaStreamDestroy(x);
        delete S;
        return cuda_fail(e, "cudaStreamCreate");
    }
    {
        // request outputs and uploads come from the device's default memory
        // pool; keep up to the budget mapped in it, so that the memory of
        // released requests serves the next ones instead of being returned
        // to the driver at every synchronisation and mapped again
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = 0, want = (uint64_t)opts->budget_bytes;
            if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess && keep < want)
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
        }
        cudaGetLastError();
    }
    S->th = std::thread(scheduler, S);
    *out = S;
    return FEM_OK;
}

int fem_serve_submit(fem_server* S, const fem_request* q, uint64_t* ticket) {
    if (!S || !q || !ticket) return fail(FEM_EINVAL, "NULL argument");
    const double t_in = now_us(S);   // latency includes the copy of the inputs
    if (q->kind != FEM_REQ_ASSEMBLE && q->kind != FEM_REQ_REASSEMBLE) return fail(FEM_EINVAL, "unknown request kind");
    if (q->which <= 0 || q->which > 7) return fail(FEM_EINVAL, "which must be a nonzero mask of FEM_MAT_M|K|T");
    if (q->which & 6) {
        if (!q->k) return fail(FEM_EINVAL, "K or T requested without a coefficient law");
        int rc = validate_coeff(q->k);
        if (rc) return rc;
        if (!q->u) return fail(FEM_EINVAL, "K or T requested without u");
    }
    auto r = std::make_unique<Request>();
    r->kind = q->kind;
    r->which = q->which;
    if (q->k) r->k = *q->k;
    else std::memset(&r->k, 0, sizeof r->k);
    size_t n = 0, nnz_bound = 0;
    int prec = S->opts.prec;
    if (q->kind == FEM_REQ_ASSEMBLE) {
        if (!q->desc) return fail(FEM_EINVAL, "ASSEMBLE needs a mesh description");
        const fem_mesh_desc& d = *q->desc;
        if ((d.dim != 2 && d.dim != 3) || d.order < 1 || d.order > 3 || d.n_nodes <= 0 || d.n_elems < 0 ||
            !d.coords || (d.n_elems > 0 && !d.conn) || (d.mem != FEM_MEM_HOST && d.mem != FEM_MEM_DEVICE))
            return fail(FEM_EINVAL, "bad mesh description");
        const size_t np = nlocal(d.dim, d.order);
        r->desc = d;
        r->coords.resize((size_t)d.n_nodes * d.dim);
        r->conn.resize((size_t)d.n_elems * np);
        if (d.mem == FEM_MEM_DEVICE) {
            cudaError_t e = cudaMemcpy(r->coords.data(), d.coords, sizeof(double) * r->coords.size(), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && !r->conn.empty())
                e = cudaMemcpy(r->conn.data(), d.conn, sizeof(int32_t) * r->conn.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "copy mesh description");
        } else {
            std::memcpy(r->coords.data(), d.coords, sizeof(double) * r->coords.size());
            if (!r->conn.empty()) std::memcpy(r->conn.data(), d.conn, sizeof(int32_t) * r->conn.size());
        }
        n = (size_t)d.n_nodes;
        nnz_bound = std::min((size_t)d.n_elems * np * np, n * n);
        r->est_bytes = mesh_estimate(d, prec);
    } else {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->meshes.find(q->mesh_id);
        if (it == S->meshes.end() || !it->second.mesh || it->second.evicted)
            return fail(FEM_EINVAL, "unknown, evicted or not yet assembled mesh id");
        n = (size_t)it->second.mesh->n;
        nnz_bound = (size_t)it->second.mesh->nnz;
        r->mesh_id = q->mesh_id;
    }
    int nout = 0;
    for (int i = 0; i < 3; ++i) nout += (q->which >> i) & 1;
    r->out_bytes = esz_of(prec) * std::max<size_t>(nnz_bound, 1) * nout;
    r->est_bytes += r->out_bytes;
    if (r->est_bytes > S->opts.budget_bytes)
        return fail(FEM_EBUSY, "request needs " + std::to_string(r->est_bytes) + " device bytes, the budget is " +
                                   std::to_string(S->opts.budget_bytes));
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    r->done = ev;
    if (q->which & 6) {
        r->u_n = n;
        r->u_pin = static_cast<double*>(S->pinned.get(sizeof(double) * n, r->u_cls));
        if (r->u_pin) std::memcpy(r->u_pin, q->u, sizeof(double) * n);
        else r->u.assign(q->u, q->u + n);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->pending >= (size_t)std::max(S->opts.max_queue, 1)) {
        cudaEventDestroy(ev);
        drop_inputs(S, *r);
        return fail(FEM_EBUSY, "queue full (" + std::to_string(S->pending) + " pending requests)");
    }
    if (r->kind == FEM_REQ_REASSEMBLE) {
        auto it = S->meshes.find(r->mesh_id);
        if (it == S->meshes.end() || !it->second.mesh || it->second.evicted) {
            cudaEventDestroy(ev);
            drop_inputs(S, *r);
            return fail(FEM_EINVAL, "unknown, evicted or not yet assembled mesh id");
        }
    }
    r->ticket = S->next_ticket++;
    r->t_submit = t_in;
    *ticket = r->ticket;
    Request& rr = *r;
    S->reqs[r->ticket] = std::move(r);
    ++S->pending;
    enqueue_request(S, rr);
    S->cv_work.notify_one();
    return FEM_OK;
}

int fem_serve_poll(fem_server* S, uint64_t ticket, int timeout_us, fem_result* out) {
    if (!S || !out) return fail(FEM_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(FEM_EINVAL, "unknown ticket");
    Request& r = *it->second;
    if (r.state != DONE && timeout_us > 0) {
        const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us);
        while (r.state != DONE)
            if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
    }
    if (r.state != DONE) {
        if (timeout_us <= 0) return FEM_EAGAIN;
        return fail(FEM_ETIMEOUT, "request not finished within the timeout");
    }
    std::memset(out, 0, sizeof(*out));
    out->status = r.status;
    out->mesh_id = r.mesh_id;
    auto m = S->meshes.find(r.mesh_id);
    if (r.status == FEM_OK && m != S->meshes.end() && m->second.mesh) {
        const fem_mesh* mesh = m->second.mesh;
        out->n = mesh->n;
        out->nnz = mesh->nnz;
        out->prec = mesh_prec(S->opts.prec, mesh);
        out->d_row_ptr = mesh->row_ptr.as<int32_t>();
        out->d_col_idx = mesh->col_idx.as<int32_t>();
        out->d_vM = r.out[0].ptr;
        out->d_vK = r.out[1].ptr;
        out->d_vT = r.out[2].ptr;
    }
    out->t_submit_us = r.t_submit;
    out->t_start_us = r.t_start;
    out->t_done_us = r.t_done;
    if (r.status != FEM_OK) set_error(r.msg);
    return FEM_OK;
}

int fem_serve_next_done(fem_server* S, int timeout_us, uint64_t* ticket) {
    if (!S || !ticket) return fail(FEM_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
    for (;;) {
        // skip tickets released meanwhile
        while (!S->done_order.empty() && !S->reqs.count(S->done_order.front())) S->done_order.pop_front();
        if (!S->done_order.empty()) {
            *ticket = S->done_order.front();
            S->done_order.pop_front();
            return FEM_OK;
        }
        if (timeout_us <= 0) return FEM_EAGAIN;
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            while (!S->done_order.empty() && !S->reqs.count(S->done_order.front())) S->done_order.pop_front();
            if (S->done_order.empty()) return fail(FEM_ETIMEOUT, "no request finished within the timeout");
        }
    }
}

int fem_serve_release(fem_server* S, uint64_t ticket) {
    if (!S) return fail(FEM_EINVAL, "NULL server");
    std::unique_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(FEM_EINVAL, "unknown ticket");
        if (it->second->state != DONE) return fail(FEM_ESTATE, "request still pending or running");
        r = std::move(it->second);
        S->reqs.erase(it);
        S->in_use -= std::min(S->in_use, r->out_bytes);
        if (S->done_order.size() > 2 * S->reqs.size() + 4096) {
            // drop released tickets (clients that poll by ticket never drain it)
            std::deque<uint64_t> keep;
            for (uint64_t t : S->done_order)
                if (S->reqs.count(t)) keep.push_back(t);
            S->done_order.swap(keep);
        }
    }
    for (auto& b : r->out) buf_free(b, nullptr);
    if (r->done) cudaEventDestroy(r->done);
    S->cv_work.notify_one();
    return FEM_OK;
}

int fem_serve_evict(fem_server* S, uint64_t mesh_id) {
    if (!S) return fail(FEM_EINVAL, "NULL server");
    Resident res;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->meshes.find(mesh_id);
        if (it == S->meshes.end() || !it->second.mesh) return fail(FEM_EINVAL, "unknown or not yet assembled mesh id");
        if (it->second.busy) return fail(FEM_ESTATE, "a request of this mesh is in flight");
        // its pending requests fail now
        Resident& rs = it->second;
        std::vector<uint64_t> drop(rs.waiting.begin(), rs.waiting.end());
        if (rs.in_ready) {
            S->ready.erase(rs.ready_ticket);
            drop.push_back(rs.ready_ticket);
        }
        for (uint64_t t : drop) {
            --S->pending;
            finish(S, *S->reqs[t], FEM_EINVAL, "mesh was evicted before the request started");
        }
        rs.waiting.clear();
        rs.in_ready = false;
        res = it->second;
        S->in_use -= std::min(S->in_use, res.bytes);
        S->meshes.erase(it);
        S->batch_stale = true;
        if (S->building || S->batch_index.count(mesh_id)) {
            // the fused batch may reference the mesh: the scheduler destroys
            // it together with the batch
            S->graveyard.emplace_back(res.mesh, res.u);
            res.u = fem::DevBuf();
            res.mesh = nullptr;
        }
    }
    if (res.mesh) {
        buf_free(res.u, nullptr);
        fem_mesh_destroy(res.mesh);
    }
    S->cv_work.notify_one();
    return FEM_OK;
}

int fem_serve_stats(fem_server* S, fem_serve_counters* out) {
    if (!S || !out) return fail(FEM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->pending = (int)S->pending;
    out->inflight = S->inflight;
    out->resident_meshes = (int)S->meshes.size();
    out->bytes_in_use = S->in_use;
    out->peak_bytes = S->peak;
    out->single_launches = S->n_single;
    out->fused_launches = S->n_fused;
    out->fused_requests = S->n_fused_req;
    out->batch_builds = S->n_builds;
    out->host_start_us = S->host_start_us;
    return FEM_OK;
}

int fem_serve_destroy(fem_server* S) {
    if (!S) return FEM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto st : S->streams) cudaStreamSynchronize(st);
    if (S->bstream) cudaStreamSynchronize(S->bstream);
    if (S->batch) fem_batch_destroy(S->batch);
    S->batch = nullptr;
    for (auto& d : S->graveyard) {
        buf_free(d.second, nullptr);
        fem_mesh_destroy(d.first);
    }
    S->graveyard.clear();
    for (auto& kv : S->reqs) {
        for (auto& b : kv.second->out) buf_free(b, nullptr);
        if (kv.second->done) cudaEventDestroy(kv.second->done);
        drop_inputs(S, *kv.second);
    }
    S->pinned.clear();
    for (auto& kv : S->meshes) {
        buf_free(kv.second.u, nullptr);
        if (kv.second.mesh) fem_mesh_destroy(kv.second.mesh);
    }
    for (auto st : S->streams) cudaStreamDestroy(st);
    if (S->bstream) cudaStreamDestroy(S->bstream);
    delete S;
    return FEM_OK;
}

}  // extern "C"
