// noalloc.cu -- an FP64 reassembly entry point that allocates no device
// memory: its scratch (the element matrices V between the element product
// and the CSR sum) lives in a fixed, file-scope device array instead of
// memory taken from the allocator.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example a solver loop whose memory budget is fixed up front by a
// framework that owns the whole device pool, or a latency-critical service
// loop in which a driver allocation (which may synchronise the device) is not
// acceptable.  They still pass their own inputs and outputs; the mesh handle,
// its geometry and its pattern were created earlier by the ordinary calls.
//
// The array is part of the library: every GPU that loads the library holds
// it until the process exits.  The driver loads the array's module into a
// device's memory when the first call on that device looks up its address
// (with CUDA's default lazy module loading); that first call therefore makes
// one driver allocation, which may synchronise the device, and should come
// before any stream capture and outside latency-critical loops.  Later calls
// on the device allocate nothing.  All calls share it and it keeps
// the last call's contents; every entry of V is overwritten before it is
// read, so nothing has to start at zero.  Calls whose GPU work overlaps (on
// different streams, or from different threads) race on the array.
#include <cstring>
#include <mutex>

#include "fem_internal.h"

namespace fem {

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FEM_NOALLOC_SCRATCH_BYTES];

std::mutex g_na_mu;
void* g_na_ptr[64] = {};   // device address of the array, per device (set up once)

// A pointer the caller passes must be device memory of the current device
// (or managed memory): a host pointer handed to the kernels would fault.
// cudaPointerGetAttributes only reads the driver's records; it allocates
// nothing.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Host code cannot use the array's name as a device address; fetch the real
// address once per device, with that device current.
int noalloc_setup(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (dev < 0 || dev >= 64) return fail(FEM_EINVAL, "device index out of range");
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        int rc = tables_init_simt();   // reference tables: a symbol copy, no allocation
        if (rc) return rc;
        g_na_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_na_ptr[dev]);
    return FEM_OK;
}

}  // namespace

}  // namespace fem

using namespace fem;

extern "C" int fem_assemble_all_noalloc(fem_mesh* m, const fem_coeff* k, const double* d_u, double* d_vM,
                                        double* d_vK, double* d_vT, void* stream) {
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    if (!d_vM && !d_vK && !d_vT) return FEM_OK;
    if (d_vK || d_vT) {
        int rc0 = validate_coeff(k);
        if (rc0) return rc0;
        if (!d_u) return fail(FEM_EINVAL, "u is NULL");
    }
    const size_t nsym = (size_t)m->np * (m->np + 1) / 2, nt = (size_t)m->np * m->np;
    // M and K interleaved in one array (K at the odd positions), then T
    const size_t bMK = (d_vM || d_vK) ? 2 * sizeof(double) * (size_t)m->E * nsym : 0;
    const size_t bT = d_vT ? sizeof(double) * (size_t)m->E * nt : 0;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t need = up(bMK) + up(bT);
    if (need > (size_t)FEM_NOALLOC_SCRATCH_BYTES)
        return fail(FEM_EINVAL, "mesh too large for fem_assemble_all_noalloc: needs " + std::to_string(need) +
                                    " bytes of scratch, the fixed array holds " +
                                    std::to_string((size_t)FEM_NOALLOC_SCRATCH_BYTES));
    int dev = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    if (m->device != dev)
        return fail(FEM_EINVAL, "fem_assemble_all_noalloc: the mesh lives on device " + std::to_string(m->device) +
                                    ", the current device is " + std::to_string(dev));
    const void* ptrs[4] = {(d_vK || d_vT) ? d_u : nullptr, d_vM, d_vK, d_vT};
    for (const void* p : ptrs)
        if (p && !on_device(p, dev))
            return fail(FEM_EINVAL, "fem_assemble_all_noalloc takes device pointers of the current device only");
    unsigned char* base = nullptr;
    int rc = noalloc_setup(dev, &base);
    if (rc) return rc;
    double* VM = d_vM ? reinterpret_cast<double*>(base) : nullptr;
    double* VK = d_vK ? reinterpret_cast<double*>(base) + 1 : nullptr;
    double* VT = d_vT ? reinterpret_cast<double*>(base + up(bMK)) : nullptr;
    const CoeffDev kd = coeff_to_device(k);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = element_simt_fp64(*m, kd, d_u, VM, VK, VT, s))) return rc;
    return scatter_fp64(*m, VM, VK, VT, d_vM, d_vK, d_vT, p1_factored(*m), s);
}
