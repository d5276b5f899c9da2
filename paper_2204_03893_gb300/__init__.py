"""Python binding of libfem (include/fem.h): loop-free finite element
reassembly of M, K(u) and the Newton tangent T(u) on one GB300 GPU.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libfem.so.  There is no CPU fallback; if the shared library is
missing, importing the functions raises.  PyTorch is used only by the
optional helpers in :mod:`.torch_api` for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

__all__ = [
    "FemError", "lib", "library_path", "fem_mesh_desc", "fem_coeff", "fem_mesh_info", "fem_csr_pattern",
    "fem_allocator", "fem_mesh_create", "fem_mesh_destroy", "fem_mesh_get_info", "fem_symbolic",
    "fem_get_slot_map", "fem_copy_pattern", "fem_assemble_mass", "fem_assemble_stiffness", "fem_assemble_tangent",
    "fem_assemble_all", "fem_assemble_mass_u", "fem_mesh_set_conductivity", "fem_reference_tables", "fem_set_allocator", "fem_last_error", "fem_version",
    "fem_device_status", "fem_batch_create", "fem_batch_launch", "fem_batch_get_info", "fem_batch_destroy",
    "fem_batch_opts", "fem_batch_info", "fem_serve_opts", "fem_request", "fem_result", "fem_serve_counters",
    "fem_serve_create", "fem_serve_submit", "fem_serve_poll", "fem_serve_next_done", "fem_serve_release",
    "fem_serve_evict",
    "fem_serve_stats", "fem_serve_destroy", "FEM_REQ_ASSEMBLE", "FEM_REQ_REASSEMBLE", "fem_form_elements", "fem_sum_elements", "fem_chunk_plan", "fem_form_elements_range",
    "fem_sum_elements_range", "coeff", "FEM_MAT_M", "FEM_MAT_K", "FEM_MAT_T", "FEM_OK", "FEM_EINVAL", "FEM_ENOMEM", "FEM_EDEGENERATE", "FEM_ECUDA",
    "FEM_EBUSY", "FEM_EAGAIN", "FEM_ETIMEOUT", "FEM_ESTATE", "FEM_FP64", "FEM_TF32X3", "FEM_FP32", "FEM_BF16X3",
    "FEM_BF16X6",
    "FEM_MEM_HOST", "FEM_MEM_DEVICE", "FEM_K_POLY", "FEM_K_SIN", "FEM_K_PWLIN",
]

FEM_OK, FEM_EINVAL, FEM_ENOMEM, FEM_EDEGENERATE, FEM_ECUDA = 0, -1, -2, -3, -4
FEM_EBUSY, FEM_EAGAIN, FEM_ETIMEOUT, FEM_ESTATE = -5, -6, -7, -8
FEM_FP64, FEM_TF32X3, FEM_FP32, FEM_BF16X3, FEM_BF16X6 = 0, 1, 2, 3, 4
FEM_MEM_HOST, FEM_MEM_DEVICE = 0, 1
FEM_K_POLY, FEM_K_SIN, FEM_K_PWLIN = 0, 1, 2
FEM_MAT_M, FEM_MAT_K, FEM_MAT_T = 1, 2, 4
FEM_REQ_ASSEMBLE, FEM_REQ_REASSEMBLE = 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.environ.get("FEM_LIBRARY", os.path.join(_HERE, "libfem.so"))


class FemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfem error {code}: {msg}")
        self.code = code


class fem_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("order", C.c_int), ("n_nodes", C.c_int64), ("n_elems", C.c_int64),
                ("coords", C.c_void_p), ("conn", C.c_void_p), ("mem", C.c_int), ("qdeg", C.c_int),
                ("mass_coeff", C.c_double)]


class fem_coeff(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("p", C.c_double * 16)]


class fem_mesh_info(C.Structure):
    _fields_ = [("dim", C.c_int), ("order", C.c_int), ("n_p", C.c_int), ("n_q", C.c_int),
                ("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("nnz", C.c_int64), ("n_flagged", C.c_int64),
                ("device_bytes", C.c_size_t)]


class fem_csr_pattern(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("d_row_ptr", C.c_void_p), ("d_col_idx", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class fem_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class fem_heat_report(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("krylov_iters", C.c_int), ("converged", C.c_int), ("pad", C.c_int),
                ("residual0", C.c_double), ("residual", C.c_double), ("max_krylov_relres", C.c_double)]


class fem_batch_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("tune", C.c_int), ("use_graph", C.c_int), ("reserved", C.c_int)]


class fem_batch_info(C.Structure):
    _fields_ = [("n_meshes", C.c_int), ("kernels_per_launch", C.c_int), ("tc_tiles", C.c_int),
                ("simt_blocks", C.c_int), ("sum_chunks", C.c_int), ("sum_block", C.c_int), ("simt_grid", C.c_int),
                ("tuned", C.c_int), ("graph", C.c_int), ("tuned_ms", C.c_double)]


class fem_serve_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("max_inflight", C.c_int), ("n_streams", C.c_int), ("max_queue", C.c_int),
                ("budget_bytes", C.c_size_t), ("fuse_min", C.c_int), ("reserved", C.c_int)]


class fem_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("which", C.c_int), ("mesh_id", C.c_uint64),
                ("desc", C.POINTER(fem_mesh_desc)), ("k", C.POINTER(fem_coeff)), ("u", C.c_void_p)]


class fem_result(C.Structure):
    _fields_ = [("status", C.c_int), ("prec", C.c_int), ("mesh_id", C.c_uint64), ("n", C.c_int64),
                ("nnz", C.c_int64), ("d_row_ptr", C.c_void_p), ("d_col_idx", C.c_void_p), ("d_vM", C.c_void_p),
                ("d_vK", C.c_void_p), ("d_vT", C.c_void_p), ("t_submit_us", C.c_double),
                ("t_start_us", C.c_double), ("t_done_us", C.c_double)]


class fem_serve_counters(C.Structure):
    _fields_ = [("pending", C.c_int), ("inflight", C.c_int), ("resident_meshes", C.c_int),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t), ("single_launches", C.c_int64),
                ("fused_launches", C.c_int64), ("fused_requests", C.c_int64), ("batch_builds", C.c_int64),
                ("host_start_us", C.c_double)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "fem_mesh_create": ([C.POINTER(fem_mesh_desc), C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "fem_mesh_destroy": ([C.c_void_p], C.c_int),
    "fem_mesh_get_info": ([C.c_void_p, C.POINTER(fem_mesh_info)], C.c_int),
    "fem_symbolic": ([C.c_void_p, C.c_void_p, C.POINTER(fem_csr_pattern)], C.c_int),
    "fem_get_slot_map": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_copy_pattern": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_assemble_mass": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "fem_assemble_stiffness": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
                               C.c_int),
    "fem_assemble_tangent": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
                             C.c_int),
    "fem_mesh_set_conductivity": ([C.c_void_p, C.POINTER(C.c_double), C.c_void_p], C.c_int),
    "fem_assemble_mass_u": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                             C.c_void_p, C.c_void_p], C.c_int),
    "fem_assemble_all": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                          C.c_void_p, C.c_void_p], C.c_int),
    "fem_device_status": ([C.c_void_p], C.c_int),
    "fem_batch_create": ([C.POINTER(C.c_void_p), C.c_int, C.POINTER(fem_batch_opts), C.c_void_p,
                          C.POINTER(C.c_void_p)], C.c_int),
    "fem_batch_launch": ([C.c_void_p, C.POINTER(fem_coeff), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                          C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p], C.c_int),
    "fem_batch_get_info": ([C.c_void_p, C.POINTER(fem_batch_info)], C.c_int),
    "fem_batch_destroy": ([C.c_void_p], C.c_int),
    "fem_serve_create": ([C.POINTER(fem_serve_opts), C.POINTER(C.c_void_p)], C.c_int),
    "fem_serve_submit": ([C.c_void_p, C.POINTER(fem_request), C.POINTER(C.c_uint64)], C.c_int),
    "fem_serve_poll": ([C.c_void_p, C.c_uint64, C.c_int, C.POINTER(fem_result)], C.c_int),
    "fem_serve_release": ([C.c_void_p, C.c_uint64], C.c_int),
    "fem_serve_next_done": ([C.c_void_p, C.c_int, C.POINTER(C.c_uint64)], C.c_int),
    "fem_serve_evict": ([C.c_void_p, C.c_uint64], C.c_int),
    "fem_serve_stats": ([C.c_void_p, C.POINTER(fem_serve_counters)], C.c_int),
    "fem_serve_destroy": ([C.c_void_p], C.c_int),
    "fem_assemble_all_noalloc": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p], C.c_int),
    "fem_form_elements": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_int, C.c_int, C.c_void_p], C.c_int),
    "fem_law_eval": ([C.POINTER(fem_coeff), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_law_eval_fp32": ([C.POINTER(fem_coeff), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_bicgstab": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int),
                      C.POINTER(C.c_double), C.c_void_p], C.c_int),
    "fem_heat_step": ([C.c_void_p, C.POINTER(fem_coeff), C.POINTER(fem_coeff), C.c_void_p, C.c_double, C.c_void_p,
                       C.c_void_p, C.c_double, C.c_int, C.c_double, C.c_int, C.POINTER(fem_heat_report), C.c_void_p],
                      C.c_int),
    "fem_mesh_set_isoparametric": ([C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "fem_mesh_set_conductivity_field": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_boundary_facets": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "fem_get_boundary_facets": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_assemble_boundary": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p], C.c_int),
    "fem_csr_spmv": ([C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "fem_residual": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                      C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_jacobian": ([C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                      C.c_void_p, C.c_void_p], C.c_int),
    "fem_chunk_plan": ([C.c_void_p, C.c_int, C.c_size_t, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64),
                        C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "fem_form_elements_range": ([C.c_void_p, C.POINTER(fem_coeff), C.c_void_p, C.c_int, C.c_int, C.c_int64,
                                 C.c_int64, C.c_void_p], C.c_int),
    "fem_sum_elements_range": ([C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p], C.c_int),
    "fem_sum_elements": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "fem_reference_tables": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.POINTER(C.c_int)], C.c_int),
    "fem_set_allocator": ([C.POINTER(fem_allocator)], C.c_int),
    "fem_last_error": ([C.c_char_p, C.c_size_t], C.c_int),
    "fem_version": ([], C.c_char_p),
}


def lib() -> C.CDLL:
    """Loads libfem.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise FemError(FEM_EINVAL, f"{path} not found: build it with paper_2204_03893_gb300.build.build()")
            L = C.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _err() -> str:
    buf = C.create_string_buffer(1024)
    lib().fem_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc: int) -> int:
    if rc != FEM_OK:
        raise FemError(rc, _err())
    return rc


def _vp(x):
    """Pointer argument: int address, None, a ctypes object or an object
    exposing data_ptr() (torch tensors) or .ctypes (numpy arrays)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return C.cast(x, C.c_void_p).value


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return getattr(s, "cuda_stream", s)


def coeff(kind: str, params) -> fem_coeff:
    """fem_coeff from ('poly'|'sin'|'pwlin', parameters)."""
    c = fem_coeff()
    c.kind = {"poly": FEM_K_POLY, "sin": FEM_K_SIN, "pwlin": FEM_K_PWLIN}[kind]
    params = list(params)
    if kind == "poly":
        while len(params) > 1 and params[-1] == 0.0:
            params.pop()
    c.n = len(params)
    for i, v in enumerate(params):
        c.p[i] = float(v)
    return c


# ------------------------------------------------------------------ calls
def fem_mesh_create(desc: fem_mesh_desc, stream=None) -> int:
    h = C.c_void_p()
    _check(lib().fem_mesh_create(C.byref(desc), _stream(stream), C.byref(h)))
    return h.value


def fem_mesh_destroy(mesh: int) -> None:
    _check(lib().fem_mesh_destroy(mesh))


def fem_mesh_get_info(mesh: int) -> fem_mesh_info:
    info = fem_mesh_info()
    _check(lib().fem_mesh_get_info(mesh, C.byref(info)))
    return info


def fem_symbolic(mesh: int, stream=None) -> fem_csr_pattern:
    pat = fem_csr_pattern()
    _check(lib().fem_symbolic(mesh, _stream(stream), C.byref(pat)))
    return pat


def fem_copy_pattern(mesh: int, d_row_ptr, d_col_idx, stream=None) -> None:
    _check(lib().fem_copy_pattern(mesh, _vp(d_row_ptr), _vp(d_col_idx), _stream(stream)))


def fem_get_slot_map(mesh: int, d_slot, stream=None) -> None:
    _check(lib().fem_get_slot_map(mesh, _vp(d_slot), _stream(stream)))


def fem_assemble_mass(mesh: int, prec: int, values, stream=None) -> None:
    _check(lib().fem_assemble_mass(mesh, prec, _vp(values), _stream(stream)))


def fem_assemble_stiffness(mesh: int, k: fem_coeff, u, prec: int, values, stream=None) -> None:
    _check(lib().fem_assemble_stiffness(mesh, C.byref(k), _vp(u), prec, _vp(values), _stream(stream)))


def fem_assemble_tangent(mesh: int, k: fem_coeff, u, prec: int, values, stream=None) -> None:
    _check(lib().fem_assemble_tangent(mesh, C.byref(k), _vp(u), prec, _vp(values), _stream(stream)))


def fem_assemble_all(mesh: int, k, u, prec: int, vM, vK, vT, stream=None) -> None:
    _check(lib().fem_assemble_all(mesh, C.byref(k) if k is not None else None, _vp(u), prec, _vp(vM), _vp(vK),
                                  _vp(vT), _stream(stream)))


def fem_mesh_set_conductivity(mesh: int, c=None, stream=None) -> None:
    """Constant anisotropic conductivity tensor c (d x d, symmetric positive
    definite; None: the identity); recomputes the geometry cache."""
    if c is None:
        _check(lib().fem_mesh_set_conductivity(mesh, None, _stream(stream)))
        return
    flat = [float(x) for row in c for x in (row if hasattr(row, "__len__") else [row])]
    arr = (C.c_double * len(flat))(*flat)
    _check(lib().fem_mesh_set_conductivity(mesh, arr, _stream(stream)))


def fem_assemble_mass_u(mesh: int, m, d_u, d_us, prec: int, d_vMu, d_vMt, stream=None) -> None:
    """M(u) with the coefficient law m and the mass tensor times (u - u^s)
    (FEM_FP64 / FEM_FP32; device pointers only)."""
    _check(lib().fem_assemble_mass_u(mesh, C.byref(m) if m is not None else None, _vp(d_u), _vp(d_us), prec,
                                     _vp(d_vMu), _vp(d_vMt), _stream(stream)))


def fem_form_elements(mesh: int, k, d_u, prec: int, which: int, stream=None) -> None:
    _check(lib().fem_form_elements(mesh, C.byref(k) if k is not None else None, _vp(d_u), prec, which,
                                   _stream(stream)))


def fem_sum_elements(mesh: int, prec: int, d_vM, d_vK, d_vT, stream=None) -> None:
    _check(lib().fem_sum_elements(mesh, prec, _vp(d_vM), _vp(d_vK), _vp(d_vT), _stream(stream)))


FEM_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024


def fem_assemble_all_noalloc(mesh: int, k, d_u, d_vM, d_vK, d_vT, stream=None) -> None:
    """FP64 reassembly that allocates no device memory (scratch in a fixed
    library array of FEM_NOALLOC_SCRATCH_BYTES); device pointers only."""
    _check(lib().fem_assemble_all_noalloc(mesh, C.byref(k) if k is not None else None, _vp(d_u), _vp(d_vM),
                                          _vp(d_vK), _vp(d_vT), _stream(stream)))


def fem_law_eval(k, d_u, n: int, d_k, d_dk, stream=None) -> None:
    """k(u) and k'(u) of a law at n device values, in FP64 on the GPU."""
    _check(lib().fem_law_eval(C.byref(k), _vp(d_u), int(n), _vp(d_k), _vp(d_dk), _stream(stream)))

def fem_law_eval_fp32(k, d_u, n: int, d_k, d_dk, stream=None) -> None:
    """k(u) and k'(u) in FP32 with the FP32 element kernels' device code."""
    _check(lib().fem_law_eval_fp32(C.byref(k), _vp(d_u), int(n), _vp(d_k), _vp(d_dk), _stream(stream)))


def fem_bicgstab(mesh: int, d_vA, d_b, d_x, rtol: float, maxit: int, stream=None):
    """Solves A x = b in place (Jacobi-preconditioned BiCGStab); returns
    (iterations, relative residual)."""
    it, rr = C.c_int(), C.c_double()
    _check(lib().fem_bicgstab(mesh, _vp(d_vA), _vp(d_b), _vp(d_x), float(rtol), int(maxit), C.byref(it), C.byref(rr),
                              _stream(stream)))
    return it.value, rr.value


def fem_heat_step(mesh: int, k, g, d_mask, dt: float, d_us, d_u, newton_rtol: float = 1e-10, max_newton: int = 20,
                  krylov_rtol: float = 1e-12, max_krylov: int = 1000, stream=None) -> fem_heat_report:
    """One implicit Euler step (d_u: initial guess in, new state out)."""
    rep = fem_heat_report()
    _check(lib().fem_heat_step(mesh, C.byref(k), C.byref(g), _vp(d_mask), float(dt), _vp(d_us), _vp(d_u),
                               float(newton_rtol), int(max_newton), float(krylov_rtol), int(max_krylov), C.byref(rep),
                               _stream(stream)))
    return rep


def fem_mesh_set_isoparametric(mesh: int, on: bool = True, stream=None) -> None:
    _check(lib().fem_mesh_set_isoparametric(mesh, 1 if on else 0, _stream(stream)))


def fem_mesh_set_conductivity_field(mesh: int, c_field=None, stream=None) -> None:
    """c_field: (n_elems, n_q, d, d) float64 (numpy or a device tensor), or None."""
    if c_field is not None and not hasattr(c_field, "data_ptr"):
        import numpy as _np
        c_field = _np.ascontiguousarray(c_field, dtype=_np.float64)
    _check(lib().fem_mesh_set_conductivity_field(mesh, _vp(c_field), _stream(stream)))


def fem_boundary_facets(mesh: int, stream=None) -> int:
    """Finds the boundary facets once per mesh; returns their number."""
    n = C.c_int64()
    _check(lib().fem_boundary_facets(mesh, _stream(stream), C.byref(n)))
    return n.value


def fem_get_boundary_facets(mesh: int, d_elem, d_face, stream=None) -> None:
    _check(lib().fem_get_boundary_facets(mesh, _vp(d_elem), _vp(d_face), _stream(stream)))


def fem_assemble_boundary(mesh: int, g, d_u, d_mask, d_vB, d_b, stream=None) -> None:
    """B(u) (CSR values) and the boundary load b(u), FP64."""
    _check(lib().fem_assemble_boundary(mesh, C.byref(g), _vp(d_u), _vp(d_mask), _vp(d_vB), _vp(d_b),
                                       _stream(stream)))


def fem_csr_spmv(mesh: int, d_vals, alpha: float, d_x, beta: float, d_y, stream=None) -> None:
    _check(lib().fem_csr_spmv(mesh, _vp(d_vals), float(alpha), _vp(d_x), float(beta), _vp(d_y), _stream(stream)))


def fem_residual(mesh: int, d_vM, d_vK, d_b, d_u, d_us, dt: float, d_F, d_norms, stream=None) -> None:
    _check(lib().fem_residual(mesh, _vp(d_vM), _vp(d_vK), _vp(d_b), _vp(d_u), _vp(d_us), float(dt), _vp(d_F),
                              _vp(d_norms), _stream(stream)))


def fem_jacobian(mesh: int, dt: float, d_vM, d_vMt, d_vK, d_vT, d_vB, d_vJ, stream=None) -> None:
    _check(lib().fem_jacobian(mesh, float(dt), _vp(d_vM), _vp(d_vMt), _vp(d_vK), _vp(d_vT), _vp(d_vB), _vp(d_vJ),
                              _stream(stream)))


def _ptr_array(seq):
    if seq is None:
        return None
    arr = (C.c_void_p * len(seq))()
    for i, x in enumerate(seq):
        arr[i] = _vp(x)
    return arr


def fem_batch_create(meshes, opts: fem_batch_opts | None = None, stream=None) -> int:
    arr = (C.c_void_p * len(meshes))(*meshes)
    h = C.c_void_p()
    _check(lib().fem_batch_create(arr, len(meshes), C.byref(opts) if opts is not None else None, _stream(stream),
                                  C.byref(h)))
    return h.value


def fem_batch_launch(batch: int, coeffs, d_u, d_vM, d_vK, d_vT, stream=None) -> None:
    """coeffs: sequence of fem_coeff (one per mesh); the other arguments are
    sequences of device pointers / tensors (or None)."""
    karr = (fem_coeff * len(coeffs))(*coeffs) if coeffs is not None else None
    _check(lib().fem_batch_launch(batch, karr, _ptr_array(d_u), _ptr_array(d_vM), _ptr_array(d_vK),
                                  _ptr_array(d_vT), _stream(stream)))


def fem_batch_get_info(batch: int) -> fem_batch_info:
    info = fem_batch_info()
    _check(lib().fem_batch_get_info(batch, C.byref(info)))
    return info


def fem_batch_destroy(batch: int) -> None:
    _check(lib().fem_batch_destroy(batch))


def fem_serve_create(opts: fem_serve_opts) -> int:
    h = C.c_void_p()
    _check(lib().fem_serve_create(C.byref(opts), C.byref(h)))
    return h.value


def fem_serve_submit(server: int, kind: int, which: int = 7, mesh_id: int = 0, desc: fem_mesh_desc | None = None,
                     k: fem_coeff | None = None, u=None) -> int:
    """Queues one request; u is a host FP64 array (copied), desc a
    fem_mesh_desc whose buffers stay alive for the call.  Returns the ticket."""
    import numpy as np
    ua = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
    req = fem_request(kind, which, mesh_id, C.pointer(desc) if desc is not None else None,
                      C.pointer(k) if k is not None else None, ua.ctypes.data if ua is not None else None)
    t = C.c_uint64()
    _check(lib().fem_serve_submit(server, C.byref(req), C.byref(t)))
    return t.value


def fem_serve_poll(server: int, ticket: int, timeout_us: int = 0) -> fem_result | None:
    """The finished request's result, or None if it is not finished and
    timeout_us <= 0.  Raises FemError(FEM_ETIMEOUT) if a wait ran out."""
    out = fem_result()
    rc = lib().fem_serve_poll(server, ticket, timeout_us, C.byref(out))
    if rc == FEM_EAGAIN:
        return None
    _check(rc)
    return out


def fem_serve_next_done(server: int, timeout_us: int = 0) -> int | None:
    """Ticket of a finished request not returned before, in completion order;
    None if none is ready and timeout_us <= 0.  Raises FemError(FEM_ETIMEOUT)
    if a wait ran out."""
    t = C.c_uint64(0)
    rc = lib().fem_serve_next_done(server, timeout_us, C.byref(t))
    if rc == FEM_EAGAIN:
        return None
    _check(rc)
    return int(t.value)


def fem_serve_release(server: int, ticket: int) -> None:
    _check(lib().fem_serve_release(server, ticket))


def fem_serve_evict(server: int, mesh_id: int) -> None:
    _check(lib().fem_serve_evict(server, mesh_id))


def fem_serve_stats(server: int) -> fem_serve_counters:
    out = fem_serve_counters()
    _check(lib().fem_serve_stats(server, C.byref(out)))
    return out


def fem_serve_destroy(server: int) -> None:
    _check(lib().fem_serve_destroy(server))


def fem_chunk_plan(mesh: int, prec: int, target_bytes: int = 0, max_chunks: int = 64, stream=None):
    """(element bounds, slot bounds) of the chunked schedule, as lists of n+1."""
    n = C.c_int()
    eb = (C.c_int64 * (max_chunks + 1))()
    sb = (C.c_int64 * (max_chunks + 1))()
    _check(lib().fem_chunk_plan(mesh, prec, target_bytes, max_chunks, C.byref(n), eb, sb, _stream(stream)))
    return list(eb[: n.value + 1]), list(sb[: n.value + 1])


def fem_form_elements_range(mesh: int, k, d_u, prec: int, which: int, e_begin: int, e_end: int, stream=None) -> None:
    _check(lib().fem_form_elements_range(mesh, C.byref(k) if k is not None else None, _vp(d_u), prec, which,
                                         e_begin, e_end, _stream(stream)))


def fem_sum_elements_range(mesh: int, prec: int, s_begin: int, s_end: int, d_vM, d_vK, d_vT, stream=None) -> None:
    _check(lib().fem_sum_elements_range(mesh, prec, s_begin, s_end, _vp(d_vM), _vp(d_vK), _vp(d_vT),
                                        _stream(stream)))


def fem_device_status(stream=None) -> None:
    _check(lib().fem_device_status(_stream(stream)))


def fem_reference_tables(dim: int, order: int, qdeg: int = 0):
    """(xq, wq, phi, grad) of the library's reference element as numpy arrays."""
    import numpy as np
    nq = C.c_int()
    _check(lib().fem_reference_tables(dim, order, qdeg, None, None, None, None, C.byref(nq)))
    n = nq.value
    np_ = {2: (order + 1) * (order + 2) // 2, 3: (order + 1) * (order + 2) * (order + 3) // 6}[dim]
    xq = np.zeros((n, dim))
    wq = np.zeros(n)
    phi = np.zeros((n, np_))
    grad = np.zeros((n, np_, dim))
    _check(lib().fem_reference_tables(dim, order, qdeg, xq.ctypes.data, wq.ctypes.data, phi.ctypes.data,
                                      grad.ctypes.data, C.byref(nq)))
    return xq, wq, phi, grad


def fem_set_allocator(alloc: fem_allocator | None) -> None:
    _check(lib().fem_set_allocator(C.byref(alloc) if alloc is not None else None))


def fem_last_error() -> str:
    return _err()


def fem_version() -> str:
    return lib().fem_version().decode()
