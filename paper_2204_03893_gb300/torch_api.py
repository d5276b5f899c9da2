"""Convenience layer over the libfem C ABI using PyTorch for device memory and
streams.  Marshalling only: buffers are torch tensors, all computation runs
in libfem's kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import (FEM_BF16X3, FEM_BF16X6, FEM_FP32, FEM_FP64, FEM_MEM_HOST, FEM_REQ_ASSEMBLE, FEM_REQ_REASSEMBLE, FEM_TF32X3, coeff,
               fem_assemble_all, fem_assemble_mass_u, fem_copy_pattern, fem_mesh_set_conductivity, fem_get_slot_map, fem_mesh_create, fem_mesh_desc,
               fem_mesh_destroy, fem_mesh_get_info, fem_serve_create, fem_serve_destroy, fem_serve_evict,
               fem_serve_opts, fem_serve_poll, fem_serve_release, fem_serve_stats, fem_serve_submit, fem_symbolic)

PRECISIONS = {"fp64": FEM_FP64, "tf32x3": FEM_TF32X3, "fp32": FEM_FP32, "bf16x3": FEM_BF16X3, "bf16x6": FEM_BF16X6}


class FemMesh:
    """A libfem mesh handle built from host arrays (coords n x d float64,
    conn E x n_p int32)."""

    def __init__(self, d: int, p: int, coords: np.ndarray, conn: np.ndarray, mass: float = 1.0, stream=None):
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.conn = np.ascontiguousarray(conn, dtype=np.int32)
        desc = fem_mesh_desc()
        desc.dim, desc.order = d, p
        desc.n_nodes, desc.n_elems = self.coords.shape[0], self.conn.shape[0]
        desc.coords, desc.conn = self.coords.ctypes.data, self.conn.ctypes.data
        desc.mem, desc.qdeg, desc.mass_coeff = FEM_MEM_HOST, 0, float(mass)
        self.stream = stream
        self.h = fem_mesh_create(desc, stream)
        self.d, self.p = d, p
        self.n, self.E = self.coords.shape[0], self.conn.shape[0]
        self.nnz = -1

    @classmethod
    def of(cls, mesh, mass: float = 1.0, stream=None):
        return cls(mesh.d, mesh.p, mesh.coords, mesh.conn, mass, stream)

    def info(self):
        return fem_mesh_get_info(self.h)

    def symbolic(self):
        pat = fem_symbolic(self.h, self.stream)
        self.nnz = int(pat.nnz)
        return pat

    def pattern(self):
        """(row_ptr, col_idx) as int32 CUDA tensors (copies)."""
        if self.nnz < 0:
            self.symbolic()
        rp = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(max(self.nnz, 1), dtype=torch.int32, device="cuda")
        fem_copy_pattern(self.h, rp, ci, self.stream)
        return rp, ci[: self.nnz]

    def slot_map(self):
        n_p = self.conn.shape[1]
        out = torch.empty(self.E * n_p * n_p, dtype=torch.int32, device="cuda")
        fem_get_slot_map(self.h, out, self.stream)
        return out

    def assemble(self, u, kind: str, params, prec: str = "fp64", which=("M", "K", "T"), out=None):
        """CSR values of the requested matrices as CUDA tensors (or into `out`)."""
        if self.nnz < 0:
            self.symbolic()
        dt = torch.float64 if prec == "fp64" else torch.float32
        outs = {}
        for w in ("M", "K", "T"):
            if w in which:
                outs[w] = out[w] if out is not None else torch.empty(max(self.nnz, 1), dtype=dt, device="cuda")
        fem_assemble_all(self.h, coeff(kind, params), u, PRECISIONS[prec], outs.get("M"), outs.get("K"),
                         outs.get("T"), self.stream)
        return {k: v[: self.nnz] for k, v in outs.items()}

    def set_conductivity(self, c=None):
        """Constant anisotropic conductivity tensor (d x d SPD; None: identity)."""
        fem_mesh_set_conductivity(self.h, c, self.stream)
        return self

    def assemble_mass_u(self, u, us, kind: str, params, prec: str = "fp64", which=("Mu", "Mt")):
        """M(u) with the mass law (kind, params) and the mass tensor times
        (u - us), as CUDA tensors {'Mu', 'Mt'} (FP64 or FP32)."""
        if self.nnz < 0:
            self.symbolic()
        dt = torch.float64 if prec == "fp64" else torch.float32
        outs = {w: torch.empty(max(self.nnz, 1), dtype=dt, device="cuda") for w in ("Mu", "Mt") if w in which}
        fem_assemble_mass_u(self.h, coeff(kind, params), u, us, PRECISIONS[prec], outs.get("Mu"), outs.get("Mt"),
                            self.stream)
        return {k: v[: self.nnz] for k, v in outs.items()}

    def close(self):
        if getattr(self, "h", None):
            fem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """Describes library-owned device memory to torch (CUDA array interface)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2,
                                         "strides": None}


def device_view(ptr: int, n: int, dtype) -> torch.Tensor:
    """A CUDA tensor aliasing n elements at a library-owned device pointer."""
    ts = {torch.float64: "<f8", torch.float32: "<f4", torch.int32: "<i4"}[dtype]
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n, ts), device="cuda")


def mesh_desc(mesh, mass: float = 1.0):
    """(fem_mesh_desc, keep-alive arrays) for a host mesh."""
    coords = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    desc = fem_mesh_desc()
    desc.dim, desc.order = mesh.d, mesh.p
    desc.n_nodes, desc.n_elems = coords.shape[0], conn.shape[0]
    desc.coords, desc.conn = coords.ctypes.data, conn.ctypes.data
    desc.mem, desc.qdeg, desc.mass_coeff = FEM_MEM_HOST, 0, float(mass)
    return desc, (coords, conn)


_WHICH = {"M": 1, "K": 2, "T": 4}


class FemServer:
    """The request server of libfem (fem_serve_*) with torch-tensor results."""

    def __init__(self, prec: str = "tf32x3", budget_bytes: int = 8 << 30, max_inflight: int = 8, n_streams: int = 4,
                 max_queue: int = 1 << 20, fuse_min: int = 2):
        self.prec = prec
        self.h = fem_serve_create(fem_serve_opts(PRECISIONS[prec], max_inflight, n_streams, max_queue, budget_bytes,
                                                 fuse_min, 0))

    def assemble(self, mesh, kind: str = "poly", params=(1.0,), u=None, which="MKT", mass: float = 1.0) -> int:
        desc, keep = mesh_desc(mesh, mass)
        w = sum(_WHICH[c] for c in which)
        t = fem_serve_submit(self.h, FEM_REQ_ASSEMBLE, w, 0, desc, coeff(kind, params), u)
        del keep
        return t

    def reassemble(self, mesh_id: int, kind: str, params, u=None, which="MKT") -> int:
        w = sum(_WHICH[c] for c in which)
        return fem_serve_submit(self.h, FEM_REQ_REASSEMBLE, w, mesh_id, None, coeff(kind, params), u)

    def result(self, ticket: int, timeout_us: int = 60_000_000, copy: bool = True, release: bool = True):
        """Waits for the request; returns (fem_result, {"M"|"K"|"T": tensor})."""
        r = fem_serve_poll(self.h, ticket, timeout_us)
        vals = {}
        if r is not None and r.status == 0:
            dt = torch.float64 if r.prec == FEM_FP64 else torch.float32
            for name, ptr in (("M", r.d_vM), ("K", r.d_vK), ("T", r.d_vT)):
                if ptr:
                    v = device_view(ptr, int(r.nnz), dt)
                    vals[name] = v.clone() if copy else v
            torch.cuda.synchronize()
        if r is not None and release:
            fem_serve_release(self.h, ticket)
        return r, vals

    def evict(self, mesh_id: int):
        fem_serve_evict(self.h, mesh_id)

    def stats(self):
        return fem_serve_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            fem_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
