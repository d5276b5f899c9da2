"""Convenience layer over the libfem C ABI using PyTorch for device memory and
streams.  Marshalling only: buffers are torch tensors, all computation runs
in libfem's kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import (FEM_FP32, FEM_FP64, FEM_MEM_HOST, FEM_TF32X3, coeff, fem_assemble_all, fem_copy_pattern,
               fem_get_slot_map, fem_mesh_create, fem_mesh_desc, fem_mesh_destroy, fem_mesh_get_info, fem_symbolic)

PRECISIONS = {"fp64": FEM_FP64, "tf32x3": FEM_TF32X3, "fp32": FEM_FP32}


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

    def close(self):
        if getattr(self, "h", None):
            fem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
