"""CPU FP64 oracle for finite element assembly -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library (``paper_2204_03893_gb300``)
never imports, links or runs it; the two share no code.

The arithmetic lives in ``fem_oracle.c`` (plain C, FP64): Algorithm 1 of the
paper (element loop, quadrature loop, dense local matrices, scatter-add), the
tangent as the Section 5.2 conductivity tensor multiplied by u in its second
mode, the u-dependent mass with the Section 5.1 mass tensor multiplied by
u - u^s in its second mode, and its own quadrature tables, Lagrange basis and CSR construction.
This module compiles it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"poly": 0, "sin": 1, "pwlin": 2}


def build(force: bool = False) -> str:
    """Compile fem_oracle.c into liboracle.so (plain gcc, -O2, no -ffast-math;
    -fopenmp for the multi-core timing variant)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:   # OpenMP for the multi-core timing variant; without it that variant runs on one thread
            subprocess.check_call(base[:4] + ["-fopenmp"] + base[4:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.oracle_rule.argtypes = [C.c_int, C.c_int, dp, dp]
            L.oracle_rule.restype = C.c_int
            L.oracle_basis.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.oracle_basis.restype = C.c_int
            L.oracle_nlocal.argtypes = [C.c_int, C.c_int]
            L.oracle_nlocal.restype = C.c_int
            L.oracle_k.argtypes = [C.c_int, dp, C.c_int, C.c_double, dp]
            L.oracle_k.restype = C.c_double
            L.oracle_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, ip]
            L.oracle_create.restype = C.c_void_p
            L.oracle_destroy.argtypes = [C.c_void_p]
            L.oracle_nnz.argtypes = [C.c_void_p]
            L.oracle_nnz.restype = C.c_longlong
            L.oracle_pattern.argtypes = [C.c_void_p, ip, ip]
            L.oracle_element.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int, dp, C.c_int, dp, dp, dp, dp]
            L.oracle_element.restype = C.c_int
            L.oracle_geometry.argtypes = [C.c_void_p, C.c_int, dp]
            L.oracle_geometry.restype = C.c_double
            L.oracle_assemble.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, dp, C.c_int, dp] + [dp] * 6
            L.oracle_assemble.restype = C.c_int
            L.oracle_assemble_mt.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, dp, C.c_int, dp] + [dp] * 3 \
                + [C.c_int]
            L.oracle_assemble_mt.restype = C.c_int
            L.oracle_boundary_facets.argtypes = [C.c_void_p, ip, ip]
            L.oracle_boundary_facets.restype = C.c_int
            L.oracle_boundary.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, dp, dp, dp, dp, dp]
            L.oracle_boundary.restype = C.c_int
            L.oracle_residual.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, C.c_double, dp, dp]
            L.oracle_residual.restype = C.c_int
            L.oracle_jacobian.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, C.c_double, dp]
            L.oracle_jacobian.restype = C.c_int
            L.oracle_facet_rule.argtypes = [C.c_int, C.c_int, dp, dp]
            L.oracle_facet_rule.restype = C.c_int
            L.oracle_entries.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, dp, C.c_int, dp,
                                         C.c_longlong, ip, ip] + [dp] * 6
            L.oracle_entries.restype = C.c_int
            L.oracle_assemble_mass_u.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_int, dp, dp] + [dp] * 4
            L.oracle_assemble_mass_u.restype = C.c_int
            L.oracle_set_isoparametric.argtypes = [C.c_void_p, C.c_int]
            L.oracle_set_isoparametric.restype = None
            L.oracle_set_conductivity_field.argtypes = [C.c_void_p, dp]
            L.oracle_set_conductivity_field.restype = C.c_int
            L.oracle_set_conductivity.argtypes = [C.c_void_p, dp]
            L.oracle_set_conductivity.restype = None
            _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def rule(d: int, deg: int):
    """Quadrature rule of the given degree: (points (nq x d), weights (nq))."""
    L = lib()
    n = L.oracle_rule(d, deg, None, None)
    if n < 0:
        raise ValueError("no rule")
    x = np.zeros((n, d))
    w = np.zeros(n)
    L.oracle_rule(d, deg, _dp(x), _dp(w))
    return x, w


def basis(d: int, p: int, xhat):
    """Lagrange basis values (n_p) and reference gradients (n_p x d) at xhat."""
    L = lib()
    n = L.oracle_nlocal(d, p)
    xh = np.ascontiguousarray(xhat, dtype=np.float64)
    phi = np.zeros(n)
    g = np.zeros((n, d))
    if L.oracle_basis(d, p, _dp(xh), _dp(phi), _dp(g)) != n:
        raise ValueError("bad element")
    return phi, g


def kfun(kind: str, params, u: float):
    """(k(u), k'(u)) for a conductivity law."""
    cp = np.ascontiguousarray(params, dtype=np.float64)
    dk = np.zeros(1)
    v = lib().oracle_k(KIND[kind], _dp(cp), len(cp), float(u), _dp(dk))
    return v, float(dk[0])


class Oracle:
    """Oracle bound to one mesh (coords n x d float64, conn E x n_p int32)."""

    def __init__(self, d: int, p: int, coords: np.ndarray, conn: np.ndarray):
        self.d, self.p = d, p
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.conn = np.ascontiguousarray(conn, dtype=np.int32)
        self.n = self.coords.shape[0]
        self.E = self.conn.shape[0]
        self._h = lib().oracle_create(d, p, self.n, self.E, _dp(self.coords), _ip(self.conn))
        if not self._h:
            raise ValueError("invalid mesh")

    @classmethod
    def of(cls, mesh):
        return cls(mesh.d, mesh.p, mesh.coords, mesh.conn)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_destroy(h)
            self._h = None

    def set_conductivity(self, c=None):
        """Constant conductivity tensor c (d x d, SPD): the conductivity
        becomes k(u) c and A_e = B_e^-1 c B_e^-T (None: identity)."""
        cc = None if c is None else np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(self.d, self.d))
        lib().oracle_set_conductivity(self._h, _dp(cc))
        return self

    def set_isoparametric(self, on: bool = True):
        """Map every element through all its nodes (curved elements): the
        Jacobian, its determinant and A depend on the quadrature point."""
        lib().oracle_set_isoparametric(self._h, 1 if on else 0)
        return self

    def set_conductivity_field(self, cf=None):
        """Conductivity tensors per quadrature point of the degree-2p rule,
        shape (E, n_q, d, d) (None: clear)."""
        if cf is None:
            lib().oracle_set_conductivity_field(self._h, None)
            return self
        self._cf = np.ascontiguousarray(cf, dtype=np.float64)
        if lib().oracle_set_conductivity_field(self._h, _dp(self._cf)) != 0:
            raise RuntimeError("oracle_set_conductivity_field failed")
        return self

    def nnz(self) -> int:
        return int(lib().oracle_nnz(self._h))

    def pattern(self):
        nz = self.nnz()
        rp = np.zeros(self.n + 1, dtype=np.int32)
        ci = np.zeros(max(nz, 1), dtype=np.int32)
        lib().oracle_pattern(self._h, _ip(rp), _ip(ci))
        return rp, ci[:nz]

    @staticmethod
    def _deg(deg, p):
        return deg or 2 * p

    def assemble(self, u, coeff, m: float = 1.0, deg: int = 0, want_abs: bool = True):
        """Returns dict with 'M','K','T' (and 'absM','absK','absT') CSR values."""
        nz = self.nnz()
        out = {k: np.zeros(nz) for k in ("M", "K", "T")}
        if want_abs:
            out.update({k: np.zeros(nz) for k in ("absM", "absK", "absT")})
        cp = coeff.numpy()
        uu = np.ascontiguousarray(u, dtype=np.float64)
        rc = lib().oracle_assemble(self._h, self._deg(deg, self.p), float(m), KIND[coeff.kind], _dp(cp), len(cp),
                                   _dp(uu), _dp(out["M"]), _dp(out["K"]), _dp(out["T"]),
                                   _dp(out.get("absM")), _dp(out.get("absK")), _dp(out.get("absT")))
        if rc != 0:
            raise RuntimeError(f"oracle_assemble failed ({rc})")
        return out

    def assemble_mt(self, u, coeff, m: float = 1.0, deg: int = 0, threads: int = 0):
        """The multi-core timing variant: the same M, K, T (same bits) with
        the element loop on `threads` host threads (0 = all cores).  Returns
        (dict, threads used)."""
        nz = self.nnz()
        out = {k: np.zeros(nz) for k in ("M", "K", "T")}
        cp = coeff.numpy()
        uu = np.ascontiguousarray(u, dtype=np.float64)
        used = lib().oracle_assemble_mt(self._h, self._deg(deg, self.p), float(m), KIND[coeff.kind], _dp(cp),
                                        len(cp), _dp(uu), _dp(out["M"]), _dp(out["K"]), _dp(out["T"]), int(threads))
        if used < 0:
            raise RuntimeError(f"oracle_assemble_mt failed ({used})")
        return out, used

    def assemble_mass_u(self, u, us, mcoeff, deg: int = 0):
        """M(u) (mass with the coefficient law m(u)) and the mass tensor of
        Section 5.1 multiplied by z = u - us in its second mode, as CSR
        values: dict with 'Mu', 'Mt', 'absMu', 'absMt' (us may be None:
        'Mt' then is not computed)."""
        nz = self.nnz()
        out = {k: np.zeros(nz) for k in ("Mu", "absMu")}
        if us is not None:
            out.update({k: np.zeros(nz) for k in ("Mt", "absMt")})
        cp = mcoeff.numpy()
        uu = np.ascontiguousarray(u, dtype=np.float64)
        ss = None if us is None else np.ascontiguousarray(us, dtype=np.float64)
        rc = lib().oracle_assemble_mass_u(self._h, self._deg(deg, self.p), KIND[mcoeff.kind], _dp(cp), len(cp),
                                          _dp(uu), _dp(ss), _dp(out["Mu"]), _dp(out.get("Mt")),
                                          _dp(out["absMu"]), _dp(out.get("absMt")))
        if rc != 0:
            raise RuntimeError(f"oracle_assemble_mass_u failed ({rc})")
        return out

    def entries(self, rows, cols, u, coeff, m: float = 1.0, deg: int = 0):
        """Selected entries computed one by one (works at any size)."""
        r = np.ascontiguousarray(rows, dtype=np.int32)
        c = np.ascontiguousarray(cols, dtype=np.int32)
        n = len(r)
        out = {k: np.zeros(n) for k in ("M", "K", "T", "absM", "absK", "absT")}
        cp = coeff.numpy()
        uu = np.ascontiguousarray(u, dtype=np.float64)
        rc = lib().oracle_entries(self._h, self._deg(deg, self.p), float(m), KIND[coeff.kind], _dp(cp), len(cp),
                                  _dp(uu), n, _ip(r), _ip(c), *[_dp(out[k]) for k in ("M", "K", "T", "absM", "absK", "absT")])
        if rc != 0:
            raise RuntimeError("oracle_entries failed")
        return out

    def boundary_facets(self):
        """Boundary facets (faces of exactly one element) as arrays (element,
        local face = the local vertex it is opposite to), ascending."""
        nb = lib().oracle_boundary_facets(self._h, None, None)
        fe = np.zeros(max(nb, 1), dtype=np.int32)
        ff = np.zeros(max(nb, 1), dtype=np.int32)
        lib().oracle_boundary_facets(self._h, _ip(fe), _ip(ff))
        return fe[:nb], ff[:nb]

    def boundary(self, u, gcoeff):
        """Boundary matrix B_ik = int g'(u_h) phi_i phi_k dS (CSR values) and
        boundary load b_i = int g(u_h) phi_i dS over the whole boundary:
        dict with 'B', 'b', 'absB', 'absb'."""
        nz = self.nnz()
        out = {"B": np.zeros(nz), "absB": np.zeros(nz), "b": np.zeros(self.n), "absb": np.zeros(self.n)}
        cp = gcoeff.numpy()
        uu = np.ascontiguousarray(u, dtype=np.float64)
        rc = lib().oracle_boundary(self._h, KIND[gcoeff.kind], _dp(cp), len(cp), _dp(uu), _dp(out["B"]),
                                   _dp(out["b"]), _dp(out["absB"]), _dp(out["absb"]))
        if rc != 0:
            raise RuntimeError(f"oracle_boundary failed ({rc})")
        return out

    def residual(self, M, K, b, u, us, dt):
        """F = M (u - us) + dt K u - dt b and its error scale: (F, absF)."""
        F = np.zeros(self.n)
        aF = np.zeros(self.n)
        arr = [np.ascontiguousarray(x, dtype=np.float64) if x is not None else None for x in (M, K, b, u, us)]
        rc = lib().oracle_residual(self._h, *[_dp(x) for x in arr], float(dt), _dp(F), _dp(aF))
        if rc != 0:
            raise RuntimeError("oracle_residual failed")
        return F, aF

    def jacobian(self, M, Mt, K, T, B, dt):
        """J = Mt + M + dt (K + T) - dt B on the pattern (Mt, T, B may be None)."""
        J = np.zeros(self.nnz())
        arr = [np.ascontiguousarray(x, dtype=np.float64) if x is not None else None for x in (M, Mt, K, T, B)]
        if lib().oracle_jacobian(self._h, *[_dp(x) for x in arr], float(dt), _dp(J)) != 0:
            raise RuntimeError("oracle_jacobian failed")
        return J

    def heat_step(self, k, g, us, dt, m, u0=None, rtol=1e-12, maxit=30):
        """One implicit Euler step (Section 5): Newton's method on
        F(u) = M (u - us) + dt K(u) u - dt b(u) with the Jacobian
        M + dt (K + T) - dt B (constant mass m), each linear system solved by
        a sparse direct solve (scipy.sparse.linalg.spsolve, a library step).
        Returns (u, {'newton': updates, 'residuals': [||F||_2 per iterate]})."""
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        rp, ci = self.pattern()
        us = np.ascontiguousarray(us, dtype=np.float64)
        u = us.copy() if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).copy()
        res = []
        for it in range(maxit + 1):
            r = self.assemble(u, k, m=m, want_abs=False)
            bd = self.boundary(u, g)
            F, _ = self.residual(r["M"], r["K"], bd["b"], u, us, dt)
            res.append(float(np.linalg.norm(F)))
            if res[-1] <= rtol * res[0] or it == maxit:
                break
            J = self.jacobian(r["M"], None, r["K"], r["T"], bd["B"], dt)
            A = sp.csr_matrix((J, ci, rp), shape=(self.n, self.n))
            u = u - spl.spsolve(A.tocsc(), F)
        return u, {"newton": len(res) - 1, "residuals": res}

    def element(self, e: int, u, coeff, m: float = 1.0, deg: int = 0):
        """Dense local matrices (Me, Ke, Te) of element e, row = test index."""
        np_ = self.conn.shape[1]
        Me, Ke, Te = (np.zeros((np_, np_)) for _ in range(3))
        cp = coeff.numpy()
        uu = np.ascontiguousarray(u, dtype=np.float64)
        if lib().oracle_element(self._h, int(e), self._deg(deg, self.p), float(m), KIND[coeff.kind], _dp(cp), len(cp),
                                _dp(uu), _dp(Me), _dp(Ke), _dp(Te)) != 0:
            raise ValueError("bad element")
        return Me, Ke, Te

    def geometry(self, e: int):
        """(det B_e, A_e) of element e."""
        A = np.zeros((self.d, self.d))
        det = lib().oracle_geometry(self._h, int(e), _dp(A))
        return det, A


def facet_rule(d: int, p: int):
    """The oracle's facet quadrature: (points (n x (d-1)), weights)."""
    L = lib()
    xi = np.zeros(64)
    w = np.zeros(32)
    n = L.oracle_facet_rule(d, p, _dp(xi), _dp(w))
    return xi[: n * (d - 1)].reshape(n, d - 1), w[:n]


def csr_to_dense(rp, ci, vals, n):
    """Dense matrix from CSR arrays (small n only)."""
    D = np.zeros((n, n))
    for r in range(n):
        D[r, ci[rp[r]:rp[r + 1]]] = vals[rp[r]:rp[r + 1]]
    return D
