"""Pins of the oracle's FP64 error scale (absM, absK, absT).

Every FP64 parity verdict divides |gpu - oracle| by this scale, so an
inflated scale would loosen the 1e-12 bar unnoticed.  The scale of a CSR
entry is the sum, over elements and quadrature points, of the magnitudes of
the expanded product terms of that entry's quadrature sum (Section 3, step 4:
every entry of a local matrix is a quadrature sum; Algorithm 1 adds the local
matrices), with |A_ab| bounded by sqrt(A_aa A_bb) because A_e is symmetric
positive definite.  These tests fix it from outside the oracle's code:

  * P1 mass with a positive coefficient: the rules' points are interior, so
    every term w_q b_e m phi_i phi_j is positive and the scale equals M bit
    for bit; higher orders: |M| <= absM <= m sum_e b_e sum_q |w_q| for P2,
    whose basis functions stay within [-1/8, 1] on the simplex.
  * K with a constant k0 and T with k = k0 + c1 u (k' = c1), every order: the
    expanded term of S_ij = J_i A J_j^T has magnitude
    sum_ab |J_ia| |J_jb| sqrt(A_aa A_bb), which lies between
    min_c A_cc |J_i|_1 |J_j|_1 and max_c A_cc |J_i|_1 |J_j|_1.  The bracket
    is evaluated here with A_e = (B_e^T B_e)^-1 computed by numpy from the
    coordinates; on these meshes it is tight enough that both a 10x
    inflated and a 10x deflated scale fail it (checked in each test).
  * Rotating the mesh leaves b_e and A_e, hence all values and scales,
    unchanged.
"""
import numpy as np
import pytest

import meshgen as mg
import oracle as orc

CASES = {
    "tri_p1": lambda: mg.structured_tri(6, 1, 0.2, seed=5),
    "tri_p2": lambda: mg.structured_tri(5, 2, 0.2, seed=6),
    "tri_p3": lambda: mg.structured_tri(4, 3, 0.2, seed=7),
    "tet_p1": lambda: mg.structured_tet(3, 1, 0.15, seed=8),
    "tet_p2": lambda: mg.structured_tet(2, 2, 0.15, seed=9),
    "tet_p3": lambda: mg.structured_tet(2, 3, 0.15, seed=10),
}


def _dense(o, vals):
    rp, ci = o.pattern()
    return orc.csr_to_dense(rp, ci, vals, o.n)


def _geometry(mesh):
    """b_e = |det B_e| and the extreme diagonal entries of A_e = (B^T B)^-1,
    from the vertex coordinates (numpy, independent of the oracle)."""
    d = mesh.d
    X = mesh.coords[mesh.conn[:, : d + 1]]                # E x (d+1) x d
    B = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # columns x_k - x_0
    b = np.abs(np.linalg.det(B))
    A = np.linalg.inv(np.einsum("eka,ekb->eab", B, B))
    diag = np.einsum("eaa->ea", A)
    return b, diag.min(axis=1), diag.max(axis=1)


def _tables(mesh):
    x, w = orc.rule(mesh.d, 2 * mesh.p)
    phi, grad = zip(*(orc.basis(mesh.d, mesh.p, xq) for xq in x))
    return w, np.array(phi), np.array(grad)      # nq, (nq, np), (nq, np, d)


def _scatter(mesh, local):
    """Dense n x n sum over elements of local[e, a, b] at (conn[e,a], conn[e,b])."""
    n = mesh.n_nodes
    out = np.zeros((n, n))
    c = mesh.conn.astype(np.int64)
    rows = np.repeat(c[:, :, None], c.shape[1], axis=2)
    cols = np.repeat(c[:, None, :], c.shape[1], axis=1)
    np.add.at(out, (rows.ravel(), cols.ravel()), local.ravel())
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_p1_mass_scale_equals_mass_bitwise(dim):
    mesh = CASES["tri_p1" if dim == 2 else "tet_p1"]()
    o = orc.Oracle.of(mesh)
    u = mg.fourier_field(mesh.coords, 3)
    r = o.assemble(u, mg.Coeff("poly", (1.0, 0.5)), m=2.5)
    assert np.array_equal(r["absM"], r["M"])
    x, w = orc.rule(dim, 2)
    assert (w > 0).all() and (x > 0).all() and (x.sum(axis=1) < 1).all()   # interior points


def test_p2_mass_scale_bounds():
    mesh = CASES["tri_p2"]()
    o = orc.Oracle.of(mesh)
    r = o.assemble(np.zeros(mesh.n_nodes), mg.Coeff("poly", (1.0,)), m=1.5)
    b, _, _ = _geometry(mesh)
    w, _, _ = _tables(mesh)
    E, npl = mesh.conn.shape
    upper = _scatter(mesh, np.broadcast_to((1.5 * b * np.abs(w).sum())[:, None, None], (E, npl, npl)))
    aM, M = _dense(o, r["absM"]), _dense(o, r["M"])
    assert (aM >= np.abs(M) * (1 - 1e-14)).all()
    assert (aM <= upper * (1 + 1e-13)).all()
    # a scale 10x too large fails the bound
    assert (10 * aM > upper * (1 + 1e-13)).any()


def _k_bracket(mesh, k0):
    b, amin, amax = _geometry(mesh)
    w, _, grad = _tables(mesh)
    n1 = np.abs(grad).sum(axis=2)                               # |J_qi|_1, (nq, np)
    core = np.einsum("q,qi,qj->ij", np.abs(w), n1, n1)          # same for every element
    lo = _scatter(mesh, k0 * (b * amin)[:, None, None] * core[None])
    hi = _scatter(mesh, k0 * (b * amax)[:, None, None] * core[None])
    return lo, hi, amax / amin


@pytest.mark.parametrize("name", list(CASES))
def test_stiffness_scale_bracket(name):
    mesh = CASES[name]()
    o = orc.Oracle.of(mesh)
    k0 = 1.7
    r = o.assemble(mg.fourier_field(mesh.coords, 4), mg.Coeff("poly", (k0,)))
    lo, hi, ratio = _k_bracket(mesh, k0)
    aK, K = _dense(o, r["absK"]), _dense(o, r["K"])
    nz = hi > 0
    # the bracket is tight enough that a scale 10x too large or too small fails it
    assert (10 * aK[nz] > hi[nz]).any() and (aK[nz] / 10 < lo[nz]).any()
    assert np.median(ratio) < 4.0
    assert (aK[nz] >= lo[nz] * (1 - 1e-13)).all()
    assert (aK[nz] <= hi[nz] * (1 + 1e-13)).all()
    assert (aK >= np.abs(K) * (1 - 1e-13)).all()
    assert (aK[~nz] == 0).all()


@pytest.mark.parametrize("name", list(CASES))
def test_tangent_scale_bracket(name):
    mesh = CASES[name]()
    o = orc.Oracle.of(mesh)
    k0, c1 = 1.2, 0.8
    u = mg.fourier_field(mesh.coords, 5)          # values in [0, 1]
    r = o.assemble(u, mg.Coeff("poly", (k0, c1)))
    b, amin, amax = _geometry(mesh)
    w, phi, grad = _tables(mesh)
    n1 = np.abs(grad).sum(axis=2)                                  # (nq, np)
    ue = np.abs(u[mesh.conn])                                      # (E, np)
    gu = np.einsum("ql,el->eq", n1, ue)                            # sum_l |J_ql|_1 |u_l|
    core = np.einsum("q,qi,eq,qj->eij", np.abs(w), n1, gu, np.abs(phi))
    lo = _scatter(mesh, abs(c1) * (b * amin)[:, None, None] * core)
    hi = _scatter(mesh, abs(c1) * (b * amax)[:, None, None] * core)
    aT, T = _dense(o, r["absT"]), _dense(o, r["T"])
    nz = hi > 0
    assert (10 * aT[nz] > hi[nz]).any() and (aT[nz] / 10 < lo[nz]).any()
    assert (aT[nz] >= lo[nz] * (1 - 1e-13)).all()
    assert (aT[nz] <= hi[nz] * (1 + 1e-13)).all()
    assert (aT >= np.abs(T) * (1 - 1e-13)).all()


@pytest.mark.parametrize("name", ["tri_p2", "tet_p2"])
def test_scales_invariant_under_rotation(name):
    mesh = CASES[name]()
    u = mg.fourier_field(mesh.coords, 6)
    law = mg.Coeff("sin", (2.0, 1.0, 3.0))
    r0 = orc.Oracle.of(mesh).assemble(u, law)
    rng = np.random.default_rng(12)
    Q, R = np.linalg.qr(rng.standard_normal((mesh.d, mesh.d)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    rot = mg.Mesh(mesh.d, mesh.p, mesh.coords @ Q.T + 0.375, mesh.conn)
    r1 = orc.Oracle.of(rot).assemble(u, law)
    for k in ("M", "K", "T", "absM", "absK", "absT"):
        scale = np.abs(r0[k]).max()
        assert np.abs(r1[k] - r0[k]).max() <= 1e-12 * scale, k
