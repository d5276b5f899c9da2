"""Pins of the oracle's per-quadrature-point geometry (Section 7).

Isoparametric mappings make the Jacobian depend on the quadrature point:
B_q = sum_i x_i (grad phi_i(xhat_q))^T through all the element's nodes, with
det B_q and A_q = B_q^-1 c_q B_q^-T per point; an anisotropic conductivity
may also vary over the points (A_qe = B_e^-1 c_q B_e^-T).  Fixed here by:
  * an affine mesh run through the isoparametric path gives the affine
    results; a field with the same tensor at every point gives the constant
    tensor's results bit for bit;
  * curved meshes (higher-order nodes off the boundary moved, meshgen.curved)
    still tile the unit square / cube, and det B_q is a polynomial the rules
    integrate exactly (degree 2, 3, 4, 6 for P2/P3 triangles/tetrahedra), so
    sum M = m exactly; a linear u = a.x is reproduced by the isoparametric
    space, so u^T K u = k |a|^2 exactly; with c(x) = diag(1 + x, 2 - y
    (, 1 + z)) sampled at the physical quadrature points, u^T K u =
    int a^T c(x) a dx in closed form wherever the rule integrates
    c(x(xhat)) det B exactly (curved P2 triangles, affine elements);
  * K rows and T columns sum to zero; rotating the mesh and the field
    (c_q -> R c_q R^T) leaves every value unchanged; the tangent against
    exact Richardson differences.
"""
import numpy as np
import pytest

import meshgen as mg
import oracle as orc

CASES = [(2, 2), (2, 3), (3, 2), (3, 3)]


def _mesh(d, p, seed=61, curved=True):
    m = mg.structured_tri(4, p, 0.2, seed=seed) if d == 2 else mg.structured_tet(2, p, 0.15, seed=seed)
    return mg.curved(m, 0.05, seed=seed + 1) if curved else m


def _min_det(mesh):
    """Smallest det B_q over all elements and points (numpy, from the nodes)."""
    xq, _ = orc.rule(mesh.d, 2 * mesh.p)
    G = np.array([orc.basis(mesh.d, mesh.p, x)[1] for x in xq])           # (nq, np, d)
    B = np.einsum("eia,qib->eqab", mesh.coords[mesh.conn], G)
    return np.linalg.det(B).min()


def _qpoints(mesh):
    """Physical quadrature points x(xhat_q) = sum_i x_i phi_i(xhat_q): (E, nq, d)."""
    xq, _ = orc.rule(mesh.d, 2 * mesh.p)
    phi = np.array([orc.basis(mesh.d, mesh.p, x)[0] for x in xq])      # (nq, np)
    return np.einsum("qi,eid->eqd", phi, mesh.coords[mesh.conn])


@pytest.mark.parametrize("d,p", CASES)
def test_affine_mesh_through_isoparametric_path(d, p):
    m = _mesh(d, p, curved=False)
    u = mg.fourier_field(m.coords, 62)
    law = mg.Coeff("sin", (2.0, 1.0, 3.0))
    ref = orc.Oracle.of(m).assemble(u, law)
    got = orc.Oracle.of(m).set_isoparametric(True).assemble(u, law)
    for k in ("M", "K", "T", "absM", "absK", "absT"):
        assert np.abs(got[k] - ref[k]).max() <= 1e-13 * np.abs(ref[k]).max(), k


@pytest.mark.parametrize("d,p", [(2, 2), (3, 1)])
def test_constant_field_equals_constant_tensor(d, p):
    m = _mesh(d, p, curved=False)
    c = np.array([[2.0, 0.3], [0.3, 1.0]]) if d == 2 else np.array([[2.0, 0.3, 0.1], [0.3, 1.0, -0.2], [0.1, -0.2, 1.5]])
    nq = len(orc.rule(d, 2 * p)[1])
    u = mg.fourier_field(m.coords, 63)
    law = mg.Coeff("poly", (1.0, 0.5, 0.25))
    ref = orc.Oracle.of(m).set_conductivity(c).assemble(u, law)
    got = orc.Oracle.of(m).set_conductivity_field(np.broadcast_to(c, (m.n_elems, nq, d, d))).assemble(u, law)
    for k in ("M", "K", "T"):
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("d,p", CASES)
def test_curved_mesh_exact_area_and_linear_energy(d, p):
    m = _mesh(d, p)
    assert _min_det(m) > 0          # a valid (unfolded) curved mesh
    o = orc.Oracle.of(m).set_isoparametric(True)
    a = np.array([0.7, -1.3, 0.4][:d])
    u = 0.3 + m.coords @ a
    r = o.assemble(u, mg.Coeff("poly", (2.5,)), m=1.7)
    assert abs(r["M"].sum() - 1.7) <= 1e-13
    rp, ci = o.pattern()
    K = orc.csr_to_dense(rp, ci, r["K"], m.n_nodes)
    assert abs(u @ K @ u - 2.5 * (a @ a)) <= 1e-12 * 2.5 * (a @ a)
    assert np.abs(K.sum(axis=1)).max() <= 1e-12 * np.abs(K).max()
    T = orc.csr_to_dense(rp, ci, r["T"], m.n_nodes)
    assert not T.any()          # k' = 0


@pytest.mark.parametrize("d,p,curved", [(2, 2, True), (2, 1, False), (2, 3, False), (3, 1, False), (3, 2, False),
                                         (3, 3, False)])
def test_varying_field_closed_form(d, p, curved):
    """c(x) linear in x sampled at the physical points: the integrand
    a^T c(x(xhat)) a |det B| has degree p + 2(p-1) on a curved P2 triangle
    (4, exact with the 6-point rule) and degree 1 on affine elements."""
    m = _mesh(d, p, curved=curved)
    xq = _qpoints(m)
    diag = [1.0 + xq[..., 0], 2.0 - xq[..., 1]] + ([1.0 + xq[..., 2]] if d == 3 else [])
    cf = np.zeros(xq.shape[:2] + (d, d))
    for i in range(d):
        cf[..., i, i] = diag[i]
    o = orc.Oracle.of(m).set_isoparametric(curved).set_conductivity_field(cf)
    a = np.array([0.7, -1.3, 0.4][:d])
    u = m.coords @ a
    r = o.assemble(u, mg.Coeff("poly", (1.0,)))
    rp, ci = o.pattern()
    K = orc.csr_to_dense(rp, ci, r["K"], m.n_nodes)
    means = [1.5, 1.5] + ([1.5] if d == 3 else [])          # int over the unit cell of 1 + x, 2 - y, 1 + z
    exact = sum(a[i] ** 2 * means[i] for i in range(d))
    assert abs(u @ K @ u - exact) <= 1e-12 * exact
    assert np.abs(K.sum(axis=1)).max() <= 1e-12 * np.abs(K).max()


@pytest.mark.parametrize("d,p", [(2, 2), (3, 2)])
def test_rotation_invariance_with_field(d, p):
    m = _mesh(d, p)
    xq = _qpoints(m)
    cf = np.zeros(xq.shape[:2] + (d, d))
    for i in range(d):
        cf[..., i, i] = 1.0 + 0.5 * i + 0.3 * np.sin(3 * xq[..., i])
    cf[..., 0, 1] = cf[..., 1, 0] = 0.2 * xq[..., 0]
    u = mg.fourier_field(m.coords, 64)
    law = mg.Coeff("poly", (1.0, 0.5, 0.25))
    r0 = orc.Oracle.of(m).set_isoparametric(True).set_conductivity_field(cf).assemble(u, law)
    rng = np.random.default_rng(65)
    Q, R = np.linalg.qr(rng.standard_normal((d, d)))
    Q = Q * np.sign(np.diag(R))
    rot = mg.Mesh(d, p, m.coords @ Q.T + 0.25, m.conn)
    cfr = np.einsum("ab,eqbc,dc->eqad", Q, cf, Q)
    r1 = orc.Oracle.of(rot).set_isoparametric(True).set_conductivity_field(cfr).assemble(u, law)
    for k in ("M", "K", "T"):
        assert np.abs(r1[k] - r0[k]).max() <= 1e-12 * np.abs(r0[k]).max(), k


@pytest.mark.parametrize("d,p", [(2, 2), (3, 2)])
def test_curved_tangent_finite_differences(d, p):
    m = _mesh(d, p)
    o = orc.Oracle.of(m).set_isoparametric(True)
    law = mg.Coeff("poly", (1.0, 0.6, 0.3))
    u = mg.fourier_field(m.coords, 66)
    v = mg.fourier_field(m.coords, 67) - 0.5
    rp, ci = o.pattern()
    r = o.assemble(u, law)
    KT = orc.csr_to_dense(rp, ci, r["K"] + r["T"], m.n_nodes)

    def Ku(x):
        rr = o.assemble(x, law, want_abs=False)
        return orc.csr_to_dense(rp, ci, rr["K"], m.n_nodes) @ x

    h = 1e-2
    d1 = (Ku(u + h * v) - Ku(u - h * v)) / (2 * h)
    d2 = (Ku(u + 0.5 * h * v) - Ku(u - 0.5 * h * v)) / h
    fd = (4 * d2 - d1) / 3
    assert np.abs(KT @ v - fd).max() <= 1e-11 * np.abs(KT).max() * np.abs(v).max() * 10
