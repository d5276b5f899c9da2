"""Pins of the oracle's boundary terms, residual and Jacobian.

Section 5: B_ik = int_{dOmega_N} g_N'(u_h) phi_i phi_k dS is the derivative
of the boundary part of the load vector, b_i = int g_N(u_h) phi_i dS; the
implicit Euler residual is F(u) = M (u - u^s) + dt K(u) u - dt f(u) and its
Jacobian M + dt (K + T) - dt B (constant mass; T the conductivity tensor
times u).  Section 6, Experiment 2: g_N = h_c (T_a - u) + h_r (T_a^4 - u^4)
on the whole boundary.  Fixed here by:
  * boundary facet counts of the structured meshes (4N edges of an N x N
    square, 12 N^2 triangles of an N^3 cube) and the facet rule's exactness;
  * sum_ik B_ik = beta |dOmega| for g' = beta and sum_i b_i = g(c) |dOmega|
    for u = c (|dOmega| = 4 and 6: jitter moves boundary nodes tangentially);
  * closed-form boundary mass matrices assembled independently in numpy from
    boundary edges/faces found by coordinates or by counting faces: the P1
    edge matrix L/6 [2 1; 1 2], the P2 edge matrix L/30 [4 -1 2; -1 4 2;
    2 2 16], the P1 triangle matrix |T|/12 (1 + delta_ik);
  * B v = d/de b(u + e v) and J v = d/de F(u + e v), by the Richardson
    combination of central differences, exact up to rounding for these
    polynomial laws (b and F are polynomials of degree <= 4 in e);
  * F_i = 0 on interior rows for a linear u = u^s, constant k and g = 0
    (the Galerkin form reproduces the zero Laplacian of a linear field).
"""
import numpy as np
import pytest

import meshgen as mg
import oracle as orc

EXP2 = mg.Coeff("poly", (10.0 * 1000.0 + 0.8 * 5.670373e-8 * 1000.0 ** 4, -10.0, 0.0, 0.0,
                         -0.8 * 5.670373e-8))   # h_c (T_a - u) + h_r (T_a^4 - u^4), T_a = 1000


def _dense(o, vals):
    rp, ci = o.pattern()
    return orc.csr_to_dense(rp, ci, vals, o.n)


@pytest.mark.parametrize("d,p,N", [(2, 1, 5), (2, 2, 4), (2, 3, 3), (3, 1, 3), (3, 2, 2), (3, 3, 2)])
def test_boundary_facet_counts(d, p, N):
    m = mg.structured_tri(N, p, 0.2, seed=31) if d == 2 else mg.structured_tet(N, p, 0.15, seed=31)
    fe, ff = orc.Oracle.of(m).boundary_facets()
    assert len(fe) == (4 * N if d == 2 else 12 * N * N)
    assert np.all(np.diff(fe.astype(np.int64) * 4 + ff) > 0)   # ascending (element, face)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_facet_rule_exactness(p):
    x, w = orc.facet_rule(2, p)
    assert len(w) == p + 1
    for k in range(2 * p + 2):
        assert abs((w * x[:, 0] ** k).sum() - 1.0 / (k + 1)) < 1e-15
    x3, w3 = orc.facet_rule(3, p)
    assert abs(w3.sum() - 0.5) < 1e-15


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_boundary_totals(d, p):
    m = mg.structured_tri(4, p, 0.2, seed=32) if d == 2 else mg.structured_tet(2, p, 0.15, seed=32)
    o = orc.Oracle.of(m)
    area = 4.0 if d == 2 else 6.0
    r = o.boundary(np.full(m.n_nodes, 0.7), mg.Coeff("poly", (2.0, -3.0)))   # g = 2 - 3u, g' = -3
    assert abs(r["B"].sum() - (-3.0) * area) < 1e-12 * area * 3
    assert abs(r["b"].sum() - (2.0 - 3.0 * 0.7) * area) < 1e-12 * area
    assert (r["absB"] >= np.abs(r["B"]) * (1 - 1e-14)).all()


def _boundary_edges_2d(m):
    """Boundary edges of a structured unit-square mesh from coordinates: the
    vertices on each side, consecutive along it, with the P2 midpoint node."""
    X = m.coords
    nv = m.conn[:, :3]
    vert = np.unique(nv)
    edges = []
    for axis, val in ((0, 0.0), (0, 1.0), (1, 0.0), (1, 1.0)):
        on = vert[np.abs(X[vert, axis] - val) < 1e-12]
        on = on[np.argsort(X[on, 1 - axis])]
        edges += [(on[i], on[i + 1]) for i in range(len(on) - 1)]
    return edges


@pytest.mark.parametrize("p", [1, 2])
def test_closed_form_edge_mass(p):
    m = mg.structured_tri(4, p, 0.2, seed=33)
    o = orc.Oracle.of(m)
    beta = 1.7
    B = _dense(o, o.boundary(np.zeros(m.n_nodes), mg.Coeff("poly", (0.5, beta)))["B"])
    ref = np.zeros_like(B)
    mid = {}
    if p == 2:   # edge midpoint node of each element edge (local nodes 3, 4, 5: edges 01, 02, 12)
        for row in m.conn:
            for (a, b), l in zip(((0, 1), (0, 2), (1, 2)), (3, 4, 5)):
                mid[frozenset((row[a], row[b]))] = row[l]
    for a, b in _boundary_edges_2d(m):
        L = np.linalg.norm(m.coords[a] - m.coords[b])
        if p == 1:
            idx, loc = [a, b], np.array([[2.0, 1.0], [1.0, 2.0]]) * L / 6
        else:
            idx, loc = [a, b, mid[frozenset((a, b))]], np.array([[4.0, -1, 2], [-1, 4, 2], [2, 2, 16]]) * L / 30
        ref[np.ix_(idx, idx)] += beta * loc
    assert np.abs(B - ref).max() < 1e-14


def test_closed_form_triangle_mass_3d():
    m = mg.structured_tet(3, 1, 0.15, seed=34)
    o = orc.Oracle.of(m)
    beta = -2.5
    B = _dense(o, o.boundary(np.zeros(m.n_nodes), mg.Coeff("poly", (1.0, beta)))["B"])
    faces = np.sort(np.concatenate([m.conn[:, [1, 2, 3]], m.conn[:, [0, 2, 3]], m.conn[:, [0, 1, 3]],
                                    m.conn[:, [0, 1, 2]]]), axis=1)
    uniq, cnt = np.unique(faces, axis=0, return_counts=True)
    ref = np.zeros_like(B)
    for t in uniq[cnt == 1]:
        P = m.coords[t]
        area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        ref[np.ix_(t, t)] += beta * area / 12 * (np.ones((3, 3)) + np.eye(3))
    assert np.abs(B - ref).max() < 1e-14


def _richardson(f, x, v, h):
    d1 = (f(x + h * v) - f(x - h * v)) / (2 * h)
    d2 = (f(x + 0.5 * h * v) - f(x - 0.5 * h * v)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("d,p", [(2, 2), (3, 1), (3, 2)])
def test_boundary_matrix_is_derivative_of_load(d, p):
    m = mg.structured_tri(3, p, 0.2, seed=35) if d == 2 else mg.structured_tet(2, p, 0.15, seed=35)
    o = orc.Oracle.of(m)
    u = 600.0 * mg.fourier_field(m.coords, 36)        # temperatures in [0, 600]
    v = mg.fourier_field(m.coords, 37) - 0.5
    B = _dense(o, o.boundary(u, EXP2)["B"])
    fd = _richardson(lambda x: o.boundary(x, EXP2)["b"], u, v, 4.0)
    assert np.abs(B @ v - fd).max() <= 1e-9 * np.abs(B).max() * np.abs(v).max() * 10
    # a transposed or dropped g' fails: the load's derivative is not B^T v for a varying g'
    assert np.abs(B @ v).max() > 1e3 * np.abs(B @ v - fd).max()


@pytest.mark.parametrize("d,p", [(2, 2), (3, 1)])
def test_jacobian_is_derivative_of_residual(d, p):
    m = mg.structured_tri(3, p, 0.2, seed=38) if d == 2 else mg.structured_tet(2, p, 0.15, seed=38)
    o = orc.Oracle.of(m)
    k = mg.Coeff("poly", (1.5, -0.004, 3e-6))          # a quadratic k(T)
    us = 400.0 * mg.fourier_field(m.coords, 39)
    u = us + 30.0 * mg.fourier_field(m.coords, 40)
    v = mg.fourier_field(m.coords, 41) - 0.5
    dt = 10.0

    def F(x):
        r = o.assemble(x, k, m=2.4e6, want_abs=False)
        return o.residual(r["M"], r["K"], o.boundary(x, EXP2)["b"], x, us, dt)[0]

    r = o.assemble(u, k, m=2.4e6, want_abs=False)
    J = _dense(o, o.jacobian(r["M"], None, r["K"], r["T"], o.boundary(u, EXP2)["B"], dt))
    fd = _richardson(F, u, v, 2.0)
    scale = np.abs(J).max() * np.abs(v).max()
    assert np.abs(J @ v - fd).max() <= 1e-9 * scale
    # the tangent term matters here: dropping it fails the check
    J0 = _dense(o, o.jacobian(r["M"], None, r["K"], None, o.boundary(u, EXP2)["B"], dt))
    assert np.abs(J0 @ v - fd).max() > 1e3 * np.abs(J @ v - fd).max()


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_residual_interior_rows_vanish_for_linear_field(d, p):
    m = mg.structured_tri(4, p, 0.2, seed=42) if d == 2 else mg.structured_tet(3, p, 0.15, seed=42)
    o = orc.Oracle.of(m)
    g = np.array([0.3, -1.1, 0.7][:d])
    u = 0.2 + m.coords @ g
    r = o.assemble(u, mg.Coeff("poly", (2.0,)))
    F, aF = o.residual(r["M"], r["K"], None, u, u, 10.0)
    interior = np.all((m.coords > 1e-9) & (m.coords < 1 - 1e-9), axis=1)
    assert interior.sum() > 0
    assert (np.abs(F[interior]) <= 1e-12 * aF[interior]).all()
    assert np.abs(F[~interior]).max() > 1e-3      # boundary rows carry the flux
