"""Pins of the P1 structure that the FP64 P1 kernels store instead of the
element matrices themselves, checked on the oracle's element matrices
(Section 3 with P1 Lagrange elements, Section 4.2):

  * M_e is the exact P1 mass matrix m |e| (1 + delta_ij) / ((d+1)(d+2)):
    one value on the diagonal, one off it;
  * K_e = b_e (sum_q w_q k(u_q)) G A_e G^T, G the constant reference
    gradients: a scalar times the element's u-independent Gram matrix,
    also with an anisotropic conductivity in A_e;
  * T_e is rank one, t_e s_e^T with t_e = b_e G A_e G^T u_e and
    s_e[j] = sum_q w_q k'(u_q) phi_q[j];
  * the degree-2 rules have one point per vertex, equal weights and basis
    values beta + gamma [j = vertex of the point].

A slip in any of these (a transposed T, a dropped weight, a mass constant
off by the factor 2 on the diagonal) fails one of them.
"""
import math

import numpy as np
import pytest

import meshgen as mg
import oracle as orc

LAWS = [mg.Coeff("sin", (2.0, 1.0, 3.0)), mg.Coeff("poly", (1.0, 0.6, 0.3))]


def _mesh(d):
    return mg.structured_tri(6, 1, 0.2, seed=91) if d == 2 else mg.structured_tet(3, 1, 0.15, seed=92)


def _G(d):
    """Reference gradients of the P1 basis, one row per node."""
    return np.vstack([-np.ones(d), np.eye(d)])


def _element_data(o, m, e, u, law):
    d = m.d
    det, A = o.geometry(e)
    b = abs(det)
    xq, wq = orc.rule(d, 2)
    phis = np.array([orc.basis(d, 1, x)[0] for x in xq])
    ue = u[m.conn[e]]
    uq = phis @ ue
    kk = np.array([orc.kfun(law.kind, law.numpy(), v) for v in uq])
    return b, A, wq, phis, ue, kk


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("law", LAWS, ids=lambda c: c.kind)
@pytest.mark.parametrize("aniso", [False, True])
def test_p1_element_matrices_factor(d, law, aniso):
    m = _mesh(d)
    o = orc.Oracle.of(m)
    if aniso:
        c = np.array([[2.0, 0.3], [0.3, 0.7]]) if d == 2 else np.array([[2.0, 0.3, 0.1], [0.3, 0.7, -0.2],
                                                                       [0.1, -0.2, 1.3]])
        o.set_conductivity(c)
    u = mg.fourier_field(m.coords, 93 + d)
    G = _G(d)
    mass = 1.7
    for e in (0, 1, m.n_elems // 2, m.n_elems - 1):
        Me, Ke, Te = o.element(e, u, law, m=mass)
        b, A, wq, phis, ue, kk = _element_data(o, m, e, u, law)
        # exact P1 mass: two values
        vol = b / math.factorial(d)
        Mex = mass * vol * (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
        assert np.allclose(Me, Mex, rtol=1e-13, atol=0), (e, Me, Mex)
        # K: scalar times the Gram matrix
        gram = G @ A @ G.T
        kap = b * float(wq @ kk[:, 0])
        scale = np.abs(Ke).max()
        assert np.abs(Ke - kap * gram).max() <= 1e-13 * scale, e
        # T: rank one, t s^T
        t = b * (G @ A @ (G.T @ ue))
        s = (wq * kk[:, 1]) @ phis
        assert np.abs(Te - np.outer(t, s)).max() <= 1e-13 * max(np.abs(Te).max(), 1e-300), e
        # a transposed T would not match (the test can tell the factors apart)
        if np.abs(Te - Te.T).max() > 1e-6 * np.abs(Te).max():
            assert np.abs(Te.T - np.outer(t, s)).max() > 1e-9 * np.abs(Te).max()


@pytest.mark.parametrize("d", [2, 3])
def test_p1_degree2_rule_one_point_per_vertex(d):
    xq, wq = orc.rule(d, 2)
    assert len(wq) == d + 1
    assert np.allclose(wq, wq[0], rtol=1e-15, atol=0)
    phis = np.array([orc.basis(d, 1, x)[0] for x in xq])
    al, be = phis.max(), phis.min()
    assert al - be > 1e-3
    hit = np.isclose(phis, al, rtol=1e-15, atol=0)
    assert np.all(hit.sum(axis=1) == 1) and np.all(hit.sum(axis=0) == 1)   # one vertex per point and vice versa
    assert np.allclose(phis[~hit], be, rtol=1e-15, atol=0)
    # the per-vertex form of u at the points: beta sum u + gamma u_vertex
    u = np.array([0.3, -1.1, 2.4, 0.7][: d + 1])
    vert = hit.argmax(axis=1)
    assert np.allclose(phis @ u, be * u.sum() + (al - be) * u[vert], rtol=1e-14, atol=1e-15)
