"""Pins of the oracle's anisotropic conductivity (Section 7: a d x d
conductivity c gives A_e = B_e^-1 c B_e^-T; here the conductivity is
k(u) c with c constant and SPD), against the mathematics: c = I is the
isotropic oracle, c = a I scales K and T by a, a rotation of the mesh with
c rotated alike leaves every matrix unchanged (which fixes where c sits
between the inverse Jacobians), the energy of a linear field is k g^T c g
|Omega|, and the tangent is the exact Newton derivative of K(u) u."""
import math

import numpy as np
import pytest

import meshgen as mg
import oracle as orc

C2 = np.array([[2.0, 0.6], [0.6, 0.8]])
C3 = np.array([[2.0, 0.5, -0.3], [0.5, 1.2, 0.4], [-0.3, 0.4, 0.9]])


def meshes():
    return [mg.structured_tri(4, 1, 0.2, seed=81), mg.structured_tri(3, 2, 0.2, seed=82),
            mg.structured_tri(2, 3, 0.2, seed=83), mg.structured_tet(2, 1, 0.15, seed=84),
            mg.structured_tet(2, 2, 0.15, seed=85)]


def cond(d):
    return C2 if d == 2 else C3


def rotation(d):
    if d == 2:
        t = 0.7
        return np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    a = np.array([1.0, 2.0, 2.0]) / 3.0                       # unit axis, angle 1.1 (Rodrigues)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(1.1) * K + (1 - math.cos(1.1)) * K @ K


LAW = mg.Coeff("poly", (1.0, 0.5, 0.25))


@pytest.mark.parametrize("mi", range(5))
def test_identity_and_scaling(mi):
    m = meshes()[mi]
    u = mg.fourier_field(m.coords, 91)
    base = orc.Oracle.of(m).assemble(u, LAW)
    ident = orc.Oracle.of(m).set_conductivity(np.eye(m.d)).assemble(u, LAW)
    for k in ("M", "K", "T"):
        assert np.array_equal(ident[k], base[k]), k
    sc = orc.Oracle.of(m).set_conductivity(2.5 * np.eye(m.d)).assemble(u, LAW)
    assert np.array_equal(sc["M"], base["M"])
    for k in ("K", "T"):
        np.testing.assert_allclose(sc[k], 2.5 * base[k], rtol=1e-13, atol=1e-13 * np.abs(base[k]).max())


@pytest.mark.parametrize("mi", range(5))
def test_rotation_invariance(mi):
    m = meshes()[mi]
    R = rotation(m.d)
    c = cond(m.d)
    u = mg.fourier_field(m.coords, 92)
    a = orc.Oracle.of(m).set_conductivity(c).assemble(u, LAW)
    mr = mg.Mesh(d=m.d, p=m.p, coords=m.coords @ R.T, conn=m.conn, name=m.name + "_rot")
    b = orc.Oracle.of(mr).set_conductivity(R @ c @ R.T).assemble(u, LAW)
    for k in ("M", "K", "T"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-11, atol=1e-12 * np.abs(a[k]).max())
    # a tensor that is not carried along changes K: the test can fail
    bad = orc.Oracle.of(mr).set_conductivity(c).assemble(u, LAW)
    assert np.abs(bad["K"] - a["K"]).max() > 1e-3 * np.abs(a["K"]).max()


@pytest.mark.parametrize("mi", range(5))
def test_linear_field_energy(mi):
    m = meshes()[mi]
    c = cond(m.d)
    g = np.array([0.7, -1.3, 0.4])[: m.d]
    u = m.coords @ g + 0.25
    o = orc.Oracle.of(m).set_conductivity(c)
    r = o.assemble(u, mg.Coeff("poly", (1.7,)))
    rp, ci = o.pattern()
    Kd = orc.csr_to_dense(rp, ci, r["K"], o.n)
    np.testing.assert_allclose(u @ Kd @ u, 1.7 * g @ c @ g, rtol=1e-12)


@pytest.mark.parametrize("mi", range(5))
def test_tangent_is_newton_derivative(mi):
    """(K(u) + T(u)) v = d/de [K(u + e v)(u + e v)] exactly (quadratic k:
    cubic along the line, Richardson combination of central differences)."""
    m = meshes()[mi]
    c = cond(m.d)
    o = orc.Oracle.of(m).set_conductivity(c)
    rp, ci = o.pattern()
    rng = np.random.default_rng(93 + mi)
    u = mg.fourier_field(m.coords, 94)
    v = rng.standard_normal(m.n_nodes)

    def G(w):
        return orc.csr_to_dense(rp, ci, o.assemble(w, LAW, want_abs=False)["K"], o.n) @ w

    def D(h):
        return (G(u + h * v) - G(u - h * v)) / (2 * h)

    fd = (4 * D(0.05) - D(0.1)) / 3
    r = o.assemble(u, LAW)
    J = orc.csr_to_dense(rp, ci, r["K"], o.n) + orc.csr_to_dense(rp, ci, r["T"], o.n)
    np.testing.assert_allclose(J @ v, fd, rtol=1e-10, atol=1e-11 * np.abs(fd).max())
