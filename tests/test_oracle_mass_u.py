"""Pins of the oracle's u-dependent mass M(u) and mass-tensor term
Mt = (mass tensor) o_2 (u - us) (Sections 2, 5 and 5.1), against the
mathematics: a constant coefficient reduces M(u) to the already pinned
mass matrix and Mt to 0; a constant field gives closed forms; the Newton
derivative of M(u)(u - us) is M(u) + Mt exactly (Richardson combination of
central differences, exact for a residual that is cubic along a line);
both matrices are symmetric."""
import numpy as np
import pytest

import meshgen as mg
import oracle as orc


def meshes():
    return [mg.structured_tri(4, 1, 0.2, seed=11), mg.structured_tri(3, 2, 0.2, seed=12),
            mg.structured_tri(2, 3, 0.2, seed=13), mg.structured_tet(2, 1, 0.15, seed=14),
            mg.structured_tet(2, 2, 0.15, seed=15)]


def dense(o, vals):
    rp, ci = o.pattern()
    return orc.csr_to_dense(rp, ci, vals, o.n)


@pytest.mark.parametrize("mi", range(5))
def test_constant_coefficient_reduces_to_mass(mi):
    m = meshes()[mi]
    o = orc.Oracle.of(m)
    u = mg.fourier_field(m.coords, 21)
    r = o.assemble_mass_u(u, 0.7 * u, mg.Coeff("poly", (2.5,)))
    M1 = o.assemble(u, mg.Coeff("poly", (1.0,)), m=1.0)["M"]
    np.testing.assert_allclose(r["Mu"], 2.5 * M1, rtol=1e-13, atol=1e-15)
    assert abs(r["Mu"].sum() - 2.5) < 1e-13                 # sum of M = m |Omega|, |Omega| = 1
    assert np.all(r["Mt"] == 0.0)                            # m' = 0


@pytest.mark.parametrize("mi", range(5))
def test_constant_field_closed_forms(mi):
    """u = c, us = c - d: u_h = c and z_h = d, so M(u) = m(c) M_1 and
    Mt = m'(c) d M_1 (the basis sums to one), sum(Mt) = m'(c) d |Omega|."""
    m = meshes()[mi]
    o = orc.Oracle.of(m)
    c, d = 0.6, 0.25
    u = np.full(m.n_nodes, c)
    law = mg.Coeff("poly", (1.0, 0.5, 0.3))
    mc, dmc = 1.0 + 0.5 * c + 0.3 * c * c, 0.5 + 0.6 * c
    r = o.assemble_mass_u(u, u - d, law)
    M1 = o.assemble(u, mg.Coeff("poly", (1.0,)), m=1.0)["M"]
    np.testing.assert_allclose(r["Mu"], mc * M1, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["Mt"], dmc * d * M1, rtol=1e-12, atol=1e-15)
    assert abs(r["Mt"].sum() - dmc * d) < 1e-12


@pytest.mark.parametrize("mi", range(5))
def test_newton_derivative_exact(mi):
    """d/de [M(u + e v)(u + e v - us)] at e = 0 equals (M(u) + Mt) v; for a
    quadratic m the left side is cubic in e, so (4 D(h/2) - D(h)) / 3 of the
    central differences D is exact up to rounding."""
    m = meshes()[mi]
    o = orc.Oracle.of(m)
    rng = np.random.default_rng(30 + mi)
    u = mg.fourier_field(m.coords, 31)
    us = u - 0.1 * rng.standard_normal(m.n_nodes)
    v = rng.standard_normal(m.n_nodes)
    law = mg.Coeff("poly", (1.0, 0.8, -0.4))

    def G(w):
        return dense(o, o.assemble_mass_u(w, None, law)["Mu"]) @ (w - us)

    def D(h):
        return (G(u + h * v) - G(u - h * v)) / (2 * h)

    fd = (4 * D(0.05) - D(0.1)) / 3
    r = o.assemble_mass_u(u, us, law)
    J = dense(o, r["Mu"]) + dense(o, r["Mt"])
    np.testing.assert_allclose(J @ v, fd, rtol=1e-10, atol=1e-11 * np.abs(fd).max())
    # a dropped or mis-scaled tensor term fails it
    assert np.abs(dense(o, r["Mt"]) @ v).max() > 1e-3 * np.abs(fd).max()


@pytest.mark.parametrize("mi", range(5))
def test_symmetric(mi):
    m = meshes()[mi]
    o = orc.Oracle.of(m)
    u = mg.fourier_field(m.coords, 41)
    r = o.assemble_mass_u(u, 0.5 * u, mg.Coeff("sin", (2.0, 1.0, 3.0)))
    for k in ("Mu", "Mt"):
        A = dense(o, r[k])
        np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-15 * np.abs(A).max())
