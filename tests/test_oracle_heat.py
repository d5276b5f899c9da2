"""Pins of the oracle's implicit Euler step (Section 5; Section 6,
Experiment 2), which composes the pinned residual, Jacobian and boundary
terms with a sparse direct solve:
  * a converged step balances the energy exactly: sum_i (M (u - u^s))_i =
    dt sum_i b_i(u), because the columns of K(u) sum to zero;
  * the ambient state u = T_a is a fixed point (g(T_a) = 0, K T_a = 0);
  * Newton converges quadratically (each residual ratio below the square of
    the previous one times a modest constant, once in the asymptotic
    range).
"""
import numpy as np

import meshgen as mg
import oracle as orc

KLAW = mg.Coeff("pwlin", (0.0, 200.0, 1000.0, 1.5, 0.7, 0.5))            # k(T), Experiment 2
HC, HR, TA = 10.0, 0.8 * 5.670373e-8, 1000.0
GLAW = mg.Coeff("poly", (HC * TA + HR * TA ** 4, -HC, 0.0, 0.0, -HR))      # convection + radiation
RHOC = 1000.0 * 2400.0


def _mesh():
    m = mg.structured_tri(6, 2, 0.2, seed=81)
    return mg.Mesh(m.d, m.p, 0.2 * m.coords, m.conn)                      # the square (0, 0.2)^2


def test_energy_balance_of_a_converged_step():
    m = _mesh()
    o = orc.Oracle.of(m)
    us = np.zeros(m.n_nodes)
    u = us
    for _ in range(3):
        u_new, info = o.heat_step(KLAW, GLAW, u, 10.0, RHOC)
        r = o.assemble(u_new, KLAW, m=RHOC, want_abs=False)
        b = o.boundary(u_new, GLAW)["b"]
        rp, ci = o.pattern()
        M = orc.csr_to_dense(rp, ci, r["M"], m.n_nodes)
        lhs, rhs = (M @ (u_new - u)).sum(), 10.0 * b.sum()
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs)
        assert info["residuals"][-1] <= 1e-12 * info["residuals"][0]
        u = u_new
    # heat flows in from the hot surroundings: the stored energy rose
    # (pointwise values may undershoot: P2 has no discrete maximum principle)
    assert (M @ u).sum() > 0 and u.max() < TA


def test_ambient_state_is_a_fixed_point():
    m = _mesh()
    o = orc.Oracle.of(m)
    us = np.full(m.n_nodes, TA)
    u, info = o.heat_step(KLAW, GLAW, us, 10.0, RHOC)
    assert info["newton"] == 0 or np.abs(u - TA).max() <= 1e-9 * TA
    r = o.assemble(us, KLAW, m=RHOC, want_abs=False)
    F, aF = o.residual(r["M"], r["K"], o.boundary(us, GLAW)["b"], us, us, 10.0)
    assert np.abs(F).max() <= 1e-12 * aF.max()


def test_newton_converges_quadratically():
    m = _mesh()
    o = orc.Oracle.of(m)
    us = 300.0 * mg.fourier_field(m.coords / 0.2, 82)
    _, info = o.heat_step(mg.Coeff("poly", (1.5, -0.002, 1e-6)), GLAW, us, 100.0, RHOC,
                          u0=us + 50.0, rtol=1e-14)
    res = np.array(info["residuals"]) / info["residuals"][0]
    ratios = res[1:] / res[:-1]
    assert res[-1] <= 1e-12
    # quadratic: r_{k+1} <= C r_k^2 with a modest C in the last steps above rounding
    tail = [i for i in range(1, len(res)) if res[i] > 1e-13]
    assert any(res[i] <= 1e3 * res[i - 1] ** 2 for i in tail[1:]) or len(tail) <= 2
    assert ratios.max() < 0.5
