"""Pins of the CPU oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: exact
monomial integrals, exact rational reference matrices (sympy), closed-form
element matrices, conservation identities, finite differences, closed-form
nonzero counts and hand-enumerated patterns.  A plausible slip in the oracle
(a dropped weight, a transposed tangent, a wrong A_e = (B^T B)^-1, a wrong
basis gradient) fails at least one of them.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import meshgen as mg
import oracle as orc

RULES = [(2, 2, 3), (2, 4, 6), (2, 6, 12), (3, 2, 4), (3, 4, 11), (3, 6, 24)]
TYPES = [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)]


def mono_exact(alpha):
    """Integral of x^alpha over the reference simplex: prod(alpha_i!) / (|alpha|+d)!"""
    d = len(alpha)
    return math.prod(math.factorial(a) for a in alpha) / math.factorial(sum(alpha) + d)


# ---------------------------------------------------------------- P1 quadrature
@pytest.mark.parametrize("d,deg,nq", RULES)
def test_quadrature_exactness(d, deg, nq):
    x, w = orc.rule(d, deg)
    assert len(w) == nq
    assert abs(w.sum() - 1.0 / math.factorial(d)) < 1e-15
    for alpha in itertools.product(range(deg + 1), repeat=d):
        if sum(alpha) > deg:
            continue
        q = np.sum(w * np.prod(x ** np.array(alpha), axis=1))
        assert abs(q - mono_exact(alpha)) < 2e-15, (alpha, q, mono_exact(alpha))
    # points inside the simplex
    assert (x > 0).all() and (x.sum(1) < 1).all()


@pytest.mark.parametrize("d,deg,nq", RULES)
def test_quadrature_not_exact_beyond_degree(d, deg, nq):
    """The rule has exactly the stated degree (some monomial of degree+1 fails)."""
    x, w = orc.rule(d, deg)
    worst = 0.0
    for alpha in itertools.product(range(deg + 2), repeat=d):
        if sum(alpha) != deg + 1:
            continue
        q = np.sum(w * np.prod(x ** np.array(alpha), axis=1))
        worst = max(worst, abs(q - mono_exact(alpha)))
    assert worst > 1e-8


# ---------------------------------------------------------------- P2 basis
def ref_nodes(d, p):
    K = mg.local_nodes(d, p)
    return K[:, 1:].astype(float) / p


@pytest.mark.parametrize("d,p", TYPES)
def test_basis_kronecker_and_partition(d, p):
    X = ref_nodes(d, p)
    n = X.shape[0]
    for j in range(n):
        phi, g = orc.basis(d, p, X[j])
        np.testing.assert_allclose(phi, np.eye(n)[j], atol=1e-14)
    rng = np.random.default_rng(7)
    for _ in range(20):
        x = rng.dirichlet(np.ones(d + 1))[1:]
        phi, g = orc.basis(d, p, x)
        assert abs(phi.sum() - 1) < 1e-14
        np.testing.assert_allclose(g.sum(0), 0, atol=1e-13)
        # gradients against central differences of the values
        h = 1e-6
        for a in range(d):
            e = np.zeros(d)
            e[a] = h
            fd = (orc.basis(d, p, x + e)[0] - orc.basis(d, p, x - e)[0]) / (2 * h)
            np.testing.assert_allclose(g[:, a], fd, atol=1e-8)


@pytest.mark.parametrize("d,p", TYPES)
def test_basis_reproduces_polynomials(d, p):
    """sum_i f(x_i) phi_i(x) = f(x) for every polynomial f of degree <= p."""
    X = ref_nodes(d, p)
    rng = np.random.default_rng(3)
    for alpha in itertools.product(range(p + 1), repeat=d):
        if sum(alpha) > p:
            continue
        fvals = np.prod(X ** np.array(alpha), axis=1)
        for _ in range(5):
            x = rng.dirichlet(np.ones(d + 1))[1:]
            phi, _ = orc.basis(d, p, x)
            assert abs(phi @ fvals - np.prod(x ** np.array(alpha))) < 1e-13


# ---------------------------------------------------------------- P3 exact matrices
def exact_reference_matrices(d, p):
    """Exact rational reference mass matrix and gradient Gram matrices
    G_ab[i][j] = int d_a phi_i d_b phi_j, from a Lagrange basis obtained by
    solving the Vandermonde system in exact arithmetic (sympy)."""
    import sympy as sp
    xs = sp.symbols("x0:%d" % d)
    K = mg.local_nodes(d, p)
    nodes = [[sp.Rational(int(K[i, a + 1]), p) for a in range(d)] for i in range(K.shape[0])]
    monos = [m for m in itertools.product(range(p + 1), repeat=d) if sum(m) <= p]
    V = sp.Matrix([[sp.prod([nd[a] ** m[a] for a in range(d)]) for m in monos] for nd in nodes])
    Cm = V.inv()  # column i: coefficients of basis i
    basis = [sum(Cm[k, i] * sp.prod([xs[a] ** monos[k][a] for a in range(d)]) for k in range(len(monos)))
             for i in range(len(nodes))]

    def integ(expr):
        poly = sp.Poly(sp.expand(expr), *xs)
        tot = sp.Integer(0)
        for mon, coef in poly.terms():
            tot += coef * sp.Rational(math.prod(math.factorial(a) for a in mon), math.factorial(sum(mon) + d))
        return tot

    n = len(basis)
    Mref = [[integ(basis[i] * basis[j]) for j in range(n)] for i in range(n)]
    grads = [[sp.diff(b, xs[a]) for a in range(d)] for b in basis]
    G = {}
    for a in range(d):
        for b in range(d):
            G[a, b] = [[integ(grads[i][a] * grads[j][b]) for j in range(n)] for i in range(n)]
    to = lambda m: np.array([[float(v) for v in row] for row in m])
    return to(Mref), {k: to(v) for k, v in G.items()}


def single_element(d, p, verts):
    """One element with the given vertices, higher-order nodes at affine positions."""
    K = mg.local_nodes(d, p).astype(float) / p
    coords = K @ np.asarray(verts, dtype=float)
    conn = np.arange(K.shape[0], dtype=np.int32)[None, :]
    return coords, conn


CONST1 = mg.Coeff("poly", (1.0, 0.0, 0.0, 0.0, 0.0))


@pytest.mark.parametrize("d,p", TYPES)
def test_exact_reference_matrices(d, p):
    """Element mass / stiffness on reference and on a random affine element
    equal the exact rational matrices mapped by |det B| and A = (B^T B)^-1
    (rule degree 2p integrates the mass exactly and the constant-k stiffness)."""
    Mref, G = exact_reference_matrices(d, p)
    ref = np.vstack([np.zeros(d), np.eye(d)])
    rng = np.random.default_rng(11)
    for verts in (ref, ref + rng.uniform(-0.2, 0.2, ref.shape)):
        coords, conn = single_element(d, p, verts)
        o = orc.Oracle(d, p, coords, conn)
        Me, Ke, Te = o.element(0, np.zeros(coords.shape[0]), CONST1, m=1.0)
        B = (verts[1:] - verts[0]).T
        b = abs(np.linalg.det(B))
        A = np.linalg.inv(B.T @ B)
        Kexp = sum(A[a, c] * G[a, c] for a in range(d) for c in range(d)) * b
        np.testing.assert_allclose(Me, b * Mref, rtol=0, atol=1e-14 * max(1, np.abs(Mref).max()))
        np.testing.assert_allclose(Ke, Kexp, rtol=0, atol=2e-13 * np.abs(Kexp).max())
        np.testing.assert_allclose(Te, 0, atol=0)


@pytest.mark.parametrize("d", [2, 3])
def test_p1_mass_closed_form(d):
    """P1 element mass = |T|/12 (1+delta_ij) in 2D, |T|/20 (1+delta_ij) in 3D."""
    rng = np.random.default_rng(5)
    verts = np.vstack([np.zeros(d), np.eye(d)]) + rng.uniform(-0.2, 0.2, (d + 1, d))
    coords, conn = single_element(d, 1, verts)
    o = orc.Oracle(d, 1, coords, conn)
    Me, _, _ = o.element(0, np.zeros(d + 1), CONST1, m=1.0)
    vol = abs(np.linalg.det((verts[1:] - verts[0]).T)) / math.factorial(d)
    den = 12.0 if d == 2 else 20.0
    np.testing.assert_allclose(Me, vol / den * (1 + np.eye(d + 1)), rtol=1e-14)


# ---------------------------------------------------------------- P4, P5 conservation
def small_mesh(d, p, N=None, seed=0):
    if d == 2:
        return mg.structured_tri(N or 4, p, 0.2, seed=seed)
    return mg.structured_tet(N or 2, p, 0.15, seed=seed)


@pytest.mark.parametrize("d,p", TYPES)
def test_mass_total_and_stiffness_rows(d, p):
    m = small_mesh(d, p)
    o = orc.Oracle.of(m)
    rng = np.random.default_rng(1)
    u = rng.uniform(0, 1, m.n_nodes)
    coeff = mg.Coeff("poly", (1.0, 0.5, 0.25, 0.0, 0.0))
    r = o.assemble(u, coeff, m=2.5)
    assert abs(r["M"].sum() - 2.5) < 1e-13          # m |Omega|, |Omega| = 1
    rp, ci = o.pattern()
    for row in range(m.n_nodes):
        sl = slice(rp[row], rp[row + 1])
        assert abs(r["K"][sl].sum()) <= 1e-13 * r["absK"][sl].sum()
    # tangent columns sum to zero: sum_i T_ik = int k' phi_k grad u . grad(sum_i phi_i) = 0
    colsum = np.zeros(m.n_nodes)
    colabs = np.zeros(m.n_nodes)
    np.add.at(colsum, ci, r["T"])
    np.add.at(colabs, ci, r["absT"])
    assert (np.abs(colsum) <= 1e-12 * colabs + 1e-300).all()


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_constant_u(d, p):
    """u == c: T = 0 and K(u) = k(c) K_1 (K_1: the k == 1 matrix)."""
    m = small_mesh(d, p)
    o = orc.Oracle.of(m)
    c = 0.37
    coeff = mg.Coeff("sin", (2.0, 1.0, 3.0))
    r = o.assemble(np.full(m.n_nodes, c), coeff)
    r1 = o.assemble(np.zeros(m.n_nodes), CONST1)
    assert np.abs(r["T"]).max() < 1e-13 * np.abs(r["K"]).max()
    np.testing.assert_allclose(r["K"], (2.0 + math.sin(3 * c)) * r1["K"], rtol=0,
                               atol=1e-13 * np.abs(r1["K"]).max())


# ---------------------------------------------------------------- P6 tangent by finite differences
def KU(o, u, coeff):
    rp, ci = o.pattern()
    K = o.assemble(u, coeff, want_abs=False)["K"]
    y = np.zeros(o.n)
    for r in range(o.n):
        y[r] = K[rp[r]:rp[r + 1]] @ u[ci[rp[r]:rp[r + 1]]]
    return y


def matvec(o, vals, v):
    rp, ci = o.pattern()
    return np.array([vals[rp[r]:rp[r + 1]] @ v[ci[rp[r]:rp[r + 1]]] for r in range(o.n)])


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_tangent_fd_polynomial_exact(d, p):
    """(K(u)+T(u)) v = d/de [K(u+ev)(u+ev)]; for quadratic k the map is a
    cubic in e, so the Richardson combination of central differences is exact."""
    m = small_mesh(d, p, N=3 if d == 2 else 2)
    o = orc.Oracle.of(m)
    rng = np.random.default_rng(2)
    u = rng.uniform(0, 1, m.n_nodes)
    v = rng.uniform(-1, 1, m.n_nodes)
    coeff = mg.Coeff("poly", (1.0, 0.5, 0.25, 0.0, 0.0))
    r = o.assemble(u, coeff)
    lhs = matvec(o, r["K"] + r["T"], v)

    def D(h):
        return (KU(o, u + h * v, coeff) - KU(o, u - h * v, coeff)) / (2 * h)

    h = 0.5
    fd = (4 * D(h / 2) - D(h)) / 3
    assert np.abs(lhs - fd).max() <= 1e-11 * np.abs(lhs).max()
    # transposing T breaks it
    rp, ci = o.pattern()
    Td = orc.csr_to_dense(rp, ci, r["T"], o.n)
    lhs_t = matvec(o, r["K"], v) + Td.T @ v
    assert np.abs(lhs_t - fd).max() > 1e-6 * np.abs(lhs).max()


def test_tangent_fd_sin():
    m = small_mesh(2, 2, N=3)
    o = orc.Oracle.of(m)
    rng = np.random.default_rng(4)
    u = rng.uniform(0, 1, m.n_nodes)
    v = rng.uniform(-1, 1, m.n_nodes)
    coeff = mg.Coeff("sin", (2.0, 1.0, 3.0))
    r = o.assemble(u, coeff)
    lhs = matvec(o, r["K"] + r["T"], v)
    h = 1e-4
    fd = (KU(o, u + h * v, coeff) - KU(o, u - h * v, coeff)) / (2 * h)
    assert np.abs(lhs - fd).max() <= 1e-7 * np.abs(lhs).max()


def test_tangent_fd_pwlin():
    """Piecewise-linear k with all u inside one branch: quadratic in e, exact FD."""
    m = small_mesh(2, 1, N=3)
    o = orc.Oracle.of(m)
    rng = np.random.default_rng(8)
    u = rng.uniform(250, 900, m.n_nodes)      # inside (200, 1000]
    v = rng.uniform(-1, 1, m.n_nodes)
    coeff = mg.Coeff("pwlin", (0.0, 200.0, 1000.0, 1.5, 0.7, 0.5))
    r = o.assemble(u, coeff)
    lhs = matvec(o, r["K"] + r["T"], v)
    h = 1.0
    fd = (KU(o, u + h * v, coeff) - KU(o, u - h * v, coeff)) / (2 * h)
    assert np.abs(lhs - fd).max() <= 1e-10 * np.abs(lhs).max()


def test_kfun_branches():
    pw = (0.0, 200.0, 1000.0, 1.5, 0.7, 0.5)
    assert orc.kfun("pwlin", pw, -5.0) == (1.5, 0.0)
    assert orc.kfun("pwlin", pw, 0.0) == (1.5, pytest.approx(-0.004))
    assert orc.kfun("pwlin", pw, 200.0)[0] == pytest.approx(0.7)
    assert orc.kfun("pwlin", pw, 200.0)[1] == pytest.approx(-0.004)    # T2 in the first branch
    assert orc.kfun("pwlin", pw, 600.0) == (pytest.approx(0.6), pytest.approx(-0.00025))
    assert orc.kfun("pwlin", pw, 2000.0) == (0.5, 0.0)
    v, dv = orc.kfun("poly", (1.0, 0.5, 0.25, 0, 0), 2.0)
    assert (v, dv) == (3.0, 1.5)
    v, dv = orc.kfun("sin", (2.0, 1.0, 3.0), 0.5)
    assert v == pytest.approx(2 + math.sin(1.5)) and dv == pytest.approx(3 * math.cos(1.5))


# ---------------------------------------------------------------- P7 energy of a linear field
@pytest.mark.parametrize("d,p", TYPES)
def test_linear_field_energy(d, p):
    m = small_mesh(d, p)
    o = orc.Oracle.of(m)
    g = np.array([0.7, -1.3, 0.4][:d])
    u = m.coords @ g + 0.25
    kc = 1.75
    r = o.assemble(u, mg.Coeff("poly", (kc, 0, 0, 0, 0)), want_abs=False)
    e = u @ matvec(o, r["K"], u)
    assert abs(e - kc * (g @ g)) < 1e-12 * kc * (g @ g)


# ---------------------------------------------------------------- P8 config-1 exactness
def test_p1_quadratic_k_closed_form():
    """P1, k = 1 + 0.5u + 0.25u^2, 3-point degree-2 rule integrates exactly:
    K_e = (grad phi_i . grad phi_j) int_T k(u_h),
    T_e = (grad phi_i . grad u_h) int_T k'(u_h) phi_j."""
    m = mg.structured_tri(6, 1, 0.2, seed=9)
    rng = np.random.default_rng(10)
    u = rng.uniform(0, 1, m.n_nodes)
    coeff = mg.Coeff("poly", (1.0, 0.5, 0.25, 0.0, 0.0))
    o = orc.Oracle.of(m)
    for e in range(0, m.n_elems, 7):
        v = m.conn[e]
        X = m.coords[v]
        # barycentric gradients from the affine interpolation system (independent of B^-1)
        Vm = np.hstack([np.ones((3, 1)), X])
        coefs = np.linalg.solve(Vm, np.eye(3))     # column i: [c0, cx, cy] of lambda_i
        grads = coefs[1:, :].T                      # (3, 2)
        area = 0.5 * abs(np.linalg.det(Vm))
        ue = u[v]
        ik = area * (1 + 0.5 * ue.mean() + 0.25 * ((ue ** 2).sum() + ue.sum() ** 2) / 12)
        Kexp = grads @ grads.T * ik
        gu = grads.T @ ue
        ikp = np.array([0.5 * area / 3 + 0.5 * area / 12 * (ue.sum() + ue[j]) for j in range(3)])
        Texp = np.outer(grads @ gu, ikp)
        Me, Ke, Te = o.element(e, u, coeff)
        np.testing.assert_allclose(Ke, Kexp, rtol=0, atol=1e-13 * np.abs(Kexp).max())
        np.testing.assert_allclose(Te, Texp, rtol=0, atol=1e-13 * np.abs(Texp).max())


# ---------------------------------------------------------------- P9 pattern
NNZ = {
    (2, 1): lambda N: 7 * N * N + 6 * N + 1,
    (2, 2): lambda N: 46 * N * N + 16 * N + 1,
    (3, 1): lambda N: 15 * N ** 3 + 21 * N ** 2 + 9 * N + 1,
    (3, 2): lambda N: 230 * N ** 3 + 138 * N ** 2 + 24 * N + 1,
}


@pytest.mark.parametrize("d,p", list(NNZ))
def test_pattern_nnz_polynomial(d, p):
    for N in ((3, 5, 8) if d == 2 else (2, 3, 4)):
        m = mg.structured_tri(N, p) if d == 2 else mg.structured_tet(N, p)
        o = orc.Oracle.of(m)
        assert o.nnz() == NNZ[d, p](N)
        rp, ci = o.pattern()
        for r in range(m.n_nodes):
            row = ci[rp[r]:rp[r + 1]]
            assert (np.diff(row) > 0).all() and r in row


def test_pattern_two_triangles_by_hand():
    """Unit square, one cell: triangles (0,1,3), (0,3,2): every pair but {1,2}."""
    m = mg.structured_tri(1, 1, 0.0)
    assert m.conn.tolist() == [[0, 1, 3], [0, 3, 2]]
    rp, ci = orc.Oracle.of(m).pattern()
    D = np.zeros((4, 4), dtype=int)
    for r in range(4):
        D[r, ci[rp[r]:rp[r + 1]]] = 1
    exp = np.ones((4, 4), dtype=int)
    exp[1, 2] = exp[2, 1] = 0
    assert (D == exp).all()


def test_pattern_single_p2_tet_full():
    coords, conn = single_element(3, 2, np.vstack([np.zeros(3), np.eye(3)]))
    rp, ci = orc.Oracle(3, 2, coords, conn).pattern()
    assert len(ci) == 100 and (np.diff(rp) == 10).all()


def test_entries_match_full_assembly():
    m = mg.structured_tri(5, 2, 0.2, seed=3)
    o = orc.Oracle.of(m)
    u = mg.fourier_field(m.coords, 5)
    coeff = mg.Coeff("poly", (1.0, 0.0, 1.0, 0.0, 0.0))
    r = o.assemble(u, coeff)
    rp, ci = o.pattern()
    rows = np.repeat(np.arange(m.n_nodes), np.diff(rp))
    sel = np.arange(0, len(ci), 3)
    s = o.entries(rows[sel], ci[sel], u, coeff)
    for k in ("M", "K", "T", "absK"):
        assert np.array_equal(s[k], r[k][sel])     # same order of summation: bit-identical


@pytest.mark.parametrize("name", ["tri_p2", "tet_p1"])
def test_multicore_oracle_same_bits(name):
    """The multi-core timing variant forms the element matrices in parallel
    and adds them in the same element order: identical bits."""
    mesh = mg.structured_tri(7, 2, 0.2, seed=21) if name == "tri_p2" else mg.structured_tet(4, 1, 0.15, seed=22)
    o = orc.Oracle.of(mesh)
    u = mg.fourier_field(mesh.coords, 23)
    law = mg.Coeff("sin", (2.0, 1.0, 3.0))
    ref = o.assemble(u, law, want_abs=False)
    got, used = o.assemble_mt(u, law, threads=3)
    assert used >= 1
    for k in ("M", "K", "T"):
        assert np.array_equal(got[k], ref[k]), k
