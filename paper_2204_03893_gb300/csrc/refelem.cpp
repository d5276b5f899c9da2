// refelem.cpp -- reference-element tables of libfem (host, FP64).
//
// Quadrature (Section 3 step 4: Gaussian simplex rules): each rule is a
// set of symmetric orbits whose parameters are found by Gauss-Newton on the
// moment equations sum_q w_q xhat_q^alpha = int_That x^alpha for all
// |alpha| <= degree, starting from the published values to ~10 digits
// (triangles: Strang-Fix/Dunavant; tetrahedra: Keast).  The solved rule is
// accepted only if every moment residual is below 1e-14.
//
// Lagrange basis (Section 2: the basis of V_h; Section 3: phi_q and J_q
// evaluated once and for all): obtained by inverting the Vandermonde
// matrix of the monomials of degree <= p at the equispaced local nodes, in
// the local order of include/fem.h.
#include "refelem.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace fem {

namespace {

double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// Orbit kinds on barycentric coordinates.
enum OrbitKind { S3, S21, S111, S4, S31, S22, S211 };

struct Orbit {
    OrbitKind kind;
    int nparam;     // number of free position parameters
};

int orbit_nparam(OrbitKind k) {
    switch (k) {
        case S3: case S4: return 0;
        case S21: case S31: case S22: return 1;
        default: return 2;
    }
}

// Expand one orbit into barycentric points.
void orbit_points(OrbitKind k, const double* a, std::vector<std::vector<double>>& pts) {
    pts.clear();
    auto perms3 = [&](double x, double y, double z) {
        double t[3] = {x, y, z};
        int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        for (auto& p : P) {
            std::vector<double> v = {t[p[0]], t[p[1]], t[p[2]]};
            bool dup = false;
            for (auto& q : pts) dup = dup || q == v;
            if (!dup) pts.push_back(v);
        }
    };
    auto perms4 = [&](double x, double y, double z, double w) {
        double t[4] = {x, y, z, w};
        int idx[4] = {0, 1, 2, 3};
        // all 24 permutations by nested loops
        for (int i0 = 0; i0 < 4; ++i0)
            for (int i1 = 0; i1 < 4; ++i1)
                for (int i2 = 0; i2 < 4; ++i2)
                    for (int i3 = 0; i3 < 4; ++i3) {
                        if (i0 == i1 || i0 == i2 || i0 == i3 || i1 == i2 || i1 == i3 || i2 == i3) continue;
                        std::vector<double> v = {t[i0], t[i1], t[i2], t[i3]};
                        bool dup = false;
                        for (auto& q : pts) dup = dup || q == v;
                        if (!dup) pts.push_back(v);
                    }
        (void)idx;
    };
    switch (k) {
        case S3: perms3(1.0 / 3, 1.0 / 3, 1.0 / 3); break;
        case S21: perms3(a[0], a[0], 1.0 - 2.0 * a[0]); break;
        case S111: perms3(a[0], a[1], 1.0 - a[0] - a[1]); break;
        case S4: perms4(0.25, 0.25, 0.25, 0.25); break;
        case S31: perms4(a[0], a[0], a[0], 1.0 - 3.0 * a[0]); break;
        case S22: perms4(a[0], a[0], 0.5 - a[0], 0.5 - a[0]); break;
        case S211: perms4(a[0], a[0], a[1], 1.0 - 2.0 * a[0] - a[1]); break;
    }
}

struct RuleSpec {
    int d, deg;
    std::vector<OrbitKind> orbits;
    std::vector<double> theta;   // per orbit: params..., weight (weights for measure 1)
};

// Published starting values (about 10 digits); the solver refines them.
RuleSpec rule_spec(int d, int deg) {
    RuleSpec r;
    r.d = d;
    r.deg = deg;
    if (d == 2 && deg == 2) { r.orbits = {S21}; r.theta = {0.1666666667, 0.3333333333}; }
    else if (d == 2 && deg == 4) {
        r.orbits = {S21, S21};
        r.theta = {0.4459484909, 0.2233815897, 0.0915762135, 0.1099517437};
    } else if (d == 2 && deg == 6) {
        r.orbits = {S21, S21, S111};
        r.theta = {0.2492867452, 0.1167862757, 0.0630890145, 0.0508449064, 0.0531450498, 0.3103524510, 0.0828510756};
    } else if (d == 3 && deg == 2) { r.orbits = {S31}; r.theta = {0.1381966011, 0.25}; }
    else if (d == 3 && deg == 4) {
        r.orbits = {S4, S31, S22};
        r.theta = {-0.0789333333, 0.0714285714, 0.0457333333, 0.1005964238, 0.1493333333};
    } else if (d == 3 && deg == 6) {
        r.orbits = {S31, S31, S31, S211};
        r.theta = {0.2146028713, 0.0399227503, 0.0406739585, 0.0100772111, 0.3223378901, 0.0553571815,
                   0.0636610019, 0.2696723315, 0.0482142857};
    }
    return r;
}

void expand(const RuleSpec& r, const std::vector<double>& th, std::vector<double>& X, std::vector<double>& W) {
    X.clear();
    W.clear();
    size_t k = 0;
    std::vector<std::vector<double>> pts;
    for (OrbitKind o : r.orbits) {
        int np = orbit_nparam(o);
        orbit_points(o, &th[k], pts);
        double w = th[k + np];
        for (auto& p : pts) {
            for (int a = 0; a < r.d; ++a) X.push_back(p[a + 1]);
            W.push_back(w);
        }
        k += np + 1;
    }
}

// monomial exponents with |alpha| <= deg
std::vector<std::vector<int>> monomials(int d, int deg) {
    std::vector<std::vector<int>> out;
    if (d == 2) {
        for (int s = 0; s <= deg; ++s)
            for (int i = s; i >= 0; --i) out.push_back({i, s - i});
    } else {
        for (int s = 0; s <= deg; ++s)
            for (int i = s; i >= 0; --i)
                for (int j = s - i; j >= 0; --j) out.push_back({i, j, s - i - j});
    }
    return out;
}

double mono_exact(const std::vector<int>& al) {
    int s = 0;
    double num = 1.0;
    for (int a : al) { s += a; num *= fact(a); }
    return num / fact(s + (int)al.size());
}

void residual(const RuleSpec& r, const std::vector<double>& th, const std::vector<std::vector<int>>& mons,
              std::vector<double>& res) {
    std::vector<double> X, W;
    expand(r, th, X, W);
    double vol = 1.0 / fact(r.d);
    res.assign(mons.size(), 0.0);
    for (size_t m = 0; m < mons.size(); ++m) {
        double s = 0.0;
        for (size_t q = 0; q < W.size(); ++q) {
            double t = W[q] * vol;
            for (int a = 0; a < r.d; ++a) t *= std::pow(X[q * r.d + a], mons[m][a]);
            s += t;
        }
        res[m] = s - mono_exact(mons[m]);
    }
}

bool solve_small(std::vector<double>& A, std::vector<double>& b, int n) {
    // Gaussian elimination with partial pivoting, A n x n row-major
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r) if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
        b[c] = s / A[c * n + c];
    }
    return true;
}

bool solve_rule(int d, int deg, std::vector<double>& X, std::vector<double>& W) {
    RuleSpec r = rule_spec(d, deg);
    if (r.orbits.empty()) return false;
    auto mons = monomials(d, deg);
    std::vector<double> th = r.theta, res;
    int n = (int)th.size();
    int m = (int)mons.size();
    for (int it = 0; it < 40; ++it) {
        residual(r, th, mons, res);
        double nr = 0;
        for (double v : res) nr = std::max(nr, std::fabs(v));
        if (nr < 1e-17) break;
        // Jacobian by central differences
        std::vector<double> J((size_t)m * n), rp, rm;
        for (int k = 0; k < n; ++k) {
            double h = 1e-7 * std::max(1.0, std::fabs(th[k]));
            auto tp = th, tm = th;
            tp[k] += h;
            tm[k] -= h;
            residual(r, tp, mons, rp);
            residual(r, tm, mons, rm);
            for (int i = 0; i < m; ++i) J[(size_t)i * n + k] = (rp[i] - rm[i]) / (2 * h);
        }
        // normal equations (J^T J) delta = -J^T res
        std::vector<double> N((size_t)n * n, 0.0), g(n, 0.0);
        for (int a = 0; a < n; ++a) {
            for (int b = 0; b < n; ++b) {
                double s = 0;
                for (int i = 0; i < m; ++i) s += J[(size_t)i * n + a] * J[(size_t)i * n + b];
                N[a * n + b] = s;
            }
            double s = 0;
            for (int i = 0; i < m; ++i) s += J[(size_t)i * n + a] * res[i];
            g[a] = -s;
        }
        if (!solve_small(N, g, n)) return false;
        for (int k = 0; k < n; ++k) th[k] += g[k];
    }
    residual(r, th, mons, res);
    for (double v : res) if (!(std::fabs(v) < 1e-14)) return false;
    expand(r, th, X, W);
    double vol = 1.0 / fact(d);
    for (double& w : W) w *= vol;
    return true;
}

// Local nodes as barycentric multi-indices, local order of include/fem.h.
std::vector<std::vector<int>> local_nodes(int d, int p) {
    int nv = d + 1;
    std::vector<std::vector<int>> out;
    for (int a = 0; a < nv; ++a) {
        std::vector<int> k(nv, 0);
        k[a] = p;
        out.push_back(k);
    }
    if (p >= 2)
        for (int a = 0; a < nv; ++a)
            for (int b = a + 1; b < nv; ++b)
                for (int t = 1; t < p; ++t) {
                    std::vector<int> k(nv, 0);
                    k[a] = p - t;   // t=1: nearer a
                    k[b] = t;
                    out.push_back(k);
                }
    if (p == 3)
        for (int a = 0; a < nv; ++a)
            for (int b = a + 1; b < nv; ++b)
                for (int c = b + 1; c < nv; ++c) {
                    std::vector<int> k(nv, 0);
                    k[a] = k[b] = k[c] = 1;
                    out.push_back(k);
                }
    return out;
}


// Coefficients of the Lagrange basis in the monomials of degree <= p:
// Cm[m * np + i] = coefficient of monomial m in basis function i (the
// inverse of the Vandermonde matrix of the monomials at the local nodes).
bool basis_coefficients(int d, int p, std::vector<std::vector<int>>& mons, std::vector<double>& Cm, int& np) {
    auto nodes = local_nodes(d, p);
    np = (int)nodes.size();
    mons = monomials(d, p);
    const int nm = (int)mons.size();
    if (nm != np) return false;
    std::vector<double> V((size_t)np * nm);
    for (int i = 0; i < np; ++i)
        for (int m = 0; m < nm; ++m) {
            double v = 1.0;
            for (int a = 0; a < d; ++a) v *= std::pow((double)nodes[i][a + 1] / p, mons[m][a]);
            V[(size_t)i * nm + m] = v;
        }
    Cm.assign((size_t)nm * np, 0.0);
    for (int col = 0; col < np; ++col) {
        std::vector<double> A = V, b(np, 0.0);
        b[col] = 1.0;
        if (!solve_small(A, b, np)) return false;
        for (int m = 0; m < nm; ++m) Cm[(size_t)m * np + col] = b[m];
    }
    return true;
}

// Gauss-Legendre points and weights on [0, 1]: the roots of the Legendre
// polynomial P_n by Newton's method from the Chebyshev-like guesses
// cos(pi (i + 3/4) / (n + 1/2)), with P_n and P_n' from the three-term
// recurrence; weights 2 / ((1 - t^2) P_n'(t)^2), halved for [0, 1].
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    const double pi = 3.14159265358979323846;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double t = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 0 ? 1.0 : p1, pm = n == 0 ? 0.0 : p0;
            dp = n * (t * pn - pm) / (t * t - 1.0);
            const double dt = pn / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-17) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[n - 1 - i] = 0.5 * (1.0 + t);
        w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);
    }
}

}  // namespace

bool build_facets(int d, int p, FacetTab& F) {
    if ((d != 2 && d != 3) || p < 1 || p > 3) return false;
    std::vector<std::vector<int>> mons;
    std::vector<double> Cm;
    int np = 0;
    if (!basis_coefficients(d, p, mons, Cm, np)) return false;
    auto nodes = local_nodes(d, p);
    F.d = d;
    F.p = p;
    F.nfaces = d + 1;
    // reference facet rule: points xi (nq x (d-1)), weights
    std::vector<double> xi, w;
    if (d == 2) {
        gauss_legendre01(p + 1, xi, w);
    } else if (!solve_rule(2, 2 * p, xi, w)) {
        return false;
    }
    F.nq = (int)w.size();
    F.w = w;
    F.nf = 0;
    for (int f = 0; f <= d; ++f) {
        std::vector<int> fn;
        for (int i = 0; i < np; ++i)
            if (nodes[i][f] == 0) fn.push_back(i);
        if (f == 0) F.nf = (int)fn.size();
        if ((int)fn.size() != F.nf) return false;
        F.fnode.insert(F.fnode.end(), fn.begin(), fn.end());
        std::vector<int> wv;   // the face's vertices, ascending
        for (int a = 0; a <= d; ++a)
            if (a != f) wv.push_back(a);
        for (int q = 0; q < F.nq; ++q) {
            double mu[3];
            if (d == 2) {
                mu[0] = 1.0 - xi[q];
                mu[1] = xi[q];
            } else {
                mu[0] = 1.0 - xi[2 * q] - xi[2 * q + 1];
                mu[1] = xi[2 * q];
                mu[2] = xi[2 * q + 1];
            }
            double x[3] = {0.0, 0.0, 0.0};   // reference vertex 0 at the origin, vertex a at e_a
            for (int t = 0; t < d; ++t)
                if (wv[t] > 0) x[wv[t] - 1] += mu[t];
            for (int a = 0; a < F.nf; ++a) {
                double v = 0.0;
                for (size_t m = 0; m < mons.size(); ++m) {
                    double mv = 1.0;
                    for (int c = 0; c < d; ++c) mv *= std::pow(x[c], mons[m][c]);
                    v += Cm[m * np + fn[a]] * mv;
                }
                F.phi.push_back(v);
            }
        }
    }
    return true;
}

bool build_refelem(int d, int p, int qdeg, RefElem& R) {
    if ((d != 2 && d != 3) || p < 1 || p > 3) return false;
    if (qdeg == 0) qdeg = 2 * p;
    if (qdeg != 2 * p) return false;
    R.d = d;
    R.p = p;
    R.qdeg = qdeg;
    if (!solve_rule(d, qdeg, R.xq, R.wq)) return false;
    R.nq = (int)R.wq.size();
    auto nodes = local_nodes(d, p);
    R.np = (int)nodes.size();
    auto mons = monomials(d, p);
    int nm = (int)mons.size();
    if (nm != R.np) return false;
    // Vandermonde V[i][m] = x_i^mons[m]; basis coefficients C = V^-1 (columns)
    std::vector<double> V((size_t)R.np * nm);
    for (int i = 0; i < R.np; ++i)
        for (int m = 0; m < nm; ++m) {
            double v = 1.0;
            for (int a = 0; a < d; ++a) v *= std::pow((double)nodes[i][a + 1] / p, mons[m][a]);
            V[(size_t)i * nm + m] = v;
        }
    // invert by solving V C = I column by column
    std::vector<double> Cm((size_t)nm * R.np);
    for (int col = 0; col < R.np; ++col) {
        std::vector<double> A = V, b(R.np, 0.0);
        b[col] = 1.0;
        if (!solve_small(A, b, R.np)) return false;
        for (int m = 0; m < nm; ++m) Cm[(size_t)m * R.np + col] = b[m];   // coefficient m of basis col
    }
    R.phi.assign((size_t)R.nq * R.np, 0.0);
    R.grad.assign((size_t)R.nq * R.np * d, 0.0);
    for (int q = 0; q < R.nq; ++q) {
        const double* x = &R.xq[(size_t)q * d];
        for (int m = 0; m < nm; ++m) {
            double v = 1.0;
            for (int a = 0; a < d; ++a) v *= std::pow(x[a], mons[m][a]);
            double dv[3];
            for (int a = 0; a < d; ++a) {
                if (mons[m][a] == 0) { dv[a] = 0.0; continue; }
                double t = mons[m][a] * std::pow(x[a], mons[m][a] - 1);
                for (int c = 0; c < d; ++c) if (c != a) t *= std::pow(x[c], mons[m][c]);
                dv[a] = t;
            }
            for (int i = 0; i < R.np; ++i) {
                double c = Cm[(size_t)m * R.np + i];
                R.phi[(size_t)q * R.np + i] += c * v;
                for (int a = 0; a < d; ++a) R.grad[((size_t)q * R.np + i) * d + a] += c * dv[a];
            }
        }
    }
    // element product matrices
    int NS = d * (d + 1) / 2, NSYM = R.np * (R.np + 1) / 2, NT = R.np * R.np;
    R.ns = NS;
    R.nsym = NSYM;
    R.QM.assign((size_t)R.nq * NSYM, 0.0);
    R.QK.assign((size_t)R.nq * NS * NSYM, 0.0);
    R.QT.assign((size_t)R.nq * d * NT, 0.0);
    for (int q = 0; q < R.nq; ++q) {
        const double* ph = &R.phi[(size_t)q * R.np];
        const double* G = &R.grad[(size_t)q * R.np * d];
        for (int i = 0; i < R.np; ++i)
            for (int j = i; j < R.np; ++j) {
                int s = i * R.np - (i * (i - 1)) / 2 + (j - i);
                R.QM[(size_t)q * NSYM + s] = ph[i] * ph[j];
                int t = 0;
                for (int a = 0; a < d; ++a)
                    for (int b = a; b < d; ++b, ++t) {
                        double v = G[i * d + a] * G[j * d + b];
                        if (a != b) v += G[i * d + b] * G[j * d + a];
                        R.QK[((size_t)q * NS + t) * NSYM + s] = v;
                    }
            }
        for (int a = 0; a < d; ++a)
            for (int i = 0; i < R.np; ++i)
                for (int j = 0; j < R.np; ++j)
                    R.QT[((size_t)q * d + a) * NT + i * R.np + j] = G[i * d + a] * ph[j];
    }
    return true;
}

}  // namespace fem

#include <mutex>

namespace fem {

const FacetTab* facets_for_type(int t) {
    static std::once_flag flags[6];
    static FacetTab F[6];
    static bool ok[6] = {false, false, false, false, false, false};
    if (t < 0 || t > 5) return nullptr;
    std::call_once(flags[t], [t] { ok[t] = build_facets(t < 3 ? 2 : 3, t % 3 + 1, F[t]); });
    return ok[t] ? &F[t] : nullptr;
}

const RefElem* refelem_for_type(int t) {
    static std::once_flag flags[6];
    static RefElem R[6];
    static bool ok[6] = {false, false, false, false, false, false};
    if (t < 0 || t > 5) return nullptr;
    std::call_once(flags[t], [t] { ok[t] = build_refelem(t < 3 ? 2 : 3, t % 3 + 1, 0, R[t]); });
    return ok[t] ? &R[t] : nullptr;
}

}  // namespace fem
