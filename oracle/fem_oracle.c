/*
 * fem_oracle.c -- plain, slow, obviously correct CPU reference (FP64) for
 * the assembly of the mass matrix M, the conductivity matrix K(u) and the
 * Newton tangent term T(u) of a scalar heat-type problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg load it.  It shares no code, header or table with the CUDA
 * library: its quadrature tables, Lagrange basis and sparsity-pattern
 * construction are written here independently.
 *
 * What it computes (Voet, "On the fast assemblage of finite element
 * matrices with application to nonlinear heat transfer problems"):
 *
 *   - Algorithm 1 (classical assemblage, Section 3): a loop over elements
 *     e, an inner loop over quadrature nodes q, dense local matrices
 *         M_e += w_q m   phi_q phi_q^T        |det B_e|
 *         K_e += w_q k_q J_q A_e J_q^T        |det B_e|,  A_e = (B_e^T B_e)^-1
 *     (Section 3, steps 3-4, the formulas as implemented), then
 *     M(N_e,N_e) += M_e, K(N_e,N_e) += K_e.
 *   - The tangent term: the conductivity tensor of Section 5.2,
 *         C_e = sum_q w_q k'_q (J_q A_e J_q^T) o phi_q |det B_e|,
 *     multiplied by u in its second mode (Section 5, the Jacobian
 *     dF/du contains  (conductivity tensor) o_2 u):
 *         T_e[i][k] = sum_j C_e[i][j][k] u_e[j]
 *                   = sum_q w_q k'_q |det B_e| (S_q u_e)[i] phi_q[k],
 *     with S_q = J_q A_e J_q^T; row i is the test function, column k the
 *     trial direction.
 *   - The u-dependent mass M(u) (m = m(u_h)) and the Section 5.1 mass
 *     tensor multiplied by u - u^s in its second mode (oracle_assemble_mass_u).
 *   - B_e = [x_1 - x_0, ..., x_d - x_0] (Section 3 step 3, affine map).
 *   - Global assembly: every (row, col) pair of nodes that share an element
 *     is a structural nonzero (Section 3 step 2); contributions are added in
 *     ascending element order, then ascending local row, local column.
 *   - Error scale per CSR entry (absM/absK/absT): the sum over elements and
 *     quadrature nodes of the magnitudes of the expanded product terms, the
 *     natural bound for a floating-point evaluation of the same sum in any
 *     order (entries that cancel exactly, such as P2 vertex/adjacent-edge
 *     mass entries, keep a nonzero scale).
 *
 * Quadrature rules (Section 3 step 4 cites Gaussian simplex rules; weights
 * here sum to the reference measure 1/2 or 1/6):
 *   triangle: 3 points degree 2, 6 points degree 4, 12 points degree 6;
 *   tetrahedron: 4 points degree 2, 11 points degree 4, 24 points degree 6.
 * Lagrange basis on equispaced nodes, written with barycentric formulas.
 *
 * Local node order (input convention): vertices; edge nodes, edges in
 * lexicographic order of vertex pairs (a<b), for p=3 the node nearer a first;
 * face nodes (p=3), faces in lexicographic order of vertex triples.
 *
 * Conductivity laws: 0 = polynomial sum_i c_i u^i (up to 5 coefficients),
 * 1 = alpha + beta sin(gamma u), 2 = piecewise linear through m knots
 * (constant outside, the left knot of the first branch included in it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXNP 20
#define OR_MAXQ 24

/* ------------------------------------------------------------------ */
/* Quadrature: symmetric orbits on the reference simplex               */
/* ------------------------------------------------------------------ */

static int push_pt(double* xq, double* wq, int n, int d, const double* lam, double w) {
    /* lam: barycentric coordinates (d+1); reference coordinates = lam[1..d] */
    for (int a = 0; a < d; ++a) xq[n * d + a] = lam[a + 1];
    wq[n] = w;
    return n + 1;
}

/* all distinct permutations of a barycentric tuple */
static int push_orbit(double* xq, double* wq, int n, int d, const double* base, double w) {
    int nv = d + 1;
    int idx[4] = {0, 1, 2, 3};
    /* enumerate all permutations of nv items, keep distinct tuples */
    double seen[24][4];
    int nseen = 0;
    int perm[24][4];
    int np = 0;
    if (nv == 3) {
        int P[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
        for (int k = 0; k < 6; ++k) { for (int a = 0; a < 3; ++a) perm[np][a] = P[k][a]; ++np; }
    } else {
        for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) for (int c = 0; c < 4; ++c) for (int e = 0; e < 4; ++e) {
            if (a == b || a == c || a == e || b == c || b == e || c == e) continue;
            perm[np][0] = a; perm[np][1] = b; perm[np][2] = c; perm[np][3] = e; ++np;
        }
    }
    (void)idx;
    for (int k = 0; k < np; ++k) {
        double t[4];
        for (int a = 0; a < nv; ++a) t[a] = base[perm[k][a]];
        int dup = 0;
        for (int s = 0; s < nseen && !dup; ++s) {
            int same = 1;
            for (int a = 0; a < nv; ++a) if (seen[s][a] != t[a]) { same = 0; break; }
            dup = same;
        }
        if (dup) continue;
        for (int a = 0; a < nv; ++a) seen[nseen][a] = t[a];
        ++nseen;
        n = push_pt(xq, wq, n, d, t, w);
    }
    return n;
}

/* Returns the number of points of the rule of the given degree (2, 4 or 6),
 * or -1.  xq (n x d) and wq (n) may be NULL to query the size. */
int oracle_rule(int d, int deg, double* xq, double* wq) {
    double xb[OR_MAXQ * 3], wb[OR_MAXQ];
    int n = 0;
    if (d == 2) {
        const double area = 0.5;
        if (deg == 2) {
            double t[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};
            n = push_orbit(xb, wb, n, 2, t, area / 3.0);
        } else if (deg == 4) {
            /* Strang-Fix / Dunavant 6-point rule */
            double a1 = 0.445948490915965, w1 = 0.223381589678011;
            double a2 = 0.091576213509771, w2 = 0.109951743655322;
            double t1[3] = {1.0 - 2.0 * a1, a1, a1};
            double t2[3] = {1.0 - 2.0 * a2, a2, a2};
            n = push_orbit(xb, wb, n, 2, t1, area * w1);
            n = push_orbit(xb, wb, n, 2, t2, area * w2);
        } else if (deg == 6) {
            /* Dunavant 12-point rule */
            double a1 = 0.249286745170910, w1 = 0.116786275726379;
            double a2 = 0.063089014491502, w2 = 0.050844906370207;
            double b3 = 0.053145049844817, c3 = 0.310352451033784, w3 = 0.082851075618374;
            double t1[3] = {1.0 - 2.0 * a1, a1, a1};
            double t2[3] = {1.0 - 2.0 * a2, a2, a2};
            double t3[3] = {b3, c3, 1.0 - b3 - c3};
            n = push_orbit(xb, wb, n, 2, t1, area * w1);
            n = push_orbit(xb, wb, n, 2, t2, area * w2);
            n = push_orbit(xb, wb, n, 2, t3, area * w3);
        } else return -1;
    } else if (d == 3) {
        const double vol = 1.0 / 6.0;
        if (deg == 2) {
            double a = (5.0 - sqrt(5.0)) / 20.0;
            double t[4] = {1.0 - 3.0 * a, a, a, a};
            n = push_orbit(xb, wb, n, 3, t, vol / 4.0);
        } else if (deg == 4) {
            /* Keast 11-point rule (one negative weight); weights for volume 1/6 */
            double s = sqrt(5.0 / 14.0);
            double c[4] = {0.25, 0.25, 0.25, 0.25};
            double t1[4] = {11.0 / 14.0, 1.0 / 14.0, 1.0 / 14.0, 1.0 / 14.0};
            double t2[4] = {(1.0 + s) / 4.0, (1.0 + s) / 4.0, (1.0 - s) / 4.0, (1.0 - s) / 4.0};
            n = push_orbit(xb, wb, n, 3, c, -74.0 / 5625.0);
            n = push_orbit(xb, wb, n, 3, t1, 343.0 / 45000.0);
            n = push_orbit(xb, wb, n, 3, t2, 56.0 / 2250.0);
        } else if (deg == 6) {
            /* Keast 24-point rule; weights listed for volume 1, scaled below */
            double a1 = 0.214602871259151684, w1 = 0.0399227502581679;
            double a2 = 0.0406739585346113397, w2 = 0.0100772110553207;
            double a3 = 0.322337890142275646, w3 = 0.0553571815436547;
            double a4 = 0.0636610018750175299, b4 = 0.269672331458315867, w4 = 27.0 / 560.0;
            double t1[4] = {1.0 - 3.0 * a1, a1, a1, a1};
            double t2[4] = {1.0 - 3.0 * a2, a2, a2, a2};
            double t3[4] = {1.0 - 3.0 * a3, a3, a3, a3};
            double t4[4] = {1.0 - 2.0 * a4 - b4, b4, a4, a4};
            n = push_orbit(xb, wb, n, 3, t1, vol * w1);
            n = push_orbit(xb, wb, n, 3, t2, vol * w2);
            n = push_orbit(xb, wb, n, 3, t3, vol * w3);
            n = push_orbit(xb, wb, n, 3, t4, vol * w4);
        } else return -1;
    } else return -1;
    if (xq) memcpy(xq, xb, sizeof(double) * n * d);
    if (wq) memcpy(wq, wb, sizeof(double) * n);
    return n;
}

/* ------------------------------------------------------------------ */
/* Lagrange basis on the reference simplex (barycentric formulas)       */
/* ------------------------------------------------------------------ */

int oracle_nlocal(int d, int p) {
    if (d == 2) return (p + 1) * (p + 2) / 2;
    if (d == 3) return (p + 1) * (p + 2) * (p + 3) / 6;
    return -1;
}

/* gradient (w.r.t. reference coordinates) of barycentric coordinate a */
static void dlam(int d, int a, double* g) {
    for (int c = 0; c < d; ++c) g[c] = (a == 0) ? -1.0 : (c == a - 1 ? 1.0 : 0.0);
}

/* Values phi[n_p] and reference gradients grad[n_p][d] at xhat[d].
 * Returns n_p, or -1 for an unsupported (d, p). */
int oracle_basis(int d, int p, const double* xhat, double* phi, double* grad) {
    if ((d != 2 && d != 3) || p < 1 || p > 3) return -1;
    int nv = d + 1;
    double L[4], G[4][3];
    double s = 0.0;
    for (int a = 0; a < d; ++a) s += xhat[a];
    L[0] = 1.0 - s;
    for (int a = 0; a < d; ++a) L[a + 1] = xhat[a];
    for (int a = 0; a < nv; ++a) dlam(d, a, G[a]);
    int k = 0;
    /* vertices */
    for (int a = 0; a < nv; ++a, ++k) {
        double l = L[a], f, df;
        if (p == 1) { f = l; df = 1.0; }
        else if (p == 2) { f = l * (2.0 * l - 1.0); df = 4.0 * l - 1.0; }
        else { f = 0.5 * l * (3.0 * l - 1.0) * (3.0 * l - 2.0); df = 0.5 * (27.0 * l * l - 18.0 * l + 2.0); }
        phi[k] = f;
        for (int c = 0; c < d; ++c) grad[k * d + c] = df * G[a][c];
    }
    if (p >= 2) {
        for (int a = 0; a < nv; ++a) for (int b = a + 1; b < nv; ++b) {
            if (p == 2) {
                phi[k] = 4.0 * L[a] * L[b];
                for (int c = 0; c < d; ++c) grad[k * d + c] = 4.0 * (G[a][c] * L[b] + L[a] * G[b][c]);
                ++k;
            } else {
                /* node nearer a: 9/2 La Lb (3La - 1); nearer b: 9/2 La Lb (3Lb - 1) */
                for (int t = 0; t < 2; ++t) {
                    double Ln = t == 0 ? L[a] : L[b];
                    const double* Gn = t == 0 ? G[a] : G[b];
                    phi[k] = 4.5 * L[a] * L[b] * (3.0 * Ln - 1.0);
                    for (int c = 0; c < d; ++c)
                        grad[k * d + c] = 4.5 * ((G[a][c] * L[b] + L[a] * G[b][c]) * (3.0 * Ln - 1.0)
                                                 + L[a] * L[b] * 3.0 * Gn[c]);
                    ++k;
                }
            }
        }
    }
    if (p == 3) {
        for (int a = 0; a < nv; ++a) for (int b = a + 1; b < nv; ++b) for (int e = b + 1; e < nv; ++e) {
            phi[k] = 27.0 * L[a] * L[b] * L[e];
            for (int c = 0; c < d; ++c)
                grad[k * d + c] = 27.0 * (G[a][c] * L[b] * L[e] + L[a] * G[b][c] * L[e] + L[a] * L[b] * G[e][c]);
            ++k;
        }
    }
    return k;
}

/* ------------------------------------------------------------------ */
/* Conductivity law                                                     */
/* ------------------------------------------------------------------ */

double oracle_k(int kind, const double* cp, int ncp, double u, double* dk) {
    if (kind == 0) {
        double v = 0.0, dv = 0.0, pw = 1.0;
        for (int i = 0; i < ncp; ++i) {
            v += cp[i] * pw;
            if (i + 1 < ncp) dv += (double)(i + 1) * cp[i + 1] * pw;
            pw *= u;
        }
        if (dk) *dk = dv;
        return v;
    }
    if (kind == 1) {
        if (dk) *dk = cp[1] * cp[2] * cos(cp[2] * u);
        return cp[0] + cp[1] * sin(cp[2] * u);
    }
    if (kind == 2) {
        int m = ncp / 2;
        const double* t = cp;
        const double* kv = cp + m;
        if (u < t[0]) { if (dk) *dk = 0.0; return kv[0]; }
        if (u > t[m - 1]) { if (dk) *dk = 0.0; return kv[m - 1]; }
        int i = 0;
        while (i + 2 < m && u > t[i + 1]) ++i;   /* branch [t_i, t_i+1] (left-closed only for i=0) */
        double sl = (kv[i + 1] - kv[i]) / (t[i + 1] - t[i]);
        if (dk) *dk = sl;
        return kv[i] + sl * (u - t[i]);
    }
    if (dk) *dk = 0.0;
    return 0.0;
}

/* ------------------------------------------------------------------ */
/* Mesh context                                                         */
/* ------------------------------------------------------------------ */

typedef struct {
    int d, p, np, n, E;
    const double* X;     /* n x d, caller owned */
    const int* conn;     /* E x np, caller owned */
    /* pattern (built on demand) */
    int* row_ptr;
    int* col_idx;
    long long nnz;
    /* node -> element incidence, ascending element */
    int* inc_ptr;
    int* inc_el;
    /* constant conductivity tensor c (d x d, SPD; identity unless set):
     * the conductivity is k(u) c (Section 7, anisotropic conductivity) */
    double cond[3][3];
    /* per-quadrature-point geometry (Section 7): iso = 1 maps each element
     * through all its nodes, x(xhat) = sum_i x_i phi_i(xhat), so B depends
     * on the point; cfield (E x n_q x d x d, row-major per point, owned) a
     * conductivity tensor per quadrature point of the degree-2p rule */
    int iso;
    double* cfield;
} octx;

void* oracle_create(int d, int p, int n_nodes, int n_elems, const double* coords, const int* conn) {
    int np = oracle_nlocal(d, p);
    if (np < 0 || n_nodes < 0 || n_elems < 0) return NULL;
    for (long long k = 0; k < (long long)n_elems * np; ++k)
        if (conn[k] < 0 || conn[k] >= n_nodes) return NULL;
    octx* c = (octx*)calloc(1, sizeof(octx));
    c->d = d; c->p = p; c->np = np; c->n = n_nodes; c->E = n_elems;
    c->X = coords; c->conn = conn;
    c->nnz = -1;
    for (int a = 0; a < 3; ++a) c->cond[a][a] = 1.0;
    c->inc_ptr = (int*)calloc((size_t)n_nodes + 1, sizeof(int));
    for (long long k = 0; k < (long long)n_elems * np; ++k) c->inc_ptr[conn[k] + 1]++;
    for (int r = 0; r < n_nodes; ++r) c->inc_ptr[r + 1] += c->inc_ptr[r];
    c->inc_el = (int*)malloc(sizeof(int) * ((size_t)n_elems * np + 1));
    int* fill = (int*)calloc((size_t)n_nodes, sizeof(int));
    for (int e = 0; e < n_elems; ++e)
        for (int i = 0; i < np; ++i) {
            int r = conn[(long long)e * np + i];
            c->inc_el[c->inc_ptr[r] + fill[r]++] = e;
        }
    free(fill);
    return c;
}

void oracle_destroy(void* h) {
    octx* c = (octx*)h;
    if (!c) return;
    free(c->row_ptr); free(c->col_idx); free(c->inc_ptr); free(c->inc_el); free(c->cfield);
    free(c);
}

static int cmp_ll(const void* a, const void* b) {
    long long x = *(const long long*)a, y = *(const long long*)b;
    return (x > y) - (x < y);
}

/* Builds the CSR pattern: all pairs (conn[e][i], conn[e][j]), sorted, unique. */
static int build_pattern(octx* c) {
    if (c->nnz >= 0) return 0;
    long long m = (long long)c->E * c->np * c->np;
    long long* keys = (long long*)malloc(sizeof(long long) * (size_t)(m > 0 ? m : 1));
    if (!keys) return -1;
    long long k = 0;
    for (int e = 0; e < c->E; ++e)
        for (int i = 0; i < c->np; ++i)
            for (int j = 0; j < c->np; ++j)
                keys[k++] = (long long)c->conn[(long long)e * c->np + i] * c->n + c->conn[(long long)e * c->np + j];
    qsort(keys, (size_t)m, sizeof(long long), cmp_ll);
    long long u = 0;
    for (long long t = 0; t < m; ++t)
        if (t == 0 || keys[t] != keys[t - 1]) keys[u++] = keys[t];
    c->nnz = u;
    c->row_ptr = (int*)calloc((size_t)c->n + 1, sizeof(int));
    c->col_idx = (int*)malloc(sizeof(int) * (size_t)(u > 0 ? u : 1));
    for (long long t = 0; t < u; ++t) {
        int r = (int)(keys[t] / c->n);
        c->row_ptr[r + 1]++;
        c->col_idx[t] = (int)(keys[t] % c->n);
    }
    for (int r = 0; r < c->n; ++r) c->row_ptr[r + 1] += c->row_ptr[r];
    free(keys);
    return 0;
}

long long oracle_nnz(void* h) {
    octx* c = (octx*)h;
    if (build_pattern(c)) return -1;
    return c->nnz;
}

void oracle_pattern(void* h, int* row_ptr, int* col_idx) {
    octx* c = (octx*)h;
    build_pattern(c);
    memcpy(row_ptr, c->row_ptr, sizeof(int) * ((size_t)c->n + 1));
    memcpy(col_idx, c->col_idx, sizeof(int) * (size_t)c->nnz);
}

/* ------------------------------------------------------------------ */
/* Element matrices (Algorithm 1, inner loop)                           */
/* ------------------------------------------------------------------ */

typedef struct {
    int nq;
    double w[OR_MAXQ];
    double phi[OR_MAXQ][OR_MAXNP];
    double J[OR_MAXQ][OR_MAXNP][3];
} otab;

static int make_tab(int d, int p, int deg, otab* t) {
    double xq[OR_MAXQ * 3];
    int nq = oracle_rule(d, deg, xq, t->w);
    if (nq < 0) return -1;
    t->nq = nq;
    for (int q = 0; q < nq; ++q) {
        double g[OR_MAXNP * 3];
        oracle_basis(d, p, xq + q * d, t->phi[q], g);
        for (int i = 0; i < oracle_nlocal(d, p); ++i)
            for (int a = 0; a < d; ++a) t->J[q][i][a] = g[i * d + a];
    }
    return 0;
}

/* Exported: set the constant conductivity tensor (d x d row-major; NULL:
 * identity). */
void oracle_set_conductivity(void* h, const double* cd) {
    octx* c = (octx*)h;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) c->cond[a][b] = (a == b) ? 1.0 : 0.0;
    if (cd)
        for (int a = 0; a < c->d; ++a)
            for (int b = 0; b < c->d; ++b) c->cond[a][b] = cd[a * c->d + b];
}

/* det, |det| and A = B^-1 c B^-T of element e (c the conductivity tensor;
 * the identity gives (B^T B)^-1) */
static double invert_a(int d, double B[3][3], double cond[3][3], double A[3][3]);

static double geometry(const octx* c, int e, double A[3][3]) {
    int d = c->d;
    const int* v = c->conn + (long long)e * c->np;
    double B[3][3];
    for (int col = 0; col < d; ++col)
        for (int row = 0; row < d; ++row)
            B[row][col] = c->X[(long long)v[col + 1] * d + row] - c->X[(long long)v[0] * d + row];
    double cond[3][3];
    memcpy(cond, c->cond, sizeof(cond));
    return invert_a(d, B, cond, A);
}

/* det B and A = B^-1 cond B^-T (cofactor inverse) */
static double invert_a(int d, double B[3][3], double cond[3][3], double A[3][3]) {
    double det, Bi[3][3];
    if (d == 2) {
        det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
        Bi[0][0] = B[1][1] / det;  Bi[0][1] = -B[0][1] / det;
        Bi[1][0] = -B[1][0] / det; Bi[1][1] = B[0][0] / det;
    } else {
        double c00 = B[1][1] * B[2][2] - B[1][2] * B[2][1];
        double c01 = B[1][2] * B[2][0] - B[1][0] * B[2][2];
        double c02 = B[1][0] * B[2][1] - B[1][1] * B[2][0];
        det = B[0][0] * c00 + B[0][1] * c01 + B[0][2] * c02;
        /* inverse = adj(B)/det, adj = cofactor^T */
        Bi[0][0] = c00 / det;
        Bi[1][0] = c01 / det;
        Bi[2][0] = c02 / det;
        Bi[0][1] = (B[0][2] * B[2][1] - B[0][1] * B[2][2]) / det;
        Bi[1][1] = (B[0][0] * B[2][2] - B[0][2] * B[2][0]) / det;
        Bi[2][1] = (B[0][1] * B[2][0] - B[0][0] * B[2][1]) / det;
        Bi[0][2] = (B[0][1] * B[1][2] - B[0][2] * B[1][1]) / det;
        Bi[1][2] = (B[0][2] * B[1][0] - B[0][0] * B[1][2]) / det;
        Bi[2][2] = (B[0][0] * B[1][1] - B[0][1] * B[1][0]) / det;
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0;
            for (int k = 0; k < d; ++k)
                for (int l = 0; l < d; ++l) s += Bi[a][k] * cond[k][l] * Bi[b][l];
            A[a][b] = s;
        }
    return det;
}

/* The geometry at quadrature point q of element e (Section 7): B_q =
 * sum_i x_i (J_q)_i^T through all the element's nodes for an isoparametric
 * mesh (the vertices' edge vectors otherwise), and the point's conductivity
 * tensor when a field is set (the mesh's constant tensor otherwise):
 * A_q = B_q^-1 c_q B_q^-T.  Returns det B_q. */
static double geometry_q(const octx* c, const otab* t, int e, int q, double A[3][3]) {
    int d = c->d, np = c->np;
    const int* v = c->conn + (long long)e * np;
    double B[3][3];
    if (c->iso) {
        for (int row = 0; row < d; ++row)
            for (int col = 0; col < d; ++col) {
                double s = 0.0;
                for (int i = 0; i < np; ++i) s += c->X[(long long)v[i] * d + row] * t->J[q][i][col];
                B[row][col] = s;
            }
    } else {
        for (int col = 0; col < d; ++col)
            for (int row = 0; row < d; ++row)
                B[row][col] = c->X[(long long)v[col + 1] * d + row] - c->X[(long long)v[0] * d + row];
    }
    double cond[3][3];
    if (c->cfield) {
        const double* cf = c->cfield + ((long long)e * t->nq + q) * d * d;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) cond[a][b] = cf[a * d + b];
    } else {
        memcpy(cond, c->cond, sizeof(cond));
    }
    return invert_a(d, B, cond, A);
}

/* Exported: isoparametric mapping on (1) or off (0). */
void oracle_set_isoparametric(void* h, int on) { ((octx*)h)->iso = on ? 1 : 0; }

/* Exported: conductivity tensors per quadrature point of the degree-2p rule
 * (E x n_q x d x d, copied), or NULL to clear. */
int oracle_set_conductivity_field(void* h, const double* cf) {
    octx* c = (octx*)h;
    free(c->cfield);
    c->cfield = NULL;
    if (!cf) return 0;
    int nq = oracle_rule(c->d, 2 * c->p, NULL, NULL);
    size_t n = (size_t)c->E * nq * c->d * c->d;
    c->cfield = (double*)malloc(sizeof(double) * (n ? n : 1));
    if (!c->cfield) return -1;
    memcpy(c->cfield, cf, sizeof(double) * n);
    return 0;
}

/* Local matrices of element e (dense n_p x n_p, row = test index).  If
 * aM/aK/aT are given they receive the error scale of each entry: the sum of
 * the magnitudes of the fully expanded product terms of the quadrature sum,
 * with |A_ab| bounded by sqrt(A_aa A_bb) (A_e is symmetric positive
 * definite), so that entries which cancel inside the sum are judged against
 * what cancelled. */
static void element(const octx* c, const otab* t, int e, double m, int kkind, const double* kp, int nkp,
                    const double* u, double* Me, double* Ke, double* Te, double* aM, double* aK, double* aT) {
    int np = c->np, d = c->d;
    double A[3][3];
    double b = fabs(geometry(c, e, A));
    const int* v = c->conn + (long long)e * np;
    double ue[OR_MAXNP];
    for (int i = 0; i < np; ++i) ue[i] = u ? u[v[i]] : 0.0;
    memset(Me, 0, sizeof(double) * np * np);
    memset(Ke, 0, sizeof(double) * np * np);
    memset(Te, 0, sizeof(double) * np * np);
    if (aM) memset(aM, 0, sizeof(double) * np * np);
    if (aK) memset(aK, 0, sizeof(double) * np * np);
    if (aT) memset(aT, 0, sizeof(double) * np * np);
    double Ab[3][3];
    for (int a = 0; a < d; ++a)
        for (int bb = 0; bb < d; ++bb) Ab[a][bb] = sqrt(fabs(A[a][a] * A[bb][bb]));
    for (int q = 0; q < t->nq; ++q) {
        if (c->iso || c->cfield) {   /* per-point geometry (Section 7) */
            b = fabs(geometry_q(c, t, e, q, A));
            for (int a = 0; a < d; ++a)
                for (int bb = 0; bb < d; ++bb) Ab[a][bb] = sqrt(fabs(A[a][a] * A[bb][bb]));
        }
        const double* phi = t->phi[q];
        double uq = 0.0;
        for (int i = 0; i < np; ++i) uq += phi[i] * ue[i];
        double dk;
        double kq = oracle_k(kkind, kp, nkp, uq, &dk);
        /* S = J_q A J_q^T */
        double JA[OR_MAXNP][3];
        for (int i = 0; i < np; ++i)
            for (int bb = 0; bb < d; ++bb) {
                double s = 0.0;
                for (int a = 0; a < d; ++a) s += t->J[q][i][a] * A[a][bb];
                JA[i][bb] = s;
            }
        double S[OR_MAXNP][OR_MAXNP];
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                double s = 0.0;
                for (int a = 0; a < d; ++a) s += JA[i][a] * t->J[q][j][a];
                S[i][j] = s;
            }
        double Su[OR_MAXNP];
        for (int i = 0; i < np; ++i) {
            double s = 0.0;
            for (int j = 0; j < np; ++j) s += S[i][j] * ue[j];
            Su[i] = s;
        }
        double wb = t->w[q] * b;
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                Me[i * np + j] += wb * m * phi[i] * phi[j];
                Ke[i * np + j] += wb * kq * S[i][j];
                Te[i * np + j] += wb * dk * Su[i] * phi[j];
            }
        if (aM || aK || aT) {
            /* |S|_ij = sum_ab |J_ia| |A|_ab |J_jb| */
            double aS[OR_MAXNP][OR_MAXNP];
            for (int i = 0; i < np; ++i)
                for (int j = 0; j < np; ++j) {
                    double s2 = 0.0;
                    for (int a = 0; a < d; ++a)
                        for (int bb = 0; bb < d; ++bb) s2 += fabs(t->J[q][i][a]) * Ab[a][bb] * fabs(t->J[q][j][bb]);
                    aS[i][j] = s2;
                }
            double aSu[OR_MAXNP];
            for (int i = 0; i < np; ++i) {
                double s2 = 0.0;
                for (int j = 0; j < np; ++j) s2 += aS[i][j] * fabs(ue[j]);
                aSu[i] = s2;
            }
            double awb = fabs(wb);
            for (int i = 0; i < np; ++i)
                for (int j = 0; j < np; ++j) {
                    if (aM) aM[i * np + j] += fabs(wb * m * phi[i] * phi[j]);   /* |term| of Me, same rounding */
                    if (aK) aK[i * np + j] += awb * fabs(kq) * aS[i][j];
                    if (aT) aT[i * np + j] += awb * fabs(dk) * aSu[i] * fabs(phi[j]);
                }
        }
    }
}

/* Exported: local matrices of one element (for tests). */
int oracle_element(void* h, int e, int deg, double m, int kkind, const double* kp, int nkp,
                   const double* u, double* Me, double* Ke, double* Te) {
    octx* c = (octx*)h;
    otab t;
    if (make_tab(c->d, c->p, deg, &t)) return -1;
    if (e < 0 || e >= c->E) return -1;
    element(c, &t, e, m, kkind, kp, nkp, u, Me, Ke, Te, NULL, NULL, NULL);
    return 0;
}

/* Exported: |det B_e| and A_e (d x d row-major) of one element. */
double oracle_geometry(void* h, int e, double* A_out) {
    octx* c = (octx*)h;
    double A[3][3];
    double det = geometry(c, e, A);
    for (int a = 0; a < c->d; ++a)
        for (int b = 0; b < c->d; ++b) A_out[a * c->d + b] = A[a][b];
    return det;
}

static long long find_slot(const octx* c, int r, int col) {
    int lo = c->row_ptr[r], hi = c->row_ptr[r + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (c->col_idx[mid] == col) return mid;
        if (c->col_idx[mid] < col) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Algorithm 1: full assembly into the CSR pattern.  Any output may be NULL. */
int oracle_assemble(void* h, int deg, double m, int kkind, const double* kp, int nkp, const double* u,
                    double* M, double* K, double* T, double* absM, double* absK, double* absT) {
    octx* c = (octx*)h;
    if (build_pattern(c)) return -1;
    otab t;
    if (make_tab(c->d, c->p, deg, &t)) return -1;
    int np = c->np;
    size_t nz = (size_t)c->nnz;
    double* out[6] = {M, K, T, absM, absK, absT};
    for (int k = 0; k < 6; ++k) if (out[k]) memset(out[k], 0, sizeof(double) * nz);
    double Me[OR_MAXNP * OR_MAXNP], Ke[OR_MAXNP * OR_MAXNP], Te[OR_MAXNP * OR_MAXNP];
    double aMe[OR_MAXNP * OR_MAXNP], aKe[OR_MAXNP * OR_MAXNP], aTe[OR_MAXNP * OR_MAXNP];
    int want_abs = absM || absK || absT;
    for (int e = 0; e < c->E; ++e) {
        element(c, &t, e, m, kkind, kp, nkp, u, Me, Ke, Te, want_abs ? aMe : NULL, want_abs ? aKe : NULL,
                want_abs ? aTe : NULL);
        const int* v = c->conn + (long long)e * np;
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                long long s = find_slot(c, v[i], v[j]);
                if (s < 0) return -2;
                int l = i * np + j;
                if (M) M[s] += Me[l];
                if (K) K[s] += Ke[l];
                if (T) T[s] += Te[l];
                if (absM) absM[s] += aMe[l];
                if (absK) absK[s] += aKe[l];
                if (absT) absT[s] += aTe[l];
            }
    }
    return 0;
}

/* The same assembly with the element loop spread over `nthreads` host
 * threads (OpenMP; 0 = all the host's cores): every element's local
 * matrices are formed in parallel into a buffer by the same element()
 * routine, then added into the CSR values by one thread in ascending element
 * order, exactly as oracle_assemble adds them, so the results are the same
 * bits.  This is the multi-core CPU baseline (a timing reference); the
 * parity reference is oracle_assemble.  No error scales.  Returns the number
 * of threads used (negative on failure). */
int oracle_assemble_mt(void* h, int deg, double m, int kkind, const double* kp, int nkp, const double* u,
                       double* M, double* K, double* T, int nthreads) {
    octx* c = (octx*)h;
    if (build_pattern(c)) return -1;
    otab t;
    if (make_tab(c->d, c->p, deg, &t)) return -1;
    const int np = c->np;
    const size_t ne = (size_t)np * np;
    const size_t nz = (size_t)c->nnz;
    double* out[3] = {M, K, T};
    for (int k = 0; k < 3; ++k) if (out[k]) memset(out[k], 0, sizeof(double) * nz);
    double* buf = (double*)malloc(sizeof(double) * 3 * ne * (size_t)c->E);
    if (!buf && c->E > 0) return -3;
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_num_procs();
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int e = 0; e < c->E; ++e) {
        if (e == 0) used = omp_get_num_threads();
        double* b = buf + 3 * ne * (size_t)e;
        element(c, &t, e, m, kkind, kp, nkp, u, b, b + ne, b + 2 * ne, NULL, NULL, NULL);
    }
#else
    (void)nthreads;
    for (int e = 0; e < c->E; ++e) {
        double* b = buf + 3 * ne * (size_t)e;
        element(c, &t, e, m, kkind, kp, nkp, u, b, b + ne, b + 2 * ne, NULL, NULL, NULL);
    }
#endif
    for (int e = 0; e < c->E; ++e) {
        const int* v = c->conn + (long long)e * np;
        const double* b = buf + 3 * ne * (size_t)e;
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                long long s = find_slot(c, v[i], v[j]);
                if (s < 0) {
                    free(buf);
                    return -2;
                }
                int l = i * np + j;
                if (M) M[s] += b[l];
                if (K) K[s] += b[ne + l];
                if (T) T[s] += b[2 * ne + l];
            }
    }
    free(buf);
    return used;
}

/* Selected entries (rows[k], cols[k]) computed one by one: the sum over the
 * elements containing both nodes, in ascending element order.  Works at any
 * mesh size without building the pattern.  Outputs may be NULL. */
int oracle_entries(void* h, int deg, double m, int kkind, const double* kp, int nkp, const double* u,
                   long long nq, const int* rows, const int* cols,
                   double* M, double* K, double* T, double* absM, double* absK, double* absT) {
    octx* c = (octx*)h;
    otab t;
    if (make_tab(c->d, c->p, deg, &t)) return -1;
    int np = c->np;
    double Me[OR_MAXNP * OR_MAXNP], Ke[OR_MAXNP * OR_MAXNP], Te[OR_MAXNP * OR_MAXNP];
    double aMe[OR_MAXNP * OR_MAXNP], aKe[OR_MAXNP * OR_MAXNP], aTe[OR_MAXNP * OR_MAXNP];
    for (long long k = 0; k < nq; ++k) {
        int r = rows[k], col = cols[k];
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int p = c->inc_ptr[r]; p < c->inc_ptr[r + 1]; ++p) {
            int e = c->inc_el[p];
            const int* v = c->conn + (long long)e * np;
            int i = -1, j = -1;
            for (int a = 0; a < np; ++a) { if (v[a] == r) i = a; if (v[a] == col) j = a; }
            if (i < 0 || j < 0) continue;
            element(c, &t, e, m, kkind, kp, nkp, u, Me, Ke, Te, aMe, aKe, aTe);
            int l = i * np + j;
            s[0] += Me[l]; s[1] += Ke[l]; s[2] += Te[l];
            s[3] += aMe[l]; s[4] += aKe[l]; s[5] += aTe[l];
        }
        if (M) M[k] = s[0];
        if (K) K[k] = s[1];
        if (T) T[k] = s[2];
        if (absM) absM[k] = s[3];
        if (absK) absK[k] = s[4];
        if (absT) absT[k] = s[5];
    }
    return 0;
}

/* u-dependent mass and the mass tensor (Section 2 with m = m(u_h); Section 5,
 * the Jacobian term  (mass tensor) o_2 (u - u^s) + M(u); Section 5.1, the
 * local mass tensor):
 *     Mu_e        = sum_q w_q m(u_q)  phi_q phi_q^T               |det B_e|
 *     Mc_e[i][j][k] = sum_q w_q m'(u_q) phi_q[i] phi_q[j] phi_q[k] |det B_e|
 *     Mt_e[i][k]  = sum_j Mc_e[i][j][k] z_e[j],   z = u - us,
 * the tensor formed in full and then multiplied by z in its second mode,
 * assembled over ascending elements into the CSR pattern.  m is a
 * coefficient law as k (kind, parameters).  absMu/absMt receive the sums of
 * the magnitudes of the expanded terms.  Any output may be NULL; us may be
 * NULL when Mt and absMt are. */
int oracle_assemble_mass_u(void* h, int deg, int mkind, const double* mp, int nmp, const double* u,
                           const double* us, double* Mu, double* Mt, double* absMu, double* absMt) {
    octx* c = (octx*)h;
    if (build_pattern(c)) return -1;
    otab t;
    if (make_tab(c->d, c->p, deg, &t)) return -1;
    if ((Mt || absMt) && !us) return -3;
    int np = c->np;
    size_t nz = (size_t)c->nnz;
    double* out[4] = {Mu, Mt, absMu, absMt};
    for (int k = 0; k < 4; ++k) if (out[k]) memset(out[k], 0, sizeof(double) * nz);
    static double Mc[OR_MAXNP * OR_MAXNP * OR_MAXNP], aMc[OR_MAXNP * OR_MAXNP * OR_MAXNP];
    double Me[OR_MAXNP * OR_MAXNP], aMe[OR_MAXNP * OR_MAXNP], Te[OR_MAXNP * OR_MAXNP], aTe[OR_MAXNP * OR_MAXNP];
    for (int e = 0; e < c->E; ++e) {
        double A[3][3];
        double b = fabs(geometry(c, e, A));
        const int* v = c->conn + (long long)e * np;
        double ue[OR_MAXNP], ze[OR_MAXNP];
        for (int i = 0; i < np; ++i) {
            ue[i] = u[v[i]];
            ze[i] = us ? u[v[i]] - us[v[i]] : 0.0;
        }
        memset(Me, 0, sizeof(Me));
        memset(aMe, 0, sizeof(aMe));
        memset(Mc, 0, sizeof(double) * np * np * np);
        memset(aMc, 0, sizeof(double) * np * np * np);
        for (int q = 0; q < t.nq; ++q) {
            if (c->iso || c->cfield) b = fabs(geometry_q(c, &t, e, q, A));   /* per-point geometry (Section 7) */
            const double* phi = t.phi[q];
            double uq = 0.0;
            for (int i = 0; i < np; ++i) uq += phi[i] * ue[i];
            double dm;
            double mq = oracle_k(mkind, mp, nmp, uq, &dm);
            double wb = t.w[q] * b;
            for (int i = 0; i < np; ++i)
                for (int j = 0; j < np; ++j) {
                    Me[i * np + j] += wb * mq * phi[i] * phi[j];
                    aMe[i * np + j] += fabs(wb * mq * phi[i] * phi[j]);
                    for (int k = 0; k < np; ++k) {
                        Mc[(i * np + j) * np + k] += wb * dm * phi[i] * phi[j] * phi[k];
                        aMc[(i * np + j) * np + k] += fabs(wb * dm * phi[i] * phi[j] * phi[k]);
                    }
                }
        }
        /* second-mode product with z_e */
        for (int i = 0; i < np; ++i)
            for (int k = 0; k < np; ++k) {
                double s = 0.0, a = 0.0;
                for (int j = 0; j < np; ++j) {
                    s += Mc[(i * np + j) * np + k] * ze[j];
                    a += aMc[(i * np + j) * np + k] * fabs(ze[j]);
                }
                Te[i * np + k] = s;
                aTe[i * np + k] = a;
            }
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                long long s = find_slot(c, v[i], v[j]);
                if (s < 0) return -2;
                int l = i * np + j;
                if (Mu) Mu[s] += Me[l];
                if (Mt) Mt[s] += Te[l];
                if (absMu) absMu[s] += aMe[l];
                if (absMt) absMt[s] += aTe[l];
            }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Boundary terms, residual and Jacobian (Section 5; Section 6, Exp. 2) */
/* ------------------------------------------------------------------ */
/* The load vector holds f_i = int_Omega f phi_i + int_{dOmega_N} g_N(u_h)
 * phi_i dS (Section 2) and its derivative B_ik = int_{dOmega_N}
 * g_N'(u_h) phi_i phi_k dS (Section 5).  Here dOmega_N is the whole boundary
 * (Experiment 2: convection and radiation on every side), f = 0, and g_N is
 * a law of u (for Experiment 2 the polynomial h_c (T_a - u) + h_r (T_a^4 -
 * u^4)).  The boundary facets are the element faces that belong to one
 * element only; face f of an element is the face opposite its local vertex
 * f.  They are listed in ascending (element, face) order, the order in
 * which their contributions are added. */

typedef struct { int e, f; int key[3]; } oface;

static int cmp_face(const void* a, const void* b) {
    const oface* x = (const oface*)a; const oface* y = (const oface*)b;
    for (int t = 0; t < 3; ++t) if (x->key[t] != y->key[t]) return x->key[t] < y->key[t] ? -1 : 1;
    if (x->e != y->e) return x->e < y->e ? -1 : 1;
    return x->f - y->f;
}
static int cmp_ef(const void* a, const void* b) {
    const int* x = (const int*)a; const int* y = (const int*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return x[1] - y[1];
}

/* Boundary facets as (element, face) pairs in ascending order; returns the
 * count (out may be NULL: count only), -1 on allocation failure. */
int oracle_boundary_facets(void* h, int* fe, int* ff) {
    octx* c = (octx*)h;
    int d = c->d, nv = d + 1;
    long long nf = (long long)c->E * nv;
    oface* F = (oface*)malloc(sizeof(oface) * (size_t)(nf > 0 ? nf : 1));
    if (!F) return -1;
    for (int e = 0; e < c->E; ++e)
        for (int f = 0; f < nv; ++f) {
            oface* o = &F[(long long)e * nv + f];
            o->e = e; o->f = f;
            int k = 0;
            for (int a = 0; a < nv; ++a) if (a != f) o->key[k++] = c->conn[(long long)e * c->np + a];
            for (; k < 3; ++k) o->key[k] = -1;
            /* sort the face's vertex ids (at most 3) */
            for (int i = 0; i < 3; ++i) for (int j = i + 1; j < 3; ++j)
                if (o->key[j] < o->key[i]) { int t = o->key[i]; o->key[i] = o->key[j]; o->key[j] = t; }
        }
    qsort(F, (size_t)nf, sizeof(oface), cmp_face);
    int* pairs = (int*)malloc(sizeof(int) * 2 * (size_t)(nf > 0 ? nf : 1));
    int nb = 0;
    for (long long i = 0; i < nf;) {
        long long j = i + 1;
        while (j < nf && F[j].key[0] == F[i].key[0] && F[j].key[1] == F[i].key[1] && F[j].key[2] == F[i].key[2]) ++j;
        if (j - i == 1) { pairs[2 * nb] = F[i].e; pairs[2 * nb + 1] = F[i].f; ++nb; }
        i = j;
    }
    qsort(pairs, (size_t)nb, 2 * sizeof(int), cmp_ef);
    if (fe && ff) for (int i = 0; i < nb; ++i) { fe[i] = pairs[2 * i]; ff[i] = pairs[2 * i + 1]; }
    free(F); free(pairs);
    return nb;
}

/* The local nodes of face f: the nodes whose associated vertices (one for a
 * vertex node, the two ends of its edge, the three corners of its face, in
 * the local order of oracle_basis) do not include vertex f. */
static int face_nodes(int d, int p, int f, int* out) {
    int nv = d + 1, k = 0, n = 0;
    for (int a = 0; a < nv; ++a, ++k) if (a != f) out[n++] = k;
    if (p >= 2)
        for (int a = 0; a < nv; ++a) for (int b = a + 1; b < nv; ++b)
            for (int t = 0; t < p - 1; ++t, ++k) if (a != f && b != f) out[n++] = k;
    if (p == 3)
        for (int a = 0; a < nv; ++a) for (int b = a + 1; b < nv; ++b) for (int e = b + 1; e < nv; ++e, ++k)
            if (a != f && b != f && e != f) out[n++] = k;
    return n;
}

/* Quadrature on the reference facet: Gauss-Legendre with p+1 points on
 * [0, 1] (weights summing to 1) for the edges of triangles; for the
 * triangular faces of tetrahedra the triangle rule of degree 2p (weights
 * summing to 1/2).  xi: n x (d-1).  Returns n. */
static int facet_rule(int d, int p, double* xi, double* w) {
    if (d == 3) return oracle_rule(2, 2 * p, xi, w);
    static const double t2[] = {-0.57735026918962576451, 0.57735026918962576451};
    static const double w2[] = {1.0, 1.0};
    static const double t3[] = {-0.77459666924148337704, 0.0, 0.77459666924148337704};
    static const double w3[] = {0.55555555555555555556, 0.88888888888888888889, 0.55555555555555555556};
    static const double t4[] = {-0.86113631159405257522, -0.33998104358485626480, 0.33998104358485626480,
                                0.86113631159405257522};
    static const double w4[] = {0.34785484513745385737, 0.65214515486254614263, 0.65214515486254614263,
                                0.34785484513745385737};
    const double* t = p == 1 ? t2 : p == 2 ? t3 : t4;
    const double* ww = p == 1 ? w2 : p == 2 ? w3 : w4;
    int n = p + 1;
    for (int q = 0; q < n; ++q) { xi[q] = 0.5 * (1.0 + t[q]); w[q] = 0.5 * ww[q]; }
    return n;
}

/* B (CSR values of the mesh pattern) and b (n values); absB, absb receive the
 * sums of the magnitudes of the terms (the error scale).  Any output may be
 * NULL.  Returns 0, or negative on failure. */
int oracle_boundary(void* h, int gkind, const double* gp, int ngp, const double* u, double* B, double* b,
                    double* absB, double* absb) {
    octx* c = (octx*)h;
    if (build_pattern(c)) return -1;
    if (c->iso) return -3;   /* straight facets only */
    int d = c->d, p = c->p, np = c->np, nv = d + 1;
    int nb = oracle_boundary_facets(h, NULL, NULL);
    if (nb < 0) return -1;
    int* fe = (int*)malloc(sizeof(int) * (size_t)(nb + 1));
    int* ff = (int*)malloc(sizeof(int) * (size_t)(nb + 1));
    oracle_boundary_facets(h, fe, ff);
    if (B) memset(B, 0, sizeof(double) * (size_t)c->nnz);
    if (absB) memset(absB, 0, sizeof(double) * (size_t)c->nnz);
    if (b) memset(b, 0, sizeof(double) * (size_t)c->n);
    if (absb) memset(absb, 0, sizeof(double) * (size_t)c->n);
    double xi[OR_MAXQ * 2], w[OR_MAXQ];
    int nq = facet_rule(d, p, xi, w);
    for (int k = 0; k < nb; ++k) {
        int e = fe[k], f = ff[k];
        const int* v = c->conn + (long long)e * np;
        int fn[OR_MAXNP];
        int nf = face_nodes(d, p, f, fn);
        int wv[3], m = 0;
        for (int a = 0; a < nv; ++a) if (a != f) wv[m++] = a;
        /* facet measure: edge length (2D), twice the triangle's area (3D) */
        double E1[3], E2[3], J;
        for (int a = 0; a < d; ++a) E1[a] = c->X[(long long)v[wv[1]] * d + a] - c->X[(long long)v[wv[0]] * d + a];
        if (d == 2) {
            J = sqrt(E1[0] * E1[0] + E1[1] * E1[1]);
        } else {
            for (int a = 0; a < 3; ++a) E2[a] = c->X[(long long)v[wv[2]] * 3 + a] - c->X[(long long)v[wv[0]] * 3 + a];
            double cx = E1[1] * E2[2] - E1[2] * E2[1], cy = E1[2] * E2[0] - E1[0] * E2[2],
                   cz = E1[0] * E2[1] - E1[1] * E2[0];
            J = sqrt(cx * cx + cy * cy + cz * cz);
        }
        double Be[OR_MAXNP][OR_MAXNP], aBe[OR_MAXNP][OR_MAXNP], be[OR_MAXNP], abe[OR_MAXNP];
        memset(Be, 0, sizeof(Be)); memset(aBe, 0, sizeof(aBe)); memset(be, 0, sizeof(be)); memset(abe, 0, sizeof(abe));
        for (int q = 0; q < nq; ++q) {
            /* the facet point in reference coordinates of the element: the
             * barycentric combination of the face's reference vertices
             * (reference vertex 0 at the origin, vertex a at e_a) */
            double mu[3], xh[3] = {0.0, 0.0, 0.0};
            if (d == 2) { mu[0] = 1.0 - xi[q]; mu[1] = xi[q]; }
            else { mu[0] = 1.0 - xi[2 * q] - xi[2 * q + 1]; mu[1] = xi[2 * q]; mu[2] = xi[2 * q + 1]; }
            for (int t = 0; t < d; ++t) if (wv[t] > 0) xh[wv[t] - 1] += mu[t];
            double phi[OR_MAXNP], grad[OR_MAXNP * 3];
            oracle_basis(d, p, xh, phi, grad);
            double uq = 0.0;   /* the trace of u_h: face nodes only */
            for (int i = 0; i < nf; ++i) uq += phi[fn[i]] * (u ? u[v[fn[i]]] : 0.0);
            double dg;
            double gq = oracle_k(gkind, gp, ngp, uq, &dg);
            double wj = w[q] * J;
            for (int i = 0; i < nf; ++i) {
                double ti = wj * gq * phi[fn[i]];
                be[i] += ti;
                abe[i] += fabs(ti);
                for (int kk = 0; kk < nf; ++kk) {
                    double t = wj * dg * phi[fn[i]] * phi[fn[kk]];
                    Be[i][kk] += t;
                    aBe[i][kk] += fabs(t);
                }
            }
        }
        for (int i = 0; i < nf; ++i) {
            int r = v[fn[i]];
            if (b) b[r] += be[i];
            if (absb) absb[r] += abe[i];
            for (int kk = 0; kk < nf; ++kk) {
                long long s = find_slot(c, r, v[fn[kk]]);
                if (s < 0) { free(fe); free(ff); return -2; }
                if (B) B[s] += Be[i][kk];
                if (absB) absB[s] += aBe[i][kk];
            }
        }
    }
    free(fe); free(ff);
    return 0;
}

/* Residual of one implicit Euler step (Section 5):
 *   F_i = sum_j M_ij (u_j - us_j) + dt sum_j K_ij u_j - dt b_i,
 * with M, K CSR values of the mesh pattern (M may be M(u)) and b the
 * boundary load (f = 0).  absF receives the sum of the magnitudes of the
 * terms.  Columns in ascending order. */
int oracle_residual(void* h, const double* M, const double* K, const double* b, const double* u, const double* us,
                    double dt, double* F, double* absF) {
    octx* c = (octx*)h;
    if (build_pattern(c)) return -1;
    for (int r = 0; r < c->n; ++r) {
        double s = 0.0, a = 0.0;
        for (int k = c->row_ptr[r]; k < c->row_ptr[r + 1]; ++k) {
            int j = c->col_idx[k];
            double t1 = M[k] * (u[j] - us[j]), t2 = dt * K[k] * u[j];
            s += t1 + t2;
            a += fabs(t1) + fabs(t2);
        }
        double t3 = b ? dt * b[r] : 0.0;
        F[r] = s - t3;
        if (absF) absF[r] = a + fabs(t3);
    }
    return 0;
}

/* Jacobian of the residual (Section 5):
 *   J = Mt + M + dt (K + T) - dt B
 * entry by entry on the mesh pattern (Mt: the mass tensor times u - u^s, T:
 * the conductivity tensor times u; any of Mt, T, B may be NULL for zero). */
int oracle_jacobian(void* h, const double* M, const double* Mt, const double* K, const double* T, const double* B,
                    double dt, double* J) {
    octx* c = (octx*)h;
    if (build_pattern(c)) return -1;
    for (long long s = 0; s < c->nnz; ++s) {
        double kt = K[s] + (T ? T[s] : 0.0);
        J[s] = (Mt ? Mt[s] : 0.0) + M[s] + dt * kt - (B ? dt * B[s] : 0.0);
    }
    return 0;
}

/* Exported: the facet quadrature rule (for tests). */
int oracle_facet_rule(int d, int p, double* xi, double* w) {
    double x[OR_MAXQ * 2], ww[OR_MAXQ];
    int n = facet_rule(d, p, x, ww);
    if (xi) memcpy(xi, x, sizeof(double) * (size_t)n * (d - 1));
    if (w) memcpy(w, ww, sizeof(double) * (size_t)n);
    return n;
}
