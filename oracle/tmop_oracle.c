/*
 * TMOP oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of what the partially assembled TMOP
 * Newton step computes, written from the paper "Accelerating High-Order Mesh
 * Optimization Using Finite Element Partial Assembly on GPUs" (Camier,
 * Dobrev, Knupp, Kolev, Mittal, Rieben, Tomov).  Every element loop runs over
 * the full tensor-product basis (N_p basis functions at each of the N_q
 * quadrature points, no sum factorisation), so each formula can be read
 * against the paper.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this library.  It shares no code, header or table with
 * the CUDA library and neither links nor calls it.
 *
 * Conventions (readings of the paper where it is silent):
 *   - reference element [0,1]^d (Sec. 3.1); Gauss-Legendre quadrature;
 *     Lagrange basis on Gauss-Lobatto-Legendre nodes (node set not stated in
 *     the paper);
 *   - positions are stored component-major: x[a*Nx + node] (Sec. 3, the
 *     vector of all nodal positions x = {x_{a,i}});
 *   - local node and quadrature indices are lexicographic (Sec. 3.1);
 *   - fixed[a*Nx + node] != 0 marks a Dirichlet DOF: the gradient is zero
 *     there, the Hessian row and column are replaced by the identity.
 *
 * Parity pins: every function below is checked by tests/ against values the
 * paper or mathematics fixes (textbook quadrature values, complex-step
 * derivatives, zero energy of the ideal mesh, finite differences, symmetry,
 * convergence of Newton to the uniform mesh, exact remap of linear fields).
 * No function is left without such a pin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXD 3
#define OR_PI 3.14159265358979323846264338327950288L

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_INVERTED = 2, OR_ERR_MINRES = 5,
       OR_ERR_LINESEARCH = 6 };
enum { OR_TARGET_IDENTITY = 0, OR_TARGET_SIZE = 1, OR_TARGET_DISCRETE = 2 };

/* ------------------------------------------------------------------------
 * 1D quadrature and basis (Sec. 3.1, eq. B_G_1D)
 * --------------------------------------------------------------------- */

/* Legendre P_n and P_{n-1} at z by the three-term recurrence. */
static void legendre_pair(int n, long double z, long double *pn, long double *pn1)
{
    long double p0 = 1.0L, p1 = z;
    if (n == 0) { *pn = 1.0L; *pn1 = 0.0L; return; }
    for (int k = 2; k <= n; ++k) {
        long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1; p1 = p2;
    }
    *pn = p1; *pn1 = p0;
}

/* Gauss-Legendre rule with n points mapped to [0,1] (the "standard
 * quadrature rule" of Sec. 2.2 built as a tensor product in Sec. 3.1).
 * Points ascending; weights sum to 1. */
int or_gauss_legendre(int n, double *pts, double *wts)
{
    if (n < 1 || n > 64) return OR_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        long double z = cosl(OR_PI * (k + 0.75L) / (n + 0.5L));
        long double pn = 0, pn1 = 0, dp = 1;
        for (int it = 0; it < 100; ++it) {
            legendre_pair(n, z, &pn, &pn1);
            dp = n * (z * pn - pn1) / (z * z - 1.0L);
            long double dz = pn / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        legendre_pair(n, z, &pn, &pn1);
        dp = n * (z * pn - pn1) / (z * z - 1.0L);
        pts[k] = (double)((1.0L - z) / 2.0L);
        wts[k] = (double)(1.0L / ((1.0L - z * z) * dp * dp));
    }
    return OR_OK;
}

/* Gauss-Lobatto-Legendre nodes (n >= 2) on [0,1]: the end points and the
 * roots of P'_{n-1}.  Newton on P'_N uses P''_N from Legendre's equation. */
int or_gll_nodes(int n, double *pts)
{
    if (n < 2 || n > 64) return OR_ERR_ARG;
    int N = n - 1;
    pts[0] = 0.0; pts[n - 1] = 1.0;
    for (int j = 1; j < N; ++j) {
        long double z = cosl(OR_PI * j / N);
        for (int it = 0; it < 100; ++it) {
            long double pn, pn1;
            legendre_pair(N, z, &pn, &pn1);
            long double d1 = N * (z * pn - pn1) / (z * z - 1.0L);
            long double d2 = (2.0L * z * d1 - N * (N + 1.0L) * pn) / (1.0L - z * z);
            long double dz = d1 / d2;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        pts[j] = (double)((1.0L - z) / 2.0L);
    }
    return OR_OK;
}

/* Lagrange basis l_j(t) and l'_j(t) on the n nodes by the product formula
 * (Sec. 3.1: "standard 1D Lagrange polynomials"). */
void or_lagrange(int n, const double *nodes, double t, double *val, double *der)
{
    for (int j = 0; j < n; ++j) {
        double v = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) v *= (t - nodes[k]) / (nodes[j] - nodes[k]);
        val[j] = v;
        double s = 0.0;
        for (int m = 0; m < n; ++m) {
            if (m == j) continue;
            double prod = 1.0 / (nodes[j] - nodes[m]);
            for (int k = 0; k < n; ++k)
                if (k != j && k != m) prod *= (t - nodes[k]) / (nodes[j] - nodes[k]);
            s += prod;
        }
        der[j] = s;
    }
}

/* ------------------------------------------------------------------------
 * Quality metrics mu(T), dmu/dT and d2mu/dT2 (Sec. 2.2; Sec. 4.1 for mu_303)
 *
 * mu is evaluated from its definition.  The derivatives use the chain rule
 * through the invariants I1 = |T|^2, tau = det T and (3D) I2 = |cof T|^2:
 *   P = sum_u f_u dU,   K = sum_{u,v} f_uv dU (x) dV + sum_u f_u d2U.
 * K is indexed K[(a*d+b)*d*d + (c*d+e)] = d2mu / dT_ab dT_ce.
 * --------------------------------------------------------------------- */

static int lc3(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0;
    return ((i == 0 && j == 1) || (i == 1 && j == 2) || (i == 2 && j == 0)) ? 1 : -1;
}
static int lc2(int i, int j) { return (i == j) ? 0 : (i == 0 ? 1 : -1); }

static double det_def(int d, const double *T)
{
    if (d == 2) return T[0] * T[3] - T[1] * T[2];
    return T[0] * (T[4] * T[8] - T[5] * T[7]) - T[1] * (T[3] * T[8] - T[5] * T[6]) +
           T[2] * (T[3] * T[7] - T[4] * T[6]);
}

/* Inverse by the adjugate; returns det. */
static double inv_def(int d, const double *T, double *Ti)
{
    double t = det_def(d, T);
    if (d == 2) {
        Ti[0] = T[3] / t; Ti[1] = -T[1] / t; Ti[2] = -T[2] / t; Ti[3] = T[0] / t;
        return t;
    }
    Ti[0] = (T[4] * T[8] - T[5] * T[7]) / t;
    Ti[1] = (T[2] * T[7] - T[1] * T[8]) / t;
    Ti[2] = (T[1] * T[5] - T[2] * T[4]) / t;
    Ti[3] = (T[5] * T[6] - T[3] * T[8]) / t;
    Ti[4] = (T[0] * T[8] - T[2] * T[6]) / t;
    Ti[5] = (T[2] * T[3] - T[0] * T[5]) / t;
    Ti[6] = (T[3] * T[7] - T[4] * T[6]) / t;
    Ti[7] = (T[1] * T[6] - T[0] * T[7]) / t;
    Ti[8] = (T[0] * T[4] - T[1] * T[3]) / t;
    return t;
}

/* dtau/dT = cofactor matrix and d2tau/dT2 through Levi-Civita symbols. */
static void det_derivs(int d, const double *T, double *C, double *D2)
{
    int dd = d * d;
    if (d == 2) {
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double s = 0;
                for (int c = 0; c < 2; ++c)
                    for (int e = 0; e < 2; ++e) s += lc2(a, c) * lc2(b, e) * T[c * 2 + e];
                C[a * 2 + b] = s;
                for (int c = 0; c < 2; ++c)
                    for (int e = 0; e < 2; ++e)
                        D2[(a * 2 + b) * dd + c * 2 + e] = lc2(a, c) * lc2(b, e);
            }
        return;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int c = 0; c < 3; ++c)
                for (int e = 0; e < 3; ++e)
                    for (int m = 0; m < 3; ++m)
                        for (int n = 0; n < 3; ++n)
                            s += 0.5 * lc3(a, c, m) * lc3(b, e, n) * T[c * 3 + e] * T[m * 3 + n];
            C[a * 3 + b] = s;
            for (int c = 0; c < 3; ++c)
                for (int e = 0; e < 3; ++e) {
                    double t = 0;
                    for (int m = 0; m < 3; ++m)
                        for (int n = 0; n < 3; ++n)
                            t += lc3(a, c, m) * lc3(b, e, n) * T[m * 3 + n];
                    D2[(a * 3 + b) * dd + c * 3 + e] = t;
                }
        }
}

/* I2 = |cof T|^2 = (I1^2 - |T^T T|^2)/2 (3D), with first and second
 * derivatives from matrix calculus. */
static void i2_derivs(const double *T, double I1, double *I2, double *dI2, double *d2I2)
{
    double TtT[9], TTt[9], TTtT[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0, u = 0;
            for (int k = 0; k < 3; ++k) { s += T[k * 3 + i] * T[k * 3 + j]; u += T[i * 3 + k] * T[j * 3 + k]; }
            TtT[i * 3 + j] = s; TTt[i * 3 + j] = u;
        }
    double n2 = 0;
    for (int i = 0; i < 9; ++i) n2 += TtT[i] * TtT[i];
    *I2 = 0.5 * (I1 * I1 - n2);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += T[i * 3 + k] * TtT[k * 3 + j];
            TTtT[i * 3 + j] = s;
        }
    for (int i = 0; i < 9; ++i) dI2[i] = 2.0 * I1 * T[i] - 2.0 * TTtT[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double v = 4.0 * T[i * 3 + j] * T[k * 3 + l];
                    if (i == k && j == l) v += 2.0 * I1;
                    if (i == k) v -= 2.0 * TtT[l * 3 + j];
                    v -= 2.0 * T[i * 3 + l] * T[k * 3 + j];
                    if (j == l) v -= 2.0 * TTt[i * 3 + k];
                    d2I2[(i * 3 + j) * 9 + k * 3 + l] = v;
                }
}

/* mu, P = dmu/dT, K = d2mu/dT2 for metric id 2 (2D), 302, 303 (3D), 55 (any d),
 * 30355 = mu_303 + mu_55 (3D), and the shape+size metrics of Sec. 2.2
 * 7: mu = |T - T^-t|^2 and 9: mu = tau |T - T^-t|^2 (any d).  P or K may be
 * NULL.  Returns OR_ERR_ARG for an unknown (metric, d) pair and
 * OR_ERR_INVERTED when det T <= 0.
 *
 * mu_7 and mu_9 through the invariants: <T, T^-t> = tr(T^-1 T) = d, so
 * |T - T^-t|^2 = I1 - 2d + |T^-1|^2, with |T^-1|^2 = I2 / tau^2 in 3D and
 * I1 / tau^2 in 2D (the 2D cofactor is a signed permutation of T).  mu itself
 * is evaluated from the definition with the explicit inverse. */
int or_metric(int id, int d, const double *T, double *mu, double *P, double *K)
{
    int dd = d * d;
    double I1 = 0;
    for (int i = 0; i < dd; ++i) I1 += T[i] * T[i];
    double tau = det_def(d, T);
    int ok = (id == 2 && d == 2) || ((id == 302 || id == 303 || id == 30355) && d == 3) ||
             id == 55 || id == 7 || id == 9;
    if (!ok) return OR_ERR_ARG;
    if (!(tau > 0)) return OR_ERR_INVERTED;

    /* f-derivatives: u = (I1, tau, I2) -> index 0,1,2 */
    double f[3] = {0, 0, 0}, ff[3][3] = {{0}};
    double m = 0;
    int use_I2 = 0;
    if (id == 2) {
        m = I1 / (2.0 * tau) - 1.0;
        f[0] = 1.0 / (2.0 * tau);
        f[1] = -I1 / (2.0 * tau * tau);
        ff[0][1] = ff[1][0] = -1.0 / (2.0 * tau * tau);
        ff[1][1] = I1 / (tau * tau * tau);
    }
    if (id == 303 || id == 30355) {
        double c = 1.0 / (cbrt(tau) * cbrt(tau)); /* tau^(-2/3) */
        m += I1 * c / 3.0 - 1.0;
        f[0] += c / 3.0;
        f[1] += -2.0 / 9.0 * I1 * c / tau;
        ff[0][1] += -2.0 / 9.0 * c / tau;
        ff[1][0] += -2.0 / 9.0 * c / tau;
        ff[1][1] += 10.0 / 27.0 * I1 * c / (tau * tau);
    }
    if (id == 55 || id == 30355) {
        m += (tau - 1.0) * (tau - 1.0);
        f[1] += 2.0 * (tau - 1.0);
        ff[1][1] += 2.0;
    }
    if (id == 302) {
        double Ti[9];
        inv_def(3, T, Ti);
        double J = 0;
        for (int i = 0; i < 9; ++i) J += Ti[i] * Ti[i];
        m = I1 * J / 9.0 - 1.0;
        use_I2 = 1;
    }
    if (id == 7 || id == 9) {
        double Ti[9], n2 = 0;
        inv_def(d, T, Ti);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double r = T[a * d + b] - Ti[b * d + a];
                n2 += r * r;
            }
        m = (id == 7) ? n2 : tau * n2;
        if (d == 3) {
            use_I2 = 1;
        } else if (id == 7) {                /* I1 + I1/tau^2 - 4 */
            double t2 = tau * tau;
            f[0] = 1.0 + 1.0 / t2;
            f[1] = -2.0 * I1 / (t2 * tau);
            ff[0][1] = ff[1][0] = -2.0 / (t2 * tau);
            ff[1][1] = 6.0 * I1 / (t2 * t2);
        } else {                             /* tau I1 + I1/tau - 4 tau */
            double t2 = tau * tau;
            f[0] = tau + 1.0 / tau;
            f[1] = I1 - I1 / t2 - 4.0;
            ff[0][1] = ff[1][0] = 1.0 - 1.0 / t2;
            ff[1][1] = 2.0 * I1 / (t2 * tau);
        }
    }
    if (mu) *mu = m;
    if (!P && !K) return OR_OK;

    double dU[3][9], d2U[3][81];
    memset(dU, 0, sizeof(dU));
    memset(d2U, 0, sizeof(d2U));
    for (int i = 0; i < dd; ++i) dU[0][i] = 2.0 * T[i];
    for (int i = 0; i < dd; ++i) d2U[0][i * dd + i] = 2.0;
    det_derivs(d, T, dU[1], d2U[1]);
    if (use_I2) {
        double I2;
        i2_derivs(T, I1, &I2, dU[2], d2U[2]);
        double t2 = tau * tau;
        if (id == 7) {                       /* I1 + I2/tau^2 - 6 */
            f[0] = 1.0;
            f[2] = 1.0 / t2;
            f[1] = -2.0 * I2 / (t2 * tau);
            ff[2][1] = ff[1][2] = -2.0 / (t2 * tau);
            ff[1][1] = 6.0 * I2 / (t2 * t2);
        } else if (id == 9) {                /* tau I1 + I2/tau - 6 tau */
            f[0] = tau;
            f[2] = 1.0 / tau;
            f[1] = I1 - I2 / t2 - 6.0;
            ff[0][1] = ff[1][0] = 1.0;
            ff[2][1] = ff[1][2] = -1.0 / t2;
            ff[1][1] = 2.0 * I2 / (t2 * tau);
        } else {                             /* 302: I1 I2 / (9 tau^2) - 1 */
            f[0] = I2 / (9.0 * t2);
            f[2] = I1 / (9.0 * t2);
            f[1] = -2.0 * I1 * I2 / (9.0 * t2 * tau);
            ff[0][2] = ff[2][0] = 1.0 / (9.0 * t2);
            ff[0][1] = ff[1][0] = -2.0 * I2 / (9.0 * t2 * tau);
            ff[2][1] = ff[1][2] = -2.0 * I1 / (9.0 * t2 * tau);
            ff[1][1] = 2.0 * I1 * I2 / (3.0 * t2 * t2);
        }
    }
    int nu = use_I2 ? 3 : 2;
    if (P)
        for (int i = 0; i < dd; ++i) {
            double s = 0;
            for (int u = 0; u < nu; ++u) s += f[u] * dU[u][i];
            P[i] = s;
        }
    if (K)
        for (int i = 0; i < dd; ++i)
            for (int j = 0; j < dd; ++j) {
                double s = 0;
                for (int u = 0; u < nu; ++u) {
                    s += f[u] * d2U[u][i * dd + j];
                    for (int v = 0; v < nu; ++v) s += ff[u][v] * dU[u][i] * dU[v][j];
                }
                K[i * dd + j] = s;
            }
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Mesh description and full-basis tables
 * --------------------------------------------------------------------- */

typedef struct {
    int dim, order, nq1d;
    int64_t num_elems, num_nodes;
    int metric, target;
    double target_h0;          /* W = h0 * s(x)^(1/d) I for the size target */
    const int32_t *map;        /* num_elems x (order+1)^dim, lexicographic */
    const uint8_t *fixed;      /* dim*num_nodes, or NULL */
    double limit_delta;        /* > 0: limiting term xi = |x - x0|^2 / delta^2 (Sec. 3.5) */
    const double *x0;          /* reference positions of the limiting term */
    const double *eta;         /* discrete target: nodal field eta[node] on the current mesh */
    /* Newton with the discrete target: eta is remapped from (remap_x0,
     * remap_eta0) to every new position (Sec. 3.6) when remap_eta0 != NULL */
    const double *remap_x0, *remap_eta0;
    int remap_steps, remap_cg_max_it;
    double remap_cg_rtol;
} or_mesh;

typedef struct {
    int d, ni, nq, np, nqd;
    double *w;      /* nqd quadrature weights (tensor product) */
    double *phi;    /* [q][i]    basis values at quadrature points */
    double *dphi;   /* [q][i][b] reference gradients */
} or_tables;

static int tables_build(const or_mesh *M, or_tables *t)
{
    int d = M->dim, ni = M->order + 1, nq = M->nq1d;
    if (d < 2 || d > 3 || M->order < 1 || M->order > 8 || nq < 1 || nq > 16) return OR_ERR_ARG;
    double gx[16], gw[16], nodes[16], L[16][16], dL[16][16];
    or_gauss_legendre(nq, gx, gw);
    or_gll_nodes(ni, nodes);
    for (int q = 0; q < nq; ++q) or_lagrange(ni, nodes, gx[q], L[q], dL[q]);
    int np = 1, nqd = 1;
    for (int k = 0; k < d; ++k) { np *= ni; nqd *= nq; }
    t->d = d; t->ni = ni; t->nq = nq; t->np = np; t->nqd = nqd;
    t->w = malloc(sizeof(double) * nqd);
    t->phi = malloc(sizeof(double) * nqd * np);
    t->dphi = malloc(sizeof(double) * nqd * np * d);
    for (int q = 0; q < nqd; ++q) {
        int qk[3] = {q % nq, (q / nq) % nq, q / (nq * nq)};
        double w = 1;
        for (int k = 0; k < d; ++k) w *= gw[qk[k]];
        t->w[q] = w;
        for (int i = 0; i < np; ++i) {
            int ik[3] = {i % ni, (i / ni) % ni, i / (ni * ni)};
            double v = 1;
            for (int k = 0; k < d; ++k) v *= L[qk[k]][ik[k]];
            t->phi[q * np + i] = v;
            for (int b = 0; b < d; ++b) {
                double g = 1;
                for (int k = 0; k < d; ++k) g *= (k == b) ? dL[qk[k]][ik[k]] : L[qk[k]][ik[k]];
                t->dphi[(q * np + i) * d + b] = g;
            }
        }
    }
    return OR_OK;
}

static void tables_free(or_tables *t) { free(t->w); free(t->phi); free(t->dphi); }

/* Size field of the size target, s(x) = 1 + 0.5 prod_k sin(2 pi x_k). */
static double size_field(int d, const double *xq)
{
    double s = 0.5;
    for (int k = 0; k < d; ++k) s *= sin(2.0 * (double)OR_PI * xq[k]);
    return 1.0 + s;
}

/* Target matrix W at a quadrature point of element e (eq. W; Sec. 3.6:
 * recomputed from the current positions, derivative terms dW/dx dropped).
 * Size target: W = h0 s(x_q)^(1/d) I.  Discrete target: W = h0 eta(x_q)^(1/d) I
 * with eta(x_q) = sum_i eta_i w_i(chi_q), the interpolated nodal field; it
 * needs eta(x_q) > 0, else W is undefined and det W is returned as NaN (the
 * callers then treat the point as inverted).  Returns det W and W^-1. */
static double target_at(const or_mesh *M, const or_tables *t, int64_t e, const double *xw_e,
                        int q, double *Winv)
{
    int d = t->d;
    double w = 1.0;
    if (M->target == OR_TARGET_SIZE) {
        double xq[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a)
            for (int i = 0; i < t->np; ++i) xq[a] += xw_e[a * t->np + i] * t->phi[q * t->np + i];
        w = M->target_h0 * pow(size_field(d, xq), 1.0 / d);
    } else if (M->target == OR_TARGET_DISCRETE) {
        double eq = 0;
        for (int i = 0; i < t->np; ++i) eq += M->eta[M->map[e * t->np + i]] * t->phi[q * t->np + i];
        if (!(eq > 0)) {
            for (int k = 0; k < d * d; ++k) Winv[k] = NAN;
            return NAN;
        }
        w = M->target_h0 * pow(eq, 1.0 / d);
    }
    double W[9] = {0};
    for (int a = 0; a < d; ++a) W[a * d + a] = w;
    return inv_def(d, W, Winv);
}

static void gather_elem(const or_mesh *M, const or_tables *t, const double *x, int64_t e, double *xe)
{
    for (int a = 0; a < t->d; ++a)
        for (int i = 0; i < t->np; ++i)
            xe[a * t->np + i] = x[a * M->num_nodes + M->map[e * t->np + i]];
}

/* A_ab = sum_i x_{a,i} d w_i / d xbar_b (eq. A). */
static void jacobian(const or_tables *t, const double *xe, int q, double *A)
{
    int d = t->d;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0;
            for (int i = 0; i < t->np; ++i) s += xe[a * t->np + i] * t->dphi[(q * t->np + i) * d + b];
            A[a * d + b] = s;
        }
}

/* value of the element field u (d components) at point q: sum_i u_i w_i(chi_q) */
static void interp(const or_tables *t, const double *ue, int q, double *out)
{
    for (int a = 0; a < t->d; ++a) {
        double s = 0;
        for (int i = 0; i < t->np; ++i) s += ue[a * t->np + i] * t->phi[q * t->np + i];
        out[a] = s;
    }
}

static int limiting_on(const or_mesh *M) { return M->limit_delta > 0 && M->x0 != NULL; }

static void matmul(int d, const double *X, const double *Y, double *Z)
{
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0;
            for (int k = 0; k < d; ++k) s += X[i * d + k] * Y[k * d + j];
            Z[i * d + j] = s;
        }
}

static int64_t elem_at(const int64_t *elems, int64_t k) { return elems ? elems[k] : k; }

/* ------------------------------------------------------------------------
 * Objective F (eq. F_full, first term; D0 expression of Sec. 3.3)
 *   F = sum_E sum_q w_q det(W) omega mu(A W^-1), omega = 1.
 * xw: positions used for the targets (NULL = x); frozen targets make F a
 * smooth function of x for finite-difference checks.
 * Returns OR_ERR_INVERTED (F = +inf) when det A <= 0 at some point.
 * --------------------------------------------------------------------- */
int or_energy(const or_mesh *M, const double *x, const double *xw, const int64_t *elems,
              int64_t n_elems, double *F_out, double *min_det_out, double *scale_out)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    if (!xw) xw = x;
    if (!elems) n_elems = M->num_elems;
    int d = t.d;
    double *xe = malloc(sizeof(double) * d * t.np), *xwe = malloc(sizeof(double) * d * t.np);
    double *x0e = malloc(sizeof(double) * d * t.np);
    double F = 0, S = 0, mind = INFINITY;
    int inverted = 0;
    for (int64_t k = 0; k < n_elems; ++k) {
        int64_t e = elem_at(elems, k);
        gather_elem(M, &t, x, e, xe);
        gather_elem(M, &t, xw, e, xwe);
        if (limiting_on(M)) gather_elem(M, &t, M->x0, e, x0e);
        for (int q = 0; q < t.nqd; ++q) {
            double A[9], Winv[9], T[9], mu;
            jacobian(&t, xe, q, A);
            double detA = det_def(d, A);
            if (detA < mind) mind = detA;
            double detW = target_at(M, &t, e, xwe, q, Winv);
            if (!(detW > 0)) { inverted = 1; mind = -INFINITY; continue; }   /* undefined target */
            matmul(d, A, Winv, T);
            double c = t.w[q] * detW;
            S += fabs(c);
            if (!(detA > 0)) { inverted = 1; continue; }
            or_metric(M->metric, d, T, &mu, NULL, NULL);
            F += c * mu;
            if (limiting_on(M)) {          /* + integral of |x - x0|^2 / delta^2 (eq. F_full) */
                double xq[3], x0q[3], r2 = 0;
                interp(&t, xe, q, xq);
                interp(&t, x0e, q, x0q);
                for (int a = 0; a < d; ++a) r2 += (xq[a] - x0q[a]) * (xq[a] - x0q[a]);
                F += c * r2 / (M->limit_delta * M->limit_delta);
            }
        }
    }
    free(xe); free(xwe); free(x0e); tables_free(&t);
    if (min_det_out) *min_det_out = mind;
    if (scale_out) *scale_out = S;
    if (inverted) { *F_out = INFINITY; return OR_ERR_INVERTED; }
    *F_out = F;
    return OR_OK;
}

/* det A at every quadrature point of the listed elements, out[k*Nqd + q]
 * (Sec. 2.2, eq. A: A = sum_i x_{E,i} grad w_i^T, the Jacobian of the map from
 * the reference element; det A > 0 is the validity condition the line search
 * of Sec. 2.3 enforces). */
int or_det(const or_mesh *M, const double *x, const int64_t *elems, int64_t n_elems, double *out)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    if (!elems) n_elems = M->num_elems;
    double *xe = malloc(sizeof(double) * t.d * t.np);
    for (int64_t k = 0; k < n_elems; ++k) {
        gather_elem(M, &t, x, elem_at(elems, k), xe);
        for (int q = 0; q < t.nqd; ++q) {
            double A[9];
            jacobian(&t, xe, q, A);
            out[k * t.nqd + q] = det_def(t.d, A);
        }
    }
    free(xe); tables_free(&t);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Gradient (eq. vm_pa_grad with a general W):
 *   dF/dx_{a,i} = sum_q w_q det W sum_b [P(T) W^-T]_{ab} d w_i / d xbar_b,
 * assembled over elements (E-vector to L-vector), zero on fixed DOFs.
 * xw: positions used for the targets (NULL = x), as in or_energy.
 * absg (optional) receives the same sum of absolute values of every term,
 * the scale for condition-aware tolerances.
 * --------------------------------------------------------------------- */
int or_gradient(const or_mesh *M, const double *x, const double *xw, const int64_t *elems,
                int64_t n_elems, double *g, double *absg)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    if (!elems) n_elems = M->num_elems;
    int d = t.d;
    int64_t ndof = (int64_t)d * M->num_nodes;
    memset(g, 0, sizeof(double) * ndof);
    if (absg) memset(absg, 0, sizeof(double) * ndof);
    double *xe = malloc(sizeof(double) * d * t.np), *xwe = malloc(sizeof(double) * d * t.np);
    double *x0e = malloc(sizeof(double) * d * t.np);
    int rc = OR_OK;
    if (!xw) xw = x;
    for (int64_t k = 0; k < n_elems; ++k) {
        int64_t e = elem_at(elems, k);
        gather_elem(M, &t, x, e, xe);
        gather_elem(M, &t, xw, e, xwe);
        if (limiting_on(M)) gather_elem(M, &t, M->x0, e, x0e);
        for (int q = 0; q < t.nqd; ++q) {
            double A[9], Winv[9], T[9], P[9], mu;
            jacobian(&t, xe, q, A);
            double detW = target_at(M, &t, e, xwe, q, Winv);
            if (!(detW > 0)) { rc = OR_ERR_INVERTED; continue; }
            matmul(d, A, Winv, T);
            if (limiting_on(M)) {          /* d/dx_{a,i}: c 2 (x - x0)_a w_i / delta^2 */
                double xq[3], x0q[3], c2 = t.w[q] * detW * 2.0 / (M->limit_delta * M->limit_delta);
                interp(&t, xe, q, xq);
                interp(&t, x0e, q, x0q);
                for (int i = 0; i < t.np; ++i) {
                    int64_t node = M->map[e * t.np + i];
                    for (int a = 0; a < d; ++a) {
                        double term = c2 * (xq[a] - x0q[a]) * t.phi[q * t.np + i];
                        g[a * M->num_nodes + node] += term;
                        if (absg) absg[a * M->num_nodes + node] += fabs(term);
                    }
                }
            }
            if (or_metric(M->metric, d, T, &mu, P, NULL) != OR_OK) { rc = OR_ERR_INVERTED; continue; }
            double c = t.w[q] * detW, PA[9];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double s = 0;
                    for (int n = 0; n < d; ++n) s += P[a * d + n] * Winv[b * d + n];
                    PA[a * d + b] = c * s;
                }
            for (int i = 0; i < t.np; ++i) {
                int64_t node = M->map[e * t.np + i];
                for (int a = 0; a < d; ++a) {
                    double s = 0, sa = 0;
                    for (int b = 0; b < d; ++b) {
                        double term = PA[a * d + b] * t.dphi[(q * t.np + i) * d + b];
                        s += term; sa += fabs(term);
                    }
                    g[a * M->num_nodes + node] += s;
                    if (absg) absg[a * M->num_nodes + node] += sa;
                }
            }
        }
    }
    if (M->fixed)
        for (int64_t j = 0; j < ndof; ++j)
            if (M->fixed[j]) { g[j] = 0; if (absg) absg[j] = 0; }
    free(xe); free(xwe); free(x0e); tables_free(&t);
    return rc;
}

/* H^A_{ab,ce} = w_q det W sum_{n,f} K_{an,cf} W^-1_{bn} W^-1_{ef}: the
 * A-space second derivative at one point (eq. vm_pa_hess with a general W). */
static int hess_A(const or_mesh *M, const or_tables *t, int64_t e, const double *xe, int q,
                  double *HA)
{
    int d = t->d, dd = d * d;
    double A[9], Winv[9], T[9], K[81], mu;
    memset(HA, 0, sizeof(double) * dd * dd);
    jacobian(t, xe, q, A);
    double detW = target_at(M, t, e, xe, q, Winv);
    if (!(detW > 0)) return OR_ERR_INVERTED;
    matmul(d, A, Winv, T);
    int st = or_metric(M->metric, d, T, &mu, NULL, K);
    if (st != OR_OK) return st;
    double c = t->w[q] * detW;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
            for (int cc = 0; cc < d; ++cc)
                for (int ee = 0; ee < d; ++ee) {
                    double s = 0;
                    for (int n = 0; n < d; ++n)
                        for (int f = 0; f < d; ++f)
                            s += K[(a * d + n) * dd + cc * d + f] * Winv[b * d + n] * Winv[ee * d + f];
                    HA[(a * d + b) * dd + cc * d + ee] = c * s;
                }
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Hessian action (eq. vm_pa_hess):
 *   y_{a,i} = sum_{c,j} d2F / dx_{a,i} dx_{c,j} v_{c,j}
 *           = sum_q sum_{b,c,e} H^A_{ab,ce} (sum_j v_{c,j} d_e w_j) d_b w_i,
 * evaluated from x directly (no stored quadrature data).  Fixed DOFs: v is
 * zeroed there on input and y = v there on output.
 * --------------------------------------------------------------------- */
static int hessian_apply_impl(const or_mesh *M, const double *x, const double *v,
                              const int64_t *elems, int64_t n_elems, double *y, double *absy,
                              const double *HAcache)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    if (!elems) n_elems = M->num_elems;
    int d = t.d, dd = d * d;
    int64_t ndof = (int64_t)d * M->num_nodes;
    memset(y, 0, sizeof(double) * ndof);
    if (absy) memset(absy, 0, sizeof(double) * ndof);
    double *xe = malloc(sizeof(double) * d * t.np), *ve = malloc(sizeof(double) * d * t.np);
    int rc = OR_OK;
    for (int64_t k = 0; k < n_elems; ++k) {
        int64_t e = elem_at(elems, k);
        gather_elem(M, &t, x, e, xe);
        for (int a = 0; a < d; ++a)
            for (int i = 0; i < t.np; ++i) {
                int64_t j = a * M->num_nodes + M->map[e * t.np + i];
                ve[a * t.np + i] = (M->fixed && M->fixed[j]) ? 0.0 : v[j];
            }
        for (int q = 0; q < t.nqd; ++q) {
            double Winv0[9];
            if (!(target_at(M, &t, e, xe, q, Winv0) > 0)) { rc = OR_ERR_INVERTED; continue; }
            if (limiting_on(M)) {          /* eq. pa_limiting: c 2/delta^2 w_i sum_j v_{a,j} w_j */
                double Winv[9], vq[3];
                double c2 = t.w[q] * target_at(M, &t, e, xe, q, Winv) * 2.0 /
                            (M->limit_delta * M->limit_delta);
                interp(&t, ve, q, vq);
                for (int i = 0; i < t.np; ++i) {
                    int64_t node = M->map[e * t.np + i];
                    for (int a = 0; a < d; ++a) {
                        double term = c2 * vq[a] * t.phi[q * t.np + i];
                        y[a * M->num_nodes + node] += term;
                        if (absy) absy[a * M->num_nodes + node] += fabs(term);
                    }
                }
            }
            double HAl[81];
            const double *HA = HAl;
            if (HAcache) HA = HAcache + ((int64_t)e * t.nqd + q) * dd * dd;
            else if (hess_A(M, &t, e, xe, q, HAl) != OR_OK) { rc = OR_ERR_INVERTED; continue; }
            double dA[9], Y[9], aY[9];
            jacobian(&t, ve, q, dA);
            for (int r = 0; r < dd; ++r) {
                double s = 0, sa = 0;
                for (int u = 0; u < dd; ++u) { s += HA[r * dd + u] * dA[u]; sa += fabs(HA[r * dd + u] * dA[u]); }
                Y[r] = s; aY[r] = sa;
            }
            for (int i = 0; i < t.np; ++i) {
                int64_t node = M->map[e * t.np + i];
                for (int a = 0; a < d; ++a) {
                    double s = 0, sa = 0;
                    for (int b = 0; b < d; ++b) {
                        double g = t.dphi[(q * t.np + i) * d + b];
                        s += Y[a * d + b] * g; sa += aY[a * d + b] * fabs(g);
                    }
                    y[a * M->num_nodes + node] += s;
                    if (absy) absy[a * M->num_nodes + node] += sa;
                }
            }
        }
    }
    if (M->fixed)
        for (int64_t j = 0; j < ndof; ++j)
            if (M->fixed[j]) { y[j] = v[j]; if (absy) absy[j] = fabs(v[j]); }
    free(xe); free(ve); tables_free(&t);
    return rc;
}

int or_hessian_apply(const or_mesh *M, const double *x, const double *v, const int64_t *elems,
                     int64_t n_elems, double *y, double *absy)
{
    return hessian_apply_impl(M, x, v, elems, n_elems, y, absy, NULL);
}

/* Quadrature-point memo of H^A for all elements, used by the oracle's own
 * Newton solver so that MINRES does not recompute d2mu/dT2 at every
 * iteration.  The values are those hess_A returns; the apply that reads them
 * is the same loop as or_hessian_apply. */
double *or_hess_cache_build(const or_mesh *M, const double *x, int *status)
{
    or_tables t;
    *status = tables_build(M, &t);
    if (*status) return NULL;
    int dd = t.d * t.d;
    double *H = malloc(sizeof(double) * M->num_elems * t.nqd * dd * dd);
    double *xe = malloc(sizeof(double) * t.d * t.np);
    for (int64_t e = 0; e < M->num_elems; ++e) {
        gather_elem(M, &t, x, e, xe);
        for (int q = 0; q < t.nqd; ++q)
            if (hess_A(M, &t, e, xe, q, H + (e * t.nqd + q) * dd * dd) != OR_OK) *status = OR_ERR_INVERTED;
    }
    free(xe); tables_free(&t);
    return H;
}
void or_hess_cache_free(double *H) { free(H); }

int or_hessian_apply_cached(const or_mesh *M, const double *x, const double *HA, const double *v,
                            double *y)
{
    return hessian_apply_impl(M, x, v, NULL, 0, y, NULL, HA);
}

/* ------------------------------------------------------------------------
 * Hessian diagonal (Sec. 3.4, Jacobi preconditioning):
 *   diag_{a,i} = sum_q sum_{b,e} H^A_{ab,ae} d_b w_i d_e w_i, assembled;
 * absd (optional) receives the same sum of the absolute values of every
 * term, the scale of the condition-aware tolerance;
 * 1 on fixed DOFs.
 * --------------------------------------------------------------------- */
int or_hessian_diag(const or_mesh *M, const double *x, const int64_t *elems, int64_t n_elems,
                    double *diag, double *absd)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    if (!elems) n_elems = M->num_elems;
    int d = t.d, dd = d * d;
    int64_t ndof = (int64_t)d * M->num_nodes;
    memset(diag, 0, sizeof(double) * ndof);
    if (absd) memset(absd, 0, sizeof(double) * ndof);
    double *xe = malloc(sizeof(double) * d * t.np);
    int rc = OR_OK;
    for (int64_t k = 0; k < n_elems; ++k) {
        int64_t e = elem_at(elems, k);
        gather_elem(M, &t, x, e, xe);
        for (int q = 0; q < t.nqd; ++q) {
            double Winv0[9];
            if (!(target_at(M, &t, e, xe, q, Winv0) > 0)) { rc = OR_ERR_INVERTED; continue; }
            if (limiting_on(M)) {          /* c 2/delta^2 w_i^2 */
                double Winv[9];
                double c2 = t.w[q] * target_at(M, &t, e, xe, q, Winv) * 2.0 /
                            (M->limit_delta * M->limit_delta);
                for (int i = 0; i < t.np; ++i) {
                    int64_t node = M->map[e * t.np + i];
                    double ph = t.phi[q * t.np + i];
                    for (int a = 0; a < d; ++a) {
                        diag[a * M->num_nodes + node] += c2 * ph * ph;
                        if (absd) absd[a * M->num_nodes + node] += fabs(c2 * ph * ph);
                    }
                }
            }
            double HA[81];
            if (hess_A(M, &t, e, xe, q, HA) != OR_OK) { rc = OR_ERR_INVERTED; continue; }
            for (int i = 0; i < t.np; ++i) {
                int64_t node = M->map[e * t.np + i];
                const double *gi = t.dphi + (q * t.np + i) * d;
                for (int a = 0; a < d; ++a) {
                    double s = 0, sa = 0;
                    for (int b = 0; b < d; ++b)
                        for (int e2 = 0; e2 < d; ++e2) {
                            const double term = HA[(a * d + b) * dd + a * d + e2] * gi[b] * gi[e2];
                            s += term;
                            sa += fabs(term);
                        }
                    diag[a * M->num_nodes + node] += s;
                    if (absd) absd[a * M->num_nodes + node] += sa;
                }
            }
        }
    }
    if (M->fixed)
        for (int64_t j = 0; j < ndof; ++j)
            if (M->fixed[j]) {
                diag[j] = 1.0;
                if (absd) absd[j] = 1.0;
            }
    free(xe); tables_free(&t);
    return rc;
}

/* ------------------------------------------------------------------------
 * Jacobi-preconditioned MINRES (Sec. 2.3 and 3.4; Paige & Saunders 1975)
 * for H dx = b with M^-1 = 1/|diag| (1 where |diag| < 1e-300), x0 = 0.
 * Stops when the preconditioned residual estimate phibar <= rtol * beta1
 * (beta1 = ||b||_{M^-1}), or after max_it iterations (fixed_its = 1 runs
 * exactly max_it iterations).
 * --------------------------------------------------------------------- */
typedef struct {
    const or_mesh *M; const double *x; const double *HA;
} or_op;

static void op_apply(const or_op *op, const double *v, double *y)
{
    or_hessian_apply_cached(op->M, op->x, op->HA, v, y);
}

static double dotv(int64_t n, const double *a, const double *b)
{
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

int or_minres(const or_mesh *M, const double *x, const double *HA, const double *diag,
              const double *b, double rtol, int max_it, int fixed_its, double *dx,
              int *iters_out, double *resid_out)
{
    int64_t n = (int64_t)M->dim * M->num_nodes;
    or_op op = {M, x, HA};
    double *minv = malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) {
        double a = fabs(diag[i]);
        minv[i] = (a < 1e-300) ? 1.0 : 1.0 / a;
    }
    double *r1 = calloc(n, sizeof(double)), *r2 = calloc(n, sizeof(double));
    double *y = calloc(n, sizeof(double)), *v = calloc(n, sizeof(double));
    double *w1 = calloc(n, sizeof(double)), *w2 = calloc(n, sizeof(double));
    memset(dx, 0, sizeof(double) * n);
    /* Lanczos start: r1 = r2 = b, y = M^-1 b, beta1 = sqrt(b . M^-1 b) */
    for (int64_t i = 0; i < n; ++i) { r1[i] = b[i]; r2[i] = b[i]; y[i] = minv[i] * b[i]; }
    double beta1 = sqrt(dotv(n, b, y));
    double beta = beta1, beta_old = 0, dbar = 0, eps_k = 0, phibar = beta1, cs = -1, sn = 0;
    int k = 0, rc = OR_OK;
    if (beta1 > 0) {
        for (k = 1; k <= max_it; ++k) {
            /* Lanczos step: v_k = y / beta_k, y = H v_k - (beta_k/beta_{k-1}) r1 */
            for (int64_t i = 0; i < n; ++i) v[i] = y[i] / beta;
            op_apply(&op, v, y);
            if (k >= 2)
                for (int64_t i = 0; i < n; ++i) y[i] -= (beta / beta_old) * r1[i];
            double alpha = dotv(n, v, y);
            for (int64_t i = 0; i < n; ++i) y[i] -= (alpha / beta) * r2[i];
            double *tmp = r1; r1 = r2; r2 = y; y = tmp;      /* r1 <- r2, r2 <- y */
            for (int64_t i = 0; i < n; ++i) y[i] = minv[i] * r2[i];
            beta_old = beta;
            double bb = dotv(n, r2, y);
            if (bb < 0) { rc = OR_ERR_MINRES; break; }
            beta = sqrt(bb);
            /* previous Givens rotation applied to the new tridiagonal column */
            double eps_old = eps_k;
            double delta = cs * dbar + sn * alpha;
            double gbar = sn * dbar - cs * alpha;
            eps_k = sn * beta;
            dbar = -cs * beta;
            /* new rotation annihilating beta_{k+1} */
            double gamma = sqrt(gbar * gbar + beta * beta);
            if (gamma < 1e-300) gamma = 1e-300;
            cs = gbar / gamma;
            sn = beta / gamma;
            double phi = cs * phibar;
            phibar = sn * phibar;
            /* search direction and solution update */
            for (int64_t i = 0; i < n; ++i) {
                double wn = (v[i] - eps_old * w1[i] - delta * w2[i]) / gamma;
                w1[i] = w2[i]; w2[i] = wn;
                dx[i] += phi * wn;
            }
            if (!fixed_its && phibar <= rtol * beta1) break;
            if (beta == 0) break;
        }
        if (k > max_it) k = max_it;
    }
    if (iters_out) *iters_out = k;
    if (resid_out) *resid_out = (beta1 > 0) ? phibar / beta1 : 0.0;
    free(minv); free(r1); free(r2); free(y); free(v); free(w1); free(w2);
    return rc;
}

/* ------------------------------------------------------------------------
 * One Newton step with backtracking line search (Sec. 2.3, eq. nodal_solve
 * and nodal_dx):  dx = [d2F]^-1 dF by Jacobi-MINRES, x+ = x - alpha dx,
 * alpha = 1, 1/2, ... until det A(x+) > 0 at every point,
 * F(x+) < ls_factor F(x) and |dF(x+)| < ls_factor |dF(x)|.  x is overwritten
 * only when a step is accepted.
 * --------------------------------------------------------------------- */
/* ------------------------------------------------------------------------
 * Adaptive discrete target and its advection remap (Sec. 3.6)
 *
 * The discrete target reads a finite element field eta of the mesh's own
 * space (nodal values eta[node]).  The field is given on positions x0; on
 * positions x1 its values come from the pseudo-time advection
 *     d eta / dt = v . grad eta,   v = x1 - x0,   x_t = x0 + t v,  t in [0, 1],
 * discretised by Galerkin in the same space, whose basis functions move with
 * the nodes:
 *     M(x_t) d eta/dt = K(x_t) eta,
 *     M_ij = int w_i w_j dx,   K_ij = int w_i v . grad_x w_j dx   (mesh x_t),
 * integrated with the mesh's quadrature rule (grad_x = A^-T grad_xbar).
 * Pseudo-time integration: the classical fourth-order Runge-Kutta method with
 * n uniform steps; every stage solves M k = K eta with Jacobi-preconditioned
 * CG from a zero initial guess.
 * --------------------------------------------------------------------- */

static void gather_scalar(const or_mesh *M, const or_tables *t, const double *u, int64_t e, double *ue)
{
    for (int i = 0; i < t->np; ++i) ue[i] = u[M->map[e * t->np + i]];
}

/* y = M(x) u, y_i = sum_E sum_q w_q det A_q w_i(chi_q) u(chi_q).  Returns
 * OR_ERR_INVERTED (after computing y) when det A <= 0 at some point. */
int or_mass_apply(const or_mesh *M, const double *x, const double *u, double *y)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    int d = t.d, rc = OR_OK;
    memset(y, 0, sizeof(double) * M->num_nodes);
    double *xe = malloc(sizeof(double) * d * t.np), *ue = malloc(sizeof(double) * t.np);
    for (int64_t e = 0; e < M->num_elems; ++e) {
        gather_elem(M, &t, x, e, xe);
        gather_scalar(M, &t, u, e, ue);
        for (int q = 0; q < t.nqd; ++q) {
            double A[9], uq = 0;
            jacobian(&t, xe, q, A);
            double detA = det_def(d, A);
            if (!(detA > 0)) rc = OR_ERR_INVERTED;
            for (int j = 0; j < t.np; ++j) uq += ue[j] * t.phi[q * t.np + j];
            double c = t.w[q] * detA * uq;
            for (int i = 0; i < t.np; ++i) y[M->map[e * t.np + i]] += c * t.phi[q * t.np + i];
        }
    }
    free(xe); free(ue); tables_free(&t);
    return rc;
}

/* diag M(x), sum_E sum_q w_q det A_q w_i(chi_q)^2. */
int or_mass_diag(const or_mesh *M, const double *x, double *diag)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    int d = t.d, rc = OR_OK;
    memset(diag, 0, sizeof(double) * M->num_nodes);
    double *xe = malloc(sizeof(double) * d * t.np);
    for (int64_t e = 0; e < M->num_elems; ++e) {
        gather_elem(M, &t, x, e, xe);
        for (int q = 0; q < t.nqd; ++q) {
            double A[9];
            jacobian(&t, xe, q, A);
            double detA = det_def(d, A);
            if (!(detA > 0)) rc = OR_ERR_INVERTED;
            for (int i = 0; i < t.np; ++i) {
                double ph = t.phi[q * t.np + i];
                diag[M->map[e * t.np + i]] += t.w[q] * detA * ph * ph;
            }
        }
    }
    free(xe); tables_free(&t);
    return rc;
}

/* y = K(x, vel) u, y_i = sum_E sum_q w_q det A_q w_i(chi_q) vel(chi_q) . grad_x u(chi_q),
 * grad_x u = A_q^-T grad_xbar u.  vel has the layout of x. */
int or_advect_apply(const or_mesh *M, const double *x, const double *vel, const double *u, double *y)
{
    or_tables t;
    int st = tables_build(M, &t);
    if (st) return st;
    int d = t.d, rc = OR_OK;
    memset(y, 0, sizeof(double) * M->num_nodes);
    double *xe = malloc(sizeof(double) * d * t.np), *ve = malloc(sizeof(double) * d * t.np);
    double *ue = malloc(sizeof(double) * t.np);
    for (int64_t e = 0; e < M->num_elems; ++e) {
        gather_elem(M, &t, x, e, xe);
        gather_elem(M, &t, vel, e, ve);
        gather_scalar(M, &t, u, e, ue);
        for (int q = 0; q < t.nqd; ++q) {
            double A[9], Ai[9], vq[3], gref[3] = {0, 0, 0}, gx[3];
            jacobian(&t, xe, q, A);
            double detA = inv_def(d, A, Ai);
            if (!(detA > 0)) { rc = OR_ERR_INVERTED; continue; }
            interp(&t, ve, q, vq);
            for (int j = 0; j < t.np; ++j)
                for (int b = 0; b < d; ++b) gref[b] += ue[j] * t.dphi[(q * t.np + j) * d + b];
            double vg = 0;
            for (int a = 0; a < d; ++a) {          /* (A^-T gref)_a = sum_b Ai_ba gref_b */
                gx[a] = 0;
                for (int b = 0; b < d; ++b) gx[a] += Ai[b * d + a] * gref[b];
                vg += vq[a] * gx[a];
            }
            double c = t.w[q] * detA * vg;
            for (int i = 0; i < t.np; ++i) y[M->map[e * t.np + i]] += c * t.phi[q * t.np + i];
        }
    }
    free(xe); free(ve); free(ue); tables_free(&t);
    return rc;
}

/* Jacobi-preconditioned CG for M(x) k = b from k = 0.  Stops when
 * sqrt(r.z) <= rtol sqrt(b.D^-1 b) (z = D^-1 r) or after max_it iterations;
 * returns the iterations done. */
static int mass_cg(const or_mesh *M, const double *x, const double *diag, const double *b,
                   double rtol, int max_it, double *k)
{
    int64_t n = M->num_nodes;
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *Mp = malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) { k[i] = 0; r[i] = b[i]; z[i] = r[i] / diag[i]; p[i] = z[i]; }
    double rz = dotv(n, r, z), stop = rtol * rtol * rz;
    int it = 0;
    while (it < max_it && rz > stop && rz > 0) {
        or_mass_apply(M, x, p, Mp);
        double alpha = rz / dotv(n, p, Mp);
        for (int64_t i = 0; i < n; ++i) { k[i] += alpha * p[i]; r[i] -= alpha * Mp[i]; z[i] = r[i] / diag[i]; }
        double rz1 = dotv(n, r, z);
        double beta = rz1 / rz;
        rz = rz1;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        ++it;
    }
    free(r); free(z); free(p); free(Mp);
    return it;
}

/* eta1 = eta0 advected from positions x0 to x1 (see above).  cg_its (optional)
 * receives the total CG iterations.  Returns OR_ERR_INVERTED when an
 * intermediate mesh x_t has det A <= 0 at some point (eta1 then undefined). */
int or_remap(const or_mesh *M, const double *x0, const double *x1, const double *eta0, int nsteps,
             double cg_rtol, int cg_max_it, double *eta1, int *cg_its)
{
    if (nsteps < 1) return OR_ERR_ARG;
    int64_t Nx = M->num_nodes, nd = (int64_t)M->dim * Nx;
    double *v = malloc(sizeof(double) * nd), *xt = malloc(sizeof(double) * nd);
    double *diag = malloc(sizeof(double) * Nx), *rhs = malloc(sizeof(double) * Nx);
    double *es = malloc(sizeof(double) * Nx), *kk[4];
    for (int s = 0; s < 4; ++s) kk[s] = malloc(sizeof(double) * Nx);
    for (int64_t i = 0; i < nd; ++i) v[i] = x1[i] - x0[i];
    memcpy(eta1, eta0, sizeof(double) * Nx);
    const double dt = 1.0 / nsteps;
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};      /* stage times (fractions of dt) */
    const double ast[4] = {0.0, 0.5, 0.5, 1.0};      /* stage increments a_{s,s-1} */
    int rc = OR_OK, total = 0;
    for (int n = 0; n < nsteps && rc == OR_OK; ++n) {
        for (int s = 0; s < 4; ++s) {
            double tt = (n + cst[s]) * dt;
            for (int64_t i = 0; i < nd; ++i) xt[i] = x0[i] + tt * v[i];
            for (int64_t i = 0; i < Nx; ++i) es[i] = eta1[i] + (s ? ast[s] * dt * kk[s - 1][i] : 0.0);
            if (or_mass_diag(M, xt, diag) != OR_OK) { rc = OR_ERR_INVERTED; break; }
            or_advect_apply(M, xt, v, es, rhs);
            total += mass_cg(M, xt, diag, rhs, cg_rtol, cg_max_it, kk[s]);
        }
        if (rc != OR_OK) break;
        for (int64_t i = 0; i < Nx; ++i)
            eta1[i] += dt / 6.0 * (kk[0][i] + 2.0 * kk[1][i] + 2.0 * kk[2][i] + kk[3][i]);
    }
    if (cg_its) *cg_its = total;
    free(v); free(xt); free(diag); free(rhs); free(es);
    for (int s = 0; s < 4; ++s) free(kk[s]);
    return rc;
}

static int remap_on(const or_mesh *M)
{
    return M->target == OR_TARGET_DISCRETE && M->remap_eta0 != NULL && M->remap_x0 != NULL;
}

typedef struct {
    double energy, grad_norm, energy_new, grad_norm_new, alpha, min_det, minres_resid;
    int minres_iters, halvings, status;
} or_report;

int or_newton_step(const or_mesh *M, double *x, double minres_rtol, int minres_max_it,
                   int minres_fixed_its, double ls_factor, int ls_max_halvings, or_report *rep)
{
    int64_t n = (int64_t)M->dim * M->num_nodes;
    memset(rep, 0, sizeof(*rep));
    /* discrete target with a remap source: eta follows every position change
     * (Sec. 3.6), at x and at each line-search trial */
    or_mesh Mx = *M, Mt = *M;
    double *eta_x = NULL, *eta_t = NULL;
    if (remap_on(M)) {
        eta_x = malloc(sizeof(double) * M->num_nodes);
        eta_t = malloc(sizeof(double) * M->num_nodes);
        int rst = or_remap(M, M->remap_x0, x, M->remap_eta0, M->remap_steps, M->remap_cg_rtol,
                           M->remap_cg_max_it, eta_x, NULL);
        if (rst) { free(eta_x); free(eta_t); rep->status = rst; return rst; }
        Mx.eta = eta_x;
        Mt.eta = eta_t;
    }
    M = &Mx;
    double F0, mind;
    int st = or_energy(M, x, NULL, NULL, 0, &F0, &mind, NULL);
    rep->energy = F0; rep->min_det = mind;
    if (st) { rep->status = st; free(eta_x); free(eta_t); return st; }
    double *g = malloc(sizeof(double) * n), *diag = malloc(sizeof(double) * n);
    double *dx = malloc(sizeof(double) * n), *xt = malloc(sizeof(double) * n);
    or_gradient(M, x, NULL, NULL, 0, g, NULL);
    double g0 = sqrt(dotv(n, g, g));
    rep->grad_norm = g0;
    if (g0 == 0) {               /* already stationary: nothing to solve */
        rep->energy_new = F0; rep->status = OR_OK;
        free(g); free(diag); free(dx); free(xt); free(eta_x); free(eta_t);
        return OR_OK;
    }
    double *HA = or_hess_cache_build(M, x, &st);
    or_hessian_diag(M, x, NULL, 0, diag, NULL);
    int its = 0;
    double res = 0;
    int mst = or_minres(M, x, HA, diag, g, minres_rtol, minres_max_it, minres_fixed_its, dx, &its, &res);
    rep->minres_iters = its; rep->minres_resid = res;
    or_hess_cache_free(HA);
    int rc = OR_ERR_LINESEARCH;
    if (mst == OR_OK) {
        double alpha = 1.0;
        for (int h = 0; h <= ls_max_halvings; ++h, alpha *= 0.5) {
            for (int64_t i = 0; i < n; ++i) xt[i] = x[i] - alpha * dx[i];
            double F1, md1;
            const or_mesh *MT = M;
            if (eta_t) {
                if (or_remap(M, M->remap_x0, xt, M->remap_eta0, M->remap_steps, M->remap_cg_rtol,
                             M->remap_cg_max_it, eta_t, NULL) != OR_OK)
                    continue;                                   /* x_t inverted on the way */
                MT = &Mt;
            }
            int est = or_energy(MT, xt, NULL, NULL, 0, &F1, &md1, NULL);
            if (est != OR_OK || !(md1 > 0)) continue;          /* det A > 0 */
            if (!(F1 < ls_factor * F0)) continue;               /* energy */
            or_gradient(MT, xt, NULL, NULL, 0, g, NULL);
            double g1 = sqrt(dotv(n, g, g));
            if (!(g1 < ls_factor * g0)) continue;               /* gradient */
            memcpy(x, xt, sizeof(double) * n);
            rep->alpha = alpha; rep->halvings = h;
            rep->energy_new = F1; rep->grad_norm_new = g1; rep->min_det = md1;
            rc = OR_OK;
            break;
        }
    } else {
        rc = mst;
    }
    rep->status = rc;
    free(g); free(diag); free(dx); free(xt); free(eta_x); free(eta_t);
    return rc;
}
