// Host-side 1D tables of the tensor-product basis (paper Sec. 3.1,
// eq. B_G_1D): Gauss-Legendre points and weights on [0,1], Gauss-Lobatto-
// Legendre nodes, and B_qi = l_i(chi_q), G_qi = l_i'(chi_q) for the Lagrange
// polynomials l_i on those nodes.  Computed in long double, stored FP64.
#include <cmath>

#include "tmop_internal.h"

namespace tmop {

namespace {

const long double kPi = 3.141592653589793238462643383279502884L;

// (P_n(t), P_n'(t)) on [-1,1] by the Bonnet recurrence.
void legendre(int n, long double t, long double &pn, long double &dpn)
{
    long double a = 1.0L, b = t;
    if (n == 0) { pn = 1.0L; dpn = 0.0L; return; }
    for (int k = 2; k <= n; ++k) {
        const long double c = ((2.0L * k - 1.0L) * t * b - (k - 1.0L) * a) / k;
        a = b;
        b = c;
    }
    pn = b;
    dpn = n * (a - t * b) / (1.0L - t * t);
}

}  // namespace

void host_gauss_legendre(int n, double *x, double *w)
{
    for (int j = 0; j < n; ++j) {
        // Tricomi's initial guess, refined by Newton on P_n
        long double t = cosl(kPi * (4.0L * j + 3.0L) / (4.0L * n + 2.0L));
        long double pn = 0, dp = 1;
        for (int it = 0; it < 64; ++it) {
            legendre(n, t, pn, dp);
            const long double step = pn / dp;
            t -= step;
            if (fabsl(step) <= 1e-20L) break;
        }
        legendre(n, t, pn, dp);
        // ascending order on [0,1]: t_j decreases with j
        x[j] = (double)(0.5L * (1.0L - t));
        w[j] = (double)(1.0L / ((1.0L - t * t) * dp * dp));
    }
}

void host_gll_nodes(int n, double *x)
{
    const int N = n - 1;
    x[0] = 0.0;
    x[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        // interior nodes: roots of P_N', Newton with P_N'' from Legendre's equation
        long double t = cosl(kPi * j / N);
        for (int it = 0; it < 64; ++it) {
            long double pn, dp;
            legendre(N, t, pn, dp);
            const long double d2 = (2.0L * t * dp - N * (N + 1.0L) * pn) / (1.0L - t * t);
            const long double step = dp / d2;
            t -= step;
            if (fabsl(step) <= 1e-20L) break;
        }
        x[j] = (double)(0.5L * (1.0L - t));
    }
}

void host_basis_tables(int ni, int nq, double *B, double *G, double *w1d)
{
    double nodes[16], pts[16];
    host_gll_nodes(ni, nodes);
    host_gauss_legendre(nq, pts, w1d);
    // barycentric weights lambda_i = 1 / prod_{k != i} (x_i - x_k)
    long double lam[16];
    for (int i = 0; i < ni; ++i) {
        long double p = 1.0L;
        for (int k = 0; k < ni; ++k)
            if (k != i) p *= (long double)nodes[i] - nodes[k];
        lam[i] = 1.0L / p;
    }
    for (int q = 0; q < nq; ++q) {
        const long double t = pts[q];
        for (int i = 0; i < ni; ++i) {
            // l_i(t) = lambda_i prod_{k != i} (t - x_k)
            long double v = lam[i];
            for (int k = 0; k < ni; ++k)
                if (k != i) v *= t - nodes[k];
            // l_i'(t) = lambda_i sum_{m != i} prod_{k != i, m} (t - x_k)
            long double dv = 0.0L;
            for (int m = 0; m < ni; ++m) {
                if (m == i) continue;
                long double pr = 1.0L;
                for (int k = 0; k < ni; ++k)
                    if (k != i && k != m) pr *= t - nodes[k];
                dv += pr;
            }
            B[q * ni + i] = (double)v;
            G[q * ni + i] = (double)(lam[i] * dv);
        }
    }
}

// Collocated derivative on the Gauss points: D_qk = m_k'(chi_q) for the
// Lagrange polynomials m_k through the nq Gauss-Legendre points (barycentric
// form).  A polynomial of degree < nq is reproduced exactly by its values at
// the points, so G = D B for the GLL basis of any order p <= nq - 1 (the
// reference gradient of a nodal field is D applied to its values at the
// points).  Long double, stored FP64.
void host_colloc_deriv(int nq, double *D)
{
    double pts[16], w[16];
    host_gauss_legendre(nq, pts, w);
    long double lam[16];
    for (int k = 0; k < nq; ++k) {
        long double p = 1.0L;
        for (int m = 0; m < nq; ++m)
            if (m != k) p *= (long double)pts[k] - pts[m];
        lam[k] = 1.0L / p;
    }
    for (int q = 0; q < nq; ++q) {
        long double diag = 0.0L;
        for (int k = 0; k < nq; ++k) {
            if (k == q) continue;
            const long double dqk = (long double)pts[q] - pts[k];
            D[q * nq + k] = (double)(lam[k] / (lam[q] * dqk));
            diag += 1.0L / dqk;
        }
        D[q * nq + q] = (double)diag;
    }
}

}  // namespace tmop
