// Gauss-Lobatto-Legendre rule on nx points, computed on the host.
//
// The interior nodes are the roots of L'_N (N = nx-1).  They are found by
// Newton's method from the Chebyshev-Gauss-Lobatto points -cos(pi j/N), with
// L_N and its first two derivatives from the three-term Legendre recurrence and
// the Legendre differential equation.  Weights rho_i = 2/(N(N+1) L_N(xi_i)^2);
// D[i][l] = l_l'(xi_i) = L_N(xi_i)/(L_N(xi_l)(xi_i - xi_l)) off the diagonal and
// -/+ N(N+1)/4 at the two end points, 0 elsewhere on the diagonal.
#include <cmath>

#include "nek_internal.h"

namespace nek {

namespace {

// L_N(x), L_N'(x), L_N''(x) for |x| < 1 (and L_N only at |x| = 1).
void legendre3(int N, double x, double* p, double* dp, double* d2p)
{
    double pm1 = 1.0, pk = x;
    if (N == 0) pk = 1.0;
    for (int k = 1; k < N; k++) {
        double pn = ((2.0 * k + 1.0) * x * pk - k * pm1) / (k + 1.0);
        pm1 = pk;
        pk = pn;
    }
    *p = pk;
    double one_m = 1.0 - x * x;
    if (one_m > 0.0) {
        // (1-x^2) L' = N (L_{N-1} - x L_N);  (1-x^2) L'' = 2x L' - N(N+1) L
        *dp = N * (pm1 - x * pk) / one_m;
        *d2p = (2.0 * x * (*dp) - N * (N + 1.0) * pk) / one_m;
    } else {
        *dp = 0.0;
        *d2p = 0.0;
    }
}

}  // namespace

void gll_host(int nx, double* xi, double* rho, double* D)
{
    const int N = nx - 1;
    double z[kMaxNx], LN[kMaxNx];
    z[0] = -1.0;
    z[N] = 1.0;
    for (int j = 1; j < N; j++) {
        double x = -std::cos(M_PI * j / N);
        for (int it = 0; it < 100; it++) {
            double p, dp, d2p;
            legendre3(N, x, &p, &dp, &d2p);
            double dx = dp / d2p;
            x -= dx;
            if (std::fabs(dx) <= 1e-17) break;
        }
        z[j] = x;
    }
    // exact symmetry of the rule
    for (int j = 0; j < nx / 2; j++) {
        double a = 0.5 * (z[N - j] - z[j]);
        z[j] = -a;
        z[N - j] = a;
    }
    if (nx % 2) z[N / 2] = 0.0;
    for (int i = 0; i < nx; i++) {
        double p, dp, d2p;
        legendre3(N, z[i], &p, &dp, &d2p);
        LN[i] = p;
    }
    if (xi)
        for (int i = 0; i < nx; i++) xi[i] = z[i];
    if (rho)
        for (int i = 0; i < nx; i++) rho[i] = 2.0 / (N * (N + 1.0) * LN[i] * LN[i]);
    if (D) {
        for (int i = 0; i < nx; i++)
            for (int l = 0; l < nx; l++)
                D[i * nx + l] = (i == l) ? 0.0 : LN[i] / (LN[l] * (z[i] - z[l]));
        D[0] = -N * (N + 1.0) / 4.0;
        D[N * nx + N] = N * (N + 1.0) / 4.0;
    }
}

}  // namespace nek
