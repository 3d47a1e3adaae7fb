// Geometric factors of trilinear hexahedra at the GLL nodes (set-up kernel).
//
// For element corners X_q (q = di + 2dj + 4dk) the map is
// x(r,s,t) = sum_q X_q (1 + sr r)(1 + ss s)(1 + st t)/8 with s* = +-1.  Its
// columns x_r, x_s, x_t give |J| = x_r . (x_s x x_t) and the contravariant
// gradients grad r = (x_s x x_t)/|J| (cyclically), so
// G_ab = rho_i rho_j rho_k |J| grad r_a . grad r_b, stored (rr,rs,rt,ss,st,tt).
#include "nek_internal.h"

namespace nek {

struct GllParams {
    double xi[kMaxNx];
    double rho[kMaxNx];
};

__global__ void k_geom(int64_t nelt, int nx, GllParams gp, const double* __restrict__ corners,
                       double* __restrict__ G)
{
    const int64_t n3 = (int64_t)nx * nx * nx;
    const int64_t total = nelt * n3;
    for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < total;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = gid / n3;
        const int p = static_cast<int>(gid - e * n3);
        const int i = p % nx, j = (p / nx) % nx, k = p / (nx * nx);
        const double r = gp.xi[i], s = gp.xi[j], t = gp.xi[k];
        const double* X = corners + e * 24;
        double a[3] = {0, 0, 0}, b[3] = {0, 0, 0}, c[3] = {0, 0, 0};  // x_r, x_s, x_t
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const double sr = (q & 1) ? 1.0 : -1.0, ss = (q & 2) ? 1.0 : -1.0, st = (q & 4) ? 1.0 : -1.0;
            const double fr = 1.0 + sr * r, fs = 1.0 + ss * s, ft = 1.0 + st * t;
            const double dr = 0.125 * sr * fs * ft, ds = 0.125 * ss * fr * ft, dt = 0.125 * st * fr * fs;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const double xq = X[q * 3 + d];
                a[d] += dr * xq;
                b[d] += ds * xq;
                c[d] += dt * xq;
            }
        }
        const double bc0 = b[1] * c[2] - b[2] * c[1], bc1 = b[2] * c[0] - b[0] * c[2], bc2 = b[0] * c[1] - b[1] * c[0];
        const double ca0 = c[1] * a[2] - c[2] * a[1], ca1 = c[2] * a[0] - c[0] * a[2], ca2 = c[0] * a[1] - c[1] * a[0];
        const double ab0 = a[1] * b[2] - a[2] * b[1], ab1 = a[2] * b[0] - a[0] * b[2], ab2 = a[0] * b[1] - a[1] * b[0];
        const double det = a[0] * bc0 + a[1] * bc1 + a[2] * bc2;
        // G_ab = W |J| (v_a/|J|).(v_b/|J|) = W (v_a . v_b) / |J|
        const double wq = gp.rho[i] * gp.rho[j] * gp.rho[k] / det;
        double* g = G + gid * 6;
        g[0] = wq * (bc0 * bc0 + bc1 * bc1 + bc2 * bc2);
        g[1] = wq * (bc0 * ca0 + bc1 * ca1 + bc2 * ca2);
        g[2] = wq * (bc0 * ab0 + bc1 * ab1 + bc2 * ab2);
        g[3] = wq * (ca0 * ca0 + ca1 * ca1 + ca2 * ca2);
        g[4] = wq * (ca0 * ab0 + ca1 * ab1 + ca2 * ab2);
        g[5] = wq * (ab0 * ab0 + ab1 * ab1 + ab2 * ab2);
    }
}

}  // namespace nek

using namespace nek;

extern "C" nek_status nek_geom(int64_t nelt, int nx, const double* corners, double* G, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!corners || !G || !is_aligned(corners, 8) || !is_aligned(G, 16)) return NEK_ERR_INVALID_ARG;
    GllParams gp;
    gll_host(nx, gp.xi, gp.rho, nullptr);
    const int64_t total = nelt * (int64_t)nx * nx * nx;
    const int64_t nb = (total + 255) / 256;
    const int blocks = static_cast<int>(nb < 152 * 64 ? nb : 152 * 64);
    k_geom<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(nelt, nx, gp, corners, G);
    return check_launch();
}
