/*
 * Oracle for the Nekbone AX solve path: plain, slow, obviously correct FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links or calls this
 * file; only tests/, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py do.  It shares no code, header, table or constant with the CUDA
 * library.  Compiled with -ffp-contract=off so that every a*b+c is two rounded
 * operations on every host (x86_64 here, aarch64 on the GPU node).
 *
 * Paper: N. Brown, "Exploring the acceleration of Nekbone on reconfigurable
 * architectures" (arXiv 2011.04981).  Section II-B, Listing 1 gives the
 * element operator ax / ax_e / local_grad3; the same section states that the
 * CG iteration is vector operations + this operator + nearest-neighbour
 * exchange + global reductions, with a basic preconditioner.  Everything
 * the paper leaves open is read as the standard spectral-element definition;
 * each function says which reading it takes.
 *
 * OpenMP: the element loop of ref_ax, the group loop of ref_dssum and the
 * pointwise loops of ref_pcg carry "omp parallel for" pragmas.  They split
 * independent iterations only (elements, disjoint groups, points) and leave the
 * dot products serial, so a build with -fopenmp computes every value with the
 * same operations in the same order as the default build (which ignores the
 * pragmas); it exists only to time the oracle on all host cores.
 *
 * Layouts: an E-vector is [nelt][nx][nx][nx] with i fastest; the geometric
 * factors are [nelt][nx^3][6] in the order (rr, rs, rt, ss, st, tt) = g(1..6)
 * of Listing 1; D is row-major D[i*nx+l] = l_l'(xi_i) (the paper's dxm1, whose
 * transpose is dxtm1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REF_OK 0
#define REF_INVALID 1
#define REF_NOT_CONVERGED 4
#define REF_BREAKDOWN 5
#define REF_NOMEM 7

static inline int64_t at3(int i, int j, int k, int n) { return (int64_t)i + (int64_t)n * (j + (int64_t)n * k); }

/*
 * Geometric factors of a trilinear hexahedron (the paper is silent on how g is
 * formed; reading: the standard SEM metric, 6 symmetric factors times the
 * tensor GLL weight):
 *   x(r,s,t) = sum_q N_q(r,s,t) X_q,  N_q = (1 +/- r)(1 +/- s)(1 +/- t)/8,
 *   J = [x_r x_s x_t],  |J| = x_r . (x_s x x_t),
 *   grad r = (x_s x x_t)/|J|, grad s = (x_t x x_r)/|J|, grad t = (x_r x x_s)/|J|,
 *   G_ab = rho_i rho_j rho_k |J| (grad r_a . grad r_b).
 * Returns the number of nodes with |J| <= 0; *min_detj receives the minimum.
 */
int64_t ref_geom(int64_t nelt, int nx, const double* z, const double* rho, const double* corners,
                 double* G, double* min_detj)
{
    int64_t bad = 0;
    double mind = INFINITY;
    for (int64_t e = 0; e < nelt; e++) {
        const double* X = corners + e * 24;
        for (int k = 0; k < nx; k++)
            for (int j = 0; j < nx; j++)
                for (int i = 0; i < nx; i++) {
                    double r = z[i], s = z[j], t = z[k];
                    double xr[3] = {0, 0, 0}, xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
                    for (int q = 0; q < 8; q++) {
                        double sr = (q & 1) ? 1.0 : -1.0;
                        double ss = ((q >> 1) & 1) ? 1.0 : -1.0;
                        double st = ((q >> 2) & 1) ? 1.0 : -1.0;
                        double dr = sr * (1.0 + ss * s) * (1.0 + st * t) / 8.0;
                        double ds = ss * (1.0 + sr * r) * (1.0 + st * t) / 8.0;
                        double dt = st * (1.0 + sr * r) * (1.0 + ss * s) / 8.0;
                        for (int c = 0; c < 3; c++) {
                            xr[c] += dr * X[q * 3 + c];
                            xs[c] += ds * X[q * 3 + c];
                            xt[c] += dt * X[q * 3 + c];
                        }
                    }
                    double cst[3] = {xs[1] * xt[2] - xs[2] * xt[1], xs[2] * xt[0] - xs[0] * xt[2],
                                     xs[0] * xt[1] - xs[1] * xt[0]};
                    double ctr[3] = {xt[1] * xr[2] - xt[2] * xr[1], xt[2] * xr[0] - xt[0] * xr[2],
                                     xt[0] * xr[1] - xt[1] * xr[0]};
                    double crs[3] = {xr[1] * xs[2] - xr[2] * xs[1], xr[2] * xs[0] - xr[0] * xs[2],
                                     xr[0] * xs[1] - xr[1] * xs[0]};
                    double det = xr[0] * cst[0] + xr[1] * cst[1] + xr[2] * cst[2];
                    if (det < mind) mind = det;
                    if (!(det > 0.0)) bad++;
                    double gr[3], gs[3], gt[3];
                    for (int c = 0; c < 3; c++) {
                        gr[c] = cst[c] / det;
                        gs[c] = ctr[c] / det;
                        gt[c] = crs[c] / det;
                    }
                    double wq = rho[i] * rho[j] * rho[k] * det;
                    double* g = G + (e * (int64_t)nx * nx * nx + at3(i, j, k, nx)) * 6;
                    g[0] = wq * (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
                    g[1] = wq * (gr[0] * gs[0] + gr[1] * gs[1] + gr[2] * gs[2]);
                    g[2] = wq * (gr[0] * gt[0] + gr[1] * gt[1] + gr[2] * gt[2]);
                    g[3] = wq * (gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]);
                    g[4] = wq * (gs[0] * gt[0] + gs[1] * gt[1] + gs[2] * gt[2]);
                    g[5] = wq * (gt[0] * gt[0] + gt[1] * gt[1] + gt[2] * gt[2]);
                }
    }
    if (min_detj) *min_detj = mind;
    return bad;
}

/*
 * AX (Section II-B, Listing 1: ax -> ax_e -> local_grad3, the g product, and
 * local_grad3_t, which the text describes as the transposed products summed):
 *   ur(i,j,k) = sum_l D[i][l] u(l,j,k)   (mxm(dxm1,n,u,n,ur,n*n))
 *   us(i,j,k) = sum_l D[j][l] u(i,l,k)   (per k: mxm(u(:,:,k),n,dxtm1,n,us(:,:,k),n))
 *   ut(i,j,k) = sum_l D[k][l] u(i,j,l)   (mxm(u,n*n,dxtm1,n,ut,n))
 *   [wr ws wt] = [[g1 g2 g3][g2 g4 g5][g3 g5 g6]] [ur us ut]
 *   w(i,j,k) = sum_l D[l][i] wr(l,j,k) + sum_l D[l][j] ws(i,l,k) + sum_l D[l][k] wt(i,j,l)
 * Elements are independent (the outer loop of ax).
 */
int ref_ax(int64_t nelt, int nx, const double* D, const double* G, const double* u, double* w)
{
    int64_t n3 = (int64_t)nx * nx * nx;
    int status = REF_OK;
#pragma omp parallel
    {
    double* wr = (double*)malloc(sizeof(double) * n3 * 3);  /* scratch of one element (per thread) */
    if (!wr) {
#pragma omp atomic write
        status = REF_NOMEM;
    }
    double* ws = wr ? wr + n3 : NULL;
    double* wt = ws ? ws + n3 : NULL;
#pragma omp for schedule(static)
    for (int64_t e = 0; e < nelt; e++) {
        if (!wr) continue;
        const double* ue = u + e * n3;
        const double* ge = G + e * n3 * 6;
        double* we = w + e * n3;
        for (int k = 0; k < nx; k++)
            for (int j = 0; j < nx; j++)
                for (int i = 0; i < nx; i++) {
                    double ur = 0.0, us = 0.0, ut = 0.0;
                    for (int l = 0; l < nx; l++) {
                        ur += D[i * nx + l] * ue[at3(l, j, k, nx)];
                        us += D[j * nx + l] * ue[at3(i, l, k, nx)];
                        ut += D[k * nx + l] * ue[at3(i, j, l, nx)];
                    }
                    int64_t p = at3(i, j, k, nx);
                    const double* g = ge + 6 * p;
                    wr[p] = g[0] * ur + g[1] * us + g[2] * ut;
                    ws[p] = g[1] * ur + g[3] * us + g[4] * ut;
                    wt[p] = g[2] * ur + g[4] * us + g[5] * ut;
                }
        for (int k = 0; k < nx; k++)
            for (int j = 0; j < nx; j++)
                for (int i = 0; i < nx; i++) {
                    double s = 0.0;
                    for (int l = 0; l < nx; l++) s += D[l * nx + i] * wr[at3(l, j, k, nx)];
                    for (int l = 0; l < nx; l++) s += D[l * nx + j] * ws[at3(i, l, k, nx)];
                    for (int l = 0; l < nx; l++) s += D[l * nx + k] * wt[at3(i, j, l, nx)];
                    we[at3(i, j, k, nx)] = s;
                }
    }
    free(wr);
    }
    return status;
}

/* ---- gather-scatter (the exchange with neighbouring elements of Section II-B) ----
 * Reading: direct stiffness summation.  Every local node whose global id is
 * shared by m >= 2 local nodes belongs to one group; dssum replaces each member
 * by the group sum.  Groups are listed by ascending global id and members by
 * ascending local index; the sum is taken left to right in that member order.
 */
typedef struct {
    int64_t glo;
    int64_t idx;
} ref_pair;

static int cmp_pair(const void* a, const void* b)
{
    const ref_pair* x = (const ref_pair*)a;
    const ref_pair* y = (const ref_pair*)b;
    if (x->glo != y->glo) return x->glo < y->glo ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* offsets: capacity n+1, idx: capacity n.  Returns the number of groups, or -1 on
 * allocation failure. */
int64_t ref_gs_build(int64_t n, const int64_t* glo, int64_t* offsets, int64_t* idx)
{
    ref_pair* pr = (ref_pair*)malloc(sizeof(ref_pair) * (n > 0 ? n : 1));
    if (!pr) return -1;
    for (int64_t p = 0; p < n; p++) {
        pr[p].glo = glo[p];
        pr[p].idx = p;
    }
    qsort(pr, (size_t)n, sizeof(ref_pair), cmp_pair);
    int64_t ng = 0, m = 0;
    offsets[0] = 0;
    int64_t a = 0;
    while (a < n) {
        int64_t b = a + 1;
        while (b < n && pr[b].glo == pr[a].glo) b++;
        if (b - a >= 2) {
            for (int64_t q = a; q < b; q++) idx[m++] = pr[q].idx;
            offsets[++ng] = m;
        }
        a = b;
    }
    free(pr);
    return ng;
}

void ref_dssum(int64_t ngroups, const int64_t* offsets, const int64_t* idx, double* v)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < ngroups; g++) {
        double s = v[idx[offsets[g]]];
        for (int64_t o = offsets[g] + 1; o < offsets[g + 1]; o++) s += v[idx[o]];
        for (int64_t o = offsets[g]; o < offsets[g + 1]; o++) v[idx[o]] = s;
    }
}

/* c_p = 1 / (number of local copies of the global node of p): the weight that
 * turns a sum over local nodes of a consistent field into the global sum. */
void ref_inv_multiplicity(int64_t n, int64_t ngroups, const int64_t* offsets, const int64_t* idx, double* c)
{
    for (int64_t p = 0; p < n; p++) c[p] = 1.0;
    for (int64_t g = 0; g < ngroups; g++) {
        double m = (double)(offsets[g + 1] - offsets[g]);
        for (int64_t o = offsets[g]; o < offsets[g + 1]; o++) c[idx[o]] = 1.0 / m;
    }
}

/* Dirichlet mask (not in the paper; the box boundary is read as homogeneous
 * Dirichlet): v_p <- 0 where mask_p == 0. */
void ref_mask(int64_t n, const uint8_t* mask, double* v)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++)
        if (mask[p] == 0) v[p] = 0.0;
}

/*
 * Diagonal of the element operator of ref_ax, written out from the bilinear form
 * A_e[p,q] = sum_m sum_ab G_ab(m) d_a phi_p(m) d_b phi_q(m), with
 * d_r phi_ijk(l,m,n) = D[l][i] delta_mj delta_nk (and likewise for s, t):
 *   diag(i,j,k) = sum_l [ G_rr(l,j,k) D[l][i]^2 + G_ss(i,l,k) D[l][j]^2 + G_tt(i,j,l) D[l][k]^2 ]
 *               + 2 [ G_rs D[i][i] D[j][j] + G_rt D[i][i] D[k][k] + G_st D[j][j] D[k][k] ](i,j,k)
 */
void ref_diag_local(int64_t nelt, int nx, const double* D, const double* G, double* d)
{
    int64_t n3 = (int64_t)nx * nx * nx;
    for (int64_t e = 0; e < nelt; e++) {
        const double* ge = G + e * n3 * 6;
        for (int k = 0; k < nx; k++)
            for (int j = 0; j < nx; j++)
                for (int i = 0; i < nx; i++) {
                    double s = 0.0;
                    for (int l = 0; l < nx; l++) {
                        double a = D[l * nx + i], b = D[l * nx + j], c = D[l * nx + k];
                        s += ge[6 * at3(l, j, k, nx) + 0] * a * a;
                        s += ge[6 * at3(i, l, k, nx) + 3] * b * b;
                        s += ge[6 * at3(i, j, l, nx) + 5] * c * c;
                    }
                    const double* g = ge + 6 * at3(i, j, k, nx);
                    double di = D[i * nx + i], dj = D[j * nx + j], dk = D[k * nx + k];
                    s += 2.0 * (g[1] * di * dj + g[2] * di * dk + g[4] * dj * dk);
                    d[e * n3 + at3(i, j, k, nx)] = s;
                }
    }
}

/* Jacobi preconditioner (the basic preconditioner of Section II-B, read as the
 * inverse of the assembled diagonal): minv = 1/dssum(diag_local), 0 on masked
 * nodes. */
int ref_jacobi_minv(int64_t nelt, int nx, const double* D, const double* G, int64_t ngroups,
                    const int64_t* offsets, const int64_t* idx, const uint8_t* mask, double* minv)
{
    int64_t n = nelt * (int64_t)nx * nx * nx;
    ref_diag_local(nelt, nx, D, G, minv);
    ref_dssum(ngroups, offsets, idx, minv);
    for (int64_t p = 0; p < n; p++) minv[p] = mask[p] ? 1.0 / minv[p] : 0.0;
    return REF_OK;
}

static double wdot(int64_t n, const double* c, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t p = 0; p < n; p++) s += c[p] * a[p] * b[p];
    return s;
}

/*
 * Jacobi-preconditioned CG on the masked, assembled operator (Section II-B: CG
 * iterations of vector operations, AX, nearest-neighbour exchange and global
 * reductions).  Readings: b = mask.f; inner products weighted by
 * c = 1/multiplicity; stop when ||r||_c / ||b||_c <= tol.  tol <= 0 runs exactly
 * max_iter iterations.
 *   x=0, r=b, z=Minv r, p=z, rz=<r,z>
 *   repeat: w = mask(dssum(AX p)); alpha = rz/<p,w>; x += alpha p; r -= alpha w;
 *           stop test; z = Minv r; beta = <r,z>_new/rz; p = z + beta p
 */
int ref_pcg(int64_t nelt, int nx, const double* D, const double* G, int64_t ngroups, const int64_t* offsets,
            const int64_t* idx, const uint8_t* mask, const double* minv, const double* f, double* x, double tol,
            int max_iter, int* iters, double* relres, double* res_hist)
{
    int64_t n = nelt * (int64_t)nx * nx * nx;
    double* buf = (double*)malloc(sizeof(double) * (n > 0 ? n : 1) * 5);
    if (!buf) return REF_NOMEM;
    double *r = buf, *z = buf + n, *p = buf + 2 * n, *w = buf + 3 * n, *c = buf + 4 * n;
    ref_inv_multiplicity(n, ngroups, offsets, idx, c);
    for (int64_t q = 0; q < n; q++) {
        x[q] = 0.0;
        r[q] = mask[q] ? f[q] : 0.0;
        z[q] = minv[q] * r[q];
        p[q] = z[q];
    }
    double rz = wdot(n, c, r, z);
    double bnorm = sqrt(wdot(n, c, r, r));
    *iters = 0;
    *relres = 0.0;
    if (!(bnorm > 0.0)) {
        free(buf);
        return bnorm == 0.0 ? REF_OK : REF_BREAKDOWN;
    }
    int status = tol > 0.0 ? REF_NOT_CONVERGED : REF_OK;
    for (int it = 1; it <= max_iter; it++) {
        ref_ax(nelt, nx, D, G, p, w);
        ref_dssum(ngroups, offsets, idx, w);
        ref_mask(n, mask, w);
        double pw = wdot(n, c, p, w);
        if (!(pw > 0.0) || !isfinite(pw)) {
            *iters = it;
            status = REF_BREAKDOWN;
            break;
        }
        double alpha = rz / pw;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; q++) {
            x[q] += alpha * p[q];
            r[q] -= alpha * w[q];
        }
        double rr = wdot(n, c, r, r);
        *relres = sqrt(rr) / bnorm;
        if (res_hist) res_hist[it - 1] = *relres;
        *iters = it;
        if (!isfinite(*relres)) {
            status = REF_BREAKDOWN;
            break;
        }
        if (tol > 0.0 && *relres <= tol) {
            status = REF_OK;
            break;
        }
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; q++) z[q] = minv[q] * r[q];
        double rz_new = wdot(n, c, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; q++) p[q] = z[q] + beta * p[q];
    }
    free(buf);
    return status;
}
