// Jacobi preconditioner and the preconditioned CG solve on the device.
//
// The CG iteration of Section II-B (vector operations, AX, nearest-neighbour
// exchange, global reductions) runs entirely on one stream: the scalars
// alpha, beta, <r,z>, ||r|| live in device memory and every kernel reads them
// there, so the host only enqueues work and reads the residual back every
// check_every iterations.  Reductions are two-stage and deterministic (fixed
// grid per length, fixed shuffle pattern, partials summed in order by one
// block).  Once the residual test passes, or a breakdown is seen, the device
// sets a flag and all later update kernels of the call leave x untouched, so the
// result and the iteration count do not depend on check_every.
#include <algorithm>
#include <cmath>
#include <vector>

#include "nek_internal.h"
#include "nek_reduce.cuh"

namespace nek {

namespace {

struct CgScalars {
    double rz;      // <r, z>_c of the current iterate
    double pw;      // <p, w>_c
    double alpha;
    double beta;
    double rr;      // <r, r>_c
    double bnorm;   // ||b||_c
    double relres;  // ||r||_c / ||b||_c
    double tol;
    int done;       // residual test passed
    int status;     // NEK_OK or NEK_ERR_BREAKDOWN
    int iters;      // iterations completed when done/status was set
    int it;         // iterations executed so far
};

constexpr int NT = kReduceThreads;

__device__ __forceinline__ bool halted(const CgScalars* sc) { return sc->done || sc->status != NEK_OK; }

// ---------------------------------------------------------------- Jacobi
__global__ void k_diag_local(int64_t nelt, int nx, const double* __restrict__ D, const double* __restrict__ G,
                             double* __restrict__ d)
{
    const int64_t n3 = (int64_t)nx * nx * nx;
    for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < nelt * n3;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = gid / n3;
        const int p = static_cast<int>(gid - e * n3);
        const int i = p % nx, j = (p / nx) % nx, k = p / (nx * nx);
        const double* Ge = G + e * n3 * 6;
        double s = 0.0;
        for (int l = 0; l < nx; l++) {
            const double a = D[l * nx + i], b = D[l * nx + j], c = D[l * nx + k];
            s += Ge[6 * (l + nx * (j + nx * k)) + 0] * a * a;
            s += Ge[6 * (i + nx * (l + nx * k)) + 3] * b * b;
            s += Ge[6 * (i + nx * (j + nx * l)) + 5] * c * c;
        }
        const double* g = Ge + 6 * p;
        const double di = D[i * nx + i], dj = D[j * nx + j], dk = D[k * nx + k];
        s += 2.0 * (g[1] * di * dj + g[2] * di * dk + g[4] * dj * dk);
        d[gid] = s;
    }
}

__global__ void k_invert_masked(int64_t n, const uint8_t* __restrict__ mask, double* __restrict__ d)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        d[p] = mask[p] ? 1.0 / d[p] : 0.0;
}

// ---------------------------------------------------------------- CG kernels
// x = 0, r = mask.f, z = minv r, p = z; partials of <r,z>_c and <r,r>_c.
__global__ void __launch_bounds__(NT) k_cg_init(int64_t n, const double* __restrict__ c,
                                                 const uint8_t* __restrict__ mask, const double* __restrict__ minv,
                                                 const double* __restrict__ f, double* __restrict__ x,
                                                 double* __restrict__ r, double* __restrict__ z,
                                                 double* __restrict__ p, double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
    double arz = 0.0, arr = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        const double rq = mask[q] ? f[q] : 0.0;
        const double zq = minv[q] * rq;
        x[q] = 0.0;
        r[q] = rq;
        z[q] = zq;
        p[q] = zq;
        arz += c[q] * rq * zq;
        arr += c[q] * rq * rq;
    }
    double t = block_sum<NT>(arz, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
    t = block_sum<NT>(arr, sh);
    if (threadIdx.x == 0) parts[gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_cg_init_finish(const double* __restrict__ parts, int nb, double tol,
                                                        CgScalars* sc)
{
    __shared__ double sh[NT / 32];
    const double rz = sum_partials<NT>(parts, nb, sh);
    const double rr = sum_partials<NT>(parts + nb, nb, sh);
    if (threadIdx.x == 0) {
        sc->rz = rz;
        sc->rr = rr;
        sc->bnorm = sqrt(rr);
        sc->tol = tol;
        sc->it = 0;
        sc->iters = 0;
        sc->alpha = sc->beta = sc->pw = 0.0;
        sc->status = NEK_OK;
        sc->done = 0;
        sc->relres = 0.0;
        if (!(rr >= 0.0) || !isfinite(rr) || !isfinite(rz)) {
            sc->status = NEK_ERR_BREAKDOWN;
        } else if (rr == 0.0) {
            sc->done = 1;  // b = 0: x = 0 is the solution
        } else {
            sc->relres = 1.0;
        }
    }
}

// w <- mask.w ; partials of <p,w>_c
__global__ void __launch_bounds__(NT) k_cg_pw(int64_t n, const double* __restrict__ c,
                                               const uint8_t* __restrict__ mask, const double* __restrict__ p,
                                               double* __restrict__ w, double* __restrict__ parts,
                                               const CgScalars* __restrict__ sc)
{
    __shared__ double sh[NT / 32];
    if (halted(sc)) return;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        double wq = w[q];
        if (!mask[q]) {
            wq = 0.0;
            w[q] = 0.0;
        }
        acc += c[q] * p[q] * wq;
    }
    const double t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_cg_alpha(const double* __restrict__ parts, int nb, CgScalars* sc)
{
    __shared__ double sh[NT / 32];
    if (halted(sc)) return;
    const double pw = sum_partials<NT>(parts, nb, sh);
    if (threadIdx.x == 0) {
        sc->it += 1;
        sc->pw = pw;
        if (!(pw > 0.0) || !isfinite(pw)) {
            sc->status = NEK_ERR_BREAKDOWN;
            sc->iters = sc->it;
        } else {
            sc->alpha = sc->rz / pw;
        }
    }
}

// x += alpha p; r -= alpha w; z = minv r; partials of <r,r>_c and <r,z>_c
__global__ void __launch_bounds__(NT) k_cg_update(int64_t n, const double* __restrict__ c,
                                                   const double* __restrict__ minv, const double* __restrict__ p,
                                                   const double* __restrict__ w, double* __restrict__ x,
                                                   double* __restrict__ r, double* __restrict__ z,
                                                   double* __restrict__ parts, const CgScalars* __restrict__ sc)
{
    __shared__ double sh[NT / 32];
    if (halted(sc)) return;
    const double alpha = sc->alpha;
    double arr = 0.0, arz = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        x[q] = fma(alpha, p[q], x[q]);
        const double rq = fma(-alpha, w[q], r[q]);
        const double zq = minv[q] * rq;
        r[q] = rq;
        z[q] = zq;
        arr += c[q] * rq * rq;
        arz += c[q] * rq * zq;
    }
    double t = block_sum<NT>(arr, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
    t = block_sum<NT>(arz, sh);
    if (threadIdx.x == 0) parts[gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_cg_beta(const double* __restrict__ parts, int nb, CgScalars* sc)
{
    __shared__ double sh[NT / 32];
    if (halted(sc)) return;
    const double rr = sum_partials<NT>(parts, nb, sh);
    const double rz = sum_partials<NT>(parts + nb, nb, sh);
    if (threadIdx.x == 0) {
        sc->rr = rr;
        sc->relres = sqrt(rr) / sc->bnorm;
        if (!isfinite(sc->relres) || !isfinite(rz)) {
            sc->status = NEK_ERR_BREAKDOWN;
            sc->iters = sc->it;
        } else if (sc->tol > 0.0 && sc->relres <= sc->tol) {
            sc->done = 1;
            sc->iters = sc->it;
        } else {
            sc->beta = rz / sc->rz;
            sc->rz = rz;
        }
    }
}

__global__ void k_cg_p(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                       const CgScalars* __restrict__ sc)
{
    if (halted(sc)) return;
    const double beta = sc->beta;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        p[q] = fma(beta, p[q], z[q]);
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int stream_blocks(int64_t n)
{
    int64_t nb = (n + 255) / 256;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nb, 152 * 16)));
}

}  // namespace

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_jacobi_minv(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                           const uint8_t* mask, double* minv, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!gs || nelt < 0) return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (gs->npts != n) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!D || !G || !mask || !minv || !is_aligned(G, 16) || !is_aligned(minv, 8)) return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_diag_local<<<stream_blocks(n), 256, 0, s>>>(nelt, nx, D, G, minv);
    nek_status st = check_launch();
    if (st != NEK_OK) return st;
    if ((st = launch_dssum(gs, minv, s)) != NEK_OK) return st;
    k_invert_masked<<<stream_blocks(n), 256, 0, s>>>(n, mask, minv);
    return check_launch();
}

size_t nek_cg_workspace_bytes(int64_t nelt, int nx, int need_minv)
{
    if (nelt < 0 || nx < kMinNx || nx > kMaxNx) return 0;
    const size_t n = (size_t)nelt * nx * nx * nx;
    const size_t vec = align256(sizeof(double) * std::max<size_t>(n, 1));
    return vec * (need_minv ? 5 : 4) + align256(sizeof(double) * 2 * kMaxReduceBlocks) + align256(sizeof(CgScalars));
}

nek_status nek_cg_solve_ex(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                           const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                           int max_iter, void* workspace, int* iters_out, double* relres_out, nek_cg_opts* opts,
                           void* stream)
{
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!gs || nelt < 0 || max_iter < 0 || !(tol_rel >= 0.0)) return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (gs->npts != n) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!D || !G || !mask || !f || !x) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(G, 16) || !is_aligned(f, 8) || !is_aligned(x, 16) || (minv && !is_aligned(minv, 8)))
        return NEK_ERR_INVALID_ARG;
    if (workspace && !is_aligned(workspace, 256)) return NEK_ERR_INVALID_ARG;
    const int check_every = (opts && opts->check_every > 0) ? opts->check_every : 1;
    const bool time_ax = opts && opts->time_ax;
    const int ax_impl = opts ? opts->ax_impl : NEK_AX_FP64;
    const float* Gff = opts ? opts->Gff : nullptr;
    if (ax_impl != NEK_AX_FP64 && ax_impl != NEK_AX_FF) return NEK_ERR_INVALID_ARG;
    if (ax_impl == NEK_AX_FF && (!Gff || !is_aligned(Gff, 16))) return NEK_ERR_INVALID_ARG;
    if (opts) {
        opts->ax_ms_total = 0.0;
        opts->ax_launches = 0;
        opts->kernel_launches = 0;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = nek_cg_workspace_bytes(nelt, nx, minv == nullptr);
    void* ws = workspace;
    nek_status st = NEK_OK;
    if (!ws) {
        st = check_cuda(cudaMallocAsync(&ws, bytes, s));
        if (st != NEK_OK) return NEK_ERR_NOMEM;
    }
    const size_t vec = align256(sizeof(double) * n);
    char* base = static_cast<char*>(ws);
    double* r = reinterpret_cast<double*>(base);
    double* z = reinterpret_cast<double*>(base + vec);
    double* p = reinterpret_cast<double*>(base + 2 * vec);
    double* w = reinterpret_cast<double*>(base + 3 * vec);
    size_t off = 4 * vec;
    double* mv = const_cast<double*>(minv);
    if (!minv) {
        mv = reinterpret_cast<double*>(base + off);
        off += vec;
    }
    double* parts = reinterpret_cast<double*>(base + off);
    off += align256(sizeof(double) * 2 * kMaxReduceBlocks);
    CgScalars* sc = reinterpret_cast<CgScalars*>(base + off);

    const int nb = reduce_blocks(n);
    const int sb = stream_blocks(n);
    int launches = 0;
    std::vector<cudaEvent_t> ev;
    CgScalars h{};
    int it = 0;

    if (!minv) {
        if ((st = nek_jacobi_minv(gs, nelt, nx, D, G, mask, mv, stream)) != NEK_OK) goto done;
        launches += 3;
    }
    k_cg_init<<<nb, NT, 0, s>>>(n, gs->d_c, mask, mv, f, x, r, z, p, parts);
    k_cg_init_finish<<<1, NT, 0, s>>>(parts, nb, tol_rel, sc);
    launches += 2;
    if ((st = check_launch()) != NEK_OK) goto done;
    if (time_ax) {
        const int nt = std::min(max_iter, 100000);
        ev.resize(2 * (size_t)nt);
        for (auto& e : ev)
            if ((st = check_cuda(cudaEventCreate(&e))) != NEK_OK) goto done;
    }
    for (it = 1; it <= max_iter; it++) {
        const bool timed = time_ax && (size_t)(2 * it) <= ev.size();
        if (timed) cudaEventRecord(ev[2 * (it - 1)], s);
        st = ax_impl == NEK_AX_FF ? launch_ax_ff(nelt, nx, D, Gff, p, w, s) : launch_ax_fp64(nelt, nx, D, G, p, w, s);
        if (st != NEK_OK) goto done;
        if (timed) cudaEventRecord(ev[2 * (it - 1) + 1], s);
        if ((st = launch_dssum(gs, w, s)) != NEK_OK) goto done;
        k_cg_pw<<<nb, NT, 0, s>>>(n, gs->d_c, mask, p, w, parts, sc);
        k_cg_alpha<<<1, NT, 0, s>>>(parts, nb, sc);
        k_cg_update<<<nb, NT, 0, s>>>(n, gs->d_c, mv, p, w, x, r, z, parts, sc);
        k_cg_beta<<<1, NT, 0, s>>>(parts, nb, sc);
        launches += 6;
        if ((st = check_launch()) != NEK_OK) goto done;
        if (tol_rel > 0.0 && (it % check_every == 0 || it == max_iter)) {
            if ((st = check_cuda(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s))) != NEK_OK) goto done;
            if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
            if (h.done || h.status != NEK_OK) break;
        }
        if (it < max_iter) {
            k_cg_p<<<sb, 256, 0, s>>>(n, z, p, sc);
            launches += 1;
        }
    }
    if ((st = check_cuda(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s))) != NEK_OK) goto done;
    if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
    if (time_ax && opts) {
        const int nt = std::min<int>(std::min(max_iter, h.it), static_cast<int>(ev.size() / 2));
        double tot = 0.0;
        for (int q = 0; q < nt; q++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]) == cudaSuccess) tot += ms;
        }
        opts->ax_ms_total = tot;
        opts->ax_launches = nt;
    }
    if (iters_out) *iters_out = (h.done || h.status != NEK_OK) ? h.iters : h.it;
    if (relres_out) *relres_out = h.relres;
    if (h.status != NEK_OK)
        st = static_cast<nek_status>(h.status);
    else if (tol_rel > 0.0 && !h.done)
        st = NEK_ERR_NOT_CONVERGED;
done:
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (opts) opts->kernel_launches = launches;
    if (!workspace) {
        cudaFreeAsync(ws, s);
        if (st == NEK_OK) st = check_cuda(cudaStreamSynchronize(s));
    }
    return st;
}

nek_status nek_cg_solve(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                        const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                        int max_iter, void* workspace, int* iters_out, double* relres_out, void* stream)
{
    return nek_cg_solve_ex(gs, nelt, nx, D, G, mask, minv, f, x, tol_rel, max_iter, workspace, iters_out,
                           relres_out, nullptr, stream);
}

}  // extern "C"
