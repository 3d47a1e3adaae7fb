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
#include "nek_pcg.cuh"

namespace nek {

namespace {

using pcg::stream_blocks;

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

// r = mask ? f - w : 0
__global__ void k_residual(int64_t n, const uint8_t* __restrict__ mask, const double* __restrict__ f,
                           double* __restrict__ r)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        r[p] = mask[p] ? f[p] - r[p] : 0.0;
}

__global__ void k_invert_masked(int64_t n, const uint8_t* __restrict__ mask, double* __restrict__ d)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        d[p] = mask[p] ? 1.0 / d[p] : 0.0;
}

}  // namespace

nek_status launch_diag_local(int64_t nelt, int nx, const double* D, const double* G, double* d, cudaStream_t s)
{
    k_diag_local<<<stream_blocks(nelt * (int64_t)nx * nx * nx), 256, 0, s>>>(nelt, nx, D, G, d);
    return check_launch();
}

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

nek_status nek_residual(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G, const float* Gff,
                        const uint8_t* mask, const double* f, const double* x, double* r, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!gs || nelt < 0) return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (gs->npts != n) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!D || !mask || !f || !x || !r || (!G && !Gff) || x == r || f == r) return NEK_ERR_INVALID_ARG;
    if ((Gff && !is_aligned(Gff, 16)) || (!Gff && !is_aligned(G, 16)) || !is_aligned(f, 8) || !is_aligned(x, 8) ||
        !is_aligned(r, 8))
        return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    nek_status st = Gff ? launch_ax_ff(nelt, nx, D, Gff, x, r, s) : launch_ax_fp64(nelt, nx, D, G, x, r, s);
    if (st == NEK_OK) st = launch_dssum(gs, r, s);
    if (st != NEK_OK) return st;
    k_residual<<<stream_blocks(n), 256, 0, s>>>(n, mask, f, r);
    return check_launch();
}

size_t nek_cg_workspace_bytes(int64_t nelt, int nx, int need_minv)
{
    if (nelt < 0 || nx < kMinNx || nx > kMaxNx) return 0;
    const size_t n = (size_t)nelt * nx * nx * nx;
    const size_t vec = pcg::align256(sizeof(double) * std::max<size_t>(n, 1));
    // r, p, w, [minv], point flags (1 byte each), element energies, reduction
    // partials, scalars
    return vec * (need_minv ? 4 : 3) + pcg::align256(std::max<size_t>(n, 1)) +
           pcg::align256(sizeof(double) * std::max<int64_t>(nelt, 1)) +
           pcg::align256(sizeof(double) * 2 * kMaxReduceBlocks) + pcg::align256(sizeof(pcg::Scalars));
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
    if (ax_impl != NEK_AX_FP64 && ax_impl != NEK_AX_FF && ax_impl != NEK_AX_OZ) return NEK_ERR_INVALID_ARG;
    if (ax_impl == NEK_AX_OZ && !ax_oz_supported(nx)) return NEK_ERR_UNSUPPORTED_NX;
    if (ax_impl != NEK_AX_FP64 && (!Gff || !is_aligned(Gff, 16))) return NEK_ERR_INVALID_ARG;
    if (ax_impl == NEK_AX_OZ && minv && !is_aligned(minv, 16)) return NEK_ERR_INVALID_ARG;
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
    const size_t vec = pcg::align256(sizeof(double) * n);
    char* base = static_cast<char*>(ws);
    pcg::Buffers<double> b;
    b.r = reinterpret_cast<double*>(base);
    b.p = reinterpret_cast<double*>(base + vec);
    b.w = reinterpret_cast<double*>(base + 2 * vec);
    size_t off = 3 * vec;
    double* mv = const_cast<double*>(minv);
    if (!minv) {
        mv = reinterpret_cast<double*>(base + off);
        off += vec;
    }
    uint8_t* flags = reinterpret_cast<uint8_t*>(base + off);
    off += pcg::align256(n);
    double* edot = reinterpret_cast<double*>(base + off);
    off += pcg::align256(sizeof(double) * nelt);
    b.parts = reinterpret_cast<double*>(base + off);
    off += pcg::align256(sizeof(double) * 2 * kMaxReduceBlocks);
    b.sc = reinterpret_cast<pcg::Scalars*>(base + off);

    pcg::Result res;
    int extra = 0;
    if (!minv) {
        st = nek_jacobi_minv(gs, nelt, nx, D, G, mask, mv, stream);
        extra = 3;
    }
    if (st == NEK_OK) {
        st = pcg::build_flags(gs, n, mask, flags, s);
        extra += gs->ngroups > 0 ? 2 : 1;
    }
    // The float-float operator also writes element energies, which replace the
    // solve's <p,w> pass.
    const bool energies = ax_impl != NEK_AX_FP64;
    // and the direction update, where compiled
    pcg::ElementEnergies ee{edot, nelt, ax_impl == NEK_AX_OZ ? ax_oz_supported(nx) : ax_ff_dir_supported(nx)};
    if (st == NEK_OK) {
        auto ax = [&](const double* p, double* w, double* ed, const DirUpdate* dir, cudaStream_t ss) {
            return ax_impl == NEK_AX_FF   ? launch_ax_ff(nelt, nx, D, Gff, p, w, ss, nullptr, nullptr, nullptr, ed, dir)
                   : ax_impl == NEK_AX_OZ ? launch_ax_oz(nelt, nx, D, Gff, p, w, ss, ed, dir)
                                          : launch_ax_fp64(nelt, nx, D, G, p, w, ss);
        };
        st = pcg::run<double>(gs, n, gs->d_c, mask, mv, f, x, b, tol_rel, max_iter, check_every, time_ax, ax, s,
                              &res, flags, energies ? &ee : nullptr);
        if (iters_out) *iters_out = res.iters;
        if (relres_out) *relres_out = res.relres;
        if (opts) {
            opts->ax_ms_total = res.ax_ms;
            opts->ax_launches = res.ax_timed;
            opts->kernel_launches = res.launches + extra;
        }
    }
    if (!workspace) {
        cudaFreeAsync(ws, s);
        nek_status st2 = check_cuda(cudaStreamSynchronize(s));
        if (st == NEK_OK) st = st2;
    }
    return st;
}

size_t nek_cg_host_staging_bytes(int64_t nelt, int nx)
{
    if (nelt < 0 || nx < kMinNx || nx > kMaxNx) return 0;
    return 2 * pcg::align256(sizeof(double) * std::max<size_t>((size_t)nelt * nx * nx * nx, 1));
}

nek_status nek_cg_solve_host(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                             const uint8_t* mask, const double* minv, const double* f_host, double* x_host,
                             double tol_rel, int max_iter, void* workspace, void* staging, int* iters_out,
                             double* relres_out, nek_cg_opts* opts, void* stream)
{
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!gs || nelt < 0 || max_iter < 0 || !(tol_rel >= 0.0)) return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (gs->npts != n) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!f_host || !x_host || (staging && !is_aligned(staging, 256))) return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* st_buf = staging;
    nek_status st = NEK_OK;
    if (!st_buf && (st = check_cuda(cudaMallocAsync(&st_buf, nek_cg_host_staging_bytes(nelt, nx), s))) != NEK_OK)
        return NEK_ERR_NOMEM;
    double* fd = static_cast<double*>(st_buf);
    double* xd = reinterpret_cast<double*>(static_cast<char*>(st_buf) + pcg::align256(sizeof(double) * n));
    const size_t bytes = sizeof(double) * (size_t)n;
    st = check_cuda(cudaMemcpyAsync(fd, f_host, bytes, cudaMemcpyHostToDevice, s));
    if (st == NEK_OK)
        st = nek_cg_solve_ex(gs, nelt, nx, D, G, mask, minv, fd, xd, tol_rel, max_iter, workspace, iters_out,
                             relres_out, opts, stream);
    if (st == NEK_OK || st == NEK_ERR_NOT_CONVERGED || st == NEK_ERR_BREAKDOWN) {
        nek_status st2 = check_cuda(cudaMemcpyAsync(x_host, xd, bytes, cudaMemcpyDeviceToHost, s));
        if (st2 != NEK_OK) st = st2;
    }
    if (!staging) cudaFreeAsync(st_buf, s);
    nek_status st3 = check_cuda(cudaStreamSynchronize(s));
    return st == NEK_OK ? st3 : st;
}

nek_status nek_cg_solve(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                        const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                        int max_iter, void* workspace, int* iters_out, double* relres_out, void* stream)
{
    return nek_cg_solve_ex(gs, nelt, nx, D, G, mask, minv, f, x, tol_rel, max_iter, workspace, iters_out,
                           relres_out, nullptr, stream);
}

}  // extern "C"
