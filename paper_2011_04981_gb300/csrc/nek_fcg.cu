// Flexible CG with the learned element preconditioner, falling back to Jacobi.
//
// Flexible CG (Notay, 2000) tolerates a preconditioner that is not a fixed SPD
// matrix by taking the Polak-Ribiere coefficient
//   beta = <r_new - r_old, z_new> / <r_old, z_old>
// instead of <r_new, z_new>/<r_old, z_old>.  Iteration (inner products weighted
// by 1/multiplicity, as in the Jacobi-PCG solve):
//   w = mask(dssum(AX p)); alpha = <r,z>/<p,w>; x += alpha p; r_old = r;
//   r -= alpha w; stop if ||r||/||b|| <= tol; z = M(r); beta as above;
//   p = z + beta p,
// with M(r) = mask(dssum(net(r) * rms(Jacobi r) / multiplicity)).  If the
// relative residual has not fallen by `stag_factor` within the last `stag_window`
// iterations, M becomes Jacobi (z = Minv r) for the rest of the solve and the
// search direction restarts from z.
#include <vector>

#include "nek_internal.h"
#include "nek_pcg.cuh"

namespace nek {

nek_status launch_net_apply_tc(int64_t nelt, const float* theta, const float* xin, const float* scale,
                               const double* c, double* z, cudaStream_t s);
nek_status launch_net_apply(int64_t nelt, const float* theta, const float* xin, const float* scale, const double* c,
                            double* z, cudaStream_t s);
nek_status launch_net_prep(int64_t nelt, const double* r, const double* minv, float* xin, float* scale,
                           cudaStream_t s);

namespace {

constexpr int NT = kReduceThreads;

struct FScal {
    double rz, pw, alpha, beta, rr, bnorm, relres, num;
};

// w <- mask.w, partial <p,w>
__global__ void __launch_bounds__(NT) kf_pw(int64_t n, const double* __restrict__ c, const uint8_t* __restrict__ mask,
                                            const double* __restrict__ p, double* __restrict__ w,
                                            double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
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

__global__ void __launch_bounds__(NT) kf_alpha(const double* __restrict__ parts, int nb, FScal* sc)
{
    __shared__ double sh[NT / 32];
    const double pw = sum_partials<NT>(parts, nb, sh);
    if (threadIdx.x == 0) {
        sc->pw = pw;
        sc->alpha = sc->rz / pw;
    }
}

// x += alpha p; r_old = r; r -= alpha w; partial <r,r>
__global__ void __launch_bounds__(NT) kf_update(int64_t n, const double* __restrict__ c,
                                                const double* __restrict__ p, const double* __restrict__ w,
                                                double* __restrict__ x, double* __restrict__ r,
                                                double* __restrict__ r_old, double* __restrict__ parts,
                                                const FScal* __restrict__ sc)
{
    __shared__ double sh[NT / 32];
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        x[q] = fma(alpha, p[q], x[q]);
        const double ro = r[q];
        const double rq = fma(-alpha, w[q], ro);
        r_old[q] = ro;
        r[q] = rq;
        acc += c[q] * rq * rq;
    }
    const double t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) kf_rr(const double* __restrict__ parts, int nb, int first, FScal* sc)
{
    __shared__ double sh[NT / 32];
    const double rr = sum_partials<NT>(parts, nb, sh);
    if (threadIdx.x == 0) {
        sc->rr = rr;
        if (first) sc->bnorm = sqrt(rr);
        sc->relres = sc->bnorm > 0.0 ? sqrt(rr) / sc->bnorm : 0.0;
    }
}

// z = minv r (Jacobi)
__global__ void kf_jacobi(int64_t n, const double* __restrict__ minv, const double* __restrict__ r,
                          double* __restrict__ z)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        z[q] = minv[q] * r[q];
}

// z <- mask.z ; partials <r,z>, <r_old,z>
__global__ void __launch_bounds__(NT) kf_zdots(int64_t n, const double* __restrict__ c,
                                               const uint8_t* __restrict__ mask, const double* __restrict__ r,
                                               const double* __restrict__ r_old, double* __restrict__ z,
                                               double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
    double a = 0.0, b = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        double zq = z[q];
        if (!mask[q]) {
            zq = 0.0;
            z[q] = 0.0;
        }
        a += c[q] * r[q] * zq;
        b += c[q] * r_old[q] * zq;
    }
    double t = block_sum<NT>(a, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
    t = block_sum<NT>(b, sh);
    if (threadIdx.x == 0) parts[gridDim.x + blockIdx.x] = t;
}

// beta = (<r,z> - <r_old,z>) / rz_old (0 on restart); rz = <r,z>
__global__ void __launch_bounds__(NT) kf_beta(const double* __restrict__ parts, int nb, int restart, FScal* sc)
{
    __shared__ double sh[NT / 32];
    const double rz = sum_partials<NT>(parts, nb, sh);
    const double roz = sum_partials<NT>(parts + nb, nb, sh);
    if (threadIdx.x == 0) {
        sc->num = rz - roz;
        sc->beta = restart ? 0.0 : (rz - roz) / sc->rz;
        sc->rz = rz;
    }
}

__global__ void kf_p(int64_t n, const double* __restrict__ z, double* __restrict__ p, const FScal* __restrict__ sc)
{
    const double beta = sc->beta;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        p[q] = fma(beta, p[q], z[q]);
}

// x = 0, r = mask.f, partial <r,r>
__global__ void __launch_bounds__(NT) kf_init(int64_t n, const double* __restrict__ c,
                                              const uint8_t* __restrict__ mask, const double* __restrict__ f,
                                              double* __restrict__ x, double* __restrict__ r,
                                              double* __restrict__ r_old, double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        const double rq = mask[q] ? f[q] : 0.0;
        x[q] = 0.0;
        r[q] = rq;
        r_old[q] = 0.0;
        acc += c[q] * rq * rq;
    }
    const double t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct FLayout {
    double *r, *r_old, *z, *p, *w, *minv, *parts;
    float *xin, *scale;
    FScal* sc;
    size_t bytes;
};

FLayout f_layout(char* base, int64_t nelt, int nx, bool need_minv)
{
    FLayout L{};
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    size_t off = 0;
    auto take = [&](size_t b) {
        char* q = base ? base + off : nullptr;
        off += al256(b);
        return q;
    };
    const size_t v = sizeof(double) * std::max<int64_t>(n, 1);
    L.r = reinterpret_cast<double*>(take(v));
    L.r_old = reinterpret_cast<double*>(take(v));
    L.z = reinterpret_cast<double*>(take(v));
    L.p = reinterpret_cast<double*>(take(v));
    L.w = reinterpret_cast<double*>(take(v));
    L.minv = need_minv ? reinterpret_cast<double*>(take(v)) : nullptr;
    L.xin = reinterpret_cast<float*>(take(sizeof(float) * 2 * std::max<int64_t>(n, 1)));
    L.scale = reinterpret_cast<float*>(take(sizeof(float) * std::max<int64_t>(nelt, 1)));
    L.parts = reinterpret_cast<double*>(take(sizeof(double) * 2 * kMaxReduceBlocks));
    L.sc = reinterpret_cast<FScal*>(take(sizeof(FScal)));
    L.bytes = off;
    return L;
}

}  // namespace

}  // namespace nek

using namespace nek;

extern "C" {

size_t nek_fcg_workspace_bytes(int64_t nelt, int nx, int need_minv)
{
    if (nelt < 0 || nx < kMinNx || nx > kMaxNx) return 0;
    return f_layout(nullptr, nelt, nx, need_minv != 0).bytes;
}

nek_status nek_fcg_solve(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G, const float* Gff,
                         const uint8_t* mask, const double* minv, const float* theta, const double* f, double* x,
                         double tol_rel, int max_iter, int stag_window, double stag_factor, void* workspace,
                         nek_fcg_info* info, void* stream)
{
    if (info) *info = nek_fcg_info{};
    if (nx != 8) return NEK_ERR_UNSUPPORTED_NX;  // the network is built for 8^3 element blocks
    if (!gs || nelt < 0 || max_iter < 0 || !(tol_rel > 0.0) || stag_window < 1 || !(stag_factor > 0.0) ||
        !(stag_factor < 1.0))
        return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (gs->npts != n) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!D || !G || !mask || !f || !x || !is_aligned(G, 16) || !is_aligned(x, 8) || (Gff && !is_aligned(Gff, 16)) ||
        (minv && !is_aligned(minv, 8)) || (workspace && !is_aligned(workspace, 256)))
        return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = nek_fcg_workspace_bytes(nelt, nx, minv == nullptr);
    void* ws = workspace;
    if (!ws && check_cuda(cudaMallocAsync(&ws, bytes, s)) != NEK_OK) return NEK_ERR_NOMEM;
    FLayout L = f_layout(static_cast<char*>(ws), nelt, nx, minv == nullptr);
    const double* mv = minv;
    const int nb = reduce_blocks(n);
    const int sb = pcg::stream_blocks(n);
    nek_status st = NEK_OK;
    FScal h{};
    std::vector<double> hist;
    bool net = theta != nullptr;
    int it = 0, fell_back = 0, net_apps = 0, launches = 0;
    // one event pair per network application, read once at the end (no host
    // synchronisation inside the loop for the timing)
    std::vector<cudaEvent_t> nev;
    double net_ms = 0.0;

    auto precondition = [&](int restart) -> nek_status {
        if (net) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            const bool timed = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
            if (timed) {
                nev.push_back(e0);
                nev.push_back(e1);
            } else {
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
            }
            if (timed) cudaEventRecord(e0, s);
            nek_status sp = launch_net_prep(nelt, L.r, mv, L.xin, L.scale, s);
            if (sp == NEK_OK) sp = launch_net_apply_tc(nelt, theta, L.xin, L.scale, gs->d_c, L.z, s);
            if (sp == NEK_OK) sp = pcg::dssum<double>(gs, L.z, s);
            if (timed) cudaEventRecord(e1, s);
            if (sp != NEK_OK) return sp;
            net_apps++;
            launches += 3;
        } else {
            kf_jacobi<<<sb, 256, 0, s>>>(n, mv, L.r, L.z);
            launches += 1;
        }
        kf_zdots<<<nb, NT, 0, s>>>(n, gs->d_c, mask, L.r, L.r_old, L.z, L.parts);
        kf_beta<<<1, NT, 0, s>>>(L.parts, nb, restart, L.sc);
        launches += 2;
        return check_launch();
    };

    if (!minv) {
        if ((st = nek_jacobi_minv(gs, nelt, nx, D, G, mask, L.minv, stream)) != NEK_OK) goto done;
        mv = L.minv;
        launches += 3;
    }
    kf_init<<<nb, NT, 0, s>>>(n, gs->d_c, mask, f, x, L.r, L.r_old, L.parts);
    kf_rr<<<1, NT, 0, s>>>(L.parts, nb, 1, L.sc);
    launches += 2;
    if ((st = check_launch()) != NEK_OK) goto done;
    if ((st = check_cuda(cudaMemcpyAsync(&h, L.sc, sizeof(h), cudaMemcpyDeviceToHost, s))) != NEK_OK) goto done;
    if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
    if (!std::isfinite(h.bnorm)) {
        st = NEK_ERR_BREAKDOWN;
        goto done;
    }
    if (h.bnorm == 0.0) goto done;
    hist.push_back(1.0);
    if ((st = precondition(1)) != NEK_OK) goto done;
    cudaMemcpyAsync(L.p, L.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    for (it = 1; it <= max_iter; it++) {
        st = Gff ? launch_ax_ff(nelt, nx, D, Gff, L.p, L.w, s) : launch_ax_fp64(nelt, nx, D, G, L.p, L.w, s);
        if (st != NEK_OK) goto done;
        if ((st = pcg::dssum<double>(gs, L.w, s)) != NEK_OK) goto done;
        kf_pw<<<nb, NT, 0, s>>>(n, gs->d_c, mask, L.p, L.w, L.parts);
        kf_alpha<<<1, NT, 0, s>>>(L.parts, nb, L.sc);
        kf_update<<<nb, NT, 0, s>>>(n, gs->d_c, L.p, L.w, x, L.r, L.r_old, L.parts, L.sc);
        kf_rr<<<1, NT, 0, s>>>(L.parts, nb, 0, L.sc);
        launches += 6;
        if ((st = check_launch()) != NEK_OK) goto done;
        if ((st = check_cuda(cudaMemcpyAsync(&h, L.sc, sizeof(h), cudaMemcpyDeviceToHost, s))) != NEK_OK) goto done;
        if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
        if (!(h.pw > 0.0) || !std::isfinite(h.relres)) {  // A is SPD: p.Ap <= 0 means p = 0 or bad data
            st = NEK_ERR_BREAKDOWN;
            goto done;
        }
        hist.push_back(h.relres);
        if (h.relres <= tol_rel) break;
        int restart = 0;
        if (net && it >= stag_window && h.relres > stag_factor * hist[it - stag_window]) {
            net = false;
            fell_back = it;
            restart = 1;
        }
        if ((st = precondition(restart)) != NEK_OK) goto done;
        kf_p<<<sb, 256, 0, s>>>(n, L.z, L.p, L.sc);
        launches += 1;
    }
    if (it > max_iter) {
        it = max_iter;
        st = NEK_ERR_NOT_CONVERGED;
    }
done:
    if (!nev.empty() && cudaStreamSynchronize(s) == cudaSuccess) {
        for (size_t q = 0; q + 1 < nev.size(); q += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, nev[q], nev[q + 1]) == cudaSuccess) net_ms += ms;
        }
    }
    for (auto& e : nev) cudaEventDestroy(e);
    if (info) {
        info->iters = it;
        info->relres = h.relres;
        info->fell_back_at = fell_back;
        info->net_applications = net_apps;
        info->net_ms = net_ms;
        info->kernel_launches = launches;
    }
    if (!workspace) {
        cudaFreeAsync(ws, s);
        nek_status st2 = check_cuda(cudaStreamSynchronize(s));
        if (st == NEK_OK) st = st2;
    }
    return st;
}

}  // extern "C"
