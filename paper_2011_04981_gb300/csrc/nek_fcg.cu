// Flexible CG with the learned element preconditioner, falling back to Jacobi.
//
// Truncated flexible CG, FCG(m) (Notay, "Flexible conjugate gradients", SIAM J.
// Sci. Comput. 22, 2000), tolerates a preconditioner that is not a fixed SPD
// matrix -- here a nonlinear network -- by making every new direction
// A-orthogonal to the last m directions explicitly instead of relying on the
// short recurrence.  Iteration k (inner products weighted by 1/multiplicity, as
// in the Jacobi-PCG solve):
//   z = M(r);  p_k = z - sum_{i = k-m}^{k-1} (<z, A p_i> / <p_i, A p_i>) p_i;
//   w = mask(dssum(AX p_k));  alpha = <p_k, r> / <p_k, w>;  x += alpha p_k;
//   r -= alpha w;  stop if ||r||/||b|| <= tol,
// with M(r) = mask(dssum(net(r) * rms(Jacobi r) / multiplicity)).  m = 1 is
// flexible CG with the Polak-Ribiere-type coefficient; for a fixed SPD M every m
// gives the PCG iterates in exact arithmetic.  If the relative residual has not
// fallen by `stag_factor` within the last `stag_window` iterations, M becomes
// Jacobi (z = Minv r) for the rest of the solve and the direction window is
// emptied (a restart).
#include <vector>

#include "nek_internal.h"
#include "nek_pcg.cuh"

namespace nek {

nek_status launch_net_apply_tc5(int64_t nelt, const float* theta, const float* xin, const float* scale,
                                const double* c, double* z, cudaStream_t s);
nek_status net_tc5_take_timeout(bool* timed_out);
nek_status launch_net_apply(int64_t nelt, const float* theta, const float* xin, const float* scale, const double* c,
                            double* z, cudaStream_t s);
nek_status launch_net_prep(int64_t nelt, const double* r, const double* minv, float* xin, float* scale,
                           cudaStream_t s);

namespace {

constexpr int NT = kReduceThreads;
constexpr int kMaxTrunc = 16;

struct FScal {
    double alpha, pw, pr, rr, bnorm, relres;
    double beta[kMaxTrunc];      // coefficients of the window's directions
    double pwv[kMaxTrunc + 1];   // <p_i, A p_i> per ring slot
};

// Ring slots of the directions the new one is orthogonalised against.
struct Window {
    int n;
    int slot[kMaxTrunc];
};

// x = 0, r = mask.f, partial <r,r>
__global__ void __launch_bounds__(NT) kf_init(int64_t n, const double* __restrict__ c,
                                              const uint8_t* __restrict__ mask, const double* __restrict__ f,
                                              double* __restrict__ x, double* __restrict__ r,
                                              double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        const double rq = mask[q] ? f[q] : 0.0;
        x[q] = 0.0;
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

// z <- mask.z; partials of <z, W_i> for the window's M slots (parts[i * nb + block]).
// M is a template parameter so that the M loads of a point are independent
// registers and all in flight together.
template <int M>
__global__ void __launch_bounds__(NT) kf_zdots(int64_t n, const double* __restrict__ c,
                                               const uint8_t* __restrict__ mask, double* __restrict__ z,
                                               const double* __restrict__ Wbase, int64_t stride, Window win,
                                               double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
    const double* W[M > 0 ? M : 1];
#pragma unroll
    for (int i = 0; i < M; i++) W[i] = Wbase + win.slot[i] * stride;
    double acc[M > 0 ? M : 1];
#pragma unroll
    for (int i = 0; i < M; i++) acc[i] = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        double zq = z[q];
        const double cq = c[q];
        double wv[M > 0 ? M : 1];
#pragma unroll
        for (int i = 0; i < M; i++) wv[i] = W[i][q];
        if (!mask[q]) {
            zq = 0.0;
            z[q] = 0.0;
        }
        const double cz = cq * zq;
#pragma unroll
        for (int i = 0; i < M; i++) acc[i] += cz * wv[i];
    }
#pragma unroll
    for (int i = 0; i < M; i++) {
        const double t = block_sum<NT>(acc[i], sh);
        if (threadIdx.x == 0) parts[i * gridDim.x + blockIdx.x] = t;
    }
}

// beta_i = <z, W_i> / <p_i, W_i>
__global__ void __launch_bounds__(NT) kf_betas(const double* __restrict__ parts, int nb, Window win, FScal* sc)
{
    __shared__ double sh[NT / 32];
    for (int i = 0; i < win.n; i++) {
        const double d = sum_partials<NT>(parts + i * nb, nb, sh);
        if (threadIdx.x == 0) sc->beta[i] = d / sc->pwv[win.slot[i]];
    }
}

// P_cur = z - sum_i beta_i P_i (the window's M directions)
template <int M>
__global__ void kf_p(int64_t n, const double* __restrict__ z, double* __restrict__ Pbase, int64_t stride, int cur,
                     Window win, const FScal* __restrict__ sc)
{
    double beta[M > 0 ? M : 1];
    const double* P[M > 0 ? M : 1];
#pragma unroll
    for (int i = 0; i < M; i++) {
        beta[i] = sc->beta[i];
        P[i] = Pbase + win.slot[i] * stride;
    }
    double* pc = Pbase + cur * stride;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        double pv[M > 0 ? M : 1];
#pragma unroll
        for (int i = 0; i < M; i++) pv[i] = P[i][q];
        double v = z[q];
#pragma unroll
        for (int i = 0; i < M; i++) v = fma(-beta[i], pv[i], v);
        pc[q] = v;
    }
}

// The window-length dispatch of kf_zdots and kf_p (0 <= win.n <= kMaxTrunc).
template <int M>
nek_status window_kernels(int64_t n, int nb, int sb, const double* c, const uint8_t* mask, double* z,
                          double* P, double* W, int64_t stride, int cur, const Window& win, double* parts,
                          FScal* sc, cudaStream_t s, int* launches)
{
    if constexpr (M < kMaxTrunc) {
        if (win.n != M)
            return window_kernels<M + 1>(n, nb, sb, c, mask, z, P, W, stride, cur, win, parts, sc, s, launches);
    }
    kf_zdots<M><<<nb, NT, 0, s>>>(n, c, mask, z, W, stride, win, parts);
    if (M > 0) kf_betas<<<1, NT, 0, s>>>(parts, nb, win, sc);
    kf_p<M><<<sb, 256, 0, s>>>(n, z, P, stride, cur, win, sc);
    *launches += M > 0 ? 3 : 2;
    return check_launch();
}

// w <- mask.w; partials <p,w> and <p,r>
__global__ void __launch_bounds__(NT) kf_pw(int64_t n, const double* __restrict__ c, const uint8_t* __restrict__ mask,
                                            const double* __restrict__ p, double* __restrict__ w,
                                            const double* __restrict__ r, double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
    double a = 0.0, b = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        double wq = w[q];
        if (!mask[q]) {
            wq = 0.0;
            w[q] = 0.0;
        }
        const double cp = c[q] * p[q];
        a += cp * wq;
        b += cp * r[q];
    }
    double t = block_sum<NT>(a, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
    t = block_sum<NT>(b, sh);
    if (threadIdx.x == 0) parts[gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) kf_alpha(const double* __restrict__ parts, int nb, int cur, FScal* sc)
{
    __shared__ double sh[NT / 32];
    const double pw = sum_partials<NT>(parts, nb, sh);
    const double pr = sum_partials<NT>(parts + nb, nb, sh);
    if (threadIdx.x == 0) {
        sc->pw = pw;
        sc->pr = pr;
        sc->pwv[cur] = pw;
        sc->alpha = pr / pw;
    }
}

// x += alpha p; r -= alpha w; partial <r,r>
__global__ void __launch_bounds__(NT) kf_update(int64_t n, const double* __restrict__ c,
                                                const double* __restrict__ p, const double* __restrict__ w,
                                                double* __restrict__ x, double* __restrict__ r,
                                                double* __restrict__ parts, const FScal* __restrict__ sc)
{
    __shared__ double sh[NT / 32];
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        x[q] = fma(alpha, p[q], x[q]);
        const double rq = fma(-alpha, w[q], r[q]);
        r[q] = rq;
        acc += c[q] * rq * rq;
    }
    const double t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct FLayout {
    double *r, *z, *P, *W, *minv, *parts;
    int64_t stride;  // doubles between ring slots
    float *xin, *scale;
    FScal* sc;
    size_t bytes;
};

FLayout f_layout(char* base, int64_t nelt, int nx, bool need_minv, int m)
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
    L.stride = static_cast<int64_t>(al256(v) / sizeof(double));
    L.r = reinterpret_cast<double*>(take(v));
    L.z = reinterpret_cast<double*>(take(v));
    L.P = reinterpret_cast<double*>(take(al256(v) * (m + 1)));
    L.W = reinterpret_cast<double*>(take(al256(v) * (m + 1)));
    L.minv = need_minv ? reinterpret_cast<double*>(take(v)) : nullptr;
    L.xin = reinterpret_cast<float*>(take(sizeof(float) * 2 * std::max<int64_t>(n, 1)));
    L.scale = reinterpret_cast<float*>(take(sizeof(float) * std::max<int64_t>(nelt, 1)));
    L.parts = reinterpret_cast<double*>(take(sizeof(double) * kMaxTrunc * kMaxReduceBlocks));
    L.sc = reinterpret_cast<FScal*>(take(sizeof(FScal)));
    L.bytes = off;
    return L;
}

}  // namespace

}  // namespace nek

using namespace nek;

extern "C" {

size_t nek_fcg_trunc_workspace_bytes(int64_t nelt, int nx, int need_minv, int truncation)
{
    if (nelt < 0 || nx < kMinNx || nx > kMaxNx || truncation < 1 || truncation > kMaxTrunc) return 0;
    return f_layout(nullptr, nelt, nx, need_minv != 0, truncation).bytes;
}

size_t nek_fcg_workspace_bytes(int64_t nelt, int nx, int need_minv)
{
    return nek_fcg_trunc_workspace_bytes(nelt, nx, need_minv, 1);
}

nek_status nek_fcg_solve_trunc(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                               const float* Gff, const uint8_t* mask, const double* minv, const float* theta,
                               const double* f, double* x, double tol_rel, int max_iter, int truncation,
                               int stag_window, double stag_factor, void* workspace, nek_fcg_info* info, void* stream)
{
    if (info) *info = nek_fcg_info{};
    if (nx != 8) return NEK_ERR_UNSUPPORTED_NX;  // the network is built for 8^3 element blocks
    if (!gs || nelt < 0 || max_iter < 0 || !(tol_rel > 0.0) || stag_window < 1 || !(stag_factor > 0.0) ||
        !(stag_factor < 1.0) || truncation < 1 || truncation > kMaxTrunc)
        return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (gs->npts != n) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!D || !G || !mask || !f || !x || !is_aligned(G, 16) || !is_aligned(x, 8) || (Gff && !is_aligned(Gff, 16)) ||
        (minv && !is_aligned(minv, 8)) || (workspace && !is_aligned(workspace, 256)))
        return NEK_ERR_INVALID_ARG;
    const int m = truncation;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = nek_fcg_trunc_workspace_bytes(nelt, nx, minv == nullptr, m);
    void* ws = workspace;
    if (!ws && check_cuda(cudaMallocAsync(&ws, bytes, s)) != NEK_OK) return NEK_ERR_NOMEM;
    FLayout L = f_layout(static_cast<char*>(ws), nelt, nx, minv == nullptr, m);
    const double* mv = minv;
    const int nb = reduce_blocks(n);
    const int sb = pcg::stream_blocks(n);
    nek_status st = NEK_OK;
    FScal h{};
    std::vector<double> hist;
    bool net = theta != nullptr;
    int it = 0, fell_back = 0, net_apps = 0, launches = 0;
    // ring of the last m directions: slot of direction k is k mod (m + 1); `have`
    // directions are in the window (0 after a restart)
    int have = 0;
    // one event pair per network application, read once at the end (no host
    // synchronisation inside the loop for the timing)
    std::vector<cudaEvent_t> nev;
    double net_ms = 0.0;

    auto precondition = [&]() -> nek_status {
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
            if (sp == NEK_OK) sp = launch_net_apply_tc5(nelt, theta, L.xin, L.scale, gs->d_c, L.z, s);
            if (sp == NEK_OK) sp = pcg::dssum<double>(gs, L.z, s);
            if (timed) cudaEventRecord(e1, s);
            if (sp != NEK_OK) return sp;
            net_apps++;
            launches += 3;
        } else {
            kf_jacobi<<<sb, 256, 0, s>>>(n, mv, L.r, L.z);
            launches += 1;
        }
        return check_launch();
    };

    if (!minv) {
        if ((st = nek_jacobi_minv(gs, nelt, nx, D, G, mask, L.minv, stream)) != NEK_OK) goto done;
        mv = L.minv;
        launches += 3;
    }
    kf_init<<<nb, NT, 0, s>>>(n, gs->d_c, mask, f, x, L.r, L.parts);
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
    for (it = 1; it <= max_iter; it++) {
        // the new direction: z = M(r), made A-orthogonal to the window
        if ((st = precondition()) != NEK_OK) goto done;
        const int cur = it % (m + 1);
        Window win{};
        win.n = have;
        for (int i = 0; i < have; i++) win.slot[i] = ((it - 1 - i) % (m + 1) + (m + 1)) % (m + 1);
        if ((st = window_kernels<0>(n, nb, sb, gs->d_c, mask, L.z, L.P, L.W, L.stride, cur, win, L.parts, L.sc, s,
                                     &launches)) != NEK_OK)
            goto done;
        double* p = L.P + cur * L.stride;
        double* w = L.W + cur * L.stride;
        st = Gff ? launch_ax_ff(nelt, nx, D, Gff, p, w, s) : launch_ax_fp64(nelt, nx, D, G, p, w, s);
        if (st != NEK_OK) goto done;
        if ((st = pcg::dssum<double>(gs, w, s)) != NEK_OK) goto done;
        kf_pw<<<nb, NT, 0, s>>>(n, gs->d_c, mask, p, w, L.r, L.parts);
        kf_alpha<<<1, NT, 0, s>>>(L.parts, nb, cur, L.sc);
        kf_update<<<nb, NT, 0, s>>>(n, gs->d_c, p, w, x, L.r, L.parts, L.sc);
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
        have = have < m ? have + 1 : m;
        if (net && it >= stag_window && h.relres > stag_factor * hist[it - stag_window]) {
            net = false;
            fell_back = it;
            have = 0;  // restart: the Jacobi directions start a new window
        }
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
    if (net_apps > 0) {  // a bounded wait inside the network kernel that ran out
        bool to = false;
        if (cudaStreamSynchronize(s) == cudaSuccess && net_tc5_take_timeout(&to) == NEK_OK && to)
            st = NEK_ERR_TIMEOUT;
    }
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

nek_status nek_fcg_solve(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G, const float* Gff,
                         const uint8_t* mask, const double* minv, const float* theta, const double* f, double* x,
                         double tol_rel, int max_iter, int stag_window, double stag_factor, void* workspace,
                         nek_fcg_info* info, void* stream)
{
    return nek_fcg_solve_trunc(gs, nelt, nx, D, G, Gff, mask, minv, theta, f, x, tol_rel, max_iter, 1, stag_window,
                               stag_factor, workspace, info, stream);
}

}  // extern "C"
