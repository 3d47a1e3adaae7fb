// Status handling, GLL, mask, gather-scatter plan and dssum, weighted dot.
#include <cuda.h>  // CUcontext / CUresult types only: the two driver calls below are fetched at run time

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "nek_internal.h"
#include "nek_pcg.cuh"
#include "nek_reduce.cuh"

namespace nek {

namespace {
thread_local char g_last_error[256] = "";
}

nek_status cuda_fail(cudaError_t e)
{
    const char* s = cudaGetErrorString(e);
    std::strncpy(g_last_error, s ? s : "unknown CUDA error", sizeof(g_last_error) - 1);
    g_last_error[sizeof(g_last_error) - 1] = '\0';
    return NEK_ERR_CUDA;
}

int reduce_blocks(int64_t n)
{
    int64_t b = (n + kReduceThreads * 4 - 1) / (kReduceThreads * 4);
    if (b < 1) b = 1;
    if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
    return static_cast<int>(b);
}

// ------------------------------------------------------------------ mask
__global__ void k_mask(int64_t n, const uint8_t* __restrict__ mask, double* __restrict__ v)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        if (mask[p] == 0) v[p] = 0.0;
}

nek_status launch_mask(int64_t n, const uint8_t* mask, double* v, cudaStream_t s)
{
    if (n == 0) return NEK_OK;
    int64_t nb = (n + 255) / 256;
    int blocks = static_cast<int>(std::min<int64_t>(nb, 152 * 32));
    k_mask<<<blocks, 256, 0, s>>>(n, mask, v);
    return check_launch();
}

// ------------------------------------------------------------------ dssum
// One thread per group: left-to-right sum over members (ascending local index),
// then the sum is written back to every member.  Groups are disjoint.
nek_status launch_dssum(const nek_gs* gs, double* v, cudaStream_t s) { return pcg::dssum<double>(gs, v, s); }

// ------------------------------------------------------------------ dot
__global__ void __launch_bounds__(kReduceThreads) k_dot_c_partials(int64_t n, const double* __restrict__ c,
                                                                   const double* __restrict__ a,
                                                                   const double* __restrict__ b,
                                                                   double* __restrict__ parts)
{
    __shared__ double sh[kReduceThreads / 32];
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)kReduceThreads + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kReduceThreads)
        acc += c[p] * a[p] * b[p];
    double t = block_sum<kReduceThreads>(acc, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kReduceThreads) k_sum_partials(const double* __restrict__ parts, int nparts,
                                                                 double* __restrict__ out)
{
    __shared__ double sh[kReduceThreads / 32];
    double t = sum_partials<kReduceThreads>(parts, nparts, sh);
    if (threadIdx.x == 0) out[0] = t;
}

// Scratch of nek_dot_c_noalloc: one partial sum per reduction block.  It is part
// of the library image, so every GPU that loads the library holds these
// kNoAllocPartials doubles (9.5 KB) until the process exits, and all calls on a
// device share them.
constexpr int kNoAllocPartials = kMaxReduceBlocks;
constexpr int64_t kNoAllocMaxPoints = (int64_t(1) << 31) - 1;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;

// Per device: the array's device address and the id of the context it was
// looked up in.  cudaDeviceReset destroys the primary context (and with it the
// module that holds the array); the next context can place the array
// elsewhere, so an address is reused only while the context id is unchanged.
struct NoAllocSlot {
    double* ptr = nullptr;
    unsigned long long ctx_id = 0;
};
NoAllocSlot g_noalloc_slot[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the calling thread's current context, 0 if there is none (driver
// entry points fetched through the runtime, so the library does not link
// libcuda itself).
nek_status current_context_id(unsigned long long* id)
{
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        nek_status st = check_cuda(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        if (st == NEK_OK) st = check_cuda(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (st != NEK_OK) return st;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) return NEK_ERR_CUDA;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return NEK_ERR_CUDA;
    if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return NEK_ERR_CUDA;
    return NEK_OK;
}

// Device address of g_noalloc_partials on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress (which may load the module) the first time a device is
// used, and again only if that device's context has been replaced since.
nek_status noalloc_scratch(double** out)
{
    int dev = 0;
    nek_status st = check_cuda(cudaGetDevice(&dev));
    if (st != NEK_OK) return st;
    if (dev < 0 || dev >= kMaxDevices) return NEK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocSlot& slot = g_noalloc_slot[dev];
    unsigned long long id = 0;
    if ((st = current_context_id(&id)) != NEK_OK) return st;
    if (!slot.ptr || id == 0 || id != slot.ctx_id) {
        void* p = nullptr;
        if ((st = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_partials))) != NEK_OK) return st;
        if ((st = current_context_id(&id)) != NEK_OK) return st;  // the lookup made the primary context current
        slot.ptr = static_cast<double*>(p);
        slot.ctx_id = id;
    }
    *out = slot.ptr;
    return NEK_OK;
}
}  // namespace

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_dot_c_noalloc(int64_t n, const double* c, const double* a, const double* b, double* result,
                             void* stream)
{
    if (n < 0 || !result || !is_aligned(result, 8)) return NEK_ERR_INVALID_ARG;
    if (n > kNoAllocMaxPoints) return NEK_ERR_TOO_LARGE;
    if (n > 0 && (!c || !a || !b || !is_aligned(c, 8) || !is_aligned(a, 8) || !is_aligned(b, 8)))
        return NEK_ERR_INVALID_ARG;
    double* parts = nullptr;
    nek_status st = noalloc_scratch(&parts);
    if (st != NEK_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = reduce_blocks(n);  // <= kNoAllocPartials; every partial read below is written first
    k_dot_c_partials<<<nb, kReduceThreads, 0, s>>>(n, c, a, b, parts);
    st = check_launch();
    if (st != NEK_OK) return st;
    k_sum_partials<<<1, kReduceThreads, 0, s>>>(parts, nb, result);
    return check_launch();
}

const char* nek_status_string(int status)
{
    switch (status) {
        case NEK_OK: return "NEK_OK";
        case NEK_ERR_INVALID_ARG: return "NEK_ERR_INVALID_ARG";
        case NEK_ERR_UNSUPPORTED_NX: return "NEK_ERR_UNSUPPORTED_NX";
        case NEK_ERR_CUDA: return "NEK_ERR_CUDA";
        case NEK_ERR_NOT_CONVERGED: return "NEK_ERR_NOT_CONVERGED";
        case NEK_ERR_BREAKDOWN: return "NEK_ERR_BREAKDOWN";
        case NEK_ERR_TIMEOUT: return "NEK_ERR_TIMEOUT";
        case NEK_ERR_NOMEM: return "NEK_ERR_NOMEM";
        case NEK_ERR_TOO_LARGE: return "NEK_ERR_TOO_LARGE";
        default: return "NEK_ERR_UNKNOWN";
    }
}

const char* nek_last_error(void) { return g_last_error; }

int nek_version(void) { return 100; }

nek_status nek_gll(int nx, double* xi, double* rho, double* D)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    gll_host(nx, xi, rho, D);
    return NEK_OK;
}

nek_status nek_mask(int64_t n, const uint8_t* mask, double* v, void* stream)
{
    if (n < 0) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!mask || !v || !is_aligned(v, 8)) return NEK_ERR_INVALID_ARG;
    return launch_mask(n, mask, v, static_cast<cudaStream_t>(stream));
}

nek_status nek_gs_create(int64_t nelt, int nx, const int64_t* glo, nek_gs** out)
{
    if (!out) return NEK_ERR_INVALID_ARG;
    *out = nullptr;
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (n >= (int64_t(1) << 31)) return NEK_ERR_TOO_LARGE;
    if (n > 0 && !glo) return NEK_ERR_INVALID_ARG;
    return gs_create_flat(n, glo, out);
}

}  // extern "C"

namespace nek {

// Plan from a flat list of n global ids (the grouping does not depend on how the
// points are split into elements).
nek_status gs_create_flat(int64_t n, const int64_t* glo, nek_gs** out)
{
    *out = nullptr;
    int64_t gmax = -1;
    for (int64_t p = 0; p < n; p++) {
        if (glo[p] < 0) return NEK_ERR_INVALID_ARG;
        gmax = std::max(gmax, glo[p]);
    }
    std::vector<int32_t> offsets(1, 0), members;
    std::vector<double> c(static_cast<size_t>(n), 1.0);
    try {
        if (gmax < 4 * n + 1024) {
            // counting sort on the global id: members come out in ascending local index
            std::vector<int32_t> cnt(static_cast<size_t>(gmax + 1), 0);
            for (int64_t p = 0; p < n; p++) cnt[glo[p]]++;
            std::vector<int32_t> start(static_cast<size_t>(gmax + 1), -1);
            int32_t m = 0;
            for (int64_t g = 0; g <= gmax; g++)
                if (cnt[g] >= 2) {
                    start[g] = m;
                    m += cnt[g];
                    offsets.push_back(m);
                }
            members.resize(static_cast<size_t>(m));
            for (int64_t p = 0; p < n; p++) {
                const int64_t g = glo[p];
                c[p] = 1.0 / cnt[g];
                if (start[g] >= 0) members[start[g]++] = static_cast<int32_t>(p);
            }
        } else {
            std::vector<std::pair<int64_t, int32_t>> pr(static_cast<size_t>(n));
            for (int64_t p = 0; p < n; p++) pr[p] = {glo[p], static_cast<int32_t>(p)};
            std::sort(pr.begin(), pr.end());
            int64_t a = 0;
            while (a < n) {
                int64_t b = a + 1;
                while (b < n && pr[b].first == pr[a].first) b++;
                for (int64_t q = a; q < b; q++) c[pr[q].second] = 1.0 / double(b - a);
                if (b - a >= 2) {
                    for (int64_t q = a; q < b; q++) members.push_back(pr[q].second);
                    offsets.push_back(static_cast<int32_t>(members.size()));
                }
                a = b;
            }
        }
    } catch (const std::bad_alloc&) {
        return NEK_ERR_NOMEM;
    }
    nek_gs* gs = new (std::nothrow) nek_gs();
    if (!gs) return NEK_ERR_NOMEM;
    gs->npts = n;
    gs->ngroups = static_cast<int64_t>(offsets.size()) - 1;
    gs->nshared = static_cast<int64_t>(members.size());
    gs->d_offsets = nullptr;
    gs->d_members = nullptr;
    gs->d_c = nullptr;
    gs->d_partials = nullptr;
    nek_status st = NEK_OK;
    if ((st = check_cuda(cudaMalloc(&gs->d_offsets, sizeof(int32_t) * offsets.size()))) != NEK_OK) goto fail;
    if ((st = check_cuda(cudaMalloc(&gs->d_members, sizeof(int32_t) * std::max<size_t>(members.size(), 1)))) != NEK_OK)
        goto fail;
    if ((st = check_cuda(cudaMalloc(&gs->d_c, sizeof(double) * std::max<int64_t>(n, 1)))) != NEK_OK) goto fail;
    if ((st = check_cuda(cudaMemcpy(gs->d_offsets, offsets.data(), sizeof(int32_t) * offsets.size(),
                                    cudaMemcpyHostToDevice))) != NEK_OK)
        goto fail;
    if (!members.empty() &&
        (st = check_cuda(cudaMemcpy(gs->d_members, members.data(), sizeof(int32_t) * members.size(),
                                    cudaMemcpyHostToDevice))) != NEK_OK)
        goto fail;
    if (n > 0 &&
        (st = check_cuda(cudaMemcpy(gs->d_c, c.data(), sizeof(double) * n, cudaMemcpyHostToDevice))) != NEK_OK)
        goto fail;
    *out = gs;
    return NEK_OK;
fail:
    nek_gs_destroy(gs);
    return st;
}

}  // namespace nek

extern "C" {

nek_status nek_gs_destroy(nek_gs* gs)
{
    if (!gs) return NEK_OK;
    cudaFree(gs->d_offsets);
    cudaFree(gs->d_members);
    cudaFree(gs->d_c);
    cudaFree(gs->d_partials);
    delete gs;
    return NEK_OK;
}

nek_status nek_gs_info(const nek_gs* gs, int64_t* npts, int64_t* ngroups, int64_t* nshared)
{
    if (!gs) return NEK_ERR_INVALID_ARG;
    if (npts) *npts = gs->npts;
    if (ngroups) *ngroups = gs->ngroups;
    if (nshared) *nshared = gs->nshared;
    return NEK_OK;
}

nek_status nek_gs_export(const nek_gs* gs, int64_t* offsets_host, int64_t* members_host)
{
    if (!gs || !offsets_host || (gs->nshared > 0 && !members_host)) return NEK_ERR_INVALID_ARG;
    std::vector<int32_t> o(static_cast<size_t>(gs->ngroups + 1)), m(static_cast<size_t>(gs->nshared));
    nek_status st = check_cuda(cudaMemcpy(o.data(), gs->d_offsets, sizeof(int32_t) * o.size(), cudaMemcpyDeviceToHost));
    if (st != NEK_OK) return st;
    if (!m.empty()) {
        st = check_cuda(cudaMemcpy(m.data(), gs->d_members, sizeof(int32_t) * m.size(), cudaMemcpyDeviceToHost));
        if (st != NEK_OK) return st;
    }
    for (size_t q = 0; q < o.size(); q++) offsets_host[q] = o[q];
    for (size_t q = 0; q < m.size(); q++) members_host[q] = m[q];
    return NEK_OK;
}

nek_status nek_ax_ff_energy(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                            double* edot, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Gff || !u || !w || !edot) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(D, 8) || !is_aligned(Gff, 16) || !is_aligned(u, 8) || !is_aligned(w, 8) || !is_aligned(edot, 8))
        return NEK_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)nelt * nx * nx * nx, ebytes = sizeof(double) * (size_t)nelt;
    if (ranges_overlap(u, bytes, w, bytes) || ranges_overlap(edot, ebytes, u, bytes) ||
        ranges_overlap(edot, ebytes, w, bytes))
        return NEK_ERR_INVALID_ARG;
    return launch_ax_ff(nelt, nx, D, Gff, u, w, static_cast<cudaStream_t>(stream), nullptr, nullptr, nullptr, edot);
}

nek_status nek_dssum(const nek_gs* gs, double* v, void* stream)
{
    if (!gs) return NEK_ERR_INVALID_ARG;
    if (gs->npts == 0) return NEK_OK;
    if (!v || !is_aligned(v, 8)) return NEK_ERR_INVALID_ARG;
    return launch_dssum(gs, v, static_cast<cudaStream_t>(stream));
}

nek_status nek_gs_inv_multiplicity(const nek_gs* gs, double* c, void* stream)
{
    if (!gs) return NEK_ERR_INVALID_ARG;
    if (gs->npts == 0) return NEK_OK;
    if (!c) return NEK_ERR_INVALID_ARG;
    return check_cuda(cudaMemcpyAsync(c, gs->d_c, sizeof(double) * gs->npts, cudaMemcpyDeviceToDevice,
                                      static_cast<cudaStream_t>(stream)));
}

nek_status nek_dot_c(const nek_gs* gs, const double* a, const double* b, double* result, void* stream)
{
    if (!gs || !result || !is_aligned(result, 8)) return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (gs->npts > 0 && (!a || !b || !is_aligned(a, 8) || !is_aligned(b, 8))) return NEK_ERR_INVALID_ARG;
    if (!gs->d_partials) {
        nek_status st = check_cuda(cudaMalloc(&const_cast<nek_gs*>(gs)->d_partials, sizeof(double) * kMaxReduceBlocks));
        if (st != NEK_OK) return NEK_ERR_NOMEM;
    }
    const int nb = reduce_blocks(gs->npts);
    k_dot_c_partials<<<nb, kReduceThreads, 0, s>>>(gs->npts, gs->d_c, a, b, gs->d_partials);
    nek_status st = check_launch();
    if (st != NEK_OK) return st;
    k_sum_partials<<<1, kReduceThreads, 0, s>>>(gs->d_partials, nb, result);
    return check_launch();
}

}  // extern "C"
