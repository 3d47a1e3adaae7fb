// Elements-per-CTA selection for the AX kernels.
//
// Every AX kernel is compiled for several elements-per-CTA counts (1, 2, 4 where
// the thread count and shared memory allow).  The count changes only how
// elements are grouped into CTAs, never the arithmetic on an element, so all
// variants give bit-identical results; it trades occupancy against how much of
// a CTA's load phase overlaps other CTAs' compute.  nek_tune_ax times the
// variants on the caller's data and keeps the fastest for later launches.  The
// float-float kernel has two forms (plain, and with element energies for the
// solve), each tuned on its own: their register allocations differ.
#include <algorithm>
#include <atomic>

#include "nek_internal.h"

namespace nek {

namespace {
std::atomic<int> g_epb[3][kMaxNx + 1];  // NEK_AX_FP64, NEK_AX_FF, kAxFfEnergy
}

int tuned_epb(int impl, int nx)
{
    if (impl < 0 || impl > kAxFfEnergy || nx < 0 || nx > kMaxNx) return 0;
    return g_epb[impl][nx].load(std::memory_order_relaxed);
}

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_set_ax_epb(int impl, int nx, int epb)
{
    if (impl != NEK_AX_FP64 && impl != NEK_AX_FF && impl != NEK_AX_FF_ENERGY) return NEK_ERR_INVALID_ARG;
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (epb != 0 && !(impl == NEK_AX_FP64 ? ax_fp64_epb_fits(nx, epb) : ax_ff_epb_fits(nx, epb)))
        return NEK_ERR_INVALID_ARG;  // not one of the compiled counts, or too many threads / too much smem
    g_epb[impl][nx].store(epb, std::memory_order_relaxed);
    if (impl == NEK_AX_FF) g_epb[kAxFfEnergy][nx].store(epb, std::memory_order_relaxed);
    return NEK_OK;
}

int nek_get_ax_epb(int impl, int nx)
{
    return impl == NEK_AX_FP64 || impl == NEK_AX_FF || impl == NEK_AX_FF_ENERGY ? tuned_epb(impl, nx) : 0;
}

nek_status nek_tune_ax(int impl, int64_t nelt, int nx, const double* D, const void* Gx, const double* u, double* w,
                       int* epb_out, float* ms_out, void* stream)
{
    if (impl != NEK_AX_FP64 && impl != NEK_AX_FF) return NEK_ERR_INVALID_ARG;
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt <= 0 || !D || !Gx || !u || !w || !is_aligned(Gx, 16) || !is_aligned(u, 16) || !is_aligned(w, 16))
        return NEK_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)nelt * nx * nx * nx;
    if (ranges_overlap(u, bytes, w, bytes)) return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    constexpr int kReps = 7;  // individually timed launches per candidate; the median is kept
    cudaEvent_t ev[kReps + 1] = {};
    double* edot = nullptr;  // element energies of the float-float solve form
    nek_status st = NEK_OK;
    for (int r = 0; r <= kReps && st == NEK_OK; r++) st = check_cuda(cudaEventCreate(&ev[r]));
    if (st == NEK_OK && impl == NEK_AX_FF)
        if (check_cuda(cudaMalloc(&edot, sizeof(double) * (size_t)nelt)) != NEK_OK) st = NEK_ERR_NOMEM;
    int best_plain = 0;
    float best_plain_ms = 0.f;
    const int nforms = impl == NEK_AX_FF ? 2 : 1;
    for (int form = 0; form < nforms && st == NEK_OK; form++) {
        int best = 0;
        float best_ms = 0.f;
        const int cand[3] = {1, 2, 4};
        for (int c = 0; c < 3 && st == NEK_OK; c++) {
            auto run = [&]() {
                return impl == NEK_AX_FF
                           ? launch_ax_ff_epb(cand[c], nelt, nx, D, static_cast<const float*>(Gx), u, w, s, nullptr,
                                              nullptr, nullptr, form ? edot : nullptr)
                           : launch_ax_fp64_epb(cand[c], nelt, nx, D, static_cast<const double*>(Gx), u, w, s);
            };
            nek_status sv = run();
            if (sv == NEK_ERR_INVALID_ARG) continue;  // this count does not fit this nx
            if (sv != NEK_OK) {
                st = sv;
                break;
            }
            if ((st = run()) != NEK_OK) break;
            cudaEventRecord(ev[0], s);
            for (int r = 0; r < kReps && st == NEK_OK; r++) {
                st = run();
                cudaEventRecord(ev[r + 1], s);
            }
            if (st != NEK_OK) break;
            if ((st = check_cuda(cudaEventSynchronize(ev[kReps]))) != NEK_OK) break;
            float t[kReps];
            for (int r = 0; r < kReps; r++) cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]);
            std::sort(t, t + kReps);
            const float ms = t[kReps / 2];
            if (best == 0 || ms < best_ms) {
                best = cand[c];
                best_ms = ms;
            }
        }
        if (st == NEK_OK && best == 0) st = NEK_ERR_INVALID_ARG;
        if (st != NEK_OK) break;
        g_epb[form ? kAxFfEnergy : impl][nx].store(best, std::memory_order_relaxed);
        if (form == 0) {
            best_plain = best;
            best_plain_ms = best_ms;
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (edot) cudaFree(edot);
    if (st != NEK_OK) return st;
    if (epb_out) *epb_out = best_plain;
    if (ms_out) *ms_out = best_plain_ms;
    return NEK_OK;
}

}  // extern "C"
