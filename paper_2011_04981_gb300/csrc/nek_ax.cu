// AX operator, native FP64 (Section II-B, Listing 1 of arXiv 2011.04981).
//
// Per element the operator is
//   ur = D_r u, us = D_s u, ut = D_t u             (local_grad3)
//   [wr ws wt] = G [ur us ut]                        (the pointwise g product)
//   w = D_r^T wr + D_s^T ws + D_t^T wt               (local_grad3_t)
// with D_r acting on i, D_s on j and D_t on k of the [k][j][i] block.
//
// Kernel layout: a CTA owns EPB elements and has nx*nx*EPB threads; thread
// (e, i, j) keeps the k-line u(i,j,:) and the t-results wt(i,j,:) in registers
// and walks the k planes.  The u block of every element is staged in shared
// memory once (one coalesced read of u: the FPGA design's single read of every
// grid point of u becomes one pass through HBM here) so that the r- and
// s-contractions read it from shared memory in their own order, which is what
// the per-matmul reorder buffers of the FPGA design (Section III) achieve.
// ws goes to shared memory as it is produced; wr is kept in registers until
// every thread has finished reading u, then overwrites the u block, so each
// element needs 2*nx^3 doubles of shared memory.  G is streamed from HBM exactly
// once, w written exactly once.
#include <algorithm>

#include "nek_internal.h"

namespace nek {

namespace {

// Elements per CTA for each nx, chosen so that nx*nx*EPB threads fill whole
// warps as far as possible and several CTAs fit on one SM.
constexpr int ax_epb(int nx)
{
    return nx == 2 ? 32 : nx == 3 ? 32 : nx == 4 ? 8 : nx == 5 ? 16 : nx == 6 ? 8 : nx == 7 ? 8 : nx == 8 ? 4
         : nx == 9 ? 4 : nx == 10 ? 4 : nx == 11 ? 2 : nx == 12 ? 2 : nx == 13 ? 2 : 1;
}

template <int NX, int EPB>
constexpr size_t ax_smem_bytes()
{
    return sizeof(double) * (size_t)(NX * NX + 2 * EPB * NX * NX * NX + 1);
}

template <int NX, int EPB>
__global__ void __launch_bounds__(NX* NX* EPB) k_ax_fp64(int64_t nelt, const double* __restrict__ D,
                                                          const double* __restrict__ G,
                                                          const double* __restrict__ u, double* __restrict__ w)
{
    constexpr int N2 = NX * NX, N3 = NX * NX * NX, NT = N2 * EPB;
    constexpr int DPAD = (N2 + 1) & ~1;  // keep the element blocks 16-byte aligned
    extern __shared__ double smem[];
    double* sD = smem;
    double* sA = smem + DPAD;     // u, then wr   [EPB][N3]
    double* sB = sA + EPB * N3;   // ws           [EPB][N3]

    const int tid = threadIdx.x;
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int ne = static_cast<int>(nelt - e0 < EPB ? nelt - e0 : EPB);

    for (int q = tid; q < N2; q += NT) sD[q] = D[q];
    if ((reinterpret_cast<uintptr_t>(u + e0 * N3) & 15) == 0) {  // 16-byte aligned block start: vector loads
        const double2* src = reinterpret_cast<const double2*>(u + e0 * N3);
        double2* dst = reinterpret_cast<double2*>(sA);
        const int nv = (ne * N3) / 2;
        for (int q = tid; q < nv; q += NT) dst[q] = __ldg(src + q);
        if ((ne * N3) & 1) {
            if (tid == 0) sA[ne * N3 - 1] = __ldg(u + e0 * N3 + ne * N3 - 1);
        }
    } else {
        const double* src = u + e0 * N3;
        for (int q = tid; q < ne * N3; q += NT) sA[q] = __ldg(src + q);
    }
    __syncthreads();

    const int el = tid / N2;
    const int q2 = tid - el * N2;
    const int i = q2 % NX, j = q2 / NX;
    const bool active = el < ne;
    double* ue = sA + el * N3;
    double* se = sB + el * N3;

    double ul[NX], wr[NX], wt[NX];
    if (active) {
#pragma unroll
        for (int l = 0; l < NX; l++) ul[l] = ue[i + NX * (j + NX * l)];
        const double* Ge = G + (e0 + el) * (int64_t)N3 * 6;
#pragma unroll
        for (int k = 0; k < NX; k++) {
            const int p = i + NX * (j + NX * k);
            double ar = 0.0, as = 0.0, at = 0.0;
#pragma unroll
            for (int l = 0; l < NX; l++) {
                ar = fma(sD[i * NX + l], ue[l + NX * (j + NX * k)], ar);
                as = fma(sD[j * NX + l], ue[i + NX * (l + NX * k)], as);
                at = fma(sD[k * NX + l], ul[l], at);
            }
            const double2* g2 = reinterpret_cast<const double2*>(Ge + 6 * p);
            const double2 g01 = __ldg(g2), g23 = __ldg(g2 + 1), g45 = __ldg(g2 + 2);
            wr[k] = fma(g01.x, ar, fma(g01.y, as, g23.x * at));
            se[p] = fma(g01.y, ar, fma(g23.y, as, g45.x * at));
            wt[k] = fma(g23.x, ar, fma(g45.x, as, g45.y * at));
        }
    }
    __syncthreads();  // every thread is done reading u
    if (active) {
#pragma unroll
        for (int k = 0; k < NX; k++) ue[i + NX * (j + NX * k)] = wr[k];
    }
    __syncthreads();
    if (active) {
        double* we = w + (e0 + el) * (int64_t)N3;
#pragma unroll
        for (int k = 0; k < NX; k++) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < NX; l++) {
                s = fma(sD[l * NX + i], ue[l + NX * (j + NX * k)], s);
                s = fma(sD[l * NX + j], se[i + NX * (l + NX * k)], s);
                s = fma(sD[l * NX + k], wt[l], s);
            }
            we[i + NX * (j + NX * k)] = s;
        }
    }
}

template <int NX, int EPB>
nek_status launch_ax_variant(int64_t nelt, const double* D, const double* G, const double* u, double* w,
                             cudaStream_t s)
{
    constexpr size_t smem = ax_smem_bytes<NX, EPB>();
    static std::atomic<uint64_t> configured{0};
    nek_status st = ensure_dyn_smem(k_ax_fp64<NX, EPB>, smem, configured);
    if (st != NEK_OK) return st;
    const int64_t blocks = (nelt + EPB - 1) / EPB;
    if (blocks > 0x7fffffff) return NEK_ERR_TOO_LARGE;
    k_ax_fp64<NX, EPB><<<(unsigned)blocks, NX * NX * EPB, smem, s>>>(nelt, D, G, u, w);
    return check_launch();
}

template <int NX, int EPB>
constexpr bool ax_fits()
{
    return NX * NX * EPB <= 1024 && ax_smem_bytes<NX, EPB>() <= 227 * 1024;
}

template <int NX>
nek_status launch_ax_nx(int epb, int64_t nelt, const double* D, const double* G, const double* u, double* w,
                        cudaStream_t s)
{
    if (epb <= 0) epb = ax_epb(NX);
    switch (epb) {
        case 1:
            if constexpr (ax_fits<NX, 1>()) return launch_ax_variant<NX, 1>(nelt, D, G, u, w, s);
            break;
        case 2:
            if constexpr (ax_fits<NX, 2>()) return launch_ax_variant<NX, 2>(nelt, D, G, u, w, s);
            break;
        case 4:
            if constexpr (ax_fits<NX, 4>()) return launch_ax_variant<NX, 4>(nelt, D, G, u, w, s);
            break;
        default:
            break;
    }
    if constexpr (ax_epb(NX) != 1 && ax_epb(NX) != 2 && ax_epb(NX) != 4)
        return launch_ax_variant<NX, ax_epb(NX)>(nelt, D, G, u, w, s);
    return NEK_ERR_INVALID_ARG;
}

}  // namespace

nek_status launch_ax_fp64_epb(int epb, int64_t nelt, int nx, const double* D, const double* G, const double* u,
                              double* w, cudaStream_t s)
{
    switch (nx) {
        case 2: return launch_ax_nx<2>(epb, nelt, D, G, u, w, s);
        case 3: return launch_ax_nx<3>(epb, nelt, D, G, u, w, s);
        case 4: return launch_ax_nx<4>(epb, nelt, D, G, u, w, s);
        case 5: return launch_ax_nx<5>(epb, nelt, D, G, u, w, s);
        case 6: return launch_ax_nx<6>(epb, nelt, D, G, u, w, s);
        case 7: return launch_ax_nx<7>(epb, nelt, D, G, u, w, s);
        case 8: return launch_ax_nx<8>(epb, nelt, D, G, u, w, s);
        case 9: return launch_ax_nx<9>(epb, nelt, D, G, u, w, s);
        case 10: return launch_ax_nx<10>(epb, nelt, D, G, u, w, s);
        case 11: return launch_ax_nx<11>(epb, nelt, D, G, u, w, s);
        case 12: return launch_ax_nx<12>(epb, nelt, D, G, u, w, s);
        case 13: return launch_ax_nx<13>(epb, nelt, D, G, u, w, s);
        case 14: return launch_ax_nx<14>(epb, nelt, D, G, u, w, s);
        case 15: return launch_ax_nx<15>(epb, nelt, D, G, u, w, s);
        case 16: return launch_ax_nx<16>(epb, nelt, D, G, u, w, s);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
}

namespace {
template <int NX>
bool ax_fits_rt(int epb)
{
    return (epb == 1 && ax_fits<NX, 1>()) || (epb == 2 && ax_fits<NX, 2>()) || (epb == 4 && ax_fits<NX, 4>());
}
}  // namespace

bool ax_fp64_epb_fits(int nx, int epb)
{
    switch (nx) {
        case 2: return ax_fits_rt<2>(epb);
        case 3: return ax_fits_rt<3>(epb);
        case 4: return ax_fits_rt<4>(epb);
        case 5: return ax_fits_rt<5>(epb);
        case 6: return ax_fits_rt<6>(epb);
        case 7: return ax_fits_rt<7>(epb);
        case 8: return ax_fits_rt<8>(epb);
        case 9: return ax_fits_rt<9>(epb);
        case 10: return ax_fits_rt<10>(epb);
        case 11: return ax_fits_rt<11>(epb);
        case 12: return ax_fits_rt<12>(epb);
        case 13: return ax_fits_rt<13>(epb);
        case 14: return ax_fits_rt<14>(epb);
        case 15: return ax_fits_rt<15>(epb);
        case 16: return ax_fits_rt<16>(epb);
        default: return false;
    }
}

nek_status launch_ax_fp64(int64_t nelt, int nx, const double* D, const double* G, const double* u, double* w,
                          cudaStream_t s)
{
    return launch_ax_fp64_epb(tuned_epb(NEK_AX_FP64, nx), nelt, nx, D, G, u, w, s);
}

}  // namespace nek

using namespace nek;

extern "C" nek_status nek_ax(int64_t nelt, int nx, const double* D, const double* G, const double* u, double* w,
                             void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !G || !u || !w) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(D, 8) || !is_aligned(G, 16) || !is_aligned(u, 8) || !is_aligned(w, 8))
        return NEK_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)nelt * nx * nx * nx;
    if (ranges_overlap(u, bytes, w, bytes)) return NEK_ERR_INVALID_ARG;
    return launch_ax_fp64(nelt, nx, D, G, u, w, static_cast<cudaStream_t>(stream));
}
