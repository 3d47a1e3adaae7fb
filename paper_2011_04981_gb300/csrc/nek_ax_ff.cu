// AX operator to FP64 accuracy on the FP32 pipes: the FP64 -> float-pair
// split of the geometric factors, the nx dispatch of the launchers and the
// C entry points.  The kernels and the arithmetic are described in
// nek_ax_ff_kernels.cuh.
#include "nek_ax_ff_kernels.cuh"

namespace nek {

namespace {

// G (FP64, [e][p][6]) -> float-float [e][p][12] = (h0,l0,h1,l1,...,h5,l5).
__global__ void k_g_to_ff(int64_t npts, const double* __restrict__ G, float2* __restrict__ Gff)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npts * 6;
         q += (int64_t)gridDim.x * blockDim.x)
        Gff[q] = split_double(G[q]);
}

int ff_group(int nx) { return nx <= 7 ? 0 : nx <= 9 ? 1 : nx <= 11 ? 2 : nx <= 13 ? 3 : 4; }

}  // namespace

nek_status launch_ax_ff_epb(int epb, int64_t nelt, int nx, const double* D, const float* Gff, const double* u,
                            double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                            const uint8_t* pdone, double* edot, const DirUpdate* dir)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    switch (ff_group(nx)) {
        case 0: return launch_ax_ff_group_a(nx, epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 1: return launch_ax_ff_group_b(nx, epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 2: return launch_ax_ff_group_c(nx, epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 3: return launch_ax_ff_group_d(nx, epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        default: return launch_ax_ff_group_e(nx, epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
    }
}

bool ax_ff_epb_fits(int nx, int epb)
{
    if (nx < kMinNx || nx > kMaxNx) return false;
    switch (ff_group(nx)) {
        case 0: return ax_ff_fits_group_a(nx, epb);
        case 1: return ax_ff_fits_group_b(nx, epb);
        case 2: return ax_ff_fits_group_c(nx, epb);
        case 3: return ax_ff_fits_group_d(nx, epb);
        default: return ax_ff_fits_group_e(nx, epb);
    }
}

nek_status launch_ax_ff(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                        cudaStream_t s, const int32_t* l2g, const int32_t* eprob, const uint8_t* pdone,
                        double* edot, const DirUpdate* dir)
{
    return launch_ax_ff_epb(tuned_epb(edot ? kAxFfEnergy : NEK_AX_FF, nx), nelt, nx, D, Gff, u, w, s, l2g, eprob,
                            pdone, edot, dir);
}

bool ax_ff_dir_supported(int nx) { return nx >= kMinNx && nx <= kMaxNx; }

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_geom_ff(int64_t nelt, int nx, const double* G, float* Gff, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!G || !Gff || !is_aligned(G, 8) || !is_aligned(Gff, 16)) return NEK_ERR_INVALID_ARG;
    const int64_t npts = nelt * (int64_t)nx * nx * nx;
    if (ranges_overlap(G, sizeof(double) * 6 * npts, Gff, sizeof(float) * 12 * npts)) return NEK_ERR_INVALID_ARG;
    const int64_t nb = (npts * 6 + 255) / 256;
    const int blocks = static_cast<int>(nb < 152 * 32 ? nb : 152 * 32);
    k_g_to_ff<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(npts, G, reinterpret_cast<float2*>(Gff));
    return check_launch();
}

nek_status nek_ax_ff(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                     void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Gff || !u || !w) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(D, 8) || !is_aligned(Gff, 16) || !is_aligned(u, 8) || !is_aligned(w, 8))
        return NEK_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)nelt * nx * nx * nx;
    if (ranges_overlap(u, bytes, w, bytes)) return NEK_ERR_INVALID_ARG;
    return launch_ax_ff(nelt, nx, D, Gff, u, w, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
