// Float-float AX launchers for nx = 8, 9 (kernels in nek_ax_ff_kernels.cuh).
#include "nek_ax_ff_kernels.cuh"

namespace nek {

nek_status launch_ax_ff_group_b(int nx, int epb, int64_t nelt, const double* D, const float* Gff, const double* u,
                                  double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                                  const uint8_t* pdone, double* edot, const DirUpdate* dir)
{
    switch (nx) {
        case 8: return launch_ax_ff_nx<8>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 9: return launch_ax_ff_nx<9>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
}

bool ax_ff_fits_group_b(int nx, int epb)
{
    switch (nx) {
        case 8: return ff_fits_rt<8>(epb);
        case 9: return ff_fits_rt<9>(epb);
        default: return false;
    }
}

}  // namespace nek
