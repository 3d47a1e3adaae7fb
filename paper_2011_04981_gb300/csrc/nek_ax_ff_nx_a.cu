// Float-float AX launchers for nx = 2, 3, 4, 5, 6, 7 (kernels in nek_ax_ff_kernels.cuh).
#include "nek_ax_ff_kernels.cuh"

namespace nek {

nek_status launch_ax_ff_group_a(int nx, int epb, int64_t nelt, const double* D, const float* Gff, const double* u,
                                  double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                                  const uint8_t* pdone, double* edot, const DirUpdate* dir)
{
    switch (nx) {
        case 2: return launch_ax_ff_nx<2>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 3: return launch_ax_ff_nx<3>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 4: return launch_ax_ff_nx<4>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 5: return launch_ax_ff_nx<5>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 6: return launch_ax_ff_nx<6>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        case 7: return launch_ax_ff_nx<7>(epb, nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
}

bool ax_ff_fits_group_a(int nx, int epb)
{
    switch (nx) {
        case 2: return ff_fits_rt<2>(epb);
        case 3: return ff_fits_rt<3>(epb);
        case 4: return ff_fits_rt<4>(epb);
        case 5: return ff_fits_rt<5>(epb);
        case 6: return ff_fits_rt<6>(epb);
        case 7: return ff_fits_rt<7>(epb);
        default: return false;
    }
}

}  // namespace nek
