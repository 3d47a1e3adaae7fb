// Internal declarations shared by the translation units of libnekax.so.
#pragma once

#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nekax.h"

namespace nek {

constexpr int kMinNx = 2;
constexpr int kMaxNx = 16;

struct DirUpdate;   // below
struct DirUpdateF;  // below

// Record a CUDA error in the calling thread's last-error slot and map it to NEK_ERR_CUDA.
nek_status cuda_fail(cudaError_t e);
inline nek_status check_cuda(cudaError_t e) { return e == cudaSuccess ? NEK_OK : cuda_fail(e); }
inline nek_status check_launch() { return check_cuda(cudaGetLastError()); }

inline bool is_aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (the attribute belongs to the device's context: set
// on one GPU only, a launch with more than 48 KB on another would fail).
// done_mask: one bit per device ordinal (< 64), static storage of the caller.
template <class K>
nek_status ensure_dyn_smem(K kernel, size_t bytes, std::atomic<uint64_t>& done_mask)
{
    int dev = 0;
    nek_status st = check_cuda(cudaGetDevice(&dev));
    if (st != NEK_OK) return st;
    const uint64_t bit = dev >= 0 && dev < 64 ? (uint64_t(1) << dev) : 0;
    if (bit && (done_mask.load(std::memory_order_acquire) & bit)) return NEK_OK;
    st = check_cuda(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (st == NEK_OK && bit) done_mask.fetch_or(bit, std::memory_order_release);
    return st;
}
inline bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb)
{
    uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// Gather-scatter plan from a flat list of n non-negative global ids (n < 2^31).
nek_status gs_create_flat(int64_t n, const int64_t* glo, nek_gs** out);

// Host GLL rule: ascending nodes, weights, D[i*nx+l] = l_l'(xi_i).
void gll_host(int nx, double* xi, double* rho, double* D);

// Elements per CTA of the AX kernels: 0 = built-in default, else the value chosen
// by nek_tune_ax for (impl, nx); impl kAxFfEnergy is the float-float kernel in
// its element-energy form.
constexpr int kAxFfEnergy = NEK_AX_FF_ENERGY;
int tuned_epb(int impl, int nx);
bool ax_fp64_epb_fits(int nx, int epb);
bool ax_ff_epb_fits(int nx, int epb);
nek_status launch_ax_fp64_epb(int epb, int64_t nelt, int nx, const double* D, const double* G, const double* u,
                              double* w, cudaStream_t s);
// l2g (optional): u is then a unique-node vector and element point p of the
// launch reads u[l2g[p]] (the gather Q u of the unique-node form).
// eprob, pdone (optional, batched solves): problem of each element of the
// launch and one byte per problem, nonzero once it has finished; CTAs whose
// elements all belong to finished problems do nothing.
// edot (optional, nelt doubles): edot[e] = u_e . w_e, the element's energy
// (u_e gathered through l2g when given), summed in an order fixed by nx alone
// (with eprob/pdone, skipped elements' entries are left as they were).
nek_status launch_ax_ff_epb(int epb, int64_t nelt, int nx, const double* D, const float* Gff, const double* u,
                            double* w, cudaStream_t s, const int32_t* l2g = nullptr, const int32_t* eprob = nullptr,
                            const uint8_t* pdone = nullptr, double* edot = nullptr,
                            const DirUpdate* dir = nullptr);

// Kernel launchers (arguments already validated).
nek_status launch_ax_fp64(int64_t nelt, int nx, const double* D, const double* G, const double* u, double* w,
                          cudaStream_t s);
// dir (optional, with edot, without l2g / eprob, where ax_ff_dir_supported):
// the direction update above; u is then ignored (the input is dir->p).
nek_status launch_ax_ff(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                        cudaStream_t s, const int32_t* l2g = nullptr, const int32_t* eprob = nullptr,
                        const uint8_t* pdone = nullptr, double* edot = nullptr, const DirUpdate* dir = nullptr);
// The tcgen05 form of the reduced-precision operator (BF16 / FP16, nx 2..11).  edot (optional): element
// energies; dir (optional, with edot): the FP32 direction update below, input dir->p (u ignored).
bool ax_lowp_tc5_supported(int nx, int precision);
nek_status launch_ax_lowp_tc5(int precision, int64_t nelt, int nx, const double* D, const void* Glp,
                              const float* gscale, const float* u, float* w, cudaStream_t s, double* edot = nullptr,
                              const DirUpdateF* dir = nullptr);
// edot (optional, nelt doubles): per-element energies u_e . w_e in FP64; dir (optional, with edot): the
// FP32 direction update (DirUpdateF), input dir->p (u ignored).
nek_status launch_ax_lowp(int prec, int64_t nelt, int nx, const double* D, const void* Glp, const float* gscale,
                          const float* u, float* w, cudaStream_t s, double* edot = nullptr,
                          const DirUpdateF* dir = nullptr);
nek_status launch_mask(int64_t n, const uint8_t* mask, double* v, cudaStream_t s);
// Diagonal of the element operators (before summation over shared nodes).
nek_status launch_diag_local(int64_t nelt, int nx, const double* D, const double* G, double* d, cudaStream_t s);
nek_status launch_dssum(const nek_gs* gs, double* v, cudaStream_t s);

// Device scalars of the PCG loop (nek_pcg.cuh).
struct PcgScalars {
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
    int xpend;      // this iteration's x += alpha p is still to be applied
};

// The PCG direction update done by the float-float operator as it loads its
// input (the solve's separate x / direction pass then disappears): on every
// point of the launch, x += alpha p (old p) while sc->xpend is set, then
// p = minv r + beta p while the solve goes on (not done, no breakdown), and
// the operator is applied to the new p, which it also writes back to p.
struct DirUpdate {
    double* p;
    const double* r;
    const double* minv;
    double* x;
    const PcgScalars* sc;
};
// The same update on FP32 vectors (the inner solve of defect correction), with alpha and beta rounded to
// float and the operations of that solve's own update, x = fma(alpha, p, x) and p = fma(beta, p, minv r).
struct DirUpdateF {
    float* p;
    const float* r;
    const float* minv;
    float* x;
    const PcgScalars* sc;
};
// True where launch_ax_ff supports dir (every nx of the float-float kernels).
bool ax_ff_dir_supported(int nx);

// The tensor-core FP64-accurate operator (nek_ax_oz): even nx up to 10.  Goz from nek_geom_oz; u, w
// 16-byte aligned.  edot (optional): element energies, as for launch_ax_ff; dir (optional, with edot):
// the direction update, input dir->p (u ignored), every array 16-byte aligned.
bool ax_oz_supported(int nx);
nek_status launch_ax_oz(int64_t nelt, int nx, const double* D, const float* Goz, const double* u, double* w,
                        cudaStream_t s, double* edot = nullptr, const DirUpdate* dir = nullptr);
nek_status launch_ax_oz_ex(int64_t nelt, int nx, const double* D, const float* Goz, const double* u, double* w,
                           cudaStream_t s, long long wait_ns, int arrivals, double* edot, const DirUpdate* dir);

// Deterministic block-partial reductions use this fixed grid for a given length.
int reduce_blocks(int64_t n);
constexpr int kReduceThreads = 256;
constexpr int kMaxReduceBlocks = 152 * 8;

}  // namespace nek

// Gather-scatter plan (opaque to callers).
struct nek_gs {
    int64_t npts;      // local points
    int64_t ngroups;   // groups with >= 2 members
    int64_t nshared;   // local points that belong to a group
    int32_t* d_offsets;  // ngroups+1
    int32_t* d_members;  // nshared
    double* d_c;         // npts: 1/multiplicity
    double* d_partials;  // scratch for nek_dot_c (kMaxReduceBlocks doubles), lazily allocated
};
