/*
 * nekax: GB300 (sm_103a) spectral-element Poisson operator and Jacobi-PCG solve.
 *
 * C ABI of libnekax.so.  Every entry point takes plain pointers and sizes, never
 * throws, and reports failure through a nek_status return code.  Arguments are
 * validated on the host before anything is launched; on a validation failure
 * nothing is enqueued and no output is touched.
 *
 * The operator is Nekbone's AX as given in Section II-B, Listing 1 of
 * N. Brown, "Exploring the acceleration of Nekbone on reconfigurable
 * architectures" (arXiv 2011.04981): per element,
 *     w = Dr^T (G (D u))  summed over the three reference directions,
 * with the derivative matrix applied along r, s and t of the nx^3 block, the
 * 3x3 symmetric geometric factors applied pointwise and the transposed
 * contractions summed back.  The surrounding solve (gather-scatter, mask,
 * Jacobi-preconditioned CG) is the CG iteration the same section describes.
 *
 * Conventions shared by all entry points:
 *   - nx is the number of GLL points per direction (order nx-1), 2 <= nx <= 16;
 *   - an E-vector holds nelt*nx^3 doubles, element-major, [e][k][j][i] with i
 *     fastest (Fortran u(nx,nx,nx,nelt));
 *   - the geometric factors G are [e][k][j][i][6] in the order
 *     (rr, rs, rt, ss, st, tt) = g(1..6) of Listing 1;
 *   - D is nx*nx doubles, row-major, D[i*nx + l] = l_l'(xi_i) (Nekbone's dxm1
 *     read row-wise, i.e. the memory of dxtm1);
 *   - "device" pointers are CUDA device (or managed) memory owned by the caller;
 *     E-vector and G pointers must be 16-byte aligned, D 8-byte aligned;
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     calls are asynchronous unless stated otherwise.
 */
#ifndef NEKAX_H
#define NEKAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NEK_OK = 0,
    NEK_ERR_INVALID_ARG = 1,    /* null/misaligned pointer, negative size, aliasing */
    NEK_ERR_UNSUPPORTED_NX = 2, /* nx outside [2, 16] */
    NEK_ERR_CUDA = 3,           /* a CUDA call failed; see nek_last_error() */
    NEK_ERR_NOT_CONVERGED = 4,  /* CG reached max_iter before tol */
    NEK_ERR_BREAKDOWN = 5,      /* CG: p.Ap <= 0 or a non-finite scalar */
    NEK_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
    NEK_ERR_NOMEM = 7,          /* host or device allocation failed */
    NEK_ERR_TOO_LARGE = 8       /* problem exceeds an index-width limit */
} nek_status;

/* Human-readable name of a status code (static string, never NULL). */
const char* nek_status_string(int status);

/* Text of the last CUDA error seen by this thread inside the library ("" if none). */
const char* nek_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int nek_version(void);

/* ---------------------------------------------------------------- set-up ---
 * GLL rule on nx points (host, synchronous).  xi, rho: nx doubles each,
 * ascending nodes and weights; D: nx*nx doubles, D[i*nx+l] = l_l'(xi_i).  Any
 * output pointer may be NULL.  The paper takes dxm1/dxtm1 as given (Listing 1);
 * these are the standard Gauss-Lobatto-Legendre collocation objects.
 */
nek_status nek_gll(int nx, double* xi, double* rho, double* D);

/*
 * Geometric factors of trilinear hexahedra (device, async).
 *   corners: device, nelt*8*3 doubles; corner q = di + 2 dj + 4 dk of element e
 *            is the vertex at reference (2di-1, 2dj-1, 2dk-1), xyz fastest.
 *   G:       device output, nelt*nx^3*6 doubles (layout above).
 * G_ab = rho_i rho_j rho_k |J| (grad r_a . grad r_b) at every GLL node, the 6
 * factors Listing 1 multiplies by (the paper does not say how they are built).
 * Elements with a non-positive Jacobian still produce finite-or-not values;
 * the caller checks its mesh.
 */
nek_status nek_geom(int64_t nelt, int nx, const double* corners, double* G, void* stream);

/* ------------------------------------------------------------------ AX ---
 * w = AX(u) on every element (Section II-B, Listing 1: ax, ax_e, local_grad3
 * and the transposed local_grad3_t), FP64 throughout.
 *   nelt >= 0 elements (0 is a no-op), 2 <= nx <= 16;
 *   D: device, nx*nx; G: device, nelt*nx^3*6; u: device, in; w: device, out.
 *   u and w must not overlap.  Async on stream.
 * Native FP64 arithmetic on the double-precision pipe.
 */
nek_status nek_ax(int64_t nelt, int nx, const double* D, const double* G, const double* u, double* w,
                  void* stream);

/*
 * Geometric factors split into float pairs for nek_ax_ff (device, async):
 * Gff[e][p][2a] + Gff[e][p][2a+1] = G[e][p][a] to ~2^-48 relative, a = 0..5,
 * i.e. 12 floats (48 bytes) per point, the same size as the FP64 layout.
 * G: device, 8-byte aligned; Gff: device, 16-byte aligned, must not overlap G.
 * Values must lie in the normal FP32 range (|g| in about [1e-30, 1e30]).
 */
nek_status nek_geom_ff(int64_t nelt, int nx, const double* G, float* Gff, void* stream);

/*
 * w = AX(u) to FP64 accuracy computed on the FP32 pipes (the operator of
 * Section II-B, Listing 1, in float-float arithmetic).  Same arguments and
 * layouts as nek_ax except Gff (from nek_geom_ff); u, w 8-byte aligned, no
 * overlap.  Every value is carried as a pair of floats (~48 significant bits)
 * and every sum is formed with exact residual tracking; the result matches the
 * FP64 operator to ~1e-14 relative in the max norm.  Element blocks whose
 * largest |u| is below ~1e-30 (or contain non-finite values) are not covered by
 * that accuracy statement.  Async on stream.
 */
nek_status nek_ax_ff(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                     void* stream);

/* ------------------------------------------------------- gather-scatter ---
 * Direct stiffness summation over shared face, edge and corner nodes (the
 * nearest-neighbour exchange of Section II-B).  A plan groups every local node
 * whose global id is shared by two or more local nodes; groups are ordered by
 * ascending global id and members by ascending local index, and dssum replaces
 * each member by the left-to-right sum of its group in that order, so results
 * are bit-reproducible.
 *
 * nek_gs_create: glo_num_host is a HOST array of nelt*nx^3 non-negative global
 * ids (copied; the caller keeps ownership).  Synchronous.  *out receives a
 * handle owned by the caller, released with nek_gs_destroy.  Needs
 * nelt*nx^3 < 2^31.
 */
typedef struct nek_gs nek_gs;

nek_status nek_gs_create(int64_t nelt, int nx, const int64_t* glo_num_host, nek_gs** out);
nek_status nek_gs_destroy(nek_gs* gs);

/* Sizes of a plan: local points, groups, local points that belong to a group. */
nek_status nek_gs_info(const nek_gs* gs, int64_t* npts, int64_t* ngroups, int64_t* nshared);

/* Copy the plan's groups to HOST arrays: offsets (ngroups+1) and members
 * (nshared), both int64.  Synchronous. */
nek_status nek_gs_export(const nek_gs* gs, int64_t* offsets_host, int64_t* members_host);

/* v <- dssum(v) in place on an E-vector (device).  Async. */
nek_status nek_dssum(const nek_gs* gs, double* v, void* stream);

/* c[p] = 1 / multiplicity of the global node of p (device output, npts doubles). */
nek_status nek_gs_inv_multiplicity(const nek_gs* gs, double* c, void* stream);

/* ---------------------------------------------------------------- mask ---
 * v_p <- 0 where mask_p == 0 (homogeneous Dirichlet nodes; the paper's test case
 * is not specified, the box boundary is read as Dirichlet).  n points, device. */
nek_status nek_mask(int64_t n, const uint8_t* mask, double* v, void* stream);

/* ----------------------------------------------------- Jacobi / vectors ---
 * Jacobi preconditioner (the "simple preconditioner" of Section II-B read as
 * the inverse assembled diagonal): minv = mask ? 1/dssum(diag_e(A)) : 0.
 * All pointers device; async. */
nek_status nek_jacobi_minv(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                           const uint8_t* mask, double* minv, void* stream);

/* result[0] = sum_p c_p a_p b_p with c = 1/multiplicity (the global inner
 * product of two consistent fields; Section II-B's MPI_Allreduce becomes a
 * device reduction on one GPU).  a, b, result device; deterministic for a given
 * npts.  Uses library-owned scratch for per-block partial sums (allocated on the
 * first call for a plan and kept with it).  Async. */
nek_status nek_dot_c(const nek_gs* gs, const double* a, const double* b, double* result, void* stream);

/* Allocation-free form of nek_dot_c for callers that must not allocate device
 * memory, e.g. code running between the set-up and tear-down of a host
 * framework that owns every device allocation, or a control loop that may not
 * call cudaMalloc/cudaFree (they synchronise the device).  The paper has no
 * counterpart; it is an interface convenience.
 *   n: number of points, 0 <= n <= 2^31-1 (larger n returns NEK_ERR_TOO_LARGE);
 *   c: weights (e.g. nek_gs_inv_multiplicity), a, b: inputs, result: output
 *      (1 double) -- all device pointers owned by the caller.
 *   result[0] = sum_p c_p a_p b_p, computed by the same kernels and grid as
 *   nek_dot_c, so the two agree bit for bit on the same inputs.
 * The per-block partial sums live in a fixed 9.5 KB array inside the library
 * (held on every GPU that loads it until the process exits); nothing is
 * allocated or freed.  The first call on a device looks the array's device
 * address up (which can load the library's GPU module); make that first call
 * before any stream capture.  All calls on a device share the array: calls that
 * overlap on the GPU (different streams, no ordering) race and may return wrong
 * sums.  Async on stream.
 */
nek_status nek_dot_c_noalloc(int64_t n, const double* c, const double* a, const double* b, double* result,
                             void* stream);

/* ----------------------------------------------------------------- CG ---
 * Jacobi-preconditioned conjugate gradients on the masked, assembled operator
 * (Section II-B: vector operations, AX, nearest-neighbour exchange and global
 * reductions per iteration):
 *   b = mask.f, x = 0, r = b, z = Minv r, p = z;
 *   per iteration: w = mask(dssum(AX p)); alpha = <r,z>/<p,w>; x += alpha p;
 *   r -= alpha w; stop if ||r||/||b|| <= tol_rel; z = Minv r;
 *   beta = <r,z>new/<r,z>old; p = z + beta p.
 * Inner products are weighted by 1/multiplicity.
 *   gs, D, G, mask, f, x: as above (device); f is an E-vector (consistent or
 *     not; only its masked values are used); x is the output E-vector.
 *   minv: device Jacobi inverse diagonal, or NULL to build it internally.
 *   tol_rel > 0: stop at convergence, NEK_ERR_NOT_CONVERGED after max_iter;
 *   tol_rel == 0: run exactly max_iter iterations and return NEK_OK.
 *   workspace: device, >= nek_cg_workspace_bytes(...) bytes 256-aligned, or
 *     NULL to allocate (stream-ordered) and free inside the call.
 *   iters_out, relres_out: host, may be NULL.
 * Synchronizes the stream before returning (it reads the residual).  Returns
 * NEK_ERR_BREAKDOWN if p.Ap <= 0 or a scalar becomes non-finite.
 */
size_t nek_cg_workspace_bytes(int64_t nelt, int nx, int need_minv);

typedef enum {
    NEK_AX_FP64 = 0, /* nek_ax: native FP64 */
    NEK_AX_FF = 1    /* nek_ax_ff: FP64-accurate float-float on the FP32 pipes; needs Gff */
} nek_ax_impl;

typedef struct {
    int check_every;     /* residual read-back period in iterations (>=1; default 1) */
    int time_ax;         /* nonzero: record CUDA events around every AX launch */
    double ax_ms_total;  /* out: summed AX kernel time when time_ax */
    int ax_launches;     /* out: number of AX launches */
    int kernel_launches; /* out: kernels this call enqueued */
    int ax_impl;         /* nek_ax_impl; default NEK_AX_FP64 */
    const float* Gff;    /* device, from nek_geom_ff, required for NEK_AX_FF */
} nek_cg_opts;

nek_status nek_cg_solve(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                        const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                        int max_iter, void* workspace, int* iters_out, double* relres_out, void* stream);

/* Same as nek_cg_solve with options (opts may be NULL). */
nek_status nek_cg_solve_ex(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                           const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                           int max_iter, void* workspace, int* iters_out, double* relres_out, nek_cg_opts* opts,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NEKAX_H */
