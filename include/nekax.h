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
 *     G pointers must be 16-byte aligned, E-vectors and D 8-byte aligned
 *     (unless an entry point states otherwise);
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

/* Which AX operator a call uses. */
typedef enum {
    NEK_AX_FP64 = 0,      /* nek_ax: native FP64 */
    NEK_AX_FF = 1,        /* nek_ax_ff: FP64-accurate float-float on the FP32 pipes; needs Gff */
    NEK_AX_FF_ENERGY = 2, /* nek_ax_ff's element-energy form (nek_ax_ff_energy and the solves):
                             for nek_set_ax_epb / nek_get_ax_epb only */
    NEK_AX_OZ = 3         /* nek_ax_oz: FP64-accurate with the contractions on the tensor cores; needs
                             the split of nek_geom_oz; even nx up to 10 */
} nek_ax_impl;

/* Opaque gather-scatter plan (see nek_gs_create). */
typedef struct nek_gs nek_gs;

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

/*
 * nek_ax_ff plus the element energies edot[e] = u_e . w_e = u_e^T A_e u_e
 * (FP64 products and sums; each element's sum runs in an order fixed by nx
 * alone, so it does not depend on the tuned elements per CTA).  Summed over
 * elements this is the CG's <p, A p> (Section II-B's inner product of the
 * direction with the assembled operator applied to it) for a p that is
 * continuous across elements and zero on masked nodes; the FP64 solve with
 * NEK_AX_FF takes its <p,w> this way.  edot: device, nelt doubles, 8-byte
 * aligned, not overlapping u or w.  Async on stream.
 */
nek_status nek_ax_ff_energy(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                            double* edot, void* stream);

/*
 * Geometric factors split into float pairs for nek_ax_oz (device, async): the
 * values of nek_geom_ff with two adjacent points interleaved,
 * Goz[e][q][c] = (hi of G[e][2q][c], hi of G[e][2q+1][c], lo of G[e][2q][c],
 * lo of G[e][2q+1][c]) for c = 0..5 (48 bytes per point).  nx as nek_ax_oz;
 * G: device, 8-byte aligned; Goz: device, 16-byte aligned, must not overlap G.
 */
nek_status nek_geom_oz(int64_t nelt, int nx, const double* G, float* Goz, void* stream);

/*
 * w = AX(u) to FP64 accuracy with the contractions on the tensor cores
 * (tcgen05 BF16 MMAs, FP32 tensor-memory accumulators): the operator of
 * Section II-B, Listing 1.  Per element, u and then the pointwise products
 * G (ur, us, ut) are scaled to the element's largest magnitude and split into
 * six 8-bit BF16 digits each (D likewise); every digit product is summed
 * exactly, level by level, by the tensor cores, and the levels are recombined
 * into float pairs on the CUDA cores; the G product is float-float.  Layouts
 * as nek_ax except Goz (from nek_geom_oz); u and w device, 16-byte aligned, no
 * overlap; nx even and at most 10, else NEK_ERR_UNSUPPORTED_NX.  The result
 * matches the FP64 operator to ~1e-14 relative in the max norm of each element
 * (the error scales with the element's largest |u|: parts of an element far
 * below it keep less relative accuracy); the same range caveats as nek_ax_ff.
 * Every wait of the kernel on its tensor-core work is bounded (~2 s); one that
 * runs out leaves NaN in the outputs of the elements it had not finished (see
 * nek_ax_oz_selftest).  Async on stream.
 */
nek_status nek_ax_oz(int64_t nelt, int nx, const double* D, const float* Goz, const double* u, double* w,
                     void* stream);

/* Self-test of the bounded waits of nek_ax_oz's kernel: runs it on three nx = 4
 * elements (zero D, G and u, so w = 0) with every mbarrier wait bounded by
 * wait_us microseconds (1 .. 2e6).  force_timeout != 0 makes the mbarrier
 * expect one arrival more than the kernel's MMAs ever give, so every wait runs
 * out: the kernel must then set its flag, write NaN into its elements' outputs,
 * free its tensor memory and return.  *timed_out receives whether the flag was
 * set.  Returns NEK_ERR_TIMEOUT when it was (and the output was poisoned),
 * NEK_OK when the kernel finished normally, NEK_ERR_CUDA if the flag and the
 * output disagree.  No paper counterpart: failure detection of the library.
 * Allocates and synchronises the device; for tests. */
nek_status nek_ax_oz_selftest(int force_timeout, int64_t wait_us, int* timed_out);

/* ------------------------------------------------------------ tuning ---
 * The AX kernels group elements into CTAs; the group size (1, 2 or 4 elements
 * per CTA where threads and shared memory allow) changes only occupancy, never
 * the arithmetic, so results are bit-identical.  nek_tune_ax times each size on
 * the given data (synchronously; u, G/Gff, w as for nek_ax / nek_ax_ff with
 * impl = NEK_AX_FP64 / NEK_AX_FF, 16-byte aligned; the median of 7
 * individually timed launches) and keeps the fastest for all later launches of
 * that (impl, nx) in this process; *epb_out and *ms_out (nullable) receive it
 * and its time per launch.  For NEK_AX_FF the form with
 * element energies that nek_cg_solve_ex uses is tuned too (kept on its own,
 * not reported).  nek_set_ax_epb sets the size
 * directly (0 restores the built-in default; a size that does not fit the
 * kernel's thread or shared-memory limits for that nx is NEK_ERR_INVALID_ARG;
 * NEK_AX_FF sets both float-float forms, NEK_AX_FF_ENERGY the energy form
 * only); nek_get_ax_epb reads it back (0 = the built-in default).
 * These settings are process-wide.  No paper counterpart: the paper picks its
 * FPGA kernel count by hand (Section IV).
 */
nek_status nek_tune_ax(int impl, int64_t nelt, int nx, const double* D, const void* Gx, const double* u, double* w,
                       int* epb_out, float* ms_out, void* stream);
nek_status nek_set_ax_epb(int impl, int nx, int epb);
int nek_get_ax_epb(int impl, int nx);

/* ---------------------------------------------- reduced-precision AX ---
 * The paper's further work (Section V) names single and half precision for the
 * AX kernel.  These entry points run the operator with its contraction inputs
 * (u, D and the intermediate wr, ws, wt) rounded to FP32, BF16 or FP16 and FP32
 * accumulation; u and w are FP32 E-vectors.
 */
typedef enum { NEK_PREC_F32 = 0, NEK_PREC_BF16 = 1, NEK_PREC_F16 = 2 } nek_precision;

/* Bytes of one stored value of a precision (4, 2, 2), 0 for an unknown one. */
size_t nek_lowp_bytes_per_value(int precision);

/* G (FP64 [e][p][6]) -> Glp [e][p][6] in `precision` scaled per element by
 * gscale[e], a power of two >= max |G_e| (so |Glp| <= 1).  Glp: device,
 * nelt*nx^3*6 values, 4-byte aligned; gscale: device, nelt floats.  Async. */
nek_status nek_geom_lowp(int64_t nelt, int nx, int precision, const double* G, void* Glp, float* gscale,
                         void* stream);

/* w = AX(u) in reduced precision: u scaled per element by a power of two and
 * rounded, D rounded, FP32 sums, wr/ws/wt rounded before the transposed
 * contractions, output rescaled to FP32.  D: device FP64 (rounded in the
 * kernel); Glp, gscale from nek_geom_lowp; u, w: device FP32, no overlap.
 * Async. */
nek_status nek_ax_lowp(int64_t nelt, int nx, int precision, const double* D, const void* Glp, const float* gscale,
                       const float* u, float* w, void* stream);

/* Same operator with the D-contractions on the tensor cores (precision
 * NEK_PREC_BF16 or NEK_PREC_F16 only, else NEK_ERR_INVALID_ARG): each
 * contraction is a 16 x 16 x 16 product per plane of the element (nx padded
 * with zeros), mma.sync m16n8k16 with FP32 accumulation.  Same rounding points
 * and the same error bound as nek_ax_lowp; only the order of the FP32
 * additions inside a contraction differs.  Arguments as nek_ax_lowp. */
nek_status nek_ax_lowp_tc(int64_t nelt, int nx, int precision, const double* D, const void* Glp,
                          const float* gscale, const float* u, float* w, void* stream);

/* Same operator with the D-contractions on the 5th-generation tensor cores
 * (tcgen05 BF16 / FP16 MMAs, FP32 accumulators in tensor memory): per element,
 * each direction's contraction is one 128 x 16 x 16 product of the element's
 * lines (nx points padded to 16) with rnd(D).  precision NEK_PREC_BF16 or
 * NEK_PREC_F16 (else NEK_ERR_INVALID_ARG), nx 2..11 (else
 * NEK_ERR_UNSUPPORTED_NX).  Same rounding points and error bound as
 * nek_ax_lowp; only the order of the FP32 additions inside a contraction
 * differs.  Every wait on the tensor cores is bounded (~2 s); one that runs out
 * leaves NaN in the affected outputs.  Arguments as nek_ax_lowp. */
nek_status nek_ax_lowp_tc5(int64_t nelt, int nx, int precision, const double* D, const void* Glp,
                           const float* gscale, const float* u, float* w, void* stream);

/* Defect correction (iterative refinement) to FP64 accuracy: the residual
 * r = mask(f - dssum(AX x)), its norm, inner products and the update x += d are
 * FP64 on the GPU (AX through nek_ax_ff when Gff is given, else nek_ax); each
 * correction solves A d = r/||r|| by Jacobi-PCG with FP32 vectors and the
 * reduced-precision operator (nek_ax_lowp_tc5 for BF16 / FP16 at nx up to 11,
 * else nek_ax_lowp) until its relative residual is <= inner_tol (or max_inner
 * iterations); that operator also applies the inner solve's x / direction update
 * as it loads p, with the FP32 operations of the update (five kernels an inner
 * iteration).  Stops when ||r||_c/||b||_c <= tol_rel (NEK_OK) or after max_outer
 * corrections (NEK_ERR_NOT_CONVERGED).  workspace: device, >=
 * nek_cg_mixed_workspace_bytes(...) bytes, 256-aligned, or NULL.  Synchronous.
 */
typedef struct {
    int outer_iters;     /* corrections applied */
    int inner_iters;     /* inner PCG iterations, summed */
    double relres;       /* final ||r||_c / ||b||_c (FP64 residual) */
    int kernel_launches; /* kernels enqueued */
} nek_mixed_info;

size_t nek_cg_mixed_workspace_bytes(int64_t nelt, int nx, int need_minv);

nek_status nek_cg_solve_mixed(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                              const float* Gff, int precision, const void* Glp, const float* gscale,
                              const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                              double inner_tol, int max_outer, int max_inner, void* workspace,
                              nek_mixed_info* info, void* stream);

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

/* Residual of the masked, assembled system (the quantity Section II-B's CG
 * iteration drives to zero): r = mask.(f - dssum(AX x)), AX through nek_ax_ff
 * when Gff is given, else nek_ax with G.  f, x, r: device E-vectors, r must not
 * overlap f or x.  Async. */
nek_status nek_residual(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G, const float* Gff,
                        const uint8_t* mask, const double* f, const double* x, double* r, void* stream);

/* ----------------------------------------------------- Jacobi / vectors ---
 * Jacobi preconditioner (Section II-B's basic preconditioner, read as the
 * inverse assembled diagonal): minv = mask ? 1/dssum(diag_e(A)) : 0.
 * All pointers device; async. */
nek_status nek_jacobi_minv(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                           const uint8_t* mask, double* minv, void* stream);

/* result[0] = sum_p c_p a_p b_p with c = 1/multiplicity (the global inner
 * product of two consistent fields; Section II-B's MPI_Allreduce becomes a
 * device reduction on one GPU).  a, b, result device, 8-byte aligned;
 * deterministic for a given npts.  Uses library-owned scratch for per-block partial sums (allocated on the
 * first call for a plan and kept with it).  Async. */
nek_status nek_dot_c(const nek_gs* gs, const double* a, const double* b, double* result, void* stream);

/* Allocation-free form of nek_dot_c for callers that must not allocate device
 * memory, e.g. code running between the set-up and tear-down of a host
 * framework that owns every device allocation, or a control loop that may not
 * call cudaMalloc/cudaFree (they synchronise the device).  The paper has no
 * counterpart; it is an interface convenience.
 *   n: number of points, 0 <= n <= 2^31-1 (larger n returns NEK_ERR_TOO_LARGE);
 *   c: weights (e.g. nek_gs_inv_multiplicity), a, b: inputs, result: output
 *      (1 double) -- all device pointers owned by the caller, 8-byte aligned
 *      (else NEK_ERR_INVALID_ARG); n = 0 writes 0.
 *   result[0] = sum_p c_p a_p b_p, computed by the same kernels and grid as
 *   nek_dot_c, so the two agree bit for bit on the same inputs.
 * The per-block partial sums live in a fixed 9.5 KB array inside the library
 * (held on every GPU that loads it until the process exits); nothing is
 * allocated or freed.  The first call on a device looks the array's device
 * address up (which can load the library's GPU module); make that first call
 * before any stream capture.  The address is kept per device together with the
 * id of the context it belongs to; after cudaDeviceReset the next call is a
 * first call again.  All calls on a device share the array: calls that
 * overlap on the GPU (different streams, no ordering) race and may return wrong
 * sums.  Async on stream.
 */
nek_status nek_dot_c_noalloc(int64_t n, const double* c, const double* a, const double* b, double* result,
                             void* stream);

/* ---------------------------------------------------- batched solves ---
 * Many independent problems solved together by Jacobi-PCG (no paper
 * counterpart: the paper runs one mesh).  Problems are laid out back to back in
 * one E-vector space in the order given, which must be sorted by nx
 * (non-decreasing); problem q holds nelt[q]*nx[q]^3 points and its G block is
 * [nelt[q]][nx[q]^3][6] at the same offset (x6).  glo_num_host concatenates each
 * problem's own global ids (each starting anywhere >= 0; they are made disjoint
 * internally).  All points together must be < 2^31.  The handle owns the
 * gather-scatter plan over all problems, the reduction chunk table and one D per
 * distinct nx.  Synchronous.  Within an nx, ordering the problems by size
 * (smallest first) lets the solve stop launching the operator over the
 * problems that have finished (the small ones usually finish first).
 */
typedef struct nek_batch nek_batch;

typedef struct {
    int iterations_run;  /* iterations executed for the batch (max over problems) */
    int converged;       /* problems that met tol */
    int kernel_launches; /* kernels enqueued, counting those inside graph replays */
    int graph_launches;  /* CUDA graph replays */
} nek_batch_stats;

nek_status nek_batch_create(int nprob, const int64_t* nelt, const int* nx, const int64_t* glo_num_host,
                            nek_batch** out);
nek_status nek_batch_destroy(nek_batch* b);
nek_status nek_batch_info(const nek_batch* b, int64_t* npts, int* ngroups, int* nchunks);
/* The plan over all problems (owned by the batch), e.g. for nek_gs_inv_multiplicity. */
const nek_gs* nek_batch_gs(const nek_batch* b);
size_t nek_batch_workspace_bytes(const nek_batch* b, int need_minv);
/* Jacobi inverse diagonal of every problem (device, async). */
nek_status nek_batch_jacobi_minv(const nek_batch* b, const double* G, const uint8_t* mask, double* minv,
                                 void* stream);
/*
 * Jacobi-PCG on every problem at once, each with its own scalars and stopping
 * test (same iteration and rules as nek_cg_solve).  AX is nek_ax_ff when Gff
 * (the batch's G split by nek_geom_ff) is given, else nek_ax.  After one eager
 * iteration, iters_per_graph (> 0) iterations are captured into a CUDA graph
 * and replayed until every problem has stopped or max_iter is reached (0 = no
 * graph; < 0 = the rest of the solve as ONE graph launch: the iteration is the
 * body of a conditional WHILE node whose condition a kernel at the end of the
 * body sets on the device from the count of unfinished problems and the
 * iteration budget, so the host waits once, for the end of the solve).  iters_host, relres_host, status_host: HOST arrays of nprob entries,
 * nullable.  Returns NEK_OK if all problems converged (or tol_rel == 0),
 * NEK_ERR_NOT_CONVERGED / NEK_ERR_BREAKDOWN if any did not.  Synchronous.
 */
nek_status nek_batch_cg_solve(const nek_batch* b, const double* G, const float* Gff, const uint8_t* mask,
                              const double* minv, const double* f, double* x, double tol_rel, int max_iter,
                              int iters_per_graph, void* workspace, int* iters_host, double* relres_host,
                              int* status_host, nek_batch_stats* stats, void* stream);

/* ------------------------------------------- learned preconditioner ---
 * No counterpart in the paper (its solver uses Nekbone's fixed preconditioner).
 * A per-element network for nx = 8 element blocks (8^3 points): input channels
 * r/rms(r) and (Minv r)/rms(Minv r) of the element; three 3x3x3 convolutions
 * with zero padding inside the element, 16 hidden channels, GELU after the first
 * two; weights rounded to BF16, FP32 activations and accumulation.  Parameters
 * theta: nek_net_param_count() FP32 values, W1 [16][2][27], b1 [16],
 * W2 [16][16][27], b2 [16], W3 [1][16][27], b3 [1]; tap t = (dk+1)*9 + (dj+1)*3
 * + (di+1) reads point (i+di, j+dj, k+dk).  All pointers device; async unless
 * stated.
 */
int nek_net_param_count(void);

/* xin[e][0][p] = r/rms_e(r), xin[e][1][p] = (minv r)/rms_e(minv r) (0 where the
 * rms is 0); scale[e] = rms_e(minv r).  r, minv: FP64 E-vectors (nx = 8). */
nek_status nek_net_prep(int64_t nelt, int nx, const double* r, const double* minv, float* xin, float* scale,
                        void* stream);

/* Training target of the network for one (x_k, x*) pair of the solver: target[e][p] =
 * (xs - xk)[e][p] / scale[e] (the error in units of the element's rms(minv r), FP64
 * arithmetic, one FP32 rounding; 0 where scale[e] is 0).  xs, xk: FP64 E-vectors
 * (nx = 8); scale: from nek_net_prep; target: nelt*512 floats. */
nek_status nek_net_target(int64_t nelt, int nx, const double* xs, const double* xk, const float* scale,
                          float* target, void* stream);

/* z[e][p] = net(xin[e])[p] * scale[e] * c[e][p] (FP64 out; c = 1/multiplicity). */
nek_status nek_net_apply(int64_t nelt, int nx, const float* theta, const float* xin, const float* scale,
                         const double* c, double* z, void* stream);

/* Same as nek_net_apply on the 5th-generation tensor cores (tcgen05): each
 * 3x3x3 convolution is an implicit GEMM of 128 x 16 x 16 MMAs per tap with the
 * activations and weights in shared memory and the FP32 accumulators in tensor
 * memory.  The network input and the two hidden activations are rounded to BF16
 * (nearest even) before each convolution, products are exact and sums FP32.
 * Same arguments and errors; xin 4-byte, c and z 8-byte aligned.  A bounded wait
 * inside the kernel that runs out (about 2 s) writes NaN into its element's z and
 * sets a flag that nek_fcg_solve_trunc reports as NEK_ERR_TIMEOUT.
 * nek_fcg_solve(_trunc) uses this form. */
nek_status nek_net_apply_bf16(int64_t nelt, int nx, const float* theta, const float* xin, const float* scale,
                              const double* c, double* z, void* stream);

/* Self-test of the bounded waits of nek_net_apply_bf16's kernel: runs it on two
 * elements (zero weights and inputs, so z = 0) with every mbarrier wait bounded
 * by wait_us microseconds (1 .. 2e6).  force_timeout != 0 makes the mbarrier
 * expect one arrival more than the kernel's MMAs ever give, so every wait runs
 * out: the kernel must then set its flag, write NaN into its element's output,
 * free its tensor memory and return.  *timed_out receives whether the flag was
 * set.  Returns NEK_ERR_TIMEOUT when it was (and the output was poisoned),
 * NEK_OK when the kernel finished normally, NEK_ERR_CUDA if the flag and the
 * output disagree.  No paper counterpart: failure detection of the library.
 * Allocates and synchronises the device; for tests. */
nek_status nek_net_tc_selftest(int force_timeout, int64_t wait_us, int* timed_out);

/* The same network and rounding on the warp-level tensor-core MMA (mma.sync
 * m16n8k16, BF16 x BF16 -> FP32), kept for comparison with the tcgen05 form. */
nek_status nek_net_apply_bf16_mma(int64_t nelt, int nx, const float* theta, const float* xin, const float* scale,
                                  const double* c, double* z, void* stream);

/* Training on a batch of `batch` samples (xin [batch][2][512], target
 * [batch][512]): loss = mean_b |y_b - t_b|^2/|t_b|^2 (device float, nullable)
 * and its gradient (grad: NPARAM floats, summed over the batch in a fixed
 * order).  nek_net_forward_batch writes y [batch][512].  workspace: device,
 * >= nek_net_train_workspace_bytes(batch) bytes, 256-aligned. */
size_t nek_net_train_workspace_bytes(int batch);
nek_status nek_net_forward_batch(int batch, const float* theta, const float* xin, float* y, void* workspace,
                                 void* stream);
nek_status nek_net_train_grad(int batch, const float* theta, const float* xin, const float* target, float* grad,
                              float* loss, void* workspace, void* stream);

/* Same with the loss measured in each sample's element energy norm:
 * loss = mean_b (y_b - t_b)^T A_b (y_b - t_b) / t_b^T A_b t_b, where A_b is the
 * element operator of sample b given by its FP32 geometric factors Glp32
 * [batch][512][6] with per-sample scales gscale [batch] (nek_geom_lowp layout
 * with NEK_PREC_F32) and D (device FP64, nx = 8).  The norm ignores the
 * constants, which an element-local prediction cannot fix, and weights the
 * high-frequency error a local preconditioner must remove. */
nek_status nek_net_train_grad_energy(int batch, const float* theta, const float* xin, const float* target,
                                     const double* D, const float* Glp32, const float* gscale, float* grad,
                                     float* loss, void* workspace, void* stream);

/* One Adam step (Kingma & Ba) on n parameters; step >= 1 is the step count used
 * for bias correction. */
nek_status nek_adam_step(int n, float* theta, const float* grad, float* m, float* v, float lr, float beta1,
                         float beta2, float eps, int step, void* stream);

/*
 * Truncated flexible CG, FCG(m) (Notay 2000), preconditioned by the network,
 * M(r) = mask(dssum(nek_net_apply_bf16(r))): each new direction is z = M(r)
 * made A-orthogonal to the last m directions, alpha = <p, r>/<p, A p>.  The
 * network is not a fixed SPD operator, so the short recurrence of CG loses
 * orthogonality over long solves; the explicit window restores it (m = 1 is
 * flexible CG with the Polak-Ribiere-type coefficient).  Falls back to Jacobi
 * (emptying the window) when the relative residual has not fallen by
 * stag_factor (0 < stag_factor < 1) in the last stag_window iterations.  theta
 * NULL runs the same loop with Jacobi throughout (for a fixed SPD
 * preconditioner every m gives the PCG iterates in exact arithmetic).  AX is
 * nek_ax_ff when Gff is given, else nek_ax.  nx must be 8; 1 <= truncation
 * <= 16 (else NEK_ERR_INVALID_ARG).  workspace: device, >=
 * nek_fcg_trunc_workspace_bytes(...) bytes (it holds 2 (m + 1) E-vectors for
 * the directions and their images), 256-aligned, or NULL to allocate inside the
 * call.  Synchronous.  nek_fcg_solve is nek_fcg_solve_trunc with m = 1.
 */
typedef struct {
    int iters;            /* iterations run */
    double relres;        /* final ||r||_c/||b||_c */
    int fell_back_at;     /* iteration at which Jacobi took over (0 = never) */
    int net_applications; /* network preconditioner applications */
    double net_ms;        /* GPU time of those applications */
    int kernel_launches;
} nek_fcg_info;

size_t nek_fcg_workspace_bytes(int64_t nelt, int nx, int need_minv);
size_t nek_fcg_trunc_workspace_bytes(int64_t nelt, int nx, int need_minv, int truncation);
nek_status nek_fcg_solve_trunc(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                               const float* Gff, const uint8_t* mask, const double* minv, const float* theta,
                               const double* f, double* x, double tol_rel, int max_iter, int truncation,
                               int stag_window, double stag_factor, void* workspace, nek_fcg_info* info, void* stream);
nek_status nek_fcg_solve(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G, const float* Gff,
                         const uint8_t* mask, const double* minv, const float* theta, const double* f, double* x,
                         double tol_rel, int max_iter, int stag_window, double stag_factor, void* workspace,
                         nek_fcg_info* info, void* stream);

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

typedef struct {
    int check_every;     /* residual read-back period in iterations (>=1; default 1) */
    int time_ax;         /* nonzero: record CUDA events around every AX launch */
    double ax_ms_total;  /* out: summed AX kernel time when time_ax */
    int ax_launches;     /* out: number of AX launches */
    int kernel_launches; /* out: kernels this call enqueued */
    int ax_impl;         /* nek_ax_impl; default NEK_AX_FP64 */
    const float* Gff;    /* device, 16-byte aligned: from nek_geom_ff, required for NEK_AX_FF; from
                            nek_geom_oz, required for NEK_AX_OZ (which also needs minv, when given,
                            16-byte aligned) */
} nek_cg_opts;

nek_status nek_cg_solve(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                        const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                        int max_iter, void* workspace, int* iters_out, double* relres_out, void* stream);

/* Same as nek_cg_solve with options (opts may be NULL). */
nek_status nek_cg_solve_ex(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                           const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                           int max_iter, void* workspace, int* iters_out, double* relres_out, nek_cg_opts* opts,
                           void* stream);

/* Same solve with f and x in HOST memory (pinned or pageable), for callers
 * whose right-hand side and solution live on the host: f_host is copied to the
 * device, the solve of nek_cg_solve_ex runs, and x is copied back to x_host;
 * the call returns once x_host holds the result (also on NOT_CONVERGED and
 * BREAKDOWN, which leave the last iterate there).  The copies are part of the
 * call, one cudaMemcpyAsync each way on `stream`.
 *   f_host, x_host: host, nelt*nx^3 doubles each, E-vector layout.
 *   staging: device, >= nek_cg_host_staging_bytes(nelt, nx) bytes,
 *     256-aligned (device copies of f and x), or NULL to allocate
 *     (stream-ordered) and free inside the call.
 *   Every other argument as nek_cg_solve_ex.  Synchronous.
 */
size_t nek_cg_host_staging_bytes(int64_t nelt, int nx);

nek_status nek_cg_solve_host(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                             const uint8_t* mask, const double* minv, const double* f_host, double* x_host,
                             double tol_rel, int max_iter, void* workspace, void* staging, int* iters_out,
                             double* relres_out, nek_cg_opts* opts, void* stream);

/* ------------------------------------------------- unique-node vectors ---
 * The solve on unique-node ("L-") vectors: every global node is stored once,
 * ordered by ascending global id.  With Q the map from unique nodes to element
 * points (u_local[p] = u[l2g[p]]), the assembled operator of Section II-B's
 * AX plus nearest-neighbour exchange is w = Q^T AX Q u: AX gathers its input
 * through l2g (inside the kernel), and the copies of each node are summed in
 * ascending local index, the order of nek_dssum.  CG vectors then have the
 * unique length and inner products need no 1/multiplicity weight.
 *
 * nek_lvec_create: glo_num [npts] (host, >= 0) and mask [npts] (host; copies
 *   of a node must agree, else NEK_ERR_INVALID_ARG).  npts < 2^31
 *   (NEK_ERR_TOO_LARGE).  The plan owns its device arrays; free it with
 *   nek_lvec_destroy.  nek_lvec_size: unique nodes (-1 for NULL).
 * nek_lvec_scatter: uE = Q uL.  nek_lvec_restrict: uL[g] = uE at the first
 *   copy of g (the inverse of scatter on consistent E-vectors).
 *   nek_lvec_assemble: wL = Q^T wE.  All device, asynchronous, no aliasing.
 * nek_lvec_ax_ff: wL = Q^T AX Q uL with the FP64-accurate operator of
 *   nek_ax_ff (Gff from nek_geom_ff), unmasked; wE is caller-provided device
 *   scratch of npts doubles.
 * nek_lvec_jacobi_minv: minvL = 1 / diag(Q^T A Q), 0 on Dirichlet nodes;
 *   scratchE: npts doubles.
 * nek_lvec_cg_solve: Jacobi-PCG of nek_cg_solve on L-vectors (fL, xL, minvL
 *   of nek_lvec_size entries), AX as in nek_lvec_ax_ff.  opts (nullable):
 *   check_every, time_ax and the outputs; ax_impl and Gff in opts are ignored.
 *   workspace: >= nek_lvec_cg_workspace_bytes(lv) bytes, 256-aligned, or NULL.
 *   Same stopping rules, statuses and synchronisation as nek_cg_solve.
 */
typedef struct nek_lvec nek_lvec;

nek_status nek_lvec_create(int64_t npts, const int64_t* glo_num, const uint8_t* mask, nek_lvec** out);
nek_status nek_lvec_destroy(nek_lvec* lv);
int64_t nek_lvec_size(const nek_lvec* lv);
nek_status nek_lvec_scatter(const nek_lvec* lv, const double* uL, double* uE, void* stream);
nek_status nek_lvec_restrict(const nek_lvec* lv, const double* uE, double* uL, void* stream);
nek_status nek_lvec_assemble(const nek_lvec* lv, const double* wE, double* wL, void* stream);
nek_status nek_lvec_ax_ff(const nek_lvec* lv, int64_t nelt, int nx, const double* D, const float* Gff,
                          const double* uL, double* wL, double* wE, void* stream);
nek_status nek_lvec_jacobi_minv(const nek_lvec* lv, int64_t nelt, int nx, const double* D, const double* G,
                                double* minvL, double* scratchE, void* stream);
size_t nek_lvec_cg_workspace_bytes(const nek_lvec* lv);
nek_status nek_lvec_cg_solve(const nek_lvec* lv, int64_t nelt, int nx, const double* D, const float* Gff,
                             const double* minvL, const double* fL, double* xL, double tol_rel, int max_iter,
                             void* workspace, int* iters_out, double* relres_out, nek_cg_opts* opts, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NEKAX_H */
