// Reduced-precision AX and the FP64 defect-correction solve around it.
//
// The paper's further work (Section V of arXiv 2011.04981) names single, half
// and fixed-point precision for the AX kernel.  Here the operator's
// contractions take their inputs in FP32, BF16 or FP16 and accumulate in FP32:
//   u_q = rnd(u / s_u)          s_u = per-element power of two >= max|u|
//   D_q = rnd(D)
//   ur = D_q u_q etc.           FP32 sums of products of rounded inputs
//   [wr ws wt] = G_q [ur us ut] G_q = rnd(G / s_G), s_G per-element power of two
//   w  = s_u s_G sum_a D_q^T rnd(w_a)
// with rnd() rounding to the storage type (identity for FP32).  Products of two
// BF16/FP16 values are exact in FP32, so this is the arithmetic of a
// tensor-core contraction with FP32 accumulation.  u and w stay FP32; G is
// stored in the reduced type, 6 values per point plus one FP32 scale per
// element, so one apply moves 4 + 6 s + 4 bytes per point (32 B for FP32,
// 20 B for BF16/FP16).
//
// The solve is iterative refinement (defect correction): the residual
// r = mask(f - dssum(AX x)), its norm, the inner products and the update of x
// are FP64 on the GPU; each correction d solves A d = r / ||r|| approximately by
// Jacobi-PCG with FP32 vectors and the reduced-precision operator.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nek_internal.h"
#include "nek_pcg.cuh"

namespace nek {

namespace {

template <class S>
struct Lp;
template <>
struct Lp<float> {
    __device__ static __forceinline__ float rnd(float x) { return x; }
    __device__ static __forceinline__ float to_f(float v) { return v; }
    __device__ static __forceinline__ float from_f(float x) { return x; }
};
template <>
struct Lp<__nv_bfloat16> {
    __device__ static __forceinline__ float rnd(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
    __device__ static __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
    __device__ static __forceinline__ float bits_to_f(unsigned short h) { return __uint_as_float((unsigned)h << 16); }
};
template <>
struct Lp<__half> {
    __device__ static __forceinline__ float rnd(float x) { return __half2float(__float2half_rn(x)); }
    __device__ static __forceinline__ float to_f(__half v) { return __half2float(v); }
    __device__ static __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
    __device__ static __forceinline__ float bits_to_f(unsigned short h) { return __half2float(__ushort_as_half(h)); }
};

// slot[key] = max(slot[key], v) for v >= 0, one shared-memory atomic per key per warp.
__device__ __forceinline__ void segmented_max_to_smem(int key, float v, float* slot)
{
    // Lanes beyond a partial last warp do not exist, so only the active lanes are named.
    const unsigned same = __match_any_sync(__activemask(), key);
    const unsigned m = __reduce_max_sync(same, __float_as_uint(v));
    if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMax(reinterpret_cast<unsigned*>(slot + key), m);
}

// Smallest power of two >= m (m > 0), as a float; 1 for m == 0.
__device__ __forceinline__ float pow2_ceil(float m)
{
    if (!(m > 0.f)) return 1.f;
    int e;
    const float f = frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, f == 0.5f ? e - 1 : e);
}

constexpr int lp_epb(int nx)
{
    return nx == 2 ? 32 : nx == 3 ? 32 : nx == 4 ? 8 : nx == 5 ? 16 : nx == 6 ? 8 : nx == 7 ? 8 : nx == 8 ? 4
         : nx == 9 ? 4 : nx == 10 ? 4 : nx == 11 ? 2 : nx == 12 ? 2 : nx == 13 ? 2 : 1;
}

// D rows padded to a multiple of 4 floats so a row is read with 16-byte broadcast loads.
constexpr int lp_row(int nx) { return (nx + 3) & ~3; }

template <int NX, int EPB>
constexpr size_t lp_smem_bytes()
{
    // rnd(D) and rnd(D)^T (padded rows), three [EPB][N3] float blocks, per-element maxima
    return sizeof(float) * (size_t)(2 * NX * lp_row(NX) + 3 * EPB * NX * NX * NX + EPB + 4);
}

// Six G values of point p as floats (3 paired loads where alignment allows).
template <class S>
struct GLoad;
template <>
struct GLoad<float> {
    __device__ static __forceinline__ void get(const float* __restrict__ g, bool al8, float* v)
    {
        if (al8) {
            const float2* g2 = reinterpret_cast<const float2*>(g);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const float2 t = __ldg(g2 + q);
                v[2 * q] = t.x;
                v[2 * q + 1] = t.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 6; q++) v[q] = __ldg(g + q);
        }
    }
};
template <class H>
struct GLoad16 {
    // 6 values of 2 bytes at a 4-byte aligned address (12 p bytes from a 4-byte aligned base)
    __device__ static __forceinline__ void get(const H* __restrict__ g, bool, float* v)
    {
        const unsigned* g4 = reinterpret_cast<const unsigned*>(g);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const unsigned t = __ldg(g4 + q);
            v[2 * q] = Lp<H>::bits_to_f(static_cast<unsigned short>(t & 0xffffu));
            v[2 * q + 1] = Lp<H>::bits_to_f(static_cast<unsigned short>(t >> 16));
        }
    }
};
template <>
struct GLoad<__nv_bfloat16> : GLoad16<__nv_bfloat16> {
};
template <>
struct GLoad<__half> : GLoad16<__half> {
};

// out[o] = sum_l M[o][l] x[l], l ascending (one FP32 FMA chain per output); M rows
// are read as 16-byte broadcasts from shared memory (every lane reads the same row).
template <int NX>
__device__ __forceinline__ void line_apply(const float* __restrict__ M, const float (&x)[NX], float (&out)[NX])
{
    constexpr int R = lp_row(NX);
#pragma unroll
    for (int o = 0; o < NX; o++) {
        // Load each row of M just before its use: hoisted ahead (within or across
        // calls), the nx^2 values of M would crowd the lines out of registers.
        asm volatile("" ::: "memory");
        float acc = 0.f;
#pragma unroll
        for (int l4 = 0; l4 < R / 4; l4++) {
            const float4 m = reinterpret_cast<const float4*>(M + o * R)[l4];
            const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (4 * l4 + c < NX) acc = fmaf(mv[c], x[4 * l4 + c], acc);
        }
        out[o] = acc;
    }
}

// Line-pass form: every contraction is done by a thread that holds one whole
// line of nx values in registers and produces the nx results of that line
// (nx^2 FMAs per nx shared-memory reads).  Thread (a, b) of an element owns the
// r-line (j, k) = (a, b), the s-line (i, k) = (a, b) and the t-line
// (i, j) = (a, b).  Phase 1 writes ur and us to shared memory and keeps ut in
// registers; the pointwise G product runs on the t-lines; phase 2 sums the
// r- and s-contributions through shared memory and adds the t-contribution in
// registers before the store.
// MODE kLowpEnergy: edot[e] = sum over the element's points of u w (each
// thread's nx terms summed in FP32, the element's threads in FP64), which the
// inner solve uses for <p,w> (see nek_pcg.cuh).  MODE kLowpDir: the same, and
// the inner solve's x / direction update (DirUpdateF) is applied as the
// element's input is loaded: x += alpha p, p = minv r + beta p with that
// solve's own FP32 operations, and the operator is applied to the new p.
constexpr int kLowpPlain = 0, kLowpEnergy = 1, kLowpDir = 2;
template <class S, int NX, int EPB, int MODE>
__global__ void __launch_bounds__(NX* NX* EPB) k_ax_lowp(int64_t nelt, const double* __restrict__ D,
                                                          const S* __restrict__ Glp,
                                                          const float* __restrict__ gscale,
                                                          const float* __restrict__ u, float* __restrict__ w,
                                                          double* __restrict__ edot, DirUpdateF dir)
{
    using L = Lp<S>;
    constexpr int N2 = NX * NX, N3 = NX * NX * NX, NT = N2 * EPB, R = lp_row(NX);
    extern __shared__ __align__(16) float fsm[];
    float* sD = fsm;                 // [NX][R]  rnd(D)[o][l]
    float* sDT = sD + NX * R;        // [NX][R]  rnd(D)[l][o] at o*R + l
    float* sU = sDT + NX * R;        // [EPB][N3] u_q, later the r+s part of w
    float* sR = sU + EPB * N3;       // [EPB][N3] ur, then wr
    float* sS = sR + EPB * N3;       // [EPB][N3] us, then ws
    float* sMax = sS + EPB * N3;     // [EPB]

    const int tid = threadIdx.x;
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int ne = static_cast<int>(nelt - e0 < EPB ? nelt - e0 : EPB);

    for (int q = tid; q < NX * R; q += NT) {
        const int o = q / R, l = q - o * R;
        sD[q] = l < NX ? L::rnd((float)D[o * NX + l]) : 0.f;
        sDT[q] = l < NX ? L::rnd((float)D[l * NX + o]) : 0.f;
    }
    for (int q = tid; q < EPB; q += NT) sMax[q] = 0.f;
    if constexpr (MODE == kLowpDir) {
        const bool dx = dir.sc->xpend != 0, dp = !(dir.sc->done || dir.sc->status != NEK_OK);
        const float alpha = (float)dir.sc->alpha, beta = (float)dir.sc->beta;
        float* pb = dir.p + e0 * N3;
        float* xb = dir.x + e0 * N3;
        const float* rb = dir.r + e0 * N3;
        const float* mb = dir.minv + e0 * N3;
        const int nq = ne * N3;
        constexpr int KB = 4;  // points per batch: a batch's loads are issued before its stores
        for (int q0 = tid; q0 < nq; q0 += KB * NT) {
            float po[KB], rv[KB], mv[KB], xv[KB];
#pragma unroll
            for (int k = 0; k < KB; k++) {
                const int q = q0 + k * NT < nq ? q0 + k * NT : q0;
                po[k] = pb[q];
                rv[k] = __ldg(rb + q);
                mv[k] = __ldg(mb + q);
                xv[k] = dx ? xb[q] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < KB; k++) {
                const int q = q0 + k * NT;
                if (q < nq) {
                    if (dx) xb[q] = fmaf(alpha, po[k], xv[k]);
                    float v = po[k];
                    if (dp) {
                        v = fmaf(beta, po[k], mv[k] * rv[k]);
                        pb[q] = v;
                    }
                    sU[q] = v;
                }
            }
        }
    } else {
        const float* src = u + e0 * N3;
        for (int q = tid; q < ne * N3; q += NT) sU[q] = __ldg(src + q);
    }
    __syncthreads();

    const int el = tid / N2;
    const int q2 = tid - el * N2;
    const int a = q2 % NX, b = q2 / NX;
    const bool active = el < ne;
    float* ue = sU + el * N3;
    float* re = sR + el * N3;
    float* se = sS + el * N3;
    {
        float m = 0.f;
        if (active) {
#pragma unroll
            for (int l = 0; l < NX; l++) m = fmaxf(m, fabsf(ue[l * N2 + b * NX + a]));
        }
        segmented_max_to_smem(el, m, sMax);
    }
    __syncthreads();
    const float su = pow2_ceil(sMax[el]);
    {
        const float inv = 1.f / su;  // a power of two: exact
        if (active) {
#pragma unroll
            for (int l = 0; l < NX; l++) {
                const int p = l * N2 + b * NX + a;
                ue[p] = L::rnd(ue[p] * inv);
            }
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- phase 1
    float ut[NX];
    if (active) {
        float x[NX], y[NX];
#pragma unroll
        for (int l = 0; l < NX; l++) x[l] = ue[b * N2 + a * NX + l];  // r-line (j,k) = (a,b)
        line_apply<NX>(sD, x, y);
#pragma unroll
        for (int o = 0; o < NX; o++) re[b * N2 + a * NX + o] = y[o];
#pragma unroll
        for (int l = 0; l < NX; l++) x[l] = ue[b * N2 + l * NX + a];  // s-line (i,k) = (a,b)
        line_apply<NX>(sD, x, y);
#pragma unroll
        for (int o = 0; o < NX; o++) se[b * N2 + o * NX + a] = y[o];
#pragma unroll
        for (int l = 0; l < NX; l++) x[l] = ue[l * N2 + b * NX + a];  // t-line (i,j) = (a,b)
        line_apply<NX>(sD, x, ut);
    }
    __syncthreads();

    // ---------------------------------------------------------------- G product on the t-lines
    float wt[NX];
    if (active) {
        const S* Ge = Glp + (e0 + el) * (int64_t)N3 * 6;
        const bool al8 = (reinterpret_cast<uintptr_t>(Glp) & 7) == 0;
#pragma unroll
        for (int k = 0; k < NX; k++) {
            const int p = k * N2 + b * NX + a;
            const float ar = re[p], as = se[p], at = ut[k];
            float g[6];
            GLoad<S>::get(Ge + 6 * p, al8, g);
            re[p] = L::rnd(fmaf(g[0], ar, fmaf(g[1], as, g[2] * at)));
            se[p] = L::rnd(fmaf(g[1], ar, fmaf(g[3], as, g[4] * at)));
            wt[k] = L::rnd(fmaf(g[2], ar, fmaf(g[4], as, g[5] * at)));
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- phase 2
    float os[NX];
    if (active) {
        float x[NX], y[NX];
#pragma unroll
        for (int l = 0; l < NX; l++) x[l] = re[b * N2 + a * NX + l];  // r-line of wr
        line_apply<NX>(sDT, x, y);
#pragma unroll
        for (int o = 0; o < NX; o++) ue[b * N2 + a * NX + o] = y[o];  // u is dead: reuse for w
#pragma unroll
        for (int l = 0; l < NX; l++) x[l] = se[b * N2 + l * NX + a];  // s-line of ws
        line_apply<NX>(sDT, x, os);
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int o = 0; o < NX; o++) ue[b * N2 + o * NX + a] += os[o];
    }
    __syncthreads();
    float energy = 0.f;  // this thread's nx terms u w in FP32, then FP64 across the element
    if (active) {
        float ot[NX];
        line_apply<NX>(sDT, wt, ot);
        const float scale = su * gscale[e0 + el];
        float* we = w + (e0 + el) * (int64_t)N3;
        const float* ug = u + (e0 + el) * (int64_t)N3;
        // with the direction update: the p written above
        const float* pg = MODE == kLowpDir ? dir.p + (e0 + el) * (int64_t)N3 : nullptr;
#pragma unroll
        for (int k = 0; k < NX; k++) {
            const int p = k * N2 + b * NX + a;
            const float wv = (ue[p] + ot[k]) * scale;
            we[p] = wv;
            // (written by another thread of the block before the barriers above: a plain load)
            if constexpr (MODE == kLowpDir) energy = fmaf(pg[p], wv, energy);
            if constexpr (MODE == kLowpEnergy) energy = fmaf(__ldg(ug + p), wv, energy);
        }
    }
    if constexpr (MODE != kLowpPlain)
        element_sums<N2, EPB>(pcg::to_f64(energy), reinterpret_cast<double*>(sR), edot + e0, ne);
}

template <class S, int NX, int MODE>
nek_status launch_lowp_kernel(int64_t nelt, const double* D, const void* Glp, const float* gscale, const float* u,
                              float* w, double* edot, const DirUpdateF& dir, cudaStream_t s)
{
    constexpr int EPB = lp_epb(NX);
    constexpr size_t smem = lp_smem_bytes<NX, EPB>();
    static std::atomic<uint64_t> configured{0};
    nek_status st = ensure_dyn_smem(k_ax_lowp<S, NX, EPB, MODE>, smem, configured);
    if (st != NEK_OK) return st;
    const int64_t blocks = (nelt + EPB - 1) / EPB;
    if (blocks > 0x7fffffff) return NEK_ERR_TOO_LARGE;
    k_ax_lowp<S, NX, EPB, MODE><<<(unsigned)blocks, NX * NX * EPB, smem, s>>>(
        nelt, D, static_cast<const S*>(Glp), gscale, u, w, edot, dir);
    return check_launch();
}

template <class S, int NX>
nek_status launch_lowp_nx(int64_t nelt, const double* D, const void* Glp, const float* gscale, const float* u,
                          float* w, double* edot, const DirUpdateF* dir, cudaStream_t s)
{
    const DirUpdateF none{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (edot && dir) return launch_lowp_kernel<S, NX, kLowpDir>(nelt, D, Glp, gscale, u, w, edot, *dir, s);
    return edot ? launch_lowp_kernel<S, NX, kLowpEnergy>(nelt, D, Glp, gscale, u, w, edot, none, s)
                : launch_lowp_kernel<S, NX, kLowpPlain>(nelt, D, Glp, gscale, u, w, nullptr, none, s);
}

template <class S>
nek_status launch_lowp_t(int64_t nelt, int nx, const double* D, const void* Glp, const float* gscale,
                         const float* u, float* w, double* edot, const DirUpdateF* dir, cudaStream_t s)
{
    switch (nx) {
        case 2: return launch_lowp_nx<S, 2>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 3: return launch_lowp_nx<S, 3>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 4: return launch_lowp_nx<S, 4>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 5: return launch_lowp_nx<S, 5>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 6: return launch_lowp_nx<S, 6>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 7: return launch_lowp_nx<S, 7>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 8: return launch_lowp_nx<S, 8>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 9: return launch_lowp_nx<S, 9>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 10: return launch_lowp_nx<S, 10>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 11: return launch_lowp_nx<S, 11>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 12: return launch_lowp_nx<S, 12>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 13: return launch_lowp_nx<S, 13>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 14: return launch_lowp_nx<S, 14>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 15: return launch_lowp_nx<S, 15>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 16: return launch_lowp_nx<S, 16>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
}

}  // namespace

nek_status launch_ax_lowp_tc(int prec, int64_t nelt, int nx, const double* D, const void* Glp, const float* gscale,
                             const float* u, float* w, cudaStream_t s);

nek_status launch_ax_lowp(int prec, int64_t nelt, int nx, const double* D, const void* Glp, const float* gscale,
                          const float* u, float* w, cudaStream_t s, double* edot, const DirUpdateF* dir)
{
    switch (prec) {
        case NEK_PREC_F32: return launch_lowp_t<float>(nelt, nx, D, Glp, gscale, u, w, edot, dir, s);
        case NEK_PREC_BF16: return launch_lowp_t<__nv_bfloat16>(nelt, nx, D, Glp, gscale, u, w, edot, dir, s);
        case NEK_PREC_F16: return launch_lowp_t<__half>(nelt, nx, D, Glp, gscale, u, w, edot, dir, s);
        default: return NEK_ERR_INVALID_ARG;
    }
}

namespace {

// One block per element: s_G = pow2_ceil(max |G_e|); Glp = rnd(G / s_G).
template <class S>
__global__ void k_geom_lowp(int64_t nelt, int n6, const double* __restrict__ G, S* __restrict__ Glp,
                            float* __restrict__ gscale)
{
    __shared__ float smax;
    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        if (threadIdx.x == 0) smax = 0.f;
        __syncthreads();
        float m = 0.f;
        for (int q = threadIdx.x; q < n6; q += blockDim.x) m = fmaxf(m, fabsf((float)G[e * n6 + q]));
        atomicMax(reinterpret_cast<int*>(&smax), __float_as_int(m));
        __syncthreads();
        const float sc = pow2_ceil(smax);
        for (int q = threadIdx.x; q < n6; q += blockDim.x) Glp[e * n6 + q] = Lp<S>::from_f((float)(G[e * n6 + q] / sc));
        if (threadIdx.x == 0) gscale[e] = sc;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- defect correction
struct MixScalars {
    double bnorm, rnorm, relres;
};

constexpr int NT = kReduceThreads;

// x = 0; r = mask.f; partials of <r,r>_c
__global__ void __launch_bounds__(NT) k_mix_init(int64_t n, const double* __restrict__ c,
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

// r = mask.(f - w); partials of <r,r>_c
__global__ void __launch_bounds__(NT) k_mix_residual(int64_t n, const double* __restrict__ c,
                                                      const uint8_t* __restrict__ mask, const double* __restrict__ f,
                                                      const double* __restrict__ w, double* __restrict__ r,
                                                      double* __restrict__ parts)
{
    __shared__ double sh[NT / 32];
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        const double rq = mask[q] ? f[q] - w[q] : 0.0;
        r[q] = rq;
        acc += c[q] * rq * rq;
    }
    const double t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_mix_norm(const double* __restrict__ parts, int nb, int first,
                                                  MixScalars* ms)
{
    __shared__ double sh[NT / 32];
    const double rr = sum_partials<NT>(parts, nb, sh);
    if (threadIdx.x == 0) {
        ms->rnorm = sqrt(rr);
        if (first) ms->bnorm = ms->rnorm;
        ms->relres = ms->bnorm > 0.0 ? ms->rnorm / ms->bnorm : 0.0;
    }
}

// r32 = r / ||r||
__global__ void k_mix_scale_down(int64_t n, const double* __restrict__ r, float* __restrict__ r32,
                                 const MixScalars* __restrict__ ms)
{
    const double inv = ms->rnorm > 0.0 ? 1.0 / ms->rnorm : 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        r32[q] = (float)(r[q] * inv);
}

// x += ||r|| d
__global__ void k_mix_update_x(int64_t n, const float* __restrict__ d, double* __restrict__ x,
                               const MixScalars* __restrict__ ms)
{
    const double s = ms->rnorm;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        x[q] = fma(s, (double)d[q], x[q]);
}

__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        b[q] = (float)a[q];
}

struct MixLayout {
    double *r, *w, *minv64;
    float *d, *minv, *c;
    uint8_t* flags;  // owner / free byte per point for the inner solve's inner products
    pcg::Buffers<float> b;
    double* edot;  // element energies of the inner operator (its <p,w>)
    double* parts;
    MixScalars* ms;
    size_t bytes;
};

MixLayout mix_layout(void* base_, int64_t nelt, int64_t n, bool need_minv)
{
    using pcg::align256;
    MixLayout L{};
    char* base = static_cast<char*>(base_);
    const size_t v8 = align256(sizeof(double) * std::max<int64_t>(n, 1));
    const size_t v4 = align256(sizeof(float) * std::max<int64_t>(n, 1));
    size_t off = 0;
    auto take = [&](size_t b) {
        char* p = base ? base + off : nullptr;
        off += b;
        return p;
    };
    L.r = reinterpret_cast<double*>(take(v8));
    L.w = reinterpret_cast<double*>(take(v8));
    L.minv64 = need_minv ? reinterpret_cast<double*>(take(v8)) : nullptr;
    L.d = reinterpret_cast<float*>(take(v4));
    L.minv = reinterpret_cast<float*>(take(v4));
    L.c = reinterpret_cast<float*>(take(v4));
    L.flags = reinterpret_cast<uint8_t*>(take(align256(std::max<int64_t>(n, 1))));
    L.b.r = reinterpret_cast<float*>(take(v4));
    L.b.p = reinterpret_cast<float*>(take(v4));
    L.b.w = reinterpret_cast<float*>(take(v4));
    L.b.parts = reinterpret_cast<double*>(take(align256(sizeof(double) * 2 * kMaxReduceBlocks)));
    L.b.sc = reinterpret_cast<pcg::Scalars*>(take(align256(sizeof(pcg::Scalars))));
    L.edot = reinterpret_cast<double*>(take(align256(sizeof(double) * std::max<int64_t>(nelt, 1))));
    L.parts = reinterpret_cast<double*>(take(align256(sizeof(double) * kMaxReduceBlocks)));
    L.ms = reinterpret_cast<MixScalars*>(take(align256(sizeof(MixScalars))));
    L.bytes = off;
    return L;
}

}  // namespace

}  // namespace nek

using namespace nek;

extern "C" {

size_t nek_lowp_bytes_per_value(int precision)
{
    return precision == NEK_PREC_F32 ? 4 : (precision == NEK_PREC_BF16 || precision == NEK_PREC_F16) ? 2 : 0;
}

nek_status nek_geom_lowp(int64_t nelt, int nx, int precision, const double* G, void* Glp, float* gscale,
                         void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0 || nek_lowp_bytes_per_value(precision) == 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!G || !Glp || !gscale || !is_aligned(G, 8) || !is_aligned(Glp, 4) || !is_aligned(gscale, 4))
        return NEK_ERR_INVALID_ARG;
    const int n6 = 6 * nx * nx * nx;
    const int blocks = static_cast<int>(nelt < 152 * 16 ? nelt : 152 * 16);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (precision) {
        case NEK_PREC_F32: k_geom_lowp<float><<<blocks, 256, 0, s>>>(nelt, n6, G, static_cast<float*>(Glp), gscale); break;
        case NEK_PREC_BF16:
            k_geom_lowp<__nv_bfloat16><<<blocks, 256, 0, s>>>(nelt, n6, G, static_cast<__nv_bfloat16*>(Glp), gscale);
            break;
        default: k_geom_lowp<__half><<<blocks, 256, 0, s>>>(nelt, n6, G, static_cast<__half*>(Glp), gscale); break;
    }
    return check_launch();
}

nek_status nek_ax_lowp_tc(int64_t nelt, int nx, int precision, const double* D, const void* Glp,
                          const float* gscale, const float* u, float* w, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0 || (precision != NEK_PREC_BF16 && precision != NEK_PREC_F16)) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Glp || !gscale || !u || !w) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(D, 8) || !is_aligned(Glp, 4) || !is_aligned(u, 4) || !is_aligned(w, 4)) return NEK_ERR_INVALID_ARG;
    const size_t bytes = sizeof(float) * (size_t)nelt * nx * nx * nx;
    if (ranges_overlap(u, bytes, w, bytes)) return NEK_ERR_INVALID_ARG;
    return launch_ax_lowp_tc(precision, nelt, nx, D, Glp, gscale, u, w, static_cast<cudaStream_t>(stream));
}

nek_status nek_ax_lowp(int64_t nelt, int nx, int precision, const double* D, const void* Glp, const float* gscale,
                       const float* u, float* w, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0 || nek_lowp_bytes_per_value(precision) == 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Glp || !gscale || !u || !w) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(D, 8) || !is_aligned(Glp, 4) || !is_aligned(u, 4) || !is_aligned(w, 4)) return NEK_ERR_INVALID_ARG;
    const size_t bytes = sizeof(float) * (size_t)nelt * nx * nx * nx;
    if (ranges_overlap(u, bytes, w, bytes)) return NEK_ERR_INVALID_ARG;
    return launch_ax_lowp(precision, nelt, nx, D, Glp, gscale, u, w, static_cast<cudaStream_t>(stream));
}

size_t nek_cg_mixed_workspace_bytes(int64_t nelt, int nx, int need_minv)
{
    if (nelt < 0 || nx < kMinNx || nx > kMaxNx) return 0;
    return mix_layout(nullptr, nelt, nelt * (int64_t)nx * nx * nx, need_minv != 0).bytes;
}

nek_status nek_cg_solve_mixed(const nek_gs* gs, int64_t nelt, int nx, const double* D, const double* G,
                              const float* Gff, int precision, const void* Glp, const float* gscale,
                              const uint8_t* mask, const double* minv, const double* f, double* x, double tol_rel,
                              double inner_tol, int max_outer, int max_inner, void* workspace,
                              nek_mixed_info* info, void* stream)
{
    if (info) *info = nek_mixed_info{};
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!gs || nelt < 0 || max_outer < 0 || max_inner < 1 || !(tol_rel > 0.0) || !(inner_tol > 0.0) ||
        !(inner_tol < 1.0) || nek_lowp_bytes_per_value(precision) == 0)
        return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * (int64_t)nx * nx * nx;
    if (gs->npts != n) return NEK_ERR_INVALID_ARG;
    if (n == 0) return NEK_OK;
    if (!D || !G || !Glp || !gscale || !mask || !f || !x) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(G, 16) || !is_aligned(f, 8) || !is_aligned(x, 16) || (Gff && !is_aligned(Gff, 16)) ||
        (minv && !is_aligned(minv, 8)) || !is_aligned(Glp, 4))
        return NEK_ERR_INVALID_ARG;
    if (workspace && !is_aligned(workspace, 256)) return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = nek_cg_mixed_workspace_bytes(nelt, nx, minv == nullptr);
    void* ws = workspace;
    nek_status st = NEK_OK;
    if (!ws) {
        if (check_cuda(cudaMallocAsync(&ws, bytes, s)) != NEK_OK) return NEK_ERR_NOMEM;
    }
    MixLayout L = mix_layout(ws, nelt, n, minv == nullptr);
    const double* mv = minv;
    const int nb = reduce_blocks(n);
    const int sb = pcg::stream_blocks(n);
    MixScalars h{};
    int outer = 0, inner_total = 0, launches = 0;
    auto ax64 = [&](const double* p, double* w) {
        return Gff ? launch_ax_ff(nelt, nx, D, Gff, p, w, s) : launch_ax_fp64(nelt, nx, D, G, p, w, s);
    };
    // the inner operator: the tcgen05 form where it applies (BF16 / FP16, nx up to 11), else the CUDA-core one
    const bool tc5 = ax_lowp_tc5_supported(nx, precision);
    // (both take the inner solve's x / direction update)
    auto ax_lo = [&](const float* p, float* w, double* ed, const DirUpdateF* dir, cudaStream_t ss) {
        return tc5 ? launch_ax_lowp_tc5(precision, nelt, nx, D, Glp, gscale, p, w, ss, ed, dir)
                   : launch_ax_lowp(precision, nelt, nx, D, Glp, gscale, p, w, ss, ed, dir);
    };

    if (!minv) {
        if ((st = nek_jacobi_minv(gs, nelt, nx, D, G, mask, L.minv64, stream)) != NEK_OK) goto done;
        mv = L.minv64;
        launches += 3;
    }
    k_d2f<<<sb, 256, 0, s>>>(n, mv, L.minv);
    k_d2f<<<sb, 256, 0, s>>>(n, gs->d_c, L.c);
    if ((st = pcg::build_flags(gs, n, mask, L.flags, s)) != NEK_OK) goto done;
    launches += gs->ngroups > 0 ? 2 : 1;
    k_mix_init<<<nb, NT, 0, s>>>(n, gs->d_c, mask, f, x, L.r, L.parts);
    k_mix_norm<<<1, NT, 0, s>>>(L.parts, nb, 1, L.ms);
    launches += 4;
    if ((st = check_launch()) != NEK_OK) goto done;
    for (;;) {
        if ((st = check_cuda(cudaMemcpyAsync(&h, L.ms, sizeof(h), cudaMemcpyDeviceToHost, s))) != NEK_OK) goto done;
        if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
        if (!std::isfinite(h.relres)) {
            st = NEK_ERR_BREAKDOWN;
            goto done;
        }
        if (h.relres <= tol_rel || h.bnorm == 0.0) break;
        if (outer >= max_outer) {
            st = NEK_ERR_NOT_CONVERGED;
            goto done;
        }
        outer++;
        // the inner right-hand side goes to b.w: pcg::run reads it once, at initialisation
        k_mix_scale_down<<<sb, 256, 0, s>>>(n, L.r, L.b.w, L.ms);
        launches += 1;
        {
            pcg::Result res;
            const pcg::ElementEnergies ee{L.edot, nelt, true};  // the operator's energies give <p,w>
            nek_status si = pcg::run<float>(gs, n, L.c, mask, L.minv, L.b.w, L.d, L.b, inner_tol, max_inner, 10,
                                           false, ax_lo, s, &res, L.flags, &ee);
            inner_total += res.iters;
            launches += res.launches;
            if (si == NEK_ERR_BREAKDOWN || si == NEK_ERR_CUDA) {
                st = si;
                goto done;
            }
        }
        k_mix_update_x<<<sb, 256, 0, s>>>(n, L.d, x, L.ms);
        if ((st = ax64(x, L.w)) != NEK_OK) goto done;
        if ((st = pcg::dssum<double>(gs, L.w, s)) != NEK_OK) goto done;
        k_mix_residual<<<nb, NT, 0, s>>>(n, gs->d_c, mask, f, L.w, L.r, L.parts);
        k_mix_norm<<<1, NT, 0, s>>>(L.parts, nb, 0, L.ms);
        launches += 5;
        if ((st = check_launch()) != NEK_OK) goto done;
    }
done:
    if (info) {
        info->outer_iters = outer;
        info->inner_iters = inner_total;
        info->relres = h.relres;
        info->kernel_launches = launches;
    }
    if (!workspace) {
        cudaFreeAsync(ws, s);
        nek_status st2 = check_cuda(cudaStreamSynchronize(s));
        if (st == NEK_OK) st = st2;
    }
    return st;
}

}  // extern "C"
