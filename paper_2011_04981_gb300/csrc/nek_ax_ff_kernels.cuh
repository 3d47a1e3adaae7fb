// AX operator to FP64 accuracy on the FP32 pipes (float-float arithmetic).
//
// Same operator as nek_ax (Section II-B, Listing 1 of arXiv 2011.04981).  On
// GB300 the FP64 pipe runs 2 DFMA/clk/SM against 128 FFMA/clk/SM, so native
// FP64 AX is bound by the FP64 pipe at ~8% of the HBM roofline.  This kernel
// keeps every value as an unevaluated pair hi + lo of floats (about 48
// significant bits) and does all arithmetic on the FP32 pipes, two k-planes per
// instruction with the packed f32x2 operations of sm_100+.
//
// Contractions use an offset accumulator.  For a sum y = sum_l a_l b_l whose
// terms are bounded by B (sum_l |a_l||b_l| <= B), the running sum is kept as
// S = sigma + partial with sigma = 1.5 * 2^m and 2^m > 2B, so S stays in the
// binade [2^m, 2^(m+1)) and every rounding of S is to the same grid 2^(m-23):
//   t = fma(ah, bh, S);  d = S - t (exact);  r = fma(ah, bh, d)
// gives the residual of the exact product to 2^-24 of itself (|r| <= 2^(m-24)).
// The residuals are summed the same way on a second offset S2 = sigma * 2^-18
// (grid 2^(m-41)), whose own exact residuals and the cross products
// ah*bl + al*bh go to a plain float c.  The result is (S - sigma) + (S2 - sigma2)
// + c, all exact differences, with an absolute error of about n * 2^(m-48),
// i.e. 2^-44 B.  Bounds come from the element maximum of |u| (|wr|,|ws|,|wt| in
// the second phase) times the absolute row (column) sums of D.
//
// The pointwise geometric product uses Dekker products (FMA-exact) and Knuth
// two-sums.  Inputs: u and w in FP64, D in FP64 (split on load), G pre-split by
// nek_geom_ff into [e][p][12] floats (48 B per point, the same HBM traffic as
// FP64 G).
//
// Two kernel families: k_ax_ff walks (i, j) columns (or groups of planes
// above nx = 12) with u, wr, ws, wt as float pairs in shared memory; k_ax_ffi
// (nx = 10 and 12) keeps k-plane pairs as float4 so one load feeds a packed
// instruction, and spreads an element's (column, k-pair) items over whole
// warps.  Both take a compile-time load mode (plain, gathered, skipping
// finished problems, with element energies, with the solve's direction update).
//
// This header holds the kernels and their launch templates; the per-nx
// launchers are compiled in nek_ax_ff_nx_*.cu (a few nx each, so the build's
// translation units compile in parallel) and nek_ax_ff.cu dispatches to them.
#pragma once

#include <type_traits>

#include "nek_ff.cuh"
#include "nek_internal.h"
#include "nek_reduce.cuh"

namespace nek {

namespace {

// ---------------------------------------------------------------- f32 / f32x2 arithmetic
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

template <class T>
__device__ __forceinline__ T splat(float x);
template <>
__device__ __forceinline__ float splat<float>(float x) { return x; }
template <>
__device__ __forceinline__ float2 splat<float2>(float x) { return make_float2(x, x); }

template <class T>
__device__ __forceinline__ T vzero() { return splat<T>(0.f); }

// Knuth two-sum: s + e = a + b exactly.
template <class T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e)
{
    s = vadd(a, b);
    const T bb = vsub(s, a);
    e = vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
}

// 1.5 * 2^(floor(log2 b) + 2): offset whose binade holds any partial sum bounded by b.
__device__ __forceinline__ float offset_for(float b)
{
    return __fmul_rn(__int_as_float(__float_as_int(b) & 0x7F800000), 6.0f);
}

template <class T>
struct OffsetAcc {
    T S, S2, c0, c1, c2, s1;
    __device__ __forceinline__ void init(T sigma)
    {
        s1 = sigma;
        S = s1;
        S2 = vmul(sigma, splat<T>(3.814697265625e-06f));  // sigma * 2^-18
        c0 = vzero<T>();
        c1 = vzero<T>();
        c2 = vzero<T>();
    }
    // += (ah + al) * (bh + bl).  S, S2, c0, c1 and c2 each carry a one-operation
    // recurrence, so consecutive terms overlap in the pipeline.
    __device__ __forceinline__ void add(T ah, T al, T bh, T bl)
    {
        const T t = vfma(ah, bh, S);
        const T d = vsub(S, t);
        const T r = vfma(ah, bh, d);
        const T t2 = vadd(S2, r);
        const T d2 = vsub(S2, t2);
        const T r2 = vadd(r, d2);
        c0 = vadd(c0, r2);
        c1 = vfma(ah, bl, c1);
        c2 = vfma(al, bh, c2);
        S = t;
        S2 = t2;
    }
    __device__ __forceinline__ void finish(T& hi, T& lo) const
    {
        const T H1 = vsub(S, s1);
        const T H2 = vsub(S2, vmul(s1, splat<T>(3.814697265625e-06f)));
        T e;
        two_sum(H1, H2, hi, e);
        lo = vadd(e, vadd(c0, vadd(c1, c2)));
    }
};

// Dekker product with FMA: p + e = (ah + al)(bh + bl) to ~2^-48.
template <class T>
__device__ __forceinline__ void df_mul(T ah, T al, T bh, T bl, T& p, T& e)
{
    p = vmul(ah, bh);
    e = vfma(ah, bh, vneg(p));
    e = vfma(ah, bl, e);
    e = vfma(al, bh, e);
}

// (ah,al)(xh,xl) + (bh,bl)(yh,yl) + (ch,cl)(zh,zl) as an unevaluated pair.
template <class T>
__device__ __forceinline__ void df_dot3(T ah, T al, T xh, T xl, T bh, T bl, T yh, T yl, T ch, T cl, T zh, T zl,
                                        T& h, T& l)
{
    T p1, e1, p2, e2, p3, e3, s, f1, f2;
    df_mul(ah, al, xh, xl, p1, e1);
    df_mul(bh, bl, yh, yl, p2, e2);
    df_mul(ch, cl, zh, zl, p3, e3);
    two_sum(p1, p2, s, f1);
    two_sum(s, p3, h, f2);
    l = vadd(vadd(vadd(e1, e2), vadd(e3, f1)), f2);
}


__device__ __forceinline__ float absmax_bits(float a, float b) { return fmaxf(fabsf(a), b); }

// slot[key] = max(slot[key], v) for v >= 0, one shared-memory atomic per key per warp.
__device__ __forceinline__ void segmented_max_to_smem(int key, float v, float* slot)
{
    // Lanes beyond a partial last warp do not exist, so only the active lanes are named.
    const unsigned same = __match_any_sync(__activemask(), key);
    const unsigned m = __reduce_max_sync(same, __float_as_uint(v));
    if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMax(reinterpret_cast<unsigned*>(slot + key), m);
}

// Lane access for the 1- and 2-wide forms.
template <class T>
struct Lanes;
template <>
struct Lanes<float> {
    static constexpr int W = 1;
    __device__ static __forceinline__ float get(float v, int) { return v; }
    __device__ static __forceinline__ void set(float& v, int, float x) { v = x; }
};
template <>
struct Lanes<float2> {
    static constexpr int W = 2;
    __device__ static __forceinline__ float get(float2 v, int q) { return q ? v.y : v.x; }
    __device__ static __forceinline__ void set(float2& v, int q, float x)
    {
        if (q)
            v.y = x;
        else
            v.x = x;
    }
};

template <int NX>
constexpr int ff_epb();

template <int NX, int EPB>
constexpr size_t ff_smem_bytes()
{
    // four float2 blocks [EPB][N3] (u, wr, ws, wt), D and D^T as float2 pairs,
    // rowabs, colabs and the per-element maxima.
    return sizeof(float2) * (4 * EPB * NX * NX * NX + 2 * NX * NX) + sizeof(float) * (2 * NX + 4 * EPB + 4) + 16;
}

// k-planes per thread.  Up to nx = 12 a thread walks its whole (i, j) column
// (measured fastest: the per-thread set-up is amortised over nx planes); above,
// columns are split into groups of 4 planes (3 at nx = 13) so that one element
// spreads over up to 1024 threads.
constexpr int ff_ppt(int nx) { return nx <= 12 ? nx : nx == 13 ? 3 : 4; }
constexpr int ff_groups(int nx) { return (nx + ff_ppt(nx) - 1) / ff_ppt(nx); }
constexpr int ff_threads_per_elem(int nx) { return nx * nx * ff_groups(nx); }

// Default elements per CTA: at least ~128 threads per CTA, 1, 2 or 4 where
// possible; nx = 10 and 12 run the item-mapped kernel with 128 and 144 threads
// per element, whose measured best counts are 1 and 4 (the tuner may change them).
template <int NX>
constexpr int ff_epb()
{
    if constexpr (NX == 10) return 1;
    if constexpr (NX == 12) return 4;
    return ff_threads_per_elem(NX) >= 128 ? 1 : ff_threads_per_elem(NX) >= 64 ? 2 : 4;
}

// CTAs per SM the register budget is set for: about 16 resident warps.
template <int NX, int EPB>
constexpr int ff_min_blocks()
{
    constexpr int warps = (NX * NX * EPB * ff_groups(NX) + 31) / 32;
    return warps >= 16 ? 1 : (16 / warps > 4 ? 4 : 16 / warps);
}

// Thread (e, i, j, g) computes the W-wide k-groups of planes [g*PPT, g*PPT + PPT)
// of element e.
// Load modes of the float-float kernels: plain w = AX u; GATHER: u is a
// unique-node vector read through l2g (element point p reads u[l2g[p]]); SKIP:
// a CTA whose elements all belong to finished problems (eprob: problem of each
// element, pdone: one byte per problem) returns at once (batched solves); DOT:
// plain, and each element's energy u_e . (A_e u_e) is written to edot[e] (the
// CG's <p, Ap> is their sum, see the solve); SKIP_DOT, GATHER_DOT: energies
// with the skip (batched solves) or the gather (unique-node solves); DIR_DOT:
// energies, the input being the solve's direction after the update that the
// kernel applies as it loads it (DirUpdate).
constexpr int kModePlain = 0, kModeGather = 1, kModeSkip = 2, kModeDot = 3, kModeSkipDot = 4, kModeGatherDot = 5,
              kModeDirDot = 6;
constexpr bool mode_skips(int m) { return m == kModeSkip || m == kModeSkipDot; }
constexpr bool mode_gathers(int m) { return m == kModeGather || m == kModeGatherDot; }
constexpr bool mode_energies(int m)
{
    return m == kModeDot || m == kModeSkipDot || m == kModeGatherDot || m == kModeDirDot;
}

// True when every element of the CTA belongs to a finished problem.
template <int MODE>
__device__ __forceinline__ bool cta_skipped(const int32_t* __restrict__ eprob, const uint8_t* __restrict__ pdone,
                                            int64_t e0, int ne)
{
    if constexpr (!mode_skips(MODE)) {
        return false;
    } else {
        bool all_done = true;
        for (int q = 0; q < ne; q++) all_done = all_done && pdone[eprob[e0 + q]] != 0;
        return all_done;
    }
}

// Reads the launch's input points q in [0, count) of the CTA (local index q of
// element block e0) and hands each value to stage(q, value): u[q] directly,
// through l2g in the gather modes, and in DIR_DOT the solve's direction after
// the update (x += alpha p, p = minv r + beta p, both written back), four
// points per thread at a time with all loads issued before the stores (one
// point at a time, each load would wait for the previous point's stores).
template <int MODE, int NT, class Stage>
__device__ __forceinline__ void load_input(int tid, int count, int64_t first, const double* __restrict__ u,
                                           const int32_t* __restrict__ l2g, const DirUpdate& dir, Stage&& stage)
{
    if constexpr (MODE == kModeDirDot) {
        const bool dx = dir.sc->xpend != 0, dp = !(dir.sc->done || dir.sc->status != NEK_OK);
        const double da = dir.sc->alpha, db = dir.sc->beta;
        constexpr int B = 4;
        for (int q0 = tid; q0 < count; q0 += B * NT) {
            double pv[B], xv[B], mv[B], rv[B];
#pragma unroll
            for (int m = 0; m < B; m++) {
                const int q = q0 + m * NT;
                const int64_t g = first + (q < count ? q : 0);
                pv[m] = dir.p[g];
                xv[m] = dx ? dir.x[g] : 0.0;
                mv[m] = dir.minv[g];
                rv[m] = dir.r[g];
            }
#pragma unroll
            for (int m = 0; m < B; m++) {
                const int q = q0 + m * NT;
                if (q >= count) break;
                const int64_t g = first + q;
                double val = pv[m];
                if (dx) dir.x[g] = fma(da, val, xv[m]);
                if (dp) {
                    val = fma(db, val, mv[m] * rv[m]);
                    dir.p[g] = val;
                }
                stage(q, val);
            }
        }
    } else {
        for (int q = tid; q < count; q += NT)
            stage(q, mode_gathers(MODE) ? __ldg(u + __ldg(l2g + first + q)) : __ldg(u + first + q));
    }
}

// The input value at local point p of an element whose first point is `first`,
// read again for the energy: DIR_DOT reads the direction this kernel wrote
// (plain loads), the gather modes go through l2g.
template <int MODE>
__device__ __forceinline__ double reread_input(int64_t first, int p, const double* __restrict__ u,
                                               const int32_t* __restrict__ l2g, const DirUpdate& dir)
{
    if constexpr (MODE == kModeDirDot)
        return dir.p[first + p];
    else if constexpr (mode_gathers(MODE))
        return __ldg(u + __ldg(l2g + first + p));
    else
        return __ldg(u + first + p);
}

template <int NX, int EPB, int MODE>
__global__ void __launch_bounds__(NX* NX* ff_groups(NX)* EPB, (ff_min_blocks<NX, EPB>()))
    k_ax_ff(int64_t nelt, const double* __restrict__ D, const float4* __restrict__ Gff,
            const double* __restrict__ u, double* __restrict__ w, const int32_t* __restrict__ l2g,
            const int32_t* __restrict__ eprob, const uint8_t* __restrict__ pdone, double* __restrict__ edot,
            DirUpdate dir)
{
    using T = typename std::conditional<(NX % 2 == 0), float2, float>::type;
    using L = Lanes<T>;
    constexpr int W = L::W;
    constexpr int PPT = ff_ppt(NX), NG = ff_groups(NX);
    constexpr int N2 = NX * NX, N3 = NX * NX * NX, TPE = N2 * NG, NT = TPE * EPB;
    static_assert(PPT % W == 0, "plane groups hold whole k-pairs");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sU = reinterpret_cast<float2*>(smem_raw);  // [EPB][N3] u (hi, lo)
    float2* sWr = sU + EPB * N3;                       // [EPB][N3] wr
    float2* sWs = sWr + EPB * N3;                      // [EPB][N3] ws
    float2* sWt = sWs + EPB * N3;                      // [EPB][N3] wt
    float2* sD = sWt + EPB * N3;                       // D[i][l]   at i*NX+l
    float2* sDT = sD + N2;                             // D[k][l]   at l*NX+k
    float* sRow = reinterpret_cast<float*>(sDT + N2);  // sum_l |D[q][l]|
    float* sCol = sRow + NX;                           // sum_l |D[l][q]|
    float* sMax = sCol + NX;  // [EPB][4]: max |u|, |wr|, |ws|, |wt| (non-negative floats, compared as ints)

    const int tid = threadIdx.x;
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int ne = static_cast<int>(nelt - e0 < EPB ? nelt - e0 : EPB);
    if (cta_skipped<MODE>(eprob, pdone, e0, ne)) return;  // uniform over the CTA, before any barrier

    for (int q = tid; q < N2; q += NT) {
        const float2 d = split_double(D[q]);
        sD[q] = d;
        sDT[(q % NX) * NX + q / NX] = d;
    }
    for (int q = tid; q < 4 * EPB; q += NT) sMax[q] = 0.f;
    load_input<MODE, NT>(tid, ne * N3, e0 * N3, u, l2g, dir, [&](int q, double v) { sU[q] = split_double(v); });
    __syncthreads();
    for (int q = tid; q < NX; q += NT) {
        float r = 0.f, c = 0.f;
        for (int l = 0; l < NX; l++) {
            r += fabsf(sD[q * NX + l].x);
            c += fabsf(sD[l * NX + q].x);
        }
        // inflate for the lo parts and the rounding of the sums themselves
        sRow[q] = r * 1.0001f;
        sCol[q] = c * 1.0001f;
    }

    const int el = tid / TPE;
    const int q3 = tid - el * TPE;
    const int g = q3 / N2;
    const int q2 = q3 - g * N2;
    const int i = q2 % NX, j = q2 / NX;
    const int kbeg = g * PPT;
    const int kend = kbeg + PPT < NX ? kbeg + PPT : NX;
    const bool active = el < ne;
    const float2* ue = sU + el * N3;
    {
        float m = 0.f;
        if (active)
            for (int k = kbeg; k < kend; k++) m = absmax_bits(ue[i + NX * (j + NX * k)].x, m);
        segmented_max_to_smem(4 * el, m, sMax);
    }
    __syncthreads();

    // ------------------------------------------------------------- phase 1
    float mx_r = 0.f, mx_s = 0.f, mx_t = 0.f;
    if (active) {
        const float umax = sMax[4 * el] * 1.0001f;
        const T sig_r = splat<T>(offset_for(sRow[i] * umax));
        const T sig_s = splat<T>(offset_for(sRow[j] * umax));
        const float4* Ge = Gff + (e0 + el) * (int64_t)N3 * 3;
        float2* wre = sWr + el * N3;
        float2* wse = sWs + el * N3;
        float2* wte = sWt + el * N3;
#pragma unroll 1
        for (int k0 = kbeg; k0 < kend; k0 += W) {
            OffsetAcc<T> ar, as, at;
            T sig_t;
#pragma unroll
            for (int q = 0; q < W; q++) L::set(sig_t, q, offset_for(sRow[k0 + q] * umax));
            ar.init(sig_r);
            as.init(sig_s);
            at.init(sig_t);
#pragma unroll 2
            for (int l = 0; l < NX; l++) {
                T uh, ul, vh, vl, dh, dl;
#pragma unroll
                for (int q = 0; q < W; q++) {
                    const float2 a = ue[l + NX * (j + NX * (k0 + q))];
                    const float2 b = ue[i + NX * (l + NX * (k0 + q))];
                    const float2 d = sDT[l * NX + k0 + q];
                    L::set(uh, q, a.x);
                    L::set(ul, q, a.y);
                    L::set(vh, q, b.x);
                    L::set(vl, q, b.y);
                    L::set(dh, q, d.x);
                    L::set(dl, q, d.y);
                }
                const float2 dr = sD[i * NX + l], ds = sD[j * NX + l], uc = ue[i + NX * (j + NX * l)];
                ar.add(splat<T>(dr.x), splat<T>(dr.y), uh, ul);
                as.add(splat<T>(ds.x), splat<T>(ds.y), vh, vl);
                at.add(dh, dl, splat<T>(uc.x), splat<T>(uc.y));
            }
            T urh, url, ush, usl, uth, utl;
            ar.finish(urh, url);
            as.finish(ush, usl);
            at.finish(uth, utl);
            // geometric factors of the W points: g[2a], g[2a+1] = hi, lo of factor a
            T gf[12];
#pragma unroll
            for (int q = 0; q < W; q++) {
                const int p = i + NX * (j + NX * (k0 + q));
                const float4 a = __ldg(Ge + 3 * p), b = __ldg(Ge + 3 * p + 1), c = __ldg(Ge + 3 * p + 2);
                L::set(gf[0], q, a.x); L::set(gf[1], q, a.y); L::set(gf[2], q, a.z); L::set(gf[3], q, a.w);
                L::set(gf[4], q, b.x); L::set(gf[5], q, b.y); L::set(gf[6], q, b.z); L::set(gf[7], q, b.w);
                L::set(gf[8], q, c.x); L::set(gf[9], q, c.y); L::set(gf[10], q, c.z); L::set(gf[11], q, c.w);
            }
            T wrh, wrl, wsh, wsl, wth, wtl;
            df_dot3(gf[0], gf[1], urh, url, gf[2], gf[3], ush, usl, gf[4], gf[5], uth, utl, wrh, wrl);
            df_dot3(gf[2], gf[3], urh, url, gf[6], gf[7], ush, usl, gf[8], gf[9], uth, utl, wsh, wsl);
            df_dot3(gf[4], gf[5], urh, url, gf[8], gf[9], ush, usl, gf[10], gf[11], uth, utl, wth, wtl);
#pragma unroll
            for (int q = 0; q < W; q++) {
                const int p = i + NX * (j + NX * (k0 + q));
                wre[p] = make_float2(L::get(wrh, q), L::get(wrl, q));
                wse[p] = make_float2(L::get(wsh, q), L::get(wsl, q));
                wte[p] = make_float2(L::get(wth, q), L::get(wtl, q));
                mx_r = absmax_bits(L::get(wrh, q), mx_r);
                mx_s = absmax_bits(L::get(wsh, q), mx_s);
                mx_t = absmax_bits(L::get(wth, q), mx_t);
            }
        }
    }
    segmented_max_to_smem(4 * el + 1, mx_r, sMax);
    segmented_max_to_smem(4 * el + 2, mx_s, sMax);
    segmented_max_to_smem(4 * el + 3, mx_t, sMax);
    __syncthreads();

    // ------------------------------------------------------------- phase 2
    double energy = 0.0;  // kModeDot: sum of u . w over this thread's points
    if (active) {
        const float2* wre = sWr + el * N3;
        const float2* wse = sWs + el * N3;
        const float2* wte = sWt + el * N3;
        const float mwr = sMax[4 * el + 1] * 1.0001f, mws = sMax[4 * el + 2] * 1.0001f,
                    mwt = sMax[4 * el + 3] * 1.0001f;
        const float bij = sCol[i] * mwr + sCol[j] * mws;
        double* we = w + (e0 + el) * (int64_t)N3;
#pragma unroll 1
        for (int k0 = kbeg; k0 < kend; k0 += W) {
            T sig;
#pragma unroll
            for (int q = 0; q < W; q++) L::set(sig, q, offset_for(bij + sCol[k0 + q] * mwt));
            OffsetAcc<T> acc;
            acc.init(sig);
#pragma unroll 2
            for (int l = 0; l < NX; l++) {
                T ah, al, bh, bl, dh, dl;
#pragma unroll
                for (int q = 0; q < W; q++) {
                    const float2 a = wre[l + NX * (j + NX * (k0 + q))];
                    const float2 b = wse[i + NX * (l + NX * (k0 + q))];
                    const float2 d = sD[l * NX + k0 + q];
                    L::set(ah, q, a.x);
                    L::set(al, q, a.y);
                    L::set(bh, q, b.x);
                    L::set(bl, q, b.y);
                    L::set(dh, q, d.x);
                    L::set(dl, q, d.y);
                }
                const float2 ci = sD[l * NX + i], cj = sD[l * NX + j], tc = wte[i + NX * (j + NX * l)];
                acc.add(splat<T>(ci.x), splat<T>(ci.y), ah, al);
                acc.add(splat<T>(cj.x), splat<T>(cj.y), bh, bl);
                acc.add(dh, dl, splat<T>(tc.x), splat<T>(tc.y));
            }
            T hi, lo;
            acc.finish(hi, lo);
#pragma unroll
            for (int q = 0; q < W; q++) {
                const int p = i + NX * (j + NX * (k0 + q));
                const double wv = join_pair(L::get(hi, q), L::get(lo, q));
                we[p] = wv;
                if constexpr (mode_energies(MODE))
                    energy = fma(reread_input<MODE>((e0 + el) * (int64_t)N3, p, u, l2g, dir), wv, energy);
            }
        }
    }
    if constexpr (mode_energies(MODE)) element_sums<TPE, EPB>(energy, reinterpret_cast<double*>(sU), edot + e0, ne);
}

// ------------------------------------------------------------------------
// nx = 10 and 12: operands laid out for the packed f32x2 instructions.
//
// Shared memory holds u, wr and ws as float4 (h_k, h_k+1, l_k, l_k+1) per
// (k-pair, j, i), so one 16-byte load gives both packed operands of a term; D is
// kept pre-splatted (h, h, l, l), for the t-direction as k-pair tables, and for
// the r-contraction transposed, so that a warp reads it across i without bank
// conflicts; wt goes to a fourth block, read back by columns in phase 2.
template <int NX>
constexpr size_t kpair_smem_bytes(int epb)
{
    // U4, WR4, WS4: [EPB][NX/2][NX][NX] float4 = 3 * 8 B per point; WT2 [EPB][N3]
    // float2; DS [NX][NX], DP / DPT [NX][NX/2], DSt [NX][NX] float4; rowabs,
    // colabs, maxima.
    return sizeof(float4) * (3 * (size_t)epb * (NX / 2) * NX * NX + 3 * NX * NX) +
           sizeof(float2) * (size_t)epb * NX * NX * NX + sizeof(float) * (2 * NX + 4 * (size_t)epb + 4) + 16;
}

// Item mapping: the TPE threads of an element take its (column, k-pair) items
// q = t, t + TPE, ...  At nx = 10, 128 threads share 500 items (at most 4
// each): one column per thread would make a 100-thread CTA run a fourth warp on
// 4 lanes, a quarter of its issue slots.  At nx = 12, 144 threads take one
// column each (6 items); with four elements per CTA that is 18 full warps.  A
// thread reads the column values of the t-contraction from shared memory (one
// 16-byte load per k-pair) instead of holding a column in registers.
constexpr int ffi_tpe(int nx) { return nx == 12 ? 144 : 128; }

// CTAs per SM the register budget is set for: 20 resident warps (96 registers
// a thread at one element per CTA; the kernel then spills 4-8 bytes).
template <int NX, int EPB>
constexpr int ffi_min_blocks()
{
    constexpr int warps = (ffi_tpe(NX) * EPB + 31) / 32;
    return warps >= 20 ? 1 : 20 / warps;
}

template <int NX, int EPB, int MODE>
__global__ void __launch_bounds__(ffi_tpe(NX) * EPB, (ffi_min_blocks<NX, EPB>()))
    k_ax_ffi(int64_t nelt, const double* __restrict__ D, const float4* __restrict__ Gff,
             const double* __restrict__ u, double* __restrict__ w, const int32_t* __restrict__ l2g,
             const int32_t* __restrict__ eprob, const uint8_t* __restrict__ pdone, double* __restrict__ edot,
             DirUpdate dir)
{
    static_assert(NX % 2 == 0 && NX <= 12, "even nx up to 12");
    using T = float2;
    constexpr int NP = NX / 2, N2 = NX * NX, N3 = NX * NX * NX, PB = NP * N2;
    constexpr int TPE = ffi_tpe(NX), NT = TPE * EPB, NITEM = NP * N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* U4 = reinterpret_cast<float4*>(smem_raw);  // [EPB][NP][NX][NX]
    float4* WR4 = U4 + EPB * PB;
    float4* WS4 = WR4 + EPB * PB;
    float2* WT2 = reinterpret_cast<float2*>(WS4 + EPB * PB);  // [EPB][N3] wt (h, l)
    float4* DS = reinterpret_cast<float4*>(WT2 + EPB * N3);    // DS[a*NX+b] = (Dh,Dh,Dl,Dl) of D[a][b]
    float4* DP = DS + N2;              // DP[l*NP+kp]  = (Dh[2kp][l], Dh[2kp+1][l], Dl[2kp][l], Dl[2kp+1][l])
    float4* DPT = DP + NX * NP;        // DPT[l*NP+kp] = (Dh[l][2kp], Dh[l][2kp+1], Dl[l][2kp], Dl[l][2kp+1])
    float4* DSt = DPT + NX * NP;       // DSt[b*NX+a] = DS[a*NX+b]: the r-contraction's row of D read across i
    float* sRow = reinterpret_cast<float*>(DSt + N2);
    float* sCol = sRow + NX;
    float* sMax = sCol + NX;

    const int tid = threadIdx.x;
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int ne = static_cast<int>(nelt - e0 < EPB ? nelt - e0 : EPB);
    if (cta_skipped<MODE>(eprob, pdone, e0, ne)) return;  // uniform over the CTA, before any barrier

    for (int q = tid; q < N2; q += NT) {
        const int a = q / NX, b = q % NX;
        const float2 d = split_double(D[q]);
        DS[q] = make_float4(d.x, d.x, d.y, d.y);
        DSt[b * NX + a] = make_float4(d.x, d.x, d.y, d.y);
        float* dp = reinterpret_cast<float*>(DP + b * NP + a / 2);  // D[a][b]: k = a, l = b
        dp[a & 1] = d.x;
        dp[2 + (a & 1)] = d.y;
        float* dt = reinterpret_cast<float*>(DPT + a * NP + b / 2);  // D[a][b]: l = a, k = b
        dt[b & 1] = d.x;
        dt[2 + (b & 1)] = d.y;
    }
    for (int q = tid; q < 4 * EPB; q += NT) sMax[q] = 0.f;
    load_input<MODE, NT>(tid, ne * N3, e0 * N3, u, l2g, dir, [&](int q, double val) {
        const int el = q / N3, p = q - el * N3;
        const int k = p / N2, ji = p - k * N2;
        const float2 v = split_double(val);
        float* dst = reinterpret_cast<float*>(U4 + el * PB + (k / 2) * N2 + ji);
        dst[k & 1] = v.x;
        dst[2 + (k & 1)] = v.y;
    });
    __syncthreads();
    for (int q = tid; q < NX; q += NT) {
        float r = 0.f, c = 0.f;
        for (int l = 0; l < NX; l++) {
            r += fabsf(DS[q * NX + l].x);
            c += fabsf(DS[l * NX + q].x);
        }
        sRow[q] = r * 1.0001f;
        sCol[q] = c * 1.0001f;
    }

    const int el = tid / TPE;
    const int t = tid - el * TPE;
    const bool active = el < ne;
    const float4* ue = U4 + el * PB;
    {
        float m = 0.f;
        if (active)
            for (int q = t; q < PB; q += TPE) {
                const float4 v = ue[q];
                m = absmax_bits(v.x, absmax_bits(v.y, m));
            }
        segmented_max_to_smem(4 * el, m, sMax);
    }
    __syncthreads();

    // ------------------------------------------------------------- phase 1
    float mx_r = 0.f, mx_s = 0.f, mx_t = 0.f;
    if (active) {
        const float umax = sMax[4 * el] * 1.0001f;
        const float4* Ge = Gff + (e0 + el) * (int64_t)N3 * 3;
        float4* wre = WR4 + el * PB;
        float4* wse = WS4 + el * PB;
        float2* wte = WT2 + el * N3;
#pragma unroll 1
        for (int q = t; q < NITEM; q += TPE) {
            const int kp = q / N2, c = q - kp * N2;
            const int i = c % NX, j = c / NX, k0 = 2 * kp;
            OffsetAcc<T> ar, as, at;
            ar.init(splat<T>(offset_for(sRow[i] * umax)));
            as.init(splat<T>(offset_for(sRow[j] * umax)));
            at.init(make_float2(offset_for(sRow[k0] * umax), offset_for(sRow[k0 + 1] * umax)));
            const float4* ur = ue + kp * N2 + j * NX;  // u(l, j, k0..k0+1) at ur[l]
            const float4* us = ue + kp * N2 + i;       // u(i, l, k0..k0+1) at us[l * NX]
            const float4* uc = ue + c;                 // u(i, j, 2m..2m+1) at uc[m * N2]
            float4 cu = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int l = 0; l < NX; l++) {
                if ((l & 1) == 0) cu = uc[(l >> 1) * N2];
                const float ch = (l & 1) ? cu.y : cu.x, cl = (l & 1) ? cu.w : cu.z;
                const float4 a = ur[l], b = us[l * NX];
                const float4 dr = DSt[l * NX + i], ds = DS[j * NX + l], dt = DP[l * NP + kp];
                ar.add(make_float2(dr.x, dr.y), make_float2(dr.z, dr.w), make_float2(a.x, a.y),
                       make_float2(a.z, a.w));
                as.add(make_float2(ds.x, ds.y), make_float2(ds.z, ds.w), make_float2(b.x, b.y),
                       make_float2(b.z, b.w));
                at.add(make_float2(dt.x, dt.y), make_float2(dt.z, dt.w), make_float2(ch, ch), make_float2(cl, cl));
            }
            T urh, url, ush, usl, uth, utl;
            ar.finish(urh, url);
            as.finish(ush, usl);
            at.finish(uth, utl);
            T gf[12];
#pragma unroll
            for (int qq = 0; qq < 2; qq++) {
                const int p = c + N2 * (k0 + qq);
                const float4 a = __ldg(Ge + 3 * p), b = __ldg(Ge + 3 * p + 1), cc = __ldg(Ge + 3 * p + 2);
                const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                for (int g = 0; g < 12; g++) {
                    if (qq)
                        gf[g].y = v[g];
                    else
                        gf[g].x = v[g];
                }
            }
            T wrh, wrl, wsh, wsl, wth, wtl;
            df_dot3(gf[0], gf[1], urh, url, gf[2], gf[3], ush, usl, gf[4], gf[5], uth, utl, wrh, wrl);
            df_dot3(gf[2], gf[3], urh, url, gf[6], gf[7], ush, usl, gf[8], gf[9], uth, utl, wsh, wsl);
            df_dot3(gf[4], gf[5], urh, url, gf[8], gf[9], ush, usl, gf[10], gf[11], uth, utl, wth, wtl);
            wre[kp * N2 + c] = make_float4(wrh.x, wrh.y, wrl.x, wrl.y);
            wse[kp * N2 + c] = make_float4(wsh.x, wsh.y, wsl.x, wsl.y);
            wte[c + N2 * k0] = make_float2(wth.x, wtl.x);
            wte[c + N2 * (k0 + 1)] = make_float2(wth.y, wtl.y);
            mx_r = absmax_bits(wrh.x, absmax_bits(wrh.y, mx_r));
            mx_s = absmax_bits(wsh.x, absmax_bits(wsh.y, mx_s));
            mx_t = absmax_bits(wth.x, absmax_bits(wth.y, mx_t));
        }
    }
    segmented_max_to_smem(4 * el + 1, mx_r, sMax);
    segmented_max_to_smem(4 * el + 2, mx_s, sMax);
    segmented_max_to_smem(4 * el + 3, mx_t, sMax);
    __syncthreads();

    // ------------------------------------------------------------- phase 2
    double energy = 0.0;  // energy modes: sum of u . w over this thread's points
    if (active) {
        const float4* wre = WR4 + el * PB;
        const float4* wse = WS4 + el * PB;
        const float2* wte = WT2 + el * N3;
        const float mwr = sMax[4 * el + 1] * 1.0001f, mws = sMax[4 * el + 2] * 1.0001f,
                    mwt = sMax[4 * el + 3] * 1.0001f;
        double* we = w + (e0 + el) * (int64_t)N3;
        const int64_t ef = (e0 + el) * (int64_t)N3;  // the element's first point
#pragma unroll 1
        for (int q = t; q < NITEM; q += TPE) {
            const int kp = q / N2, c = q - kp * N2;
            const int i = c % NX, j = c / NX, k0 = 2 * kp;
            const int p0 = c + N2 * k0;
            double u0 = 0.0, u1 = 0.0;
            if constexpr (mode_energies(MODE)) {  // issued here, used after the contraction
                u0 = reread_input<MODE>(ef, p0, u, l2g, dir);
                u1 = reread_input<MODE>(ef, p0 + N2, u, l2g, dir);
            }
            const float bij = sCol[i] * mwr + sCol[j] * mws;
            OffsetAcc<T> acc;
            acc.init(make_float2(offset_for(bij + sCol[k0] * mwt), offset_for(bij + sCol[k0 + 1] * mwt)));
            const float4* rr = wre + kp * N2 + j * NX;  // wr(l, j, k0..k0+1) at rr[l]
            const float4* ss = wse + kp * N2 + i;       // ws(i, l, k0..k0+1) at ss[l * NX]
            const float2* tt = wte + c;                 // wt(i, j, l) at tt[l * N2]
#pragma unroll
            for (int l = 0; l < NX; l++) {
                const float4 a = rr[l], b = ss[l * NX];
                const float4 ci = DS[l * NX + i], cj = DS[l * NX + j], dk = DPT[l * NP + kp];
                acc.add(make_float2(ci.x, ci.y), make_float2(ci.z, ci.w), make_float2(a.x, a.y),
                        make_float2(a.z, a.w));
                acc.add(make_float2(cj.x, cj.y), make_float2(cj.z, cj.w), make_float2(b.x, b.y),
                        make_float2(b.z, b.w));
                const float2 tc = tt[l * N2];
                acc.add(make_float2(dk.x, dk.y), make_float2(dk.z, dk.w), make_float2(tc.x, tc.x),
                        make_float2(tc.y, tc.y));
            }
            T hi, lo;
            acc.finish(hi, lo);
            const double w0 = join_pair(hi.x, lo.x), w1 = join_pair(hi.y, lo.y);
            we[p0] = w0;
            we[p0 + N2] = w1;
            if constexpr (mode_energies(MODE)) energy = fma(u1, w1, fma(u0, w0, energy));
        }
    }
    if constexpr (mode_energies(MODE)) element_sums<TPE, EPB>(energy, reinterpret_cast<double*>(U4), edot + e0, ne);
}

// The k-pair layout (k_ax_ffi) is used where it measured faster than the
// column walk on GB300 (nx = 10: 34.0 vs 25.6 GDOF/s; nx = 12: 26.5 vs 23.2;
// nx = 8: 32.1 vs 36.4 with an earlier form of the layout).  The choice is
// fixed per nx, never tuned at run time, because the two orders of summation
// round differently.
template <int NX>
constexpr bool ff_item_layout()
{
    return NX == 10 || NX == 12;
}

template <int NX, int EPB>
constexpr size_t ff_variant_smem()
{
    if constexpr (ff_item_layout<NX>())
        return kpair_smem_bytes<NX>(EPB);
    else
        return ff_smem_bytes<NX, EPB>();
}

template <int NX, int EPB, int MODE>
nek_status launch_ax_ff_kernel(int64_t nelt, const double* D, const float* Gff, const double* u, double* w,
                               cudaStream_t s, const int32_t* l2g, const int32_t* eprob, const uint8_t* pdone,
                               double* edot, const DirUpdate* dir = nullptr)
{
    constexpr size_t smem = ff_variant_smem<NX, EPB>();
    static std::atomic<uint64_t> configured{0};
    const int64_t blocks = (nelt + EPB - 1) / EPB;
    if (blocks > 0x7fffffff) return NEK_ERR_TOO_LARGE;
    if constexpr (ff_item_layout<NX>()) {
        nek_status st = ensure_dyn_smem(k_ax_ffi<NX, EPB, MODE>, smem, configured);
        if (st != NEK_OK) return st;
        k_ax_ffi<NX, EPB, MODE><<<(unsigned)blocks, ffi_tpe(NX) * EPB, smem, s>>>(
            nelt, D, reinterpret_cast<const float4*>(Gff), u, w, l2g, eprob, pdone, edot, dir ? *dir : DirUpdate{});
    } else {
        nek_status st = ensure_dyn_smem(k_ax_ff<NX, EPB, MODE>, smem, configured);
        if (st != NEK_OK) return st;
        k_ax_ff<NX, EPB, MODE><<<(unsigned)blocks, ff_threads_per_elem(NX) * EPB, smem, s>>>(
            nelt, D, reinterpret_cast<const float4*>(Gff), u, w, l2g, eprob, pdone, edot, dir ? *dir : DirUpdate{});
    }
    return check_launch();
}

template <int NX, int EPB>
nek_status launch_ax_ff_variant(int64_t nelt, const double* D, const float* Gff, const double* u, double* w,
                                cudaStream_t s, const int32_t* l2g, const int32_t* eprob, const uint8_t* pdone,
                                double* edot, const DirUpdate* dir)
{
    if (dir) {
        if (!edot || l2g || eprob) return NEK_ERR_INVALID_ARG;
        return launch_ax_ff_kernel<NX, EPB, kModeDirDot>(nelt, D, Gff, dir->p, w, s, nullptr, nullptr, nullptr,
                                                         edot, dir);
    }
    if (l2g && edot)
        return launch_ax_ff_kernel<NX, EPB, kModeGatherDot>(nelt, D, Gff, u, w, s, l2g, nullptr, nullptr, edot);
    if (l2g)
        return launch_ax_ff_kernel<NX, EPB, kModeGather>(nelt, D, Gff, u, w, s, l2g, nullptr, nullptr, nullptr);
    if (eprob && pdone && edot)
        return launch_ax_ff_kernel<NX, EPB, kModeSkipDot>(nelt, D, Gff, u, w, s, nullptr, eprob, pdone, edot);
    if (eprob && pdone)
        return launch_ax_ff_kernel<NX, EPB, kModeSkip>(nelt, D, Gff, u, w, s, nullptr, eprob, pdone, nullptr);
    if (edot) return launch_ax_ff_kernel<NX, EPB, kModeDot>(nelt, D, Gff, u, w, s, nullptr, nullptr, nullptr, edot);
    return launch_ax_ff_kernel<NX, EPB, kModePlain>(nelt, D, Gff, u, w, s, nullptr, nullptr, nullptr, nullptr);
}

template <int NX, int EPB>
constexpr bool ff_fits()
{
    constexpr int threads = ff_item_layout<NX>() ? ffi_tpe(NX) * EPB : ff_threads_per_elem(NX) * EPB;
    return threads <= 1024 && ff_variant_smem<NX, EPB>() <= 227 * 1024;
}

template <int NX>
nek_status launch_ax_ff_nx(int epb, int64_t nelt, const double* D, const float* Gff, const double* u, double* w,
                           cudaStream_t s, const int32_t* l2g, const int32_t* eprob, const uint8_t* pdone,
                           double* edot, const DirUpdate* dir)
{
    if (epb <= 0) epb = ff_epb<NX>();
    switch (epb) {
        case 1:
            if constexpr (ff_fits<NX, 1>())
                return launch_ax_ff_variant<NX, 1>(nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
            break;
        case 2:
            if constexpr (ff_fits<NX, 2>())
                return launch_ax_ff_variant<NX, 2>(nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
            break;
        case 4:
            if constexpr (ff_fits<NX, 4>())
                return launch_ax_ff_variant<NX, 4>(nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
            break;
        default:
            break;
    }
    if constexpr (ff_epb<NX>() != 1 && ff_epb<NX>() != 2 && ff_epb<NX>() != 4)
        return launch_ax_ff_variant<NX, ff_epb<NX>()>(nelt, D, Gff, u, w, s, l2g, eprob, pdone, edot, dir);
    return NEK_ERR_INVALID_ARG;
}

template <int NX>
bool ff_fits_rt(int epb)
{
    return (epb == 1 && ff_fits<NX, 1>()) || (epb == 2 && ff_fits<NX, 2>()) || (epb == 4 && ff_fits<NX, 4>());
}

}  // namespace

// Per-nx launchers and fit checks (nek_ax_ff_nx_<group>.cu: a = nx 2-7, b = 8-9,
// c = 10-11, d = 12-13, e = 14-16).
nek_status launch_ax_ff_group_a(int nx, int epb, int64_t nelt, const double* D, const float* Gff, const double* u,
                                  double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                                  const uint8_t* pdone, double* edot, const DirUpdate* dir);
bool ax_ff_fits_group_a(int nx, int epb);
nek_status launch_ax_ff_group_b(int nx, int epb, int64_t nelt, const double* D, const float* Gff, const double* u,
                                  double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                                  const uint8_t* pdone, double* edot, const DirUpdate* dir);
bool ax_ff_fits_group_b(int nx, int epb);
nek_status launch_ax_ff_group_c(int nx, int epb, int64_t nelt, const double* D, const float* Gff, const double* u,
                                  double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                                  const uint8_t* pdone, double* edot, const DirUpdate* dir);
bool ax_ff_fits_group_c(int nx, int epb);
nek_status launch_ax_ff_group_d(int nx, int epb, int64_t nelt, const double* D, const float* Gff, const double* u,
                                  double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                                  const uint8_t* pdone, double* edot, const DirUpdate* dir);
bool ax_ff_fits_group_d(int nx, int epb);
nek_status launch_ax_ff_group_e(int nx, int epb, int64_t nelt, const double* D, const float* Gff, const double* u,
                                  double* w, cudaStream_t s, const int32_t* l2g, const int32_t* eprob,
                                  const uint8_t* pdone, double* edot, const DirUpdate* dir);
bool ax_ff_fits_group_e(int nx, int epb);

}  // namespace nek
