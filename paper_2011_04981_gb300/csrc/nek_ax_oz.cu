// AX to FP64 accuracy with its contractions on the tensor cores (tcgen05):
// the operands split into BF16 digits, every digit product summed exactly per
// level in FP32 tensor-memory accumulators, the levels recombined into float
// pairs on the CUDA cores.
//
// Same operator as nek_ax (Section II-B, Listing 1 of arXiv 2011.04981), per
// element:
//   phase 1   ur = (I x I x D) u,  us = (I x D x I) u,  ut = (D x I x I) u
//             (wr, ws, wt) = G (ur, us, ut), pointwise, in float-float
//   phase 2   w = (I x I x D^T) wr + (I x D^T x I) ws + (D^T x I x I) wt
//
// Digits (the error-free splitting of Ozaki, Ogita, Oishi and Rump 2012, with
// BF16 digits).  Within an element every input value x of a phase is scaled
// by 2^-E (|x| < 2^E over the element) and split by round-to-grid extraction
// into six digits, x 2^-E = q_0 + ... + q_5 + O(2^-47) with
// q_a = d_a 2^(-8(a+1)), |d_a| <= 256: each digit is exact in BF16.  D is split
// the same way (digits p_b of D 2^-Ed, stored times 2^16).  A digit product
// q_a p_b 2^16 is an exact FP32 value on the grid 2^(-8L) of its level
// L = a + b, and a level's sum over the 8 NX products of a K row stays below
// 2^21 grid units, so the tensor core's FP32 accumulation of a level is exact
// in any order.  Levels 0..7 go to separate accumulator columns.
//
// MMA operands (one element at a time per CTA; M = 128 lines, K = N = 8 NX):
//   A, one buffer per direction: row = one of the element's NX^2 lines along
//     the contracted direction (rows above NX^2 are not read back); K = (point
//     l on the line, digit a): each 16-byte core-matrix row is one point's six
//     digits and two zeros, so a point's digits are written as one 16-byte
//     store per direction.  K-adjacent core matrices are 144 bytes apart
//     (128 + 16) so that a warp's stores spread over the banks.
//   B: row n = 16 (o / 2) + 2 L + (o mod 2) for output index o and level L,
//     K = (l, a): p_{L-a} of D[o][l] (D[l][o] in phase 2), zero where L - a is
//     not a digit index.  Two outputs of one level sit in adjacent columns, so
//     one 16-column TMEM load gives both lanes of a packed f32x2 operand.
//   Accumulator (TMEM): lane = line, column n as above; the three directions
//     side by side (24 NX of 256 columns).
//
// Recombination of one output from its exact levels x_0..x_7: with
// sigma = 1.5 * 2^k and 2^(k-1) above every partial sum,
//   T_0 = sigma + x_0, T_L = T_{L-1} + x_L (L = 1..3) stay in sigma's binade,
//   e_L = x_L - (T_L - T_{L-1}) is exact, hi = T_3 - sigma (a multiple of
//   ulp(sigma)), E = e_1 + e_2 + e_3 (exact), s = x_4 + x_5 + x_6 + x_7.
// Phase 1 hands the G product the pair (S, T + s) with S + T = hi + E exactly
// (Fast2Sum; exact because |E| < 2 ulp(sigma) <= |hi| or hi = 0).  Phase 2
// keeps (hi, E, s) per direction: the three his and the three Es each sum
// exactly, then one TwoSum gives the output pair.  The result carries about
// 2^-47 of the element's scale, like the float-float kernel.
//
// Work split (256 threads): every point-wise stage works on pairs of adjacent
// points (p, p + 1) in the two lanes of packed f32x2 operations, so vector
// loads give packed operands directly: u as two doubles, G in the pair-
// interleaved layout of nek_geom_oz, the exchange arrays likewise.  Thread
// lanes read TMEM lanes 32 (warp mod 4) + lane, the line of every direction;
// the two warps that share a lane range take alternate 16-column chunks.  For
// the s and t lines, adjacent lines hold adjacent points, so the two TMEM
// lanes of a point pair swap one value each (a shuffle) and store whole pairs.
//
// Stages per element: the u digits, phase-1 MMAs (one thread issues,
// committed to an mbarrier), recombination into the exchange array (over the
// A buffers, whose MMAs have completed), the G product with its pairs
// renormalised by TwoSum (the digit bound needs |low| <= ulp(high) / 2, which
// cancellation among the three products can break), the digits of wr, ws, wt,
// phase-2 MMAs, recombination, and the sum of the three directions written as
// doubles.  CTAs are persistent (two per SM, bound by the 256 TMEM columns
// each takes) and hold the B matrices of D for the whole launch; G of the
// element and u of the next one are prefetched into L2.
//
// Every mbarrier wait is bounded (~2 s of global time).  A wait that runs out
// sets a device flag, writes NaN into every output of the CTA's remaining
// elements, waits once more for the MMAs in flight, frees the CTA's TMEM and
// returns.
#include <cuda_bf16.h>

#include "nek_ff.cuh"
#include "nek_internal.h"
#include "nek_tc5.cuh"

namespace nek {

namespace {

constexpr int kNT = 256;               // 8 warps; warps w and w + 4 share TMEM lanes 32 (w mod 4) ..
constexpr int kLbo = 144;              // A: bytes between K-adjacent core matrices
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitNs = 2000000000LL;

__device__ int g_ax_oz_timeout = 0;    // set by a bounded wait that ran out

// Modes: the plain operator; with element energies u_e . w_e; with the CG direction update on the input
// (x += alpha p, p = minv r + beta p, the operator applied to the new p) and the energies p_e . w_e.
constexpr int kOzPlain = 0, kOzEnergy = 1, kOzDir = 2;

// The direction update's scalars, read once per launch.
struct OzDir {
    double alpha, beta;
    bool dx, dp;  // x is updated; p is replaced
};

template <int NX>
struct Oz {
    static_assert(NX % 2 == 0 && NX >= 2 && NX <= 10, "even nx up to 10");
    static constexpr int N2 = NX * NX, N3 = N2 * NX, NPP = N3 / 2;
    static constexpr int NCOL = 8 * NX;        // MMA N and TMEM columns per direction
    static constexpr int KSTEP = NX / 2;       // MMAs per direction (K = 8 NX, 16 per MMA)
    static constexpr int SBO = NX * kLbo;      // A: bytes between 8-row groups
    static constexpr int ABYTES = 16 * SBO;    // A: 128 rows of one direction
    static constexpr int BSBO = NX * 128;      // B: bytes between 8-row groups
    static constexpr int BBYTES = NX * NX * 128;
    static constexpr int NPR = (NPP + kNT - 1) / kNT;  // point pairs per thread
    static constexpr uint32_t IDESC = tc5::idesc_bf16_f32(128, NCOL);
    // exchange arrays over the A buffers: phase 1 [3][NPP] float4, phase 2 [3][NPP] float4 + [3][NPP] float2
    static_assert(3 * NPP * 24 <= 3 * ABYTES, "exchange fits over the A buffers");
    static_assert(3 * ABYTES <= 16 * 65536, "digit-row offsets / 16 fit 16 bits");
};

struct OzMisc {
    unsigned long long mbar;
    uint32_t tmem;
    int ed;            // D < 2^ed
    float sig[2];      // recombination offsets of phase 1 and phase 2
    float red[2][8];   // per-warp maxima: [0] |u|, [1] |wr|, |ws|, |wt|
    int flag[2];       // a wait of phase 1 / phase 2 ran out
    double rs[10], cs[10];  // absolute row / column sums of D
    double esum[8];         // per-warp parts of an element's energy
};

template <int NX>
constexpr size_t oz_smem_bytes()
{
    // at least 80 KB, so that at most two CTAs (2 x 256 TMEM columns) share an SM
    constexpr size_t need = 3 * (size_t)Oz<NX>::ABYTES + 2 * (size_t)Oz<NX>::BBYTES + sizeof(OzMisc);
    return need > 81920 ? need : 81920;
}

// ---------------------------------------------------------------- f32x2 arithmetic
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sp2(float x) { return make_float2(x, x); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e)
{
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void df_mul2(float2 ah, float2 al, float2 bh, float2 bl, float2& p, float2& e)
{
    p = mul2(ah, bh);
    e = fma2(ah, bh, make_float2(-p.x, -p.y));
    e = fma2(ah, bl, e);
    e = fma2(al, bh, e);
}
// (ah,al)(xh,xl) + (bh,bl)(yh,yl) + (ch,cl)(zh,zl) as an unevaluated pair.
__device__ __forceinline__ void df_dot3_2(float2 ah, float2 al, float2 xh, float2 xl, float2 bh, float2 bl, float2 yh,
                                          float2 yl, float2 ch, float2 cl, float2 zh, float2 zl, float2& h, float2& l)
{
    float2 p1, e1, p2, e2, p3, e3, s, f1, f2;
    df_mul2(ah, al, xh, xl, p1, e1);
    df_mul2(bh, bl, yh, yl, p2, e2);
    df_mul2(ch, cl, zh, zl, p3, e3);
    two_sum2(p1, p2, s, f1);
    two_sum2(s, p3, h, f2);
    l = add2(add2(add2(e1, e2), add2(e3, f1)), f2);
}

// ---------------------------------------------------------------- digits
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float2 add_(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 sub_(float2 a, float2 b) { return sub2(a, b); }
template <class T>
__device__ __forceinline__ T spl(float x);
template <>
__device__ __forceinline__ float spl<float>(float x) { return x; }
template <>
__device__ __forceinline__ float2 spl<float2>(float x) { return make_float2(x, x); }

// y + yl (|y + yl| < ~1, |yl| <= ulp(y) / 2) -> q_0..q_5 on the grids 2^-8, ..., 2^-48:
// round-to-grid by adding and subtracting 1.5 * 2^(23 - 8(a+1)); the remainders are exact.
template <class T>
__device__ __forceinline__ void digits6(T y, T yl, T (&q)[6])
{
    const T c0 = spl<T>(49152.f), c1 = spl<T>(192.f), c2 = spl<T>(0.75f), c3 = spl<T>(0.0029296875f),
            c4 = spl<T>(1.1444091796875e-05f), c5 = spl<T>(4.470348358154296875e-08f);
    q[0] = sub_(add_(y, c0), c0);
    y = sub_(y, q[0]);
    q[1] = sub_(add_(y, c1), c1);
    y = sub_(y, q[1]);
    q[2] = sub_(add_(y, c2), c2);
    y = sub_(y, q[2]);
    y = add_(y, yl);
    q[3] = sub_(add_(y, c3), c3);
    y = sub_(y, q[3]);
    q[4] = sub_(add_(y, c4), c4);
    y = sub_(y, q[4]);
    q[5] = sub_(add_(y, c5), c5);
}

// Digits are exact BF16 values: the upper 16 bits of their FP32 encoding.
__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi)
{
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
// The 16-byte digit rows of the two points of a packed pair.
__device__ __forceinline__ void digit_rows(const float2 (&q)[6], uint4& r0, uint4& r1)
{
    r0 = make_uint4(bf16_pair(q[0].x, q[1].x), bf16_pair(q[2].x, q[3].x), bf16_pair(q[4].x, q[5].x), 0u);
    r1 = make_uint4(bf16_pair(q[0].y, q[1].y), bf16_pair(q[2].y, q[3].y), bf16_pair(q[4].y, q[5].y), 0u);
}

// |m| < 2^return (0 for m == 0); m >= 0.
__device__ __forceinline__ int exp_bound(float m)
{
    if (m == 0.f) return 0;
    const int e = (int)((__float_as_uint(m) >> 23) & 0xFF);
    return (e > 0 ? e : 1) - 126;
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }  // -126..127

// (double)f * 2^X through the bit pattern (f normal; zero and FP32-denormal give 0).
__device__ __forceinline__ double widen_scaled(float f, int X)
{
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7FFFFFFFu;
    if (a < 0x00800000u) return 0.0;
    const unsigned hi = (u & 0x80000000u) | (((a >> 23) + 896u + (unsigned)X) << 20) | ((a & 0x7FFFFFu) >> 3);
    const unsigned lo = (a & 0x7u) << 29;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// Max over the CTA of non-negative v (one barrier); red: 8 floats of shared memory.
__device__ __forceinline__ float block_max(float v, float* red)
{
    const unsigned x = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(v));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __uint_as_float(x);
    __syncthreads();
    float m = red[0];
#pragma unroll
    for (int q = 1; q < kNT / 32; q++) m = fmaxf(m, red[q]);
    return m;
}

// Byte offset of (row, chunk) in one direction's A buffer.
template <int NX>
__host__ __device__ constexpr int a_off(int row, int chunk)
{
    return (row >> 3) * Oz<NX>::SBO + chunk * kLbo + (row & 7) * 16;
}

// Packed recombination of two outputs (lanes .x, .y) from their levels x[0..7]:
// hi (multiple of ulp(sig)), E (exact), s (levels 4..7).
__device__ __forceinline__ void recombine(const float2 (&x)[8], float2 sig, float2& hi, float2& E, float2& s)
{
    const float2 t0 = add2(x[0], sig);
    const float2 t1 = add2(t0, x[1]);
    const float2 e1 = sub2(x[1], sub2(t1, t0));
    const float2 t2 = add2(t1, x[2]);
    const float2 e2 = sub2(x[2], sub2(t2, t1));
    const float2 t3 = add2(t2, x[3]);
    const float2 e3 = sub2(x[3], sub2(t3, t2));
    hi = sub2(t3, sig);
    E = add2(add2(e1, e2), e3);
    s = add2(x[6], x[7]);
    s = add2(x[5], s);
    s = add2(x[4], s);
}

// Recombine this lane's TMEM lane m (line m of every direction) into the exchange
// arrays, indexed by point pair: phase 1 XA[d][pp] = (S(p), S(p+1), lo(p), lo(p+1)),
// phase 2 XA[d][pp] = (hi, hi, E, E) and XS[d][pp] = (s, s).  The two warps of a
// lane range take alternate 32-column blocks (HALF: which), one TMEM wait per
// block; warps whose lanes hold no line return at once (warp-uniform).
template <int NX, bool PHASE2, int HALF>
__device__ __forceinline__ void readout(uint32_t lane_addr, float sig, unsigned char* __restrict__ X, int m)
{
    using C = Oz<NX>;
    constexpr int N2 = C::N2, NPP = C::NPP, NCOL = C::NCOL;
    constexpr int NCH = 3 * NCOL / 16;  // 16-column chunks over the three directions
    if ((m & ~31) >= N2) return;
    const float2 s2 = sp2(sig);
    float4* XA = reinterpret_cast<float4*>(X);
    float* XAf = reinterpret_cast<float*>(X);
    float* XSf = reinterpret_cast<float*>(X + 3 * NPP * 16);
    const bool valid = m < N2;
    // lane m's lines: r (j,k) = m; s (i,k) = m; t (i,j) = m
    const int pr = NX * m, ps = (m % NX) + N2 * (m / NX), pt = m;
#pragma unroll
    for (int ch = HALF; ch < NCH; ch += 2) {
        const int d = (16 * ch) / NCOL, o = 2 * (((16 * ch) % NCOL) / 16);  // outputs o, o + 1 of direction d
        uint32_t r[16];
        tc5::tmem_ld16(lane_addr + (uint32_t)(16 * ch), r);
        float2 x[8];
#pragma unroll
        for (int L = 0; L < 8; L++) x[L] = make_float2(__uint_as_float(r[2 * L]), __uint_as_float(r[2 * L + 1]));
        float2 hi, E, sm;
        recombine(x, s2, hi, E, sm);
        float2 A0, A1;  // phase 1: S, lo; phase 2: hi, E
        if (!PHASE2) {
            // Fast2Sum(hi, E) -> (S, T); the pair (S, T + s)
            A0 = add2(hi, E);
            A1 = add2(sub2(E, sub2(A0, hi)), sm);
        } else {
            A0 = hi;
            A1 = E;
        }
        if (!valid) continue;
        if (d == 0) {
            // line (j,k) = m: outputs o, o + 1 are the two points of pair (o + NX m) / 2
            const int pp = (o + pr) >> 1;
            XA[pp] = make_float4(A0.x, A0.y, A1.x, A1.y);
            if (PHASE2) reinterpret_cast<float2*>(XSf)[pp] = sm;
        } else {
            // s: points (i, o, k), (i, o + 1, k); t: points (i, j, o), (i, j, o + 1); each is lane i mod 2 of its
            // pair
            const int p0 = d == 1 ? ps + NX * o : pt + N2 * o;
            const int p1 = p0 + (d == 1 ? NX : N2);
            const int b0 = 4 * (d * NPP + (p0 >> 1)) + (p0 & 1), b1 = 4 * (d * NPP + (p1 >> 1)) + (p1 & 1);
            XAf[b0] = A0.x;
            XAf[b0 + 2] = A1.x;
            XAf[b1] = A0.y;
            XAf[b1 + 2] = A1.y;
            if (PHASE2) {
                XSf[2 * (d * NPP + (p0 >> 1)) + (p0 & 1)] = sm.x;
                XSf[2 * (d * NPP + (p1 >> 1)) + (p1 & 1)] = sm.y;
            }
        }
    }
}

// One thread waits for the commit of the MMAs; a barrier hands the outcome to the CTA.
__device__ __forceinline__ bool cta_wait_mma(uint32_t mbar, uint32_t parity, long long wait_ns, int* flag)
{
    if (threadIdx.x == 0) *flag = tc5::mbar_wait_bounded(mbar, parity, wait_ns) ? 0 : 1;
    __syncthreads();
    return *flag == 0;
}

// Stage 1: element e's input as float pairs of this thread's point pairs (lane .x: point 2 pp, .y: 2 pp + 1)
// and the element's exponent bound (one barrier).  With the direction update the input is the new p: each
// point does x += alpha p (old p) and p = minv r + beta p with the operations of the CG's own update, and
// writes both back.
template <int NX, int MODE>
__device__ __forceinline__ int load_u(const double* __restrict__ u, int64_t e, int tid, float2 (&uh)[Oz<NX>::NPR],
                                      float2 (&ul)[Oz<NX>::NPR], float* red, const DirUpdate& dir, const OzDir& dv)
{
    using C = Oz<NX>;
    constexpr int NPR = C::NPR;
    const int64_t first = e * C::N3;
    double2 v[NPR];
    if constexpr (MODE == kOzDir) {
        // all loads before the first store (the arrays may alias as far as the compiler knows)
        double2* p2 = reinterpret_cast<double2*>(dir.p + first);
        double2* x2 = reinterpret_cast<double2*>(dir.x + first);
        double2 rv[NPR], mv[NPR], xv[NPR];
#pragma unroll
        for (int q = 0; q < NPR; q++) {
            const int pp = tid + kNT * q < C::NPP ? tid + kNT * q : 0;
            v[q] = p2[pp];
            rv[q] = reinterpret_cast<const double2*>(dir.r + first)[pp];
            mv[q] = reinterpret_cast<const double2*>(dir.minv + first)[pp];
            xv[q] = dv.dx ? x2[pp] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int q = 0; q < NPR; q++) {
            const int pp = tid + kNT * q;
            if (pp < C::NPP) {
                if (dv.dx) x2[pp] = make_double2(fma(dv.alpha, v[q].x, xv[q].x), fma(dv.alpha, v[q].y, xv[q].y));
                if (dv.dp) {
                    v[q] = make_double2(fma(dv.beta, v[q].x, mv[q].x * rv[q].x),
                                        fma(dv.beta, v[q].y, mv[q].y * rv[q].y));
                    p2[pp] = v[q];
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < NPR; q++) {
            const int pp = tid + kNT * q < C::NPP ? tid + kNT * q : 0;
            v[q] = __ldg(reinterpret_cast<const double2*>(u + first) + pp);
        }
    }
    float mu = 0.f;
#pragma unroll
    for (int q = 0; q < NPR; q++) {
        float2 a = make_float2(0.f, 0.f), b = a;
        if (tid + kNT * q < C::NPP) {
            a = split_double(v[q].x);
            b = split_double(v[q].y);
        }
        uh[q] = make_float2(a.x, b.x);
        ul[q] = make_float2(a.y, b.y);
        mu = fmaxf(mu, fmaxf(fabsf(a.x), fabsf(b.x)));
    }
    return exp_bound(block_max(mu, red));
}

// Issued by the whole of warp 0 (converged); lane 0 alone issues each MMA and the commit.
template <int NX>
__device__ __forceinline__ void issue_phase(uint32_t tmem, uint32_t a_base, uint32_t b_base, uint32_t mbar)
{
    using C = Oz<NX>;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const uint64_t ad = tc5::smem_desc(a_base + (uint32_t)(d * C::ABYTES), kLbo, C::SBO);
        const uint64_t bd = tc5::smem_desc(b_base, 128, C::BSBO);
#pragma unroll
        for (int s = 0; s < C::KSTEP; s++)
            tc5::mma_bf16_lane0(tmem + (uint32_t)(d * C::NCOL), ad + (uint64_t)((2 * s * kLbo) >> 4),
                                bd + (uint64_t)((2 * s * 128) >> 4), C::IDESC, s > 0 ? 1u : 0u);
    }
    tc5::mma_commit_lane0(mbar);
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// arrivals: arrivals the mbarrier expects per phase (1: the commit of the MMAs;
// 2 never completes, which the self-test uses to make every wait run out).
template <int NX, int MODE>
__global__ void __launch_bounds__(kNT, 2)
    k_ax_oz(int64_t nelt, const double* __restrict__ D, const float4* __restrict__ Goz,
            const double* __restrict__ u, double* __restrict__ w, double* __restrict__ edot, DirUpdate dir,
            long long wait_ns, int arrivals)
{
    using C = Oz<NX>;
    constexpr int N2 = C::N2, N3 = C::N3, NPP = C::NPP, NPR = C::NPR;
    extern __shared__ __align__(128) unsigned char oz_raw[];
    unsigned char* A = oz_raw;                        // [3][ABYTES] digit rows; between MMAs the exchange arrays
    unsigned char* B1 = A + 3 * C::ABYTES;            // phase 1: digits of D
    unsigned char* B2 = B1 + C::BBYTES;               // phase 2: digits of D^T
    OzMisc& M = *reinterpret_cast<OzMisc*>(B2 + C::BBYTES);
    const float4* XA = reinterpret_cast<const float4*>(A);
    const float2* XS = reinterpret_cast<const float2*>(A + 3 * NPP * 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- set-up: D's exponent bound, recombination offsets, the B matrices, mbarrier, TMEM
    if (tid < NX) {
        double r = 0.0, c = 0.0;
        for (int l = 0; l < NX; l++) {
            r += fabs(D[tid * NX + l]);
            c += fabs(D[l * NX + tid]);
        }
        M.rs[tid] = r;
        M.cs[tid] = c;
    }
    __syncthreads();
    if (tid == 0) {
        double dmax = 0.0, rmax = 0.0, cmax = 0.0;
        for (int q = 0; q < N2; q++) dmax = fmax(dmax, fabs(D[q]));
        for (int q = 0; q < NX; q++) {
            rmax = fmax(rmax, M.rs[q]);
            cmax = fmax(cmax, M.cs[q]);
        }
        int ed = 0;
        frexp(dmax, &ed);  // dmax < 2^ed
        M.ed = ed;
        // bound on any partial sum of levels, in level-0 grid units: 2^16 sum_l (|y| + 2^-8)(|D|/2^ed + 2^-8)
        for (int ph = 0; ph < 2; ph++) {
            const double b = 65536.0 * 1.005 * (ldexp(ph == 0 ? rmax : cmax, -ed) + NX * 0.005);
            int k = 0;
            frexp(b, &k);  // b < 2^k: sigma = 1.5 * 2^(k+1) keeps sigma +- b in one binade
            M.sig[ph] = (float)ldexp(1.5, k + 1);
        }
        tc5::mbar_init(tc5::smem_u32(&M.mbar), arrivals);
    }
    __syncthreads();
    for (int q = tid; q < N2; q += kNT) {
        const int r = q / NX, c = q % NX;
        const float2 hl = split_double(ldexp(D[q], -M.ed));
        float p[6];
        digits6(hl.x, hl.y, p);
#pragma unroll
        for (int L = 0; L < 8; L++) {
            float v[8];
#pragma unroll
            for (int a = 0; a < 8; a++) v[a] = (a < 6 && L - a >= 0 && L - a < 6) ? __fmul_rn(p[L - a], 65536.f) : 0.f;
            const uint4 row = make_uint4(bf16_pair(v[0], v[1]), bf16_pair(v[2], v[3]), bf16_pair(v[4], v[5]),
                                         bf16_pair(v[6], v[7]));
            // phase 1: output o = r, K chunk l = c; phase 2: o = c, l = r
            const int n1 = 16 * (r >> 1) + 2 * L + (r & 1), n2 = 16 * (c >> 1) + 2 * L + (c & 1);
            *reinterpret_cast<uint4*>(B1 + (n1 >> 3) * C::BSBO + c * 128 + (n1 & 7) * 16) = row;
            *reinterpret_cast<uint4*>(B2 + (n2 >> 3) * C::BSBO + r * 128 + (n2 & 7) * 16) = row;
        }
    }
    if (warp == 0) tc5::tmem_alloc(&M.tmem, kTmemCols);
    tc5::fence_async_smem();
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tmem = M.tmem;
    const uint32_t mbar = tc5::smem_u32(&M.mbar);
    const uint32_t a_base = tc5::smem_u32(A), b1 = tc5::smem_u32(B1), b2 = tc5::smem_u32(B2);
    const int m = 32 * (warp & 3) + lane, half = warp >> 2;  // TMEM lane (= line) of this thread
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const int ed = M.ed;
    const float sig1 = M.sig[0], sig2 = M.sig[1];
    OzDir dv{0.0, 0.0, false, false};
    if constexpr (MODE == kOzDir) {
        dv.alpha = dir.sc->alpha;
        dv.beta = dir.sc->beta;
        dv.dx = dir.sc->xpend != 0;
        dv.dp = !(dir.sc->done || dir.sc->status != NEK_OK);
    }
    // this thread's point pairs pp = tid + kNT q (points 2 pp, 2 pp + 1: i even, i + 1 on the same lines
    // of the r direction): byte offsets / 16 of their digit rows in the three A buffers, two to a word
    uint32_t offw[NPR][3];
#pragma unroll
    for (int q = 0; q < NPR; q++) {
        const int pp = tid + kNT * q;
        const int p = 2 * (pp < NPP ? pp : 0);
        const int i = p % NX, j = (p / NX) % NX, k = p / N2;
        const int o[6] = {a_off<NX>(j + NX * k, i), a_off<NX>(j + NX * k, i + 1),
                          C::ABYTES + a_off<NX>(i + NX * k, j), C::ABYTES + a_off<NX>(i + 1 + NX * k, j),
                          2 * C::ABYTES + a_off<NX>(i + NX * j, k), 2 * C::ABYTES + a_off<NX>(i + 1 + NX * j, k)};
#pragma unroll
        for (int d = 0; d < 3; d++) offw[q][d] = (uint32_t)(o[2 * d] >> 4) | ((uint32_t)(o[2 * d + 1] >> 4) << 16);
    }
    uint32_t parity = 0;
    // stage 1 of the first element: u as float pairs of point pairs, the element's exponent bound
    float2 uh[NPR], ul[NPR];
    int eu = 0;
    if ((int64_t)blockIdx.x < nelt) {
        for (int q = tid; q < (48 * N3 + 127) / 128; q += kNT)
            prefetch_l2(reinterpret_cast<const unsigned char*>(Goz + blockIdx.x * (int64_t)NPP * 6) + 128 * q);
        eu = load_u<NX, MODE>(u, blockIdx.x, tid, uh, ul, M.red[0], dir, dv);
    }

    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        const float4* Ge = Goz + e * (int64_t)NPP * 6;
        const int64_t en = e + gridDim.x;  // this CTA's next element
        // ---- stage 2: u's digit rows into the three A buffers
        {
            const float2 su = sp2(pow2f(-eu));
#pragma unroll
            for (int q = 0; q < NPR; q++) {
                if (tid + kNT * q < NPP) {
                    float2 dg[6];
                    digits6(mul2(uh[q], su), mul2(ul[q], su), dg);
                    uint4 r0, r1;
                    digit_rows(dg, r0, r1);
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        *reinterpret_cast<uint4*>(A + ((offw[q][d] & 0xFFFFu) << 4)) = r0;
                        *reinterpret_cast<uint4*>(A + ((offw[q][d] >> 16) << 4)) = r1;
                    }
                }
            }
        }
        // ---- phase-1 MMAs
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
        if (warp == 0) {
            issue_phase<NX>(tmem, a_base, b1, mbar);
            __syncwarp();
        }
        // while the MMAs run: G of the first point pair into registers, u of the next element into L2
        float4 g0[6];
        if (tid < NPP) {
#pragma unroll
            for (int c = 0; c < 6; c++) g0[c] = __ldg(Ge + 6 * tid + c);
        }
        if (en < nelt) {
            const double* nxt = MODE == kOzDir ? dir.p : u;
            for (int q = tid; q < (8 * N3 + 127) / 128; q += kNT) {
                prefetch_l2(reinterpret_cast<const unsigned char*>(nxt + en * N3) + 128 * q);
                if constexpr (MODE == kOzDir) {
                    prefetch_l2(reinterpret_cast<const unsigned char*>(dir.r + en * N3) + 128 * q);
                    prefetch_l2(reinterpret_cast<const unsigned char*>(dir.minv + en * N3) + 128 * q);
                    if (dv.dx) prefetch_l2(reinterpret_cast<const unsigned char*>(dir.x + en * N3) + 128 * q);
                }
            }
        }
        if (!cta_wait_mma(mbar, parity, wait_ns, &M.flag[0])) goto timed_out;
        parity ^= 1u;
        tc5::fence_after();
        // ---- stage 3: levels -> (S, lo) pairs of ur, us, ut in XA (the A buffers are free again)
        if (half)
            readout<NX, false, 1>(lane_addr, sig1, A, m);
        else
            readout<NX, false, 0>(lane_addr, sig1, A, m);
        tc5::fence_before();
        __syncthreads();
        // ---- stage 4: (wr, ws, wt) = G (ur, us, ut) in float-float, renormalised
        {
            float2 wh[3][NPR], wl[3][NPR];
            float mw = 0.f;
#pragma unroll
            for (int q = 0; q < NPR; q++) {
                const int pp = tid + kNT * q;
                if (pp < NPP) {
                    float4 x[3], g[6];
#pragma unroll
                    for (int d = 0; d < 3; d++) x[d] = XA[d * NPP + pp];
#pragma unroll
                    for (int c = 0; c < 6; c++) g[c] = q == 0 ? g0[c] : __ldg(Ge + 6 * pp + c);
                    // g[c] = (G_c hi of p, p + 1; G_c lo of p, p + 1); x[d] = (S of p, p + 1; lo of p, p + 1)
#define OZ_H(v) make_float2((v).x, (v).y)
#define OZ_L(v) make_float2((v).z, (v).w)
                    df_dot3_2(OZ_H(g[0]), OZ_L(g[0]), OZ_H(x[0]), OZ_L(x[0]), OZ_H(g[1]), OZ_L(g[1]), OZ_H(x[1]),
                              OZ_L(x[1]), OZ_H(g[2]), OZ_L(g[2]), OZ_H(x[2]), OZ_L(x[2]), wh[0][q], wl[0][q]);
                    df_dot3_2(OZ_H(g[1]), OZ_L(g[1]), OZ_H(x[0]), OZ_L(x[0]), OZ_H(g[3]), OZ_L(g[3]), OZ_H(x[1]),
                              OZ_L(x[1]), OZ_H(g[4]), OZ_L(g[4]), OZ_H(x[2]), OZ_L(x[2]), wh[1][q], wl[1][q]);
                    df_dot3_2(OZ_H(g[2]), OZ_L(g[2]), OZ_H(x[0]), OZ_L(x[0]), OZ_H(g[4]), OZ_L(g[4]), OZ_H(x[1]),
                              OZ_L(x[1]), OZ_H(g[5]), OZ_L(g[5]), OZ_H(x[2]), OZ_L(x[2]), wh[2][q], wl[2][q]);
#undef OZ_H
#undef OZ_L
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        // renormalise: after cancellation among the three products the low part can exceed
                        // ulp(high), and the digits need |low| <= ulp(high) / 2 to stay within 8 bits
                        two_sum2(wh[d][q], wl[d][q], wh[d][q], wl[d][q]);
                        mw = fmaxf(mw, fmaxf(fabsf(wh[d][q].x), fabsf(wh[d][q].y)));
                    }
                }
            }
            const int ew = exp_bound(block_max(mw, M.red[1]));  // after this barrier XA is no longer read
            const int eu_e = eu;  // stage 1 of the next element replaces eu below
            // ---- stage 5: digit rows of wr -> A_r, ws -> A_s, wt -> A_t
            const float2 sw = sp2(pow2f(-ew));
#pragma unroll
            for (int q = 0; q < NPR; q++) {
                if (tid + kNT * q < NPP) {
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        float2 dg[6];
                        digits6(mul2(wh[d][q], sw), mul2(wl[d][q], sw), dg);
                        uint4 r0, r1;
                        digit_rows(dg, r0, r1);
                        *reinterpret_cast<uint4*>(A + ((offw[q][d] & 0xFFFFu) << 4)) = r0;
                        *reinterpret_cast<uint4*>(A + ((offw[q][d] >> 16) << 4)) = r1;
                    }
                }
            }
            // ---- phase-2 MMAs
            tc5::fence_async_smem();
            tc5::fence_before();
            __syncthreads();
            tc5::fence_after();
            if (warp == 0) {
                issue_phase<NX>(tmem, a_base, b2, mbar);
                __syncwarp();
            }
            // while the MMAs run: stage 1 of the next element, and its G into L2
            if (en < nelt) {
                for (int q = tid; q < (48 * N3 + 127) / 128; q += kNT)
                    prefetch_l2(reinterpret_cast<const unsigned char*>(Goz + en * (int64_t)NPP * 6) + 128 * q);
                eu = load_u<NX, MODE>(u, en, tid, uh, ul, M.red[0], dir, dv);
            }
            if (!cta_wait_mma(mbar, parity, wait_ns, &M.flag[1])) goto timed_out;
            parity ^= 1u;
            tc5::fence_after();
            // ---- stage 6: levels -> (hi, E, s) of the three directions in XA, XS
            if (half)
                readout<NX, true, 1>(lane_addr, sig2, A, m);
            else
                readout<NX, true, 0>(lane_addr, sig2, A, m);
            tc5::fence_before();
            __syncthreads();
            // ---- stage 7: w = (his + Es + ss of the three directions) * 2^(eu + ew + 2 ed - 32); the his
            // and the Es sum exactly, TwoSum joins them
            const int xs = eu_e + ew + 2 * ed - 32;
            double2* we = reinterpret_cast<double2*>(w + e * N3);
            double energy = 0.0;  // this thread's part of the element's input . w, in a fixed order
            double2 iv[NPR];      // the input at this thread's points (u, or the p written in stage 1), loaded
                                  // before any store of w, which the compiler cannot order past them
            if constexpr (MODE != kOzPlain) {
#pragma unroll
                for (int q = 0; q < NPR; q++) {
                    const int pp = tid + kNT * q < NPP ? tid + kNT * q : 0;
                    iv[q] = MODE == kOzDir ? reinterpret_cast<const double2*>(dir.p + e * N3)[pp]
                                           : __ldg(reinterpret_cast<const double2*>(u + e * N3) + pp);
                }
            }
#pragma unroll
            for (int q = 0; q < NPR; q++) {
                const int pp = tid + kNT * q;
                if (pp < NPP) {
                    const float4 a = XA[pp], b = XA[NPP + pp], c = XA[2 * NPP + pp];
                    const float2 sa = XS[pp], sb = XS[NPP + pp], sc = XS[2 * NPP + pp];
                    const float2 H = add2(add2(make_float2(a.x, a.y), make_float2(b.x, b.y)), make_float2(c.x, c.y));
                    const float2 Es = add2(add2(make_float2(a.z, a.w), make_float2(b.z, b.w)), make_float2(c.z, c.w));
                    const float2 ss = add2(add2(sa, sb), sc);
                    float2 S, T;
                    two_sum2(H, Es, S, T);
                    const float2 lo = add2(T, ss);
                    const double2 wv = make_double2(__dadd_rn(widen_scaled(S.x, xs), widen_scaled(lo.x, xs)),
                                                    __dadd_rn(widen_scaled(S.y, xs), widen_scaled(lo.y, xs)));
                    we[pp] = wv;
                    if constexpr (MODE != kOzPlain) {
                        energy = fma(iv[q].x, wv.x, energy);
                        energy = fma(iv[q].y, wv.y, energy);
                    }
                }
            }
            if constexpr (MODE != kOzPlain) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) energy += __shfl_xor_sync(0xFFFFFFFFu, energy, o);
                if (lane == 0) M.esum[warp] = energy;
            }
            __syncthreads();  // the exchange arrays are read before the next element's digits overwrite them
            if constexpr (MODE != kOzPlain) {
                if (tid == 0) {
                    double t = 0.0;
#pragma unroll
                    for (int q = 0; q < kNT / 32; q++) t += M.esum[q];
                    edot[e] = t;
                }
            }
        }
        continue;
    timed_out:
        // a wait ran out: flag it, poison the outputs this CTA still owes, wait once more for
        // the MMAs in flight, then leave the element loop (TMEM is freed below)
        if (tid == 0) atomicExch(&g_ax_oz_timeout, 1);
        for (int64_t e2 = e; e2 < nelt; e2 += gridDim.x)
            for (int p = tid; p < N3; p += kNT) w[e2 * N3 + p] = __longlong_as_double(0x7FF8000000000000LL);
        if (tid == 0) tc5::mbar_wait_bounded(mbar, parity, wait_ns);
        __syncthreads();
        break;
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (warp == 0) tc5::tmem_dealloc(tmem, kTmemCols);
}

// G (FP64, [e][p][6]) -> pairs of points interleaved: Goz[e][pp][c] = (hi of G_c at
// points 2 pp and 2 pp + 1, lo at the same two points), split as split_double does.
__global__ void k_g_to_oz(int64_t nq, const double* __restrict__ G, float4* __restrict__ Goz)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pp = q / 6;
        const int c = (int)(q - 6 * pp);
        const float2 a = split_double(G[12 * pp + c]), b = split_double(G[12 * pp + 6 + c]);
        Goz[q] = make_float4(a.x, b.x, a.y, b.y);
    }
}

int oz_sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                      cudaSuccess && v > 0)
            n = v;
        else
            n = 152;
    }
    return n;
}

template <int NX, int MODE>
nek_status launch_oz_mode(int64_t nelt, const double* D, const float* Goz, const double* u, double* w, double* edot,
                          const DirUpdate& dir, cudaStream_t s, long long wait_ns, int arrivals)
{
    static std::atomic<uint64_t> configured{0};
    constexpr size_t smem = oz_smem_bytes<NX>();
    nek_status st = ensure_dyn_smem(k_ax_oz<NX, MODE>, smem, configured);
    if (st != NEK_OK) return st;
    const int64_t cap = 2 * (int64_t)oz_sm_count();
    const int grid = static_cast<int>(nelt < cap ? nelt : cap);
    k_ax_oz<NX, MODE><<<grid, kNT, smem, s>>>(nelt, D, reinterpret_cast<const float4*>(Goz), u, w, edot, dir, wait_ns,
                                              arrivals);
    return check_launch();
}

template <int NX>
nek_status launch_oz_nx(int64_t nelt, const double* D, const float* Goz, const double* u, double* w, double* edot,
                        const DirUpdate* dir, cudaStream_t s, long long wait_ns, int arrivals)
{
    if (dir) return launch_oz_mode<NX, kOzDir>(nelt, D, Goz, u, w, edot, *dir, s, wait_ns, arrivals);
    const DirUpdate none{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (edot) return launch_oz_mode<NX, kOzEnergy>(nelt, D, Goz, u, w, edot, none, s, wait_ns, arrivals);
    return launch_oz_mode<NX, kOzPlain>(nelt, D, Goz, u, w, nullptr, none, s, wait_ns, arrivals);
}

}  // namespace

bool ax_oz_supported(int nx) { return nx >= 2 && nx <= 10 && nx % 2 == 0; }

nek_status launch_ax_oz_ex(int64_t nelt, int nx, const double* D, const float* Goz, const double* u, double* w,
                           cudaStream_t s, long long wait_ns, int arrivals, double* edot, const DirUpdate* dir)
{
    switch (nx) {
        case 2: return launch_oz_nx<2>(nelt, D, Goz, u, w, edot, dir, s, wait_ns, arrivals);
        case 4: return launch_oz_nx<4>(nelt, D, Goz, u, w, edot, dir, s, wait_ns, arrivals);
        case 6: return launch_oz_nx<6>(nelt, D, Goz, u, w, edot, dir, s, wait_ns, arrivals);
        case 8: return launch_oz_nx<8>(nelt, D, Goz, u, w, edot, dir, s, wait_ns, arrivals);
        case 10: return launch_oz_nx<10>(nelt, D, Goz, u, w, edot, dir, s, wait_ns, arrivals);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
}

nek_status launch_ax_oz(int64_t nelt, int nx, const double* D, const float* Goz, const double* u, double* w,
                        cudaStream_t s, double* edot, const DirUpdate* dir)
{
    return launch_ax_oz_ex(nelt, nx, D, Goz, u, w, s, kWaitNs, 1, edot, dir);
}

// Reads and clears the flag that a bounded wait of the kernel ran out (synchronous).
nek_status ax_oz_take_timeout(bool* was_set)
{
    int v = 0;
    const int zero = 0;
    nek_status st = check_cuda(cudaMemcpyFromSymbol(&v, g_ax_oz_timeout, sizeof(int)));
    if (st == NEK_OK && v) st = check_cuda(cudaMemcpyToSymbol(g_ax_oz_timeout, &zero, sizeof(int)));
    *was_set = v != 0;
    return st;
}

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_geom_oz(int64_t nelt, int nx, const double* G, float* Goz, void* stream)
{
    if (!ax_oz_supported(nx)) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!G || !Goz || !is_aligned(G, 8) || !is_aligned(Goz, 16)) return NEK_ERR_INVALID_ARG;
    const int64_t npts = nelt * (int64_t)nx * nx * nx;
    if (ranges_overlap(G, sizeof(double) * 6 * npts, Goz, sizeof(float) * 12 * npts)) return NEK_ERR_INVALID_ARG;
    const int64_t nq = npts / 2 * 6;
    const int64_t nb = (nq + 255) / 256;
    const int blocks = static_cast<int>(nb < 152 * 32 ? nb : 152 * 32);
    k_g_to_oz<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(nq, G, reinterpret_cast<float4*>(Goz));
    return check_launch();
}

nek_status nek_ax_oz(int64_t nelt, int nx, const double* D, const float* Goz, const double* u, double* w,
                     void* stream)
{
    if (!ax_oz_supported(nx)) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Goz || !u || !w || !is_aligned(D, 8) || !is_aligned(Goz, 16) || !is_aligned(u, 16) ||
        !is_aligned(w, 16))
        return NEK_ERR_INVALID_ARG;
    const int64_t npts = nelt * (int64_t)nx * nx * nx;
    if (ranges_overlap(u, sizeof(double) * npts, w, sizeof(double) * npts)) return NEK_ERR_INVALID_ARG;
    return launch_ax_oz(nelt, nx, D, Goz, u, w, static_cast<cudaStream_t>(stream), nullptr, nullptr);
}

nek_status nek_ax_oz_selftest(int force_timeout, int64_t wait_us, int* timed_out)
{
    if (!timed_out || wait_us < 1 || wait_us > 2000000) return NEK_ERR_INVALID_ARG;
    *timed_out = 0;
    bool stale = false;
    nek_status st = ax_oz_take_timeout(&stale);  // clear a flag left by an earlier call
    if (st != NEK_OK) return st;
    // three nx = 4 elements with zero D, G and u: w = 0 unless a wait ran out (then w is NaN)
    constexpr int nx = 4, ne = 3, n3 = nx * nx * nx;
    double* dbuf = nullptr;
    float* gff = nullptr;
    const size_t nd = nx * nx + 2 * (size_t)ne * n3;
    if (check_cuda(cudaMalloc(&dbuf, sizeof(double) * nd)) != NEK_OK) return NEK_ERR_NOMEM;
    if (check_cuda(cudaMalloc(&gff, sizeof(float) * 12 * ne * n3)) != NEK_OK) {
        cudaFree(dbuf);
        return NEK_ERR_NOMEM;
    }
    st = check_cuda(cudaMemset(dbuf, 0, sizeof(double) * nd));
    if (st == NEK_OK) st = check_cuda(cudaMemset(gff, 0, sizeof(float) * 12 * ne * n3));
    double* w = dbuf + nx * nx + ne * n3;
    if (st == NEK_OK)
        st = launch_ax_oz_ex(ne, nx, dbuf, gff, dbuf + nx * nx, w, nullptr, wait_us * 1000LL, force_timeout ? 2 : 1,
                             nullptr, nullptr);
    if (st == NEK_OK) st = check_cuda(cudaDeviceSynchronize());
    bool to = false;
    if (st == NEK_OK) st = ax_oz_take_timeout(&to);
    double w0 = 0.0;
    if (st == NEK_OK) st = check_cuda(cudaMemcpy(&w0, w, sizeof(double), cudaMemcpyDeviceToHost));
    cudaFree(gff);
    cudaFree(dbuf);
    if (st != NEK_OK) return st;
    *timed_out = to ? 1 : 0;
    if (to != (w0 != w0)) return NEK_ERR_CUDA;  // the flag and the poisoned output must agree
    return to ? NEK_ERR_TIMEOUT : NEK_OK;
}

}  // extern "C"
