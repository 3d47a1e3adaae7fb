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
//   B: row n = (output index o, level L), K = (l, a): p_{L-a} of D[o][l]
//     (D[l][o] in phase 2), zero where L - a is not a digit index.
//   Accumulator (TMEM): lane = line, column 8 o + L = level L of output o on
//     the line; the three directions side by side (24 NX of 256 columns).
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
// Stages per element (128 threads; thread m reads TMEM lane m, the line m of
// every direction): the u digits (point-strided, two points per packed f32x2
// lane pair), phase-1 MMAs (one thread issues, committed to an mbarrier),
// recombination into a float-pair exchange array (over the A buffers, whose
// MMAs have completed), the G product (point-strided), its pairs renormalised
// by TwoSum (the digit bound needs |low| <= ulp(high) / 2, which cancellation
// among the three products can break), the digits of wr, ws, wt, phase-2 MMAs, recombination, and the sum of the three directions written
// as doubles.  CTAs are persistent (two per SM, bound by the 256 TMEM columns
// each takes) and hold the B matrices of D for the whole launch.
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

constexpr int kNT = 128;               // 4 warps: one per 32-lane TMEM sub-partition
constexpr int kLbo = 144;              // A: bytes between K-adjacent core matrices
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitNs = 2000000000LL;

__device__ int g_ax_oz_timeout = 0;    // set by a bounded wait that ran out

template <int NX>
struct Oz {
    static_assert(NX % 2 == 0 && NX >= 2 && NX <= 10, "even nx up to 10");
    static constexpr int N2 = NX * NX, N3 = N2 * NX;
    static constexpr int NCOL = 8 * NX;        // MMA N and TMEM columns per direction
    static constexpr int KSTEP = NX / 2;       // MMAs per direction (K = 8 NX, 16 per MMA)
    static constexpr int SBO = NX * kLbo;      // A: bytes between 8-row groups
    static constexpr int ABYTES = 16 * SBO;    // A: 128 rows of one direction
    static constexpr int BSBO = NX * 128;      // B: bytes between 8-row groups
    static constexpr int BBYTES = NX * NX * 128;
    static constexpr int NPAIR = (N3 + 2 * kNT - 1) / (2 * kNT);  // point pairs per thread
    static constexpr uint32_t IDESC = tc5::idesc_bf16_f32(128, NCOL);
};

struct OzMisc {
    unsigned long long mbar;
    uint32_t tmem;
    int ed;            // D < 2^ed
    float sig[2];      // recombination offsets of phase 1 and phase 2
    float red[2][4];   // per-warp maxima: [0] |u|, [1] |wr|, |ws|, |wt|
    double rs[10], cs[10];  // absolute row / column sums of D
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

// y + yl (|y + yl| < ~1, yl below ulp(y)) -> q_0..q_5 on the grids 2^-8, ..., 2^-48:
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
__device__ __forceinline__ uint4 digit_row(float q0, float q1, float q2, float q3, float q4, float q5)
{
    return make_uint4(bf16_pair(q0, q1), bf16_pair(q2, q3), bf16_pair(q4, q5), 0u);
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

// Max over the CTA of non-negative v (one barrier); red: 4 floats of shared memory.
__device__ __forceinline__ float block_max(float v, float* red)
{
    const unsigned x = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(v));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __uint_as_float(x);
    __syncthreads();
    return fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
}

// Byte offset of (row, chunk) in one direction's A buffer.
template <int NX>
__device__ __forceinline__ int a_off(int row, int chunk)
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

// Thread m (< NX^2) reads its TMEM lane (line m of every direction) and
// recombines the 3 NX outputs: phase 1 stores float pairs X2[d][point], phase 2
// (hi, E, s, 0) in X4[d][point].  Warps with no line return at once
// (warp-uniform); the others load their lanes whole.
template <int NX, bool PHASE2>
__device__ __forceinline__ void readout(uint32_t lane_addr, float sig, unsigned char* __restrict__ X, int m)
{
    using C = Oz<NX>;
    constexpr int N2 = C::N2, N3 = C::N3;
    if ((m & ~31) >= N2) return;
    const float2 s2 = sp2(sig);
    float2* X2 = reinterpret_cast<float2*>(X);
    float4* X4 = reinterpret_cast<float4*>(X);
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int c = 0; c < NX / 2; c++) {
            uint32_t r[16];
            tc5::tmem_ld16(lane_addr + (uint32_t)(d * C::NCOL + 16 * c), r);
            if (m < N2) {
                float2 x[8];
#pragma unroll
                for (int L = 0; L < 8; L++) x[L] = make_float2(__uint_as_float(r[L]), __uint_as_float(r[8 + L]));
                float2 hi, E, sm;
                recombine(x, s2, hi, E, sm);
                const int o = 2 * c;
                // points of outputs o and o + 1 on line m
                const int p = d == 0 ? o + NX * m : d == 1 ? (m % NX) + N2 * (m / NX) + NX * o : m + N2 * o;
                const int step = d == 0 ? 1 : d == 1 ? NX : N2;
                if (!PHASE2) {
                    // Fast2Sum(hi, E) -> (S, T); the pair (S, T + s)
                    const float2 S = add2(hi, E);
                    const float2 lo = add2(sub2(E, sub2(S, hi)), sm);
                    if (d == 0) {
                        *reinterpret_cast<float4*>(X2 + p) = make_float4(S.x, lo.x, S.y, lo.y);
                    } else {
                        X2[d * N3 + p] = make_float2(S.x, lo.x);
                        X2[d * N3 + p + step] = make_float2(S.y, lo.y);
                    }
                } else {
                    X4[d * N3 + p] = make_float4(hi.x, E.x, sm.x, 0.f);
                    X4[d * N3 + p + step] = make_float4(hi.y, E.y, sm.y, 0.f);
                }
            }
        }
    }
}

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
            tc5::mma_bf16(tmem + (uint32_t)(d * C::NCOL), ad + (uint64_t)((2 * s * kLbo) >> 4),
                          bd + (uint64_t)((2 * s * 128) >> 4), C::IDESC, s > 0 ? 1u : 0u);
    }
    tc5::mma_commit(mbar);
}

// arrivals: arrivals the mbarrier expects per phase (1: the commit of the MMAs;
// 2 never completes, which the self-test uses to make every wait run out).
template <int NX>
__global__ void __launch_bounds__(kNT, 2)
    k_ax_oz(int64_t nelt, const double* __restrict__ D, const float4* __restrict__ Gff,
            const double* __restrict__ u, double* __restrict__ w, long long wait_ns, int arrivals)
{
    using C = Oz<NX>;
    constexpr int N2 = C::N2, N3 = C::N3, NPAIR = C::NPAIR;
    extern __shared__ __align__(128) unsigned char oz_raw[];
    unsigned char* A = oz_raw;                        // [3][ABYTES] digit rows; between MMAs the exchange X
    unsigned char* B1 = A + 3 * C::ABYTES;            // phase 1: digits of D
    unsigned char* B2 = B1 + C::BBYTES;               // phase 2: digits of D^T
    OzMisc& M = *reinterpret_cast<OzMisc*>(B2 + C::BBYTES);
    const float2* X = reinterpret_cast<const float2*>(A);  // phase-1 exchange: [3][N3] float pairs
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
            *reinterpret_cast<uint4*>(B1 + r * C::BSBO + c * 128 + L * 16) = row;  // n = (o = r, L), K = (l = c, a)
            *reinterpret_cast<uint4*>(B2 + c * C::BSBO + r * 128 + L * 16) = row;  // n = (o = c, L), K = (l = r, a)
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
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
    const int ed = M.ed;
    const float sig1 = M.sig[0], sig2 = M.sig[1];
    uint32_t parity = 0;

    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        const double* ue = u + e * N3;
        const float4* Ge = Gff + e * (int64_t)N3 * 3;
        // ---- stage 1: u as float pairs (lane .x: point p0, .y: p1 = p0 + 128)
        float2 uh[NPAIR], ul[NPAIR];
        float mu = 0.f;
#pragma unroll
        for (int r = 0; r < NPAIR; r++) {
            const int p0 = tid + 2 * kNT * r, p1 = p0 + kNT;
            const float2 a = p0 < N3 ? split_double(ue[p0]) : make_float2(0.f, 0.f);
            const float2 b = p1 < N3 ? split_double(ue[p1]) : make_float2(0.f, 0.f);
            uh[r] = make_float2(a.x, b.x);
            ul[r] = make_float2(a.y, b.y);
            mu = fmaxf(mu, fmaxf(fabsf(a.x), fabsf(b.x)));
        }
        const int eu = exp_bound(block_max(mu, M.red[0]));
        // ---- stage 2: u's digit rows into the three A buffers
        {
            const float2 su = sp2(pow2f(-eu));
#pragma unroll
            for (int r = 0; r < NPAIR; r++) {
                float2 q[6];
                digits6(mul2(uh[r], su), mul2(ul[r], su), q);
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int p = tid + 2 * kNT * r + kNT * h;
                    if (p < N3) {
                        const uint4 row = h ? digit_row(q[0].y, q[1].y, q[2].y, q[3].y, q[4].y, q[5].y)
                                            : digit_row(q[0].x, q[1].x, q[2].x, q[3].x, q[4].x, q[5].x);
                        const int i = p % NX, j = (p / NX) % NX, k = p / N2;
                        *reinterpret_cast<uint4*>(A + a_off<NX>(j + NX * k, i)) = row;
                        *reinterpret_cast<uint4*>(A + C::ABYTES + a_off<NX>(i + NX * k, j)) = row;
                        *reinterpret_cast<uint4*>(A + 2 * C::ABYTES + a_off<NX>(i + NX * j, k)) = row;
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
            if (lane == 0) issue_phase<NX>(tmem, a_base, b1, mbar);
            __syncwarp();
        }
        bool ok = tc5::mbar_wait_bounded(mbar, parity, wait_ns);
        if (__syncthreads_or(!ok)) goto timed_out;
        parity ^= 1u;
        tc5::fence_after();
        // ---- stage 3: levels -> float pairs ur, us, ut in X (the A buffers are free again)
        readout<NX, false>(lane_addr, sig1, A, tid);
        tc5::fence_before();
        __syncthreads();
        // ---- stage 4: (wr, ws, wt) = G (ur, us, ut) in float-float
        {
            float2 wh[3][NPAIR], wl[3][NPAIR];
            float mw = 0.f;
#pragma unroll
            for (int r = 0; r < NPAIR; r++) {
                const int p0 = tid + 2 * kNT * r, p1 = p0 + kNT;
                float2 a[3][2];  // [direction][lane]: (hi, lo) of ur, us, ut
                float4 g[3][2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int p = h ? p1 : p0;
                    const bool v = p < N3;
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        a[d][h] = v ? X[d * N3 + p] : make_float2(0.f, 0.f);
                        g[d][h] = v ? __ldg(Ge + 3 * p + d) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                // G factors g0..g5 as (hi, lo) pairs: g[0] = (g0h, g0l, g1h, g1l), g[1] = (g2, g3), g[2] = (g4, g5)
                const float2 g0h = make_float2(g[0][0].x, g[0][1].x), g0l = make_float2(g[0][0].y, g[0][1].y);
                const float2 g1h = make_float2(g[0][0].z, g[0][1].z), g1l = make_float2(g[0][0].w, g[0][1].w);
                const float2 g2h = make_float2(g[1][0].x, g[1][1].x), g2l = make_float2(g[1][0].y, g[1][1].y);
                const float2 g3h = make_float2(g[1][0].z, g[1][1].z), g3l = make_float2(g[1][0].w, g[1][1].w);
                const float2 g4h = make_float2(g[2][0].x, g[2][1].x), g4l = make_float2(g[2][0].y, g[2][1].y);
                const float2 g5h = make_float2(g[2][0].z, g[2][1].z), g5l = make_float2(g[2][0].w, g[2][1].w);
                const float2 rh = make_float2(a[0][0].x, a[0][1].x), rl = make_float2(a[0][0].y, a[0][1].y);
                const float2 sh = make_float2(a[1][0].x, a[1][1].x), sl = make_float2(a[1][0].y, a[1][1].y);
                const float2 th = make_float2(a[2][0].x, a[2][1].x), tl = make_float2(a[2][0].y, a[2][1].y);
                df_dot3_2(g0h, g0l, rh, rl, g1h, g1l, sh, sl, g2h, g2l, th, tl, wh[0][r], wl[0][r]);
                df_dot3_2(g1h, g1l, rh, rl, g3h, g3l, sh, sl, g4h, g4l, th, tl, wh[1][r], wl[1][r]);
                df_dot3_2(g2h, g2l, rh, rl, g4h, g4l, sh, sl, g5h, g5l, th, tl, wh[2][r], wl[2][r]);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    // renormalise: after cancellation among the three products the low part can exceed
                    // ulp(high), and the digits need |low| <= ulp(high) / 2 to stay within 8 bits
                    two_sum2(wh[d][r], wl[d][r], wh[d][r], wl[d][r]);
                    mw = fmaxf(mw, fmaxf(fabsf(wh[d][r].x), fabsf(wh[d][r].y)));
                }
            }
            const int ew = exp_bound(block_max(mw, M.red[1]));  // after this barrier X is no longer read
            // ---- stage 5: digit rows of wr -> A_r, ws -> A_s, wt -> A_t
            const float2 sw = sp2(pow2f(-ew));
#pragma unroll
            for (int r = 0; r < NPAIR; r++) {
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    float2 q[6];
                    digits6(mul2(wh[d][r], sw), mul2(wl[d][r], sw), q);
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int p = tid + 2 * kNT * r + kNT * h;
                        if (p < N3) {
                            const uint4 row = h ? digit_row(q[0].y, q[1].y, q[2].y, q[3].y, q[4].y, q[5].y)
                                                : digit_row(q[0].x, q[1].x, q[2].x, q[3].x, q[4].x, q[5].x);
                            const int i = p % NX, j = (p / NX) % NX, k = p / N2;
                            const int row_d = d == 0 ? j + NX * k : d == 1 ? i + NX * k : i + NX * j;
                            const int chunk = d == 0 ? i : d == 1 ? j : k;
                            *reinterpret_cast<uint4*>(A + d * C::ABYTES + a_off<NX>(row_d, chunk)) = row;
                        }
                    }
                }
            }
            // ---- phase-2 MMAs
            tc5::fence_async_smem();
            tc5::fence_before();
            __syncthreads();
            tc5::fence_after();
            if (warp == 0) {
                if (lane == 0) issue_phase<NX>(tmem, a_base, b2, mbar);
                __syncwarp();
            }
            ok = tc5::mbar_wait_bounded(mbar, parity, wait_ns);
            if (__syncthreads_or(!ok)) goto timed_out;
            parity ^= 1u;
            tc5::fence_after();
            // ---- stage 6: levels -> float pairs of the three direction sums in X
            readout<NX, true>(lane_addr, sig2, A, tid);
            tc5::fence_before();
            __syncthreads();
            // ---- stage 7: w = (his + Es + ss of the three directions) * 2^(eu + ew + 2 ed - 32); the his
            // and the Es sum exactly, TwoSum joins them
            const int xs = eu + ew + 2 * ed - 32;
            const float4* X4 = reinterpret_cast<const float4*>(A);
            double* we = w + e * N3;
            for (int p = tid; p < N3; p += kNT) {
                const float4 a = X4[p], b = X4[N3 + p], c = X4[2 * N3 + p];
                const float H = __fadd_rn(__fadd_rn(a.x, b.x), c.x);
                const float Es = __fadd_rn(__fadd_rn(a.y, b.y), c.y);
                const float ss = __fadd_rn(__fadd_rn(a.z, b.z), c.z);
                const float S = __fadd_rn(H, Es);
                const float bb = __fsub_rn(S, H);
                const float T = __fadd_rn(__fsub_rn(H, __fsub_rn(S, bb)), __fsub_rn(Es, bb));
                we[p] = __dadd_rn(widen_scaled(S, xs), widen_scaled(__fadd_rn(T, ss), xs));
            }
        }
        continue;
    timed_out:
        // a wait ran out: flag it, poison the outputs this CTA still owes, wait once more for
        // the MMAs in flight, then leave the element loop (TMEM is freed below)
        if (tid == 0) atomicExch(&g_ax_oz_timeout, 1);
        for (int64_t e2 = e; e2 < nelt; e2 += gridDim.x)
            for (int p = tid; p < N3; p += kNT) w[e2 * N3 + p] = __longlong_as_double(0x7FF8000000000000LL);
        tc5::mbar_wait_bounded(mbar, parity, wait_ns);
        break;
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (warp == 0) tc5::tmem_dealloc(tmem, kTmemCols);
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

template <int NX>
nek_status launch_oz_nx(int64_t nelt, const double* D, const float* Gff, const double* u, double* w,
                        cudaStream_t s, long long wait_ns, int arrivals)
{
    static std::atomic<uint64_t> configured{0};
    constexpr size_t smem = oz_smem_bytes<NX>();
    nek_status st = ensure_dyn_smem(k_ax_oz<NX>, smem, configured);
    if (st != NEK_OK) return st;
    const int64_t cap = 2 * (int64_t)oz_sm_count();
    const int grid = static_cast<int>(nelt < cap ? nelt : cap);
    k_ax_oz<NX><<<grid, kNT, smem, s>>>(nelt, D, reinterpret_cast<const float4*>(Gff), u, w, wait_ns, arrivals);
    return check_launch();
}

}  // namespace

bool ax_oz_supported(int nx) { return nx >= 2 && nx <= 10 && nx % 2 == 0; }

nek_status launch_ax_oz_ex(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                           cudaStream_t s, long long wait_ns, int arrivals)
{
    switch (nx) {
        case 2: return launch_oz_nx<2>(nelt, D, Gff, u, w, s, wait_ns, arrivals);
        case 4: return launch_oz_nx<4>(nelt, D, Gff, u, w, s, wait_ns, arrivals);
        case 6: return launch_oz_nx<6>(nelt, D, Gff, u, w, s, wait_ns, arrivals);
        case 8: return launch_oz_nx<8>(nelt, D, Gff, u, w, s, wait_ns, arrivals);
        case 10: return launch_oz_nx<10>(nelt, D, Gff, u, w, s, wait_ns, arrivals);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
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

nek_status nek_ax_oz(int64_t nelt, int nx, const double* D, const float* Gff, const double* u, double* w,
                     void* stream)
{
    if (!ax_oz_supported(nx)) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Gff || !u || !w || !is_aligned(D, 8) || !is_aligned(Gff, 16) || !is_aligned(u, 8) ||
        !is_aligned(w, 8))
        return NEK_ERR_INVALID_ARG;
    const int64_t npts = nelt * (int64_t)nx * nx * nx;
    if (ranges_overlap(u, sizeof(double) * npts, w, sizeof(double) * npts)) return NEK_ERR_INVALID_ARG;
    return launch_ax_oz_ex(nelt, nx, D, Gff, u, w, static_cast<cudaStream_t>(stream), kWaitNs, 1);
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
        st = launch_ax_oz_ex(ne, nx, dbuf, gff, dbuf + nx * nx, w, nullptr, wait_us * 1000LL, force_timeout ? 2 : 1);
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
