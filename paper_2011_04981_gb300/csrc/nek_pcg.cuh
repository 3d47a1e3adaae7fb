// Preconditioned CG on the device, generic over the vector storage type V
// (double for the FP64 solve, float for the inner solve of the defect
// correction).  Scalars and all inner products are accumulated in double.
//
// One iteration (the CG iteration of Section II-B of arXiv 2011.04981:
// operator, nearest-neighbour exchange, reductions, vector updates):
//   w = AX p (caller's operator) ; w = dssum(w) ; w = mask.w ; pw = <p,w>_c
//   alpha = rz/pw ; x += alpha p ; r -= alpha w ; z = minv r ; rr = <r,r>_c ;
//   rz' = <r,z>_c ; stop if sqrt(rr)/||b|| <= tol ; beta = rz'/rz ; p = z + beta p
// The kernels split this so that p is read by one vector kernel only:
// k_update does r -= alpha w and the two sums (z = minv r formed on the fly,
// never stored); k_p then does x += alpha p with the old p and p = minv r +
// beta p.  Every value is computed by the same operations as in the order
// above, so the split changes no result, and it saves 8 bytes per point and
// iteration (the second read of p; z's write and read become reads of minv
// and r).
// With point flags the mask is applied where w is used (k_update, and the flag
// test of <p,w>), so nothing writes w after the operator and dssum.
//
// Operators that report element energies (ElementEnergies) save the <p,w>
// pass: <p, mask.dssum(A_L p)>_c = sum over elements of p_e . (A_e p_e),
// because p holds the same value in every copy of a node and is zero on masked
// nodes (z = minv r and r vanish there).  The operator writes those energies
// and k_alpha sums them.  An operator that can also apply k_p's x / direction
// update as it loads p (ElementEnergies::fused_dir; DirUpdate, or DirUpdateF for
// FP32 vectors) takes over that pass: the loop then runs operator, dssum,
// k_alpha, k_update, k_beta, and k_p runs once after it for the last x update.
// Reductions use a fixed grid per length and a fixed shuffle tree, so results
// are deterministic.  Once the residual test passes, or a breakdown is seen, a
// device flag makes every later update kernel of the call return at once.
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "nek_ff.cuh"
#include "nek_internal.h"
#include "nek_reduce.cuh"

namespace nek {
namespace pcg {

using Scalars = PcgScalars;

constexpr int NT = kReduceThreads;

__device__ __forceinline__ bool halted(const Scalars* sc) { return sc->done || sc->status != NEK_OK; }

// (double)x with integer operations only, exact for every float (normal,
// subnormal, zero, inf, nan).  The FP32 -> FP64 conversion instruction runs on
// the FP64 pipe, which the double-precision dot products of the float solve
// already load; this keeps it to the DFMA of each product.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned sgn = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    unsigned hi, lo;
    if (e != 0u && e != 0xFFu) {  // normal: exponent rebiased 127 -> 1023, mantissa 23 -> 52 bits
        hi = sgn | ((e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    } else if (e == 0xFFu) {  // inf, nan (payload kept)
        hi = sgn | 0x7FF00000u | (m >> 3);
        lo = m << 29;
    } else if (m == 0u) {  // signed zero
        hi = sgn;
        lo = 0u;
    } else {  // subnormal m * 2^-149 = 1.f * 2^(p-149) with the leading one at bit p
        const int p = 31 - __clz(m);
        const unsigned long long f = static_cast<unsigned long long>(m ^ (1u << p)) << (52 - p);
        hi = sgn | (static_cast<unsigned>(p + 874) << 20) | static_cast<unsigned>(f >> 32);
        lo = static_cast<unsigned>(f);
    }
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// Inner-product weight of entry q: 1/multiplicity on E-vectors, 1 when c is
// null (unique-node vectors, where every node is stored once).
template <class V>
__device__ __forceinline__ double cw(const V* __restrict__ c, int64_t q)
{
    return c ? to_f64(c[q]) : 1.0;
}

// Point flags (optional, one byte per point): bit 0 = free (the mask), bit 1 =
// owner (exactly one copy of every global node).  With flags the inner products
// sum over owner copies, which is the 1/multiplicity-weighted sum over all
// copies (copies hold bit-identical values) read from 1 byte instead of 8.
constexpr uint8_t kFree = 1, kOwner = 2;

template <class V>
__device__ __forceinline__ double weight(const V* __restrict__ c, const uint8_t* __restrict__ flags, int64_t q)
{
    return flags ? ((flags[q] & kOwner) ? 1.0 : 0.0) : cw(c, q);
}

__device__ __forceinline__ bool is_free(const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flags,
                                        int64_t q)
{
    return flags ? (flags[q] & kFree) != 0 : mask[q] != 0;
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

inline int stream_blocks(int64_t n)
{
    int64_t nb = (n + 255) / 256;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nb, 152 * 16)));
}

namespace {

// Groups [g_begin, g_end) of a plan summed by the threads tid, tid + stride,
// ...: one thread per group, a left-to-right sum over members (ascending local
// index) written back to every member; groups are disjoint.  A thread takes
// four groups at a time and issues each level of their loads (offsets, the
// first two members, their values) together before any store; members beyond
// the second (edge and corner nodes) follow in order.
template <class V>
__device__ __forceinline__ void dssum_groups(int64_t g_begin, int64_t g_end, int64_t tid, int64_t stride,
                                             const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                                             V* __restrict__ v)
{
    constexpr int B = 4;
    for (int64_t g0 = g_begin + tid; g0 < g_end; g0 += B * stride) {
        int a[B], b[B], m0[B], m1[B];
        V s[B];
#pragma unroll
        for (int k = 0; k < B; k++) {
            const int64_t g = g0 + k * stride < g_end ? g0 + k * stride : g0;  // in bounds; unused when past
            a[k] = off[g];
            b[k] = off[g + 1];
        }
#pragma unroll
        for (int k = 0; k < B; k++) {
            m0[k] = mem[a[k]];
            m1[k] = mem[a[k] + 1];  // every group has at least two members
        }
#pragma unroll
        for (int k = 0; k < B; k++) s[k] = v[m0[k]] + v[m1[k]];
#pragma unroll
        for (int k = 0; k < B; k++) {
            if (g0 + k * stride >= g_end) break;
            for (int o = a[k] + 2; o < b[k]; o++) s[k] += v[mem[o]];
            v[m0[k]] = s[k];
            v[m1[k]] = s[k];
            for (int o = a[k] + 2; o < b[k]; o++) v[mem[o]] = s[k];
        }
    }
}

template <class V>
__global__ void k_dssum_t(int64_t ngroups, const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                          V* __restrict__ v)
{
    dssum_groups<V>(0, ngroups, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, off,
                    mem, v);
}

template <class V>
nek_status dssum(const nek_gs* gs, V* v, cudaStream_t s)
{
    if (!gs || gs->ngroups == 0) return NEK_OK;  // no plan: the operator is already assembled
    const int64_t nb = (gs->ngroups + 255) / 256;
    k_dssum_t<V><<<static_cast<int>(std::min<int64_t>(nb, 152 * 64)), 256, 0, s>>>(gs->ngroups, gs->d_offsets,
                                                                                 gs->d_members, v);
    return check_launch();
}

// x = 0, r = mask.f, p = z = minv r; partials of <r,z>_c and <r,r>_c.
template <class V>
__global__ void __launch_bounds__(NT) k_init(int64_t n, const V* __restrict__ c, const uint8_t* __restrict__ mask,
                                              const V* __restrict__ minv, const V* __restrict__ f, V* __restrict__ x,
                                              V* __restrict__ r, V* __restrict__ p, double* __restrict__ parts,
                                              const uint8_t* __restrict__ flags)
{
    __shared__ double sh[NT / 32];
    double arz = 0.0, arr = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += (int64_t)gridDim.x * NT) {
        const V rq = is_free(mask, flags, q) ? f[q] : V(0);
        const V zq = minv[q] * rq;
        x[q] = V(0);
        r[q] = rq;
        p[q] = zq;
        const double wq = weight(c, flags, q);
        arz += wq * to_f64(rq) * to_f64(zq);
        arr += wq * to_f64(rq) * to_f64(rq);
    }
    double t = block_sum<NT>(arz, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
    t = block_sum<NT>(arr, sh);
    if (threadIdx.x == 0) parts[gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_init_finish(const double* __restrict__ parts, int nb, double tol,
                                                     Scalars* sc)
{
    __shared__ double sh[NT / 32];
    const double rz = sum_partials<NT>(parts, nb, sh);
    const double rr = sum_partials<NT>(parts + nb, nb, sh);
    if (threadIdx.x == 0) {
        sc->rz = rz;
        sc->rr = rr;
        sc->bnorm = sqrt(rr);
        sc->tol = tol;
        sc->it = 0;
        sc->iters = 0;
        sc->alpha = sc->beta = sc->pw = 0.0;
        sc->xpend = 0;
        sc->status = NEK_OK;
        sc->done = 0;
        sc->relres = 0.0;
        if (!(rr >= 0.0) || !isfinite(rr) || !isfinite(rz)) {
            sc->status = NEK_ERR_BREAKDOWN;
        } else if (rr == 0.0) {
            sc->done = 1;  // b = 0: x = 0 is the solution
        } else {
            sc->relres = 1.0;
        }
    }
}

// w <- mask.w ; partials of <p,w>_c
template <class V>
__global__ void __launch_bounds__(NT) k_pw(int64_t n, const V* __restrict__ c, const uint8_t* __restrict__ mask,
                                            const V* __restrict__ p, V* __restrict__ w, double* __restrict__ parts,
                                            const Scalars* __restrict__ sc, const uint8_t* __restrict__ flags)
{
    __shared__ double sh[NT / 32];
    if (halted(sc)) return;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * NT;
    if (flags) {
        // read-only (the mask is applied by k_update), so the unrolled loads of
        // consecutive iterations can all be in flight
#pragma unroll 4
        for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += stride) {
            const uint8_t fq = flags[q];
            const V pq = p[q];  // loaded whatever the flags say, so it is not held back behind them
            const V wq = w[q];
            if ((fq & (kFree | kOwner)) == (kFree | kOwner)) acc += to_f64(pq) * to_f64(wq);
        }
    } else {
        for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += stride) {
            V wq = w[q];
            if (!mask[q]) {
                wq = V(0);
                w[q] = V(0);
            }
            acc += cw(c, q) * to_f64(p[q]) * to_f64(wq);
        }
    }
    const double t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
}

// NTA threads sum the nb partials (1024 for the nelt element energies, whose
// loads then overlap better).
template <int NTA = NT>
__global__ void __launch_bounds__(NTA) k_alpha(const double* __restrict__ parts, int nb, Scalars* sc)
{
    __shared__ double sh[NTA / 32];
    if (halted(sc)) {
        if (threadIdx.x == 0) sc->xpend = 0;
        return;
    }
    const double pw = sum_partials<NTA>(parts, nb, sh);
    if (threadIdx.x == 0) {
        sc->it += 1;
        sc->pw = pw;
        if (!(pw > 0.0) || !isfinite(pw)) {
            sc->status = NEK_ERR_BREAKDOWN;
            sc->iters = sc->it;
            sc->xpend = 0;
        } else {
            sc->alpha = sc->rz / pw;
            sc->xpend = 1;
        }
    }
}

// r -= alpha mask.w; partials of <r,r>_c and <r,z>_c with z = minv r (not stored)
// (s_hi + s_lo) + s_c += r^2 in float pairs: r = rh + rl split by integer operations (|r - rh - rl| <=
// 2^-46 |r|), r^2 = rh^2 (exact as the float pair p + e) + 2 rh rl; p summed with TwoSum into s_hi + s_lo,
// e + 2 rh rl into s_c.  For sums of ~100 terms a thread: good to ~2^-40 of the sum.
__device__ __forceinline__ void sq_pair_add(double r, float& s_hi, float& s_lo, float& s_c)
{
    const float2 h = split_double(r);
    const float pr = __fmul_rn(h.x, h.x);
    const float t = __fmaf_rn(2.f * h.x, h.y, __fmaf_rn(h.x, h.x, -pr));
    const float sn = __fadd_rn(s_hi, pr);
    const float bb = __fsub_rn(sn, s_hi);
    s_lo = __fadd_rn(s_lo, __fadd_rn(__fsub_rn(s_hi, __fsub_rn(sn, bb)), __fsub_rn(pr, bb)));
    s_hi = sn;
    s_c = __fadd_rn(s_c, t);
}

template <class V>
__global__ void __launch_bounds__(NT) k_update(int64_t n, const V* __restrict__ c, const V* __restrict__ minv,
                                                const V* __restrict__ w, V* __restrict__ r, double* __restrict__ parts,
                                                const Scalars* __restrict__ sc, const uint8_t* __restrict__ flags,
                                                const uint8_t* __restrict__ mask)
{
    __shared__ double sh[NT / 32];
    if (halted(sc)) return;
    const V alpha = (V)sc->alpha;
    double arr = 0.0, arz = 0.0;
    const int64_t stride = (int64_t)gridDim.x * NT;
    if (flags && std::is_same<V, float>::value) {
        if constexpr (std::is_same<V, float>::value) {  // (instantiated for FP32 vectors only)
            // FP32 vectors (the inner solve of defect correction, run to a relative
            // residual of about 1e-2): each thread sums its ~100 positive terms in
            // FP32 with FMAs and hands one double to the block's FP64 reduction
            float frr = 0.f, frz = 0.f;
            auto point = [&](uint32_t fq, float wq, float ro, float mq) {
                if (!(fq & kFree)) wq = 0.f;  // the mask
                const float rq = fmaf(-(float)alpha, wq, ro);
                const float zq = mq * rq;
                if (fq & kOwner) {
                    frr = fmaf(rq, rq, frr);
                    frz = fmaf(rq, zq, frz);
                }
                return rq;
            };
            const uintptr_t al = reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(r) |
                                 reinterpret_cast<uintptr_t>(minv);
            if ((al & 15) == 0 && (reinterpret_cast<uintptr_t>(flags) & 3) == 0) {
                // four consecutive points per access (16-byte vectors, one 32-bit word of flags); the last n % 4
                // points by block 0
                const int64_t n4 = n >> 2;
                const float4* w4 = reinterpret_cast<const float4*>(w);
                const float4* m4 = reinterpret_cast<const float4*>(minv);
                float4* r4 = reinterpret_cast<float4*>(r);
                const uint32_t* f4 = reinterpret_cast<const uint32_t*>(flags);
                for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n4; q += stride) {
                    const uint32_t fq = f4[q];
                    const float4 wv = w4[q], mv = m4[q], ro = r4[q];
                    float4 rn;
                    rn.x = point(fq & 0xffu, wv.x, ro.x, mv.x);
                    rn.y = point((fq >> 8) & 0xffu, wv.y, ro.y, mv.y);
                    rn.z = point((fq >> 16) & 0xffu, wv.z, ro.z, mv.z);
                    rn.w = point(fq >> 24, wv.w, ro.w, mv.w);
                    r4[q] = rn;
                }
                if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
                    const int64_t q = 4 * n4 + threadIdx.x;
                    r[q] = point(flags[q], w[q], r[q], minv[q]);
                }
            } else {
#pragma unroll 4
                for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += stride)
                    r[q] = point(flags[q], w[q], r[q], minv[q]);
            }
            arr = to_f64(frr);
            arz = to_f64(frz);
        }
    } else if (flags) {
        // r and <r,z> in FP64; <r,r> (used only for the residual test and the reported norm) exactly enough on
        // the FP32 pipes, so that GB300's 2-per-clock FP64 pipe carries three operations a point, not four:
        // r = rh + rl split by integer operations (|r - rh - rl| <= 2^-46 |r|), r^2 = rh^2 (exact as the
        // float pair p + e) + 2 rh rl, the p summed with TwoSum, the rest in plain floats: each thread's sum
        // is good to ~2^-40 of itself
        float s_hi = 0.f, s_lo = 0.f, s_c = 0.f;
#pragma unroll 4
        for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += stride) {
            const uint8_t fq = flags[q];
            V wq = w[q];
            if (!(fq & kFree)) wq = V(0);  // the mask
            const V rq = fma(-alpha, wq, r[q]);
            const V zq = minv[q] * rq;
            r[q] = rq;
            if (fq & kOwner) {
                arz += to_f64(rq) * to_f64(zq);
                if constexpr (std::is_same<V, double>::value) {
                    sq_pair_add(rq, s_hi, s_lo, s_c);
                } else {
                    const double rd = to_f64(rq);
                    arr += rd * rd;
                }
            }
        }
        if constexpr (std::is_same<V, double>::value) arr = (widen(s_hi) + widen(s_lo)) + widen(s_c);
    } else {
        for (int64_t q = blockIdx.x * (int64_t)NT + threadIdx.x; q < n; q += stride) {
            V wv = w[q];
            if (!mask[q]) wv = V(0);  // the mask (already applied when k_pw ran)
            const V rq = fma(-alpha, wv, r[q]);
            const V zq = minv[q] * rq;
            r[q] = rq;
            const double wq = cw(c, q);
            arr += wq * to_f64(rq) * to_f64(rq);
            arz += wq * to_f64(rq) * to_f64(zq);
        }
    }
    double t = block_sum<NT>(arr, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = t;
    t = block_sum<NT>(arz, sh);
    if (threadIdx.x == 0) parts[gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_beta(const double* __restrict__ parts, int nb, Scalars* sc)
{
    __shared__ double sh[NT / 32];
    if (halted(sc)) return;
    const double rr = sum_partials<NT>(parts, nb, sh);
    const double rz = sum_partials<NT>(parts + nb, nb, sh);
    if (threadIdx.x == 0) {
        sc->rr = rr;
        sc->relres = sqrt(rr) / sc->bnorm;
        if (!isfinite(sc->relres) || !isfinite(rz)) {
            sc->status = NEK_ERR_BREAKDOWN;
            sc->iters = sc->it;
        } else if (sc->tol > 0.0 && sc->relres <= sc->tol) {
            sc->done = 1;
            sc->iters = sc->it;
        } else {
            sc->beta = rz / sc->rz;
            sc->rz = rz;
        }
    }
}

// x += alpha p (old p) while xpend is set; then, when the iteration goes on and
// update_p is set, p = minv r + beta p.
template <class V>
__global__ void k_p(int64_t n, const V* __restrict__ minv, const V* __restrict__ r, V* __restrict__ x,
                    V* __restrict__ p, const Scalars* __restrict__ sc, int update_p)
{
    const bool do_x = sc->xpend != 0;
    const bool do_p = update_p && !halted(sc);
    const V alpha = (V)sc->alpha, beta = (V)sc->beta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (do_x && do_p) {
#pragma unroll 4
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) {
            const V pq = p[q];
            x[q] = fma(alpha, pq, x[q]);
            p[q] = fma(beta, pq, minv[q] * r[q]);
        }
    } else if (do_x) {
#pragma unroll 4
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride)
            x[q] = fma(alpha, p[q], x[q]);
    } else if (do_p) {  // not reached: an iteration that goes on has a pending x update
#pragma unroll 4
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride)
            p[q] = fma(beta, p[q], minv[q] * r[q]);
    }
}

}  // namespace

template <class V>
struct Buffers {
    V *r, *p, *w;
    double* parts;  // 2 * kMaxReduceBlocks
    Scalars* sc;
};

struct Result {
    int iters = 0;
    double relres = 0.0;
    int launches = 0;
    double ax_ms = 0.0;
    int ax_timed = 0;
};

// The element-energy path (see the top of this file): the operator writes
// edot[e] = p_e . (A_e p_e) for its nelt elements (k_update applies the mask,
// from the point flags or the mask array).  fused_dir: the operator also
// applies the x / direction update as it loads p (DirUpdate for FP64 vectors,
// DirUpdateF for FP32), so k_p runs once, after the loop, for the last x update.
struct ElementEnergies {
    double* edot;
    int64_t nelt;
    bool fused_dir = false;
};

namespace {

// One flag byte per point of an E-vector plan: kFree from the mask; kOwner on
// points in no group and on the first member of every group.
__global__ void k_flags_init(int64_t n, const uint8_t* __restrict__ mask, uint8_t* __restrict__ flags)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        flags[q] = (mask[q] ? kFree : 0) | kOwner;
}

__global__ void k_flags_groups(int64_t ngroups, const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                               uint8_t* __restrict__ flags)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x)
        for (int32_t m = off[g] + 1; m < off[g + 1]; m++) flags[mem[m]] &= static_cast<uint8_t>(~kOwner);
}

}  // namespace

// Fills flags (n bytes) for the plan gs and the mask.
inline nek_status build_flags(const nek_gs* gs, int64_t n, const uint8_t* mask, uint8_t* flags, cudaStream_t s)
{
    k_flags_init<<<stream_blocks(n), 256, 0, s>>>(n, mask, flags);
    if (gs && gs->ngroups > 0)
        k_flags_groups<<<stream_blocks(gs->ngroups), 256, 0, s>>>(gs->ngroups, gs->d_offsets, gs->d_members, flags);
    return check_launch();
}

// Runs PCG from x = 0.  `ax(p, w, edot, dir, stream)` applies the element
// operator, which gs then sums over shared nodes; with gs null, ax applies the
// assembled operator itself.  edot is ee->edot on the element-energy path (ee
// non-null), else null; dir is the direction update the operator applies
// first (ee->fused_dir), else null.  c null weights every entry by 1.
// tol > 0: stop at convergence (NEK_ERR_NOT_CONVERGED after max_iter);
// tol == 0: exactly max_iter iterations.  Leaves the stream synchronised.
template <class V, class AxFn>
nek_status run(const nek_gs* gs, int64_t n, const V* c, const uint8_t* mask, const V* minv, const V* f, V* x,
               const Buffers<V>& b, double tol, int max_iter, int check_every, bool time_ax, AxFn&& ax,
               cudaStream_t s, Result* res, const uint8_t* flags = nullptr, const ElementEnergies* ee = nullptr)
{
    const int nb = reduce_blocks(n);
    const int sb = stream_blocks(n);
    int launches = 0;
    const bool fused = ee && ee->fused_dir;
    using Dir = typename std::conditional<std::is_same<V, double>::value, DirUpdate, DirUpdateF>::type;
    const Dir dir{b.p, b.r, minv, x, b.sc};
    std::vector<cudaEvent_t> ev;
    Scalars h{};
    nek_status st = NEK_OK;
    k_init<V><<<nb, NT, 0, s>>>(n, c, mask, minv, f, x, b.r, b.p, b.parts, flags);
    k_init_finish<<<1, NT, 0, s>>>(b.parts, nb, tol, b.sc);
    launches += 2;
    if ((st = check_launch()) != NEK_OK) goto done;
    if (time_ax) {
        ev.resize(2 * (size_t)std::min(max_iter, 100000));
        for (auto& e : ev)
            if ((st = check_cuda(cudaEventCreate(&e))) != NEK_OK) goto done;
    }
    for (int it = 1; it <= max_iter; it++) {
        const bool timed = time_ax && (size_t)(2 * it) <= ev.size();
        if (timed) cudaEventRecord(ev[2 * (it - 1)], s);
        if ((st = ax(b.p, b.w, ee ? ee->edot : nullptr, fused ? &dir : nullptr, s)) != NEK_OK) goto done;
        if (timed) cudaEventRecord(ev[2 * (it - 1) + 1], s);
        if ((st = dssum<V>(gs, b.w, s)) != NEK_OK) goto done;
        if (ee) {
            k_alpha<1024><<<1, 1024, 0, s>>>(ee->edot, static_cast<int>(ee->nelt), b.sc);
        } else {
            k_pw<V><<<nb, NT, 0, s>>>(n, c, mask, b.p, b.w, b.parts, b.sc, flags);
            k_alpha<><<<1, NT, 0, s>>>(b.parts, nb, b.sc);
            launches += 1;
        }
        k_update<V><<<nb, NT, 0, s>>>(n, c, minv, b.w, b.r, b.parts, b.sc, flags, mask);
        k_beta<<<1, NT, 0, s>>>(b.parts, nb, b.sc);
        launches += 5;  // the operator, dssum, k_alpha, k_update, k_beta
        if (!fused) {
            k_p<V><<<sb, 256, 0, s>>>(n, minv, b.r, x, b.p, b.sc, it < max_iter ? 1 : 0);
            launches += 1;
        }
        if ((st = check_launch()) != NEK_OK) goto done;
        if (tol > 0.0 && (it % check_every == 0 || it == max_iter)) {
            if ((st = check_cuda(cudaMemcpyAsync(&h, b.sc, sizeof(h), cudaMemcpyDeviceToHost, s))) != NEK_OK) goto done;
            if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
            if (h.done || h.status != NEK_OK) break;
        }
    }
    if (fused) {  // the last iteration's x += alpha p (nothing when it was applied or never due)
        k_p<V><<<sb, 256, 0, s>>>(n, minv, b.r, x, b.p, b.sc, 0);
        launches += 1;
        if ((st = check_launch()) != NEK_OK) goto done;
    }
    if ((st = check_cuda(cudaMemcpyAsync(&h, b.sc, sizeof(h), cudaMemcpyDeviceToHost, s))) != NEK_OK) goto done;
    if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
    if (time_ax) {
        const int nt = std::min<int>(std::min(max_iter, h.it), static_cast<int>(ev.size() / 2));
        double tot = 0.0;
        for (int q = 0; q < nt; q++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]) == cudaSuccess) tot += ms;
        }
        res->ax_ms = tot;
        res->ax_timed = nt;
    }
    res->iters = (h.done || h.status != NEK_OK) ? h.iters : h.it;
    res->relres = h.relres;
    if (h.status != NEK_OK)
        st = static_cast<nek_status>(h.status);
    else if (tol > 0.0 && !h.done)
        st = NEK_ERR_NOT_CONVERGED;
done:
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    res->launches = launches;
    return st;
}

}  // namespace pcg
}  // namespace nek
