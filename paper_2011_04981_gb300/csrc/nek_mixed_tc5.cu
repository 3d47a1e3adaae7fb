// Reduced-precision AX (BF16 / FP16 operands) with the D-contractions on the
// 5th-generation tensor cores (tcgen05, FP32 accumulators in tensor memory).
// Same arithmetic as the CUDA-core form (nek_mixed.cu) and the mma.sync form
// (nek_mixed_tc.cu):
//   u_q = rnd(u / s_u), D_q = rnd(D), FP32 sums of exact products,
//   [wr ws wt] = rnd(G_q [ur us ut]) in FP32, w = s_u s_G ((w_r + w_s) + w_t),
// only the order of the FP32 additions inside a contraction differs.
//
// One element at a time per CTA of 128 threads (persistent over elements):
//   A, one buffer per direction: row m = line m of the element along the
//     contracted direction (NX^2 <= 128 rows used), K = the line's NX points
//     padded to 16 with zeros: two 16-byte core-matrix rows per line, written
//     by the thread that owns the line from the element's u in shared memory.
//   B = rnd(D) (phase 2: rnd(D)^T), 16 x 16 padded.
//   Accumulator: lane = line, 16 columns per direction (48 of the CTA's 64).
// Each phase is three MMAs of 128 x 16 x 16, issued by warp 0 (lane 0's
// predicate) and committed to one mbarrier; thread m reads TMEM lane m (its
// line of each direction) into FP32 point arrays in shared memory, and the
// pointwise stages (G product, the final sum and scaling) run point-strided.
//
// Three forms: the plain operator; with element energies u_e . w_e (the inner
// solve's <p,w>); and with energies and the PCG direction update of the inner
// solve done as the element's input is loaded (x += alpha p, p = minv r + beta p
// with that solve's own FP32 operations; the operator is applied to the new p),
// which takes the solve's separate x / direction pass over the vectors away.
//
// Every wait on the mbarrier is bounded (~2 s of global time); a wait that
// runs out writes NaN into the CTA's remaining outputs, waits once more for its
// MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nek_internal.h"
#include "nek_reduce.cuh"
#include "nek_tc5.cuh"

#include <algorithm>

namespace nek {

namespace {

constexpr int kT5 = 128;
constexpr uint32_t kCols5 = 64;
constexpr long long kWait5 = 2000000000LL;
constexpr uint32_t kHint5 = 200;  // ns a try may suspend the waiting thread: the MMAs take well under 1 us
constexpr int kLpPlain = 0, kLpEnergy = 1, kLpDir = 2;  // operator forms (MODE)

template <class S>
struct Lp5;
template <>
struct Lp5<__nv_bfloat16> {
    static constexpr uint32_t kFmt = 1;  // instruction-descriptor A / B format: BF16
    __device__ static __forceinline__ unsigned short bits(float x)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    }
    __device__ static __forceinline__ float from_bits(unsigned short h) { return __uint_as_float((unsigned)h << 16); }
};
template <>
struct Lp5<__half> {
    static constexpr uint32_t kFmt = 0;  // FP16
    __device__ static __forceinline__ unsigned short bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
    __device__ static __forceinline__ float from_bits(unsigned short h) { return __half2float(__ushort_as_half(h)); }
};

// kind::f16 instruction descriptor: FP32 D, A and B of format fmt, K-major, M = 128, N = 16.
constexpr uint32_t idesc_lowp(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
}

constexpr int kABytes = 16 * 256;  // one direction's A: 16 groups of 8 rows x 2 chunks of 16 bytes
constexpr int kBBytes = 2 * 256;   // 16 rows x 2 chunks

// Byte size of the three point arrays [3][N3] floats, rounded up to 16 so that the 8-byte mbarrier and
// the doubles after them stay aligned for every nx.
template <int NX>
constexpr size_t tc5_x_bytes()
{
    return (sizeof(float) * 3 * (size_t)NX * NX * NX + 15) & ~size_t(15);
}
// The point arrays (the element's u, then ur us ut, wr ws wt, the parts of w), A [3], B [2], then 64 bytes
// of scalars and 32 of per-warp energies: 25.4 KB at nx = 10, so that 8 CTAs fit on an SM.
template <int NX>
constexpr size_t tc5_smem_bytes()
{
    return 3 * kABytes + 2 * kBBytes + tc5_x_bytes<NX>() + 96;
}

__device__ int g_lowp_tc5_timeout = 0;

// Byte offset of (row, chunk) in an A or B buffer (K-major, no swizzle).
__device__ __forceinline__ int rc_off(int row, int chunk) { return (row >> 3) * 256 + chunk * 128 + (row & 7) * 16; }

// Round the 16 line values v[0..NX) (zero beyond) to S and store them as row `row` of a buffer.
template <class S, int NX>
__device__ __forceinline__ void store_row(unsigned char* buf, int row, const float (&v)[NX])
{
    uint32_t h[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const float a = 2 * q < NX ? v[2 * q] : 0.f, b = 2 * q + 1 < NX ? v[2 * q + 1] : 0.f;
        h[q] = (uint32_t)Lp5<S>::bits(a) | ((uint32_t)Lp5<S>::bits(b) << 16);
    }
    *reinterpret_cast<uint4*>(buf + rc_off(row, 0)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(buf + rc_off(row, 1)) = make_uint4(h[4], h[5], h[6], h[7]);
}

// Max over the CTA of non-negative v (one barrier).
__device__ __forceinline__ float cta_max(float v, float* red)
{
    const unsigned x = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(v));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = __uint_as_float(x);
    __syncthreads();
    return fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
}

// Smallest power of two >= m (m > 0), 1 for m == 0 (the CUDA-core form's scale).
__device__ __forceinline__ float pow2_up(float m)
{
    if (!(m > 0.f)) return 1.f;
    int e;
    const float f = frexpf(m, &e);
    return ldexpf(1.f, f == 0.5f ? e - 1 : e);
}

// Six G values of point p as floats (12 bytes at a 4-byte aligned address).
template <class S>
__device__ __forceinline__ void g_load(const S* __restrict__ g, float (&v)[6])
{
    const unsigned* g4 = reinterpret_cast<const unsigned*>(g);
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const unsigned t = __ldg(g4 + q);
        v[2 * q] = Lp5<S>::from_bits(static_cast<unsigned short>(t & 0xffffu));
        v[2 * q + 1] = Lp5<S>::from_bits(static_cast<unsigned short>(t >> 16));
    }
}

// Warp 0, converged: the three MMAs of a phase (one per direction) and their commit.
__device__ __forceinline__ void issue3(uint32_t tmem, uint32_t a_base, uint32_t b_base, uint32_t idesc, uint32_t mbar)
{
    const uint64_t bd = tc5::smem_desc(b_base, 128, 256);
#pragma unroll
    for (int d = 0; d < 3; d++)
        tc5::mma_bf16_lane0(tmem + 16u * d, tc5::smem_desc(a_base + (uint32_t)(d * kABytes), 128, 256), bd, idesc, 0u);
    tc5::mma_commit_lane0(mbar);
}

template <class S, int NX, int MODE>
__global__ void __launch_bounds__(kT5, MODE == kLpDir ? 6 : 4)
    k_ax_lowp_tc5(int64_t nelt, const double* __restrict__ D, const S* __restrict__ Glp,
                  const float* __restrict__ gscale, const float* __restrict__ u, float* __restrict__ w,
                  double* __restrict__ edot, DirUpdateF dir, long long wait_ns)
{
    constexpr int N2 = NX * NX, N3 = N2 * NX;
    constexpr uint32_t IDESC = idesc_lowp(Lp5<S>::kFmt);
    extern __shared__ __align__(128) unsigned char lp5_raw[];
    unsigned char* A = lp5_raw;                                        // [3][kABytes]
    unsigned char* B1 = A + 3 * kABytes;                               // rnd(D)
    unsigned char* B2 = B1 + kBBytes;                                  // rnd(D)^T
    float* X = reinterpret_cast<float*>(B2 + kBBytes);                // [3][N3] u; ur us ut; wr ws wt; w parts
    float* sU = X;                                                     // the element's u until the first readout
    unsigned char* tail = B2 + kBBytes + tc5_x_bytes<NX>();            // 16-byte aligned
    unsigned long long* mbar_p = reinterpret_cast<unsigned long long*>(tail);
    uint32_t* tmem_p = reinterpret_cast<uint32_t*>(tail + 8);
    float* red = reinterpret_cast<float*>(tail + 16);                  // [4]
    int* flag = reinterpret_cast<int*>(tail + 32);
    double* esum = reinterpret_cast<double*>(tail + 64);               // [4]
    const int tid = threadIdx.x, warp = tid >> 5;

    // ---- set-up: rnd(D) and its transpose as B operands, mbarrier, TMEM
    for (int q = tid; q < 16 * 16; q += kT5) {
        const int n = q >> 4, k = q & 15;
        const float d1 = (n < NX && k < NX) ? (float)D[n * NX + k] : 0.f;
        const float d2 = (n < NX && k < NX) ? (float)D[k * NX + n] : 0.f;
        unsigned short* b1 = reinterpret_cast<unsigned short*>(B1 + rc_off(n, k >> 3)) + (k & 7);
        unsigned short* b2 = reinterpret_cast<unsigned short*>(B2 + rc_off(n, k >> 3)) + (k & 7);
        *b1 = Lp5<S>::bits(d1);
        *b2 = Lp5<S>::bits(d2);
    }
    if (tid == 0) tc5::mbar_init(tc5::smem_u32(mbar_p), 1);
    if (warp == 0) tc5::tmem_alloc(tmem_p, kCols5);
    tc5::fence_async_smem();
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tmem = *tmem_p, mbar = tc5::smem_u32(mbar_p);
    const uint32_t a_base = tc5::smem_u32(A), b1 = tc5::smem_u32(B1), b2 = tc5::smem_u32(B2);
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
    const int m = tid;  // this thread's line (TMEM lane) in every direction
    const bool line = m < N2;
    const int la = m % NX, lb = m / NX;  // r-line (j,k) = (la, lb); s-line (i,k) = (la, lb); t-line (i,j) = (la, lb)
    uint32_t parity = 0;
    // the direction update: x += alpha p while an x update is pending, p = minv r + beta p while the solve goes on
    bool dx = false, dp = false;
    float alpha = 0.f, beta = 0.f;
    if constexpr (MODE == kLpDir) {
        dx = dir.sc->xpend != 0;
        dp = !(dir.sc->done || dir.sc->status != NEK_OK);
        alpha = (float)dir.sc->alpha;
        beta = (float)dir.sc->beta;
    }

    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        // the next element's inputs and G into L2 while this one is processed
        if (e + gridDim.x < nelt) {
            const int64_t o = (e + gridDim.x) * N3;
            const unsigned char* gn = reinterpret_cast<const unsigned char*>(Glp + o * 6);
            for (int q = tid; q < (4 * N3 + 127) / 128; q += kT5) {
                if constexpr (MODE == kLpDir) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const unsigned char*>(dir.p + o) + 128 * q));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const unsigned char*>(dir.r + o) + 128 * q));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const unsigned char*>(dir.minv + o) + 128 * q));
                    if (dx)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const unsigned char*>(dir.x + o) + 128 * q));
                } else {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const unsigned char*>(u + o) + 128 * q));
                }
            }
            for (int q = tid; q < (12 * N3 + 127) / 128; q += kT5)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(gn + 128 * q));
        }
        // ---- u (with the direction update: the new p) into shared memory, the element's scale s_u
        float mx = 0.f;
        if constexpr (MODE == kLpDir) {
            float* pe = dir.p + e * N3;
            float* xe = dir.x + e * N3;
            const float* re = dir.r + e * N3;
            const float* me = dir.minv + e * N3;
            constexpr int KB = 4;  // points per batch: a batch's loads are issued before its stores
            for (int q0 = tid; q0 < N3; q0 += KB * kT5) {
                float po[KB], rv[KB], mv[KB], xv[KB];
#pragma unroll
                for (int k = 0; k < KB; k++) {
                    const int q = q0 + k * kT5 < N3 ? q0 + k * kT5 : q0;
                    po[k] = pe[q];
                    rv[k] = __ldg(re + q);
                    mv[k] = __ldg(me + q);
                    xv[k] = dx ? xe[q] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < KB; k++) {
                    const int q = q0 + k * kT5;
                    if (q < N3) {
                        if (dx) xe[q] = fmaf(alpha, po[k], xv[k]);
                        float v = po[k];
                        if (dp) {
                            v = fmaf(beta, po[k], mv[k] * rv[k]);
                            pe[q] = v;
                        }
                        sU[q] = v;
                        mx = fmaxf(mx, fabsf(v));
                    }
                }
            }
        } else {
            const float* ue = u + e * N3;
            for (int q = tid; q < N3; q += kT5) {
                const float v = __ldg(ue + q);
                sU[q] = v;
                mx = fmaxf(mx, fabsf(v));
            }
        }
        const float su = pow2_up(cta_max(mx, red));
        const float inv = 1.f / su;  // a power of two: exact
        // ---- A rows: this thread's three lines of rnd(u / s_u)
        if (line) {
            float v[NX];
#pragma unroll
            for (int l = 0; l < NX; l++) v[l] = sU[lb * N2 + la * NX + l] * inv;
            store_row<S, NX>(A, m, v);
#pragma unroll
            for (int l = 0; l < NX; l++) v[l] = sU[lb * N2 + l * NX + la] * inv;
            store_row<S, NX>(A + kABytes, m, v);
#pragma unroll
            for (int l = 0; l < NX; l++) v[l] = sU[l * N2 + lb * NX + la] * inv;
            store_row<S, NX>(A + 2 * kABytes, m, v);
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
        if (warp == 0) {
            issue3(tmem, a_base, b1, IDESC, mbar);
            __syncwarp();
        }
        if (tid == 0) *flag = tc5::mbar_wait_bounded(mbar, parity, wait_ns, kHint5) ? 0 : 1;
        __syncthreads();
        if (*flag) goto timed_out;
        parity ^= 1u;
        tc5::fence_after();
        // ---- ur, us, ut into the point arrays
        if ((m & ~31) < N2) {  // warp-uniform: lanes beyond NX^2 read padding and store nothing
#pragma unroll
            for (int d = 0; d < 3; d++) {
                float v[16];
                tc5::tmem_ld16(lane_addr + 16u * d, v);
                if (line) {
#pragma unroll
                    for (int o = 0; o < NX; o++) {
                        const int p = d == 0 ? lb * N2 + la * NX + o : d == 1 ? lb * N2 + o * NX + la : o * N2 + lb * NX + la;
                        X[d * N3 + p] = v[o];
                    }
                }
            }
        }
        tc5::fence_before();
        __syncthreads();
        // ---- wr, ws, wt = rnd(G_q [ur us ut]) in FP32, in place
        {
            const S* Ge = Glp + e * (int64_t)N3 * 6;
            for (int p = tid; p < N3; p += kT5) {
                const float ar = X[p], as = X[N3 + p], at = X[2 * N3 + p];
                float g[6];
                g_load<S>(Ge + 6 * p, g);
                X[p] = Lp5<S>::from_bits(Lp5<S>::bits(fmaf(g[0], ar, fmaf(g[1], as, g[2] * at))));
                X[N3 + p] = Lp5<S>::from_bits(Lp5<S>::bits(fmaf(g[1], ar, fmaf(g[3], as, g[4] * at))));
                X[2 * N3 + p] = Lp5<S>::from_bits(Lp5<S>::bits(fmaf(g[2], ar, fmaf(g[4], as, g[5] * at))));
            }
        }
        __syncthreads();
        // ---- A rows of wr (r-lines), ws (s-lines), wt (t-lines)
        if (line) {
            float v[NX];
#pragma unroll
            for (int l = 0; l < NX; l++) v[l] = X[lb * N2 + la * NX + l];
            store_row<S, NX>(A, m, v);
#pragma unroll
            for (int l = 0; l < NX; l++) v[l] = X[N3 + lb * N2 + l * NX + la];
            store_row<S, NX>(A + kABytes, m, v);
#pragma unroll
            for (int l = 0; l < NX; l++) v[l] = X[2 * N3 + l * N2 + lb * NX + la];
            store_row<S, NX>(A + 2 * kABytes, m, v);
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
        if (warp == 0) {
            issue3(tmem, a_base, b2, IDESC, mbar);
            __syncwarp();
        }
        if (tid == 0) *flag = tc5::mbar_wait_bounded(mbar, parity, wait_ns, kHint5) ? 0 : 1;
        __syncthreads();
        if (*flag) goto timed_out;
        parity ^= 1u;
        tc5::fence_after();
        // ---- the three directions' parts of w into the point arrays
        if ((m & ~31) < N2) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                float v[16];
                tc5::tmem_ld16(lane_addr + 16u * d, v);
                if (line) {
#pragma unroll
                    for (int o = 0; o < NX; o++) {
                        const int p = d == 0 ? lb * N2 + la * NX + o : d == 1 ? lb * N2 + o * NX + la : o * N2 + lb * NX + la;
                        X[d * N3 + p] = v[o];
                    }
                }
            }
        }
        tc5::fence_before();
        __syncthreads();
        // ---- w = s_u s_G ((w_r + w_s) + w_t)
        {
            const float scale = su * gscale[e];
            float* we = w + e * N3;
            float energy = 0.f;  // this thread's terms u w in FP32, then FP64 across the element
            for (int p = tid; p < N3; p += kT5) {
                const float wv = ((X[p] + X[N3 + p]) + X[2 * N3 + p]) * scale;
                we[p] = wv;
                // the input at p: with the direction update the p this thread wrote above (a plain load)
                if constexpr (MODE == kLpDir) energy = fmaf(dir.p[e * N3 + p], wv, energy);
                if constexpr (MODE == kLpEnergy) energy = fmaf(__ldg(u + e * N3 + p), wv, energy);
            }
            if constexpr (MODE != kLpPlain) {
                double t = (double)energy;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
                if ((tid & 31) == 0) esum[warp] = t;
            }
        }
        __syncthreads();  // u and the point arrays are read before the next element overwrites them
        if constexpr (MODE != kLpPlain) {
            if (tid == 0) edot[e] = (esum[0] + esum[1]) + (esum[2] + esum[3]);
        }
        continue;
    timed_out:
        if (tid == 0) atomicExch(&g_lowp_tc5_timeout, 1);
        for (int64_t e2 = e; e2 < nelt; e2 += gridDim.x)
            for (int p = tid; p < N3; p += kT5) w[e2 * N3 + p] = __int_as_float(0x7FC00000);
        if (tid == 0) tc5::mbar_wait_bounded(mbar, parity, wait_ns);
        __syncthreads();
        break;
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (warp == 0) tc5::tmem_dealloc(tmem, kCols5);
}

// CTAs of `threads` threads with `dyn_smem` bytes of dynamic shared memory that fit on one SM together
// (registers in 256-register warp allocations, shared memory with the per-CTA reservation, threads), at
// most cap; 1 if an attribute cannot be read.
int resident_ctas(const void* kernel, int threads, size_t dyn_smem, int cap)
{
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0, regs_sm = 0, rsv = 0, thr_sm = 0;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 1;
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int n = cap;
    n = std::min(n, thr_sm / threads);
    if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
    n = std::min(n, (int)(smem_sm / (dyn_smem + fa.sharedSizeBytes + (size_t)rsv)));
    return n < 1 ? 1 : n;
}

int tc5_sm_count()
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

template <class S, int NX, int MODE>
nek_status launch_tc5_kernel(int64_t nelt, const double* D, const void* Glp, const float* gscale, const float* u,
                             float* w, double* edot, const DirUpdateF& dir, cudaStream_t s)
{
    static std::atomic<uint64_t> configured{0};
    constexpr size_t smem = tc5_smem_bytes<NX>();
    nek_status st = ensure_dyn_smem(k_ax_lowp_tc5<S, NX, MODE>, smem, configured);
    if (st != NEK_OK) return st;
    // shared memory over L1, so that the CTAs the grid is sized for all fit
    static std::atomic<uint64_t> carved{0};
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !(carved.load() & (uint64_t(1) << dev))) {
            st = check_cuda(cudaFuncSetAttribute(k_ax_lowp_tc5<S, NX, MODE>,
                                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            if (st != NEK_OK) return st;
            carved.fetch_or(uint64_t(1) << dev);
        }
    }
    // persistent CTAs: as many as are resident on an SM at once, from the kernel's registers and shared
    // memory and the device's limits (at most 8, whose 64 TMEM columns fill the 512)
    static int per_sm = 0;
    if (!per_sm) per_sm = resident_ctas(reinterpret_cast<const void*>(k_ax_lowp_tc5<S, NX, MODE>), kT5, smem, 8);
    const int64_t cap = (int64_t)per_sm * tc5_sm_count();
    const int grid = static_cast<int>(nelt < cap ? nelt : cap);
    k_ax_lowp_tc5<S, NX, MODE><<<grid, kT5, smem, s>>>(nelt, D, static_cast<const S*>(Glp), gscale, u, w, edot, dir,
                                                        kWait5);
    return check_launch();
}

template <class S, int NX>
nek_status launch_tc5_nx(int64_t nelt, const double* D, const void* Glp, const float* gscale, const float* u,
                         float* w, double* edot, const DirUpdateF* dir, cudaStream_t s)
{
    const DirUpdateF none{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (edot && dir) return launch_tc5_kernel<S, NX, kLpDir>(nelt, D, Glp, gscale, u, w, edot, *dir, s);
    return edot ? launch_tc5_kernel<S, NX, kLpEnergy>(nelt, D, Glp, gscale, u, w, edot, none, s)
                : launch_tc5_kernel<S, NX, kLpPlain>(nelt, D, Glp, gscale, u, w, nullptr, none, s);
}

template <class S>
nek_status launch_tc5_t(int64_t nelt, int nx, const double* D, const void* Glp, const float* gscale, const float* u,
                        float* w, double* edot, const DirUpdateF* dir, cudaStream_t s)
{
    switch (nx) {
        case 2: return launch_tc5_nx<S, 2>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 3: return launch_tc5_nx<S, 3>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 4: return launch_tc5_nx<S, 4>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 5: return launch_tc5_nx<S, 5>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 6: return launch_tc5_nx<S, 6>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 7: return launch_tc5_nx<S, 7>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 8: return launch_tc5_nx<S, 8>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 9: return launch_tc5_nx<S, 9>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 10: return launch_tc5_nx<S, 10>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        case 11: return launch_tc5_nx<S, 11>(nelt, D, Glp, gscale, u, w, edot, dir, s);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
}

}  // namespace

bool ax_lowp_tc5_supported(int nx, int precision)
{
    return nx >= 2 && nx <= 11 && (precision == NEK_PREC_BF16 || precision == NEK_PREC_F16);
}

nek_status launch_ax_lowp_tc5(int precision, int64_t nelt, int nx, const double* D, const void* Glp,
                              const float* gscale, const float* u, float* w, cudaStream_t s, double* edot,
                              const DirUpdateF* dir)
{
    if (precision == NEK_PREC_BF16) return launch_tc5_t<__nv_bfloat16>(nelt, nx, D, Glp, gscale, u, w, edot, dir, s);
    if (precision == NEK_PREC_F16) return launch_tc5_t<__half>(nelt, nx, D, Glp, gscale, u, w, edot, dir, s);
    return NEK_ERR_INVALID_ARG;
}

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_ax_lowp_tc5(int64_t nelt, int nx, int precision, const double* D, const void* Glp,
                           const float* gscale, const float* u, float* w, void* stream)
{
    if (nx < 2 || nx > 11) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0 || !ax_lowp_tc5_supported(nx, precision)) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Glp || !gscale || !u || !w) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(D, 8) || !is_aligned(Glp, 4) || !is_aligned(u, 4) || !is_aligned(w, 4)) return NEK_ERR_INVALID_ARG;
    const size_t bytes = sizeof(float) * (size_t)nelt * nx * nx * nx;
    if (ranges_overlap(u, bytes, w, bytes)) return NEK_ERR_INVALID_ARG;
    return launch_ax_lowp_tc5(precision, nelt, nx, D, Glp, gscale, u, w, static_cast<cudaStream_t>(stream), nullptr);
}

}  // extern "C"
