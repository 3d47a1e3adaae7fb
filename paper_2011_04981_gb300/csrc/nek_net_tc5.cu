// Learned-preconditioner inference on the 5th-generation tensor cores (tcgen05):
// BF16 operands in shared memory, FP32 accumulators in tensor memory (TMEM).
//
// Each 3x3x3 convolution of the per-element network is an implicit GEMM with
// M = output points, K = 16 input channels of one tap, N = 16 output channels,
// accumulated over the 27 taps.  The activations of one element are kept in
// shared memory on a zero-padded 10 x 10 x 10 grid of 16-byte rows (8 BF16
// channels per row; the 16 channels are two such arrays, the two K halves of
// the MMA's A operand):
//     row (i', j', k') at byte 16 * (10 * L + i'),  L = 10 k' + j' + 1,
// i' = i + 1 etc., plus one guard line (L = 0 and L = 101) at each end.  An M = 128
// tile covers 16 consecutive "padded lines" L_out = 10 k + j' of the output
// (8 points each, the i direction); for tap (di, dj, dk) the A rows of those 16
// lines are 16 lines of the grid at the uniform line stride, shifted by
// 10 (1 + dk) + dj lines and 1 + di rows, so every tap is one descriptor with the
// same strides (SBO = 160 B between 8-row groups, LBO = the K-half array size).
// The 80 padded output lines (k = 0..7, j' = 0..9) make 5 tiles; rows on the
// padding lines j' = 0, 9 compute garbage from in-range addresses and are
// dropped by the epilogue.  Per element and layer: 5 x 27 MMAs of
// 128 x 16 x 16 issued by one thread, committed to an mbarrier.
//
// The epilogue reads each thread's TMEM lane (one output row) with tcgen05.ld,
// adds the bias, applies GELU in FP32, rounds to BF16 and writes the row back
// into the same grid (the next layer's input; every MMA of the layer has
// completed by then).  The last layer writes z = y * scale * c in FP64.
//
// Numerics are those of nek_net_apply_bf16's contract: BF16 weights, the input
// and both hidden activations rounded to BF16 (nearest even) before each
// convolution, products exact and sums FP32 in the tensor core.
//
// Every wait on the mbarrier is bounded (~2 s of global time).  A wait that runs
// out sets a device flag (read by nek_fcg_solve_trunc, which returns
// NEK_ERR_TIMEOUT), writes NaN into the element's output (so the solve that uses
// it stops on a non-finite value), waits once more, frees the CTA's TMEM and
// returns.
#include <cuda_bf16.h>

#include "nek_internal.h"

namespace nek {

namespace {

constexpr int NP = 512, CIN = 2, CH = 16;
constexpr int NPARAM_TC5 = CH * CIN * 27 + CH + CH * CH * 27 + CH + CH * 27 + 1;
constexpr int OW1 = 0, OB1 = OW1 + CH * CIN * 27, OW2 = OB1 + CH, OB2 = OW2 + CH * CH * 27, OW3 = OB2 + CH,
              OB3 = OW3 + CH * 27;
constexpr int NT5 = 128;            // 4 warps: one per 32-lane TMEM sub-partition
constexpr int kLines = 102;         // 100 grid lines + 2 guard lines
constexpr int kHalfBytes = kLines * 10 * 16;  // one K half of the activation grid: 16320 B
constexpr int kTapBytes = 512;      // B operand of one tap: 16 rows (n) x 16 channels (k), two K halves
constexpr int kTiles = 5;           // 80 padded output lines / 16
constexpr uint32_t kTmemCols = 128; // 5 tiles x 16 columns, rounded up to a power of two
constexpr long long kWaitNs = 2000000000LL;  // default bound of every mbarrier wait

// 32-bit instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

struct __align__(128) Tc5Smem {
    __nv_bfloat16 act[2 * kLines * 10 * 8];  // [K half][line][row][8 channels]
    __nv_bfloat16 w[3 * 27 * 2 * 16 * 8];     // [layer][tap][K half][n][8 channels]
    float b1[16], b2[16], b3[4];
    unsigned long long mbar;
    uint32_t tmem_base;
};

__device__ int g_net_tc5_timeout = 0;  // set by a bounded wait that ran out

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float gelu5(float v) { return 0.5f * v * (1.f + erff(v * 0.70710678118654752f)); }

// Shared-memory matrix descriptor (no swizzle): start address, LBO (K direction),
// SBO (M/N direction, 8-row groups), all >> 4; the fixed value 1 in bits 46-48.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_bf16_tmem(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase with parity `parity`; false if it did not complete
// within kWaitNs.  Each try may suspend the thread (up to the hint, 20 us) until
// the phase completes, so waiting threads do not take issue slots from the
// other CTAs on the SM; the clock is read every 64 tries.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long wait_ns)
{
    const long long t0 = global_ns();
    for (int tries = 1;; tries++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P1;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, %3;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(20000)
            : "memory");
        if (done) return true;
        if ((tries & 63) == 0 && global_ns() - t0 > wait_ns) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; q++) v[q] = __uint_as_float(r[q]);
}

// Byte offset of grid row (i', j', k') in one K half.
__device__ __forceinline__ int grid_row(int ip, int jp, int kp) { return 16 * (10 * (10 * kp + jp + 1) + ip); }

// arrivals: arrivals the mbarrier expects per phase (1: the commit of the MMAs;
// the self-test passes 2, which no phase ever gets, so every wait runs out).
__global__ void __launch_bounds__(NT5, 3) k_net_apply_tc5(int64_t nelt, const float* __restrict__ theta,
                                                         const float* __restrict__ xin,
                                                         const float* __restrict__ scale,
                                                         const double* __restrict__ c, double* __restrict__ z,
                                                         long long wait_ns, int arrivals)
{
    extern __shared__ __align__(128) unsigned char raw5[];
    Tc5Smem& S = *reinterpret_cast<Tc5Smem*>(raw5);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* act = reinterpret_cast<unsigned char*>(S.act);

    // ---- set-up: weights as BF16 B operands, zero grid, biases, mbarrier, TMEM
    for (int q = tid; q < 3 * 27 * 2 * 16 * 8; q += NT5) {
        const int k8 = q & 7, n = (q >> 3) & 15, h = (q >> 7) & 1, t = (q >> 8) % 27, l = (q >> 8) / 27;
        const int ch = 8 * h + k8;
        float v = 0.f;
        if (l == 0 && ch < CIN) v = theta[OW1 + (n * CIN + ch) * 27 + t];
        if (l == 1) v = theta[OW2 + (n * CH + ch) * 27 + t];
        if (l == 2 && n == 0) v = theta[OW3 + ch * 27 + t];
        S.w[q] = __float2bfloat16_rn(v);
    }
    for (int q = tid; q < 2 * kLines * 10 * 8 / 8; q += NT5) reinterpret_cast<uint4*>(S.act)[q] = make_uint4(0, 0, 0, 0);
    if (tid < CH) {
        S.b1[tid] = __bfloat162float(__float2bfloat16_rn(theta[OB1 + tid]));
        S.b2[tid] = __bfloat162float(__float2bfloat16_rn(theta[OB2 + tid]));
    }
    if (tid == 0) {
        S.b3[0] = __bfloat162float(__float2bfloat16_rn(theta[OB3]));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar)), "r"(arrivals) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const uint32_t mbar = smem_u32(&S.mbar);
    const uint32_t act_base = smem_u32(S.act), w_base = smem_u32(S.w);
    // descriptors of the grid's first row (LBO = one K half, SBO = one line) and of layer 0, tap 0
    const uint64_t a_desc0 = smem_desc(act_base, kHalfBytes, 160);
    const uint64_t b_desc0 = smem_desc(w_base, 256, 128);
    uint32_t parity = 0;
    // This thread's TMEM lane: row m of every tile (warp w owns lanes 32 w .. 32 w + 31).
    const int m = 32 * warp + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
    bool failed = false;  // uniform across the CTA (decided by __syncthreads_or)

    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        // input: channels 0, 1 of the interior rows (rounded to BF16), channels 2..15 zero
        for (int p = tid; p < NP; p += NT5) {
            const int i = p & 7, j = (p >> 3) & 7, k = p >> 6;
            const __nv_bfloat162 x01 = __floats2bfloat162_rn(xin[(e * CIN + 0) * NP + p], xin[(e * CIN + 1) * NP + p]);
            const int off = grid_row(i + 1, j + 1, k + 1);
            uint4 h0 = make_uint4(*reinterpret_cast<const uint32_t*>(&x01), 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(act + off) = h0;
            *reinterpret_cast<uint4*>(act + kHalfBytes + off) = make_uint4(0, 0, 0, 0);
        }
        const double sc = (double)scale[e];
        for (int layer = 0; layer < 3; layer++) {
            fence_async_smem();  // the grid's rows, written by this CTA's threads, are read by the tensor core
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (warp == 0) {
                if (lane == 0) {
                    // descriptors advance by (byte offset >> 4) in their start-address field
                    const uint64_t b_layer = b_desc0 + (uint64_t)((layer * 27 * kTapBytes) >> 4);
#pragma unroll 1
                    for (int tile = 0; tile < kTiles; tile++) {
                        const uint64_t a_tile = a_desc0 + (uint64_t)(16 * tile * 10);  // 16 lines of 160 B
                        const uint32_t d = tmem + 16u * (uint32_t)tile;
#pragma unroll
                        for (int t = 0; t < 27; t++) {
                            const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
                            // first row of the tile's A rows: line 11 + 10 dk + dj, row 1 + di (in 16-byte units)
                            const int a_off = 10 * (11 + 10 * dk + dj) + 1 + di;
                            mma_bf16_tmem(d, a_tile + (uint64_t)a_off, b_layer + (uint64_t)(t * (kTapBytes >> 4)),
                                          t > 0 ? 1u : 0u);
                        }
                    }
                    mma_commit(mbar);
                }
                __syncwarp();
            }
            bool ok = mbar_wait_bounded(mbar, parity, wait_ns);
            if (__syncthreads_or(!ok)) {
                // a wait ran out: flag it, poison the element's output, wait once more for the MMAs in
                // flight, then leave the element loop (TMEM is freed below)
                failed = true;
                if (tid == 0) {
                    atomicExch(&g_net_tc5_timeout, 1);
                    z[e * NP] = __longlong_as_double(0x7FF8000000000000LL);
                }
                mbar_wait_bounded(mbar, parity, wait_ns);
                break;
            }
            parity ^= 1u;
            tc_fence_after();
#pragma unroll 1
            for (int tile = 0; tile < kTiles; tile++) {
                float v[16];
                tmem_ld16(lane_addr + 16u * (uint32_t)tile, v);
                const int lout = 16 * tile + (m >> 3), i = m & 7, jp = lout % 10, k = lout / 10;
                if (jp < 1 || jp > 8) continue;  // a padding line of the output: dropped
                if (layer < 2) {
                    const float* b = layer == 0 ? S.b1 : S.b2;
                    uint32_t packed[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const __nv_bfloat162 h2 =
                            __floats2bfloat162_rn(gelu5(v[2 * q] + b[2 * q]), gelu5(v[2 * q + 1] + b[2 * q + 1]));
                        packed[q] = *reinterpret_cast<const uint32_t*>(&h2);
                    }
                    const int off = grid_row(i + 1, jp, k + 1);
                    *reinterpret_cast<uint4*>(act + off) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    *reinterpret_cast<uint4*>(act + kHalfBytes + off) =
                        make_uint4(packed[4], packed[5], packed[6], packed[7]);
                } else {
                    const int p = i + 8 * (jp - 1) + 64 * k;
                    z[e * NP + p] = (double)(v[0] + S.b3[0]) * sc * c[e * NP + p];
                }
            }
            tc_fence_before();
        }
        if (failed) break;
        __syncthreads();  // the next element's input overwrites the grid
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

int sm_count()
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

}  // namespace

nek_status launch_net_apply_tc5_ex(int64_t nelt, const float* theta, const float* xin, const float* scale,
                                   const double* c, double* z, cudaStream_t s, long long wait_ns, int arrivals)
{
    static std::atomic<uint64_t> configured{0};
    nek_status st = ensure_dyn_smem(k_net_apply_tc5, sizeof(Tc5Smem), configured);
    if (st != NEK_OK) return st;
    const int64_t cap = 3 * (int64_t)sm_count();
    const int grid = static_cast<int>(nelt < cap ? nelt : cap);
    k_net_apply_tc5<<<grid, NT5, sizeof(Tc5Smem), s>>>(nelt, theta, xin, scale, c, z, wait_ns, arrivals);
    return check_launch();
}

nek_status launch_net_apply_tc5(int64_t nelt, const float* theta, const float* xin, const float* scale,
                                const double* c, double* z, cudaStream_t s)
{
    return launch_net_apply_tc5_ex(nelt, theta, xin, scale, c, z, s, kWaitNs, 1);
}

// Reads and clears the flag that a bounded wait of the kernel ran out (synchronous).
nek_status net_tc5_take_timeout(bool* timed_out)
{
    int v = 0, zero = 0;
    nek_status st = check_cuda(cudaMemcpyFromSymbol(&v, g_net_tc5_timeout, sizeof(int)));
    if (st == NEK_OK && v) st = check_cuda(cudaMemcpyToSymbol(g_net_tc5_timeout, &zero, sizeof(int)));
    *timed_out = v != 0;
    return st;
}

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_net_apply_bf16(int64_t nelt, int nx, const float* theta, const float* xin, const float* scale,
                              const double* c, double* z, void* stream)
{
    if (nx != 8) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!theta || !xin || !scale || !c || !z || !is_aligned(xin, 4) || !is_aligned(z, 8) || !is_aligned(c, 8))
        return NEK_ERR_INVALID_ARG;
    return launch_net_apply_tc5(nelt, theta, xin, scale, c, z, static_cast<cudaStream_t>(stream));
}

nek_status nek_net_tc_selftest(int force_timeout, int64_t wait_us, int* timed_out)
{
    if (!timed_out || wait_us < 1 || wait_us > 2000000) return NEK_ERR_INVALID_ARG;
    *timed_out = 0;
    bool stale = false;
    nek_status st = net_tc5_take_timeout(&stale);  // clear a flag left by an earlier call
    if (st != NEK_OK) return st;
    // two elements with zero weights and inputs: z = 0 unless the wait ran out (then z[0] is NaN)
    const int64_t ne = 2;
    float* buf = nullptr;
    double* dbuf = nullptr;
    const size_t nf = NPARAM_TC5 + ne * CIN * NP + ne;
    if ((st = check_cuda(cudaMalloc(&buf, sizeof(float) * nf))) != NEK_OK) return NEK_ERR_NOMEM;
    if ((st = check_cuda(cudaMalloc(&dbuf, sizeof(double) * 2 * ne * NP))) != NEK_OK) {
        cudaFree(buf);
        return NEK_ERR_NOMEM;
    }
    st = check_cuda(cudaMemset(buf, 0, sizeof(float) * nf));
    if (st == NEK_OK) st = check_cuda(cudaMemset(dbuf, 0, sizeof(double) * 2 * ne * NP));
    if (st == NEK_OK)
        st = launch_net_apply_tc5_ex(ne, buf, buf + NPARAM_TC5, buf + NPARAM_TC5 + ne * CIN * NP, dbuf,
                                     dbuf + ne * NP, nullptr, wait_us * 1000LL, force_timeout ? 2 : 1);
    if (st == NEK_OK) st = check_cuda(cudaDeviceSynchronize());
    bool to = false;
    if (st == NEK_OK) st = net_tc5_take_timeout(&to);
    double z0 = 0.0;
    if (st == NEK_OK) st = check_cuda(cudaMemcpy(&z0, dbuf + ne * NP, sizeof(double), cudaMemcpyDeviceToHost));
    cudaFree(buf);
    cudaFree(dbuf);
    if (st != NEK_OK) return st;
    *timed_out = to ? 1 : 0;
    if (to != (z0 != z0)) return NEK_ERR_CUDA;  // the flag and the poisoned output must agree
    return to ? NEK_ERR_TIMEOUT : NEK_OK;
}

}  // extern "C"
