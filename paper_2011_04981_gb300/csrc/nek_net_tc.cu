// Learned-preconditioner inference on the warp-level tensor-core MMA (mma.sync;
// BF16 in, FP32 accumulate): nek_net_apply_bf16_mma, kept beside the tcgen05
// form of nek_net_apply_bf16 (nek_net_tc5.cu) for comparison.
//
// Each 3x3x3 convolution of the per-element network is an implicit GEMM:
// rows = the 512 points of the element, K = 16 input channels per tap (the two
// input channels are padded with zeros to 16), 27 taps accumulated, N = 16
// output channels (8 for the last layer, of which only channel 0 is real).  A
// warp owns four tiles of 16 points; per tap it loads the B fragment of the
// tap's weights once (ldmatrix.x4), and for each tile the A fragment of the 16
// shifted points with one ldmatrix.x4 whose rows are gathered per lane (a point
// outside the element reads an all-zero row, which is the zero padding), then
// issues mma.sync.m16n8k16 (BF16 x BF16 -> FP32) for each half of N; the four
// tiles are four independent accumulation chains.  The epilogue adds
// the bias and applies GELU in FP32 and stores the activations back to shared
// memory as BF16, the next layer's A operand.
//
// Numerics: the weights are the same BF16-rounded values as nek_net_apply; the
// network input and the two hidden activations are rounded to BF16 (round to
// nearest even) before each convolution; sums are FP32.
#include <cuda_bf16.h>

#include "nek_internal.h"

namespace nek {

namespace {

constexpr int NXN = 8, NP = 512, CIN = 2, CH = 16;
constexpr int OW1 = 0, OB1 = OW1 + CH * CIN * 27, OW2 = OB1 + CH, OB2 = OW2 + CH * CH * 27, OW3 = OB2 + CH,
              OB3 = OW3 + CH * 27;
constexpr int RS = 24;  // activation row stride in BF16 values (48 B: ldmatrix rows land on distinct banks)
constexpr int NT_TC = 256;

__device__ __forceinline__ float gelu_tc(float v) { return 0.5f * v * (1.f + erff(v * 0.70710678118654752f)); }

struct TcSmem {
    __nv_bfloat16 x[(NP + 1) * RS];   // input, channels 0..1 (2..15 zero); row NP is all zero
    __nv_bfloat16 a1[(NP + 1) * RS];  // first hidden layer
    __nv_bfloat16 a2[(NP + 1) * RS];  // second hidden layer
    __nv_bfloat16 w1[27 * 16 * 16];   // [tap][n = cout][k = cin], cin 2..15 zero
    __nv_bfloat16 w2[27 * 16 * 16];
    __nv_bfloat16 w3[27 * 8 * 16];    // n = 0 is the output channel, 1..7 zero
    float b1[16], b2[16], b3[4];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

// d += a (16x16, row) * b (16x8, col); BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// W [CO][CI][27] (FP32) -> sW [27][NR][16] BF16 (zero beyond CI and CO).
template <int CI, int CO, int NR>
__device__ __forceinline__ void stage_w(const float* __restrict__ W, __nv_bfloat16* sW)
{
    for (int q = threadIdx.x; q < 27 * NR * 16; q += blockDim.x) {
        const int k = q % 16, n = (q / 16) % NR, t = q / (16 * NR);
        const float v = (k < CI && n < CO) ? W[(n * CI + k) * 27 + t] : 0.f;
        sW[q] = __float2bfloat16_rn(v);
    }
}

// Per-lane A-row data of the warp's NTL tiles (tile q starts at point p0 + 128 q):
// the byte offset of the lane's row (plus its K half) and the 27-bit mask of the
// taps that stay inside the element.  The same for every layer and element.
template <int NTL>
struct TileRows {
    uint32_t off[NTL];
    uint32_t valid[NTL];
    uint32_t zero_off;  // the all-zero row NP, same K half
    __device__ __forceinline__ TileRows(int p0, int lane)
    {
        const int mrow = (lane & 7) + 8 * ((lane >> 3) & 1);
        const uint32_t kofs = 2u * (uint32_t)(8 * (lane >> 4));
        zero_off = 2u * (uint32_t)(NP * RS) + kofs;
#pragma unroll
        for (int q = 0; q < NTL; q++) {
            const int p = p0 + 128 * q + mrow;
            const int i = p & 7, j = (p >> 3) & 7, k = p >> 6;
            off[q] = 2u * (uint32_t)(p * RS) + kofs;
            uint32_t m = 0;
            for (int t = 0; t < 27; t++) {
                const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
                if ((unsigned)(i + di) < 8u && (unsigned)(j + dj) < 8u && (unsigned)(k + dk) < 8u) m |= 1u << t;
            }
            valid[q] = m;
        }
    }
};

// One layer for the warp's NTL point tiles: acc[q][h] += sum_taps
// A_shift(16 x 16) W_tap(16 x 8h..8h+7).  The tiles give NTL independent
// accumulation chains, and each tap's B fragment is loaded once for all of them.
// NH = 2 (16 outputs) or 1 (8 outputs).
template <int NH, int WROWS, int NTL>
__device__ __forceinline__ void conv_tiles(const __nv_bfloat16* act, const __nv_bfloat16* w, const TileRows<NTL>& R,
                                           int lane, float (&acc)[NTL][2][4])
{
    const uint32_t abase = smem_u32(act);
    // B rows: n = (lane & 7) + 8 * (lane >> 4) (x4) or (lane & 7) (x2); k offset 8 * ((lane >> 3) & 1)
    const int bn = NH == 2 ? (lane & 7) + 8 * (lane >> 4) : (lane & 7);
    const uint32_t bbase = smem_u32(w) + 2u * (uint32_t)(bn * 16 + 8 * ((lane >> 3) & 1));
#pragma unroll
    for (int q = 0; q < NTL; q++)
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int r = 0; r < 4; r++) acc[q][h][r] = 0.f;
#pragma unroll 3
    for (int t = 0; t < 27; t++) {
        const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
        const int shift = 2 * RS * (di + 8 * dj + 64 * dk);  // byte offset of the tap's neighbour row
        const uint32_t baddr = bbase + 2u * (uint32_t)(t * WROWS * 16);
        uint32_t b0, b1, b2 = 0, b3 = 0;
        if constexpr (NH == 2)
            ldsm_x4(baddr, b0, b1, b2, b3);  // (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
        else
            ldsm_x2(baddr, b0, b1);
#pragma unroll
        for (int q = 0; q < NTL; q++) {
            const uint32_t off = ((R.valid[q] >> t) & 1u) ? R.off[q] + (uint32_t)shift : R.zero_off;
            uint32_t a0, a1, a2, a3;
            ldsm_x4(abase + off, a0, a1, a2, a3);
            mma_bf16(acc[q][0], a0, a1, a2, a3, b0, b1);
            if constexpr (NH == 2) mma_bf16(acc[q][1], a0, a1, a2, a3, b2, b3);
        }
    }
}

// bias + GELU, rounded to BF16, into rows p0 + (lane / 4) and p0 + 8 + (lane / 4) of out.
__device__ __forceinline__ void store_hidden(const float (&acc)[2][4], const float* bias, __nv_bfloat16* out, int p0,
                                             int lane)
{
    const int r0 = p0 + (lane >> 2), r1 = r0 + 8;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int n = 8 * h + 2 * (lane & 3);
        const __nv_bfloat162 v0 = __floats2bfloat162_rn(gelu_tc(acc[h][0] + bias[n]), gelu_tc(acc[h][1] + bias[n + 1]));
        const __nv_bfloat162 v1 = __floats2bfloat162_rn(gelu_tc(acc[h][2] + bias[n]), gelu_tc(acc[h][3] + bias[n + 1]));
        *reinterpret_cast<__nv_bfloat162*>(out + r0 * RS + n) = v0;
        *reinterpret_cast<__nv_bfloat162*>(out + r1 * RS + n) = v1;
    }
}

__global__ void __launch_bounds__(NT_TC, 2) k_net_apply_tc(int64_t nelt, const float* __restrict__ theta,
                                                        const float* __restrict__ xin,
                                                        const float* __restrict__ scale,
                                                        const double* __restrict__ c, double* __restrict__ z)
{
    extern __shared__ __align__(16) unsigned char raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    stage_w<CIN, CH, 16>(theta + OW1, S.w1);
    stage_w<CH, CH, 16>(theta + OW2, S.w2);
    stage_w<CH, 1, 8>(theta + OW3, S.w3);
    if (tid < CH) {
        S.b1[tid] = __bfloat162float(__float2bfloat16_rn(theta[OB1 + tid]));
        S.b2[tid] = __bfloat162float(__float2bfloat16_rn(theta[OB2 + tid]));
    }
    if (tid == 0) S.b3[0] = __bfloat162float(__float2bfloat16_rn(theta[OB3]));
    // zero rows, and input channels 2..RS-1 (never written afterwards)
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int q = tid; q < (NP + 1) * RS; q += NT_TC) {
        if (q / RS == NP || q % RS >= CIN) S.x[q] = zero;
        if (q / RS == NP) {
            S.a1[q] = zero;
            S.a2[q] = zero;
        }
    }
    const TileRows<4> rows(16 * warp, lane);
    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        __syncthreads();  // previous element done with every buffer
        for (int p = tid; p < NP; p += NT_TC) {
            S.x[p * RS + 0] = __float2bfloat16_rn(xin[(e * CIN + 0) * NP + p]);
            S.x[p * RS + 1] = __float2bfloat16_rn(xin[(e * CIN + 1) * NP + p]);
        }
        __syncthreads();
        // warp w owns the tiles starting at points 16 w + 128 q, q = 0..3
        float acc[4][2][4];
        conv_tiles<2, 16, 4>(S.x, S.w1, rows, lane, acc);
#pragma unroll
        for (int q = 0; q < 4; q++) store_hidden(acc[q], S.b1, S.a1, 16 * warp + 128 * q, lane);
        __syncthreads();
        conv_tiles<2, 16, 4>(S.a1, S.w2, rows, lane, acc);
#pragma unroll
        for (int q = 0; q < 4; q++) store_hidden(acc[q], S.b2, S.a2, 16 * warp + 128 * q, lane);
        __syncthreads();
        const double sc = (double)scale[e];
        conv_tiles<1, 8, 4>(S.a2, S.w3, rows, lane, acc);
        if ((lane & 3) == 0) {  // column n = 0 of the accumulators: rows lane/4 and lane/4 + 8 of each tile
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int p0 = 16 * warp + 128 * q + (lane >> 2), p1 = p0 + 8;
                z[e * NP + p0] = (double)(acc[q][0][0] + S.b3[0]) * sc * c[e * NP + p0];
                z[e * NP + p1] = (double)(acc[q][0][2] + S.b3[0]) * sc * c[e * NP + p1];
            }
        }
    }
}

}  // namespace

nek_status launch_net_apply_tc(int64_t nelt, const float* theta, const float* xin, const float* scale,
                               const double* c, double* z, cudaStream_t s)
{
    static std::atomic<uint64_t> configured{0};
    nek_status st = ensure_dyn_smem(k_net_apply_tc, sizeof(TcSmem), configured);
    if (st != NEK_OK) return st;
    const int grid = static_cast<int>(nelt < 152 * 2 ? nelt : 152 * 2);
    k_net_apply_tc<<<grid, NT_TC, sizeof(TcSmem), s>>>(nelt, theta, xin, scale, c, z);
    return check_launch();
}

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_net_apply_bf16_mma(int64_t nelt, int nx, const float* theta, const float* xin, const float* scale,
                                  const double* c, double* z, void* stream)
{
    if (nx != NXN) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!theta || !xin || !scale || !c || !z) return NEK_ERR_INVALID_ARG;
    return launch_net_apply_tc(nelt, theta, xin, scale, c, z, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
