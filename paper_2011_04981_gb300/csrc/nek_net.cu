// Learned element preconditioner: a small 3D convolutional network applied to
// every nx = 8 element block, its training kernels, and flexible CG using it.
//
// The network (no counterpart in the paper, which uses Nekbone's fixed
// preconditioner): input channels r/rms(r) and (Jacobi r)/rms(Jacobi r) of one
// element; three 3x3x3 convolutions with zero padding inside the element,
// 16 hidden channels and GELU after the first two; BF16 weights (FP32 master
// copy, rounded when staged), FP32 activations and accumulation.  The output,
// times rms(Jacobi r) and 1/multiplicity, summed over elements by dssum and
// masked, is the preconditioned residual.
//
// Parameter vector (FP32): W1 [16][2][27], b1 [16], W2 [16][16][27], b2 [16],
// W3 [1][16][27], b3 [1]; tap t = (dk+1)*9 + (dj+1)*3 + (di+1) reads the point
// (i+di, j+dj, k+dk).
#include <cuda_bf16.h>

#include <vector>

#include "nek_internal.h"
#include "nek_pcg.cuh"

namespace nek {

namespace {

constexpr int NXN = 8, NP = 512, CIN = 2, CH = 16;
constexpr int OW1 = 0, OB1 = OW1 + CH * CIN * 27, OW2 = OB1 + CH, OB2 = OW2 + CH * CH * 27, OW3 = OB2 + CH,
              OB3 = OW3 + CH * 27, NPARAM = OB3 + 1;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float gelu(float v) { return 0.5f * v * (1.f + erff(v * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float v)
{
    return 0.5f * (1.f + erff(v * 0.70710678118654752f)) + v * expf(-0.5f * v * v) * 0.39894228040143268f;
}

// Weights staged in shared memory as [cin][27][cout] (BF16-rounded floats).
template <int CI, int CO>
__device__ __forceinline__ void stage_weights(const float* __restrict__ W, float* sW)
{
    for (int q = threadIdx.x; q < CI * 27 * CO; q += blockDim.x) {
        const int o = q % CO, t = (q / CO) % 27, c = q / (CO * 27);
        sW[q] = bf16r(W[(o * CI + c) * 27 + t]);
    }
}

// acc[o] = bias[o] + sum_c sum_t W[o][c][t] x[c][p + t] for point p = (i, j, k).
template <int CI, int CO>
__device__ __forceinline__ void conv_point(const float* xin, const float* sW, const float* sb, int i, int j, int k,
                                           float (&acc)[CO])
{
#pragma unroll
    for (int o = 0; o < CO; o++) acc[o] = sb[o];
#pragma unroll
    for (int t = 0; t < 27; t++) {
        const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
        const int ii = i + di, jj = j + dj, kk = k + dk;
        if (ii < 0 || ii >= NXN || jj < 0 || jj >= NXN || kk < 0 || kk >= NXN) continue;
        const int q = ii + NXN * (jj + NXN * kk);
#pragma unroll 4
        for (int c = 0; c < CI; c++) {
            const float xv = xin[c * NP + q];
            const float* w = sW + (c * 27 + t) * CO;
#pragma unroll
            for (int o = 0; o < CO; o++) acc[o] = fmaf(w[o], xv, acc[o]);
        }
    }
}

// Two points per thread, p and p + NP/2 (planes k and k + 4): every weight read
// from shared memory feeds two FMAs.
template <int CI, int CO>
__device__ __forceinline__ void conv_2pts(const float* xin, const float* sW, const float* sb, int i, int j, int k,
                                          float (&acc0)[CO], float (&acc1)[CO])
{
#pragma unroll
    for (int o = 0; o < CO; o++) acc0[o] = acc1[o] = sb[o];
#pragma unroll
    for (int t = 0; t < 27; t++) {
        const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
        const int ii = i + di, jj = j + dj, k0 = k + dk, k1 = k + 4 + dk;
        if (ii < 0 || ii >= NXN || jj < 0 || jj >= NXN) continue;
        const bool v0 = k0 >= 0, v1 = k1 < NXN;  // k0 < 8 and k1 >= 0 always hold for k in [0,4)
        const int q0 = ii + NXN * (jj + NXN * k0), q1 = ii + NXN * (jj + NXN * k1);
#pragma unroll 4
        for (int c = 0; c < CI; c++) {
            const float x0 = v0 ? xin[c * NP + q0] : 0.f;
            const float x1 = v1 ? xin[c * NP + q1] : 0.f;
            const float* w = sW + (c * 27 + t) * CO;
#pragma unroll
            for (int o = 0; o < CO; o++) {
                const float wo = w[o];
                acc0[o] = fmaf(wo, x0, acc0[o]);
                acc1[o] = fmaf(wo, x1, acc1[o]);
            }
        }
    }
}

// ------------------------------------------------------------------ prep
// xin[e][0][p] = r/rms(r), xin[e][1][p] = (minv r)/rms(minv r); scale[e] = rms(minv r).
// One warp per element: lane l holds points l + 32 q (q = 0..15, coalesced), sums
// its FP64 squares, the warp sums the lanes with a fixed shuffle tree, and lane 0
// forms the two RMS values and their reciprocals (FP64 square root and division
// on one lane); no block-wide barrier, so the warps of a CTA work on different
// elements independently.
constexpr int kPrepWarps = 8;

__global__ void __launch_bounds__(32 * kPrepWarps) k_net_prep(int64_t nelt, const double* __restrict__ r,
                                                               const double* __restrict__ minv,
                                                               float* __restrict__ xin, float* __restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    for (int64_t e = (int64_t)blockIdx.x * kPrepWarps + (threadIdx.x >> 5); e < nelt;
         e += (int64_t)gridDim.x * kPrepWarps) {
        double rv[NP / 32], jv[NP / 32];
#pragma unroll
        for (int q = 0; q < NP / 32; q++) {
            const int64_t o = e * NP + lane + 32 * q;
            rv[q] = r[o];
            jv[q] = minv[o] * rv[q];
        }
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int q = 0; q < NP / 32; q++) {
            a += rv[q] * rv[q];
            b += jv[q] * jv[q];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        double ia = 0.0, ib = 0.0;
        if (lane == 0) {
            const double ra = sqrt(a / NP), rb = sqrt(b / NP);
            ia = ra > 0.0 ? 1.0 / ra : 0.0;
            ib = rb > 0.0 ? 1.0 / rb : 0.0;
            scale[e] = (float)rb;
        }
        ia = __shfl_sync(0xffffffffu, ia, 0);
        ib = __shfl_sync(0xffffffffu, ib, 0);
#pragma unroll
        for (int q = 0; q < NP / 32; q++) {
            xin[(e * CIN + 0) * NP + lane + 32 * q] = (float)(rv[q] * ia);
            xin[(e * CIN + 1) * NP + lane + 32 * q] = (float)(jv[q] * ib);
        }
    }
}

// ------------------------------------------------------------------ inference
struct ApplySmem {
    float x[CIN * NP];
    float a1[CH * NP];
    float a2[CH * NP];
    float w1[CIN * 27 * CH];
    float w2[CH * 27 * CH];
    float w3[CH * 27];
    float b1[CH], b2[CH], b3[4];
};

// z[e][p] = net(xin[e])[p] * scale[e] * c[e][p] (FP64 out).  NP/2 threads per
// element, each computing points p and p + NP/2.
constexpr int NT_APPLY = NP / 2;
__global__ void __launch_bounds__(NT_APPLY) k_net_apply(int64_t nelt, const float* __restrict__ theta,
                                                        const float* __restrict__ xin,
                                                        const float* __restrict__ scale,
                                                        const double* __restrict__ c, double* __restrict__ z)
{
    extern __shared__ __align__(16) unsigned char raw[];
    ApplySmem& S = *reinterpret_cast<ApplySmem*>(raw);
    stage_weights<CIN, CH>(theta + OW1, S.w1);
    stage_weights<CH, CH>(theta + OW2, S.w2);
    stage_weights<CH, 1>(theta + OW3, S.w3);
    if (threadIdx.x < CH) {
        S.b1[threadIdx.x] = bf16r(theta[OB1 + threadIdx.x]);
        S.b2[threadIdx.x] = bf16r(theta[OB2 + threadIdx.x]);
    }
    if (threadIdx.x == 0) S.b3[0] = bf16r(theta[OB3]);
    const int p = threadIdx.x, p1 = p + NT_APPLY;
    const int i = p % NXN, j = (p / NXN) % NXN, k = p / (NXN * NXN);  // k in [0, 4)
    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        __syncthreads();
        S.x[p] = xin[(e * CIN + 0) * NP + p];
        S.x[p1] = xin[(e * CIN + 0) * NP + p1];
        S.x[NP + p] = xin[(e * CIN + 1) * NP + p];
        S.x[NP + p1] = xin[(e * CIN + 1) * NP + p1];
        __syncthreads();
        {
            float a0[CH], a1[CH];
            conv_2pts<CIN, CH>(S.x, S.w1, S.b1, i, j, k, a0, a1);
#pragma unroll
            for (int o = 0; o < CH; o++) {
                S.a1[o * NP + p] = gelu(a0[o]);
                S.a1[o * NP + p1] = gelu(a1[o]);
            }
        }
        __syncthreads();
        {
            float a0[CH], a1[CH];
            conv_2pts<CH, CH>(S.a1, S.w2, S.b2, i, j, k, a0, a1);
#pragma unroll
            for (int o = 0; o < CH; o++) {
                S.a2[o * NP + p] = gelu(a0[o]);
                S.a2[o * NP + p1] = gelu(a1[o]);
            }
        }
        __syncthreads();
        float y0[1], y1[1];
        conv_2pts<CH, 1>(S.a2, S.w3, S.b3, i, j, k, y0, y1);
        z[e * NP + p] = (double)y0[0] * (double)scale[e] * c[e * NP + p];
        z[e * NP + p1] = (double)y1[0] * (double)scale[e] * c[e * NP + p1];
    }
}

// ------------------------------------------------------------------ training
// Forward over a batch of B samples keeping the pre-activations h1, h2 and y.
__global__ void __launch_bounds__(NP) k_net_fwd_train(int B, const float* __restrict__ theta,
                                                      const float* __restrict__ xin, float* __restrict__ h1,
                                                      float* __restrict__ h2, float* __restrict__ y)
{
    extern __shared__ __align__(16) unsigned char raw[];
    ApplySmem& S = *reinterpret_cast<ApplySmem*>(raw);
    stage_weights<CIN, CH>(theta + OW1, S.w1);
    stage_weights<CH, CH>(theta + OW2, S.w2);
    stage_weights<CH, 1>(theta + OW3, S.w3);
    if (threadIdx.x < CH) {
        S.b1[threadIdx.x] = bf16r(theta[OB1 + threadIdx.x]);
        S.b2[threadIdx.x] = bf16r(theta[OB2 + threadIdx.x]);
    }
    if (threadIdx.x == 0) S.b3[0] = bf16r(theta[OB3]);
    const int p = threadIdx.x;
    const int i = p % NXN, j = (p / NXN) % NXN, k = p / (NXN * NXN);
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        __syncthreads();
        S.x[p] = xin[(b * CIN + 0) * NP + p];
        S.x[NP + p] = xin[(b * CIN + 1) * NP + p];
        __syncthreads();
        {
            float acc[CH];
            conv_point<CIN, CH>(S.x, S.w1, S.b1, i, j, k, acc);
#pragma unroll
            for (int o = 0; o < CH; o++) {
                h1[((int64_t)b * CH + o) * NP + p] = acc[o];
                S.a1[o * NP + p] = gelu(acc[o]);
            }
        }
        __syncthreads();
        {
            float acc[CH];
            conv_point<CH, CH>(S.a1, S.w2, S.b2, i, j, k, acc);
#pragma unroll
            for (int o = 0; o < CH; o++) {
                h2[((int64_t)b * CH + o) * NP + p] = acc[o];
                S.a2[o * NP + p] = gelu(acc[o]);
            }
        }
        __syncthreads();
        float yo[1];
        conv_point<CH, 1>(S.a2, S.w3, S.b3, i, j, k, yo);
        y[(int64_t)b * NP + p] = yo[0];
    }
}

// Per sample: loss_b = |y - t|^2 / |t|^2 ; dy = (2/B) (y - t) / |t|^2.
__global__ void __launch_bounds__(NP) k_net_loss(int B, const float* __restrict__ y, const float* __restrict__ t,
                                                 float* __restrict__ dy, float* __restrict__ loss_b)
{
    __shared__ float sh[2][NP / 32];
    const int p = threadIdx.x;
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        const float d = y[(int64_t)b * NP + p] - t[(int64_t)b * NP + p];
        const float tv = t[(int64_t)b * NP + p];
        float a = d * d, c = tv * tv;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if ((p & 31) == 0) {
            sh[0][p >> 5] = a;
            sh[1][p >> 5] = c;
        }
        __syncthreads();
        float num = 0.f, den = 0.f;
        for (int q = 0; q < NP / 32; q++) {
            num += sh[0][q];
            den += sh[1][q];
        }
        __syncthreads();
        den = den > 0.f ? den : 1.f;
        dy[(int64_t)b * NP + p] = 2.f / (float)B * d / den;
        if (p == 0) loss_b[b] = num / den;
    }
}

// d = y - t (FP32, in place into d)
__global__ void k_net_diff(int64_t n, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ d)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        d[q] = y[q] - t[q];
}

// Per sample: loss_b = d.Ad / t.At ; dy = (2/B) Ad / t.At  (A = the sample element's operator).
__global__ void __launch_bounds__(NP) k_net_energy_loss(int B, const float* __restrict__ d, const float* __restrict__ Ad,
                                                        const float* __restrict__ t, const float* __restrict__ At,
                                                        float* __restrict__ dy, float* __restrict__ loss_b)
{
    __shared__ float sh[2][NP / 32];
    const int p = threadIdx.x;
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        const int64_t o = (int64_t)b * NP + p;
        float a = d[o] * Ad[o], c = t[o] * At[o];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, s);
            c += __shfl_xor_sync(0xffffffffu, c, s);
        }
        if ((p & 31) == 0) {
            sh[0][p >> 5] = a;
            sh[1][p >> 5] = c;
        }
        __syncthreads();
        float num = 0.f, den = 0.f;
        for (int q = 0; q < NP / 32; q++) {
            num += sh[0][q];
            den += sh[1][q];
        }
        __syncthreads();
        den = den > 0.f ? den : 1.f;
        dy[o] = 2.f / (float)B * Ad[o] / den;
        if (p == 0) loss_b[b] = num / den;
    }
}

struct BwdSmem {
    float x[CIN * NP];
    float a1[CH * NP];
    float g2[CH * NP];  // a2, then dh2
    float g1[CH * NP];  // dh1
    float dy[NP];
    float w2[CH * 27 * CH];  // [c][t][o]
    float w3[CH * 27];       // [c][t]
};

// d/dx of sum_p g[o][p] * conv(x)[o][p] at input channel c, point q:
// sum_o sum_t W[o][c][t] g[o][q - t]  (W staged as [c][t][o])
template <int CO>
__device__ __forceinline__ float convT_point(const float* g, const float* sW, int c, int i, int j, int k)
{
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < 27; t++) {
        const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
        const int ii = i - di, jj = j - dj, kk = k - dk;
        if (ii < 0 || ii >= NXN || jj < 0 || jj >= NXN || kk < 0 || kk >= NXN) continue;
        const int q = ii + NXN * (jj + NXN * kk);
        const float* w = sW + (c * 27 + t) * CO;
#pragma unroll
        for (int o = 0; o < CO; o++) s = fmaf(w[o], g[o * NP + q], s);
    }
    return s;
}

// dW[o][c][t] = sum_p g[o][p] x[c][p + t] for a 4x4 (o, c) tile and one tap per thread.
template <int CI>
__device__ __forceinline__ void wgrad_tiles(const float* g, const float* x, int CO, float* out /*[CO][CI][27]*/)
{
    const int otiles = (CO + 3) / 4, ctiles = (CI + 3) / 4;
    const int ntask = otiles * ctiles * 27;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        const int t = task % 27, ct = (task / 27) % ctiles, ot = task / (27 * ctiles);
        const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
        float acc[4][4] = {};
        for (int p = 0; p < NP; p++) {
            const int i = p % NXN, j = (p / NXN) % NXN, k = p / (NXN * NXN);
            const int ii = i + di, jj = j + dj, kk = k + dk;
            if (ii < 0 || ii >= NXN || jj < 0 || jj >= NXN || kk < 0 || kk >= NXN) continue;
            const int q = ii + NXN * (jj + NXN * kk);
            float gv[4], xv[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                const int o = ot * 4 + a, c = ct * 4 + a;
                gv[a] = o < CO ? g[o * NP + p] : 0.f;
                xv[a] = c < CI ? x[c * NP + q] : 0.f;
            }
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int bb = 0; bb < 4; bb++) acc[a][bb] = fmaf(gv[a], xv[bb], acc[a][bb]);
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int bb = 0; bb < 4; bb++) {
                const int o = ot * 4 + a, c = ct * 4 + bb;
                if (o < CO && c < CI) out[(o * CI + c) * 27 + t] = acc[a][bb];
            }
    }
}

// Backward for one sample per block iteration: per-sample gradient vector gs[b][NPARAM].
__global__ void __launch_bounds__(NP) k_net_bwd(int B, const float* __restrict__ theta,
                                                const float* __restrict__ xin, const float* __restrict__ h1,
                                                const float* __restrict__ h2, const float* __restrict__ dy,
                                                float* __restrict__ gs)
{
    extern __shared__ __align__(16) unsigned char raw[];
    BwdSmem& S = *reinterpret_cast<BwdSmem*>(raw);
    stage_weights<CH, CH>(theta + OW2, S.w2);
    stage_weights<CH, 1>(theta + OW3, S.w3);
    const int p = threadIdx.x;
    const int i = p % NXN, j = (p / NXN) % NXN, k = p / (NXN * NXN);
    __shared__ float red[CH][NP / 32];
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        float* g = gs + (int64_t)b * NPARAM;
        __syncthreads();
        S.x[p] = xin[(b * CIN + 0) * NP + p];
        S.x[NP + p] = xin[(b * CIN + 1) * NP + p];
        S.dy[p] = dy[(int64_t)b * NP + p];
#pragma unroll
        for (int o = 0; o < CH; o++) {
            S.a1[o * NP + p] = gelu(h1[((int64_t)b * CH + o) * NP + p]);
            S.g2[o * NP + p] = gelu(h2[((int64_t)b * CH + o) * NP + p]);
        }
        __syncthreads();
        // layer 3: dW3 = sum_p dy a2(p + t); db3 = sum dy
        wgrad_tiles<CH>(S.dy, S.g2, 1, g + OW3);
        __syncthreads();
        // dh2 = gelu'(h2) * convT(dy; W3)
#pragma unroll
        for (int c = 0; c < CH; c++) {
            const float v = convT_point<1>(S.dy, S.w3, c, i, j, k);
            S.g2[c * NP + p] = v * gelu_grad(h2[((int64_t)b * CH + c) * NP + p]);
        }
        __syncthreads();
        // layer 2: dW2 = sum_p dh2 a1(p + t)
        wgrad_tiles<CH>(S.g2, S.a1, CH, g + OW2);
        // dh1 = gelu'(h1) * convT(dh2; W2)
#pragma unroll 4
        for (int c = 0; c < CH; c++) {
            const float v = convT_point<CH>(S.g2, S.w2, c, i, j, k);
            S.g1[c * NP + p] = v * gelu_grad(h1[((int64_t)b * CH + c) * NP + p]);
        }
        __syncthreads();
        // layer 1: dW1 = sum_p dh1 x(p + t)
        wgrad_tiles<CIN>(S.g1, S.x, CH, g + OW1);
        // biases: sums over the block's points (fixed shuffle tree)
        {
            float v3 = S.dy[p];
            float v2[CH], v1[CH];
#pragma unroll
            for (int o = 0; o < CH; o++) {
                v2[o] = S.g2[o * NP + p];
                v1[o] = S.g1[o * NP + p];
            }
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                v3 += __shfl_xor_sync(0xffffffffu, v3, s);
#pragma unroll
                for (int o = 0; o < CH; o++) {
                    v2[o] += __shfl_xor_sync(0xffffffffu, v2[o], s);
                    v1[o] += __shfl_xor_sync(0xffffffffu, v1[o], s);
                }
            }
            __syncthreads();
            if ((p & 31) == 0) {
                red[0][p >> 5] = v3;
            }
            __syncthreads();
            if (p == 0) {
                float s = 0.f;
                for (int q = 0; q < NP / 32; q++) s += red[0][q];
                g[OB3] = s;
            }
            __syncthreads();
            if ((p & 31) == 0)
                for (int o = 0; o < CH; o++) red[o][p >> 5] = v2[o];
            __syncthreads();
            if (p < CH) {
                float s = 0.f;
                for (int q = 0; q < NP / 32; q++) s += red[p][q];
                g[OB2 + p] = s;
            }
            __syncthreads();
            if ((p & 31) == 0)
                for (int o = 0; o < CH; o++) red[o][p >> 5] = v1[o];
            __syncthreads();
            if (p < CH) {
                float s = 0.f;
                for (int q = 0; q < NP / 32; q++) s += red[p][q];
                g[OB1 + p] = s;
            }
        }
    }
}

// grad[q] = sum_b gs[b][q] in order; loss = sum_b loss_b / B.
__global__ void k_net_reduce(int B, const float* __restrict__ gs, const float* __restrict__ loss_b,
                             float* __restrict__ grad, float* __restrict__ loss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < NPARAM) {
        float s = 0.f;
        for (int b = 0; b < B; b++) s += gs[(int64_t)b * NPARAM + q];
        grad[q] = s;
    }
    if (q == 0 && loss) {
        float s = 0.f;
        for (int b = 0; b < B; b++) s += loss_b[b];
        loss[0] = s / (float)B;
    }
}

__global__ void k_adam(int n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    th[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

std::atomic<uint64_t> g_apply_conf{0}, g_fwd_conf{0}, g_bwd_conf{0};

int grid_for(int64_t n) { return static_cast<int>(n < 152 * 2 ? n : 152 * 2); }

}  // namespace

nek_status launch_net_apply(int64_t nelt, const float* theta, const float* xin, const float* scale, const double* c,
                            double* z, cudaStream_t s)
{
    nek_status st = ensure_dyn_smem(k_net_apply, sizeof(ApplySmem), g_apply_conf);
    if (st != NEK_OK) return st;
    k_net_apply<<<static_cast<int>(nelt < 152 * 2 ? nelt : 152 * 2), NT_APPLY, sizeof(ApplySmem), s>>>(nelt, theta,
                                                                                                  xin, scale, c, z);
    return check_launch();
}

// target[e][p] = (xs - xk)[e][p] / scale[e] (FP64 difference and quotient, one FP32 rounding); 0 where
// the element's scale is 0.
__global__ void k_net_target(int64_t n, const double* __restrict__ xs, const double* __restrict__ xk,
                             const float* __restrict__ scale, float* __restrict__ target)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const double s = (double)scale[q / NP];
        target[q] = s > 0.0 ? (float)((xs[q] - xk[q]) / s) : 0.f;
    }
}

nek_status launch_net_prep(int64_t nelt, const double* r, const double* minv, float* xin, float* scale,
                           cudaStream_t s)
{
    const int64_t nb = (nelt + kPrepWarps - 1) / kPrepWarps;
    k_net_prep<<<static_cast<int>(nb < 152 * 16 ? nb : 152 * 16), 32 * kPrepWarps, 0, s>>>(nelt, r, minv, xin, scale);
    return check_launch();
}

}  // namespace nek

using namespace nek;

namespace {

inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct TrainLayout {
    float *h1, *h2, *y, *dy, *lossb, *gs, *d, *Ad, *At;
    size_t bytes;
};

TrainLayout train_layout(char* base, int B)
{
    TrainLayout L{};
    size_t off = 0;
    auto take = [&](size_t n) {
        char* q = base ? base + off : nullptr;
        off += al256(n);
        return reinterpret_cast<float*>(q);
    };
    L.h1 = take(sizeof(float) * (size_t)B * CH * NP);
    L.h2 = take(sizeof(float) * (size_t)B * CH * NP);
    L.y = take(sizeof(float) * (size_t)B * NP);
    L.dy = take(sizeof(float) * (size_t)B * NP);
    L.lossb = take(sizeof(float) * (size_t)B);
    L.gs = take(sizeof(float) * (size_t)B * NPARAM);
    L.d = take(sizeof(float) * (size_t)B * NP);
    L.Ad = take(sizeof(float) * (size_t)B * NP);
    L.At = take(sizeof(float) * (size_t)B * NP);
    L.bytes = off;
    return L;
}

}  // namespace

extern "C" {

int nek_net_param_count(void) { return NPARAM; }

nek_status nek_net_prep(int64_t nelt, int nx, const double* r, const double* minv, float* xin, float* scale,
                        void* stream)
{
    if (nx != NXN) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!r || !minv || !xin || !scale) return NEK_ERR_INVALID_ARG;
    return launch_net_prep(nelt, r, minv, xin, scale, static_cast<cudaStream_t>(stream));
}

nek_status nek_net_target(int64_t nelt, int nx, const double* xs, const double* xk, const float* scale,
                          float* target, void* stream)
{
    if (nx != NXN) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!xs || !xk || !scale || !target) return NEK_ERR_INVALID_ARG;
    const int64_t n = nelt * NP;
    k_net_target<<<pcg::stream_blocks(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, xs, xk, scale, target);
    return check_launch();
}

nek_status nek_net_apply(int64_t nelt, int nx, const float* theta, const float* xin, const float* scale,
                         const double* c, double* z, void* stream)
{
    if (nx != NXN) return NEK_ERR_UNSUPPORTED_NX;
    if (nelt < 0) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!theta || !xin || !scale || !c || !z) return NEK_ERR_INVALID_ARG;
    return launch_net_apply(nelt, theta, xin, scale, c, z, static_cast<cudaStream_t>(stream));
}

size_t nek_net_train_workspace_bytes(int batch) { return batch > 0 ? train_layout(nullptr, batch).bytes : 0; }

nek_status nek_net_forward_batch(int batch, const float* theta, const float* xin, float* y, void* workspace,
                                 void* stream)
{
    if (batch <= 0 || !theta || !xin || !y || !workspace || !is_aligned(workspace, 256)) return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TrainLayout L = train_layout(static_cast<char*>(workspace), batch);
    nek_status st = ensure_dyn_smem(k_net_fwd_train, sizeof(ApplySmem), g_fwd_conf);
    if (st != NEK_OK) return st;
    k_net_fwd_train<<<grid_for(batch), NP, sizeof(ApplySmem), s>>>(batch, theta, xin, L.h1, L.h2, y);
    return check_launch();
}

nek_status nek_net_train_grad(int batch, const float* theta, const float* xin, const float* target, float* grad,
                              float* loss, void* workspace, void* stream)
{
    if (batch <= 0 || !theta || !xin || !target || !grad || !workspace || !is_aligned(workspace, 256))
        return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TrainLayout L = train_layout(static_cast<char*>(workspace), batch);
    nek_status st0 = ensure_dyn_smem(k_net_fwd_train, sizeof(ApplySmem), g_fwd_conf);
    if (st0 == NEK_OK) st0 = ensure_dyn_smem(k_net_bwd, sizeof(BwdSmem), g_bwd_conf);
    if (st0 != NEK_OK) return st0;
    k_net_fwd_train<<<grid_for(batch), NP, sizeof(ApplySmem), s>>>(batch, theta, xin, L.h1, L.h2, L.y);
    k_net_loss<<<grid_for(batch), NP, 0, s>>>(batch, L.y, target, L.dy, L.lossb);
    k_net_bwd<<<grid_for(batch), NP, sizeof(BwdSmem), s>>>(batch, theta, xin, L.h1, L.h2, L.dy, L.gs);
    k_net_reduce<<<(NPARAM + 255) / 256, 256, 0, s>>>(batch, L.gs, L.lossb, grad, loss);
    return check_launch();
}

nek_status nek_net_train_grad_energy(int batch, const float* theta, const float* xin, const float* target,
                                     const double* D, const float* Glp32, const float* gscale, float* grad,
                                     float* loss, void* workspace, void* stream)
{
    if (batch <= 0 || !theta || !xin || !target || !D || !Glp32 || !gscale || !grad || !workspace ||
        !is_aligned(workspace, 256))
        return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TrainLayout L = train_layout(static_cast<char*>(workspace), batch);
    nek_status st0 = ensure_dyn_smem(k_net_fwd_train, sizeof(ApplySmem), g_fwd_conf);
    if (st0 == NEK_OK) st0 = ensure_dyn_smem(k_net_bwd, sizeof(BwdSmem), g_bwd_conf);
    if (st0 != NEK_OK) return st0;
    const int64_t n = (int64_t)batch * NP;
    k_net_fwd_train<<<grid_for(batch), NP, sizeof(ApplySmem), s>>>(batch, theta, xin, L.h1, L.h2, L.y);
    k_net_diff<<<pcg::stream_blocks(n), 256, 0, s>>>(n, L.y, target, L.d);
    nek_status st = check_launch();
    if (st != NEK_OK) return st;
    if ((st = launch_ax_lowp(NEK_PREC_F32, batch, NXN, D, Glp32, gscale, L.d, L.Ad, s)) != NEK_OK) return st;
    if ((st = launch_ax_lowp(NEK_PREC_F32, batch, NXN, D, Glp32, gscale, target, L.At, s)) != NEK_OK) return st;
    k_net_energy_loss<<<grid_for(batch), NP, 0, s>>>(batch, L.d, L.Ad, target, L.At, L.dy, L.lossb);
    k_net_bwd<<<grid_for(batch), NP, sizeof(BwdSmem), s>>>(batch, theta, xin, L.h1, L.h2, L.dy, L.gs);
    k_net_reduce<<<(NPARAM + 255) / 256, 256, 0, s>>>(batch, L.gs, L.lossb, grad, loss);
    return check_launch();
}

nek_status nek_adam_step(int n, float* theta, const float* grad, float* m, float* v, float lr, float beta1,
                         float beta2, float eps, int step, void* stream)
{
    if (n <= 0 || !theta || !grad || !m || !v || step < 1 || !(lr > 0.f)) return NEK_ERR_INVALID_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, theta, grad, m, v, lr, beta1, beta2,
                                                                           eps, c1, c2);
    return check_launch();
}

}  // extern "C"
