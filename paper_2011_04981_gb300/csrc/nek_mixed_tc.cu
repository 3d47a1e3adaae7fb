// Reduced-precision AX (BF16 / FP16 operands) with the D-contractions on the
// tensor cores: every contraction of the element is a 16 x 16 x 16 matrix
// product per plane (nx padded to 16 with zeros), mma.sync.m16n8k16 with FP32
// accumulation.  Same arithmetic as the CUDA-core form (nek_mixed.cu):
//   u_q = rnd(u / s_u), D_q = rnd(D), FP32 sums of exact products,
//   [wr ws wt] = rnd(G_q [ur us ut]) in FP32, w = s_u s_G sum_a D_q^T w_a,
// only the order of the FP32 additions inside a contraction differs.
//
// One CTA of four warps per element (grid-stride over elements).  Shared
// memory holds u_q as U[k][j][i] and wt as WT[k][j][i] (16^3 each, zero
// padded), and an FP32 block X[k][j][i] (nx^3) that carries ut, then the
// r- and s-parts of w, then w.  With A = rows i, the contractions are
//   ur(i,j) = D_q[i][l] U[k][j][l]         (A: D_q,       B: rows of U[k])
//   us(i,j) = U[k][l][i] D_q[j][l]         (A: U[k]^T,    B: D_q)
//   ut(i,k) = U[l][j][i] D_q[k][l]         (A: U[.][j]^T, B: D_q), per j
// and in phase 2, for plane k, C(i,j) = D_q[l][i] wr(l,j) + ws(i,l) D_q[l][j]
// from the warp's plane buffers, and per j the t-part U-like sum over planes.
// A warp handles the planes k and the lines j congruent to its index mod 4.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "nek_internal.h"

namespace nek {

namespace {

constexpr int TCW = 4;  // warps per element

template <class S>
struct TcType;
template <>
struct TcType<__nv_bfloat16> {
    __device__ static __forceinline__ __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
    __device__ static __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ float bits_to_f(unsigned short h) { return __uint_as_float((unsigned)h << 16); }
    __device__ static __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
    {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};
template <>
struct TcType<__half> {
    __device__ static __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
    __device__ static __forceinline__ float to_f(__half v) { return __half2float(v); }
    __device__ static __forceinline__ float bits_to_f(unsigned short h) { return __half2float(__ushort_as_half(h)); }
    __device__ static __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
    {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm4(uint32_t a, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void ldsm4t(uint32_t a, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// Lane address offsets (in elements of a 16 x 16 tile with row stride `rs`):
//   A from row-major M[m][k] (ldmatrix):           row (L&7) + 8((L>>3)&1), col 8(L>>4)
//   A from T[k][m], A[m][k] = T[k][m] (.trans):    row (L&7) + 8(L>>4),     col 8((L>>3)&1)
//   B (both n-halves) from [n][k] storage:         row (L&7) + 8(L>>4),     col 8((L>>3)&1)
__device__ __forceinline__ int a_row(int L) { return (L & 7) + 8 * ((L >> 3) & 1); }
__device__ __forceinline__ int a_col(int L) { return 8 * (L >> 4); }
__device__ __forceinline__ int t_row(int L) { return (L & 7) + 8 * (L >> 4); }
__device__ __forceinline__ int t_col(int L) { return 8 * ((L >> 3) & 1); }

template <class S, int NX>
struct TcSmemLp {
    S U[16 * 16 * 16];        // u_q[k][j][i], zero outside nx^3
    S WT[16 * 16 * 16];       // rnd(wt)[k][j][i], zero outside nx^3
    S PR[TCW][16 * 16];       // per warp: rnd(wr) of its current plane at [j][i]
    S PS[TCW][16 * 16];       // per warp: rnd(ws) of its current plane at [j][i]
    S DQ[16 * 16];            // D_q[a][b] at [a][b], zero padded
    S DQT[16 * 16];           // D_q[b][a] at [a][b]
    float X[NX * NX * NX];    // ut, then the r+s part of w, then w (FP32, [k][j][i])
    float red[TCW];
};

template <class S, int NX>
__global__ void __launch_bounds__(32 * TCW) k_ax_lowp_tc(int64_t nelt, const double* __restrict__ D,
                                                         const S* __restrict__ Glp,
                                                         const float* __restrict__ gscale,
                                                         const float* __restrict__ u, float* __restrict__ w)
{
    using T = TcType<S>;
    constexpr int N2 = NX * NX, N3 = NX * NX * NX, NT = 32 * TCW;
    constexpr int PER = (N3 + NT - 1) / NT;  // u values per thread
    extern __shared__ __align__(16) unsigned char raw[];
    TcSmemLp<S, NX>& sm = *reinterpret_cast<TcSmemLp<S, NX>*>(raw);
    const int tid = threadIdx.x, L = tid & 31, wp = tid >> 5;
    const int g = L >> 2, c = L & 3;

    // zero padding (never overwritten outside nx^3) and D_q, D_q^T
    {
        const S zero = T::from_f(0.f);
        for (int q = tid; q < 16 * 16 * 16; q += NT) {
            sm.U[q] = zero;
            sm.WT[q] = zero;
        }
        for (int q = tid; q < 256; q += NT) {
            const int a = q >> 4, b = q & 15;
            sm.DQ[q] = (a < NX && b < NX) ? T::from_f((float)D[a * NX + b]) : zero;
            sm.DQT[q] = (a < NX && b < NX) ? T::from_f((float)D[b * NX + a]) : zero;
        }
    }
    __syncthreads();
    // constant fragments: D_q and D_q^T as A (row-major) and as B ([n][k] storage)
    uint32_t AD[4], ADT[4], BD[4], BDT[4];
    ldsm4(smem_addr(sm.DQ + a_row(L) * 16 + a_col(L)), AD);
    ldsm4(smem_addr(sm.DQT + a_row(L) * 16 + a_col(L)), ADT);
    ldsm4(smem_addr(sm.DQ + t_row(L) * 16 + t_col(L)), BD);     // B[l][n] = D_q[n][l]
    ldsm4(smem_addr(sm.DQT + t_row(L) * 16 + t_col(L)), BDT);   // B[l][n] = D_q[l][n]

    for (int64_t e = blockIdx.x; e < nelt; e += gridDim.x) {
        // ---------------------------------------------------------- stage u_q
        float uv[PER];
        float m = 0.f;
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const int q = tid + r * NT;
            uv[r] = q < N3 ? __ldg(u + e * N3 + q) : 0.f;
            m = fmaxf(m, fabsf(uv[r]));
        }
        m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
        if (L == 0) sm.red[wp] = m;
        __syncthreads();  // also: the previous element is done with U, WT, X
        float mx = 0.f;
#pragma unroll
        for (int q = 0; q < TCW; q++) mx = fmaxf(mx, sm.red[q]);
        float su = 1.f;
        if (mx > 0.f) {
            int ex;
            const float f = frexpf(mx, &ex);
            su = ldexpf(1.f, f == 0.5f ? ex - 1 : ex);
        }
        const float inv = 1.f / su;
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const int q = tid + r * NT;
            if (q < N3) {
                const int i = q % NX, j = (q / NX) % NX, k = q / N2;
                sm.U[(k * 16 + j) * 16 + i] = T::from_f(uv[r] * inv);
            }
        }
        __syncthreads();

        // ---------------------------------------------------------- ut, per line j
        for (int j = wp; j < NX; j += TCW) {
            uint32_t a[4];
            ldsm4t(smem_addr(sm.U + (t_row(L) * 16 + j) * 16 + t_col(L)), a);  // A[i][l] = U[l][j][i]
            float acc[2][4] = {};
            T::mma(acc[0], a, BD[0], BD[1]);
            T::mma(acc[1], a, BD[2], BD[3]);
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int i = g + 8 * (r >> 1), k = 8 * h + 2 * c + (r & 1);
                    if (i < NX && k < NX) sm.X[(k * NX + j) * NX + i] = acc[h][r];
                }
        }
        __syncthreads();

        // ---------------------------------------------------------- planes k
        const S* Ge = Glp + e * (int64_t)N3 * 6;
        S* pr = sm.PR[wp];
        S* ps = sm.PS[wp];
        for (int k = wp; k < NX; k += TCW) {
            const S* Uk = sm.U + k * 256;
            uint32_t bu[4], au[4];
            ldsm4(smem_addr(Uk + t_row(L) * 16 + t_col(L)), bu);   // B[l][j] = U[k][j][l]
            ldsm4t(smem_addr(Uk + t_row(L) * 16 + t_col(L)), au);  // A[i][l] = U[k][l][i]
            float ur[2][4] = {}, us[2][4] = {};
            T::mma(ur[0], AD, bu[0], bu[1]);
            T::mma(ur[1], AD, bu[2], bu[3]);
            T::mma(us[0], au, BD[0], BD[1]);
            T::mma(us[1], au, BD[2], BD[3]);
            // geometric product at the fragment's points (i, j) of plane k
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int i = g + 8 * (r >> 1), j = 8 * h + 2 * c + (r & 1);
                    float wr = 0.f, ws = 0.f, wt = 0.f;
                    if (i < NX && j < NX) {
                        const int p = (k * NX + j) * NX + i;
                        const float at = sm.X[p];
                        const unsigned* g4 = reinterpret_cast<const unsigned*>(Ge + 6 * p);
                        float gg[6];
#pragma unroll
                        for (int q = 0; q < 3; q++) {
                            const unsigned t = __ldg(g4 + q);
                            gg[2 * q] = T::bits_to_f(static_cast<unsigned short>(t & 0xffffu));
                            gg[2 * q + 1] = T::bits_to_f(static_cast<unsigned short>(t >> 16));
                        }
                        const float ar = ur[h][r], as = us[h][r];
                        wr = fmaf(gg[0], ar, fmaf(gg[1], as, gg[2] * at));
                        ws = fmaf(gg[1], ar, fmaf(gg[3], as, gg[4] * at));
                        wt = fmaf(gg[2], ar, fmaf(gg[4], as, gg[5] * at));
                    }
                    pr[j * 16 + i] = T::from_f(wr);
                    ps[j * 16 + i] = T::from_f(ws);
                    sm.WT[(k * 16 + j) * 16 + i] = T::from_f(wt);
                }
            __syncwarp();
            uint32_t bw[4], aw[4];
            ldsm4(smem_addr(pr + t_row(L) * 16 + t_col(L)), bw);   // B[l][j] = wr(l, j)
            ldsm4t(smem_addr(ps + t_row(L) * 16 + t_col(L)), aw);  // A[i][l] = ws(i, l)
            float acc[2][4] = {};
            T::mma(acc[0], ADT, bw[0], bw[1]);
            T::mma(acc[1], ADT, bw[2], bw[3]);
            T::mma(acc[0], aw, BDT[0], BDT[1]);
            T::mma(acc[1], aw, BDT[2], BDT[3]);
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int i = g + 8 * (r >> 1), j = 8 * h + 2 * c + (r & 1);
                    if (i < NX && j < NX) sm.X[(k * NX + j) * NX + i] = acc[h][r];
                }
            __syncwarp();  // the plane buffers are rewritten for the next plane
        }
        __syncthreads();

        // ---------------------------------------------------------- t-part and scale, per line j
        const float scale = su * gscale[e];
        for (int j = wp; j < NX; j += TCW) {
            uint32_t a[4];
            ldsm4t(smem_addr(sm.WT + (t_row(L) * 16 + j) * 16 + t_col(L)), a);  // A[i][l] = wt(i, j, l)
            float acc[2][4] = {};
            T::mma(acc[0], a, BDT[0], BDT[1]);
            T::mma(acc[1], a, BDT[2], BDT[3]);
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int i = g + 8 * (r >> 1), k = 8 * h + 2 * c + (r & 1);
                    if (i < NX && k < NX) {
                        const int p = (k * NX + j) * NX + i;
                        sm.X[p] = (sm.X[p] + acc[h][r]) * scale;
                    }
                }
        }
        __syncthreads();
        for (int q = tid; q < N3; q += NT) w[e * N3 + q] = sm.X[q];
    }
}

template <class S, int NX>
nek_status launch_tc_nx(int64_t nelt, const double* D, const void* Glp, const float* gscale, const float* u, float* w,
                        cudaStream_t s)
{
    constexpr size_t smem = sizeof(TcSmemLp<S, NX>);
    static std::atomic<uint64_t> configured{0};
    nek_status st0 = ensure_dyn_smem(k_ax_lowp_tc<S, NX>, smem, configured);
    if (st0 != NEK_OK) return st0;
    static std::atomic<int> per_sm_cache{0};  // resident CTAs per SM (the same on every GB300)
    int per_sm = per_sm_cache.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        nek_status so =
            check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_lowp_tc<S, NX>, 32 * TCW, smem));
        if (so != NEK_OK) return so;
        if (per_sm < 1) per_sm = 1;
        per_sm_cache.store(per_sm, std::memory_order_relaxed);
    }
    int dev = 0, sms = 0;
    nek_status st = check_cuda(cudaGetDevice(&dev));
    if (st == NEK_OK) st = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (st != NEK_OK) return st;
    const int64_t grid = std::min<int64_t>(nelt, (int64_t)per_sm * sms);
    k_ax_lowp_tc<S, NX><<<(unsigned)grid, 32 * TCW, smem, s>>>(nelt, D, static_cast<const S*>(Glp), gscale, u, w);
    return check_launch();
}

template <class S>
nek_status launch_tc_t(int64_t nelt, int nx, const double* D, const void* Glp, const float* gscale, const float* u,
                       float* w, cudaStream_t s)
{
    switch (nx) {
        case 2: return launch_tc_nx<S, 2>(nelt, D, Glp, gscale, u, w, s);
        case 3: return launch_tc_nx<S, 3>(nelt, D, Glp, gscale, u, w, s);
        case 4: return launch_tc_nx<S, 4>(nelt, D, Glp, gscale, u, w, s);
        case 5: return launch_tc_nx<S, 5>(nelt, D, Glp, gscale, u, w, s);
        case 6: return launch_tc_nx<S, 6>(nelt, D, Glp, gscale, u, w, s);
        case 7: return launch_tc_nx<S, 7>(nelt, D, Glp, gscale, u, w, s);
        case 8: return launch_tc_nx<S, 8>(nelt, D, Glp, gscale, u, w, s);
        case 9: return launch_tc_nx<S, 9>(nelt, D, Glp, gscale, u, w, s);
        case 10: return launch_tc_nx<S, 10>(nelt, D, Glp, gscale, u, w, s);
        case 11: return launch_tc_nx<S, 11>(nelt, D, Glp, gscale, u, w, s);
        case 12: return launch_tc_nx<S, 12>(nelt, D, Glp, gscale, u, w, s);
        case 13: return launch_tc_nx<S, 13>(nelt, D, Glp, gscale, u, w, s);
        case 14: return launch_tc_nx<S, 14>(nelt, D, Glp, gscale, u, w, s);
        case 15: return launch_tc_nx<S, 15>(nelt, D, Glp, gscale, u, w, s);
        case 16: return launch_tc_nx<S, 16>(nelt, D, Glp, gscale, u, w, s);
        default: return NEK_ERR_UNSUPPORTED_NX;
    }
}

}  // namespace

nek_status launch_ax_lowp_tc(int prec, int64_t nelt, int nx, const double* D, const void* Glp, const float* gscale,
                             const float* u, float* w, cudaStream_t s)
{
    switch (prec) {
        case NEK_PREC_BF16: return launch_tc_t<__nv_bfloat16>(nelt, nx, D, Glp, gscale, u, w, s);
        case NEK_PREC_F16: return launch_tc_t<__half>(nelt, nx, D, Glp, gscale, u, w, s);
        default: return NEK_ERR_INVALID_ARG;
    }
}

}  // namespace nek
