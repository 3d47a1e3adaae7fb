// Many independent Poisson problems solved together by Jacobi-PCG.
//
// The problems (any element counts, nx in [2,16]) are laid out back to back in
// one E-vector space, sorted by nx, so that
//   - AX is one launch per nx group (elements are independent, the operator does
//     not care which problem an element belongs to); with the float-float
//     operator, CTAs whose elements all belong to finished problems return at
//     once, so the operator's work follows the problems still iterating;
//   - gather-scatter is one plan over all problems (each problem's global ids
//     are offset past the previous problem's);
//   - vector updates and inner products run over fixed-size chunks that never
//     straddle two problems: every chunk writes one partial per inner product,
//     and one warp per problem sums its chunks' partials in order, so every
//     problem gets its own deterministic scalars (alpha, beta, residual).
// A problem whose residual test passes (or that breaks down) is frozen by a
// per-problem flag: later update kernels skip its chunks, so its solution and
// iteration count are exactly those of a solve on its own.  One iteration for
// all problems is about ten kernels; `iters_per_graph` iterations are captured
// once into a CUDA graph and replayed, with a device counter of unfinished
// problems read back after each replay.  With iters_per_graph < 0 the whole
// solve is one graph launch: the iteration is the body of a conditional WHILE
// node, and a one-thread kernel at the end of the body sets the loop condition
// from the device's count of unfinished problems and an iteration counter, so
// the host neither waits nor launches anything until the solve has finished.
#include <algorithm>
#include <new>
#include <vector>

#include "nek_internal.h"
#include "nek_pcg.cuh"

namespace nek {

namespace {

constexpr int kChunk = 4096;   // points per reduction chunk
constexpr int kGChunk = 2048;  // gather-scatter groups per dssum chunk
constexpr int BT = 256;       // threads per chunk block

struct BScal {
    double rz, pw, alpha, beta, rr, bnorm, relres;
    int done, status, iters, it;
    int xpend;  // this iteration's x += alpha p is still to be applied (kb_p)
};

struct Group {
    int nx;
    int64_t elem0, nelt;  // element range of the group
    int64_t pt0;          // first point of the group
    double* D;            // device nx*nx (owned)
};

__device__ __forceinline__ bool bhalted(const BScal& s) { return s.done || s.status != NEK_OK; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NA>
__device__ __forceinline__ void chunk_reduce(double (&acc)[NA], double* parts, int nchunks, int cid)
{
    __shared__ double sh[NA][BT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < NA; a++) {
        const double v = warp_sum(acc[a]);
        if (lane == 0) sh[a][wid] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int a = 0; a < NA; a++) {
            double t = lane < BT / 32 ? sh[a][lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) parts[a * nchunks + cid] = t;
        }
    }
}

// x = 0; r = mask.f; p = z = minv r; partials <r,z>, <r,r>
__global__ void __launch_bounds__(BT) kb_init(const int64_t* __restrict__ ch_begin, const int32_t* __restrict__ ch_prob,
                                              int nchunks, const uint8_t* __restrict__ flags,
                                              const double* __restrict__ minv,
                                              const double* __restrict__ f, double* __restrict__ x,
                                              double* __restrict__ r, double* __restrict__ p,
                                              double* __restrict__ parts)
{
    const int64_t a = ch_begin[blockIdx.x], b = ch_begin[blockIdx.x + 1];
    double acc[2] = {0.0, 0.0};
    for (int64_t q = a + threadIdx.x; q < b; q += BT) {
        const uint8_t fq = flags[q];
        const double rq = (fq & pcg::kFree) ? f[q] : 0.0;
        const double zq = minv[q] * rq;
        x[q] = 0.0;
        r[q] = rq;
        p[q] = zq;
        if (fq & pcg::kOwner) {  // owner copies: the 1/multiplicity-weighted sums
            acc[0] += rq * zq;
            acc[1] += rq * rq;
        }
    }
    chunk_reduce<2>(acc, parts, nchunks, blockIdx.x);
}

// Chunk of block b: clist[b] when the host passes a compacted list of the
// chunks of unfinished problems, else b.
__device__ __forceinline__ int chunk_of(const int32_t* __restrict__ clist)
{
    return clist ? clist[blockIdx.x] : static_cast<int>(blockIdx.x);
}

// one warp per problem: sums its partials [c0, c1) in order
template <class I>
__device__ __forceinline__ double prob_sum(const double* __restrict__ parts, I c0, I c1)
{
    const int lane = threadIdx.x & 31;
    double v = 0.0;
#pragma unroll 4
    for (I q = c0 + lane; q < c1; q += 32) v += parts[q];
    return warp_sum(v);
}

__global__ void kb_init_finish(int nprob, const int* __restrict__ pch, const double* __restrict__ parts, int nchunks,
                               double tol, BScal* __restrict__ sc, int* __restrict__ active)
{
    const int pid = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (pid >= nprob) return;
    const double rz = prob_sum(parts, pch[pid], pch[pid + 1]);
    const double rr = prob_sum(parts + nchunks, pch[pid], pch[pid + 1]);
    if ((threadIdx.x & 31) == 0) {
        BScal s{};
        s.rz = rz;
        s.rr = rr;
        s.bnorm = sqrt(rr);
        s.relres = 1.0;
        s.status = NEK_OK;
        if (!(rr >= 0.0) || !isfinite(rr) || !isfinite(rz)) {
            s.status = NEK_ERR_BREAKDOWN;
        } else if (rr == 0.0) {
            s.done = 1;
            s.relres = 0.0;
        }
        sc[pid] = s;
        if (!bhalted(s)) atomicAdd(active, 1);
    }
}

// w <- mask.w ; partial <p,w>
__global__ void __launch_bounds__(BT) kb_pw(const int64_t* __restrict__ ch_begin, const int32_t* __restrict__ ch_prob,
                                            int nchunks, const uint8_t* __restrict__ flags,
                                            const double* __restrict__ p,
                                            double* __restrict__ w, double* __restrict__ parts,
                                            const BScal* __restrict__ sc, const int32_t* __restrict__ clist)
{
    const int c = chunk_of(clist);
    if (bhalted(sc[ch_prob[c]])) return;
    const int64_t a = ch_begin[c], b = ch_begin[c + 1];
    double acc[1] = {0.0};
    for (int64_t q = a + threadIdx.x; q < b; q += BT) {
        const uint8_t fq = flags[q];
        const double pq = p[q];  // loaded whatever the flags say, so it is not held back behind them
        const double wq = w[q];  // read-only: kb_update applies the mask
        if ((fq & (pcg::kFree | pcg::kOwner)) == (pcg::kFree | pcg::kOwner)) acc[0] += pq * wq;
    }
    chunk_reduce<1>(acc, parts, nchunks, c);
}

// pw from the chunk partials of kb_pw or, with edot, from the element energies
// of the float-float operator (problem p's elements are [pel[p], pel[p+1]))
__global__ void kb_alpha(int nprob, const int* __restrict__ pch, const double* __restrict__ parts,
                         BScal* __restrict__ sc, int* __restrict__ active, const int64_t* __restrict__ pel,
                         const double* __restrict__ edot)
{
    const int pid = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (pid >= nprob) return;
    if (bhalted(sc[pid])) {
        if ((threadIdx.x & 31) == 0) sc[pid].xpend = 0;
        return;
    }
    const double pw = edot ? prob_sum(edot, pel[pid], pel[pid + 1]) : prob_sum(parts, pch[pid], pch[pid + 1]);
    if ((threadIdx.x & 31) == 0) {
        BScal& s = sc[pid];
        s.it += 1;
        s.pw = pw;
        if (!(pw > 0.0) || !isfinite(pw)) {
            s.status = NEK_ERR_BREAKDOWN;
            s.iters = s.it;
            s.xpend = 0;
            atomicSub(active, 1);
        } else {
            s.alpha = s.rz / pw;
            s.xpend = 1;
        }
    }
}

// r -= alpha w; partials <r,r>, <r,z> with z = minv r (not stored); x and p
// are updated by kb_p, so p is read by one vector kernel only (the same split
// as the single-problem solve, with the same results)
__global__ void __launch_bounds__(BT) kb_update(const int64_t* __restrict__ ch_begin,
                                                const int32_t* __restrict__ ch_prob, int nchunks,
                                                const uint8_t* __restrict__ flags, const double* __restrict__ minv,
                                                const double* __restrict__ w, double* __restrict__ r,
                                                double* __restrict__ parts, const BScal* __restrict__ sc,
                                                const int32_t* __restrict__ clist)
{
    const int c = chunk_of(clist);
    const BScal& s = sc[ch_prob[c]];
    if (bhalted(s)) return;
    const double alpha = s.alpha;
    const int64_t a = ch_begin[c], b = ch_begin[c + 1];
    double acc[2] = {0.0, 0.0};
    // <r,r> in float pairs on the FP32 pipes, as the single-problem solve's r update does
    float s_hi = 0.f, s_lo = 0.f, s_c = 0.f;
    for (int64_t q = a + threadIdx.x; q < b; q += BT) {
        const uint8_t fq = flags[q];
        double wq = w[q];  // loaded whatever the flags say
        if (!(fq & pcg::kFree)) wq = 0.0;  // the mask
        const double rq = fma(-alpha, wq, r[q]);
        const double zq = minv[q] * rq;
        r[q] = rq;
        if (fq & pcg::kOwner) {
            pcg::sq_pair_add(rq, s_hi, s_lo, s_c);
            acc[1] += rq * zq;
        }
    }
    acc[0] = (widen(s_hi) + widen(s_lo)) + widen(s_c);
    chunk_reduce<2>(acc, parts, nchunks, c);
}

__global__ void kb_beta(int nprob, const int* __restrict__ pch, const double* __restrict__ parts, int nchunks,
                        BScal* __restrict__ sc, int* __restrict__ active)
{
    const int pid = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (pid >= nprob || bhalted(sc[pid])) return;
    const double rr = prob_sum(parts, pch[pid], pch[pid + 1]);
    const double rz = prob_sum(parts + nchunks, pch[pid], pch[pid + 1]);
    if ((threadIdx.x & 31) == 0) {
        BScal& s = sc[pid];
        s.rr = rr;
        s.relres = sqrt(rr) / s.bnorm;
        if (!isfinite(s.relres) || !isfinite(rz)) {
            s.status = NEK_ERR_BREAKDOWN;
            s.iters = s.it;
            atomicSub(active, 1);
        } else {
            s.beta = rz / s.rz;
            s.rz = rz;
        }
    }
}

// Loop control of the one-launch solve (end of the WHILE body): counts the
// iteration and keeps looping while problems are unfinished and the iteration
// budget lasts.
__global__ void kb_loop_ctl(cudaGraphConditionalHandle h, const int* __restrict__ active, int* __restrict__ iters,
                            int budget)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int n = *iters + 1;
        *iters = n;
        cudaGraphSetConditional(h, (*active > 0 && n < budget) ? 1u : 0u);
    }
}

// per-problem convergence test, kept separate from kb_beta so the tolerance is
// a kernel argument of the captured graph; pdone[p] = 1 once p has finished
// (the operator then skips p's elements)
__global__ void kb_test(int nprob, double tol, BScal* __restrict__ sc, int* __restrict__ active,
                        uint8_t* __restrict__ pdone)
{
    const int pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= nprob) return;
    BScal& s = sc[pid];
    if (!bhalted(s) && tol > 0.0 && s.relres <= tol && s.it > 0) {
        s.done = 1;
        s.iters = s.it;
        atomicSub(active, 1);
    }
    pdone[pid] = bhalted(s) ? 1 : 0;
}

// x += alpha p (old p) while the problem's x update is pending; p = minv r +
// beta p while it goes on
// dssum over the groups of the problems still going: block b sums the groups
// of chunk b unless its problem has finished (its vectors are frozen then).
__global__ void __launch_bounds__(BT) kb_dssum(const int64_t* __restrict__ gch_begin,
                                               const int32_t* __restrict__ gch_prob, const uint8_t* __restrict__ pdone,
                                               const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                                               double* __restrict__ v, const int32_t* __restrict__ glist)
{
    const int g = chunk_of(glist);
    if (pdone[gch_prob[g]]) return;
    pcg::dssum_groups<double>(gch_begin[g], gch_begin[g + 1], threadIdx.x, BT, off, mem, v);
}

__global__ void __launch_bounds__(BT) kb_p(const int64_t* __restrict__ ch_begin, const int32_t* __restrict__ ch_prob,
                                           const double* __restrict__ minv, const double* __restrict__ r,
                                           double* __restrict__ x, double* __restrict__ p,
                                           const BScal* __restrict__ sc, const int32_t* __restrict__ clist)
{
    const int c = chunk_of(clist);
    const BScal& s = sc[ch_prob[c]];
    const bool do_x = s.xpend != 0, do_p = !bhalted(s);
    const double alpha = s.alpha, beta = s.beta;
    const int64_t a = ch_begin[c], b = ch_begin[c + 1];
    if (do_x && do_p) {
        for (int64_t q = a + threadIdx.x; q < b; q += BT) {
            const double pq = p[q];
            x[q] = fma(alpha, pq, x[q]);
            p[q] = fma(beta, pq, minv[q] * r[q]);
        }
    } else if (do_x) {
        for (int64_t q = a + threadIdx.x; q < b; q += BT) x[q] = fma(alpha, p[q], x[q]);
    }
}

__global__ void k_bdiag_local(int64_t nelt, int nx, const double* __restrict__ D, const double* __restrict__ G,
                              double* __restrict__ d)
{
    const int64_t n3 = (int64_t)nx * nx * nx;
    for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < nelt * n3;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = gid / n3;
        const int p = static_cast<int>(gid - e * n3);
        const int i = p % nx, j = (p / nx) % nx, k = p / (nx * nx);
        const double* Ge = G + e * n3 * 6;
        double s = 0.0;
        for (int l = 0; l < nx; l++) {
            const double a = D[l * nx + i], b = D[l * nx + j], cc = D[l * nx + k];
            s += Ge[6 * (l + nx * (j + nx * k)) + 0] * a * a;
            s += Ge[6 * (i + nx * (l + nx * k)) + 3] * b * b;
            s += Ge[6 * (i + nx * (j + nx * l)) + 5] * cc * cc;
        }
        const double* g = Ge + 6 * p;
        const double di = D[i * nx + i], dj = D[j * nx + j], dk = D[k * nx + k];
        s += 2.0 * (g[1] * di * dj + g[2] * di * dk + g[4] * dj * dk);
        d[gid] = s;
    }
}

__global__ void k_binvert(int64_t n, const uint8_t* __restrict__ mask, double* __restrict__ d)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        d[p] = mask[p] ? 1.0 / d[p] : 0.0;
}

}  // namespace

}  // namespace nek

struct nek_batch {
    int nprob;
    int64_t npts, nelt_total;
    nek_gs* gs;
    std::vector<nek::Group> groups;
    std::vector<int64_t> prob_pt0;  // first point of each problem, nprob+1
    std::vector<int64_t> prob_el0;  // first element of each problem, nprob+1
    std::vector<int> prob_group;    // group (nx run) of each problem
    int nchunks;
    int64_t* d_ch_begin;  // nchunks+1
    int32_t* d_ch_prob;   // nchunks
    int* d_pch;           // nprob+1: chunk range of each problem
    int32_t* d_elem_prob; // nelt_total: problem of each element
    int64_t* d_pel;       // nprob+1: element range of each problem
    int ngchunks;         // chunks of the gather-scatter groups, each within one problem
    int64_t* d_gch_begin; // ngchunks+1: first group of each chunk
    int32_t* d_gch_prob;  // ngchunks: problem of each chunk
    std::vector<int32_t> h_ch_prob, h_gch_prob;  // the same two maps on the host
};

using namespace nek;

namespace {

inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct BLayout {
    double *r, *p, *w, *minv, *parts, *edot;
    BScal* sc;
    int* active;
    uint8_t* pdone;  // nprob: 1 once a problem has finished (converged or broken down)
    uint8_t* flags;  // npts: owner / free byte per point (inner-product weights and the mask)
    int32_t* clist;  // nchunks: chunks of the unfinished problems, for the vector kernels
    int32_t* glist;  // ngchunks: the same for the gather-scatter chunks
    size_t bytes;
};

BLayout b_layout(char* base, const nek_batch* b, bool need_minv)
{
    BLayout L{};
    size_t off = 0;
    auto take = [&](size_t n) {
        char* q = base ? base + off : nullptr;
        off += al256(n);
        return q;
    };
    const size_t v = sizeof(double) * std::max<int64_t>(b->npts, 1);
    L.r = reinterpret_cast<double*>(take(v));
    L.p = reinterpret_cast<double*>(take(v));
    L.w = reinterpret_cast<double*>(take(v));
    L.minv = need_minv ? reinterpret_cast<double*>(take(v)) : nullptr;
    L.parts = reinterpret_cast<double*>(take(sizeof(double) * 2 * (size_t)b->nchunks));
    L.edot = reinterpret_cast<double*>(take(sizeof(double) * std::max<int64_t>(b->nelt_total, 1)));
    L.sc = reinterpret_cast<BScal*>(take(sizeof(BScal) * (size_t)b->nprob));
    L.active = reinterpret_cast<int*>(take(sizeof(int) * 4));  // [0] unfinished problems, [1] loop iterations
    L.pdone = reinterpret_cast<uint8_t*>(take(static_cast<size_t>(b->nprob)));
    L.flags = reinterpret_cast<uint8_t*>(take(static_cast<size_t>(b->npts)));
    L.clist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * std::max(b->nchunks, 1)));
    L.glist = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * std::max(b->ngchunks, 1)));
    L.bytes = off;
    return L;
}

}  // namespace

extern "C" {

nek_status nek_batch_create(int nprob, const int64_t* nelt, const int* nx, const int64_t* glo_num_host,
                            nek_batch** out)
{
    if (!out) return NEK_ERR_INVALID_ARG;
    *out = nullptr;
    if (nprob <= 0 || !nelt || !nx || !glo_num_host) return NEK_ERR_INVALID_ARG;
    int64_t npts = 0, nel = 0;
    for (int q = 0; q < nprob; q++) {
        if (nx[q] < kMinNx || nx[q] > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
        if (nelt[q] <= 0) return NEK_ERR_INVALID_ARG;
        if (q > 0 && nx[q] < nx[q - 1]) return NEK_ERR_INVALID_ARG;  // problems must be sorted by nx
        npts += nelt[q] * (int64_t)nx[q] * nx[q] * nx[q];
        nel += nelt[q];
    }
    if (npts >= (int64_t(1) << 31)) return NEK_ERR_TOO_LARGE;
    nek_batch* b = new (std::nothrow) nek_batch();
    if (!b) return NEK_ERR_NOMEM;
    b->nprob = nprob;
    b->npts = npts;
    b->nelt_total = nel;
    b->gs = nullptr;
    b->d_ch_begin = nullptr;
    b->d_ch_prob = nullptr;
    b->d_pch = nullptr;
    b->d_elem_prob = nullptr;
    b->d_pel = nullptr;
    b->ngchunks = 0;
    b->d_gch_begin = nullptr;
    b->d_gch_prob = nullptr;
    nek_status st = NEK_OK;
    try {
        // global ids of all problems in one space: problem q's ids are offset by
        // the sum of the previous problems' (max id + 1)
        std::vector<int64_t> glo(static_cast<size_t>(npts));
        std::vector<int64_t> ch_begin;
        std::vector<int32_t> ch_prob;
        std::vector<int> pch(1, 0);
        std::vector<int32_t> elem_prob(static_cast<size_t>(nel));
        std::vector<int64_t> pel(1, 0);
        std::vector<int64_t> gch_begin;  // group chunks: groups of problem q follow those of q - 1
        std::vector<int32_t> gch_prob;
        std::vector<int32_t> mult;       // multiplicity of each global id of one problem
        int64_t gtot = 0;
        b->prob_pt0.assign(1, 0);
        b->prob_el0.assign(1, 0);
        int64_t pt = 0, goff = 0, el = 0;
        for (int q = 0; q < nprob; q++) {
            const int64_t n = nelt[q] * (int64_t)nx[q] * nx[q] * nx[q];
            int64_t gmax = -1;
            for (int64_t k = 0; k < n; k++) {
                const int64_t g = glo_num_host[pt + k];
                if (g < 0) throw 1;
                glo[pt + k] = g + goff;
                gmax = std::max(gmax, g);
            }
            // the plan orders groups by global id, and problem q's ids follow q - 1's: its groups are the
            // next (number of its ids with two or more copies)
            mult.assign(static_cast<size_t>(gmax + 1), 0);
            for (int64_t k = 0; k < n; k++) mult[glo_num_host[pt + k]]++;
            int64_t ngq = 0;
            for (int32_t c : mult) ngq += c >= 2;
            for (int64_t a = gtot; a < gtot + ngq; a += kGChunk) {
                gch_begin.push_back(a);
                gch_prob.push_back(q);
            }
            gtot += ngq;
            for (int64_t a = pt; a < pt + n; a += kChunk) {
                ch_begin.push_back(a);
                ch_prob.push_back(q);
            }
            pch.push_back(static_cast<int>(ch_begin.size()));
            for (int64_t k = 0; k < nelt[q]; k++) elem_prob[el + k] = q;
            pel.push_back(el + nelt[q]);
            if (b->groups.empty() || b->groups.back().nx != nx[q]) b->groups.push_back(Group{nx[q], el, 0, pt, nullptr});
            b->prob_group.push_back(static_cast<int>(b->groups.size()) - 1);
            b->groups.back().nelt += nelt[q];
            goff += gmax + 1;
            pt += n;
            el += nelt[q];
            b->prob_pt0.push_back(pt);
            b->prob_el0.push_back(el);
        }
        ch_begin.push_back(npts);
        b->nchunks = static_cast<int>(ch_prob.size());
        if ((st = gs_create_flat(npts, glo.data(), &b->gs)) != NEK_OK) throw 3;
        if (b->gs->ngroups != gtot) throw 3;  // the plan's grouping must be the one counted above
        gch_begin.push_back(gtot);
        b->ngchunks = static_cast<int>(gch_prob.size());
        b->h_ch_prob = ch_prob;
        b->h_gch_prob = gch_prob;
        if ((st = check_cuda(cudaMalloc(&b->d_gch_begin, sizeof(int64_t) * gch_begin.size()))) != NEK_OK) throw 3;
        if ((st = check_cuda(cudaMalloc(&b->d_gch_prob, sizeof(int32_t) * std::max<size_t>(gch_prob.size(), 1)))) !=
            NEK_OK)
            throw 3;
        if ((st = check_cuda(cudaMemcpy(b->d_gch_begin, gch_begin.data(), sizeof(int64_t) * gch_begin.size(),
                                        cudaMemcpyHostToDevice))) != NEK_OK)
            throw 3;
        if (!gch_prob.empty() &&
            (st = check_cuda(cudaMemcpy(b->d_gch_prob, gch_prob.data(), sizeof(int32_t) * gch_prob.size(),
                                        cudaMemcpyHostToDevice))) != NEK_OK)
            throw 3;
        if ((st = check_cuda(cudaMalloc(&b->d_ch_begin, sizeof(int64_t) * ch_begin.size()))) != NEK_OK) throw 3;
        if ((st = check_cuda(cudaMalloc(&b->d_ch_prob, sizeof(int32_t) * ch_prob.size()))) != NEK_OK) throw 3;
        if ((st = check_cuda(cudaMalloc(&b->d_pch, sizeof(int) * pch.size()))) != NEK_OK) throw 3;
        if ((st = check_cuda(cudaMalloc(&b->d_elem_prob, sizeof(int32_t) * elem_prob.size()))) != NEK_OK) throw 3;
        if ((st = check_cuda(cudaMalloc(&b->d_pel, sizeof(int64_t) * pel.size()))) != NEK_OK) throw 3;
        if ((st = check_cuda(cudaMemcpy(b->d_pel, pel.data(), sizeof(int64_t) * pel.size(), cudaMemcpyHostToDevice))) !=
            NEK_OK)
            throw 3;
        if ((st = check_cuda(cudaMemcpy(b->d_elem_prob, elem_prob.data(), sizeof(int32_t) * elem_prob.size(),
                                        cudaMemcpyHostToDevice))) != NEK_OK)
            throw 3;
        cudaMemcpy(b->d_ch_begin, ch_begin.data(), sizeof(int64_t) * ch_begin.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(b->d_ch_prob, ch_prob.data(), sizeof(int32_t) * ch_prob.size(), cudaMemcpyHostToDevice);
        if ((st = check_cuda(cudaMemcpy(b->d_pch, pch.data(), sizeof(int) * pch.size(), cudaMemcpyHostToDevice))) !=
            NEK_OK)
            throw 3;
        for (auto& g : b->groups) {
            double Dh[kMaxNx * kMaxNx];
            gll_host(g.nx, nullptr, nullptr, Dh);
            if ((st = check_cuda(cudaMalloc(&g.D, sizeof(double) * g.nx * g.nx))) != NEK_OK) throw 3;
            if ((st = check_cuda(cudaMemcpy(g.D, Dh, sizeof(double) * g.nx * g.nx, cudaMemcpyHostToDevice))) != NEK_OK)
                throw 3;
        }
    } catch (const std::bad_alloc&) {
        st = NEK_ERR_NOMEM;
    } catch (int code) {
        if (code == 1) st = NEK_ERR_INVALID_ARG;
        if (st == NEK_OK) st = NEK_ERR_CUDA;
    }
    if (st != NEK_OK) {
        nek_batch_destroy(b);
        return st;
    }
    *out = b;
    return NEK_OK;
}

nek_status nek_batch_destroy(nek_batch* b)
{
    if (!b) return NEK_OK;
    nek_gs_destroy(b->gs);
    cudaFree(b->d_ch_begin);
    cudaFree(b->d_ch_prob);
    cudaFree(b->d_pch);
    cudaFree(b->d_elem_prob);
    cudaFree(b->d_pel);
    cudaFree(b->d_gch_begin);
    cudaFree(b->d_gch_prob);
    for (auto& g : b->groups) cudaFree(g.D);
    delete b;
    return NEK_OK;
}

nek_status nek_batch_info(const nek_batch* b, int64_t* npts, int* ngroups, int* nchunks)
{
    if (!b) return NEK_ERR_INVALID_ARG;
    if (npts) *npts = b->npts;
    if (ngroups) *ngroups = static_cast<int>(b->groups.size());
    if (nchunks) *nchunks = b->nchunks;
    return NEK_OK;
}

const nek_gs* nek_batch_gs(const nek_batch* b) { return b ? b->gs : nullptr; }

size_t nek_batch_workspace_bytes(const nek_batch* b, int need_minv)
{
    if (!b) return 0;
    return b_layout(nullptr, b, need_minv != 0).bytes;
}

nek_status nek_batch_jacobi_minv(const nek_batch* b, const double* G, const uint8_t* mask, double* minv,
                                 void* stream)
{
    if (!b || !G || !mask || !minv || !is_aligned(G, 16) || !is_aligned(minv, 8)) return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (const auto& g : b->groups) {
        const int64_t n = g.nelt * (int64_t)g.nx * g.nx * g.nx;
        const int64_t nb = (n + 255) / 256;
        k_bdiag_local<<<static_cast<int>(std::min<int64_t>(nb, 152 * 16)), 256, 0, s>>>(
            g.nelt, g.nx, g.D, G + g.pt0 * 6, minv + g.pt0);
    }
    nek_status st = check_launch();
    if (st != NEK_OK) return st;
    if ((st = pcg::dssum<double>(b->gs, minv, s)) != NEK_OK) return st;
    k_binvert<<<pcg::stream_blocks(b->npts), 256, 0, s>>>(b->npts, mask, minv);
    return check_launch();
}

nek_status nek_batch_cg_solve(const nek_batch* b, const double* G, const float* Gff, const uint8_t* mask,
                              const double* minv, const double* f, double* x, double tol_rel, int max_iter,
                              int iters_per_graph, void* workspace, int* iters_host, double* relres_host,
                              int* status_host, nek_batch_stats* stats, void* stream)
{
    if (stats) *stats = nek_batch_stats{};
    if (!b || !G || !mask || !f || !x || max_iter < 0 || !(tol_rel >= 0.0)) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(G, 16) || !is_aligned(x, 16) || !is_aligned(f, 8) || (Gff && !is_aligned(Gff, 16)) ||
        (minv && !is_aligned(minv, 8)) || (workspace && !is_aligned(workspace, 256)))
        return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = nek_batch_workspace_bytes(b, minv == nullptr);
    void* ws = workspace;
    if (!ws && check_cuda(cudaMallocAsync(&ws, bytes, s)) != NEK_OK) return NEK_ERR_NOMEM;
    BLayout L = b_layout(static_cast<char*>(ws), b, minv == nullptr);
    nek_status st = NEK_OK;
    const double* mv = minv;
    const int nc = b->nchunks, np = b->nprob;
    const int wblocks = (np + 7) / 8;  // 8 warps (problems) per 256-thread block
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int it_done = 0, launches = 0, graph_launches = 0;
    int active = 0;
    const int per_graph = iters_per_graph > 0 ? iters_per_graph : 0;
    bool device_loop = false;  // the one-launch solve ran (or there was nothing left to run)
    bool lists_changed = false;

    // Per group, the elements before ax_first[g] belong to finished problems only,
    // and the operator is launched from there on.  With the problems of a group
    // ordered by size (the larger need more iterations), the launches shrink as
    // the small ones finish; ax_first is advanced at graph boundaries.
    std::vector<int64_t> ax_first(b->groups.size(), 0);
    // The vector kernels and dssum run over compacted lists of the chunks of the
    // problems still going (L.clist / L.glist), rebuilt by the host at graph
    // boundaries; until the first rebuild (and in the one-launch solve) every
    // chunk is launched and the finished problems' blocks return at once.
    bool use_lists = false;
    int n_act = nc, n_gact = b->ngchunks;
    std::vector<int32_t> h_clist, h_glist;
    int iter_launches = 0;  // launches enqueued by the last one_iteration
    auto one_iteration = [&](cudaStream_t ss) -> nek_status {
        iter_launches = 0;
        for (size_t gi = 0; gi < b->groups.size(); gi++) {
            // the group's elements from the first one of a problem still going (see ax_first)
            const auto& g = b->groups[gi];
            const int64_t f0 = ax_first[gi];
            if (f0 >= g.nelt) continue;
            const int64_t pt = g.pt0 + f0 * (int64_t)g.nx * g.nx * g.nx;
            nek_status sa = Gff ? launch_ax_ff(g.nelt - f0, g.nx, g.D, Gff + pt * 12, L.p + pt, L.w + pt, ss, nullptr,
                                               b->d_elem_prob + g.elem0 + f0, L.pdone, L.edot + g.elem0 + f0)
                                : launch_ax_fp64(g.nelt - f0, g.nx, g.D, G + pt * 6, L.p + pt, L.w + pt, ss);
            if (sa != NEK_OK) return sa;
            iter_launches++;
        }
        const int32_t* cl = use_lists ? L.clist : nullptr;
        const int32_t* gl = use_lists ? L.glist : nullptr;
        if (n_gact > 0)
            kb_dssum<<<n_gact, BT, 0, ss>>>(b->d_gch_begin, b->d_gch_prob, L.pdone, b->gs->d_offsets,
                                            b->gs->d_members, L.w, gl);
        // the float-float operator writes element energies, which give <p,w> (no kb_pw pass)
        if (!Gff) kb_pw<<<n_act, BT, 0, ss>>>(b->d_ch_begin, b->d_ch_prob, nc, L.flags, L.p, L.w, L.parts, L.sc, cl);
        kb_alpha<<<wblocks, 256, 0, ss>>>(np, b->d_pch, L.parts, L.sc, L.active, b->d_pel, Gff ? L.edot : nullptr);
        kb_update<<<n_act, BT, 0, ss>>>(b->d_ch_begin, b->d_ch_prob, nc, L.flags, mv, L.w, L.r, L.parts, L.sc, cl);
        kb_beta<<<wblocks, 256, 0, ss>>>(np, b->d_pch, L.parts, nc, L.sc, L.active);
        kb_test<<<(np + 255) / 256, 256, 0, ss>>>(np, tol_rel, L.sc, L.active, L.pdone);
        kb_p<<<n_act, BT, 0, ss>>>(b->d_ch_begin, b->d_ch_prob, mv, L.r, x, L.p, L.sc, cl);
        iter_launches += (n_gact > 0 ? 1 : 0) + (Gff ? 0 : 1) + 5;
        return check_launch();
    };
    int graph_iter_launches = 0;  // launches in one replay of the captured graph
    // (Re)captures per_graph iterations with the current ax_first on a private
    // stream (the caller's may be the legacy default stream, which cannot be
    // captured); nothing runs during capture.  The graph is launched on the
    // caller's stream.
    auto capture = [&]() -> nek_status {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        cudaStream_t cs = nullptr;
        nek_status r = check_cuda(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        if (r != NEK_OK) return r;
        r = check_cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        graph_iter_launches = 0;
        if (r == NEK_OK) {
            for (int k = 0; k < per_graph && r == NEK_OK; k++) {
                r = one_iteration(cs);
                graph_iter_launches += iter_launches;
            }
            cudaError_t ce = cudaStreamEndCapture(cs, &graph);
            if (r == NEK_OK) r = check_cuda(ce);
        }
        cudaStreamDestroy(cs);
        if (r == NEK_OK) r = check_cuda(cudaGraphInstantiate(&gexec, graph, 0));
        return r;
    };
    // Advances ax_first past the finished problems at the start of each group
    // (pdone on the host); true when a group's launch shrank by an eighth or
    // more since the last capture, which is then worth a new graph.
    std::vector<uint8_t> hdone(static_cast<size_t>(np), 0);
    auto advance_windows = [&]() -> bool {
        bool shrunk = false;
        for (size_t gi = 0; gi < b->groups.size(); gi++) {
            const auto& g = b->groups[gi];
            int64_t f0 = g.nelt;
            for (int q = 0; q < np; q++) {
                if (b->prob_group[q] != static_cast<int>(gi) || hdone[q]) continue;
                f0 = b->prob_el0[q] - g.elem0;  // the group's first problem still going
                break;
            }
            if (f0 - ax_first[gi] >= std::max<int64_t>(1, g.nelt / 8)) {
                ax_first[gi] = f0;
                shrunk = true;
            }
        }
        return shrunk;
    };
    // Rebuilds the chunk lists from the finished problems (hdone).  Only when
    // either list is an eighth or more shorter than the one in use are both
    // uploaded, and the graph is then recaptured with the new grid sizes, so a
    // graph never runs with a list other than the one it was captured for.
    auto shrink_lists = [&]() -> nek_status {
        h_clist.clear();
        h_glist.clear();
        for (int c = 0; c < nc; c++)
            if (!hdone[b->h_ch_prob[c]]) h_clist.push_back(c);
        for (int g = 0; g < b->ngchunks; g++)
            if (!hdone[b->h_gch_prob[g]]) h_glist.push_back(g);
        const int na = static_cast<int>(h_clist.size()), ng = static_cast<int>(h_glist.size());
        if (na > n_act - std::max(1, n_act / 8) && ng > n_gact - std::max(1, n_gact / 8)) return NEK_OK;
        if (na > 0) {
            nek_status r = check_cuda(cudaMemcpyAsync(L.clist, h_clist.data(), sizeof(int32_t) * na,
                                                      cudaMemcpyHostToDevice, s));
            if (r != NEK_OK) return r;
        }
        if (ng > 0) {
            nek_status r = check_cuda(cudaMemcpyAsync(L.glist, h_glist.data(), sizeof(int32_t) * ng,
                                                      cudaMemcpyHostToDevice, s));
            if (r != NEK_OK) return r;
        }
        n_act = na;
        n_gact = ng;
        use_lists = true;
        lists_changed = true;
        return NEK_OK;
    };

    if (!minv) {
        if ((st = nek_batch_jacobi_minv(b, G, mask, L.minv, stream)) != NEK_OK) goto done;
        mv = L.minv;
        launches += static_cast<int>(b->groups.size()) + 2;
    }
    cudaMemsetAsync(L.active, 0, sizeof(int), s);
    if ((st = pcg::build_flags(b->gs, b->npts, mask, L.flags, s)) != NEK_OK) goto done;
    launches += b->gs->ngroups > 0 ? 2 : 1;
    kb_init<<<nc, BT, 0, s>>>(b->d_ch_begin, b->d_ch_prob, nc, L.flags, mv, f, x, L.r, L.p, L.parts);
    kb_init_finish<<<wblocks, 256, 0, s>>>(np, b->d_pch, L.parts, nc, tol_rel, L.sc, L.active);
    kb_test<<<(np + 255) / 256, 256, 0, s>>>(np, tol_rel, L.sc, L.active, L.pdone);  // initial pdone
    launches += 3;
    if ((st = check_launch()) != NEK_OK) goto done;
    // first iteration eagerly (configures every kernel before any capture)
    if (max_iter > 0) {
        if ((st = one_iteration(s)) != NEK_OK) goto done;
        it_done = 1;
        launches += iter_launches;
    }
    if (iters_per_graph < 0 && it_done < max_iter) {
        device_loop = true;
        // the remaining iterations in one graph launch (device-side WHILE loop)
        if ((st = check_cuda(cudaMemcpyAsync(&active, L.active, sizeof(int), cudaMemcpyDeviceToHost, s))) != NEK_OK)
            goto done;
        if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
        if (active > 0) {
            int body_launches = 0;
            if ((st = check_cuda(cudaMemsetAsync(L.active + 1, 0, sizeof(int), s))) != NEK_OK) goto done;
            if ((st = check_cuda(cudaGraphCreate(&graph, 0))) != NEK_OK) goto done;
            cudaGraphConditionalHandle cond;
            if ((st = check_cuda(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault))) !=
                NEK_OK)
                goto done;
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = cond;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode;
            if ((st = check_cuda(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp))) != NEK_OK) goto done;
            {
                cudaStream_t cs = nullptr;
                st = check_cuda(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
                if (st == NEK_OK)
                    st = check_cuda(cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr,
                                                                  0, cudaStreamCaptureModeThreadLocal));
                if (st == NEK_OK) {
                    st = one_iteration(cs);
                    body_launches = iter_launches + 1;
                    if (st == NEK_OK) {
                        kb_loop_ctl<<<1, 32, 0, cs>>>(cond, L.active, L.active + 1, max_iter - it_done);
                        st = check_launch();
                    }
                    cudaGraph_t body = nullptr;
                    cudaError_t ce = cudaStreamEndCapture(cs, &body);
                    if (st == NEK_OK) st = check_cuda(ce);
                }
                if (cs) cudaStreamDestroy(cs);
            }
            if (st != NEK_OK) goto done;
            if ((st = check_cuda(cudaGraphInstantiate(&gexec, graph, 0))) != NEK_OK) goto done;
            if ((st = check_cuda(cudaGraphLaunch(gexec, s))) != NEK_OK) goto done;
            int loops = 0;
            if ((st = check_cuda(cudaMemcpyAsync(&loops, L.active + 1, sizeof(int), cudaMemcpyDeviceToHost, s))) !=
                NEK_OK)
                goto done;
            if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
            it_done += loops;
            launches += loops * body_launches;
            graph_launches = 1;
        }
    }
    if (!device_loop && per_graph > 0 && it_done < max_iter)
        if ((st = capture()) != NEK_OK) goto done;
    while (!device_loop && it_done < max_iter) {
        if ((st = check_cuda(cudaMemcpyAsync(&active, L.active, sizeof(int), cudaMemcpyDeviceToHost, s))) != NEK_OK)
            goto done;
        if ((st = check_cuda(cudaMemcpyAsync(hdone.data(), L.pdone, static_cast<size_t>(np),
                                             cudaMemcpyDeviceToHost, s))) != NEK_OK)
            goto done;
        if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
        if (active <= 0) break;
        lists_changed = false;
        if ((st = shrink_lists()) != NEK_OK) goto done;
        if ((advance_windows() || lists_changed) && gexec)
            if ((st = capture()) != NEK_OK) goto done;
        if (gexec && it_done + per_graph <= max_iter) {
            if ((st = check_cuda(cudaGraphLaunch(gexec, s))) != NEK_OK) goto done;
            it_done += per_graph;
            launches += graph_iter_launches;
            graph_launches++;
        } else {
            if ((st = one_iteration(s)) != NEK_OK) goto done;
            it_done += 1;
            launches += iter_launches;
        }
    }
    {
        std::vector<BScal> h(static_cast<size_t>(np));
        if ((st = check_cuda(cudaMemcpyAsync(h.data(), L.sc, sizeof(BScal) * np, cudaMemcpyDeviceToHost, s))) !=
            NEK_OK)
            goto done;
        if ((st = check_cuda(cudaStreamSynchronize(s))) != NEK_OK) goto done;
        int nconv = 0, nbreak = 0;
        for (int q = 0; q < np; q++) {
            const bool stopped = h[q].done || h[q].status != NEK_OK;
            if (iters_host) iters_host[q] = stopped ? h[q].iters : h[q].it;
            if (relres_host) relres_host[q] = h[q].relres;
            int sq = h[q].status != NEK_OK ? h[q].status : (h[q].done || tol_rel == 0.0) ? NEK_OK : NEK_ERR_NOT_CONVERGED;
            if (status_host) status_host[q] = sq;
            nconv += h[q].done;
            nbreak += h[q].status != NEK_OK;
        }
        if (nbreak) st = NEK_ERR_BREAKDOWN;
        else if (tol_rel > 0.0 && nconv < np) st = NEK_ERR_NOT_CONVERGED;
        if (stats) {
            stats->iterations_run = it_done;
            stats->converged = nconv;
            stats->kernel_launches = launches;
            stats->graph_launches = graph_launches;
        }
    }
done:
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (!workspace) {
        cudaFreeAsync(ws, s);
        nek_status st2 = check_cuda(cudaStreamSynchronize(s));
        if (st == NEK_OK) st = st2;
    }
    return st;
}

}  // extern "C"
