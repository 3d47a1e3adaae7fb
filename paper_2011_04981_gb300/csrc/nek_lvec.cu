// Unique-node ("L-vector") form of the operator and of the Jacobi-PCG solve.
//
// The E-vector solve of Section II-B stores every element's nx^3 nodes, so a
// node shared by m elements is stored m times and every vector operation of CG
// touches all copies; the nearest-neighbour exchange (dssum) then makes the
// copies agree.  Here every global node is stored once, in ascending global id.
// With Q the local-to-unique map (u_local[p] = u[l2g[p]]), the element operator
// becomes w = Q^T AX Q u: the AX kernel gathers its input through l2g, writes
// the element results to an E-vector scratch, and one kernel sums each node's
// copies (ascending local index, the order of dssum).  CG then runs on vectors
// of the unique length with plain (unweighted) inner products, so its iterates
// equal those of the E-vector solve up to rounding: x_E = Q x_L.
//
// Index arrays are int32: npts < 2^31.
#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "nek_internal.h"
#include "nek_pcg.cuh"

struct nek_lvec {
    int64_t npts;      // local (E-vector) points
    int64_t nl;        // unique nodes
    int32_t* d_l2g;    // [npts] unique index of each local point
    int32_t* d_off;    // [nl + 1] copies of unique node g: d_mem[d_off[g] .. d_off[g+1])
    int32_t* d_mem;    // [npts] local points grouped by unique node, ascending within a node
    uint8_t* d_mask;   // [nl] 1 = free node, 0 = Dirichlet node
};

namespace nek {

namespace {

using pcg::stream_blocks;

__global__ void k_lv_scatter(int64_t npts, const int32_t* __restrict__ l2g, const double* __restrict__ uL,
                             double* __restrict__ uE)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x)
        uE[p] = __ldg(uL + __ldg(l2g + p));
}

__global__ void k_lv_restrict(int64_t nl, const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                              const double* __restrict__ uE, double* __restrict__ uL)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nl; g += (int64_t)gridDim.x * blockDim.x)
        uL[g] = uE[mem[off[g]]];
}

// wL[g] = sum of wE over the copies of g, left to right in ascending local index.
__global__ void k_lv_assemble(int64_t nl, const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                              const double* __restrict__ wE, double* __restrict__ wL)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nl; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = __ldg(off + g), b = __ldg(off + g + 1);
        double s = __ldg(wE + __ldg(mem + a));
        for (int32_t m = a + 1; m < b; m++) s += __ldg(wE + __ldg(mem + m));
        wL[g] = s;
    }
}

// minvL[g] = 1 / (sum of the element diagonals over the copies of g), 0 on Dirichlet nodes.
__global__ void k_lv_invert(int64_t nl, const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                            const uint8_t* __restrict__ mask, const double* __restrict__ dE,
                            double* __restrict__ minvL)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nl; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = off[g], b = off[g + 1];
        double s = dE[mem[a]];
        for (int32_t m = a + 1; m < b; m++) s += dE[mem[m]];
        minvL[g] = mask[g] ? 1.0 / s : 0.0;
    }
}

template <class T>
nek_status upload(T** dst, const std::vector<T>& src)
{
    *dst = nullptr;
    const size_t bytes = sizeof(T) * std::max<size_t>(src.size(), 1);
    nek_status st = check_cuda(cudaMalloc(reinterpret_cast<void**>(dst), bytes));
    if (st != NEK_OK) return st;
    if (!src.empty()) st = check_cuda(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return st;
}

bool lvec_ok(const nek_lvec* lv, int64_t nelt, int nx)
{
    return lv && nelt >= 0 && nx >= kMinNx && nx <= kMaxNx && lv->npts == nelt * (int64_t)nx * nx * nx;
}

// edot (optional): element energies uL_e . (A_e uL_e) of the gathered field.
nek_status lvec_ax(const nek_lvec* lv, int64_t nelt, int nx, const double* D, const float* Gff, const double* uL,
                   double* wL, double* wE, cudaStream_t s, double* edot = nullptr)
{
    nek_status st = launch_ax_ff(nelt, nx, D, Gff, uL, wE, s, lv->d_l2g, nullptr, nullptr, edot);
    if (st != NEK_OK) return st;
    k_lv_assemble<<<stream_blocks(lv->nl), 256, 0, s>>>(lv->nl, lv->d_off, lv->d_mem, wE, wL);
    return check_launch();
}

}  // namespace

}  // namespace nek

using namespace nek;

extern "C" {

nek_status nek_lvec_create(int64_t npts, const int64_t* glo_num, const uint8_t* mask, nek_lvec** out)
{
    if (!out) return NEK_ERR_INVALID_ARG;
    *out = nullptr;
    if (npts < 0 || (npts > 0 && (!glo_num || !mask))) return NEK_ERR_INVALID_ARG;
    if (npts >= (int64_t(1) << 31)) return NEK_ERR_TOO_LARGE;
    std::vector<int32_t> l2g, off, mem;
    std::vector<uint8_t> mk;
    try {
        l2g.resize(static_cast<size_t>(npts));
        mem.resize(static_cast<size_t>(npts));
        off.push_back(0);
        int64_t gmax = -1;
        for (int64_t p = 0; p < npts; p++) {
            if (glo_num[p] < 0) return NEK_ERR_INVALID_ARG;
            gmax = std::max(gmax, glo_num[p]);
        }
        // order[q] = local points sorted by (global id, local index)
        std::vector<int32_t> order(static_cast<size_t>(npts));
        if (gmax < 4 * npts + 1024) {
            std::vector<int32_t> start(static_cast<size_t>(gmax + 2), 0);  // counting sort on the global id
            for (int64_t p = 0; p < npts; p++) start[glo_num[p] + 1]++;
            for (int64_t g = 0; g <= gmax; g++) start[g + 1] += start[g];
            for (int64_t p = 0; p < npts; p++) order[start[glo_num[p]]++] = static_cast<int32_t>(p);
        } else {
            std::vector<std::pair<int64_t, int32_t>> pr(static_cast<size_t>(npts));
            for (int64_t p = 0; p < npts; p++) pr[p] = {glo_num[p], static_cast<int32_t>(p)};
            std::sort(pr.begin(), pr.end());
            for (int64_t q = 0; q < npts; q++) order[q] = pr[q].second;
        }
        int64_t a = 0;
        while (a < npts) {
            const int64_t ga = glo_num[order[a]];
            int64_t b = a + 1;
            while (b < npts && glo_num[order[b]] == ga) b++;
            const int32_t g = static_cast<int32_t>(off.size() - 1);
            const uint8_t m0 = mask[order[a]] ? 1 : 0;
            for (int64_t q = a; q < b; q++) {
                const int32_t p = order[q];
                if ((mask[p] ? 1 : 0) != m0) return NEK_ERR_INVALID_ARG;  // copies disagree on the boundary
                l2g[p] = g;
                mem[q] = p;
            }
            mk.push_back(m0);
            off.push_back(static_cast<int32_t>(b));
            a = b;
        }
    } catch (const std::bad_alloc&) {
        return NEK_ERR_NOMEM;
    }
    nek_lvec* lv = new (std::nothrow) nek_lvec();
    if (!lv) return NEK_ERR_NOMEM;
    lv->npts = npts;
    lv->nl = static_cast<int64_t>(mk.size());
    lv->d_l2g = lv->d_off = lv->d_mem = nullptr;
    lv->d_mask = nullptr;
    nek_status st = upload(&lv->d_l2g, l2g);
    if (st == NEK_OK) st = upload(&lv->d_off, off);
    if (st == NEK_OK) st = upload(&lv->d_mem, mem);
    if (st == NEK_OK) st = upload(&lv->d_mask, mk);
    if (st != NEK_OK) {
        nek_lvec_destroy(lv);
        return st == NEK_ERR_CUDA ? NEK_ERR_NOMEM : st;
    }
    *out = lv;
    return NEK_OK;
}

nek_status nek_lvec_destroy(nek_lvec* lv)
{
    if (!lv) return NEK_OK;
    cudaFree(lv->d_l2g);
    cudaFree(lv->d_off);
    cudaFree(lv->d_mem);
    cudaFree(lv->d_mask);
    delete lv;
    return NEK_OK;
}

int64_t nek_lvec_size(const nek_lvec* lv) { return lv ? lv->nl : -1; }

nek_status nek_lvec_scatter(const nek_lvec* lv, const double* uL, double* uE, void* stream)
{
    if (!lv) return NEK_ERR_INVALID_ARG;
    if (lv->npts == 0) return NEK_OK;
    if (!uL || !uE || !is_aligned(uL, 8) || !is_aligned(uE, 8)) return NEK_ERR_INVALID_ARG;
    if (ranges_overlap(uL, sizeof(double) * lv->nl, uE, sizeof(double) * lv->npts)) return NEK_ERR_INVALID_ARG;
    k_lv_scatter<<<stream_blocks(lv->npts), 256, 0, static_cast<cudaStream_t>(stream)>>>(lv->npts, lv->d_l2g, uL,
                                                                                         uE);
    return check_launch();
}

nek_status nek_lvec_restrict(const nek_lvec* lv, const double* uE, double* uL, void* stream)
{
    if (!lv) return NEK_ERR_INVALID_ARG;
    if (lv->nl == 0) return NEK_OK;
    if (!uL || !uE || !is_aligned(uL, 8) || !is_aligned(uE, 8)) return NEK_ERR_INVALID_ARG;
    if (ranges_overlap(uL, sizeof(double) * lv->nl, uE, sizeof(double) * lv->npts)) return NEK_ERR_INVALID_ARG;
    k_lv_restrict<<<stream_blocks(lv->nl), 256, 0, static_cast<cudaStream_t>(stream)>>>(lv->nl, lv->d_off,
                                                                                        lv->d_mem, uE, uL);
    return check_launch();
}

nek_status nek_lvec_assemble(const nek_lvec* lv, const double* wE, double* wL, void* stream)
{
    if (!lv) return NEK_ERR_INVALID_ARG;
    if (lv->nl == 0) return NEK_OK;
    if (!wL || !wE || !is_aligned(wL, 8) || !is_aligned(wE, 8)) return NEK_ERR_INVALID_ARG;
    if (ranges_overlap(wL, sizeof(double) * lv->nl, wE, sizeof(double) * lv->npts)) return NEK_ERR_INVALID_ARG;
    k_lv_assemble<<<stream_blocks(lv->nl), 256, 0, static_cast<cudaStream_t>(stream)>>>(lv->nl, lv->d_off,
                                                                                        lv->d_mem, wE, wL);
    return check_launch();
}

nek_status nek_lvec_ax_ff(const nek_lvec* lv, int64_t nelt, int nx, const double* D, const float* Gff,
                          const double* uL, double* wL, double* wE, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!lvec_ok(lv, nelt, nx)) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Gff || !uL || !wL || !wE) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(D, 8) || !is_aligned(Gff, 16) || !is_aligned(uL, 8) || !is_aligned(wL, 8) || !is_aligned(wE, 8))
        return NEK_ERR_INVALID_ARG;
    const size_t bl = sizeof(double) * lv->nl, be = sizeof(double) * lv->npts;
    if (ranges_overlap(uL, bl, wL, bl) || ranges_overlap(uL, bl, wE, be) || ranges_overlap(wL, bl, wE, be))
        return NEK_ERR_INVALID_ARG;
    return lvec_ax(lv, nelt, nx, D, Gff, uL, wL, wE, static_cast<cudaStream_t>(stream));
}

nek_status nek_lvec_jacobi_minv(const nek_lvec* lv, int64_t nelt, int nx, const double* D, const double* G,
                                double* minvL, double* scratchE, void* stream)
{
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!lvec_ok(lv, nelt, nx)) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !G || !minvL || !scratchE || !is_aligned(G, 8) || !is_aligned(minvL, 8) || !is_aligned(scratchE, 8))
        return NEK_ERR_INVALID_ARG;
    if (ranges_overlap(minvL, sizeof(double) * lv->nl, scratchE, sizeof(double) * lv->npts))
        return NEK_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    nek_status st = launch_diag_local(nelt, nx, D, G, scratchE, s);
    if (st != NEK_OK) return st;
    k_lv_invert<<<stream_blocks(lv->nl), 256, 0, s>>>(lv->nl, lv->d_off, lv->d_mem, lv->d_mask, scratchE, minvL);
    return check_launch();
}

size_t nek_lvec_cg_workspace_bytes(const nek_lvec* lv)
{
    if (!lv) return 0;
    const size_t vec = pcg::align256(sizeof(double) * std::max<int64_t>(lv->nl, 1));
    return 3 * vec + pcg::align256(sizeof(double) * std::max<int64_t>(lv->npts, 1)) +
           pcg::align256(sizeof(double) * std::max<int64_t>(lv->npts, 1)) +  // element energies (<= npts)
           pcg::align256(sizeof(double) * 2 * kMaxReduceBlocks) + pcg::align256(sizeof(pcg::Scalars));
}

nek_status nek_lvec_cg_solve(const nek_lvec* lv, int64_t nelt, int nx, const double* D, const float* Gff,
                             const double* minvL, const double* fL, double* xL, double tol_rel, int max_iter,
                             void* workspace, int* iters_out, double* relres_out, nek_cg_opts* opts, void* stream)
{
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    if (nx < kMinNx || nx > kMaxNx) return NEK_ERR_UNSUPPORTED_NX;
    if (!lvec_ok(lv, nelt, nx) || max_iter < 0 || !(tol_rel >= 0.0)) return NEK_ERR_INVALID_ARG;
    if (nelt == 0) return NEK_OK;
    if (!D || !Gff || !minvL || !fL || !xL) return NEK_ERR_INVALID_ARG;
    if (!is_aligned(Gff, 16) || !is_aligned(minvL, 8) || !is_aligned(fL, 8) || !is_aligned(xL, 8))
        return NEK_ERR_INVALID_ARG;
    if (workspace && !is_aligned(workspace, 256)) return NEK_ERR_INVALID_ARG;
    const int check_every = (opts && opts->check_every > 0) ? opts->check_every : 1;
    const bool time_ax = opts && opts->time_ax;
    if (opts) {
        opts->ax_ms_total = 0.0;
        opts->ax_launches = 0;
        opts->kernel_launches = 0;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = nek_lvec_cg_workspace_bytes(lv);
    void* ws = workspace;
    nek_status st = NEK_OK;
    if (!ws) {
        st = check_cuda(cudaMallocAsync(&ws, bytes, s));
        if (st != NEK_OK) return NEK_ERR_NOMEM;
    }
    const size_t vec = pcg::align256(sizeof(double) * lv->nl);
    char* base = static_cast<char*>(ws);
    pcg::Buffers<double> b;
    b.r = reinterpret_cast<double*>(base);
    b.p = reinterpret_cast<double*>(base + vec);
    b.w = reinterpret_cast<double*>(base + 2 * vec);
    double* wE = reinterpret_cast<double*>(base + 3 * vec);
    size_t off = 3 * vec + pcg::align256(sizeof(double) * lv->npts);
    double* edot = reinterpret_cast<double*>(base + off);  // nelt entries
    off += pcg::align256(sizeof(double) * lv->npts);
    b.parts = reinterpret_cast<double*>(base + off);
    off += pcg::align256(sizeof(double) * 2 * kMaxReduceBlocks);
    b.sc = reinterpret_cast<pcg::Scalars*>(base + off);

    pcg::Result res;
    // the operator's element energies give <p,w> (p is zero on masked nodes)
    auto ax = [&](const double* p, double* w, double* ed, const DirUpdate*, cudaStream_t ss) {
        return lvec_ax(lv, nelt, nx, D, Gff, p, w, wE, ss, ed);
    };
    const pcg::ElementEnergies ee{edot, nelt};
    st = pcg::run<double>(nullptr, lv->nl, static_cast<const double*>(nullptr), lv->d_mask, minvL, fL, xL, b, tol_rel,
                          max_iter, check_every, time_ax, ax, s, &res, nullptr, &ee);
    if (iters_out) *iters_out = res.iters;
    if (relres_out) *relres_out = res.relres;
    if (opts) {
        opts->ax_ms_total = res.ax_ms;
        opts->ax_launches = res.ax_timed;
        opts->kernel_launches = res.launches;  // AX + assembly take the two slots of AX + dssum
    }
    if (!workspace) {
        cudaFreeAsync(ws, s);
        nek_status st2 = check_cuda(cudaStreamSynchronize(s));
        if (st == NEK_OK) st = st2;
    }
    return st;
}

}  // extern "C"
