// op2.cu -- the indirect edge-to-cell increment of the paper's OP2 example
// (Sec. 3.1): every edge i adds edge[i] to its two cells, in the sequential
// order "second end, then first end, edge by edge".
//
// Two kernels:
//   ordered -- a plan lists, for every cell, the edges that increment it in
//              exactly that sequential order (a stable counting sort of the
//              contributions, built once on the host).  One thread per cell
//              starts from the cell's value and adds its edges in list order in
//              FP64, so the result is the same bits as the sequential loop and
//              does not depend on the launch (the reproducible reading of the
//              loop, Sec. 3.1).  Where no cell has more than 8 contributions
//              (and the table stays within twice the list's size), the lists
//              are stored as D = 4 or 8 slots per cell, slot-major, padded with
//              -1: a thread's index loads are then coalesced and need no row
//              pointer first, one dependent load fewer.
//   atomic  -- one thread per edge, two FP64 atomicAdds: no plan, but the
//              order of the additions (and so the rounding) varies from run to
//              run -- the precision-for-speed switch Sec. 3.1 anticipates.
#include <algorithm>
#include <new>
#include <vector>

#include "internal.cuh"

namespace pencil {
namespace {

__global__ void __launch_bounds__(256)
    op2_ordered_kernel(const int *__restrict__ rowptr, const int *__restrict__ col,
                       const double *__restrict__ edge, double *__restrict__ cell, int ncells) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    double acc = cell[c];
    const int k1 = __ldg(rowptr + c + 1);
    // groups of up to 4 contributions: all their index and value loads are
    // issued before the additions, which stay in list order
    for (int k = __ldg(rowptr + c); k < k1; k += 4) {
        const int n = min(4, k1 - k);
        int e[4];
        double v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) e[j] = j < n ? __ldg(col + k + j) : 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = j < n ? __ldg(edge + e[j]) : 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < n) acc = __dadd_rn(acc, v[j]);
    }
    cell[c] = acc;
}

// The same additions from the slot-major table: slot s of cell c at
// ell[s * ncells + c], -1 past the cell's last contribution.
template <int D>
__global__ void __launch_bounds__(256)
    op2_ordered_ell_kernel(const int *__restrict__ ell, const double *__restrict__ edge, double *__restrict__ cell,
                           int ncells) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    double acc = cell[c];
    int e[D];
#pragma unroll
    for (int s = 0; s < D; ++s) e[s] = __ldg(ell + (size_t)s * ncells + c);
    double v[D];
#pragma unroll
    for (int s = 0; s < D; ++s) v[s] = e[s] >= 0 ? __ldg(edge + e[s]) : 0.0;
#pragma unroll
    for (int s = 0; s < D; ++s)
        if (e[s] >= 0) acc = __dadd_rn(acc, v[s]);
    cell[c] = acc;
}

__global__ void __launch_bounds__(256)
    op2_atomic_kernel(const int *__restrict__ e2c, const double *__restrict__ edge,
                      double *__restrict__ cell, int nedges) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nedges) return;
    const double e = __ldg(edge + i);
    const int2 cc = __ldg(reinterpret_cast<const int2 *>(e2c) + i);
    atomicAdd(cell + cc.y, e);
    atomicAdd(cell + cc.x, e);
}

}  // namespace
}  // namespace pencil

using namespace pencil;

struct pencil_op2_plan {
    int ncells = 0, nedges = 0;
    int ell_d = 0;          // slots per cell of the table (4 or 8), or 0: the lists below
    int *ell = nullptr;     // device, ell_d * ncells edge indices, slot-major, -1 padded
    int *rowptr = nullptr;  // device, ncells + 1 (without the table)
    int *col = nullptr;     // device, 2 * nedges edge indices, per cell in sequential order (without the table)
    int *e2c = nullptr;     // device, 2 * nedges
};

extern "C" {

int pencil_op2_plan_create(int ncells, int nedges, const int *e2c, pencil_op2_plan **out) {
    if (!out) return PENCIL_ERR_NULL;
    *out = nullptr;
    if (ncells <= 0 || nedges < 0 || nedges > (1 << 29)) return PENCIL_ERR_ARG;
    if (nedges > 0 && !e2c) return PENCIL_ERR_NULL;
    std::vector<int> count((size_t)ncells + 1, 0);
    for (long long t = 0; t < 2ll * nedges; ++t) {
        const int c = e2c[t];
        if (c < 0 || c >= ncells) return PENCIL_ERR_ARG;
        ++count[(size_t)c + 1];
    }
    for (int c = 0; c < ncells; ++c) count[(size_t)c + 1] += count[c];
    std::vector<int> col((size_t)2 * nedges > 0 ? (size_t)2 * nedges : 1);
    std::vector<int> pos(count.begin(), count.end() - 1);
    for (int i = 0; i < nedges; ++i) {  // sequential order: second end, then first end
        col[(size_t)pos[e2c[2 * i + 1]]++] = i;
        col[(size_t)pos[e2c[2 * i]]++] = i;
    }
    int maxdeg = 0;
    for (int c = 0; c < ncells; ++c) maxdeg = std::max(maxdeg, count[(size_t)c + 1] - count[c]);
    const int d = maxdeg == 0 ? 0 : (maxdeg <= 4 ? 4 : (maxdeg <= 8 ? 8 : 0));
    std::vector<int> ell;
    if (d > 0 && (size_t)d * ncells <= (size_t)4 * nedges) {
        ell.assign((size_t)d * ncells, -1);
        for (int c = 0; c < ncells; ++c)
            for (int j = count[c]; j < count[(size_t)c + 1]; ++j)
                ell[(size_t)(j - count[c]) * ncells + c] = col[(size_t)j];
    }
    pencil_op2_plan *p = new (std::nothrow) pencil_op2_plan;
    if (!p) return PENCIL_ERR_NOMEM;
    p->ncells = ncells;
    p->nedges = nedges;
    cudaError_t e = cudaSuccess;
    if (!ell.empty()) {
        p->ell_d = d;
        e = cudaMalloc(&p->ell, sizeof(int) * ell.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->ell, ell.data(), sizeof(int) * ell.size(), cudaMemcpyHostToDevice);
    } else {
        e = cudaMalloc(&p->rowptr, sizeof(int) * ((size_t)ncells + 1));
        if (e == cudaSuccess) e = cudaMalloc(&p->col, sizeof(int) * col.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(p->rowptr, count.data(), sizeof(int) * ((size_t)ncells + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->e2c, sizeof(int) * ((size_t)2 * nedges + 2));
    if (e == cudaSuccess && nedges > 0)
        e = cudaMemcpy(p->e2c, e2c, sizeof(int) * (size_t)2 * nedges, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->ell);
        cudaFree(p->rowptr);
        cudaFree(p->col);
        cudaFree(p->e2c);
        delete p;
        return e == cudaErrorMemoryAllocation ? PENCIL_ERR_NOMEM : cuda_fail(e);
    }
    *out = p;
    return PENCIL_OK;
}

int pencil_op2_inc(const pencil_op2_plan *p, const double *edge, double *cell, int mode, void *stream) {
    if (!p || !edge || !cell) return PENCIL_ERR_NULL;
    if (mode != PENCIL_OP2_ORDERED && mode != PENCIL_OP2_ATOMIC) return PENCIL_ERR_ARG;
    const uintptr_t eb = (uintptr_t)edge, cb = (uintptr_t)cell;
    const size_t en = sizeof(double) * (size_t)p->nedges, cn = sizeof(double) * (size_t)p->ncells;
    if (en && eb < cb + cn && cb < eb + en) return PENCIL_ERR_ALIAS;
    cudaPointerAttributes a;
    for (const void *q : {(const void *)edge, (const void *)cell}) {
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return PENCIL_ERR_PTR;
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return PENCIL_ERR_PTR;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == PENCIL_OP2_ORDERED) {
        const unsigned blocks = (unsigned)((p->ncells + 255) / 256);
        if (p->ell_d == 4)
            op2_ordered_ell_kernel<4><<<blocks, 256, 0, s>>>(p->ell, edge, cell, p->ncells);
        else if (p->ell_d == 8)
            op2_ordered_ell_kernel<8><<<blocks, 256, 0, s>>>(p->ell, edge, cell, p->ncells);
        else
            op2_ordered_kernel<<<blocks, 256, 0, s>>>(p->rowptr, p->col, edge, cell, p->ncells);
    } else if (p->nedges > 0) {
        op2_atomic_kernel<<<(p->nedges + 255) / 256, 256, 0, s>>>(p->e2c, edge, cell, p->nedges);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_op2_plan_destroy(pencil_op2_plan *p) {
    if (!p) return PENCIL_OK;
    cudaFree(p->ell);
    cudaFree(p->rowptr);
    cudaFree(p->col);
    cudaFree(p->e2c);
    delete p;
    return PENCIL_OK;
}

}  // extern "C"
