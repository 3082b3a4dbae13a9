// The device handle of the hmat library (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hmat.h"
#include "hmat_internal.h"
#include "kernels.h"
#include "mdf.h"

namespace hmat_internal {

// Text of the last CUDA error seen in this thread (hmat_last_cuda_error).
std::string &last_cuda_error();

inline bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    last_cuda_error() = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

}  // namespace hmat_internal

#define CK(call)                                                             \
    do {                                                                     \
        if (!hmat_internal::cuda_ok((call), #call)) return HMAT_ERR_CUDA;    \
    } while (0)

// One packed operator piece: indices, typed panels and work buffers.  The
// library's own forms are one segment; a paper variant is one or two segments
// whose products add up (paper_forms.cpp).
struct HmatSegment {
    hmat_internal::DevIndex ix;
    hmat_internal::DevPanels P;
    hmat_internal::Store store = hmat_internal::Store::DF;
    int64_t partials_n = 0, glen = 0;
};

struct hmat_t {
    using DevIndex = hmat_internal::DevIndex;
    using DevPanels = hmat_internal::DevPanels;
    using Store = hmat_internal::Store;
    using SolverScalars = hmat_internal::SolverScalars;
    int device = 0;
    int precision = 0;
    int method3_c = 0;
    int64_t n = 0;
    const int32_t *perm = nullptr;  // [n] cluster order -> original index (device)
    HmatSegment seg[2];             // the iterated operator A~ (seg[1] adds into seg[0]'s y)
    int nseg = 1;
    HmatSegment seg64;              // the FP64 H-matrix of the true residual (Section 4.1.3)
    std::vector<void *> allocs;
    // HMAT_ERR_TIMEOUT from a bounded device wait of one of the handle's kernels
    // (mapped pinned memory: the kernels write it, the host reads it at the
    // next call or at hmat_check)
    int32_t *status_host = nullptr, *status_dev = nullptr;
    std::vector<int64_t> prob_off;  // problem p owns [prob_off[p], prob_off[p+1]) (batch handles)
    // GMRES buffers (first GMRES solve; sized for the restart length m)
    struct Gmres {
        int m = 0;
        double *V = nullptr, *w = nullptr, *r = nullptr, *b = nullptr, *x = nullptr, *part = nullptr, *partials = nullptr;
        double *x0 = nullptr, *r0 = nullptr, *d = nullptr;  // the run's start and the correction d = x - x0
        hmat_internal::GmresState *G = nullptr, *G_host = nullptr;
        cudaGraphExec_t graph = nullptr;
        int graph_m = 0, graph_limit = -1;
        std::vector<void *> mine;
    } gm;
    hmat_internal::MdfBufs mdf;     // many-column double-float product (first use)
    bool mrhs = false;              // BF16 handle with the many-right-hand-side tensor-core product
    hmat_internal::MrhsIndex mx;    // its indices (upload) and buffers (first use)
    // buffers of the many-system solver, sized for `cap` right-hand sides
    struct Multi {
        int cap = 0;
        double *b = nullptr, *x = nullptr, *r = nullptr, *rt = nullptr, *p = nullptr, *v = nullptr, *s = nullptr,
               *t = nullptr, *y = nullptr, *stage = nullptr, *partials = nullptr;
        hmat_internal::SysDesc *sys = nullptr;
        hmat_internal::SysScalars *S = nullptr, *S_host = nullptr;
        int32_t *cols = nullptr, *cols_host = nullptr;  // the columns of a true-residual pass (device, pinned)
        cudaGraphExec_t graph = nullptr;
        int graph_k = 0, graph_limit = -1, graph_nrhs = 0;
        std::vector<void *> mine;
    } multi;
    // solver state, cluster order
    double *b = nullptr, *x = nullptr, *r = nullptr, *rt = nullptr, *p = nullptr, *v = nullptr, *s = nullptr,
           *t = nullptr, *y = nullptr;
    double *partials = nullptr;  // 2 x vec_blocks: grid reductions of the vector kernels
    double *dpart = nullptr;     // 2 x nleaves: per-work-item sums of the fused dot products
    SolverScalars *S = nullptr;
    SolverScalars *S_host = nullptr;  // pinned
    double *stage_in = nullptr, *stage_out = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_k = 0, graph_limit = -1;
    // a run as one graph: a WHILE node over batches of graph_k iterations
    cudaGraphExec_t loop_graph = nullptr;
    int loop_k = 0, loop_limit = -1;
    // sizes
    int64_t panel_bytes = 0, panel_bytes64 = 0, index_bytes = 0;
    int64_t panel_bytes_mrhs = 0;  // W tiles of the many-right-hand-side projection (BF16 handles)
    int64_t stored_entries = 0, phase1_entries = 0, phase2_entries = 0, partials_n = 0, rank_sum = 0;
    int64_t phase1_bytes = 0, phase2_bytes = 0;

    ~hmat_t() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (graph) cudaGraphExecDestroy(graph);
        if (multi.graph) cudaGraphExecDestroy(multi.graph);
        if (gm.graph) cudaGraphExecDestroy(gm.graph);
        if (gm.G_host) cudaFreeHost(gm.G_host);
        if (multi.S_host) cudaFreeHost(multi.S_host);
        if (multi.cols_host) cudaFreeHost(multi.cols_host);
        if (loop_graph) cudaGraphExecDestroy(loop_graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (void *a : allocs) cudaFree(a);
        if (S_host) cudaFreeHost(S_host);
        if (status_host) cudaFreeHost(status_host);
        cudaSetDevice(cur);
    }

    template <class T>
    int alloc(T **ptr, size_t bytes) {
        void *q = nullptr;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            hmat_internal::last_cuda_error() = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            return HMAT_ERR_NOMEM;
        }
        allocs.push_back(q);
        *ptr = (T *)q;
        return HMAT_OK;
    }
    // release one allocation made by alloc()
    void release(void *q) {
        if (!q) return;
        for (size_t k = 0; k < allocs.size(); ++k)
            if (allocs[k] == q) {
                cudaFree(q);
                allocs.erase(allocs.begin() + k);
                return;
            }
    }
    template <class T>
    int upload(T **ptr, const void *host, size_t bytes) {
        int st = alloc(ptr, bytes);
        if (st != HMAT_OK) return st;
        if (bytes) CK(cudaMemcpy(*ptr, host, bytes, cudaMemcpyHostToDevice));
        return HMAT_OK;
    }
};

// A timeout recorded by a bounded device wait of the handle's kernels, taken
// (cleared) by the call that reports it; HMAT_OK when there is none.
inline int take_status(hmat_t *h) {
    volatile int32_t *s = h->status_host;
    if (!s || *s == 0) return HMAT_OK;
    const int e = *s;
    *s = 0;
    return e;
}
