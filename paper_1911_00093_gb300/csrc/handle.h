// The device handle of the hmat library (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hmat.h"
#include "hmat_internal.h"
#include "kernels.h"

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

struct hmat_t {
    using DevIndex = hmat_internal::DevIndex;
    using DevPanels = hmat_internal::DevPanels;
    using Store = hmat_internal::Store;
    using SolverScalars = hmat_internal::SolverScalars;
    int device = 0;
    int precision = 0;
    Store store = Store::DF, store64 = Store::DF;
    bool separate64 = false;
    DevIndex ix;
    DevPanels P, P64;
    std::vector<void *> allocs;
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
    // sizes
    int64_t panel_bytes = 0, panel_bytes64 = 0, index_bytes = 0;
    int64_t stored_entries = 0, phase1_entries = 0, phase2_entries = 0, partials_n = 0, rank_sum = 0;
    int64_t glen = 0;  // operand slots of the phase-2 buffers

    ~hmat_t() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (graph) cudaGraphExecDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (void *a : allocs) cudaFree(a);
        if (S_host) cudaFreeHost(S_host);
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
    template <class T>
    int upload(T **ptr, const void *host, size_t bytes) {
        int st = alloc(ptr, bytes);
        if (st != HMAT_OK) return st;
        if (bytes) CK(cudaMemcpy(*ptr, host, bytes, cudaMemcpyHostToDevice));
        return HMAT_OK;
    }
};

