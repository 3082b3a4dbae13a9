// Launch wrappers of the device kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hmat_internal {

// Device-resident packing indices (shared by every precision copy of a handle).
struct DevIndex {
    int32_t n = 0, nleaves = 0, nlr = 0, nbig = 0, ntasks = 0;
    const int32_t *perm = nullptr;  // [n]
    const P1Desc *p1 = nullptr;     // [nleaves]
    const P1Run *p1_runs = nullptr;
    const XDst *xdst = nullptr;
    const LrDesc *lr = nullptr;     // [nlr]
    const int32_t *gdst = nullptr;
    const int32_t *red_big = nullptr, *red_tasks = nullptr;
    const P2Desc *p2 = nullptr;     // [nleaves]
    int32_t max_leaf = 0;           // rows of the widest leaf cluster
    int32_t max_ld2 = 0;            // widest phase-2 panel (entries)
};

// One precision copy of the panels plus its work buffers.
struct DevPanels {
    Store store = Store::DF;
    const void *q1 = nullptr;  // phase-1 panels
    const void *p2 = nullptr;  // phase-2 panels
    void *xs = nullptr;        // source-vector operand, cluster order (n entries of the operand type)
    void *part = nullptr;      // projection partial sums of multi-cluster blocks
    void *g = nullptr;         // phase-2 operand buffers (glen entries of the operand type)
};

// Operand bytes per entry for a store (x and t copies).
inline size_t operand_bytes(Store s) { return s == Store::F32 || s == Store::BF16 ? 4 : 8; }
inline size_t partial_bytes(Store s) { return s == Store::F32 || s == Store::BF16 ? 4 : 8; }

// Source-vector operand from an FP64 vector: src_perm != nullptr gathers
// x[src_perm[p]] (original order in), otherwise x is already in cluster order.
void launch_prep(Store s, const DevIndex &ix, const double *x, const int32_t *src_perm, void *xs,
                 cudaStream_t st);
struct SolverScalars;
// skipS/mode: a solver's product is skipped once its run has stopped (mode 1:
// flag set; mode 2: flag set or stop at the ||s|| check); mode 0 never skips.
void launch_phase1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st);
// t of the blocks spanning several leaf clusters, scattered into g (no launch when there is none)
void launch_reduce(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st);
// y[p] (cluster order) or y[out_perm[p]] (original order) = (A~ x)_p; dotmode 1/2
// also computes alpha (w = r~) or omega (w = s) of Algorithm 1 into Sd
void launch_phase2(Store s, const DevIndex &ix, const DevPanels &P, double *y, const int32_t *out_perm,
                   const SolverScalars *skipS, int mode, cudaStream_t st, const double *w = nullptr,
                   int dotmode = 0, SolverScalars *Sd = nullptr, double *dpart = nullptr);

// ---- BiCG-STAB vector kernels (FP64) ----
struct SolverScalars {
    double rho, rho_prev, alpha, omega;
    double rtv, ts, tt, snorm2, rnorm2, bnorm2, stop2;
    int32_t iter_in_run;  // 0 before the first iteration of a run
    int32_t flag;         // 0 running, 1 stop (converged this run), >1 an hmat_status error
    int32_t iters;        // iterations of this run
    int32_t stop_on_s;    // 1 if the run stopped at the ||s|| check
    unsigned int ticket;  // last-block counter of the fused reductions
    int32_t nmv;          // products with the iterated operator, excluding r_0
};

constexpr int kVecThreads = 256;
int vec_blocks(int64_t n);

// iteration budget test and count; then p = r (first iteration of a run) or
// p = r + beta (p - omega v), with the operand copy of p
void launch_count_iter(SolverScalars *S, int iter_limit, cudaStream_t st);
void launch_update_p(Store s, int64_t n, const double *r, double *p, const double *v, void *ps,
                     SolverScalars *S, cudaStream_t st);
// s = r - alpha v, operand copy of s, ||s||^2 and the stop check (x += alpha p on a stop)
void launch_update_s(Store s, int64_t n, const double *r, const double *v, double *svec, void *ss,
                     double *x, const double *p, SolverScalars *S, double *partials, cudaStream_t st);
// x += alpha p + omega s; r = s - omega t; rho = r~ . r, ||r||^2, stop check;
// counts the next iteration when the run goes on
void launch_update_xr(int64_t n, double *x, const double *p, const double *svec, const double *t, double *r,
                      const double *rt, SolverScalars *S, double *partials, int iter_limit, cudaStream_t st);
// r = b - y; r~ = r; ||r||^2 into S->rnorm2 and rho = r~ . r; resets the run state;
// iter_limit >= 0 starts a run (counts its first iteration)
void launch_residual(int64_t n, const double *b, const double *y, double *r, double *rt, SolverScalars *S,
                     double *partials, int iter_limit, cudaStream_t st);
// gather / scatter between original and cluster order
void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst_perm, cudaStream_t st);
void launch_scatter(int64_t n, const int32_t *perm, const double *src_perm, double *dst, cudaStream_t st);

}  // namespace hmat_internal
