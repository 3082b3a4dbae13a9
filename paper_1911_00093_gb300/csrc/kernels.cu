// Launchers of the product kernels for the library's own stores (DF, F64, F32,
// BF16) and the BiCG-STAB vector kernels (sm_103a).  The paper's variants
// (stores PM, PS, PM1, PS2) are instantiated in kernels_table1.cu.
#include "product.cuh"

namespace hmat_internal {

// ------------------------------------------------------------------------
// product launchers
// ------------------------------------------------------------------------
#define HMAT_DISPATCH(S, CALL)                                    \
    switch (S) {                                                  \
    case Store::DF: { constexpr Store SS = Store::DF; CALL; } break;   \
    case Store::F64: { constexpr Store SS = Store::F64; CALL; } break; \
    case Store::F32: { constexpr Store SS = Store::F32; CALL; } break; \
    case Store::BF16: { constexpr Store SS = Store::BF16; CALL; } break; \
    default: break;                                               \
    }

// the paper's variants keep x in FP64 (their FP32 copies are made in phase 1)
static Store operand_store(Store s) { return is_table1(s) ? Store::F64 : s; }

void launch_prep(Store s, const DevIndex &ix, const double *x, const int32_t *src_perm, void *xs, cudaStream_t st) {
    int blocks = grid_for(ix.n, 256, 4096);
    HMAT_DISPATCH(operand_store(s),
                  launch_pdl(k_prep<SS>, dim3(blocks), dim3(256), st, ix.n, x, src_perm, (typename Tr<SS>::Op *)xs));
}

void launch_phase1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st, const SysScalars *sys) {
    if (is_table1(s)) return launch_phase1_table1(s, ix, P, skipS, mode, st, sys);
    HMAT_DISPATCH(s, phase1_launch<SS>(ix, P, skipS, mode, st, sys));
}

float time_phase1(Store s, const DevIndex &ix, const DevPanels &P, int reps, cudaStream_t st) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    launch_phase1(s, ix, P, nullptr, 0, st);  // warm-up
    cudaEventRecord(a, st);
    for (int k = 0; k < reps; ++k) launch_phase1(s, ix, P, nullptr, 0, st);
    cudaEventRecord(b, st);
    float ms = -1.f;
    if (cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms < 0.f ? -1.f : 1e3f * ms / (float)reps;
}

int phase1_default_threads(Store s) {
    switch (s) {
    case Store::BF16: return p1_threads<Store::BF16>();
    default: return 256;
    }
}

void launch_reduce(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st, const SysScalars *sys) {
    if (is_table1(s)) return launch_reduce_table1(s, ix, P, skipS, mode, st, sys);
    HMAT_DISPATCH(s, reduce_launch<SS>(ix, P, skipS, mode, st, sys));
}

void launch_phase2(Store s, const DevIndex &ix, const DevPanels &P, double *y, const int32_t *out_perm, int accum,
                   const SolverScalars *skipS, int mode, cudaStream_t st, const double *w, int dotmode,
                   double *dpart, const SysScalars *sys) {
    if (is_table1(s))
        return launch_phase2_table1(s, ix, P, y, out_perm, accum, skipS, mode, st, w, dotmode, dpart, sys);
    HMAT_DISPATCH(s, phase2_launch<SS>(ix, P, y, out_perm, accum, skipS, mode, st, w, dotmode, dpart, sys));
}


// ------------------------------------------------------------------------
// BiCG-STAB vector kernels: FP64 arithmetic, deterministic two-stage
// reductions (per block: warp butterflies, then the warps in order; then the
// last block sums the block partials in block order)
// ------------------------------------------------------------------------
namespace {

// Every thread gets the CTA's sums: the first warp adds 8 consecutive values
// per lane, then a butterfly over its lanes (FP64 additions run at about one
// per clock per SM on GB300, so few warp-wide ones: 13 per sum).
// sh: NV * kVecThreads doubles; ends with a barrier.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double *sh) {
    constexpr int PER = kVecThreads / 32;
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * kVecThreads + threadIdx.x] = v[q];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = 0.0;
            for (int k = 0; k < PER; ++k) t += sh[q * kVecThreads + threadIdx.x * PER + k];
            for (int m = 16; m >= 1; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
            if (threadIdx.x == 0) sh[q * kVecThreads] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = sh[q * kVecThreads];
    __syncthreads();
}

// Block partials -> last block; returns true in the last block, where tot[] holds the totals.
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double *partials, SolverScalars *S, double *sh) {
    __shared__ bool am_last;
    block_reduce<NV>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[q * gridDim.x + blockIdx.x] = v[q];
        __threadfence();
        unsigned int t = atomicAdd(&S->ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double w[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        w[q] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) w[q] += __ldcg(&partials[q * gridDim.x + b]);
    }
    block_reduce<NV>(w, sh);
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = w[q];
    if (threadIdx.x == 0) S->ticket = 0u;
    return true;
}

// The expansion's shares of an inner product (ndp work items, NV products laid
// out one after the other) added in a fixed order: every CTA gets the same bits.
template <int NV>
__device__ __forceinline__ void share_sum(const double *__restrict__ dpart, int ndp, double (&v)[NV], double *sh) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        v[q] = 0.0;
        for (int k = threadIdx.x; k < ndp; k += blockDim.x) v[q] += __ldg(dpart + (size_t)q * ndp + k);
    }
    block_reduce<NV>(v, sh);  // ends with a barrier: sh is free for the caller
}

__device__ __forceinline__ bool run_stopped(const SolverScalars *S) {
    return *(volatile const int32_t *)&S->flag != 0;
}

// Starts an iteration: the budget test, then the count (an iteration whose rho
// test fails is counted, one refused by the budget is not).
__global__ void k_count_iter(SolverScalars *S, int iter_limit) {
    if (S->flag != 0) return;
    if (S->iters >= iter_limit) S->flag = HMAT_ERR_MAXIT;
    else S->iters += 1;
}

template <Store ST>
__global__ void __launch_bounds__(kVecThreads) k_update_p(int n, const double *__restrict__ r, double *__restrict__ p,
                                                          const double *__restrict__ v, typename Tr<ST>::Op *__restrict__ ps,
                                                          SolverScalars *S) {
    if (run_stopped(S)) return;
    const double rho = S->rho;
    const bool first = S->iter_in_run == 0;
    if (!isfinite(rho) || rho == 0.0) {  // Algorithm 1: rho_{i-1} = 0 -> the method fails
        if (blockIdx.x == 0 && threadIdx.x == 0) S->flag = isfinite(rho) ? HMAT_ERR_BREAKDOWN_RHO : HMAT_ERR_NONFINITE;
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) S->nmv += 1;  // v = A p follows
    const double beta = first ? 0.0 : (rho / S->rho_prev) * (S->alpha / S->omega);
    const double omega = S->omega;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double pv = p_next(first, r[i], p[i], v[i], beta, omega);
        p[i] = pv;
        if constexpr (ST == Store::DF) ps[i] = split_double(pv);
        else if constexpr (ST == Store::F64) ps[i] = pv;
        else ps[i] = __double2float_rn(pv);
    }
}

template <Store ST>
__global__ void __launch_bounds__(kVecThreads) k_update_s(int n, const double *__restrict__ r, const double *__restrict__ v,
                                                          double *__restrict__ s, typename Tr<ST>::Op *__restrict__ ss,
                                                          SolverScalars *S, double *partials,
                                                          const double *__restrict__ dpart, int ndp) {
    __shared__ double sh[kVecThreads];
    if (run_stopped(S)) return;
    // alpha = rho / (r~ . v) (Algorithm 1), the same in every CTA
    double rtv[1];
    share_sum<1>(dpart, ndp, rtv, sh);
    const double alpha = S->rho / rtv[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->rtv = rtv[0];
        S->alpha = alpha;
        if (!isfinite(alpha)) S->flag = HMAT_ERR_NONFINITE;
    }
    if (!isfinite(alpha)) return;
    double a[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double sv = r[i] - alpha * v[i];
        s[i] = sv;
        a[0] += sv * sv;
        if constexpr (ST == Store::DF) ss[i] = split_double(sv);
        else if constexpr (ST == Store::F64) ss[i] = sv;
        else ss[i] = __double2float_rn(sv);
    }
    if (grid_reduce<1>(a, partials, S, sh) && threadIdx.x == 0) {
        S->snorm2 = a[0];
        if (!isfinite(a[0])) S->flag = HMAT_ERR_NONFINITE;
        else if (a[0] <= S->stop2) S->stop_on_s = 1;
        else S->nmv += 1;  // t = A s follows
    }
}

__global__ void __launch_bounds__(kVecThreads) k_update_xr(int n, double *__restrict__ x, const double *__restrict__ p,
                                                           const double *__restrict__ s, const double *__restrict__ t,
                                                           double *__restrict__ r, const double *__restrict__ rt,
                                                           SolverScalars *S, double *partials,
                                                           const double *__restrict__ dpart, int ndp, int iter_limit) {
    __shared__ double sh[2 * kVecThreads];
    if (run_stopped(S)) return;
    const bool at_s = S->stop_on_s != 0;
    const double alpha = S->alpha;
    double omega = 0.0;
    if (!at_s) {  // omega = (t . s) / (t . t) (Algorithm 1), the same in every CTA
        double d[2];
        share_sum<2>(dpart, ndp, d, sh);
        omega = d[1] == 0.0 ? 0.0 : d[0] / d[1];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            S->ts = d[0];
            S->tt = d[1];
            S->omega = omega;
            if (!isfinite(omega)) S->flag = HMAT_ERR_NONFINITE;
        }
        if (!isfinite(omega)) return;
    }
    double a[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double sv = s[i];
        x[i] = x[i] + alpha * p[i] + omega * sv;
        double rv = at_s ? sv : sv - omega * t[i];
        r[i] = rv;
        a[0] += rt[i] * rv;
        a[1] += rv * rv;
    }
    if (grid_reduce<2>(a, partials, S, sh) && threadIdx.x == 0) {
        S->rho_prev = S->rho;
        S->rho = a[0];
        S->rnorm2 = a[1];
        S->iter_in_run += 1;
        if (at_s) {
            S->rnorm2 = S->snorm2;
            S->flag = 1;
        } else if (!isfinite(a[1])) {
            S->flag = HMAT_ERR_NONFINITE;
        } else if (a[1] <= S->stop2) {
            S->flag = 1;
        } else if (omega == 0.0) {
            S->flag = HMAT_ERR_BREAKDOWN_OMEGA;
        } else if (S->iters >= iter_limit) {  // the next iteration is over budget
            S->flag = HMAT_ERR_MAXIT;
        } else {
            S->iters += 1;
        }
    }
}

__global__ void __launch_bounds__(kVecThreads) k_residual(int n, const double *__restrict__ b, const double *__restrict__ y,
                                                          double *__restrict__ r, double *__restrict__ rt,
                                                          SolverScalars *S, double *partials, int iter_limit) {
    __shared__ double sh[kVecThreads];
    double a[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double rv = b[i] - (y ? y[i] : 0.0);
        r[i] = rv;
        rt[i] = rv;
        a[0] += rv * rv;
    }
    if (grid_reduce<1>(a, partials, S, sh) && threadIdx.x == 0) {
        if (iter_limit < 0) {  // a true residual: keep the state of the run it follows
            S->run_flag = S->flag;
            S->run_rnorm2 = S->rnorm2;
        }
        S->rnorm2 = a[0];
        S->rho = a[0];
        S->iter_in_run = 0;
        S->stop_on_s = 0;
        S->flag = isfinite(a[0]) ? 0 : HMAT_ERR_NONFINITE;
        if (iter_limit >= 0 && S->flag == 0) {  // a run starts: count its first iteration
            if (S->iters >= iter_limit) S->flag = HMAT_ERR_MAXIT;
            else S->iters += 1;
        }
    }
}

__global__ void k_gather(int n, const int32_t *__restrict__ perm, const double *__restrict__ src, double *__restrict__ dst) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) dst[p] = src[perm[p]];
}
__global__ void k_scatter(int n, const int32_t *__restrict__ perm, const double *__restrict__ src, double *__restrict__ dst) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) dst[perm[p]] = src[p];
}

}  // namespace

int vec_blocks(int64_t n) { return grid_for(n, kVecThreads, 4 * 152); }

void launch_count_iter(SolverScalars *S, int iter_limit, cudaStream_t st) { k_count_iter<<<1, 1, 0, st>>>(S, iter_limit); }

namespace {
__global__ void k_loop_condition(SolverScalars *S, cudaGraphConditionalHandle cond, int max_loops) {
    const int loops = ++S->loops;
    cudaGraphSetConditional(cond, (S->flag == 0 && loops < max_loops) ? 1u : 0u);
}
}  // namespace

void launch_loop_condition(SolverScalars *S, cudaGraphConditionalHandle cond, int max_loops, cudaStream_t st) {
    k_loop_condition<<<1, 1, 0, st>>>(S, cond, max_loops);
}

void launch_update_p(Store s, int64_t n, const double *r, double *p, const double *v, void *ps, SolverScalars *S,
                     cudaStream_t st) {
    HMAT_DISPATCH(operand_store(s), (k_update_p<SS><<<vec_blocks(n), kVecThreads, 0, st>>>((int)n, r, p, v,
                                                                           (typename Tr<SS>::Op *)ps, S)));
}

void launch_update_s(Store s, int64_t n, const double *r, const double *v, double *svec, void *ss,
                     SolverScalars *S, double *partials, const double *dpart, int ndp, cudaStream_t st) {
    HMAT_DISPATCH(operand_store(s), (k_update_s<SS><<<vec_blocks(n), kVecThreads, 0, st>>>(
                                        (int)n, r, v, svec, (typename Tr<SS>::Op *)ss, S, partials, dpart, ndp)));
}

void launch_update_xr(int64_t n, double *x, const double *p, const double *svec, const double *t, double *r,
                      const double *rt, SolverScalars *S, double *partials, const double *dpart, int ndp,
                      int iter_limit, cudaStream_t st) {
    k_update_xr<<<vec_blocks(n), kVecThreads, 0, st>>>((int)n, x, p, svec, t, r, rt, S, partials, dpart, ndp,
                                                       iter_limit);
}

void launch_residual(int64_t n, const double *b, const double *y, double *r, double *rt, SolverScalars *S,
                     double *partials, int iter_limit, cudaStream_t st) {
    k_residual<<<vec_blocks(n), kVecThreads, 0, st>>>((int)n, b, y, r, rt, S, partials, iter_limit);
}

void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst_perm, cudaStream_t st) {
    k_gather<<<grid_for(n, 256, 4096), 256, 0, st>>>((int)n, perm, src, dst_perm);
}

void launch_scatter(int64_t n, const int32_t *perm, const double *src_perm, double *dst, cudaStream_t st) {
    k_scatter<<<grid_for(n, 256, 4096), 256, 0, st>>>((int)n, perm, src_perm, dst);
}

}  // namespace hmat_internal
