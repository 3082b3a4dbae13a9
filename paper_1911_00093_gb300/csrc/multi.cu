// Many independent BiCG-STAB recurrences (Algorithm 1) advanced together: the
// right-hand sides of one H-matrix, or the problems of a block-diagonal batch
// handle, or both.  Every system owns a contiguous range of the stacked vectors
// (cluster order) and its own scalars; each vector kernel runs over a 2-D grid
// (blocks of a system x systems) and reduces its inner products per system with
// a fixed-order tree and the system's last block (deterministic).  All the
// decisions of a run -- stop, breakdown, true-residual acceptance, restart --
// are taken on the device, so the host only asks whether a system still runs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "hmat.h"
#include "kernels.h"

namespace hmat_internal {

namespace {

constexpr int kT = kVecThreads;

__device__ __forceinline__ bool sys_idle(const SysScalars &s) { return s.state != 0 || s.flag != 0; }

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * kT + threadIdx.x] = v[q];
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < NV; ++q) sh[q * kT + threadIdx.x] += sh[q * kT + threadIdx.x + s];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = sh[q * kT];
}

// Per-system two-stage reduction: block partials, then the system's last block
// adds them in block order.  Returns true in that block (totals in v).
template <int NV>
__device__ bool sys_reduce(double (&v)[NV], double *partials, SysScalars &S, double *sh) {
    __shared__ bool am_last;
    block_sum<NV>(v, sh);
    const int nb = gridDim.x;
    double *mine = partials + (size_t)blockIdx.y * NV * nb;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) mine[q * nb + blockIdx.x] = v[q];
        __threadfence();
        am_last = atomicAdd(&S.ticket, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double w[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        w[q] = 0.0;
        for (int b = threadIdx.x; b < nb; b += kT) w[q] += __ldcg(&mine[q * nb + b]);
    }
    __syncthreads();
    block_sum<NV>(w, sh);
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = w[q];
    if (threadIdx.x == 0) S.ticket = 0u;
    return true;
}

#define SYS_RANGE                                                     \
    const SysDesc sd = sys[blockIdx.y];                               \
    const int64_t i0 = sd.off;                                        \
    const int stride = gridDim.x * kT;                                \
    const int first = blockIdx.x * kT + threadIdx.x

// Start a run (counting its first iteration) from r = b - y: r~ = r, rho = ||r||^2.
// A run stops at ||r|| <= max(tol ||b||, inner_tol ||r_start||); a restart, which
// follows a failed true residual, always iterates (its stop is then tol ||b||
// alone should inner_tol be 1 or more).
__device__ void start_run(SysScalars &S, double rn, double tol, double inner_tol, int iter_limit, bool restart) {
    S.rnorm2 = rn;
    S.rho = rn;
    S.iter_in_run = 0;
    S.stop_on_s = 0;
    S.stop2 = fmax(tol * tol * S.bnorm2, inner_tol * inner_tol * rn);
    if (restart && rn <= S.stop2) S.stop2 = tol * tol * S.bnorm2;
    if (!isfinite(rn)) S.flag = HMAT_ERR_NONFINITE;
    else if (S.bnorm2 == 0.0 || rn <= S.stop2) S.flag = 1;  // nothing to iterate
    else if (S.iters >= iter_limit) S.flag = HMAT_ERR_MAXIT;
    else { S.flag = 0; S.iters += 1; }
}

// mode 0: ||b||^2 of every system (state reset);
// mode 1: r = b - y, r~ = r and a run starts (y = A~ x, the iterated operator);
// mode 2: the true residual r = b - y (y = the FP64 H-matrix times x) decides
//         acceptance (Section 4.1.3), the run's error, or a restart from r, for
//         every system whose run has stopped (the others keep iterating).
__global__ void __launch_bounds__(kT) k_mresidual(const SysDesc *__restrict__ sys, SysScalars *Sa, int mode,
                                                  const double *__restrict__ b, const double *__restrict__ y,
                                                  double *__restrict__ x, double *__restrict__ r,
                                                  double *__restrict__ rt, double *partials, double tol,
                                                  double inner_tol, int iter_limit, int max_restarts) {
    __shared__ double sh[kT];
    SysScalars &S = Sa[blockIdx.y];
    if (mode != 0 && S.state != 0) return;
    if (mode == 2 && S.flag == 0) return;  // its run goes on: no true residual yet
    SYS_RANGE;
    if (mode == 2 && S.bnorm2 == 0.0) {  // b = 0: x = 0 is the solution
        for (int i = first; i < sd.n; i += stride) x[i0 + i] = 0.0;
    }
    double a[1] = {0.0};
    for (int i = first; i < sd.n; i += stride) {
        const double rv = b[i0 + i] - (mode == 0 ? 0.0 : y[i0 + i]);
        if (mode != 0) {
            r[i0 + i] = rv;
            rt[i0 + i] = rv;
        }
        a[0] += rv * rv;
    }
    if (!sys_reduce<1>(a, partials, S, sh) || threadIdx.x != 0) return;
    const double rn = a[0];
    if (mode == 0) {
        S.bnorm2 = rn;
        S.state = isfinite(rn) ? 0 : 2;
        S.flag = isfinite(rn) ? 0 : HMAT_ERR_NONFINITE;
        S.iters = 0;
        S.restarts = 0;
        S.nmv = 0;
        S.nmv64 = 0;
        S.relres_true = 0.0;
        S.relres_inner = 0.0;
        return;
    }
    if (mode == 1) {
        start_run(S, rn, tol, inner_tol, iter_limit, false);
        return;
    }
    S.nmv64 += 1;
    S.relres_inner = S.bnorm2 > 0.0 ? sqrt(S.rnorm2 / S.bnorm2) : 0.0;
    const double rel = S.bnorm2 > 0.0 ? sqrt(rn / S.bnorm2) : 0.0;
    S.relres_true = rel;
    if (!isfinite(rel)) {
        S.flag = HMAT_ERR_NONFINITE;
        S.state = 2;
    } else if (rel <= tol) {
        S.flag = HMAT_OK;
        S.state = 1;
    } else if (S.flag > 1) {
        S.state = 2;  // the run ended on an error
    } else if (S.restarts >= max_restarts) {
        S.flag = HMAT_ERR_MAXIT;
        S.state = 2;
    } else {
        S.restarts += 1;
        start_run(S, rn, tol, inner_tol, iter_limit, true);
        if (S.flag > 1) S.state = 2;
    }
}

// The budget test and count of the next iteration of every running system
// (a restarted run's first iteration is counted by k_mresidual).
__global__ void k_mupdate_p(const SysDesc *__restrict__ sys, SysScalars *Sa, const double *__restrict__ r,
                            double *__restrict__ p, const double *__restrict__ v) {
    SysScalars &S = Sa[blockIdx.y];
    if (sys_idle(S)) return;
    const double rho = S.rho;
    if (!isfinite(rho) || rho == 0.0) {  // Algorithm 1: rho_{i-1} = 0 -> the method fails
        if (blockIdx.x == 0 && threadIdx.x == 0) S.flag = isfinite(rho) ? HMAT_ERR_BREAKDOWN_RHO : HMAT_ERR_NONFINITE;
        return;
    }
    SYS_RANGE;
    const bool firstit = S.iter_in_run == 0;
    const double beta = firstit ? 0.0 : (rho / S.rho_prev) * (S.alpha / S.omega);
    const double omega = S.omega;
    for (int i = first; i < sd.n; i += stride) {
        const int64_t k = i0 + i;
        p[k] = firstit ? r[k] : r[k] + beta * (p[k] - omega * v[k]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) S.nmv += 1;  // v = A p follows
}

// mode 1: alpha = rho / (r~ . v);  mode 2: omega = (t . s) / (t . t) (skipped
// after a stop at the ||s|| check)
__global__ void __launch_bounds__(kT) k_mdots(const SysDesc *__restrict__ sys, SysScalars *Sa, int mode,
                                              const double *__restrict__ a_, const double *__restrict__ b_,
                                              double *partials) {
    __shared__ double sh[2 * kT];
    SysScalars &S = Sa[blockIdx.y];
    if (sys_idle(S) || (mode == 2 && S.stop_on_s)) return;
    SYS_RANGE;
    double a[2] = {0.0, 0.0};
    for (int i = first; i < sd.n; i += stride) {
        const double u = a_[i0 + i], w = b_[i0 + i];
        a[0] += u * w;
        a[1] += w * w;
    }
    if (!sys_reduce<2>(a, partials, S, sh) || threadIdx.x != 0) return;
    if (mode == 1) {
        S.alpha = S.rho / a[0];
        if (!isfinite(S.alpha)) S.flag = HMAT_ERR_NONFINITE;
    } else {
        S.omega = a[1] == 0.0 ? 0.0 : a[0] / a[1];
        if (!isfinite(S.omega)) S.flag = HMAT_ERR_NONFINITE;
    }
}

// s = r - alpha v, ||s||^2 and the stop check
__global__ void __launch_bounds__(kT) k_mupdate_s(const SysDesc *__restrict__ sys, SysScalars *Sa,
                                                  const double *__restrict__ r, const double *__restrict__ v,
                                                  double *__restrict__ s, double *partials) {
    __shared__ double sh[kT];
    SysScalars &S = Sa[blockIdx.y];
    if (sys_idle(S)) return;
    SYS_RANGE;
    const double alpha = S.alpha;
    double a[1] = {0.0};
    for (int i = first; i < sd.n; i += stride) {
        const double sv = r[i0 + i] - alpha * v[i0 + i];
        s[i0 + i] = sv;
        a[0] += sv * sv;
    }
    if (!sys_reduce<1>(a, partials, S, sh) || threadIdx.x != 0) return;
    S.snorm2 = a[0];
    if (!isfinite(a[0])) S.flag = HMAT_ERR_NONFINITE;
    else if (a[0] <= S.stop2) S.stop_on_s = 1;
    else S.nmv += 1;  // t = A s follows
}

// x += alpha p + omega s; r = s - omega t; rho = r~ . r, ||r||^2, stop check;
// counts the next iteration when the run goes on
__global__ void __launch_bounds__(kT) k_mupdate_xr(const SysDesc *__restrict__ sys, SysScalars *Sa,
                                                   double *__restrict__ x, const double *__restrict__ p,
                                                   const double *__restrict__ s, const double *__restrict__ t,
                                                   double *__restrict__ r, const double *__restrict__ rt,
                                                   double *partials, int iter_limit) {
    __shared__ double sh[2 * kT];
    SysScalars &S = Sa[blockIdx.y];
    if (sys_idle(S)) return;
    SYS_RANGE;
    const bool at_s = S.stop_on_s != 0;
    const double alpha = S.alpha, omega = at_s ? 0.0 : S.omega;
    double a[2] = {0.0, 0.0};
    for (int i = first; i < sd.n; i += stride) {
        const int64_t k = i0 + i;
        const double sv = s[k];
        x[k] = x[k] + alpha * p[k] + omega * sv;
        const double rv = at_s ? sv : sv - omega * t[k];
        r[k] = rv;
        a[0] += rt[k] * rv;
        a[1] += rv * rv;
    }
    if (!sys_reduce<2>(a, partials, S, sh) || threadIdx.x != 0) return;
    S.rho_prev = S.rho;
    S.rho = a[0];
    S.rnorm2 = a[1];
    S.iter_in_run += 1;
    if (at_s) {
        S.rnorm2 = S.snorm2;
        S.flag = 1;
    } else if (!isfinite(a[1])) {
        S.flag = HMAT_ERR_NONFINITE;
    } else if (a[1] <= S.stop2) {
        S.flag = 1;
    } else if (omega == 0.0) {
        S.flag = HMAT_ERR_BREAKDOWN_OMEGA;
    } else if (S.iters >= iter_limit) {
        S.flag = HMAT_ERR_MAXIT;
    } else {
        S.iters += 1;
    }
}

// x (or b) of every system from original to cluster order and back; column k of
// an N x nrhs block uses the same permutation
__global__ void k_mgather(int64_t n, int nrhs, const int32_t *__restrict__ perm, const double *__restrict__ src,
                          double *__restrict__ dst) {
    const int64_t total = n * nrhs;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = q / n, p = q - k * n;
        dst[q] = src[k * n + perm[p]];
    }
}
__global__ void k_mscatter(int64_t n, int nrhs, const int32_t *__restrict__ perm, const double *__restrict__ src,
                           double *__restrict__ dst) {
    const int64_t total = n * nrhs;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = q / n, p = q - k * n;
        dst[k * n + perm[p]] = src[q];
    }
}

}  // namespace

int multi_blocks_x(int64_t max_n, int nsys) {
    int64_t b = (max_n + kT - 1) / kT;
    const int64_t cap = std::max<int64_t>(1, 4096 / std::max(1, nsys));
    if (b > cap) b = cap;
    return (int)std::max<int64_t>(b, 1);
}

void launch_mresidual(const MultiGrid &g, int mode, const double *b, const double *y, double *x, double *r, double *rt,
                      double tol, double inner_tol, int iter_limit, int max_restarts, cudaStream_t st) {
    k_mresidual<<<dim3(g.bx, g.nsys), kT, 0, st>>>(g.sys, g.S, mode, b, y, x, r, rt, g.partials, tol, inner_tol,
                                                    iter_limit, max_restarts);
}

void launch_miteration_vec(const MultiGrid &g, int step, const MultiVecs &v, int iter_limit, cudaStream_t st) {
    const dim3 grid(g.bx, g.nsys);
    switch (step) {
    case 0: k_mupdate_p<<<grid, kT, 0, st>>>(g.sys, g.S, v.r, v.p, v.v); break;
    case 1: k_mdots<<<grid, kT, 0, st>>>(g.sys, g.S, 1, v.rt, v.v, g.partials); break;
    case 2: k_mupdate_s<<<grid, kT, 0, st>>>(g.sys, g.S, v.r, v.v, v.s, g.partials); break;
    case 3: k_mdots<<<grid, kT, 0, st>>>(g.sys, g.S, 2, v.s, v.t, g.partials); break;
    case 4:
        k_mupdate_xr<<<grid, kT, 0, st>>>(g.sys, g.S, v.x, v.p, v.s, v.t, v.r, v.rt, g.partials, iter_limit);
        break;
    }
}

void launch_mgather(int64_t n, int nrhs, const int32_t *perm, const double *src, double *dst, cudaStream_t st) {
    const int64_t total = n * nrhs;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
    k_mgather<<<blocks, 256, 0, st>>>(n, nrhs, perm, src, dst);
}

void launch_mscatter(int64_t n, int nrhs, const int32_t *perm, const double *src, double *dst, cudaStream_t st) {
    const int64_t total = n * nrhs;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
    k_mscatter<<<blocks, 256, 0, st>>>(n, nrhs, perm, src, dst);
}

}  // namespace hmat_internal
