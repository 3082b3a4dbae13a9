// Restarted GMRES(m) on the device (a second Krylov method on the same
// products; Section 4.5 names other solvers as the next step): Arnoldi with
// classical Gram-Schmidt applied twice (CGS2), Givens rotations on the
// Hessenberg matrix, x += V y at the end of each cycle.  Every reduction is a
// fixed-order two-stage sum (deterministic); the rotations, the stop test and
// the triangular solve run in one thread on the device, so a whole cycle of m
// steps is one graph launch and the host reads the state once per cycle.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "hmat.h"
#include "kernels.h"

namespace hmat_internal {

namespace {

constexpr int kT = kVecThreads;

__device__ __forceinline__ void bsum(double &v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    v = sh[0];
    __syncthreads();
}

// ||a||^2 over the grid; true in the last block (total in v)
__device__ bool grid_sum(double &v, double *partials, unsigned int *ticket, double *sh) {
    __shared__ bool am_last;
    bsum(v, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v;
        __threadfence();
        am_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double w = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kT) w += __ldcg(&partials[b]);
    bsum(w, sh);
    v = w;
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// mode 2: ||b||;
// mode 3: the true residual r = b - y (y = A64 x), which also starts the next
//         run on the correction equation A~ d = r (its stop: max(tol ||b||,
//         inner_tol ||r||));
// mode 1: r = b - y between the cycles of a run (b = the run's r_0, y = A~ (x - x_0))
__global__ void __launch_bounds__(kT) k_g_residual(int n, int mode, const double *__restrict__ b,
                                                   const double *__restrict__ y, double *__restrict__ r,
                                                   GmresState *G, double tol, double inner_tol) {
    __shared__ double sh[kT];
    double a = 0.0;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        const double rv = b[i] - (mode == 2 ? 0.0 : y[i]);
        if (mode != 2) r[i] = rv;
        a += rv * rv;
    }
    if (!grid_sum(a, G->partials, &G->ticket, sh) || threadIdx.x != 0) return;
    if (mode == 2) {
        G->bnorm2 = a;
    } else if (mode == 1) {
        G->rnorm = sqrt(a);
    } else {
        G->relres_true = sqrt(a / G->bnorm2);
        G->nmv64 += 1;
        G->rnorm = sqrt(a);
        G->stop = fmax(tol * sqrt(G->bnorm2), inner_tol * sqrt(a));
        G->run_over = 0;
    }
}
// d = x - x_0
__global__ void k_g_diff(int n, const double *__restrict__ x, const double *__restrict__ x0, double *__restrict__ d) {
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) d[i] = x[i] - x0[i];
}

// A cycle starts from r: beta = ||r|| (known from the residual kernel), the run
// ends if beta is below its stop (or the budget is spent), else v_0 = r / beta.
__global__ void k_g_start_cycle(GmresState *G, int m, int maxit) {
    const double beta = G->rnorm;
    G->j = 0;
    if (!isfinite(beta)) {
        G->status = HMAT_ERR_NONFINITE;
        G->run_over = 1;
    } else if (beta <= G->stop) {
        G->run_over = 1;
    } else if (G->it >= maxit) {
        G->status = HMAT_ERR_MAXIT;
        G->run_over = 1;
    }
    G->s.flag = G->run_over ? 1 : 0;  // the products of a finished cycle are skipped
    for (int i = 0; i <= m; ++i) G->g[i] = 0.0;
    G->g[0] = beta;
}
__global__ void k_g_scale0(int n, const double *__restrict__ r, double *__restrict__ v0, const GmresState *G) {
    if (G->s.flag) return;
    const double inv = 1.0 / G->rnorm;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) v0[i] = r[i] * inv;
}

// partial inner products of w with columns 0..j of V: grid (blocks, j + 1)
__global__ void __launch_bounds__(kT) k_g_dots(int n, const double *__restrict__ V, int ldv,
                                               const double *__restrict__ w, const GmresState *G, int jj,
                                               double *__restrict__ part) {
    __shared__ double sh[kT];
    if (G->s.flag) return;
    const double *v = V + (size_t)blockIdx.y * ldv;
    double a = 0.0;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) a += v[i] * w[i];
    bsum(a, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = a;
    (void)jj;
}
// h_pass[i] = sum of the partials in block order; h[i] accumulates the passes
__global__ void __launch_bounds__(kT) k_g_dots_fin(int nb, const double *__restrict__ part, GmresState *G, int pass) {
    __shared__ double sh[kT];
    if (G->s.flag) return;
    const int i = blockIdx.x;
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += kT) a += part[(size_t)i * nb + b];
    bsum(a, sh);
    if (threadIdx.x == 0) {
        G->hp[i] = a;
        G->h[i] = (pass == 0 ? 0.0 : G->h[i]) + a;
    }
}
// w -= V h_pass (columns 0..jj)
__global__ void k_g_orth(int n, const double *__restrict__ V, int ldv, double *__restrict__ w, const GmresState *G,
                         int jj) {
    if (G->s.flag) return;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        double s = w[i];
        for (int c = 0; c <= jj; ++c) s -= G->hp[c] * V[(size_t)c * ldv + i];
        w[i] = s;
    }
}
// ||w||, column jj of the Hessenberg matrix, the rotations, the residual
// estimate |g_{jj+1}| and the stop test of this step
__global__ void __launch_bounds__(kT) k_g_rotate(int n, const double *__restrict__ w, GmresState *G, int jj, int m,
                                                 int maxit) {
    __shared__ double sh[kT];
    if (G->s.flag) return;
    double a = 0.0;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) a += w[i] * w[i];
    if (!grid_sum(a, G->partials, &G->ticket, sh) || threadIdx.x != 0) return;
    const double hn = sqrt(a);
    double *col = G->H + (size_t)jj * (m + 1);
    for (int i = 0; i <= jj; ++i) col[i] = G->h[i];
    col[jj + 1] = hn;
    for (int i = 0; i < jj; ++i) {
        const double x0 = col[i], x1 = col[i + 1];
        col[i] = G->cs[i] * x0 + G->sn[i] * x1;
        col[i + 1] = -G->sn[i] * x0 + G->cs[i] * x1;
    }
    const double den = sqrt(col[jj] * col[jj] + col[jj + 1] * col[jj + 1]);
    G->cs[jj] = den == 0.0 ? 1.0 : col[jj] / den;
    G->sn[jj] = den == 0.0 ? 0.0 : col[jj + 1] / den;
    col[jj] = den;
    col[jj + 1] = 0.0;
    G->g[jj + 1] = -G->sn[jj] * G->g[jj];
    G->g[jj] = G->cs[jj] * G->g[jj];
    const double resid = fabs(G->g[jj + 1]);
    G->it += 1;
    G->s.nmv += 1;
    G->j = jj + 1;
    G->hn = hn;
    G->resid = resid;
    if (!isfinite(resid)) {
        G->status = HMAT_ERR_NONFINITE;
        G->s.flag = 1;
    } else if (hn == 0.0 || resid <= G->stop || jj + 1 == m || G->it >= maxit) {
        G->s.flag = 1;  // the cycle ends here
    }
}
// v_{jj+1} = w / h_{jj+1,jj} (when the cycle goes on)
__global__ void k_g_scale(int n, const double *__restrict__ w, double *__restrict__ vnext, const GmresState *G) {
    if (G->s.flag) return;
    const double inv = 1.0 / G->hn;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) vnext[i] = w[i] * inv;
}
// y = R^-1 g over the columns built (one thread), then x += V y
__global__ void k_g_solve(GmresState *G, int m) {
    const int jend = G->run_over ? 0 : G->j;
    for (int i = jend - 1; i >= 0; --i) {
        double s = G->g[i];
        for (int k = i + 1; k < jend; ++k) s -= G->H[(size_t)k * (m + 1) + i] * G->y[k];
        const double d = G->H[(size_t)i * (m + 1) + i];
        G->y[i] = d == 0.0 ? 0.0 : s / d;
    }
    G->jend = jend;
}
__global__ void k_g_update_x(int n, const double *__restrict__ V, int ldv, double *__restrict__ x, const GmresState *G) {
    const int jend = G->jend;
    if (jend == 0) return;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        double s = x[i];
        for (int c = 0; c < jend; ++c) s += V[(size_t)c * ldv + i] * G->y[c];
        x[i] = s;
    }
}

}  // namespace

int gmres_blocks(int64_t n) { return vec_blocks(n); }

void launch_g_diff(int64_t n, const double *x, const double *x0, double *d, cudaStream_t st) {
    k_g_diff<<<vec_blocks(n), kT, 0, st>>>((int)n, x, x0, d);
}

void launch_g_residual(int64_t n, int mode, const double *b, const double *y, double *r, GmresState *G, double tol,
                       double inner_tol, cudaStream_t st) {
    k_g_residual<<<vec_blocks(n), kT, 0, st>>>((int)n, mode, b, y, r, G, tol, inner_tol);
}
void launch_g_start_cycle(int64_t n, const double *r, double *v0, GmresState *G, int m, int maxit, cudaStream_t st) {
    k_g_start_cycle<<<1, 1, 0, st>>>(G, m, maxit);
    k_g_scale0<<<vec_blocks(n), kT, 0, st>>>((int)n, r, v0, G);
}
void launch_g_arnoldi(int64_t n, const double *V, int ldv, double *w, GmresState *G, int jj, int m, int maxit,
                      double *part, cudaStream_t st) {
    const int nb = vec_blocks(n);
    for (int pass = 0; pass < 2; ++pass) {
        k_g_dots<<<dim3(nb, jj + 1), kT, 0, st>>>((int)n, V, ldv, w, G, jj, part);
        k_g_dots_fin<<<jj + 1, kT, 0, st>>>(nb, part, G, pass);
        k_g_orth<<<nb, kT, 0, st>>>((int)n, V, ldv, w, G, jj);
    }
    k_g_rotate<<<nb, kT, 0, st>>>((int)n, w, G, jj, m, maxit);
    k_g_scale<<<nb, kT, 0, st>>>((int)n, w, const_cast<double *>(V) + (size_t)(jj + 1) * ldv, G);
}
void launch_g_finish_cycle(int64_t n, const double *V, int ldv, double *x, GmresState *G, int m, cudaStream_t st) {
    k_g_solve<<<1, 1, 0, st>>>(G, m);
    k_g_update_x<<<vec_blocks(n), kT, 0, st>>>((int)n, V, ldv, x, G);
}

}  // namespace hmat_internal
