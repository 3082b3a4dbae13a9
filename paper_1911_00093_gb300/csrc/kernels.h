// Launch wrappers of the device kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hmat_internal {

// One launch of the projection over items [begin, begin + count) of its work
// list with CTAs of nt threads (64, 128 or 256).
struct P1Plan {
    int32_t begin = 0, count = 0, nt = 0;
};
constexpr int kP1MaxRuns = 8;

// Device-resident packing indices (shared by every precision copy of a handle).
struct DevIndex {
    int32_t n = 0, nleaves = 0, nlr = 0, nbig = 0, ntasks = 0;
    const int32_t *perm = nullptr;  // [n]
    const P1Desc *p1 = nullptr;     // [nleaves]
    const int32_t *tofs = nullptr;  // LrDesc::boff: T offsets of each block's per-cluster projections
    const XDst *xdst = nullptr;
    const int32_t *xsel = nullptr;  // local indices of the column-subset operand slices
    const LrDesc *lr = nullptr;     // [nlr]
    const int32_t *gdst = nullptr;
    const int32_t *red_big = nullptr, *red_tasks = nullptr;
    const RedDirect *red_direct = nullptr;  // [ndirect]
    int32_t ndirect = 0;
    const P2Desc *p2 = nullptr;     // [nleaves]
    const double *tscale = nullptr; // per-rank factors of LrDesc::toff (paper's Methods 2 and 3)
    const GroupDesc *groups = nullptr;  // row groups of the row-group expansion
    int32_t ngroups = 0;
    int32_t nsm = 1;                // SMs of the device (row-group grid = nsm x kP2gBlocks)
    // projection plan (hmat_autotune): nruns == 0 is one launch over p1 in cluster
    // order at the store's default CTA size; else the runs over p1_sorted (the
    // clusters sorted by panel width) or p1
    const P1Desc *p1_sorted = nullptr;
    int32_t nruns = 0;
    P1Plan runs[kP1MaxRuns];
    int32_t max_leaf = 0;           // rows of the widest leaf cluster
    int32_t max_ld2 = 0;            // widest phase-2 panel (entries)
};

struct SolverScalars;
struct SysScalars;

// Programmatic dependent launch (sm_90 and later).  The product kernels (operand
// copy, projection, reduction, expansion) are launched with programmatic stream
// serialization: the CTAs of a kernel may be scheduled while its predecessor in
// the stream drains, once every CTA of the predecessor has started (pdl_trigger,
// at the top of each such kernel).  Before pdl_wait() a kernel reads only
// immutable data (index arrays, panels) and writes nothing; pdl_wait()
// (griddepcontrol.wait) returns once every preceding kernel of the stream has
// completed and its memory operations are visible.  Every such kernel executes
// pdl_wait() before it exits, on every path, so completion stays transitive
// along the stream.  Measured at level 6: the BF16 product through hmat_matvec
// 85.1 -> 77.5 us, FP64 231.7 -> 223.8 us; the solver's vector kernels launched
// the same way made the BF16 solve slower (8.4 -> 9.1 ms), so they are not.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kern, args...);  // a failed launch is reported by cudaGetLastError
}
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// One precision copy of the panels plus its work buffers.
struct DevPanels {
    Store store = Store::DF;
    const void *q1 = nullptr;  // phase-1 panels
    const void *p2 = nullptr;  // phase-2 panels
    void *xs = nullptr;        // source-vector operand, cluster order (n entries of the operand type)
    void *part = nullptr;      // T: every leaf column cluster's projections t_{m,kappa}, panel column order
    void *g = nullptr;         // phase-2 operand buffers (glen entries of the operand type)
};

// The expansion runs as persistent warps over groups of up to four rows of one
// leaf row cluster (k_phase2g), kP2gBlocks CTAs per SM, each lane with two
// vectors of each row in flight.  Measured at L6 against the launch shapes it
// replaced (BF16 expansion): 51.0 us for row groups, 57.7 for row-persistent
// warps, 61.7 for one CTA per leaf row cluster, 100.5 for a bulk-copy pipeline
// through shared memory; two vectors in flight at 3 CTAs per SM against one at
// 4: FP64 pairs 117.0 against 124.2 us, FP32 60.5 against 63.5, BF16 38.9
// against 39.2.
constexpr int kP2gBlocks = 3;
// Work items (CTAs) of the expansion; a solver expansion leaves one pair of
// inner-product shares per item in dpart.
inline int phase2_items(const DevIndex &ix) { return ix.nsm * kP2gBlocks; }

// Operand bytes per entry for a store (x and t copies).
inline size_t operand_bytes(Store s) { return s == Store::F32 || s == Store::BF16 ? 4 : 8; }
inline size_t partial_bytes(Store s) { return s == Store::F32 || s == Store::BF16 ? 4 : 8; }
inline bool table1_store(Store s) { return s == Store::PM || s == Store::PS || s == Store::PM1 || s == Store::PS2; }

// Mean microseconds of the projection (every run of ix's plan) over reps
// launches, CUDA events on st (the autotuner's measurement).
float time_phase1(Store s, const DevIndex &ix, const DevPanels &P, int reps, cudaStream_t st);
// default CTA size of a store's projection
int phase1_default_threads(Store s);

// Source-vector operand from an FP64 vector: src_perm != nullptr gathers
// x[src_perm[p]] (original order in), otherwise x is already in cluster order.
void launch_prep(Store s, const DevIndex &ix, const double *x, const int32_t *src_perm, void *xs,
                 cudaStream_t st);
struct SolverScalars;
// skipS/mode: a solver's product is skipped once its run has stopped (mode 1:
// flag set; mode 2: flag set or stop at the ||s|| check); mode 0 never skips.
// sys != nullptr (many-system solver): the work items of a problem whose system
// sys[problem] has stopped are skipped (the problem index of an item is in the
// pad fields of its descriptor)
void launch_phase1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st, const SysScalars *sys = nullptr);
// t of the blocks spanning several leaf clusters, scattered into g (no launch when there is none)
void launch_reduce(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st, const SysScalars *sys = nullptr);
// y[p] (cluster order) or y[out_perm[p]] (original order) = (A~ x)_p, or
// y[.] += (A~ x)_p when accum is set (the second segment of a paper variant);
// dotmode 1/2 also leaves, per work item k, w . y in dpart[k] and y . y in
// dpart[items + k] (items = phase2_items; w = r~ for alpha, w = s for omega of
// Algorithm 1)
void launch_phase2(Store s, const DevIndex &ix, const DevPanels &P, double *y, const int32_t *out_perm, int accum,
                   const SolverScalars *skipS, int mode, cudaStream_t st, const double *w = nullptr,
                   int dotmode = 0, double *dpart = nullptr, const SysScalars *sys = nullptr);
// the same for the paper's stores (kernels_table1.cu)
void launch_phase1_table1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                          cudaStream_t st, const SysScalars *sys);
void launch_reduce_table1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                          cudaStream_t st, const SysScalars *sys);
void launch_phase2_table1(Store s, const DevIndex &ix, const DevPanels &P, double *y, const int32_t *out_perm,
                          int accum, const SolverScalars *skipS, int mode, cudaStream_t st, const double *w,
                          int dotmode, double *dpart, const SysScalars *sys);

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
    int32_t loops;        // batches of iterations the device loop of a run has replayed
    int32_t run_flag;     // the flag of the run a true residual follows (kept by that residual)
    double run_rnorm2;    // its ||r||^2 at the end of the run
};

constexpr int kVecThreads = 256;
int vec_blocks(int64_t n);
// The end of one batch of iterations inside a run's device loop (a conditional
// WHILE graph node): counts the batch and keeps looping while the run goes on
// and fewer than max_loops batches have run.
void launch_loop_condition(SolverScalars *S, cudaGraphConditionalHandle cond, int max_loops, cudaStream_t st);

// ---- restarted GMRES(m) (gmres.cu) ----
constexpr int kGmresMaxM = 64;
struct GmresState {
    SolverScalars s;  // s.flag: the current cycle has ended (its remaining products skip); s.nmv: Arnoldi steps
    double bnorm2, rnorm, stop, hn, resid, relres_true;
    int32_t j, jend, it, status, run_over, nmv64;
    unsigned int ticket;
    int32_t pad;
    double *partials;  // grid-reduction scratch (vec_blocks entries)
    double H[(kGmresMaxM + 1) * kGmresMaxM], cs[kGmresMaxM], sn[kGmresMaxM], g[kGmresMaxM + 1], y[kGmresMaxM];
    double h[kGmresMaxM + 1], hp[kGmresMaxM + 1];
};
// mode 2: ||b||; 3: true residual r = b - y, which starts the next run; 1: r = b - y
// between cycles (b = the run's r_0, y = A~ (x - x_0))
void launch_g_diff(int64_t n, const double *x, const double *x0, double *d, cudaStream_t st);
void launch_g_residual(int64_t n, int mode, const double *b, const double *y, double *r, GmresState *G, double tol,
                       double inner_tol, cudaStream_t st);
// a cycle starts from r (or the run ends): v_0 = r / ||r||
void launch_g_start_cycle(int64_t n, const double *r, double *v0, GmresState *G, int m, int maxit, cudaStream_t st);
// step jj after w = A v_jj: CGS2 against v_0..v_jj, column jj of H, rotations, v_{jj+1}
void launch_g_arnoldi(int64_t n, const double *V, int ldv, double *w, GmresState *G, int jj, int m, int maxit,
                      double *part, cudaStream_t st);
// y = R^-1 g, x += V y
void launch_g_finish_cycle(int64_t n, const double *V, int ldv, double *x, GmresState *G, int m, cudaStream_t st);

// ---- product for many right-hand sides on the tensor cores (mrhs.cu, BF16 panels) ----
// Bounded device waits: a wait that runs out writes HMAT_ERR_TIMEOUT to *status
// (mapped host memory of the handle) and the kernel gives up its work.
struct PipeCtl {
    int32_t *status = nullptr;
    long long wait_limit = 0;  // SM clock cycles per wait
    int32_t withhold = 0;      // tests: the projection issues no copies, so its waits run out
    int32_t pad = 0;
};
constexpr long long kDefaultWaitCycles = 2000000000ll;  // about one second at the SM clock
constexpr int kMrhsCols = 64;  // right-hand sides per pass
struct MrhsSrc {
    int32_t row;  // row of U feeding this operand slot (x row, t row, or the zero row)
    int32_t exp;  // power of two of the stored array the slot multiplies
};
// One column cluster sigma of the projection: the rank rows of every low-rank
// block whose column cluster is sigma, stacked (R rows), times x_sigma.
struct MrhsSig {
    int64_t woff;   // first element of its W tile (K-major core matrices, kpad x npad; TF32: two per chunk)
    int32_t xbeg;   // first source row (cluster order)
    int32_t xlen;   // |sigma|
    int32_t kpad;   // xlen rounded up to 16
    int32_t npad;   // R rounded up to 16
    int32_t R;      // rank rows
    int32_t tbeg;   // first t row (within T) of its rank rows
};
struct MrhsIndex {
    const MrhsSrc *src = nullptr;    // [glen]
    const MrhsSig *sigs = nullptr;   // [nsig]
    const void *wt = nullptr;        // W tiles of the column clusters (BF16, or TF32 high/low pairs)
    int32_t nsig = 0, max_npad = 16;
    bool tf32 = false;               // FP32 panels: kind::tf32 MMAs on TF32 high/low parts
    int64_t urows = 0;               // rows of U (n + ranks + 1)
    float *U = nullptr;              // [urows][64]: x rows, then t rows, then a zero row
    PipeCtl ctl;
};
constexpr int kMrhsMaxRows = 128;  // rank rows of one projection item (tensor-memory columns)
// raise the shared-memory limits of the two kernels (once per device, at upload)
cudaError_t mrhs_prepare();
// y(:, k) = A~ x(:, k), k < nrhs <= 64, cluster order, columns ldx / ldy apart
void launch_mrhs_product(const DevIndex &ix, const MrhsIndex &mx, const DevPanels &P, const double *x, int64_t ldx,
                         double *y, int64_t ldy, int nrhs, cudaStream_t st);

// ---- many systems at once (multi.cu) ----
struct SysDesc {
    int64_t off;  // first entry of the system in the stacked vectors (cluster order)
    int32_t n;    // its length
    int32_t pad;
};
struct SysScalars {
    double rho, rho_prev, alpha, omega, snorm2, rnorm2, bnorm2, stop2, relres_true, relres_inner;
    int32_t flag;        // run: 0 running, 1 stopped (converged), >1 an hmat_status error
    int32_t state;       // 0 active, 1 accepted, 2 finished with the error in flag
    int32_t iters, iter_in_run, stop_on_s, restarts, nmv, nmv64;
    unsigned int ticket;
    int32_t pad;
};
struct MultiGrid {
    const SysDesc *sys = nullptr;
    SysScalars *S = nullptr;
    double *partials = nullptr;  // nsys x 2 x bx
    int bx = 1, nsys = 0;
};
struct MultiVecs {
    double *x, *r, *rt, *p, *v, *s, *t;
};
int multi_blocks_x(int64_t max_n, int nsys);
// mode 0: ||b||^2 and a state reset; 1: r = b - y and a run starts; 2: true
// residual r = b - y, acceptance at tol, error or restart (Section 4.1.3)
void launch_mresidual(const MultiGrid &g, int mode, const double *b, const double *y, double *x, double *r, double *rt,
                      double tol, double inner_tol, int iter_limit, int max_restarts, cudaStream_t st);
// the vector steps of one iteration: 0 p update, 1 alpha, 2 s update, 3 omega, 4 x/r update
void launch_miteration_vec(const MultiGrid &g, int step, const MultiVecs &v, int iter_limit, cudaStream_t st);
// column-wise permutation of an n x nrhs block: dst[k n + p] = src[k n + perm[p]] and back
void launch_mgather(int64_t n, int nrhs, const int32_t *perm, const double *src, double *dst, cudaStream_t st);
void launch_mscatter(int64_t n, int nrhs, const int32_t *perm, const double *src, double *dst, cudaStream_t st);

// iteration budget test and count; then p = r (first iteration of a run) or
// p = r + beta (p - omega v), with the operand copy of p
void launch_count_iter(SolverScalars *S, int iter_limit, cudaStream_t st);
void launch_update_p(Store s, int64_t n, const double *r, double *p, const double *v, void *ps,
                     SolverScalars *S, cudaStream_t st);
// alpha = rho / (r~ . v) from the expansion's shares (ndp work items); s = r -
// alpha v, operand copy of s, ||s||^2 and the stop check
void launch_update_s(Store s, int64_t n, const double *r, const double *v, double *svec, void *ss,
                     SolverScalars *S, double *partials, const double *dpart, int ndp, cudaStream_t st);
// omega = (t . s) / (t . t) from the expansion's shares; x += alpha p + omega s;
// r = s - omega t; rho = r~ . r, ||r||^2, stop check; counts the next iteration
// when the run goes on
void launch_update_xr(int64_t n, double *x, const double *p, const double *svec, const double *t, double *r,
                      const double *rt, SolverScalars *S, double *partials, const double *dpart, int ndp,
                      int iter_limit, cudaStream_t st);
// r = b - y; r~ = r; ||r||^2 into S->rnorm2 and rho = r~ . r; resets the run state;
// iter_limit >= 0 starts a run (counts its first iteration)
void launch_residual(int64_t n, const double *b, const double *y, double *r, double *rt, SolverScalars *S,
                     double *partials, int iter_limit, cudaStream_t st);
// gather / scatter between original and cluster order
void launch_gather(int64_t n, const int32_t *perm, const double *src, double *dst_perm, cudaStream_t st);
void launch_scatter(int64_t n, const int32_t *perm, const double *src_perm, double *dst, cudaStream_t st);

}  // namespace hmat_internal
