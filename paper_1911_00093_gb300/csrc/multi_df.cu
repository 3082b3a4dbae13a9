// The double-float H-matrix product of several columns at once: the FP64
// operator of a many-column hmat_matvec and of the many-system solver's true
// residuals (Section 4.1.3), on the FP64 panels stored as double-float pairs.
//
// The one-column kernels (product.cuh) stream every panel vector from HBM once
// per column and are bound by that stream.  Here each CTA (projection) or warp
// (expansion) applies the panel vectors it loads to NC columns at once, and the
// work items of the NC-column batches of one cluster or row group are adjacent,
// so the batches after the first find the panel in L1 or L2: the panels come
// from HBM about once per pass of kMdfCols columns, and the kernels are bound by
// the double-float arithmetic on the FP32 pipe instead.
//
// Per column, every sum is formed in the order of the one-column kernels:
// projection rows in order, renormalised after each 8 rows; the reduction's
// per-block order over its leaf clusters; each expansion lane's panel vectors
// in order, renormalised after each kFoldVecs vectors, and the same butterfly
// over the lanes.  So each column is bit for bit the one-column product.
#include "mdf.h"
#include "product.cuh"

namespace hmat_internal {

namespace {

constexpr int kMdfP1Cols = 4;       // columns of a projection CTA
constexpr int kMdfP1Threads = 128;
constexpr int kMdfP1Blocks = 6;     // resident CTAs per SM the registers are held to
constexpr int kMdfP2Cols = 4;       // columns of an expansion warp
constexpr int kMdfP2Threads = 256;
constexpr int kMdfP2Warps = kMdfP2Threads / 32;
constexpr int kMdfP2Blocks = 2;     // resident CTAs per SM (persistent grid)
static_assert(kMdfCols % kMdfP1Cols == 0 && kMdfCols % kMdfP2Cols == 0,
              "a pass's column batches stay inside the buffers");

struct MdfArgs {
    const double *x;          // column 0 of x and y
    double *y;
    float2 *xs, *part, *g;    // the pass's buffers (column c of the pass at c * ld..)
    int64_t ldx, ldy, ldxs, ldt, ldg;
    int ncols;                // columns of this pass (<= kMdfCols)
    int cbase;                // column c of the pass is column cbase + c of x and y ...
    const int32_t *cols;      // ... or cols[c] when the pass runs over a list
    const SysScalars *sys;    // system (problem 0, column 0), or null
    int sysmode, nprob;
};

// the x / y column (and system column) of the pass's column c
__device__ __forceinline__ int col_of(const MdfArgs &a, int c) { return a.cols ? __ldg(a.cols + c) : a.cbase + c; }

// the column's system does not need this product (see launch_mdf_product)
__device__ __forceinline__ bool col_idle(const MdfArgs &a, int c, int prob) {
    if (a.sys == nullptr || a.sysmode == 0) return false;
    const SysScalars &q = a.sys[(size_t)col_of(a, c) * a.nprob + prob];
    return a.sysmode == 1 ? (q.state != 0 || q.flag != 0) : (q.state != 0 || q.flag == 0);
}

// bit c: column c0 + c is in the pass and its system needs the product
template <int NC>
__device__ __forceinline__ unsigned col_mask(const MdfArgs &a, int c0, int prob) {
    unsigned m = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c)
        if (c0 + c < a.ncols && !col_idle(a, c0 + c, prob)) m |= 1u << c;
    return m;
}

__device__ __forceinline__ int4 ld_panel(const char *p) { return __ldg(reinterpret_cast<const int4 *>(p)); }

// operand copies: every column's x split into double-float pairs
__global__ void k_mdf_prep(MdfArgs a, int n) {
    const int c = blockIdx.y;
    const double *x = a.x + (size_t)col_of(a, c) * a.ldx;
    float2 *xs = a.xs + (size_t)c * a.ldxs;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) xs[p] = split_double(x[p]);
}

// phase 1: CTA (leaf column cluster kappa, batch of NC columns) -> T_kappa of
// the batch's columns and their dense-block operand slices (eq. 9/22, 21)
template <int NC>
__global__ void __launch_bounds__(kMdfP1Threads, kMdfP1Blocks) k_mdf_phase1(MdfArgs a, const P1Desc *__restrict__ desc,
                                                                 const XDst *__restrict__ xdst,
                                                                 const int32_t *__restrict__ xsel,
                                                                 const void *__restrict__ q1) {
    constexpr int NT = kMdfP1Threads;
    __shared__ float2 xk[kMaxLeaf * NC];  // x_kappa of the batch's columns, [row][column]
    const int ncb = (a.ncols + NC - 1) / NC;
    const int item = blockIdx.x / ncb, c0 = (blockIdx.x - item * ncb) * NC;
    const P1Desc d = desc[item];
    const unsigned mask = col_mask<NC>(a, c0, d.pad[0]);  // (pad[0]: the item's problem)
    if (mask == 0) return;
    const int xlen = d.xlen;
    for (int t = threadIdx.x; t < xlen * NC; t += NT) {
        const int j = t / NC, c = t - j * NC;
        xk[t] = (mask >> c) & 1u ? a.xs[(size_t)(c0 + c) * a.ldxs + d.xbeg + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int nvec = d.ld / 2;
    const char *base = (const char *)q1 + (size_t)d.off * 8;
    const size_t row_bytes = (size_t)d.ld * 8;
    for (int vc = threadIdx.x; vc < nvec; vc += NT) {
        DF acc[NC][2];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c][0] = acc[c][1] = DF{0.f, 0.f};
        const char *col = base + (size_t)vc * 16;
        auto mac = [&](int4 raw, int j) {
            const float4 v = *reinterpret_cast<float4 *>(&raw);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float2 x = xk[j * NC + c];
                df_fma(acc[c][0], v.x, v.y, x.x, x.y);
                df_fma(acc[c][1], v.z, v.w, x.x, x.y);
            }
        };
        int j = 0;
        for (; j + 8 <= xlen; j += 8) {
            int4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = ld_panel(col + (size_t)(j + u) * row_bytes);
#pragma unroll
            for (int u = 0; u < 8; ++u) mac(raw[u], j + u);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                renorm(acc[c][0]);
                renorm(acc[c][1]);
            }
        }
        if (j < xlen) {  // the last rows, no renormalisation before the output's
            const int rem = xlen - j;
            int4 raw[7];
#pragma unroll
            for (int u = 0; u < 7; ++u)
                raw[u] = u < rem ? ld_panel(col + (size_t)(j + u) * row_bytes) : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 7; ++u) {
                if (u >= rem) break;
                mac(raw[u], j + u);
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (!((mask >> c) & 1u)) continue;
            renorm(acc[c][0]);
            renorm(acc[c][1]);
            *reinterpret_cast<float4 *>(a.part + (size_t)(c0 + c) * a.ldt + d.tbeg + (size_t)vc * 2) =
                make_float4(acc[c][0].s, acc[c][0].c, acc[c][1].s, acc[c][1].c);
        }
    }
    // the dense-block operands fed by x_kappa, scaled by 2^e
    const int xdcnt = d.xdcnt;
    for (int t = threadIdx.x; t < xdcnt * xlen; t += NT) {
        const int k = t / xlen, j = t - k * xlen;
        const XDst xd = xdst[d.xdbeg + k];
        if (j >= xd.cnt) continue;
        const int src = xd.sel < 0 ? j : __ldg(xsel + xd.sel + j);
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if ((mask >> c) & 1u)
                a.g[(size_t)(c0 + c) * a.ldg + xd.goff + j] = scale_op<Store::DF>(xk[src * NC + c], xd.scale);
    }
}

// reduce: CTA row blockIdx.y = one column; the one-column reduction's work
// split and order (k_reduce)
__global__ void __launch_bounds__(kRedThreads) k_mdf_reduce(MdfArgs a, int nbig, int ntasks, int ndirect,
                                                            const int32_t *__restrict__ big,
                                                            const int32_t *__restrict__ tasks,
                                                            const RedDirect *__restrict__ direct,
                                                            const LrDesc *__restrict__ lr,
                                                            const int32_t *__restrict__ gdst,
                                                            const int32_t *__restrict__ tofs,
                                                            const double *__restrict__ tscale) {
    using RT = typename RedT<Store::DF>::T;
    __shared__ RT red[kRedThreads];
    const int c = blockIdx.y;
    const float2 *part = a.part + (size_t)c * a.ldt;
    float2 *g = a.g + (size_t)c * a.ldg;
    if ((int)blockIdx.x < nbig) {
        const LrDesc ld = lr[big[blockIdx.x]];
        if (col_idle(a, c, ld.pad)) return;  // (pad: the block's problem; CTA-uniform)
        const int32_t *to = tofs + ld.boff;
        const int32_t *gd = gdst + ld.gbeg;
        for (int l0 = 0; l0 < ld.rank; l0 += 32) {
            const int rr = min(32, ld.rank - l0);
            int rp = 1;
            while (rp < rr) rp <<= 1;
            const int G = kRedThreads / rp, gi = threadIdx.x / rp, l = threadIdx.x % rp;
            RT acc;
            red_zero<Store::DF>(acc);
            if (l < rr) {
                const float2 *src = part + l0 + l;
                for (int k = gi; k < ld.cnt; k += G) red_add_part<Store::DF>(acc, src[__ldg(to + k)]);
            }
            red[threadIdx.x] = acc;
            __syncthreads();
            for (int half = G >> 1; half >= 1; half >>= 1) {
                if (gi < half) {
                    RT s = red[threadIdx.x];
                    red_add<Store::DF>(s, red[threadIdx.x + half * rp]);
                    red[threadIdx.x] = s;
                }
                __syncthreads();
            }
            for (int idx = threadIdx.x; idx < ld.gcnt * rr; idx += kRedThreads) {
                const int k = idx / rr, ll = idx - k * rr;
                g[__ldg(gd + k) + l0 + ll] = part_to_op<Store::DF>(red_to_part<Store::DF>(red[ll]), ld.scale);
            }
            __syncthreads();
        }
        return;
    }
    const int task_blocks = (ntasks + kRedThreads - 1) / kRedThreads;
    if ((int)blockIdx.x >= nbig + task_blocks) {  // a rank of a single-leaf block: t_m = 2^e T entry
        const int i = ((int)blockIdx.x - nbig - task_blocks) * kRedThreads + threadIdx.x;
        if (i >= ndirect) return;
        const int4 r = __ldg(reinterpret_cast<const int4 *>(direct) + i);  // (tsrc, gdst, scale, prob)
        if (col_idle(a, c, r.w)) return;
        g[r.y] = part_to_op<Store::DF>(part[r.x], r.z);
        return;
    }
    const int task = ((int)blockIdx.x - nbig) * kRedThreads + threadIdx.x;
    if (task >= ntasks) return;
    const int tq = __ldg(tasks + task);
    const LrDesc ld = lr[tq >> 6];
    if (col_idle(a, c, ld.pad)) return;
    reduce_task<Store::DF>(tq & 63, ld, gdst, tofs, part, g, tscale, nullptr);
}

// phase 2: persistent warps over (row group, batch of NC columns) items, the
// batches of one group adjacent (they share the group's panel rows in L1)
template <int NC>
__global__ void __launch_bounds__(kMdfP2Threads, kMdfP2Blocks) k_mdf_phase2(MdfArgs a, int ng,
                                                                           const GroupDesc *__restrict__ groups,
                                                                           const void *__restrict__ p2) {
    constexpr int GR = kGroupRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncb = (a.ncols + NC - 1) / NC;
    const int64_t nitems = (int64_t)ng * ncb;
    const int64_t W = (int64_t)gridDim.x * kMdfP2Warps;
    for (int64_t t = (int64_t)blockIdx.x * kMdfP2Warps + warp; t < nitems; t += W) {
        const int gi = (int)(t / ncb), c0 = (int)(t - (int64_t)gi * ncb) * NC;
        const GroupDesc cur = groups[gi];
        const unsigned mask = col_mask<NC>(a, c0, cur.pad[0]);  // (pad[0]: the group's problem)
        if (mask == 0) continue;                                // warp-uniform
        const char *base = (const char *)p2 + (size_t)cur.off * 8;
        const size_t row_bytes = (size_t)cur.ld * 8;
        const int nv = cur.ld / 2, nr = cur.nr;
        const float2 *gc = a.g + cur.goff;
        Acc<Store::DF> acc[NC][GR];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int r = 0; r < GR; ++r) acc[c][r].init();
        int nf = 0;  // vectors since the rows' last renormalisation
        for (int v = lane; v < nv; v += 32) {
            int4 raw[GR];
#pragma unroll
            for (int r = 0; r < GR; ++r)
                raw[r] = r < nr ? ld_panel(base + (size_t)r * row_bytes + (size_t)v * 16) : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float4 gv = __ldg(reinterpret_cast<const float4 *>(gc + (size_t)(c0 + c) * a.ldg + v * 2));
#pragma unroll
                for (int r = 0; r < GR; ++r) {
                    if (r >= nr) continue;
                    const float4 w = *reinterpret_cast<const float4 *>(&raw[r]);
                    df_fma(acc[c][r].a, w.x, w.y, gv.x, gv.y);
                    df_fma(acc[c][r].a, w.z, w.w, gv.z, gv.w);
                }
            }
            if (++nf == kFoldVecs) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int r = 0; r < GR; ++r) renorm(acc[c][r].a);
                nf = 0;
            }
        }
        const bool own = (lane & 7) == 0 && (lane >> 3) < nr;
        const int p = cur.p0 + (lane >> 3);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double tot = group_totals<Store::DF>(acc[c], lane);  // lanes 8r..8r+7: row r
            if (own && ((mask >> c) & 1u)) a.y[(size_t)col_of(a, c0 + c) * a.ldy + p] = tot;
        }
    }
}

}  // namespace

int mdf_launches(const DevIndex &ix, int ncols) {
    const int passes = (ncols + kMdfCols - 1) / kMdfCols;
    return passes * ((ix.nbig + ix.ntasks + ix.ndirect) ? 4 : 3);
}

void launch_mdf_product(const DevIndex &ix, const DevPanels &P, const MdfBufs &b, const double *x, int64_t ldx,
                        double *y, int64_t ldy, int ncols, const int32_t *cols, const SysScalars *sys, int sysmode,
                        int nprob, cudaStream_t st) {
    for (int k0 = 0; k0 < ncols; k0 += kMdfCols) {
        MdfArgs a;
        a.x = x;
        a.y = y;
        a.xs = (float2 *)b.xs;
        a.part = (float2 *)b.part;
        a.g = (float2 *)b.g;
        a.ldx = ldx;
        a.ldy = ldy;
        a.ldxs = b.ldxs;
        a.ldt = b.ldt;
        a.ldg = b.ldg;
        a.ncols = std::min(kMdfCols, ncols - k0);
        a.cbase = k0;
        a.cols = cols ? cols + k0 : nullptr;
        a.sys = sys;
        a.sysmode = sys ? sysmode : 0;
        a.nprob = nprob;
        const int prep_x = grid_for(ix.n, 256, 4 * ix.nsm);
        k_mdf_prep<<<dim3(prep_x, a.ncols), 256, 0, st>>>(a, ix.n);
        const int ncb1 = (a.ncols + kMdfP1Cols - 1) / kMdfP1Cols;
        k_mdf_phase1<kMdfP1Cols><<<(unsigned)ix.nleaves * ncb1, kMdfP1Threads, 0, st>>>(a, ix.p1, ix.xdst, ix.xsel,
                                                                                     P.q1);
        const int rblocks = ix.nbig + (ix.ntasks + kRedThreads - 1) / kRedThreads +
                            (ix.ndirect + kRedThreads - 1) / kRedThreads;
        if (rblocks > 0)
            k_mdf_reduce<<<dim3(rblocks, a.ncols), kRedThreads, 0, st>>>(a, ix.nbig, ix.ntasks, ix.ndirect, ix.red_big,
                                                                         ix.red_tasks, ix.red_direct, ix.lr, ix.gdst,
                                                                         ix.tofs,
                                                                         ix.tscale);
        k_mdf_phase2<kMdfP2Cols><<<ix.nsm * kMdfP2Blocks, kMdfP2Threads, 0, st>>>(a, ix.ngroups, ix.groups, P.p2);
    }
}

}  // namespace hmat_internal
