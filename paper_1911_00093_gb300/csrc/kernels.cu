// Device kernels of the H-matrix vector product and of BiCG-STAB (sm_103a).
//
// Product (Section 2.1, eq. 5-10 and 21-25), in three launches:
//   phase 1  one CTA per leaf column cluster kappa: t-partials = Q_kappa^T x_kappa,
//            Q_kappa the rows of every W_m^T (eq. 9/22) whose column cluster
//            contains kappa, row-major; each thread owns one 16-byte column vector
//            and walks the |kappa| rows (coalesced 128-bit loads, x from shared
//            memory, no cross-thread reduction);
//   reduce   one warp per low-rank block: t = 2^e sum_kappa partials, in a fixed
//            order (deterministic, no atomics on values);
//   phase 2  one CTA per leaf row cluster rho: y_rho = P_rho g_rho with P_rho the
//            rows of the dense blocks (eq. 21) and of the V_m (eq. 10/24) over rho,
//            g_rho the matching pieces of x and t staged in shared memory; one warp
//            per row; each row of y is written once by its owner (eq. 25 without
//            atomics).
// Arithmetic per store:
//   DF    panels are pairs (hi, lo); products and sums in double-float on the
//         FP32 pipe (the FP64 pipe of GB300 is ~1/60 of FP32);
//   F64   IEEE FP64 FMA;
//   F32, BF16  FP32 FMA over chunks of 8 products, chunks summed in double-float.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "hmat.h"
#include "kernels.h"

namespace hmat_internal {

namespace {

// ------------------------------------------------------------------------
// double-float helpers (error-free transformations; intrinsics keep the
// compiler from contracting or reassociating them)
// ------------------------------------------------------------------------
struct DF {
    float s, c;  // value s + c
};

__device__ __forceinline__ void two_sum_acc(DF &a, float p) {
    float t = __fadd_rn(a.s, p);
    float bb = __fsub_rn(t, a.s);
    float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    a.s = t;
    a.c = __fadd_rn(a.c, err);
}

__device__ __forceinline__ void renorm(DF &a) {
    float t = __fadd_rn(a.s, a.c);
    a.c = __fsub_rn(a.c, __fsub_rn(t, a.s));
    a.s = t;
}

// a += (ah + al) * (xh + xl), the lo*lo term (~2^-48) dropped
__device__ __forceinline__ void df_fma(DF &a, float ah, float al, float xh, float xl) {
    float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);  // exact error of the product
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    float t = __fadd_rn(a.s, p);
    float bb = __fsub_rn(t, a.s);
    float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    a.s = t;
    a.c = __fadd_rn(a.c, __fadd_rn(err, e));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    float t = __fadd_rn(a.s, b.s);
    float bb = __fsub_rn(t, a.s);
    float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bb)), __fsub_rn(b.s, bb));
    float c = __fadd_rn(__fadd_rn(a.c, b.c), err);
    DF r;
    r.s = __fadd_rn(t, c);
    r.c = __fsub_rn(c, __fsub_rn(r.s, t));
    return r;
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.s + (double)a.c; }

__device__ __forceinline__ int4 ld_stream(const void *p) { return __ldcs((const int4 *)p); }

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ float2 split_double(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return make_float2(hi, lo);
}

// ------------------------------------------------------------------------
// store traits
// ------------------------------------------------------------------------
// VW = entries per 16-byte vector; Op = operand type of x and t entries.
template <Store S> struct Tr;
template <> struct Tr<Store::DF> { static constexpr int VW = 2; using Op = float2; using Part = float2; };
template <> struct Tr<Store::F64> { static constexpr int VW = 2; using Op = double; using Part = double; };
template <> struct Tr<Store::F32> { static constexpr int VW = 4; using Op = float; using Part = float; };
template <> struct Tr<Store::BF16> { static constexpr int VW = 8; using Op = float; using Part = float; };

// per-column / per-row accumulator
template <Store S> struct Acc;
template <> struct Acc<Store::DF> {
    DF a;
    int n;
    __device__ void init() { a.s = 0.f; a.c = 0.f; n = 0; }
};
template <> struct Acc<Store::F64> {
    double a;
    __device__ void init() { a = 0.0; }
};
template <> struct Acc<Store::F32> {
    DF a;
    float ch;
    __device__ void init() { a.s = 0.f; a.c = 0.f; ch = 0.f; }
};
template <> struct Acc<Store::BF16> {
    DF a;
    float ch;
    int cnt;
    __device__ void init() { a.s = 0.f; a.c = 0.f; ch = 0.f; cnt = 0; }
};

// Multiply one 16-byte panel vector by VW operands and accumulate into VW
// separate accumulators (phase 1: one per column).
template <Store S> struct Cols;
template <> struct Cols<Store::DF> {
    __device__ static void mac(Acc<Store::DF> *acc, int4 raw, float2 x) {
        float4 v = *reinterpret_cast<float4 *>(&raw);
        df_fma(acc[0].a, v.x, v.y, x.x, x.y);
        df_fma(acc[1].a, v.z, v.w, x.x, x.y);
    }
};
template <> struct Cols<Store::F64> {
    __device__ static void mac(Acc<Store::F64> *acc, int4 raw, double x) {
        double2 v = *reinterpret_cast<double2 *>(&raw);
        acc[0].a = fma(v.x, x, acc[0].a);
        acc[1].a = fma(v.y, x, acc[1].a);
    }
};
template <> struct Cols<Store::F32> {
    __device__ static void mac(Acc<Store::F32> *acc, int4 raw, float x) {
        float4 v = *reinterpret_cast<float4 *>(&raw);
        acc[0].ch = fmaf(v.x, x, acc[0].ch);
        acc[1].ch = fmaf(v.y, x, acc[1].ch);
        acc[2].ch = fmaf(v.z, x, acc[2].ch);
        acc[3].ch = fmaf(v.w, x, acc[3].ch);
    }
};
template <> struct Cols<Store::BF16> {
    __device__ static void mac(Acc<Store::BF16> *acc, int4 raw, float x) {
        uint32_t w[4] = {(uint32_t)raw.x, (uint32_t)raw.y, (uint32_t)raw.z, (uint32_t)raw.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[2 * k].ch = fmaf(bf_lo(w[k]), x, acc[2 * k].ch);
            acc[2 * k + 1].ch = fmaf(bf_hi(w[k]), x, acc[2 * k + 1].ch);
        }
    }
};

// fold a chunk (F32/BF16) or renormalise (DF) -- called every 8 rows / products
template <Store S> __device__ __forceinline__ void fold(Acc<S> &a);
template <> __device__ __forceinline__ void fold<Store::DF>(Acc<Store::DF> &a) { renorm(a.a); }
template <> __device__ __forceinline__ void fold<Store::F64>(Acc<Store::F64> &) {}
template <> __device__ __forceinline__ void fold<Store::F32>(Acc<Store::F32> &a) { two_sum_acc(a.a, a.ch); a.ch = 0.f; }
template <> __device__ __forceinline__ void fold<Store::BF16>(Acc<Store::BF16> &a) { two_sum_acc(a.a, a.ch); a.ch = 0.f; }

// partial-sum output of a finished accumulator
template <Store S> __device__ __forceinline__ typename Tr<S>::Part to_part(Acc<S> &a);
template <> __device__ __forceinline__ float2 to_part<Store::DF>(Acc<Store::DF> &a) {
    renorm(a.a);
    return make_float2(a.a.s, a.a.c);
}
template <> __device__ __forceinline__ double to_part<Store::F64>(Acc<Store::F64> &a) { return a.a; }
template <> __device__ __forceinline__ float to_part<Store::F32>(Acc<Store::F32> &a) {
    fold<Store::F32>(a);
    return __fadd_rn(a.a.s, a.a.c);
}
template <> __device__ __forceinline__ float to_part<Store::BF16>(Acc<Store::BF16> &a) {
    fold<Store::BF16>(a);
    return __fadd_rn(a.a.s, a.a.c);
}

// skip test of the solver's products: mode 0 never, 1 on a set flag,
// 2 on a set flag or a stop at the ||s|| check
__device__ __forceinline__ bool skip_product(const SolverScalars *S, int mode) {
    if (mode == 0 || S == nullptr) return false;
    int f = *(volatile const int32_t *)&S->flag;
    if (f != 0) return true;
    return mode == 2 && *(volatile const int32_t *)&S->stop_on_s != 0;
}

// ------------------------------------------------------------------------
// source-vector operand
// ------------------------------------------------------------------------
template <Store S>
__global__ void k_prep(int n, const double *__restrict__ x, const int32_t *__restrict__ src_perm,
                       typename Tr<S>::Op *__restrict__ xs) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double v = x[src_perm ? src_perm[p] : p];
        if constexpr (S == Store::DF) xs[p] = split_double(v);
        else if constexpr (S == Store::F64) xs[p] = v;
        else xs[p] = __double2float_rn(v);
    }
}

// ------------------------------------------------------------------------
// exact power-of-two factors (|e| <= 120 is enforced at upload)
// ------------------------------------------------------------------------
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

template <Store S>
__device__ __forceinline__ typename Tr<S>::Op scale_op(typename Tr<S>::Op v, int e) {
    if constexpr (S == Store::DF) { const float f = pow2f(e); return make_float2(v.x * f, v.y * f); }
    else if constexpr (S == Store::F64) return v * pow2d(e);
    else return v * pow2f(e);
}

// operand from a finished projection (scaled by 2^e, exact)
template <Store S>
__device__ __forceinline__ typename Tr<S>::Op part_to_op(typename Tr<S>::Part p, int e) {
    if constexpr (S == Store::DF) { const float f = pow2f(e); return make_float2(p.x * f, p.y * f); }
    else if constexpr (S == Store::F64) return p * pow2d(e);
    else return p * pow2f(e);
}

// accumulator of the completing work item's fixed-order reduction
template <Store S> struct RedT { using T = DF; };
template <> struct RedT<Store::F64> { using T = double; };

template <Store S> __device__ __forceinline__ void red_zero(typename RedT<S>::T &a) {
    if constexpr (S == Store::F64) a = 0.0; else { a.s = 0.f; a.c = 0.f; }
}
template <Store S> __device__ __forceinline__ void red_add_part(typename RedT<S>::T &a, typename Tr<S>::Part p) {
    if constexpr (S == Store::F64) a += p;
    else if constexpr (S == Store::DF) a = df_add(a, DF{p.x, p.y});
    else two_sum_acc(a, p);
}
template <Store S> __device__ __forceinline__ void red_add(typename RedT<S>::T &a, typename RedT<S>::T b) {
    if constexpr (S == Store::F64) a += b; else a = df_add(a, b);
}
template <Store S>
__device__ __forceinline__ typename RedT<S>::T red_xor(typename RedT<S>::T a, int m, bool upper) {
    typename RedT<S>::T b;
    if constexpr (S == Store::F64) b = __shfl_xor_sync(0xffffffffu, a, m);
    else { b.s = __shfl_xor_sync(0xffffffffu, a.s, m); b.c = __shfl_xor_sync(0xffffffffu, a.c, m); }
    if (upper) { red_add<S>(b, a); return b; }
    red_add<S>(a, b);
    return a;
}

template <Store S> __device__ __forceinline__ typename Tr<S>::Part red_to_part(typename RedT<S>::T a) {
    if constexpr (S == Store::F64) return a;
    else if constexpr (S == Store::DF) { renorm(a); return make_float2(a.s, a.c); }
    else return __fadd_rn(a.s, a.c);
}

// ------------------------------------------------------------------------
// phase 1: per leaf column cluster kappa
// ------------------------------------------------------------------------
constexpr int kP1Threads = 256;

template <Store S>
__global__ void __launch_bounds__(kP1Threads) k_phase1(const P1Desc *__restrict__ desc, const P1Run *__restrict__ runs,
                                                        const XDst *__restrict__ xdst, const LrDesc *__restrict__ lr,
                                                        const int32_t *__restrict__ gdst, const void *__restrict__ q1,
                                                        const typename Tr<S>::Op *__restrict__ xs,
                                                        typename Tr<S>::Part *__restrict__ part,
                                                        typename Tr<S>::Op *__restrict__ g, const SolverScalars *S_,
                                                        int mode) {
    using Op = typename Tr<S>::Op;
    using Part = typename Tr<S>::Part;
    constexpr int VW = Tr<S>::VW;
    __shared__ Op xk[kMaxLeaf];  // x_kappa, broadcast to every thread
    if (skip_product(S_, mode)) return;
    const P1Desc d = desc[blockIdx.x];
    for (int j = threadIdx.x; j < d.xlen; j += blockDim.x) xk[j] = xs[d.xbeg + j];
    __syncthreads();

    // projections (eq. 9/22): thread = one 16-byte column vector, walk the rows
    const int nvec = d.ld / VW;
    const char *base = (const char *)q1 + (size_t)d.off * (16 / VW);
    const size_t row_bytes = (size_t)d.ld * (16 / VW);
    for (int vc = threadIdx.x; vc < nvec; vc += blockDim.x) {
        Acc<S> acc[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[e].init();
        const char *col = base + (size_t)vc * 16;
        int j = 0;
        for (; j + 8 <= d.xlen; j += 8) {
            int4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = ld_stream(col + (size_t)(j + u) * row_bytes);
#pragma unroll
            for (int u = 0; u < 8; ++u) Cols<S>::mac(acc, raw[u], xk[j + u]);
#pragma unroll
            for (int e = 0; e < VW; ++e) fold<S>(acc[e]);
        }
        for (; j < d.xlen; ++j) {
            int4 raw = ld_stream(col + (size_t)j * row_bytes);
            Cols<S>::mac(acc, raw, xk[j]);
        }
        const int c0 = vc * VW;
        if (c0 >= d.R) continue;
        const P1Run *rk = runs + d.rbeg;
        int lo = 0, hi = d.rcnt - 1;  // run holding column c0
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldg(&rk[mid].col0) <= c0) lo = mid;
            else hi = mid - 1;
        }
        P1Run rn = rk[lo];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            const int c = c0 + e;
            if (c < d.R) {
                while (c >= rn.col0 + rn.len) rn = rk[++lo];
                const int l = c - rn.col0;
                const Part pv = to_part<S>(acc[e]);
                if (rn.poff >= 0) {
                    part[rn.poff + l] = pv;
                } else {  // final: 2^e t to every leaf row cluster of the block
                    const LrDesc ld = lr[rn.q];
                    const Op o = part_to_op<S>(pv, ld.scale);
                    for (int k = 0; k < ld.gcnt; ++k) g[gdst[ld.gbeg + k] + l] = o;
                }
            }
        }
    }

    // the dense-block operands fed by x_kappa (eq. 21 inputs), scaled by 2^e
    for (int t = threadIdx.x; t < d.xdcnt * d.xlen; t += blockDim.x) {
        const int k = t / d.xlen, j = t - k * d.xlen;
        const XDst x = xdst[d.xdbeg + k];
        g[x.goff + j] = scale_op<S>(xk[j], x.scale);
    }
}

// ------------------------------------------------------------------------
// reduce: t of the blocks spanning several leaf clusters, in a fixed order,
// scattered to the operand buffers.  Blocks over >= kRedBigCnt clusters get a
// whole CTA (kernel blocks [0, nbig)); the others are split into one task per
// rank, one lane each.
// ------------------------------------------------------------------------
constexpr int kRedThreads = 256;

template <Store S>
__global__ void __launch_bounds__(kRedThreads) k_reduce(int nbig, int ntasks, const int32_t *__restrict__ big,
                                                         const int32_t *__restrict__ tasks,
                                                         const LrDesc *__restrict__ lr, const int32_t *__restrict__ gdst,
                                                         const typename Tr<S>::Part *__restrict__ part,
                                                         typename Tr<S>::Op *__restrict__ g, const SolverScalars *S_,
                                                         int mode) {
    using Op = typename Tr<S>::Op;
    using RT = typename RedT<S>::T;
    __shared__ RT red[kRedThreads];
    if (skip_product(S_, mode)) return;
    if ((int)blockIdx.x < nbig) {
        const LrDesc ld = lr[big[blockIdx.x]];
        for (int l0 = 0; l0 < ld.rank; l0 += 32) {
            const int rr = min(32, ld.rank - l0);
            int rp = 1;
            while (rp < rr) rp <<= 1;
            const int G = kRedThreads / rp, gi = threadIdx.x / rp, l = threadIdx.x % rp;
            RT a;
            red_zero<S>(a);
            if (l < rr) {
                const typename Tr<S>::Part *src = part + ld.boff + l0 + l;
#pragma unroll 4
                for (int k = gi; k < ld.cnt; k += G) red_add_part<S>(a, src[(size_t)k * ld.rank]);
            }
            red[threadIdx.x] = a;
            __syncthreads();
            for (int half = G >> 1; half >= 1; half >>= 1) {
                if (gi < half) {
                    RT c = red[threadIdx.x];
                    red_add<S>(c, red[threadIdx.x + half * rp]);
                    red[threadIdx.x] = c;
                }
                __syncthreads();
            }
            // every thread scatters: destination k, rank l
            for (int idx = threadIdx.x; idx < ld.gcnt * rr; idx += kRedThreads) {
                const int k = idx / rr, ll = idx - k * rr;
                g[gdst[ld.gbeg + k] + l0 + ll] = part_to_op<S>(red_to_part<S>(red[ll]), ld.scale);
            }
            __syncthreads();
        }
        return;
    }
    // the other blocks: one lane per (block, rank), a sequential sum over the
    // block's leaf clusters (independent loads) and the scatter of that rank
    const int task = ((int)blockIdx.x - nbig) * kRedThreads + threadIdx.x;
    if (task >= ntasks) return;
    const int tq = __ldg(tasks + task);
    const LrDesc ld = lr[tq >> 6];
    const int l = tq & 63;
    const typename Tr<S>::Part *src = part + ld.boff + l;
    RT a;
    red_zero<S>(a);
#pragma unroll 4
    for (int k = 0; k < ld.cnt; ++k) red_add_part<S>(a, src[(size_t)k * ld.rank]);
    const Op o = part_to_op<S>(red_to_part<S>(a), ld.scale);
    for (int k = 0; k < ld.gcnt; ++k) g[gdst[ld.gbeg + k] + l] = o;
}

// ------------------------------------------------------------------------
// phase 2: per leaf row cluster, y_rho = P_rho g_rho
// ------------------------------------------------------------------------
constexpr int kP2Threads = 256;
constexpr int kP2Warps = kP2Threads / 32;

// The VW operands matching one 16-byte panel vector, loaded as vectors through
// L1 (operand buffers are 16-byte aligned per row cluster).
template <Store S> struct GV;
template <> struct GV<Store::DF> {
    float4 v;  // (hi, lo) of two operands
    __device__ static GV load(const float2 *p) { GV r; r.v = __ldg(reinterpret_cast<const float4 *>(p)); return r; }
};
template <> struct GV<Store::F64> {
    double2 v;
    __device__ static GV load(const double *p) { GV r; r.v = __ldg(reinterpret_cast<const double2 *>(p)); return r; }
};
template <> struct GV<Store::F32> {
    float4 v;
    __device__ static GV load(const float *p) { GV r; r.v = __ldg(reinterpret_cast<const float4 *>(p)); return r; }
};
template <> struct GV<Store::BF16> {
    float4 a, b;
    __device__ static GV load(const float *p) {
        GV r;
        r.a = __ldg(reinterpret_cast<const float4 *>(p));
        r.b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        return r;
    }
};

// Multiply one 16-byte panel vector by its VW operands (one row).
template <Store S>
__device__ __forceinline__ void row_mac(Acc<S> &acc, int4 raw, const GV<S> &gv);
template <>
__device__ __forceinline__ void row_mac<Store::DF>(Acc<Store::DF> &acc, int4 raw, const GV<Store::DF> &gv) {
    float4 v = *reinterpret_cast<float4 *>(&raw);
    const float4 x = gv.v;
    df_fma(acc.a, v.x, v.y, x.x, x.y);
    df_fma(acc.a, v.z, v.w, x.z, x.w);
    if (++acc.n == 4) { renorm(acc.a); acc.n = 0; }
}
template <>
__device__ __forceinline__ void row_mac<Store::F64>(Acc<Store::F64> &acc, int4 raw, const GV<Store::F64> &gv) {
    double2 v = *reinterpret_cast<double2 *>(&raw);
    acc.a = fma(v.x, gv.v.x, acc.a);
    acc.a = fma(v.y, gv.v.y, acc.a);
}
template <>
__device__ __forceinline__ void row_mac<Store::F32>(Acc<Store::F32> &acc, int4 raw, const GV<Store::F32> &gv) {
    float4 v = *reinterpret_cast<float4 *>(&raw);
    const float4 x = gv.v;
    float c = 0.f;
    c = fmaf(v.x, x.x, c);
    c = fmaf(v.y, x.y, c);
    c = fmaf(v.z, x.z, c);
    c = fmaf(v.w, x.w, c);
    two_sum_acc(acc.a, c);  // one chunk of 4 products
}
template <>
__device__ __forceinline__ void row_mac<Store::BF16>(Acc<Store::BF16> &acc, int4 raw, const GV<Store::BF16> &gv) {
    const float4 x0 = gv.a, x1 = gv.b;
    float c = acc.ch;
    c = fmaf(bf_lo((uint32_t)raw.x), x0.x, c);
    c = fmaf(bf_hi((uint32_t)raw.x), x0.y, c);
    c = fmaf(bf_lo((uint32_t)raw.y), x0.z, c);
    c = fmaf(bf_hi((uint32_t)raw.y), x0.w, c);
    c = fmaf(bf_lo((uint32_t)raw.z), x1.x, c);
    c = fmaf(bf_hi((uint32_t)raw.z), x1.y, c);
    c = fmaf(bf_lo((uint32_t)raw.w), x1.z, c);
    c = fmaf(bf_hi((uint32_t)raw.w), x1.w, c);
    acc.ch = c;
    if (++acc.cnt == 4) { two_sum_acc(acc.a, acc.ch); acc.ch = 0.f; acc.cnt = 0; }  // chunk of 32
}

// the lane partial of one row as a reduction accumulator
template <Store S>
__device__ __forceinline__ typename RedT<S>::T row_partial(Acc<S> &a) {
    if constexpr (S == Store::F64) return a.a;
    else {
        if constexpr (S == Store::BF16) { two_sum_acc(a.a, a.ch); a.ch = 0.f; }
        renorm(a.a);
        return a.a;
    }
}

// BiCG-STAB scalars fused into the expansion of a solver product (Algorithm 1):
//   dotmode 1: alpha = rho / (r~ . v)          (w = r~, y = v)
//   dotmode 2: omega = (t . s) / (t . t)       (w = s,  y = t)
// Each work item adds its rows in a fixed order; the last one to finish (integer
// ticket, no waiting) adds the per-item sums in work-item order.
__device__ void fused_dots(const P2Desc &d, double out, const double *__restrict__ w, int dotmode, SolverScalars *Sd,
                           double *dpart) {
    __shared__ double dsm[2][kMaxLeaf];
    __shared__ double tot[2][kP2Threads];
    __shared__ bool am_last;
    const int t = threadIdx.x;
    if (t < kMaxLeaf) {
        const bool live = t < d.ylen;
        const double wv = live ? w[d.ybeg + t] : 0.0;
        dsm[0][t] = live ? wv * out : 0.0;
        dsm[1][t] = live ? out * out : 0.0;
    }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < d.ylen; ++i) { a += dsm[0][i]; b += dsm[1][i]; }
        dpart[blockIdx.x] = a;
        dpart[gridDim.x + blockIdx.x] = b;
        __threadfence();
        am_last = atomicAdd(&Sd->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int k = t; k < (int)gridDim.x; k += blockDim.x) {
        a += __ldcg(&dpart[k]);
        b += __ldcg(&dpart[gridDim.x + k]);
    }
    tot[0][t] = a;
    tot[1][t] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) { tot[0][t] += tot[0][t + s]; tot[1][t] += tot[1][t + s]; }
        __syncthreads();
    }
    if (t == 0) {
        const double wy = tot[0][0], yy = tot[1][0];
        if (dotmode == 1) {
            Sd->rtv = wy;
            Sd->alpha = Sd->rho / wy;
            if (!isfinite(Sd->alpha)) Sd->flag = HMAT_ERR_NONFINITE;
        } else {
            Sd->ts = wy;
            Sd->tt = yy;
            Sd->omega = yy == 0.0 ? 0.0 : wy / yy;
            if (!isfinite(Sd->omega)) Sd->flag = HMAT_ERR_NONFINITE;
        }
        Sd->ticket = 0u;
    }
}


// Row totals of a phase-2 work item: each warp adds its rows' lane partials with
// a fixed butterfly; lane 0 writes y.  Returns this thread's row value (rows in
// thread order: thread t holds row t) through shared memory for the fused dots.
template <Store S, int MR>
__device__ __forceinline__ double phase2_epilogue(const P2Desc &d, Acc<S> (&acc)[MR], double *__restrict__ y,
                                                  const int32_t *__restrict__ out_perm, double *rowval) {
    using RT = typename RedT<S>::T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int rr = 0; rr < MR; ++rr) {
        const int i = warp + rr * kP2Warps;
        if (i < d.ylen) {
            RT a = row_partial<S>(acc[rr]);
            for (int m = 1; m < 32; m <<= 1) a = red_xor<S>(a, m, (lane & m) != 0);
            double out;
            if constexpr (S == Store::F64) out = a;
            else out = df_to_double(a);
            if (lane == 0) {
                const int p = d.ybeg + i;
                y[out_perm ? out_perm[p] : p] = out;
                rowval[i] = out;
            }
        }
    }
    __syncthreads();
    return threadIdx.x < d.ylen ? rowval[threadIdx.x] : 0.0;
}

template <Store S, int MR>
__global__ void __launch_bounds__(kP2Threads, MR == 4 ? 3 : 2) k_phase2(const P2Desc *__restrict__ desc,
                                                                       const void *__restrict__ p2,
                                                                       const typename Tr<S>::Op *__restrict__ g,
                                                                       double *__restrict__ y,
                                                                       const int32_t *__restrict__ out_perm,
                                                                       const SolverScalars *S_, int mode,
                                                                       const double *__restrict__ w, int dotmode,
                                                                       SolverScalars *Sd, double *dpart) {
    using Op = typename Tr<S>::Op;
    constexpr int VW = Tr<S>::VW;
    __shared__ double rowval[kMaxLeaf];
    if (skip_product(S_, mode)) return;
    const P2Desc d = desc[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t esz = 16 / VW;
    const char *base = (const char *)p2 + (size_t)d.off * esz;
    const size_t row_bytes = (size_t)d.ld * esz;
    const Op *gr = g + d.goff;  // operands of this row cluster, read through L1 by every warp

    Acc<S> acc[MR];
#pragma unroll
    for (int r = 0; r < MR; ++r) acc[r].init();
    const int nv = d.ld / VW;
    int v = lane;
    // two vectors per row in flight per iteration
    for (; v + 32 < nv; v += 64) {
        int4 ra[MR], rb[MR];
#pragma unroll
        for (int rr = 0; rr < MR; ++rr) {
            const int i = warp + rr * kP2Warps;
            const char *p = base + (size_t)i * row_bytes + (size_t)v * 16;
            ra[rr] = i < d.ylen ? ld_stream(p) : make_int4(0, 0, 0, 0);
            rb[rr] = i < d.ylen ? ld_stream(p + 32 * 16) : make_int4(0, 0, 0, 0);
        }
        const GV<S> ga = GV<S>::load(gr + v * VW), gb = GV<S>::load(gr + (v + 32) * VW);
#pragma unroll
        for (int rr = 0; rr < MR; ++rr)
            if (warp + rr * kP2Warps < d.ylen) { row_mac<S>(acc[rr], ra[rr], ga); row_mac<S>(acc[rr], rb[rr], gb); }
    }
    if (v < nv) {
        int4 ra[MR];
#pragma unroll
        for (int rr = 0; rr < MR; ++rr) {
            const int i = warp + rr * kP2Warps;
            ra[rr] = i < d.ylen ? ld_stream(base + (size_t)i * row_bytes + (size_t)v * 16) : make_int4(0, 0, 0, 0);
        }
        const GV<S> ga = GV<S>::load(gr + v * VW);
#pragma unroll
        for (int rr = 0; rr < MR; ++rr)
            if (warp + rr * kP2Warps < d.ylen) row_mac<S>(acc[rr], ra[rr], ga);
    }
    const double out = phase2_epilogue<S, MR>(d, acc, y, out_perm, rowval);
    if (dotmode != 0) fused_dots(d, out, w, dotmode, Sd, dpart);
}

int grid_for(int64_t n, int threads, int cap) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

// ------------------------------------------------------------------------
// product launchers
// ------------------------------------------------------------------------
#define HMAT_DISPATCH(S, CALL)                                    \
    switch (S) {                                                  \
    case Store::DF: { constexpr Store SS = Store::DF; CALL; } break;   \
    case Store::F64: { constexpr Store SS = Store::F64; CALL; } break; \
    case Store::F32: { constexpr Store SS = Store::F32; CALL; } break; \
    case Store::BF16: { constexpr Store SS = Store::BF16; CALL; } break; \
    }

void launch_prep(Store s, const DevIndex &ix, const double *x, const int32_t *src_perm, void *xs, cudaStream_t st) {
    int blocks = grid_for(ix.n, 256, 4096);
    HMAT_DISPATCH(s, (k_prep<SS><<<blocks, 256, 0, st>>>(ix.n, x, src_perm, (typename Tr<SS>::Op *)xs)));
}

void launch_phase1(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st) {
    HMAT_DISPATCH(s, (k_phase1<SS><<<ix.nleaves, kP1Threads, 0, st>>>(
                         ix.p1, ix.p1_runs, ix.xdst, ix.lr, ix.gdst, P.q1, (const typename Tr<SS>::Op *)P.xs,
                         (typename Tr<SS>::Part *)P.part, (typename Tr<SS>::Op *)P.g, skipS, mode)));
}

void launch_reduce(Store s, const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode,
                   cudaStream_t st) {
    const int blocks = ix.nbig + (ix.ntasks + kRedThreads - 1) / kRedThreads;
    if (blocks == 0) return;
    HMAT_DISPATCH(s, (k_reduce<SS><<<blocks, kRedThreads, 0, st>>>(
                         ix.nbig, ix.ntasks, ix.red_big, ix.red_tasks, ix.lr, ix.gdst,
                         (const typename Tr<SS>::Part *)P.part, (typename Tr<SS>::Op *)P.g, skipS, mode)));
}


void launch_phase2(Store s, const DevIndex &ix, const DevPanels &P, double *y, const int32_t *out_perm,
                   const SolverScalars *skipS, int mode, cudaStream_t st, const double *w, int dotmode,
                   SolverScalars *Sd, double *dpart) {
    if (ix.max_leaf <= 4 * kP2Warps) {
        HMAT_DISPATCH(s, (k_phase2<SS, 4><<<ix.nleaves, kP2Threads, 0, st>>>(
                             ix.p2, P.p2, (const typename Tr<SS>::Op *)P.g, y, out_perm, skipS, mode, w, dotmode, Sd,
                             dpart)));
    } else {
        HMAT_DISPATCH(s, (k_phase2<SS, kMaxLeaf / kP2Warps><<<ix.nleaves, kP2Threads, 0, st>>>(
                             ix.p2, P.p2, (const typename Tr<SS>::Op *)P.g, y, out_perm, skipS, mode, w, dotmode, Sd,
                             dpart)));
    }
}


// ------------------------------------------------------------------------
// BiCG-STAB vector kernels: FP64 arithmetic, deterministic two-stage
// reductions (per-block tree, then the last block sums the block partials in
// block order)
// ------------------------------------------------------------------------
namespace {

template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double *sh) {
    // sh: NV * kVecThreads doubles
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * kVecThreads + threadIdx.x] = v[q];
    __syncthreads();
    for (int s = kVecThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < NV; ++q) sh[q * kVecThreads + threadIdx.x] += sh[q * kVecThreads + threadIdx.x + s];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = sh[q * kVecThreads];
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
        double pv = first ? r[i] : r[i] + beta * (p[i] - omega * v[i]);
        p[i] = pv;
        if constexpr (ST == Store::DF) ps[i] = split_double(pv);
        else if constexpr (ST == Store::F64) ps[i] = pv;
        else ps[i] = __double2float_rn(pv);
    }
}

template <Store ST>
__global__ void __launch_bounds__(kVecThreads) k_update_s(int n, const double *__restrict__ r, const double *__restrict__ v,
                                                          double *__restrict__ s, typename Tr<ST>::Op *__restrict__ ss,
                                                          SolverScalars *S, double *partials) {
    __shared__ double sh[kVecThreads];
    if (run_stopped(S)) return;
    const double alpha = S->alpha;
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
                                                           SolverScalars *S, double *partials, int iter_limit) {
    __shared__ double sh[2 * kVecThreads];
    if (run_stopped(S)) return;
    const bool at_s = S->stop_on_s != 0;
    const double alpha = S->alpha, omega = at_s ? 0.0 : S->omega;
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

void launch_update_p(Store s, int64_t n, const double *r, double *p, const double *v, void *ps, SolverScalars *S,
                     cudaStream_t st) {
    HMAT_DISPATCH(s, (k_update_p<SS><<<vec_blocks(n), kVecThreads, 0, st>>>((int)n, r, p, v,
                                                                           (typename Tr<SS>::Op *)ps, S)));
}

void launch_update_s(Store s, int64_t n, const double *r, const double *v, double *svec, void *ss, double *,
                     const double *, SolverScalars *S, double *partials, cudaStream_t st) {
    HMAT_DISPATCH(s, (k_update_s<SS><<<vec_blocks(n), kVecThreads, 0, st>>>((int)n, r, v, svec,
                                                                           (typename Tr<SS>::Op *)ss, S, partials)));
}

void launch_update_xr(int64_t n, double *x, const double *p, const double *svec, const double *t, double *r,
                      const double *rt, SolverScalars *S, double *partials, int iter_limit, cudaStream_t st) {
    k_update_xr<<<vec_blocks(n), kVecThreads, 0, st>>>((int)n, x, p, svec, t, r, rt, S, partials, iter_limit);
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
