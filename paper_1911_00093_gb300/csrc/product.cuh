// Device code of the H-matrix vector product (sm_103a), shared by the
// translation units that instantiate it for each store (kernels.cu: the
// library's own forms; kernels_table1.cu: the paper's variants).
//
// Product (Section 2.1, eq. 5-10 and 21-25), in three launches:
//   phase 1  one CTA per leaf column cluster kappa (128 threads for BF16 panels,
//            else 256): T_kappa = Q_kappa^T x_kappa, Q_kappa the rows of every
//            W_m^T (eq. 9/22) whose column cluster contains kappa, row-major; each
//            thread owns one 16-byte column vector and walks the |kappa| rows
//            (coalesced 128-bit loads, x from shared memory, no cross-thread
//            reduction) and stores its sums as whole vectors, so T_kappa is
//            written contiguously;
//   reduce   t = 2^e sum_kappa T_kappa entries of every block, in a fixed order: a
//            lane per (block, rank), a CTA per block over 32 or more clusters
//            (deterministic, no atomics on values), scattered to the operands;
//   phase 2  y_rho = P_rho g_rho with P_rho the rows of the dense blocks (eq. 21)
//            and of the V_m (eq. 10/24) over rho, g_rho the matching pieces of x
//            and t; a warp per row, each row of y written once by its owner (eq. 25
//            without atomics): by default persistent warps over groups of four
//            rows of one cluster sharing each operand load.
// Arithmetic per store:
//   DF    panels are pairs (hi, lo); products and sums in double-float on the
//         FP32 pipe (the FP64 pipe of GB300 is ~1/60 of FP32);
//   F64   IEEE FP64 FMA;
//   F32, BF16  FP32 FMA over chunks of 8 products, chunks summed in double-float;
//   PM, PS, PM1, PS2  FP32 panels with the arithmetic of Table 1 (Section 3):
//         FP64 operands and FP64 sums, products of two FP32 values rounded to
//         FP32 where Table 1 puts both in FP32 (classes of paper_forms.cpp).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>

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

// Algorithm 1's search direction, p = r + beta (p - omega v), or r at a run's
// first iteration, with explicit roundings (no contraction choices left to the
// compiler)
__device__ __forceinline__ double p_next(bool first, double r, double p, double v, double beta, double omega) {
    return first ? r : __fma_rn(beta, __fma_rn(-omega, v, p), r);
}

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
// The primary templates describe the paper's variants (FP32 panels, FP64
// operands, partial sums and accumulators).
constexpr bool is_table1(Store s) { return s == Store::PM || s == Store::PS || s == Store::PM1 || s == Store::PS2; }
// class S products (FP32 x FP32 rounded to FP32) in phase 2
constexpr bool s_class_expansion(Store s) { return s == Store::PS || s == Store::PM1; }
// FP32 operand x in phase 1 (Method 1-Single and Method 2-Single)
constexpr bool fp32_source(Store s) { return s == Store::PS || s == Store::PS2; }
template <Store S> struct Tr { static constexpr int VW = 4; using Op = double; using Part = double; };
template <> struct Tr<Store::DF> { static constexpr int VW = 2; using Op = float2; using Part = float2; };
template <> struct Tr<Store::F64> { static constexpr int VW = 2; using Op = double; using Part = double; };
template <> struct Tr<Store::F32> { static constexpr int VW = 4; using Op = float; using Part = float; };
template <> struct Tr<Store::BF16> { static constexpr int VW = 8; using Op = float; using Part = float; };

// per-column / per-row accumulator
template <Store S> struct Acc {
    double a;  // FP64 sums
    float f;   // FP32 projection z_m of Method 1
    __device__ void init() { a = 0.0; f = 0.f; }
};
template <> struct Acc<Store::DF> {
    DF a;
    __device__ void init() { a.s = 0.f; a.c = 0.f; }
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
    __device__ void init() { a.s = 0.f; a.c = 0.f; ch = 0.f; }
};

// Multiply one 16-byte panel vector by VW operands and accumulate into VW
// separate accumulators (phase 1: one per column).
template <Store S> struct Cols {
    __device__ static void mac(Acc<S> *acc, int4 raw, double x) {
        const float4 v = *reinterpret_cast<float4 *>(&raw);
        const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if constexpr (S == Store::PM) {           // FP32 W promoted, FP64 x and z
                acc[e].a = fma((double)w[e], x, acc[e].a);
            } else if constexpr (S == Store::PS) {    // FP32 W, x and z (Method 1-Single)
                acc[e].f = __fadd_rn(acc[e].f, __fmul_rn(w[e], (float)x));
            } else if constexpr (S == Store::PM1) {   // z = fl32(z + W x), right side FP64 (Method 1-Mixed)
                acc[e].f = __double2float_rn(__dadd_rn((double)acc[e].f, __dmul_rn((double)w[e], x)));
            } else {                                  // PS2: FP32 product into FP64 z (Method 2-Single)
                acc[e].a = __dadd_rn(acc[e].a, (double)__fmul_rn(w[e], (float)x));
            }
        }
    }
};
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
template <Store S> __device__ __forceinline__ void fold(Acc<S> &) {}
template <> __device__ __forceinline__ void fold<Store::DF>(Acc<Store::DF> &a) { renorm(a.a); }
template <> __device__ __forceinline__ void fold<Store::F64>(Acc<Store::F64> &) {}
template <> __device__ __forceinline__ void fold<Store::F32>(Acc<Store::F32> &a) { two_sum_acc(a.a, a.ch); a.ch = 0.f; }
template <> __device__ __forceinline__ void fold<Store::BF16>(Acc<Store::BF16> &a) { two_sum_acc(a.a, a.ch); a.ch = 0.f; }

// partial-sum output of a finished accumulator
template <Store S> __device__ __forceinline__ typename Tr<S>::Part to_part(Acc<S> &a) {
    if constexpr (S == Store::PS || S == Store::PM1) return (double)a.f;
    else return a.a;
}
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

// the many-system solver: the work item belongs to a problem whose system has
// stopped (its run ended or it finished), so its products are not needed
__device__ __forceinline__ bool item_idle(const SysScalars *sys, int prob) {
    if (sys == nullptr) return false;
    const SysScalars &q = sys[prob];
    return q.state != 0 || q.flag != 0;
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
    pdl_trigger();
    pdl_wait();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double v = x[src_perm ? src_perm[p] : p];
        if constexpr (S == Store::DF) xs[p] = split_double(v);
        else if constexpr (S == Store::F64 || is_table1(S)) xs[p] = v;
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
    else if constexpr (S == Store::F64 || is_table1(S)) return v * pow2d(e);
    else return v * pow2f(e);
}

// operand from a finished projection (scaled by 2^e, exact)
template <Store S>
__device__ __forceinline__ typename Tr<S>::Op part_to_op(typename Tr<S>::Part p, int e) {
    if constexpr (S == Store::DF) { const float f = pow2f(e); return make_float2(p.x * f, p.y * f); }
    else if constexpr (S == Store::F64 || is_table1(S)) return p * pow2d(e);
    else return p * pow2f(e);
}

// t = d_l z_l of the Method 2/3 structure V' D W' (eq. 23), when the block has factors
template <Store S>
__device__ __forceinline__ typename Tr<S>::Op apply_d(typename Tr<S>::Op o, const LrDesc &ld, int l,
                                                      const double *__restrict__ tscale) {
    if constexpr (S == Store::F64 || is_table1(S)) {
        if (ld.toff >= 0) return o * __ldg(tscale + ld.toff + l);
    }
    return o;
}

// accumulator of the completing work item's fixed-order reduction
template <Store S> struct RedT { using T = DF; };
template <> struct RedT<Store::F64> { using T = double; };
template <> struct RedT<Store::PM> { using T = double; };
template <> struct RedT<Store::PS> { using T = double; };
template <> struct RedT<Store::PM1> { using T = double; };
template <> struct RedT<Store::PS2> { using T = double; };
constexpr bool red_double(Store s) { return s == Store::F64 || is_table1(s); }

// Method 1's z_m stays FP32 across the partial sums of its leaf clusters:
// FP32 additions (Single), FP64 additions rounded to FP32 (Mixed)
__device__ __forceinline__ double red_m1(Store s, double a, double b) {
    return s == Store::PS ? (double)__fadd_rn((float)a, (float)b) : (double)__double2float_rn(a + b);
}

template <Store S> __device__ __forceinline__ void red_zero(typename RedT<S>::T &a) {
    if constexpr (red_double(S)) a = 0.0; else { a.s = 0.f; a.c = 0.f; }
}
template <Store S> __device__ __forceinline__ void red_add_part(typename RedT<S>::T &a, typename Tr<S>::Part p) {
    if constexpr (S == Store::PS || S == Store::PM1) a = red_m1(S, a, p);
    else if constexpr (red_double(S)) a += p;
    else if constexpr (S == Store::DF) a = df_add(a, DF{p.x, p.y});
    else two_sum_acc(a, p);
}
template <Store S> __device__ __forceinline__ void red_add(typename RedT<S>::T &a, typename RedT<S>::T b) {
    if constexpr (S == Store::PS || S == Store::PM1) a = red_m1(S, a, b);
    else if constexpr (red_double(S)) a += b;
    else a = df_add(a, b);
}
template <Store S>
__device__ __forceinline__ typename RedT<S>::T red_xor(typename RedT<S>::T a, int m, bool upper) {
    typename RedT<S>::T b;
    if constexpr (red_double(S)) b = __shfl_xor_sync(0xffffffffu, a, m);
    else { b.s = __shfl_xor_sync(0xffffffffu, a.s, m); b.c = __shfl_xor_sync(0xffffffffu, a.c, m); }
    // row sums of phase 2 are FP64 additions for every FP64-accumulated store
    // (Table 1 puts y^_m in FP64, also for Method 1)
    if constexpr (red_double(S)) return upper ? b + a : a + b;
    else {
        if (upper) { red_add<S>(b, a); return b; }
        red_add<S>(a, b);
        return a;
    }
}

template <Store S> __device__ __forceinline__ typename Tr<S>::Part red_to_part(typename RedT<S>::T a) {
    if constexpr (red_double(S)) return a;
    else if constexpr (S == Store::DF) { renorm(a); return make_float2(a.s, a.c); }
    else return __fadd_rn(a.s, a.c);
}

// ------------------------------------------------------------------------
// phase 1: per leaf column cluster kappa
// ------------------------------------------------------------------------
// 128 threads for BF16 panels (8 columns per thread: most clusters need fewer
// than 128 threads, and small CTAs let more clusters stream at once), else 256
template <Store S> constexpr int p1_threads() { return S == Store::BF16 ? 128 : 256; }
// resident CTAs per SM the register budget is held to: 64 registers a thread
// (BF16, FP32), 51 for the others (8 CTAs of 128 threads for BF16, 4 or 5 of 256
// for the others; the tuned CTA sizes keep the same budget per thread)
template <Store S, int NT> constexpr int p1_min_blocks() {
    return (65536 / (NT * (S == Store::BF16 || S == Store::F32 ? 64 : 51))) < 32
               ? 65536 / (NT * (S == Store::BF16 || S == Store::F32 ? 64 : 51))
               : 32;
}
constexpr int kP1SmemXd = 64;     // dense-operand slices staged in shared memory

// One leaf column cluster of the projection, its x slice and dense slices
// already staged in shared memory (xds null: read them from global memory):
// the column vectors' dot products with x_kappa, stored in panel column order
// at T + d.tbeg (each thread its VW consecutive sums: 16 or 32 contiguous bytes,
// a warp 512 or 1024), then the dense-block operand slices.
template <Store S, int NT>
__device__ __forceinline__ void p1_cluster(const P1Desc &d, const typename Tr<S>::Op *xk, const XDst *xds,
                                           const XDst *__restrict__ xdst, const int32_t *__restrict__ xsel,
                                           const void *__restrict__ q1, typename Tr<S>::Part *__restrict__ part,
                                           typename Tr<S>::Op *__restrict__ g) {
    using Part = typename Tr<S>::Part;
    constexpr int VW = Tr<S>::VW;
    static_assert(sizeof(Part) * VW % 16 == 0, "a thread's sums are whole 16-byte vectors");
    const int nvec = d.ld / VW, xlen = d.xlen;
    const char *base = (const char *)q1 + (size_t)d.off * (16 / VW);
    const size_t row_bytes = (size_t)d.ld * (16 / VW);

    // projections (eq. 9/22): thread = one 16-byte column vector, walk the rows
    for (int vc = threadIdx.x; vc < nvec; vc += NT) {
        Acc<S> acc[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[e].init();
        const char *col = base + (size_t)vc * 16;
        int j = 0;
        for (; j + 8 <= xlen; j += 8) {
            int4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = ld_stream(col + (size_t)(j + u) * row_bytes);
#pragma unroll
            for (int u = 0; u < 8; ++u) Cols<S>::mac(acc, raw[u], xk[j + u]);
#pragma unroll
            for (int e = 0; e < VW; ++e) fold<S>(acc[e]);
        }
        if constexpr (is_table1(S)) {  // FP64-pipe bound: the last rows one at a time
            for (; j < xlen; ++j) Cols<S>::mac(acc, ld_stream(col + (size_t)j * row_bytes), xk[j]);
        } else if (j < xlen) {  // the last rows: one batch of loads in flight, the same sums in row order
            const int rem = xlen - j;
            int4 raw[7];
#pragma unroll
            for (int u = 0; u < 7; ++u)
                raw[u] = u < rem ? ld_stream(col + (size_t)(j + u) * row_bytes) : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 7; ++u) {
                if (u >= rem) break;  // CTA-uniform: no multiply-adds on the padding
                Cols<S>::mac(acc, raw[u], xk[j + u]);
            }
        }
        // t_{m,kappa} of the vector's VW columns (zero past R: the panel's padding)
        Part out[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) out[e] = to_part<S>(acc[e]);
        uint32_t w[sizeof(out) / 4];
        memcpy(w, out, sizeof(out));
        int4 *dst = reinterpret_cast<int4 *>(part + d.tbeg + (size_t)vc * VW);
#pragma unroll
        for (int u = 0; u < (int)(sizeof(out) / 16); ++u)
            dst[u] = make_int4((int)w[4 * u], (int)w[4 * u + 1], (int)w[4 * u + 2], (int)w[4 * u + 3]);
    }

    // the dense-block operands fed by x_kappa (eq. 21 inputs), scaled by 2^e: a
    // whole slice, or the listed entries of a column subset
    const int xdcnt = d.xdcnt;
    for (int t = threadIdx.x; t < xdcnt * xlen; t += NT) {
        const int k = t / xlen, j = t - k * xlen;
        const XDst x = xds ? xds[k] : xdst[d.xdbeg + k];
        if (j < x.cnt) g[x.goff + j] = scale_op<S>(xk[x.sel < 0 ? j : __ldg(xsel + x.sel + j)], x.scale);
    }
}

template <Store S, int NT = p1_threads<S>()>
__global__ void __launch_bounds__(NT, (p1_min_blocks<S, NT>())) k_phase1(int base, const P1Desc *__restrict__ desc,
                                                        const XDst *__restrict__ xdst, const int32_t *__restrict__ xsel,
                                                        const void *__restrict__ q1,
                                                        const typename Tr<S>::Op *__restrict__ xs,
                                                        typename Tr<S>::Part *__restrict__ part,
                                                        typename Tr<S>::Op *__restrict__ g, const SolverScalars *S_,
                                                        int mode, const SysScalars *sys) {
    using Op = typename Tr<S>::Op;
    __shared__ Op xk[kMaxLeaf];  // x_kappa, broadcast to every thread
    // the cluster's dense-operand descriptors, loaded with x_kappa so that the
    // slice loop's lookups stay on chip (global reads past the limit)
    __shared__ XDst xds[kP1SmemXd];
    pdl_trigger();
    const P1Desc d = desc[base + blockIdx.x];
    const bool xd_sm = d.xdcnt <= kP1SmemXd;
    if (xd_sm)
        for (int j = threadIdx.x; j < d.xdcnt; j += NT) xds[j] = xdst[d.xdbeg + j];
    pdl_wait();  // x, the flags and the outputs belong to earlier kernels
    if (skip_product(S_, mode) || item_idle(sys, d.pad[0])) return;  // (pad[0]: the item's problem)
    for (int j = threadIdx.x; j < d.xlen; j += NT) {
        if constexpr (fp32_source(S)) xk[j] = (double)__double2float_rn(xs[d.xbeg + j]);  // Section 3.5
        else xk[j] = xs[d.xbeg + j];
    }
    __syncthreads();
    p1_cluster<S, NT>(d, xk, xd_sm ? xds : nullptr, xdst, xsel, q1, part, g);
}

// ------------------------------------------------------------------------
// reduce: every block's t_m = sum of its per-cluster projections
// t_{m,kappa} (eq. 9), in a fixed order, scaled by 2^e (and d_l, eq. 23) and
// scattered to the operand buffers of its leaf row clusters.  Blocks over
// >= kRedBigCnt leaf clusters get a whole CTA (kernel blocks [0, nbig)), their
// T offsets and destinations staged in shared memory; the others are split into
// one task per rank, kRedTasks tasks per thread (one term and no sum when the
// column cluster is a leaf), except the ranks of blocks inside one leaf column
// cluster and one leaf row cluster (no factors d_l): those are direct copies
// from T to their operand slot, one record each (the last kernel blocks).
// ------------------------------------------------------------------------
constexpr int kRedThreads = 128;
constexpr int kRedTasks = 1;     // independent tasks per thread of the small blocks
constexpr int kRedStage = 256;   // T offsets / destinations of a big block staged on chip

template <Store S>
__device__ __forceinline__ void reduce_task(int l, const LrDesc &ld, const int32_t *__restrict__ gdst,
                                            const int32_t *__restrict__ tofs,
                                            const typename Tr<S>::Part *__restrict__ part,
                                            typename Tr<S>::Op *__restrict__ g, const double *__restrict__ tscale,
                                            const SysScalars *sys) {
    using RT = typename RedT<S>::T;
    if (item_idle(sys, ld.pad)) return;
    const typename Tr<S>::Part *src = part + l;
    const int32_t *to = tofs + ld.boff;
    typename Tr<S>::Part t;
    if (ld.cnt == 1) {  // the column cluster is a leaf: t_m is its one projection
        t = src[__ldg(to)];
    } else {
        RT a;
        red_zero<S>(a);
#pragma unroll 4
        for (int k = 0; k < ld.cnt; ++k) red_add_part<S>(a, src[__ldg(to + k)]);
        t = red_to_part<S>(a);
    }
    const typename Tr<S>::Op o = apply_d<S>(part_to_op<S>(t, ld.scale), ld, l, tscale);
    for (int k = 0; k < ld.gcnt; ++k) g[gdst[ld.gbeg + k] + l] = o;
}

static_assert(sizeof(RedDirect) == 16 && offsetof(RedDirect, gdst) == 4 && offsetof(RedDirect, scale) == 8 &&
                  offsetof(RedDirect, prob) == 12,
              "RedDirect is read as one int4 (tsrc, gdst, scale, prob)");

template <Store S>
__global__ void __launch_bounds__(kRedThreads) k_reduce(int nbig, int ntasks, int ndirect,
                                                         const int32_t *__restrict__ big,
                                                         const int32_t *__restrict__ tasks,
                                                         const RedDirect *__restrict__ direct,
                                                         const LrDesc *__restrict__ lr, const int32_t *__restrict__ gdst,
                                                         const int32_t *__restrict__ tofs,
                                                         const typename Tr<S>::Part *__restrict__ part,
                                                         typename Tr<S>::Op *__restrict__ g,
                                                         const double *__restrict__ tscale, const SolverScalars *S_,
                                                         int mode, const SysScalars *sys) {
    using RT = typename RedT<S>::T;
    __shared__ RT red[kRedThreads];
    __shared__ int32_t sto[kRedStage], sgd[kRedStage];
    pdl_trigger();
    if ((int)blockIdx.x < nbig) {
        const LrDesc ld = lr[big[blockIdx.x]];
        const bool st_to = ld.cnt <= kRedStage, st_gd = ld.gcnt <= kRedStage;
        if (st_to)
            for (int k = threadIdx.x; k < ld.cnt; k += kRedThreads) sto[k] = __ldg(tofs + ld.boff + k);
        if (st_gd)
            for (int k = threadIdx.x; k < ld.gcnt; k += kRedThreads) sgd[k] = __ldg(gdst + ld.gbeg + k);
        pdl_wait();  // T, the flags and g belong to earlier kernels
        if (skip_product(S_, mode) || item_idle(sys, ld.pad)) return;  // (pad: the block's problem; CTA-uniform)
        __syncthreads();
        const int32_t *to = st_to ? sto : tofs + ld.boff;  // generic pointers: shared or global
        const int32_t *gd = st_gd ? sgd : gdst + ld.gbeg;
        for (int l0 = 0; l0 < ld.rank; l0 += 32) {
            const int rr = min(32, ld.rank - l0);
            int rp = 1;
            while (rp < rr) rp <<= 1;
            const int G = kRedThreads / rp, gi = threadIdx.x / rp, l = threadIdx.x % rp;
            RT a;
            red_zero<S>(a);
            if (l < rr) {
                const typename Tr<S>::Part *src = part + l0 + l;
#pragma unroll 8
                for (int k = gi; k < ld.cnt; k += G) red_add_part<S>(a, src[to[k]]);
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
                g[gd[k] + l0 + ll] = apply_d<S>(part_to_op<S>(red_to_part<S>(red[ll]), ld.scale), ld, l0 + ll, tscale);
            }
            __syncthreads();
        }
        return;
    }
    const int task_blocks = (ntasks + kRedThreads * kRedTasks - 1) / (kRedThreads * kRedTasks);
    if ((int)blockIdx.x >= nbig + task_blocks) {  // a rank of a single-leaf block: t_m = 2^e T entry
        const int i = ((int)blockIdx.x - nbig - task_blocks) * kRedThreads + threadIdx.x;
        int4 r = make_int4(0, 0, 0, 0);  // (tsrc, gdst, scale, prob) of RedDirect
        if (i < ndirect) r = __ldg(reinterpret_cast<const int4 *>(direct) + i);
        pdl_wait();  // T, the flags and g belong to earlier kernels
        if (i >= ndirect || skip_product(S_, mode) || item_idle(sys, r.w)) return;
        g[r.y] = part_to_op<S>(part[r.x], r.z);
        return;
    }
    // the other blocks: one lane per (block, rank), a sequential sum over the
    // block's leaf clusters (independent loads) and the scatter of that rank
    const int t0 = ((int)blockIdx.x - nbig) * kRedThreads * kRedTasks + threadIdx.x;
    int tq[kRedTasks];
    LrDesc ld[kRedTasks];
#pragma unroll
    for (int u = 0; u < kRedTasks; ++u) {
        const int task = t0 + u * kRedThreads;
        tq[u] = task < ntasks ? __ldg(tasks + task) : -1;
        if (tq[u] >= 0) ld[u] = lr[tq[u] >> 6];
    }
    pdl_wait();  // T, the flags and g belong to earlier kernels
    if (skip_product(S_, mode)) return;
#pragma unroll
    for (int u = 0; u < kRedTasks; ++u)
        if (tq[u] >= 0) reduce_task<S>(tq[u] & 63, ld[u], gdst, tofs, part, g, tscale, sys);
}

// ------------------------------------------------------------------------
// phase 2: per leaf row cluster, y_rho = P_rho g_rho
// ------------------------------------------------------------------------
constexpr int kP2Threads = 256;
constexpr int kP2Warps = kP2Threads / 32;

// The VW operands matching one 16-byte panel vector, loaded as vectors through
// L1 (operand buffers are 16-byte aligned per row cluster).
template <Store S> struct GV {  // paper's variants: four FP64 operands
    double2 a, b;
    __device__ static GV load(const double *p) {
        GV r;
        r.a = __ldg(reinterpret_cast<const double2 *>(p));
        r.b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        return r;
    }
};
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
__device__ __forceinline__ void row_mac(Acc<S> &acc, int4 raw, const GV<S> &gv) {
    const float4 v = *reinterpret_cast<float4 *>(&raw);
    const double x[4] = {gv.a.x, gv.a.y, gv.b.x, gv.b.y};
    const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if constexpr (s_class_expansion(S))  // FP32 x FP32 rounded to FP32, added in FP64
            acc.a = __dadd_rn(acc.a, (double)__fmul_rn(w[e], (float)x[e]));
        else                                 // FP32 promoted, FP64 operand and sum
            acc.a = fma((double)w[e], x[e], acc.a);
    }
}
// One panel vector of a row: the row-group expansion advances its rows in step
// and folds the double-float and BF16 accumulators itself (fold<S>) after every
// kFoldVecs vectors
constexpr int kFoldVecs = 4;
template <Store S>
__device__ __forceinline__ void row_mac_nofold(Acc<S> &acc, int4 raw, const GV<S> &gv) {
    if constexpr (S == Store::DF) {
        float4 v = *reinterpret_cast<float4 *>(&raw);
        df_fma(acc.a, v.x, v.y, gv.v.x, gv.v.y);
        df_fma(acc.a, v.z, v.w, gv.v.z, gv.v.w);
    } else if constexpr (S == Store::BF16) {
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
    } else {
        row_mac<S>(acc, raw, gv);
    }
}
template <Store S> constexpr bool row_folds() { return S == Store::DF || S == Store::BF16; }
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

// the lane partial of one row as a reduction accumulator
template <Store S>
__device__ __forceinline__ typename RedT<S>::T row_partial(Acc<S> &a) {
    if constexpr (red_double(S)) return a.a;
    else {
        if constexpr (S == Store::BF16) { two_sum_acc(a.a, a.ch); a.ch = 0.f; }
        renorm(a.a);
        return a.a;
    }
}

// Row-group expansion: persistent warps over groups of up to four consecutive
// rows of one leaf row cluster, so each 16-byte operand vector g_rho is loaded
// once for the group's rows.

// Totals of a group's four rows from the lanes' partials with 12 shuffles
// instead of four butterflies of 5: the xor-16 step keeps rows 0-1 in the lower
// half-warp and rows 2-3 in the upper, the xor-8 step one row per quarter, and
// xor 4, 2, 1 finish it.  Every pairing adds the lower lane's value first, in
// the canonical order (16, 8, 4, 2, 1), so lanes 8r..8r+7 hold exactly row r's
// canonical total (the canonical butterfly: lane partials paired at xor 16, 8,
// 4, 2, 1, the lower lane's value first).  Rows past the group's end are zero
// and unused.
template <Store S>
__device__ __forceinline__ double group_totals(Acc<S> (&acc)[kGroupRows], int lane) {
    static_assert(kGroupRows == 4, "the transposed reduction is written for four rows");
    using RT = typename RedT<S>::T;
    RT a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = row_partial<S>(acc[r]);
    auto shfl = [](RT v, int m) {
        RT w;
        if constexpr (red_double(S)) w = __shfl_xor_sync(0xffffffffu, v, m);
        else { w.s = __shfl_xor_sync(0xffffffffu, v.s, m); w.c = __shfl_xor_sync(0xffffffffu, v.c, m); }
        return w;
    };
    // (lower lane's value) + (upper lane's value), as red_xor adds them
    auto add = [](RT lo, RT hi) {
        if constexpr (red_double(S)) return lo + hi;
        else { red_add<S>(lo, hi); return lo; }
    };
    const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
    // xor 16: send the rows the other half keeps
    const RT r0 = shfl(up16 ? a[0] : a[2], 16), r1 = shfl(up16 ? a[1] : a[3], 16);
    const RT k0 = up16 ? add(r0, a[2]) : add(a[0], r0);
    const RT k1 = up16 ? add(r1, a[3]) : add(a[1], r1);
    // xor 8: one row per quarter-warp
    const RT rv = shfl(up8 ? k0 : k1, 8);
    RT k = up8 ? add(rv, k1) : add(k0, rv);
    for (int m = 4; m >= 1; m >>= 1) k = red_xor<S>(k, m, (lane & m) != 0);
    if constexpr (red_double(S)) return k;
    else return df_to_double(k);
}

static_assert(sizeof(GroupDesc) == 32 && offsetof(GroupDesc, goff) == 8 && offsetof(GroupDesc, nr) == 20,
              "GroupDesc is read as eight 32-bit words");
// a GroupDesc from its words 0..5, held one per lane in lanes 0..5
__device__ __forceinline__ GroupDesc group_from_words(int32_t word) {
    GroupDesc d;
    const uint32_t lo = (uint32_t)__shfl_sync(0xffffffffu, word, 0);
    const uint32_t hi = (uint32_t)__shfl_sync(0xffffffffu, word, 1);
    d.off = (int64_t)(((uint64_t)hi << 32) | lo);
    d.goff = __shfl_sync(0xffffffffu, word, 2);
    d.ld = __shfl_sync(0xffffffffu, word, 3);
    d.p0 = __shfl_sync(0xffffffffu, word, 4);
    d.nr = __shfl_sync(0xffffffffu, word, 5);
    d.pad[0] = d.pad[1] = 0;
    return d;
}

template <Store S>
__global__ void __launch_bounds__(kP2Threads, kP2gBlocks) k_phase2g(
    int ng, const GroupDesc *__restrict__ groups, const void *__restrict__ p2, const typename Tr<S>::Op *__restrict__ g,
    double *__restrict__ y, const int32_t *__restrict__ out_perm, int accum, const SolverScalars *S_, int mode,
    const double *__restrict__ w, int dotmode, double *dpart,
    const SysScalars *sys) {
    constexpr int VW = Tr<S>::VW;
    constexpr size_t esz = 16 / VW;
    constexpr int GR = kGroupRows;
    __shared__ double wsum[2][kP2Warps];
    pdl_trigger();
    pdl_wait();  // g, y, w and the flags belong to earlier kernels
    if (skip_product(S_, mode)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = gridDim.x * kP2Warps;
    // lane 8r owns row r of a group (r < nr): its output index, w and (accum)
    // old y are loaded at the group's start, so the epilogue waits on no load
    double dw = 0.0, dy = 0.0;
    int t = blockIdx.x * kP2Warps + warp;
    // the next group's descriptor travels as one word per lane (lanes 0..5)
    // while this group streams, then is broadcast: one register, not six
    const int32_t *gwords = reinterpret_cast<const int32_t *>(groups);
    // (word 6, pad[0], is the group's problem: lane 6 carries it for the skip test)
    const int nw = sys ? 7 : 6;
    int32_t word = (lane < nw && t < ng) ? __ldg(gwords + (size_t)t * 8 + lane) : 0;
    GroupDesc cur = group_from_words(word);
    int prob = sys ? __shfl_sync(0xffffffffu, word, 6) : 0;
    for (; t < ng; t += W) {
        word = (lane < nw && t + W < ng) ? __ldg(gwords + (size_t)(t + W) * 8 + lane) : 0;
        if (item_idle(sys, prob)) {  // warp-uniform: the group's problem has stopped
            cur = group_from_words(word);
            prob = sys ? __shfl_sync(0xffffffffu, word, 6) : 0;
            continue;
        }
        const bool own = (lane & 7) == 0 && (lane >> 3) < cur.nr;
        const int p = cur.p0 + (lane >> 3);
        int q = p;
        double wl = 0.0, yl = 0.0;
        if (own) {
            if (out_perm) q = __ldg(out_perm + p);
            if (dotmode != 0) wl = __ldg(w + p);
            if (accum) yl = y[q];  // a later segment adds to the earlier ones' rows
        }
        const char *base = (const char *)p2 + (size_t)cur.off * esz;
        const size_t row_bytes = (size_t)cur.ld * esz;
        const typename Tr<S>::Op *gr = g + cur.goff;
        const int nv = cur.ld / VW, nr = cur.nr;
        Acc<S> acc[GR];
#pragma unroll
        for (int r = 0; r < GR; ++r) acc[r].init();
        int nf = 0;  // vectors since the rows' last fold (the rows advance in step)
        int v = lane;
        // two vectors per row in flight (v and v + 32), used in order: the same sums
        for (; v + 32 < nv; v += 64) {
            int4 raw[GR], raw2[GR];
#pragma unroll
            for (int r = 0; r < GR; ++r) {
                raw[r] = r < nr ? ld_stream(base + (size_t)r * row_bytes + (size_t)v * 16) : make_int4(0, 0, 0, 0);
                raw2[r] = r < nr ? ld_stream(base + (size_t)r * row_bytes + (size_t)(v + 32) * 16) : make_int4(0, 0, 0, 0);
            }
            const GV<S> gv = GV<S>::load(gr + v * VW), gv2 = GV<S>::load(gr + (v + 32) * VW);
#pragma unroll
            for (int r = 0; r < GR; ++r)
                if (r < nr) row_mac_nofold<S>(acc[r], raw[r], gv);
            if constexpr (row_folds<S>()) {
                if (++nf == kFoldVecs) {
#pragma unroll
                    for (int r = 0; r < GR; ++r) fold<S>(acc[r]);
                    nf = 0;
                }
            }
#pragma unroll
            for (int r = 0; r < GR; ++r)
                if (r < nr) row_mac_nofold<S>(acc[r], raw2[r], gv2);
            if constexpr (row_folds<S>()) {
                if (++nf == kFoldVecs) {
#pragma unroll
                    for (int r = 0; r < GR; ++r) fold<S>(acc[r]);
                    nf = 0;
                }
            }
        }
        for (; v < nv; v += 32) {
            int4 raw[GR];
#pragma unroll
            for (int r = 0; r < GR; ++r)
                raw[r] = r < nr ? ld_stream(base + (size_t)r * row_bytes + (size_t)v * 16) : make_int4(0, 0, 0, 0);
            const GV<S> gv = GV<S>::load(gr + v * VW);
#pragma unroll
            for (int r = 0; r < GR; ++r)
                if (r < nr) row_mac_nofold<S>(acc[r], raw[r], gv);
            if constexpr (row_folds<S>()) {
                if (++nf == kFoldVecs) {
#pragma unroll
                    for (int r = 0; r < GR; ++r) fold<S>(acc[r]);
                    nf = 0;
                }
            }
        }
        // lanes 8r..8r+7 end with row r's total, the same bits as the
        // canonical butterfly (group_totals)
        const double mine = group_totals<S>(acc, lane);
        if (own) {
            const double out = accum ? yl + mine : mine;
            y[q] = out;
            if (dotmode != 0) {
                dw += wl * out;
                dy += out * out;
            }
        }
        cur = group_from_words(word);
        prob = sys ? __shfl_sync(0xffffffffu, word, 6) : 0;
    }
    if (dotmode == 0) return;
    // the warp's share: the owner lanes 0, 8, 16, 24 in lane order
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int r = 0; r < GR; ++r) {
        a += __shfl_sync(0xffffffffu, dw, 8 * r);
        b += __shfl_sync(0xffffffffu, dy, 8 * r);
    }
    if (lane == 0) {
        wsum[0][warp] = a;
        wsum[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int k = 0; k < kP2Warps; ++k) { sa += wsum[0][k]; sb += wsum[1][k]; }
        dpart[blockIdx.x] = sa;
        dpart[gridDim.x + blockIdx.x] = sb;
    }
}

int grid_for(int64_t n, int threads, int cap) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// launches of one store's product kernels (the dispatchers pick the store)
template <Store SS, int NT>
void phase1_run(const P1Desc *list, int base, int count, const DevIndex &ix, const DevPanels &P,
                const SolverScalars *skipS, int mode, cudaStream_t st, const SysScalars *sys) {
    launch_pdl(k_phase1<SS, NT>, dim3(count), dim3(NT), st, base, list, ix.xdst, ix.xsel, P.q1,
               (const typename Tr<SS>::Op *)P.xs, (typename Tr<SS>::Part *)P.part, (typename Tr<SS>::Op *)P.g, skipS,
               mode, sys);
}

// The projection: one launch per run of the work list (one run over the
// clusters in order by default; the tuned plan's runs over the list sorted by
// panel width, each with its CTA size).  The paper's variants keep one CTA size.
template <Store SS>
void phase1_launch(const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode, cudaStream_t st,
                   const SysScalars *sys) {
    if constexpr (is_table1(SS)) {
        phase1_run<SS, p1_threads<SS>()>(ix.p1, 0, ix.nleaves, ix, P, skipS, mode, st, sys);
    } else {
        if (ix.nruns == 0) {
            phase1_run<SS, p1_threads<SS>()>(ix.p1, 0, ix.nleaves, ix, P, skipS, mode, st, sys);
            return;
        }
        const P1Desc *list = ix.p1_sorted ? ix.p1_sorted : ix.p1;
        for (int r = 0; r < ix.nruns; ++r) {
            const P1Plan &u = ix.runs[r];
            if (u.count <= 0) continue;
            if (u.nt == 64) phase1_run<SS, 64>(list, u.begin, u.count, ix, P, skipS, mode, st, sys);
            else if (u.nt == 128) phase1_run<SS, 128>(list, u.begin, u.count, ix, P, skipS, mode, st, sys);
            else phase1_run<SS, 256>(list, u.begin, u.count, ix, P, skipS, mode, st, sys);
        }
    }
}

template <Store SS>
void reduce_launch(const DevIndex &ix, const DevPanels &P, const SolverScalars *skipS, int mode, cudaStream_t st,
                   const SysScalars *sys) {
    const int blocks = ix.nbig + (ix.ntasks + kRedThreads * kRedTasks - 1) / (kRedThreads * kRedTasks) +
                       (ix.ndirect + kRedThreads - 1) / kRedThreads;
    if (blocks == 0) return;
    launch_pdl(k_reduce<SS>, dim3(blocks), dim3(kRedThreads), st, ix.nbig, ix.ntasks, ix.ndirect, ix.red_big,
               ix.red_tasks, ix.red_direct, ix.lr,
               ix.gdst, ix.tofs, (const typename Tr<SS>::Part *)P.part, (typename Tr<SS>::Op *)P.g, ix.tscale, skipS,
               mode, sys);
}

template <Store SS>
void phase2_launch(const DevIndex &ix, const DevPanels &P, double *y, const int32_t *out_perm, int accum,
                   const SolverScalars *skipS, int mode, cudaStream_t st, const double *w, int dotmode,
                   double *dpart, const SysScalars *sys) {
    launch_pdl(k_phase2g<SS>, dim3(phase2_items(ix)), dim3(kP2Threads), st, ix.ngroups, ix.groups, P.p2,
               (const typename Tr<SS>::Op *)P.g, y, out_perm, accum, skipS, mode, w, dotmode, dpart, sys);
}

}  // namespace

}  // namespace hmat_internal
