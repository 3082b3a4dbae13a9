// The product for many right-hand sides at once (up to 64 per pass) with BF16
// panels on the tensor cores: every block's product is a small dense GEMM
// (mma.sync m16n8k16, BF16 inputs, FP32 accumulation).  The operands x and t
// stay FP32 in memory; staged into shared memory, each is split into a BF16 high
// part and a BF16 remainder that are both multiplied (two MMAs), so the only
// rounding to BF16 is the panels' own.
//
// The data flow is the single-vector one with every operand widened to a row of
// 64 right-hand sides (U: the source rows x_p, then the rank rows t of the
// low-rank blocks, then one zero row):
//   projection, one CTA per leaf column cluster kappa: T_kappa = Q_kappa^T X_kappa
//     (M = ranks in tiles of 16, N = 64, K = |kappa| <= 64), each rank row
//     written to its block's t row (single-cluster blocks) or partial row;
//   reduction: partial rows of multi-cluster blocks added in cluster order;
//   expansion, one CTA per leaf row cluster rho: Y_rho = P_rho G_rho (M = |rho| <= 64,
//     N = 64, K = the panel width in chunks of 64) with G_rho's rows gathered from
//     U by an index per panel column (x rows for dense blocks, t rows for
//     low-rank ones) and scaled by the stored array's power of two.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "hmat.h"
#include "kernels.h"

namespace hmat_internal {

namespace {

constexpr int kNR = kMrhsCols;  // right-hand sides per pass (floats per U row)
constexpr int kPadH = 8;        // BF16 padding per shared-memory row: conflict-free ldmatrix
constexpr int kKC = 64;         // expansion K chunk
constexpr int kThreads = 128;   // four warps

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
// d += a b: A 16 x 16 row-major, B 16 x 8 column-major, BF16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
// four FP32 values -> BF16 high parts and BF16 remainders (v = hi + lo to ~2^-17)
__device__ __forceinline__ void split4(float4 u, uint2 &hi, uint2 &lo) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(u.x), h1 = __float2bfloat16_rn(u.y);
    const __nv_bfloat16 h2 = __float2bfloat16_rn(u.z), h3 = __float2bfloat16_rn(u.w);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(u.x - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(u.y - __bfloat162float(h1));
    const __nv_bfloat16 l2 = __float2bfloat16_rn(u.z - __bfloat162float(h2));
    const __nv_bfloat16 l3 = __float2bfloat16_rn(u.w - __bfloat162float(h3));
    hi = make_uint2(pack_bf16(h0, h1), pack_bf16(h2, h3));
    lo = make_uint2(pack_bf16(l0, l1), pack_bf16(l2, l3));
}

__device__ __forceinline__ float pow2f_(int e) { return __int_as_float((e + 127) << 23); }

// x rows of U: U[p][k] = x[k * ldx + p] for k < nrhs, 0 above (cluster order)
__global__ void k_mrhs_prep(int64_t n, int nrhs, const double *__restrict__ x, int64_t ldx, float *__restrict__ U) {
    const int64_t total = n * kNR;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = q / kNR;
        const int k = (int)(q - p * kNR);
        U[q] = k < nrhs ? (float)x[(int64_t)k * ldx + p] : 0.f;
    }
}

__global__ void __launch_bounds__(kThreads) k_mrhs_phase1(const P1Desc *__restrict__ desc, const P1Run *__restrict__ runs,
                                                           const int32_t *__restrict__ tbase,
                                                           const uint16_t *__restrict__ q1, const float *__restrict__ U,
                                                           float *__restrict__ part, float *__restrict__ T) {
    __shared__ __align__(16) uint16_t sXh[kMaxLeaf][kNR + kPadH];
    __shared__ __align__(16) uint16_t sXl[kMaxLeaf][kNR + kPadH];
    __shared__ __align__(16) uint16_t sQ[kMaxLeaf][64 + kPadH];
    const P1Desc d = desc[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tig = lane & 3;
    const int mi = lane >> 3, r8 = lane & 7;
    const int KS = (d.xlen + 15) & ~15;  // rows padded to whole k16 steps
    // X_kappa split into BF16 high / low parts
    for (int idx = tid; idx < KS * (kNR / 4); idx += kThreads) {
        const int j = idx / (kNR / 4), q = idx - j * (kNR / 4);
        float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < d.xlen) u = __ldg(reinterpret_cast<const float4 *>(U + (size_t)(d.xbeg + j) * kNR) + q);
        uint2 hi, lo;
        split4(u, hi, lo);
        *reinterpret_cast<uint2 *>(&sXh[j][q * 4]) = hi;
        *reinterpret_cast<uint2 *>(&sXl[j][q * 4]) = lo;
    }
    for (int m0 = 0; m0 < d.R; m0 += 64) {
        __syncthreads();  // X staged / the previous chunk's Q consumed
        for (int idx = tid; idx < KS * 8; idx += kThreads) {
            const int j = idx >> 3, v = idx & 7, c = m0 + v * 8;
            int4 val = make_int4(0, 0, 0, 0);
            if (j < d.xlen && c < d.ld)
                val = __ldcs(reinterpret_cast<const int4 *>(q1 + (size_t)d.off + (size_t)j * d.ld + c));
            *reinterpret_cast<int4 *>(&sQ[j][v * 8]) = val;
        }
        __syncthreads();
        const int mw = m0 + 16 * warp;  // this warp's 16 ranks
        if (mw >= d.R) continue;
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
        for (int ks = 0; ks < KS; ks += 16) {
            uint32_t a[4];  // A = Q^T (ranks x rows): transposed loads of the row-major panel
            ldsm_x4_t(a, &sQ[ks + r8 + (mi >> 1) * 8][16 * warp + (mi & 1) * 8]);
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint32_t bh[4], bl[4];
                ldsm_x4_t(bh, &sXh[ks + r8 + (mi & 1) * 8][np * 16 + (mi >> 1) * 8]);
                ldsm_x4_t(bl, &sXl[ks + r8 + (mi & 1) * 8][np * 16 + (mi >> 1) * 8]);
                mma_bf16(acc[2 * np], a, bh[0], bh[1]);
                mma_bf16(acc[2 * np + 1], a, bh[2], bh[3]);
                mma_bf16(acc[2 * np], a, bl[0], bl[1]);
                mma_bf16(acc[2 * np + 1], a, bl[2], bl[3]);
            }
        }
        // rank rows g and g + 8 of the tile: to the block's t row or partial row
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int c = mw + g + 8 * half;
            if (c >= d.R) continue;
            const P1Run *rk = runs + d.rbeg;
            int lo = 0, hi = d.rcnt - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&rk[mid].col0) <= c) lo = mid;
                else hi = mid - 1;
            }
            const P1Run rn = rk[lo];
            const int l = c - rn.col0;
            float *dst = rn.poff >= 0 ? part + (size_t)(rn.poff + l) * kNR : T + (size_t)(__ldg(tbase + rn.q) + l) * kNR;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
                *reinterpret_cast<float2 *>(dst + nt * 8 + 2 * tig) = make_float2(acc[nt][2 * half], acc[nt][2 * half + 1]);
        }
    }
}

// t rows of the blocks spanning several leaf clusters: partial rows added in
// cluster order; one thread per (block, rank, 4 right-hand sides)
__global__ void k_mrhs_reduce(int ntasks, const int32_t *__restrict__ tasks, const LrDesc *__restrict__ lr,
                              const int32_t *__restrict__ tbase, const float *__restrict__ part, float *__restrict__ T) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t task = idx / (kNR / 4);
    if (task >= ntasks) return;
    const int q4 = (int)(idx - task * (kNR / 4));
    const int tq = __ldg(tasks + task);
    const LrDesc d = lr[tq >> 6];
    const int l = tq & 63;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < d.cnt; ++k) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(part + (size_t)(d.boff + (size_t)k * d.rank + l) * kNR) + q4);
        a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
    }
    reinterpret_cast<float4 *>(T + (size_t)(__ldg(tbase + (tq >> 6)) + l) * kNR)[q4] = a;
}

__global__ void __launch_bounds__(kThreads) k_mrhs_phase2(const P2Desc *__restrict__ desc, const MrhsSrc *__restrict__ src,
                                                           const uint16_t *__restrict__ p2, const float *__restrict__ U,
                                                           double *__restrict__ y, int64_t ldy, int nrhs) {
    __shared__ __align__(16) uint16_t sA[kMaxLeaf][kKC + kPadH];
    __shared__ __align__(16) uint16_t sBh[kKC][kNR + kPadH];
    __shared__ __align__(16) uint16_t sBl[kKC][kNR + kPadH];
    const P2Desc d = desc[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tig = lane & 3;
    const int mi = lane >> 3, r8 = lane & 7;
    const int MS = (d.ylen + 15) >> 4;  // m16 tiles of rows
    float acc[4][2][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
    for (int c0 = 0; c0 < d.ld; c0 += kKC) {
        __syncthreads();  // the previous chunk consumed
        for (int idx = tid; idx < MS * 16 * (kKC / 8); idx += kThreads) {
            const int i = idx / (kKC / 8), v = idx - i * (kKC / 8), c = c0 + v * 8;
            int4 val = make_int4(0, 0, 0, 0);
            if (i < d.ylen && c < d.ld)
                val = __ldcs(reinterpret_cast<const int4 *>(p2 + (size_t)d.off + (size_t)i * d.ld + c));
            *reinterpret_cast<int4 *>(&sA[i][v * 8]) = val;
        }
        for (int idx = tid; idx < kKC * (kNR / 4); idx += kThreads) {
            const int kr = idx / (kNR / 4), q = idx - kr * (kNR / 4), c = c0 + kr;
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < d.ld) {
                const MrhsSrc s = src[d.goff + c];
                u = __ldg(reinterpret_cast<const float4 *>(U + (size_t)s.row * kNR) + q);
                const float f = pow2f_(s.exp);
                u.x *= f; u.y *= f; u.z *= f; u.w *= f;
            }
            uint2 hi, lo;
            split4(u, hi, lo);
            *reinterpret_cast<uint2 *>(&sBh[kr][q * 4]) = hi;
            *reinterpret_cast<uint2 *>(&sBl[kr][q * 4]) = lo;
        }
        __syncthreads();
        const int kend = min(kKC, d.ld - c0);
        for (int ks = 0; ks < kend; ks += 16) {
            uint32_t bh[4], bl[4];  // this warp's 16 right-hand sides
            ldsm_x4_t(bh, &sBh[ks + r8 + (mi & 1) * 8][16 * warp + (mi >> 1) * 8]);
            ldsm_x4_t(bl, &sBl[ks + r8 + (mi & 1) * 8][16 * warp + (mi >> 1) * 8]);
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                if (mt >= MS) break;
                uint32_t a[4];
                ldsm_x4(a, &sA[mt * 16 + r8 + (mi & 1) * 8][ks + (mi >> 1) * 8]);
                mma_bf16(acc[mt][0], a, bh[0], bh[1]);
                mma_bf16(acc[mt][1], a, bh[2], bh[3]);
                mma_bf16(acc[mt][0], a, bl[0], bl[1]);
                mma_bf16(acc[mt][1], a, bl[2], bl[3]);
            }
        }
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        if (mt >= MS) break;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int i = mt * 16 + g + 8 * half;
            if (i >= d.ylen) continue;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int k = 16 * warp + nt * 8 + 2 * tig;
                if (k < nrhs) y[(int64_t)k * ldy + d.ybeg + i] = acc[mt][nt][2 * half];
                if (k + 1 < nrhs) y[(int64_t)(k + 1) * ldy + d.ybeg + i] = acc[mt][nt][2 * half + 1];
            }
        }
    }
}

}  // namespace

void launch_mrhs_product(const DevIndex &ix, const MrhsIndex &mx, const DevPanels &P, const double *x, int64_t ldx,
                         double *y, int64_t ldy, int nrhs, cudaStream_t st) {
    const int64_t total = (int64_t)ix.n * kNR;
    const int pb = (int)std::min<int64_t>((total + 255) / 256, 8192);
    k_mrhs_prep<<<pb, 256, 0, st>>>(ix.n, nrhs, x, ldx, mx.U);
    k_mrhs_phase1<<<ix.nleaves, kThreads, 0, st>>>(ix.p1, ix.p1_runs, mx.tbase, (const uint16_t *)P.q1, mx.U,
                                                   mx.part, mx.U + (size_t)ix.n * kNR);
    if (mx.ntasks > 0) {
        const int64_t threads = (int64_t)mx.ntasks * (kNR / 4);
        k_mrhs_reduce<<<(int)((threads + 255) / 256), 256, 0, st>>>(mx.ntasks, mx.tasks, ix.lr, mx.tbase, mx.part,
                                                                      mx.U + (size_t)ix.n * kNR);
    }
    k_mrhs_phase2<<<ix.nleaves, kThreads, 0, st>>>(ix.p2, mx.src, (const uint16_t *)P.p2, mx.U, y, ldy, nrhs);
}

}  // namespace hmat_internal
