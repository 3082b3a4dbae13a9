// The product for many right-hand sides at once (up to 64 per pass) with BF16
// panels on the fifth-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory).  Every operand row U[p] holds the 64 right-hand sides of one
// source entry in FP32: the x rows (cluster order), then the t rows of the
// low-rank blocks, then one zero row.  Staged into shared memory, each operand
// is split into a BF16 high part and a BF16 remainder (v = hi + lo to about
// 2^-17), stacked as the 128 rows of the MMA's A operand, so one MMA multiplies
// both parts and the only rounding to BF16 is the panels' own:
//
//   projection, one CTA per column cluster sigma that has low-rank blocks
//     (eq. 9, all of sigma's blocks at once, over all of sigma's columns):
//     D (128 x R_sigma) = [X_hi; X_lo]^T (sigma) * W_sigma^T, W_sigma the rank
//     rows of every block whose column cluster is sigma, so every t row is
//     complete (no partial sums, no reduction);  t = D[m] + D[m + 64];
//   expansion, one CTA per leaf row cluster rho (eq. 10, 21, 24-25):
//     D (128 x |rho|) = [G_hi; G_lo]^T * P_rho^T, with G_rho's rows gathered from U
//     by an index per panel column and scaled by the stored array's power of
//     two, P_rho the rows of the phase-2 panel;  y = D[m] + D[m + 64].
//
// Both operands are K-major without swizzle: 8 x 8 BF16 core matrices of 128
// contiguous bytes, core (r/8, k/8) at ((k/8) * R/8 + r/8) * 128 bytes, so the
// descriptors' leading (K) stride is R/8 * 128 bytes and the stride (M/N) one
// 128 bytes.  K runs in chunks of 64 through one buffer per CTA: a chunk's MMAs
// finish before the next chunk is staged over it, and the other CTAs on the SM
// (4 or 8, as many as its tensor memory serves) fill the gap.  The projection's
// W tiles are stored in that layout (packed at upload) and arrive by one bulk
// copy per chunk; the expansion's panel rows arrive by 16-byte cp.async.
// Every wait is bounded: a wait that runs out records HMAT_ERR_TIMEOUT in
// *ctl.status, the CTA stops issuing work, lets what it issued finish, frees its
// tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "hmat.h"
#include "kernels.h"

namespace hmat_internal {

namespace {

constexpr int kNR = kMrhsCols;     // right-hand sides per pass (floats per U row)
constexpr int kThreads = 128;      // four warps: warp w reads tensor-memory lanes 32w..32w+31
constexpr int kKC = 64;            // K chunk, BF16 panels (128 bytes a row)
constexpr int kM = 2 * kNR;        // MMA rows: high parts 0..63, remainders 64..127
constexpr int kABytes = kM * 128;  // one A chunk (16 KB)
// FP32 panels (TF, kind::tf32): a K chunk of 32 entries fills the same 128 bytes a row
template <bool TF> constexpr int kc_max() { return TF ? 32 : kKC; }
constexpr long long kDrainCycles = 4000000000ll;        // ~2 s: issued work always finishes long before
constexpr int kEpiStride = 33;     // floats per right-hand side in the epilogue's exchange (no bank conflicts)

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, version 1 (sm_100 family)
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((sa(p) >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// instruction descriptor of kind::tf32: TF32 A and B (both K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mb_init(uint64_t *b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sa(dst)),
                 "l"(src), "r"(bytes), "r"(sa(bar))
                 : "memory");
}
// 16 bytes global -> shared, zero-filled when `valid` is false (nothing is read then)
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(bar)) : "memory");
}
// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float pow2f_(int e) { return __int_as_float((e + 127) << 23); }

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
// FP32 -> TF32 (10 fraction bits), round to nearest, ties away from zero: the
// FP32 bit pattern with the low 13 bits cleared
__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}
// v = hi + lo + O(2^-22 |v|), both TF32
__device__ __forceinline__ void split_tf32(float v, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(v);
    lo = to_tf32(v - __uint_as_float(hi));
}

// Bounded wait on an mbarrier phase; false when this CTA gave up (here or in
// another thread), the timeout recorded.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, const PipeCtl &ctl, volatile int *abort_flag) {
    const long long t0 = clock64();
    while (!mb_test(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > ctl.wait_limit) {
            *abort_flag = 1;
            if (ctl.status) *(volatile int32_t *)ctl.status = HMAT_ERR_TIMEOUT;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void drain_bar(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mb_test(bar, parity) && clock64() - t0 < kDrainCycles) {
    }
}

// One A chunk: operands k0 .. k0 + kc - 1 (kc a multiple of 16), 64 right-hand
// sides each; operand kk's value for right-hand side m is get(kk) [m]; its high
// part goes to row m, its remainder to row m + 64 (BF16 parts, or TF32 parts for
// FP32 panels).  A task is one core-matrix row (16 bytes: 8 BF16 or 4 TF32
// operands of one right-hand side): 16-byte stores, and the 32 threads of a
// warp read 32 consecutive floats of a U row.
template <bool TF, class Row>
__device__ __forceinline__ void stage_a(unsigned char *A, int kc, Row row) {
    constexpr int EPC = TF ? 4 : 8;  // operands per 16-byte core-matrix row
    for (int task = threadIdx.x; task < kNR * (kc / EPC); task += kThreads) {
        const int m = task % kNR, ki = task / kNR;
        uint32_t hi[4], lo[4];
        if constexpr (TF) {
#pragma unroll
            for (int e = 0; e < 4; ++e) split_tf32(row(ki * 4 + e, m), hi[e], lo[e]);
        } else {
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float2 v;
                v.x = row(ki * 8 + e, m);
                v.y = row(ki * 8 + e + 1, m);
                const __nv_bfloat16 h0 = __float2bfloat16_rn(v.x), h1 = __float2bfloat16_rn(v.y);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(v.x - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(v.y - __bfloat162float(h1));
                hi[e / 2] = pack_bf16(h0, h1);
                lo[e / 2] = pack_bf16(l0, l1);
            }
        }
        *reinterpret_cast<uint4 *>(A + (size_t)(ki * (kM / 8) + m / 8) * 128 + (m % 8) * 16) =
            make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4 *>(A + (size_t)(ki * (kM / 8) + (m + kNR) / 8) * 128 + (m % 8) * 16) =
            make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// The MMAs of one K chunk: steps of 32 bytes of K (16 BF16 or 8 TF32 entries),
// N split at 256 (the instruction's limit); D columns [0, npad) of the CTA's
// tensor memory.  FP32 panels: B holds the panel's TF32 high parts, B + kc *
// npad * 4 its remainders, and each step multiplies A by both.
template <bool TF>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, const unsigned char *A, const unsigned char *B, int kc,
                                            int npad, bool first) {
    const uint32_t lboA = (kM / 8) * 128, lboB = (uint32_t)(npad / 8) * 128;
    const int steps = TF ? kc / 8 : kc / 16;
    const unsigned char *Blo = B + (size_t)kc * npad * 4;
    for (int ks = 0; ks < steps; ++ks) {
        const uint64_t ad = sdesc(A + (size_t)ks * 2 * lboA, lboA, 128);
        for (int n0 = 0; n0 < npad; n0 += 256) {
            const int nn = min(256, npad - n0);
            const size_t boff = (size_t)ks * 2 * lboB + (size_t)(n0 / 8) * 128;
            const uint64_t bd = sdesc(B + boff, lboB, 128);
            if constexpr (TF) {
                mma_tf32(tmem + (uint32_t)n0, ad, bd, idesc_tf32(kM, nn), !(first && ks == 0));
                mma_tf32(tmem + (uint32_t)n0, ad, sdesc(Blo + boff, lboB, 128), idesc_tf32(kM, nn), true);
            } else {
                mma_bf16(tmem + (uint32_t)n0, ad, bd, idesc_bf16(kM, nn), !(first && ks == 0));
            }
        }
    }
}

// Per-CTA state of the MMA pipeline, the same in every thread: mbarrier phases
// consumed so far and, in thread 0, what it issued and has not yet waited for.
struct Pipe {
    uint64_t *bfull, *mdone;
    uint32_t nb = 0, nm = 0;    // phases of bfull / mdone consumed
    bool mma_pending = false;   // a chunk's MMAs were due since the last wait on mdone
    // (thread 0) issued work whose completion it has not seen, and its phase
    bool copy_inflight = false, mma_inflight = false;
    uint32_t copy_phase = 0, mma_phase = 0;
};

// One GEMM D (128 x npad, tensor memory) = A B^T over K = kpad in chunks of
// kc_max<TF>() entries, single-buffered: the MMAs of a chunk finish before the
// next chunk (or the next item) is staged over them.  bulk_bytes(c, kc) > 0:
// thread 0 brings B in by one bulk copy from bulk_src(c) (else stage_b(c, kc)
// issues cp.async in every thread, and post_b(c, kc) then rewrites what the
// thread copied); stage_a(c, kc) writes A.  False when the CTA gave up.
template <bool TF, class BulkBytes, class BulkSrc, class StageB, class PostB, class StageA>
__device__ __forceinline__ bool item_gemm(uint32_t tmem, unsigned char *A, unsigned char *B, int kpad, int npad,
                                          BulkBytes bulk_bytes, BulkSrc bulk_src, StageB stage_b, PostB post_b,
                                          StageA stage_a, Pipe &p, const PipeCtl &ctl, volatile int *abort_flag) {
    constexpr int KC = kc_max<TF>();
    const int nch = (kpad + KC - 1) / KC;
    for (int c = 0; c < nch; ++c) {
        const int kc = min(KC, kpad - c * KC);
        if (p.mma_pending) {  // the buffers (and, at an item's start, D) are free again
            if (wait_bar(p.mdone, p.nm & 1, ctl, abort_flag)) p.mma_inflight = false;
            ++p.nm;
            p.mma_pending = false;
        }
        __syncthreads();
        if (*abort_flag) return false;
        const uint32_t bytes = bulk_bytes(c, kc);
        if (bytes > 0) {
            if (threadIdx.x == 0 && !ctl.withhold) {
                mb_arrive_expect_tx(p.bfull, bytes);
                bulk_copy(B, bulk_src(c), bytes, p.bfull);
                p.copy_inflight = true;
                p.copy_phase = p.nb;
            }
        } else {
            stage_b(c, kc);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        stage_a(c, kc);
        if (bytes == 0) {
            asm volatile("cp.async.wait_all;" ::: "memory");
            post_b(c, kc);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A (and B) visible to the tensor cores
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            const bool ok = bytes == 0 || wait_bar(p.bfull, p.nb & 1, ctl, abort_flag);
            if (bytes > 0 && ok) p.copy_inflight = false;
            if (ok) {
                tc_fence_after();
                issue_chunk<TF>(tmem, A, B, kc, npad, c == 0);
                mma_commit(p.mdone);
                p.mma_inflight = true;
                p.mma_phase = p.nm;
            }
        }
        if (bytes > 0) ++p.nb;
        p.mma_pending = true;
    }
    if (wait_bar(p.mdone, p.nm & 1, ctl, abort_flag)) p.mma_inflight = false;  // D complete
    ++p.nm;
    p.mma_pending = false;
    __syncthreads();
    return !*abort_flag;
}

// After a give-up: thread 0 lets the copy and the MMAs it issued and has not
// seen complete finish, before the buffers and the tensor memory are released.
__device__ __forceinline__ void pipe_drain(const Pipe &p) {
    if (threadIdx.x != 0) return;
    if (p.copy_inflight) drain_bar(p.bfull, p.copy_phase & 1);
    if (p.mma_inflight) drain_bar(p.mdone, p.mma_phase & 1);
}

// D (128 x ncols, FP32) -> out(row, m, value) for rows [0, nrows): the high part
// (lanes 0..63, warps 0-1) plus the remainder (lanes 64..127, warps 2-3, handed
// over through shared memory E), written by warps 0-1.
template <class Out>
__device__ __forceinline__ void epilogue(uint32_t tmem, int nrows, float *E, Out out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    tc_fence_after();
    for (int c0 = 0; c0 < nrows; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
        if (warp >= 2)
#pragma unroll
            for (int j = 0; j < 32; ++j) E[(32 * (warp - 2) + lane) * kEpiStride + j] = v[j];
        __syncthreads();
        if (warp < 2) {
            const int m = 32 * warp + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (c0 + j < nrows) out(c0 + j, m, v[j] + E[m * kEpiStride + j]);
        }
        __syncthreads();
    }
    tc_fence_before();  // the tensor-memory reads precede the next item's MMAs
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// projection: persistent CTAs over the column-cluster items (static round
// robin over items sorted by size, largest first)
// ---------------------------------------------------------------------------
constexpr int kProjCtasPerSm = 4;          // x kProjCols tensor-memory columns each
constexpr int kProjCols = kMrhsMaxRows;    // an item's rank rows (<= 128)
constexpr int kExpCtasPerSm = 8;
constexpr int kExpCols = kMaxLeaf;         // a leaf row cluster's rows (<= 64)
// Dynamic shared memory: the tiles (FP32 panels: TF32 high and low B tiles),
// raised so that no more CTAs fit on an SM than its 512 tensor-memory columns
// serve (228 KB per SM, 1 KB reserved per CTA)
template <bool TF>
constexpr size_t kProjSmem = std::max<size_t>((size_t)kABytes + (TF ? 2 : 1) * (size_t)kProjCols * 128, 52 * 1024);
template <bool TF>
constexpr size_t kExpSmem = std::max<size_t>((size_t)kABytes + (TF ? 2 : 1) * (size_t)kExpCols * 128 +
                                                  kc_max<TF>() * sizeof(MrhsSrc),
                                              26 * 1024);
static_assert((228 * 1024) / (kProjSmem<false> + 2048) <= 512 / kProjCols, "projection CTAs per SM vs tensor memory");
static_assert((228 * 1024) / (kProjSmem<true> + 2048) <= 512 / kProjCols, "projection CTAs per SM vs tensor memory");
static_assert((228 * 1024) / (kExpSmem<false> + 2048) <= 512 / kExpCols, "expansion CTAs per SM vs tensor memory");
static_assert((228 * 1024) / (kExpSmem<true> + 2048) <= 512 / kExpCols, "expansion CTAs per SM vs tensor memory");

// W tiles: BF16 (uint16_t) for BF16 panels; for FP32 panels each chunk's TF32
// high-part tile followed by its remainder tile (uint32_t)
template <bool TF> using WElem = typename std::conditional<TF, uint32_t, uint16_t>::type;

template <bool TF>
__global__ void __launch_bounds__(kThreads) k_mrhs_proj(int nsig, const MrhsSig *__restrict__ sigs,
                                                         const WElem<TF> *__restrict__ wt, const float *__restrict__ U,
                                                         float *__restrict__ T, PipeCtl ctl) {
    constexpr int KC = kc_max<TF>();
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tbase;
    __shared__ int abort_flag;
    unsigned char *A = smem, *B = smem + kABytes;
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&tbase, kProjCols);
    if (threadIdx.x == 0) {
        mb_init(&bars[0], 1);
        mb_init(&bars[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    Pipe p;
    p.bfull = &bars[0];
    p.mdone = &bars[1];
    for (int it = blockIdx.x; it < nsig; it += gridDim.x) {
        const MrhsSig sg = sigs[it];
        const bool ok = item_gemm<TF>(
            tmem, A, B, sg.kpad, sg.npad,
            [&](int, int kc) { return (uint32_t)kc * (uint32_t)sg.npad * (TF ? 8u : 2u); },
            [&](int c) { return (const void *)(wt + sg.woff + (size_t)c * KC * sg.npad * (TF ? 2 : 1)); },
            [](int, int) {}, [](int, int) {},
            [&](int c, int kc) {
                const int k0 = c * KC;
                stage_a<TF>(A, kc, [&](int kk, int m) {
                    const int j = k0 + kk;
                    return j < sg.xlen ? __ldg(U + (size_t)(sg.xbeg + j) * kNR + m) : 0.f;
                });
            },
            p, ctl, &abort_flag);
        if (!ok) break;
        epilogue(tmem, sg.R, reinterpret_cast<float *>(smem),
                 [&](int r, int m, float v) { T[(size_t)(sg.tbeg + r) * kNR + m] = v; });
    }
    if (abort_flag) pipe_drain(p);
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_free(tmem, kProjCols);
}

// ---------------------------------------------------------------------------
// expansion: persistent CTAs over the leaf row clusters (round robin)
// ---------------------------------------------------------------------------
template <bool TF>
__global__ void __launch_bounds__(kThreads) k_mrhs_expand(int nitems, const P2Desc *__restrict__ desc,
                                                           const MrhsSrc *__restrict__ src, const void *__restrict__ p2v,
                                                           const float *__restrict__ U, double *__restrict__ y,
                                                           int64_t ldy, int nrhs, PipeCtl ctl) {
    constexpr int KC = kc_max<TF>();
    constexpr int EPC = TF ? 4 : 8;  // panel entries per 16-byte piece
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tbase;
    __shared__ int abort_flag;
    unsigned char *A = smem, *B = smem + kABytes;
    MrhsSrc *ssrc = reinterpret_cast<MrhsSrc *>(smem + kABytes + (TF ? 2 : 1) * (size_t)kExpCols * 128);
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&tbase, kExpCols);
    if (threadIdx.x == 0) {
        mb_init(&bars[0], 1);
        mb_init(&bars[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    Pipe p;
    p.bfull = &bars[0];
    p.mdone = &bars[1];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const P2Desc d = desc[it];
        const int npad = (d.ylen + 15) & ~15, kpad = (d.ld + 15) & ~15;
        const MrhsSrc *sr = src + d.goff;
        const unsigned char *panel = (const unsigned char *)p2v + (size_t)d.off * (TF ? 4 : 2);
        const size_t prow = (size_t)d.ld * (TF ? 4 : 2);  // bytes per panel row
        const bool ok = item_gemm<TF>(
            tmem, A, B, kpad, npad, [](int, int) { return 0u; }, [](int) { return (const void *)nullptr; },
            [&](int c, int kc) {  // B: the panel rows, zero past |rho| and past ld
                const int k0 = c * KC;
                for (int t = threadIdx.x; t < npad * (kc / EPC); t += kThreads) {
                    const int i = t % npad, ki = t / npad, k = k0 + EPC * ki;
                    const bool in = i < d.ylen && k < d.ld;
                    cp_async16(B + (size_t)(ki * (npad / 8) + i / 8) * 128 + (i % 8) * 16,
                               in ? (const void *)(panel + (size_t)i * prow + (size_t)k * (TF ? 4 : 2))
                                  : (const void *)panel,
                               in);
                }
                if (threadIdx.x < kc) {  // the chunk's gather indices
                    const int k = k0 + threadIdx.x;
                    ssrc[threadIdx.x] = k < d.ld ? sr[k] : MrhsSrc{-1, 0};
                }
            },
            [&](int, int kc) {  // FP32 panels: split each piece this thread copied into TF32 parts
                if constexpr (TF) {
                    for (int t = threadIdx.x; t < npad * (kc / EPC); t += kThreads) {
                        const int i = t % npad, ki = t / npad;
                        const size_t off = (size_t)(ki * (npad / 8) + i / 8) * 128 + (i % 8) * 16;
                        const float4 v = *reinterpret_cast<const float4 *>(B + off);
                        uint4 hi, lo;
                        split_tf32(v.x, hi.x, lo.x);
                        split_tf32(v.y, hi.y, lo.y);
                        split_tf32(v.z, hi.z, lo.z);
                        split_tf32(v.w, hi.w, lo.w);
                        *reinterpret_cast<uint4 *>(B + off) = hi;
                        *reinterpret_cast<uint4 *>(B + (size_t)kc * npad * 4 + off) = lo;
                    }
                }
            },
            [&](int, int kc) {  // A: the operands G gathered from U, times their power of two
                __syncthreads();
                stage_a<TF>(A, kc, [&](int kk, int m) {
                    const MrhsSrc s = ssrc[kk];
                    return s.row < 0 ? 0.f : __ldg(U + (size_t)s.row * kNR + m) * pow2f_(s.exp);
                });
            },
            p, ctl, &abort_flag);
        if (!ok) break;
        epilogue(tmem, d.ylen, reinterpret_cast<float *>(smem), [&](int r, int m, float v) {
            if (m < nrhs) y[(int64_t)m * ldy + d.ybeg + r] = (double)v;
        });
    }
    if (abort_flag) pipe_drain(p);
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_free(tmem, kExpCols);
}

// x rows of U: U[p][k] = x[k * ldx + p] for k < nrhs, 0 above (cluster order)
__global__ void k_mrhs_prep(int64_t n, int nrhs, const double *__restrict__ x, int64_t ldx, float *__restrict__ U) {
    const int64_t total = n * kNR;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = q / kNR;
        const int k = (int)(q - p * kNR);
        U[q] = k < nrhs ? (float)x[(int64_t)k * ldx + p] : 0.f;
    }
}

}  // namespace

cudaError_t mrhs_prepare() {
    cudaError_t e = cudaSuccess;
    auto raise = [&](const void *k, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    raise((const void *)k_mrhs_proj<false>, kProjSmem<false>);
    raise((const void *)k_mrhs_expand<false>, kExpSmem<false>);
    raise((const void *)k_mrhs_proj<true>, kProjSmem<true>);
    raise((const void *)k_mrhs_expand<true>, kExpSmem<true>);
    return e;
}

void launch_mrhs_product(const DevIndex &ix, const MrhsIndex &mx, const DevPanels &P, const double *x, int64_t ldx,
                         double *y, int64_t ldy, int nrhs, cudaStream_t st) {
    const int64_t total = (int64_t)ix.n * kNR;
    const int pb = (int)std::min<int64_t>((total + 255) / 256, 8192);
    k_mrhs_prep<<<pb, 256, 0, st>>>(ix.n, nrhs, x, ldx, mx.U);
    const int gp = std::min(mx.nsig, ix.nsm * kProjCtasPerSm), ge = std::min<int>(ix.nleaves, ix.nsm * kExpCtasPerSm);
    if (mx.tf32) {  // FP32 panels
        if (mx.nsig > 0)
            k_mrhs_proj<true><<<gp, kThreads, kProjSmem<true>, st>>>(mx.nsig, mx.sigs, (const uint32_t *)mx.wt, mx.U,
                                                                     mx.U + (size_t)ix.n * kNR, mx.ctl);
        k_mrhs_expand<true><<<ge, kThreads, kExpSmem<true>, st>>>(ix.nleaves, ix.p2, mx.src, P.p2, mx.U, y, ldy, nrhs,
                                                                  mx.ctl);
        return;
    }
    if (mx.nsig > 0)
        k_mrhs_proj<false><<<gp, kThreads, kProjSmem<false>, st>>>(mx.nsig, mx.sigs, (const uint16_t *)mx.wt, mx.U,
                                                                   mx.U + (size_t)ix.n * kNR, mx.ctl);
    k_mrhs_expand<false><<<ge, kThreads, kExpSmem<false>, st>>>(ix.nleaves, ix.p2, mx.src, P.p2, mx.U, y, ldy, nrhs,
                                                                mx.ctl);
}

}  // namespace hmat_internal
