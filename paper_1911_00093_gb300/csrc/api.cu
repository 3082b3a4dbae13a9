// C ABI of the hmat library: upload, product, BiCG-STAB driver, introspection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "hmat.h"
#include "hmat_internal.h"
#include "kernels.h"
#include "handle.h"

using namespace hmat_internal;

namespace {

// Where a caller's vector lives: *on_device = false for host memory (the call
// stages it), true for device or managed memory the kernels can read directly.
// Device memory of another GPU than the handle's is rejected (HMAT_ERR_ARG):
// the kernels would otherwise read or write a peer's memory.
int vector_location(const void *p, int device, bool *on_device) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *on_device = false;
        return HMAT_OK;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != device) return HMAT_ERR_ARG;
    *on_device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    return HMAT_OK;
}

Store store_of(int precision) {
    switch (precision) {
    case HMAT_FP64: return Store::DF;
    case HMAT_FP64_DFMA: return Store::F64;
    case HMAT_FP32: return Store::F32;
    default: return Store::BF16;
    }
}

bool is_table1_precision(int precision) { return precision >= HMAT_M1_SINGLE && precision <= HMAT_M3_DENSE; }

}  // namespace

namespace {

// y = A~ x for one vector with the segments of an operator, everything on the device.
//   x_src != nullptr: source gathered through src_perm (or copied) into the operand copy; else it is ready
//   out_perm != nullptr: y written in original order
// The segments' expansions add up in y; the last one also leaves the shares of
// Algorithm 1's inner products in dpart (dotmode 1: r~ . v, v . v; 2: s . t, t . t).
// sys != nullptr: the work items of problems whose system sys[problem] has
// stopped are skipped (their rows of y are left as they were).
void enqueue_segments(const HmatSegment *seg, int nseg, const double *x_src, const int32_t *src_perm, double *y,
                      const int32_t *out_perm, const SolverScalars *skipS, int mode, cudaStream_t st,
                      const double *w = nullptr, int dotmode = 0, double *dpart = nullptr,
                      const SysScalars *sys = nullptr) {
    if (x_src) launch_prep(seg[0].store, seg[0].ix, x_src, src_perm, seg[0].P.xs, st);
    for (int k = 0; k < nseg; ++k) {
        launch_phase1(seg[k].store, seg[k].ix, seg[k].P, skipS, mode, st, sys);
        launch_reduce(seg[k].store, seg[k].ix, seg[k].P, skipS, mode, st, sys);
    }
    for (int k = 0; k < nseg; ++k) {
        const bool last = k == nseg - 1;
        launch_phase2(seg[k].store, seg[k].ix, seg[k].P, y, out_perm, k > 0, skipS, mode, st, last ? w : nullptr,
                      last ? dotmode : 0, dpart, sys);
    }
}

int product_launches(const HmatSegment *seg, int nseg) {
    int n = 1;  // operand copy
    for (int k = 0; k < nseg; ++k) n += (seg[k].ix.nbig + seg[k].ix.ntasks + seg[k].ix.ndirect) ? 3 : 2;
    return n;
}

// Device copies of a layout's indices (perm is the handle's).
int upload_index(hmat_t *h, const Layout &L, HmatSegment &g) {
    DevIndex &ix = g.ix;
    ix.n = (int32_t)L.n;
    ix.nleaves = L.nleaves;
    ix.nlr = (int32_t)L.lr.size();
    ix.nbig = (int32_t)L.red_big.size();
    ix.ntasks = (int32_t)L.red_tasks.size();
    ix.ndirect = (int32_t)L.red_direct.size();
    ix.max_leaf = L.max_leaf;
    ix.max_ld2 = L.max_ld2;
    ix.perm = h->perm;
    int32_t *gdst = nullptr, *red_big = nullptr, *red_tasks = nullptr, *tofs = nullptr;
    P1Desc *p1 = nullptr;
    XDst *xdst = nullptr;
    int32_t *xsel = nullptr;
    LrDesc *lr = nullptr;
    P2Desc *p2 = nullptr;
    double *tscale = nullptr;
    GroupDesc *groups = nullptr;
    RedDirect *red_direct = nullptr;
    int st;
    // the problem of every work item (pad fields): a batch's solver skips the
    // items of the problems whose systems have stopped
    std::vector<P1Desc> p1h = L.p1;
    std::vector<GroupDesc> grh = L.groups;
    std::vector<LrDesc> lrh = L.lr;
    auto prob_of = [&](int64_t row) {
        return (int32_t)(std::upper_bound(h->prob_off.begin(), h->prob_off.end(), row) - h->prob_off.begin() - 1);
    };
    for (size_t k = 0; k < p1h.size(); ++k) {
        p1h[k].pad[0] = prob_of(p1h[k].xbeg);
        for (int r = 0; r < p1h[k].rcnt; ++r) lrh[L.p1_runs[p1h[k].rbeg + r].q].pad = p1h[k].pad[0];
    }
    for (GroupDesc &gd : grh) {
        gd.pad[0] = prob_of(gd.p0);
        gd.pad[1] = 0;
    }
    std::vector<RedDirect> rdh = L.red_direct;
    for (size_t k = 0; k < rdh.size(); ++k) rdh[k].prob = lrh[L.red_direct_q[k]].pad;
    if ((st = h->upload(&p1, p1h.data(), sizeof(P1Desc) * p1h.size())) ||
        (st = h->upload(&xdst, L.xdst.data(), sizeof(XDst) * L.xdst.size())) ||
        (st = h->upload(&xsel, L.xsel.data(), 4 * L.xsel.size())) ||
        (st = h->upload(&lr, lrh.data(), sizeof(LrDesc) * lrh.size())) ||
        (st = h->upload(&gdst, L.gdst.data(), 4 * L.gdst.size())) ||
        (st = h->upload(&tofs, L.tofs.data(), 4 * L.tofs.size())) ||
        (st = h->upload(&red_big, L.red_big.data(), 4 * L.red_big.size())) ||
        (st = h->upload(&red_tasks, L.red_tasks.data(), 4 * L.red_tasks.size())) ||
        (st = h->upload(&red_direct, rdh.data(), sizeof(RedDirect) * rdh.size())) ||
        (st = h->upload(&p2, L.p2.data(), sizeof(P2Desc) * L.p2.size())) ||
        (st = h->upload(&tscale, L.tscale.data(), 8 * L.tscale.size())) ||
        (st = h->upload(&groups, grh.data(), sizeof(GroupDesc) * grh.size()))) {
        return st;
    }
    ix.p1 = p1; ix.tofs = tofs; ix.xdst = xdst; ix.xsel = xsel; ix.lr = lr; ix.gdst = gdst; ix.p2 = p2;
    ix.red_big = red_big; ix.red_tasks = red_tasks; ix.red_direct = red_direct;
    ix.tscale = L.tscale.empty() ? nullptr : tscale;
    ix.groups = groups;
    ix.ngroups = (int32_t)L.groups.size();
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    ix.nsm = std::max(1, nsm);
    g.partials_n = L.npart;
    g.glen = L.glen;
    h->index_bytes += (int64_t)(sizeof(P1Desc) * L.p1.size() + 4 * L.tofs.size() +
                                sizeof(XDst) * L.xdst.size() + 4 * L.xsel.size() + sizeof(LrDesc) * L.lr.size() +
                                4 * L.gdst.size() +
                                sizeof(P2Desc) * L.p2.size() + 4 * (L.red_big.size() + L.red_tasks.size()) +
                                sizeof(RedDirect) * L.red_direct.size() +
                                8 * L.tscale.size() +
                                sizeof(GroupDesc) * L.groups.size());
    return HMAT_OK;
}

// Typed panels of one store plus its work buffers; shared_xs != nullptr reuses
// another segment's operand copy of x (same cluster order, FP64).
int alloc_panels(hmat_t *h, const BlobView &v, const Layout &L, Store s, DevPanels &P, int64_t *bytes_out,
                 void *shared_xs = nullptr) {
    P.store = s;
    const size_t es = store_bytes(s);
    const size_t b1 = (size_t)L.p1_elems * es, b2 = (size_t)L.p2_elems * es;
    std::vector<char> host;
    try {
        host.resize(b1 + b2);
    } catch (const std::bad_alloc &) {
        return HMAT_ERR_NOMEM;
    }
    fill_panels(v, L, s, host.data(), host.data() + b1);
    void *q1 = nullptr, *p2 = nullptr;
    int st = h->upload(&q1, host.data(), b1);
    if (st) return st;
    st = h->upload(&p2, host.data() + b1, b2);
    if (st) return st;
    P.q1 = q1;
    P.p2 = p2;
    if (shared_xs) {
        P.xs = shared_xs;
    } else {
        st = h->alloc(&P.xs, (size_t)L.n * operand_bytes(s));
        if (st) return st;
    }
    st = h->alloc(&P.part, (size_t)std::max<int64_t>(L.npart, 1) * partial_bytes(s));
    if (st) return st;
    st = h->alloc(&P.g, (size_t)std::max<int64_t>(L.glen, 1) * operand_bytes(s));
    if (st) return st;
    CK(cudaMemset(P.g, 0, (size_t)std::max<int64_t>(L.glen, 1) * operand_bytes(s)));  // zero padding columns
    *bytes_out += (int64_t)(b1 + b2);
    return HMAT_OK;
}

// Indices of the tensor-core product for many right-hand sides (BF16 handles).
// The low-rank blocks are grouped by column cluster sigma (in (begin, end)
// order; blocks in their order) into work items of at most kMrhsMaxRows rank rows; an
// item's t rows are consecutive in T, and its W tile holds the rank rows of its
// blocks restricted to sigma -- the BF16 values of the phase-1 panels, W_m / 2^e
// -- as K-major 8 x 8 core matrices, core (n/8, k/8) at (k/8 * npad/8 + n/8),
// zero past |sigma| and past the item's rows.  Plus the U row and power of two
// feeding every operand slot of the expansion.
// FP32 -> TF32 on the host as the device's cvt.rna does it: round to nearest,
// ties away from zero, the low 13 bits cleared (finite values of pow2-scaled panels)
uint32_t tf32_bits(float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    return (b + 0x1000u) & ~0x1FFFu;
}
float bits_float(uint32_t b) {
    float v;
    std::memcpy(&v, &b, 4);
    return v;
}

int upload_mrhs_index(hmat_t *h, const BlobView &v, const Layout &L, bool tf32) {
    MrhsIndex &mx = h->mx;
    const size_t nlr = L.lr.size();
    // blob block and W exponent of each low-rank block, from its phase-1 slices
    std::vector<int64_t> blk(nlr, -1);
    std::vector<int32_t> ew(nlr, 0);
    for (size_t k = 0; k < L.p1.size(); ++k) {
        const P1Desc &d = L.p1[k];
        for (int r = 0; r < d.rcnt; ++r) {
            const P1Run &run = L.p1_runs[d.rbeg + r];
            const Layout::Slice &sl = L.p1_slices[L.p1_slice_ptr[k] + r];
            blk[run.q] = sl.block;
            ew[run.q] = sl.scale;
        }
    }
    std::vector<std::pair<std::pair<int64_t, int64_t>, int32_t>> order;  // ((begin, end) of sigma, block)
    order.reserve(nlr);
    for (size_t q = 0; q < nlr; ++q) {
        if (blk[q] < 0) return HMAT_ERR_BAD_LAYOUT;
        const int64_t *e = v.blocks + 8 * blk[q];
        order.push_back({{e[2], e[3]}, (int32_t)q});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const auto &a, const auto &b) { return a.first < b.first; });
    std::vector<int32_t> tbase(nlr, 0);
    std::vector<MrhsSig> sigs;
    std::vector<std::pair<size_t, size_t>> members;  // each item's range in `order`
    int64_t trows = 0, woff = 0;
    int32_t max_npad = 16;
    for (size_t a = 0; a < order.size();) {
        size_t b = a;
        int32_t R = 0;
        while (b < order.size() && order[b].first == order[a].first &&
               R + L.lr[order[b].second].rank <= kMrhsMaxRows) {
            tbase[order[b].second] = (int32_t)(trows + R);
            R += L.lr[order[b].second].rank;
            ++b;
        }
        if (b == a) return HMAT_ERR_UNSUPPORTED;  // (a rank above kMrhsMaxRows)
        MrhsSig sg;
        sg.woff = woff;
        sg.xbeg = (int32_t)order[a].first.first;
        sg.xlen = (int32_t)(order[a].first.second - order[a].first.first);
        sg.kpad = (sg.xlen + 15) & ~15;
        sg.npad = (R + 15) & ~15;
        sg.R = R;
        sg.tbeg = (int32_t)trows;
        sigs.push_back(sg);
        members.push_back({a, b});
        max_npad = std::max(max_npad, sg.npad);
        woff += (int64_t)sg.kpad * sg.npad * (tf32 ? 2 : 1);
        trows += R;
        a = b;
    }
    const int64_t zero_row = L.n + trows;
    if (zero_row + 1 > (int64_t(1) << 31) - 16) return HMAT_ERR_UNSUPPORTED;
    // the device takes the items round robin: largest (K x N) first
    std::vector<size_t> by_size(sigs.size());
    for (size_t k = 0; k < by_size.size(); ++k) by_size[k] = k;
    std::stable_sort(by_size.begin(), by_size.end(), [&](size_t x, size_t y) {
        return (int64_t)sigs[x].kpad * sigs[x].npad > (int64_t)sigs[y].kpad * sigs[y].npad;
    });
    // BF16 tiles: core (n/8, k/8) at (k/8 * npad/8 + n/8); TF32 (FP32 panels):
    // per 32-entry K chunk a high-part tile, core (n/8, kk/4) at (kk/4 * npad/8 +
    // n/8), then the remainders' tile of the same chunk
    std::vector<uint16_t> wt(tf32 ? 8 : (size_t)std::max<int64_t>(woff, 8), 0);
    std::vector<uint32_t> wt32(tf32 ? (size_t)std::max<int64_t>(woff, 8) : 8, 0);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t s = 0; s < (int64_t)sigs.size(); ++s) {
        const MrhsSig &sg = sigs[s];
        int32_t n = 0;
        for (size_t o = members[s].first; o < members[s].second; ++o) {
            const int32_t q = order[o].second;
            const int64_t *e = v.blocks + 8 * blk[q];
            const int64_t m = e[1] - e[0], cols = e[3] - e[2], r = e[5];
            const double *W = v.data + e[6] + m * r;  // W_m, r x cols row-major
            const double inv = std::ldexp(1.0, -ew[q]);
            for (int64_t l = 0; l < r; ++l, ++n)
                for (int64_t k = 0; k < cols; ++k) {
                    if (!tf32) {
                        wt[sg.woff + ((k / 8) * (sg.npad / 8) + n / 8) * 64 + (n % 8) * 8 + (k % 8)] =
                            bf16_bits(W[l * cols + k] * inv);
                        continue;
                    }
                    const float w = (float)(W[l * cols + k] * inv);  // the FP32 panel's value
                    const uint32_t hi = tf32_bits(w), lo = tf32_bits(w - bits_float(hi));
                    const int64_t c = k / 32, kk = k % 32, kc = std::min<int64_t>(32, sg.kpad - c * 32);
                    const int64_t at = sg.woff + c * 32 * 2 * sg.npad + ((kk / 4) * (sg.npad / 8) + n / 8) * 32 +
                                       (n % 8) * 4 + (kk % 4);
                    wt32[at] = hi;
                    wt32[at + kc * sg.npad] = lo;
                }
        }
    }
    std::vector<MrhsSrc> src((size_t)L.glen, MrhsSrc{(int32_t)zero_row, 0});
    for (size_t k = 0; k < L.p1.size(); ++k) {
        const P1Desc &d = L.p1[k];
        for (int e = 0; e < d.xdcnt; ++e) {
            const XDst &x = L.xdst[d.xdbeg + e];
            for (int j = 0; j < x.cnt; ++j)
                src[x.goff + j] = MrhsSrc{d.xbeg + (x.sel < 0 ? j : L.xsel[x.sel + j]), x.scale};
        }
    }
    for (size_t q = 0; q < nlr; ++q) {
        const LrDesc &d = L.lr[q];
        for (int k = 0; k < d.gcnt; ++k)
            for (int l = 0; l < d.rank; ++l)
                src[L.gdst[d.gbeg + k] + l] = MrhsSrc{(int32_t)(L.n + tbase[q] + l), d.scale};
    }
    MrhsSrc *dsrc = nullptr;
    MrhsSig *dsig = nullptr;
    void *dwt = nullptr;
    int st;
    std::vector<MrhsSig> sorted(sigs.size());
    for (size_t k = 0; k < by_size.size(); ++k) sorted[k] = sigs[by_size[k]];
    if ((st = h->upload(&dsrc, src.data(), sizeof(MrhsSrc) * src.size())) ||
        (st = h->upload(&dsig, sorted.data(), sizeof(MrhsSig) * sorted.size())) ||
        (st = tf32 ? h->upload(&dwt, wt32.data(), 4 * wt32.size()) : h->upload(&dwt, wt.data(), 2 * wt.size())))
        return st;
    CK(mrhs_prepare());
    mx.src = dsrc;
    mx.sigs = dsig;
    mx.wt = dwt;
    mx.tf32 = tf32;
    mx.nsig = (int32_t)sigs.size();
    mx.max_npad = max_npad;
    mx.urows = zero_row + 1;
    mx.ctl.status = h->status_dev;
    mx.ctl.wait_limit = kDefaultWaitCycles;
    h->index_bytes += (int64_t)(sizeof(MrhsSrc) * src.size() + sizeof(MrhsSig) * sigs.size());
    h->panel_bytes_mrhs = tf32 ? 4 * (int64_t)wt32.size() : 2 * (int64_t)wt.size();
    h->mrhs = true;
    return HMAT_OK;
}

void add_stats(hmat_t *h, const Layout &L, Store s) {
    h->stored_entries += L.stored_entries;
    h->phase1_entries += L.phase1_entries;
    h->phase2_entries += L.phase2_entries;
    h->phase1_bytes += L.phase1_entries * (int64_t)store_bytes(s);
    h->phase2_bytes += L.phase2_entries * (int64_t)store_bytes(s);
    h->partials_n += L.npart;
    h->rank_sum += L.rank_sum;
}

// A handle over a validated view; `offsets` delimits its problems (one problem:
// {0, n}; a block-diagonal batch: one range per problem).
int upload_view(const BlobView &v, int32_t precision, int32_t method3_c, const std::vector<int64_t> &offsets,
                hmat_handle *out) {
    int st = HMAT_OK;
    std::unique_ptr<hmat_t> hp;
    try {
        hp.reset(new hmat_t());
        hmat_t *h = hp.get();
        h->prob_off = offsets;
        Layout L;
        st = build_layout(v, L);
        if (st == HMAT_OK) st = check_layout(L);
        if (st != HMAT_OK) return st;
        CK(cudaGetDevice(&h->device));
        CK(cudaHostAlloc((void **)&h->status_host, sizeof(int32_t), cudaHostAllocMapped));
        *(volatile int32_t *)h->status_host = 0;
        CK(cudaHostGetDevicePointer((void **)&h->status_dev, h->status_host, 0));
        h->precision = precision;
        h->method3_c =
            (precision == HMAT_M3 || precision == HMAT_M3_TRUNC || precision == HMAT_M3_DENSE) ? method3_c : 0;
        h->n = L.n;
        int32_t *perm = nullptr;
        if ((st = h->upload(&perm, L.perm.data(), 4 * L.perm.size()))) return st;
        h->perm = perm;
        h->index_bytes = 4 * (int64_t)L.perm.size();

        if (!is_table1_precision(precision)) {
            // one layout; the FP64 operator shares its indices (DF panels, or the
            // F64 panels themselves for the FP64 FMA form)
            HmatSegment &g = h->seg[0];
            h->nseg = 1;
            g.store = store_of(precision);
            if ((st = upload_index(h, L, g))) return st;
            add_stats(h, L, g.store);
            if ((st = alloc_panels(h, v, L, g.store, g.P, &h->panel_bytes))) return st;
            h->seg64.ix = g.ix;
            h->seg64.partials_n = g.partials_n;
            h->seg64.glen = g.glen;
            if ((precision == HMAT_BF16 || precision == HMAT_FP32) &&
                (st = upload_mrhs_index(h, v, L, precision == HMAT_FP32)))
                return st;
            if (precision == HMAT_FP64 || precision == HMAT_FP64_DFMA) {
                h->seg64.store = g.store;
                h->seg64.P = g.P;
                h->panel_bytes64 = h->panel_bytes;
            } else {
                h->seg64.store = Store::DF;
                if ((st = alloc_panels(h, v, L, Store::DF, h->seg64.P, &h->panel_bytes64))) return st;
            }
        } else {
            // the paper's variant: derived segments, plus the FP64 H-matrix
            // (Method 1-Double) for the true residual
            DerivedSegment dseg[2];
            Store dstore[2];
            int nseg = 0;
            if ((st = derive_table1(v, precision, method3_c, dseg, dstore, &nseg))) return st;
            h->nseg = nseg;
            for (int k = 0; k < nseg; ++k) {
                Layout Lk;
                st = build_layout(dseg[k].view, Lk);
                if (st == HMAT_OK) st = check_layout(Lk);
                if (st != HMAT_OK) return st;
                HmatSegment &g = h->seg[k];
                g.store = dstore[k];
                if ((st = upload_index(h, Lk, g))) return st;
                add_stats(h, Lk, g.store);
                if ((st = alloc_panels(h, dseg[k].view, Lk, g.store, g.P, &h->panel_bytes,
                                       k > 0 ? h->seg[0].P.xs : nullptr)))
                    return st;
            }
            HmatSegment &g = h->seg64;
            g.store = Store::F64;
            if ((st = upload_index(h, L, g))) return st;
            if ((st = alloc_panels(h, v, L, g.store, g.P, &h->panel_bytes64))) return st;
        }
        // solver vectors and scratch
        const size_t nb = 8 * (size_t)L.n;
        double **vecs[] = {&h->b, &h->x, &h->r, &h->rt, &h->p, &h->v, &h->s, &h->t, &h->y, &h->stage_in, &h->stage_out};
        for (double **pp : vecs)
            if ((st = h->alloc(pp, nb))) return st;
        if ((st = h->alloc(&h->partials, sizeof(double) * 2 * (size_t)vec_blocks(L.n))) ||
            (st = h->alloc(&h->dpart, sizeof(double) * 2 * (size_t)phase2_items(h->seg[0].ix))) ||
            (st = h->alloc(&h->S, sizeof(SolverScalars)))) {
            return st;
        }
        CK(cudaMemset(h->S, 0, sizeof(SolverScalars)));
        CK(cudaMemset(h->p, 0, nb));
        CK(cudaMemset(h->v, 0, nb));
        CK(cudaHostAlloc((void **)&h->S_host, sizeof(SolverScalars), cudaHostAllocDefault));
        CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        CK(cudaDeviceSynchronize());
    } catch (const std::bad_alloc &) {
        return HMAT_ERR_NOMEM;
    }
    *out = hp.release();
    return HMAT_OK;
}

int upload_impl(const void *blob, size_t blob_bytes, int32_t precision, int32_t method3_c, hmat_handle *out) {
    if (!blob || !out) return HMAT_ERR_ARG;
    if (precision < HMAT_FP64 || precision > HMAT_M3_DENSE) return HMAT_ERR_ARG;
    *out = nullptr;
    BlobView v;
    int st = parse_blob(blob, blob_bytes, v);
    if (st != HMAT_OK) return st;
    return upload_view(v, precision, method3_c, {0, v.h->n}, out);
}

}  // namespace

extern "C" int hmat_upload(const void *blob, size_t blob_bytes, int32_t precision, hmat_handle *out) {
    return upload_impl(blob, blob_bytes, precision, 0, out);
}

extern "C" int hmat_upload_batch(const void *const *blobs, const size_t *blob_bytes, int32_t count, int32_t precision,
                                 int32_t method3_c, hmat_handle *out) {
    if (!blobs || !blob_bytes || !out || count < 1) return HMAT_ERR_ARG;
    if (precision < HMAT_FP64 || precision > HMAT_M3_DENSE) return HMAT_ERR_ARG;
    *out = nullptr;
    try {
        std::vector<BlobView> views(count);
        for (int32_t p = 0; p < count; ++p) {
            if (!blobs[p]) return HMAT_ERR_ARG;
            int st = parse_blob(blobs[p], blob_bytes[p], views[p]);
            if (st != HMAT_OK) return st;
        }
        CombinedBlob cb;
        int st = combine_blobs(views.data(), count, cb);
        if (st != HMAT_OK) return st;
        return upload_view(cb.view, precision, method3_c, cb.offsets, out);
    } catch (const std::bad_alloc &) {
        return HMAT_ERR_NOMEM;
    }
}

extern "C" int hmat_problems(hmat_handle h, int32_t *count, int64_t *offsets) {
    if (!h || !count) return HMAT_ERR_ARG;
    *count = (int32_t)h->prob_off.size() - 1;
    if (offsets)
        for (size_t k = 0; k < h->prob_off.size(); ++k) offsets[k] = h->prob_off[k];
    return HMAT_OK;
}

extern "C" int hmat_upload_ex(const void *blob, size_t blob_bytes, int32_t precision, int32_t method3_c,
                              hmat_handle *out) {
    return upload_impl(blob, blob_bytes, precision, method3_c, out);
}

extern "C" int hmat_destroy(hmat_handle h) {
    delete h;
    return HMAT_OK;
}

namespace {

int multi_matvec(hmat_t *h, const HmatSegment *seg, int nseg, const double *x, double *y, int32_t nrhs,
                 cudaStream_t st);

int matvec_impl(hmat_handle h, const double *x, double *y, int32_t nrhs, void *stream, bool fp64) {
    if (!h || !x || !y || nrhs < 1) return HMAT_ERR_ARG;
    if (int e = take_status(h)) return e;  // a wait of an earlier product ran out
    cudaStream_t st = (cudaStream_t)stream;
    const HmatSegment *seg = fp64 ? &h->seg64 : h->seg;
    const int nseg = fp64 ? 1 : h->nseg;
    if (nrhs >= 2 && ((!fp64 && h->mrhs) || (nseg == 1 && seg->store == Store::DF)))
        return multi_matvec(h, seg, nseg, x, y, nrhs, st);
    const int64_t n = h->n;
    bool dx = false, dy = false;
    if (int rc_ = vector_location(x, h->device, &dx)) return rc_;
    if (int rc_ = vector_location(y, h->device, &dy)) return rc_;
    for (int32_t k = 0; k < nrhs; ++k) {
        const double *xk = x + (size_t)k * n;
        double *yk = y + (size_t)k * n;
        const double *src = xk;
        if (!dx) {
            CK(cudaMemcpyAsync(h->stage_in, xk, 8 * n, cudaMemcpyHostToDevice, st));
            src = h->stage_in;
        }
        double *dst = dy ? yk : h->stage_out;
        enqueue_segments(seg, nseg, src, h->perm, dst, h->perm, nullptr, 0, st);
        CK(cudaGetLastError());
        if (!dy) {
            CK(cudaMemcpyAsync(yk, h->stage_out, 8 * n, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        } else if (!dx) {
            CK(cudaStreamSynchronize(st));  // the host input may be reused by the caller
        }
    }
    return HMAT_OK;
}

// One iteration of Algorithm 1 on the device (every kernel returns at once
// after the run has stopped).
void enqueue_iteration(hmat_t *h, int iter_limit, cudaStream_t st) {
    const int64_t n = h->n;
    const Store s = h->seg[0].store;
    void *xs = h->seg[0].P.xs;  // operand copy shared by the segments
    // v = A p, with alpha = rho / (r~ . v)
    launch_update_p(s, n, h->r, h->p, h->v, xs, h->S, st);
    enqueue_segments(h->seg, h->nseg, nullptr, nullptr, h->v, nullptr, h->S, 1, st, h->rt, 1, h->dpart);
    const int ndp = phase2_items(h->seg[h->nseg - 1].ix);  // work items of the expansion that leaves the shares
    launch_update_s(s, n, h->r, h->v, h->s, xs, h->S, h->partials, h->dpart, ndp, st);
    // t = A s, with omega = (t . s) / (t . t)
    enqueue_segments(h->seg, h->nseg, nullptr, nullptr, h->t, nullptr, h->S, 2, st, h->s, 2, h->dpart);
    launch_update_xr(n, h->x, h->p, h->s, h->t, h->r, h->rt, h->S, h->partials, h->dpart, ndp, iter_limit, st);
}

int read_scalars(hmat_t *h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h->S_host, h->S, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return HMAT_OK;
}

int ensure_graph(hmat_t *h, int k, int iter_limit) {
    if (h->graph && h->graph_k == k && h->graph_limit == iter_limit) return HMAT_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < k; ++i) enqueue_iteration(h, iter_limit, h->cap_stream);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (!hmat_internal::cuda_ok(e, "cudaStreamEndCapture")) return HMAT_ERR_CUDA;
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (!hmat_internal::cuda_ok(e, "cudaGraphInstantiate")) return HMAT_ERR_CUDA;
    h->graph_k = k;
    h->graph_limit = iter_limit;
    return HMAT_OK;
}

// A run of Algorithm 1 as one graph launch: a conditional WHILE node whose body
// is k iterations and the loop condition, so the host waits once per run
// instead of once per batch.  The condition stops after iter_limit / k + 2
// batches whatever the flag says (the iteration budget ends a run before).
int ensure_loop_graph(hmat_t *h, int k, int iter_limit) {
    if (h->loop_graph && h->loop_k == k && h->loop_limit == iter_limit) return HMAT_OK;
    if (h->loop_graph) {
        cudaGraphExecDestroy(h->loop_graph);
        h->loop_graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int i = 0; i < k; ++i) enqueue_iteration(h, iter_limit, h->cap_stream);
            launch_loop_condition(h->S, cond, iter_limit / k + 2, h->cap_stream);
            cudaGraph_t out = nullptr;
            e = cudaStreamEndCapture(h->cap_stream, &out);
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->loop_graph, g, 0);
    cudaGraphDestroy(g);
    if (!hmat_internal::cuda_ok(e, "device loop graph")) return HMAT_ERR_CUDA;
    h->loop_k = k;
    h->loop_limit = iter_limit;
    return HMAT_OK;
}

}  // namespace

extern "C" int hmat_matvec(hmat_handle h, const double *x, double *y, int32_t nrhs, void *stream) {
    return matvec_impl(h, x, y, nrhs, stream, false);
}

extern "C" int hmat_matvec_fp64(hmat_handle h, const double *x, double *y, int32_t nrhs, void *stream) {
    return matvec_impl(h, x, y, nrhs, stream, true);
}

extern "C" void hmat_solve_opts_default(hmat_solve_opts *o) {
    if (!o) return;
    o->tol = 1e-8;
    o->inner_tol = 0.0;
    o->maxit = 1000;
    o->max_restarts = 30;
    o->check_every = 1;
    o->use_graph = 2;
}

static int bicgstab_ex_impl(hmat_handle h, const double *b, double *x, const hmat_solve_opts *opts_in,
                            void *stream, hmat_solve_info *info) {
    if (!h || !b || !x) return HMAT_ERR_ARG;
    hmat_solve_opts o;
    hmat_solve_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0.0) || !(o.inner_tol >= 0.0) || o.maxit < 0 || o.max_restarts < 0 || o.check_every < 1)
        return HMAT_ERR_ARG;
    hmat_solve_info loc{};
    hmat_solve_info &inf = info ? *info : loc;
    std::memset(&inf, 0, sizeof(inf));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->n;
    bool db = false, dx = false;
    if (int rc_ = vector_location(b, h->device, &db)) return rc_;
    if (int rc_ = vector_location(x, h->device, &dx)) return rc_;
    // kernels per product (source operand, projection, reduction when some block
    // spans several leaf clusters, expansion) and per iteration (p update, two
    // products without operand preparation whose expansions also give alpha and
    // omega, s update, x/r update with the count of the next iteration)
    const int kProductLaunches = product_launches(h->seg, h->nseg);
    const int kProduct64Launches = product_launches(&h->seg64, 1);
    const int kIterationLaunches = 3 + 2 * (kProductLaunches - 1);
    const double *bsrc = b;
    if (!db) {
        CK(cudaMemcpyAsync(h->stage_in, b, 8 * n, cudaMemcpyHostToDevice, st));
        bsrc = h->stage_in;
    }
    launch_gather(n, h->perm, bsrc, h->b, st);
    int launches = 1;
    const double *xsrc = x;
    if (!dx) {
        CK(cudaMemcpyAsync(h->stage_out, x, 8 * n, cudaMemcpyHostToDevice, st));
        xsrc = h->stage_out;
    }
    launch_gather(n, h->perm, xsrc, h->x, st);
    CK(cudaMemsetAsync(h->S, 0, sizeof(SolverScalars), st));
    // ||x_0|| (a zero initial guess needs no product for r_0 = b), then ||b||
    // ||x_0||^2, then ||b||^2 (the second keeps the first in run_rnorm2): one read
    launch_residual(n, h->x, nullptr, h->r, h->rt, h->S, h->partials, -1, st);
    launch_residual(n, h->b, nullptr, h->r, h->rt, h->S, h->partials, -1, st);
    launches += 3;
    int rc = read_scalars(h, st);
    if (rc) return rc;
    const bool x0_zero = h->S_host->run_rnorm2 == 0.0;
    const double bnorm2 = h->S_host->rnorm2;
    int status = HMAT_OK;
    if (!std::isfinite(bnorm2)) {
        status = HMAT_ERR_NONFINITE;
        inf.relres_true = NAN;
    } else if (bnorm2 == 0.0) {
        CK(cudaMemsetAsync(h->x, 0, 8 * n, st));
        inf.relres_true = 0.0;
    } else {
        // first run: r_0 = b - A~ x_0 with the iterated operator (Algorithm 1); for
        // x_0 = 0 that is b exactly, without the product
        if (x0_zero) {
            launch_residual(n, h->b, nullptr, h->r, h->rt, h->S, h->partials, o.maxit, st);  // run 1 starts
            launches += 1;
        } else {
            enqueue_segments(h->seg, h->nseg, h->x, nullptr, h->y, nullptr, nullptr, 0, st);
            launch_residual(n, h->b, h->y, h->r, h->rt, h->S, h->partials, o.maxit, st);  // run 1 starts
            launches += kProductLaunches + 1;
        }
        CK(cudaGetLastError());
        // the state a run starts from is read from the device only when the host
        // does not know it already: ||r_0||^2 is ||b||^2 for x_0 = 0, and a restart
        // starts from the true residual just read (a start that fails -- budget --
        // leaves every kernel of the run a no-op, and the flag shows at the end)
        bool start_known = x0_zero;
        double start_rnorm2 = bnorm2;
        for (;;) {
            // a run: its stop threshold, then batches of iterations until its flag is set
            int start_flag = 0;
            if (!start_known) {
                if ((rc = read_scalars(h, st))) return rc;
                start_flag = h->S_host->flag;
                start_rnorm2 = h->S_host->rnorm2;
            }
            bool read_after_run = false;
            if (start_flag == 0) {
                double stop2 = std::max(o.tol * o.tol * bnorm2, o.inner_tol * o.inner_tol * start_rnorm2);
                CK(cudaMemcpyAsync(&h->S->stop2, &stop2, sizeof(double), cudaMemcpyHostToDevice, st));
                if (o.use_graph == 2) {  // the whole run on the device
                    if ((rc = ensure_loop_graph(h, o.check_every, o.maxit))) return rc;
                    CK(cudaMemsetAsync(&h->S->loops, 0, sizeof(int32_t), st));
                    CK(cudaGraphLaunch(h->loop_graph, st));
                }
                for (; o.use_graph != 2;) {
                    launches += o.check_every * kIterationLaunches;
                    if (o.use_graph) {
                        if ((rc = ensure_graph(h, o.check_every, o.maxit))) return rc;
                        CK(cudaGraphLaunch(h->graph, st));
                    } else {
                        for (int i = 0; i < o.check_every; ++i) enqueue_iteration(h, o.maxit, st);
                        CK(cudaGetLastError());
                    }
                    if ((rc = read_scalars(h, st))) return rc;
                    read_after_run = true;
                    if (h->S_host->flag != 0) break;
                }
            }
            // true residual with the FP64 H-matrix (Section 4.1.3); r~ = r for a
            // restart; the residual kernel first keeps the run's flag and ||r||^2
            enqueue_segments(&h->seg64, 1, h->x, nullptr, h->y, nullptr, nullptr, 0, st);
            launch_residual(n, h->b, h->y, h->r, h->rt, h->S, h->partials, -1, st);
            launches += kProduct64Launches + 1;
            inf.matvecs_fp64 += 1;
            if ((rc = read_scalars(h, st))) return rc;
            int flag = h->S_host->run_flag;
            if (start_flag == 0 && o.use_graph == 2) {
                launches += h->S_host->loops * (o.check_every * kIterationLaunches + 1);
                if (flag == 0) flag = HMAT_ERR_MAXIT;  // the loop bound ended it: count it as the budget
            } else if (start_flag != 0 && !read_after_run) {
                flag = start_flag;
            }
            inf.relres_inner = std::sqrt(h->S_host->run_rnorm2 / bnorm2);
            inf.iters = h->S_host->iters;
            const double rel = std::sqrt(h->S_host->rnorm2 / bnorm2);
            inf.relres_true = rel;
            if (flag != 1) { status = flag; break; }
            if (!std::isfinite(rel)) { status = HMAT_ERR_NONFINITE; break; }
            if (rel <= o.tol) { status = HMAT_OK; break; }
            if (inf.restarts >= o.max_restarts) { status = HMAT_ERR_MAXIT; break; }
            inf.restarts += 1;
            launch_count_iter(h->S, o.maxit, st);  // the restarted run starts
            launches += 1;
            start_known = true;
            start_rnorm2 = h->S_host->rnorm2;
        }
    }
    // products with the iterated operator: r_0, then two per iteration except a stop at ||s||
    double *xo = dx ? x : h->stage_out;
    launch_scatter(n, h->perm, h->x, xo, st);
    launches += 1;
    inf.launches = launches;
    if (!dx) CK(cudaMemcpyAsync(x, h->stage_out, 8 * n, cudaMemcpyDeviceToHost, st));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    inf.iters = h->S_host->iters;
    inf.matvecs = bnorm2 > 0.0 && std::isfinite(bnorm2) ? (x0_zero ? 0 : 1) + h->S_host->nmv : 0;
    inf.status = status;
    return status;
}

extern "C" int hmat_bicgstab(hmat_handle h, const double *b, double *x, double tol, int32_t maxit, void *stream,
                             hmat_solve_info *info) {
    hmat_solve_opts o;
    hmat_solve_opts_default(&o);
    o.tol = tol;
    o.maxit = maxit;
    return hmat_bicgstab_ex(h, b, x, &o, stream, info);
}

namespace {

// Buffers of the many-system solver for nrhs right-hand sides (kept while they fit).
int multi_ensure(hmat_t *h, int nrhs) {
    auto &m = h->multi;
    if (m.cap >= nrhs) return HMAT_OK;
    for (void *q : m.mine) h->release(q);
    m.mine.clear();
    if (m.graph) {
        cudaGraphExecDestroy(m.graph);
        m.graph = nullptr;
    }
    if (m.S_host) {
        cudaFreeHost(m.S_host);
        m.S_host = nullptr;
    }
    if (m.cols_host) {
        cudaFreeHost(m.cols_host);
        m.cols_host = nullptr;
    }
    m.cap = 0;
    const int nprob = (int)h->prob_off.size() - 1;
    const int nsys = nprob * nrhs;
    const size_t vb = 8 * (size_t)h->n * nrhs;
    int64_t maxn = 0;
    for (int p = 0; p < nprob; ++p) maxn = std::max(maxn, h->prob_off[p + 1] - h->prob_off[p]);
    const int bx = multi_blocks_x(maxn, nsys);
    double **vecs[] = {&m.b, &m.x, &m.r, &m.rt, &m.p, &m.v, &m.s, &m.t, &m.y, &m.stage};
    int st;
    for (double **pp : vecs) {
        if ((st = h->alloc(pp, vb))) return st;
        m.mine.push_back(*pp);
    }
    if ((st = h->alloc(&m.partials, sizeof(double) * 2 * (size_t)bx * nsys))) return st;
    m.mine.push_back(m.partials);
    if ((st = h->alloc(&m.S, sizeof(SysScalars) * (size_t)nsys))) return st;
    m.mine.push_back(m.S);
    if ((st = h->alloc(&m.cols, sizeof(int32_t) * (size_t)nrhs))) return st;
    m.mine.push_back(m.cols);
    std::vector<SysDesc> sys(nsys);
    for (int k = 0; k < nrhs; ++k)
        for (int p = 0; p < nprob; ++p) {
            SysDesc &d = sys[(size_t)k * nprob + p];
            d.off = (int64_t)k * h->n + h->prob_off[p];
            d.n = (int32_t)(h->prob_off[p + 1] - h->prob_off[p]);
            d.pad = 0;
        }
    if ((st = h->upload(&m.sys, sys.data(), sizeof(SysDesc) * sys.size()))) return st;
    m.mine.push_back(m.sys);
    CK(cudaMemset(m.S, 0, sizeof(SysScalars) * (size_t)nsys));
    CK(cudaMemset(m.p, 0, vb));
    CK(cudaMemset(m.v, 0, vb));
    CK(cudaHostAlloc((void **)&m.S_host, sizeof(SysScalars) * (size_t)nsys, cudaHostAllocDefault));
    CK(cudaHostAlloc((void **)&m.cols_host, sizeof(int32_t) * (size_t)nrhs, cudaHostAllocDefault));
    m.cap = nrhs;
    return HMAT_OK;
}

MultiGrid multi_grid(hmat_t *h, int nrhs) {
    MultiGrid g;
    const int nprob = (int)h->prob_off.size() - 1;
    int64_t maxn = 0;
    for (int p = 0; p < nprob; ++p) maxn = std::max(maxn, h->prob_off[p + 1] - h->prob_off[p]);
    g.nsys = nprob * nrhs;
    g.bx = multi_blocks_x(maxn, g.nsys);
    g.sys = h->multi.sys;
    g.S = h->multi.S;
    g.partials = h->multi.partials;
    return g;
}

// The many-column double-float product serves a one-segment double-float
// operator (the FP64 handle's own, every handle's FP64 copy but the Table 1
// variants') once its buffers exist.
bool mdf_serves(const hmat_t *h, const HmatSegment *seg, int nseg, int nrhs) {
    return nrhs >= 2 && nseg == 1 && seg->store == Store::DF && h->mdf.cap > 0;
}

// y(:, k) = A x(:, k) for every column, cluster order (a block-diagonal batch is one operator)
// The products of every system's column; skip_stopped (the products inside an
// iteration): the work items of problems whose system has stopped are skipped,
// so a batch costs less as its problems converge.
void multi_products(hmat_t *h, const HmatSegment *seg, int nseg, const double *x, double *y, int nrhs,
                    cudaStream_t st, bool skip_stopped = false) {
    if (seg == h->seg && h->mrhs && h->mx.U && nrhs >= 2) {  // tensor cores, 64 columns per pass
        for (int k0 = 0; k0 < nrhs; k0 += kMrhsCols)
            launch_mrhs_product(h->seg[0].ix, h->mx, h->seg[0].P, x + (size_t)k0 * h->n, h->n, y + (size_t)k0 * h->n,
                                h->n, std::min(kMrhsCols, nrhs - k0), st);
        return;
    }
    const size_t count = h->prob_off.size() - 1;  // problems: system (p, k) is k * count + p
    if (mdf_serves(h, seg, nseg, nrhs)) {  // double-float panels, kMdfCols columns per pass
        launch_mdf_product(seg->ix, seg->P, h->mdf, x, h->n, y, h->n, nrhs, nullptr,
                           skip_stopped ? h->multi.S : nullptr, 1, (int)count, st);
        return;
    }
    for (int k = 0; k < nrhs; ++k)
        enqueue_segments(seg, nseg, x + (size_t)k * h->n, nullptr, y + (size_t)k * h->n, nullptr, nullptr, 0, st,
                         nullptr, 0, nullptr, skip_stopped ? h->multi.S + (size_t)k * count : nullptr);
}

int multi_product_launches(hmat_t *h, const HmatSegment *seg, int nseg, int nrhs) {
    if (seg == h->seg && h->mrhs && h->mx.U && nrhs >= 2)
        return ((nrhs + kMrhsCols - 1) / kMrhsCols) * (h->mx.nsig > 0 ? 3 : 2);
    if (mdf_serves(h, seg, nseg, nrhs)) return mdf_launches(seg->ix, nrhs);
    return nrhs * product_launches(seg, nseg);
}

// buffers of the many-column double-float product (first use), sized by the
// FP64 copy's index (the handle's own double-float segment shares it); column
// strides are multiples of 32 entries (16-byte vector access)
int mdf_buffers(hmat_t *h) {
    auto &b = h->mdf;
    if (b.cap > 0 || h->seg64.store != Store::DF) return HMAT_OK;
    auto up = [](int64_t v) { return (std::max<int64_t>(v, 1) + 31) / 32 * 32; };
    const int64_t ld[3] = {up(h->n), up(h->seg64.partials_n), up(h->seg64.glen)};
    void **buf[3] = {&b.xs, &b.part, &b.g};
    for (int k = 0; k < 3; ++k) {
        const size_t bytes = 8 * (size_t)kMdfCols * ld[k];
        if (int st = h->alloc(buf[k], bytes)) return st;
        CK(cudaMemset(*buf[k], 0, bytes));  // the operands' padding columns stay zero
    }
    b.ldxs = ld[0];
    b.ldt = ld[1];
    b.ldg = ld[2];
    b.cap = kMdfCols;
    return HMAT_OK;
}

// buffers of the tensor-core product (first many-right-hand-side solve)
int mrhs_buffers(hmat_t *h) {
    if (!h->mrhs || h->mx.U) return HMAT_OK;
    float *U = nullptr;
    int st;
    if ((st = h->alloc(&U, sizeof(float) * kMrhsCols * (size_t)h->mx.urows))) return st;
    CK(cudaMemset(U, 0, sizeof(float) * kMrhsCols * (size_t)h->mx.urows));  // the zero row stays zero
    h->mx.U = U;
    return HMAT_OK;
}

void multi_iteration(hmat_t *h, const MultiGrid &g, int nrhs, int iter_limit, cudaStream_t st) {
    auto &m = h->multi;
    const MultiVecs v{m.x, m.r, m.rt, m.p, m.v, m.s, m.t};
    launch_miteration_vec(g, 0, v, iter_limit, st);  // p
    multi_products(h, h->seg, h->nseg, m.p, m.v, nrhs, st, true);
    launch_miteration_vec(g, 1, v, iter_limit, st);  // alpha
    launch_miteration_vec(g, 2, v, iter_limit, st);  // s
    multi_products(h, h->seg, h->nseg, m.s, m.t, nrhs, st, true);
    launch_miteration_vec(g, 3, v, iter_limit, st);  // omega
    launch_miteration_vec(g, 4, v, iter_limit, st);  // x, r
}

// The systems' scalars to the host: whether a system still iterates, and the
// columns (right-hand sides) with a system whose run has stopped and that
// awaits its true residual (ncols of them in multi.cols_host).
int multi_read(hmat_t *h, int nsys, int nrhs, cudaStream_t st, bool *running, int *ncols) {
    CK(cudaMemcpyAsync(h->multi.S_host, h->multi.S, sizeof(SysScalars) * (size_t)nsys, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *running = false;
    *ncols = 0;
    const int count = nsys / nrhs;  // problems: system (p, k) is k * count + p
    for (int k = 0; k < nrhs; ++k) {
        bool waits = false;
        for (int p = 0; p < count; ++p) {
            const SysScalars &q = h->multi.S_host[(size_t)k * count + p];
            if (q.state == 0 && q.flag == 0) *running = true;
            if (q.state == 0 && q.flag != 0) waits = true;
        }
        if (waits) h->multi.cols_host[(*ncols)++] = k;
    }
    return HMAT_OK;
}

// The true residuals (Section 4.1.3) of the systems whose run has stopped, in
// the ncols columns listed by multi_read: FP64 products of those columns, then
// acceptance, the run's error, or a restart from the true residual, decided per
// system on the device; the other systems are left as they are.
int multi_true_residuals(hmat_t *h, const MultiGrid &g, int ncols, const hmat_solve_opts &o, cudaStream_t st,
                         int *launches) {
    auto &m = h->multi;
    const HmatSegment *seg = &h->seg64;
    const int count = (int)(h->prob_off.size() - 1);
    // the many-column product over the list (its work items of the other
    // systems skipped), or one column at a time when a single right-hand side of
    // a one-problem handle is listed (the same bits, no unused column batch)
    if (seg->store == Store::DF && h->mdf.cap > 0 && (ncols >= 2 || count > 1)) {
        CK(cudaMemcpyAsync(m.cols, m.cols_host, sizeof(int32_t) * (size_t)ncols, cudaMemcpyHostToDevice, st));
        launch_mdf_product(seg->ix, seg->P, h->mdf, m.x, h->n, m.y, h->n, ncols, m.cols, m.S, 2, count, st);
        *launches += mdf_launches(seg->ix, ncols);
    } else {
        for (int j = 0; j < ncols; ++j) {
            const size_t k = (size_t)m.cols_host[j] * h->n;
            enqueue_segments(seg, 1, m.x + k, nullptr, m.y + k, nullptr, nullptr, 0, st);
        }
        *launches += ncols * product_launches(seg, 1);
    }
    launch_mresidual(g, 2, m.b, m.y, m.x, m.r, m.rt, o.tol, o.inner_tol, o.maxit, o.max_restarts, st);
    *launches += 1;
    CK(cudaGetLastError());
    return HMAT_OK;
}

// Several columns through the tensor-core product (seg = the handle's
// operator) or the many-column double-float product (a double-float operator):
// original order in and out, host or device pointers.
int multi_matvec(hmat_t *h, const HmatSegment *seg, int nseg, const double *x, double *y, int32_t nrhs,
                 cudaStream_t st) {
    int rc;
    if ((rc = multi_ensure(h, nrhs)) || (rc = mrhs_buffers(h)) || (rc = mdf_buffers(h))) return rc;
    auto &m = h->multi;
    const int64_t n = h->n;
    const size_t vb = 8 * (size_t)n * nrhs;
    bool dx = false, dy = false;
    if (int rc_ = vector_location(x, h->device, &dx)) return rc_;
    if (int rc_ = vector_location(y, h->device, &dy)) return rc_;
    const double *src = x;
    if (!dx) {
        CK(cudaMemcpyAsync(m.stage, x, vb, cudaMemcpyHostToDevice, st));
        src = m.stage;
    }
    launch_mgather(n, nrhs, h->perm, src, m.x, st);
    multi_products(h, seg, nseg, m.x, m.y, nrhs, st);
    double *dst = dy ? y : m.stage;
    launch_mscatter(n, nrhs, h->perm, m.y, dst, st);
    if (!dy) CK(cudaMemcpyAsync(y, m.stage, vb, cudaMemcpyDeviceToHost, st));
    CK(cudaGetLastError());
    if (!dx || !dy) {
        CK(cudaStreamSynchronize(st));
        return take_status(h);  // the call waited for its products
    }
    return HMAT_OK;
}

}  // namespace

static int bicgstab_multi_impl(hmat_handle h, const double *b, double *x, int32_t nrhs,
                               const hmat_solve_opts *opts_in, void *stream, hmat_solve_info *infos) {
    if (!h || !b || !x || nrhs < 1) return HMAT_ERR_ARG;
    hmat_solve_opts o;
    hmat_solve_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0.0) || !(o.inner_tol >= 0.0) || o.maxit < 0 || o.max_restarts < 0 || o.check_every < 1)
        return HMAT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = multi_ensure(h, nrhs);
    if (rc) return rc;
    if (nrhs >= 2 && ((rc = mrhs_buffers(h)) || (rc = mdf_buffers(h)))) return rc;
    auto &m = h->multi;
    const MultiGrid g = multi_grid(h, nrhs);
    const int64_t n = h->n;
    const size_t vb = 8 * (size_t)n * nrhs;
    bool db = false, dx = false;
    if (int rc_ = vector_location(b, h->device, &db)) return rc_;
    if (int rc_ = vector_location(x, h->device, &dx)) return rc_;
    // products per iteration: two per column; every launch of a product is counted
    const int per_pass = multi_product_launches(h, h->seg, h->nseg, nrhs);
    int launches = 0;
    const double *bsrc = b;
    if (!db) {
        CK(cudaMemcpyAsync(m.stage, b, vb, cudaMemcpyHostToDevice, st));
        bsrc = m.stage;
    }
    launch_mgather(n, nrhs, h->perm, bsrc, m.b, st);
    const double *xsrc = x;
    if (!dx) {  // stream order: the gather of b has read the stage buffer by then
        CK(cudaMemcpyAsync(m.stage, x, vb, cudaMemcpyHostToDevice, st));
        xsrc = m.stage;
    }
    launch_mgather(n, nrhs, h->perm, xsrc, m.x, st);
    launch_mresidual(g, 0, m.b, nullptr, m.x, m.r, m.rt, o.tol, o.inner_tol, o.maxit, o.max_restarts, st);
    multi_products(h, h->seg, h->nseg, m.x, m.y, nrhs, st);
    launch_mresidual(g, 1, m.b, m.y, m.x, m.r, m.rt, o.tol, o.inner_tol, o.maxit, o.max_restarts, st);
    launches += 4 + per_pass;
    CK(cudaGetLastError());
    // Each host read (after every batch of check_every iterations) lists the
    // systems whose run has stopped since.  With several right-hand sides and a
    // double-float FP64 copy their true residuals decide at once (accept, finish
    // on an error, or restart from the true residual) while the other systems
    // keep iterating, so no system waits for the slowest one; otherwise they
    // wait until no system iterates.  Either way every system goes through the
    // same steps: only the time at which its next run starts differs.
    const bool early = nrhs >= 2 && h->seg64.store == Store::DF && h->mdf.cap > 0;
    bool running = false;
    int nwait = 0;
    if ((rc = multi_read(h, g.nsys, nrhs, st, &running, &nwait))) return rc;
    while (running || nwait > 0) {
        if (nwait > 0 && (early || !running)) {
            if ((rc = multi_true_residuals(h, g, nwait, o, st, &launches))) return rc;
            if (!running) {  // nothing iterates: the read tells which systems restarted
                if ((rc = multi_read(h, g.nsys, nrhs, st, &running, &nwait))) return rc;
                continue;
            }
        }
        if (o.use_graph) {
            if (!(m.graph && m.graph_k == o.check_every && m.graph_limit == o.maxit && m.graph_nrhs == nrhs)) {
                if (m.graph) {
                    cudaGraphExecDestroy(m.graph);
                    m.graph = nullptr;
                }
                cudaGraph_t gr = nullptr;
                CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
                for (int i = 0; i < o.check_every; ++i) multi_iteration(h, g, nrhs, o.maxit, h->cap_stream);
                cudaError_t e = cudaStreamEndCapture(h->cap_stream, &gr);
                if (!hmat_internal::cuda_ok(e, "cudaStreamEndCapture")) return HMAT_ERR_CUDA;
                e = cudaGraphInstantiate(&m.graph, gr, 0);
                cudaGraphDestroy(gr);
                if (!hmat_internal::cuda_ok(e, "cudaGraphInstantiate")) return HMAT_ERR_CUDA;
                m.graph_k = o.check_every;
                m.graph_limit = o.maxit;
                m.graph_nrhs = nrhs;
            }
            CK(cudaGraphLaunch(m.graph, st));
        } else {
            for (int i = 0; i < o.check_every; ++i) multi_iteration(h, g, nrhs, o.maxit, st);
            CK(cudaGetLastError());
        }
        launches += o.check_every * (5 + 2 * per_pass);
        if ((rc = multi_read(h, g.nsys, nrhs, st, &running, &nwait))) return rc;
    }
    double *xo = dx ? x : m.stage;
    launch_mscatter(n, nrhs, h->perm, m.x, xo, st);
    launches += 1;
    if (!dx) CK(cudaMemcpyAsync(x, m.stage, vb, cudaMemcpyDeviceToHost, st));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    int worst = HMAT_OK;
    for (int k = 0; k < g.nsys; ++k) {
        const SysScalars &S = m.S_host[k];
        const int status = S.state == 1 ? HMAT_OK : (S.flag > 1 ? S.flag : HMAT_ERR_MAXIT);
        if (status != HMAT_OK && worst == HMAT_OK) worst = status;
        if (infos) {
            hmat_solve_info &inf = infos[k];
            std::memset(&inf, 0, sizeof(inf));
            inf.status = status;
            inf.iters = S.iters;
            inf.restarts = S.restarts;
            inf.matvecs = S.bnorm2 > 0.0 && std::isfinite(S.bnorm2) ? 1 + S.nmv : 0;
            inf.matvecs_fp64 = S.nmv64;
            inf.launches = launches;
            inf.relres_true = S.relres_true;
            inf.relres_inner = S.relres_inner;
        }
    }
    return worst;
}

namespace {

int gmres_ensure(hmat_t *h, int m) {
    auto &g = h->gm;
    if (g.m == m) return HMAT_OK;
    for (void *q : g.mine) h->release(q);
    g.mine.clear();
    if (g.graph) {
        cudaGraphExecDestroy(g.graph);
        g.graph = nullptr;
    }
    if (g.G_host) {
        cudaFreeHost(g.G_host);
        g.G_host = nullptr;
    }
    g.m = 0;
    const size_t n = (size_t)h->n;
    const int nb = vec_blocks(h->n);
    int st;
    double **vecs[] = {&g.w, &g.r, &g.b, &g.x, &g.x0, &g.r0, &g.d};
    if ((st = h->alloc(&g.V, 8 * n * (m + 1)))) return st;
    g.mine.push_back(g.V);
    for (double **pp : vecs) {
        if ((st = h->alloc(pp, 8 * n))) return st;
        g.mine.push_back(*pp);
    }
    if ((st = h->alloc(&g.part, sizeof(double) * (size_t)nb * (m + 1))) ||
        (st = h->alloc(&g.partials, sizeof(double) * (size_t)nb)) || (st = h->alloc(&g.G, sizeof(GmresState))))
        return st;
    g.mine.push_back(g.part);
    g.mine.push_back(g.partials);
    g.mine.push_back(g.G);
    CK(cudaHostAlloc((void **)&g.G_host, sizeof(GmresState), cudaHostAllocDefault));
    g.m = m;
    return HMAT_OK;
}

int gmres_read(hmat_t *h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h->gm.G_host, h->gm.G, offsetof(GmresState, H), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return HMAT_OK;
}

}  // namespace

static int gmres_impl(hmat_handle h, const double *b, double *x, int32_t m, const hmat_solve_opts *opts_in,
                      void *stream, hmat_solve_info *info) {
    if (!h || !b || !x || m < 1 || m > kGmresMaxM) return HMAT_ERR_ARG;
    hmat_solve_opts o;
    hmat_solve_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0.0) || !(o.inner_tol >= 0.0) || o.maxit < 0 || o.max_restarts < 0) return HMAT_ERR_ARG;
    hmat_solve_info loc{};
    hmat_solve_info &inf = info ? *info : loc;
    std::memset(&inf, 0, sizeof(inf));
    cudaStream_t st = (cudaStream_t)stream;
    int rc = gmres_ensure(h, m);
    if (rc) return rc;
    auto &g = h->gm;
    const int64_t n = h->n;
    bool db = false, dx = false;
    if (int rc_ = vector_location(b, h->device, &db)) return rc_;
    if (int rc_ = vector_location(x, h->device, &dx)) return rc_;
    const int per_product = product_launches(h->seg, h->nseg), per_product64 = product_launches(&h->seg64, 1);
    int launches = 0, products = 0;
    // state: zero, then the scratch pointer
    CK(cudaMemsetAsync(g.G, 0, sizeof(GmresState), st));
    CK(cudaMemcpyAsync(&g.G->partials, &g.partials, sizeof(double *), cudaMemcpyHostToDevice, st));
    const double *bsrc = b;
    if (!db) {
        CK(cudaMemcpyAsync(h->stage_in, b, 8 * n, cudaMemcpyHostToDevice, st));
        bsrc = h->stage_in;
    }
    launch_gather(n, h->perm, bsrc, g.b, st);
    const double *xsrc = x;
    if (!dx) {
        CK(cudaMemcpyAsync(h->stage_out, x, 8 * n, cudaMemcpyHostToDevice, st));
        xsrc = h->stage_out;
    }
    launch_gather(n, h->perm, xsrc, g.x, st);
    launch_g_residual(n, 2, g.b, nullptr, nullptr, g.G, o.tol, o.inner_tol, st);
    launches += 3;
    if ((rc = gmres_read(h, st))) return rc;
    const double bnorm2 = g.G_host->bnorm2;
    int status = HMAT_OK;
    if (!std::isfinite(bnorm2)) {
        status = HMAT_ERR_NONFINITE;
        inf.relres_true = NAN;
    } else if (bnorm2 == 0.0) {
        CK(cudaMemsetAsync(g.x, 0, 8 * n, st));
    } else {
        // the first run starts from the true residual r_0 = b - A64 x_0
        enqueue_segments(&h->seg64, 1, g.x, nullptr, g.w, nullptr, nullptr, 0, st);
        launch_g_residual(n, 3, g.b, g.w, g.r0, g.G, o.tol, o.inner_tol, st);
        launches += per_product64 + 1;
        if ((rc = gmres_read(h, st))) return rc;
        for (;;) {
            const double rel = g.G_host->relres_true;
            inf.relres_true = rel;
            if (!std::isfinite(rel)) { status = HMAT_ERR_NONFINITE; break; }
            if (rel <= o.tol) { status = HMAT_OK; break; }
            // a run on the correction equation A~ d = r_0 from x_0 = x
            CK(cudaMemcpyAsync(g.x0, g.x, 8 * n, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(g.r, g.r0, 8 * n, cudaMemcpyDeviceToDevice, st));
            for (;;) {
                // a cycle of at most m Arnoldi steps, one graph launch
                launch_g_start_cycle(n, g.r, g.V, g.G, m, o.maxit, st);
                launches += 2;
                if (!(g.graph && g.graph_m == m && g.graph_limit == o.maxit)) {
                    if (g.graph) {
                        cudaGraphExecDestroy(g.graph);
                        g.graph = nullptr;
                    }
                    cudaGraph_t gr = nullptr;
                    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
                    for (int jj = 0; jj < m; ++jj) {
                        enqueue_segments(h->seg, h->nseg, g.V + (size_t)jj * n, nullptr, g.w, nullptr, &g.G->s, 1,
                                         h->cap_stream);
                        launch_g_arnoldi(n, g.V, (int)n, g.w, g.G, jj, m, o.maxit, g.part, h->cap_stream);
                    }
                    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &gr);
                    if (!hmat_internal::cuda_ok(e, "cudaStreamEndCapture")) return HMAT_ERR_CUDA;
                    e = cudaGraphInstantiate(&g.graph, gr, 0);
                    cudaGraphDestroy(gr);
                    if (!hmat_internal::cuda_ok(e, "cudaGraphInstantiate")) return HMAT_ERR_CUDA;
                    g.graph_m = m;
                    g.graph_limit = o.maxit;
                }
                CK(cudaGraphLaunch(g.graph, st));
                launch_g_finish_cycle(n, g.V, (int)n, g.x, g.G, m, st);
                launches += m * (per_product + 8) + 2;
                if ((rc = gmres_read(h, st))) return rc;
                if (g.G_host->run_over || g.G_host->status != HMAT_OK) break;
                // the next cycle starts from r_0 - A~ (x - x_0)
                launch_g_diff(n, g.x, g.x0, g.d, st);
                enqueue_segments(h->seg, h->nseg, g.d, nullptr, g.w, nullptr, nullptr, 0, st);
                launch_g_residual(n, 1, g.r0, g.w, g.r, g.G, o.tol, o.inner_tol, st);
                launches += per_product + 2;
                products += 1;
            }
            // true residual with the FP64 H-matrix (Section 4.1.3): accept, or the next run's r_0
            enqueue_segments(&h->seg64, 1, g.x, nullptr, g.w, nullptr, nullptr, 0, st);
            launch_g_residual(n, 3, g.b, g.w, g.r0, g.G, o.tol, o.inner_tol, st);
            launches += per_product64 + 1;
            if ((rc = gmres_read(h, st))) return rc;
            inf.relres_true = g.G_host->relres_true;
            if (!std::isfinite(g.G_host->relres_true)) { status = HMAT_ERR_NONFINITE; break; }
            if (g.G_host->relres_true <= o.tol) { status = HMAT_OK; break; }
            if (g.G_host->status != HMAT_OK) { status = g.G_host->status; break; }
            if (inf.restarts >= o.max_restarts) { status = HMAT_ERR_MAXIT; break; }
            inf.restarts += 1;
        }
    }
    double *xo = dx ? x : h->stage_out;
    launch_scatter(n, h->perm, g.x, xo, st);
    launches += 1;
    if (!dx) CK(cudaMemcpyAsync(x, h->stage_out, 8 * n, cudaMemcpyDeviceToHost, st));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    inf.status = status;
    inf.iters = g.G_host->it;
    inf.matvecs = g.G_host->s.nmv + products;
    inf.matvecs_fp64 = g.G_host->nmv64;
    inf.launches = launches;
    inf.relres_inner = bnorm2 > 0.0 ? g.G_host->rnorm / std::sqrt(bnorm2) : 0.0;
    return status;
}

extern "C" int hmat_info(hmat_handle h, hmat_handle_info *out) {
    if (!h || !out) return HMAT_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->precision = h->precision;
    out->nleaves = h->seg64.ix.nleaves;
    out->panel_bytes = h->panel_bytes;
    out->panel_bytes_fp64 = h->panel_bytes64;
    out->index_bytes = h->index_bytes;
    out->stored_entries = h->stored_entries;
    out->phase1_entries = h->phase1_entries;
    out->phase2_entries = h->phase2_entries;
    out->partials = h->partials_n;
    out->rank_sum = h->rank_sum;
    out->phase1_bytes = h->phase1_bytes;
    out->phase2_bytes = h->phase2_bytes;
    out->stored_bytes = h->phase1_bytes + h->phase2_bytes;
    out->segments = h->nseg;
    out->method3_c = h->method3_c;
    return HMAT_OK;
}

static int time_matvec_impl(hmat_handle h, int32_t iters, int32_t fp64, void *stream, double *ms_out) {
    if (!h || !ms_out || iters < 1) return HMAT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const HmatSegment *seg = fp64 ? &h->seg64 : h->seg;
    const int nseg = fp64 ? 1 : h->nseg;
    const int64_t n = h->n;
    // a fixed source vector: x = 1 in cluster order
    std::vector<double> ones(n, 1.0);
    CK(cudaMemcpyAsync(h->stage_in, ones.data(), 8 * n, cudaMemcpyHostToDevice, st));
    // the launches of a solver product: the expansion also leaves the shares of
    // Algorithm 1's inner products (in the handle's solver scratch)
    cudaEvent_t ev[5];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    double tot[5] = {0, 0, 0, 0, 0};
    for (int it = 0; it < iters; ++it) {
        CK(cudaEventRecord(ev[0], st));
        launch_prep(seg[0].store, seg[0].ix, h->stage_in, nullptr, seg[0].P.xs, st);
        CK(cudaEventRecord(ev[1], st));
        for (int k = 0; k < nseg; ++k) launch_phase1(seg[k].store, seg[k].ix, seg[k].P, nullptr, 0, st);
        CK(cudaEventRecord(ev[2], st));
        for (int k = 0; k < nseg; ++k) launch_reduce(seg[k].store, seg[k].ix, seg[k].P, nullptr, 0, st);
        CK(cudaEventRecord(ev[3], st));
        for (int k = 0; k < nseg; ++k) {
            const bool last = k == nseg - 1;
            launch_phase2(seg[k].store, seg[k].ix, seg[k].P, h->stage_out, nullptr, k > 0, nullptr, 0, st,
                          last ? h->stage_in : nullptr, last ? 1 : 0, h->dpart);
        }
        CK(cudaEventRecord(ev[4], st));
        CK(cudaEventSynchronize(ev[4]));
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
            tot[k] += ms;
        }
        float all = 0.f;
        CK(cudaEventElapsedTime(&all, ev[0], ev[4]));
        tot[4] += all;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    for (int k = 0; k < 5; ++k) ms_out[k] = tot[k] / iters;
    return HMAT_OK;
}

extern "C" const char *hmat_strerror(int status) {
    switch (status) {
    case HMAT_OK: return "ok";
    case HMAT_ERR_ARG: return "invalid argument";
    case HMAT_ERR_BAD_LAYOUT: return "serialized H-matrix failed validation";
    case HMAT_ERR_NOMEM: return "out of memory";
    case HMAT_ERR_CUDA: return "CUDA runtime error";
    case HMAT_ERR_BREAKDOWN_RHO: return "BiCG-STAB breakdown: rho = 0";
    case HMAT_ERR_BREAKDOWN_OMEGA: return "BiCG-STAB breakdown: omega = 0";
    case HMAT_ERR_MAXIT: return "iteration budget exhausted";
    case HMAT_ERR_NONFINITE: return "non-finite value";
    case HMAT_ERR_RANGE: return "value out of range for the precision form";
    case HMAT_ERR_UNSUPPORTED: return "unsupported size";
    case HMAT_ERR_TIMEOUT: return "a bounded wait inside a kernel ran out (the product was abandoned)";
    default: return "unknown status";
    }
}

std::string &hmat_internal::last_cuda_error() {
    static thread_local std::string s;
    return s;
}

extern "C" const char *hmat_last_cuda_error(void) { return hmat_internal::last_cuda_error().c_str(); }

// ---- entry points that report the timeouts of bounded device waits ----
namespace {
// a synchronous call's own status, unless one of its products (or an earlier
// asynchronous product) recorded a timeout: then that product's result was not
// valid and whatever followed from it is reported as the timeout
int with_status(hmat_handle h, int rc, hmat_solve_info *info, int ninfo) {
    const int e = take_status(h);
    if (e != HMAT_OK) {
        rc = e;
        for (int k = 0; info && k < ninfo; ++k) info[k].status = e;
    }
    return rc;
}
}  // namespace

extern "C" int hmat_bicgstab_ex(hmat_handle h, const double *b, double *x, const hmat_solve_opts *opts_in, void *stream,
                                hmat_solve_info *info) {
    if (h)
        if (int e = take_status(h)) return e;
    const int rc = bicgstab_ex_impl(h, b, x, opts_in, stream, info);
    return h ? with_status(h, rc, info, 1) : rc;
}

extern "C" int hmat_bicgstab_multi(hmat_handle h, const double *b, double *x, int32_t nrhs,
                                   const hmat_solve_opts *opts_in, void *stream, hmat_solve_info *infos) {
    if (h)
        if (int e = take_status(h)) return e;
    const int rc = bicgstab_multi_impl(h, b, x, nrhs, opts_in, stream, infos);
    return h ? with_status(h, rc, infos, nrhs > 0 ? nrhs : 0) : rc;
}

extern "C" int hmat_gmres(hmat_handle h, const double *b, double *x, int32_t m, const hmat_solve_opts *opts_in,
                          void *stream, hmat_solve_info *info) {
    if (h)
        if (int e = take_status(h)) return e;
    const int rc = gmres_impl(h, b, x, m, opts_in, stream, info);
    return h ? with_status(h, rc, info, 1) : rc;
}

extern "C" int hmat_time_matvec(hmat_handle h, int32_t iters, int32_t fp64, void *stream, double *ms_out) {
    if (h)
        if (int e = take_status(h)) return e;
    const int rc = time_matvec_impl(h, iters, fp64, stream, ms_out);
    return h ? with_status(h, rc, nullptr, 0) : rc;
}

extern "C" int hmat_check(hmat_handle h, void *stream) {
    if (!h) return HMAT_ERR_ARG;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return take_status(h);
}

extern "C" int hmat_set_wait_limit(hmat_handle h, int64_t cycles, int32_t withhold) {
    if (!h || cycles < 1) return HMAT_ERR_ARG;
    h->mx.ctl.wait_limit = cycles;
    h->mx.ctl.withhold = withhold ? 1 : 0;
    // solver graphs captured the old values: capture them again at their next use
    if (h->multi.graph) {
        cudaGraphExecDestroy(h->multi.graph);
        h->multi.graph = nullptr;
        h->multi.graph_k = 0;
        h->multi.graph_limit = -1;
    }
    return HMAT_OK;
}

// ---- the projection's plan, chosen by measurement ----
namespace {

constexpr int kTuneBuckets = 5;
constexpr int kBucketVec[kTuneBuckets] = {32, 64, 128, 256, 0};  // column vectors per row (0: no bound)
constexpr int kTuneSizes[3] = {64, 128, 256};

int bucket_of(int nvec) {
    for (int b = 0; b < kTuneBuckets - 1; ++b)
        if (nvec <= kBucketVec[b]) return b;
    return kTuneBuckets - 1;
}

// The plan of the sorted work list: one run per stretch of buckets with the same size.
void sorted_plan(DevIndex &t, const int32_t (&begin)[kTuneBuckets + 1], const int (&nt)[kTuneBuckets]) {
    t.nruns = 0;
    for (int b = 0; b < kTuneBuckets; ++b) {
        const int cnt = begin[b + 1] - begin[b];
        if (cnt == 0) continue;
        if (t.nruns > 0 && t.runs[t.nruns - 1].nt == nt[b]) {
            t.runs[t.nruns - 1].count += cnt;
        } else {
            t.runs[t.nruns].begin = begin[b];
            t.runs[t.nruns].count = cnt;
            t.runs[t.nruns].nt = nt[b];
            ++t.nruns;
        }
    }
}

int tune_segment(hmat_t *h, HmatSegment &g, int reps, cudaStream_t st, hmat_tune_report *rep) {
    DevIndex &ix = g.ix;
    if (table1_store(g.store) || ix.nleaves == 0) return HMAT_OK;
    const int VW = g.store == Store::BF16 ? 8 : g.store == Store::F32 ? 4 : 2;
    std::vector<P1Desc> d((size_t)ix.nleaves);
    CK(cudaMemcpy(d.data(), ix.p1, sizeof(P1Desc) * d.size(), cudaMemcpyDeviceToHost));
    // the work list sorted by bucket (stable: cluster order inside a bucket)
    std::vector<P1Desc> sorted;
    sorted.reserve(d.size());
    int32_t begin[kTuneBuckets + 1] = {0};
    for (int b = 0; b < kTuneBuckets; ++b) {
        begin[b] = (int32_t)sorted.size();
        for (const P1Desc &e : d)
            if (bucket_of(e.ld / VW) == b) sorted.push_back(e);
    }
    begin[kTuneBuckets] = (int32_t)sorted.size();
    P1Desc *dsorted = nullptr;
    int st2;
    if ((st2 = h->upload(&dsorted, sorted.data(), sizeof(P1Desc) * sorted.size()))) return st2;
    DevIndex base = ix;
    base.nruns = 0;
    base.p1_sorted = nullptr;
    const float t_default = time_phase1(g.store, base, g.P, reps, st);
    if (t_default < 0.f) return HMAT_ERR_CUDA;
    const int def = phase1_default_threads(g.store);
    int nt[kTuneBuckets];
    for (int &v : nt) v = def;
    double us[kTuneBuckets][3] = {};
    DevIndex t = base;
    t.p1_sorted = dsorted;
    sorted_plan(t, begin, nt);
    float best = time_phase1(g.store, t, g.P, reps, st);
    for (int pass = 0; pass < 2; ++pass) {
        bool changed = false;
        for (int b = 0; b < kTuneBuckets; ++b) {
            if (begin[b + 1] == begin[b]) continue;
            for (int c = 0; c < 3; ++c) {
                if (kTuneSizes[c] == nt[b]) {
                    us[b][c] = best;
                    continue;
                }
                int trial[kTuneBuckets];
                for (int k = 0; k < kTuneBuckets; ++k) trial[k] = nt[k];
                trial[b] = kTuneSizes[c];
                sorted_plan(t, begin, trial);
                const float tt = time_phase1(g.store, t, g.P, reps, st);
                if (tt < 0.f) return HMAT_ERR_CUDA;
                us[b][c] = tt;
                if (tt < best * 0.99f) {
                    best = tt;
                    nt[b] = kTuneSizes[c];
                    changed = true;
                }
            }
        }
        if (!changed) break;
    }
    const bool use_sorted = best < t_default * 0.98f;
    if (use_sorted) {
        sorted_plan(ix, begin, nt);
        ix.p1_sorted = dsorted;
    } else {
        ix.nruns = 0;
        ix.p1_sorted = nullptr;
    }
    if (rep) {
        rep->nbuckets = kTuneBuckets;
        rep->sorted = use_sorted ? 1 : 0;
        rep->default_us = t_default;
        rep->tuned_us = use_sorted ? best : t_default;
        for (int b = 0; b < kTuneBuckets; ++b) {
            rep->bucket[b].vec_max = kBucketVec[b];
            rep->bucket[b].clusters = begin[b + 1] - begin[b];
            rep->bucket[b].threads = use_sorted ? nt[b] : def;
            rep->bucket[b].pad = 0;
            for (int c = 0; c < 3; ++c) rep->bucket[b].us[c] = us[b][c];
        }
    }
    return HMAT_OK;
}

}  // namespace

extern "C" int hmat_autotune(hmat_handle h, int32_t reps, void *stream, hmat_tune_report *out) {
    if (!h || reps < 1) return HMAT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (out) std::memset(out, 0, sizeof(*out));
    int rc = tune_segment(h, h->seg[0], reps, st, out);
    if (rc) return rc;
    const bool fp64_form = h->precision == HMAT_FP64 || h->precision == HMAT_FP64_DFMA;
    if (fp64_form) h->seg64.ix = h->seg[0].ix;  // the same operator
    else if ((rc = tune_segment(h, h->seg64, reps, st, nullptr))) return rc;
    // solver graphs captured the old launches: capture them again at their next use
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; h->graph_k = 0; h->graph_limit = -1; }
    if (h->loop_graph) { cudaGraphExecDestroy(h->loop_graph); h->loop_graph = nullptr; h->loop_k = 0; h->loop_limit = -1; }
    if (h->multi.graph) { cudaGraphExecDestroy(h->multi.graph); h->multi.graph = nullptr; h->multi.graph_k = 0; h->multi.graph_limit = -1; }
    if (h->gm.graph) { cudaGraphExecDestroy(h->gm.graph); h->gm.graph = nullptr; h->gm.graph_m = 0; h->gm.graph_limit = -1; }
    return HMAT_OK;
}
