// The paper's own precision variants (Section 3, Table 1), derived on the host
// at upload from the FP64 H-matrix as Section 4.1.3 prescribes: generate in
// FP64, factor the low-rank blocks (Methods 2 and 3), then convert.
//
// A variant is run as one or two segments over the same cluster tree.  Each
// segment is a derived block list (not a cover of I x J) whose entries all use
// one arithmetic class; the product is y = sum over segments of P_s g_s, the
// second segment adding into the y the first one wrote.
//
//   variant          segment A                       segment B
//   Method 1-Single  all blocks, class S             -
//   Method 1-Mixed   dense blocks, class M           low-rank V_m, W_m, class M1
//   Method 2-Double  all blocks (V' D W'), FP64      -
//   Method 2-Single  dense blocks, class S           low-rank V' D W', class S2
//   Method 2-Mixed   all blocks (V' D W'), class M   -
//   Method 3         dense + ranks with d_i >= d_max 10^-c (eq. 20), FP64
//                                                    ranks with d_i < d_max 10^-c (eq. 19), class M
//   dense split      dense columns with weight       the other dense columns and every
//   (Section 4.5)    >= d_max 10^-c, FP64            low-rank V' D W', class M
//     (a dense column's weight is max_i |a_ij|, d_max the largest near-field
//     entry; a block whose columns fall on both sides is stored as two column
//     subsets, kind 2 blocks with their column lists)
//
// Classes (what the kernels compute per stored entry p and operand):
//   FP64  p FP64, x FP64, FP64 products and sums;
//   M     p FP32 promoted to FP64, x FP64, FP64 products and sums;
//   S     p FP32 times FP32 x, product rounded to FP32, then added in FP64
//         (low-rank z_m of Method 1-Single accumulated in FP32);
//   M1    Method 1-Mixed's projection: z_m = fl32(z_m + p x) with the right side
//         in FP64; its expansion multiplies FP32 V_m by FP32 z_m (class S);
//   S2    Method 2-Single's low-rank block: projection in class S summed into an
//         FP64 z_m, expansion in class M.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hmat.h"
#include "hmat_internal.h"

namespace hmat_internal {

namespace {

bool is_table1(int precision) { return precision >= HMAT_M1_SINGLE && precision <= HMAT_M3_DENSE; }

// FP32 storage must not overflow; underflow is the precision loss the variant accepts
bool fits_fp32(const double *a, int64_t cnt) {
    for (int64_t k = 0; k < cnt; ++k)
        if (std::fabs(a[k]) > (double)FLT_MAX) return false;
    return true;
}

struct SegBuilder {
    DerivedSegment *seg;
    void add_dense(const int64_t *e, const double *src) {
        const int64_t m = e[1] - e[0], n = e[3] - e[2];
        const int64_t off = (int64_t)seg->data.size();
        seg->data.insert(seg->data.end(), src, src + m * n);
        seg->blocks.insert(seg->blocks.end(), {e[0], e[1], e[2], e[3], 0, 0, off, 0});
        seg->toff.push_back(-1);
    }
    // the columns `js` (ascending, block-local) of a dense block, as a kind 2 block
    void add_dense_cols(const int64_t *e, const double *src, const std::vector<int64_t> &js) {
        const int64_t m = e[1] - e[0], n = e[3] - e[2], k = (int64_t)js.size();
        const int64_t off = (int64_t)seg->data.size();
        seg->data.resize(off + m * k);
        for (int64_t i = 0; i < m; ++i)
            for (int64_t c = 0; c < k; ++c) seg->data[off + i * k + c] = src[i * n + js[c]];
        const int64_t coff = (int64_t)seg->dcols.size();
        for (int64_t j : js) seg->dcols.push_back((int32_t)(e[2] + j));
        seg->blocks.insert(seg->blocks.end(), {e[0], e[1], e[2], e[3], 2, k, off, coff});
        seg->toff.push_back(-1);
    }
    // low-rank block with the ranks `ls` of (V, W) (V #I x r row-major, W r x #J
    // row-major); `d` non-null attaches the per-rank factors d_l to t (eq. 23)
    void add_lr(const int64_t *e, const double *V, const double *W, int64_t r, const std::vector<int64_t> &ls,
                const double *d) {
        const int64_t m = e[1] - e[0], n = e[3] - e[2], rs = (int64_t)ls.size();
        if (rs == 0) return;
        const int64_t off = (int64_t)seg->data.size();
        seg->data.resize(off + rs * (m + n));
        double *Vs = seg->data.data() + off, *Ws = Vs + m * rs;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t k = 0; k < rs; ++k) Vs[i * rs + k] = V[i * r + ls[k]];
        for (int64_t k = 0; k < rs; ++k)
            std::memcpy(Ws + k * n, W + ls[k] * n, sizeof(double) * n);
        seg->blocks.insert(seg->blocks.end(), {e[0], e[1], e[2], e[3], 1, rs, off, 0});
        if (d) {
            seg->toff.push_back((int64_t)seg->tval.size());
            for (int64_t k = 0; k < rs; ++k) seg->tval.push_back(d[ls[k]]);
        } else {
            seg->toff.push_back(-1);
        }
    }
};

void finish(DerivedSegment &s, const BlobView &v) {
    s.hdr = *v.h;
    s.hdr.nblocks = (int64_t)s.toff.size();
    s.hdr.ndata = (int64_t)s.data.size();
    s.view.h = &s.hdr;
    s.view.perm = v.perm;
    s.view.clusters = v.clusters;
    s.view.blocks = s.blocks.data();
    s.view.data = s.data.data();
    s.view.leaf_begin = v.leaf_begin;
    s.view.pow2 = false;
    s.view.toff = s.toff.data();
    s.view.tval = s.tval.data();
    s.view.dcols = s.dcols.data();
}

}  // namespace

int derive_table1(const BlobView &v, int precision, int c, DerivedSegment (&seg)[2], Store (&store)[2], int *nseg,
                  std::string *why) {
    if (!is_table1(precision)) return HMAT_ERR_ARG;
    const bool m3 = precision == HMAT_M3 || precision == HMAT_M3_TRUNC;
    const bool split_dense = precision == HMAT_M3_DENSE;
    if ((m3 || split_dense) && (c < -1 || c > 16)) {
        if (why) *why = "Method 3 c outside [-1, 16]";
        return HMAT_ERR_ARG;
    }
    for (auto &s : seg) s = DerivedSegment();
    const bool m1 = precision == HMAT_M1_SINGLE || precision == HMAT_M1_MIXED;
    // segment of the dense blocks / of the low-rank ranks, and the classes
    int dense_seg = 0, lr_seg = 0;
    switch (precision) {
    case HMAT_M1_SINGLE: store[0] = Store::PS; store[1] = Store::PS; break;
    case HMAT_M1_MIXED: store[0] = Store::PM; store[1] = Store::PM1; lr_seg = 1; break;
    case HMAT_M2_DOUBLE: store[0] = Store::F64; store[1] = Store::F64; break;
    case HMAT_M2_SINGLE: store[0] = Store::PS; store[1] = Store::PS2; lr_seg = 1; break;
    case HMAT_M2_MIXED: store[0] = Store::PM; store[1] = Store::PM; break;
    case HMAT_M3: store[0] = Store::F64; store[1] = Store::PM; break;
    case HMAT_M3_TRUNC: store[0] = Store::F64; store[1] = Store::F64; break;
    case HMAT_M3_DENSE: store[0] = Store::F64; store[1] = Store::PM; lr_seg = 1; break;
    }
    // dense split: the threshold on the column weights, from the largest entry
    // of the near field (every dense block)
    double dense_thr = 0.0;
    if (split_dense) {
        double dmax = 0.0;
        for (int64_t b = 0; b < v.h->nblocks; ++b) {
            const int64_t *e = v.blocks + 8 * b;
            if (e[4] != 0) continue;
            const double *a = v.data + e[6];
            for (int64_t k = 0; k < (e[1] - e[0]) * (e[3] - e[2]); ++k) dmax = std::max(dmax, std::fabs(a[k]));
        }
        dense_thr = dmax * std::pow(10.0, -(double)c);
    }
    std::vector<int64_t> j64, j32;
    SegBuilder sb[2] = {{&seg[0]}, {&seg[1]}};
    std::vector<double> Vp, Wp, d;
    std::vector<int64_t> lsA, lsB;
    const double *data = v.data;
    for (int64_t b = 0; b < v.h->nblocks; ++b) {
        const int64_t *e = v.blocks + 8 * b;
        const int64_t m = e[1] - e[0], n = e[3] - e[2], r = e[5];
        const double *src = data + e[6];
        if (e[4] == 0) {
            if (split_dense) {
                // a column is FP64 iff max_i |a_ij| >= d_max 10^-c (eq. 19-20 on W' = I)
                j64.clear();
                j32.clear();
                for (int64_t j = 0; j < n; ++j) {
                    double w = 0.0;
                    for (int64_t i = 0; i < m; ++i) w = std::max(w, std::fabs(src[i * n + j]));
                    (w >= dense_thr ? j64 : j32).push_back(j);
                }
                for (int64_t j : j32)
                    for (int64_t i = 0; i < m; ++i)
                        if (std::fabs(src[i * n + j]) > (double)FLT_MAX) {
                            if (why) *why = "dense block outside the FP32 range";
                            return HMAT_ERR_RANGE;
                        }
                if (j32.empty()) sb[0].add_dense(e, src);
                else if (j64.empty()) sb[1].add_dense(e, src);
                else {
                    sb[0].add_dense_cols(e, src, j64);
                    sb[1].add_dense_cols(e, src, j32);
                }
                continue;
            }
            if (store[dense_seg] != Store::F64 && !fits_fp32(src, m * n)) {
                if (why) *why = "dense block outside the FP32 range";
                return HMAT_ERR_RANGE;
            }
            sb[dense_seg].add_dense(e, src);
            continue;
        }
        if (r == 0) continue;
        const double *V = src, *W = src + m * r;
        lsA.clear();
        lsB.clear();
        if (m1) {
            if (!fits_fp32(V, m * r) || !fits_fp32(W, r * n)) {
                if (why) *why = "low-rank factor outside the FP32 range";
                return HMAT_ERR_RANGE;
            }
            for (int64_t l = 0; l < r; ++l) lsA.push_back(l);
            sb[lr_seg].add_lr(e, V, W, r, lsA, nullptr);
            continue;
        }
        // Method 2/3 structure V' D W' (eq. 11-16): D_V and D_W hold the max-abs
        // of each column of V_m / row of W_m, V' = V D_V^-1, W' = D_W^-1 W,
        // D_m = D_V D_W; all in FP64, converted afterwards
        Vp.resize(m * r);
        Wp.resize(r * n);
        d.resize(r);
        for (int64_t l = 0; l < r; ++l) {
            double dv = 0.0, dw = 0.0;
            for (int64_t i = 0; i < m; ++i) dv = std::max(dv, std::fabs(V[i * r + l]));
            for (int64_t j = 0; j < n; ++j) dw = std::max(dw, std::fabs(W[l * n + j]));
            if (!(dv > 0.0) || !(dw > 0.0)) {
                if (why) *why = "zero low-rank vector: D_m of eq. (14)-(15) is singular";
                return HMAT_ERR_RANGE;
            }
            for (int64_t i = 0; i < m; ++i) Vp[i * r + l] = V[i * r + l] / dv;
            for (int64_t j = 0; j < n; ++j) Wp[l * n + j] = W[l * n + j] / dw;
            d[l] = dv * dw;
            if (!std::isfinite(d[l])) {
                if (why) *why = "D_m entry overflows FP64";
                return HMAT_ERR_RANGE;
            }
        }
        if (m3) {
            // eq. (19)-(20): rank l in FP64 iff d_l >= d_max 10^-c
            double dmax = 0.0;
            for (int64_t l = 0; l < r; ++l) dmax = std::max(dmax, d[l]);
            const double thr = dmax * std::pow(10.0, -(double)c);
            for (int64_t l = 0; l < r; ++l) (d[l] >= thr ? lsA : lsB).push_back(l);
        } else {
            for (int64_t l = 0; l < r; ++l) lsA.push_back(l);
        }
        if (precision == HMAT_M3) {
            sb[0].add_lr(e, Vp.data(), Wp.data(), r, lsA, d.data());
            sb[1].add_lr(e, Vp.data(), Wp.data(), r, lsB, d.data());
        } else if (precision == HMAT_M3_TRUNC) {
            sb[0].add_lr(e, Vp.data(), Wp.data(), r, lsA, d.data());  // Section 4.5: lsB deleted
        } else {
            sb[lr_seg].add_lr(e, Vp.data(), Wp.data(), r, lsA, d.data());
        }
    }
    int k = 0;
    for (int s = 0; s < 2; ++s) {
        if (seg[s].toff.empty()) continue;
        if (k != s) {
            seg[k] = std::move(seg[s]);
            store[k] = store[s];
        }
        ++k;
    }
    for (int s = 0; s < k; ++s) finish(seg[s], v);
    *nseg = k;
    if (k == 0) {
        if (why) *why = "no blocks";
        return HMAT_ERR_BAD_LAYOUT;
    }
    return HMAT_OK;
}

}  // namespace hmat_internal

namespace hmat_internal {

// A batch of independent problems as one block-diagonal operator: the problems'
// index spaces are concatenated (problem p owns rows and columns [off_p, off_p +
// n_p) in both orders), their blocks shifted onto the diagonal.  Each view must
// have been validated by parse_blob.
int combine_blobs(const BlobView *views, int count, CombinedBlob &out, std::string *why) {
    if (count < 1) return HMAT_ERR_ARG;
    out = CombinedBlob();
    int64_t n = 0, nb = 0, nd = 0;
    for (int p = 0; p < count; ++p) {
        n += views[p].h->n;
        nb += views[p].h->nblocks;
        nd += views[p].h->ndata;
    }
    if (n > (int64_t(1) << 30)) {
        if (why) *why = "batch too large";
        return HMAT_ERR_UNSUPPORTED;
    }
    out.perm.resize(n);
    out.blocks.resize(8 * nb);
    out.data.resize(nd);
    out.offsets.assign(1, 0);
    out.view.leaf_begin.clear();
    int64_t on = 0, ob = 0, od = 0;
    for (int p = 0; p < count; ++p) {
        const BlobView &v = views[p];
        const int64_t np = v.h->n, nbp = v.h->nblocks, ndp = v.h->ndata;
        for (int64_t i = 0; i < np; ++i) out.perm[on + i] = on + v.perm[i];
        for (int64_t b = 0; b < nbp; ++b) {
            const int64_t *e = v.blocks + 8 * b;
            int64_t *o = out.blocks.data() + 8 * (ob + b);
            o[0] = e[0] + on; o[1] = e[1] + on; o[2] = e[2] + on; o[3] = e[3] + on;
            o[4] = e[4]; o[5] = e[5]; o[6] = e[6] + od; o[7] = e[7];
        }
        std::copy(v.data, v.data + ndp, out.data.begin() + od);
        for (size_t l = 0; l + 1 < v.leaf_begin.size(); ++l) out.view.leaf_begin.push_back(on + v.leaf_begin[l]);
        on += np;
        ob += nbp;
        od += ndp;
        out.offsets.push_back(on);
    }
    out.view.leaf_begin.push_back(n);
    out.hdr = *views[0].h;
    out.hdr.n = n;
    out.hdr.nblocks = nb;
    out.hdr.ndata = nd;
    out.view.h = &out.hdr;
    out.view.perm = out.perm.data();
    out.view.clusters = nullptr;  // not used past validation
    out.view.blocks = out.blocks.data();
    out.view.data = out.data.data();
    return HMAT_OK;
}

}  // namespace hmat_internal

extern "C" int hmat_form_stats_get(const void *blob, size_t blob_bytes, int32_t precision, int32_t method3_c,
                                   hmat_form_stats *out) {
    using namespace hmat_internal;
    if (!blob || !out || precision < HMAT_FP64 || precision > HMAT_M3_DENSE) return HMAT_ERR_ARG;
    BlobView v;
    int st = parse_blob(blob, blob_bytes, v);
    if (st != HMAT_OK) return st;
    std::memset(out, 0, sizeof(*out));
    try {
        DerivedSegment seg[2];
        Store store[2];
        int nseg = 1;
        const BlobView *views[2] = {&v, nullptr};
        if (precision >= HMAT_M1_SINGLE) {
            st = derive_table1(v, precision, method3_c, seg, store, &nseg, nullptr);
            if (st != HMAT_OK) return st;
            for (int k = 0; k < nseg; ++k) views[k] = &seg[k].view;
        }
        out->segments = nseg;
        for (int k = 0; k < nseg; ++k) {
            const BlobView &w = *views[k];
            Layout L;
            if ((st = build_layout(w, L)) != HMAT_OK || (st = check_layout(L)) != HMAT_OK) return st;
            out->blocks[k] = w.h->nblocks;
            for (int64_t b = 0; b < w.h->nblocks; ++b) {
                const int64_t *e = w.blocks + 8 * b;
                const int64_t m = e[1] - e[0], n = e[3] - e[2];
                if (block_is_dense(e)) {
                    out->dense_entries[k] += m * dense_width(e);
                    if (e[4] == 2) out->column_subsets[k] += 1;
                } else {
                    out->lr_ranks[k] += e[5];
                    out->lr_entries[k] += e[5] * (m + n);
                }
            }
            out->selected_operands[k] = (int64_t)L.xsel.size();
        }
    } catch (const std::bad_alloc &) {
        return HMAT_ERR_NOMEM;
    }
    return HMAT_OK;
}
