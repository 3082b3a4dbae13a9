// Validation of the serialized H-matrix and its packing into the two work
// lists the GPU kernels stream:
//   phase 1, per leaf column cluster kappa: the rows of every W_m (eq. 9/22)
//     whose column cluster contains kappa, as one row-major |kappa| x R panel;
//   phase 2, per leaf row cluster rho: the rows of every dense block A|^m
//     (eq. 21) and of every V_m (eq. 10/24) whose row cluster contains rho, as
//     one row-major |rho| x K panel.
// Every entry of the blob lands in exactly one panel, so one product reads
// each stored value once.  Each array (dense block, V_m, W_m) is divided by
// 2^floor(log2 max|array|) before conversion; the kernels undo it exactly.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hmat.h"
#include "hmat_internal.h"

namespace hmat_internal {

namespace {

bool fail(std::string *why, const char *msg) {
    if (why) *why = msg;
    return false;
}

int exponent_of_max(const double *a, int64_t cnt) {
    double mx = 0.0;
    for (int64_t k = 0; k < cnt; ++k) mx = std::max(mx, std::fabs(a[k]));
    if (mx == 0.0) return 0;
    int e;
    std::frexp(mx, &e);  // mx = f 2^e, 0.5 <= f < 1
    return e - 1;
}

int64_t roundup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Round an FP64 value to the nearest BF16 (ties to even) and return its 16 bits.
uint16_t to_bf16(double v) {
    uint64_t bits;
    std::memcpy(&bits, &v, 8);
    uint64_t mag = bits & 0x7FFFFFFFFFFFFFFFull;
    if (mag == 0) return (uint16_t)((bits >> 48) & 0x8000);
    // keep 7 explicit fraction bits of the 52: round the low 45 bits to even
    const uint64_t low = (uint64_t(1) << 45) - 1;
    uint64_t keep_lsb = (bits >> 45) & 1;
    uint64_t r = bits + (low >> 1) + keep_lsb;
    r &= ~low;
    double d;
    std::memcpy(&d, &r, 8);
    float f = (float)d;  // exact: 8 significant bits inside the FP32 range
    uint32_t fb;
    std::memcpy(&fb, &f, 4);
    return (uint16_t)(fb >> 16);
}

template <class T> struct Writer;
template <> struct Writer<double> {
    static void put(double *p, int64_t k, double v) { p[k] = v; }
};
template <> struct Writer<float> {
    static void put(float *p, int64_t k, double v) { p[k] = (float)v; }
};
struct DFPair { float hi, lo; };
template <> struct Writer<DFPair> {
    static void put(DFPair *p, int64_t k, double v) {
        float hi = (float)v;
        float lo = (float)(v - (double)hi);
        p[k].hi = hi;
        p[k].lo = lo;
    }
};
template <> struct Writer<uint16_t> {
    static void put(uint16_t *p, int64_t k, double v) { p[k] = to_bf16(v); }
};

template <class T>
void fill_typed(const BlobView &v, const Layout &L, T *q1, T *p2) {
    const int64_t *bt = v.blocks;
    const double *data = v.data;
    const int64_t n1 = (int64_t)L.p1.size();
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t w = 0; w < n1; ++w) {
        const P1Desc &d = L.p1[w];
        T *base = q1 + d.off;
        for (int64_t k = 0; k < (int64_t)d.xlen * d.ld; ++k) Writer<T>::put(base, k, 0.0);
        for (int64_t s = L.p1_slice_ptr[w]; s < L.p1_slice_ptr[w + 1]; ++s) {
            const Layout::Slice &sl = L.p1_slices[s];
            const int64_t *e = bt + 8 * sl.block;
            const int64_t m = e[1] - e[0], n = e[3] - e[2], r = e[5];
            const double *W = data + e[6] + m * r;  // W_m, r x n row-major
            const double inv = std::ldexp(1.0, -sl.scale);
            for (int64_t j = 0; j < d.xlen; ++j)
                for (int64_t l = 0; l < sl.ncols; ++l)
                    Writer<T>::put(base, j * d.ld + sl.col0 + l, W[l * n + sl.row0 + j] * inv);
        }
    }
    const int64_t n2 = (int64_t)L.p2.size();
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t w = 0; w < n2; ++w) {
        const P2Desc &d = L.p2[w];
        T *base = p2 + d.off;
        for (int64_t k = 0; k < (int64_t)d.ylen * d.ld; ++k) Writer<T>::put(base, k, 0.0);
        for (int64_t s = L.p2_slice_ptr[w]; s < L.p2_slice_ptr[w + 1]; ++s) {
            const Layout::Slice &sl = L.p2_slices[s];
            const int64_t *e = bt + 8 * sl.block;
            const int64_t r = e[5];
            const double *src = data + e[6];
            const int64_t ld_src = sl.kind == 0 ? dense_width(e) : r;  // dense row-major, V_m row-major m x r
            const double inv = std::ldexp(1.0, -sl.scale);
            for (int64_t i = 0; i < d.ylen; ++i)
                for (int64_t k = 0; k < sl.ncols; ++k)
                    Writer<T>::put(base, i * d.ld + sl.col0 + k, src[(sl.row0 + i) * ld_src + k] * inv);
        }
    }
}

}  // namespace

int parse_blob(const void *blob, size_t bytes, BlobView &v, std::string *why) {
    if (!blob) return HMAT_ERR_ARG;
    if (bytes < (size_t)kBlobHeaderBytes) return fail(why, "blob shorter than its header"), HMAT_ERR_BAD_LAYOUT;
    if (((uintptr_t)blob & 7) != 0) return fail(why, "blob not 8-byte aligned"), HMAT_ERR_ARG;
    const BlobHeader *h = (const BlobHeader *)blob;
    if (std::memcmp(h->magic, kBlobMagic, 8) != 0) return fail(why, "bad magic"), HMAT_ERR_BAD_LAYOUT;
    if (h->version != 1 || h->header_bytes != (uint32_t)kBlobHeaderBytes)
        return fail(why, "unsupported version"), HMAT_ERR_BAD_LAYOUT;
    const int64_t n = h->n, nc = h->nclusters, nb = h->nblocks, nd = h->ndata;
    if (n < 1 || n > (int64_t(1) << 30) || nc < 1 || nc > 2 * n || nb < 1 || nd < 0 || nd > (int64_t(1) << 40))
        return fail(why, "bad counts"), HMAT_ERR_BAD_LAYOUT;
    if (h->total_bytes < kBlobHeaderBytes || (uint64_t)h->total_bytes > (uint64_t)bytes)
        return fail(why, "total_bytes exceeds the buffer"), HMAT_ERR_BAD_LAYOUT;
    auto section_ok = [&](int64_t off, int64_t len) {
        return off >= kBlobHeaderBytes && (off & 7) == 0 && len >= 0 && off <= h->total_bytes &&
               len <= h->total_bytes - off;
    };
    if (!section_ok(h->off_perm, 8 * n) || !section_ok(h->off_clusters, 32 * nc) ||
        !section_ok(h->off_blocks, 64 * nb) || !section_ok(h->off_data, 8 * nd))
        return fail(why, "section outside the blob"), HMAT_ERR_BAD_LAYOUT;
    const char *base = (const char *)blob;
    v.h = h;
    v.perm = (const int64_t *)(base + h->off_perm);
    v.clusters = (const int64_t *)(base + h->off_clusters);
    v.blocks = (const int64_t *)(base + h->off_blocks);
    v.data = (const double *)(base + h->off_data);

    // permutation
    std::vector<char> seen(n, 0);
    for (int64_t p = 0; p < n; ++p) {
        int64_t q = v.perm[p];
        if (q < 0 || q >= n || seen[q]) return fail(why, "perm is not a permutation"), HMAT_ERR_BAD_LAYOUT;
        seen[q] = 1;
    }
    // cluster tree
    const int64_t *cl = v.clusters;
    if (cl[0] != 0 || cl[1] != n) return fail(why, "cluster 0 is not the root"), HMAT_ERR_BAD_LAYOUT;
    std::vector<char> parent_seen(nc, 0);
    std::vector<int64_t> leaves;
    int64_t max_leaf = 0;
    for (int64_t k = 0; k < nc; ++k) {
        int64_t b = cl[4 * k], e = cl[4 * k + 1], c0 = cl[4 * k + 2], c1 = cl[4 * k + 3];
        if (b < 0 || e > n || b >= e) return fail(why, "bad cluster range"), HMAT_ERR_BAD_LAYOUT;
        if (c0 < 0 || c1 < 0) {
            if (c0 != -1 || c1 != -1) return fail(why, "half leaf"), HMAT_ERR_BAD_LAYOUT;
            leaves.push_back(k);
            max_leaf = std::max(max_leaf, e - b);
            continue;
        }
        if (c0 <= k || c1 <= k || c0 >= nc || c1 >= nc || parent_seen[c0] || parent_seen[c1])
            return fail(why, "bad cluster children"), HMAT_ERR_BAD_LAYOUT;
        parent_seen[c0] = parent_seen[c1] = 1;
        if (cl[4 * c0] != b || cl[4 * c0 + 1] != cl[4 * c1] || cl[4 * c1 + 1] != e)
            return fail(why, "children do not split the parent"), HMAT_ERR_BAD_LAYOUT;
    }
    for (int64_t k = 1; k < nc; ++k)
        if (!parent_seen[k]) return fail(why, "cluster without a parent"), HMAT_ERR_BAD_LAYOUT;
    if (max_leaf > kMaxLeaf) return fail(why, "leaf cluster larger than 64"), HMAT_ERR_UNSUPPORTED;
    std::sort(leaves.begin(), leaves.end(), [&](int64_t a, int64_t b) { return cl[4 * a] < cl[4 * b]; });
    v.leaf_begin.clear();
    for (int64_t k : leaves) v.leaf_begin.push_back(cl[4 * k]);
    v.leaf_begin.push_back(n);
    for (size_t i = 0; i + 1 < v.leaf_begin.size(); ++i)
        if (cl[4 * leaves[i] + 1] != v.leaf_begin[i + 1]) return fail(why, "leaves do not tile"), HMAT_ERR_BAD_LAYOUT;
    auto is_boundary = [&](int64_t x) {
        return std::binary_search(v.leaf_begin.begin(), v.leaf_begin.end(), x);
    };
    // blocks
    const int64_t nleaves = (int64_t)leaves.size();
    std::vector<std::vector<std::pair<int64_t, int64_t>>> rowcov(nleaves);
    int64_t area = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t *e = v.blocks + 8 * b;
        int64_t is = e[0], ie = e[1], js = e[2], je = e[3], kind = e[4], r = e[5], off = e[6];
        if (is < 0 || ie > n || is >= ie || js < 0 || je > n || js >= je)
            return fail(why, "bad block range"), HMAT_ERR_BAD_LAYOUT;
        if (!is_boundary(is) || !is_boundary(ie) || !is_boundary(js) || !is_boundary(je))
            return fail(why, "block not aligned to leaf clusters"), HMAT_ERR_BAD_LAYOUT;
        int64_t m = ie - is, w = je - js, cnt;
        if (kind == 0) {
            if (r != 0) return fail(why, "dense block with a rank"), HMAT_ERR_BAD_LAYOUT;
            cnt = m * w;
        } else if (kind == 1) {
            if (r < 0 || r > std::min(m, w)) return fail(why, "rank > min(#I,#J)"), HMAT_ERR_BAD_LAYOUT;
            cnt = r * (m + w);
        } else {
            return fail(why, "bad block kind"), HMAT_ERR_BAD_LAYOUT;
        }
        if (off < 0 || off > nd || cnt > nd - off) return fail(why, "block data outside the blob"), HMAT_ERR_BAD_LAYOUT;
        area += m * w;
        int64_t l0 = std::lower_bound(v.leaf_begin.begin(), v.leaf_begin.end(), is) - v.leaf_begin.begin();
        int64_t l1 = std::lower_bound(v.leaf_begin.begin(), v.leaf_begin.end(), ie) - v.leaf_begin.begin();
        for (int64_t l = l0; l < l1; ++l) rowcov[l].push_back({js, je});
    }
    if (area != n * n) return fail(why, "blocks do not cover I x J (eq. 1-2)"), HMAT_ERR_BAD_LAYOUT;
    for (auto &lst : rowcov) {
        std::sort(lst.begin(), lst.end());
        int64_t at = 0;
        for (auto &iv : lst) {
            if (iv.first != at) return fail(why, "blocks overlap or leave a gap (eq. 1-2)"), HMAT_ERR_BAD_LAYOUT;
            at = iv.second;
        }
        if (at != n) return fail(why, "row not covered (eq. 2)"), HMAT_ERR_BAD_LAYOUT;
    }
    for (int64_t k = 0; k < nd; ++k)
        if (!std::isfinite(v.data[k])) return fail(why, "non-finite value"), HMAT_ERR_BAD_LAYOUT;
    return HMAT_OK;
}

int build_layout(const BlobView &v, Layout &L, std::string *why) {
    const int64_t n = v.h->n, nb = v.h->nblocks;
    const int64_t nleaves = (int64_t)v.leaf_begin.size() - 1;
    L = Layout();
    L.n = n;
    L.nleaves = (int32_t)nleaves;
    L.perm.resize(n);
    for (int64_t p = 0; p < n; ++p) L.perm[p] = (int32_t)v.perm[p];
    L.leaf_begin.resize(nleaves + 1);
    for (int64_t l = 0; l <= nleaves; ++l) L.leaf_begin[l] = (int32_t)v.leaf_begin[l];
    for (int64_t l = 0; l < nleaves; ++l) L.max_leaf = std::max<int32_t>(L.max_leaf, L.leaf_begin[l + 1] - L.leaf_begin[l]);

    auto leaf_index = [&](int64_t x) {
        return (int64_t)(std::lower_bound(v.leaf_begin.begin(), v.leaf_begin.end(), x) - v.leaf_begin.begin());
    };

    // exponents, low-rank block numbering
    std::vector<int32_t> eD(nb, 0), eU(nb, 0), eV(nb, 0), lrq(nb, -1);
    std::vector<int64_t> lr_blocks;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t *e = v.blocks + 8 * b;
        int64_t m = e[1] - e[0], w = e[3] - e[2], r = e[5];
        const double *d = v.data + e[6];
        L.stored_entries += block_is_dense(e) ? m * dense_width(e) : r * (m + w);
        if (block_is_dense(e)) {
            if (v.pow2) eD[b] = exponent_of_max(d, m * dense_width(e));
        } else if (r > 0) {
            if (v.pow2) {
                eU[b] = exponent_of_max(d, m * r);
                eV[b] = exponent_of_max(d + m * r, r * w);
            }
            lrq[b] = (int32_t)lr_blocks.size();
            lr_blocks.push_back(b);
            L.rank_sum += r;
        }
        if (std::abs(eD[b]) > kMaxScaleExp || std::abs(eU[b]) > kMaxScaleExp || std::abs(eV[b]) > kMaxScaleExp ||
            std::abs(eU[b] + eV[b]) > kMaxScaleExp) {
            if (why) *why = "panel exponent out of range";
            return HMAT_ERR_RANGE;
        }
    }
    const int64_t nlr = (int64_t)lr_blocks.size();

    // phase 2 first: panel columns and operand buffers g per leaf row cluster
    std::vector<std::vector<int64_t>> by_row(nleaves);
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t *e = v.blocks + 8 * b;
        if (e[4] == 1 && e[5] == 0) continue;
        for (int64_t l = leaf_index(e[0]); l < leaf_index(e[1]); ++l) by_row[l].push_back(b);
    }
    // column of block b in the panel of leaf rho, in block order per rho
    std::vector<std::vector<std::pair<int64_t, int32_t>>> col_of(nleaves);
    L.p2.resize(nleaves);
    L.p2_slice_ptr.assign(nleaves + 1, 0);
    int64_t off = 0, goff = 0;
    for (int64_t k = 0; k < nleaves; ++k) {
        P2Desc &d = L.p2[k];
        d.ybeg = (int32_t)v.leaf_begin[k];
        d.ylen = (int32_t)(v.leaf_begin[k + 1] - v.leaf_begin[k]);
        int64_t col = 0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int64_t b : by_row[k]) {
                const int64_t *e = v.blocks + 8 * b;
                if ((block_is_dense(e) ? 0 : 1) != pass) continue;
                const int32_t len = (int32_t)(pass == 0 ? dense_width(e) : e[5]);
                col_of[k].push_back({b, (int32_t)col});
                L.p2_slices.push_back({b, (int32_t)col, len, (int32_t)(d.ybeg - e[0]), pass, pass == 0 ? eD[b] : eU[b]});
                col += len;
            }
        }
        d.K = (int32_t)col;
        d.ld = (int32_t)roundup(std::max<int64_t>(col, 1), kPadElems);
        d.off = off;
        d.goff = (int32_t)goff;
        d.pad = 0;
        off += (int64_t)d.ld * d.ylen;
        goff += d.ld;
        L.phase2_entries += col * d.ylen;
        L.max_ld2 = std::max(L.max_ld2, d.ld);
        L.p2_slice_ptr[k + 1] = (int64_t)L.p2_slices.size();
    }
    if (goff > (int64_t(1) << 31) - 16) { if (why) *why = "operand buffer too large"; return HMAT_ERR_UNSUPPORTED; }
    L.rows.resize(n);
    for (int64_t k = 0; k < nleaves; ++k) {
        const P2Desc &d = L.p2[k];
        for (int i = 0; i < d.ylen; ++i) L.rows[d.ybeg + i] = RowDesc{d.off + (int64_t)i * d.ld, d.goff, d.ld};
        for (int i = 0; i < d.ylen; i += kGroupRows)
            L.groups.push_back(GroupDesc{d.off + (int64_t)i * d.ld, d.goff, d.ld, d.ybeg + i,
                                         std::min(kGroupRows, d.ylen - i), {0, 0}});
    }
    L.p2_elems = off;
    L.glen = goff;
    auto column_in = [&](int64_t rho, int64_t b) {
        const auto &lst = col_of[rho];
        for (const auto &pr : lst)
            if (pr.first == b) return pr.second;
        return -1;
    };

    // low-rank descriptors: operand destinations in every leaf row cluster of the block
    std::vector<int64_t> kfirst(nb, 0), kcnt(nb, 0);
    L.lr.resize(nlr);
    int64_t ntofs = 0;
    std::vector<int64_t> direct_q;
    for (int64_t q = 0; q < nlr; ++q) {
        const int64_t b = lr_blocks[q];
        const int64_t *e = v.blocks + 8 * b;
        LrDesc &d = L.lr[q];
        kfirst[b] = leaf_index(e[2]);
        kcnt[b] = leaf_index(e[3]) - kfirst[b];
        d.rank = (int32_t)e[5];
        d.cnt = (int32_t)kcnt[b];
        d.scale = eU[b] + eV[b];
        d.boff = (int32_t)ntofs;  // filled with the phase-1 panels below
        ntofs += kcnt[b];
        if (ntofs > (int64_t(1) << 31) - 16) { if (why) *why = "too many projection terms"; return HMAT_ERR_UNSUPPORTED; }
        d.gbeg = (int32_t)L.gdst.size();
        for (int64_t rho = leaf_index(e[0]); rho < leaf_index(e[1]); ++rho) {
            int32_t c = column_in(rho, b);
            if (c < 0) { if (why) *why = "internal: block missing from a row panel"; return HMAT_ERR_BAD_LAYOUT; }
            L.gdst.push_back(L.p2[rho].goff + c);
        }
        d.gcnt = (int32_t)L.gdst.size() - d.gbeg;
        d.toff = -1;
        d.pad = 0;
        if (v.toff && v.toff[b] >= 0) {
            if (L.tscale.size() + e[5] > (size_t(1) << 31) - 16) { if (why) *why = "too many rank factors"; return HMAT_ERR_UNSUPPORTED; }
            d.toff = (int32_t)L.tscale.size();
            L.tscale.insert(L.tscale.end(), v.tval + v.toff[b], v.tval + v.toff[b] + e[5]);
        }
        // the reduction's work: a CTA for a block over many leaf clusters; a
        // direct copy per rank for a block inside one leaf column cluster and one
        // leaf row cluster (its records follow once T is laid out); else a lane
        // per rank
        if (kcnt[b] >= kRedBigCnt) {
            L.red_big.push_back((int32_t)q);
        } else if (kcnt[b] == 1 && d.gcnt == 1 && d.toff < 0) {
            direct_q.push_back(q);
        } else {
            if (q >= (int64_t(1) << 25) || e[5] > 63) { if (why) *why = "reduction task out of range"; return HMAT_ERR_UNSUPPORTED; }
            for (int64_t l = 0; l < e[5]; ++l) L.red_tasks.push_back((int32_t)((q << 6) | l));
        }
    }
    L.tofs.assign((size_t)ntofs, -1);

    // phase 1: low-rank blocks per leaf column cluster (block order), and the
    // dense-block operand slices each leaf column cluster feeds
    std::vector<std::vector<int64_t>> by_col(nleaves), dense_by_col(nleaves);
    for (int64_t q = 0; q < nlr; ++q) {
        const int64_t b = lr_blocks[q];
        for (int64_t l = kfirst[b]; l < kfirst[b] + kcnt[b]; ++l) by_col[l].push_back(b);
    }
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t *e = v.blocks + 8 * b;
        if (!block_is_dense(e)) continue;
        for (int64_t l = leaf_index(e[2]); l < leaf_index(e[3]); ++l) dense_by_col[l].push_back(b);
    }
    L.p1.resize(nleaves);
    L.p1_slice_ptr.assign(nleaves + 1, 0);
    off = 0;
    int64_t tbeg = 0;
    for (int64_t k = 0; k < nleaves; ++k) {
        P1Desc &d = L.p1[k];
        d.xbeg = (int32_t)v.leaf_begin[k];
        d.xlen = (int32_t)(v.leaf_begin[k + 1] - v.leaf_begin[k]);
        d.rbeg = (int32_t)L.p1_runs.size();
        int64_t col = 0;
        for (int64_t b : by_col[k]) {
            const int64_t *e = v.blocks + 8 * b;
            const int64_t r = e[5];
            const LrDesc &ld = L.lr[lrq[b]];
            P1Run run;
            run.col0 = (int32_t)col;
            run.len = (int32_t)r;
            run.q = lrq[b];
            run.pad = 0;
            L.tofs[ld.boff + (k - kfirst[b])] = (int32_t)(tbeg + col);
            L.p1_runs.push_back(run);
            L.p1_slices.push_back({b, (int32_t)col, (int32_t)r, (int32_t)(d.xbeg - e[2]), 1, eV[b]});
            col += r;
        }
        d.rcnt = (int32_t)L.p1_runs.size() - d.rbeg;
        d.R = (int32_t)col;
        d.ld = (int32_t)roundup(std::max<int64_t>(col, 1), kPadElems);
        d.off = off;
        off += (int64_t)d.ld * d.xlen;
        d.tbeg = (int32_t)tbeg;
        tbeg += d.ld;
        if (tbeg > (int64_t(1) << 31) - 16) { if (why) *why = "too many projections"; return HMAT_ERR_UNSUPPORTED; }
        d.xdbeg = (int32_t)L.xdst.size();
        for (int64_t b : dense_by_col[k]) {
            const int64_t *e = v.blocks + 8 * b;
            // the block's stored columns inside kappa: all of them (kind 0), or
            // the listed ones [a, a + cnt) of its column list (kind 2)
            int32_t a = (int32_t)(d.xbeg - e[2]), cnt = d.xlen, sel = -1;
            if (e[4] == 2) {
                const int32_t *cl = v.dcols + e[7], *ce = cl + e[5];
                const int32_t *lo = std::lower_bound(cl, ce, d.xbeg), *hi = std::lower_bound(cl, ce, d.xbeg + d.xlen);
                a = (int32_t)(lo - cl);
                cnt = (int32_t)(hi - lo);
                if (cnt == 0) continue;
                sel = (int32_t)L.xsel.size();
                for (const int32_t *q = lo; q < hi; ++q) L.xsel.push_back(*q - d.xbeg);
            }
            for (int64_t rho = leaf_index(e[0]); rho < leaf_index(e[1]); ++rho) {
                int32_t c = column_in(rho, b);
                if (c < 0) { if (why) *why = "internal: dense block missing from a row panel"; return HMAT_ERR_BAD_LAYOUT; }
                L.xdst.push_back({(int32_t)(L.p2[rho].goff + c + a), eD[b], cnt, sel});
            }
        }
        d.xdcnt = (int32_t)L.xdst.size() - d.xdbeg;
        d.pad[0] = 0;
        L.phase1_entries += col * d.xlen;
        L.max_ld1 = std::max(L.max_ld1, d.ld);
        L.max_runs1 = std::max(L.max_runs1, d.rcnt);
        L.p1_slice_ptr[k + 1] = (int64_t)L.p1_slices.size();
    }
    L.p1_elems = off;
    L.npart = tbeg;
    for (int64_t q : direct_q) {
        const LrDesc &d = L.lr[q];
        for (int32_t l = 0; l < d.rank; ++l) {
            L.red_direct.push_back({L.tofs[d.boff] + l, L.gdst[d.gbeg] + l, d.scale, 0});
            L.red_direct_q.push_back((int32_t)q);
        }
    }
    return HMAT_OK;
}

int check_layout(const Layout &L, std::string *why) {
    // every index the kernels form stays inside its buffer, and every operand
    // slot of g is written exactly once per product
    auto bad = [&](const char *m) { if (why) *why = m; return HMAT_ERR_BAD_LAYOUT; };
    if ((int64_t)L.p1.size() != L.nleaves || (int64_t)L.p2.size() != L.nleaves) return bad("work list size");
    std::vector<uint8_t> gw((size_t)L.glen, 0);
    for (const P2Desc &d : L.p2) {
        if (d.ylen < 1 || d.ylen > kMaxLeaf || d.ybeg < 0 || (int64_t)d.ybeg + d.ylen > L.n) return bad("p2 rows");
        if (d.K < 0 || d.ld < d.K || d.ld % kPadElems || d.off % kPadElems || d.goff % kPadElems) return bad("p2 stride");
        if (d.off < 0 || d.off + (int64_t)d.ylen * d.ld > L.p2_elems) return bad("p2 extent");
        if (d.goff < 0 || (int64_t)d.goff + d.ld > L.glen) return bad("p2 operands");
        for (int c = d.K; c < d.ld; ++c) gw[d.goff + c] = 2;  // zero padding, never written
    }
    for (const LrDesc &d : L.lr) {
        if (d.rank < 1 || d.cnt < 1 || std::abs(d.scale) > kMaxScaleExp) return bad("lr desc");
        if (d.boff < 0 || (int64_t)d.boff + d.cnt > (int64_t)L.tofs.size()) return bad("lr projections");
        for (int k = 0; k < d.cnt; ++k)
            if (L.tofs[d.boff + k] < 0 || (int64_t)L.tofs[d.boff + k] + d.rank > L.npart) return bad("lr projection range");
        if (d.gbeg < 0 || d.gcnt < 1 || (int64_t)d.gbeg + d.gcnt > (int64_t)L.gdst.size()) return bad("lr dst");
        if (d.toff < -1 || (d.toff >= 0 && (int64_t)d.toff + d.rank > (int64_t)L.tscale.size())) return bad("lr factors");
        for (int k = 0; k < d.gcnt; ++k) {
            int32_t g0 = L.gdst[d.gbeg + k];
            if (g0 < 0 || (int64_t)g0 + d.rank > L.glen) return bad("lr dst range");
            for (int l = 0; l < d.rank; ++l) {
                if (gw[g0 + l]) return bad("operand slot written twice");
                gw[g0 + l] = 1;
            }
        }
    }
    for (const P1Desc &d : L.p1) {
        if (d.xlen < 1 || d.xlen > kMaxLeaf || d.xbeg < 0 || (int64_t)d.xbeg + d.xlen > L.n) return bad("p1 rows");
        if (d.R < 0 || d.ld < d.R || d.ld % kPadElems || d.off % kPadElems) return bad("p1 stride");
        if (d.off < 0 || d.off + (int64_t)d.xlen * d.ld > L.p1_elems) return bad("p1 extent");
        if (d.tbeg < 0 || d.tbeg % kPadElems || (int64_t)d.tbeg + d.ld > L.npart) return bad("p1 projection output");
        if (d.rbeg < 0 || d.rcnt < 0 || (int64_t)d.rbeg + d.rcnt > (int64_t)L.p1_runs.size()) return bad("p1 runs");
        if (d.R > 0 && d.rcnt < 1) return bad("p1 empty runs");
        int64_t at = 0;
        for (int r = 0; r < d.rcnt; ++r) {
            const P1Run &u = L.p1_runs[d.rbeg + r];
            if (u.col0 != at || u.len < 1 || u.q < 0 || u.q >= (int32_t)L.lr.size()) return bad("p1 runs do not tile");
            const LrDesc &ld = L.lr[u.q];
            if (u.len != ld.rank) return bad("p1 run rank");
            bool listed = false;  // the block finds this cluster's projection where it is written
            for (int k = 0; k < ld.cnt && !listed; ++k) listed = L.tofs[ld.boff + k] == d.tbeg + u.col0;
            if (!listed) return bad("p1 run projection");
            at += u.len;
        }
        if (at != d.R) return bad("p1 runs do not cover R");
        if (d.xdbeg < 0 || d.xdcnt < 0 || (int64_t)d.xdbeg + d.xdcnt > (int64_t)L.xdst.size()) return bad("p1 xdst");
        for (int k = 0; k < d.xdcnt; ++k) {
            const XDst &x = L.xdst[d.xdbeg + k];
            if (x.cnt < 1 || x.cnt > d.xlen || (x.sel < 0 && (x.sel != -1 || x.cnt != d.xlen))) return bad("xdst count");
            if (x.goff < 0 || (int64_t)x.goff + x.cnt > L.glen || std::abs(x.scale) > kMaxScaleExp) return bad("xdst range");
            if (x.sel >= 0) {
                if ((int64_t)x.sel + x.cnt > (int64_t)L.xsel.size()) return bad("xdst selection");
                for (int j = 0; j < x.cnt; ++j)
                    if (L.xsel[x.sel + j] < 0 || L.xsel[x.sel + j] >= d.xlen) return bad("xdst selection entry");
            }
            for (int j = 0; j < x.cnt; ++j) {
                if (gw[x.goff + j]) return bad("operand slot written twice");
                gw[x.goff + j] = 1;
            }
        }
    }
    for (int64_t k = 0; k < L.glen; ++k)
        if (!gw[k]) return bad("operand slot never written");
    size_t multi = 0, multi_ranks = 0;
    for (const LrDesc &d : L.lr)
        if (d.cnt < kRedBigCnt) multi_ranks += d.rank;
        else if (d.cnt >= kRedBigCnt) ++multi;
    if (multi != L.red_big.size() || multi_ranks != L.red_tasks.size() + L.red_direct.size() ||
        L.red_direct_q.size() != L.red_direct.size())
        return bad("reduction lists");
    for (size_t k = 0; k < L.red_direct.size(); ++k) {  // the block's own projection and slot, one per rank
        const RedDirect &r = L.red_direct[k];
        const int32_t q = L.red_direct_q[k];
        if (q < 0 || q >= (int32_t)L.lr.size()) return bad("red direct block");
        const LrDesc &d = L.lr[q];
        const int64_t l = (int64_t)r.tsrc - L.tofs[d.boff];
        if (d.cnt != 1 || d.gcnt != 1 || d.toff >= 0 || r.scale != d.scale || l < 0 || l >= d.rank ||
            (int64_t)r.gdst != (int64_t)L.gdst[d.gbeg] + l || r.tsrc < 0 || r.tsrc >= L.npart || r.gdst < 0 ||
            r.gdst >= L.glen)
            return bad("red direct");
    }
    for (int32_t q : L.red_big) if (q < 0 || q >= (int32_t)L.lr.size() || L.lr[q].cnt < kRedBigCnt) return bad("red big");
    for (int32_t t : L.red_tasks) {
        const int32_t q = t >> 6, l = t & 63;
        if (q < 0 || q >= (int32_t)L.lr.size() || L.lr[q].cnt >= kRedBigCnt || l >= L.lr[q].rank)
            return bad("red task");
    }
    if ((int64_t)L.rows.size() != L.n) return bad("rows size");
    {  // row groups: cover every row once, inside its cluster's panel
        int64_t covered = 0;
        for (const GroupDesc &gd : L.groups) {
            if (gd.nr < 1 || gd.nr > kGroupRows || gd.p0 < 0 || (int64_t)gd.p0 + gd.nr > L.n) return bad("group rows");
            const RowDesc &r0 = L.rows[gd.p0], &r1 = L.rows[gd.p0 + gd.nr - 1];
            if (gd.off != r0.off || gd.goff != r0.goff || gd.ld != r0.ld || r1.goff != gd.goff ||
                r1.off != gd.off + (int64_t)(gd.nr - 1) * gd.ld)
                return bad("group desc");
            if (gd.p0 != covered) return bad("groups do not tile the rows");
            covered += gd.nr;
        }
        if (covered != L.n) return bad("groups do not cover the rows");
    }
    for (const P2Desc &d : L.p2)
        for (int i = 0; i < d.ylen; ++i) {
            const RowDesc &r = L.rows[d.ybeg + i];
            if (r.off != d.off + (int64_t)i * d.ld || r.goff != d.goff || r.ld != d.ld) return bad("row desc");
        }
    if ((int64_t)L.perm.size() != L.n) return bad("perm size");
    for (int32_t q : L.perm) if (q < 0 || q >= L.n) return bad("perm entry");
    return HMAT_OK;
}

size_t store_bytes(Store s) {
    switch (s) {
    case Store::F64: return 8;
    case Store::DF: return 8;
    case Store::F32: return 4;
    case Store::BF16: return 2;
    case Store::PM: case Store::PS: case Store::PM1: case Store::PS2: return 4;
    }
    return 0;
}

void fill_panels(const BlobView &v, const Layout &L, Store s, void *q1, void *p2) {
    switch (s) {
    case Store::F64: fill_typed<double>(v, L, (double *)q1, (double *)p2); break;
    case Store::DF: fill_typed<DFPair>(v, L, (DFPair *)q1, (DFPair *)p2); break;
    case Store::F32: fill_typed<float>(v, L, (float *)q1, (float *)p2); break;
    case Store::BF16: fill_typed<uint16_t>(v, L, (uint16_t *)q1, (uint16_t *)p2); break;
    case Store::PM: case Store::PS: case Store::PM1: case Store::PS2:
        fill_typed<float>(v, L, (float *)q1, (float *)p2);
        break;
    }
}

uint16_t bf16_bits(double v) { return to_bf16(v); }

}  // namespace hmat_internal

extern "C" int hmat_blob_stats_get(const void *blob, size_t blob_bytes, hmat_blob_stats *out) {
    if (!blob || !out) return HMAT_ERR_ARG;
    hmat_internal::BlobView v;
    int st = hmat_internal::parse_blob(blob, blob_bytes, v);
    if (st != HMAT_OK) return st;
    {
        hmat_internal::Layout L;  // the packing upload would use, with its invariants
        st = hmat_internal::build_layout(v, L);
        if (st == HMAT_OK) st = hmat_internal::check_layout(L);
        if (st != HMAT_OK) return st;
    }
    std::memset(out, 0, sizeof(*out));
    out->n = v.h->n;
    out->nclusters = v.h->nclusters;
    out->nblocks = v.h->nblocks;
    out->nleaves = (int64_t)v.leaf_begin.size() - 1;
    for (int64_t b = 0; b < v.h->nblocks; ++b) {
        const int64_t *e = v.blocks + 8 * b;
        int64_t m = e[1] - e[0], w = e[3] - e[2], r = e[5];
        if (e[4] == 0) {
            out->dense_blocks++;
            out->dense_entries += m * w;
        } else {
            out->lr_blocks++;
            out->lr_entries += r * (m + w);
            out->rank_sum += r;
            out->rank_max = std::max(out->rank_max, r);
        }
    }
    return HMAT_OK;
}
