// Host builder of the FP64 H-matrix of a collocation BEM kernel and writer of
// the serialized layout (format version 1, described in include/hmat.h).
//
// The H-matrix recipe is the one the paper takes from the HACApK library
// (Section 4.1.3): a geometric cluster tree, a block partition M that covers
// I x J exactly once (eq. 1-2), dense blocks A|^m and low-rank blocks V_m W_m
// (eq. 3-4) obtained by adaptive cross approximation (Section 1).  Build flags
// keep FP contraction off so that the arithmetic is reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "hmat.h"
#include "hmat_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Node {
    int64_t begin, end, child0, child1;
    double lo[3], hi[3];
};

struct BlockRec {
    int64_t is, ie, js, je;
    int kind;        // 0 dense, 1 low rank
    int64_t rank;
    std::vector<double> data;
};

// Collocation kernel in original indices.
struct Kernel {
    const double *c;
    const double *area;
    double operator()(int64_t i, int64_t j) const {
        if (i == j) return std::sqrt(area[i] / kPi) / 2.0;
        double dx = c[3 * i + 0] - c[3 * j + 0];
        double dy = c[3 * i + 1] - c[3 * j + 1];
        double dz = c[3 * i + 2] - c[3 * j + 2];
        double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        return area[j] / (4.0 * kPi * r);
    }
};

double diag_len(const Node &k) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = k.hi[d] - k.lo[d];
        s += e * e;
    }
    return std::sqrt(s);
}

double gap_len(const Node &a, const Node &b) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        if (a.hi[d] < b.lo[d]) g = b.lo[d] - a.hi[d];
        else if (b.hi[d] < a.lo[d]) g = a.lo[d] - b.hi[d];
        s += g * g;
    }
    return std::sqrt(s);
}

class TreeBuilder {
  public:
    TreeBuilder(int64_t n, const double *c, int64_t leaf) : n_(n), c_(c), leaf_(leaf) {}

    // Preorder cluster numbering (a node, then its left subtree, then its right).
    void build(std::vector<int64_t> &perm, std::vector<Node> &nodes) {
        perm.resize(n_);
        for (int64_t i = 0; i < n_; ++i) perm[i] = i;
        std::vector<int64_t> scratch(n_);
        struct Task { int64_t begin, end, parent; int side; };
        std::vector<Task> stack;
        stack.push_back({0, n_, -1, 0});
        while (!stack.empty()) {
            Task t = stack.back();
            stack.pop_back();
            int64_t id = (int64_t)nodes.size();
            nodes.push_back(Node{t.begin, t.end, -1, -1, {0, 0, 0}, {0, 0, 0}});
            if (t.parent >= 0) (t.side == 0 ? nodes[t.parent].child0 : nodes[t.parent].child1) = id;
            Node &k = nodes[id];
            for (int d = 0; d < 3; ++d) { k.lo[d] = INFINITY; k.hi[d] = -INFINITY; }
            for (int64_t p = t.begin; p < t.end; ++p) {
                const double *x = c_ + 3 * perm[p];
                for (int d = 0; d < 3; ++d) {
                    k.lo[d] = std::min(k.lo[d], x[d]);
                    k.hi[d] = std::max(k.hi[d], x[d]);
                }
            }
            if (t.end - t.begin <= leaf_) continue;
            int axis = 0;
            double ext = k.hi[0] - k.lo[0];
            for (int d = 1; d < 3; ++d)
                if (k.hi[d] - k.lo[d] > ext) { ext = k.hi[d] - k.lo[d]; axis = d; }
            double mid = 0.5 * (k.lo[axis] + k.hi[axis]);
            int64_t left = 0;
            for (int64_t p = t.begin; p < t.end; ++p)
                if (c_[3 * perm[p] + axis] <= mid) ++left;
            int64_t split;
            if (left == 0 || left == t.end - t.begin) {
                // degenerate midpoint: median of the (coordinate, index) order
                const double *cc = c_;
                std::sort(perm.begin() + t.begin, perm.begin() + t.end, [cc, axis](int64_t a, int64_t b) {
                    double ca = cc[3 * a + axis], cb = cc[3 * b + axis];
                    if (ca != cb) return ca < cb;
                    return a < b;
                });
                split = t.begin + (t.end - t.begin) / 2;
            } else {
                int64_t a = t.begin, b = t.begin + left;
                for (int64_t p = t.begin; p < t.end; ++p) {
                    int64_t q = perm[p];
                    if (c_[3 * q + axis] <= mid) scratch[a++] = q;
                    else scratch[b++] = q;
                }
                std::copy(scratch.begin() + t.begin, scratch.begin() + t.end, perm.begin() + t.begin);
                split = t.begin + left;
            }
            // right task below left so that the left subtree is numbered first
            stack.push_back({split, t.end, id, 1});
            stack.push_back({t.begin, split, id, 0});
        }
    }

  private:
    int64_t n_;
    const double *c_;
    int64_t leaf_;
};

// Block recursion in depth-first order, children in order.
void partition(const std::vector<Node> &nodes, double eta, std::vector<BlockRec> &out) {
    std::vector<std::pair<int64_t, int64_t>> stack;
    stack.push_back({0, 0});
    while (!stack.empty()) {
        auto [t, s] = stack.back();
        stack.pop_back();
        const Node &a = nodes[t], &b = nodes[s];
        double dist = gap_len(a, b);
        double dmin = std::min(diag_len(a), diag_len(b));
        if (dist > 0.0 && dmin <= eta * dist) {
            out.push_back(BlockRec{a.begin, a.end, b.begin, b.end, 1, 0, {}});
            continue;
        }
        bool tl = a.child0 < 0, sl = b.child0 < 0;
        if (tl && sl) {
            out.push_back(BlockRec{a.begin, a.end, b.begin, b.end, 0, 0, {}});
            continue;
        }
        int64_t tc[2] = {t, -1}, sc[2] = {s, -1};
        int nt = 1, ns = 1;
        if (!tl) { tc[0] = a.child0; tc[1] = a.child1; nt = 2; }
        if (!sl) { sc[0] = b.child0; sc[1] = b.child1; ns = 2; }
        for (int i = nt - 1; i >= 0; --i)
            for (int j = ns - 1; j >= 0; --j) stack.push_back({tc[i], sc[j]});
    }
}

// Adaptive cross approximation with partial pivoting of the m x n block
// entry(i, j).  Factors are kept column by column (u_l of length m, v_l of
// length n) and the approximant is sum_l u_l v_l^T.  Pivoting: start at row 0;
// column pivot = largest unused |row residual| (first on ties); a zero residual
// row is retired and the first unused row is tried; next row pivot = largest
// unused |u| (first on ties).  Stop when ||u|| ||v|| <= eps ||S||_F (running
// Frobenius norm of the approximant) or at rank min(m, n).
template <class Entry>
int64_t aca(int64_t m, int64_t n, const Entry &entry, double eps, std::vector<double> &U,
            std::vector<double> &V) {
    const int64_t rmax = std::min(m, n);
    std::vector<char> row_done(m, 0), col_done(n, 0);
    std::vector<double> row(n);
    U.clear();
    V.clear();
    int64_t r = 0, pr = 0;
    double fro2 = 0.0;
    while (r < rmax) {
        for (int64_t j = 0; j < n; ++j) {
            double s = entry(pr, j);
            for (int64_t l = 0; l < r; ++l) s -= U[l * m + pr] * V[l * n + j];
            row[j] = s;
        }
        row_done[pr] = 1;
        int64_t pc = -1;
        double best = -1.0;
        for (int64_t j = 0; j < n; ++j)
            if (!col_done[j] && std::fabs(row[j]) > best) { best = std::fabs(row[j]); pc = j; }
        if (pc < 0) break;
        if (row[pc] == 0.0) {
            int64_t nxt = -1;
            for (int64_t i = 0; i < m; ++i)
                if (!row_done[i]) { nxt = i; break; }
            if (nxt < 0) break;
            pr = nxt;
            continue;
        }
        const double pivot = row[pc];
        col_done[pc] = 1;
        U.resize((r + 1) * m);
        V.resize((r + 1) * n);
        double *u = U.data() + r * m, *v = V.data() + r * n;
        for (int64_t j = 0; j < n; ++j) v[j] = row[j] / pivot;
        for (int64_t i = 0; i < m; ++i) {
            double s = entry(i, pc);
            for (int64_t l = 0; l < r; ++l) s -= U[l * m + i] * V[l * n + pc];
            u[i] = s;
        }
        double uu = 0.0, vv = 0.0;
        for (int64_t i = 0; i < m; ++i) uu += u[i] * u[i];
        for (int64_t j = 0; j < n; ++j) vv += v[j] * v[j];
        double cross = 0.0;
        for (int64_t l = 0; l < r; ++l) {
            double ul = 0.0, vl = 0.0;
            for (int64_t i = 0; i < m; ++i) ul += U[l * m + i] * u[i];
            for (int64_t j = 0; j < n; ++j) vl += V[l * n + j] * v[j];
            cross += ul * vl;
        }
        fro2 += uu * vv + 2.0 * cross;
        ++r;
        if (std::sqrt(uu) * std::sqrt(vv) <= eps * std::sqrt(fro2)) break;
        int64_t nr = -1;
        best = -1.0;
        for (int64_t i = 0; i < m; ++i)
            if (!row_done[i] && std::fabs(u[i]) > best) { best = std::fabs(u[i]); nr = i; }
        if (nr < 0) break;
        pr = nr;
    }
    return r;
}

void fill(BlockRec &b, const Kernel &K, const std::vector<int64_t> &perm, double eps) {
    const int64_t m = b.ie - b.is, n = b.je - b.js;
    const int64_t *rows = perm.data() + b.is, *cols = perm.data() + b.js;
    auto entry = [&](int64_t i, int64_t j) { return K(rows[i], cols[j]); };
    if (b.kind == 1) {
        std::vector<double> U, V;
        int64_t r = aca(m, n, entry, eps, U, V);
        if (r * (m + n) >= m * n) {
            b.kind = 0;  // the factors would not be smaller than the block
        } else {
            b.rank = r;
            b.data.resize(r * (m + n));
            for (int64_t i = 0; i < m; ++i)
                for (int64_t l = 0; l < r; ++l) b.data[i * r + l] = U[l * m + i];  // V_m, #I x r
            std::copy(V.begin(), V.end(), b.data.begin() + m * r);              // W_m, r x #J
            return;
        }
    }
    b.rank = 0;
    b.data.resize(m * n);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) b.data[i * n + j] = entry(i, j);
}

int64_t align64(int64_t x) { return (x + 63) & ~int64_t(63); }

}  // namespace

namespace hmat_internal {

int plan_build(int64_t n, const double *centroids, const double *areas, int32_t leaf, double eta, double aca_eps,
               BuildPlan &plan) {
    if (!centroids || !areas || n < 1 || leaf < 1 || leaf > kMaxLeaf || !(eta >= 0.0) || !(aca_eps > 0.0) ||
        !std::isfinite(eta) || !std::isfinite(aca_eps))
        return HMAT_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (!std::isfinite(areas[i]) || areas[i] < 0.0) return HMAT_ERR_ARG;
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(centroids[3 * i + d])) return HMAT_ERR_ARG;
    }
    try {
        std::vector<Node> nodes;
        TreeBuilder(n, centroids, leaf).build(plan.perm, nodes);
        std::vector<BlockRec> blocks;
        partition(nodes, eta, blocks);
        plan.clusters.resize(4 * nodes.size());
        for (size_t k = 0; k < nodes.size(); ++k) {
            plan.clusters[4 * k + 0] = nodes[k].begin;
            plan.clusters[4 * k + 1] = nodes[k].end;
            plan.clusters[4 * k + 2] = nodes[k].child0;
            plan.clusters[4 * k + 3] = nodes[k].child1;
        }
        plan.blocks.resize(4 * blocks.size());
        plan.lowrank.resize(blocks.size());
        for (size_t b = 0; b < blocks.size(); ++b) {
            plan.blocks[4 * b + 0] = blocks[b].is;
            plan.blocks[4 * b + 1] = blocks[b].ie;
            plan.blocks[4 * b + 2] = blocks[b].js;
            plan.blocks[4 * b + 3] = blocks[b].je;
            plan.lowrank[b] = (uint8_t)blocks[b].kind;
        }
        plan.n = n;
        plan.leaf = leaf;
        plan.eta = eta;
        plan.aca_eps = aca_eps;
    } catch (const std::bad_alloc &) {
        return HMAT_ERR_NOMEM;
    }
    return HMAT_OK;
}

int serialize_blob(const BuildPlan &plan, const std::vector<int64_t> &kind, const std::vector<int64_t> &rank,
                   char **out, size_t *out_bytes, std::vector<int64_t> &data_off, int64_t *off_data_bytes) {
    const int64_t n = plan.n, nb = (int64_t)kind.size(), nc = (int64_t)plan.clusters.size() / 4;
    int64_t ndata = 0, dense_entries = 0, lr_entries = 0, rank_sum = 0, rank_max = 0;
    data_off.resize(nb);
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t *e = plan.blocks.data() + 4 * b;
        const int64_t m = e[1] - e[0], w = e[3] - e[2];
        const int64_t cnt = kind[b] == 0 ? m * w : rank[b] * (m + w);
        data_off[b] = ndata;
        ndata += cnt;
        if (kind[b] == 0) dense_entries += cnt;
        else {
            lr_entries += cnt;
            rank_sum += rank[b];
            rank_max = std::max(rank_max, rank[b]);
        }
    }
    const int64_t off_perm = kBlobHeaderBytes;
    const int64_t off_clusters = align64(off_perm + 8 * n);
    const int64_t off_blocks = align64(off_clusters + 32 * nc);
    const int64_t off_data = align64(off_blocks + 64 * nb);
    const int64_t total = align64(off_data + 8 * ndata);
    char *buf = (char *)std::calloc((size_t)total, 1);
    if (!buf) return HMAT_ERR_NOMEM;
    BlobHeader hdr{};
    std::memcpy(hdr.magic, kBlobMagic, 8);
    hdr.version = 1;
    hdr.header_bytes = kBlobHeaderBytes;
    hdr.n = n;
    hdr.nclusters = nc;
    hdr.nblocks = nb;
    hdr.ndata = ndata;
    hdr.leaf = plan.leaf;
    hdr.eta = plan.eta;
    hdr.aca_eps = plan.aca_eps;
    hdr.off_perm = off_perm;
    hdr.off_clusters = off_clusters;
    hdr.off_blocks = off_blocks;
    hdr.off_data = off_data;
    hdr.total_bytes = total;
    hdr.dense_entries = dense_entries;
    hdr.lr_entries = lr_entries;
    hdr.rank_sum = rank_sum;
    hdr.rank_max = rank_max;
    std::memcpy(buf, &hdr, sizeof(hdr));
    std::memcpy(buf + off_perm, plan.perm.data(), 8 * n);
    std::memcpy(buf + off_clusters, plan.clusters.data(), 32 * nc);
    int64_t *bt = (int64_t *)(buf + off_blocks);
    for (int64_t b = 0; b < nb; ++b) {
        int64_t *e = bt + 8 * b;
        const int64_t *pe = plan.blocks.data() + 4 * b;
        e[0] = pe[0]; e[1] = pe[1]; e[2] = pe[2]; e[3] = pe[3];
        e[4] = kind[b]; e[5] = kind[b] == 0 ? 0 : rank[b]; e[6] = data_off[b]; e[7] = 0;
    }
    *out = buf;
    *out_bytes = (size_t)total;
    *off_data_bytes = off_data;
    return HMAT_OK;
}

int host_block_data(const BuildPlan &plan, int64_t b, const double *centroids, const double *areas, int64_t *kind,
                    int64_t *rank, std::vector<double> &data) {
    try {
        const int64_t *e = plan.blocks.data() + 4 * b;
        BlockRec r{e[0], e[1], e[2], e[3], (int)plan.lowrank[b], 0, {}};
        fill(r, Kernel{centroids, areas}, plan.perm, plan.aca_eps);
        *kind = r.kind;
        *rank = r.rank;
        data = std::move(r.data);
    } catch (const std::bad_alloc &) {
        return HMAT_ERR_NOMEM;
    }
    return HMAT_OK;
}

}  // namespace hmat_internal

extern "C" int hmat_build(int64_t n, const double *centroids, const double *areas, int32_t leaf, double eta,
                          double aca_eps, void **blob, size_t *blob_bytes) {
    if (!blob || !blob_bytes) return HMAT_ERR_ARG;
    hmat_internal::BuildPlan plan;
    int st = hmat_internal::plan_build(n, centroids, areas, leaf, eta, aca_eps, plan);
    if (st != HMAT_OK) return st;
    try {
        const int64_t nb = (int64_t)plan.lowrank.size();
        std::vector<BlockRec> blocks(nb);
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t *e = plan.blocks.data() + 4 * b;
            blocks[b] = BlockRec{e[0], e[1], e[2], e[3], (int)plan.lowrank[b], 0, {}};
        }
        Kernel K{centroids, areas};
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t b = 0; b < nb; ++b) fill(blocks[b], K, plan.perm, aca_eps);
        std::vector<int64_t> kind(nb), rank(nb), off;
        for (int64_t b = 0; b < nb; ++b) {
            kind[b] = blocks[b].kind;
            rank[b] = blocks[b].rank;
        }
        char *buf = nullptr;
        size_t total = 0;
        int64_t off_data = 0;
        st = hmat_internal::serialize_blob(plan, kind, rank, &buf, &total, off, &off_data);
        if (st != HMAT_OK) return st;
        double *data = (double *)(buf + off_data);
        for (int64_t b = 0; b < nb; ++b)
            std::memcpy(data + off[b], blocks[b].data.data(), 8 * blocks[b].data.size());
        *blob = buf;
        *blob_bytes = total;
        return HMAT_OK;
    } catch (const std::bad_alloc &) {
        return HMAT_ERR_NOMEM;
    }
}

extern "C" void hmat_blob_free(void *blob) { std::free(blob); }
