// Internal declarations of the hmat library (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace hmat_internal {

constexpr int kMaxLeaf = 64;               // rows of a leaf cluster the kernels accept
constexpr int kBlobHeaderBytes = 256;
constexpr char kBlobMagic[8] = {'H', 'M', 'A', 'T', 'B', 'L', 'B', '1'};
constexpr int kPadElems = 8;               // row strides are multiples of 8 entries (16 B of BF16)

struct BlobHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int64_t n, nclusters, nblocks, ndata, leaf;
    double eta, aca_eps;
    int64_t off_perm, off_clusters, off_blocks, off_data, total_bytes;
    int64_t dense_entries, lr_entries, rank_sum, rank_max;
};
static_assert(sizeof(BlobHeader) <= kBlobHeaderBytes, "header too large");

// A validated, read-only view of a blob.
struct BlobView {
    const BlobHeader *h = nullptr;
    const int64_t *perm = nullptr;
    const int64_t *clusters = nullptr;  // [nc][4]
    const int64_t *blocks = nullptr;    // [nb][8]
    const double *data = nullptr;
    std::vector<int64_t> leaf_begin;    // nleaves + 1 boundaries of the leaf clusters
};

// Validate a blob; on success fill `view`.  Returns an hmat_status.
int parse_blob(const void *blob, size_t bytes, BlobView &view, std::string *why = nullptr);

// ---- packed device layout (host-side description) ----
// Phase 1 (projection t = W x), one work item per leaf column cluster kappa:
// a row-major |kappa| x R panel whose column c holds one rank vector of one
// low-rank block restricted to kappa; its R dot products with x_kappa go, per
// block (a run of r columns), either straight to t (a block whose column
// cluster is kappa itself) or to the block's partial sums.
struct P1Desc {
    int64_t off;   // element offset of the panel
    int32_t R;     // columns
    int32_t ld;    // row stride (R rounded up to kPadElems)
    int32_t rbeg;  // first output run (Run: dst = first column, src = first output index,
                   // info = kind (0 t, 1 partial) | (scale exponent + 512) << 8)
    int32_t xbeg;  // first row of kappa (cluster order)
    int32_t xlen;  // rows of kappa
    int32_t rcnt;  // output runs
};
// Reduction of the partials of one low-rank block spanning several leaf
// clusters: t[toff + l] = 2^scale sum_k partial[boff + k rank + l].
struct RdDesc {
    int32_t boff;   // first partial (block-major: cnt rows of rank values)
    int32_t cnt;    // number of leaf clusters kappa inside sigma
    int32_t toff;   // first t entry of the block
    int32_t rank;
    int32_t scale;  // exponent e
    int32_t pad[3];
};
// Phase 2 (expansion y = D x + V t), one work item per leaf row cluster rho:
// a row-major |rho| x K panel; columns come in runs (dense block slices reading
// the source vector, then low-rank slices reading t).
struct P2Desc {
    int64_t off;
    int32_t K;
    int32_t ld;
    int32_t rbeg;  // first run
    int32_t rcnt;  // runs
    int32_t ybeg;  // first row (cluster order)
    int32_t ylen;
};
struct Run {
    int32_t dst;    // first column of the run in the panel
    int32_t src;    // first source index: cluster-order x index (kind 0) or t index (kind 1)
    int32_t len;
    int32_t info;   // kind | (scale exponent + 512) << 8
};

struct Layout {
    int64_t n = 0;
    int32_t nleaves = 0;
    std::vector<int32_t> perm;        // perm[p] = original index
    std::vector<int32_t> leaf_begin;  // nleaves + 1
    std::vector<P1Desc> p1;
    std::vector<RdDesc> rd;
    std::vector<Run> p1_runs;
    std::vector<P2Desc> p2;
    std::vector<Run> runs;
    int64_t p1_elems = 0, p2_elems = 0;
    int64_t npart = 0, tlen = 0;
    int32_t max_runs = 0, max_ld2 = 0, max_ld1 = 0, max_runs1 = 0;
    int64_t stored_entries = 0, phase1_entries = 0, phase2_entries = 0, rank_sum = 0;
    // source of each packed entry, used to fill typed panels without
    // materialising an FP64 copy: per P1/P2 work item, the list of block slices
    struct Slice {
        int64_t block;   // blob block index
        int32_t col0;    // first panel column
        int32_t ncols;   // columns
        int32_t row0;    // first row of the block covered by the work item
        int32_t kind;    // 0 dense (row-major D rows), 1 LR factor V_m rows (phase 2) / W_m^T rows (phase 1)
        int32_t scale;   // exponent e of the stored array: value / 2^e is packed
    };
    std::vector<int64_t> p1_slice_ptr, p2_slice_ptr;
    std::vector<Slice> p1_slices, p2_slices;
};

int build_layout(const BlobView &v, Layout &L, std::string *why = nullptr);
// Bounds invariants of every index the kernels form (defence in depth).
int check_layout(const Layout &L, std::string *why = nullptr);

// Fill typed panels from the blob according to the layout.
enum class Store { F64, DF, F32, BF16 };
size_t store_bytes(Store s);
void fill_panels(const BlobView &v, const Layout &L, Store s, void *q1, void *p2);

}  // namespace hmat_internal
