// Internal declarations of the hmat library (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

struct hmat_build_device_info;

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

// Cluster tree and block partition of the collocation H-matrix (host), the
// part of the build shared by the host builder and the device ACA builder.
struct BuildPlan {
    int64_t n = 0;
    int32_t leaf = 0;
    double eta = 0.0, aca_eps = 0.0;
    std::vector<int64_t> perm;      // cluster order -> original index
    std::vector<int64_t> clusters;  // [nc][4] begin, end, child0, child1
    std::vector<int64_t> blocks;    // [nb][4] i_s, i_e, j_s, j_e (partition order)
    std::vector<uint8_t> lowrank;   // per block: 1 admissible (ACA), 0 dense
};
// Validates the arguments as hmat_build does.
int plan_build(int64_t n, const double *centroids, const double *areas, int32_t leaf, double eta, double aca_eps,
               BuildPlan &plan);
// A blob buffer (calloc'ed) with header, perm, clusters and block table written
// for the given kinds (0 dense, 1 low rank) and ranks; data_off[b] is block b's
// first value, the data section starts at *off_data_bytes and is left zero.
int serialize_blob(const BuildPlan &plan, const std::vector<int64_t> &kind, const std::vector<int64_t> &rank,
                   char **out, size_t *out_bytes, std::vector<int64_t> &data_off, int64_t *off_data_bytes);

// The host builder's ACA and dense fill of block b of the plan (kind 0 dense,
// 1 low rank; data as in the blob).
int host_block_data(const BuildPlan &plan, int64_t b, const double *centroids, const double *areas, int64_t *kind,
                    int64_t *rank, std::vector<double> &data);

// A validated, read-only view of a blob.
struct BlobView {
    const BlobHeader *h = nullptr;
    const int64_t *perm = nullptr;
    const int64_t *clusters = nullptr;  // [nc][4]
    const int64_t *blocks = nullptr;    // [nb][8]
    const double *data = nullptr;
    std::vector<int64_t> leaf_begin;    // nleaves + 1 boundaries of the leaf clusters
    // derived block lists of the paper's variants (not set for a parsed blob):
    bool pow2 = true;                   // false: arrays stored unscaled
    const int64_t *toff = nullptr;      // per block: first tval of its ranks, or -1
    const double *tval = nullptr;       // d_l of eq. (14)-(16) multiplied into t (eq. 23)
    // kind 2 blocks (a dense block restricted to some of its columns, stored
    // #I x e[5] row-major): their e[5] columns, ascending, at dcols[e[7] ...]
    const int32_t *dcols = nullptr;
};

// dense blocks: kind 0 (every column) or kind 2 (the columns listed in dcols)
inline bool block_is_dense(const int64_t *e) { return e[4] == 0 || e[4] == 2; }
inline int64_t dense_width(const int64_t *e) { return e[4] == 2 ? e[5] : e[3] - e[2]; }

// Validate a blob; on success fill `view`.  Returns an hmat_status.
int parse_blob(const void *blob, size_t bytes, BlobView &view, std::string *why = nullptr);

// ---- packed device layout (host-side description) ----
// The product runs in two launches over leaf clusters.
//
// Phase 1, one work item per leaf column cluster kappa: a row-major |kappa| x R
// panel whose columns are the rank vectors of every W_m (eq. 9/22) whose column
// cluster contains kappa, restricted to kappa.  Its R dot products with x_kappa
// (the contributions t_{m,kappa} = W_m|kappa x_kappa of its blocks, in panel
// column order) are stored contiguously in the projection output T at tbeg.  A
// reduction launch then forms every block's t_m = sum over the leaf clusters
// kappa of its column cluster of t_{m,kappa}, in cluster order (one term when the
// column cluster is a leaf).  Phase 1 and the reduction write every operand
// phase 2 needs into per-row-cluster operand buffers g: the slices 2^e x_kappa
// of the dense blocks over kappa (phase 1), and each block's 2^e t for every leaf
// row cluster of the block (the reduction).
//
// Phase 2, one work item per leaf row cluster rho: a row-major |rho| x K panel
// holding the rows over rho of every dense block (eq. 21) and of every V_m
// (eq. 10/24) whose row cluster contains rho; y_rho = P_rho g_rho.
struct P1Desc {
    int64_t off;    // element offset of the panel
    int32_t R;      // columns
    int32_t ld;     // row stride (R rounded up to kPadElems)
    int32_t rbeg;   // first P1Run
    int32_t rcnt;   // runs (one per low-rank block over kappa)
    int32_t xbeg;   // first row of kappa (cluster order)
    int32_t xlen;   // rows of kappa
    int32_t xdbeg;  // first XDst (dense-block operand slices fed from x_kappa)
    int32_t xdcnt;
    int32_t tbeg;    // first entry of the cluster's projection output in T (ld entries)
    int32_t pad[1];  // on the device: pad[0] = the item's problem (batch handles)
};
struct P1Run {      // one low-rank block of a phase-1 panel (host side)
    int32_t col0;   // first panel column of the block
    int32_t len;    // rank r
    int32_t q;      // low-rank block index (LrDesc)
    int32_t pad;
};
struct LrDesc {
    int32_t boff;   // first of its cnt entries of tofs: where t_{m,kappa} starts in T, kappa in cluster order
    int32_t cnt;    // leaf clusters inside the column cluster
    int32_t rank;
    int32_t scale;  // exponent e of 2^e t
    int32_t gbeg;   // first entry of gdst (one per leaf row cluster of the block)
    int32_t gcnt;
    int32_t toff;   // first per-rank factor d_l of t = d_l z_l (eq. 23), or -1
    int32_t pad;    // on the device: the block's problem (batch handles)
};
// One rank of a low-rank block whose column cluster is a leaf and whose row
// cluster is a leaf: its t_m entry is its one projection, and it feeds one
// operand slot, so the reduction copies it without the block's descriptor.
struct RedDirect {
    int32_t tsrc;   // entry of T holding t_{m,kappa} of this rank
    int32_t gdst;   // operand slot in g
    int32_t scale;  // exponent e of 2^e t
    int32_t prob;   // on the device: the block's problem (batch handles)
};
struct XDst {
    int32_t goff;   // operand index of the slice's first entry in g
    int32_t scale;  // exponent e
    int32_t cnt;    // operands written: |kappa| for a whole slice, fewer for a column subset
    int32_t sel;    // -1: x_kappa[0..cnt) in order; else first of cnt local indices in Layout::xsel
};
struct P2Desc {
    int64_t off;    // element offset of the panel
    int32_t K;      // columns
    int32_t ld;     // row stride (K rounded up to kPadElems)
    int32_t goff;   // first operand of g_rho (ld operands, zero past K)
    int32_t ybeg;   // first row (cluster order)
    int32_t ylen;
    int32_t pad;
};

// One row of the phase-2 panels (the row-persistent expansion's work item).
struct RowDesc {
    int64_t off;    // element offset of the row
    int32_t goff;   // first operand of its leaf row cluster
    int32_t ld;     // entries (the cluster's panel stride; 0 for no row)
};

// Up to kGroupRows consecutive rows of one leaf row cluster (the row-group
// expansion's work item).
constexpr int kGroupRows = 4;
struct GroupDesc {
    int64_t off;    // element offset of the first row
    int32_t goff;   // first operand of the leaf row cluster
    int32_t ld;     // entries per row
    int32_t p0;     // first row (cluster order)
    int32_t nr;     // rows (1..kGroupRows)
    int32_t pad[2];  // on the device: pad[0] = the group's problem (batch handles)
};

constexpr int kMaxScaleExp = 120;  // |e| of every stored power-of-two scale
constexpr int kRedBigCnt = 32;     // blocks over this many leaf clusters are reduced by a whole CTA

struct Layout {
    int64_t n = 0;
    int32_t nleaves = 0;
    std::vector<int32_t> perm;        // perm[p] = original index
    std::vector<int32_t> leaf_begin;  // nleaves + 1
    std::vector<RowDesc> rows;        // [n] every row's place in the phase-2 panels (cluster order)
    std::vector<GroupDesc> groups;    // row groups of the leaf row clusters, in cluster order
    std::vector<P1Desc> p1;
    std::vector<P1Run> p1_runs;
    std::vector<XDst> xdst;
    std::vector<int32_t> xsel;       // local indices of the column-subset slices (XDst::sel)
    std::vector<LrDesc> lr;
    std::vector<int32_t> gdst;
    std::vector<P2Desc> p2;
    int64_t p1_elems = 0, p2_elems = 0;
    int64_t npart = 0, glen = 0;     // entries of T (the phase-1 panels' ld summed) and of g
    std::vector<int32_t> tofs;       // LrDesc::boff: T offsets of each block's per-cluster projections
    std::vector<double> tscale;      // per-rank factors referenced by LrDesc::toff
    std::vector<int32_t> red_big;    // multi-cluster blocks over >= kRedBigCnt clusters (a CTA each)
    std::vector<int32_t> red_tasks;  // (block << 6) | rank of the other low-rank blocks (a lane each) ...
    std::vector<RedDirect> red_direct;  // ... but the ranks of single-leaf blocks without factors d_l
    std::vector<int32_t> red_direct_q;  // (host) the low-rank block of each red_direct entry
    int32_t max_ld2 = 0, max_ld1 = 0, max_runs1 = 0, max_leaf = 0;
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
//   F64, DF, F32, BF16  the library's own forms
//   PM, PS, PM1, PS2    FP32 panels of the paper's variants (classes M, S, M1
//                       and S2 of paper_forms.cpp)
enum class Store { F64, DF, F32, BF16, PM, PS, PM1, PS2 };
size_t store_bytes(Store s);
void fill_panels(const BlobView &v, const Layout &L, Store s, void *q1, void *p2);
// the BF16 value the panels store for v (round to nearest, ties to even): its 16 bits
uint16_t bf16_bits(double v);

// One segment of a paper variant: a derived block list over the cluster tree
// of the source blob, with its own arrays (`view` points into this object).
struct DerivedSegment {
    BlobHeader hdr{};
    std::vector<int64_t> blocks;  // [nb][8] like the blob
    std::vector<double> data;
    std::vector<int64_t> toff;    // per block
    std::vector<double> tval;
    std::vector<int32_t> dcols;   // column lists of the kind 2 blocks
    BlobView view;
    DerivedSegment() = default;
    DerivedSegment(const DerivedSegment &) = delete;
    DerivedSegment &operator=(const DerivedSegment &) = delete;
    DerivedSegment(DerivedSegment &&) = default;
    DerivedSegment &operator=(DerivedSegment &&) = default;
};

// Independent problems as one block-diagonal operator (`view` points into this
// object; offsets[p] = first row of problem p, offsets[count] = n).
struct CombinedBlob {
    BlobHeader hdr{};
    std::vector<int64_t> perm, blocks, offsets;
    std::vector<double> data;
    BlobView view;
    CombinedBlob() = default;
    CombinedBlob(const CombinedBlob &) = delete;
    CombinedBlob &operator=(const CombinedBlob &) = delete;
    CombinedBlob(CombinedBlob &&) = default;
    CombinedBlob &operator=(CombinedBlob &&) = default;
};
int combine_blobs(const BlobView *views, int count, CombinedBlob &out, std::string *why = nullptr);

// Split a validated blob into the segments of a paper variant (precision
// HMAT_M1_SINGLE .. HMAT_M3, `c` of eq. 19-20 for Method 3).  Sets nseg (1 or 2)
// and the store of each segment.  Returns an hmat_status.
int derive_table1(const BlobView &v, int precision, int c, DerivedSegment (&seg)[2], Store (&store)[2], int *nseg,
                  std::string *why = nullptr);

}  // namespace hmat_internal
