// Device construction of the collocation H-matrix: the cluster tree and block
// partition come from the host planner (cheap tree work), the entries from
// the GPU -- adaptive cross approximation with partial pivoting of every
// admissible block (the low-rank factors V_m W_m of eq. 3-4, one CTA per
// block) and the dense blocks.  Every operation is the host builder's, in the
// same order (this file is compiled without FMA contraction; division and
// square root are IEEE round-to-nearest on both sides), so the blob is the host
// builder's bit for bit.  Sums the host takes in sequence (the norms of the
// stopping test) are taken by one thread each here; the argmax reductions
// keep the host's first-on-ties rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "hmat.h"
#include "hmat_internal.h"

namespace hmat_internal {

namespace {

constexpr int kAcaThreads = 256;
constexpr int kAcaRankCap = 64;  // ranks a block's workspace holds; beyond it the host finishes the block
constexpr double kPiD = 3.14159265358979323846;

struct AcaTask {
    int64_t m, n, is, js;  // block shape and first row / column (cluster order)
    int64_t uoff, voff;    // workspace of u_l (rcap x m) and v_l (rcap x n)
    int64_t foff;          // used-row / used-column flags (m + n bytes)
    int32_t rcap, rmax;    // workspace ranks; min(m, n)
};

struct PackTask {
    int64_t m, n, is, js, doff;  // block shape, first row / column, first value in the blob data
    int64_t uoff, voff;          // factors in the workspace (kind 1)
    int32_t kind, rank;          // 0: dense entries, 1: V_m then W_m from the workspace
};

// Collocation kernel in original indices (the host builder's expression).
__device__ __forceinline__ double entry(const double *__restrict__ c, const double *__restrict__ area, int64_t i,
                                        int64_t j) {
    if (i == j) return sqrt(area[i] / kPiD) / 2.0;
    const double dx = c[3 * i + 0] - c[3 * j + 0];
    const double dy = c[3 * i + 1] - c[3 * j + 1];
    const double dz = c[3 * i + 2] - c[3 * j + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    return area[j] / (4.0 * kPiD * r);
}

// (value, index) argmax over the CTA: the larger value wins, the smaller
// index on ties; value -1 / index INT64_MAX is "none".  Result in thread 0.
__device__ void argmax_cta(double &v, int64_t &idx, double *sv, int64_t *si) {
    sv[threadIdx.x] = v;
    si[threadIdx.x] = idx;
    __syncthreads();
    for (int s = kAcaThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double v2 = sv[threadIdx.x + s];
            const int64_t i2 = si[threadIdx.x + s];
            if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    v = sv[0];
    idx = si[0];
    __syncthreads();
}

// ACA with partial pivoting of one admissible block (the host builder's loop):
// row pivot 0 first; column pivot = largest unused |row residual| (first on
// ties); a zero pivot retires the row and tries the first unused one; next row
// pivot = largest unused |u| (first on ties); stop when ||u|| ||v|| <= eps
// ||S||_F with the running Frobenius norm, or at rank min(m, n).  Status:
// 0 the loop ended as on the host, 1 r (m + n) >= m n was reached (the block
// will be dense whatever follows), 2 the workspace's ranks ran out.
__global__ void __launch_bounds__(kAcaThreads) k_aca(const AcaTask *__restrict__ tasks, const double *__restrict__ c,
                                                      const double *__restrict__ area,
                                                      const int64_t *__restrict__ perm, double *ws, uint8_t *flags,
                                                      double eps, int32_t *rank_out, int32_t *status_out) {
    __shared__ double sv[kAcaThreads];
    __shared__ int64_t si[kAcaThreads];
    __shared__ double sdot[2 + 2 * kAcaRankCap];
    __shared__ double s_pivot;
    __shared__ int s_stop;
    const AcaTask T = tasks[blockIdx.x];
    const int64_t m = T.m, n = T.n;
    const int64_t *rows = perm + T.is, *cols = perm + T.js;
    double *U = ws + T.uoff, *V = ws + T.voff;
    uint8_t *rdone = flags + T.foff, *cdone = rdone + m;
    const int tid = threadIdx.x;
    for (int64_t k = tid; k < m + n; k += kAcaThreads) rdone[k] = 0;
    __syncthreads();
    int64_t r = 0, pr = 0;
    double fro2 = 0.0;  // thread 0's
    int status = 0;
    while (r < T.rmax) {
        if (r >= T.rcap) { status = 2; break; }
        double *row = V + r * n;  // the row residual, divided in place into v_r
        const int64_t gi = rows[pr];
        for (int64_t j = tid; j < n; j += kAcaThreads) {
            double s = entry(c, area, gi, cols[j]);
            for (int64_t l = 0; l < r; ++l) s -= U[l * m + pr] * V[l * n + j];
            row[j] = s;
        }
        __syncthreads();
        if (tid == 0) rdone[pr] = 1;
        double bv = -1.0;
        int64_t bi = INT64_MAX;
        for (int64_t j = tid; j < n; j += kAcaThreads)
            if (!cdone[j] && fabs(row[j]) > bv) { bv = fabs(row[j]); bi = j; }
        argmax_cta(bv, bi, sv, si);  // also orders rdone[pr] before the row search below
        if (bi == INT64_MAX) break;
        const int64_t pc = bi;
        if (row[pc] == 0.0) {
            int64_t nxt = INT64_MAX;
            for (int64_t i = tid; i < m; i += kAcaThreads)
                if (!rdone[i]) { nxt = i; break; }
            double dummy = 0.0;  // smallest unused row: an argmax with equal values picks the smallest index
            argmax_cta(dummy, nxt, sv, si);
            if (nxt == INT64_MAX) break;
            pr = nxt;
            continue;
        }
        if (tid == 0) {
            s_pivot = row[pc];
            cdone[pc] = 1;
        }
        __syncthreads();
        const double pivot = s_pivot;
        double *u = U + r * m, *v = row;
        for (int64_t j = tid; j < n; j += kAcaThreads) v[j] = row[j] / pivot;
        for (int64_t i = tid; i < m; i += kAcaThreads) {
            double s = entry(c, area, rows[i], cols[pc]);
            for (int64_t l = 0; l < r; ++l) s -= U[l * m + i] * V[l * n + pc];
            u[i] = s;
        }
        __syncthreads();
        // the stopping test's sums, each in the host's order by one thread
        if (tid == 0) {
            double a = 0.0;
            for (int64_t i = 0; i < m; ++i) a += u[i] * u[i];
            sdot[0] = a;
        } else if (tid == 1) {
            double a = 0.0;
            for (int64_t j = 0; j < n; ++j) a += v[j] * v[j];
            sdot[1] = a;
        } else if (tid - 2 < 2 * r) {
            const int64_t l = (tid - 2) >> 1;
            double a = 0.0;
            if (((tid - 2) & 1) == 0)
                for (int64_t i = 0; i < m; ++i) a += U[l * m + i] * u[i];
            else
                for (int64_t j = 0; j < n; ++j) a += V[l * n + j] * v[j];
            sdot[2 + (tid - 2)] = a;
        }
        __syncthreads();
        if (tid == 0) {
            const double uu = sdot[0], vv = sdot[1];
            double cross = 0.0;
            for (int64_t l = 0; l < r; ++l) cross += sdot[2 + 2 * l] * sdot[3 + 2 * l];
            fro2 += uu * vv + 2.0 * cross;
            s_stop = sqrt(uu) * sqrt(vv) <= eps * sqrt(fro2);
        }
        __syncthreads();
        ++r;
        if (s_stop) break;
        if (r * (m + n) >= m * n) { status = 1; break; }
        bv = -1.0;
        bi = INT64_MAX;
        for (int64_t i = tid; i < m; i += kAcaThreads)
            if (!rdone[i] && fabs(u[i]) > bv) { bv = fabs(u[i]); bi = i; }
        argmax_cta(bv, bi, sv, si);
        if (bi == INT64_MAX) break;
        pr = bi;
    }
    if (tid == 0) {
        rank_out[blockIdx.x] = (int32_t)r;
        status_out[blockIdx.x] = status;
    }
}

// Blob values of one block: the dense entries, or V_m (#I x r, row-major, from
// the columns u_l) followed by W_m (r x #J, the rows v_l).
__global__ void __launch_bounds__(kAcaThreads) k_pack(const PackTask *__restrict__ tasks,
                                                       const double *__restrict__ c, const double *__restrict__ area,
                                                       const int64_t *__restrict__ perm, const double *__restrict__ ws,
                                                       double *__restrict__ data) {
    const PackTask T = tasks[blockIdx.x];
    double *out = data + T.doff;
    if (T.kind == 1) {
        const int64_t r = T.rank;
        const double *U = ws + T.uoff, *V = ws + T.voff;
        for (int64_t k = threadIdx.x; k < T.m * r; k += kAcaThreads) {
            const int64_t i = k / r, l = k - i * r;
            out[k] = U[l * T.m + i];
        }
        for (int64_t k = threadIdx.x; k < r * T.n; k += kAcaThreads) out[T.m * r + k] = V[k];
        return;
    }
    const int64_t *rows = perm + T.is, *cols = perm + T.js;
    for (int64_t k = threadIdx.x; k < T.m * T.n; k += kAcaThreads) {
        const int64_t i = k / T.n, j = k - i * T.n;
        out[k] = entry(c, area, rows[i], cols[j]);
    }
}

// device buffers of one build, released on every path
struct DevBufs {
    std::vector<void *> p;
    ~DevBufs() {
        for (void *q : p) cudaFree(q);
    }
    template <class T> cudaError_t alloc(T **ptr, size_t bytes) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
        if (e == cudaSuccess) {
            p.push_back(q);
            *ptr = (T *)q;
        }
        return e;
    }
};

int cuda_status(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return HMAT_ERR_NOMEM;
    }
    return e == cudaSuccess ? HMAT_OK : HMAT_ERR_CUDA;
}

}  // namespace

int build_device(int64_t n, const double *centroids, const double *areas, int32_t leaf, double eta, double aca_eps,
                 void **blob, size_t *blob_bytes, hmat_build_device_info *info) {
    if (!blob || !blob_bytes) return HMAT_ERR_ARG;
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t0) { return std::chrono::duration<double, std::milli>(clk::now() - t0).count(); };
    const clk::time_point t_plan = clk::now();
    BuildPlan plan;
    int st = plan_build(n, centroids, areas, leaf, eta, aca_eps, plan);
    if (st != HMAT_OK) return st;
    const double plan_ms = ms_since(t_plan);
    clk::time_point t_stage = clk::now();
    const int64_t nb = (int64_t)plan.lowrank.size();
    // ACA tasks and their workspace
    std::vector<AcaTask> aca;
    std::vector<int64_t> aca_block;
    int64_t ws_len = 0, fl_len = 0;
    for (int64_t b = 0; b < nb; ++b) {
        if (!plan.lowrank[b]) continue;
        const int64_t *e = plan.blocks.data() + 4 * b;
        const int64_t m = e[1] - e[0], w = e[3] - e[2];
        const int64_t rmax = std::min(m, w);
        // ranks past ceil(m w / (m + w)) make the block dense, so never need storing
        const int64_t rdense = (m * w + (m + w) - 1) / (m + w);
        const int32_t rcap = (int32_t)std::min<int64_t>({rmax, rdense, (int64_t)kAcaRankCap});
        AcaTask t{m, w, e[0], e[2], ws_len, ws_len + rcap * m, fl_len, rcap, (int32_t)rmax};
        ws_len += (int64_t)rcap * (m + w);
        fl_len += m + w;
        aca.push_back(t);
        aca_block.push_back(b);
    }
    const int64_t na = (int64_t)aca.size();
    DevBufs D;
    double *dc = nullptr, *da = nullptr, *dws = nullptr, *ddata = nullptr;
    int64_t *dperm = nullptr;
    uint8_t *dfl = nullptr;
    AcaTask *dtask = nullptr;
    int32_t *drank = nullptr, *dstat = nullptr;
    cudaError_t e;
    if ((e = D.alloc(&dc, 24 * n)) || (e = D.alloc(&da, 8 * n)) || (e = D.alloc(&dperm, 8 * n)) ||
        (e = D.alloc(&dws, 8 * ws_len)) || (e = D.alloc(&dfl, fl_len)) || (e = D.alloc(&dtask, sizeof(AcaTask) * na)) ||
        (e = D.alloc(&drank, 4 * na)) || (e = D.alloc(&dstat, 4 * na)))
        return cuda_status(e);
    if ((e = cudaMemcpy(dc, centroids, 24 * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(da, areas, 8 * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(dperm, plan.perm.data(), 8 * n, cudaMemcpyHostToDevice)) ||
        (na && (e = cudaMemcpy(dtask, aca.data(), sizeof(AcaTask) * na, cudaMemcpyHostToDevice))))
        return cuda_status(e);
    const double alloc_ms = ms_since(t_stage);
    t_stage = clk::now();
    if (na) k_aca<<<(unsigned)na, kAcaThreads>>>(dtask, dc, da, dperm, dws, dfl, aca_eps, drank, dstat);
    std::vector<int32_t> hrank(na), hstat(na);
    if ((e = cudaGetLastError()) || (na && (e = cudaMemcpy(hrank.data(), drank, 4 * na, cudaMemcpyDeviceToHost))) ||
        (na && (e = cudaMemcpy(hstat.data(), dstat, 4 * na, cudaMemcpyDeviceToHost))))
        return cuda_status(e);
    const double aca_ms = ms_since(t_stage);
    t_stage = clk::now();
    // kinds and ranks as the host builder decides them; blocks whose ranks
    // outgrew the workspace are finished by the host builder's own ACA
    std::vector<int64_t> kind(nb, 0), rank(nb, 0);
    std::vector<int64_t> host_blocks;
    std::vector<std::vector<double>> host_data;
    std::vector<int32_t> task_of(nb, -1);
    for (int64_t k = 0; k < na; ++k) {
        const int64_t b = aca_block[k];
        const AcaTask &t = aca[k];
        task_of[b] = (int32_t)k;
        if (hstat[k] == 2) {
            host_blocks.push_back(b);
            continue;
        }
        if (hstat[k] == 0 && (int64_t)hrank[k] * (t.m + t.n) < t.m * t.n) {
            kind[b] = 1;
            rank[b] = hrank[k];
        }
    }
    host_data.resize(host_blocks.size());
    for (size_t k = 0; k < host_blocks.size(); ++k) {
        const int64_t b = host_blocks[k];
        st = host_block_data(plan, b, centroids, areas, &kind[b], &rank[b], host_data[k]);
        if (st != HMAT_OK) return st;
    }
    char *buf = nullptr;
    size_t total = 0;
    int64_t off_data = 0;
    std::vector<int64_t> doff;
    st = serialize_blob(plan, kind, rank, &buf, &total, doff, &off_data);
    if (st != HMAT_OK) return st;
    const int64_t ndata = (int64_t)((total - (size_t)off_data) / 8);
    std::vector<PackTask> pack;
    for (int64_t b = 0; b < nb; ++b) {
        if (std::find(host_blocks.begin(), host_blocks.end(), b) != host_blocks.end()) continue;
        const int64_t *q = plan.blocks.data() + 4 * b;
        PackTask t{q[1] - q[0], q[3] - q[2], q[0], q[2], doff[b], 0, 0, (int32_t)kind[b], (int32_t)rank[b]};
        if (kind[b] == 1) {
            t.uoff = aca[task_of[b]].uoff;
            t.voff = aca[task_of[b]].voff;
        }
        pack.push_back(t);
    }
    PackTask *dpack = nullptr;
    if ((e = D.alloc(&ddata, 8 * ndata)) || (e = D.alloc(&dpack, sizeof(PackTask) * pack.size())) ||
        (!pack.empty() && (e = cudaMemcpy(dpack, pack.data(), sizeof(PackTask) * pack.size(), cudaMemcpyHostToDevice)))) {
        std::free(buf);
        return cuda_status(e);
    }
    if (!pack.empty()) k_pack<<<(unsigned)pack.size(), kAcaThreads>>>(dpack, dc, da, dperm, dws, ddata);
    if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize())) {
        std::free(buf);
        return cuda_status(e);
    }
    const double pack_ms = ms_since(t_stage);
    const clk::time_point t_copy = clk::now();
    if ((e = cudaMemcpy(buf + off_data, ddata, 8 * ndata, cudaMemcpyDeviceToHost))) {
        std::free(buf);
        return cuda_status(e);
    }
    const double copy_ms = ms_since(t_copy);
    for (size_t k = 0; k < host_blocks.size(); ++k)
        std::memcpy(buf + off_data + 8 * doff[host_blocks[k]], host_data[k].data(), 8 * host_data[k].size());
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->aca_blocks = na;
        info->host_blocks = (int64_t)host_blocks.size();
        info->workspace_bytes = 8 * ws_len + fl_len;
        info->plan_ms = plan_ms;
        info->alloc_ms = alloc_ms;
        info->aca_ms = aca_ms;
        info->pack_ms = pack_ms;
        info->copy_ms = copy_ms;
    }
    *blob = buf;
    *blob_bytes = total;
    return HMAT_OK;
}

}  // namespace hmat_internal

extern "C" int hmat_build_device(int64_t n, const double *centroids, const double *areas, int32_t leaf, double eta,
                                 double aca_eps, void **blob, size_t *blob_bytes, hmat_build_device_info *info) {
    return hmat_internal::build_device(n, centroids, areas, leaf, eta, aca_eps, blob, blob_bytes, info);
}
