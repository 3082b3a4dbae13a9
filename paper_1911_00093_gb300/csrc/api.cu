// C ABI of the hmat library: upload, product, BiCG-STAB driver, introspection.
#include <cuda_runtime.h>

#include <algorithm>
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

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

Store store_of(int precision) {
    switch (precision) {
    case HMAT_FP64: return Store::DF;
    case HMAT_FP64_DFMA: return Store::F64;
    case HMAT_FP32: return Store::F32;
    default: return Store::BF16;
    }
}

}  // namespace

namespace {

// y = A~ x for one vector, everything on the device.
//   x_orig != nullptr: source in original order (gathered); else the operand copy P.xs is ready
//   out_perm != nullptr: y written in original order
void enqueue_product(hmat_t *h, const DevPanels &P, Store s, const double *x_src, const int32_t *src_perm,
                     double *y, const int32_t *out_perm, const SolverScalars *skipS, int mode, cudaStream_t st) {
    if (x_src) launch_prep(s, h->ix, x_src, src_perm, P.xs, st);
    launch_phase1(s, h->ix, P, skipS, mode, st);
    launch_reduce(s, h->ix, P, skipS, mode, st);
    launch_phase2(s, h->ix, P, y, out_perm, skipS, mode, st);
}

int alloc_panels(hmat_t *h, const BlobView &v, const Layout &L, Store s, DevPanels &P, int64_t *bytes_out) {
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
    st = h->alloc(&P.xs, (size_t)L.n * operand_bytes(s));
    if (st) return st;
    st = h->alloc(&P.part, (size_t)std::max<int64_t>(L.npart, 1) * partial_bytes(s));
    if (st) return st;
    st = h->alloc(&P.g, (size_t)std::max<int64_t>(L.glen, 1) * operand_bytes(s));
    if (st) return st;
    CK(cudaMemset(P.g, 0, (size_t)std::max<int64_t>(L.glen, 1) * operand_bytes(s)));  // zero padding columns
    *bytes_out = (int64_t)(b1 + b2);
    return HMAT_OK;
}

}  // namespace

extern "C" int hmat_upload(const void *blob, size_t blob_bytes, int32_t precision, hmat_handle *out) {
    if (!blob || !out) return HMAT_ERR_ARG;
    if (precision < HMAT_FP64 || precision > HMAT_BF16) return HMAT_ERR_ARG;
    *out = nullptr;
    BlobView v;
    int st = parse_blob(blob, blob_bytes, v);
    if (st != HMAT_OK) return st;
    std::unique_ptr<hmat_t> hp;
    try {
        hp.reset(new hmat_t());
        hmat_t *h = hp.get();
        Layout L;
        st = build_layout(v, L);
        if (st == HMAT_OK) st = check_layout(L);
        if (st != HMAT_OK) return st;
        CK(cudaGetDevice(&h->device));
        h->precision = precision;
        h->store = store_of(precision);
        h->store64 = precision == HMAT_FP64_DFMA ? Store::F64 : Store::DF;
        h->separate64 = !(precision == HMAT_FP64 || precision == HMAT_FP64_DFMA);
        h->stored_entries = L.stored_entries;
        h->phase1_entries = L.phase1_entries;
        h->phase2_entries = L.phase2_entries;
        h->partials_n = L.npart;
        h->glen = L.glen;
        h->rank_sum = L.rank_sum;

        // indices
        DevIndex &ix = h->ix;
        ix.n = (int32_t)L.n;
        ix.nleaves = L.nleaves;
        ix.nlr = (int32_t)L.lr.size();
        ix.nbig = (int32_t)L.red_big.size();
        ix.ntasks = (int32_t)L.red_tasks.size();
        ix.max_leaf = L.max_leaf;
        ix.max_ld2 = L.max_ld2;
        int32_t *perm = nullptr, *gdst = nullptr, *red_big = nullptr, *red_tasks = nullptr;
        P1Desc *p1 = nullptr;
        P1Run *p1_runs = nullptr;
        XDst *xdst = nullptr;
        LrDesc *lr = nullptr;
        P2Desc *p2 = nullptr;
        if ((st = h->upload(&perm, L.perm.data(), 4 * L.perm.size())) ||
            (st = h->upload(&p1, L.p1.data(), sizeof(P1Desc) * L.p1.size())) ||
            (st = h->upload(&p1_runs, L.p1_runs.data(), sizeof(P1Run) * L.p1_runs.size())) ||
            (st = h->upload(&xdst, L.xdst.data(), sizeof(XDst) * L.xdst.size())) ||
            (st = h->upload(&lr, L.lr.data(), sizeof(LrDesc) * L.lr.size())) ||
            (st = h->upload(&gdst, L.gdst.data(), 4 * L.gdst.size())) ||
            (st = h->upload(&red_big, L.red_big.data(), 4 * L.red_big.size())) ||
            (st = h->upload(&red_tasks, L.red_tasks.data(), 4 * L.red_tasks.size())) ||
            (st = h->upload(&p2, L.p2.data(), sizeof(P2Desc) * L.p2.size()))) {
            return st;
        }
        ix.perm = perm; ix.p1 = p1; ix.p1_runs = p1_runs; ix.xdst = xdst; ix.lr = lr; ix.gdst = gdst; ix.p2 = p2;
        ix.red_big = red_big; ix.red_tasks = red_tasks;
        h->index_bytes = (int64_t)(4 * L.perm.size() + sizeof(P1Desc) * L.p1.size() + sizeof(P1Run) * L.p1_runs.size() +
                                   sizeof(XDst) * L.xdst.size() + sizeof(LrDesc) * L.lr.size() + 4 * L.gdst.size() +
                                   sizeof(P2Desc) * L.p2.size() + 4 * (L.red_big.size() + L.red_tasks.size()));

        // panels
        if ((st = alloc_panels(h, v, L, h->store, h->P, &h->panel_bytes))) return st;
        if (h->separate64) {
            if ((st = alloc_panels(h, v, L, h->store64, h->P64, &h->panel_bytes64))) return st;
        } else {
            h->P64 = h->P;
            h->panel_bytes64 = h->panel_bytes;
        }
        // solver vectors and scratch
        const size_t nb = 8 * (size_t)L.n;
        double **vecs[] = {&h->b, &h->x, &h->r, &h->rt, &h->p, &h->v, &h->s, &h->t, &h->y, &h->stage_in, &h->stage_out};
        for (double **pp : vecs)
            if ((st = h->alloc(pp, nb))) return st;
        if ((st = h->alloc(&h->partials, sizeof(double) * 2 * (size_t)vec_blocks(L.n))) ||
            (st = h->alloc(&h->dpart, sizeof(double) * 2 * (size_t)L.nleaves)) ||
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

extern "C" int hmat_destroy(hmat_handle h) {
    delete h;
    return HMAT_OK;
}

namespace {

int matvec_impl(hmat_handle h, const double *x, double *y, int32_t nrhs, void *stream, bool fp64) {
    if (!h || !x || !y || nrhs < 1) return HMAT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const DevPanels &P = fp64 ? h->P64 : h->P;
    const Store s = fp64 ? h->store64 : h->store;
    const int64_t n = h->ix.n;
    const bool dx = is_device_pointer(x), dy = is_device_pointer(y);
    for (int32_t k = 0; k < nrhs; ++k) {
        const double *xk = x + (size_t)k * n;
        double *yk = y + (size_t)k * n;
        const double *src = xk;
        if (!dx) {
            CK(cudaMemcpyAsync(h->stage_in, xk, 8 * n, cudaMemcpyHostToDevice, st));
            src = h->stage_in;
        }
        double *dst = dy ? yk : h->stage_out;
        enqueue_product(h, P, s, src, h->ix.perm, dst, h->ix.perm, nullptr, 0, st);
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
    const int64_t n = h->ix.n;
    const Store s = h->store;
    launch_update_p(s, n, h->r, h->p, h->v, h->P.xs, h->S, st);
    // v = A p, with alpha = rho / (r~ . v)
    launch_phase1(s, h->ix, h->P, h->S, 1, st);
    launch_reduce(s, h->ix, h->P, h->S, 1, st);
    launch_phase2(s, h->ix, h->P, h->v, nullptr, h->S, 1, st, h->rt, 1, h->S, h->dpart);
    launch_update_s(s, n, h->r, h->v, h->s, h->P.xs, h->x, h->p, h->S, h->partials, st);
    // t = A s, with omega = (t . s) / (t . t)
    launch_phase1(s, h->ix, h->P, h->S, 2, st);
    launch_reduce(s, h->ix, h->P, h->S, 2, st);
    launch_phase2(s, h->ix, h->P, h->t, nullptr, h->S, 2, st, h->s, 2, h->S, h->dpart);
    launch_update_xr(n, h->x, h->p, h->s, h->t, h->r, h->rt, h->S, h->partials, iter_limit, st);
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
    o->use_graph = 1;
}

extern "C" int hmat_bicgstab_ex(hmat_handle h, const double *b, double *x, const hmat_solve_opts *opts_in,
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
    const int64_t n = h->ix.n;
    const bool db = is_device_pointer(b), dx = is_device_pointer(x);
    // kernels per product (source operand, projection, reduction when some block
    // spans several leaf clusters, expansion) and per iteration (p update, two
    // products without operand preparation whose expansions also give alpha and
    // omega, s update, x/r update with the count of the next iteration)
    const int kProductLaunches = (h->ix.nbig + h->ix.ntasks) ? 4 : 3;
    const int kIterationLaunches = 3 + 2 * (kProductLaunches - 1);
    const double *bsrc = b;
    if (!db) {
        CK(cudaMemcpyAsync(h->stage_in, b, 8 * n, cudaMemcpyHostToDevice, st));
        bsrc = h->stage_in;
    }
    launch_gather(n, h->ix.perm, bsrc, h->b, st);
    int launches = 1;
    const double *xsrc = x;
    if (!dx) {
        CK(cudaMemcpyAsync(h->stage_out, x, 8 * n, cudaMemcpyHostToDevice, st));
        xsrc = h->stage_out;
    }
    launch_gather(n, h->ix.perm, xsrc, h->x, st);
    CK(cudaMemsetAsync(h->S, 0, sizeof(SolverScalars), st));
    // ||b||
    launch_residual(n, h->b, nullptr, h->r, h->rt, h->S, h->partials, -1, st);
    launches += 2;
    int rc = read_scalars(h, st);
    if (rc) return rc;
    const double bnorm2 = h->S_host->rnorm2;
    int status = HMAT_OK;
    if (!std::isfinite(bnorm2)) {
        status = HMAT_ERR_NONFINITE;
        inf.relres_true = NAN;
    } else if (bnorm2 == 0.0) {
        CK(cudaMemsetAsync(h->x, 0, 8 * n, st));
        inf.relres_true = 0.0;
    } else {
        // first run: r_0 = b - A~ x_0 with the iterated operator (Algorithm 1)
        enqueue_product(h, h->P, h->store, h->x, nullptr, h->y, nullptr, nullptr, 0, st);
        launch_residual(n, h->b, h->y, h->r, h->rt, h->S, h->partials, o.maxit, st);  // run 1 starts
        launches += kProductLaunches + 1;
        CK(cudaGetLastError());
        for (;;) {
            // a run: its stop threshold, then batches of iterations until its flag is set
            // (a run whose start already failed -- budget, non-finite -- goes straight on)
            if ((rc = read_scalars(h, st))) return rc;
            if (h->S_host->flag == 0) {
                double stop2 = std::max(o.tol * o.tol * bnorm2, o.inner_tol * o.inner_tol * h->S_host->rnorm2);
                CK(cudaMemcpyAsync(&h->S->stop2, &stop2, sizeof(double), cudaMemcpyHostToDevice, st));
                for (;;) {
                    launches += o.check_every * kIterationLaunches;
                    if (o.use_graph) {
                        if ((rc = ensure_graph(h, o.check_every, o.maxit))) return rc;
                        CK(cudaGraphLaunch(h->graph, st));
                    } else {
                        for (int i = 0; i < o.check_every; ++i) enqueue_iteration(h, o.maxit, st);
                        CK(cudaGetLastError());
                    }
                    if ((rc = read_scalars(h, st))) return rc;
                    if (h->S_host->flag != 0) break;
                }
            }
            const int flag = h->S_host->flag;
            inf.relres_inner = std::sqrt(h->S_host->rnorm2 / bnorm2);
            inf.iters = h->S_host->iters;
            // true residual with the FP64 H-matrix (Section 4.1.3); r~ = r for a restart
            enqueue_product(h, h->P64, h->store64, h->x, nullptr, h->y, nullptr, nullptr, 0, st);
            launch_residual(n, h->b, h->y, h->r, h->rt, h->S, h->partials, -1, st);
            launches += kProductLaunches + 1;
            inf.matvecs_fp64 += 1;
            if ((rc = read_scalars(h, st))) return rc;
            const double rel = std::sqrt(h->S_host->rnorm2 / bnorm2);
            inf.relres_true = rel;
            if (flag != 1) { status = flag; break; }
            if (!std::isfinite(rel)) { status = HMAT_ERR_NONFINITE; break; }
            if (rel <= o.tol) { status = HMAT_OK; break; }
            if (inf.restarts >= o.max_restarts) { status = HMAT_ERR_MAXIT; break; }
            inf.restarts += 1;
            launch_count_iter(h->S, o.maxit, st);  // the restarted run starts
            launches += 1;
        }
    }
    // products with the iterated operator: r_0, then two per iteration except a stop at ||s||
    double *xo = dx ? x : h->stage_out;
    launch_scatter(n, h->ix.perm, h->x, xo, st);
    launches += 1;
    inf.launches = launches;
    if (!dx) CK(cudaMemcpyAsync(x, h->stage_out, 8 * n, cudaMemcpyDeviceToHost, st));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    inf.iters = h->S_host->iters;
    inf.matvecs = bnorm2 > 0.0 && std::isfinite(bnorm2) ? 1 + h->S_host->nmv : 0;
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

extern "C" int hmat_info(hmat_handle h, hmat_handle_info *out) {
    if (!h || !out) return HMAT_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = h->ix.n;
    out->precision = h->precision;
    out->nleaves = h->ix.nleaves;
    out->panel_bytes = h->panel_bytes;
    out->panel_bytes_fp64 = h->panel_bytes64;
    out->index_bytes = h->index_bytes;
    out->stored_entries = h->stored_entries;
    out->phase1_entries = h->phase1_entries;
    out->phase2_entries = h->phase2_entries;
    out->partials = h->partials_n;
    out->rank_sum = h->rank_sum;
    return HMAT_OK;
}

extern "C" int hmat_time_matvec(hmat_handle h, int32_t iters, int32_t fp64, void *stream, double *ms_out) {
    if (!h || !ms_out || iters < 1) return HMAT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const DevPanels &P = fp64 ? h->P64 : h->P;
    const Store s = fp64 ? h->store64 : h->store;
    const int64_t n = h->ix.n;
    // a fixed source vector: x = 1 in cluster order
    std::vector<double> ones(n, 1.0);
    CK(cudaMemcpyAsync(h->stage_in, ones.data(), 8 * n, cudaMemcpyHostToDevice, st));
    cudaEvent_t ev[5];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    double tot[5] = {0, 0, 0, 0, 0};
    for (int it = 0; it < iters; ++it) {
        CK(cudaEventRecord(ev[0], st));
        launch_prep(s, h->ix, h->stage_in, nullptr, P.xs, st);
        CK(cudaEventRecord(ev[1], st));
        launch_phase1(s, h->ix, P, nullptr, 0, st);
        CK(cudaEventRecord(ev[2], st));
        launch_reduce(s, h->ix, P, nullptr, 0, st);
        CK(cudaEventRecord(ev[3], st));
        launch_phase2(s, h->ix, P, h->stage_out, nullptr, nullptr, 0, st);
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
    default: return "unknown status";
    }
}

std::string &hmat_internal::last_cuda_error() {
    static thread_local std::string s;
    return s;
}

extern "C" const char *hmat_last_cuda_error(void) { return hmat_internal::last_cuda_error().c_str(); }
