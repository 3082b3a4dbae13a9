"""Python binding of libhmat (include/hmat.h): the GB300 H-matrix vector product
and BiCG-STAB of arXiv:1911.00093.

Argument marshalling only: every step of the product and of the solver runs in
the library's CUDA kernels.  Vectors may be torch CUDA tensors (their device
pointers are passed), torch CPU tensors or numpy arrays (host pointers, staged
by the library).  Importing fails loudly when the extension has not been built.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libhmat.so")

HMAT_OK = 0
STATUS = {0: "ok", 1: "arg", 2: "bad_layout", 3: "nomem", 4: "cuda", 5: "breakdown_rho",
          6: "breakdown_omega", 7: "maxit", 8: "nonfinite", 9: "range", 10: "unsupported", 11: "timeout"}
HMAT_ERR_TIMEOUT = 11
HMAT_FP64, HMAT_FP64_DFMA, HMAT_FP32, HMAT_BF16 = 0, 1, 2, 3
HMAT_M1_SINGLE, HMAT_M1_MIXED, HMAT_M2_DOUBLE, HMAT_M2_SINGLE, HMAT_M2_MIXED, HMAT_M3 = 4, 5, 6, 7, 8, 9
HMAT_M3_TRUNC = 10
HMAT_M3_DENSE = 11
PRECISIONS = {"fp64": HMAT_FP64, "fp64_dfma": HMAT_FP64_DFMA, "fp32": HMAT_FP32, "bf16": HMAT_BF16,
              # the paper's variants (Section 3, Table 1); Method 1-Double is "fp64_dfma"
              "m1_single": HMAT_M1_SINGLE, "m1_mixed": HMAT_M1_MIXED, "m2_double": HMAT_M2_DOUBLE,
              "m2_single": HMAT_M2_SINGLE, "m2_mixed": HMAT_M2_MIXED, "m3": HMAT_M3, "m3_trunc": HMAT_M3_TRUNC,
              "m3_dense": HMAT_M3_DENSE}

# every symbol declared in include/hmat.h
EXPORTS = ("hmat_build", "hmat_blob_free", "hmat_blob_stats_get", "hmat_upload", "hmat_destroy",
           "hmat_matvec", "hmat_matvec_fp64", "hmat_solve_opts_default", "hmat_bicgstab",
           "hmat_bicgstab_ex", "hmat_info", "hmat_time_matvec", "hmat_strerror", "hmat_last_cuda_error",
           "hmat_matvec_noalloc", "hmat_upload_ex", "hmat_upload_batch", "hmat_problems", "hmat_bicgstab_multi",
           "hmat_gmres", "hmat_build_device", "hmat_form_stats_get", "hmat_check", "hmat_set_wait_limit",
           "hmat_autotune")


class TuneBucket(C.Structure):
    _fields_ = [("vec_max", C.c_int32), ("clusters", C.c_int32), ("threads", C.c_int32), ("pad", C.c_int32),
                ("us", C.c_double * 3)]


class TuneReport(C.Structure):
    _fields_ = [("nbuckets", C.c_int32), ("sorted", C.c_int32), ("default_us", C.c_double),
                ("tuned_us", C.c_double), ("bucket", TuneBucket * 5)]


class BuildDeviceInfo(C.Structure):
    _fields_ = [("aca_blocks", C.c_int64), ("host_blocks", C.c_int64), ("workspace_bytes", C.c_int64),
                ("plan_ms", C.c_double), ("alloc_ms", C.c_double), ("aca_ms", C.c_double),
                ("pack_ms", C.c_double), ("copy_ms", C.c_double)]


class FormStats(C.Structure):
    _fields_ = [("segments", C.c_int32), ("pad", C.c_int32)] + [
        (k, C.c_int64 * 2) for k in ("blocks", "dense_entries", "lr_ranks", "lr_entries", "column_subsets",
                                     "selected_operands")]


class BlobStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("n", "nclusters", "nblocks", "nleaves", "dense_blocks", "lr_blocks",
                                         "dense_entries", "lr_entries", "rank_sum", "rank_max")]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("inner_tol", C.c_double), ("maxit", C.c_int32),
                ("max_restarts", C.c_int32), ("check_every", C.c_int32), ("use_graph", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("restarts", C.c_int32), ("matvecs", C.c_int32),
                ("matvecs_fp64", C.c_int32), ("launches", C.c_int32), ("relres_true", C.c_double),
                ("relres_inner", C.c_double)]


class HandleInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("precision", C.c_int32), ("nleaves", C.c_int32), ("panel_bytes", C.c_int64),
                ("panel_bytes_fp64", C.c_int64), ("index_bytes", C.c_int64), ("stored_entries", C.c_int64),
                ("phase1_entries", C.c_int64), ("phase2_entries", C.c_int64), ("partials", C.c_int64),
                ("rank_sum", C.c_int64), ("stored_bytes", C.c_int64), ("phase1_bytes", C.c_int64),
                ("phase2_bytes", C.c_int64), ("segments", C.c_int32), ("method3_c", C.c_int32)]


class HmatError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if status == 4 and _lib is not None:
            msg += f" ({_lib.hmat_last_cuda_error().decode()})"
        super().__init__(msg)


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libhmat.so; raises ImportError when it is missing (run __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with paper_1911_00093_gb300._build.build()")
    L = C.CDLL(_LIB_PATH)
    P, I32, I64, D, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "hmat_build": (C.c_int, [I64, P, P, I32, D, D, C.POINTER(C.c_void_p), C.POINTER(SZ)]),
        "hmat_blob_free": (None, [P]),
        "hmat_blob_stats_get": (C.c_int, [P, SZ, C.POINTER(BlobStats)]),
        "hmat_upload": (C.c_int, [P, SZ, I32, C.POINTER(C.c_void_p)]),
        "hmat_destroy": (C.c_int, [P]),
        "hmat_matvec": (C.c_int, [P, P, P, I32, P]),
        "hmat_matvec_fp64": (C.c_int, [P, P, P, I32, P]),
        "hmat_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
        "hmat_bicgstab": (C.c_int, [P, P, P, D, I32, P, C.POINTER(SolveInfo)]),
        "hmat_bicgstab_ex": (C.c_int, [P, P, P, C.POINTER(SolveOpts), P, C.POINTER(SolveInfo)]),
        "hmat_info": (C.c_int, [P, C.POINTER(HandleInfo)]),
        "hmat_time_matvec": (C.c_int, [P, I32, I32, P, C.POINTER(C.c_double)]),
        "hmat_strerror": (C.c_char_p, [C.c_int]),
        "hmat_last_cuda_error": (C.c_char_p, []),
        "hmat_matvec_noalloc": (C.c_int, [P, P, P, P]),
        "hmat_upload_ex": (C.c_int, [P, SZ, I32, I32, C.POINTER(C.c_void_p)]),
        "hmat_upload_batch": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(SZ), I32, I32, I32, C.POINTER(C.c_void_p)]),
        "hmat_problems": (C.c_int, [P, C.POINTER(I32), P]),
        "hmat_bicgstab_multi": (C.c_int, [P, P, P, I32, C.POINTER(SolveOpts), P, P]),
        "hmat_gmres": (C.c_int, [P, P, P, I32, C.POINTER(SolveOpts), P, C.POINTER(SolveInfo)]),
        "hmat_build_device": (C.c_int, [I64, P, P, I32, D, D, C.POINTER(C.c_void_p), C.POINTER(SZ),
                                        C.POINTER(BuildDeviceInfo)]),
        "hmat_form_stats_get": (C.c_int, [P, SZ, I32, I32, C.POINTER(FormStats)]),
        "hmat_check": (C.c_int, [P, P]),
        "hmat_autotune": (C.c_int, [P, I32, P, C.POINTER(TuneReport)]),
        "hmat_set_wait_limit": (C.c_int, [P, I64, I32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st, where):
    if st != HMAT_OK:
        raise HmatError(st, where)


def _ptr(a):
    """(pointer, keepalive) of a torch tensor or numpy array of float64."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError("vectors must be contiguous float64")
            return C.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return C.c_void_p(arr.ctypes.data), arr


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------------
# functions with the names of the C ABI
# ---------------------------------------------------------------------------
def hmat_build(centroids, areas, leaf=32, eta=2.0, aca_eps=1e-4) -> bytes:
    """Serialized FP64 H-matrix (format of include/hmat.h) of the collocation kernel."""
    L = load()
    c = np.ascontiguousarray(centroids, dtype=np.float64)
    a = np.ascontiguousarray(areas, dtype=np.float64)
    n = a.shape[0]
    if c.shape != (n, 3):
        raise ValueError("centroids must be (n, 3)")
    buf, size = C.c_void_p(), C.c_size_t()
    _check(L.hmat_build(n, c.ctypes.data, a.ctypes.data, int(leaf), float(eta), float(aca_eps),
                        C.byref(buf), C.byref(size)), "hmat_build")
    try:
        out = np.empty(size.value, dtype=np.uint8)  # blobs may exceed 2 GiB: copy with memmove
        C.memmove(out.ctypes.data, buf, size.value)
    finally:
        L.hmat_blob_free(buf)
    return out


def hmat_build_device(centroids, areas, leaf=32, eta=2.0, aca_eps=1e-4, info=None):
    """hmat_build with the ACA and the dense entries on the current CUDA device (the
    same blob, byte for byte); `info`, if a dict, receives the build's counts and times."""
    L = load()
    c = np.ascontiguousarray(centroids, dtype=np.float64)
    a = np.ascontiguousarray(areas, dtype=np.float64)
    n = a.shape[0]
    if c.shape != (n, 3):
        raise ValueError("centroids must be (n, 3)")
    buf, size, inf = C.c_void_p(), C.c_size_t(), BuildDeviceInfo()
    _check(L.hmat_build_device(n, c.ctypes.data, a.ctypes.data, int(leaf), float(eta), float(aca_eps),
                               C.byref(buf), C.byref(size), C.byref(inf)), "hmat_build_device")
    try:
        out = np.empty(size.value, dtype=np.uint8)
        C.memmove(out.ctypes.data, buf, size.value)
    finally:
        L.hmat_blob_free(buf)
    if isinstance(info, dict):
        info.update({k: getattr(inf, k) for k, _ in BuildDeviceInfo._fields_})
    return out


def hmat_form_stats(blob, precision="fp64", c=0) -> dict:
    """What an upload in `precision` would store (host only): per-segment counts as lists."""
    L = load()
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    s = FormStats()
    _check(L.hmat_form_stats_get(b.ctypes.data, b.nbytes, prec, int(c), C.byref(s)), "hmat_form_stats_get")
    out = {"segments": s.segments}
    for k, _ in FormStats._fields_[2:]:
        out[k] = list(getattr(s, k))[:s.segments]
    return out


def hmat_blob_stats(blob) -> dict:
    L = load()
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    s = BlobStats()
    _check(L.hmat_blob_stats_get(b.ctypes.data, b.nbytes, C.byref(s)), "hmat_blob_stats_get")
    return {k: int(getattr(s, k)) for k, _ in BlobStats._fields_}


def hmat_upload(blob, precision="fp64", c=None):
    """Device handle (int) of a blob in one precision form (a key of PRECISIONS);
    `c` is Method 3's split parameter (eq. 19-20), passed through hmat_upload_ex."""
    L = load()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    h = C.c_void_p()
    if c is None:
        _check(L.hmat_upload(b.ctypes.data, b.nbytes, prec, C.byref(h)), "hmat_upload")
    else:
        _check(L.hmat_upload_ex(b.ctypes.data, b.nbytes, prec, int(c), C.byref(h)), "hmat_upload_ex")
    return h.value


def hmat_upload_batch(blobs, precision="fp64", c=None):
    """One handle over several problems (a block-diagonal operator; vectors are the
    concatenation of the problems' vectors)."""
    L = load()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    arrs = [np.ascontiguousarray(b, dtype=np.uint8) for b in blobs]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    sizes = (C.c_size_t * len(arrs))(*[a.nbytes for a in arrs])
    h = C.c_void_p()
    _check(L.hmat_upload_batch(ptrs, sizes, len(arrs), prec, 0 if c is None else int(c), C.byref(h)),
           "hmat_upload_batch")
    return h.value


def hmat_problems(h):
    """First rows of the handle's problems plus the total (length count + 1)."""
    L = load()
    cnt = C.c_int32()
    _check(L.hmat_problems(C.c_void_p(h), C.byref(cnt), None), "hmat_problems")
    off = np.empty(cnt.value + 1, dtype=np.int64)
    _check(L.hmat_problems(C.c_void_p(h), C.byref(cnt), C.c_void_p(off.ctypes.data)), "hmat_problems")
    return off


def hmat_bicgstab_multi(h, b, x, nrhs=1, tol=1e-8, maxit=1000, stream=None, **opts):
    """Every (problem, right-hand side) system with its own recurrence; b and x are
    N x nrhs column-major (torch: a contiguous (nrhs, N) tensor).  Returns the list
    of per-system info dicts, system (p, k) at k * count + p."""
    L = load()

    def colmajor(a):  # numpy (N, nrhs) -> flat column-major FP64
        return a if hasattr(a, "data_ptr") else np.asarray(a, dtype=np.float64).ravel(order="F").copy()

    bb, xx = colmajor(b), colmajor(x)
    pb, kb = _ptr(bb)
    px, kx = _ptr(xx)
    cnt = len(hmat_problems(h)) - 1
    infos = (SolveInfo * (cnt * nrhs))()
    o = hmat_solve_opts(tol=float(tol), maxit=int(maxit), **opts)
    st = L.hmat_bicgstab_multi(C.c_void_p(h), pb, px, int(nrhs), C.byref(o), _stream_ptr(stream), infos)
    if st in (1, 3, 4):
        raise HmatError(st, "hmat_bicgstab_multi")
    if not hasattr(x, "data_ptr"):
        x[...] = kx.reshape(np.shape(x), order="F")
    out = []
    for inf in infos:
        d = {k: getattr(inf, k) for k, _ in SolveInfo._fields_}
        d["status_name"] = STATUS.get(d["status"], d["status"])
        out.append(d)
    return out


def hmat_destroy(h):
    if h:
        load().hmat_destroy(C.c_void_p(h))


def hmat_matvec(h, x, y, nrhs=1, stream=None, fp64=False):
    L = load()
    px, kx = _ptr(x)
    py, ky = _ptr(y)
    f = L.hmat_matvec_fp64 if fp64 else L.hmat_matvec
    _check(f(C.c_void_p(h), px, py, int(nrhs), _stream_ptr(stream)), "hmat_matvec")
    return y


def hmat_matvec_noalloc(h, x, y, stream=None):
    """y = A~ x through the allocation-free entry point (device pointers only)."""
    px, kx = _ptr(x)
    py, ky = _ptr(y)
    _check(load().hmat_matvec_noalloc(C.c_void_p(h), px, py, _stream_ptr(stream)), "hmat_matvec_noalloc")
    return y


def hmat_check(h, stream=None) -> int:
    """Synchronise `stream`; the status of the handle's bounded device waits since the
    last report (HMAT_ERR_TIMEOUT when one ran out, else 0), cleared."""
    return int(load().hmat_check(C.c_void_p(h), _stream_ptr(stream)))


def hmat_set_wait_limit(h, cycles, withhold=False):
    """Bound of the tensor-core product's waits in SM cycles; withhold=True makes its
    projection issue no copies, so the waits run out (tests of the timeout path)."""
    _check(load().hmat_set_wait_limit(C.c_void_p(h), int(cycles), 1 if withhold else 0), "hmat_set_wait_limit")


def hmat_autotune(h, reps=20, stream=None) -> dict:
    """Choose the projection's CTA size per panel-width bucket by measurement and
    keep the plan in the handle; returns the report of the iterated operator."""
    r = TuneReport()
    _check(load().hmat_autotune(C.c_void_p(h), int(reps), _stream_ptr(stream), C.byref(r)), "hmat_autotune")
    return {"sorted": bool(r.sorted), "default_us": r.default_us, "tuned_us": r.tuned_us,
            "buckets": [{"vec_max": b.vec_max, "clusters": b.clusters, "threads": b.threads,
                         "us_64_128_256": [b.us[0], b.us[1], b.us[2]]} for b in r.bucket[:r.nbuckets]]}


def hmat_solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    load().hmat_solve_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def hmat_bicgstab(h, b, x, tol=1e-8, maxit=1000, stream=None, **opts) -> dict:
    """Solve A~ x = b in place of x; returns the solve info as a dict (status is not raised)."""
    L = load()
    pb, kb = _ptr(b)
    px, kx = _ptr(x)
    info = SolveInfo()
    o = hmat_solve_opts(tol=float(tol), maxit=int(maxit), **opts)
    st = L.hmat_bicgstab_ex(C.c_void_p(h), pb, px, C.byref(o), _stream_ptr(stream), C.byref(info))
    if st in (1, 3, 4):
        raise HmatError(st, "hmat_bicgstab")
    if kx is not x and not hasattr(x, "data_ptr"):
        np.copyto(x, kx)
    out = {k: getattr(info, k) for k, _ in SolveInfo._fields_}
    out["status_name"] = STATUS.get(out["status"], out["status"])
    return out


def hmat_gmres(h, b, x, m=30, tol=1e-8, maxit=1000, stream=None, **opts) -> dict:
    """Restarted GMRES(m) with the handle's products; x in place; returns the info dict."""
    L = load()
    pb, kb = _ptr(b)
    px, kx = _ptr(x)
    info = SolveInfo()
    o = hmat_solve_opts(tol=float(tol), maxit=int(maxit), **opts)
    st = L.hmat_gmres(C.c_void_p(h), pb, px, int(m), C.byref(o), _stream_ptr(stream), C.byref(info))
    if st in (1, 3, 4):
        raise HmatError(st, "hmat_gmres")
    if kx is not x and not hasattr(x, "data_ptr"):
        np.copyto(x, kx)
    out = {k: getattr(info, k) for k, _ in SolveInfo._fields_}
    out["status_name"] = STATUS.get(out["status"], out["status"])
    return out


def hmat_info(h) -> dict:
    s = HandleInfo()
    _check(load().hmat_info(C.c_void_p(h), C.byref(s)), "hmat_info")
    return {k: int(getattr(s, k)) for k, _ in HandleInfo._fields_}


def hmat_time_matvec(h, iters=10, fp64=False, stream=None):
    """Mean ms per launch of [prep, projection, reduce, expansion, whole product]."""
    out = (C.c_double * 5)()
    _check(load().hmat_time_matvec(C.c_void_p(h), int(iters), int(bool(fp64)), _stream_ptr(stream), out),
           "hmat_time_matvec")
    return list(out)


def hmat_strerror(status) -> str:
    return load().hmat_strerror(int(status)).decode()


class HMatrix:
    """Owning wrapper of one uploaded handle."""

    def __init__(self, blob, precision="fp64", c=None):
        self.blob = np.ascontiguousarray(blob, dtype=np.uint8)
        self.precision = precision
        self.h = hmat_upload(self.blob, precision, c)
        self.info = hmat_info(self.h)
        self.n = self.info["n"]

    def close(self):
        if getattr(self, "h", None):
            hmat_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def matvec(self, x, y=None, stream=None, fp64=False):
        import torch
        if y is None:
            y = torch.empty_like(x) if isinstance(x, torch.Tensor) else np.empty_like(np.asarray(x, dtype=np.float64))
        nrhs = 1 if (x.ndim if hasattr(x, "ndim") else 1) == 1 else x.shape[1]
        return hmat_matvec(self.h, x, y, nrhs, stream, fp64)

    def solve(self, b, x=None, tol=1e-8, maxit=1000, stream=None, **opts):
        import torch
        if x is None:
            x = torch.zeros_like(b) if isinstance(b, torch.Tensor) else np.zeros(self.n)
        info = hmat_bicgstab(self.h, b, x, tol, maxit, stream, **opts)
        return x, info
