"""ctypes wrapper of the C oracle (hmat_oracle.c).  Test infrastructure only."""
import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmat_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# precision variants (Table 1 rows, plus data-rounding references)
M1_DOUBLE, M1_SINGLE, M1_MIXED, M2_DOUBLE, M2_SINGLE, M2_MIXED, M3, DATA_FP32, DATA_BF16, M3_TRUNC, M3_DENSE = range(11)
VARIANTS = {"M1_DOUBLE": M1_DOUBLE, "M1_SINGLE": M1_SINGLE, "M1_MIXED": M1_MIXED,
            "M2_DOUBLE": M2_DOUBLE, "M2_SINGLE": M2_SINGLE, "M2_MIXED": M2_MIXED, "M3": M3,
            "DATA_FP32": DATA_FP32, "DATA_BF16": DATA_BF16, "M3_TRUNC": M3_TRUNC, "M3_DENSE": M3_DENSE}
STATUS = {0: "ok", 1: "breakdown_rho", 2: "breakdown_omega", 3: "maxit", 4: "nonfinite"}


def build_oracle(force: bool = False) -> str:
    """Compile hmat_oracle.c into liboracle.so next to it (plain gcc, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(_LIB)
        P, D, I64, I = C.c_void_p, C.c_double, C.c_int64, C.c_int
        sig = {
            "or_kernel_entry": (D, [P, P, I64, I64]),
            "or_dense_matrix": (None, [I64, P, P, P]),
            "or_dense_matvec": (None, [I64, P, P, P]),
            "or_dense_solve": (I, [I64, P, P, P]),
            "or_admissible_boxes": (I, [P, P, P, P, D]),
            "or_aca_array": (I64, [I64, I64, P, D, I64, P, P]),
            "or_build": (P, [I64, P, P, I64, D, D]),
            "or_from_blocks": (P, [I64, I64, P, P]),
            "or_free": (None, [P]),
            "or_n": (I64, [P]), "or_nblocks": (I64, [P]), "or_nclusters": (I64, [P]),
            "or_get_perm": (None, [P, P]),
            "or_get_blocks": (None, [P, P]),
            "or_get_clusters": (None, [P, P, P]),
            "or_block_size": (I64, [P, I64]),
            "or_get_block_data": (None, [P, I64, P]),
            "or_method2_factors": (None, [P, I64, P, P, P]),
            "or_matvec": (None, [P, I, I, P, P]),
            "or_matvec_rows": (None, [P, P, I64, P, P]),
            "or_hmat_to_dense": (None, [P, P]),
            "or_bicgstab": (I, [P, I, I, P, P, D, D, I64, I64, P, I64, P]),
            "or_bicgstab_dense": (I, [I64, P, P, P, D, I64, P]),
            "or_gmres": (I, [P, I, I, I64, P, P, D, D, I64, I64, P]),
            "or_gmres_dense": (I, [I64, I64, P, P, P, D, I64, P]),
            "or_round_bf16_pow2": (None, [P, I64, P]),
            "or_set_threads": (None, [I]),
            "or_get_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def kernel_entry(centroid, area, i, j) -> float:
    c, a = _f64(centroid), _f64(area)
    return lib().or_kernel_entry(_p(c), _p(a), int(i), int(j))


def dense_matrix(centroid, area) -> np.ndarray:
    c, a = _f64(centroid), _f64(area)
    n = a.shape[0]
    A = np.empty((n, n))
    lib().or_dense_matrix(n, _p(c), _p(a), _p(A))
    return A


def dense_matvec(A, x) -> np.ndarray:
    A, x = _f64(A), _f64(x)
    y = np.empty(A.shape[0])
    lib().or_dense_matvec(A.shape[0], _p(A), _p(x), _p(y))
    return y


def dense_solve(A, b) -> np.ndarray:
    A, b = _f64(A), _f64(b)
    x = np.empty(A.shape[0])
    rc = lib().or_dense_solve(A.shape[0], _p(A), _p(b), _p(x))
    if rc != 0:
        raise ArithmeticError(f"or_dense_solve failed ({rc})")
    return x


def admissible(box_a, box_b, eta) -> bool:
    alo, ahi = _f64(box_a[0]), _f64(box_a[1])
    blo, bhi = _f64(box_b[0]), _f64(box_b[1])
    return bool(lib().or_admissible_boxes(_p(alo), _p(ahi), _p(blo), _p(bhi), float(eta)))


def aca(A, eps, rmax=None):
    """ACA with partial pivoting of an explicit block: returns (U m x r, V n x r)."""
    A = _f64(A)
    m, n = A.shape
    rmax = min(m, n) if rmax is None else int(rmax)
    U = np.zeros((max(rmax, 1), m))
    V = np.zeros((max(rmax, 1), n))
    r = lib().or_aca_array(m, n, _p(A), float(eps), rmax, _p(U), _p(V))
    return U[:r].T.copy(), V[:r].T.copy()


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (the block fill of the build and the
    product); the results are the same bits at any count."""
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def round_bf16_pow2(a):
    """The BF16 storage form of one array: s * bf16(a / s), s = 2^floor(log2 max|a|)."""
    a = _f64(a)
    out = np.empty_like(a)
    lib().or_round_bf16_pow2(_p(a), a.size, _p(out))
    return out


def dense_bicgstab(A, b, tol=1e-10, maxit=1000):
    A, b = _f64(A), _f64(b)
    x = np.zeros_like(b)
    info = np.zeros(6)
    st = lib().or_bicgstab_dense(A.shape[0], _p(A), _p(b), _p(x), float(tol), int(maxit), _p(info))
    return x, {"iters": int(info[0]), "relres": info[1], "status": STATUS[st]}


def dense_gmres(A, b, m=30, tol=1e-10, maxit=1000):
    """Restarted GMRES(m) (CGS2 Arnoldi, Givens rotations) on a dense matrix."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = _f64(b)
    x = np.zeros(A.shape[0])
    info = np.zeros(6)
    st = lib().or_gmres_dense(A.shape[0], int(m), _p(A), _p(b), _p(x), float(tol), int(maxit), _p(info))
    return x, {"iters": int(info[0]), "relres": float(info[1]), "status": STATUS[st]}


class HMatrix:
    """The oracle's own FP64 H-matrix of the collocation kernel (cluster tree,
    block partition, ACA factors), built from collocation points and areas."""

    def __init__(self, centroid, area, leaf=32, eta=2.0, eps=1e-4):
        self._c = _f64(centroid)
        self._a = _f64(area)
        self.n = int(self._a.shape[0])
        self.leaf, self.eta, self.eps = int(leaf), float(eta), float(eps)
        self._h = lib().or_build(self.n, _p(self._c), _p(self._a), self.leaf, self.eta, self.eps)
        if not self._h:
            raise MemoryError("or_build failed")

    @classmethod
    def from_blocks(cls, n, blocks):
        """A hand-written H-matrix (identity permutation): `blocks` is a list of
        (i_s, i_e, j_s, j_e, A) for a dense block A|^m, or (i_s, i_e, j_s, j_e,
        (V_m, W_m)) for a low-rank block V_m W_m (eq. 3)."""
        desc, data = [], []
        for i_s, i_e, j_s, j_e, d in blocks:
            if isinstance(d, tuple):
                V, W = _f64(d[0]), _f64(d[1])
                desc.append((i_s, i_e, j_s, j_e, 1, V.shape[1]))
                data += [V.ravel(), W.ravel()]
            else:
                desc.append((i_s, i_e, j_s, j_e, 0, 0))
                data.append(_f64(d).ravel())
        desc = np.ascontiguousarray(np.array(desc, dtype=np.int64).reshape(-1, 6))
        flat = _f64(np.concatenate(data) if data else np.zeros(1))
        self = cls.__new__(cls)
        self.n = int(n)
        self.leaf, self.eta, self.eps = 0, 0.0, 0.0
        self._h = lib().or_from_blocks(self.n, desc.shape[0], _p(desc), _p(flat))
        if not self._h:
            raise ValueError("malformed block list")
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_free(h)
            self._h = None

    # --- structure ---
    @property
    def perm(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.int64)
        lib().or_get_perm(self._h, _p(p))
        return p

    @property
    def blocks(self) -> np.ndarray:
        """(nblocks, 7) int64: i_s, i_e, j_s, j_e, kind (0 dense, 1 LR), rank, forced_dense."""
        nb = lib().or_nblocks(self._h)
        out = np.empty((nb, 7), dtype=np.int64)
        lib().or_get_blocks(self._h, _p(out))
        return out

    def clusters(self):
        nc = lib().or_nclusters(self._h)
        idx = np.empty((nc, 4), dtype=np.int64)
        box = np.empty((nc, 6))
        lib().or_get_clusters(self._h, _p(idx), _p(box))
        return idx, box

    def block_data(self, b):
        """Dense A|^m (m x n), or (V_m m x r, W_m r x n) for a low-rank block."""
        i_s, i_e, j_s, j_e, kind, r, _ = self.blocks[b]
        m, n = i_e - i_s, j_e - j_s
        cnt = lib().or_block_size(self._h, int(b))
        d = np.empty(max(cnt, 1))
        lib().or_get_block_data(self._h, int(b), _p(d))
        if kind == 0:
            return d[:m * n].reshape(m, n)
        return d[:m * r].reshape(m, r), d[m * r:m * r + r * n].reshape(r, n)

    def all_block_data(self):
        """Every block's data, in block order (list)."""
        blk = self.blocks
        out = []
        for b in range(blk.shape[0]):
            out.append(self.block_data(b))
        return out

    def method2_factors(self, b):
        i_s, i_e, j_s, j_e, kind, r, _ = self.blocks[b]
        m, n = i_e - i_s, j_e - j_s
        Vp = np.empty(max(m * r, 1)); Wp = np.empty(max(r * n, 1)); d = np.empty(max(r, 1))
        lib().or_method2_factors(self._h, int(b), _p(Vp), _p(Wp), _p(d))
        return Vp[:m * r].reshape(m, r), Wp[:r * n].reshape(r, n), d[:r]

    # --- products and solves (original panel order) ---
    def matvec(self, x, variant=M1_DOUBLE, c=0):
        x = _f64(x)
        y = np.empty(self.n)
        lib().or_matvec(self._h, int(variant), int(c), _p(x), _p(y))
        return y

    def matvec_rows(self, x, rows):
        x = _f64(x)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(rows.shape[0])
        lib().or_matvec_rows(self._h, _p(x), rows.shape[0], _p(rows), _p(out))
        return out

    def to_dense(self):
        A = np.empty((self.n, self.n))
        lib().or_hmat_to_dense(self._h, _p(A))
        return A

    def bicgstab(self, b, variant=M1_DOUBLE, c=0, tol=1e-8, inner_tol=0.0, maxit=1000,
                 maxrestart=30, x0=None, history=False):
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        info = np.zeros(6)
        hist = np.zeros(maxit) if history else None
        st = lib().or_bicgstab(self._h, int(variant), int(c), _p(b), _p(x), float(tol),
                               float(inner_tol), int(maxit), int(maxrestart),
                               _p(hist) if history else None, int(maxit) if history else 0, _p(info))
        out = {"iters": int(info[0]), "relres": float(info[1]), "status": STATUS[st],
               "restarts": int(info[3]), "matvecs": int(info[4]), "matvecs_fp64": int(info[5])}
        if history:
            out["history"] = hist[:out["iters"]]
        return x, out

    def gmres(self, b, m=30, variant=M1_DOUBLE, c=0, tol=1e-8, inner_tol=0.0, maxit=1000, maxrestart=30, x0=None):
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        info = np.zeros(6)
        st = lib().or_gmres(self._h, int(variant), int(c), int(m), _p(b), _p(x), float(tol), float(inner_tol),
                            int(maxit), int(maxrestart), _p(info))
        return x, {"iters": int(info[0]), "relres": float(info[1]), "status": STATUS[st],
                   "restarts": int(info[3]), "matvecs": int(info[4]), "matvecs_fp64": int(info[5])}

    # --- sizes ---
    def stats(self):
        blk = self.blocks
        m = blk[:, 1] - blk[:, 0]
        n = blk[:, 3] - blk[:, 2]
        dense = blk[:, 4] == 0
        lr = ~dense
        r = blk[:, 5]
        return {"n": self.n, "blocks": int(blk.shape[0]), "dense_blocks": int(dense.sum()),
                "lr_blocks": int(lr.sum()), "forced_dense": int(blk[:, 6].sum()),
                "dense_entries": int((m * n)[dense].sum()),
                "lr_entries": int((r * (m + n))[lr].sum()),
                "rank_sum": int(r[lr].sum()), "rank_max": int(r.max()) if r.size else 0}
