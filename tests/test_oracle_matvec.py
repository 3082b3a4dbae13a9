"""Pins of the oracle's H-matrix vector product (eq. 5-10, 21-25) and of its
precision variants (Table 1, eq. 11-20)."""
import numpy as np
import pytest

import synth

FP32_U = 2.0 ** -24


@pytest.mark.parametrize("level", [2, 3, 4])
def test_hmatvec_vs_dense_brute_force(hcache, oracle_mod, level):
    mesh = synth.icosphere(level)
    H = hcache(mesh)
    A = oracle_mod.dense_matrix(mesh.centroid, mesh.area)
    rng = np.random.default_rng(level)
    for x in (np.ones(mesh.n), rng.standard_normal(mesh.n)):
        y = A @ x
        yh = H.matvec(x)
        rel = np.linalg.norm(yh - y) / np.linalg.norm(y)
        assert rel <= 2 * H.eps, rel      # within the ACA tolerance
        assert rel > 1e-9                 # and the approximation is really used


def test_all_dense_partition_is_the_dense_product(oracle_mod):
    mesh = synth.icosphere(2)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area, eta=0.0)
    A = oracle_mod.dense_matrix(mesh.centroid, mesh.area)
    x = np.random.default_rng(0).standard_normal(mesh.n)
    y = A @ x
    assert np.linalg.norm(H.matvec(x) - y) <= 1e-15 * np.linalg.norm(y) * 4


def test_dense_matvec_helper_matches_numpy(oracle_mod):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((37, 37)); x = rng.standard_normal(37)
    assert np.allclose(oracle_mod.dense_matvec(A, x), A @ x, rtol=1e-14, atol=1e-13)


def test_linearity_assembly_and_rows(hcache):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    rng = np.random.default_rng(7)
    x, z = rng.standard_normal(mesh.n), rng.standard_normal(mesh.n)
    y = H.matvec(2.0 * x - 3.0 * z)
    assert np.linalg.norm(y - (2.0 * H.matvec(x) - 3.0 * H.matvec(z))) <= 1e-13 * np.linalg.norm(y)
    D = H.to_dense()
    assert np.linalg.norm(D @ x - H.matvec(x)) <= 1e-13 * np.linalg.norm(D @ x)
    rows = rng.integers(0, mesh.n, 25)
    assert np.allclose(H.matvec_rows(x, rows), H.matvec(x)[rows], rtol=1e-13, atol=1e-15)


def test_method2_scaling_eq16(hcache):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    blk = H.blocks
    lr = np.nonzero(blk[:, 4] == 1)[0]
    for b in lr[:: max(1, len(lr) // 60)]:
        Vm, Wm = H.block_data(b)
        Vp, Wp, d = H.method2_factors(b)
        assert np.array_equal(np.abs(Vp).max(axis=0), np.ones(Vm.shape[1]))   # eq. (16)
        assert np.array_equal(np.abs(Wp).max(axis=1), np.ones(Wm.shape[0]))
        assert np.allclose(Vp @ np.diag(d) @ Wp, Vm @ Wm, rtol=1e-14, atol=1e-18)
        assert np.all(d > 0)


def _table1():
    import os
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_precision.txt")
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows[f[0]] = f[1:]
    return rows


@pytest.mark.parametrize("name", ["M1_DOUBLE", "M1_SINGLE", "M1_MIXED", "M2_DOUBLE", "M2_SINGLE", "M2_MIXED"])
def test_variant_precisions_follow_table1(hcache, oracle_mod, name):
    """The source-vector columns of Table 1 decide whether a perturbation below FP32
    resolution is seen; the matrix columns decide the error size against FP64; the
    z_m column decides whether the low-rank sums add FP32 rounding of their own
    (Method 1) on top of Method 2's with the same source vector (bit-level pins of
    every cell: test_oracle_table1_cells.py)."""
    cols = _table1()[name]
    x_dense, x_lr, A_dense, W_lr, z_lr = cols[2], cols[5], cols[1], cols[4], cols[3]
    assert x_dense == x_lr
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    v = oracle_mod.VARIANTS[name]
    rng = np.random.default_rng(11)
    x = rng.uniform(1.0, 2.0, mesh.n)
    x32 = x.astype(np.float32).astype(np.float64)
    # perturb within the FP32 rounding interval of every entry
    xp = x32 + (x - x32) * 0.5 + x32 * 2.0 ** -30
    assert np.array_equal(xp.astype(np.float32).astype(np.float64), x32)
    y, yp = H.matvec(x, v), H.matvec(xp, v)
    if x_dense == "FP32":
        assert np.array_equal(y, yp)
    else:
        assert not np.array_equal(y, yp)
    y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
    rel = np.linalg.norm(y - y64) / np.linalg.norm(y64)
    if A_dense == "FP64" and W_lr == "FP64":
        assert rel <= 1e-14
    else:
        assert 1e-10 <= rel <= 1e-6       # FP32 rounding is present and within the FP32 bound
        assert rel <= 40 * FP32_U
    if z_lr == "FP32":
        # the same source and matrix precisions with an FP64 z_m (Method 2's row)
        twin = _table1()[name.replace("M1", "M2")]
        assert twin[3] == "FP64" and twin[2] == x_dense and twin[1] == A_dense
        y2 = H.matvec(x, oracle_mod.VARIANTS[name.replace("M1", "M2")])
        rel2 = np.linalg.norm(y2 - y64) / np.linalg.norm(y64)
        assert rel > 2 * rel2             # measured about 4x at level 3


def test_method3_limits(hcache, oracle_mod):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    x = np.random.default_rng(4).standard_normal(mesh.n)
    y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
    # c large: every rank FP64 -> Method 2-Double
    y3 = H.matvec(x, oracle_mod.M3, c=30)
    assert np.array_equal(y3, H.matvec(x, oracle_mod.M2_DOUBLE))
    assert np.linalg.norm(y3 - y64) <= 1e-14 * np.linalg.norm(y64)
    # c = -1: every low-rank factor FP32 but dense blocks FP64 (Section 3.3)
    e = {c: np.linalg.norm(H.matvec(x, oracle_mod.M3, c=c) - y64) / np.linalg.norm(y64) for c in (-1, 0, 1, 2, 4, 7)}
    e_mixed = np.linalg.norm(H.matvec(x, oracle_mod.M2_MIXED) - y64) / np.linalg.norm(y64)
    assert 1e-10 < e[-1] < e_mixed        # dense in FP64 removes part of the FP32 error
    assert e[7] <= e[1] <= e[-1] * 1.01   # more ranks in FP64 as c grows


def test_rank_truncation(hcache, oracle_mod):
    """Section 4.5's alternative to Method 3: ranks with d_i < d_max 10^-c are
    deleted.  Pins: nothing deleted for a large c (= Method 2-Double); every rank
    deleted for c = -1 (= the dense blocks alone, summed here from the raw block
    data); in between, what is lost is exactly the deleted ranks' d_l v'_l (w'_l x),
    and it shrinks as c grows."""
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    x = np.random.default_rng(45).standard_normal(mesh.n)
    T = oracle_mod.M3_TRUNC
    assert np.array_equal(H.matvec(x, T, c=30), H.matvec(x, oracle_mod.M2_DOUBLE))
    perm = H.perm
    xp = x[perm]
    blk = H.blocks
    y_dense = np.zeros(mesh.n)
    lost = {c: np.zeros(mesh.n) for c in (1, 3)}
    for b in range(len(blk)):
        i_s, i_e, j_s, j_e, kind, r, _ = blk[b]
        if kind == 0:
            y_dense[i_s:i_e] += H.block_data(b) @ xp[j_s:j_e]
        elif r > 0:
            Vp, Wp, d = H.method2_factors(b)
            for c in lost:
                for l in np.nonzero(d < d.max() * 10.0 ** (-c))[0]:
                    lost[c][i_s:i_e] += d[l] * Vp[:, l] * (Wp[l] @ xp[j_s:j_e])
    yd = np.empty(mesh.n)
    yd[perm] = y_dense
    assert np.linalg.norm(H.matvec(x, T, c=-1) - yd) <= 1e-14 * np.linalg.norm(yd)
    y2d = H.matvec(x, oracle_mod.M2_DOUBLE)
    errs = []
    for c in (1, 3):
        lc = np.empty(mesh.n)
        lc[perm] = lost[c]
        yt = H.matvec(x, T, c=c)
        assert np.linalg.norm((y2d - yt) - lc) <= 1e-13 * np.linalg.norm(y2d)
        errs.append(np.linalg.norm(y2d - yt))
    assert errs[1] < errs[0]


def test_dense_split(hcache, oracle_mod):
    """Section 4.5's multi-level dense blocks (Method 3's rule applied to the
    columns of the dense blocks against the largest near-field entry, the
    low-rank blocks as Method 2-Mixed).  Pins:
    a large c keeps every dense column FP64, which is Method 3 with c = -1 (dense
    FP64, low rank FP32) bit for bit; c = -1 demotes every column, which is
    Method 2-Mixed bit for bit; in between, what changes against c = 16 is exactly
    sum over the demoted columns of (fl32(a_ij) - a_ij) x_j, computed here from
    the raw block data; the error shrinks as c grows."""
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    x = np.random.default_rng(46).standard_normal(mesh.n)
    MD = oracle_mod.M3_DENSE
    y_hi = H.matvec(x, MD, c=16)
    assert np.array_equal(y_hi, H.matvec(x, oracle_mod.M3, c=-1))
    assert np.array_equal(H.matvec(x, MD, c=-1), H.matvec(x, oracle_mod.M2_MIXED))
    perm = H.perm
    xp = x[perm]
    blk = H.blocks
    dense = [b for b in range(len(blk)) if blk[b][4] == 0]
    dmax = max(np.abs(H.block_data(b)).max() for b in dense)   # the largest near-field entry
    delta = {c: np.zeros(mesh.n) for c in (0, 1, 2)}
    demoted = {c: 0 for c in delta}
    for b in dense:
        i_s, i_e, j_s, j_e, kind, r, _ = blk[b]
        A = H.block_data(b)
        w = np.abs(A).max(axis=0)
        for c in delta:
            lo = w < dmax * 10.0 ** (-c)
            demoted[c] += int(lo.sum())
            E = A.astype(np.float32).astype(np.float64) - A
            delta[c][i_s:i_e] += E[:, lo] @ xp[j_s:j_e][lo]
    y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
    # near-field column weights lie within 2e-2..1 of the self term here: c = 2 demotes nothing
    assert demoted[2] == 0 and np.array_equal(H.matvec(x, MD, c=2), y_hi)
    del delta[2]
    errs = []
    for c in delta:
        assert demoted[c] > 0
        dc = np.empty(mesh.n)
        dc[perm] = delta[c]
        yc = H.matvec(x, MD, c=c)
        # the change is reproduced to six digits (y's own rounding is ~1e-16 |y|)
        assert np.linalg.norm((yc - y_hi) - dc) <= 1e-6 * np.linalg.norm(dc)
        errs.append(np.linalg.norm(yc - y64))
    assert demoted[1] < demoted[0] and errs[1] <= errs[0]


def test_data_rounding_forms(hcache, oracle_mod):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    x = np.random.default_rng(9).standard_normal(mesh.n)
    y64 = H.matvec(x)
    r32 = np.linalg.norm(H.matvec(x, oracle_mod.DATA_FP32) - y64) / np.linalg.norm(y64)
    rbf = np.linalg.norm(H.matvec(x, oracle_mod.DATA_BF16) - y64) / np.linalg.norm(y64)
    assert 1e-10 < r32 < 1e-6
    assert 1e-5 < rbf < 1e-2
    assert rbf > 1000 * r32


def test_bf16_pow2_rounding_matches_torch_bfloat16(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    for scale in (1e-6, 1.0, 3e4):
        a = (rng.standard_normal(4000) * scale).astype(np.float32).astype(np.float64)  # FP32-exact
        got = oracle_mod.round_bf16_pow2(a)
        mx = np.abs(a).max()
        s = 2.0 ** (np.floor(np.log2(mx)))
        ref = (torch.from_numpy(a / s).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()) * s
        assert np.array_equal(got, ref)


def test_determinism(hcache, oracle_mod):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    x = np.random.default_rng(1).standard_normal(mesh.n)
    for v in range(9):
        assert np.array_equal(H.matvec(x, v, 2), H.matvec(x, v, 2))


def test_parallel_product_is_the_serial_one(hcache, oracle_mod):
    """The oracle's product runs its blocks in parallel and adds their y^_m into y
    in block order (eq. 25): every variant gives the same bits on one thread and
    on all of them, and so does a whole solve."""
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    x = np.random.default_rng(47).standard_normal(mesh.n)
    nt = oracle_mod.get_threads()
    try:
        oracle_mod.set_threads(1)
        ys = [H.matvec(x, v, 2) for v in range(11)]
        xs, info_s = H.bicgstab(synth.rhs_one_plus_half_z(mesh), tol=1e-8)
        oracle_mod.set_threads(max(4, nt))
        for v in range(11):
            assert np.array_equal(H.matvec(x, v, 2), ys[v]), v
        xp, info_p = H.bicgstab(synth.rhs_one_plus_half_z(mesh), tol=1e-8)
        assert np.array_equal(xp, xs) and info_p["iters"] == info_s["iters"]
    finally:
        oracle_mod.set_threads(nt)
