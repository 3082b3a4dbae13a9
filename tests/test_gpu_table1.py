"""GPU parity of the paper's own precision variants (Section 3, Table 1) against
the oracle's literal emulation of the same variant, element by element.

Methods 2 and 3 keep z_m and y^_m in FP64 (Table 1), and both sides round the
same FP64 values to FP32 (A|^m, V'_m = V_m D_V^-1, W'_m = D_W^-1 W_m of eq. 11-16,
the FP32 copy of x of Section 3.5, FP32 x FP32 products), so they differ only by
the order of FP64 additions: 1e-12 relative.  Method 1 keeps z_m in FP32, whose
additions depend on their order (the GPU sums per leaf cluster, then the
partial sums; the oracle runs along the row): for a general x the two agree to
FP32 accumulation accuracy only.  For a source vector with a single nonzero
entry every z_m has one term, so no FP32 addition is left to order and Method 1
must agree to 1e-12 as well; a rounding put anywhere else than Table 1 says (x
not rounded, a product not rounded, z_m kept in FP64) would show at 1e-8.
"""
import numpy as np
import pytest

import synth
from blob_util import oracle_blob
from gpu_util import lib, maxrel, need_gpu, rel

pytestmark = pytest.mark.gpu

MESHES = [synth.icosphere(3), synth.unit_cube(8), synth.two_spheres(3)]

# (form, oracle variant, Method 3's c)
VARIANTS = [("m1_single", "M1_SINGLE", None), ("m1_mixed", "M1_MIXED", None),
            ("m2_double", "M2_DOUBLE", None), ("m2_single", "M2_SINGLE", None),
            ("m2_mixed", "M2_MIXED", None),
            ("m3", "M3", -1), ("m3", "M3", 1), ("m3", "M3", 3), ("m3", "M3", 7),
            ("m3_trunc", "M3_TRUNC", 1), ("m3_trunc", "M3_TRUNC", 3),
            ("m3_dense", "M3_DENSE", 0), ("m3_dense", "M3_DENSE", 1)]
FP64_SUMS = ("M2_DOUBLE", "M2_SINGLE", "M2_MIXED", "M3", "M3_TRUNC", "M3_DENSE")


def _ids(v):
    return v[0] + ("" if v[2] is None else f"_c{v[2]}")


def _gpu_matvec(P, torch, h, x):
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    P.hmat_matvec(h, xd, yd, 1)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _check(y, ysame, y64, variant, exact=False):
    if variant in FP64_SUMS or exact:
        assert rel(y, ysame) <= 1e-12 and maxrel(y, ysame) <= 1e-11, (rel(y, ysame), maxrel(y, ysame))
    else:
        assert rel(y, ysame) <= 3e-7, rel(y, ysame)
        assert rel(y, y64) <= 1e-6, rel(y, y64)


@pytest.mark.parametrize("mesh", MESHES, ids=lambda m: m.name)
@pytest.mark.parametrize("form,variant,c", VARIANTS, ids=[_ids(v) for v in VARIANTS])
def test_table1_matvec_parity(hcache, oracle_mod, mesh, form, variant, c):
    torch = need_gpu()
    P = lib()
    H = hcache(mesh)
    h = P.hmat_upload(oracle_blob(H), form, c)
    cc = 0 if c is None else c
    try:
        rng = np.random.default_rng(mesh.n + 11)
        for x in (rng.standard_normal(mesh.n), synth.rhs_one_plus_half_z(mesh)):
            y = _gpu_matvec(P, torch, h, x)
            ysame = H.matvec(x, oracle_mod.VARIANTS[variant], cc)
            y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
            _check(y, ysame, y64, variant)
            if variant != "M2_DOUBLE" and not (variant == "M3" and cc >= 2):
                assert rel(y, y64) > 1e-12  # the FP32 data is really used (c >= 2 leaves it tiny ranks)
        # single-nonzero sources: no FP32 addition of z_m to order
        for j in rng.choice(mesh.n, 3, replace=False):
            x = np.zeros(mesh.n)
            x[j] = 1.2345678901234567
            y = _gpu_matvec(P, torch, h, x)
            _check(y, H.matvec(x, oracle_mod.VARIANTS[variant], cc), None, variant, exact=True)
    finally:
        P.hmat_destroy(h)


def test_method3_limits(hcache, oracle_mod):
    """c = -1 puts every rank in FP32 (Section 3.3); a c above every ratio
    d_max / d_i keeps every rank in FP64 and gives Method 2-Double."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    blob = oracle_blob(H)
    x = np.random.default_rng(5).standard_normal(mesh.n)
    h16 = P.hmat_upload(blob, "m3", 16)
    hm = P.hmat_upload(blob, "m3", -1)
    try:
        y16 = _gpu_matvec(P, torch, h16, x)
        assert rel(y16, H.matvec(x, oracle_mod.M2_DOUBLE)) <= 1e-12
        ym = _gpu_matvec(P, torch, hm, x)
        assert rel(ym, H.matvec(x, oracle_mod.M3, -1)) <= 1e-12
        # FP64 dense blocks and FP32 low-rank blocks: between FP64 and all-FP32 accuracy
        y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
        assert 1e-12 < rel(ym, y64) < rel(H.matvec(x, oracle_mod.M2_MIXED), y64)
    finally:
        P.hmat_destroy(h16)
        P.hmat_destroy(hm)
    with pytest.raises(P.HmatError) as e:
        P.hmat_upload(blob, "m3", 40)
    assert e.value.status == 1


def test_dense_split_limits(hcache, oracle_mod):
    """Section 4.5's dense split at its ends: c = -1 demotes every dense column
    (Method 2-Mixed), c = 16 none (Method 3 with c = -1); c = 1 stores the near
    field as two column subsets, between the two in accuracy and in bytes."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    blob = oracle_blob(H)
    x = np.random.default_rng(8).standard_normal(mesh.n)
    y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
    hs = {c: P.hmat_upload(blob, "m3_dense", c) for c in (-1, 1, 16)}
    try:
        y = {c: _gpu_matvec(P, torch, h, x) for c, h in hs.items()}
        assert rel(y[-1], H.matvec(x, oracle_mod.M2_MIXED)) <= 1e-12
        assert rel(y[16], H.matvec(x, oracle_mod.M3, -1)) <= 1e-12
        assert rel(y[1], H.matvec(x, oracle_mod.M3_DENSE, 1)) <= 1e-12
        assert rel(y[16], y64) < rel(y[1], y64) < rel(y[-1], y64)
        st = {c: P.hmat_info(h)["stored_bytes"] for c, h in hs.items()}
        assert st[-1] < st[1] < st[16]
    finally:
        for h in hs.values():
            P.hmat_destroy(h)
    with pytest.raises(P.HmatError) as e:
        P.hmat_upload(blob, "m3_dense", 17)
    assert e.value.status == 1


def test_table1_host_pointers_and_determinism(hcache, oracle_mod):
    """A two-segment variant through host pointers gives the device result's bits,
    and repeated products are bitwise identical (no atomics)."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    h = P.hmat_upload(oracle_blob(H), "m3", 2)
    try:
        x = np.random.default_rng(9).standard_normal(mesh.n)
        yd = _gpu_matvec(P, torch, h, x)
        yh = np.empty(mesh.n)
        P.hmat_matvec(h, x, yh, 1)
        assert np.array_equal(yd, yh)
        assert np.array_equal(yd, _gpu_matvec(P, torch, h, x))
        # the FP64 H-matrix of the true residual is Method 1-Double
        yf = np.empty(mesh.n)
        P.hmat_matvec(h, x, yf, 1, None, True)
        assert rel(yf, H.matvec(x, oracle_mod.M1_DOUBLE)) <= 1e-14
    finally:
        P.hmat_destroy(h)


@pytest.mark.parametrize("form,variant,c", [("m1_single", "M1_SINGLE", None), ("m1_mixed", "M1_MIXED", None),
                                            ("m2_double", "M2_DOUBLE", None), ("m2_single", "M2_SINGLE", None),
                                            ("m2_mixed", "M2_MIXED", None), ("m3", "M3", -1), ("m3", "M3", 2),
                                            ("m3_trunc", "M3_TRUNC", 3), ("m3_dense", "M3_DENSE", 1)],
                         ids=lambda v: str(v))
def test_table1_solve(hcache, oracle_mod, form, variant, c):
    """BiCG-STAB with the variant as the iterated operator and the FP64
    H-matrix's true residual (Section 4.1.3) reaches 1e-8, restarting from the
    true residual where the variant's accuracy stops the inner iteration; the
    oracle's solve with the same variant takes a similar number of iterations."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    inner = 0.0 if variant == "M2_DOUBLE" else 1e-5
    h = P.hmat_upload(oracle_blob(H), form, c)
    try:
        xd = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        info = P.hmat_bicgstab(h, torch.from_numpy(b).cuda(), xd, tol=1e-8, maxit=400, inner_tol=inner,
                               check_every=2)
        assert info["status"] == 0 and info["relres_true"] <= 1e-8, info
        x = xd.cpu().numpy()
        r = b - H.matvec(x, oracle_mod.M1_DOUBLE)
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
        _, ref = H.bicgstab(b, oracle_mod.VARIANTS[variant], 0 if c is None else c, tol=1e-8, inner_tol=inner,
                            maxit=400)
        assert ref["status"] == "ok"
        assert abs(info["iters"] - ref["iters"]) <= max(3, ref["iters"] // 4), (info["iters"], ref["iters"])
    finally:
        P.hmat_destroy(h)


def test_table1_full_size(oracle_mod):
    """Icosphere level 6 (N = 81,920), built by the library's host builder: every
    element of the GPU product of three variants against the oracle's emulation
    on its own H-matrix (the builder reproduces it exactly)."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(6)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
    x = synth.rhs_one_plus_half_z(mesh) + 0.1 * np.random.default_rng(16).standard_normal(mesh.n)
    y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
    for form, variant, c in (("m2_mixed", "M2_MIXED", None), ("m3", "M3", -1), ("m1_single", "M1_SINGLE", None),
                             ("m3_dense", "M3_DENSE", 1)):
        h = P.hmat_upload(blob, form, c)
        try:
            y = _gpu_matvec(P, torch, h, x)
            _check(y, H.matvec(x, oracle_mod.VARIANTS[variant], 0 if c is None else c), y64, variant)
        finally:
            P.hmat_destroy(h)
