"""GPU parity of hmat_matvec against the oracle, element by element, in every
precision form (tolerances: FP64 1e-13, FP32 1e-6, BF16 1e-2 relative to the
FP64 product; tighter against the oracle's product on identically rounded data)."""
import numpy as np
import pytest

import synth
from blob_util import dense_blob, oracle_blob
from gpu_util import lib, maxrel, need_gpu, rel

pytestmark = pytest.mark.gpu

MESHES = [synth.icosphere(3), synth.icosphere(4), synth.unit_cube(8), synth.two_spheres(3)]

# (form, oracle variant of the same stored data, tol vs that variant, tol vs FP64)
FORMS = [("fp64", "M1_DOUBLE", 1e-13, 1e-13),
         ("fp64_dfma", "M1_DOUBLE", 1e-14, 1e-14),
         ("fp32", "DATA_FP32", 2e-7, 1e-6),
         ("bf16", "DATA_BF16", 2e-6, 1e-2)]


def _gpu_matvec(P, torch, h, x, fp64=False):
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    P.hmat_matvec(h, xd, yd, 1, None, fp64)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("mesh", MESHES, ids=lambda m: m.name)
@pytest.mark.parametrize("form,variant,tol_same,tol64", FORMS, ids=[f[0] for f in FORMS])
def test_matvec_parity(hcache, oracle_mod, mesh, form, variant, tol_same, tol64):
    torch = need_gpu()
    P = lib()
    H = hcache(mesh)
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        rng = np.random.default_rng(mesh.n)
        for x in (rng.standard_normal(mesh.n), np.ones(mesh.n), synth.rhs_one_plus_half_z(mesh)):
            y = _gpu_matvec(P, torch, h, x)
            y64 = H.matvec(x, oracle_mod.M1_DOUBLE)
            ysame = H.matvec(x, oracle_mod.VARIANTS[variant])
            assert rel(y, ysame) <= tol_same and maxrel(y, ysame) <= 4 * tol_same, (rel(y, ysame), maxrel(y, ysame))
            assert rel(y, y64) <= tol64, rel(y, y64)
            if form not in ("fp64", "fp64_dfma"):
                assert rel(y, y64) > 1e-12  # the low-precision data is really used
    finally:
        P.hmat_destroy(h)


def test_fp64_copy_host_pointers_determinism_and_nrhs(hcache, oracle_mod):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    blob = oracle_blob(H)
    h32 = P.hmat_upload(blob, "fp32")
    h64 = P.hmat_upload(blob, "fp64")
    try:
        x = np.random.default_rng(0).standard_normal(mesh.n)
        # the FP64 copy of a low-precision handle is the FP64 form
        assert np.array_equal(_gpu_matvec(P, torch, h32, x, fp64=True), _gpu_matvec(P, torch, h64, x))
        # host pointers are staged and give the same bits; repeated calls are deterministic
        yd = _gpu_matvec(P, torch, h64, x)
        yh = np.empty(mesh.n)
        P.hmat_matvec(h64, x, yh, 1)
        assert np.array_equal(yd, yh)
        assert np.array_equal(yd, _gpu_matvec(P, torch, h64, x))
        # nrhs columns (column-major N x nrhs) = separate products
        X = np.random.default_rng(1).standard_normal((3, mesh.n))  # rows = columns of N x 3
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        P.hmat_matvec(h64, Xd, Yd, 3)
        torch.cuda.synchronize()
        for k in range(3):
            assert np.array_equal(Yd[k].cpu().numpy(), _gpu_matvec(P, torch, h64, X[k]))
    finally:
        P.hmat_destroy(h32)
        P.hmat_destroy(h64)


@pytest.mark.parametrize("case", ["single_panel", "one_leaf", "all_dense", "dense3x3"])
def test_edge_cases(oracle_mod, case):
    torch = need_gpu()
    P = lib()
    if case == "dense3x3":
        A = np.array([[2.0, 1.0, -1.0], [-1.0, -1.0, 0.0], [-1.0, 1.0, -1.0]])
        blob = dense_blob(A)
        x = np.array([0.5, -2.0, 3.0])
        ref = A @ x
    else:
        if case == "single_panel":
            mesh = synth.Mesh(tri=np.zeros((1, 3, 3)), centroid=np.zeros((1, 3)), area=np.array([0.7]), name="one")
            H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
        elif case == "one_leaf":
            mesh = synth.icosphere(0)
            H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
        else:
            mesh = synth.icosphere(2)
            H = oracle_mod.HMatrix(mesh.centroid, mesh.area, eta=0.0)
        blob = oracle_blob(H)
        x = np.random.default_rng(3).standard_normal(mesh.n)
        ref = H.matvec(x)
    for form, tol in (("fp64", 1e-13), ("fp64_dfma", 1e-15), ("fp32", 1e-6), ("bf16", 1e-2)):
        h = P.hmat_upload(blob, form)
        try:
            y = _gpu_matvec(P, torch, h, x)
            assert rel(y, ref) <= tol, (form, rel(y, ref))
        finally:
            P.hmat_destroy(h)


def test_full_size_sampled_rows(oracle_mod):
    """Icosphere level 6 (N = 81,920), the configuration the benchmark times, built by
    the library's host builder; sampled rows against the oracle's own H-matrix."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(6)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
    x = synth.rhs_one_plus_half_z(mesh) + 0.1 * np.random.default_rng(6).standard_normal(mesh.n)
    rows = np.random.default_rng(7).choice(mesh.n, 400, replace=False)
    ref = H.matvec_rows(x, rows)
    for form, tol in (("fp64", 1e-13), ("fp64_dfma", 1e-14), ("fp32", 1e-6), ("bf16", 1e-2)):
        h = P.hmat_upload(blob, form)
        try:
            y = _gpu_matvec(P, torch, h, x)
            assert maxrel(y[rows], ref) <= tol, (form, maxrel(y[rows], ref))
        finally:
            P.hmat_destroy(h)


def test_upload_rejects_bad_blob():
    need_gpu()
    P = lib()
    bad = np.zeros(512, dtype=np.uint8)
    with pytest.raises(P.HmatError) as e:
        P.hmat_upload(bad, "fp64")
    assert e.value.status == 2
