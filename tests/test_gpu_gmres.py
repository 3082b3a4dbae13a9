"""GPU restarted GMRES(m) (hmat_gmres) against the oracle's GMRES on the same
H-matrix, in FP64 and with the low-precision forms inside the FP64 true-residual
restarts."""
import numpy as np
import pytest

import synth
from blob_util import oracle_blob
from gpu_util import lib, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [20, 4])
def test_gmres_fp64_matches_oracle(hcache, oracle_mod, m):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    h = P.hmat_upload(oracle_blob(H), "fp64")
    try:
        x = np.zeros(mesh.n)
        info = P.hmat_gmres(h, b, x, m=m, tol=1e-10, maxit=2000)
        xr, ref = H.gmres(b, m=m, tol=1e-10, maxit=2000)
        assert info["status"] == 0 and ref["status"] == "ok", (info, ref)
        assert info["relres_true"] <= 1e-10
        assert abs(info["iters"] - ref["iters"]) <= max(2, ref["iters"] // 10), (info["iters"], ref["iters"])
        assert rel(x, xr) <= 1e-8
        assert np.linalg.norm(b - H.matvec(x)) / np.linalg.norm(b) <= 1.05e-10
    finally:
        P.hmat_destroy(h)


@pytest.mark.parametrize("form,opts", [("bf16", {"inner_tol": 1e-2}), ("fp32", {"inner_tol": 1e-4}),
                                       ("m2_mixed", {"inner_tol": 1e-4})])
def test_gmres_low_precision_forms_reach_fp64_residual(hcache, oracle_mod, form, opts):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        xd = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        info = P.hmat_gmres(h, torch.from_numpy(b).cuda(), xd, m=30, tol=1e-8, maxit=2000, **opts)
        x = xd.cpu().numpy()
        assert info["status"] == 0 and info["relres_true"] <= 1e-8, info
        assert np.linalg.norm(b - H.matvec(x)) / np.linalg.norm(b) <= 1.05e-8
    finally:
        P.hmat_destroy(h)


def test_gmres_statuses(hcache):
    need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    h = P.hmat_upload(oracle_blob(hcache(mesh)), "fp64")
    try:
        x = np.ones(mesh.n)
        info = P.hmat_gmres(h, np.zeros(mesh.n), x, m=10)
        assert info["status"] == 0 and info["iters"] == 0 and np.all(x == 0.0)
        x = np.zeros(mesh.n)
        info = P.hmat_gmres(h, synth.rhs_one_plus_half_z(mesh), x, m=10, tol=1e-14, maxit=3, max_restarts=0)
        assert info["status"] == 7 and info["iters"] == 3, info
        with pytest.raises(P.HmatError):
            P.hmat_gmres(h, np.ones(mesh.n), x, m=65)
    finally:
        P.hmat_destroy(h)


def test_gmres_full_size_bf16(oracle_mod):
    """Icosphere level 6 (N = 81,920), BF16 panels inside the FP64 refinement."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(6)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
    b = synth.rhs_one_plus_half_z(mesh)
    h = P.hmat_upload(blob, "bf16")
    try:
        xd = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        info = P.hmat_gmres(h, torch.from_numpy(b).cuda(), xd, m=40, tol=1e-8, maxit=2000, inner_tol=1e-2)
        assert info["status"] == 0, info
        assert np.linalg.norm(b - H.matvec(xd.cpu().numpy())) / np.linalg.norm(b) <= 1.05e-8
    finally:
        P.hmat_destroy(h)
