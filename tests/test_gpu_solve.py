"""GPU BiCG-STAB (Algorithm 1) with the FP64 true-residual acceptance of
Section 4.1.3, against the oracle's solve and closed-form electrostatics."""
import math
import os

import numpy as np
import pytest

import synth
from blob_util import dense_blob, oracle_blob
from gpu_util import lib, need_gpu, rel

pytestmark = pytest.mark.gpu


def _solve(P, torch, h, b, **kw):
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xd = torch.zeros_like(bd)
    info = P.hmat_bicgstab(h, bd, xd, **kw)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), info


@pytest.mark.parametrize("level", [3, 4])
def test_fp64_solve_matches_oracle(hcache, oracle_mod, level):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(level)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    h = P.hmat_upload(oracle_blob(H), "fp64")
    try:
        x, info = _solve(P, torch, h, b, tol=1e-8)
        assert info["status"] == 0 and info["relres_true"] <= 1e-8
        xo, io = H.bicgstab(b, tol=1e-8)
        # the iteration count of Algorithm 1 depends on the summation order of its
        # inner products: the oracle's own recurrence with the GPU's order (cluster
        # order, per-leaf-cluster partial sums) takes 14 instead of 16 iterations at
        # level 3, so only the agreement of the counts within ~20% is asserted
        assert abs(info["iters"] - io["iters"]) <= max(2, io["iters"] // 5), (info["iters"], io["iters"])
        # same algorithm and stop rule: the two 1e-8 solutions agree far below the
        # discretisation error (their difference is bounded by cond(A) * 2e-8)
        assert rel(x, xo) <= 1e-5
        # the oracle's own product confirms the true residual
        assert np.linalg.norm(b - H.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
    finally:
        P.hmat_destroy(h)


@pytest.mark.parametrize("form,opts", [("fp64", {}), ("fp64_dfma", {}), ("fp32", {}),
                                       ("fp32", {"inner_tol": 1e-4}), ("bf16", {"inner_tol": 1e-2})],
                         ids=["fp64", "fp64_dfma", "fp32", "fp32_refine", "bf16_refine"])
def test_every_form_reaches_fp64_true_residual(hcache, oracle_mod, form, opts):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        x, info = _solve(P, torch, h, b, tol=1e-8, **opts)
        assert info["status"] == 0, info
        assert info["relres_true"] <= 1e-8
        assert np.linalg.norm(b - H.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
        if form == "bf16":
            assert info["restarts"] >= 2
    finally:
        P.hmat_destroy(h)


def test_graph_batches_and_host_pointers_agree(hcache):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    h = P.hmat_upload(oracle_blob(H), "fp32")
    try:
        x1, i1 = _solve(P, torch, h, b, tol=1e-8, use_graph=0, check_every=1)
        x2, i2 = _solve(P, torch, h, b, tol=1e-8, use_graph=1, check_every=1)
        x3, i3 = _solve(P, torch, h, b, tol=1e-8, use_graph=1, check_every=5)
        xh = np.zeros(mesh.n)
        i4 = P.hmat_bicgstab(h, b.copy(), xh, tol=1e-8)
        # a whole run as one graph launch (a device-side WHILE loop over batches)
        x5, i5 = _solve(P, torch, h, b, tol=1e-8, use_graph=2, check_every=1)
        x6, i6 = _solve(P, torch, h, b, tol=1e-8, use_graph=2, check_every=4)
        for x, i in ((x2, i2), (x3, i3), (xh, i4), (x5, i5), (x6, i6)):
            assert np.array_equal(x, x1) and i["iters"] == i1["iters"]
        # the device loop also ends on the iteration budget, and with refinement runs
        _, i7 = _solve(P, torch, h, b, tol=1e-8, use_graph=2, check_every=3, maxit=5, max_restarts=0)
        assert i7["status"] == 7 and i7["iters"] == 5, i7
        x8, i8 = _solve(P, torch, h, b, tol=1e-8, use_graph=2, check_every=4, inner_tol=1e-3)
        x9, i9 = _solve(P, torch, h, b, tol=1e-8, use_graph=1, check_every=4, inner_tol=1e-3)
        assert i8["status"] == 0 and i8["restarts"] >= 1 and np.array_equal(x8, x9) and i8["iters"] == i9["iters"]
    finally:
        P.hmat_destroy(h)


def test_status_cases(hcache):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(2)
    H = hcache(mesh)
    h = P.hmat_upload(oracle_blob(H), "fp64")
    try:
        x, info = _solve(P, torch, h, np.zeros(mesh.n))
        assert info["status"] == 0 and info["iters"] == 0 and not x.any()
        x, info = _solve(P, torch, h, np.ones(mesh.n), maxit=1)
        assert info["status_name"] == "maxit" and info["iters"] == 1
        bn = np.ones(mesh.n); bn[4] = np.nan
        x, info = _solve(P, torch, h, bn)
        assert info["status_name"] == "nonfinite"
    finally:
        P.hmat_destroy(h)
    # exact rho = 0 breakdown (alpha = 1/2, omega = -1 are exact in binary arithmetic)
    A = np.array([[2.0, 1.0, -1.0], [-1.0, -1.0, 0.0], [-1.0, 1.0, -1.0]])
    for form in ("fp64", "fp64_dfma"):
        h = P.hmat_upload(dense_blob(A), form)
        try:
            x, info = _solve(P, torch, h, np.array([1.0, 0.0, 0.0]), tol=1e-12)
            assert info["status_name"] == "breakdown_rho" and info["iters"] == 2, info
        finally:
            P.hmat_destroy(h)


def test_unit_sphere_total_charge_on_gpu(hcache):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    h = P.hmat_upload(blob, "fp32")
    try:
        sigma, info = _solve(P, torch, h, synth.rhs_constant(mesh), tol=1e-8)
        assert info["status"] == 0
        q = float(np.dot(sigma, mesh.area)) / (4 * math.pi)
        assert abs(q - 1.0) <= 3e-2
    finally:
        P.hmat_destroy(h)


def test_full_size_solve_true_residual(oracle_mod):
    """Icosphere level 6 (N = 81,920): the FP64 true residual of the GPU solution,
    recomputed by the oracle's own H-matrix, meets 1e-8."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(6)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
    b = synth.rhs_one_plus_half_z(mesh)
    for form, opts in (("fp64", {}), ("bf16", {"inner_tol": 1e-2})):
        h = P.hmat_upload(blob, form)
        try:
            x, info = _solve(P, torch, h, b, tol=1e-8, **opts)
            assert info["status"] == 0, info
            assert np.linalg.norm(b - H.matvec(x)) / np.linalg.norm(b) <= 1.05e-8
        finally:
            P.hmat_destroy(h)


def test_two_spheres_level7_bf16_refinement(oracle_mod):
    """Two unit spheres at potentials +1 / -1, centres 3 apart, icosphere level 7
    each (N = 655,360): BF16 panels with power-of-two scales inside the FP64
    iterative refinement reach a true relative residual of 1e-8, checked with the
    oracle's own FP64 H-matrix; sampled rows of the FP64 product match the
    oracle; the charges approach the image-series value (golden file) and are
    opposite up to the approximation."""
    torch = need_gpu()
    P = lib()
    mesh = synth.two_spheres(7)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
    b = synth.rhs_two_spheres(mesh)
    h = P.hmat_upload(blob, "bf16")
    del blob
    try:
        rows = np.random.default_rng(77).choice(mesh.n, 300, replace=False)
        xs = np.random.default_rng(78).standard_normal(mesh.n)
        y64 = np.empty(mesh.n)
        P.hmat_matvec(h, xs, y64, 1, None, True)
        ref = H.matvec_rows(xs, rows)
        assert float(np.max(np.abs(y64[rows] - ref)) / np.max(np.abs(ref))) <= 1e-13
        x, info = _solve(P, torch, h, b, tol=1e-8, inner_tol=1e-2, maxit=2000, check_every=4)
        assert info["status"] == 0 and info["restarts"] >= 1, info
        assert np.linalg.norm(b - H.matvec(x)) / np.linalg.norm(b) <= 1.05e-8
        half = mesh.n // 2
        q1 = float(np.dot(x[:half], mesh.area[:half])) / (4 * math.pi)
        q2 = float(np.dot(x[half:], mesh.area[half:])) / (4 * math.pi)
        gold = float(open(os.path.join(os.path.dirname(__file__), "golden", "two_spheres_charge.txt")).read().split()[-1])
        assert abs(q1 / gold - 1.0) <= 1e-2, (q1, gold)
        # antisymmetric up to the H-matrix approximation (ACA eps 1e-4 breaks the mirror symmetry)
        assert abs(q1 + q2) <= 1e-3 * abs(q1), (q1, q2)
    finally:
        P.hmat_destroy(h)
