"""Pins of the oracle's BiCG-STAB (Algorithm 1) with the true-residual acceptance
of Section 4.1.3, against library solves, and of the whole oracle against
closed-form electrostatics."""
import math
import os

import numpy as np
import pytest

import synth


def test_dense_solve_matches_numpy(oracle_mod):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((60, 60)) + 8 * np.eye(60)
    b = rng.standard_normal(60)
    assert np.allclose(oracle_mod.dense_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)


def test_dense_bicgstab_matches_numpy(oracle_mod):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((80, 80)) + 10 * np.eye(80)   # nonsymmetric, well conditioned
    b = rng.standard_normal(80)
    x, info = oracle_mod.dense_bicgstab(A, b, tol=1e-13)
    assert info["status"] == "ok" and info["relres"] <= 1e-13
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


def test_rho_breakdown_is_reported(oracle_mod):
    # exact binary arithmetic: alpha_1 = 1/2, omega_1 = -1 and r~^T r_1 = 0 exactly
    A = np.array([[2.0, 1.0, -1.0], [-1.0, -1.0, 0.0], [-1.0, 1.0, -1.0]])
    b = np.array([1.0, 0.0, 0.0])
    x, info = oracle_mod.dense_bicgstab(A, b, tol=1e-12)
    assert info["status"] == "breakdown_rho" and info["iters"] == 2


def test_maxit_nonfinite_and_zero_rhs(hcache, oracle_mod):
    mesh = synth.icosphere(2)
    H = hcache(mesh)
    b = np.ones(mesh.n)
    x, info = H.bicgstab(b, maxit=1)
    assert info["status"] == "maxit" and info["iters"] == 1
    bn = b.copy(); bn[5] = np.nan
    x, info = H.bicgstab(bn)
    assert info["status"] == "nonfinite"
    x, info = H.bicgstab(np.zeros(mesh.n))
    assert info["status"] == "ok" and info["iters"] == 0 and not x.any()


def test_hmatrix_solve_matches_dense_solve_of_same_operator(hcache):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    x, info = H.bicgstab(b, tol=1e-12)
    assert info["status"] == "ok" and info["relres"] <= 1e-12
    ref = np.linalg.solve(H.to_dense(), b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def _charge(mesh, sigma):
    return float(np.dot(sigma, mesh.area))


def test_unit_sphere_uniform_density_and_total_charge(hcache):
    """phi = 1 on the unit sphere: sigma = 1 and Q = 4 pi (unit permittivity)."""
    errs = []
    for level in (2, 3, 4):
        mesh = synth.icosphere(level)
        H = hcache(mesh)
        sigma, info = H.bicgstab(synth.rhs_constant(mesh), tol=1e-10)
        assert info["status"] == "ok"
        errs.append(abs(_charge(mesh, sigma) / (4 * math.pi) - 1.0))
        assert abs(np.mean(sigma) - 1.0) < 0.06
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 3e-2


def test_unit_sphere_first_harmonic(hcache):
    """phi = 1 + z/2: the l=1 harmonic of the unit-sphere single layer has
    eigenvalue 1/3, so sigma = 1 + 1.5 z."""
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    sigma, info = H.bicgstab(synth.rhs_one_plus_half_z(mesh), tol=1e-10)
    assert info["status"] == "ok"
    z = mesh.centroid[:, 2] / np.linalg.norm(mesh.centroid, axis=1)
    a, b = np.linalg.lstsq(np.stack([np.ones_like(z), z], 1), sigma, rcond=None)[0]
    assert abs(a - 1.0) < 0.03 and abs(b / 1.5 - 1.0) < 0.03


def _two_sphere_constant():
    path = os.path.join(os.path.dirname(__file__), "golden", "two_spheres_charge.txt")
    val = float([l for l in open(path) if not l.startswith("#")][0])
    beta = math.acosh(1.5)
    series = math.sinh(beta) * sum(1.0 / math.sinh(n * beta) for n in range(1, 400))
    # method of images, iterated to convergence
    d, R = 3.0, 1.0
    q1, new1, new2 = 4 * math.pi, [(0.0, 4 * math.pi)], [(d, -4 * math.pi)]
    for _ in range(200):
        im1 = [(R * R / p, -q * R / p) for p, q in new2]
        im2 = [(d - R * R / (d - p), -q * R / (d - p)) for p, q in new1]
        q1 += sum(q for _, q in im1)
        new1, new2 = im1, im2
    assert abs(series - val) < 1e-14 and abs(q1 / (4 * math.pi) - val) < 1e-14
    return val


def test_two_spheres_charge(hcache):
    target = _two_sphere_constant()
    errs = []
    for level in (2, 3, 4):
        mesh = synth.two_spheres(level)
        H = hcache(mesh)
        sigma, info = H.bicgstab(synth.rhs_two_spheres(mesh), tol=1e-10)
        assert info["status"] == "ok"
        n2 = mesh.n // 2
        q1 = float(np.dot(sigma[:n2], mesh.area[:n2])) / (4 * math.pi)
        q2 = float(np.dot(sigma[n2:], mesh.area[n2:])) / (4 * math.pi)
        assert abs(q1 + q2) < 2 * H.eps * abs(q1)  # antisymmetric up to the ACA tolerance
        errs.append(abs(q1 / target - 1.0))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.03


def test_unit_cube_capacitance_loose(hcache):
    """Unit cube at unit potential: C ~ 0.6607 x 4 pi (literature value, an external
    constant); corners and edges make collocation converge slowly, so the pin is loose."""
    mesh = synth.unit_cube(12)
    H = hcache(mesh)
    sigma, info = H.bicgstab(synth.rhs_constant(mesh), tol=1e-10)
    assert info["status"] == "ok"
    c = _charge(mesh, sigma) / (4 * math.pi)
    assert abs(c / 0.6607 - 1.0) < 0.05


@pytest.mark.parametrize("name,c", [("M1_SINGLE", 0), ("M1_MIXED", 0), ("M2_SINGLE", 0), ("M2_MIXED", 0),
                                    ("M3", -1), ("M3", 3), ("DATA_FP32", 0)])
def test_variant_solves_reach_true_residual(hcache, oracle_mod, name, c):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    x, info = H.bicgstab(b, variant=oracle_mod.VARIANTS[name], c=c, tol=1e-8)
    assert info["status"] == "ok" and info["relres"] <= 1e-8
    x64, i64 = H.bicgstab(b, tol=1e-8)
    assert np.linalg.norm(x - x64) <= 1e-6 * np.linalg.norm(x64)


def test_bf16_refinement_reaches_fp64_accuracy(hcache, oracle_mod):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    x, info = H.bicgstab(b, variant=oracle_mod.DATA_BF16, tol=1e-8, inner_tol=1e-2)
    assert info["status"] == "ok" and info["relres"] <= 1e-8
    assert info["restarts"] >= 2          # BF16 alone stalls near 1e-3
