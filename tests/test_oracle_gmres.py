"""The oracle's restarted GMRES(m) (a second Krylov method on the same products):
pinned by properties of the method itself, not by its own code -- finite
termination on a matrix with k distinct eigenvalues, exact solves on small dense
systems against LAPACK, and agreement with the oracle's BiCG-STAB on the BEM
system."""
import numpy as np
import pytest

import synth


def test_gmres_terminates_in_k_steps_for_k_eigenvalues(oracle_mod):
    # A diagonalizable matrix with 3 distinct eigenvalues: the Krylov space has
    # dimension 3, so GMRES (restart length >= 3) finds the solution in 3 steps.
    rng = np.random.default_rng(1)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat([1.0, 2.5, -0.75], [14, 13, 13])
    A = Q @ np.diag(lam) @ Q.T
    b = rng.standard_normal(n)
    x, info = oracle_mod.dense_gmres(A, b, m=10, tol=1e-12)
    assert info["status"] == "ok" and info["iters"] == 3, info
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(x)


@pytest.mark.parametrize("m", [5, 50])
def test_gmres_dense_nonsymmetric_against_lapack(oracle_mod, m):
    rng = np.random.default_rng(m)
    n = 50
    A = rng.standard_normal((n, n)) + 8.0 * np.eye(n)
    b = rng.standard_normal(n)
    x, info = oracle_mod.dense_gmres(A, b, m=m, tol=1e-12, maxit=2000)
    assert info["status"] == "ok"
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
    if m >= n:
        assert info["iters"] <= n  # full GMRES terminates within n steps


def test_gmres_identity_one_step(oracle_mod):
    b = np.arange(1.0, 8.0)
    x, info = oracle_mod.dense_gmres(np.eye(7), b, m=3, tol=1e-14)
    assert info["iters"] == 1 and np.allclose(x, b, rtol=0, atol=1e-15)


def test_gmres_matches_bicgstab_on_the_bem_system(hcache, oracle_mod):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    b = synth.rhs_one_plus_half_z(mesh)
    xg, ig = H.gmres(b, m=20, tol=1e-10)
    xb, ib = H.bicgstab(b, tol=1e-10)
    assert ig["status"] == "ok" and ig["relres"] <= 1e-10
    assert np.linalg.norm(xg - xb) <= 1e-8 * np.linalg.norm(xb)
    # a restart length shorter than the iteration count restarts cycles and still converges
    xs, i_s = H.gmres(b, m=4, tol=1e-10, maxit=2000)
    assert i_s["status"] == "ok" and i_s["iters"] > ig["iters"]
    assert np.linalg.norm(xs - xb) <= 1e-8 * np.linalg.norm(xb)
