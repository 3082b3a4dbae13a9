"""Pins of the oracle's ACA with partial pivoting."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("k", [1, 3, 7])
def test_exact_low_rank_is_recovered(oracle_mod, k):
    rng = np.random.default_rng(k)
    A = rng.standard_normal((40, k)) @ rng.standard_normal((k, 30))
    U, V = oracle_mod.aca(A, 1e-10)
    assert U.shape[1] in (k, k + 1)
    assert np.linalg.norm(A - U @ V.T) <= 1e-12 * np.linalg.norm(A)


def test_zero_block_has_rank_zero(oracle_mod):
    U, V = oracle_mod.aca(np.zeros((10, 12)), 1e-4)
    assert U.shape[1] == 0


def test_zero_first_row_moves_on(oracle_mod):
    rng = np.random.default_rng(3)
    A = np.outer(rng.standard_normal(8), rng.standard_normal(9))
    A[0, :] = 0.0
    U, V = oracle_mod.aca(A, 1e-8)
    assert U.shape[1] >= 1
    assert np.linalg.norm(A - U @ V.T) <= 1e-13 * np.linalg.norm(A)


def test_full_rank_stops_at_min_dimension(oracle_mod):
    A = np.eye(5)
    U, V = oracle_mod.aca(A, 1e-12)
    assert U.shape[1] == 5
    assert np.allclose(U @ V.T, A, atol=1e-15)


def test_cross_interpolation_property(oracle_mod):
    # after r steps the approximant reproduces the pivot rows and columns exactly
    rng = np.random.default_rng(5)
    x = np.sort(rng.random(30)); y = np.sort(rng.random(25)) + 2.0
    A = 1.0 / np.abs(x[:, None] - y[None, :])
    U, V = oracle_mod.aca(A, 1e-6)
    S = U @ V.T
    r = U.shape[1]
    # the pivot columns are where v_l has its 1.0 entry (v_l = R / R_j*)
    piv_cols = [int(np.argmax(np.abs(V[:, l]) == 1.0)) for l in range(r)]
    for j in piv_cols:
        assert np.allclose(S[:, j], A[:, j], rtol=1e-12, atol=1e-14)
    assert np.linalg.norm(A - S) <= 1e-5 * np.linalg.norm(A)


def test_bem_blocks_meet_tolerance(hcache, oracle_mod):
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    A = oracle_mod.dense_matrix(mesh.centroid, mesh.area)
    P = A[np.ix_(H.perm, H.perm)]
    errs, e2, n2 = [], 0.0, 0.0
    for b, (i_s, i_e, j_s, j_e, kind, rank, forced) in enumerate(H.blocks):
        blk = P[i_s:i_e, j_s:j_e]
        if kind == 0:
            assert np.array_equal(H.block_data(b), blk)
            continue
        Vm, Wm = H.block_data(b)
        e = np.linalg.norm(blk - Vm @ Wm)
        errs.append(e / np.linalg.norm(blk))
        e2 += e * e
        n2 += np.linalg.norm(blk) ** 2
    errs = np.array(errs)
    # partial pivoting estimates the error from the last cross only: globally the
    # low-rank part meets eps, single blocks may miss it by a small factor
    assert np.sqrt(e2 / n2) <= 2 * H.eps
    assert np.percentile(errs, 99) <= 10 * H.eps
    assert errs.max() <= 30 * H.eps
