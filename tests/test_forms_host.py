"""The host derivation of every precision form (hmat_form_stats_get: the
segments hmat_upload_ex would pack and check, computed without a device)
against counts taken from the oracle's own H-matrix: Method 3's rank split
(eq. 19-20 on the d_l of eq. 14-16), Section 4.5's rank truncation and
dense-column split, and conservation of every stored entry."""
import numpy as np
import pytest

import synth
from blob_util import oracle_blob
from gpu_util import lib


@pytest.fixture(scope="module", params=["icosphere3", "two_spheres3", "cube8"])
def case(hcache, request):
    mesh = {"icosphere3": synth.icosphere(3), "two_spheres3": synth.two_spheres(3),
            "cube8": synth.unit_cube(8)}[request.param]
    H = hcache(mesh)
    return mesh, H, oracle_blob(H)


def _lr_split(H, c):
    """(ranks with d_l >= d_max 10^-c, the others), over every low-rank block."""
    hi = lo = 0
    blk = H.blocks
    for b in range(len(blk)):
        if blk[b][4] == 1 and blk[b][5] > 0:
            _, _, d = H.method2_factors(b)
            k = int(np.sum(d >= d.max() * 10.0 ** (-c)))
            hi += k
            lo += len(d) - k
    return hi, lo


@pytest.mark.parametrize("form", ["fp64", "fp64_dfma", "fp32", "bf16", "m1_single", "m1_mixed", "m2_double",
                                  "m2_single", "m2_mixed"])
def test_every_entry_is_stored_once(case, form):
    _, H, blob = case
    P = lib()
    st = P.hmat_blob_stats(blob)
    fs = P.hmat_form_stats(blob, form)
    assert sum(fs["dense_entries"]) == st["dense_entries"]
    assert sum(fs["lr_ranks"]) == st["rank_sum"] and sum(fs["lr_entries"]) == st["lr_entries"]
    assert sum(fs["column_subsets"]) == 0
    # Methods 1-Mixed and 2-Single keep the dense blocks and the low-rank blocks apart
    assert fs["segments"] == (2 if form in ("m1_mixed", "m2_single") else 1)


@pytest.mark.parametrize("c", [-1, 1, 3, 7])
def test_method3_rank_split(case, c):
    _, H, blob = case
    P = lib()
    hi, lo = _lr_split(H, c)
    fs = P.hmat_form_stats(blob, "m3", c)
    ranks = fs["lr_ranks"] if fs["segments"] == 2 else fs["lr_ranks"] + [0]
    if hi == 0:  # no FP64 rank: the FP64 segment holds the dense blocks only
        assert ranks[0] == 0 and ranks[1] == lo
    else:
        assert ranks == [hi, lo]
    assert fs["dense_entries"][0] == P.hmat_blob_stats(blob)["dense_entries"]
    tr = P.hmat_form_stats(blob, "m3_trunc", c)
    assert tr["segments"] == 1 and tr["lr_ranks"] == [hi]


@pytest.mark.parametrize("c", [-1, 0, 1, 2, 16])
def test_dense_column_split(case, c):
    _, H, blob = case
    P = lib()
    blk = H.blocks
    dense = [b for b in range(len(blk)) if blk[b][4] == 0]
    dmax = max(np.abs(H.block_data(b)).max() for b in dense)
    thr = dmax * 10.0 ** (-c)
    e64 = e32 = both = 0
    for b in dense:
        A = H.block_data(b)
        w = np.abs(A).max(axis=0)
        n64 = int(np.sum(w >= thr))
        e64 += A.shape[0] * n64
        e32 += A.shape[0] * (A.shape[1] - n64)
        both += int(0 < n64 < A.shape[1])
    fs = P.hmat_form_stats(blob, "m3_dense", c)
    st = P.hmat_blob_stats(blob)
    if e64 == 0:  # every column demoted: Method 2-Mixed, one segment
        assert fs["segments"] == 1 and fs["dense_entries"] == [e32]
    else:
        assert fs["segments"] == 2 and fs["dense_entries"] == [e64, e32]
        assert fs["column_subsets"] == [both, both]
        assert (fs["selected_operands"][0] > 0) == (both > 0)
    # every low-rank block as Method 2-Mixed, in the FP32 segment
    assert fs["lr_ranks"][-1] == st["rank_sum"] and sum(fs["lr_ranks"]) == st["rank_sum"]


def test_form_arguments(case):
    _, _, blob = case
    P = lib()
    for form, c in (("m3", 17), ("m3_dense", -2), ("m3_trunc", 40)):
        with pytest.raises(P.HmatError) as e:
            P.hmat_form_stats(blob, form, c)
        assert e.value.status == 1
    with pytest.raises(P.HmatError):
        P.hmat_form_stats(blob, 12)
