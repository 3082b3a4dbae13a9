"""The allocation-free product (hmat_matvec_noalloc) against the ordinary one.

Callers that cannot allocate device memory when they run the product -- a
latency-critical loop that cannot pay for a cudaMalloc, or code whose device
memory belongs to another allocator or budget -- create a handle once and then
call hmat_matvec_noalloc, whose scratch lives in a static device array of the
library.  This file is collected last so
that a run stopping at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth
from gpu_util import lib, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL = 1e-13  # the two entry points run the same kernels on the same panels


def _device(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("form", ["fp64", "fp32", "bf16"])
def test_noalloc_matches_matvec_on_two_calls(form):
    torch = need_gpu()
    P = lib()
    small, mid = synth.icosphere(3), synth.icosphere(4)
    h3 = P.hmat_upload(P.hmat_build(small.centroid, small.area), form)
    h4 = P.hmat_upload(P.hmat_build(mid.centroid, mid.area), form)
    try:
        rng = np.random.default_rng(2024)
        # two calls in a row on one handle, then another handle of another size:
        # every call must see a clean scratch, whatever the previous call left there
        for h, mesh in ((h4, mid), (h4, mid), (h3, small), (h4, mid)):
            x = _device(torch, rng.standard_normal(mesh.n))
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, np.nan)
            P.hmat_matvec(h, x, y_ref)
            P.hmat_matvec_noalloc(h, x, y)
            torch.cuda.synchronize()
            assert rel(y.cpu().numpy(), y_ref.cpu().numpy()) <= TOL
    finally:
        P.hmat_destroy(h3)
        P.hmat_destroy(h4)


def test_noalloc_rejects_host_pointers_and_oversized_handles():
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(2)
    h = P.hmat_upload(P.hmat_build(mesh.centroid, mesh.area), "fp64")
    try:
        x = np.ones(mesh.n)
        y = np.zeros(mesh.n)
        with pytest.raises(P.HmatError) as e:
            P.hmat_matvec_noalloc(h, x, y)
        assert e.value.status == 1
    finally:
        P.hmat_destroy(h)
    big = synth.icosphere(6)  # its scratch is larger than the static array
    hb = P.hmat_upload(P.hmat_build(big.centroid, big.area), "fp64")
    try:
        xd = torch.ones(big.n, dtype=torch.float64, device="cuda")
        yd = torch.zeros_like(xd)
        with pytest.raises(P.HmatError) as e:
            P.hmat_matvec_noalloc(hb, xd, yd)
        assert e.value.status == 10
    finally:
        P.hmat_destroy(hb)


def test_noalloc_paper_variants():
    """A one-segment paper variant runs through the static array like any form;
    a two-segment one (its products add two expansions) is rejected."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    x = _device(torch, np.random.default_rng(8).standard_normal(mesh.n))
    h1 = P.hmat_upload(blob, "m2_mixed")
    h2 = P.hmat_upload(blob, "m3", 1)
    try:
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, np.nan)
        P.hmat_matvec(h1, x, y_ref)
        P.hmat_matvec_noalloc(h1, x, y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), y_ref.cpu().numpy()) <= TOL
        with pytest.raises(P.HmatError) as e:
            P.hmat_matvec_noalloc(h2, x, y)
        assert e.value.status == 10
    finally:
        P.hmat_destroy(h1)
        P.hmat_destroy(h2)
