"""Failure detection of the tensor-core product without a GPU fault.

The product of many right-hand sides hands shared-memory buffers between the
copy engine, the tensor cores and the threads through mbarriers.  Every wait is
bounded; a wait that runs out records HMAT_ERR_TIMEOUT in the handle's status
word, lets the issued copies and MMAs finish, frees the tensor memory and
returns.  Here the projection is told to issue none of its copies (a completion
that nothing signals), the limit is short, and the tests check that the host
reads the status and that the context and the handle work normally afterwards.
"""
import numpy as np
import pytest

import synth
from blob_util import oracle_blob
from gpu_util import lib, need_gpu, rel

pytestmark = pytest.mark.gpu

SHORT = 200_000            # SM cycles: about 0.1 ms
DEFAULT = 2_000_000_000    # the library's default bound (about one second)


@pytest.mark.parametrize("form,data,tol", [("bf16", "DATA_BF16", 2e-5), ("fp32", "DATA_FP32", 1e-5)])
def test_tensor_core_timeout_is_reported_and_the_handle_recovers(hcache, oracle_mod, form, data, tol):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        nrhs = 3
        X = synth.rhs_normal_columns(mesh.n, nrhs, seed=7)
        Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
        Yd = torch.empty_like(Xd)
        P.hmat_set_wait_limit(h, SHORT, withhold=True)
        P.hmat_matvec(h, Xd, Yd, nrhs)                # asynchronous: reported later
        assert P.hmat_check(h) == P.HMAT_ERR_TIMEOUT
        assert P.hmat_check(h) == 0                   # taken once
        # a synchronous call (host vectors) reports its own product's timeout
        with pytest.raises(P.HmatError) as e:
            P.hmat_matvec(h, np.ascontiguousarray(X.T), np.empty((nrhs, mesh.n)), nrhs)
        assert e.value.status == P.HMAT_ERR_TIMEOUT
        # an asynchronous product's timeout is returned by the next call
        P.hmat_matvec(h, Xd, Yd, nrhs)
        torch.cuda.synchronize()
        with pytest.raises(P.HmatError) as e:
            P.hmat_matvec(h, Xd, Yd, nrhs)
        assert e.value.status == P.HMAT_ERR_TIMEOUT
        assert P.hmat_check(h) == 0                   # the refused call enqueued nothing
        # normal operation again: the context and the handle are usable
        P.hmat_set_wait_limit(h, DEFAULT, withhold=False)
        P.hmat_matvec(h, Xd, Yd, nrhs)
        assert P.hmat_check(h) == 0
        Y = Yd.cpu().numpy().T
        for k in range(nrhs):
            assert rel(Y[:, k], H.matvec(X[:, k], getattr(oracle_mod, data))) <= tol
    finally:
        P.hmat_destroy(h)


def test_many_system_solve_stops_with_timeout_and_then_converges(hcache):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(4)
    H = hcache(mesh)
    h = P.hmat_upload(oracle_blob(H), "bf16")
    try:
        nrhs = 2
        B = torch.from_numpy(np.ascontiguousarray(synth.rhs_normal_columns(mesh.n, nrhs, seed=3).T)).cuda()
        X = torch.zeros_like(B)
        P.hmat_set_wait_limit(h, SHORT, withhold=True)
        infos = P.hmat_bicgstab_multi(h, B, X, nrhs, tol=1e-8, inner_tol=1e-2)
        assert all(i["status"] == P.HMAT_ERR_TIMEOUT for i in infos)
        assert P.hmat_check(h) == 0
        P.hmat_set_wait_limit(h, DEFAULT, withhold=False)
        X.zero_()
        infos = P.hmat_bicgstab_multi(h, B, X, nrhs, tol=1e-8, inner_tol=1e-2)
        assert all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in infos)
    finally:
        P.hmat_destroy(h)


def test_wait_limit_arguments():
    need_gpu()
    P = lib()
    mesh = synth.icosphere(2)
    h = P.hmat_upload(P.hmat_build(mesh.centroid, mesh.area), "bf16")
    try:
        with pytest.raises(P.HmatError) as e:
            P.hmat_set_wait_limit(h, 0)
        assert e.value.status == 1
    finally:
        P.hmat_destroy(h)
