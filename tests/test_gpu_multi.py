"""Many BiCG-STAB recurrences at once (hmat_bicgstab_multi): the 64 right-hand
sides of one H-matrix, and a batch of 48 independent problems of uneven size in
one block-diagonal handle.  Every system must reach a true relative residual of
1e-8 (checked with the oracle's own FP64 H-matrix) and agree with the oracle's
single-system FP64 solve to the accuracy the tolerance allows."""
import numpy as np
import pytest

import synth
from blob_util import oracle_blob
from gpu_util import lib, maxrel, need_gpu, rel

pytestmark = pytest.mark.gpu


def _true_rel(H, b, x):
    return float(np.linalg.norm(b - H.matvec(x)) / np.linalg.norm(b))


@pytest.mark.parametrize("form,opts", [("fp64", {}), ("bf16", {"inner_tol": 1e-2}), ("fp32", {"inner_tol": 1e-4}),
                                       ("m2_mixed", {"inner_tol": 1e-4})])
def test_multi_rhs_small(hcache, oracle_mod, form, opts):
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    nrhs = 8
    B = synth.rhs_normal_columns(mesh.n, nrhs)  # (N, nrhs), column-major
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        X = np.zeros((mesh.n, nrhs), order="F")
        infos = P.hmat_bicgstab_multi(h, B, X, nrhs, tol=1e-8, maxit=500, check_every=2, **opts)
        assert len(infos) == nrhs
        for k in range(nrhs):
            assert infos[k]["status"] == 0 and infos[k]["relres_true"] <= 1e-8, (k, infos[k])
            assert _true_rel(H, B[:, k], X[:, k]) <= 1.05e-8
            xk, _ = H.bicgstab(B[:, k], tol=1e-10)
            assert rel(X[:, k], xk) <= 1e-6, (k, rel(X[:, k], xk))
        # device tensors give the same bits; one system alone matches the single solver's accuracy
        Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
        Xd = torch.zeros_like(Bd)
        infos_d = P.hmat_bicgstab_multi(h, Bd, Xd, nrhs, tol=1e-8, maxit=500, check_every=2, **opts)
        torch.cuda.synchronize()
        assert np.array_equal(Xd.cpu().numpy().T, X)
        assert [i["iters"] for i in infos_d] == [i["iters"] for i in infos]
    finally:
        P.hmat_destroy(h)


def test_multi_rhs_statuses(hcache):
    """A zero right-hand side is solved by x = 0 without iterating; an iteration
    budget of 2 ends the other systems with HMAT_ERR_MAXIT, each on its own."""
    need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    B = synth.rhs_normal_columns(mesh.n, 3)
    B[:, 1] = 0.0
    h = P.hmat_upload(oracle_blob(H), "fp64")
    try:
        X = np.ones((mesh.n, 3), order="F")
        infos = P.hmat_bicgstab_multi(h, B, X, 3, tol=1e-8, maxit=2, max_restarts=0)
        assert infos[1]["status"] == 0 and infos[1]["iters"] == 0 and np.all(X[:, 1] == 0.0)
        for k in (0, 2):
            assert infos[k]["status"] == 7 and infos[k]["iters"] == 2, infos[k]
    finally:
        P.hmat_destroy(h)


def test_multi_rhs_full_size_64(oracle_mod):
    """Icosphere level 6 (N = 81,920), 64 right-hand sides of N(0,1) panel
    potentials, BF16 panels inside the FP64 refinement: all 64 recurrences reach
    1e-8 (oracle FP64 H-matrix); two columns match the oracle's FP64 solve."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(6)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
    nrhs = 64
    B = synth.rhs_normal_columns(mesh.n, nrhs)
    h = P.hmat_upload(blob, "bf16")
    try:
        Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
        Xd = torch.zeros_like(Bd)
        infos = P.hmat_bicgstab_multi(h, Bd, Xd, nrhs, tol=1e-8, maxit=2000, inner_tol=1e-2, check_every=4)
        torch.cuda.synchronize()
        X = Xd.cpu().numpy().T
        assert all(i["status"] == 0 for i in infos), [i for i in infos if i["status"] != 0][:2]
        for k in range(nrhs):
            assert _true_rel(H, B[:, k], X[:, k]) <= 1.05e-8, k
        for k in (0, 37):  # tol x cond of the level-6 single layer (~ 600) bounds the difference
            xk, _ = H.bicgstab(B[:, k], tol=1e-10)
            assert rel(X[:, k], xk) <= 1e-5, (k, rel(X[:, k], xk))
    finally:
        P.hmat_destroy(h)


def test_uneven_batch_48(oracle_mod):
    """48 independent problems (unit-cube surfaces and cube-spheres, N drawn
    log-uniformly in [1280, 20480]) in one block-diagonal handle with FP32 panels:
    every problem converges to 1e-8 against its own oracle H-matrix, and the
    batch handle's product is every problem's own product."""
    torch = need_gpu()
    P = lib()
    specs = synth.uneven_batch_specs(48)
    meshes = [synth.mesh_from_spec(s) for s in specs]
    blobs = [P.hmat_build(m.centroid, m.area) for m in meshes]
    h = P.hmat_upload_batch(blobs, "fp32")
    try:
        off = P.hmat_problems(h)
        assert len(off) == 49 and off[-1] == sum(m.n for m in meshes)
        b = np.concatenate([synth.rhs_constant(m) for m in meshes])
        x = np.zeros(off[-1])
        infos = P.hmat_bicgstab_multi(h, b, x, 1, tol=1e-8, maxit=2000, inner_tol=1e-4, check_every=4)
        assert all(i["status"] == 0 for i in infos), [i for i in infos if i["status"] != 0][:2]
        xs = np.random.default_rng(48).standard_normal(off[-1])
        ys = np.empty(off[-1])
        P.hmat_matvec(h, xs, ys, 1, None, True)  # FP64 operator of the whole batch
        for p, m in enumerate(meshes):
            sl = slice(off[p], off[p + 1])
            H = oracle_mod.HMatrix(m.centroid, m.area)
            assert _true_rel(H, b[sl], x[sl]) <= 1.05e-8, (p, specs[p])
            assert rel(ys[sl], H.matvec(xs[sl])) <= 1e-13, p
    finally:
        P.hmat_destroy(h)


# (form, the oracle's rounding of the same panels, tolerance): BF16 panels with
# x / t split into BF16 high and low parts (~2^-17 each); FP32 panels and
# operands both split into TF32 high and low parts (~2^-24 each), where the
# tensor cores' FP32 accumulation over ~1,000 terms is what remains (~4e-6
# measured at level 4, against 2e-7 for the single-column FP32 product)
TC_FORMS = [("bf16", "DATA_BF16", 2e-5), ("fp32", "DATA_FP32", 1e-5)]


@pytest.mark.parametrize("mesh", [synth.icosphere(3), synth.two_spheres(3), synth.icosphere(4)], ids=lambda m: m.name)
@pytest.mark.parametrize("nrhs", [64, 5, 70])
@pytest.mark.parametrize("form,data,tol", TC_FORMS, ids=[f[0] for f in TC_FORMS])
def test_tensor_core_product_parity(hcache, oracle_mod, mesh, nrhs, form, data, tol):
    """The product of many columns on the tensor cores (BF16 panels: kind::f16;
    FP32 panels: kind::tf32 on split parts) against the oracle's product on the
    same rounded panels (FP64 arithmetic) and against the single-column GPU
    product; 5 columns leave most of a pass empty, 70 take two passes."""
    torch = need_gpu()
    P = lib()
    H = hcache(mesh)
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        X = synth.rhs_normal_columns(mesh.n, nrhs, seed=nrhs)
        Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
        Yd = torch.empty_like(Xd)
        P.hmat_matvec(h, Xd, Yd, nrhs)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy().T
        for k in sorted({0, 1, nrhs // 2, nrhs - 1}):
            yr = H.matvec(X[:, k], getattr(oracle_mod, data))
            assert rel(Y[:, k], yr) <= tol, (k, rel(Y[:, k], yr))
            y1 = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
            P.hmat_matvec(h, Xd[k].contiguous(), y1, 1)
            torch.cuda.synchronize()
            assert rel(Y[:, k], y1.cpu().numpy()) <= tol
            assert rel(Y[:, k], H.matvec(X[:, k])) <= (1e-2 if form == "bf16" else 1e-5)
        # repeated passes give the same bits (no atomics)
        Y2 = torch.empty_like(Xd)
        P.hmat_matvec(h, Xd, Y2, nrhs)
        torch.cuda.synchronize()
        assert torch.equal(Y2, Yd)
    finally:
        P.hmat_destroy(h)


@pytest.mark.parametrize("form", ["bf16", "fp32", "fp64"])
def test_autotune_keeps_the_bits(hcache, form):
    """hmat_autotune changes only how the projection is launched (CTA size per
    panel-width bucket, the work list sorted by bucket): the products, single and
    batched, give the same bits before and after, and the solves still converge."""
    torch = need_gpu()
    P = lib()
    meshes = [synth.icosphere(4), synth.icosphere(3), synth.two_spheres(3)]
    blobs = [oracle_blob(hcache(m)) for m in meshes]
    for h in (P.hmat_upload(blobs[0], form), P.hmat_upload_batch(blobs, form)):
        try:
            n = sum(m.n for m in meshes) if len(P.hmat_problems(h)) > 2 else meshes[0].n
            x = torch.from_numpy(np.random.default_rng(3).standard_normal(n)).cuda()
            y0, y1 = torch.empty_like(x), torch.empty_like(x)
            P.hmat_matvec(h, x, y0)
            rep = P.hmat_autotune(h, reps=5)
            assert len(rep["buckets"]) == 5 and rep["default_us"] > 0 and rep["tuned_us"] > 0
            assert sum(b["clusters"] for b in rep["buckets"]) == P.hmat_info(h)["nleaves"]
            assert all(b["threads"] in (64, 128, 256) for b in rep["buckets"])
            P.hmat_matvec(h, x, y1)
            torch.cuda.synchronize()
            assert torch.equal(y0, y1)
            b = torch.ones_like(x)
            xs = torch.zeros_like(x)
            opts = {"bf16": {"inner_tol": 1e-2}, "fp32": {"inner_tol": 1e-4}}.get(form, {})
            infos = P.hmat_bicgstab_multi(h, b, xs, 1, tol=1e-8, **opts)
            assert all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in infos)
        finally:
            P.hmat_destroy(h)


@pytest.mark.parametrize("form,fp64", [("fp64", False), ("bf16", True), ("fp32", True)])
@pytest.mark.parametrize("nrhs", [2, 5, 19])
def test_double_float_many_columns_bits(hcache, oracle_mod, form, fp64, nrhs):
    """Several columns of a double-float operator (the FP64 handle's own, the
    FP64 copy of a BF16 or FP32 handle) go through the many-column product: each
    CTA or warp applies its panel loads to several columns.  Every column keeps
    the one-column product's summation order, so the bits are the same; 19
    columns take two passes of 16, and a batch handle covers the problem index
    of every work item."""
    torch = need_gpu()
    P = lib()
    meshes = [synth.icosphere(3), synth.two_spheres(3)]
    Hs = [hcache(m) for m in meshes]
    for h, H in ((P.hmat_upload(oracle_blob(Hs[0]), form), Hs[0]),
                 (P.hmat_upload_batch([oracle_blob(x) for x in Hs], form), None)):
        try:
            n = P.hmat_info(h)["n"]
            X = synth.rhs_normal_columns(n, nrhs, seed=7 + nrhs)
            Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
            Yd = torch.empty_like(Xd)
            P.hmat_matvec(h, Xd, Yd, nrhs, fp64=fp64)
            Yh = np.zeros(n * nrhs)  # host buffers, staged: flat column-major
            P.hmat_matvec(h, X.ravel(order="F").copy(), Yh, nrhs, fp64=fp64)
            torch.cuda.synchronize()
            assert np.array_equal(Yd.cpu().numpy(), Yh.reshape(nrhs, n))
            for k in range(nrhs):
                y1 = torch.empty(n, dtype=torch.float64, device="cuda")
                P.hmat_matvec(h, Xd[k].contiguous(), y1, 1, fp64=fp64)
                torch.cuda.synchronize()
                assert torch.equal(Yd[k], y1), k
                if H is not None and k in (0, nrhs - 1):
                    assert rel(Yd[k].cpu().numpy(), H.matvec(X[:, k])) <= 1e-13
        finally:
            P.hmat_destroy(h)


@pytest.mark.parametrize("form,opts", [("fp64", {}), ("bf16", {"inner_tol": 1e-2}), ("fp32", {"inner_tol": 1e-4})])
def test_multi_rhs_systems_independent(hcache, form, opts):
    """A system's result does not depend on the other systems solved with it:
    the true residual of a system whose run has stopped is taken at the next
    host read and the system restarts while the others iterate, so changing the
    other right-hand sides changes when runs end around it, but not one bit of
    its own iterates, counts or residuals."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    nrhs = 8
    B1 = synth.rhs_normal_columns(mesh.n, nrhs, seed=11)
    B2 = synth.rhs_normal_columns(mesh.n, nrhs, seed=12)
    B2[:, 0] = B1[:, 0]
    B2[:, 3] *= 1e3  # a column far from the others in scale
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        out = []
        for B in (B1, B2):
            Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
            Xd = torch.zeros_like(Bd)
            infos = P.hmat_bicgstab_multi(h, Bd, Xd, nrhs, tol=1e-8, maxit=500, check_every=2, **opts)
            torch.cuda.synchronize()
            assert all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in infos), infos
            out.append((Xd[0].cpu().numpy(), infos[0]))
        assert np.array_equal(out[0][0], out[1][0])
        for key in ("iters", "restarts", "matvecs", "matvecs_fp64", "relres_true", "relres_inner"):
            assert out[0][1][key] == out[1][1][key], key
    finally:
        P.hmat_destroy(h)


def test_double_float_many_columns_full_size(oracle_mod):
    """Icosphere level 6 (N = 81,920), 18 columns (a full pass of 16 and a ragged
    one of 2) of the FP64 handle: sampled rows against the oracle's own H-matrix
    for two columns, and three columns bit for bit the one-column product."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(6)
    blob = P.hmat_build(mesh.centroid, mesh.area)
    H = oracle_mod.HMatrix(mesh.centroid, mesh.area)
    nrhs = 18
    X = synth.rhs_normal_columns(mesh.n, nrhs, seed=18)
    rows = np.random.default_rng(8).choice(mesh.n, 300, replace=False)
    h = P.hmat_upload(blob, "fp64")
    try:
        Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
        Yd = torch.empty_like(Xd)
        P.hmat_matvec(h, Xd, Yd, nrhs)
        torch.cuda.synchronize()
        for k in (0, 17):
            ref = H.matvec_rows(X[:, k], rows)
            assert maxrel(Yd[k].cpu().numpy()[rows], ref) <= 1e-13, k
        for k in (0, 15, 17):
            y1 = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
            P.hmat_matvec(h, Xd[k].contiguous(), y1, 1)
            torch.cuda.synchronize()
            assert torch.equal(Yd[k], y1), k
    finally:
        P.hmat_destroy(h)


@pytest.mark.parametrize("form,opts", [("fp64", {}), ("bf16", {"inner_tol": 1e-2})])
def test_batch_several_rhs(hcache, form, opts):
    """A block-diagonal batch of three problems with three right-hand sides each:
    nine systems whose true residuals are taken as their runs stop, over the
    listed columns, with the work items of the other problems of a column
    skipped.  Every system converges against its own problem's oracle
    H-matrix."""
    torch = need_gpu()
    P = lib()
    meshes = [synth.icosphere(3), synth.two_spheres(3), synth.cube_sphere(12)]
    Hs = [hcache(m) for m in meshes]
    nrhs = 3
    h = P.hmat_upload_batch([oracle_blob(H) for H in Hs], form)
    try:
        off = P.hmat_problems(h)
        n = off[-1]
        B = synth.rhs_normal_columns(n, nrhs, seed=33)
        X = np.zeros((n, nrhs), order="F")
        infos = P.hmat_bicgstab_multi(h, B, X, nrhs, tol=1e-8, maxit=800, check_every=2, **opts)
        cnt = len(off) - 1
        assert len(infos) == cnt * nrhs
        assert all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in infos), infos
        for p, H in enumerate(Hs):
            sl = slice(off[p], off[p + 1])
            for k in range(nrhs):
                assert _true_rel(H, B[sl, k], X[sl, k]) <= 1.05e-8, (p, k)
    finally:
        P.hmat_destroy(h)


@pytest.mark.parametrize("form,opts", [("fp64", {}), ("bf16", {"inner_tol": 1e-2})])
def test_multi_rhs_read_interval_same_bits(hcache, form, opts):
    """How often the host reads the systems' state (check_every) and whether the
    iterations replay as a graph only move the time at which a stopped system's
    true residual is taken and its next run starts, never its arithmetic: the
    same bits, counts and residuals for every system."""
    torch = need_gpu()
    P = lib()
    mesh = synth.icosphere(3)
    H = hcache(mesh)
    nrhs = 6
    B = synth.rhs_normal_columns(mesh.n, nrhs, seed=21)
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    h = P.hmat_upload(oracle_blob(H), form)
    try:
        runs = []
        for ce, ug in ((2, 1), (1, 0), (5, 1)):
            Xd = torch.zeros_like(Bd)
            infos = P.hmat_bicgstab_multi(h, Bd, Xd, nrhs, tol=1e-8, maxit=500, check_every=ce, use_graph=ug, **opts)
            torch.cuda.synchronize()
            assert all(i["status"] == 0 for i in infos), infos
            runs.append((Xd.cpu().numpy(), infos))
        for X, infos in runs[1:]:
            assert np.array_equal(X, runs[0][0])
            for a, b in zip(infos, runs[0][1]):
                for key in ("iters", "restarts", "matvecs", "matvecs_fp64", "relres_true", "relres_inner"):
                    assert a[key] == b[key], key
    finally:
        P.hmat_destroy(h)
