#!/usr/bin/env python
"""Benchmark of the GB300 H-matrix BiCG-STAB solve (arXiv:1911.00093 hot path).

Workload: unit-sphere icosphere level 6 (N = 81,920 flat panels, centroid
collocation), kernel a_ij = area_j / (4 pi |c_i - c_j|), a_ii = sqrt(area_i/pi)/2,
bisection cluster tree with leaf 32, eta = 2, ACA eps = 1e-4, right-hand side
phi_i = 1 + 0.5 z_i, stop at a true relative residual of 1e-8 (FP64 H-matrix).

One step = one whole solve (Algorithm 1 with its two H-matrix products per
iteration, the FP64 vector work and the FP64 true-residual acceptance) in the
headline mixed form; the FP64 solve and every other form are measured beside
it.  `value` is solves per second over all ranks (independent replicas under
torchrun).  Prints one JSON line on rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BiCG-STAB time to rel. residual 1e-8 & H-matvec HBM GB/s: mixed vs FP64"
UNIT = "solves/s"
# form -> (upload precision, Method 3's c, solver options); the m* forms are the
# paper's own variants (Section 3, Table 1), fp64_dfma is its Method 1-Double
FORMS = {"fp64": ("fp64", None, {}), "fp64_dfma": ("fp64_dfma", None, {}),
         "fp32": ("fp32", None, {"inner_tol": 1e-4}), "bf16": ("bf16", None, {"inner_tol": 1e-2}),
         "m1_single": ("m1_single", None, {"inner_tol": 1e-4}), "m1_mixed": ("m1_mixed", None, {"inner_tol": 1e-4}),
         "m2_double": ("m2_double", None, {}), "m2_single": ("m2_single", None, {"inner_tol": 1e-4}),
         "m2_mixed": ("m2_mixed", None, {"inner_tol": 1e-4}), "m3_c-1": ("m3", -1, {"inner_tol": 1e-4}),
         "m3_c2": ("m3", 2, {"inner_tol": 1e-4}), "m3_c3": ("m3", 3, {"inner_tol": 1e-4}),
         "m3trunc_c3": ("m3_trunc", 3, {"inner_tol": 1e-4}), "m3dense_c0": ("m3_dense", 0, {"inner_tol": 1e-4}),
         "m3dense_c1": ("m3_dense", 1, {"inner_tol": 1e-4})}
FORM_OPTS = {k: v[2] for k, v in FORMS.items()}
DEFAULT_FORMS = ("fp64,fp64_dfma,fp32,bf16,m1_single,m1_mixed,m2_double,m2_single,m2_mixed,m3_c-1,m3_c3,m3trunc_c3,"
                 "m3dense_c1")
CHECK_EVERY = 4  # iterations per graph replay between host reads of the stop flag
# The 64-system solves take each stopped system's true residual at the next host
# read, so they read more often (level 6, 64 BF16 solves: 199.6 ms at 2, 203.7 at
# 1, 207.5 at 4, 226.1 at 8; FP32 290.1 / 284.7 / 293.8 / 327.0)
MULTI_CHECK_EVERY = 2
PART_BYTES = {"fp64": 8, "fp64_dfma": 8, "fp32": 4, "bf16": 4}  # partial sums (8 for the paper's variants)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons; summary()
    keeps the samples whose timestamps fall inside the marked timed window."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.window = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(1.0)  # let the sampler start before the timed region
        except Exception:
            self.proc = None
        return self

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import datetime
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons, total = [], None, set(), 0
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            total += 1
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, cmax = float(f[2]), float(f[3])
            except ValueError:
                continue
            if self.window and not (self.window[0] - 0.05 <= ts <= self.window[1] + 0.05):
                continue
            sm.append(clk)
            smax = cmax
            for k, name in enumerate(names):
                if f[6 + k].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "samples_total": total}


class _nvtx:
    """An NVTX push/pop range (a no-op where NVTX is unavailable): the committed
    ncu summaries select the launches of one part of the bench by its range."""

    def __init__(self, torch, name):
        self.nv, self.name, self.on = torch.cuda.nvtx, name, False

    def __enter__(self):
        try:
            self.nv.range_push(self.name)
            self.on = True
        except Exception:
            pass
        return self

    def __exit__(self, *a):
        if self.on:
            self.nv.range_pop()


def _dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _profiled_traffic(kernel, level):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when
    there is none for this workload or a product source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"traffic_icosphere_L{level}.json")
    try:
        rec = json.load(open(path))
        for src, digest in rec["sources"].items():
            if hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest() != digest:
                return None
    except (OSError, ValueError, KeyError):
        return None
    return rec.get("dram_bytes_per_launch", {}).get(kernel)


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def _roofline(table, form, level, peak, peak_kind):
    """Roofline object of a form's dominant product kernel: algorithmic bytes per
    launch (stored entries at their element size plus the partial sums written, or
    plus y written) over the launch's mean CUDA-event time; traffic = ncu DRAM bytes
    per launch from the committed capture of the same source."""
    head = table[form]
    dom = "phase2" if head["kernel_ms"]["phase2"] >= head["kernel_ms"]["phase1"] else "phase1"
    achieved = head[dom + "_gbs"]
    kname = f"k_phase2g<{form}>" if dom == "phase2" else f"k_phase1<{form}>"
    return {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
            "algorithmic_bytes": head[dom + "_bytes"], "launch_us": head["kernel_ms"][dom] * 1e3,
            "traffic": _profiled_traffic(kname, level)}


def max_over_ranks(value, dist, device="cuda"):
    """The largest of every rank's value (the job's time is its slowest replica's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, seconds):
    """Whole-job throughput: every replica solves `steps` systems in at most `seconds`."""
    return world * steps / seconds


def _workload(level):
    import synth
    mesh = synth.icosphere(level)
    return mesh, synth.rhs_one_plus_half_z(mesh)


def _config(mesh, args, extra=None):
    c = {"workload": f"icosphere_L{args.level}_N{mesh.n}_leaf32_eta2_aca1e-4_phi=1+z/2_tol1e-8",
         "n": mesh.n, "headline_form": args.form, "parallelism": f"replicas{max(1, args.gpus)}",
         "l2": "inputs larger than L2 (H-matrix panels >> 129 MB; no flush)"}
    if extra:
        c.update(extra)
    return c


def run_reference(args):
    """The oracle (plain FP64 C, OpenMP over the blocks of each product) solving the
    same workload on the host cores, one whole solve per step."""
    world, rank, _ = _dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.build_oracle()
    mesh, b = _workload(args.level)
    variant = oracle.M1_DOUBLE  # the plain FP64 oracle
    H = oracle.HMatrix(mesh.centroid, mesh.area)
    threads = oracle.get_threads()
    # warm-up: a few products (a CPU program needs no more)
    for _ in range(max(0, args.warmup)):
        H.matvec(b, variant)
    times, infos = [], []
    for k in range(args.steps):
        t0 = time.perf_counter()
        x, info = H.bicgstab(b, variant=variant, tol=1e-8)
        times.append(time.perf_counter() - t0)
        infos.append(info)
    t = statistics.mean(times)
    line = {"metric": METRIC, "value": 1.0 / t, "unit": UNIT, "n_gpus": args.gpus, "steps": len(times),
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(mesh, args, {"oracle_variant": "fp64"}),
            "cpu_baseline": {"value": 1.0 / t, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{len(times)} whole oracle solves of the benchmark workload on {threads} "
                                       f"threads (iters {infos[-1]['iters']}, true relres {infos[-1]['relres']:.2e})"},
            "e2e": {"value": 1.0 / t, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline(mesh, b):
    """The oracle as it stands on this host's cores: one whole FP64 solve of the same
    workload on every core (the reported value), then one on a single thread."""
    import oracle
    oracle.build_oracle()
    H = oracle.HMatrix(mesh.centroid, mesh.area)
    threads = oracle.get_threads()
    t0 = time.perf_counter()
    x, info = H.bicgstab(b, variant=oracle.M1_DOUBLE, tol=1e-8)
    t = time.perf_counter() - t0
    try:
        oracle.set_threads(1)
        t1 = time.perf_counter()
        x1, info1 = H.bicgstab(b, variant=oracle.M1_DOUBLE, tol=1e-8)
        t1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(threads)
    return {"value": 1.0 / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one whole FP64 oracle solve of the benchmark workload on {threads} threads "
                      f"(iters {info['iters']}, true relres {info['relres']:.2e}, {t:.2f} s)",
            "single_thread": {"value": 1.0 / t1, "unit": UNIT, "cores": 1,
                              "sample": f"the same solve on one thread ({t1:.2f} s, the same bits)"}}


def _cuda_ms(torch, fn, reps):
    """Mean milliseconds of fn() over reps calls, CUDA events on the current stream."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = [fn() for _ in range(reps)]
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def run_workload(args):
    """The other configurations of the study, one JSON line each (not the headline):
    icosphere_L4 (FP64 correctness size), two_spheres_L7 (BF16 + FP64 refinement,
    N = 655,360), multirhs64 (64 right-hand sides at level 6, tensor-core products),
    batch48 (48 uneven cube / sphere problems in one block-diagonal handle);
    build_icosphere_L6 / build_batch48 (H-matrix construction, host vs device);
    matvec_protocol (Section 4.1.3's sets of repeated products, GPU and oracle)."""
    import torch
    import synth
    import paper_1911_00093_gb300 as P
    P.load()
    torch.cuda.set_device(0)
    out = {"metric": METRIC, "unit": "ms per solve", "higher_is_better": False, "data": "synthetic",
           "config": {"workload": args.workload}}
    if args.workload in ("icosphere_L4", "two_spheres_L7"):
        mesh = synth.icosphere(4) if args.workload == "icosphere_L4" else synth.two_spheres(7)
        b_np = synth.rhs_constant(mesh) if args.workload == "icosphere_L4" else synth.rhs_two_spheres(mesh)
        blob = P.hmat_build(mesh.centroid, mesh.area)
        b = torch.from_numpy(b_np).cuda()
        x = torch.zeros_like(b)
        forms = {"fp64": {}, "bf16": {"inner_tol": 1e-2}}
        out["config"]["n"] = mesh.n
        for f, opts in forms.items():
            h = P.hmat_upload(blob, f)
            def solve():
                x.zero_()
                return P.hmat_bicgstab(h, b, x, tol=1e-8, maxit=3000, check_every=CHECK_EVERY, **opts)
            solve()
            ms, infos = _cuda_ms(torch, solve, 3)
            kt = P.hmat_time_matvec(h, 10)
            info = P.hmat_info(h)
            out[f] = {"solve_ms": ms, "iters": infos[-1]["iters"], "restarts": infos[-1]["restarts"],
                      "relres_true": infos[-1]["relres_true"], "matvec_ms": kt[4],
                      "matvec_gbs": info["stored_bytes"] / (kt[4] * 1e-3) / 1e9}
            P.hmat_destroy(h)
        out["value"] = out["bf16"]["solve_ms"]
        out["speedup_bf16_vs_fp64"] = out["fp64"]["solve_ms"] / out["bf16"]["solve_ms"]
    elif args.workload == "multirhs64":
        mesh = synth.icosphere(6)
        nrhs = 64
        blob = P.hmat_build(mesh.centroid, mesh.area)
        B = torch.from_numpy(np.ascontiguousarray(synth.rhs_normal_columns(mesh.n, nrhs).T)).cuda()
        X = torch.zeros_like(B)
        res = {}
        for form, itol in (("bf16", 1e-2), ("fp32", 1e-4), ("fp64", 0.0)):
            h = P.hmat_upload(blob, form)
            def multi():
                X.zero_()
                return P.hmat_bicgstab_multi(h, B, X, nrhs, tol=1e-8, maxit=3000, inner_tol=itol,
                                             check_every=MULTI_CHECK_EVERY)
            multi()
            with _nvtx(torch, "solves64" if form == "bf16" else "solves64_" + form):
                ms, infos = _cuda_ms(torch, multi, 2)
            x1 = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
            def single():
                x1.zero_()
                return P.hmat_bicgstab(h, B[0].contiguous(), x1, tol=1e-8, maxit=3000, inner_tol=itol,
                                       check_every=CHECK_EVERY)
            single()
            ms1, info1 = _cuda_ms(torch, single, 3)
            Y = torch.empty_like(B)
            with _nvtx(torch, "product64" if form == "bf16" else "product64_" + form):
                mv_ms, _ = _cuda_ms(torch, lambda: P.hmat_matvec(h, B, Y, nrhs), 10)
            assert all(i["status"] == 0 for i in infos[-1])
            res[form] = {"solves_ms": ms, "iters_min_max": [min(i["iters"] for i in infos[-1]),
                                                            max(i["iters"] for i in infos[-1])],
                         "true_residual_products": sum(i["matvecs_fp64"] for i in infos[-1]),
                         "single_rhs_solve_ms": ms1, "single_rhs_iters": info1[-1]["iters"],
                         ("double_float_product_ms_64_columns" if form == "fp64"
                          else "tensor_core_product_ms_64_columns"): mv_ms,
                         "single_column_product_ms": P.hmat_time_matvec(h, 10)[4]}
            if form == "bf16":  # the FP64 copy of the true residuals, 64 columns at once
                with _nvtx(torch, "product64_fp64_copy"):
                    res[form]["fp64_copy_product_ms_64_columns"], _ = _cuda_ms(
                        torch, lambda: P.hmat_matvec(h, B, Y, nrhs, fp64=True), 10)
            P.hmat_destroy(h)
        out.update({"unit": "ms per 64 solves", "value": res["bf16"]["solves_ms"],
                    "config": {"workload": "icosphere_L6_64rhs_N(0,1)", "n": mesh.n, "nrhs": nrhs,
                               "form": "bf16 + FP64 refinement (fp32 beside it)",
                               "check_every": MULTI_CHECK_EVERY},
                    "iters_min_max": res["bf16"]["iters_min_max"],
                    "single_rhs_solve_ms": res["bf16"]["single_rhs_solve_ms"],
                    "single_rhs_iters": res["bf16"]["single_rhs_iters"],
                    "tensor_core_product_ms_64_columns": res["bf16"]["tensor_core_product_ms_64_columns"],
                    "single_column_product_ms": res["bf16"]["single_column_product_ms"],
                    "fp64_copy_product_ms_64_columns": res["bf16"]["fp64_copy_product_ms_64_columns"],
                    "true_residual_products": res["bf16"]["true_residual_products"],
                    "fp32": res["fp32"], "fp64": res["fp64"],
                    "speedup_bf16_vs_fp64": res["fp64"]["solves_ms"] / res["bf16"]["solves_ms"]})
    elif args.workload == "batch48":
        specs = synth.uneven_batch_specs(48)
        meshes = [synth.mesh_from_spec(sp) for sp in specs]
        blobs = [P.hmat_build(m.centroid, m.area) for m in meshes]
        b = torch.from_numpy(np.concatenate([synth.rhs_constant(m) for m in meshes])).cuda()
        x = torch.zeros_like(b)
        out["config"].update({"problems": len(meshes), "n_total": int(b.numel()),
                              "n_min_max": [min(m.n for m in meshes), max(m.n for m in meshes)]})
        out["unit"] = "ms per batch solve"
        # refinement tolerances measured best on this batch (FP32 1e-3..1e-6, BF16 1e-2 and 3e-3)
        for f, opts in (("fp64", {}), ("fp32", {"inner_tol": 1e-6}), ("bf16", {"inner_tol": 3e-3})):
            h = P.hmat_upload_batch(blobs, f)
            rep = P.hmat_autotune(h, 10)
            def solve():
                x.zero_()
                return P.hmat_bicgstab_multi(h, b, x, 1, tol=1e-8, maxit=3000, check_every=CHECK_EVERY, **opts)
            solve()
            ms, infos = _cuda_ms(torch, solve, 3)
            assert all(i["status"] == 0 for i in infos[-1])
            out[f] = {"batch_solve_ms": ms, "iters_max": max(i["iters"] for i in infos[-1]),
                      "matvec_ms": P.hmat_time_matvec(h, 10)[4], "projection_tuning": rep}
            P.hmat_destroy(h)
        out["value"] = out["fp32"]["batch_solve_ms"]
        out["speedup_fp32_vs_fp64"] = out["fp64"]["batch_solve_ms"] / out["fp32"]["batch_solve_ms"]
        out["speedup_bf16_vs_fp64"] = out["fp64"]["batch_solve_ms"] / out["bf16"]["batch_solve_ms"]
    elif args.workload == "matvec_protocol":
        # Section 4.1.3's protocol: sets of repeated products of one source vector,
        # the median set reported; the GPU forms (1000 products per set) and the FP64
        # oracle on one thread and on every host core (fewer products per set at
        # level 6, where one oracle product takes tenths of a second)
        import oracle
        oracle.build_oracle()
        threads = oracle.get_threads()
        out.update({"metric": "H-matvec time, sets of repeated products (Section 4.1.3)", "unit": "ms per product",
                    "higher_is_better": False})
        levels = {}
        for level, reps_cpu1, reps_cpun in ((4, 1000, 1000), (6, 20, 100)):
            mesh = synth.icosphere(level)
            xn = synth.rhs_one_plus_half_z(mesh)
            blob = P.hmat_build(mesh.centroid, mesh.area)
            rec = {"n": mesh.n, "sets": 10}
            xd = torch.from_numpy(xn).cuda()
            yd = torch.empty_like(xd)
            for f in ("fp64", "fp32", "bf16", "fp64_dfma"):
                h = P.hmat_upload(blob, f)
                for _ in range(20):
                    P.hmat_matvec(h, xd, yd)
                sets = [_cuda_ms(torch, lambda: P.hmat_matvec(h, xd, yd), 1000)[0] for _ in range(10)]
                info = P.hmat_info(h)
                med = statistics.median(sets)
                rec["gpu_" + f] = {"ms": med, "products_per_set": 1000, "gbs": info["stored_bytes"] / (med * 1e-3) / 1e9}
                P.hmat_destroy(h)
            H = oracle.HMatrix(mesh.centroid, mesh.area)
            for nt, reps in ((1, reps_cpu1), (threads, reps_cpun)):
                oracle.set_threads(nt)
                H.matvec(xn)
                sets = []
                for _ in range(10):
                    t0 = time.perf_counter()
                    for _ in range(reps):
                        H.matvec(xn)
                    sets.append((time.perf_counter() - t0) * 1e3 / reps)
                rec[f"oracle_{nt}_threads"] = {"ms": statistics.median(sets), "products_per_set": reps}
            oracle.set_threads(threads)
            levels[f"icosphere_L{level}"] = rec
        out.update({"value": levels["icosphere_L6"]["gpu_bf16"]["ms"], "levels": levels, "host_threads": threads,
                    "config": {"workload": "matvec_protocol icosphere L4 and L6, phi = 1 + z/2"}})
    elif args.workload in ("build_icosphere_L6", "build_batch48"):
        # H-matrix construction: the host builder (OpenMP on the host cores) against
        # the device ACA builder; both produce the same blob (checked here)
        if args.workload == "build_icosphere_L6":
            meshes = [synth.icosphere(6)]
        else:
            meshes = [synth.mesh_from_spec(sp) for sp in synth.uneven_batch_specs(48)]
        import ctypes as C
        L = P.load()
        # the library calls alone (the blob stays in the library's buffer): best of a few
        def call(fn, m, info=None):
            buf, size = C.c_void_p(), C.c_size_t()
            c = np.ascontiguousarray(m.centroid)
            a = np.ascontiguousarray(m.area)
            args = [m.n, c.ctypes.data, a.ctypes.data, 32, 2.0, 1e-4, C.byref(buf), C.byref(size)]
            if info is not None:
                args.append(C.byref(info))
            t0 = time.perf_counter()
            st = fn(*args)
            dt = (time.perf_counter() - t0) * 1e3
            assert st == 0, st
            return dt, buf, size.value
        def timed(fn, reps, info=None):
            best = None
            for _ in range(reps):
                tot, bufs = 0.0, []
                for m in meshes:
                    dt, buf, size = call(fn, m, info)
                    tot += dt
                    bufs.append((buf, size))
                for buf, _ in bufs:
                    L.hmat_blob_free(buf)
                best = tot if best is None or tot < best else best
            return best
        L.hmat_build_device.restype = C.c_int  # (signature set by load())
        timed(L.hmat_build_device, 1, P.BuildDeviceInfo())  # context and allocator warm-up
        dinfo = P.BuildDeviceInfo()
        dev_ms = timed(L.hmat_build_device, 3, dinfo)
        host_ms = timed(L.hmat_build, 2)
        same = all(np.array_equal(P.hmat_build_device(m.centroid, m.area), P.hmat_build(m.centroid, m.area))
                   for m in meshes[:4])
        out.update({"metric": "H-matrix construction (cluster tree, partition, ACA, dense blocks)",
                    "unit": "ms", "value": dev_ms, "host_ms": host_ms, "speedup_device_vs_host": host_ms / dev_ms,
                    "host_threads": os.cpu_count(), "identical_blobs_checked": same,
                    "last_device_build": {k: getattr(dinfo, k) for k, _ in P.BuildDeviceInfo._fields_}})
        out["config"].update({"problems": len(meshes), "n_total": int(sum(m.n for m in meshes))})
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=6)
    ap.add_argument("--form", default="bf16", choices=list(FORM_OPTS))
    ap.add_argument("--forms", default=DEFAULT_FORMS, help="forms measured beside the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--matvec-iters", type=int, default=50)
    ap.add_argument("--use-graph", type=int, default=2, choices=[0, 1, 2],
                    help="graph mode of the solves: 2 one conditional-loop graph per run (default); 1 a graph "
                         "per batch of iterations, whose kernels ncu profiles one by one; 0 stream launches")
    ap.add_argument("--workload", default="icosphere_L6",
                    choices=["icosphere_L6", "icosphere_L4", "two_spheres_L7", "multirhs64", "batch48",
                             "build_icosphere_L6", "build_batch48", "matvec_protocol"],
                    help="icosphere_L6 is the benchmark; the others print one informative line each")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "icosphere_L6":
        return run_workload(args)

    import torch
    world, rank, local = _dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1911_00093_gb300 as P
    P.load()

    mesh, b_np = _workload(args.level)
    t0 = time.perf_counter()
    blob = P.hmat_build(mesh.centroid, mesh.area)
    build_s = time.perf_counter() - t0
    stats = P.hmat_blob_stats(blob)
    forms = [f for f in args.forms.split(",") if f]
    if args.form not in forms:
        forms.append(args.form)
    handles, tune = {}, {}
    stream = torch.cuda.current_stream()
    for f in forms:
        handles[f] = P.hmat_upload(blob, FORMS[f][0], FORMS[f][1])
        tune[f] = P.hmat_autotune(handles[f], 10, stream)  # the projection's plan, by measurement
    b = torch.from_numpy(b_np).cuda()
    x = torch.zeros_like(b)

    def solve(form):
        x.zero_()
        return P.hmat_bicgstab(handles[form], b, x, tol=1e-8, maxit=2000, stream=stream, check_every=CHECK_EVERY,
                               use_graph=args.use_graph, **FORM_OPTS[form])

    def timed(form, steps, warmup, clk=None, tag=None):
        for _ in range(warmup):
            info = solve(form)
            if info["status"] != 0:
                raise RuntimeError(f"{form} solve failed: {info}")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.time()
        with _nvtx(torch, tag or f"solves_{form}"):
            ev0.record(stream)
            infos = [solve(form) for _ in range(steps)]
            ev1.record(stream)
        torch.cuda.synchronize()
        if clk is not None:
            clk.mark(w0, time.time())
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
        return ms, infos

    # ---- headline: the mixed-form solve, clocks sampled during the timed region ----
    with ClockSampler(local) as clk:
        ms, infos = timed(args.form, args.steps, max(3, args.warmup), clk, tag="headline")
    clocks = clk.summary()
    if any(i["status"] != 0 or i["relres_true"] > 1e-8 for i in infos):
        raise RuntimeError(f"headline solve did not reach the tolerance: {infos[-1]}")
    ms_per_step = ms / args.steps
    value = job_rate(world, args.steps, ms / 1e3)
    launches = int(sum(i["launches"] for i in infos))

    # ---- every form: solve time and product throughput ----
    hbm_peak, peak_kind = _peaks()
    table = {}
    for f in forms:
        fms, finf = timed(f, max(3, args.steps // 2), 2)
        info = P.hmat_info(handles[f])
        with _nvtx(torch, "products"):
            kt = P.hmat_time_matvec(handles[f], args.matvec_iters, False, stream)
        # algorithmic bytes: stored entries at their element size, plus the
        # projections T written (projection) and y written once per segment (expansion)
        p1_bytes = info["phase1_bytes"] + info["partials"] * PART_BYTES.get(f, 8)
        p2_bytes = info["phase2_bytes"] + 8 * info["n"] * info["segments"]
        table[f] = {"solve_ms": fms / max(3, args.steps // 2), "iters": finf[-1]["iters"],
                    "restarts": finf[-1]["restarts"], "relres_true": finf[-1]["relres_true"],
                    "matvec_ms": kt[4], "kernel_ms": {"prep": kt[0], "phase1": kt[1], "reduce": kt[2], "phase2": kt[3]},
                    "matvec_gbs": info["stored_bytes"] / (kt[4] * 1e-3) / 1e9,
                    "phase1_gbs": p1_bytes / (kt[1] * 1e-3) / 1e9, "phase2_gbs": p2_bytes / (kt[3] * 1e-3) / 1e9,
                    "phase1_bytes": p1_bytes, "phase2_bytes": p2_bytes,
                    "stored_bytes": info["stored_bytes"], "panel_bytes": info["panel_bytes"],
                    "segments": info["segments"]}
    roofline = _roofline(table, args.form, args.level, hbm_peak, peak_kind)
    roofline_fp64 = _roofline(table, "fp64", args.level, hbm_peak, peak_kind) if "fp64" in table else None

    # ---- end to end through the C ABI with pinned host buffers ----
    bh = torch.from_numpy(b_np.copy()).pin_memory()
    xh = torch.zeros(mesh.n, dtype=torch.float64).pin_memory()
    P.hmat_bicgstab(handles[args.form], bh, xh, tol=1e-8, maxit=2000, check_every=CHECK_EVERY, **FORM_OPTS[args.form])
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_steps = args.steps
    for _ in range(e2e_steps):
        xh.zero_()
        P.hmat_bicgstab(handles[args.form], bh, xh, tol=1e-8, maxit=2000, check_every=CHECK_EVERY, **FORM_OPTS[args.form])
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = {"value": job_rate(world, e2e_steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 16 * mesh.n,
           "d2h_bytes_per_step": 8 * mesh.n}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mesh, b_np)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"bf16": "bf16+f64", "fp64": "f64", "fp64_dfma": "f64", "m2_double": "f64"}.get(args.form, "f32+f64"),
                "data": "synthetic",
                "config": _config(mesh, args, {"blob_stats": stats, "host_build_s": round(build_s, 3),
                                               "solve_graph_mode": args.use_graph}),
                "fp64_solve_ms": table.get("fp64", {}).get("solve_ms"),
                "fp32_solve_ms": table.get("fp32", {}).get("solve_ms"),
                "fp64_dfma_solve_ms": table.get("fp64_dfma", {}).get("solve_ms"),
                "speedup_vs_fp64_solve": (table["fp64"]["solve_ms"] / ms_per_step) if "fp64" in table else None,
                "forms": table, "roofline": roofline, "roofline_fp64": roofline_fp64, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches, "projection_tuning": tune.get(args.form),
                "solve_info": {k: infos[-1][k] for k in ("iters", "restarts", "matvecs", "matvecs_fp64", "relres_true")}}
        print(json.dumps(line))
    for h in handles.values():
        P.hmat_destroy(h)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
