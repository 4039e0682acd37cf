"""Benchmark of the GCA-H^2 hot path on one B300 (or N replicas).

Workload: the 20480-triangle unit sphere (icosahedron refined five times)
and the same sphere radially perturbed by 0.1 sin(3 theta) cos(2 phi);
leaf size 64, eta = 2, 4 x 4 Gauss points per box face (k = 96), ACA
tolerance 1e-8, Sauter-Schwab order 5; 16 right-hand sides N(0, 1), seed 0.

One step = the whole hot path on both meshes: gca_build_batch (boxes, box
quadrature, Green matrices + ACA per level, nested bases, coupling and
near-field entries, panel copies in three precisions) followed by the
batched H^2 products y_i = G_i x_i (both meshes in one persistent launch)
in float64, float32 and bfloat16 and the transposed product in float32.  Inputs are resident in HBM when the timed region starts; the
stored matrices (>= 480 MB per mesh in float32) exceed the 126 MB L2, so
no flush is needed between products.

The headline `value` is the algorithmic HBM throughput of the float32
product (bytes of V, E, S, N once plus x read and y written, divided by the
product's device time).  `build_s` is the device time of building both
meshes.  Under torchrun every rank runs the same workload on its own GPU
(weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --profile f32|f64|bf16|build [--steps K] [--warmup W]
"""

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = ("GCA-H² build s & matvec GB/s (frac HBM peak), FP32/BF16 vs FP64 at stated err")
MESHES = ("sphere20480", "perturbed20480")
PARAMS = dict(leaf_size=64, eta=2.0, box_gauss_m=4, aca_tol=1e-8, sauter_q=5)
NRHS = 16
FLOPS_PER_EVAL = 11  # 3 differences, 5 for |d|^2, 1 rsqrt, 2 multiply-accumulate
# float32 operations (an FMA counted as 2) of one float-pair evaluation of the
# coupling entries: 50 additions, multiplications and rsqrt plus 12 FMAs
FLOPS_PER_SPLIT_EVAL = 74


def config(extra=None):
    c = {"workload": "sphere20480+perturbed20480 (2 meshes x 20480 triangles)",
         "leaf_size": 64, "eta": 2.0, "box_gauss_m": 4, "aca_tol": 1e-8, "sauter_q": 5,
         "nrhs": NRHS, "l2": "no flush: stored matrices exceed the 126 MB L2",
         "step": "gca_build_batch (2 meshes) + h2_matvec_batch f64/f32/bf16 + h2_matvec_transpose_batch f32"}
    if extra:
        c.update(extra)
    return c


def product_bytes(st, prec, n, R):
    sm = {"f64": 8, "f32": 4, "bf16": 2}[prec]
    sv = 8 if prec == "f64" else 4
    return (sm * (st["v_entries"] + st["e_entries"] + st["s_entries"])
            + sv * st["n_entries"] + 2 * sv * n * R)


# floating-point operations of one evaluation of g and dg/dn at a (triangle
# point, box point) pair of a Green matrix: difference 3, |d|^2 5, rsqrt 1,
# 1/|d|^3 2, <n, d> 5, two weighted accumulations 4
FLOPS_PER_GREEN_EVAL = 20


def green_aca_flops(tree, rank, k):
    """FP64 work of the Green-matrix + ACA phase, per cluster with a basis:
    7 k rows evaluations of the Green matrix (rows = |tau-hat| at leaves,
    r_1 + r_2 above) and, after pivot t, the rank-one update of the residual
    over the rows and columns not yet eliminated, 2 (rows - t - 1)
    (2k - t - 1) flops, plus the update of the interpolation matrix V^ on
    the same rows, 2 (rows - t - 1) t flops (V^ = U L^-1 kept current)."""
    c0, c1 = tree["child0"], tree["child1"]
    total = 0
    for c in range(1, len(c0)):
        r = int(rank[c])
        if r == 0:
            continue
        rows = int(tree["end"][c] - tree["begin"][c]) if c0[c] < 0 else int(rank[c0[c]] + rank[c1[c]])
        t = np.arange(r)
        act = rows - t - 1
        total += FLOPS_PER_GREEN_EVAL * 7 * k * rows + int(np.sum(2 * act * (2 * k - t - 1) + 2 * act * t))
    return int(total)


def build_evals(st, q):
    # coupling blocks come in mirrored pairs (S_{sigma tau} = S_{tau sigma}^T):
    # every distinct entry is evaluated once
    regular = 49 * (st["s_entries"] // 2 + st["n_singular"][0])
    singular = q ** 3 * (2 * st["n_singular"][1] + 5 * st["n_singular"][2]
                         + 6 * st["n_singular"][3])
    return {"couple_entries": 49 * (st["s_entries"] // 2), "near_entries": 49 * st["n_singular"][0],
            "singular": singular, "total": regular + singular}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the kernel on the 20480-triangle sphere alone, with the
# sha256 of the kernel's source file at capture time: reported only while the
# source is unchanged, scaled to the timed launch by its algorithmic bytes.
TRAFFIC = {
    "couple_entries": ("paper_1810_08429_b300/csrc/build.cu",
                       "923b1a936e03ad55214e453c632ecbec573480ead4ab6c8f2d834eff239e2297", 582.87e6),
    # the nine level launches of one mesh's build move 133.45 MB in all; a
    # batch step of the two meshes runs their jobs in 11 common launches:
    # 2 x 133.45 MB / 11 per launch
    "green_aca": ("paper_1810_08429_b300/csrc/build.cu",
                  "923b1a936e03ad55214e453c632ecbec573480ead4ab6c8f2d834eff239e2297", 2 * 133.454e6 / 11),
    "near_entries": ("paper_1810_08429_b300/csrc/build.cu",
                     "923b1a936e03ad55214e453c632ecbec573480ead4ab6c8f2d834eff239e2297", 27.44e6),
    "mv_persistent.f32": ("paper_1810_08429_b300/csrc/matvec.cu",
                          "25516c3710cefbe2a445b57e64cca9b76d169bc949d6a3f85171933ff6d8c049", 476.22e6),
    "mv_persistent.bf16": ("paper_1810_08429_b300/csrc/matvec.cu",
                           "25516c3710cefbe2a445b57e64cca9b76d169bc949d6a3f85171933ff6d8c049", 269.98e6),
}


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks of the default
    process group (the values themselves when there is none)."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_gbs(bytes_per_rank, ms_max, world):
    """Whole-job throughput: every rank's bytes over the slowest rank's time."""
    return world * bytes_per_rank / (ms_max * 1e-3) / 1e9


def captured_traffic(name):
    import hashlib
    if name not in TRAFFIC:
        return None
    path, sha, byt = TRAFFIC[name]
    with open(os.path.join(ROOT, path), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != sha:
            return None
    return byt


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        env = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS")
        return int(env) if env and env.isdigit() else (os.cpu_count() or 1)


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def kernel_evals(tree, rank, k, n_entries, n_singular, s_entries, q):
    """Kernel evaluations of a GCA-H^2 construction, the build's unit of work:
    7 k per row of every Green matrix (g and dg/dn share one distance; rows =
    |tau-hat| at leaves, r_1 + r_2 above, for every cluster with a basis),
    49 per coupling entry and per disjoint near entry, and the Sauter-Schwab
    points of every touching entry (q^3 per region: the integral over the
    radial variable of each Sauter-Schwab region is exact, 1/3; 2, 5, 6
    regions for a common vertex, a common edge, identical triangles)."""
    c0, c1 = tree["child0"], tree["child1"]
    green = 0
    for c in range(1, len(c0)):
        if rank[c] == 0:
            continue
        rows = int(tree["end"][c] - tree["begin"][c]) if c0[c] < 0 else int(rank[c0[c]] + rank[c1[c]])
        green += 7 * k * rows
    regular = 49 * (int(s_entries) + int(n_entries - sum(n_singular[1:])))
    singular = q ** 3 * (2 * n_singular[1] + 5 * n_singular[2] + 6 * n_singular[3])
    return int(green + regular + singular)


def oracle_leg(mesh="sphere1280", reps=5):
    """One timing of the oracle on a bounded sample (run in a child process
    whose BLAS thread count the parent sets): its own GCA-H^2 of a smaller
    sphere with the workload's parameters, then float64 products with 16
    RHS.  Returns build and product seconds, bytes and kernel evaluations."""
    from oracle import gca as ogca, h2 as oh2
    from oracle.galerkin import shared_vertices
    from oracle.params import Params as OParams
    v, t = synth.mesh_for_config(mesh)
    p = OParams(**PARAMS)
    x = synth.normal_rhs(len(t), NRHS, seed=0)
    t0 = time.perf_counter()
    H = ogca.build_h2(v, t, p)
    tb = time.perf_counter() - t0
    oh2.matvec(H, x)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oh2.matvec(H, x)
        times.append(time.perf_counter() - t0)
    st = oh2.storage(H)
    byt = 8 * st["total"] + 2 * 8 * len(t) * NRHS
    ii, jj = [], []
    for (tt, ss) in H.near:
        a = H.tree["perm"][H.tree["begin"][tt]:H.tree["end"][tt]]
        b = H.tree["perm"][H.tree["begin"][ss]:H.tree["end"][ss]]
        ii.append(np.repeat(a, len(b)))
        jj.append(np.tile(b, len(a)))
    sv = shared_vertices(np.asarray(t), np.concatenate(ii), np.concatenate(jj))
    nsing = [int(np.sum(sv == c)) for c in range(4)]
    evals = kernel_evals(H.tree, H.bases.rank, 6 * p.box_gauss_m ** 2, st["N"], nsing, st["S"], p.sauter_q)
    return {"build_s": tb, "matvec_s": statistics.median(times), "bytes": byt, "evals": evals,
            "n": len(t), "mesh": mesh, "threads": blas_threads()}


def oracle_sample():
    """The oracle timed on one thread (BLAS and OpenMP limited to 1 in a child
    process) and on all of the host's cores (a child process with the
    library defaults)."""
    out = {"cores": os.cpu_count() or 1, "cpu_model": cpu_model()}
    for label, limit in (("single_thread", "1"), ("all_cores", None)):
        env = dict(os.environ)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            if limit:
                env[var] = limit
            else:
                env.pop(var, None)
        res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg"], env=env,
                             capture_output=True, text=True, check=True)
        leg = json.loads(res.stdout.strip().splitlines()[-1])
        leg["gbs"] = leg["bytes"] / leg["matvec_s"] / 1e9
        leg["build_evals_per_s"] = leg["evals"] / leg["build_s"]
        out[label] = leg
    out["n"] = out["all_cores"]["n"]
    out["build_kernel_evals"] = out["all_cores"]["evals"]
    return out


def run_reference(args):
    """CPU oracle arm: same metric, unit and config; bounded oracle samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mesh = "sphere1280"
    from oracle import gca as ogca, h2 as oh2
    from oracle.params import Params as OParams
    v, t = synth.mesh_for_config(mesh)
    H = ogca.build_h2(v, t, OParams(**PARAMS))
    st = oh2.storage(H)
    x = synth.normal_rhs(len(t), NRHS, seed=0)
    byt = 8 * st["total"] + 2 * 8 * len(t) * NRHS
    for _ in range(args.warmup):
        oh2.matvec(H, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oh2.matvec(H, x)
    dt = (time.perf_counter() - t0) / args.steps
    value = byt / dt / 1e9
    sample = (f"oracle float64 H2 product, 16 RHS, on its own GCA-H2 of the {len(t)}-triangle "
              f"sphere built with the workload's parameters (build not timed)")
    threads = blas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"sample_mesh": mesh}),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads,
                             "kind": "oracle", "sample": sample, "cpu_model": cpu_model(),
                             "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Small case for kernel captures: the 20480-triangle sphere alone, built
    once (or `steps` times for --profile build), then `steps` products in one
    precision with 16 right-hand sides.  Prints one line; not a bench value."""
    import torch

    import paper_1810_08429_b300 as gca
    prm = gca.Params(**PARAMS)
    if args.profile in ("p1", "p1c"):
        # the nodal basis on the 20480-triangle sphere (flat or curved triangles)
        v, t = synth.mesh_for_config(MESHES[0])
        tree = gca.tree_build_points(v, PARAMS["leaf_size"])
        mids = synth.edge_midpoints_for_config(MESHES[0])
        for _ in range(max(args.steps, 1)):
            if args.profile == "p1":
                h = gca.build_p1(v, t, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
            else:
                h = gca.build_p1_curved(v, t, mids, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
            h.free()
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "n": len(v)}), flush=True)
        return
    if args.profile == "build2":
        # the bench's two meshes as one batch (their cross approximations share
        # the level launches)
        meshes = [synth.mesh_for_config(m) for m in MESHES]
        trees = [gca.tree_build(v, t, PARAMS["leaf_size"]) for v, t in meshes]
        for _ in range(max(args.steps, 1)):
            b = gca.build_batch(meshes, trees, prm)
            b.free()
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "meshes": len(meshes)}), flush=True)
        return
    v, t = synth.mesh_for_config(MESHES[0])
    tree = gca.tree_build(v, t, PARAMS["leaf_size"])
    h = gca.build(v, t, tree, prm)
    if args.profile == "build":
        for _ in range(args.steps):
            h.free()
            h = gca.build(v, t, tree, prm)
    else:
        dt = torch.float64 if args.profile == "f64" else torch.float32
        x = torch.from_numpy(synth.normal_rhs(len(t), NRHS, seed=0)).to("cuda", dt)
        y = torch.empty((NRHS, len(t)), dtype=dt, device="cuda").t()
        for _ in range(args.warmup + args.steps):
            h.matvec(x, args.profile, out=y)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "n": len(t), "status": h.status()}), flush=True)


def time_products(fn, K, W, stream):
    """Median device time (ms) of fn() over K runs after W warm-ups, CUDA
    events on the launching stream."""
    import torch
    for _ in range(W):
        fn()
    ts = []
    for _ in range(K):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def leg_errors(ys, ref):
    """Largest relative 2-norm error per right-hand side against `ref`."""
    return max(float(((y.double() - r).norm(dim=0) / r.norm(dim=0)).max()) for y, r in zip(ys, ref))


def run_legs(gca, batch, meshes, stats, n, args, dev, stream, hbm_peak):
    """Products outside the step: R = 1 and R = 4 on the bench's two meshes
    (float32, bfloat16; where the product streams the blocks with little
    arithmetic per byte), and the 81920-triangle sphere with 64 right-hand
    sides in float64, float32 and bfloat16 (built with the bench parameters).
    Each: median of K products after W warm-ups, algorithmic GB/s, fraction
    of HBM, error against the float64 product of the same right-hand sides."""
    import torch
    K, W = max(args.steps, 3), max(args.warmup, 3)
    legs = {}
    for R in (1, 4):
        x64 = [torch.from_numpy(synth.normal_rhs(len(t), R, seed=R)).to(dev) for _, t in meshes]
        x32 = [x.float() for x in x64]
        ref = batch.matvec(x64, "f64")
        for prec in ("f32", "bf16"):
            outs = [torch.empty((R, len(t)), dtype=torch.float32, device=dev).t() for _, t in meshes]
            ms = time_products(lambda: batch.matvec(x32, prec, outs=outs), K, W, stream)
            byt = sum(product_bytes(s, prec, n, R) for s in stats)
            legs[f"{prec}.R{R}"] = {"GB/s": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm_peak,
                                    "us_both_meshes": ms * 1e3, "err_vs_f64": leg_errors(outs, ref)}
    v, t = synth.mesh_for_config("sphere81920")
    tree = gca.tree_build(v, t, PARAMS["leaf_size"])
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    h = gca.build(v, t, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
    b.record(stream)
    b.synchronize()
    st = h.stats()
    R = 64
    x64 = torch.from_numpy(synth.normal_rhs(len(t), R, seed=0)).to(dev)
    x32 = x64.float()
    y64 = torch.empty((R, len(t)), dtype=torch.float64, device=dev).t()
    cfg3 = {"workload": "sphere81920, leaf 64, eta 2, m 4, tol 1e-8, 64 RHS N(0,1)",
            "build_s": a.elapsed_time(b) * 1e-3}
    for prec in ("f64", "f32", "bf16"):
        xin = x64 if prec == "f64" else x32
        out = y64 if prec == "f64" else torch.empty((R, len(t)), dtype=torch.float32, device=dev).t()
        ms = time_products(lambda: h.matvec(xin, prec, out=out), K, W, stream)
        byt = product_bytes(st, prec, len(t), R)
        cfg3[prec] = {"GB/s": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm_peak, "ms": ms,
                      "err_vs_f64": 0.0 if prec == "f64" else leg_errors([out], [y64])}
    h.check()
    legs["sphere81920.R64"] = cfg3
    del h
    # the single layer's entries in float64 arithmetic (GCA_F64_ENTRIES, the
    # paper's precision for the near-singular quadrature) beside the float-pair
    # default: the same batch build of the bench's two meshes
    trees = [gca.tree_build(v, t, PARAMS["leaf_size"]) for v, t in meshes]
    gca.profile_enable(True)
    a.record(stream)
    b64 = gca.build_batch(meshes, trees, gca.Params(**PARAMS, flags=gca.F64_ENTRIES))
    b.record(stream)
    b.synchronize()
    ph64 = gca.profile_read()
    gca.profile_enable(False)
    legs["f64_entries.sphere20480x2"] = {
        "workload": "the bench's two meshes, gca_build_batch with GCA_F64_ENTRIES",
        "build_s": a.elapsed_time(b) * 1e-3,
        "phases_ms": {k: round(ph64[k][1], 3) for k in ("couple_entries", "near_entries", "singular") if k in ph64}}
    b64.free()
    del b64
    # the double-layer operator K on the perturbed 20480-triangle sphere (its
    # row bases are the single layer's, its column bases its own)
    v, t = meshes[1]
    tree = gca.tree_build(v, t, PARAMS["leaf_size"])
    a.record(stream)
    hd = gca.build_double_layer(v, t, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
    b.record(stream)
    b.synchronize()
    st = hd.stats()
    cs = hd.column_stats()
    R = NRHS
    x64 = torch.from_numpy(synth.normal_rhs(len(t), R, seed=0)).to(dev)
    x32 = x64.float()
    dlg = {"workload": "double layer, perturbed20480, leaf 64, eta 2, m 4, tol 1e-8, 16 RHS N(0,1)",
           "build_s": a.elapsed_time(b) * 1e-3, "rank_sum_rows": st["rank_sum"], "rank_sum_cols": cs["rank_sum"]}
    ref = {}
    for tr in (False, True):
        y64 = torch.empty((R, len(t)), dtype=torch.float64, device=dev).t()
        for prec in ("f64", "f32", "bf16"):
            xin = x64 if prec == "f64" else x32
            out = y64 if prec == "f64" else torch.empty((R, len(t)), dtype=torch.float32, device=dev).t()
            ms = time_products(lambda: hd.matvec(xin, prec, transpose=tr, out=out), K, W, stream)
            sm = {"f64": 8, "f32": 4, "bf16": 2}[prec]
            sv = 8 if prec == "f64" else 4
            byt = (sm * (st["v_entries"] + st["e_entries"] + cs["w_entries"] + cs["f_entries"] + st["s_entries"])
                   + sv * st["n_entries"] + 2 * sv * len(t) * R)
            key = prec + (".T" if tr else "")
            dlg[key] = {"GB/s": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm_peak, "ms": ms,
                        "err_vs_f64": 0.0 if prec == "f64" else leg_errors([out], [y64])}
    hd.check()
    legs["double_layer.perturbed20480.R16"] = dlg
    del hd
    # the collocation variant on the 20480-triangle sphere: one integral per
    # entry; its entry phases beside the Galerkin single layer's (same mesh)
    v, t = meshes[0]
    tree = gca.tree_build(v, t, PARAMS["leaf_size"])
    gca.profile_enable(True)
    hg = gca.build(v, t, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
    torch.cuda.synchronize()
    ph_g = gca.profile_read()
    del hg
    a.record(stream)
    hc = gca.build_collocation(v, t, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
    b.record(stream)
    b.synchronize()
    ph_c = gca.profile_read()
    gca.profile_enable(False)
    st = hc.stats()
    cs = hc.column_stats()
    ent = lambda ph, names: sum(ph.get(nm, (0, 0.0))[1] for nm in names)  # noqa: E731
    colg = {"workload": "collocation at centroids, sphere20480, leaf 64, eta 2, m 4, tol 1e-8, 16 RHS N(0,1)",
            "build_s": a.elapsed_time(b) * 1e-3,
            "entries_ms": ent(ph_c, ("col_couple_entries", "col_near_entries")),
            "galerkin_entries_ms": ent(ph_g, ("couple_entries", "near_entries", "singular")),
            "green_aca_ms": ent(ph_c, ("green_aca",)), "galerkin_green_aca_ms": ent(ph_g, ("green_aca",))}
    x64 = torch.from_numpy(synth.normal_rhs(len(t), NRHS, seed=0)).to(dev)
    x32 = x64.float()
    for tr in (False, True):
        y64 = torch.empty((NRHS, len(t)), dtype=torch.float64, device=dev).t()
        for prec in ("f64", "f32", "bf16"):
            xin = x64 if prec == "f64" else x32
            out = y64 if prec == "f64" else torch.empty((NRHS, len(t)), dtype=torch.float32, device=dev).t()
            ms = time_products(lambda: hc.matvec(xin, prec, transpose=tr, out=out), K, W, stream)
            sm = {"f64": 8, "f32": 4, "bf16": 2}[prec]
            sv = 8 if prec == "f64" else 4
            byt = (sm * (st["v_entries"] + st["e_entries"] + cs["w_entries"] + cs["f_entries"] + st["s_entries"])
                   + sv * st["n_entries"] + 2 * sv * len(t) * NRHS)
            colg[prec + (".T" if tr else "")] = {"GB/s": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm_peak,
                                                  "ms": ms,
                                                  "err_vs_f64": 0.0 if prec == "f64" else leg_errors([out], [y64])}
    hc.check()
    legs["collocation.sphere20480.R16"] = colg
    del hc
    # the nodal (piecewise linear) basis of Sect. 5 on the 20480-triangle
    # sphere: 10242 vertex indices, entries summed over triangle pairs of the
    # support unions
    v, t = meshes[0]
    tree = gca.tree_build_points(v, PARAMS["leaf_size"])
    gca.profile_enable(True)
    a.record(stream)
    hp = gca.build_p1(v, t, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
    b.record(stream)
    b.synchronize()
    ph_p = gca.profile_read()
    gca.profile_enable(False)
    st = hp.stats()
    p1g = {"workload": "nodal basis, sphere20480 (10242 vertices), leaf 64, eta 2, m 4, tol 1e-8, 16 RHS N(0,1)",
           "build_s": a.elapsed_time(b) * 1e-3, "rank_sum": st["rank_sum"],
           "phases_ms": {k: round(ms, 3) for k, (_, ms) in ph_p.items()},
           "regular_pairs": st["n_singular"][0], "touching_pairs": st["n_singular"][1:]}
    nv = len(v)
    x64 = torch.from_numpy(synth.normal_rhs(nv, NRHS, seed=0)).to(dev)
    x32 = x64.float()
    y64 = torch.empty((NRHS, nv), dtype=torch.float64, device=dev).t()
    for prec in ("f64", "f32", "bf16"):
        xin = x64 if prec == "f64" else x32
        out = y64 if prec == "f64" else torch.empty((NRHS, nv), dtype=torch.float32, device=dev).t()
        ms = time_products(lambda: hp.matvec(xin, prec, out=out), K, W, stream)
        byt = product_bytes(st, prec, nv, NRHS)
        p1g[prec] = {"GB/s": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm_peak, "ms": ms,
                     "err_vs_f64": 0.0 if prec == "f64" else leg_errors([out], [y64])}
    hp.check()
    legs["p1.sphere20480.R16"] = p1g
    del hp
    # the nodal basis on curved triangles (Sect. 6): the same mesh with the
    # surface points over its edges
    mids = synth.edge_midpoints_for_config(MESHES[0])
    gca.profile_enable(True)
    a.record(stream)
    hq = gca.build_p1_curved(v, t, mids, tree, gca.Params(**PARAMS, flags=gca.DROP_EXPORT))
    b.record(stream)
    b.synchronize()
    ph_q = gca.profile_read()
    gca.profile_enable(False)
    st = hq.stats()
    p1c = {"workload": "nodal basis on curved triangles, sphere20480 (10242 vertices), leaf 64, eta 2, m 4, "
                       "tol 1e-8, 16 RHS N(0,1)",
           "build_s": a.elapsed_time(b) * 1e-3, "rank_sum": st["rank_sum"],
           "phases_ms": {k: round(ms, 3) for k, (_, ms) in ph_q.items()},
           "touching_pairs": st["n_singular"][1:]}
    y64 = torch.empty((NRHS, nv), dtype=torch.float64, device=dev).t()
    for prec in ("f64", "f32", "bf16"):
        xin = x64 if prec == "f64" else x32
        out = y64 if prec == "f64" else torch.empty((NRHS, nv), dtype=torch.float32, device=dev).t()
        ms = time_products(lambda: hq.matvec(xin, prec, out=out), K, W, stream)
        byt = product_bytes(st, prec, nv, NRHS)
        p1c[prec] = {"GB/s": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm_peak, "ms": ms,
                     "err_vs_f64": 0.0 if prec == "f64" else leg_errors([out], [y64])}
    hq.check()
    legs["p1_curved.sphere20480.R16"] = p1c
    del hq
    legs["error_vs_storage.sphere5120"] = error_vs_storage(gca, dev)
    return legs


def error_vs_storage(gca, dev, iters=25):
    """The comparison of the paper's Fig. 1-3 on the 5120-triangle sphere
    (leaf 32, eta 2): pure Green quadrature (m = 2, 3, 4), single-level GCA
    and GCA-H^2 (m = 3, tolerances 1e-4, 1e-6, 1e-8).  Per run: stored
    coefficients (bases, transfers, couplings or factors, near field), build
    seconds (device stream), and ||G~ - G_ref||_2 / ||G_ref||_2 by power
    iteration with the GPU products, G_ref the GCA-H^2 at m = 6, tolerance
    1e-12 (its own error is far below the others')."""
    import torch
    v, t = synth.mesh_for_config("sphere5120")
    tree = gca.tree_build(v, t, 32)
    n = len(t)

    def prm(m, tol):
        return gca.Params(leaf_size=32, eta=2.0, box_gauss_m=m, aca_tol=tol, sauter_q=5, flags=gca.DROP_EXPORT)

    def timed(fn, m, tol):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        h = fn(v, t, tree, prm(m, tol))
        b.record()
        b.synchronize()
        return h, a.elapsed_time(b) * 1e-3

    ref, _ = timed(gca.build, 6, 1e-12)

    def err(h):
        x = torch.randn(n, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
        lam = 0.0
        for _ in range(iters):
            x = x / x.norm()
            r = ref.matvec(x, "f64") - h.matvec(x, "f64")
            y = ref.matvec(r, "f64", transpose=True) - h.matvec(r, "f64", transpose=True)
            lam = float(y.norm())
            x = y
        z = torch.randn(n, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
        for _ in range(iters):
            z = z / z.norm()
            z = ref.matvec(ref.matvec(z, "f64"), "f64", transpose=True)
        return (lam / float(z.norm())) ** 0.5

    rows = []
    runs = [("green_quadrature", gca.build_green_quadrature, m, 1e-6) for m in (2, 3, 4)]
    runs += [(kind, fn, 3, tol) for tol in (1e-4, 1e-6, 1e-8)
             for kind, fn in (("single_level_gca", gca.build_single_level), ("gca_h2", gca.build))]
    for kind, fn, m, tol in runs:
        h, bs = timed(fn, m, tol)
        st = h.stats()
        rows.append({"method": kind, "m": m, "tol": tol if kind != "green_quadrature" else None,
                     "stored_entries": st["v_entries"] + st["e_entries"] + st["s_entries"] + st["n_entries"],
                     "build_s": bs, "rel_spectral_error": err(h)})
        del h
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-leg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--profile", choices=["f64", "f32", "bf16", "build", "build2", "p1", "p1c"], default=None,
                    help="run the small single-mesh case used for kernel captures")
    args = ap.parse_args()
    if args.oracle_leg:
        print(json.dumps(oracle_leg()), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile:
        run_profile(args)
        return

    import torch
    import torch.distributed as dist

    import paper_1810_08429_b300 as gca

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # workload, host side
    meshes, trees = [], []
    for name in MESHES:
        v, t = synth.mesh_for_config(name)
        meshes.append((v, t))
        trees.append(gca.tree_build(v, t, PARAMS["leaf_size"]))
    n = meshes[0][1].shape[0]
    prm = gca.Params(**PARAMS)
    xs64 = [torch.from_numpy(synth.normal_rhs(len(t), NRHS, seed=0)).to(dev) for _, t in meshes]
    xs32 = [x.float() for x in xs64]
    ys = {p: [torch.empty((NRHS, len(t)), dtype=torch.float64 if p == "f64" else torch.float32,
                          device=dev).t() for _, t in meshes] for p in ("f64", "f32", "bf16", "f32T")}

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    marks = []
    batch = None

    def step(record):
        nonlocal batch
        # the previous step's batch is freed inside the step but outside the
        # build's window (cudaFree of its buffers synchronises the device);
        # explicitly, since the batch and its handle views form a reference
        # cycle that the garbage collector would otherwise break at a random
        # point (inside some other timed window)
        if batch is not None:
            batch.free()
        batch = None
        a = ev()
        batch = gca.build_batch(meshes, trees, prm)
        if record:
            marks.append(("build", a, ev()))
        for p, xs, tr_ in (("f64", xs64, False), ("f32", xs32, False), ("bf16", xs32, False),
                           ("f32T", xs32, True)):
            a = ev()
            batch.matvec(xs, "f32" if p == "f32T" else p, transpose=tr_, outs=ys[p])
            if record:
                marks.append((p, a, ev()))
        return batch.handles

    hs = None
    gc.disable()  # no collection inside the timed windows (the batches are freed explicitly)
    for _ in range(args.warmup):
        hs = step(False)
    stats = [h.stats() for h in hs]
    ranks = [h.export(("rank",))["rank"] for h in hs]
    aca_flops = [green_aca_flops(tr, r, s["k"]) for tr, r, s in zip(trees, ranks, stats)]
    gpu_evals = sum(kernel_evals(tr, r, s["k"], s["n_entries"], s["n_singular"], s["s_entries"],
                                 PARAMS["sauter_q"]) for tr, r, s in zip(trees, ranks, stats))
    fp64_peak, fp32_peak = gca.peak_probe()
    torch.cuda.synchronize()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    gca.profile_enable(True)
    with ClockSampler(local) as clocks:
        t_start = ev()
        for _ in range(args.steps):
            hs = step(True)
        t_end = ev()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    gca.profile_enable(False)
    phases = gca.profile_read()
    gc.enable()
    total_ms = t_start.elapsed_time(t_end)
    clk = clocks.summary()

    agg = {}
    for name, a, b in marks:
        key = name.split(".")[0]
        agg.setdefault(key, 0.0)
        agg[key] += a.elapsed_time(b)
    K = args.steps
    nm = len(MESHES)
    bytes_by = {p: sum(product_bytes(s, p if p != "f32T" else "f32", n, NRHS) for s in stats)
                for p in ("f64", "f32", "bf16", "f32T")}
    # replicas: the slowest rank's times, every rank's bytes (`value` and the
    # other throughputs below are whole-job figures)
    keys = ["total"] + list(bytes_by) + ["build"]
    worst = dict(zip(keys, max_over_ranks([total_ms] + [agg[p] for p in bytes_by] + [agg["build"]], dev)))
    total_ms = worst["total"]
    agg["build"] = worst["build"]
    gbs = {p: whole_job_gbs(bytes_by[p] * K, worst[p], 1) for p in bytes_by}
    hbm_peak, peak_kind = measured_peaks()

    # accuracy of the reduced-precision products against the float64 product
    errs = {}
    for p in ("f32", "bf16"):
        e = 0.0
        for i in range(nm):
            ref = ys["f64"][i]
            e = max(e, float(((ys[p][i].double() - ref).norm(dim=0) / ref.norm(dim=0)).max()))
        errs[p] = e

    # dominant kernel of the step, and of the product: algorithmic work of the
    # phase over the timed region divided by the phase's device time
    dom = max(phases, key=lambda k: phases[k][1])
    evals = [build_evals(s, PARAMS["sauter_q"]) for s in stats]

    def roofline_for(name):
        launches, ms = phases[name]
        if name.startswith("mv_"):
            stage, prec = name.split(".")[0], name.split(".")[1]
            sm = {"f64": 8, "f32": 4, "bf16": 2}[prec]
            sv = 8 if prec == "f64" else 4
            per = {"mv_persistent": lambda s: product_bytes(s, prec, n, NRHS)}[stage]
            byt = K * sum(per(s) for s in stats)
            ach = byt / (ms * 1e-3) / 1e9
            tr = captured_traffic(name)
            if tr is not None:  # captured on mesh 0 alone; the launch covers every mesh
                tr = tr * sum(per(s) for s in stats) / per(stats[0])
            return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                    "unit": "GB/s", "frac": ach / hbm_peak, "traffic": tr,
                    "traffic_unit": "bytes per launch",
                    "launches_per_step": launches / K, "peak_kind": peak_kind}
        fp32 = name == "couple_entries"  # float-pair arithmetic on the FP32 pipe
        if name in evals[0]:
            per_eval = FLOPS_PER_SPLIT_EVAL if fp32 else FLOPS_PER_EVAL
            flops = K * per_eval * sum(e[name] for e in evals)
            ach = flops / (ms * 1e-3) / 1e12
        elif name == "green_aca":
            ach = K * sum(aca_flops) / (ms * 1e-3) / 1e12
        else:
            ach = None
        pk = (fp32_peak if fp32 else fp64_peak) / 1e12
        kind = "fp32" if fp32 else "fp64"
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": pk,
                "unit": f"TFLOP/s ({kind})", "frac": (ach / pk) if ach else None,
                "traffic": captured_traffic(name),
                "traffic_unit": ("bytes per launch (two meshes, scaled from one mesh's capture)"
                                 if name == "green_aca" else "bytes per launch (mesh 0)"),
                "launches_per_step": launches / K,
                "peak_kind": f"measured by gca_peak_probe ({kind} FMA chains)"}

    mv_dom = max((k for k in phases if k.startswith("mv_") and ".f32" in k and not k.endswith(".T")),
                 key=lambda k: phases[k][1])

    # end to end through the public API with host buffers (f32 product)
    e2e_ms = []
    h2d = d2h = 0
    # x and y live in page-locked host memory; the product's gather and
    # scatter kernels read and write them in place over the bus
    pin_x = []
    for x in xs32:
        px = torch.empty((x.shape[1], x.shape[0]), dtype=torch.float32).pin_memory().t()
        px.copy_(x.cpu())
        pin_x.append(px)
    pin_y = [torch.empty((NRHS, len(t)), dtype=torch.float32).pin_memory().t() for _, t in meshes]
    for it in range(args.warmup + K):
        a = ev()
        batch.matvec(pin_x, "f32", outs=pin_y)
        b = ev()
        b.synchronize()
        if it >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    h2d = sum(x.numel() * 4 for x in xs32)
    d2h = h2d
    e2e_val = whole_job_gbs(bytes_by["f32"], max_over_ranks([statistics.median(e2e_ms)], dev)[0], 1)

    launches_per_step = sum(l for (l, _) in phases.values()) / K

    # the other product legs: few right-hand sides on the same two meshes, and
    # the 81920-triangle precision configuration (64 right-hand sides)
    with ClockSampler(local) as clocks_legs:
        legs = run_legs(gca, batch, meshes, stats, n, args, dev, stream, hbm_peak)
    legs["clocks"] = clocks_legs.summary()

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        o = oracle_sample()
        allc, one = o["all_cores"], o["single_thread"]
        cpu = {"value": allc["gbs"], "unit": "GB/s", "cores": allc["threads"], "kind": "oracle",
               "sample": (f"oracle float64 H2 product (16 RHS) on its own GCA-H2 of the "
                          f"{o['n']}-triangle sphere built with the workload's parameters; "
                          f"timed on all cores ({allc['threads']} BLAS threads) and on one thread"),
               "cpu_model": o["cpu_model"], "host_cores": o["cores"],
               "single_thread": {"value": one["gbs"], "unit": "GB/s", "cores": 1,
                                 "build_s": one["build_s"],
                                 "build_evals_per_s": one["build_evals_per_s"]},
               "all_cores": {"value": allc["gbs"], "unit": "GB/s", "cores": allc["threads"],
                             "build_s": allc["build_s"],
                             "build_evals_per_s": allc["build_evals_per_s"]},
               "build_kernel_evals": o["build_kernel_evals"],
               "build_unit": "kernel evaluations (7 k per Green-matrix row, 49 per regular entry, "
                             "q^3 per Sauter-Schwab region)"}
    line = {
        "metric": METRIC, "value": gbs["f32"] * world, "unit": "GB/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": total_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config({"parallelism": f"replicas{world}"}),
        "build_s": agg["build"] / K * 1e-3,
        "build_evals_per_s": gpu_evals / (agg["build"] / K * 1e-3),
        "build_kernel_evals": gpu_evals,
        "matvec": {p: {"GB/s": gbs[p], "frac_hbm": gbs[p] / hbm_peak,
                       "ms_both_meshes": agg[p] / K} for p in gbs},
        "err_vs_f64": errs,
        "matvec_legs": legs,
        "roofline": roofline_for(dom),
        "roofline_matvec": roofline_for(mv_dom),
        "peaks": {"hbm_gbs": hbm_peak, "hbm_kind": peak_kind, "fp64_tflops": fp64_peak / 1e12,
                  "fp32_tflops": fp32_peak / 1e12},
        "phases_ms_per_step": {k: v[1] / K for k, v in sorted(phases.items())},
        "clocks": clk,
        "e2e": {"value": e2e_val * world, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * K,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
