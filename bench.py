"""Benchmark of the H2 double-layer matrix-vector product u2 = M u1.

Headline (default): the level-8 icosphere (655,362 boundary nodes, 1,310,720
triangles), Chebyshev order m = 5, leaf size 64, eta = 2, 16 right-hand sides
(u1 = z plus 15 seeded smooth magnetisation states), the mixed form: coupling,
transfer and leaf-basis products in FP32 on the CUDA cores, the Lindholm near
field, the solid-angle diagonal and the final per-node sums in FP64.  One step
= one full product of the 16 right-hand sides (input gather, upward pass,
coupling, downward pass, near field, leaf expansion).  The plain FP64 form of
the same product is timed beside it.

Forms (same GPU, each against the FP64 form of its own workload and r):
the 1000 x 1000 x 10 film (r = 1), the 3:2:1 ellipsoid (r = 32), the level-8
icosphere (r = 16), eight uneven meshes of 5k-100k nodes in ONE batched launch
(r = 1) and the 64 x 64-per-face cube (r = 1), in FP64, FP32, 3xTF32 and BF16
hi + lo (tensor cores) and, labelled separately, the FP32 pair near field.

Prints one JSON line.  `value` is boundary DOF/s = N * r / t_step over all
ranks (each rank runs its own replica of the problem: weak scaling, no
data-path collective).  `e2e` is the same metric through the C ABI with host
buffers (host -> device copy, product, device -> host copy per step).
Relative errors are against the CPU oracle's H2 product on sampled rows (all
nodes of a few leaves spread over the tree).  `cpu_baseline` and
`--impl reference` time the CPU oracle (plain C, OpenMP) on the host cores:
exact rows of M (Lindholm entries and Psi, O(T) per row) for seeded nodes,
applied to the same right-hand sides.

Reproduce a single form: python bench.py --workload ellipsoid --precision
bf16x3 --r 32 --no-forms (see --help).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "H² double-layer matvec boundary DOF/s at rel.err≤1e-5; mixed+batched vs FP64"
UNIT = "boundary DOF/s"
HBM_GBS_FALLBACK = 6800.0
# FP64 FMA issue rate of a GB300 SM: 2 per clock (1.26 TFLOP/s nominal over
# 152 SMs at 2070 MHz); FP32 CUDA-core FMA: 128 per clock per SM.  The paired
# near field spends 12 FP32 instructions per entry and right-hand side.
N_SM = 152
FP64_FMA_PER_CLK_SM = 2
FP32_FMA_PER_CLK_SM = 128
PAIR_INSTR_PER_MAC = 12
PASS_NAMES = {0: "gather", 1: "up_leaf", 2: "up_transfer", 3: "coupling", 4: "down_transfer",
              5: "leaf_near", 6: "leaf_expand", 7: "flow", 8: "split_near", 9: "split_far", 10: "split_add"}
KERNEL_NAMES = {0: "k_prologue", 7: "k_seg (dataflow, whole product)", 8: "k_near_items (split form near field)",
                9: "k_seg (split form far field)", 10: "k_add"}

# fp32-onfly: FP32 far field with the coupling blocks evaluated in the product;
# fp32-pair, bf16x3-pair: the near field of split-form products (r > 8) in
# FP32 pairs with error-free products and sums (FP64-equivalent, <= n * 2^-48 per row of n terms)
PRECISIONS = ("fp64", "fp32", "tf32x3", "bf16x3", "fp32-onfly", "fp32-pair", "bf16x3-pair")
DTYPES = {"fp64": "f64", "fp32": "f32+f64", "tf32x3": "tf32x3+f64", "bf16x3": "bf16x3+f64",
          "fp32-onfly": "f32+f64", "fp32-pair": "f32+f32x2+f64", "bf16x3-pair": "bf16x3+f32x2+f64"}
# the forms of each workload beside the headline (precision, right-hand sides);
# "<precision>@<eps>": the far field recompressed algebraically with relative
# threshold eps (h2_params.recompress_eps) before it is stored
FORMS = {
    "ico8": [("fp64", 16), ("bf16x3", 16), ("tf32x3", 16), ("fp32-pair", 16)],
    "ellipsoid": [("fp64", 32), ("fp32", 32), ("bf16x3", 32), ("tf32x3", 32), ("fp32-pair", 32)],
    "film": [("fp64", 1), ("fp32", 1), ("bf16x3", 1), ("tf32x3", 1), ("fp32-onfly", 1), ("fp64@1e-6", 1),
             ("fp32@1e-6", 1)],
    "batch8": [("fp64", 1), ("fp32", 1), ("bf16x3", 1)],
    "cube64": [("fp64", 1), ("fp32", 1), ("fp64@1e-8", 1), ("fp32@1e-6", 1), ("fp64", 16), ("fp32", 16),
               ("bf16x3", 16)],
}


def split_form(precision: str):
    """(precision without the recompression threshold, threshold or 0)."""
    if "@" in precision:
        base, eps = precision.split("@")
        return base, float(eps)
    return precision, 0.0
WORKLOADS = sorted(set(synth.WORKLOADS) | {"batch8"})
DEFAULT_R = {"ico3": 2, "ico8": 16, "ellipsoid": 32}   # the workloads' own counts (others: 1)


def workload_meshes(name: str):
    """(meshes, m, leaf, eta, note) of a named workload; batch8 = the eight uneven meshes."""
    if name == "batch8":
        ms = synth.workloads.multi_mesh_set()
        return ms, 5, 64, 2.0, "8 meshes: cubes n = 29, 40, 64, 90, 128; icospheres L5, L6; cube-sphere 70"
    w = synth.make_workload(name)
    return [w.mesh], w.m, w.leaf, w.eta, w.note


def workload_rhs(name: str, meshes, r: int):
    """The workload's seeded right-hand sides, one (r, N) array per mesh (the
    recipes of synth.workloads; other counts r: seeded smooth states)."""
    seed = 1811
    mesh = meshes[0]
    if name == "batch8":
        return [np.ascontiguousarray(synth.smooth_states(mm, r, seed + i)) for i, mm in enumerate(meshes)]
    if name == "ico8":   # u1 = z (uniform magnetisation along z) plus r - 1 smooth states
        u = np.atleast_2d(synth.uniform_rhs_magnetisation(mesh))
        if r > 1:
            u = np.vstack([u, synth.smooth_states(mesh, r - 1, seed)])
    elif name == "film" and r == 1:
        u = synth.uniform_rhs(mesh.n_vertices, 1, seed)
    elif name == "cube64" and r == 1:
        u = synth.normal_dot_field(mesh, seed)
    elif name == "ico3" and r == 2:
        u = np.vstack([synth.gaussian_rhs(mesh.n_vertices, 1, seed), np.ones((1, mesh.n_vertices))])
    else:
        u = synth.smooth_states(mesh, r, seed)
    return [np.ascontiguousarray(np.atleast_2d(u), dtype=np.float64)]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_GBS_FALLBACK, "sm_max_mhz": 2070.0}, "fallback"


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self) -> dict:
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def sample_nodes(n_vertices: int, count: int, seed: int) -> np.ndarray:
    return np.sort(np.random.default_rng(seed).choice(n_vertices, size=min(count, n_vertices), replace=False))


def exact_rows_rate(mesh, u1, budget_s: float, batch: int = 16, seed: int = 1811):
    """The CPU oracle's exact rows of M (Lindholm entries and Psi, O(T) per row)
    for batches of seeded nodes, applied to the r right-hand sides, until
    `budget_s` has passed: boundary DOF/s = rows x r / seconds."""
    import oracle
    oracle.build()
    r = u1.shape[0]
    done, el, k = 0, 0.0, 0
    while el < budget_s or k == 0:
        rows = sample_nodes(mesh.n_vertices, batch, seed + k)
        t0 = time.perf_counter()
        R = oracle.dense_rows(mesh.xyz, mesh.tri, rows)
        _ = R @ u1.T
        el += time.perf_counter() - t0
        done += rows.size
        k += 1
    return done * r / el, oracle.num_threads(), done, el


def oracle_sampled_rows(mesh, m, leaf, eta, u1, n_leaves: int):
    """The oracle's H2 product (direct Chebyshev bases, exact near entries, the
    diagonal) at every node of `n_leaves` leaves spread over its tree."""
    import oracle
    oracle.build()
    o = oracle.H2Oracle(mesh.xyz, mesh.tri, m, leaf, eta, store=False)
    tr = o.tree()
    leaves = [c for c in range(len(tr["size"])) if tr["child0"][c] < 0]
    pick = sorted({leaves[int(i)] for i in np.linspace(0, len(leaves) - 1, n_leaves)})
    rows = np.concatenate([tr["perm"][tr["start"][c]:tr["start"][c] + tr["size"][c]] for c in pick])
    t0 = time.perf_counter()
    ref = o.rows(u1, rows)
    el = time.perf_counter() - t0
    o.close()
    return rows, ref, el


def err_pair(y, ref):
    """(max over right-hand sides of the relative L2 error, of the relative max-norm error)."""
    l2 = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    mx = np.max(np.abs(y - ref), axis=1) / np.max(np.abs(ref), axis=1)
    return float(np.max(l2)), float(np.max(mx))


def max_over_ranks(t: float, dist, device) -> float:
    """The slowest rank's time (the job's time: every rank's step ends behind
    a barrier); `dist` None is a single process."""
    if dist is None:
        return t
    import torch
    x = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def replica_rate(units_per_rank: float, world: int, t_job: float) -> float:
    """Whole-job throughput of `world` replicas, each processing
    `units_per_rank` units per step, with the job's step time."""
    return units_per_rank * world / t_job


def run_reference(args, rank, world):
    """The tier's reference arm: the CPU oracle on the host cores, same
    workload, metric and unit; each step = exact rows of M for 16 seeded nodes
    (a different set per step) applied to the r right-hand sides."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    r = args.r if args.r > 0 else DEFAULT_R.get(args.workload, 1)
    meshes, m, leaf, eta, _ = workload_meshes(args.workload)
    us = workload_rhs(args.workload, meshes, r)
    batch = 16
    n = 0
    el = 0.0
    for step in range(args.warmup + args.steps):
        mesh, u1 = meshes[step % len(meshes)], us[step % len(meshes)]
        rows = sample_nodes(mesh.n_vertices, batch, 1811 + step)
        t0 = time.perf_counter()
        R = oracle.dense_rows(mesh.xyz, mesh.tri, rows)
        _ = R @ u1.T
        t = time.perf_counter() - t0
        if step >= args.warmup:
            el += t
            n += rows.size
    value = n * r / el
    sample = (f"per step: exact rows of M (Lindholm entries and Psi, O(T) per row) at {batch} seeded nodes "
              f"of the {args.workload} workload applied to its {r} right-hand sides (CPU oracle, plain C + "
              f"OpenMP, FP64)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": int(sum(mm.n_vertices for mm in meshes)), "m": m,
                       "leaf": leaf, "eta": eta, "r": r, "precision": getattr(args, "precision", "fp32")},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_ops(pkg, geoms, m, leaf, eta, precision, r):
    precision, eps = split_form(precision)
    base = precision.split("-")[0]
    pair = precision.endswith("-pair") and r > 8   # the paired near field needs split-form products
    return [pkg.Operator(g, m=m, leaf=leaf, eta=eta,
                         precision={"fp64": pkg.FP64, "fp32": pkg.FP32, "tf32x3": pkg.TF32X3,
                                    "bf16x3": pkg.BF16X3}[base], max_rhs=r,
                         coupling=pkg.COUPLING_ON_THE_FLY if precision == "fp32-onfly" else pkg.COUPLING_STORED,
                         near_field=pkg.NEAR_F32PAIR if pair else pkg.NEAR_FP64, recompress_eps=eps) for g in geoms]


def run_products(pkg, ops, xs, ys, stream_ptr):
    if len(ops) == 1:
        pkg.h2_matvec(ops[0].handle, xs[0].data_ptr(), ys[0].data_ptr(), xs[0].shape[0], stream_ptr)
    else:
        pkg.h2_matvec_batched([o.handle for o in ops], [x.data_ptr() for x in xs], [y.data_ptr() for y in ys],
                              [x.shape[0] for x in xs], stream_ptr)


def time_products(pkg, torch, ops, xs, ys, steps, warmup, barrier=None):
    """`steps` products timed with CUDA events on the launching stream, after
    `warmup` untimed ones (inputs resident in device memory)."""
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    for _ in range(max(warmup, 3)):
        run_products(pkg, ops, xs, ys, sp)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run_products(pkg, ops, xs, ys, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    status = pkg.h2_device_status(ops[0].handle)
    if status != 0:
        raise RuntimeError(f"device-side wait gave up during the benchmark ({status})")
    return e0.elapsed_time(e1) / 1e3 / steps


def pass_profile(pkg, op, x, y, r, steps):
    """Per-launch CUDA-event times of `steps` products (h2_profile_*): each
    kernel timed by events recorded around it on the stream it runs on."""
    import ctypes
    import torch
    L = pkg.load()
    sp = int(torch.cuda.current_stream().cuda_stream)
    L.h2_profile_enable(ctypes.c_void_p(op.handle), 1)
    for _ in range(steps):
        pkg.h2_matvec(op.handle, x.data_ptr(), y.data_ptr(), r, sp)
    cap = 64
    kind = (ctypes.c_int32 * cap)()
    ms = (ctypes.c_double * cap)()
    byt = (ctypes.c_int64 * cap)()
    macs = (ctypes.c_int64 * cap)()
    grid = (ctypes.c_int32 * cap)()
    ncalls = ctypes.c_int32()
    nent = ctypes.c_int32()
    L.h2_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 7
    rc = L.h2_profile_read(ctypes.c_void_p(op.handle), cap, kind, ms, byt, macs, grid,
                           ctypes.byref(ncalls), ctypes.byref(nent))
    L.h2_profile_enable(ctypes.c_void_p(op.handle), 0)
    passes = []
    if rc == 0 and ncalls.value > 0:
        for i in range(min(nent.value, cap)):
            passes.append({"launch": i, "kind": int(kind[i]), "pass": PASS_NAMES.get(kind[i], str(kind[i])),
                           "ms": ms[i] / ncalls.value, "bytes": byt[i], "macs_per_rhs": macs[i],
                           "grid": grid[i]})
    return passes


def roofline_of(launch, r, precision, peaks, peak_src, workload):
    """Roofline of one launch: algorithmic bytes (matrix bytes read once) and
    flops (2 per stored entry and right-hand side) per launch over its
    CUDA-event duration, against the bound that is closer to its peak."""
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", HBM_GBS_FALLBACK))
    fp64_peak = N_SM * FP64_FMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    fp32_peak = N_SM * FP32_FMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12
    pair_peak = N_SM * FP32_FMA_PER_CLK_SM / PAIR_INSTR_PER_MAC * 2 * sm_max * 1e6 / 1e12
    k = launch["kind"]
    if k in (8, 9, 10):   # the split form runs products of at most 16 right-hand sides
        r = min(r, 16)
    t = launch["ms"] / 1e3
    gbs = launch["bytes"] / t / 1e9
    tfl = 2.0 * launch["macs_per_rhs"] * r / t / 1e12
    if k == 8:   # the split form's near field: FP64 FMAs, or the paired form's FP32 instructions
        pair = precision.endswith("-pair")
        alu_peak, alu_name = (pair_peak, f"FP32 pipe at {PAIR_INSTR_PER_MAC} instructions per multiply-add "
                                         f"({N_SM} SMs x {FP32_FMA_PER_CLK_SM}/{PAIR_INSTR_PER_MAC} x 2 x {sm_max:.0f} MHz)") \
            if pair else (fp64_peak, f"FP64 FMA rate derived from unit counts: {N_SM} SMs x {FP64_FMA_PER_CLK_SM} "
                                     f"FMA/clk x 2 x {sm_max:.0f} MHz (microbenchmark: 1.257 TFLOP/s)")
    elif split_form(precision)[0] == "fp64":
        alu_peak, alu_name = fp64_peak, (f"FP64 FMA rate derived from unit counts: {N_SM} SMs x "
                                         f"{FP64_FMA_PER_CLK_SM} FMA/clk x 2 x {sm_max:.0f} MHz "
                                         f"(microbenchmark: 1.257 TFLOP/s)")
    else:
        alu_peak, alu_name = fp32_peak, (f"FP32 FMA rate derived from unit counts: {N_SM} SMs x "
                                         f"{FP32_FMA_PER_CLK_SM} FMA/clk x 2 x {sm_max:.0f} MHz")
    hbm_frac, alu_frac = gbs / hbm, tfl / alu_peak
    name = KERNEL_NAMES.get(k, f"k_seg ({launch['pass']})")
    if alu_frac > hbm_frac:
        rf = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_frac,
              "traffic": None, "peak_source": alu_name, "kernel": name, "hbm_gbs": gbs,
              "hbm_frac_of_measured": hbm_frac}
    else:
        rf = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_frac,
              "traffic": None, "peak_source": f"{peak_src} hbm_gbs (copy, burst)", "kernel": name,
              "alu_tflops": tfl, "alu_frac": alu_frac}
    rf["launch_ms"] = launch["ms"]
    rf["algorithmic_bytes"] = launch["bytes"]
    rf["algorithmic_flops"] = 2.0 * launch["macs_per_rhs"] * r
    # DRAM bytes per launch from an ncu capture (profiles/), used only while
    # the kernel source is the one that was captured
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f)
        src = os.path.join(ROOT, "paper_1811_05731_gb300", "csrc", "h2_matvec.cu")
        with open(src, "rb") as f:
            sha = hashlib.sha1(f.read()).hexdigest()
        key = f"{workload}/{precision}/r{r}/{launch['pass']}"
        if key in tr and tr.get("kernel_source_sha1") == sha:
            rf["traffic"] = tr[key]
    return rf


def bench_form(pkg, torch, name, meshes, geoms, m, leaf, eta, us, precision, steps, warmup, peaks, peak_src,
               refs, barrier=None, keep=False):
    """Times one form (operators of `precision` for r = us[0].shape[0]) and
    returns its record; `refs` maps mesh index -> (rows, oracle rows)."""
    r = us[0].shape[0]
    ops = make_ops(pkg, geoms, m, leaf, eta, precision, r)
    xs = [torch.from_numpy(u).cuda() for u in us]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    t = time_products(pkg, torch, ops, xs, ys, steps, warmup, barrier)
    dof = sum(mm.n_vertices for mm in meshes) * r
    rec = {"workload": name, "precision": precision, "r": r, "value": dof / t, "ms_per_step": t * 1e3,
           "dtype": DTYPES[split_form(precision)[0]],
           "launch": "batched (one persistent launch)" if len(ops) > 1 else "single"}
    sts = [o.stats() for o in ops]
    rec["bytes_streamed"] = int(sum(s["bytes_streamed"] for s in sts))
    rec["assemble_seconds"] = float(sum(s["assemble_seconds"] for s in sts))
    if split_form(precision)[1] > 0:
        rec["recompress_eps"] = split_form(precision)[1]
        rec["mean_rank"] = [sts[0]["mean_rank_row"], sts[0]["mean_rank_col"]]
    if len(ops) == 1:
        passes = pass_profile(pkg, ops[0], xs[0], ys[0], r, 3)
        rec["passes"] = [{k: p[k] for k in ("pass", "ms", "bytes", "grid")} for p in passes]
        dom = max((p for p in passes if p["kind"] != 0), key=lambda p: p["ms"], default=None)
        if dom:
            rec["roofline"] = roofline_of(dom, r, precision, peaks, peak_src, name)
    else:   # the batched launch: gathers + one dataflow kernel, timed as a whole
        launch = {"kind": 7, "pass": "flow", "ms": t * 1e3, "bytes": rec["bytes_streamed"],
                  "macs_per_rhs": int(sum(s["macs_per_rhs"] for s in sts)), "grid": 0}
        rec["roofline"] = roofline_of(launch, r, precision, peaks, peak_src, name)
        rec["roofline"]["kernel"] = "k_seg (batched dataflow launch; time includes the 8 input gathers)"
    if refs:
        e2, em = [], []
        for i, (rows, ref) in refs.items():
            y = ys[i].cpu().numpy()[:, rows]
            a, b = err_pair(y, ref)
            e2.append(a)
            em.append(b)
        rec["rel_err_vs_fp64_oracle"] = max(e2)
        rec["maxnorm_err_vs_fp64_oracle"] = max(em)
        rec["meets_metric_tolerance"] = max(e2) <= (1e-8 if split_form(precision)[0] == "fp64" else 1e-5)
        if split_form(precision)[1] > 0:   # recompressed: the error includes the recompression's own
            rec["meets_metric_tolerance"] = max(e2) <= max(1e-8 if precision.startswith("fp64") else 1e-5,
                                                          split_form(precision)[1])
        rec["err_rows"] = int(sum(len(rows) for rows, _ in refs.values()))
    out = (rec, ops, xs, ys) if keep else (rec, None, None, None)
    if not keep:
        del ops, xs, ys
        torch.cuda.empty_cache()
    return out


def bench_fem(pkg, torch, n, steps, peaks):
    """The finite-element half of the field evaluation (h2_fem_solve) on the
    unit ball (the [-1, 1]^3 grid of n^3 cells, six tetrahedra each, mapped
    radially), uniform magnetisation along z: u1 Neumann solve, u2 boundary
    values through the H2 product (m = 4, leaf 64, FP64), u2 Dirichlet solve,
    energy.  One step = one field evaluation; CG to |r| <= 1e-10 |b|."""
    from synth import volume as vm
    xyz, tets = vm.ball_tets(n)
    surf, nodes = vm.boundary_surface(xyz, tets)
    g = pkg.Geometry(surf.xyz, surf.tri)
    op = pkg.Operator(g, m=4, leaf=64)
    F = pkg.Fem(xyz, tets, nodes)
    M = torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64).repeat(len(tets), 1).cuda()
    F.solve(op, M, tol=1e-10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        _, _, rep = F.solve(op, M, tol=1e-10)
    t = (time.perf_counter() - t0) / steps
    # CSR entries: each tetrahedron edge couples two nodes (both directions) plus the diagonal
    edges = np.unique(np.sort(np.concatenate([tets[:, [a, b]] for a in range(4) for b in range(a + 1, 4)]), axis=1),
                      axis=0)
    nnz = 2 * len(edges) + len(xyz)
    iters = rep["iters_u1"] + rep["iters_u2"]
    # per CG iteration: the CSR values and column indices once, ~10 vector passes of 8 bytes
    cg_bytes = iters * (12 * nnz + 4 * len(xyz) + 80 * len(xyz))
    hbm = float(peaks.get("hbm_gbs", HBM_GBS_FALLBACK))
    return {"workload": f"fem_ball{n}", "vertices": int(len(xyz)), "tetrahedra": int(len(tets)),
            "surface_nodes": int(len(nodes)), "ms_per_step": t * 1e3,
            "cg_iterations": [rep["iters_u1"], rep["iters_u2"]],
            "resid": [rep["resid_u1"], rep["resid_u2"]], "energy": rep["energy"],
            "err_vs_one_third": abs(rep["energy"] - 1.0 / 3.0), "volume_dof_per_s": len(xyz) / t,
            "timing": "host wall clock around the synchronous call (two CG solves with residual reads, one H2 product)",
            "cg_gbs_lower_bound": cg_bytes / t / 1e9, "cg_hbm_frac_lower_bound": cg_bytes / t / 1e9 / hbm}


def run_gpu(args, rank, local, world):
    import torch
    import paper_1811_05731_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    peaks, peak_src = measured_peaks()
    name = args.workload
    r = args.r if args.r > 0 else DEFAULT_R.get(name, 1)
    meshes, m, leaf, eta, note = workload_meshes(name)
    us = workload_rhs(name, meshes, r)
    geoms = [pkg.Geometry(mm.xyz, mm.tri) for mm in meshes]

    def barrier():
        if dist is not None:
            dist.barrier()

    # oracle rows for the errors (CPU, before any timing)
    want_err = not args.no_errors and rank == 0
    refs_cache = {}

    def refs_for(wname, wmeshes, wus, wm, wleaf, weta):
        key = (wname, wus[0].shape[0])
        if not want_err:
            return {}
        if key not in refs_cache:
            nl = 1 if len(wmeshes) > 1 else args.err_leaves
            refs_cache[key] = {i: oracle_sampled_rows(mm, wm, wleaf, weta, u, nl)[:2]
                               for i, (mm, u) in enumerate(zip(wmeshes, wus))}
        return refs_cache[key]

    refs = refs_for(name, meshes, us, m, leaf, eta)

    # headline form: device-resident inputs, K timed steps, clocks sampled meanwhile
    with ClockSampler(local) as clk:
        head, ops, xs, ys = bench_form(pkg, torch, name, meshes, geoms, m, leaf, eta, us, args.precision,
                                       args.steps, args.warmup, peaks, peak_src, refs, barrier, keep=True)
    t_step = max_over_ranks(head["ms_per_step"] / 1e3, dist, "cuda")
    N = sum(mm.n_vertices for mm in meshes)
    value = replica_rate(N * r, world, t_step)
    st = ops[0].stats()
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)

    # end to end through the C ABI with pinned host buffers (copies in the timed region)
    e2e = None
    if len(ops) == 1:
        xh = torch.from_numpy(us[0]).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        for _ in range(2):
            pkg.h2_matvec(ops[0].handle, xh.data_ptr(), yh.data_ptr(), r, sp)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            pkg.h2_matvec(ops[0].handle, xh.data_ptr(), yh.data_ptr(), r, sp)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3 / args.steps, dist, "cuda")
        e2e = {"value": replica_rate(N * r, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": 8 * N * r,
               "d2h_bytes_per_step": 8 * N * r}
    n_launch = st["n_launches_matvec"] if len(ops) == 1 else len(ops) + 1
    del ops, xs, ys
    torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    clocks = clk.summary()
    forms = []
    if not args.no_forms and world == 1:
        # the FP64 form of the headline's workload and r first, then the others
        plan = [(name, "fp64", r)] if args.precision != "fp64" else []
        for wname in ([name] if args.forms_only_workload else [name] + [w for w in FORMS if w != name]):
            for prec, rr in FORMS.get(wname, []):
                if (wname, prec, rr) not in plan and not (wname == name and prec == args.precision and rr == r):
                    plan.append((wname, prec, rr))
        cur, wgeoms = None, None
        for wname, prec, rr in plan:
            if cur is None or cur[0] != wname:   # one workload's meshes and geometries at a time
                wgeoms = None
                cur = (wname,) + workload_meshes(wname)
                wgeoms = geoms if wname == name else [pkg.Geometry(mm.xyz, mm.tri) for mm in cur[1]]
            _, wmeshes, wm, wleaf, weta, _ = cur
            wus = workload_rhs(wname, wmeshes, rr)
            wrefs = refs_for(wname, wmeshes, wus, wm, wleaf, weta)
            rec, _, _, _ = bench_form(pkg, torch, wname, wmeshes, wgeoms, wm, wleaf, weta, wus, prec,
                                      min(args.steps, 10), 3, peaks, peak_src, wrefs)
            forms.append(rec)
            print(json.dumps({"form": rec["workload"], "precision": prec, "r": rr, "ms": rec["ms_per_step"]}),
                  file=sys.stderr, flush=True)
        allf = forms + [head]
        for f in forms:
            same = next((e["value"] for e in allf if e["workload"] == f["workload"] and e["precision"] == "fp64"
                         and e["r"] == f["r"]), None)
            if same:
                f["speedup_vs_fp64_same_workload_r"] = f["value"] / same
        fp64_head = next((f for f in forms if f["workload"] == name and f["precision"] == "fp64" and f["r"] == r),
                         None)
        if fp64_head:
            head["speedup_vs_fp64_same_workload_r"] = head["value"] / fp64_head["value"]

    cpu = None
    cpu_by = {}
    if not args.no_cpu_baseline and world == 1:
        rate, cores, n, el = exact_rows_rate(meshes[0], us[0], args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"exact rows of M (Lindholm entries and Psi, O(T) per row) at {n} seeded nodes of the "
                         f"{name} workload ({meshes[0].n_vertices} nodes) applied to its {r} right-hand sides, "
                         f"{el:.1f} s of CPU oracle work (plain C + OpenMP, FP64)"}
        if forms:
            for wname in [w for w in FORMS if w != name and w != "batch8"]:
                wmeshes = workload_meshes(wname)[0]
                rr = FORMS[wname][0][1]
                wus = workload_rhs(wname, wmeshes, rr)
                wr, _, wn, wel = exact_rows_rate(wmeshes[0], wus[0], 2.0)
                cpu_by[f"{wname}/r{rr}"] = {"value": wr, "rows": wn, "seconds": wel}

    fem_rec = None
    if not args.no_forms and world == 1:
        fem_rec = bench_fem(pkg, torch, 48, 5, peaks)

    cfg = {"workload": name, "N": N, "triangles": int(sum(mm.n_triangles for mm in meshes)), "m": m,
           "leaf": leaf, "eta": eta, "r": r, "precision": args.precision, "schedule": "flow",
           "note": note, "parallelism": f"replicas x{world}",
           "l2": f"inputs larger than L2: {head['bytes_streamed'] / 1e6:.0f} MB of matrices streamed per step "
                 f"(L2 129 MB), no flush"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic (seeded meshes and right-hand sides, synth/)",
        "config": cfg,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": n_launch * args.steps,
        "rel_err_vs_fp64_oracle": head.get("rel_err_vs_fp64_oracle"),
        "maxnorm_err_vs_fp64_oracle": head.get("maxnorm_err_vs_fp64_oracle"),
        "err_rows": head.get("err_rows"),
        "speedup_vs_fp64_same_workload_r": head.get("speedup_vs_fp64_same_workload_r"),
        "roofline": head.get("roofline"),
        "passes": head.get("passes"),
        "cpu_baseline": cpu,
        "cpu_oracle_by_workload": cpu_by,
        "forms": forms,
        "fem": fem_rec,
        "h2": {k: st[k] for k in ("n_clusters", "n_levels", "n_far_blocks", "n_near_blocks",
                                  "near_entries", "bytes_streamed", "macs_per_rhs",
                                  "compression_ratio", "assemble_seconds")},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="h2bem", choices=["h2bem", "reference"])
    ap.add_argument("--workload", default="ico8", choices=WORKLOADS)
    ap.add_argument("--precision", default="fp32", choices=list(PRECISIONS))
    ap.add_argument("--r", type=int, default=0, help="right-hand sides (0: the workload's own count)")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of CPU oracle work for cpu_baseline")
    ap.add_argument("--err-leaves", type=int, default=2, help="leaves whose rows the oracle computes for errors")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms and workloads")
    ap.add_argument("--forms-only-workload", action="store_true", help="forms of the headline workload only")
    ap.add_argument("--no-errors", action="store_true", help="skip the relative errors against the oracle")
    args = ap.parse_args()
    rank, local, world = rank_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, local, world)


if __name__ == "__main__":
    main()
