"""Benchmark of the H2 double-layer matrix-vector product u2 = M u1.

Workload (default): the surface of the unit cube with a structured 64 x 64
grid per face (24,578 boundary nodes, 49,152 triangles), Chebyshev order
m = 4, leaf size 64, eta = 2, FP64, one right-hand side u1 = n . m for a
seeded smooth unit magnetisation field m.  One step = one full matvec
(gather, upward pass, coupling, downward pass, leaf expansion + near field).

Prints one JSON line.  `value` is boundary DOF/s = N * r / t_step over all
ranks (each rank runs its own replica of the problem: weak scaling, no
data-path collective).  `e2e` is the same metric through the C ABI with host
buffers (host -> device copy, product, device -> host copy per step).
`--impl reference` times the CPU oracle (plain C, OpenMP) on the host cores.
"""
from __future__ import annotations

import argparse
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
# FP64 FMA issue rate of a GB300 SM: 2 per clock (1.25 TFLOP/s nominal over
# 152 SMs at 2070 MHz); FP32 CUDA-core FMA: 128 per clock per SM.
N_SM = 152
FP64_FMA_PER_CLK_SM = 2
FP32_FMA_PER_CLK_SM = 128
PASS_NAMES = {0: "gather", 1: "up_leaf", 2: "up_transfer", 3: "coupling", 4: "down_transfer",
              5: "leaf_near", 6: "leaf_expand", 7: "flow"}

# fp32-onfly: FP32 far field with the coupling blocks evaluated in the product;
# fp32-pair, bf16x3-pair: the near field of split-form products (r > 8) in
# FP32 pairs with error-free products and sums (FP64-equivalent, <= n * 2^-48 per row of n terms)
PRECISIONS = ("fp64", "fp32", "tf32x3", "bf16x3", "fp32-onfly", "fp32-pair", "bf16x3-pair")
DTYPES = {"fp64": "f64", "fp32": "f32+f64", "tf32x3": "tf32x3+f64", "bf16x3": "bf16x3+f64",
          "fp32-onfly": "f32+f64", "fp32-pair": "f32+f32x2+f64", "bf16x3-pair": "bf16x3+f32x2+f64"}
# reduced-precision and batched forms timed beside the headline form (same
# workload, same GPU): (precision, right-hand sides)
FORMS = [("fp32", 1), ("tf32x3", 1), ("bf16x3", 1), ("fp32-onfly", 1), ("fp64", 32), ("fp32", 32),
         ("fp32-onfly", 32), ("tf32x3", 32),
         ("bf16x3", 32), ("fp32-pair", 32), ("bf16x3-pair", 32)]


def workload_inputs(name: str, r: int):
    """The named synthetic workload; r > 0 replaces its right-hand sides by r
    seeded smooth magnetisation states u1 = n . m_c."""
    w = synth.make_workload(name)
    u1 = w.u1 if r <= 0 else synth.smooth_states(w.mesh, r, 1811)
    return w, np.ascontiguousarray(np.atleast_2d(u1), dtype=np.float64)


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


def cpu_oracle_rate(mesh, m, leaf, eta, u1, budget_s: float):
    """The CPU oracle's H2 product (plain C + OpenMP), timed on this host's cores."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.H2Oracle(mesh.xyz, mesh.tri, m, leaf, eta)
    setup = time.perf_counter() - t0
    y = o.matvec(u1)
    n = 0
    t0 = time.perf_counter()
    while True:
        y = o.matvec(u1)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 1000:
            break
    rate = mesh.n_vertices * u1.shape[0] * n / el
    return rate, oracle.num_threads(), n, el, setup, y


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
    if rank != 0:
        return
    w, u1 = workload_inputs(args.workload, args.r)
    mesh, m, leaf, eta = w.mesh, w.m, w.leaf, w.eta
    import oracle
    oracle.build()
    o = oracle.H2Oracle(mesh.xyz, mesh.tri, m, leaf, eta)
    for _ in range(args.warmup):
        o.matvec(u1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.matvec(u1)
    el = time.perf_counter() - t0
    value = mesh.n_vertices * u1.shape[0] * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": mesh.n_vertices, "m": m, "leaf": leaf,
                       "eta": eta, "r": int(u1.shape[0]), "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} full H2 matvecs of the {args.workload} workload "
                                       f"(CPU oracle, plain C + OpenMP, FP64)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_form(pkg, torch, g, w, u1_np, precision, schedule, steps, warmup, barrier=None):
    """Builds the operator of one form and times `steps` matvecs with CUDA
    events on the launching stream (inputs resident in device memory)."""
    r = u1_np.shape[0]
    base = precision.split("-")[0]
    pair = precision.endswith("-pair") and r > 8   # the paired near field needs split-form products
    op = pkg.Operator(g, m=w.m, leaf=w.leaf, eta=w.eta, precision={"fp64": pkg.FP64, "fp32": pkg.FP32,
                      "tf32x3": pkg.TF32X3, "bf16x3": pkg.BF16X3}[base], max_rhs=r,
                      schedule=pkg.SCHEDULE_FLOW if schedule == "flow" else pkg.SCHEDULE_LEVELS,
                      coupling=pkg.COUPLING_ON_THE_FLY if precision == "fp32-onfly" else pkg.COUPLING_STORED,
                      near_field=pkg.NEAR_F32PAIR if pair else pkg.NEAR_FP64)
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    x = torch.from_numpy(u1_np).cuda()
    y = torch.empty_like(x)
    for _ in range(max(warmup, 3)):
        pkg.h2_matvec(op.handle, x.data_ptr(), y.data_ptr(), r, sp)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        pkg.h2_matvec(op.handle, x.data_ptr(), y.data_ptr(), r, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    status = pkg.h2_device_status(op.handle)
    if status != 0:
        raise RuntimeError(f"device-side wait gave up during the benchmark ({status})")
    return op, x, y, e0.elapsed_time(e1) / 1e3 / steps


def pass_profile(pkg, op, x, y, r, steps):
    """Per-launch CUDA-event times of `steps` matvecs (h2_profile_*)."""
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
        for i in range(nent.value):
            passes.append({"launch": i, "pass": PASS_NAMES.get(kind[i], str(kind[i])),
                           "ms": ms[i] / ncalls.value, "bytes": byt[i], "macs_per_rhs": macs[i],
                           "grid": grid[i]})
    return passes


def rel_err(y, ref):
    return float(np.max(np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def run_gpu(args, rank, local, world):
    import torch
    import paper_1811_05731_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    w, u1_np = workload_inputs(args.workload, args.r)
    mesh = w.mesh
    N = mesh.n_vertices
    r = u1_np.shape[0]
    g = pkg.Geometry(mesh.xyz, mesh.tri)

    def barrier():
        if dist is not None:
            dist.barrier()

    # headline form: device-resident inputs, K timed steps, clocks sampled meanwhile
    with ClockSampler(local) as clk:
        op, x, y, t_step = time_form(pkg, torch, g, w, u1_np, args.precision, args.schedule, args.steps,
                                     args.warmup, barrier)
    t_step = max_over_ranks(t_step, dist, "cuda")
    value = replica_rate(N * r, world, t_step)
    st = op.stats()
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)

    # end to end through the C ABI with pinned host buffers (copies in the timed region)
    xh = torch.from_numpy(u1_np).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        pkg.h2_matvec(op.handle, xh.data_ptr(), yh.data_ptr(), r, sp)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        pkg.h2_matvec(op.handle, xh.data_ptr(), yh.data_ptr(), r, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3 / args.steps, dist, "cuda")

    passes = pass_profile(pkg, op, x, y, r, args.steps)
    y_np = y.cpu().numpy()
    del op

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, peak_src = measured_peaks()
    clocks = clk.summary()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", HBM_GBS_FALLBACK))
    fp64_peak = N_SM * FP64_FMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    fp32_peak = N_SM * FP32_FMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12
    roofline = None

    def kname(p):
        return "k_seg dataflow (whole product)" if p["pass"] == "flow" else f"k_seg ({p['pass']})"

    if passes:
        dom = max(passes, key=lambda p: p["ms"])
        t = dom["ms"] / 1e3
        gbs = dom["bytes"] / t / 1e9
        flops = 2.0 * dom["macs_per_rhs"] * r
        alu_peak = fp64_peak if args.precision == "fp64" else fp32_peak
        tfl = flops / t / 1e12
        hbm_frac = gbs / hbm
        alu_frac = tfl / alu_peak
        if alu_frac > hbm_frac:
            roofline = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s",
                        "frac": alu_frac, "traffic": None,
                        "peak_source": f"{'FP64' if args.precision == 'fp64' else 'FP32'} FMA rate derived from "
                                       f"unit counts: {N_SM} SMs x "
                                       f"{FP64_FMA_PER_CLK_SM if args.precision == 'fp64' else FP32_FMA_PER_CLK_SM}"
                                       f" FMA/clk x 2 x {sm_max:.0f} MHz (microbenchmark: 1.257 TFLOP/s FP64)",
                        "kernel": kname(dom), "hbm_gbs": gbs, "hbm_frac_of_measured": hbm_frac}
        else:
            roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_frac,
                        "traffic": None, "peak_source": f"{peak_src} hbm_gbs",
                        "kernel": kname(dom), "alu_tflops": tfl, "alu_frac": alu_frac}
        # DRAM bytes per launch from an ncu capture (profiles/), used only while
        # the kernel source is the one that was captured
        tpath = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tpath):
            import hashlib
            with open(tpath) as f:
                tr = json.load(f)
            src = os.path.join(ROOT, "paper_1811_05731_gb300", "csrc", "h2_matvec.cu")
            with open(src, "rb") as f:
                sha = hashlib.sha1(f.read()).hexdigest()
            key = f"{args.workload}/{args.precision}/r{r}/{dom['pass']}"
            if key in tr and tr.get("kernel_source_sha1") == sha:
                roofline["traffic"] = tr[key]

    # the oracle (FP64, CPU) for relative errors, one product per r
    refs = {}
    oracle_obj = None
    if not args.no_errors:
        import oracle
        oracle.build()
        oracle_obj = oracle.H2Oracle(mesh.xyz, mesh.tri, w.m, w.leaf, w.eta)
        refs[r] = oracle_obj.matvec(u1_np)

    forms = []
    if not args.no_forms and world == 1:
        for prec, rr in [(args.precision, r)] + [f for f in FORMS if f != (args.precision, r)]:
            _, u = workload_inputs(args.workload, rr if rr > 1 else args.r)
            opf, xf, yf, tf = time_form(pkg, torch, g, w, u, prec, args.schedule, min(args.steps, 20), 3)
            ent = {"precision": prec, "r": int(u.shape[0]), "value": N * u.shape[0] / tf,
                   "ms_per_step": tf * 1e3, "dtype": DTYPES[prec]}
            if oracle_obj is not None:
                if u.shape[0] not in refs:
                    refs[u.shape[0]] = oracle_obj.matvec(u)
                ent["rel_err_vs_fp64_oracle"] = rel_err(yf.cpu().numpy(), refs[u.shape[0]])
            forms.append(ent)
            del opf
        fp64_1 = next((f["value"] for f in forms if f["precision"] == "fp64" and f["r"] == 1), None)
        for f in forms:
            if fp64_1:
                f["speedup_vs_fp64_r1"] = f["value"] / fp64_1
            same = next((e["value"] for e in forms if e["precision"] == "fp64" and e["r"] == f["r"]), None)
            if same:
                f["speedup_vs_fp64_same_r"] = f["value"] / same

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, cores, n, el, setup, y_ref = cpu_oracle_rate(mesh, w.m, w.leaf, w.eta, u1_np, args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} full H2 matvecs of the same workload in {el:.1f} s (oracle setup "
                         f"{setup:.1f} s not timed)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "triangles": mesh.n_triangles, "m": w.m,
                   "leaf": w.leaf, "eta": w.eta, "r": r, "precision": args.precision,
                   "schedule": args.schedule,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2: {st['bytes_streamed'] / 1e6:.0f} MB of matrices "
                         f"streamed per step (L2 129 MB), no flush"},
        "clocks": clocks,
        "e2e": {"value": replica_rate(N * r, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": 8 * N * r,
                "d2h_bytes_per_step": 8 * N * r},
        "gpu_launches": st["n_launches_matvec"] * args.steps,
        "rel_err_vs_fp64_oracle": rel_err(y_np, refs[r]) if r in refs else None,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "forms": forms,
        "passes": passes,
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
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="h2bem", choices=["h2bem", "reference"])
    ap.add_argument("--workload", default="cube64", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS))
    ap.add_argument("--r", type=int, default=0)
    ap.add_argument("--schedule", default="flow", choices=["flow", "levels"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the reduced-precision and batched forms")
    ap.add_argument("--no-errors", action="store_true", help="skip the relative errors against the oracle")
    args = ap.parse_args()
    rank, local, world = rank_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, local, world)


if __name__ == "__main__":
    main()
