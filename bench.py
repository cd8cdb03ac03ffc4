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

WORKLOADS = {
    # name: (mesh builder, m, leaf, eta, r, rhs builder)
    "cube64": (lambda: synth.cube_surface(64), 4, 64, 2.0, 1,
               lambda mesh, r: synth.normal_dot_field(mesh, 1811)),
    "ico3": (lambda: synth.icosphere(3), 3, 32, 2.0, 1,
             lambda mesh, r: synth.gaussian_rhs(mesh.n_vertices, r, 1811)),
}


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


def run_reference(args, rank, world):
    if rank != 0:
        return
    build, m, leaf, eta, r, rhs = WORKLOADS[args.workload]
    mesh = build()
    u1 = np.atleast_2d(rhs(mesh, r))
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


def run_gpu(args, rank, local, world):
    import torch
    import paper_1811_05731_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    build, m, leaf, eta, r, rhs = WORKLOADS[args.workload]
    if args.r:
        r = args.r
    mesh = build()
    N = mesh.n_vertices
    u1_np = np.ascontiguousarray(np.atleast_2d(rhs(mesh, r)), dtype=np.float64)
    r = u1_np.shape[0]
    prec = pkg.FP32 if args.precision == "fp32" else pkg.FP64
    g = pkg.Geometry(mesh.xyz, mesh.tri)
    op = pkg.Operator(g, m=m, leaf=leaf, eta=eta, precision=prec, max_rhs=r,
                      schedule=pkg.SCHEDULE_FLOW if args.schedule == "flow" else pkg.SCHEDULE_LEVELS)
    st = op.stats()
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    x = torch.from_numpy(u1_np).cuda()
    y = torch.empty_like(x)

    def step():
        pkg.h2_matvec(op.handle, x.data_ptr(), y.data_ptr(), r, sp)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # device-timed region (matrices streamed per step exceed the L2 cache)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    t_step = e0.elapsed_time(e1) / 1e3 / args.steps
    if dist is not None:
        t = torch.tensor([t_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    value = N * r * world / t_step

    # end to end through the C ABI with pinned host buffers
    xh = torch.from_numpy(u1_np).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        pkg.h2_matvec(op.handle, xh.data_ptr(), yh.data_ptr(), r, sp)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        pkg.h2_matvec(op.handle, xh.data_ptr(), yh.data_ptr(), r, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3 / args.steps
    if dist is not None:
        t = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())

    # per-pass CUDA-event timing over a second run of the same K steps
    import ctypes
    L = pkg.load()
    L.h2_profile_enable(ctypes.c_void_p(op.handle), 1)
    for _ in range(args.steps):
        step()
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
    y_np = y.cpu().numpy()

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
    # group launches by pass kind; the dominant kind is the one with most time
    by_kind = {}
    for p in passes:
        d = by_kind.setdefault(p["pass"], {"ms": 0.0, "bytes": 0, "macs": 0, "launches": 0})
        d["ms"] += p["ms"]
        d["bytes"] += p["bytes"]
        d["macs"] += p["macs_per_rhs"]
        d["launches"] += 1
    def kname(p):
        return "k_flow (whole product)" if p["pass"] == "flow" else f"k_pass ({p['pass']})"

    if passes:
        dom = max((p for p in passes), key=lambda p: p["ms"])
        t = dom["ms"] / 1e3
        gbs = dom["bytes"] / t / 1e9
        flops = 2.0 * dom["macs_per_rhs"] * r
        alu_peak = fp64_peak if prec == pkg.FP64 else fp32_peak
        tfl = flops / t / 1e12
        hbm_frac = gbs / hbm
        alu_frac = tfl / alu_peak
        if alu_frac > hbm_frac:
            roofline = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s",
                        "frac": alu_frac, "traffic": None,
                        "peak_source": f"{'FP64' if prec == pkg.FP64 else 'FP32'} FMA rate: "
                                       f"{N_SM} SMs x {FP64_FMA_PER_CLK_SM if prec == pkg.FP64 else FP32_FMA_PER_CLK_SM}"
                                       f" FMA/clk x 2 x {sm_max:.0f} MHz",
                        "kernel": kname(dom), "hbm_gbs": gbs, "hbm_frac_of_measured": hbm_frac}
        else:
            roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_frac,
                        "traffic": None, "peak_source": f"{peak_src} hbm_gbs",
                        "kernel": kname(dom), "alu_tflops": tfl, "alu_frac": alu_frac}
        tpath = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tpath):
            with open(tpath) as f:
                tr = json.load(f)
            key = f"{args.workload}/{args.precision}/r{r}/{dom['pass']}"
            if key in tr:
                roofline["traffic"] = tr[key]

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, cores, n, el, setup, y_ref = cpu_oracle_rate(mesh, m, leaf, eta, u1_np, args.cpu_budget)
        err = float(np.max(np.linalg.norm(y_np - y_ref, axis=1) / np.linalg.norm(y_ref, axis=1)))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} full H2 matvecs of the same workload in {el:.1f} s (oracle setup "
                         f"{setup:.1f} s not timed)",
               "rel_err_gpu_vs_oracle": err}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == pkg.FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "triangles": mesh.n_triangles, "m": m,
                   "leaf": leaf, "eta": eta, "r": r, "precision": args.precision,
                   "schedule": args.schedule,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2: {st['bytes_streamed'] / 1e6:.0f} MB of matrices "
                         f"streamed per step (L2 129 MB), no flush"},
        "clocks": clocks,
        "e2e": {"value": N * r * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * N * r,
                "d2h_bytes_per_step": 8 * N * r},
        "gpu_launches": st["n_launches_matvec"] * args.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
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
    ap.add_argument("--workload", default="cube64", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--r", type=int, default=0)
    ap.add_argument("--schedule", default="flow", choices=["flow", "levels"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank, local, world = rank_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, local, world)


if __name__ == "__main__":
    main()
