"""Benchmark: reassembly of M, K(u) and the Newton tangent T(u) into CSR on
GB300, elements per second.

One step = one reassembly of all three matrices (element formation V = X Q
on the tensor cores + the deterministic segmented CSR sum) for a fresh
nodal field u, with the mesh geometry and the CSR pattern cached (they are
computed once per mesh and reported separately).  Workload: the unit square
1024 x 1024 grid of 2 097 152 jittered P2 triangles, 6-point degree-4 rule,
k(u) = 1 + u^2, u a smooth 8-mode random Fourier field; synthetic, seeded.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N>1) every rank reassembles its own mesh (independent
problems, no data-path collective; weak scaling); rank 0 prints one JSON line.
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

import meshgen as mg  # noqa: E402

METRIC = "K(u)+M reassembly elements/s, % HBM/TC roofline; served p50/p99 latency"
WORKLOAD = "tri_p2_1024"
WORKLOAD_DESC = ("unit square 1024x1024 grid, 2,097,152 P2 triangles (6 dofs/elem, 4,198,401 dofs), "
                 "jitter 0.2h, 6-point degree-4 rule, u = 8-mode Fourier field, k(u) = 1 + u^2; "
                 "M, K(u) and tangent T(u) reassembled into CSR (nnz 48,250,881) per step")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32x3", choices=["tf32x3", "fp32", "fp64"])
    ap.add_argument("--scale", type=int, default=None, help="override grid size N (not a bench line)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, f in enumerate(fl) if f.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def kernel_traffic(kernel: str, src: str):
    """DRAM bytes per launch from a committed ncu summary, only if the
    kernel's source is unchanged since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2204_03893_gb300", "csrc", src), "rb").read()).hexdigest()[:16]
    if d.get("src_sha") != h:
        return None
    return d.get("bytes_per_launch")


def cpu_baseline_oracle(budget_s: float = 12.0):
    """The oracle (single-threaded C, Algorithm 1) reassembling M, K, T on a
    bounded sample of the same recipe: a 256x256-cell P2 triangle mesh."""
    import oracle as orc
    wl = mg.workload(WORKLOAD, scale=256)
    o = orc.Oracle.of(wl.mesh)
    o.nnz()   # pattern once (not timed: cached like the GPU pattern)
    t0 = time.perf_counter()
    n = 0
    while True:
        o.assemble(wl.u, wl.coeff, want_abs=False)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n * wl.mesh.n_elems / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} reassemblies of M,K,T on tri_p2 N=256 ({wl.mesh.n_elems} elements), "
                      f"pattern cached, {dt:.1f} s single-threaded"}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle as orc
    # size each step so that warmup + steps take about a minute
    probe = mg.workload(WORKLOAD, scale=16)
    po = orc.Oracle.of(probe.mesh)
    po.nnz()
    t0 = time.perf_counter()
    po.assemble(probe.u, probe.coeff, want_abs=False)
    rate = probe.mesh.n_elems / max(time.perf_counter() - t0, 1e-6)
    per_step = 60.0 / max(args.steps + args.warmup, 1)
    N = int(max(4, min(256, (per_step * rate / 2.0) ** 0.5)))
    wl = mg.workload(WORKLOAD, scale=N)
    o = orc.Oracle.of(wl.mesh)
    o.nnz()
    for _ in range(args.warmup):
        o.assemble(wl.u, wl.coeff, want_abs=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.assemble(wl.u, wl.coeff, want_abs=False)
    dt = time.perf_counter() - t0
    val = args.steps * wl.mesh.n_elems / dt
    line = {"metric": METRIC, "value": val, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "sample_N": N,
                       "sample_elements": wl.mesh.n_elems},
            "cpu_baseline": {"value": val, "unit": "elements/s", "cores": 1, "kind": "oracle",
                             "sample": f"tri_p2 N={N} ({wl.mesh.n_elems} elements) per step, pattern cached"},
            "e2e": {"value": val, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2204_03893_gb300 as F
    from paper_2204_03893_gb300 import build as fbuild
    from paper_2204_03893_gb300.torch_api import PRECISIONS, FemMesh

    fbuild.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    wl = mg.workload(WORKLOAD, scale=args.scale)
    E = wl.mesh.n_elems
    prec = PRECISIONS[args.prec]
    dt = torch.float64 if args.prec == "fp64" else torch.float32
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        fm = FemMesh.of(wl.mesh, stream=stream)
        torch.cuda.synchronize()
        t_mesh = time.perf_counter() - t0
        t0 = time.perf_counter()
        fm.symbolic()
        torch.cuda.synchronize()
        t_sym = time.perf_counter() - t0
        nnz = fm.nnz
        # a ring of nodal fields (fresh u every step, resident in HBM)
        us = [torch.tensor(mg.fourier_field(wl.mesh.coords, 1000 + 97 * rank + s), dtype=torch.float64,
                           device="cuda") for s in range(4)]
        out = {k: torch.empty(nnz, dtype=dt, device="cuda") for k in "MKT"}
        k = F.coeff(wl.coeff.kind, wl.coeff.params)
        which = F.FEM_MAT_M | F.FEM_MAT_K | F.FEM_MAT_T

        def step(i, ev=None):
            if ev is not None:
                ev[0].record(stream)
            F.fem_form_elements(fm.h, k, us[i % len(us)], prec, which, sh)
            if ev is not None:
                ev[1].record(stream)
            F.fem_sum_elements(fm.h, prec, out["M"], out["K"], out["T"], sh)
            if ev is not None:
                ev[2].record(stream)

        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize()
        F.fem_device_status(sh)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as clk:
            t_start = torch.cuda.Event(enable_timing=True)
            t_end = torch.cuda.Event(enable_timing=True)
            t_start.record(stream)
            for i in range(args.steps):
                step(i, evs[i])
            t_end.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        F.fem_device_status(sh)
        total_ms = t_start.elapsed_time(t_end)
        form_ms = [e[0].elapsed_time(e[1]) for e in evs]
        sum_ms = [e[1].elapsed_time(e[2]) for e in evs]
        if dist:
            tt = torch.tensor([total_ms], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            total_ms = float(tt.item())
        ms_per_step = total_ms / args.steps
        value = world * E * args.steps / (total_ms / 1e3)

        # FP64 plain path on the same workload (one-matrix-at-a-time reference point)
        fp64 = None
        if not args.no_fp64 and args.prec != "fp64":
            u64 = torch.tensor(wl.u, dtype=torch.float64, device="cuda")
            o64 = {kk: torch.empty(nnz, dtype=torch.float64, device="cuda") for kk in "MKT"}
            for _ in range(2):
                F.fem_assemble_mass(fm.h, F.FEM_FP64, o64["M"], sh)
                F.fem_assemble_stiffness(fm.h, k, u64, F.FEM_FP64, o64["K"], sh)
                F.fem_assemble_tangent(fm.h, k, u64, F.FEM_FP64, o64["T"], sh)
            torch.cuda.synchronize()
            n64 = 5
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(n64):
                F.fem_assemble_mass(fm.h, F.FEM_FP64, o64["M"], sh)
                F.fem_assemble_stiffness(fm.h, k, u64, F.FEM_FP64, o64["K"], sh)
                F.fem_assemble_tangent(fm.h, k, u64, F.FEM_FP64, o64["T"], sh)
            b.record(stream)
            torch.cuda.synchronize()
            ms64 = a.elapsed_time(b) / n64
            fp64 = {"value": E / (ms64 / 1e3), "unit": "elements/s", "ms_per_step": ms64,
                    "mode": "FEM_FP64 SIMT, one matrix per call (3 calls, 6 launches)"}
            del o64

        # end to end through the C ABI with pinned host buffers
        e2e = None
        if not args.no_e2e:
            uh = [torch.empty(wl.mesh.n_nodes, dtype=torch.float64, pin_memory=True) for _ in range(2)]
            for i, x in enumerate(uh):
                x.copy_(us[i].cpu())
            oh = {kk: torch.empty(nnz, dtype=dt, pin_memory=True) for kk in "MKT"}
            n_e2e = max(3, min(args.steps, 20))
            F.fem_assemble_all(fm.h, k, uh[0], prec, oh["M"], oh["K"], oh["T"], sh)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(n_e2e):
                F.fem_assemble_all(fm.h, k, uh[i % 2], prec, oh["M"], oh["K"], oh["T"], sh)
            torch.cuda.synchronize()
            te = time.perf_counter() - t0
            esz = 8 if args.prec == "fp64" else 4
            e2e = {"value": world * E * n_e2e / te, "unit": "elements/s", "steps": n_e2e,
                   "h2d_bytes_per_step": wl.mesh.n_nodes * 8, "d2h_bytes_per_step": 3 * nnz * esz,
                   "api": "fem_assemble_all with pinned host u and host CSR values (library-staged copies)"}

    if rank != 0:
        return 0

    # roofline of the dominant kernel (algorithmic bytes per launch / mean launch time)
    n_p, nsym, nt = 6, 21, 36
    esz = 8 if args.prec == "fp64" else 4
    n = wl.mesh.n_nodes
    bytes_form = E * (n_p * 4 + (1 + 3) * esz + (2 * nsym + nt) * esz) + n * 8
    bytes_sum = (nnz + 1) * 4 + E * n_p * n_p * 4 + E * (2 * nsym + nt) * esz + 3 * nnz * esz
    mf, ms = statistics.mean(form_ms), statistics.mean(sum_ms)
    kernels = {
        "element_form": {"kernel": "element_tc_kernel" if args.prec == "tf32x3" else "element_simt_kernel",
                         "src": "element_tc.cu" if args.prec == "tf32x3" else "element_simt.cu",
                         "ms": mf, "bytes": bytes_form},
        "csr_sum": {"kernel": "scatter_kernel", "src": "scatter.cu", "ms": ms, "bytes": bytes_sum},
    }
    dom = max(kernels.values(), key=lambda d: d["ms"])
    peak, peak_kind = measured_peaks()
    achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
    traffic = kernel_traffic(dom["kernel"] + ":" + args.prec, dom["src"])
    roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": achieved, "peak": peak,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs copy)" if peak_kind == "measured" else peak_kind,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": dom["bytes"]}
    phases = {name: {"ms": d["ms"], "GB/s": d["bytes"] / (d["ms"] / 1e3) / 1e9,
                     "frac_hbm": d["bytes"] / (d["ms"] / 1e3) / 1e9 / peak} for name, d in kernels.items()}

    cpu = None if args.no_cpu_baseline else cpu_baseline_oracle()
    line = {
        "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.scale is None else f"{WORKLOAD}@N={args.scale}",
                   "desc": WORKLOAD_DESC, "precision": args.prec,
                   "element_product": "tcgen05 kind::tf32 x3 (Xhi Qhi + Xhi Qlo + Xlo Qhi), FP32 accumulate in TMEM"
                   if args.prec == "tf32x3" else args.prec,
                   "elements": E, "nnz": nnz, "l2": "inputs larger than L2 (per-step traffic > 2 GB; no explicit flush)",
                   "parallelism": f"{world} independent meshes, one per GPU" if world > 1 else "single GPU"},
        "roofline": roofline, "phases": phases,
        "setup_once_per_mesh_ms": {"mesh_create_geometry": 1e3 * t_mesh, "symbolic_pattern": 1e3 * t_sym},
        "cpu_baseline": cpu, "e2e": e2e, "fp64_plain": fp64, "clocks": clk.summary(),
        "gpu_launches": 2 * args.steps,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.impl == "reference" else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
