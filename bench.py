#!/usr/bin/env python
"""Benchmark of the global stiffness-matrix build (integrate + assemble).

Workload: the 1M-brick mesh -- a 100^3 grid of 8-node trilinear bricks on the
unit cube (1,030,301 nodes), interior nodes jittered by +-0.25 h, random node and
element numbering, c_e ~ lognormal(0, 1), 2x2x2 Gauss (seeded synthetic data).
A step is one numeric build of the lower-CSR values of K with the pattern
cached (the symbolic phase is timed separately as the cold build).

`value` is elements/s of the mixed-precision build (FP32 with FP64 Jacobians for
distorted elements), inputs resident in HBM, L2 flushed before every step.
The FP64 build, the cold build and the end-to-end build through the host-buffer
C-ABI call are reported beside it.  Multi-GPU runs are independent replicas.
"""
import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "1M-hex8: 100^3 unit-cube bricks, jitter 0.25h, permuted, c~lognormal(0,1), 2x2x2 Gauss"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=100, help="grid cells per axis (100 = the 1M-brick workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the 512-mesh batched build and the 27M-brick budgeted build")
    ap.add_argument("--once", choices=["mixed", "fp64"], default=None,
                    help="profiling mode: build K twice in this precision and exit (no timing, no JSON)")
    ap.add_argument("--workload", choices=["hex", "tet"], default="hex",
                    help="--once only: the 1M-brick workload or the 3.07M-tet workload")
    ap.add_argument("--patch-entries", type=int, default=0, help="--once only: plan patch size (0 = default)")
    ap.add_argument("--block-threads", type=int, default=0, help="--once only: threads per block (0 = default)")
    ap.add_argument("--operator", choices=["stiffness", "elasticity"], default="stiffness",
                    help="--once only: the scalar stiffness matrix or the elasticity operator")
    ap.add_argument("--backward", action="store_true",
                    help="--once only: run the backward pass (fem_vjp, seeded upstream) instead of the build")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def init_dist(world):
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist
    return None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, n = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            n += 1
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": n}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources that determine the patch kernel's code and its plan's layout
KERNEL_SOURCES = ("element.cuh", "mesh.cuh", "numeric.cu", "numeric.cuh", "phases.cuh", "symbolic.cu")


def source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1501_04784_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel, {}).get(workload_key)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def algorithmic_bytes(n_nodes, n_elems, npe, nnz, xsize, csize, vsize):
    # coordinates + connectivity + c_e read, CSR values written
    return n_nodes * 3 * xsize + n_elems * npe * 4 + n_elems * csize + nnz * vsize


# FP32 FLOPs of one brick element in the sum-factorised form (an FMA counts 2):
# 12 edge vectors (36), Jacobian rows at the 8 points (216), per point cofactor
# rows, determinant, reciprocal, 6 Gram entries scaled (8 x 73 = 584), distortion
# test (17), axis sums (12), 3 diagonal-direction tables (120), 3 cross tables
# (300), 36 packed entries of 9 terms scaled by c/8 (648).
BRICK_FLOPS = 36 + 216 + 584 + 17 + 12 + 120 + 300 + 648
SMS, FP32_LANES = 152, 128

# FP32 FLOPs of one brick of the elasticity operator, lower triangle only (an FMA
# counts 2): 12 edge vectors (36); per Gauss point the 3 rows of 2J from the edges
# (81), cofactor rows (27), determinant (5), scale 1/(8|d|) (6) -> 8 x 119 = 952;
# gradient vectors of the 8 nodes (8 x 120 = 960) and their scaled copies
# (8 x 24 = 192); 36 blocks of 9 products accumulated (8 x 1296 = 10368); the
# Lame combination lambda P + mu P^T + mu tr(P) I of 36 blocks (36 x 33 = 1188).
ELASTIC_BRICK_FLOPS = 36 + 952 + 960 + 192 + 10368 + 1188


def cpu_baseline(m, target_s=12.0):
    """The FP64 oracle (Algorithm 1 as written, single thread) on a bounded sample
    of the workload's elements: whole passes over growing prefixes until ~target_s."""
    import numpy as np
    import oracle
    oracle.build()
    n = 4096
    spent = 0.0
    while True:
        t0 = time.perf_counter()
        oracle.build_K(m.npe, m.X, m.E[:n], m.c[:n])
        dt = time.perf_counter() - t0
        spent += dt
        if spent + 2.5 * dt > target_s or n >= m.n_elems:
            break
        n = min(2 * n, m.n_elems)
    return {"value": n / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {m.n_elems} elements of the workload: element loop + stable sort/reduce to CSR, FP64, 1 thread",
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_error(m, rowptr, col, builds, n_rows=2000, seed=12):
    """Accuracy of the timed builds, from the same leg as the CPU baseline: the
    oracle's exact rows of n_rows random nodes (all elements touching them), against
    each build, as the largest |K_ij - K*_ij| / sum_e sqrt(k_aa k_bb) (the per-entry
    Cauchy-Schwarz scale of the contributions).  builds = {name: (vals, X, c)},
    X and c as that build read them."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    rows = np.unique(rng.choice(m.n_nodes, n_rows, replace=False))
    touch = np.isin(m.E, rows).any(axis=1)
    rp, cl = rowptr, col
    out = {}
    for name, (vals, X, c) in builds.items():
        sub = oracle.build_K(m.npe, np.asarray(X, np.float64), m.E[touch], np.asarray(c, np.float64)[touch])
        worst = 0.0
        for r in rows:
            a, b = sub["rowptr"][r], sub["rowptr"][r + 1]
            g0, g1 = rp[r], rp[r + 1]
            if not np.array_equal(cl[g0:g1], sub["col"][a:b]):
                worst = float("inf")
                break
            err = np.abs(vals[g0:g1].astype(np.float64) - sub["vals"][a:b]) / np.maximum(sub["cs"][a:b], 1e-300)
            worst = max(worst, float(err.max()))
        out[name] = worst
    out["rows_sampled"] = int(len(rows))
    out["metric"] = "max |K - K_oracle| / sum_e sqrt(k_aa k_bb) over the sampled rows"
    return out


# --------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    import meshgen
    from paper_1501_04784_gb300 import _build, fem

    rank, world, local = dist_env()
    dist = init_dist(world)
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        _build.build()
    barrier(dist)

    m = meshgen.config_mesh(1, nx=args.n)
    E = torch.from_numpy(m.E).cuda()
    X64 = torch.from_numpy(m.X).cuda()
    c64 = torch.from_numpy(m.c).cuda()
    Xf, cf = X64.float(), c64.float()
    stream = torch.cuda.current_stream()

    # cold build: handle creation (validation + locality order) + symbolic + first numeric build
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh = fem.Mesh(E, m.n_nodes, X=X64)
    nnz = mesh.pattern()
    vals = torch.empty(nnz, dtype=torch.float32, device="cuda")
    mesh.build_K(Xf, cf, "mixed", out=vals)
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t0
    info = mesh.info()

    # tuner (untimed): assembly tile and threads per block on the real inputs
    tuning = mesh.autotune(Xf, cf, "mixed")
    info = mesh.info()
    vals = torch.empty(nnz, dtype=torch.float32, device="cuda")

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def timed(prec, X, c, out, steps, mh=None):
        mh = mh or mesh
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            mh.build_K(X, c, prec, out=out)
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    for _ in range(args.warmup):
        mesh.build_K(Xf, cf, "mixed", out=vals)
    torch.cuda.synchronize()

    clk = Clocks(local) if rank == 0 else None
    barrier(dist)
    torch.cuda.synchronize()
    fem.launch_count(reset=True)
    ms = timed("mixed", Xf, cf, vals, args.steps)
    launches = fem.launch_count()
    torch.cuda.synchronize()
    barrier(dist)
    clocks = clk.stop() if clk else None

    total_s = sum(ms) / 1e3
    max_total = max_over_ranks(dist, total_s)
    elems_all = sum_over_ranks(dist, float(m.n_elems * args.steps))
    value = elems_all / max_total
    ms_step = statistics.mean(ms)

    # FP64 build beside it
    vals64 = torch.empty(nnz, dtype=torch.float64, device="cuda")
    for _ in range(3):
        mesh.build_K(X64, c64, "fp64", out=vals64)
    steps64 = max(3, min(args.steps, 20))
    ms64 = timed("fp64", X64, c64, vals64, steps64)
    fp64_eps = m.n_elems / (statistics.mean(ms64) / 1e3)

    # the mass operator on the same mesh and tuned tile (Section 5's other matrix)
    mass_mesh = fem.Mesh(E, m.n_nodes, X=X64, operator_kind=1, patch_entries=tuning["patch_entries"],
                         block_threads=tuning["block_threads"])
    mass_mesh.pattern()
    for _ in range(3):
        mass_mesh.build_K(Xf, cf, "mixed", out=vals)
    ms_mass = timed("mixed", Xf, cf, vals, max(3, min(args.steps, 20)), mass_mesh)
    mass_mesh.close()

    # end to end through the host-buffer C-ABI call (pinned inputs and outputs)
    e2e = None
    if not args.no_e2e:
        Xh = Xf.cpu().pin_memory()
        ch = cf.cpu().pin_memory()
        vh = torch.empty(nnz, dtype=torch.float32).pin_memory()
        for _ in range(3):
            mesh.build_K_host(Xh, ch, "mixed", out=vh)
        ne = max(3, min(args.steps, 30))
        t0 = time.perf_counter()
        for _ in range(ne):
            mesh.build_K_host(Xh, ch, "mixed", out=vh)
        dt_serial = (time.perf_counter() - t0) / ne
        # the asynchronous host entry point on three streams (the mesh's three
        # staging slots): each step still copies its inputs in and its result
        # out, but a step's copy-in and build overlap the earlier steps' copy-out
        vh2 = [vh] + [torch.empty(nnz, dtype=torch.float32).pin_memory() for _ in range(2)]
        st2 = [torch.cuda.Stream() for _ in range(3)]
        for k in range(6):
            mesh.build_K_host_async(Xh, ch, "mixed", out=vh2[k % 3], stream=st2[k % 3])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(ne):
            mesh.build_K_host_async(Xh, ch, "mixed", out=vh2[k % 3], stream=st2[k % 3])
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / ne
        mesh.sync()
        # host-resident K: the kernel writes the values straight into the pinned
        # host buffer (the path a matrix larger than device memory takes)
        dmesh = fem.Mesh(E, m.n_nodes, X=X64, host_direct=1, patch_entries=tuning["patch_entries"],
                         block_threads=tuning["block_threads"])
        dmesh.pattern()
        for _ in range(3):
            dmesh.build_K_host(Xh, ch, "mixed", out=vh)
        t0 = time.perf_counter()
        for _ in range(ne):
            dmesh.build_K_host(Xh, ch, "mixed", out=vh)
        dt_direct = (time.perf_counter() - t0) / ne
        dmesh.close()
        e2e = {"value": m.n_elems / dt, "unit": "elements/s", "h2d_bytes_per_step": Xh.nbytes + ch.nbytes,
               "d2h_bytes_per_step": nnz * 4,
               "api": "fem_build_K_host_async, three streams (copy-in and build of a step overlap the earlier copy-outs)",
               "serial": {"value": m.n_elems / dt_serial, "api": "fem_build_K_host (synchronous)"},
               "host_resident": {"value": m.n_elems / dt_direct, "ms_per_step": dt_direct * 1e3,
                                 "api": "fem_build_K_host with host_direct: values written by the kernel into "
                                        "pinned host memory, no device copy of K"}}

    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(m.n_nodes, m.n_elems, 8, nnz, 4, 4, 4)
    alg64 = algorithmic_bytes(m.n_nodes, m.n_elems, 8, nnz, 8, 8, 8)
    achieved = alg / (ms_step / 1e3) / 1e9
    # the profiled DRAM traffic of the same kernel sources, workload and patch size
    wkey = f"hex8_n{args.n}_mixed_p{(tuning or {}).get('patch_entries', 0)}"
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12          # TFLOP/s at the sampled clock
    alu_achieved = BRICK_FLOPS * m.n_elems / (ms_step / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": round(alu_achieved, 3), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
            "frac": round(alu_achieved / alu_peak, 4), "traffic": profiled_traffic("k_patch", wkey),
            "peak_source": f"derived: {SMS} SMs x {FP32_LANES} FP32 lanes x 2 FLOP x {sm_mhz:.0f} MHz (sampled)",
            "kernel": "k_patch (fused integrate + assemble)", "flops_per_element": BRICK_FLOPS,
            "algorithmic_flops_per_launch": BRICK_FLOPS * m.n_elems,
            "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "peak_source": peak_kind, "algorithmic_bytes_per_launch": alg}}
    if roof["traffic"]:
        # DRAM bytes the kernel really moves (ncu) over the launch time measured here
        roof["hbm"]["dram_gbs"] = round(roof["traffic"] / (ms_step / 1e3) / 1e9, 1)
        roof["hbm"]["dram_frac"] = round(roof["hbm"]["dram_gbs"] / peak, 4)

    if rank == 0:
        out = {
            "metric": "global-K build elements/s (integrate+assemble), % HBM roofline, mixed vs FP64",
            "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f64 Jacobians of distorted elements)", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD if args.n == 100 else f"{args.n}^3 bricks", "n_elems": m.n_elems,
                       "n_nodes": m.n_nodes, "nnz": nnz, "precision": "mixed", "pattern": "cached",
                       "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) before every step"},
            "hbm_frac": round(achieved / peak, 4),
            "fp64": {"value": fp64_eps, "unit": "elements/s", "ms_per_step": statistics.mean(ms64),
                     "hbm_frac": round(alg64 / (statistics.mean(ms64) / 1e3) / 1e9 / peak, 4),
                     "mixed_speedup": value / world / fp64_eps},
            "mass": {"value": m.n_elems / (statistics.mean(ms_mass) / 1e3), "unit": "elements/s",
                     "ms_per_step": statistics.mean(ms_mass), "operator": "consistent mass matrix, mixed"},
            "cold_build": {"value": m.n_elems / cold_s, "unit": "elements/s", "seconds": cold_s,
                           "includes": "validation, locality order, pattern, plan, first numeric build"},
            "plan": {k: info[k] for k in ("n_patches", "closure_elems", "n_colors", "plan_bytes")},
            "tuning": tuning,
            "roofline": roof, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        }
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(m)
            rowptr, col = mesh.get_pattern()
            mesh.build_K(Xf, cf, "mixed", out=vals)  # vals held the mass matrix since
            out["error"] = oracle_error(m, rowptr.cpu().numpy(), col.cpu().numpy(), {
                "mixed": (vals.cpu().numpy(), m.X.astype(np.float32), m.c.astype(np.float32)),
                "fp64": (vals64.cpu().numpy(), m.X, m.c)})
    mesh.close()
    if not args.no_workloads:
        extra = other_workloads(flush, stream)
        if rank == 0:
            out["workloads"] = extra
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


# -------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle (the plain FP64 CPU program of Algorithm 1) on the host cores,
    each step one bounded slice of the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import meshgen
    import oracle
    oracle.build()
    m = meshgen.config_mesh(1, nx=args.n)
    per_step = 8192
    off = 0

    def step():
        nonlocal off
        lo = off % max(1, m.n_elems - per_step)
        oracle.build_K(m.npe, m.X, m.E[lo:lo + per_step], m.c[lo:lo + per_step])
        off += per_step

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": "global-K build elements/s (integrate+assemble), % HBM roofline, mixed vs FP64",
        "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD if args.n == 100 else f"{args.n}^3 bricks", "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} consecutive elements of the workload per step (rotating)"},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def other_workloads(flush, stream):
    """The batched and the large workload beside the headline (mixed precision, pattern
    cached, L2 flushed before every timed build): 512 uneven brick meshes in one
    persistent launch replayed from a CUDA graph, and 300^3 bricks built in patch
    groups under a 16 GB library budget, with its backward pass."""
    import numpy as np
    import torch

    import meshgen
    from paper_1501_04784_gb300 import fem

    def dev(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt)

    def timed(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return statistics.median([a.elapsed_time(b) for a, b in evs])

    out = {}
    ms = meshgen.batch_meshes()
    meshes = [fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64)) for m in ms]
    Xs = [dev(m.X, torch.float32) for m in ms]
    cs = [dev(m.c, torch.float32) for m in ms]
    vals = [torch.empty(mesh.pattern(), dtype=torch.float32, device="cuda") for mesh in meshes]
    nel = sum(m.n_elems for m in ms)
    t = timed(lambda: fem.build_K_batched(meshes, Xs, cs, "mixed", out=vals), 10)
    out["batched"] = {"workload": f"{len(ms)} uneven brick meshes, {nel} elements, one graph launch",
                      "value": nel / (t / 1e3), "unit": "elements/s", "ms_per_step": t,
                      "launch": fem.batched_config(meshes, "mixed")}
    for mesh in meshes:
        mesh.close()
    del meshes, Xs, cs, vals
    m = meshgen.config_mesh(4)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), mem_budget_bytes=16 << 30)
    nnz = mesh.pattern()
    X, c = dev(m.X, torch.float32), dev(m.c, torch.float32)
    v = torch.empty(nnz, dtype=torch.float32, device="cuda")
    t = timed(lambda: mesh.build_K(X, c, "mixed", out=v), 3)
    info = mesh.info()
    out["large"] = {"workload": "300^3 bricks (27M elements), 16 GB library budget", "value": m.n_elems / (t / 1e3),
                    "unit": "elements/s", "ms_per_step": t, "patch_groups": info["n_groups"],
                    "plan_bytes": info["plan_bytes"]}
    # its backward: dL/dX (FP32) and dL/dc of L = sum G_ij K_ij, G seeded standard normal
    G = torch.randn(nnz, generator=torch.Generator(device="cuda").manual_seed(21), device="cuda")
    tb = timed(lambda: mesh.vjp(X, c, G, "mixed"), 3)
    mesh.sync()
    out["large"]["backward"] = {"value": m.n_elems / (tb / 1e3), "unit": "elements/s", "ms_per_step": tb,
                                "library_bytes": mesh.info()["live_bytes"]}
    mesh.close()
    del mesh, X, c, v, G
    out["elastic"] = elastic_workloads(timed, dev)
    out["backward"] = backward_workloads(timed, dev)
    return out


def backward_workloads(timed, dev):
    """The backward pass (fem_vjp: dL/dX and dL/dc of L = sum over stored entries
    G_ij K_ij) on the 1M-brick mesh, for the stiffness operator in both precisions
    and for the elasticity and mass operators in mixed precision, and on the
    3.07M-tet mesh for the stiffness and elasticity operators in mixed precision; G is a seeded standard
    normal upstream on K's pattern.  Algorithmic bytes: X, E, c and G read once,
    dX and dc written once."""
    import numpy as np
    import torch

    import meshgen
    from paper_1501_04784_gb300 import fem

    res = {}
    for op, key, idx in ((0, "stiffness", 1), (2, "elasticity", 1), (1, "mass", 1), (0, "stiffness_tet", 2),
                         (2, "elasticity_tet", 2)):
        m = meshgen.config_mesh(idx)
        mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), operator_kind=op)
        nnz = mesh.pattern()
        c = meshgen.lame(m) if op == 2 else m.c
        G = np.random.default_rng(21).standard_normal(nnz)
        name = "1M-hex8 " if idx == 1 else "3.07M-tet4 "
        r = {"workload": name + key.split("_")[0] + " backward (dL/dX, dL/dc)", "nnz": nnz}
        for prec in (("mixed", "fp64") if key == "stiffness" else ("mixed",)):
            dt = torch.float32 if prec == "mixed" else torch.float64
            w = 4 if prec == "mixed" else 8
            X, cd, Gd = dev(m.X, dt), dev(c, dt), dev(G, dt)
            t = timed(lambda: mesh.vjp(X, cd, Gd, prec), 10)
            mesh.sync()
            nb = (m.n_nodes * 3 * w * 2 + m.n_elems * m.npe * 4 + cd.numel() * w * 2 + nnz * w)
            r[prec] = {"value": m.n_elems / (t / 1e3), "unit": "elements/s", "ms_per_step": t,
                       "algorithmic_bytes": nb, "achieved_gbs": nb / (t / 1e3) / 1e9}
            del X, cd, Gd
        res[key] = r
        mesh.close()
        del mesh
    return res


def elastic_workloads(timed, dev):
    """The elasticity operator (three DOFs per node, operator_kind 2) on the 1M-brick
    mesh (mixed and FP64) and the 3.07M-tet mesh (mixed): Lame parameters from a
    seeded Poisson ratio in [0.1, 0.45] and Young's modulus c_e."""
    import torch

    import meshgen
    from paper_1501_04784_gb300 import fem

    res = {}
    for key, idx in (("hex", 1), ("tet", 2)):
        m = meshgen.config_mesh(idx)
        lame = meshgen.lame(m)
        mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), operator_kind=2)
        nnz = mesh.pattern()
        X, c = dev(m.X, torch.float32), dev(lame, torch.float32)
        v = torch.empty(nnz, dtype=torch.float32, device="cuda")
        t = timed(lambda: mesh.build_K(X, c, "mixed", out=v), 10)
        mesh.sync()
        r = {"workload": ("1M-hex8" if idx == 1 else "3.07M-tet4") + " elasticity, 3 DOFs per node",
             "value": m.n_elems / (t / 1e3), "unit": "elements/s", "ms_per_step": t, "nnz": nnz,
             "dof_entries_per_s": nnz / (t / 1e3), "n_patches": mesh.info()["n_patches"],
             "closure_elems": mesh.info()["closure_elems"]}
        if idx == 1:
            r["alu"] = {"flops_per_element": ELASTIC_BRICK_FLOPS,
                        "achieved_tflops": ELASTIC_BRICK_FLOPS * m.n_elems / (t / 1e3) / 1e12,
                        "frac_of_fp32_peak_2070mhz": ELASTIC_BRICK_FLOPS * m.n_elems / (t / 1e3)
                        / (SMS * FP32_LANES * 2 * 2070e6)}
            X64, c64 = dev(m.X, torch.float64), dev(lame, torch.float64)
            v64 = torch.empty(nnz, dtype=torch.float64, device="cuda")
            t64 = timed(lambda: mesh.build_K(X64, c64, "fp64", out=v64), 3)
            mesh.sync()
            r["fp64"] = {"value": m.n_elems / (t64 / 1e3), "unit": "elements/s", "ms_per_step": t64}
            del X64, c64, v64
        res[key] = r
        mesh.close()
        del mesh, X, c, v
    return res


def run_once(args):
    """Two builds of one workload, for a profiler to capture the second one."""
    import torch

    import meshgen
    from paper_1501_04784_gb300 import _build, fem
    _build.build()
    m = meshgen.config_mesh(1 if args.workload == "hex" else 2)
    E = torch.from_numpy(m.E).cuda()
    elastic = args.operator == "elasticity"
    X64 = torch.from_numpy(m.X).cuda()
    c64 = torch.from_numpy(meshgen.lame(m) if elastic else m.c).cuda()
    mesh = fem.Mesh(E, m.n_nodes, X=X64, patch_entries=args.patch_entries, block_threads=args.block_threads,
                    operator_kind=2 if elastic else 0)
    nnz = mesh.pattern()
    X, c = (X64.float(), c64.float()) if args.once == "mixed" else (X64, c64)
    v = torch.empty(nnz, dtype=X.dtype, device="cuda")
    if args.backward:
        import numpy as np
        G = torch.from_numpy(np.random.default_rng(21).standard_normal(nnz)).cuda().to(X.dtype)
    for _ in range(2):
        if args.backward:
            mesh.vjp(X, c, G, args.once)
        else:
            mesh.build_K(X, c, args.once, out=v)
    torch.cuda.synchronize()
    mesh.sync()
    what = "backward" if args.backward else "built"
    print(f"{what} {args.workload} {args.operator} {args.once}: nnz {nnz}, patches {mesh.info()['n_patches']}")


if __name__ == "__main__":
    a = parse()
    if a.once:
        run_once(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
