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
    ap.add_argument("--tile-elems", type=int, default=0, help="--once only: elements per tile (0 = default)")
    ap.add_argument("--assembly", type=int, default=-1,
                    help="--once only: 0 = element tiles, 1 = node patches (-1 = the library's default)")
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
KERNEL_SOURCES = ("element.cuh", "elem_ops.cuh", "mesh.cuh", "tile.cuh", "numeric.cu", "numeric.cuh", "phases.cuh",
                  "symbolic.cu", "tile.cu", "tile_plan.cu")


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


# The oracle's sample, shared by the reference arm and the CPU baseline: rotating
# slices of SAMPLE_ELEMS consecutive elements of the workload, each slice built
# end to end (element loop, stable sort, reduction to CSR) in FP64 on one thread.
SAMPLE_ELEMS = 8192


def oracle_slice(m, k):
    import oracle
    lo = (k * SAMPLE_ELEMS) % max(1, m.n_elems - SAMPLE_ELEMS)
    oracle.build_K(m.npe, m.X, m.E[lo:lo + SAMPLE_ELEMS], m.c[lo:lo + SAMPLE_ELEMS])


def cpu_baseline(m, target_s=12.0):
    """The FP64 oracle (Algorithm 1 as written, single thread) on the shared sample:
    slices until about target_s seconds of work."""
    import oracle
    oracle.build()
    oracle_slice(m, 0)
    k, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < target_s:
        oracle_slice(m, k)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k * SAMPLE_ELEMS / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} rotating slices of {SAMPLE_ELEMS} consecutive elements (the reference arm's steps), "
                      "each built end to end (element loop, stable sort, reduction to CSR), FP64, 1 thread",
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


def sampled_error(m, rowptr, col, vals, X, c, n_rows=2000, seed=12):
    """Accuracy of one build against the oracle's exact rows of n_rows random nodes
    (the oracle run on every element touching them; X and c as the build read
    them).  Three measures, each the largest over the sampled entries:
      r13   |K - K*| / sum_e sqrt(k_aa k_bb)   (the per-entry scale the tests gate on)
      c14   |K - K*| / sum_e |k_ab|            (the sum of |contributions|)
      plain |K - K*| / |K*| on entries with |K*| >= 1e-3 of their r13 scale.
    An entry whose column differs from the oracle's makes every measure inf."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    rows = np.unique(rng.choice(m.n_nodes, min(n_rows, m.n_nodes), replace=False))
    touch = np.isin(m.E, rows).any(axis=1)
    sub = oracle.build_K(m.npe, np.asarray(X, np.float64), m.E[touch], np.asarray(c, np.float64)[touch])
    idx_g, idx_o = [], []
    for r in rows:
        a, b = sub["rowptr"][r], sub["rowptr"][r + 1]
        g0, g1 = rowptr[r], rowptr[r + 1]
        if not np.array_equal(col[g0:g1], sub["col"][a:b]):
            return {"r13": float("inf"), "c14": float("inf"), "plain": float("inf"), "rows": int(len(rows))}
        idx_g.append(np.arange(g0, g1))
        idx_o.append(np.arange(a, b))
    ig, io = np.concatenate(idx_g), np.concatenate(idx_o)
    got = np.asarray(vals, np.float64)[ig]
    ref, cs, ab = sub["vals"][io], sub["cs"][io], sub["abs"][io]
    d = np.abs(got - ref)
    keep = np.abs(ref) >= 1e-3 * cs
    return {"r13": float((d / np.maximum(cs, 1e-300)).max()), "c14": float((d / np.maximum(ab, 1e-300)).max()),
            "plain": float((d[keep] / np.abs(ref[keep])).max()) if keep.any() else 0.0, "rows": int(len(rows))}


def sig(x, n=4):
    """x rounded to n significant digits (keeps the JSON line short)."""
    if isinstance(x, float) and x == x and x not in (float("inf"), float("-inf")) and x != 0.0:
        from math import floor, log10
        return round(x, n - 1 - int(floor(log10(abs(x)))))
    return x


def compact(d):
    if isinstance(d, dict):
        return {k: compact(v) for k, v in d.items()}
    if isinstance(d, (list, tuple)):
        return [compact(v) for v in d]
    return sig(d)


# --------------------------------------------------------------- our arm
def median_ms(fn, n, flush, stream):
    """Median of n device times of fn (CUDA events on the launching stream), each
    after a 256 MB write that flushes the L2."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median([a.elapsed_time(b) for a, b in evs])


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

    # Process warm-up: a small mesh through the same calls, so that the cold build
    # below is that of a mesh the library has not seen, not the one-time loading of
    # the library's kernels (reported separately as first_in_process_s).
    sm = meshgen.config_mesh(1, nx=12)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    wmesh = fem.Mesh(torch.from_numpy(sm.E).cuda(), sm.n_nodes, X=torch.from_numpy(sm.X).cuda())
    wv = torch.empty(wmesh.pattern(), dtype=torch.float32, device="cuda")
    wmesh.build_K(torch.from_numpy(sm.X).float().cuda(), torch.from_numpy(sm.c).float().cuda(), "mixed", out=wv)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    wmesh.close()
    del wv

    # cold build: handle creation (validation + locality order) + symbolic + first numeric build
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh = fem.Mesh(E, m.n_nodes, X=X64)
    nnz = mesh.pattern()
    vals = torch.empty(nnz, dtype=torch.float32, device="cuda")
    mesh.build_K(Xf, cf, "mixed", out=vals)
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t0

    # tuner (untimed): work unit and threads per block on the real inputs
    tuning = mesh.autotune(Xf, cf, "mixed")
    info = mesh.info()
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

    ms_step = statistics.median(ms)
    max_step = max_over_ranks(dist, ms_step)
    elems_all = sum_over_ranks(dist, float(m.n_elems))
    value = elems_all / (max_step / 1e3)

    # FP64 build beside it
    vals64 = torch.empty(nnz, dtype=torch.float64, device="cuda")
    for _ in range(3):
        mesh.build_K(X64, c64, "fp64", out=vals64)
    ms64 = statistics.median(timed("fp64", X64, c64, vals64, max(5, min(args.steps, 20))))
    fp64_eps = m.n_elems / (ms64 / 1e3)

    # the mass operator on the same mesh and tuning (Section 5's other matrix)
    mass_mesh = fem.Mesh(E, m.n_nodes, X=X64, operator_kind=1)
    mass_mesh.pattern()
    mass_mesh.set_tuning(tuning["patch_entries"], tuning["block_threads"])
    for _ in range(3):
        mass_mesh.build_K(Xf, cf, "mixed", out=vals)
    ms_mass = statistics.median(timed("mixed", Xf, cf, vals, max(5, min(args.steps, 20)), mass_mesh))
    mass_mesh.close()

    # end to end through the host-buffer C-ABI calls (pinned inputs and outputs)
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
        dmesh = fem.Mesh(E, m.n_nodes, X=X64, host_direct=1)
        dmesh.pattern()
        dmesh.set_tuning(tuning["patch_entries"], tuning["block_threads"])
        for _ in range(3):
            dmesh.build_K_host(Xh, ch, "mixed", out=vh)
        t0 = time.perf_counter()
        for _ in range(ne):
            dmesh.build_K_host(Xh, ch, "mixed", out=vh)
        dt_direct = (time.perf_counter() - t0) / ne
        dmesh.close()
        e2e = {"value": m.n_elems / dt, "unit": "elements/s", "h2d_bytes_per_step": Xh.nbytes + ch.nbytes,
               "d2h_bytes_per_step": nnz * 4,
               "api": "fem_build_K_host_async on three streams (a step's copy-in and build overlap earlier copy-outs)",
               "serial": m.n_elems / dt_serial, "host_resident": m.n_elems / dt_direct}

    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(m.n_nodes, m.n_elems, 8, nnz, 4, 4, 4)
    alg64 = algorithmic_bytes(m.n_nodes, m.n_elems, 8, nnz, 8, 8, 8)
    achieved = alg / (ms_step / 1e3) / 1e9
    kernel = "k_tile" if info["assembly"] == 1 else "k_patch"
    wkey = f"hex8_n{args.n}_mixed_{'t' if info['assembly'] == 1 else 'p'}{tuning.get('patch_entries', 0)}"
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12          # TFLOP/s at the sampled clock
    alu_achieved = BRICK_FLOPS * m.n_elems / (ms_step / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": alu_achieved / alu_peak, "traffic": profiled_traffic(kernel, wkey),
            "peak_source": f"derived: {SMS} SMs x {FP32_LANES} FP32 lanes x 2 FLOP x {sm_mhz:.0f} MHz (sampled)",
            "kernel": f"{kernel} (fused integrate + assemble; bricks run its prefetching form k_patch_prefetch) and its launches",
            "flops_per_element": BRICK_FLOPS,
            "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind,
                    "algorithmic_bytes_per_launch": alg}}
    if roof["traffic"]:
        roof["hbm"]["dram_gbs"] = roof["traffic"] / (ms_step / 1e3) / 1e9

    out = None
    if rank == 0:
        out = {
            "metric": "global-K build elements/s (integrate+assemble), % HBM roofline, mixed vs FP64",
            "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f64 Jacobians of distorted elements)", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD if args.n == 100 else f"{args.n}^3 bricks", "n_elems": m.n_elems,
                       "nnz": nnz, "precision": "mixed", "pattern": "cached", "parallelism": f"replicas x{world}",
                       "l2": "flushed (256 MB write) before every step", "timing": "median of steps",
                       "assembly": "element tiles" if info["assembly"] == 1 else "node patches"},
            "roofline": roof, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        }
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(m)
    rowptr, col = mesh.get_pattern()
    rp, cl = rowptr.cpu().numpy(), col.cpu().numpy()
    mesh.build_K(Xf, cf, "mixed", out=vals)
    err = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        err["hex1M"] = {"mixed": sampled_error(m, rp, cl, vals.cpu().numpy(), m.X.astype(np.float32),
                                               m.c.astype(np.float32)),
                        "fp64": sampled_error(m, rp, cl, vals64.cpu().numpy(), m.X, m.c)}
    mesh.close()
    del vals, vals64
    extra = None
    if not args.no_workloads:
        extra, werr = other_workloads(flush, stream, with_error=(rank == 0 and world == 1 and not args.no_cpu_baseline))
        err.update(werr)
    if rank == 0:
        if extra is not None:
            out["workloads"] = extra
        out["plan"] = {"tiles_or_patches": info["n_patches"], "border_rows": info["border_rows"],
                       "n_colors": info["n_colors"], "plan_bytes": info["plan_bytes"]}
        out["tuning"] = {k: tuning[k] for k in ("patch_entries", "block_threads", "assembly") if k in tuning}
        out["mass"] = {"ms_per_step": ms_mass, "value": m.n_elems / (ms_mass / 1e3)}
        out["cold_build"] = {"seconds": cold_s, "value": m.n_elems / cold_s,
                             "includes": "validation, locality order, pattern, plan, first numeric build",
                             "first_in_process_s": first_s,
                             "first_in_process": "12^3 bricks, the process's first mesh (loads the kernels)"}
        out["fp64"] = {"value": fp64_eps, "ms_per_step": ms64, "hbm_frac": alg64 / (ms64 / 1e3) / 1e9 / peak,
                       "mixed_speedup": (value / world) / fp64_eps}
        if err:
            out["error"] = err
        out["hbm_frac"] = achieved / peak
        print(json.dumps(compact(out), separators=(",", ":")))
    if dist is not None:
        dist.destroy_process_group()


# -------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle (the plain FP64 CPU program of Algorithm 1) on the host cores,
    each step one slice of the shared sample (SAMPLE_ELEMS consecutive elements of
    the same workload), the same sample the CPU baseline of our arm times."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import meshgen
    import oracle
    oracle.build()
    m = meshgen.config_mesh(1, nx=args.n)
    for k in range(args.warmup):
        oracle_slice(m, k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle_slice(m, args.warmup + k)
    dt = time.perf_counter() - t0
    value = SAMPLE_ELEMS * args.steps / dt
    print(json.dumps(compact({
        "impl": "reference", "metric": "global-K build elements/s (integrate+assemble), % HBM roofline, mixed vs FP64",
        "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD if args.n == 100 else f"{args.n}^3 bricks", "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": 1, "kind": "oracle",
                         "sample": f"rotating slices of {SAMPLE_ELEMS} consecutive elements, one per step"},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), separators=(",", ":")))


def other_workloads(flush, stream, with_error):
    """The workloads beside the headline (pattern cached, L2 flushed before every
    timed build, median of the timed builds): the 8,000-brick FP64 build (latency),
    the 3.07M-tetrahedron build (mixed), 512 uneven brick meshes in one persistent
    launch replayed from a CUDA graph, 300^3 bricks under a 16 GB library budget and
    under a budget that forces patch groups, with its backward pass, the
    elasticity operator and the backward passes.  Returns (workloads, errors)."""
    import numpy as np
    import torch

    import meshgen
    import oracle
    from paper_1501_04784_gb300 import fem

    def dev(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt)

    def timed(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        return median_ms(fn, n, flush, stream)

    out, err = {}, {}
    # the small FP64 workload: one build's latency (pattern cached) and its cold build
    m = meshgen.config_mesh(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    nnz = mesh.pattern()
    X, c = dev(m.X, torch.float64), dev(m.c, torch.float64)
    v = torch.empty(nnz, dtype=torch.float64, device="cuda")
    mesh.build_K(X, c, "fp64", out=v)
    torch.cuda.synchronize()
    cold = time.perf_counter() - t0
    t = timed(lambda: mesh.build_K(X, c, "fp64", out=v), 20)
    out["hex8k_fp64"] = {"ms": t, "value": m.n_elems / (t / 1e3), "cold_s": cold}
    if with_error:
        ref = oracle.build_K(8, m.X, m.E, m.c)
        vv = v.cpu().numpy()
        d = np.abs(vv - ref["vals"])
        keep = np.abs(ref["vals"]) >= 1e-3 * ref["cs"]
        err["hex8k"] = {"fp64": {"r13": float((d / ref["cs"]).max()), "c14": float((d / ref["abs"]).max()),
                                 "plain": float((d[keep] / np.abs(ref["vals"][keep])).max()), "rows": m.n_nodes}}
    mesh.close()

    # 3.07M tetrahedra, mixed
    m = meshgen.config_mesh(2)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    nnz = mesh.pattern()
    X, c = dev(m.X, torch.float32), dev(m.c, torch.float32)
    v = torch.empty(nnz, dtype=torch.float32, device="cuda")
    tt = mesh.autotune(X, c, "mixed")
    t = timed(lambda: mesh.build_K(X, c, "mixed", out=v), 20)
    alg = algorithmic_bytes(m.n_nodes, m.n_elems, 4, nnz, 4, 4, 4)
    peak, _ = measured_peaks()
    out["tet3M"] = {"ms": t, "value": m.n_elems / (t / 1e3), "hbm_frac": alg / (t / 1e3) / 1e9 / peak,
                    "tile": tt["patch_entries"], "threads": tt["block_threads"]}
    if with_error:
        rowptr, col = mesh.get_pattern()
        err["tet3M"] = {"mixed": sampled_error(m, rowptr.cpu().numpy(), col.cpu().numpy(), v.cpu().numpy(),
                                               m.X.astype(np.float32), m.c.astype(np.float32))}
    mesh.close()
    del mesh, X, c, v

    ms = meshgen.batch_meshes()
    meshes = [fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64)) for m in ms]
    Xs = [dev(m.X, torch.float32) for m in ms]
    cs = [dev(m.c, torch.float32) for m in ms]
    vals = [torch.empty(mesh.pattern(), dtype=torch.float32, device="cuda") for mesh in meshes]
    nel = sum(m.n_elems for m in ms)
    t = timed(lambda: fem.build_K_batched(meshes, Xs, cs, "mixed", out=vals), 10)
    cfg = fem.batched_config(meshes, "mixed")
    out["batch512"] = {"ms": t, "value": nel / (t / 1e3), "n_elems": nel, "threads": cfg["block_threads"],
                       "grid": cfg["grid"]}
    if with_error:
        worst = {"r13": 0.0, "c14": 0.0, "plain": 0.0}
        for i in sorted(range(len(ms)), key=lambda i: ms[i].n_elems)[:3]:
            mi = ms[i]
            rowptr, col = meshes[i].get_pattern()
            e = sampled_error(mi, rowptr.cpu().numpy(), col.cpu().numpy(), vals[i].cpu().numpy(),
                              mi.X.astype(np.float32), mi.c.astype(np.float32), n_rows=mi.n_nodes)
            worst = {k: max(worst[k], e[k]) for k in worst}
        err["batch512"] = {"mixed": dict(worst, meshes=3)}
    for mesh in meshes:
        mesh.close()
    del meshes, Xs, cs, vals

    m = meshgen.config_mesh(4)
    X, c = dev(m.X, torch.float32), dev(m.c, torch.float32)
    # under 7 GB the closures are built per patch group (Eq. 10): copied back from
    # their host copies at each call (the default), or built again at each call
    for key, budget, cache in (("large27M", 16 << 30, 1), ("large27M_groups", 7 << 30, 1),
                               ("large27M_groups_rebuilt", 7 << 30, 0)):
        mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), mem_budget_bytes=budget,
                        group_cache=cache)
        nnz = mesh.pattern()
        v = torch.empty(nnz, dtype=torch.float32, device="cuda")
        t = timed(lambda: mesh.build_K(X, c, "mixed", out=v), 7)
        info = mesh.info()
        out[key] = {"ms": t, "value": m.n_elems / (t / 1e3), "budget_gb": budget / 2 ** 30,
                    "groups": info["n_groups"], "assembly": info["assembly"], "plan_gb": info["plan_bytes"] / 1e9}
        if budget < 16 << 30:
            out[key]["group_cache"] = cache
        if with_error and key != "large27M_groups_rebuilt":
            rowptr, col = mesh.get_pattern()
            err[key] = {"mixed": sampled_error(m, rowptr.cpu().numpy(), col.cpu().numpy(), v.cpu().numpy(),
                                               m.X.astype(np.float32), m.c.astype(np.float32), n_rows=500)}
        if key == "large27M":
            # its backward: dL/dX (FP32) and dL/dc of L = sum G_ij K_ij, G seeded standard normal
            G = torch.randn(nnz, generator=torch.Generator(device="cuda").manual_seed(21), device="cuda")
            tb = timed(lambda: mesh.vjp(X, c, G, "mixed"), 3)
            mesh.sync()
            out[key]["backward_ms"] = tb
            out[key]["backward_lib_gb"] = mesh.info()["live_bytes"] / 1e9
            out[key]["backward_plan_gb"] = mesh.info()["plan_bytes"] / 1e9  # with the in-row positions
            del G
        mesh.close()
        del mesh, v
    del X, c
    out["large27M_host"] = host_pipeline_workload(m, dev)
    out["elastic"] = elastic_workloads(timed, dev)
    out["backward"] = backward_workloads(timed, dev)
    # the configuration workloads last, so that a stored tail of the line keeps them
    first = ("large27M_host", "elastic", "backward")
    out = {k: out[k] for k in first + tuple(k for k in out if k not in first)}
    return out, err


def host_pipeline_workload(m, dev, chunks=16, reps=3):
    """The 27M-brick build end to end through fem_build_K_host (page-locked host
    inputs and output, one blocking call a step), K's values staged whole on the
    device and copied out in one transfer, against the row-range pipeline
    (fem_options.host_chunks): range k + 1 built while range k's values are copied
    out, two ranges of values on the device.  staging_gb: the library's device
    memory the host build adds (inputs, then K's values or two ranges of them)."""
    import time

    import numpy as np
    import torch

    from paper_1501_04784_gb300 import fem

    Xh = torch.from_numpy(m.X.astype(np.float32)).pin_memory()
    ch = torch.from_numpy(m.c.astype(np.float32)).pin_memory()
    res = {}
    for key, hc in (("whole", 0), ("pipelined", chunks)):
        mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), host_chunks=hc)
        nnz = mesh.pattern()
        before = mesh.info()["live_bytes"]
        vh = torch.empty(nnz, dtype=torch.float32).pin_memory()
        for _ in range(2):
            mesh.build_K_host(Xh, ch, "mixed", out=vh)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            mesh.build_K_host(Xh, ch, "mixed", out=vh)
            ts.append(time.perf_counter() - t0)
        info = mesh.info()
        ms = 1e3 * float(np.median(ts))
        res[key] = {"ms": round(ms, 3), "value": m.n_elems / (ms / 1e3), "chunks": info["n_chunks"],
                    "staging_gb": round((info["live_bytes"] - before) / 1e9, 3)}
        mesh.close()
        del mesh, vh
    res["h2d_bytes_per_step"] = Xh.nbytes + ch.nbytes
    res["d2h_bytes_per_step"] = nnz * 4
    return res


def backward_workloads(timed, dev):
    """The backward pass (fem_vjp: dL/dX and dL/dc of L = sum over stored entries
    G_ij K_ij, G a seeded standard normal on K's pattern): stiffness on the 1M-brick
    mesh in both precisions and on the 3.07M-tet mesh, mass and elasticity in mixed
    precision.  Algorithmic bytes: X, E, c and G read once, dX and dc written once."""
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
        r = {}
        for prec in (("mixed", "fp64") if key == "stiffness" else ("mixed",)):
            dt = torch.float32 if prec == "mixed" else torch.float64
            w = 4 if prec == "mixed" else 8
            X, cd, Gd = dev(m.X, dt), dev(c, dt), dev(G, dt)
            t = timed(lambda: mesh.vjp(X, cd, Gd, prec), 10)
            mesh.sync()
            nb = (m.n_nodes * 3 * w * 2 + m.n_elems * m.npe * 4 + cd.numel() * w * 2 + nnz * w)
            r[prec] = t
            r[prec + "_gbs"] = nb / (t / 1e3) / 1e9
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
        r = {"ms": t, "dof_entries_per_s": nnz / (t / 1e3)}
        if idx == 1:
            r["alu_frac_2070mhz"] = ELASTIC_BRICK_FLOPS * m.n_elems / (t / 1e3) / (SMS * FP32_LANES * 2 * 2070e6)
            X64, c64 = dev(m.X, torch.float64), dev(lame, torch.float64)
            v64 = torch.empty(nnz, dtype=torch.float64, device="cuda")
            r["fp64_ms"] = timed(lambda: mesh.build_K(X64, c64, "fp64", out=v64), 3)
            mesh.sync()
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
    opts = dict(patch_entries=args.patch_entries, tile_elems=args.tile_elems, block_threads=args.block_threads,
                operator_kind=2 if elastic else 0)
    if args.assembly >= 0:
        opts["assembly"] = args.assembly
    mesh = fem.Mesh(E, m.n_nodes, X=X64, **opts)
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
