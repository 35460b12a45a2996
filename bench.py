"""Benchmark of the Brillouin-operator apply on GB300.

Workload (default): one application of D_B to a Gaussian spinor field on a
32^3 x 64 lattice (antiperiodic in t) with synthetic links exp(i 0.3 H), the
hopping fields stored in FP32 ("f32-full"), FP32 spinors and arithmetic.
A step is one apply over the whole lattice; the link precompute (path sums +
SU(3) projection) runs once per gauge field, before timing.

Metric: algorithmic GB/s = (40 unique hopping fields + spinor in + out per
site) x V / time; the hopping fields alone are ~6 GB, far above L2, so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode f32-full]
                    [--nrhs 1] [--impl native|reference] [--sweep] [--no-solve]

The default line also carries the solver half of the metric ("solve"): time to
a true FP64 relative residual of 1e-10 on 16^3x32 (FP64 BiCGstab vs FP64
defect correction around FP32 BiCGstab) and on 24^3x48 (12 point sources
solved together vs FP64 one after the other).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_BENCH = (32, 32, 32, 64)
BC = (1, 1, 1, -1)
EPS = 0.3
SEED = 1015

LINK_BYTES = {  # bytes per site of the 40 stored hopping fields
    "f64-full": 40 * 144, "f32-full": 40 * 72, "f32-2row": 40 * 48, "f32-8param": 40 * 32,
    "f16-full": 40 * 36, "f16-2row": 40 * 24, "f16-8param": 40 * 16,
    # FP16 hopping fields with FP16 spinors (52 bytes per site and RHS: 12 half2 + one FP32 scale)
    "f16h-full": 40 * 36, "f16h-2row": 40 * 24, "f16h-8param": 40 * 16,
}
# Algorithmic flops per site and right-hand side, the method's count:
#   80 hops x 4 spins x one 3x3 complex mat-vec (9 complex multiplies x 6 +
#   6 complex adds x 2 = 66 flops)                                  = 21,120
#   + 24 (1 + n) real adds per hop of class n into the lambda and the
#   n gamma_mu accumulators of its class (sum over the 80 hops)     =  7,104
#   + class scaling (4 classes x 5 accumulators x 24 multiplies)    =    480
#   + summing the 4 classes (5 accumulators x 3 x 24 adds)          =    360
#   + gamma combine (4 x 24 adds) and the diagonal (24 x 2)         =    144
#                                                                   = 29,208
# plus 42 flops per use of a 2-row field (third row = conj(r0 x r1), 80 uses).
# The 8-parameter decoders are not counted (their cost is the format's).
FLOPS_PER_SITE = 29208
FLOPS_2ROW = 80 * 42
# what the kernels execute: 80 hops x 4 spins x 9 complex MACs as 8 flops
# each, + per (d, -d) pair of class n the sum and difference of the two colour
# products (2 x 24 FMAs), the lambda term (24) and the gamma terms (24 n), +
# the diagonal (24); FMA = 2 flops
IMPL_FLOPS_PER_SITE = 34032


def method_flops(mode):
    return FLOPS_PER_SITE + (FLOPS_2ROW if mode.endswith("2row") else 0)


def spinor_bytes(mode):
    # in + out per site and RHS
    return 2 * (192 if mode.startswith("f64") else 52 if mode.startswith("f16h") else 96)


def site_bytes(mode, nrhs):
    return LINK_BYTES[mode] + nrhs * spinor_bytes(mode)


KERNEL_SOURCES = ["paper_1012_3615_gb300/csrc/dslash_kernel.cuh", "paper_1012_3615_gb300/csrc/dslash_pair.cuh",
                  "paper_1012_3615_gb300/csrc/links.cuh", "paper_1012_3615_gb300/csrc/common.cuh"]
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x (FMA = 2) x max SM clock


def alu_peaks():
    """FP32 (packed FMA) and FP64 FMA peaks of this GPU, measured by the
    library's own microbenchmark (bri_alu_peak) at the clocks it runs at"""
    from paper_1012_3615_gb300.core import alu_peak

    return {"f32": alu_peak("f32"), "f64": alu_peak("f64")}


def kernel_hash():
    """Hash of the stencil sources with comments and blank space removed, so
    that an edit of a comment does not retire the committed ncu counters."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_traffic(mode, nrhs, shape, lattice):
    """DRAM bytes per launch of the apply kernel from the committed ncu summary
    (profiles/dslash_traffic.json), if it was taken on the current kernel
    sources with the same storage mode, RHS count and launch shape; else None.
    A capture on a smaller lattice is scaled by the number of sites."""
    p = os.path.join(ROOT, "profiles", "dslash_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    for e in d.get("captures", []):
        if e.get("mode") == mode and e.get("nrhs") == nrhs and e.get("launch_shape") == shape:
            v_cap = 1
            for t in e["lattice"]:
                v_cap *= t
            v = 1
            for t in lattice:
                v *= t
            return e["dram_bytes_per_launch"] * v / v_cap
    return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during timing."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [t.strip() for t in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "native" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(pg, value, device=None):
    """Maximum of a float over all ranks (identity on one process)."""
    if pg is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg, device=None):
    if pg is not None:
        import torch

        t = torch.zeros(1, device=device)
        pg.all_reduce(t)


# ---------------------------------------------------------------------------------
def cpu_baseline(mode, seconds=15.0):
    """The oracle (as it stands) timed on the host cores on a bounded sample:
    a 16^3 x 8 lattice with the same link distribution, FP64 apply with the
    oracle's hops prebuilt (the hop build is not part of a step)."""
    import numpy as np

    import oracle
    from paper_1012_3615_gb300 import synth

    L = (16, 16, 16, 8)
    U = synth.random_su3_links(L, EPS, SEED)
    psi = synth.gaussian_spinor(L, 1, SEED + 1)[0]
    W = oracle.build_hops(L, U)
    V = synth.volume(L)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.apply(L, BC, W, 0.0, psi)
        n += 1
        if time.perf_counter() - t0 > seconds or n >= 50:
            break
    dt = (time.perf_counter() - t0) / n
    gbs = site_bytes(mode, 1) * V / dt / 1e9  # the metric's bytes (workload storage mode)
    return {"value": gbs, "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "FP64 oracle apply on a 16^3x8 lattice (same link and source distribution), %d applies, "
                      "%.3f s each, hops prebuilt" % (n, dt), "ms_per_apply": dt * 1e3}


def reference_arm(args, world, rank, pg):
    """--impl reference: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1012_3615_gb300 import synth

    L = (16, 16, 16, 8)
    U = synth.random_su3_links(L, EPS, SEED)
    psi = synth.gaussian_spinor(L, 1, SEED + 1)[0]
    W = oracle.build_hops(L, U)
    V = synth.volume(L)
    for _ in range(args.warmup):
        oracle.apply(L, BC, W, 0.0, psi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.apply(L, BC, W, 0.0, psi)
    dt = (time.perf_counter() - t0) / args.steps
    # the same metric as the native arm: the workload's algorithmic bytes per
    # site (its storage mode) times the sites processed, per second
    gbs = site_bytes(args.mode, 1) * V / dt / 1e9
    LB = tuple(args.lattice) if args.lattice else L_BENCH
    sample = ("each step one FP64 oracle apply on a 16^3x8 sub-lattice (same link and source "
              "distribution), hops prebuilt; %d timed steps" % args.steps)
    line = {
        "impl": "reference", "metric": "D_B apply GB/s", "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "D_B apply, %s lattice, antiperiodic t, links exp(i0.3H), Gaussian spinors"
                               % "x".join(str(v) for v in LB),
                   "lattice": list(LB), "nrhs": 1, "hop_storage": args.mode, "sample": sample,
                   "parallelism": "single"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------
def time_apply(op, x, out, mode, nrhs, steps, warmup, stream):
    import torch

    prec = mode.split("-")[0]
    for _ in range(warmup):
        op.apply(x, 0.0, prec=prec, out=out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        op.apply(x, 0.0, prec=prec, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps  # ms per apply


def rel_err_vs_fp64(op, x, y, prec):
    """max |y - y64| / max |y64|, y64 the library's FP64 apply of the same input
    (m0 = 0; the tests hold the FP64 apply to 1e-13 of the oracle): the
    per-element error of a reduced-precision storage mode at full size."""
    import torch

    if prec == "f16h":
        x, y = op.from_h16(x), op.from_h16(y)
    x64 = x.to(torch.complex128)
    y64 = op.apply(x64, 0.0, prec="f64")
    e = ((y.to(torch.complex128) - y64).abs().max() / y64.abs().max()).item()
    del x64, y64
    return e


def native(args, world, rank, local, pg):
    import numpy as np
    import torch

    from paper_1012_3615_gb300 import Brillouin, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.solve_only:
        if rank == 0:
            print(json.dumps({"metric": "mixed/batched vs FP64 solve time to 1e-10", "unit": "s",
                              "solve": solve_bench(args, dev)}), flush=True)
        return
    mode, nrhs = args.mode, args.nrhs
    prec, comp = mode.split("-")
    L = tuple(args.lattice) if args.lattice else L_BENCH
    V = synth.volume(L)
    U = synth.random_su3_links_torch(L, EPS, SEED + rank, device=dev)
    op = Brillouin(L, BC)
    op.build_hops(U, prec=prec, comp=comp)
    del U
    sdt = torch.complex128 if prec == "f64" else torch.complex64
    x = synth.gaussian_spinor_torch(L, nrhs, SEED + 100 + rank, device=dev, dtype=sdt)
    out = torch.empty_like(x)
    if args.threads is not None:
        op.set_threads(prec, nrhs, args.threads)
    elif args.tune:
        op.tune(prec, nrhs)
    stream = torch.cuda.current_stream()
    time_apply(op, x, out, mode, nrhs, 1, args.warmup, stream)  # warm-up (untimed)

    clocks = ClockSampler(local)
    barrier(pg, dev)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    n0 = op.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        op.apply(x, 0.0, prec=prec, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg, dev)
    t_wall = time.perf_counter() - t_wall
    launches = op.kernel_launches() - n0
    ms = e0.elapsed_time(e1) / args.steps
    ck = clocks.stop()
    ms_max = max_over_ranks(pg, ms, dev)

    bytes_step = site_bytes(mode, nrhs) * V
    value = bytes_step * world / (ms_max * 1e-3) / 1e9
    peak, peak_kind = load_peaks()
    dslash_gbs = bytes_step / (ms * 1e-3) / 1e9

    # end to end through the public API with host buffers (pinned): bri_apply_host
    # copies the input in, applies and copies the result out (copies overlapping
    # the stencil slab by slab); every step synchronises
    xh = x.cpu().pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    e2e_steps = max(10, min(args.steps, 30))
    op.apply_host(xh, 0.0, prec=prec, out=oh)  # staging buffers allocated outside the timing
    torch.cuda.synchronize()
    step_s = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        op.apply_host(xh, 0.0, prec=prec, out=oh)
        torch.cuda.synchronize()
        step_s.append(time.perf_counter() - t0)
    # the median step: a single slow host copy (another tenant on the host) does not set the number
    e2e_s = sorted(step_s)[len(step_s) // 2]
    e2e = {"value": bytes_step / e2e_s / 1e9 * world, "unit": "GB/s",
           "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
           "d2h_bytes_per_step": int(oh.numel() * oh.element_size()), "ms_per_step": e2e_s * 1e3,
           "ms_per_step_mean": sum(step_s) / len(step_s) * 1e3, "steps": e2e_steps, "statistic": "median step"}

    flops = method_flops(mode) * nrhs * V / (ms * 1e-3) / 1e12
    impl_flops = IMPL_FLOPS_PER_SITE * nrhs * V / (ms * 1e-3) / 1e12
    peaks = alu_peaks()
    alu_peak_v = peaks["f64"] if prec == "f64" else peaks["f32"]
    line = {
        "metric": "D_B apply GB/s", "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic",
        "config": {"workload": "D_B apply, %s lattice, antiperiodic t, links exp(i0.3H), Gaussian spinors"
                               % "x".join(str(v) for v in L),
                   "lattice": list(L), "nrhs": nrhs, "hop_storage": mode, "threads_per_block": op.threads(prec, nrhs),
                   "l2": "inputs larger than L2 (hopping fields %.1f GB)" % (LINK_BYTES[mode] * V / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": dslash_gbs, "peak": peak, "unit": "GB/s",
                     "frac": dslash_gbs / peak,
                     "traffic": measured_traffic(mode, nrhs, op.threads(prec, nrhs), L),
                     "peak_kind": peak_kind + " hbm_gbs (copy)",
                     "algorithmic_bytes_per_launch": bytes_step, "tflops": flops,
                     "alu": {"achieved_tflops": flops, "flops_per_site": method_flops(mode),
                             "peak_tflops": alu_peak_v, "frac": flops / alu_peak_v,
                             "peak_kind": "measured (bri_alu_peak: %s FMA chains on every SM)"
                                          % ("FP64" if prec == "f64" else "packed FP32"),
                             "impl_tflops": impl_flops, "impl_flops_per_site": IMPL_FLOPS_PER_SITE,
                             "impl_frac": impl_flops / alu_peak_v,
                             "measured_peaks_tflops": peaks, "fp32_nominal_tflops": FP32_NOMINAL_TFLOPS},
                     "kernel_hash": kernel_hash()},
        "e2e": e2e,
        "accuracy": {"max_rel_err": rel_err_vs_fp64(op, x, out, prec) if prec != "f64" else 0.0,
                     "vs": "FP64 apply of the same input on the same fields (max |out - out64| / max |out64|)"},
        "gpu_launches": int(launches),
        "clocks": ck,
        "wall_s_timed": t_wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(mode, seconds=args.cpu_seconds)
    if args.sweep:
        sweep = {}
        for m in ["f64-full", "f32-full", "f32-2row", "f32-8param", "f16-full", "f16-2row", "f16-8param",
                  "f16h-2row"]:
            for nr in ([1] if m.startswith("f64") else [1, 4, 12, 24]):
                p, c = m.split("-")
                if p != "f64":
                    op.store_hops("f16" if p == "f16h" else p, c)
                sd = torch.complex128 if p == "f64" else torch.complex64
                xx = synth.gaussian_spinor_torch(L, nr, SEED + 7, device=dev, dtype=sd)
                if p == "f16h":
                    xx = op.to_h16(xx)
                oo = torch.empty_like(xx)
                if p == "f16h":
                    pass  # one kernel form, no launch shapes
                elif args.threads is not None:
                    op.set_threads(p, nr, args.threads)
                else:
                    op.tune(p, nr)
                t = time_apply(op, xx, oo, m, nr, 3 if p == "f64" else 10, 2, stream)
                b = site_bytes(m, nr) * V
                sweep["%s/n%d" % (m, nr)] = {"ms": t, "ms_per_rhs": t / nr, "GB/s": b / (t * 1e-3) / 1e9,
                                             "frac_hbm": b / (t * 1e-3) / 1e9 / peak,
                                             "TFLOP/s": method_flops(m) * nr * V / (t * 1e-3) / 1e12}
                if nr == 1 and p != "f64":
                    sweep["%s/n%d" % (m, nr)]["max_rel_err"] = rel_err_vs_fp64(op, xx, oo, p)
                del xx, oo
        line["sweep"] = sweep
    if not args.no_solve and world == 1:
        del x, out
        torch.cuda.empty_cache()
        line["solve"] = solve_bench(args, dev)
    if args.rows:
        torch.cuda.empty_cache()
        line["rows"] = rows_bench(dev)
    if args.study:
        torch.cuda.empty_cache()
        line["study"] = study_bench(dev)
    if rank == 0:
        print(json.dumps(line), flush=True)


def rows_bench(dev):
    """Timings of the other rows of the path, on their own workloads:
    hop precompute (path sums + SU(3) projection, FP64) on 32^3x64 and 8^4,
    the FP64 apply on 8^4 (the parity workload, 10 applies), and the fermion
    force d Re(chi^dagger D psi)/dU plus d(phi^dagger (D^dagger D)^-1 phi)/dU on 12^4."""
    import torch

    from paper_1012_3615_gb300 import Brillouin, synth

    out = {}

    def timed(fn, reps=1):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    for L, eps in (((32, 32, 32, 64), 0.3), ((8, 8, 8, 8), 0.3)):
        U = synth.random_su3_links_torch(L, eps, SEED + 7, device=dev)
        op = Brillouin(L, BC)
        op.build_hops(U)  # warm-up (allocations)
        ms, _ = timed(lambda: op.build_hops(U))
        V = synth.volume(L)
        out["hop_precompute_%s" % "x".join(map(str, L))] = {
            "ms": ms, "projections_per_s": 36 * V / (ms * 1e-3), "sites": V}
        if L == (8, 8, 8, 8):
            psi = synth.gaussian_spinor_torch(L, 1, SEED + 8, device=dev)
            o = torch.empty_like(psi)
            op.apply(psi, 0.0, out=o)
            ms, _ = timed(lambda: op.apply(psi, 0.0, out=o), reps=10)
            out["apply_fp64_8x8x8x8"] = {"ms": ms, "GB/s": site_bytes("f64-full", 1) * V / (ms * 1e-3) / 1e9,
                                          "TFLOP/s": method_flops("f64-full") * V / (ms * 1e-3) / 1e12}
        del op, U
        torch.cuda.empty_cache()
    L = (12, 12, 12, 12)
    U = synth.random_su3_links_torch(L, 0.3, SEED + 9, device=dev)
    op = Brillouin(L, BC)
    op.build_hops(U)
    chi, psi = synth.gaussian_spinor_torch(L, 2, SEED + 10, device=dev)
    chi, psi = chi.contiguous(), psi.contiguous()
    op.force(chi, psi)
    ms, _ = timed(lambda: op.force(chi, psi))
    out["force_12x12x12x12"] = {"ms": ms}
    t0 = time.perf_counter()
    dU, info = op.force_inverse(chi, m0=0.0, tol=1e-10)
    torch.cuda.synchronize()
    out["force_inverse_12x12x12x12"] = {"seconds": time.perf_counter() - t0, "iters_second_solve": info["iters"],
                                        "status": info["status"], "solves": "FP64 BiCGstab"}
    op.store_hops("f32", "full")
    t0 = time.perf_counter()
    dU, info = op.force_inverse(chi, m0=0.0, tol=1e-10)
    torch.cuda.synchronize()
    out["force_inverse_12x12x12x12_mixed"] = {"seconds": time.perf_counter() - t0,
                                              "iters_second_solve": info["iters"],
                                              "outer_second_solve": info["outer_iters"], "status": info["status"],
                                              "solves": "FP64 defect correction around FP32 BiCGstab"}
    return out


def solve_bench(args, dev):
    """Solver workloads: time to a true FP64 relative residual of 1e-10, each
    timed solve after an untimed one of the same shape cut short (maxit 20),
    which sets up the work spaces and captures the CUDA graphs; nvidia-smi
    clocks are sampled during each workload.
    A: 16^3x32, m0 = -0.05, links exp(i0.4H), Z2 source, hopping fields in FP32
       2-row form (and FP16 2-row): FP64 BiCGstab vs FP64 defect correction
       around FP32 BiCGstab (FP32 and FP16 fields).
    B: 24^3x48, m0 = 0, links exp(i0.35H), the 12 spin-colour point sources at
       one random site: batched defect correction of all 12 together (FP16
       2-row fields, mode 3; FP32 2-row fields, mode 4) vs the FP64 solves of
       the sources one after the other (the first --fp64-sources of them)."""
    import numpy as np
    import torch

    from paper_1012_3615_gb300 import Brillouin, synth

    def run(op, b, m0, mode):
        op.solve(b, m0=m0, tol=1e-10, maxit=20, mode=mode)  # warm-up: work spaces, CUDA graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info = op.solve(b, m0=m0, tol=1e-10, maxit=20000, mode=mode)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"seconds": dt, "iters": [i["iters"] for i in info], "outer": [i["outer_iters"] for i in info],
                "true_resid_max": max(i["true_resid"] for i in info),
                "status": sorted(set(i["status"] for i in info))}

    out = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    L = (16, 16, 16, 32)
    U = synth.random_su3_links_torch(L, 0.4, SEED + 2, device=dev)
    op = Brillouin(L, BC)
    op.build_hops(U, prec="f32", comp="2row")
    op.store_hops("f16", "2row")
    b = torch.as_tensor(synth.z2_spinor(L, 1, SEED + 3), device=dev)
    res = {"workload": "16^3x32, m0=-0.05, links exp(i0.4H), Z2 source, hops FP32 2-row / FP16 2-row"}
    for mode, name in ((0, "fp64"), (1, "mixed_f32"), (2, "mixed_f16")):
        res[name] = run(op, b, -0.05, mode)
    res["speedup_mixed_f32_vs_fp64"] = res["fp64"]["seconds"] / res["mixed_f32"]["seconds"]
    res["speedup_mixed_f16_vs_fp64"] = res["fp64"]["seconds"] / res["mixed_f16"]["seconds"]
    res["clocks"] = clocks.stop()
    out["solve_16x16x16x32"] = res
    del op, U
    torch.cuda.empty_cache()
    if not args.solve_small:
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        L = (24, 24, 24, 48)
        V = synth.volume(L)
        U = synth.random_su3_links_torch(L, 0.35, SEED + 4, device=dev)
        op = Brillouin(L, BC)
        op.build_hops(U, prec="f16", comp="2row")
        x0 = int(np.random.default_rng(SEED + 5).integers(0, V))
        b = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device=dev)
        for s_ in range(4):
            for c in range(3):
                b[3 * s_ + c, x0, s_, c] = 1.0
        res = {"workload": "24^3x48, m0=0, links exp(i0.35H), 12 spin-colour point sources at site %d" % x0}
        res["batched_12_f16_fields"] = run(op, b, 0.0, 3)
        op.store_hops("f32", "2row")
        res["batched_12_f32_fields"] = run(op, b, 0.0, 4)
        nf = max(1, min(12, args.fp64_sources))
        res["fp64_sequential"] = run(op, b[:nf].contiguous(), 0.0, 0)
        res["fp64_sequential"]["sources"] = nf
        t64 = res["fp64_sequential"]["seconds"] * 12.0 / nf
        res["fp64_12_sources_seconds"] = t64
        res["fp64_12_sources_kind"] = "measured" if nf == 12 else "%d of 12 sources measured, scaled by 12/%d" % (nf, nf)
        res["speedup_batched_f16_vs_fp64"] = t64 / res["batched_12_f16_fields"]["seconds"]
        res["speedup_batched_f32_vs_fp64"] = t64 / res["batched_12_f32_fields"]["seconds"]
        res["clocks"] = clocks.stop()
        out["solve_24x24x24x48_12_point_sources"] = res
        del op, U
        torch.cuda.empty_cache()
    return out


def study_bench(dev):
    """Comparisons between members of the operator class on one synthetic field
    (12^4, links exp(i0.3H), antiperiodic t), Wilson against Brillouin:
    A (Sec. 7.4): smallest, 10th and largest eigenvalue of D^dagger D at
      m0 = -1 (the shifted overlap kernel, rho = 1; FP32 Lanczos, tol 1e-6), the condition numbers with
      and without the 9 lowest modes, and the sign-function polynomial degree
      for eps = 1e-10 after deflating 9 modes (FP32 polynomial), with the time
      of one overlap application.
    B (Sec. 6.4, Sec. 8): BiCGstab (FP64, true residual 1e-10, Z2 source) for
      each operator at its own "critical" bare mass -- where the smallest
      eigenvalue of D^dagger D is smallest on this volume -- and 0.1 above it:
      iterations and time.
    C (Sec. 7.2, 7.3): non-normality ||[D^dagger, D] eta|| and Ginsparg-Wilson
      violation at that mass, on the links, after one APE step, and with the
      clover term."""
    import numpy as np
    import torch

    from paper_1012_3615_gb300 import Brillouin, synth
    from paper_1012_3615_gb300.core import WEIGHTS

    L = (12, 12, 12, 12)
    U = synth.random_su3_links_torch(L, 0.3, SEED + 11, device=dev)
    b = torch.as_tensor(synth.z2_spinor(L, 1, SEED + 12), device=dev)
    psi = synth.gaussian_spinor_torch(L, 1, SEED + 13, device=dev)
    out = {"lattice": list(L), "links": "exp(i0.3H)"}
    for name in ("wilson", "brillouin"):
        op = Brillouin(L, BC)
        op.set_weights(*WEIGHTS[name])
        op.build_hops(U, prec="f32", comp="full")
        r = {}
        ev, lmax, info = op.eigs_ddag_d(10, m0=-1.0, max_krylov=3000, tol=1e-6, prec="f32")
        r["ritz_m0_-1"] = {"lambda_1": ev[0], "lambda_10": ev[9], "lambda_max": lmax,
                           "cond": lmax / ev[0], "cond_without_9": lmax / ev[9],
                           "krylov_dim": info["krylov_dim"], "status": info["status"]}
        ov = op.overlap_setup(rho=1.0, nlow=9, eps=1e-10, max_krylov=3000, tol=1e-10, prec="f32")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op.overlap(psi)
        torch.cuda.synchronize()
        r["overlap_rho_1_nlow_9"] = dict(ov, apply_seconds=time.perf_counter() - t0)

        def lmin(m0):
            e, _, _ = op.eigs_ddag_d(1, m0=m0, max_krylov=2000, tol=1e-2, prec="f32")
            return e[0]

        # the bare mass where the smallest eigenvalue of D^dagger D is smallest
        # (on a finite volume it stays above the lowest-momentum gap): golden
        # section over [-0.6, 0.3]; then solve there and 0.1 above it
        g = (5 ** 0.5 - 1) / 2
        a_, b_ = -0.6, 0.3
        c_, d_ = b_ - g * (b_ - a_), a_ + g * (b_ - a_)
        fc_, fd_ = lmin(c_), lmin(d_)
        for _ in range(14):
            if fc_ < fd_:
                b_, d_, fd_ = d_, c_, fc_
                c_ = b_ - g * (b_ - a_)
                fc_ = lmin(c_)
            else:
                a_, c_, fc_ = c_, d_, fd_
                d_ = a_ + g * (b_ - a_)
                fd_ = lmin(d_)
        mstar = 0.5 * (a_ + b_)
        for tag, m0 in (("solve_at_gap_minimum", mstar), ("solve_0.1_above", mstar + 0.1)):
            lm = lmin(m0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, inf = op.solve(b, m0=m0, tol=1e-10, maxit=20000, mode=0)
            torch.cuda.synchronize()
            r[tag] = {"m0": m0, "lambda_min": lm, "iters": inf[0]["iters"], "applies": 2 * inf[0]["iters"],
                      "status": inf[0]["status"], "true_resid": inf[0]["true_resid"],
                      "seconds": time.perf_counter() - t0}
        # Sec. 7.2 / 7.3: non-normality ||(D^dag D - D D^dag) eta|| (mass independent)
        # and the Ginsparg-Wilson violation ||(D g5 + g5 D - D g5 D) eta|| at the
        # operator's own critical mass, for unit Gaussian eta, on these links and
        # on one APE step (alpha = 0.72) with and without the clover term
        g5 = torch.tensor([1, 1, -1, -1], dtype=torch.complex128, device=dev).view(1, 1, 4, 1)
        etas = synth.gaussian_spinor_torch(L, 4, SEED + 14, device=dev)
        etas = etas / etas.reshape(4, -1).norm(dim=1).view(4, 1, 1, 1)

        def measures(m_gw):
            nn, gw = [], []
            for k in range(4):
                e = etas[k:k + 1].contiguous()
                De, Dde = op.apply(e, 0.0), op.apply(e, 0.0, dagger=True)
                nn.append((op.apply(De, 0.0, dagger=True) - op.apply(Dde, 0.0)).norm().item())
                Dm = op.apply(e, m_gw)
                gw.append((op.apply((g5 * e).contiguous(), m_gw) + g5 * Dm
                           - op.apply((g5 * Dm).contiguous(), m_gw)).norm().item())
            return float(np.mean(nn)), float(np.mean(gw))

        r["non_normality"], r["gw_violation_at_gap_minimum"] = measures(mstar)
        V1 = op.ape_smear(U, 0.72, 1)
        op.build_hops(V1, prec="f32", comp="full")
        r["ape1_csw0"] = dict(zip(("non_normality", "gw_violation"), measures(mstar)))
        op.set_clover(1.0)
        r["ape1_csw1"] = dict(zip(("non_normality", "gw_violation"), measures(mstar)))
        op.set_clover(0.0)
        out[name] = r
        del op
        torch.cuda.empty_cache()
    w, br = out["wilson"], out["brillouin"]
    out["brillouin_over_wilson"] = {
        "iterations_at_gap_minimum": br["solve_at_gap_minimum"]["iters"] / w["solve_at_gap_minimum"]["iters"],
        "iterations_0.1_above": br["solve_0.1_above"]["iters"] / w["solve_0.1_above"]["iters"],
        "solve_time_at_gap_minimum": br["solve_at_gap_minimum"]["seconds"] / w["solve_at_gap_minimum"]["seconds"],
        "lambda_max_m0_-1": br["ritz_m0_-1"]["lambda_max"] / w["ritz_m0_-1"]["lambda_max"],
        "cond_without_9": br["ritz_m0_-1"]["cond_without_9"] / w["ritz_m0_-1"]["cond_without_9"],
        "sign_degree": br["overlap_rho_1_nlow_9"]["degree"] / w["overlap_rho_1_nlow_9"]["degree"],
        "non_normality": br["non_normality"] / w["non_normality"],
        "non_normality_ape1_csw1": br["ape1_csw1"]["non_normality"] / w["ape1_csw1"]["non_normality"],
        "gw_violation": br["gw_violation_at_gap_minimum"] / w["gw_violation_at_gap_minimum"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--mode", default="f32-full", choices=sorted(LINK_BYTES))
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="leave out the solver workloads (time to 1e-10)")
    ap.add_argument("--solve-small", action="store_true", help="only the 16^3x32 solver workload")
    ap.add_argument("--solve-only", action="store_true",
                    help="run only the solver workloads and print their results (no apply timing)")
    ap.add_argument("--fp64-sources", type=int, default=12,
                    help="point sources of the 24^3x48 workload solved in FP64 for the comparison (1-12)")
    ap.add_argument("--rows", action="store_true", help="add hop precompute, FP64 apply and force timings")
    ap.add_argument("--study", action="store_true",
                    help="add the Wilson / Brillouin comparison (Sec. 7.4 spectra, overlap degree, solver iterations)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--lattice", type=lambda t: [int(v) for v in t.split(",")], default=None,
                    help="lattice extents x,y,z,t (default 32,32,32,64)")
    ap.add_argument("--tune", action="store_true", help="run the launch-shape tuner before timing")
    ap.add_argument("--threads", type=int, default=None,
                    help="fixed launch shape (threads per block; 0 = shared-memory tiled kernel); skips the tuner")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank, pg)
    else:
        native(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
