#!/usr/bin/env python3
"""Benchmark of the w-product hot path on GB300.

Workload ("hsi-256x256x192-L3"): two synthetic hyperspectral-shaped cubes
A, B in R^{256x256x192} (rank-20 products of Gaussian factors with smooth
spectral tubes plus 1% noise, min-max normalised; seeds 0 and 1), L = 3.
One step = one pass of the hot path over that input:
    C   = A *w B               (mixed-precision face-products, default bf16x3)
    C_r = rank-20 w-svd of A   (when the library provides it)
    C_s = rank-20 sp-w-svd of A
`value` is the w-product throughput in TFLOP/s counting the algorithmic
2 n1 n2 n4 p flops once; the w-svd / sp-w-svd times are reported beside it,
and the same w-product in plain FP32 is timed in a second loop for the
mixed-vs-FP32 comparison, with both errors against the FP64 oracle.

Protocol: inputs resident in HBM; W >= 3 untimed warm-up steps; a 512 MiB
buffer is written between timed steps to flush the 129 MB L2; every timed
interval is a pair of CUDA events on the launching stream; per-kernel times
come from the library's own event profiler (wp_profile_*).  SM clocks are
sampled with nvidia-smi during the timed loop.  Under torchrun every rank runs
its own independent replica (weak scaling); the time is the max over ranks.

`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="hsi-256x256x192-L3", n1=256, n2=256, n4=256, p=192, L=3, r=20)
METRIC = "w-product TFLOP/s & w-svd ms at 256x256x192; mixed vs FP32 at <=1e-5 rel err"
FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", default="bf16x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-timings", action="store_true",
                    help="print the oracle's timings on this host as JSON and exit (used by the cpu baseline)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-launch and deblurring measurements")
    ap.add_argument("--profile-case", choices=["lift", "gemm", "gemm_large", "sgemm", "wprod", "wprod_fp8", "jacobi", "jacobi_row_split",
                                               "batched", "glift", "jacobi_global", "wprod_fused", "wprod_lift", "wprod_lift_L1",
                                               "lift_inverse"],
                    default=None,
                    help="run one small invocation of one kernel (for ncu captures) and exit")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(values, device=None):
    """Element-wise MAX of a list of floats over all ranks (identity when not
    distributed): the step time of a weak-scaling run is the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def inputs(np_dtype=np.float32, with_clean=False):
    from paper_2601_08228_gb300 import synth
    w = WORKLOAD
    A, Ac = synth.hsi_cube(w["n1"], w["n2"], w["p"], seed=0, dtype=np_dtype, return_clean=True)
    B = synth.hsi_cube(w["n2"], w["n4"], w["p"], seed=1, dtype=np_dtype)
    return (A, B, Ac) if with_clean else (A, B)


def wprod_flops():
    w = WORKLOAD
    return 2.0 * w["n1"] * w["n2"] * w["n4"] * w["p"]


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- peaks / roofline

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d["bf16_tflops_sustained"], "sm_max_mhz": d.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


def fp32_simt_peak_tflops(sm_count, mhz):
    """2 flops (FMA) x 128 FP32 lanes per SM x SMs x clock."""
    return 2.0 * 128 * sm_count * mhz * 1e6 / 1e12


def _src_hash(fname):
    path = os.path.join(ROOT, "paper_2601_08228_gb300", "csrc", fname)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16] if os.path.exists(path) else None


def ncu_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` at this workload, from
    the table in profiles/ncu_traffic.md, or None when the entry is absent or
    the kernel's source file changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == kernel:
            src, sha, val = cells[1], cells[2], cells[3]
            if _src_hash(src) != sha:
                return None
            try:
                return float(val)
            except ValueError:
                return None
    return None


# ---------------------------------------------------------------------------- reference arm

# The oracle's w-svd and sp-w-svd are timed on a bounded sample of the
# workload: the first SAMPLE_P frontal slices of A (256 x 256 x SAMPLE_P,
# L = 3), whose SAMPLE_P wavelet-domain slices (sp-w-svd: SAMPLE_P / 4) are
# 1 / SAMPLE_SCALE of the full workload's; the per-slice SVDs dominate the
# oracle's time, so the full-workload time is estimated as SAMPLE_SCALE x.
SAMPLE_P = 48
SAMPLE_SCALE = WORKLOAD["p"] // SAMPLE_P
SAMPLE_DESC = (f"w-product: the full 256x256x192 workload; w-svd / sp-w-svd: a 256x256x{SAMPLE_P} sub-cube "
               f"(the first {SAMPLE_P} frontal slices of A, L = 3, rank 20) scaled x{SAMPLE_SCALE} to the full workload")


def _median_time(fn, reps, budget_s):
    """Median wall time of up to `reps` calls (at least one; stops once the
    calls so far have used `budget_s`)."""
    times = []
    t_all = time.perf_counter()
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget_s:
            break
    return statistics.median(times), len(times)


def oracle_timings(reps=5, budget_s=12.0):
    """The FP64 oracle on this host: w-product TFLOP/s on the full workload,
    w-svd / sp-w-svd ms estimated from the sub-cube sample (medians)."""
    import oracle as O
    A, B = inputs(np.float64)
    w = WORKLOAD
    L, r = w["L"], w["r"]
    As = np.ascontiguousarray(A[:SAMPLE_P])
    O.wprod(A, B, L)                       # first-touch / thread-pool start-up
    t_prod, n_prod = _median_time(lambda: O.wprod(A, B, L), reps, budget_s)
    t_svd, n_svd = _median_time(lambda: O.wsvd(As, L, r), reps, budget_s)
    t_sp, n_sp = _median_time(lambda: O.spwsvd(As, L, r), reps, budget_s)
    return {"wprod_tflops": wprod_flops() / t_prod / 1e12, "wprod_ms": 1e3 * t_prod,
            "wsvd_ms": 1e3 * t_svd * SAMPLE_SCALE, "spwsvd_ms": 1e3 * t_sp * SAMPLE_SCALE,
            "reps": {"wprod": n_prod, "wsvd": n_svd, "spwsvd": n_sp}, "threads": _blas_threads()}


def _oracle_timings_subprocess(threads):
    """oracle_timings() in a fresh interpreter, with the BLAS thread count
    fixed by environment before NumPy loads (None: the library default)."""
    env = dict(os.environ)
    if threads is not None:
        for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            env[var] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-timings"]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    if out.returncode != 0 or not lines:
        return {"error": (out.stderr or out.stdout)[-300:]}
    d = json.loads(lines[-1])
    if threads is not None:
        d["threads"] = threads
    return d


def run_reference(args):
    import oracle as O
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    A, B = inputs(np.float64)
    w = WORKLOAD
    L, r = w["L"], w["r"]
    As = np.ascontiguousarray(A[:SAMPLE_P])
    t_prod = t_svd = t_sp = 0.0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.wprod(A, B, L)
        t1 = time.perf_counter()
        O.wsvd(As, L, r)
        t2 = time.perf_counter()
        O.spwsvd(As, L, r)
        t3 = time.perf_counter()
        if i >= args.warmup:
            t_prod += t1 - t0
            t_svd += (t2 - t1) * SAMPLE_SCALE
            t_sp += (t3 - t2) * SAMPLE_SCALE
    value = wprod_flops() * args.steps / t_prod / 1e12
    cores = _blas_threads()
    step_ms = 1e3 * (t_prod + t_svd + t_sp) / args.steps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["workload"], "n1": w["n1"], "n2": w["n2"], "n4": w["n4"], "p": w["p"],
                       "L": w["L"], "rank": r, "l2": "n/a (CPU)"},
            "parts_ms": {"wprod": 1e3 * t_prod / args.steps, "wsvd": 1e3 * t_svd / args.steps,
                         "spwsvd": 1e3 * t_sp / args.steps},
            "wsvd_ms": 1e3 * t_svd / args.steps,
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": SAMPLE_DESC + "; every step one pass of all three"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads") for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


def cpu_baseline_sample():
    """The oracle on the host cores, all cores and one core (medians of 5;
    see oracle_timings for the sample)."""
    allc = _oracle_timings_subprocess(None)
    one = _oracle_timings_subprocess(1)
    cpu = _cpu_model()
    if "error" in allc:
        return {"value": None, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle", "error": allc["error"]}
    return {"value": allc["wprod_tflops"], "unit": "TFLOP/s", "cores": allc["threads"], "kind": "oracle",
            "sample": SAMPLE_DESC + "; medians of 5", "wsvd_ms": allc["wsvd_ms"], "spwsvd_ms": allc["spwsvd_ms"],
            "all_cores": allc, "one_core": one, "cpu_model": cpu, "host_cpus": os.cpu_count(),
            "numpy": np.__version__, "blas": _blas_name()}


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _blas_name():
    try:
        cfg = np.show_config(mode="dicts")
        return cfg["Build Dependencies"]["blas"]["name"] + " " + str(cfg["Build Dependencies"]["blas"].get("version"))
    except Exception:
        return "unknown"


# ---------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_2601_08228_gb300 import capi

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    capi.lib()
    w = WORKLOAD
    L, r = w["L"], w["r"]
    A_h, B_h, Ac_h = inputs(np.float32, with_clean=True)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    prec = args.prec
    try:
        capi.wp_wprod(A, B, L, prec=prec)
    except capi.WPError as e:
        if e.status != 12:
            raise
        prec = "fp32"
    have_wsvd = True
    try:
        capi.wp_wsvd(A, L, r)
    except capi.WPError as e:
        if e.status != 12:
            raise
        have_wsvd = False
    torch.cuda.synchronize()

    C = torch.empty((w["p"], w["n1"], w["n4"]), dtype=torch.float32, device="cuda")
    ws_prod = torch.empty(capi.wp_wprod_workspace(w["n1"], w["n2"], w["n4"], w["p"], L, prec), dtype=torch.uint8,
                          device="cuda")
    stream = torch.cuda.current_stream()

    def step(ev):
        ev[0].record(stream)
        capi.wp_wprod(A, B, L, prec=prec, out=C, ws=ws_prod)
        ev[1].record(stream)
        if have_wsvd:
            capi.wp_wsvd(A, L, r)
            ev[2].record(stream)
            capi.wp_wsvd(A, L, r, sparse=True)
            ev[3].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step([torch.cuda.Event(enable_timing=True) for _ in range(4)])
    # one untimed step with every launch bracketed by events: the per-kernel
    # breakdown and the dominant kernel
    capi.wp_profile_begin()
    flush.zero_()
    step([torch.cuda.Event(enable_timing=True) for _ in range(4)])
    torch.cuda.synchronize()
    prof_step = capi.wp_profile_end()
    dominant = max(prof_step.items(), key=lambda kv: kv[1][1])[0]
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches0 = capi.wp_launch_count()
    capi.wp_jacobi_stats()          # clear the sweep counters
    with ClockSampler(local) as clk:
        # timed region: events around the dominant kernel's launches only, so
        # that they do not separate the other kernels of the step
        capi.wp_profile_only(dominant)
        capi.wp_profile_begin()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            step(events[i])
        torch.cuda.synchronize()
        prof = capi.wp_profile_end()
        capi.wp_profile_only(None)
    launches = capi.wp_launch_count() - launches0
    tot_sw, max_sw = capi.wp_jacobi_stats()
    jac = {"total_sweeps": tot_sw, "max_sweeps": max_sw}
    t_prod = sum(e[0].elapsed_time(e[1]) for e in events) / 1e3
    t_wsvd = sum(e[1].elapsed_time(e[2]) for e in events) / 1e3 if have_wsvd else 0.0
    t_sp = sum(e[2].elapsed_time(e[3]) for e in events) / 1e3 if have_wsvd else 0.0
    t_step = t_prod + t_wsvd + t_sp
    t_prod, t_step = reduce_max([t_prod, t_step], device="cuda")
    value = ws * args.steps * wprod_flops() / t_prod / 1e12

    # FP32 comparison loop (same protocol), and errors against the oracle
    fp32 = _time_loop(lambda: capi.wp_wprod(A, B, L, prec="fp32", out=C, ws=_ws(capi, w, L, "fp32")), flush,
                      args.warmup, args.steps)
    C_mixed = capi.wp_wprod(A, B, L, prec=prec).cpu().numpy()
    C_fp32 = capi.wp_wprod(A, B, L, prec="fp32").cpu().numpy()

    # e2e through the public call with host buffers: H2D inputs, w-product, D2H result
    e2e = _e2e(capi, A_h, B_h, L, prec, args.warmup, args.steps)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    Cref = O.wprod(A_h, B_h, L)
    err_mixed = O.rel_fro(C_mixed, Cref)
    err_fp32 = O.rel_fro(C_fp32, Cref)
    svd_quality = _svd_quality(capi, O, A, A_h, Ac_h, L) if have_wsvd else None
    clocks = clk.summary()
    peaks = measured_peaks()
    sm = torch.cuda.get_device_properties(local).multi_processor_count
    roof = _roofline(prof, peaks, sm, args.steps, have_wsvd, jac)
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3",
                                                          "fp8": "fp8e4m3"}[prec],
        "data": "synthetic",
        "config": {"workload": w["workload"], "n1": w["n1"], "n2": w["n2"], "n4": w["n4"], "p": w["p"],
                   "L": w["L"], "rank": r, "prec": prec, "l2": "flushed between steps (512 MiB write)"},
        "parts_ms": {"wprod": 1e3 * t_prod / args.steps, "wsvd": 1e3 * t_wsvd / args.steps if have_wsvd else None,
                     "spwsvd": 1e3 * t_sp / args.steps if have_wsvd else None},
        "wsvd_ms": 1e3 * t_wsvd / args.steps if have_wsvd else None,
        "fp32_tflops": args.steps * wprod_flops() / fp32 / 1e12,
        "rel_err": {"mixed": err_mixed, "fp32": err_fp32,
                    "wsvd_r20": svd_quality["wsvd"]["r20"]["rel_err"] if svd_quality else None,
                    "spwsvd_r20": svd_quality["spwsvd"]["r20"]["rel_err"] if svd_quality else None},
        "svd_quality": svd_quality,
        "roofline": roof,
        "kernels_ms_per_step": {k: v[1] for k, v in prof_step.items()},
        "jacobi_sweeps": jac,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    if not args.no_extras:
        line["extras"] = _extras(capi, args)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


_WS_CACHE = {}


def _ws(capi, w, L, prec):
    import torch
    key = (L, prec)
    if key not in _WS_CACHE:
        _WS_CACHE[key] = torch.empty(capi.wp_wprod_workspace(w["n1"], w["n2"], w["n4"], w["p"], L, prec),
                                     dtype=torch.uint8, device="cuda")
    return _WS_CACHE[key]


def _wprod_kernels(capi, reps=10):
    """ms per call and TFLOP/s of each tensor-core w-product kernel (1 fused
    inverse-lift epilogue, 2 persistent GEMM + inverse lift, 3 lifted operands
    + fused epilogue) on the benchmark's A, B at L = 1, 2, 3, and the kernel
    wp_wprod picks by its rule."""
    import torch
    w = WORKLOAD
    A, B = (torch.from_numpy(x).cuda() for x in inputs(np.float32))
    C = torch.empty((w["p"], w["n1"], w["n4"]), device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    res = {}
    for L in (1, 2, 3):
        ws = torch.empty(capi.wp_wprod_workspace(w["n1"], w["n2"], w["n4"], w["p"], L, "bf16x3"),
                         dtype=torch.uint8, device="cuda")
        row = {}
        for v in ("fused", "persistent", "lifted", None):
            capi.wp_plan_clear()
            if v:
                capi.wp_plan_set(w["n1"], w["n2"], w["n4"], w["p"], L, "bf16x3", v)
            fn = lambda: capi.wp_wprod(A, B, L, prec="bf16x3", out=C, ws=ws)
            t = _time_loop(fn, flush, 3, reps) / reps
            row[v or "rule"] = {"ms": t * 1e3, "tflops": wprod_flops() / t / 1e12}
        capi.wp_plan_clear()
        capi.wp_profile_begin()
        capi.wp_wprod(A, B, L, prec="bf16x3", out=C, ws=ws)
        names = capi.wp_profile_end()
        row["rule_picks"] = ("lifted" if any(k.startswith("tc_wprod_lift") for k in names) else
                             "fused" if any(k.startswith("tc_gemm_ilift") for k in names) else "persistent")
        res[f"L{L}"] = row
    return res


def _time_loop(fn, flush, warmup, steps):
    import torch
    for _ in range(warmup):
        flush.zero_()
        fn()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b) / 1e3
    return total


def _e2e(capi, A_h, B_h, L, prec, warmup, steps):
    """The w-product end to end through the public host-buffer call
    (wp_wprod_host): pinned A, B in, C out, the copies of every step inside
    the timed region (overlapped with the product chunk by chunk)."""
    import torch
    w = WORKLOAD
    Ap = torch.from_numpy(A_h).pin_memory()
    Bp = torch.from_numpy(B_h).pin_memory()
    Cp = torch.empty((w["p"], w["n1"], w["n4"]), dtype=torch.float32).pin_memory()
    need = capi.wp_wprod_host_workspace(w["n1"], w["n2"], w["n4"], w["p"], L, prec)
    wsb = torch.empty(need, dtype=torch.uint8, device="cuda")

    def one():
        capi.wp_wprod_host(Ap, Bp, L, prec=prec, out=Cp, ws=wsb)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        one()
    b.record()
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3
    bi, bo = Ap.numel() * 4 + Bp.numel() * 4, Cp.numel() * 4
    link = _host_link(bi, bo)
    val = steps * wprod_flops() / t / 1e12
    link["e2e_frac_of_bound"] = val / link["bound_tflops"]
    return {"value": val, "unit": "TFLOP/s", "call": "wp_wprod_host",
            "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "host_link": link}


def _svd_quality(capi, O, A_dev, A_h, Ac_h, L):
    """Rank 5 / 10 / 20 w-svd and sp-w-svd of the workload cube against the
    FP64 oracle on the same FP32 input: relative error of the reconstruction
    and of the retained singular values, and the reconstruction PSNR against
    the input cube and against the clean (noise-free) cube, for the GPU and
    for the oracle."""
    A64, Ac64 = A_h.astype(np.float64), Ac_h.astype(np.float64)
    out = {}
    for sparse, fn, name in ((False, O.wsvd, "wsvd"), (True, O.spwsvd, "spwsvd")):
        per = {}
        for r in (5, 10, 20):
            C, _, S, _ = capi.wp_wsvd(A_dev, L, r, sparse=sparse, factors=True)
            Cg, Sg = C.cpu().numpy().astype(np.float64), S.cpu().numpy().astype(np.float64)
            Cr, _, Sr, _ = fn(A64, L, r, return_factors=True)
            per[f"r{r}"] = {"rel_err": O.rel_fro(Cg, Cr), "sigma_rel_err": O.rel_fro(Sg, Sr),
                            "psnr": O.psnr(Cg, A64), "oracle_psnr": O.psnr(Cr, A64),
                            "psnr_vs_clean": O.psnr(Cg, Ac64), "oracle_psnr_vs_clean": O.psnr(Cr, Ac64)}
        out[name] = per
    return out


def _host_link(bytes_in, bytes_out, reps=5):
    """Pinned host <-> device copy rates on this machine: H2D of bytes_in and D2H
    of bytes_out alone, and both at once on two streams (the ceiling of an
    end-to-end step that streams its inputs in and its result out)."""
    import torch
    hi = torch.empty(bytes_in // 4, dtype=torch.float32).pin_memory()
    di = torch.empty(bytes_in // 4, dtype=torch.float32, device="cuda")
    ho = torch.empty(bytes_out // 4, dtype=torch.float32).pin_memory()
    do = torch.empty(bytes_out // 4, dtype=torch.float32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def both():
        with torch.cuda.stream(s1):
            di.copy_(hi, non_blocking=True)
        with torch.cuda.stream(s2):
            ho.copy_(do, non_blocking=True)

    t_in = timed(lambda: di.copy_(hi, non_blocking=True))
    t_out = timed(lambda: ho.copy_(do, non_blocking=True))
    t_both = timed(both)
    return {"h2d_gbs": bytes_in / t_in / 1e9, "d2h_gbs": bytes_out / t_out / 1e9, "duplex_ms": 1e3 * t_both,
            "bound_tflops": wprod_flops() / t_both / 1e12}


def _fp8_peak():
    """Dense FP8 (E4M3) tensor rate on this GPU: torch._scaled_mm on 8192^3
    (cuBLASLt), CUDA events over 20 launches after 3 warm-up launches."""
    import torch
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        f = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            f()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            f()
        e1.record()
        torch.cuda.synchronize()
        return {"tflops": 20 * 2.0 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12, "how": "torch._scaled_mm 8192^3 E4M3"}
    except Exception as e:   # reported, not fatal
        return {"tflops": None, "error": str(e)[:200]}


def _roofline(prof, peaks, sm_count, steps, have_wsvd, jac=None):
    """Roofline entry for the kernel with the largest share of the step."""
    if not prof:
        return None
    w = WORKLOAD
    name, (launches, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    avg_s = ms / launches / 1e3
    plane_a, plane_b, plane_c = w["n1"] * w["n2"], w["n2"] * w["n4"], w["n1"] * w["n4"]
    if name.startswith("lift"):
        # bytes per step of that kernel / launches per step; each element read + written once
        per_step_elems = {"lift_forward": plane_a + plane_b + (3 * plane_a if have_wsvd else 0),
                          "lift_inverse": plane_c + (2 * plane_a if have_wsvd else 0)}.get(name, plane_a)
        bytes_per_launch = 8.0 * w["p"] * per_step_elems / (launches / steps)
        ach = bytes_per_launch / avg_s / 1e9
        peak = peaks["hbm_gbs"]
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": ncu_traffic(name), "peak_source": peaks["source"] + " hbm_gbs"}
    if name.startswith("sgemm"):
        flops = wprod_flops()
        ach = flops / avg_s / 1e12
        peak = fp32_simt_peak_tflops(sm_count, peaks["sm_max_mhz"])
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": ncu_traffic(name),
                "peak_source": f"FP32 SIMT 2*128*{sm_count} SMs*{peaks['sm_max_mhz']:.0f} MHz"}
    if name.startswith("tc_gemm"):
        flops = wprod_flops()
        ach = flops / avg_s / 1e12
        peak = peaks["bf16_tflops_sustained"]
        return {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": ncu_traffic(name), "peak_source": peaks["source"] + " bf16 sustained"}
    if name == "jacobi_svd" and jac is not None:
        # algorithmic flops: per sweep of one slice, (n-1) rounds x n/2 pairs x
        # m rows x 8 (dot product 2, plane rotation 6) plus 2 m n for the norms
        n, m = w["n2"], w["n1"]
        per_sweep = (n - 1) * (n // 2) * m * 8 + 2 * m * n
        flops = jac["total_sweeps"] * per_sweep
        ach = flops / (ms / 1e3) / 1e12
        peak = fp32_simt_peak_tflops(sm_count, peaks["sm_max_mhz"])
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": ncu_traffic(name),
                "peak_source": f"FP32 SIMT 2*128*{sm_count} SMs*{peaks['sm_max_mhz']:.0f} MHz",
                "work": f"{jac['total_sweeps']} slice-sweeps x {per_sweep} flops"}
    return {"kernel": name, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": ncu_traffic(name), "avg_launch_ms": avg_s * 1e3}


def _extras(capi, args):
    """Two further workloads timed with the same event protocol: the batched
    launch over 4096 uneven items (w-product + rank-8 w-svd per item, one
    CUDA graph) and one 512x512x128 deblurring gradient step (BF16x3)."""
    import torch
    import oracle as O
    from paper_2601_08228_gb300 import synth
    out = {}
    items = synth.batch_items(count=4096, seed=1)
    dev = []
    for it in items:
        A = torch.from_numpy(it["A"]).cuda()
        dev.append(dict(A=A, B=torch.from_numpy(it["B"]).cuda(),
                        C=torch.empty((it["p"], it["n1"], it["n4"]), device="cuda"), C_r=torch.empty_like(A),
                        L=it["L"], r=8))
    bl = capi.BatchedLaunch(dev, tune=True)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bl.run()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    a.record()
    for _ in range(reps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3 / reps
    out["batched_4096"] = {"tensors_per_s": 4096 / t, "ms": t * 1e3, "graph": True,
                           "gemm_threads": bl.plan.gemm_threads, "svd_threads": bl.plan.svd_threads,
                           "svd_kernel": "lane-group" if bl.plan.svd_group else "block-cyclic"}
    del dev, bl, g
    # the w-svd and sp-w-svd of the workload with the Jacobi SVD's QR preconditioning switched
    # off (the timed steps run with it on): time and sweeps per slice of both variants
    from paper_2601_08228_gb300 import synth as _s
    Aw = torch.from_numpy(_s.hsi_cube(256, 256, 192, seed=0, dtype=np.float32)).cuda()
    pre = {}
    for on in (True, False):
        capi.wp_set_jacobi_precondition(on)
        for sp in (False, True):
            for _ in range(2):
                capi.wp_wsvd(Aw, 3, 20, sparse=sp)
            torch.cuda.synchronize()
            capi.wp_jacobi_stats()
            a.record()
            for _ in range(5):
                capi.wp_wsvd(Aw, 3, 20, sparse=sp)
            b.record()
            torch.cuda.synchronize()
            tot, mx = capi.wp_jacobi_stats()
            nsl = 48 if sp else 192
            pre[f"{'spwsvd' if sp else 'wsvd'}_{'qr' if on else 'plain'}"] = {
                "ms": a.elapsed_time(b) / 5, "sweeps_per_slice": tot / (5 * nsl), "max_sweeps": mx}
    capi.wp_set_jacobi_precondition(True)
    out["jacobi_qr_preconditioning"] = pre
    # the same calls (QR on) with the row-split block kernel instead of the
    # column-split one
    ker = {}
    for split in (True, False):
        capi.wp_set_jacobi_column_split(split)
        for sp in (False, True):
            for _ in range(2):
                capi.wp_wsvd(Aw, 3, 20, sparse=sp)
            torch.cuda.synchronize()
            capi.wp_jacobi_stats()
            a.record()
            for _ in range(5):
                capi.wp_wsvd(Aw, 3, 20, sparse=sp)
            b.record()
            torch.cuda.synchronize()
            tot, mx = capi.wp_jacobi_stats()
            nsl = 48 if sp else 192
            ker[f"{'spwsvd' if sp else 'wsvd'}_{'column_split' if split else 'row_split'}"] = {
                "ms": a.elapsed_time(b) / 5, "sweeps_per_slice": tot / (5 * nsl), "max_sweeps": mx}
    capi.wp_set_jacobi_column_split(True)
    out["jacobi_kernels"] = ker
    del Aw
    # the three BF16x3 w-product kernels at the benchmark's slice shape for
    # L = 1, 2, 3 (forced through the plan cache; L2 flushed before each call)
    out["wprod_kernels"] = _wprod_kernels(capi)
    # deblurring step at 512 x 512 x 128, L = 4
    n, p, L = 512, 128, 4
    K = synth.blur_operator(n, p, dtype=np.float32)
    Xt = synth.hsi_cube(n, n, p, rank=8, noise=0.0, seed=2, dtype=np.float32)
    Y = O.wprod(K, Xt, L)
    Y = (Y + 0.01 * Y.std() * synth.unit_noise(Y.shape, 3)).astype(np.float32)
    Kd, Yd = torch.from_numpy(K).cuda(), torch.from_numpy(Y).cuda()
    X = torch.zeros_like(Yd)
    ws = torch.empty(capi.wp_deblur_workspace(n, n, p, L, "bf16x3"), dtype=torch.uint8, device="cuda")
    eta = 1.0 / (2.0 * (1.0 + 1e-3))
    for _ in range(3):
        capi.wp_deblur_step(Kd, Yd, X, L, 1e-3, eta, prec="bf16x3", ws=ws)
    torch.cuda.synchronize()
    a.record()
    for _ in range(10):
        capi.wp_deblur_step(Kd, Yd, X, L, 1e-3, eta, prec="bf16x3", ws=ws)
    b.record()
    torch.cuda.synchronize()
    step = a.elapsed_time(b) / 10
    out["deblur_512x512x128"] = {"ms_per_step": step, "ms_200_steps": 200 * step,
                                 "tflops": 2 * 2 * n ** 3 * p / (step / 1e3) / 1e12, "prec": "bf16x3"}
    del Kd, Yd, X, ws
    # wpinv of 192 slices of 256 x 192, iid N(0, 1) (wavelet slices with
    # condition numbers near 14), L = 3, one refinement step.  The HSI cube
    # itself is no pinv workload in FP32: its s_L slices reach condition
    # numbers of 1e7 and the cut-off falls inside a dense part of the spectrum.
    A_h = np.random.default_rng(4).standard_normal((192, 256, 192)).astype(np.float32)
    Ad = torch.from_numpy(A_h).cuda()
    wsp = torch.empty(capi.wp_wpinv_workspace(256, 192, 192, 3), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        X = capi.wp_wpinv(Ad, 3, refine_iters=1, ws=wsp)
    torch.cuda.synchronize()
    a.record()
    for _ in range(5):
        X = capi.wp_wpinv(Ad, 3, refine_iters=1, ws=wsp)
    b.record()
    torch.cuda.synchronize()
    t_pinv = a.elapsed_time(b) / 5
    err_pinv = O.rel_fro(X.cpu().numpy(), O.wpinv(A_h, 3))
    out["wpinv_256x192x192_L3"] = {"ms": t_pinv, "refine_iters": 1, "rel_err": err_pinv}
    del Ad, X, wsp
    # two-sided pseudo-inverse deblurring (Sec. IV-C) at the shapes of the
    # paper's three scenes (synthetic clean cubes blurred by the paper's linear
    # blur, b = 10).  The operators are the same in every band, so each tube
    # group's result depends only on that group of B: the oracle runs on the
    # first `og` groups (a bounded sample) and is compared with the same
    # slices of the GPU result.  PaviaU (610 rows) and Botswana (1476 rows)
    # have slices beyond a cluster's shared memory: global-memory Jacobi.
    for key, (n1, n2, p, L, og) in (("deblur_pinv_512x217x204_L2", (512, 217, 204, 2, 51)),
                                    ("deblur_pinv_610x340x102_L1", (610, 340, 102, 1, 8)),
                                    ("deblur_pinv_1476x256x144_L4", (1476, 256, 144, 4, 1))):
        Xc = synth.hsi_cube(n1, n2, p, rank=20, noise=0.0, seed=6)
        AV, AH = synth.linear_blur_operator(n1, p), synth.linear_blur_operator(n2, p)
        Bb = O.wprod(O.wprod(AV, Xc, L), O.transpose(AH), L)
        AVd, AHd, Bd = (torch.from_numpy(x.astype(np.float32)).cuda() for x in (AV, AH, Bb))
        wsd = torch.empty(capi.wp_deblur_pinv_workspace(n1, n2, p, L), dtype=torch.uint8, device="cuda")
        Xd = capi.wp_deblur_pinv(AVd, AHd, Bd, L, ws=wsd)
        torch.cuda.synchronize()
        a.record()
        for _ in range(3):
            Xd = capi.wp_deblur_pinv(AVd, AHd, Bd, L, ws=wsd)
        b.record()
        torch.cuda.synchronize()
        Xg = Xd.cpu().numpy()
        ns = og << L
        rt = max(n1, n2) * 1.1920929e-7
        ref = O.deblur_pinv(AV[:ns], AH[:ns], Bb[:ns], L, rtol=rt)
        # the oracle on the FP32-rounded operators and data: what FP32 inputs allow
        ref32 = O.deblur_pinv(AV[:ns].astype(np.float32), AH[:ns].astype(np.float32), Bb[:ns].astype(np.float32),
                              L, rtol=rt)
        out[key] = {"ms": a.elapsed_time(b) / 3, "refine_iters": 2, "sample_slices": ns,
                    "rel_err": O.rel_fro(Xg[:ns], ref), "rel_err_vs_fp32_input_oracle": O.rel_fro(Xg[:ns], ref32),
                    "psnr_vs_clean": O.psnr(Xg[:ns], Xc[:ns]), "oracle_psnr_vs_clean": O.psnr(ref, Xc[:ns]),
                    "fp32_input_oracle_psnr_vs_clean": O.psnr(ref32, Xc[:ns]),
                    "blurred_psnr_vs_clean": O.psnr(Bb[:ns], Xc[:ns])}
        del AVd, AHd, Bd, Xd, wsd
    # precision study: A 1024x1024x256 by B 1024x512x256, per-slice 10^U[-3,3] scales, L = 4
    A, B = synth.scaled_pair(1024, 1024, 512, 256, seed=0)
    ref = O.wprod(A, B, 4)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    flops = 2.0 * 1024 * 1024 * 512 * 256
    study = {}
    for prec in ("fp32", "bf16x3", "bf16", "fp8"):
        Cd = torch.empty((256, 1024, 512), device="cuda")
        wsb = torch.empty(capi.wp_wprod_workspace(1024, 1024, 512, 256, 4, prec), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            capi.wp_wprod(Ad, Bd, 4, prec=prec, out=Cd, ws=wsb)
        torch.cuda.synchronize()
        a.record()
        for _ in range(3):
            capi.wp_wprod(Ad, Bd, 4, prec=prec, out=Cd, ws=wsb)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 3 / 1e3
        study[prec] = {"tflops": flops / t / 1e12, "ms": t * 1e3,
                       "rel_err": O.rel_fro(Cd.cpu().numpy(), ref)}
        # the face-product kernel alone (one more call with events around every launch)
        capi.wp_profile_begin()
        capi.wp_wprod(Ad, Bd, 4, prec=prec, out=Cd, ws=wsb)
        kern = capi.wp_profile_end()
        gemm = {k: v for k, v in kern.items() if "gemm" in k}
        if gemm:
            name, (_, ms) = max(gemm.items(), key=lambda kv: kv[1][1])
            study[prec]["gemm_kernel"] = name
            study[prec]["gemm_ms"] = ms
            study[prec]["gemm_tflops"] = flops / (ms / 1e3) / 1e12
        del Cd, wsb
    peaks = measured_peaks()
    fp8 = _fp8_peak()
    for prec in ("bf16", "bf16x3"):
        if "gemm_tflops" in study[prec]:
            study[prec]["gemm_frac"] = study[prec]["gemm_tflops"] / peaks["bf16_tflops"]
            study[prec]["gemm_peak"] = f"{peaks['source']} bf16 burst {peaks['bf16_tflops']}"
    if "gemm_tflops" in study["fp8"] and fp8.get("tflops"):
        study["fp8"]["gemm_frac"] = study["fp8"]["gemm_tflops"] / fp8["tflops"]
        study["fp8"]["gemm_peak"] = f"measured FP8 {fp8['tflops']:.0f} ({fp8['how']})"
    # each face-product kernel against its own roofline: it reads both operands
    # once (bytes per element: BF16 2, BF16x3 hi + lo 4, E4M3 1) and writes C
    # (FP32) once; ceiling = min(tensor peak / products per output, intensity x HBM)
    per_slice_elems = 1024 * 1024 + 1024 * 512
    for prec, ebytes, nprod, tpeak in (("bf16", 2, 1, peaks["bf16_tflops"]), ("bf16x3", 4, 3, peaks["bf16_tflops"]),
                                       ("fp8", 1, 1, fp8.get("tflops"))):
        if "gemm_tflops" not in study[prec] or not tpeak:
            continue
        gbytes = 256.0 * (per_slice_elems * ebytes + 1024 * 512 * 4)
        inten = flops / gbytes
        ceil_ = min(tpeak / nprod, inten * peaks["hbm_gbs"] / 1e3)
        study[prec]["gemm_bytes"] = gbytes
        study[prec]["gemm_flop_per_byte"] = inten
        study[prec]["gemm_roofline_tflops"] = ceil_
        study[prec]["gemm_frac_of_roofline"] = study[prec]["gemm_tflops"] / ceil_
        study[prec]["gemm_roofline_bound"] = "tensor" if tpeak / nprod <= inten * peaks["hbm_gbs"] / 1e3 else "hbm"
        if nprod > 1:
            study[prec]["tensor_issued_tflops"] = nprod * study[prec]["gemm_tflops"]
            study[prec]["tensor_issued_frac"] = nprod * study[prec]["gemm_tflops"] / tpeak
    out["fp8_peak"] = fp8
    out["precision_1024x1024x256_by_1024x512x256_L4"] = study
    return out


def run_profile_case(case):
    """One small invocation of one kernel family, for ncu captures (inputs
    larger than L2 where DRAM counters matter, a few GB at most)."""
    import torch
    from paper_2601_08228_gb300 import capi, synth
    capi.lib()
    if case == "lift":
        x = torch.rand((768, 256, 256), device="cuda")      # 201 MB > L2
        capi.wp_lift_forward(x, 3)
    elif case == "gemm":
        A = torch.rand((192, 256, 256), device="cuda")
        B = torch.rand((192, 256, 256), device="cuda")
        capi.wp_facewise(A, B, prec="bf16x3")
    elif case == "gemm_large":
        # the precision study's face-product shape (1024 x 1024 by 1024 x 512), 64 slices: 1.1 GB
        A = torch.rand((64, 1024, 1024), device="cuda")
        B = torch.rand((64, 1024, 512), device="cuda")
        for prec in ("bf16", "bf16x3"):
            capi.wp_facewise(A, B, prec=prec)
    elif case == "sgemm":
        # FP32 SIMT face-product of the benchmark's shape: 192 slices of 256 x 256 (2 x 50 MB in)
        A = torch.rand((192, 256, 256), device="cuda")
        B = torch.rand((192, 256, 256), device="cuda")
        capi.wp_facewise(A, B, prec="fp32")
    elif case == "wprod":
        A, B = (torch.from_numpy(x).cuda() for x in inputs(np.float32))
        capi.wp_wprod(A, B, WORKLOAD["L"], prec="bf16x3")
    elif case == "wprod_fp8":
        # the precision study's slice shapes at 64 slices (A 268 MB, B 134 MB), L = 4
        A, B = synth.scaled_pair(1024, 1024, 512, 64, seed=0)
        capi.wp_wprod(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 4, prec="fp8")
    elif case in ("jacobi", "jacobi_row_split"):
        # 72 slices of 256 x 256: 2-CTA clusters as in the full workload, one wave;
        # jacobi_row_split: the same call on the row-split block kernel
        A = torch.from_numpy(synth.hsi_cube(256, 256, 72, seed=0, dtype=np.float32)).cuda()
        capi.wp_set_jacobi_column_split(case == "jacobi")
        capi.wp_wsvd(A, 3, 20)
    elif case == "glift":
        # general operators (CDF-5/3-style predict + update, Sec. II-A Eq. 2), 192 x 256 x 256, L = 3 (50 MB in)
        ops = [((-1, (0.5, 0.5)), (0, (0.25, 0.25)))] * 3
        x = torch.from_numpy(synth.hsi_cube(256, 256, 192, seed=0, dtype=np.float32)).cuda()
        capi.wp_glift(x, 3, ops)
    elif case == "jacobi_global":
        # w-svd of 4 slices of 1476 x 256 (L = 2): beyond a cluster's shared memory
        A = torch.from_numpy(synth.hsi_cube(1476, 256, 4, seed=0, dtype=np.float32)).cuda()
        capi.wp_wsvd(A, 2, 20)
    elif case == "wprod_fused":
        # the fused inverse-lift epilogue kernel at the benchmark's shape (forced through the plan cache)
        A, B = (torch.from_numpy(x).cuda() for x in inputs(np.float32))
        w = WORKLOAD
        capi.wp_plan_set(w["n1"], w["n2"], w["n4"], w["p"], w["L"], "bf16x3", "fused")
        capi.wp_wprod(A, B, w["L"], prec="bf16x3")
    elif case in ("wprod_lift", "wprod_lift_L1"):
        # the kernel that lifts the spatial operands in its producer warps, at the benchmark's
        # shape (L = 3, forced) or at L = 1 (where the dispatch rule picks it)
        A, B = (torch.from_numpy(x).cuda() for x in inputs(np.float32))
        w = WORKLOAD
        L = w["L"] if case == "wprod_lift" else 1
        capi.wp_plan_set(w["n1"], w["n2"], w["n4"], w["p"], L, "bf16x3", "lifted")
        capi.wp_wprod(A, B, L, prec="bf16x3")
    elif case == "lift_inverse":
        # exported Mallat-order inverse at L = 4: 256 slices of 1024 x 512 (537 MB in)
        y = torch.rand((256, 1024, 512), device="cuda")
        capi.wp_lift_inverse(y, 4)
    elif case == "batched":
        items = synth.batch_items(count=64, seed=1)
        dev = []
        for it in items:
            A = torch.from_numpy(it["A"]).cuda()
            dev.append(dict(A=A, B=torch.from_numpy(it["B"]).cuda(),
                            C=torch.empty((it["p"], it["n1"], it["n4"]), device="cuda"), C_r=torch.empty_like(A),
                            L=it["L"], r=8))
        capi.BatchedLaunch(dev).run()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "ok": True}))


def main():
    args = parse_args()
    if args.oracle_timings:
        print(json.dumps(oracle_timings()), flush=True)
        return
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
