#!/usr/bin/env python3
"""Benchmark of all-to-all convergent cross mapping on GB300.

One step is one pass of the whole hot path over the calcium-imaging-shaped
workload (50,000 series x 1,500 steps, inputs resident in HBM):
  optimal E of every series (simplex, E = 1..20, Tp_sel = 1)
  -> exact neighbour tables (k = E*+1) of every library
  -> lookup + Pearson for all 2.5e9 (library, target) pairs (tau = 1, Tp = 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line.  `value` is CCM pairs/s of the plain FP32 path, timed
with CUDA events on the launching stream over K steps; the mixed-precision
forms are reported beside it: "mixed" (FP32 distances and moments, targets
stored as scaled FP16) and "mixed_bf16" (targets stored as BF16), each with
its measured |drho| against the plain run and the FP64 oracle.  With N > 1
(torchrun) the one problem is split by library rows, one contiguous block per
rank with every series replicated (strong scaling, no data exchange); the
step time is the maximum over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2105_12301_gb300 import inputs, ranks  # noqa: E402

METRIC = ("CCM pairs/s (lib×target, L=1500) + kNN rows/s; mixed vs plain at "
          "|Δrho|≤1e-4")
UNIT = "pairs/s"
E_MAX, TAU, TP, TP_SEL = 20, 1, 0, 1

# DRAM bytes per lookup_kernel launch from an ncu capture (profiles/), valid
# only for the kernel source it was taken on.
LOOKUP_TRAFFIC = {"source_sha1": "96ae46fe3bbb3501da94cf80d5d6b420501ededf",
                  "bytes_per_launch": 26020115763}  # mean of the 5 launches of one step


def workload(name):
    if name == "calcium50k":
        return 50000, 1500
    if name == "calcium2k":
        return 2000, 1500
    raise ValueError(name)


def workload_config(name, N, L, world_size):
    return {
        "workload": "calcium-imaging-shaped all-to-all CCM, %d series x %d steps "
                    "(Lorenz-63 driver + AR(1), exp-filtered, z-normalised)" % (N, L),
        "n_series": N, "series_len": L, "pairs_per_step": N * N,
        "E_range": [1, E_MAX], "tau": TAU, "Tp": TP, "Tp_sel": TP_SEL,
        "libraries": "all series", "targets": "all series",
        "parallelism": ("library rows split in contiguous blocks, one per GPU, all series "
                        "replicated (no exchange)") if world_size > 1 else "single GPU",
        "l2": "inputs larger than L2 (300 MB series, 10 GB rho, GB-scale tables); no flush",
    }


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- CPU baseline

def sample_rows(N, n_libs):
    return np.linspace(0, N - 1, n_libs).astype(int)


def cpu_sample(X, n_libs, threads):
    """The FP64 oracle on n_libs libraries (sample_rows) x all targets,
    optimal E included; returns (pairs/s, seconds, [(E*, rho row)])."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    rows = sample_rows(X.shape[0], n_libs)

    def one(i):
        e, _ = oracle.optimal_E(X[i], E_MAX, TAU, TP_SEL)
        return e, oracle.ccm_row(X[i], X, e, TAU, TP)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, rows))
    dt = time.perf_counter() - t0
    return n_libs * X.shape[0] / dt, dt, res


def drho_stats(a, b):
    """max and 99th percentile of |a - b| over the pairs where both are
    numbers, and how many pairs that is."""
    ok = np.isfinite(a) & np.isfinite(b)
    d = np.abs(a[ok].astype(np.float64) - b[ok].astype(np.float64))
    return {"max": float(d.max(initial=0.0)),
            "p99": float(np.percentile(d, 99)) if d.size else 0.0,
            "pairs": int(d.size)}


def run_reference(args):
    rank, size = ranks.init("gloo")
    if rank != 0:
        return
    N, L = workload(args.workload)
    X = inputs.calcium(N, L)
    cores = os.cpu_count() or 1
    threads = cores
    n_libs = threads
    for _ in range(args.warmup):
        cpu_sample(X, max(1, threads // 4), threads)
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, _ = cpu_sample(X, n_libs, threads)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    sample = ("%d libraries x all %d targets per step (optimal E over 1..%d + CCM row), "
              "%d threads" % (n_libs, N, E_MAX, threads))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, N, L, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------- GPU arm

def source_sha1(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def run_gb300(args):
    from paper_2105_12301_gb300 import edm

    rank, size = ranks.init()
    _, _, local = ranks.world()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, L = workload(args.workload)
    X = inputs.calcium(N, L)
    Xg = torch.from_numpy(X).to(dev)
    # one problem split by library rows (every rank holds all series)
    b, e = ranks.row_block(N, rank, size)
    Xlib = Xg[b:e]
    rho = torch.empty((e - b, N), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(prec):
        E_opt, _ = edm.edm_simplex_optimal_E(Xlib, E_MAX, TAU, TP_SEL, with_rho=False)
        edm.edm_ccm_all(Xlib, Xg, E_opt, TAU, TP, prec, out=rho)
        return E_opt

    def timed(prec, warmup, steps, profile=False):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize(dev)
        if profile:
            edm.edm_profile_enable(True, dev)
        launches0 = edm.edm_kernel_launches(dev)
        ranks.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            E_opt = step(prec)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ranks.barrier()
        ms = e0.elapsed_time(e1) / steps
        launches = edm.edm_kernel_launches(dev) - launches0
        edm.edm_ctx_sync(dev)
        return ms, launches, E_opt

    # roofline denominator: this GPU's shared-memory gather bandwidth
    smem_peak_gbs = edm.edm_probe_smem_bandwidth(200.0, dev) / 1e9

    clocks = ClockSampler(local)
    clocks.start()
    ms, launches, E_opt = timed(args.precision, args.warmup, args.steps, profile=True)
    clk = clocks.stop()
    ms_max = ranks.max_over_ranks(ms, dev)
    pairs = float(N) * N                  # the whole job: every rank's row block
    value = pairs / (ms_max / 1e3)

    # per-kernel device times of the timed steps
    prof = {k: edm.edm_profile_read(k, dev) for k in ("sweep_kernel", "sweep_long_kernel", "simplex_finish_kernel",
                                      "ccm_table_kernel", "lookup_kernel", "target_store_kernel",
                                      "target_mean_kernel", "target_sums_kernel",
                                      "group_libs_kernel")}
    edm.edm_profile_enable(False, dev)
    # the rows of the FP64 band and brute-force fallbacks, counted on one
    # extra untimed step
    edm.edm_set_option("diagnostics", 1, dev)
    edm.edm_fallback_counts(dev)
    step(args.precision)
    fb_band, fb_brute = edm.edm_fallback_counts(dev)
    edm.edm_set_option("diagnostics", 0, dev)
    E_np = E_opt.cpu().numpy().astype(np.int64)
    n_lib = L - (E_np - 1) * TAU - TP                       # rows per library table
    k_lib = E_np + 1
    bpv = 4 if args.precision == "fp32" else 2
    # algorithmic shared-memory gather bytes of one step: one stored target
    # value per (query row, neighbour) of every (library, target) pair; the
    # table broadcast and the observation reads are overhead, not counted
    lookup_bytes = float(np.sum(n_lib * k_lib)) * N * bpv     # this rank's libraries
    lk_ms, lk_n = prof["lookup_kernel"]
    lk_avg_ms = lk_ms / max(lk_n, 1)
    achieved_gbs = lookup_bytes * args.steps / (lk_ms / 1e3) / 1e9 if lk_ms > 0 else None
    sweep_rows = sum(max(0, L - (E - 1) * TAU - TP_SEL) for E in range(1, E_MAX + 1)
                     if L - (E - 1) * TAU - TP_SEL >= E + 2) * (e - b)
    table_rows = float(np.sum(n_lib))
    knn_ms = (prof["sweep_kernel"][0] + prof["sweep_long_kernel"][0] +
              prof["ccm_table_kernel"][0]) / args.steps
    knn_rows_per_s = (sweep_rows + table_rows) / (knn_ms / 1e3) if knn_ms > 0 else None
    lookup_src = os.path.join(ROOT, "paper_2105_12301_gb300", "csrc", "lookup.cu")
    traffic = (LOOKUP_TRAFFIC["bytes_per_launch"]
               if LOOKUP_TRAFFIC["source_sha1"] == source_sha1(lookup_src) else None)
    roofline = {
        "bound": "smem", "kernel": "lookup_kernel",
        "achieved": achieved_gbs, "peak": smem_peak_gbs, "unit": "GB/s",
        "frac": (achieved_gbs / smem_peak_gbs) if achieved_gbs and smem_peak_gbs else None,
        "traffic": traffic,
        "peak_source": "measured: edm_probe_smem_bandwidth (conflict-free 128-B row gathers, "
                       "all SMs, this run)",
        "algorithmic_bytes_per_launch": lookup_bytes * args.steps / max(lk_n, 1),
        "avg_launch_ms": lk_avg_ms,
        "nominal_peak_at_sampled_clock_gbs": (152 * 128 * clk["sm_mhz"] * 1e6 / 1e9) if clk else None,
    }
    # the optimal-E sweep against FP32 issue: 3 lane-ops (sub, fma, compare)
    # per candidate, query row and E; peak = SMs x 128 lanes x sampled clock
    sw_ms = prof["sweep_kernel"][0] / args.steps
    sweep_ops = 3.0 * (e - b) * sum(max(0, L - (E - 1) * TAU - TP_SEL) * max(0, L - (E - 1) * TAU - TP_SEL - 1)
                                    for E in range(1, E_MAX + 1)
                                    if L - (E - 1) * TAU - TP_SEL >= E + 2)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * 128 * (clk["sm_mhz"] if clk else 2070.0) * 1e6
    roofline_sweep = {
        "bound": "alu", "kernel": "sweep_kernel",
        "achieved": sweep_ops / (sw_ms / 1e3) / 1e12 if sw_ms > 0 else None,
        "peak": alu_peak / 1e12, "unit": "Tops/s (FP32 lane-ops)",
        "frac": (sweep_ops / (sw_ms / 1e3)) / alu_peak if sw_ms > 0 else None,
        "peak_source": "derived: SMs x 128 FP32 lanes x sampled SM clock",
        "algorithmic_ops_per_step": sweep_ops,
    }
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": size,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f32+bf16-targets",
        "data": "synthetic",
        "config": workload_config(args.workload, N, L, size),
        "gpu_launches": int(launches),
        "clocks": clk,
        "knn_rows_per_s": knn_rows_per_s,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "roofline": roofline,
        "roofline_sweep": roofline_sweep,
        "E_opt_hist": np.bincount(E_np, minlength=E_MAX + 1)[1:].tolist(),
        "fp64_fallbacks": {"band_rows": fb_band, "brute_rows": fb_brute,
                           "rows_selected": int(sweep_rows + table_rows),
                           "note": "query rows (per E) whose exact neighbour set needed the FP64 "
                                   "band, and of those a full FP64 scan; one untimed step, "
                                   "this rank's libraries"},
    }

    cores = os.cpu_count() or 1
    rows = sample_rows(e - b, 3 * cores)        # the libraries the oracle samples (this block)
    plain_rows = rho[torch.from_numpy(rows).to(dev)].cpu().numpy()

    def lookup_roofline(prof_run, bytes_per_value, clk_run):
        lk_ms_run, lk_n_run = prof_run["lookup_kernel"]
        lk_bytes = float(np.sum(n_lib * k_lib)) * N * bytes_per_value
        ach = lk_bytes * steps_run[0] / (lk_ms_run / 1e3) / 1e9 if lk_ms_run > 0 else None
        return {"bound": "smem", "kernel": "lookup_kernel", "achieved": ach,
                "peak": smem_peak_gbs, "unit": "GB/s",
                "frac": ach / smem_peak_gbs if ach and smem_peak_gbs else None,
                "traffic": None,
                "peak_source": roofline["peak_source"],
                "algorithmic_bytes_per_launch": lk_bytes * steps_run[0] / max(lk_n_run, 1),
                "avg_launch_ms": lk_ms_run / max(lk_n_run, 1),
                "nominal_peak_at_sampled_clock_gbs":
                    (152 * 128 * clk_run["sm_mhz"] * 1e6 / 1e9) if clk_run else None}

    steps_run = [0]
    mixed_rows = {}
    if args.mixed and args.precision == "fp32":
        # the 16-bit target storages, each on its own timed steps with its own
        # clock record and per-kernel split
        for key, prec, dtype in (("mixed", "fp16", "f32+fp16-targets"),
                                 ("mixed_bf16", "bf16", "f32+bf16-targets")):
            steps_m = max(3, args.steps // 4)
            steps_run[0] = steps_m
            clocks_m = ClockSampler(local)
            clocks_m.start()
            ms_m, _, E_m = timed(prec, 1, steps_m, profile=True)
            clk_m = clocks_m.stop()
            ms_m = ranks.max_over_ranks(ms_m, dev)
            prof_m = {k: edm.edm_profile_read(k, dev) for k in prof}
            edm.edm_profile_enable(False, dev)
            assert torch.equal(E_m.cpu(), E_opt.cpu())
            mixed_rows[key] = rho[torch.from_numpy(rows).to(dev)].cpu().numpy()
            out[key] = {
                "value": pairs / (ms_m / 1e3), "unit": UNIT, "ms_per_step": ms_m,
                "steps": steps_m, "dtype": dtype, "clocks": clk_m,
                "kernel_ms_per_step": {k: v[0] / steps_m for k, v in prof_m.items() if v[1]},
                "roofline": lookup_roofline(prof_m, 2, clk_m),
                "drho_vs_plain": drho_stats(mixed_rows[key], plain_rows),
                "drho_sample": "%d libraries (evenly spaced) x all %d targets" % (len(rows), N),
            }
        out["mixed"]["tolerance"] = ("FP16 target storage: |drho| <= 5e-4 against the FP64 oracle "
                                     "(tests); drho_vs_plain / drho_vs_oracle measured here")
        out["mixed_bf16"]["tolerance"] = ("BF16 target storage: |drho| <= 1e-3 against the FP64 "
                                          "oracle for >= 300 library points (tests)")

    if args.e2e:
        # public API end to end, every step: pinned host series up
        # (edm_upload_series), optimal E, tables, lookup, rho streamed down
        # block by block as it is finished (edm_ccm_all_host)
        X_h = torch.from_numpy(X).pin_memory()
        rho_h = torch.empty((e - b, N), dtype=torch.float32, pin_memory=True)
        steps_e2e = max(1, args.steps)

        def e2e_step():
            edm.edm_upload_series(X_h, Xg)
            E_opt, _ = edm.edm_simplex_optimal_E(Xlib, E_MAX, TAU, TP_SEL, with_rho=False)
            edm.edm_ccm_all_host(Xlib, Xg, E_opt, rho, rho_h, TAU, TP, args.precision)

        e2e_step()
        torch.cuda.synchronize(dev)
        ranks.barrier()
        launches_e0 = edm.edm_kernel_launches(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps_e2e):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_e = ranks.max_over_ranks(e0.elapsed_time(e1) / steps_e2e, dev)
        edm.edm_ctx_sync(dev)
        out["e2e"] = {"value": pairs / (ms_e / 1e3), "unit": UNIT,
                      "h2d_bytes_per_step": int(X_h.numel() * 4) * size,    # every rank uploads all series
                      "d2h_bytes_per_step": int(N) * N * 4,                # all row blocks together
                      "ms_per_step": ms_e,
                      "steps": steps_e2e,
                      "gpu_launches": int(edm.edm_kernel_launches(dev) - launches_e0),
                      "api": "edm_upload_series -> edm_simplex_optimal_E -> edm_ccm_all_host"}
        del rho_h

    if args.cpu_baseline and rank == 0 and size == 1:
        v, dt, res = cpu_sample(X, len(rows), cores)
        out["cpu_baseline"] = {
            "value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d libraries x all %d targets (optimal E over 1..%d + CCM row), %.1f s"
                      % (len(rows), N, E_MAX, dt)}
        # the same libraries against the GPU rows of the timed runs, where the
        # oracle's E* equals the GPU's (the oracle used its own E*)
        same = [r for r, (e, _) in enumerate(res) if e == int(E_np[rows[r]])]
        ref = np.stack([res[r][1] for r in same]) if same else np.zeros((0, N))
        out["drho_vs_oracle"] = {"libraries": len(same), "fp32": drho_stats(plain_rows[same], ref)}
        for key in mixed_rows:
            out["drho_vs_oracle"][out[key]["dtype"]] = drho_stats(mixed_rows[key][same], ref)
            out[key]["drho_vs_oracle"] = out["drho_vs_oracle"][out[key]["dtype"]]
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------ other workloads

def sync_time(fn, dev, stream, steps):
    """Mean milliseconds of fn() over `steps` calls, CUDA events on `stream`."""
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / steps


def log(msg):
    sys.stderr.write("[bench %.0fs] %s\n" % (time.perf_counter() - T_START, msg))
    sys.stderr.flush()


T_START = time.perf_counter()


def run_batched_workload(args):
    """256 independent all-to-all CCM problems of uneven N and L (optimal E,
    then CCM), in three modes: "batched" (optimal E through the work-queue
    launches, CCM over concurrent streams, both graph-captured), "streams"
    (every instance its own launches, spread over concurrent streams,
    graph-captured) and "per_instance" (every instance's launches one after
    another on one stream)."""
    from paper_2105_12301_gb300 import edm
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    Ns, Ls = inputs.uneven_batch_shapes()
    probs, E_out, pairs = [], [], 0.0
    for i, (N, L) in enumerate(zip(Ns, Ls)):
        X = torch.from_numpy(inputs.uneven_batch_instance(i, N, L)).to(dev)
        E = torch.empty(int(N), dtype=torch.int32, device=dev)
        rho = torch.empty((int(N), int(N)), dtype=torch.float32, device=dev)
        probs.append({"X": X, "tau": TAU, "Tp": TP, "E_lib": E, "rho": rho})
        E_out.append(E)
        pairs += float(N) * float(N)
    log("generated %d instances, %.3g pairs" % (len(probs), pairs))

    def opt_E():
        edm.edm_simplex_optimal_E_batched(probs, E_MAX, TP_SEL, out=E_out)

    out = {"metric": METRIC, "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
           "config": {"workload": "256 independent coupled-logistic CCM problems, N log-uniform "
                                  "in [32, 2048], L log-uniform in [200, 5000], noise 0.02",
                      "pairs_per_step": pairs, "E_range": [1, E_MAX], "tau": TAU, "Tp": TP,
                      "Tp_sel": TP_SEL}}
    for mode, opts in (("batched", {"batch_graph": 1, "batch_streams": 8, "batch_queue": 1}),
                       ("streams", {"batch_graph": 1, "batch_streams": 8, "batch_queue": 0}),
                       ("per_instance", {"batch_graph": 0, "batch_streams": 1, "batch_queue": 0})):
        for k, v in opts.items():
            edm.edm_set_option(k, v, dev)
        opt_E()
        ms_E = sync_time(opt_E, dev, stream, max(1, args.steps))
        log("%s optimal E %.1f ms" % (mode, ms_E))
        rec = {"optimal_E_ms": ms_E}
        for prec in ("fp32", "bf16"):
            def ccm():
                edm.edm_ccm_batched(probs, prec)
            for _ in range(max(1, args.warmup)):
                ccm()
            ms = sync_time(ccm, dev, stream, max(1, args.steps))
            edm.edm_ctx_sync(dev)
            log("%s ccm %s %.1f ms" % (mode, prec, ms))
            rec[prec] = {"ccm_ms": ms, "value": pairs / ((ms + ms_E) / 1e3),
                         "ms_per_step": ms + ms_E}
        out[mode] = rec
    out["value"] = out["batched"]["fp32"]["value"]
    out["ms_per_step"] = out["batched"]["fp32"]["ms_per_step"]
    print(json.dumps(out), flush=True)


def run_libsweep_workload(args):
    """Library-length convergence: 2,000 coupled-logistic series x 10,000
    steps; E per library from the full-length simplex, then all-to-all CCM on
    the window [0, L_lib) for L_lib = 100 .. 10,000."""
    from paper_2105_12301_gb300 import edm
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    X = inputs.logistic_long()
    N, L = X.shape
    Xg = torch.from_numpy(X).to(dev)
    log("generated %d x %d" % (N, L))
    ms_E = sync_time(lambda: edm.edm_simplex_optimal_E(Xg, E_MAX, TAU, TP_SEL, with_rho=False),
                     dev, stream, 1)
    log("optimal E %.1f ms" % ms_E)
    E_full, _ = edm.edm_simplex_optimal_E(Xg, E_MAX, TAU, TP_SEL, with_rho=False)
    rho = torch.empty((N, N), dtype=torch.float32, device=dev)
    sizes = {}
    kernels = ("ccm_table_kernel", "lookup_kernel", "group_libs_kernel", "target_store_kernel")
    smem_gbs = edm.edm_probe_smem_bandwidth(200.0, dev) / 1e9
    l2_gbs = edm.edm_probe_l2_bandwidth(200.0, dev) / 1e9
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    E_np = E_full.cpu().numpy().astype(np.int64)
    for L_lib in (100, 300, 1000, 3000, 10000):
        for prec in ("fp32", "bf16"):
            def one():
                edm.edm_ccm_window(Xg, 0, L_lib, E_full, TAU, TP, prec, out=rho)
            one()
            ms = sync_time(one, dev, stream, max(1, args.steps))
            edm.edm_profile_enable(True, dev)
            one()
            split = {k: edm.edm_profile_read(k, dev)[0] for k in kernels}
            edm.edm_profile_enable(False, dev)
            edm.edm_ctx_sync(dev)
            # rooflines: the lookup's gathers (n k b bytes per pair) against
            # shared memory while a tile fits it (<= 3,300 points), else
            # against L2; the table builder against FP32 issue (E subs and
            # FMAs plus a compare per candidate)
            n_lib = np.maximum(L_lib - (E_np - 1) * TAU - TP, 0)
            ok = n_lib >= E_np + 2
            bpv = 4 if prec == "fp32" else 2
            lk_bytes = float(np.sum((n_lib * (E_np + 1))[ok])) * N * bpv
            tiled = L_lib <= 3300
            peak = smem_gbs if tiled else l2_gbs
            lk_ms = split["lookup_kernel"]
            tb_ops = float(np.sum((n_lib * (n_lib - 1) * (2 * E_np + 1))[ok]))
            tb_ms = split["ccm_table_kernel"]
            alu_peak = n_sm * 128 * 2.07e9
            sizes.setdefault(str(L_lib), {})[prec] = {
                "value": N * N / (ms / 1e3), "ms": ms, "kernel_ms": split,
                "lookup_roofline": {"bound": "smem" if tiled else "l2",
                                    "achieved_gbs": lk_bytes / (lk_ms / 1e3) / 1e9 if lk_ms else None,
                                    "peak_gbs": peak,
                                    "frac": lk_bytes / (lk_ms / 1e3) / 1e9 / peak if lk_ms else None},
                "table_roofline": {"bound": "alu", "lane_ops": tb_ops,
                                   "frac": tb_ops / (tb_ms / 1e3) / alu_peak if tb_ms else None}}
            log("window %d %s %.1f ms %s" % (L_lib, prec, ms, split))
    out = {"metric": METRIC, "unit": UNIT, "higher_is_better": True, "n_gpus": 1,
           "data": "synthetic", "value": sizes["10000"]["fp32"]["value"],
           "config": {"workload": "library-length sweep, %d coupled-logistic series x %d steps, "
                                  "windows [0, L_lib)" % (N, L), "pairs_per_size": N * N},
           "optimal_E_ms": ms_E, "per_library_size": sizes,
           "peaks": {"smem_gather_gbs": smem_gbs, "l2_gather_gbs": l2_gbs,
                     "fp32_issue_lane_ops_per_s": n_sm * 128 * 2.07e9},
           "E_opt_hist": np.bincount(E_full.cpu().numpy(), minlength=E_MAX + 1)[1:].tolist()}
    print(json.dumps(out), flush=True)


def run_paper_micro_workload(args):
    """The shapes of the paper's micro-benchmarks (section 4): exact all-kNN
    of series of 10^4 steps for E = 1..20 (16 series, so the GPU is filled),
    and the lookup of 10 libraries against 10^5 targets of 10^4 steps."""
    from paper_2105_12301_gb300 import edm
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    L = 10000
    X = inputs.logistic_long(N=16, L=L)
    Xg = torch.from_numpy(X).to(dev)
    knn = {}
    for E in range(1, E_MAX + 1):
        def one():
            edm.edm_knn(Xg, E, TAU, 0, with_dist=True)
        one()
        ms = sync_time(one, dev, stream, 1)
        rows = X.shape[0] * (L - (E - 1) * TAU)
        knn[str(E)] = {"ms": ms, "rows_per_s": rows / (ms / 1e3)}
        log("knn E=%d %.1f ms" % (E, ms))
    # the paper's two-kernel route (Algorithms 1-2: the n x n distance matrix
    # written to memory, then per-row selection), same results, as a baseline
    knn_mat = {}
    for E in (1, 2, 4, 8, 12, 16, 20):
        def one():
            edm.edm_knn_materialized(Xg, E, TAU, 0, with_dist=True)
        one()
        edm.edm_profile_enable(True, dev)
        ms = sync_time(one, dev, stream, 1)
        split = {k: edm.edm_profile_read(k, dev)[0] for k in ("dmat_kernel", "knn_from_dmat_kernel")}
        edm.edm_profile_enable(False, dev)
        edm.edm_ctx_sync(dev)
        rows = X.shape[0] * (L - (E - 1) * TAU)
        n = L - (E - 1) * TAU
        knn_mat[str(E)] = {"ms": ms, "rows_per_s": rows / (ms / 1e3), "kernel_ms": split,
                           "matrix_bytes_written": 4.0 * n * n * X.shape[0],
                           "fused_ms": knn[str(E)]["ms"]}
        log("knn materialised E=%d %.1f ms %s" % (E, ms, split))
    Y = inputs.ar1_series(100000, L, 2105)
    log("generated targets %s" % (Y.shape,))
    Yg = torch.from_numpy(Y).to(dev)
    del Y
    E_lib = torch.full((X.shape[0],), 3, dtype=torch.int32, device=dev)
    lib = Xg[:10].contiguous()
    rho = torch.empty((10, Yg.shape[0]), dtype=torch.float32, device=dev)
    lookup = {}
    for prec in ("fp32", "bf16"):
        def one():
            edm.edm_ccm_all(lib, Yg, E_lib[:10].contiguous(), TAU, TP, prec, out=rho)
        one()
        edm.edm_profile_enable(True, dev)
        ms = sync_time(one, dev, stream, 1)
        split = {k: edm.edm_profile_read(k, dev)[0] for k in
                 ("target_store_kernel", "ccm_table_kernel", "lookup_kernel")}
        edm.edm_profile_enable(False, dev)
        edm.edm_ctx_sync(dev)
        lookup[prec] = {"ms": ms, "pairs_per_s": 10 * Yg.shape[0] / (ms / 1e3), "kernel_ms": split}
        log("lookup %s %.1f ms %s" % (prec, ms, split))
    out = {"metric": "kNN rows/s and CCM pairs/s at the paper's micro-benchmark shapes",
           "unit": "rows/s, pairs/s", "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "knn: 16 coupled-logistic series x 10,000 steps, E = 1..20, exact "
                                  "order; lookup: 10 libraries (E = 3) x 100,000 AR(1) targets x "
                                  "10,000 steps", "tau": TAU, "Tp": TP},
           "knn": knn, "knn_materialized": knn_mat, "lookup": lookup}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["calcium50k", "calcium2k", "batched", "libsweep",
                                           "paper-micro"], default="calcium50k")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched_workload(args)
    elif args.workload == "libsweep":
        run_libsweep_workload(args)
    elif args.workload == "paper-micro":
        run_paper_micro_workload(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
