#!/usr/bin/env python3
"""Benchmark: multi-mass Wilson solve time to a 1e-10 true residual, and the
hop (dslash) kernels' throughput against the measured GB300 peaks.

One step = the paper's single-mass multi-mass scheme (even-odd
preconditioning, FP64 defect correction around a reduced-precision
BiCGstab, Lagrange initial guesses, masses heaviest first) for every source
of the workload, the sources batched into multimass_solve calls.  The line
also carries the end-to-end time through the public API with host inputs
and outputs, a roofline entry for each hop class that takes a large share
of the step (the inner hop against HBM, the FP64 residual hop against the
FP64 pipe), the FP64 oracle's time on the host cores, the solution error
against stored oracle solutions per mass, and the multi-shift BiCGstab-M
baseline (FP64 and double-float) on the same GPU.

Default workload (--config c5): 48^3 x 96 lattice, synthetic SU(3) links
exp(i 0.7 H), antiperiodic in time, 12 spin-colour point sources at site 0,
16 masses m0 = 0.5 * 0.04^(i/15), FP16-storage inner solves (FP32
arithmetic), FP64 residual recomputation, accumulator and reductions.
--config c3 selects 24^3 x 64, eps 0.5, 12 point sources, 8 masses
m0 = 0.40 .. 0.05, FP32 inner; --config c2 16^3 x 32, one Z2 source (its
working set fits in the 129 MB L2); --outer df the double-float outer loop.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank solves its own
replica of the workload (the solve does not shard: replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "multi-mass solve time to 1e-10 true residual; dslash GB/s vs GB300 HBM peak"
UNIT = "s"
MASSES = [0.40, 0.35, 0.30, 0.25, 0.20, 0.15, 0.10, 0.05]
CONFIGS = {
    "c3": dict(name="24^3x64, 12 spin-colour point sources x 8 masses (m0 0.40..0.05), eps 0.5",
               dims=(24, 24, 24, 64), eps=0.5, seed=3, sources="points12"),
    "c2": dict(name="16^3x32, 1 Z2 source x 8 masses (m0 0.40..0.05), eps 0.5",
               dims=(16, 16, 16, 32), eps=0.5, seed=2, sources="z2"),
    "c1": dict(name="8^4, 1 point source x 4 masses (m0 0.5, 0.3, 0.2, 0.1), eps 0.3",
               dims=(8, 8, 8, 8), eps=0.3, seed=1, sources="point1", masses=[0.5, 0.3, 0.2, 0.1]),
    # 10.6M sites: 16 solutions per source take 33 GB in canonical FP64 and,
    # with the guess through the last 6 masses, 14 GB inside the solver, so
    # the sources go three at a time (223 GB on the device).  Measured on
    # this workload, FP64 outer loop: three sources per call 4.4% faster
    # than two, 4 inner iterations per captured graph 2.5% faster than 8,
    # the Lagrange guess through the last 6 masses 0.7% faster than through
    # the last 8 and 2% faster than through the last 10; FP16 inner solves
    # refined in FP32 segments to 1e-7 take 216 outer steps per step
    # against 289 for one FP16 solve per outer step (7.29 s against 8.29 s
    # with the guess through 8 masses).  The end-to-end run writes the
    # solutions of a call to 98 GB of page-locked host memory
    "c5": dict(name="48^3x96, 12 spin-colour point sources x 16 masses (m0 0.5*0.04^(i/15)), eps 0.7",
               dims=(48, 48, 48, 96), eps=0.7, seed=5, sources="points12",
               masses=[0.5 * 0.04 ** (i / 15.0) for i in range(16)], inner="f16", source_batch=3,
               graph_iters=4, guess_max=6, inner_refine=1, pinned_gb=128, baseline_sources=1, e2e_steps=3),
}
# algorithmic bytes of one hop: per output site 8 links (12 reals: the
# minimum the method must read), per output site and rhs one input spinor
# (each read once) and one output spinor
LINK_B = {"f64": 96, "df": 96, "f32": 48, "f16": 24}
SPINOR_B = {"f64": 192, "df": 192, "f32": 96, "f16": 52}
FLOP_SITE = 1320   # per hop output site and rhs
# DRAM bytes (read + write) per launch of the timed hop kernel from one ncu
# capture, keyed by (precision, autotuner variant, rhs per launch): (half-
# lattice sites of the captured case, bytes).  Traffic scales with sites.
# An entry is valid only for the kernel as it was when captured; remove it
# when that kernel changes.
HOP_TRAFFIC = {("f16", 105, 3): (1048576, 617.48e6), ("f16", 106, 3): (1048576, 617.32e6),
               ("f64", 101, 3): (442368, 1013.01e6), ("f64", 103, 3): (442368, 1024.87e6)}
# FP64 pipe utilisation of the FP64 hop in the same captures
FP64_PIPE = {(101, 3): "92.6% busy in an ncu capture of this variant on 24^3x64, 3 rhs",
             (103, 3): "92.6% busy in an ncu capture of this variant on 24^3x64, 3 rhs"}
# FP64 FMA rate of one GB300 (TFLOP/s, 2 flops per FMA): 152 SMs x 2 FP64
# FMA per clock x 2.07 GHz, the unit count and clock of the part
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
GOLDEN = os.path.join(ROOT, "tests", "golden")


def sources(cfg):
    from paper_1103_5103_gb300 import synth
    d = cfg["dims"]
    if cfg["sources"] == "points12":
        return [synth.point_source(d, s, c) for s in range(4) for c in range(3)]
    if cfg["sources"] == "point1":
        return [synth.point_source(d)]
    return [synth.z2_source(d, seed=3)]


def host_cpu():
    """Host CPU model (lscpu) and logical core count, for the CPU baseline."""
    model = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return f"{model}, {os.cpu_count()} logical cores"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup(backend: str = "nccl"):
    """Replicas only: one independent copy of the workload per rank.  The
    process group carries just the barriers and the max-over-ranks timing
    (NCCL on GPUs; gloo for the CPU tests of this host logic)."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_counts(config):
    """The FP64 oracle's own per-mass BiCGstab iterations and restarts for
    this workload, from tests/golden/<config>_oracle_multimass.json (written
    by tests/golden/make_oracle_multimass.py, which calls only the oracle),
    averaged over the point sources it recorded.  None if there is no such
    file."""
    path = os.path.join(GOLDEN, f"{config}_oracle_multimass.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)
    recs = [r for r in gold["sources"].values() if None not in r["iterations"]]
    if not recs:
        return None
    n = len(gold["masses"])
    iters = [float(np.mean([r["iterations"][i] for r in recs])) for i in range(n)]
    rest = [float(np.mean([r["restarts"][i] for r in recs])) for i in range(n)]
    return {"iterations": iters, "restarts": rest, "sources": sorted(int(k) for k in gold["sources"]),
            "file": os.path.relpath(path, ROOT)}


def oracle_sample(cfg, U, b, iteration=True):
    """Time the FP64 oracle as it stands on this workload's field: one
    application of M_prec and, with iteration, one call of its even-odd
    BiCGstab limited to one iteration (initial residual, the iteration --
    two M_prec and the vector updates --, the restart check and the final
    residual: five applications).  Returns (seconds per M_prec, seconds per
    BiCGstab iteration or None, seconds spent)."""
    from oracle import oracle as O
    dims = cfg["dims"]
    m = cfg.get("masses", MASSES)[-1]
    bp = O.eo_source(U, dims, b, m)
    t0 = time.perf_counter()
    O.apply(O.OP_MPREC, U, dims, bp, O.kappa(m))
    t1 = time.perf_counter()
    if not iteration:
        return t1 - t0, None, t1 - t0
    _, st = O.bicgstab(O.OP_MPREC, U, dims, bp, O.kappa(m), tol=1e-30, maxiter=1)
    t2 = time.perf_counter()
    assert st["iterations"] == 1
    t_mprec = t1 - t0
    return t_mprec, max((t2 - t1) - 3.0 * t_mprec, 0.0), t2 - t0


def oracle_workload_seconds(counts, n_src, t_mprec, t_iter):
    """Oracle time for the whole workload: per source and mass, its
    iterations x t_iter plus the applications around them (initial and final
    residual, one per restart, and the even-odd source, reconstruction and
    full residual, three half-cost full-lattice hops)."""
    per_src = sum(it * t_iter + (4.5 + r) * t_mprec for it, r in zip(counts["iterations"], counts["restarts"]))
    return n_src * per_src


def oracle_threads():
    from oracle import oracle as O
    return O.set_threads(os.cpu_count() or 1)


def run_reference(args, cfg):
    ws, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1103_5103_gb300 import synth
    counts = oracle_counts(args.config) if not getattr(args, "dims", "") else None
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          "no oracle iteration count stored for this workload (tests/golden); the oracle "
                          "cannot run a full step in the time a bench run has"}))
        return
    U = synth.gauge_field(cfg["dims"], cfg["eps"], seed=cfg["seed"])
    bs = sources(cfg)
    threads = oracle_threads()
    # once: the cost of a BiCGstab iteration relative to an application of
    # M_prec; then each step times one application (a few seconds on 48^3x96)
    t_m0, t_it0, _ = oracle_sample(cfg, U, bs[0])
    q = t_it0 / t_m0
    times, last = [], None
    for k in range(args.warmup + args.steps):
        t_m = oracle_sample(cfg, U, bs[0], iteration=False)[0]
        last = (t_m, q * t_m)
        if k >= args.warmup:
            times.append(oracle_workload_seconds(counts, len(bs), last[0], last[1]))
    v = float(np.mean(times))
    its = int(round(len(bs) * sum(counts["iterations"])))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "sources": len(bs), "masses": list(cfg.get("masses", MASSES)),
                       "tol": 1e-10},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": v, "unit": UNIT, "host": host_cpu(),
                             "sample": f"per step, one FP64 oracle M_prec application timed on {threads} host "
                                       f"threads ({last[0]:.2f} s in the last step); one oracle BiCGstab "
                                       f"iteration (two M_prec and its vector updates) costs {q:.2f} of them, "
                                       f"timed once; scaled by the oracle's own {its} iterations for the "
                                       f"workload (mean over the sources {counts['sources']} in "
                                       f"{counts['file']}, times {len(bs)} sources) plus its per-mass operator "
                                       f"applications"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _used_bytes(torch):
    free, total = torch.cuda.mem_get_info()
    return total - free


def roofline_entries(prof, inner, outer, V, peak, peak_kind, nb, hop_variant, outer_variant):
    """One entry per hop class from the solve's live CUDA-event timings: the
    inner hop (D_oe p, the first hop of every inner BiCGstab iteration) is
    bound by HBM bandwidth; the FP64 residual hop (D_oe x, the first hop of
    every outer check) by the FP64 pipe, whose FMA rate GB300 cuts to 1/57
    of FP32.  Each entry also gives the class's estimated share of the step:
    its mean launch time times its launches per step (four hops per inner
    iteration, two per outer check)."""
    out = {}
    pi = prof[inner]
    if pi["launches"]:
        sites = pi["sites"] / pi["launches"]
        site_rhs = pi["site_rhs"] / pi["launches"]
        byts = sites * 8 * LINK_B[inner] + site_rhs * 2 * SPINOR_B[inner]
        avg = pi["ms"] / pi["launches"] / 1e3
        ach = byts / avg / 1e9
        l2 = byts < 129e6
        traffic = None
        if (inner, hop_variant, nb) in HOP_TRAFFIC:
            sites_cap, bytes_cap = HOP_TRAFFIC[(inner, hop_variant, nb)]
            traffic = bytes_cap * (V // 2) / sites_cap
        out["inner"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                        # a hop whose operands fit in the 129 MB L2 is latency-bound:
                        # no HBM fraction is quoted for it
                        "frac": None if l2 else ach / peak, "l2_resident": l2, "traffic": traffic,
                        "kernel": f"k_hop<{inner}> (D_oe p, first hop of each inner BiCGstab iteration), "
                                  f"autotuned variant {hop_variant}, {site_rhs / sites:.0f} rhs per launch",
                        "peak_kind": peak_kind, "bytes_per_launch": byts, "avg_launch_us": avg * 1e6,
                        "timed_launches": pi["launches"], "gflops_1320": FLOP_SITE * site_rhs / avg / 1e9}
    po = prof["outer"]
    if po["launches"]:
        site_rhs = po["site_rhs"] / po["launches"]
        avg = po["ms"] / po["launches"] / 1e3
        tf = FLOP_SITE * site_rhs / avg / 1e12
        if outer == "f64":
            otraffic = None
            if ("f64", outer_variant, nb) in HOP_TRAFFIC:
                sites_cap, bytes_cap = HOP_TRAFFIC[("f64", outer_variant, nb)]
                otraffic = bytes_cap * (V // 2) / sites_cap
            out["outer"] = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tf / FP64_PEAK_TFLOPS, "traffic": otraffic,
                            "fp64_pipe": FP64_PIPE.get((outer_variant, nb)),
                            "kernel": f"k_hop<f64> (D_oe x, first hop of each outer FP64 residual check), "
                                      f"variant {outer_variant}, {site_rhs / (po['sites'] / po['launches']):.2f} "
                                      f"rhs per launch on average",
                            "peak_kind": "FP64 FMA rate from the unit count and clock (152 SMs x 2 FMA/clk "
                                         "x 2.07 GHz)",
                            "flops_per_site": FLOP_SITE, "avg_launch_us": avg * 1e6,
                            "timed_launches": po["launches"]}
        else:
            out["outer"] = {"bound": "alu", "achieved": tf, "peak": None, "unit": "TFLOP/s", "frac": None,
                            "traffic": None, "kernel": "k_hop_rolled<df> (double-float residual hop; FP32-issue "
                                                       "bound)", "avg_launch_us": avg * 1e6,
                            "timed_launches": po["launches"]}
    return out


def golden_errors(config, xs_by_source, masses, dev):
    """Relative l2 error of GPU solutions against the oracle's solutions
    (polished to 1e-13) stored at sampled sites in tests/golden, per mass:
    {source: [error per mass]} for the sources given and recorded."""
    import torch
    path = os.path.join(GOLDEN, f"{config}_oracle_multimass.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)
    sites = torch.tensor(gold["sites"], dtype=torch.long, device=dev)
    out = {}
    for k, xs in xs_by_source.items():
        rec = gold["sources"].get(str(k))
        if rec is None:
            continue
        errs = []
        for i, m in enumerate(masses):
            ref = rec["x"][i]
            if ref is None:
                errs.append(None)
                continue
            want = np.array(ref)[..., 0] + 1j * np.array(ref)[..., 1]
            got = xs[i][sites].cpu().numpy().reshape(len(gold["sites"]), 12)
            errs.append(float(np.linalg.norm(got - want) / np.linalg.norm(want)))
        out[str(k)] = errs
    return out


def run_ours(args, cfg):
    import torch
    from paper_1103_5103_gb300 import api, synth

    ws, rank, local = dist_setup()
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    dims = cfg["dims"]
    masses = list(cfg.get("masses", MASSES))
    inner = args.inner or cfg.get("inner", "f32")
    outer = args.outer
    t0 = time.time()
    U = synth.gauge_field(dims, cfg["eps"], seed=cfg["seed"])
    bs_h = sources(cfg)
    gen_s = time.time() - t0
    torch.cuda.synchronize()
    mem0 = _used_bytes(torch)
    lat = api.Lattice(dims)
    U_dev = torch.from_numpy(U).to(dev)
    V = lat.volume
    nr, nm = len(bs_h), len(masses)
    nb = args.source_batch or cfg.get("source_batch", nr)
    batches = [list(range(i, min(nr, i + nb))) for i in range(0, nr, nb)]
    # workers: batches solved at the same time, each on its own stream and
    # gauge handle (a handle serialises its calls), with its own solution
    # buffers; the FP64 residual hops of one overlap the inner solves of
    # another when they run on a small grid (outer_blocks_per_sm)
    nw = max(1, min(len(batches), args.streams or cfg.get("streams", 1)))
    # links of the two precisions the solve uses
    refine = args.inner_refine if args.inner_refine is not None else cfg.get("inner_refine", 0)
    refine = int(refine) if inner == "f16" else 0
    gs = [api.Gauge(lat, U_dev, precs=tuple(sorted({inner, outer} | ({"f32"} if refine else set()))))
          for _ in range(nw)]
    g = gs[0]
    bs = [torch.from_numpy(b).to(dev) for b in bs_h]
    # solution buffers for one batch of sources per worker, reused by its batches
    xs_w = [[[torch.empty((V, 4, 3), dtype=torch.complex128, device=dev) for _ in masses] for _ in range(nb)]
            for _ in range(nw)]
    xs = xs_w[0]
    ob = args.outer_blocks if args.outer_blocks >= 0 else cfg.get("outer_blocks", 0)
    graph_iters = args.graph_iters if args.graph_iters is not None else cfg.get("graph_iters", 8)
    guess_max = args.guess_max if args.guess_max is not None else cfg.get("guess_max", 0)
    pinned_gb = args.pinned_gb if args.pinned_gb is not None else cfg.get("pinned_gb", 24.0)
    prm = api.params(inner_prec=inner, rhs_block=args.rhs_block, outer_prec=outer,
                     inner_tol=args.inner_tol, reliable=int(args.reliable), guess_max=guess_max,
                     verify_full=int(args.verify_full), outer_blocks_per_sm=ob if outer == "f64" else 0,
                     graph_iters=graph_iters, inner_refine=refine,
                     inner_solver=api.SOLVER_CG if args.inner_solver == "cg" else api.SOLVER_BICGSTAB,
                     mode={"graph": api.MODE_GRAPH, "persistent": api.MODE_PERSISTENT, "host": api.MODE_HOST}[args.mode])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    wstreams = [stream] if nw == 1 else [torch.cuda.Stream(device=dev) for _ in range(nw)]
    owner = {bi: bi % nw for bi in range(len(batches))}   # batch -> worker

    def solve_batch(bi, srcs=None, outs=None):
        w = owner[bi]
        rows = batches[bi]
        _, st = api.multimass_solve(gs[w], srcs or [bs[r] for r in rows], masses, prm,
                                    xs=outs or xs_w[w][:len(rows)], stream=wstreams[w])
        return st

    def run_batches(fn):
        """fn(bi) for every batch: in order on one stream, or batch bi on
        worker bi % nw, the workers in threads of their own (the library
        releases the interpreter lock in every call).  The workers' streams
        start after the work already queued on the main stream, and the
        main stream waits for all of them."""
        if nw == 1:
            return [fn(bi) for bi in range(len(batches))]
        ev0 = torch.cuda.Event()
        ev0.record(stream)
        for ws_ in wstreams:
            ws_.wait_event(ev0)
        out, errs = [None] * len(batches), []

        def work(w):
            try:
                for bi in range(w, len(batches), nw):
                    out[bi] = fn(bi)
            except BaseException as e:   # re-raised in the main thread
                errs.append(e)
        th = [threading.Thread(target=work, args=(w,)) for w in range(nw)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errs:
            raise errs[0]
        for ws_ in wstreams:
            ev = torch.cuda.Event()
            ev.record(ws_)
            stream.wait_event(ev)
        return out

    def step():
        st = []
        for r in run_batches(solve_batch):
            st += r
        return st

    # the first pass runs the batches one after another: each handle tunes
    # its hop variants on its first call, with CUDA-event timings that
    # concurrent work would disturb
    for bi in range(len(batches)):
        solve_batch(bi)
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    footprint = _used_bytes(torch) - mem0
    # timed region: flush L2 before each step (inputs are also larger than L2)
    barrier(ws)
    torch.cuda.synchronize()
    for gw in gs:
        api.profile_enable(gw, True)
    launches0 = api.launch_count()
    clocks = ClockSampler(dev.index or 0)
    step_ms = []
    all_stats = None
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if args.ncu_step and k == 0:
            torch.cuda.profiler.start()   # with ncu --profile-from-start off: capture this step only
        a.record(stream)
        all_stats = step()
        b.record(stream)
        b.synchronize()
        if args.ncu_step and k == 0:
            torch.cuda.profiler.stop()
        step_ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = (api.launch_count() - launches0) / max(1, args.steps)
    prof = api.profile_read(g)   # worker 0's handle
    for gw in gs:
        api.profile_enable(gw, False)
    hop_variant = api.autotune(g, inner, nb)[0]   # the cached choices the solves used
    outer_variant = (7000 + 100 * min(nb, 2) + ob) if (ob and outer == "f64") else api.autotune(g, outer, nb)[0]
    barrier(ws)
    t_step = max_over_ranks(float(np.mean(step_ms)) / 1e3, ws)

    # end to end through the public API, inputs in and results out of
    # page-locked host memory.  When every solution of a batch fits in
    # 24 GB of pinned memory the solver reads the sources from and writes
    # the solutions to host memory itself (unified addressing over the
    # host link); otherwise each batch's sources are copied in and every
    # solution is copied out through an 8 GB pinned ring.  The copy path is
    # also timed, for comparison.
    e2e_steps = max(1, min(args.steps, cfg.get("e2e_steps", args.steps)))
    bs_pin = [torch.from_numpy(b).pin_memory() for b in bs_h]
    x_bytes = V * 12 * 16
    h2d = sum(b.numel() * 16 for b in bs_pin)
    d2h = nr * nm * x_bytes

    def e2e_copy():
        # an 8 GB pinned ring per worker for the solutions
        n_slots = max(1, min(nr * nm, (8 << 30) // x_bytes // nw))
        slots = [[torch.empty((V, 4, 3), dtype=torch.complex128, pin_memory=True) for _ in range(n_slots)]
                 for _ in range(nw)]
        count = [0] * nw

        def one(bi):
            w = owner[bi]
            with torch.cuda.stream(wstreams[w]):
                for r in batches[bi]:
                    bs[r].copy_(bs_pin[r], non_blocking=True)
                st = solve_batch(bi)
                for j in range(len(batches[bi])):
                    for i in range(nm):
                        slots[w][count[w] % n_slots].copy_(xs_w[w][j][i], non_blocking=True)
                        count[w] += 1
            return st

        times = []
        for _ in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run_batches(one)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
        return float(np.mean(times)) / 1e3

    def e2e_zero_copy():
        xh = [[[torch.empty((V, 4, 3), dtype=torch.complex128, pin_memory=True) for _ in masses] for _ in range(nb)]
              for _ in range(nw)]
        times = []
        for _ in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run_batches(lambda bi: solve_batch(bi, [bs_pin[r] for r in batches[bi]],
                                               xh[owner[bi]][:len(batches[bi])]))
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
        return float(np.mean(times)) / 1e3

    zero_copy = nw * nb * nm * x_bytes <= pinned_gb * (1 << 30)
    t_e2e_copy = max_over_ranks(e2e_copy(), ws)
    t_e2e = max_over_ranks(e2e_zero_copy(), ws) if zero_copy else t_e2e_copy

    # solution error against the oracle's stored solutions (untimed): the
    # last batch is still in xs; the first batch is solved once more
    errors = None
    if rank == 0 and not args.dims:
        torch.cuda.synchronize()
        last = len(batches) - 1
        errors = golden_errors(args.config, {r: xs_w[owner[last]][j] for j, r in enumerate(batches[last])},
                               masses, dev) or {}
        if last > 0:
            solve_batch(0)
            torch.cuda.synchronize()
            errors.update(golden_errors(args.config, {r: xs_w[owner[0]][j] for j, r in enumerate(batches[0])},
                                        masses, dev) or {})

    peak, peak_kind = measured_peaks()
    roof = roofline_entries(prof, inner, outer, V, peak, peak_kind, nb, hop_variant, outer_variant)
    iters = sum(st["iterations"] for row in all_stats for st in row)
    restarts = sum(st["restarts"] for row in all_stats for st in row)
    # launches per step of each hop class: four hops per inner iteration of a
    # batch (the slowest rhs sets the batch's count), two per outer check
    inner_hops = 4 * sum(max(all_stats[r][i]["iterations"] for r in rows) for rows in batches for i in range(nm))
    outer_hops = 2 * sum(max(all_stats[r][i]["restarts"] for r in rows) for rows in batches for i in range(nm))
    for key, n_h in (("inner", inner_hops), ("outer", outer_hops)):
        if key in roof:
            roof[key]["launches_per_step_est"] = n_h
            roof[key]["step_share_est"] = n_h * roof[key]["avg_launch_us"] * 1e-6 / t_step
    dominant = max(roof, key=lambda k: roof[k]["step_share_est"]) if roof else None
    worst = max(st["true_relres"] for row in all_stats for st in row)
    per_mass = {}
    for i, m in enumerate(masses):
        e = {"iterations": int(sum(all_stats[r][i]["iterations"] for r in range(nr))),
             "restarts": int(sum(all_stats[r][i]["restarts"] for r in range(nr))),
             "seconds": float(sum(all_stats[rows[0]][i]["seconds"] for rows in batches)),
             "max_true_relres": float(max(all_stats[r][i]["true_relres"] for r in range(nr)))}
        if errors:
            e["oracle_error"] = {k: v[i] for k, v in errors.items()}
        per_mass[f"{m:.4g}"] = e

    dtype = {"f16": "f16 storage, f32 arithmetic", "f32": "f32", "f64": "f64"}[inner]
    line = {
        "metric": METRIC, "value": t_step, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{outer} outer loop; inner solves in {dtype}", "data": "synthetic",
        "config": {"workload": cfg["name"], "sources": nr, "source_batch": nb, "masses": masses,
                   "inner_prec": inner, "outer_prec": outer,
                   "outer_arithmetic": ("FP64 residual recomputation b - M x, FP64 solution accumulator, FP64 "
                                        "global reductions") if outer == "f64" else
                                       "double-float (about 48-bit) residual, accumulator and reconstruction",
                   "inner_tol": args.inner_tol or "library default", "mode": args.mode,
                   "graph_iters": graph_iters,
                   "inner_refine": ("FP16 segments, inner residual recomputed in FP32 between them, to "
                                    f"{args.inner_tol or 1e-7:g} of each outer residual") if refine else None,
                   "guess_max": guess_max or "all earlier masses",
                   "outer_loop": "reliable updates" if args.reliable else "restarted defect correction",
                   "inner_solver": "CG on the normal equations" if args.inner_solver == "cg" else "BiCGstab",
                   "full_residual": "recomputed with a hop D_eo x_o" if args.verify_full else
                                    "even half from the last FP64 check, odd half from the reconstruction",
                   "concurrent_batches": nw, "outer_blocks_per_sm": ob if outer == "f64" else None,
                   "tol": 1e-10, "l2": "flushed (256 MB write) before every step; working set > L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "e2e": {"value": t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "transfer": ("the solver reads the sources from and writes the solutions to page-locked host "
                             "memory (unified addressing)") if zero_copy else
                            "cudaMemcpy from pinned sources and to an 8 GB pinned ring",
                "steps": e2e_steps, "explicit_copies_value": t_e2e_copy},
        "gpu_launches": int(round(launches)),
        "roofline": dict(roof[dominant], hop_class=dominant) if dominant else None,
        "rooflines": roof,
        "clocks": clk,
        "iterations_per_step": int(iters), "restarts_per_step": int(restarts), "max_true_relres": worst,
        "per_mass": per_mass,
        "device_memory_gb": footprint / 1e9,
        "gauge_generation_s": gen_s,
    }
    if errors:
        line["oracle_error_max"] = max(e for v in errors.values() for e in v if e is not None)
        line["oracle_error_sources"] = sorted(int(k) for k in errors)
    if rank == 0 and ws == 1 and not args.no_baseline:
        # BiCGstab-M on the same GPU, same sources and masses (context for the
        # paper's comparison; not part of the timed step), with its vectors
        # and hops in FP64 and in double-float.  Each on a fresh handle with
        # only the links it uses, so its footprint is its own.
        for gw in gs:
            gw.close()
        del g, gs, xs, xs_w
        # with rhat = b a point source breaks the recurrences down at once
        # (<b, r_1> = 0): such sources get a Gaussian shadow residual
        point = cfg["sources"].startswith("point")
        shadow = torch.from_numpy(synth.gaussian_source(dims, seed=cfg["seed"] + 1000)).to(dev) if point else None
        nsrc = min(nr, args.baseline_sources or cfg.get("baseline_sources", nr))
        for key, bo, precs in (("bicgstab_m_fp64", "f64", ("f64",)), ("bicgstab_m_df", "df", ("df", "f32"))):
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            mem1 = _used_bytes(torch)
            gm = api.Gauge(lat, U_dev, precs=precs)
            prm_m = api.params(shadow=shadow, outer_prec=bo)
            t_m, it_m, worst_m, mem_m, polished = 0.0, 0, 0.0, 0, 0
            per_shift = None
            for r in range(nsrc):
                xm = [torch.empty((V, 4, 3), dtype=torch.complex128, device=dev) for _ in masses]
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                stm = api.bicgstab_m_solve(gm, bs[r], xm, masses, prm_m, check=False)
                torch.cuda.synchronize()
                t_m += time.perf_counter() - t0
                mem_m = max(mem_m, _used_bytes(torch) - mem1)
                it_m += max(s["iterations"] for s in stm)
                worst_m = max(worst_m, max(s["true_relres"] for s in stm))
                per_shift = [int(s["iterations"]) for s in stm]
                polished += sum(1 for s in stm if s["restarts"] > 0)
                del xm
            gm.close()
            del gm
            line[key] = {"seconds_per_step": t_m * nr / nsrc, "sources_run": nsrc,
                         "vectors_and_hops": "double-float" if bo == "df" else "FP64",
                         "iterations_per_source": it_m / nsrc, "max_true_relres": worst_m,
                         "iterations_per_mass_last_source": per_shift,
                         "shadow_residual": "Gaussian noise" if point else "b",
                         "masses_polished_by_single_mass": polished,
                         "device_memory_gb": mem_m / 1e9,
                         "speedup_of_single_mass_scheme": (t_m * nr / nsrc) / t_step}
    if rank == 0 and ws == 1 and not args.no_cpu:
        counts = oracle_counts(args.config) if not args.dims else None
        threads = oracle_threads()
        t_mprec, t_iter, spent = oracle_sample(cfg, U, bs_h[0])
        if counts is not None:
            its = int(round(nr * sum(counts["iterations"])))
            v = oracle_workload_seconds(counts, nr, t_mprec, t_iter)
            src = (f"the oracle's own {its} iterations for the workload (mean over the sources "
                   f"{counts['sources']} in {counts['file']}, times {nr} sources)")
        else:
            # no stored oracle count for this lattice: the step's own inner
            # iteration count stands in (said so in the sample string)
            v = iters * t_iter + nr * nm * 4.5 * t_mprec
            src = f"this run's {iters} inner iterations (no stored oracle count for this lattice)"
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "host": host_cpu(),
                                "sample": f"one FP64 oracle M_prec application ({t_mprec:.2f} s) and one oracle "
                                          f"BiCGstab iteration ({t_iter:.2f} s: two M_prec and the vector "
                                          f"updates) on {threads} host threads, {spent:.1f} s in all; scaled by "
                                          f"{src} plus the per-mass operator applications"}
        if threads > 1:
            # the same estimate on one thread: one application of M_prec
            # timed there; an iteration's two applications take that time,
            # its vector updates (not threaded in the oracle) the time above
            from oracle import oracle as O
            O.set_threads(1)
            t1 = oracle_sample(cfg, U, bs_h[0], iteration=False)[0]
            O.set_threads(threads)
            t_iter1 = t_iter + 2.0 * (t1 - t_mprec)
            v1 = (oracle_workload_seconds(counts, nr, t1, t_iter1) if counts is not None
                  else iters * t_iter1 + nr * nm * 4.5 * t1)
            line["cpu_baseline"]["single_thread"] = {
                "value": v1, "unit": UNIT, "cores": 1, "mprec_s": t1,
                "sample": f"one M_prec application on one thread ({t1:.2f} s); a BiCGstab iteration "
                          f"{t_iter1:.2f} s; the workload scaled as above"}
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="c5")
    ap.add_argument("--inner", choices=["f32", "f16", "f64"], default=None,
                    help="inner precision (default: the workload's, f32 unless it names one)")
    ap.add_argument("--outer", choices=["f64", "df"], default="f64",
                    help="precision of the residual recomputation, accumulator and reconstruction")
    ap.add_argument("--streams", type=int, default=0,
                    help="batches solved at the same time on their own streams and handles (default: the "
                         "workload's, else 1)")
    ap.add_argument("--outer-blocks", type=int, default=-1,
                    help="FP64 residual hops as a grid-stride kernel of this many blocks per SM (0: full grid; "
                         "default: the workload's)")
    ap.add_argument("--pinned-gb", type=float, default=None,
                    help="page-locked host memory the end-to-end run may use for one batch's solutions: "
                         "within it the solver writes them to host memory itself, beyond it they are copied "
                         "out through an 8 GB ring")
    ap.add_argument("--graph-iters", type=int, default=None,
                    help="inner iterations per captured CUDA graph (default: the workload's, else 8)")
    ap.add_argument("--guess-max", type=int, default=None,
                    help="earlier masses the Lagrange guess uses (0: all, the paper's choice; default: the "
                         "workload's, else 0)")
    ap.add_argument("--inner-refine", type=int, choices=[0, 1], default=None,
                    help="FP16 inner solves in FP16 segments with FP32 residual recomputation between them "
                         "(default: the workload's, else 0)")
    ap.add_argument("--verify-full", action="store_true",
                    help="recompute the even half of the full residual with one more hop per mass")
    ap.add_argument("--rhs-block", type=int, default=0)
    ap.add_argument("--inner-tol", type=float, default=0.0)
    ap.add_argument("--mode", choices=["graph", "persistent", "host"], default="graph")
    ap.add_argument("--inner-solver", choices=["bicgstab", "cg"], default="bicgstab")
    ap.add_argument("--dims", default="",
                    help="run the workload on another lattice, e.g. 32x32x32x64 (profiling of a smaller case)")
    ap.add_argument("--reliable", action="store_true",
                    help="reliable updates instead of restarted defect correction in the mixed-precision loop")
    ap.add_argument("--baseline-sources", type=int, default=0,
                    help="sources for the BiCGstab-M comparison (default: the workload's, else all)")
    ap.add_argument("--source-batch", type=int, default=0,
                    help="sources per multimass_solve call (default: the workload's, else all)")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ncu-step", action="store_true",
                    help="bracket the first timed step with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    cfg = dict(CONFIGS[args.config])
    if args.dims:
        # profiling aid: the workload's sources, masses and precisions on a
        # smaller lattice (the line's workload name says so)
        cfg["dims"] = tuple(int(v) for v in args.dims.split("x"))
        cfg["name"] = cfg["name"] + f", run on {args.dims}"
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
