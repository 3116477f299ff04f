"""Benchmark: batched LAD-LASSO fits on one GB300 (or N, one process each).

Workload (default): 4096 row-subset problems of a shared 2000 x 32 N(0,1)
matrix, n ~ U{50..2000}, p ~ U{4..32}, 16 lambdas from lambda_max down to
1e-3 lambda_max with warm starts.  One step = lambda_max + lambda path +
the full fit (coordinate descent, ternary chop, exact polish) of every
(problem, lambda) pair, all in this library's kernels.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (bounded samples of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_15649_gb300 import synth  # noqa: E402

def workload(B: int, L: int) -> str:
    """The batched workload's name with the problem and path sizes in use
    (4096 and 16 by default)."""
    return (f"batched {B} problems, shared X 2000x32, n~U[50,2000], p~U[4,32], "
            f"L={L} (1e-3 path)")
METRIC = "LAD-LASSO fits/s (certified, rel. obj err <= 1e-5 vs FP64 oracle)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--problems", type=int, default=4096)
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--parity-sample", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-thread", action="store_true", help="skip the thread-per-fit comparison")
    ap.add_argument("--thread-full", action="store_true",
                    help="time the thread-per-fit kernel on the headline workload itself (minutes) "
                         "instead of the 608-problem subset")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson arrival trace")
    ap.add_argument("--serve-rate", type=float, default=20000.0, help="requests/s offered")
    ap.add_argument("--serve-light-rate", type=float, default=1000.0,
                    help="requests/s of a second trace offered below capacity (0: none)")
    ap.add_argument("--serve-light-seconds", type=float, default=3.0)
    ap.add_argument("--serve-classes", action="store_true",
                    help="also serve the trace with slot classes (ClassedServer)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 20000 x 128 block-per-fit measurement")
    ap.add_argument("--large-problems", type=int, default=256)
    ap.add_argument("--large-lambdas", type=int, default=32)
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the option variants timed beside the headline (four-section chop, "
                         "chop off, looser descent)")
    ap.add_argument("--no-cv", action="store_true",
                    help="skip the cross-validation measurement (256 data sets x 5 folds x 16 lambdas)")
    ap.add_argument("--no-diff", action="store_true",
                    help="skip the forward + adjoint measurement (512 x 400/100 x 16)")
    ap.add_argument("--no-tune", action="store_true", help="library's default launch shape")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step eagerly instead of replaying a CUDA graph")
    ap.add_argument("--shard", default="weak", choices=["weak", "cost"],
                    help="N > 1: weak = a batch of --problems per rank (default); cost = one "
                         "batch of --problems split across ranks in contiguous shares balanced "
                         "by n*p*L (strong scaling)")
    ap.add_argument("--launch", default=None,
                    help="fixed launch shape GxF/oW (threads per fit, fits per block, work "
                         "order), e.g. 32x3/o0; skips the autotuner")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """FP64 CPU oracle on bounded samples of the same workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    batch = synth.batched(B=args.problems, seed=1)
    cores = os.cpu_count() or 1
    per_step = max(4, min(64, cores * 2))
    lm = []
    for q in range(per_step * (args.steps + args.warmup)):
        lm.append(oracle.lambda_max(*oracle.problem(batch, q % args.problems)))
    times = []
    for s in range(args.warmup + args.steps):
        qs = np.arange(s * per_step, (s + 1) * per_step) % args.problems
        expo = np.arange(args.L) / max(1, args.L - 1)  # lambda_max down to 1e-3 lambda_max
        lams = np.array(lm[s * per_step:(s + 1) * per_step])[:, None] * (1e-3 ** expo)[None, :]
        lam_full = np.zeros((args.problems, args.L))
        lam_full[qs] = lams
        t0 = time.perf_counter()
        r = oracle.fit_batch(batch, lam_full, problems=qs, nthreads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
        used = r["threads"]
    fits = per_step * args.L
    v = fits / statistics.median(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "fits/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.problems, args.L), "sample": f"{per_step} problems x {args.L} lambdas per step"},
            "cpu_baseline": {"value": v, "unit": "fits/s", "cores": used, "kind": "oracle",
                             "sample": f"{per_step} problems x {args.L} lambdas per step"},
            "e2e": {"value": v, "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm

def log2_histogram(a) -> dict:
    """Counts of the values of `a` in the buckets [0], [1], [2, 3], [4, 7],
    ... (powers of two); edges are the buckets' lower ends."""
    a = np.asarray(a).ravel()
    top = int(a.max()) if a.size else 0
    edges = [0, 1]
    while edges[-1] <= top:
        edges.append(edges[-1] * 2)
    counts = np.histogram(a, bins=np.array(edges, dtype=np.float64) - 0.5)[0]
    return {"lower_edges": edges[:-1], "counts": counts.astype(int).tolist()}


def batch_rows(batch, q):
    """Design rows and targets of problem q of a batch whose slots are rows
    of X (row_idx None)."""
    o0, o1 = int(batch["offsets"][q]), int(batch["offsets"][q + 1])
    return batch["X"][o0:o1], batch["y"][o0:o1]


def row_updates(batch, counters, B):
    """Row-updates per launch: one row's part in one 1-D weighted-median
    step (an axis step, a chop probe's axis step or a polish edge search),
    i.e. n x the fit's 1-D steps (counter slot 5), summed over fits."""
    n = np.diff(batch["offsets"])[:B].astype(np.float64)
    sel = counters[:, :, 5].astype(np.float64)
    return float(np.sum(sel * n[:, None]))


def smem_bytes(batch, counters, B):
    """Algorithmic shared-memory bytes per launch of the one-warp fit kernel:
    every selection pass reads each row's column element and residual (8 B
    a row; counter slot 4 counts passes) and every 1-D step ends with the
    residual update, which reads both and writes the residual (12 B a row;
    slot 5 counts steps).  20 B per row-update when a step takes one pass."""
    n = np.diff(batch["offsets"])[:B].astype(np.float64)
    passes = counters[:, :, 4].astype(np.float64)
    sel = counters[:, :, 5].astype(np.float64)
    return float(np.sum((8.0 * passes + 12.0 * sel) * n[:, None]))


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2510_15649_gb300 import build as _b
    if rank == 0:
        _b.build()
    if dist is not None:
        dist.barrier()
    from paper_2510_15649_gb300 import ladlasso as ll

    B, L = args.problems, args.L
    shard = (0, B)
    if args.shard == "cost":
        # strong scaling: one batch, each rank fits a contiguous share whose
        # cost (n * p * L per problem) is within one problem of 1/world
        from paper_2510_15649_gb300.dist import cost_share
        batch, shard = cost_share(synth.batched(B=B, seed=1), L, rank, world)
        B = shard[1] - shard[0]
    else:
        batch = synth.batched(B=B, seed=1 + 1000 * rank)  # weak scaling: one batch per rank
    dev = torch.device("cuda", local)
    pr = ll.Problems.from_numpy(batch, device=dev)
    ws = ll.workspace(pr, L)
    out = dict(b=torch.empty((B, L, pr.P), device=dev), obj=torch.empty((B, L), device=dev),
               status=torch.empty((B, L), dtype=torch.int32, device=dev),
               counters=torch.empty((B, L, 8), dtype=torch.int32, device=dev))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # launch shape: autotuned on the problem set (outside the timed region)
    launch, tuned = None, {}
    if args.launch:
        g_, rest = args.launch.split("x")
        f_, o_ = rest.split("/o")
        launch = ll.Launch(int(g_), int(f_), int(o_))
    elif not args.no_tune:
        from paper_2510_15649_gb300 import tune
        lam0 = ll.lambda_path(ll.lambda_max(pr, ws), L, 1e-3)
        # timed on the whole problem set: a sample times the tail differently
        # (half the problems picked 5 fits per block, 6 % slower on the set)
        launch, tuned = tune.autotune(pr, lam0, sample_problems=B, repeats=1)
        log(f"autotune {launch} {tuned}")

    lmax_buf = torch.empty(B, device=dev)
    lam_buf = torch.empty((B, L), device=dev)

    def eager_step():
        lmax_buf.copy_(ll.lambda_max(pr, ws))
        lam_buf.copy_(ll.lambda_path(lmax_buf, L, 1e-3))
        ll.fit(pr, lam_buf, ws=ws, out=out, launch=launch)
        return lam_buf

    # the step (lambda_max, path, fit: five launches) captured once in a CUDA
    # graph and replayed; eager if capture is unavailable
    step, graph_note = eager_step, "eager (--no-graph)"
    if not args.no_graph:
        try:
            sg = torch.cuda.Stream()
            sg.wait_stream(stream)
            with torch.cuda.stream(sg):
                eager_step()  # sets launch attributes outside capture
            stream.wait_stream(sg)
            torch.cuda.synchronize()
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cg, capture_error_mode="relaxed"):
                eager_step()

            def graph_step():
                cg.replay()
                return lam_buf
            step, graph_note = graph_step, "CUDA graph replay"
        except Exception as ex:  # report, keep the eager step
            step, graph_note = eager_step, f"eager (capture failed: {ex})"
            torch.cuda.synchronize()

    launches_per_step = 6  # 2 offset checks, lambda_max, lambda_path, work order, fit
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        lam = step()
    torch.cuda.synchronize()
    log(f"warmup {args.warmup} steps {time.perf_counter() - t0:.2f}s")
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush between timed steps (outside the events)
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lam = step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    t_step = statistics.median(times)
    log(f"timed steps {times}")
    from paper_2510_15649_gb300.dist import max_over_ranks
    t_step = max_over_ranks(t_step, dist, dev)  # the slowest rank sets the job time
    st = out["status"].cpu().numpy()
    cnt = out["counters"].cpu().numpy()
    certified = int(np.sum((st & 3) == 0))
    fits = B * L
    from paper_2510_15649_gb300.dist import sum_over_ranks
    certified_all = sum_over_ranks(certified, dist, dev)  # the fits every rank certified
    value = certified_all / t_step
    coverage_ok = None
    if args.shard == "cost":
        # the shares reassemble the batch: every problem fitted by exactly one rank
        from paper_2510_15649_gb300.dist import covered_once
        coverage_ok = covered_once(shard[0], shard[1], args.problems, dist, dev)

    # kernel-only time of the fit launch (events on the launching stream)
    lam_fixed = lam.clone()
    kt = []
    for _ in range(3):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ll.fit(pr, lam_fixed, ws=ws, out=out, launch=launch)
        e1.record(stream)
        torch.cuda.synchronize()
        kt.append(e0.elapsed_time(e1) / 1e3)
    t_fit = statistics.median(kt)
    log(f"fit kernel {kt}")

    # end to end through the public API with pinned host buffers
    hX = torch.as_tensor(batch["X"]).pin_memory()
    hy = torch.as_tensor(batch["y"]).pin_memory()
    hri = torch.as_tensor(batch["row_idx"]).pin_memory()
    hoff = torch.as_tensor(batch["offsets"]).pin_memory()
    hp = torch.as_tensor(batch["p"]).pin_memory()
    hb = torch.empty((B, L, pr.P)).pin_memory()
    hobj = torch.empty((B, L)).pin_memory()
    hst = torch.empty((B, L), dtype=torch.int32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (hX, hy, hri, hoff, hp))
    d2h = sum(t.numel() * t.element_size() for t in (hb, hobj, hst))
    et = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p2 = ll.Problems(X=hX.to(dev, non_blocking=True), y=hy.to(dev, non_blocking=True),
                         offsets=hoff.to(dev, non_blocking=True),
                         row_idx=hri.to(dev, non_blocking=True), p=hp.to(dev, non_blocking=True),
                         P=pr.P, n_max=pr.n_max)
        lm = ll.lambda_max(p2, ws)
        lam2 = ll.lambda_path(lm, L, 1e-3)
        o2 = ll.fit(p2, lam2, ws=ws, launch=launch)
        hb.copy_(o2["b"], non_blocking=True)
        hobj.copy_(o2["obj"], non_blocking=True)
        hst.copy_(o2["status"], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        et.append(e0.elapsed_time(e1) / 1e3)
    t_e2e = max_over_ranks(statistics.median(et), dist, dev)
    log(f"e2e {et}")

    line = {"metric": METRIC, "value": value, "unit": "fits/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "higher_is_better": True, "scaling": "strong" if args.shard == "cost" else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload(args.problems, L), "problems_per_gpu": B, "lambdas": L,
                       "fits_per_gpu": fits, "l2": "flushed between timed steps (256 MB write)",
                       "step": graph_note,
                       "launch": None if launch is None else {
                           "group_threads": launch.group_threads,
                           "fits_per_block": launch.fits_per_block,
                           "work_order": launch.work_order,
                           "autotune_ms": {f"{c.group_threads}x{c.fits_per_block}/o{c.work_order}":
                                           round(1e3 * t, 2) for c, t in tuned.items()}}},
            "certified_fraction": certified / fits,
            "gpu_launches": launches_per_step * args.steps,
            "problems_per_s": (args.problems if args.shard == "cost" else B * world) / t_step,
            "e2e": {"value": certified_all / t_e2e, "unit": "fits/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}
    if args.shard == "cost":
        line["config"].update(shard="cost", problems_total=args.problems,
                              rank0_share=list(shard), coverage_ok=coverage_ok)

    # parity on a sample of fits against the FP64 oracle
    if rank == 0 and args.parity_sample > 0:
        import oracle
        oracle.build()
        bh = out["b"].cpu().numpy()
        lh = lam.cpu().numpy()
        rng = np.random.default_rng(123)
        qs = sorted(rng.choice(B, args.parity_sample, replace=False).tolist())
        worst = 0.0
        fails = 0
        for q in qs:
            X, y = oracle.problem(batch, q)
            ref = oracle.fit_path(X, y, lh[q].astype(np.float64))
            for l in range(L):
                fg = oracle.objective(X, y, bh[q, l, :X.shape[1]].astype(np.float64), float(lh[q, l]))
                e = abs(fg - ref["f"][l]) / max(1.0, ref["f"][l])
                worst = max(worst, e)
                fails += e > 1e-5
        line["parity_sample"] = {"problems": qs, "fits": len(qs) * L, "worst_rel_obj": worst,
                                 "fails": int(fails)}

    # roofline of the fit kernel: shared-memory bandwidth, the bound for
    # designs held in shared memory.  Algorithmic bytes from the kernel's own
    # pass and step counters (smem_bytes) against 32 banks x 4 B per clock
    # per SM at the sampled clock; the ALU view (6 flops per row-update
    # against the FP32 FMA peak) is reported beside it
    ru = row_updates(batch, cnt, B)
    sb = smem_bytes(batch, cnt, B)
    clk_s = clk.summary()
    mhz = clk_s.get("sm_mhz") or 1900.0
    smem_peak = 152 * 32 * 4 * mhz * 1e6 / 1e9
    smem_ach = sb / t_fit / 1e9
    line["roofline"] = {"bound": "smem", "achieved": smem_ach, "peak": smem_peak,
                        "unit": "GB/s", "frac": smem_ach / smem_peak, "traffic": None,
                        "peak_source": "152 SMs x 128 B/clock x sampled SM clock",
                        "kernel": "fit_block_kernel", "kernel_ms": 1e3 * t_fit,
                        "bytes_per_launch": sb, "row_updates_per_launch": ru,
                        "bytes_per_row_update": sb / max(1.0, ru)}
    flops_per_ru = 6.0  # key (div+add), weight accumulate/compare, residual FMA
    alu_ach = flops_per_ru * ru / t_fit / 1e12
    alu_peak = 152 * 128 * 2 * mhz * 1e6 / 1e12  # FP32 FMA lanes x clock
    line["roofline_alu"] = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak,
                            "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
                            "flops_per_row_update": flops_per_ru, "kernel": "fit_block_kernel"}
    line["clocks"] = clk_s
    # per-fit counters of the last timed step (work the method did)
    def pct(a):
        return {"mean": float(np.mean(a)), "p50": float(np.percentile(a, 50)),
                "p99": float(np.percentile(a, 99)), "max": float(np.max(a))}
    fl = cnt[..., 3]
    line["counters"] = {"sweeps": pct(cnt[..., 0]), "chop_probes": pct(cnt[..., 1]),
                        "polish_pivots": pct(cnt[..., 2]),
                        "selection_passes_per_select": float(cnt[..., 4].sum() / max(1, cnt[..., 5].sum())),
                        "ccd_point_optimal": float(np.mean((fl & 1) != 0)),
                        "chop_ran": float(np.mean((fl & 2) != 0)),
                        "chop_point_optimal": float(np.mean((fl & 4) != 0)),
                        # SM cycles per fit spent in descent + chop and in the
                        # basis / polish work (counter slots 6 and 7)
                        "descent_chop_cycle_share": float(
                            cnt[..., 6].astype(np.float64).sum()
                            / max(1.0, cnt[..., 6:8].astype(np.float64).sum())),
                        "histograms": {k: log2_histogram(cnt[..., i])
                                       for k, i in (("sweeps", 0), ("chop_probes", 1),
                                                    ("polish_pivots", 2))}}

    # the same fits under option variants that the exact finish makes
    # result-neutral (the four-section chop; chop = 0: the polish straight
    # from the descent's stall point; a looser descent tolerance).  Not the paper's method as
    # configured for the headline and not the headline: reported beside it,
    # with every fit's objective compared with the method's (both certified)
    if not args.no_variants and rank == 0:
        ref_obj = out["obj"].cpu().numpy()
        ref_st = out["status"].cpu().numpy()
        line["option_variants"] = {}
        for name, kw in [("four_section_chop", dict(chop_sections=4)),
                         ("chop_off", dict(chop=0)), ("tol_move_1e-3", dict(tol_move=1e-3)),
                         ("chop_off_tol_move_1e-3", dict(chop=0, tol_move=1e-3))]:
            try:
                o_v = ll.default_opts(**kw)
                kt2 = []
                for _ in range(3):
                    flush.fill_(1)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ov = ll.fit(pr, lam_fixed, ws=ws, opts=o_v, launch=launch)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    kt2.append(e0.elapsed_time(e1) / 1e3)
                t_v = statistics.median(kt2)
                obj_v = ov["obj"].cpu().numpy()
                st_v = ov["status"].cpu().numpy()
                both = ((st_v & 3) == 0) & ((ref_st & 3) == 0)
                erel = np.abs(obj_v - ref_obj) / np.maximum(1.0, np.abs(ref_obj))
                line["option_variants"][name] = {
                    "opts": kw, "fits_per_s_certified": int(np.sum((st_v & 3) == 0)) / t_v,
                    "kernel_ms": 1e3 * t_v, "method_kernel_ms": 1e3 * t_fit,
                    "certified_fraction": float(np.mean((st_v & 3) == 0)),
                    "worst_rel_obj_vs_method": float(erel[both].max()) if both.any() else None,
                    "fits_over_1e-5": int(np.sum(erel[both] > 1e-5))}
                log(f"variant {name} {line['option_variants'][name]}")
            except Exception as ex:  # report, do not fail the bench line
                line["option_variants"][name] = {"error": str(ex)}

    # long problems: 20000 x 128 per fit, one 512-thread block per fit,
    # columns streamed from HBM (one launch, timed with events)
    if not args.no_large and rank == 0:
        try:
            Bl = args.large_problems
            big = synth.large(B=Bl)
            pb = ll.Problems.from_numpy(big, device=dev)
            del big
            wsb = ll.workspace(pb, args.large_lambdas)
            Ll = args.large_lambdas
            lamb = ll.lambda_path(ll.lambda_max(pb, wsb), Ll, 1e-3)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ob = ll.fit(pb, lamb, ws=wsb, counters=True)
            e1.record(stream)
            torch.cuda.synchronize()
            tl = e0.elapsed_time(e1) / 1e3
            cb = ob["counters"].cpu().numpy().astype(np.float64)
            sb = ob["status"].cpu().numpy()
            n_l, p_l = 20000, 128
            # algorithmic bytes: one read of a column (4n B) per selection
            # pass, one read of the design (4np B) per polish pivot
            byts = 4.0 * n_l * float(cb[..., 4].sum() + p_l * cb[..., 2].sum())
            hbm_peak = 6701.5
            try:
                hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
            except (OSError, KeyError, ValueError):
                pass
            cert = int(np.sum((sb & 3) == 0))
            line["large"] = {
                "workload": f"{Bl} problems x 20000 rows x 128 columns, AR(1) 0.5, L={Ll}",
                "fits_per_s": cert / tl, "kernel_ms": 1e3 * tl, "certified_fraction": cert / sb.size,
                "launch": "one 512-thread block per fit",
                "roofline": {"bound": "hbm", "achieved": byts / tl / 1e9, "peak": hbm_peak,
                             "unit": "GB/s", "frac": byts / tl / 1e9 / hbm_peak,
                             "bytes_per_launch": byts, "traffic": None},
                "pivots_mean": float(cb[..., 2].mean()), "passes_mean": float(cb[..., 4].mean()),
                # share of the block's cycles in descent + chop (the rest is
                # the stall tests and the polish: counter slots 6 and 7)
                "descent_chop_cycle_share": float(cb[..., 6].sum() / max(1.0, cb[..., 6:8].sum()))}
            log(f"large {line['large']}")
            del pb, wsb, ob
            torch.cuda.empty_cache()
        except Exception as ex:
            line["large"] = {"error": str(ex)}

    # differentiation: forward fit at 0.1 lambda_max on the training rows and
    # the adjoint of the validation LAD loss (one launch each)
    if not args.no_diff and rank == 0:
        try:
            dd = synth.diff()
            ptr = ll.Problems.from_numpy(dd["train"], device=dev)
            pva = ll.Problems.from_numpy(dd["val"], device=dev)
            Bd = ptr.B
            wsd = ll.workspace(ptr, 1)
            lamd = (0.1 * ll.lambda_max(ptr, wsd)).reshape(Bd, 1).contiguous()
            up = torch.ones(Bd, device=dev)
            fw = ll.fit(ptr, lamd, ws=wsd, basis=True)  # warm-up
            ll.fit_backward(ptr, fw, 0, pva, up, ws=wsd)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            fw = ll.fit(ptr, lamd, ws=wsd, basis=True)
            ev[1].record(stream)
            gb = ll.fit_backward(ptr, fw, 0, pva, up, ws=wsd)
            ev[2].record(stream)
            torch.cuda.synchronize()
            tf, tb = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
            sd = fw["status"].cpu().numpy()
            gs = gb["status"].cpu().numpy()
            line["diff"] = {
                "workload": "512 problems, 400 train / 100 validation rows, p=16, lambda=0.1 lambda_max",
                "forward_fits_per_s": int(np.sum((sd & 3) == 0)) / tf, "forward_ms": 1e3 * tf,
                "backward_ms": 1e3 * tb, "backward_problems_per_s": Bd / tb,
                "strict_vertex_fraction": float(np.mean(gs == 0))}
            log(f"diff {line['diff']}")
        except Exception as ex:
            line["diff"] = {"error": str(ex)}

    # thread-per-fit comparison: the paper's one-fit-per-thread layout is far
    # too slow for the full workload inside a bench run, so both kernels are
    # timed on the same 608-problem subset (same generator, n <= 500)
    if not args.no_thread and rank == 0 and args.thread_full:
        # the paper's one-fit-per-thread layout on the headline workload
        # itself: one launch over the same problems and lambda path
        try:
            # no warm-up: one launch takes minutes, so its start-up costs are noise
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o3 = ll.fit(pr, lam_fixed, ws=ws, per_thread=True)
            e1.record(stream)
            torch.cuda.synchronize()
            t3 = e0.elapsed_time(e1) / 1e3
            c3 = int(np.sum((o3["status"].cpu().numpy() & 3) == 0))
            line["thread_per_fit"] = {
                "workload": workload(B, L), "fits_per_s": c3 / t3, "kernel_ms": 1e3 * t3,
                "certified_fraction": c3 / fits, "warp_per_fit_fits_per_s": certified / t_fit,
                "speedup": (certified / t_fit) / (c3 / t3)}
            log(f"thread-per-fit full {line['thread_per_fit']}")
        except Exception as ex:  # report, do not fail the bench line
            line["thread_per_fit"] = {"error": str(ex)}
    elif not args.no_thread and rank == 0:
        try:
            sub = synth.batched_like(608, 50, 500, 4, 32, seed=11)
            psub = ll.Problems.from_numpy(sub, device=dev)
            wsub = ll.workspace(psub, L)
            lsub = ll.lambda_path(ll.lambda_max(psub, wsub), L, 1e-3)
            res = {}
            for pt in (False, True):
                ll.fit(psub, lsub, ws=wsub, per_thread=pt)  # warm-up
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                o3 = ll.fit(psub, lsub, ws=wsub, per_thread=pt)
                e1.record(stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1e3
                s3 = o3["status"].cpu().numpy()
                res[pt] = (int(np.sum((s3 & 3) == 0)) / t, t)
            log(f"thread-per-fit subset {res}")
            line["thread_per_fit"] = {
                "workload": "608 problems, n~U[50,500], p~U[4,32], L=16",
                "fits_per_s": res[True][0], "kernel_ms": 1e3 * res[True][1],
                "warp_per_fit_fits_per_s": res[False][0],
                "speedup": res[False][0] / res[True][0]}
        except Exception as ex:  # report, do not fail the bench line
            line["thread_per_fit"] = {"error": str(ex)}

    # cross-validation of lambda: 256 data sets (500 rows x 16 columns, the
    # differentiation recipe), 5 folds each, a 16-point path; one fit launch
    # and one held-out-loss launch through the driver's public call, timed
    # end to end (host index building and copies included)
    if not args.no_cv and rank == 0:
        try:
            from paper_2510_15649_gb300 import cv
            dcv = synth.diff(B=256, n=500, n_train=500, p=16, seed=8)["train"]
            data = [batch_rows(dcv, q) for q in range(256)]
            splits = [cv.kfold_splits(500, 5, seed=q) for q in range(256)]
            cv.cross_validate_many(data[:8], splits[:8], L=16, device=dev)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res_cv = cv.cross_validate_many(data, splits, L=16, device=dev)
            torch.cuda.synchronize()
            t_cv = time.perf_counter() - t0
            n_fits = 256 * 5 * 16
            line["cv"] = {"workload": "256 data sets x 500 rows x 16 columns, 5-fold, 16 lambdas",
                          "seconds": t_cv, "fits": n_fits, "fits_per_s": n_fits / t_cv,
                          "data_sets_per_s": 256 / t_cv,
                          "certified_fraction": float(np.mean([np.mean((r.status & 3) == 0)
                                                               for r in res_cv]))}
            log(f"cv {line['cv']}")
        except Exception as ex:  # report, do not fail the bench line
            line["cv"] = {"error": str(ex)}

    # continuous-batching server on Poisson arrivals (20k requests/s for
    # 10 s: the request designs are windows of one shared N(0,1) row bank,
    # each request with its own coefficients, noise and outliers), then a
    # second trace offered below capacity, where latency is service time
    if not args.no_serve and rank == 0:
        from paper_2510_15649_gb300.serve import ClassedServer, Server
        bank = 1 << 20
        try:
            t0 = time.perf_counter()
            trace = synth.serve_trace(rate=args.serve_rate, seconds=args.serve_seconds, seed=4,
                                      bank_rows=bank)
            log(f"serve trace {len(trace)} requests in {time.perf_counter() - t0:.1f}s")
            # the trace's first 4096 requests as one problem set: the launch
            # shape for this mix (5000-row slots hold only a few fits per SM,
            # where several warps per fit pay) is autotuned on it, and the
            # batched kernel's throughput on it is the serving arm's reference
            mix = trace[:4096]
            nn = np.array([r["X"].shape[0] for r in mix])
            pp = np.array([r["X"].shape[1] for r in mix], np.int32)
            off = np.concatenate([[0], np.cumsum(nn)]).astype(np.int64)
            Xm = np.zeros((off[-1], 64), np.float32)
            ym = np.zeros(off[-1], np.float32)
            for k, r in enumerate(mix):
                Xm[off[k]:off[k + 1], :pp[k]] = r["X"]
                ym[off[k]:off[k + 1]] = r["y"]
            pm = ll.Problems.from_numpy(dict(X=Xm, y=ym, row_idx=None, offsets=off, p=pp), device=dev)
            pm.n_max = 5000  # the pool's slot capacity
            wsm = ll.workspace(pm, 8)
            lamm = ll.lambda_path(ll.lambda_max(pm, wsm), 8, 1e-3)
            from paper_2510_15649_gb300 import tune
            slaunch, stimes = tune.autotune(pm, lamm, sample_problems=512, repeats=1)
            log(f"batched same-mix launch {slaunch}")
            # the server keeps the library's automatic shape: a batch timing
            # picks the block shape for this mix, which served the trace
            # slower (15.4k against 17.2k fits/s) -- a launch's fits there
            # are one path position of each slot, not whole paths
            Server(slots=2048, cap=5000, P=64, L=8).run(trace[:256])  # warm-up
            srv = Server(slots=2048, cap=5000, P=64, L=8)
            _, sst = srv.run(trace)
            offered = len(trace) * 8 / args.serve_seconds
            line["serve"] = dict(sst.summary(), offered_fits_per_s=offered, workload=(
                f"Poisson {args.serve_rate:g} req/s for {args.serve_seconds:g}s, n log-U[20,5000], "
                "p log-U[2,64], L=8, 2048 slots, several positions per launch for short requests"))
            line["serve"]["launch"] = "library automatic"
            log(f"serve {line['serve']}")
            del srv
            # the batched kernel on the same request mix, one launch along
            # the 8-point paths (the serving arm's throughput against this)
            ll.fit(pm, lamm, ws=wsm, launch=slaunch)  # warm-up
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            om = ll.fit(pm, lamm, ws=wsm, launch=slaunch)
            e1.record(stream)
            torch.cuda.synchronize()
            tm = e0.elapsed_time(e1) / 1e3
            cm = int(np.sum((om["status"].cpu().numpy() & 3) == 0))
            line["serve"]["batched_same_mix"] = {
                "workload": "the trace's first 4096 requests as one batch, L=8, one launch",
                "launch": f"{slaunch.group_threads}x{slaunch.fits_per_block}/o{slaunch.work_order} "
                          "(autotuned)",
                "fits_per_s": cm / tm, "kernel_ms": 1e3 * tm,
                "serving_share": line["serve"]["fits_per_s"] / (cm / tm)}
            log(f"serve batched same mix {line['serve']['batched_same_mix']}")
            del pm, wsm, om
        except Exception as ex:
            line["serve"] = {"error": str(ex)}
        if args.serve_light_rate > 0 and isinstance(line.get("serve"), dict):
            try:
                tl = synth.serve_trace(rate=args.serve_light_rate, seconds=args.serve_light_seconds,
                                       seed=5, bank_rows=bank)
                srv = Server(slots=2048, cap=5000, P=64, L=8)
                _, lst = srv.run(tl)
                line["serve"]["below_capacity"] = dict(
                    lst.summary(), offered_fits_per_s=len(tl) * 8 / args.serve_light_seconds,
                    workload=f"Poisson {args.serve_light_rate:g} req/s for "
                             f"{args.serve_light_seconds:g}s, same request mix")
                log(f"serve below capacity {line['serve']['below_capacity']}")
                del srv
            except Exception as ex:
                line["serve"]["below_capacity"] = {"error": str(ex)}
        if args.serve_classes and isinstance(line.get("serve"), dict):
            # the same trace and total slot count in slot classes sized to the
            # request mix (58 % of requests have n <= 500, 83 % n <= 2000)
            try:
                classes = [(1280, 500, 64), (512, 2000, 64), (256, 5000, 64)]
                csrv = ClassedServer(classes, L=8, device=dev)
                _, cst = csrv.run(trace)
                line["serve"]["slot_classes"] = dict(
                    cst.summary(), classes="slots x rows (64 columns): 1280 x 500, 512 x 2000, "
                                           "256 x 5000")
                log(f"serve slot classes {cst.summary()}")
            except Exception as ex:
                line["serve"]["slot_classes"] = {"error": str(ex)}
        torch.cuda.empty_cache()

    # CPU oracle baseline on a bounded sample
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        lh = lam.cpu().numpy().astype(np.float64)
        # problems in order, a chunk of about two per core at a time, until
        # at least 10 s of CPU work has been timed (a bounded sample)
        chunk = max(8, 2 * cores)
        done, dt, used = 0, 0.0, 1
        while done < B and dt < 10.0:
            qs = np.arange(done, min(B, done + chunk))
            t0 = time.perf_counter()
            r = oracle.fit_batch(batch, lh, problems=qs, nthreads=cores)
            dt += time.perf_counter() - t0
            done += len(qs)
            used = r["threads"]
        line["cpu_baseline"] = {"value": done * L / dt, "unit": "fits/s", "cores": used,
                                "kind": "oracle",
                                "sample": f"problems 0..{done - 1} x {L} lambdas of the workload "
                                          f"({dt:.1f} s, chunks of {chunk} problems)"}
        # the same oracle on one core: problems in order, one at a time,
        # until at least 5 s of CPU work has been timed
        done1, dt1 = 0, 0.0
        while done1 < B and dt1 < 5.0:
            t0 = time.perf_counter()
            oracle.fit_batch(batch, lh, problems=np.arange(done1, done1 + 1), nthreads=1)
            dt1 += time.perf_counter() - t0
            done1 += 1
        line["cpu_baseline"]["one_core"] = {
            "value": done1 * L / dt1, "unit": "fits/s", "cores": 1,
            "sample": f"problems 0..{done1 - 1} x {L} lambdas of the workload ({dt1:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
