"""Continuous-batching server for LAD-LASSO fits on one GPU.

Requests (one fit each: X [n, p], y [n]) arrive over time.  The server keeps
a device pool of S fixed-capacity slots (cap rows x P columns each) and runs
the request loop on the host:

  admit     arrivals whose time has come take a free slot while the device
            memory they need (n * p floats) fits the pool's budget; the rows
            (X and y) of every request admitted at once are packed into one
            staging buffer, copied to the device in one transfer and
            scattered into their slots; their lambda_max and lambda path
            computed on the device, b zeroed
  step      one launch of ladlasso_fit_batched over all S slots: every
            active request advances along its lambda path, warm-started from
            its previous b -- one position, or several when it is small
            against the launch's largest request (`positions`), so that
            short requests finish in few launches; positions not taken and
            idle slots are passed with lambda = NaN (idle slots with 0 rows)
  retire    requests whose path is done copy b and F to the host and free
            their slot; latency = arrival -> result on the host

Requests that arrive while others are on the GPU join at the next step, so
work from different requests overlaps inside every launch.  `ClassedServer`
runs the same loop over several pools of different slot sizes (slot
classes): a request takes a slot of the smallest class that holds it, so
short requests do not reserve a long request's shared memory.  A request's
results equal those of fitting it alone along the same path (same kernel,
same per-fit arithmetic).  All arithmetic runs in the CUDA library; this
module only moves data and keeps the schedule.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ladlasso as ll


def admission_offsets(slots: np.ndarray, cap: int, S: int) -> np.ndarray:
    """Offsets of the problem set made of the given (sorted) slots of a pool
    of S slots of cap rows: slot k starts at k * cap and the set ends at the
    pool's row count S * cap, as the library requires of a problem set's
    last offset."""
    ss = np.asarray(slots, np.int64)
    return np.append(ss * cap, np.int64(S) * cap)


@dataclass
class Result:
    """One served request: its fitted path and when it arrived and finished."""
    rid: int
    b: np.ndarray          # [L, p]
    obj: np.ndarray        # [L]
    status: np.ndarray     # [L]
    lambdas: np.ndarray    # [L]
    t_arrival: float
    t_done: float


@dataclass
class ServeStats:
    """Counts and latencies of one Server.run."""
    completed: int = 0
    fits: int = 0          # fits with valid input (status without BAD_INPUT)
    bad_fits: int = 0
    steps: int = 0
    wall: float = 0.0
    latencies: list = field(default_factory=list)
    max_active: int = 0
    queued_max: int = 0

    def summary(self) -> dict:
        """Requests, fits, fits/s and p50/p99 latency (ms) as a dict."""
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return dict(requests=self.completed, fits=self.fits, bad_fits=self.bad_fits, steps=self.steps,
                    seconds=self.wall, fits_per_s=self.fits / max(self.wall, 1e-9),
                    p50_ms=1e3 * float(np.percentile(lat, 50)),
                    p99_ms=1e3 * float(np.percentile(lat, 99)),
                    max_active=self.max_active, max_queued=self.queued_max)


class Server:
    """Slot pool + request loop.  `budget_floats` bounds the total n * p of
    the active requests (device-memory admission)."""

    def __init__(self, slots: int = 1024, cap: int = 5000, P: int = 64, L: int = 8,
                 ratio: float = 1e-3, budget_floats: int | None = None, device="cuda",
                 opts: ll.Opts | None = None, positions_per_step: int | None = None,
                 launch: ll.Launch | None = None):
        self.S, self.cap, self.P, self.L, self.ratio = slots, cap, P, L, ratio
        self.launch = launch  # launch shape of the fit (None: the library's choice)
        # most path positions one slot advances in one launch (1: every
        # slot one position per step)
        self.K = L if positions_per_step is None else max(1, min(L, positions_per_step))
        self.dev = torch.device(device)
        self.opts = opts
        self.budget = budget_floats if budget_floats is not None else slots * cap * P
        S, dev = slots, self.dev
        self.X = torch.zeros((S * cap, P), dtype=torch.float32, device=dev)
        self.y = torch.zeros(S * cap, dtype=torch.float32, device=dev)
        self.offsets = torch.arange(S + 1, dtype=torch.int64, device=dev) * cap
        self.n_rows = torch.zeros(S, dtype=torch.int32, device=dev)
        self.p = torch.ones(S, dtype=torch.int32, device=dev)
        K = self.K
        self.b_state = torch.zeros((S, P), dtype=torch.float32, device=dev)  # warm start
        self.b = torch.zeros((S, K, P), dtype=torch.float32, device=dev)
        self.obj = torch.zeros((S, K), dtype=torch.float32, device=dev)
        self.status = torch.zeros((S, K), dtype=torch.int32, device=dev)
        self.lam_step = torch.full((S, K), float("nan"), dtype=torch.float32, device=dev)
        self.pr = ll.Problems(X=self.X, y=self.y, offsets=self.offsets, p=self.p, P=P,
                              n_max=cap, n_rows=self.n_rows)
        self.ws = ll.workspace(self.pr, K)
        # host mirrors
        self.h_n = np.zeros(S, np.int32)
        self.h_p = np.ones(S, np.int32)
        self.h_pos = np.zeros(S, np.int32)
        self.h_rid = np.full(S, -1, np.int64)
        self.h_lam = np.zeros((S, L), np.float32)
        self.h_b = np.zeros((S, L, P), np.float32)
        self.h_obj = np.zeros((S, L), np.float32)
        self.h_st = np.zeros((S, L), np.int32)
        self.h_k = np.zeros(S, np.int32)          # positions taken by the last launch
        self.h_bstate = np.zeros((S, P), np.float32)
        self.used = 0
        self.free = list(range(S - 1, -1, -1))
        self._stage = None     # host staging of admitted rows (see _staging)
        self._stage_t = None
        # each pool works on a stream of its own, so the steps of several
        # pools (slot classes) can overlap on the device
        self.stream = torch.cuda.Stream(self.dev) if self.dev.type == "cuda" else None

    def _on_stream(self):
        import contextlib
        return torch.cuda.stream(self.stream) if self.stream is not None else contextlib.nullcontext()

    # ---------------------------------------------------------------- admit
    def _staging(self, rows: int) -> np.ndarray:
        """Host staging rows (P columns of X, then y), pinned on a CUDA
        device so the copy is asynchronous; grown geometrically, reused."""
        if self._stage is None or self._stage.shape[0] < rows:
            cap = max(rows, 2 * (0 if self._stage is None else self._stage.shape[0]), 1024)
            t = torch.empty((cap, self.P + 1), dtype=torch.float32,
                            pin_memory=self.dev.type == "cuda")
            self._stage_t, self._stage = t, t.numpy()
        return self._stage

    def _admit(self, reqs, rids):
        with self._on_stream():
            return self._admit_on_stream(reqs, rids)

    def _admit_on_stream(self, reqs, rids):
        slots, ns = [], []
        for r, rid in zip(reqs, rids):
            s = self.free.pop()
            n, p = r["X"].shape
            self.h_n[s], self.h_p[s], self.h_pos[s], self.h_rid[s] = n, p, 0, rid
            self.used += n * p
            slots.append(s)
            ns.append(n)
        # every admitted request's rows packed into one staging buffer, one
        # host-to-device copy, then scattered into the slots on the device
        tot = int(sum(ns))
        if tot:
            st = self._staging(tot)
            o = 0
            for r, n in zip(reqs, ns):
                p = r["X"].shape[1]
                st[o:o + n, :p] = r["X"]
                st[o:o + n, p:self.P] = 0.0
                st[o:o + n, self.P] = r["y"]
                o += n
            dest = np.concatenate([np.arange(s * self.cap, s * self.cap + n, dtype=np.int64)
                                   for s, n in zip(slots, ns)])
            rows = self._stage_t[:tot].to(self.dev, non_blocking=True)
            dest_t = torch.from_numpy(dest).to(self.dev, non_blocking=True)
            self.X.index_copy_(0, dest_t, rows[:, :self.P])
            self.y.index_copy_(0, dest_t, rows[:, self.P].contiguous())
        self.n_rows.copy_(torch.from_numpy(self.h_n), non_blocking=True)
        self.p.copy_(torch.from_numpy(self.h_p), non_blocking=True)
        # lambda_max and the path of the new requests, on the device: the new
        # slots as one problem set; a problem set's last offset must be the
        # pool's row count, so the last new slot's range runs to the end of
        # the pool (its n_rows still bounds the rows it uses)
        ss = np.array(sorted(slots), np.int64)
        offs = torch.from_numpy(admission_offsets(ss, self.cap, self.S)).to(self.dev)
        sub = ll.Problems(X=self.X, y=self.y, offsets=offs,
                          p=torch.from_numpy(self.h_p[ss]).to(self.dev), P=self.P,
                          n_max=self.cap,
                          n_rows=torch.from_numpy(self.h_n[ss]).to(self.dev))
        lmax = ll.lambda_max(sub, self.ws)
        lam = ll.lambda_path(lmax, self.L, self.ratio)
        self.h_lam[ss] = lam.cpu().numpy()
        self.h_bstate[ss] = 0.0  # a new request starts from b = 0
        return slots

    # ---------------------------------------------------------------- step
    def _active(self) -> np.ndarray:
        return np.nonzero(self.h_rid >= 0)[0]

    def positions(self, active: np.ndarray) -> np.ndarray:
        """Path positions each active slot advances in the next launch: a
        launch lasts about as long as one position of its largest request
        (work n * p), so a slot whose request is w times smaller takes up
        to w positions (at least 1, at most K and what is left of its
        path) and a short request finishes in one or two launches instead
        of idling through L of them."""
        w = self.h_n[active].astype(np.float64) * self.h_p[active]
        k = np.floor(w.max() / np.maximum(w, 1.0)).astype(np.int64)
        return np.clip(k, 1, np.minimum(self.K, self.L - self.h_pos[active])).astype(np.int32)

    def _launch(self) -> bool:
        """One fit launch advancing every active slot by its share of path
        positions (positions), warm-started from its last b; positions a
        slot does not take this step are passed as NaN, which the library
        skips.  False when no slot is active."""
        active = self._active()
        if len(active) == 0:
            return False
        k = self.positions(active)
        self.h_k[:] = 0
        self.h_k[active] = k
        lam = np.full((self.S, self.K), np.nan, np.float32)
        for s, ks in zip(active, k):
            lam[s, :ks] = self.h_lam[s, self.h_pos[s]:self.h_pos[s] + ks]
        with self._on_stream():
            self.lam_step.copy_(torch.from_numpy(lam), non_blocking=True)
            self.b_state.copy_(torch.from_numpy(self.h_bstate), non_blocking=True)
            ll.fit(self.pr, self.lam_step, b_init=self.b_state, ws=self.ws, opts=self.opts,
                   out=dict(b=self.b, obj=self.obj, status=self.status), launch=self.launch)
        return True

    def _collect(self, st: ServeStats, arrive: dict, results: list) -> None:
        """After a launch: copy the step's results, advance the active slots,
        retire the requests whose path is done."""
        active = self._active()
        if self.stream is not None:
            self.stream.synchronize()
        bh = self.b.cpu().numpy()
        oh = self.obj.cpu().numpy()
        sh = self.status.cpu().numpy()
        for s in active:
            ks, pos = int(self.h_k[s]), int(self.h_pos[s])
            self.h_b[s, pos:pos + ks] = bh[s, :ks]
            self.h_obj[s, pos:pos + ks] = oh[s, :ks]
            self.h_st[s, pos:pos + ks] = sh[s, :ks]
            self.h_bstate[s] = bh[s, ks - 1]  # the next launch starts here
            valid = (sh[s, :ks] & 2) == 0
            st.fits += int(valid.sum())
            st.bad_fits += int((~valid).sum())
        self.h_pos[active] += self.h_k[active]
        done = active[self.h_pos[active] >= self.L]
        tnow = time.perf_counter()
        for s in done:
            rid = int(self.h_rid[s])
            p = int(self.h_p[s])
            results.append(Result(rid=rid, b=self.h_b[s, :, :p].copy(),
                                  obj=self.h_obj[s].copy(), status=self.h_st[s].copy(),
                                  lambdas=self.h_lam[s].copy(), t_arrival=arrive[rid],
                                  t_done=tnow))
            st.latencies.append(tnow - arrive[rid])
            self.used -= int(self.h_n[s]) * p
            self.h_rid[s] = -1
            self.h_n[s] = 0
            self.free.append(int(s))
            st.completed += 1
        if len(done):
            self.n_rows.copy_(torch.from_numpy(self.h_n), non_blocking=True)

    # ---------------------------------------------------------------- run
    def run(self, trace: list, time_scale: float = 1.0) -> tuple:
        """Serve `trace` (list of dicts with t, X, y), arrivals replayed in
        real time scaled by time_scale.  Returns (results, ServeStats)."""
        return serve_pools([self], trace, time_scale, self.budget)


def serve_pools(pools: list, trace: list, time_scale: float, budget: int) -> tuple:
    """The request loop over one or more slot pools (ordered from the
    smallest slot capacity up).  Arrivals queue in order; the queue's head
    takes a free slot of the first pool whose slots hold it (cap rows, P
    columns) while the active requests' n * p stays within `budget`.  Each
    step launches every pool with active slots, then collects their
    results.  Returns (results, ServeStats)."""
    st = ServeStats()
    results = []
    t0 = time.perf_counter()
    arrive = {i: t0 + trace[i]["t"] * time_scale for i in range(len(trace))}
    queue = []
    nxt = 0
    while nxt < len(trace) or queue or any(len(pl._active()) for pl in pools):
        now = time.perf_counter()
        while nxt < len(trace) and arrive[nxt] <= now:
            queue.append(nxt)
            nxt += 1
        st.queued_max = max(st.queued_max, len(queue))
        plan = [([], []) for _ in pools]
        free_left = [len(pl.free) for pl in pools]
        used = sum(pl.used for pl in pools)
        extra = 0
        while queue:
            i = queue[0]
            n, p = trace[i]["X"].shape
            holders = [k for k, pl in enumerate(pools) if n <= pl.cap and p <= pl.P]
            if not holders:
                raise ValueError(f"request {i} ({n}x{p}) exceeds the slot capacity")
            if n * p > budget:
                raise ValueError(f"request {i} ({n}x{p}) exceeds the memory budget "
                                 f"of {budget} floats on its own")
            k = next((k for k in holders if free_left[k] > 0), None)
            if k is None:
                break  # every pool that holds it is full: wait for a slot
            if used + extra + n * p > budget:
                break  # device-memory admission: wait for requests to retire
            queue.pop(0)
            plan[k][0].append(trace[i])
            plan[k][1].append(i)
            free_left[k] -= 1
            extra += n * p
        for pl, (reqs, rids) in zip(pools, plan):
            if reqs:
                with ll._nvtx("serve_admit"):
                    pl._admit(reqs, rids)
        n_active = sum(len(pl._active()) for pl in pools)
        if n_active == 0:
            if queue:
                # nothing runs, so every slot and the whole budget are free and
                # the head request (which fits a class and the budget) would
                # have been admitted: the bookkeeping is broken, and waiting
                # would never end
                raise RuntimeError("serving stalled: requests wait, nothing runs and "
                                   "none can be admitted")
            if nxt < len(trace):  # idle until the next arrival
                time.sleep(max(0.0, min(arrive[nxt] - time.perf_counter(), 1e-3)))
            continue
        st.max_active = max(st.max_active, n_active)
        with ll._nvtx("serve_step"):
            launched = [pl for pl in pools if pl._launch()]
            st.steps += 1
            for pl in launched:
                pl._collect(st, arrive, results)
    st.wall = time.perf_counter() - t0
    return results, st


class ClassedServer:
    """Slot classes: one pool per (slots, cap, P) class, ordered by slot
    size.  A request takes a slot of the smallest class that holds it (a
    larger class when that one is full), so short requests do not reserve a
    long request's shared memory and more fits run at once; every step
    launches each class with active slots.  `budget_floats` bounds the total
    n * p of the active requests over all classes."""

    def __init__(self, classes: list, L: int = 8, ratio: float = 1e-3,
                 budget_floats: int | None = None, device="cuda", opts: ll.Opts | None = None):
        cl = sorted(classes, key=lambda c: (c[1] * c[2], c[1], c[2]))
        if not cl:
            raise ValueError("no slot classes")
        self.pools = [Server(slots=sl, cap=cap, P=P, L=L, ratio=ratio, device=device, opts=opts)
                      for sl, cap, P in cl]
        self.budget = budget_floats if budget_floats is not None else \
            sum(sl * cap * P for sl, cap, P in cl)

    def run(self, trace: list, time_scale: float = 1.0) -> tuple:
        """As Server.run, over every class."""
        return serve_pools(self.pools, trace, time_scale, self.budget)


def serve_distributed(server, trace: list, rank: int, world: int, dist=None,
                      time_scale: float = 1.0, device=None) -> tuple:
    """Serve one arrival trace on `world` GPUs, one process each: every
    rank computes the same routing (dist.route_requests by n * p), serves
    its own requests in its own pool (`server`: a Server or ClassedServer
    on this rank's GPU) with their arrival times kept, and the report is
    merged over ranks -- fits and requests summed, the wall time the
    slowest rank's, latencies pooled for p50/p99 (`device`: where the
    process group's reductions run, the rank's GPU under NCCL).  Returns
    (this rank's results with their request ids in the whole trace, merged
    ServeStats)."""
    from .dist import gather_lists, max_over_ranks, route_requests, sum_over_ranks
    sizes = [r["X"].shape[0] * r["X"].shape[1] for r in trace]
    route = route_requests(sizes, world)
    mine = [i for i in range(len(trace)) if route[i] == rank]
    results, st = server.run([trace[i] for i in mine], time_scale)
    for r in results:
        r.rid = mine[r.rid]
    dv = device
    merged = ServeStats(
        completed=int(sum_over_ranks(st.completed, dist, dv)),
        fits=int(sum_over_ranks(st.fits, dist, dv)),
        bad_fits=int(sum_over_ranks(st.bad_fits, dist, dv)),
        steps=int(max_over_ranks(st.steps, dist, dv)), wall=max_over_ranks(st.wall, dist, dv),
        latencies=gather_lists(st.latencies, dist),
        max_active=int(sum_over_ranks(st.max_active, dist, dv)),
        queued_max=int(max_over_ranks(st.queued_max, dist, dv)))
    return results, merged
