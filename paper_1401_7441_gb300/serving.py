"""Serving form: a continuous-batching request loop for H phi + sparse H/S.

Requests (systems of 50-5,000 atoms shaped like the 64-atom workload, radii 5-8 bohr)
arrive on a Poisson stream.  About 30 % reuse a resident system: a *perturbed* geometry
(atoms displaced, support functions moved onto the new locregs by lsw_reformat, the
paper's reuse across geometry steps) or a *charged* variant (the same geometry and
support functions under a shifted potential, the paper's reuse from neutral to charged
systems).  The loop

* prepares each arrived request on host threads (geometry, keys and plans are built in
  the library on a setup stream),
* admits prepared requests while their device memory fits an HBM budget, evicting idle
  resident systems least recently used first,
* enqueues each admitted request on its own CUDA stream (H phi, then H/S, then the
  copy of H and S to pinned host memory), so the work of requests in flight overlaps
  on the device,
* polls events, records each response's latency and keeps the finished system and its
  support functions resident for later reuse.

All device work is the library's (lsw_*); this module schedules it.
"""
from __future__ import annotations

import copy
import math
import queue
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field

import numpy as np

from . import build as _build
from . import inputs as I
from . import lsw

DENSITY = 64 / 30.0 ** 3          # atoms per bohr^3 of the 64-atom workload
RADII = (5.0, 6.0, 7.0, 8.0)
SLAB_MB = 2048                    # H/S panel budget of a served system (library option "slab_mb")
CACHE_SLACK = 40e9                # bytes PyTorch may keep cached but unused between requests


@dataclass
class Request:
    rid: int
    t_arrival: float               # seconds after the start of the stream
    kind: str                      # "new" | "perturb" | "charged"
    n_atoms: int
    seed: int
    parent: int | None = None      # rid of the request whose system is reused


@dataclass
class Result:
    rid: int
    kind: str
    n_sf: int
    t_arrival: float
    t_admit: float
    t_done: float
    H: np.ndarray
    S: np.ndarray
    e_kin: np.ndarray
    e_pot: np.ndarray

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def request_stream(n_requests, rate=20.0, atoms=(50, 5000), reuse_frac=0.3, seed=5005):
    """Poisson arrivals (mean ``rate``/s), log-uniform atom counts, ``reuse_frac`` of the
    requests reusing an earlier new request (half perturbed, half charged)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out, news = [], []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate)
        if news and rng.random() < reuse_frac:
            parent = int(news[rng.integers(len(news))])
            kind = "perturb" if rng.random() < 0.5 else "charged"
            n = out[parent].n_atoms
        else:
            parent, kind = None, "new"
            n = int(round(math.exp(rng.uniform(math.log(atoms[0]), math.log(atoms[1])))))
            news.append(rid)
        out.append(Request(rid, t, kind, n, int(rng.integers(1 << 30)), parent))
    return out


def new_workload(n_atoms, seed) -> I.Workload:
    cube = (n_atoms / DENSITY) ** (1.0 / 3.0)
    return I.atoms_cube("serve_%d" % n_atoms, seed, n_atoms, cube, list(RADII), lambda r: 2.0,
                        0.25, 0.0, pair_mode=lsw.LSW_PAIR_SUM_OF_RADII, precision="fp32")


def perturbed(wl: I.Workload, seed, sigma=0.05) -> I.Workload:
    """Atoms displaced by N(0, sigma) bohr; wells move with their atoms."""
    w2 = copy.deepcopy(wl)
    rng = np.random.default_rng(seed)
    d = rng.normal(0.0, sigma, size=wl.pos.shape)
    lim = wl.h * (wl.N[0] - 1)
    w2.pos = np.clip(wl.pos + d, 0.0, lim)
    w2.wells = wl.wells.copy()
    w2.wells[:, :3] = w2.pos
    return w2


def charged(wl: I.Workload, seed) -> I.Workload:
    """The same system under V shifted by one smooth seeded Gaussian (w = 5 bohr)."""
    w2 = copy.deepcopy(wl)
    u = I.uniform(seed, 11, 1)[0]
    centre = 0.5 * wl.h * (np.asarray(wl.N) - 1)
    extra = np.array([[centre[0], centre[1], centre[2], -0.5 + u, 5.0]])   # depth D in [-0.5, 0.5]
    w2.wells = np.vstack([wl.wells, extra])
    return w2


@dataclass
class _Entry:
    """A system on the device (resident between requests)."""
    rid: int
    wl: I.Workload
    system: lsw.System
    phi: object                     # torch tensor, layout off_L
    busy: bool = False
    bytes: int = 0


@dataclass
class _Job:
    req: Request
    wl: I.Workload
    system: lsw.System | None = None
    parent: _Entry | None = None
    est_bytes: int = 0
    t_ready: float = 0.0
    stream: object = None
    event: object = None
    t_admit: float = 0.0
    bufs: dict = field(default_factory=dict)
    entry: _Entry | None = None


def _keys_to_g(keys):
    if len(keys) == 0:
        return np.zeros(0, np.int64)
    lens = keys[:, 1] - keys[:, 0] + 1
    starts = np.repeat(keys[:, 0] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    return starts + np.arange(int(lens.sum()), dtype=np.int64)


class Server:
    """Continuous-batching loop on one GPU (see the module docstring)."""

    def __init__(self, device=0, budget_bytes=150e9, precision=lsw.LSW_FP32, streams=4, host_threads=4,
                 graphs=True):
        import torch
        _build.build()
        self.torch = torch
        self.device = device
        self.budget = float(budget_bytes)
        self.precision = precision
        self.dt = torch.float64 if precision == lsw.LSW_FP64 else torch.float32
        self.es = 8 if precision == lsw.LSW_FP64 else 4
        torch.cuda.set_device(device)
        self.setup_stream = torch.cuda.Stream(device)
        self.ctx = lsw.lsw_ctx_create(device, self.setup_stream.cuda_stream)
        self.streams = [torch.cuda.Stream(device) for _ in range(streams)]
        self.host_threads = host_threads
        self.graphs = graphs
        self.resident: "OrderedDict[int, _Entry]" = OrderedDict()
        self.used = 0
        self._ready, self._inflight = [], []

    def _retry_oom(self, fn):
        """fn(), and once more after PyTorch's cached blocks went back to the driver if the
        library ran out of device memory (a library call that fails for memory fails before
        it enqueues anything; the cache holds the tensors of finished requests, which the
        library's own allocations cannot use)."""
        try:
            return fn()
        except lsw.LswError as e:
            if "out of memory" not in str(e):
                raise
            self.torch.cuda.empty_cache()
            try:
                return fn()
            except lsw.LswError as e2:
                free, total = self.torch.cuda.mem_get_info()

                def held(jobs):
                    systems = {id(j.system): j.system for j in jobs if getattr(j, "system", None) is not None}
                    return len(systems), sum(lsw.lsw_workspace_bytes(x.sys) for x in systems.values()) / 1e9

                rs = {id(e.system): e.system for e in self.resident.values()}
                raise lsw.LswError(e2.status, "%s (device free %.1f of %.1f GB; PyTorch reserved %.1f GB, allocated "
                                   "%.1f GB; budget used %.1f of %.1f GB; systems prepared %d (%.1f GB), in flight %d "
                                   "(%.1f GB), resident %d (%.1f GB))"
                                   % (e2, free / 1e9, total / 1e9, self.torch.cuda.memory_reserved() / 1e9,
                                      self.torch.cuda.memory_allocated() / 1e9, self.used / 1e9, self.budget / 1e9,
                                      *held(list(self._ready)), *held(list(self._inflight)), len(rs),
                                      sum(lsw.lsw_workspace_bytes(x.sys) for x in rs.values()) / 1e9)) from e2

    # ---------------------------------------------------------------- host preparation
    def _prepare(self, job: _Job):
        wl = job.wl
        if job.req.kind == "charged" and job.parent is not None:
            job.system = job.parent.system            # same geometry: reuse the system
        else:
            job.system = self._retry_oom(lambda: lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf,
                                                            wl.pair_cutoff, wl.pair_mode, wl.lprime_margin, 0,
                                                            self.precision, ctx=self.ctx))
            # H/S panels of at most SLAB_MB per system (allocated when the system first runs,
            # counted by lsw_workspace_bytes before that)
            lsw.lsw_set_option(job.system.sys, "slab_mb", SLAB_MB)
            if not self.graphs:
                lsw.lsw_set_option(job.system.sys, "graph", 0)
        S = job.system
        V_elems = int(np.prod(wl.V_shape))
        own = 0 if job.system is (job.parent.system if job.parent else None) else lsw.lsw_workspace_bytes(S.sys)
        job.est_bytes = own + self.es * (S.total_Lp + V_elems + (0 if job.req.kind == "charged" else S.total_L)) \
            + 16 * len(S.col) + 16 * S.n_sf
        job.t_ready = time.perf_counter()

    # ---------------------------------------------------------------- device work
    def _launch(self, job: _Job, stream):
        torch = self.torch
        S, wl = job.system, job.wl
        job.stream = stream
        lsw.lsw_system_set_stream(S.sys, stream.cuda_stream)
        with torch.cuda.stream(stream):
            if job.req.kind == "charged" and job.parent is not None:
                phi = job.parent.phi
            else:
                phi = torch.zeros(S.total_L, dtype=self.dt, device="cuda")
                if job.req.kind == "perturb" and job.parent is not None:
                    P = job.parent
                    shift = (np.rint(wl.pos / wl.h) - np.rint(P.wl.pos / P.wl.h)).astype(np.int32)
                    lsw.lsw_system_set_stream(P.system.sys, stream.cuda_stream)
                    lsw.lsw_reformat(S.sys, P.system.sys, shift, P.phi, phi)
                else:
                    atoms = sorted(set(int(a) for a in S.sf_atom))
                    cg = {a: _keys_to_g(S.keys(a, 0, 0)) for a in atoms}
                    fg = {a: _keys_to_g(S.keys(a, 0, 1)) for a in atoms}
                    I.fill_phi(wl, phi, S.off_L, S.sf_atom, cg, fg)
            V = I.potential_fast(wl, "cuda").to(self.dt)
            lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
            hphi = torch.empty(S.total_Lp, dtype=self.dt, device="cuda")
            ek = torch.empty(S.n_sf, dtype=torch.float64, device="cuda")
            ep = torch.empty(S.n_sf, dtype=torch.float64, device="cuda")
            nnz = max(1, len(S.col))
            H = torch.empty(nnz, dtype=torch.float64, device="cuda")
            Sm = torch.empty(nnz, dtype=torch.float64, device="cuda")
            lsw.lsw_apply_hamiltonian(S.sys, phi, hphi, ek, ep)
            self._retry_oom(lambda: lsw.lsw_build_matrices(S.sys, phi, hphi, H, Sm))
            out = {k: torch.empty(v.numel(), dtype=torch.float64, pin_memory=True)
                   for k, v in (("H", H), ("S", Sm), ("ek", ek), ("ep", ep))}
            for k, v in (("H", H), ("S", Sm), ("ek", ek), ("ep", ep)):
                out[k].copy_(v, non_blocking=True)
            job.event = torch.cuda.Event()
            job.event.record(stream)
        job.bufs = dict(phi=phi, V=V, hphi=hphi, ek=ek, ep=ep, H=H, Sm=Sm, out=out)

    def _finish(self, job: _Job, t0) -> Result:
        S = job.system
        out = job.bufs["out"]
        res = Result(job.req.rid, job.req.kind, S.n_sf, job.req.t_arrival, job.t_admit - t0,
                     time.perf_counter() - t0, out["H"].numpy()[:len(S.col)].copy(),
                     out["S"].numpy()[:len(S.col)].copy(), out["ek"].numpy().copy(), out["ep"].numpy().copy())
        lsw.lsw_sync(S.sys, 600.0)                  # device-side checks of this request
        phi = job.bufs["phi"]
        if job.parent is not None:
            job.parent.busy = False
        if job.req.kind == "charged" and job.parent is not None:
            self.used -= job.est_bytes
        else:
            ent = _Entry(job.req.rid, job.wl, S, phi, False, 0)
            ent.bytes = lsw.lsw_workspace_bytes(S.sys) + self.es * S.total_L
            self.used += ent.bytes - job.est_bytes
            self.resident[job.req.rid] = ent
        job.bufs = {}
        # PyTorch caches freed blocks per stream; past CACHE_SLACK of cached, unused bytes
        # they go back to the driver, where the library's own allocations can use them
        torch = self.torch
        if torch.cuda.memory_reserved() - torch.cuda.memory_allocated() > CACHE_SLACK:
            torch.cuda.empty_cache()
        return res

    def _evict(self, need):
        """Drop idle resident systems (least recently used first) until need fits."""
        for rid in list(self.resident.keys()):
            if self.used + need <= self.budget:
                return True
            ent = self.resident[rid]
            if ent.busy:
                continue
            del self.resident[rid]
            self.used -= ent.bytes
            ent.system.close()
            ent.phi = None
            # the evicted request's tensors go back to the driver, where the library's own
            # allocations (workspace, panels) can use them
            torch = getattr(self, "torch", None)
            if torch is not None:
                torch.cuda.empty_cache()
        return self.used + need <= self.budget

    def _admit(self, cand, inflight, max_inflight):
        """Admit prepared jobs (in arrival order) while a stream is free and their memory
        fits the budget after evicting idle resident systems; returns the admitted jobs.

        A job larger than the whole budget can never run: that is an error.  While work
        is in flight a job that does not fit waits for it (first come, first served);
        when nothing is in flight nothing would release memory for it, so later jobs
        that fit go first."""
        admitted = []
        for job in cand:
            if len(inflight) + len(admitted) >= max_inflight:
                break
            if job.est_bytes > self.budget:
                raise RuntimeError("request %d needs %.3f GB, more than the whole %.3f GB budget"
                                   % (job.req.rid, job.est_bytes / 1e9, self.budget / 1e9))
            if not self._evict(job.est_bytes):
                if inflight or admitted:
                    break
                continue
            busy = {id(j.stream) for j in list(inflight) + admitted}
            free = [st for st in self.streams if id(st) not in busy]
            if not free:
                break
            job.stream = free[0]
            job.t_admit = time.perf_counter()
            self.used += job.est_bytes
            admitted.append(job)
        return admitted

    # ---------------------------------------------------------------- the loop
    def run(self, requests, realtime=True, max_inflight=None):
        """Serve ``requests`` (sorted by arrival); returns results in completion order.

        Worker threads build each arrived request's system (host), and, once the
        request is admitted, its device inputs and its enqueued work (on its own
        stream); this thread admits under the budget and polls completions."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        tasks: "queue.Queue" = queue.Queue()
        ready: list[_Job] = []
        lock = threading.Lock()
        inflight: list[_Job] = []
        self._ready, self._inflight = ready, inflight      # for the out-of-memory report
        results: list[Result] = []
        errors: list[BaseException] = []
        max_inflight = max_inflight or len(self.streams)
        wl_of = {}
        t0 = time.perf_counter()
        stop = threading.Event()

        def worker():
            torch.cuda.set_device(self.device)
            while not stop.is_set():
                try:
                    kind, job = tasks.get(timeout=0.01)
                except queue.Empty:
                    continue
                try:
                    if kind == "prep":
                        self._prepare(job)
                        with lock:
                            ready.append(job)
                    else:
                        self._launch(job, job.stream)
                        job.bufs["launched"] = True
                except BaseException as e:      # surfaced by the loop
                    errors.append(e)

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.host_threads)]
        for th in threads:
            th.start()
        nxt = 0
        waiting = []
        try:
            while len(results) < len(reqs):
                if errors:
                    raise errors[0]
                now = time.perf_counter() - t0
                while nxt < len(reqs) and (not realtime or reqs[nxt].t_arrival <= now):
                    waiting.append(reqs[nxt])
                    nxt += 1
                still = []
                for r in waiting:
                    if r.kind == "new" or r.parent is None:
                        wl_of[r.rid] = new_workload(r.n_atoms, r.seed)
                        tasks.put(("prep", _Job(r, wl_of[r.rid])))
                        continue
                    par = self.resident.get(r.parent)
                    if par is None or par.busy:
                        if par is None and _done(results, r.parent) and r.parent in wl_of:
                            # parent evicted: serve it as a fresh system of that geometry
                            base = wl_of[r.parent]
                            wl = perturbed(base, r.seed) if r.kind == "perturb" else charged(base, r.seed)
                            wl_of[r.rid] = wl
                            tasks.put(("prep", _Job(Request(r.rid, r.t_arrival, "new", r.n_atoms, r.seed), wl)))
                            continue
                        still.append(r)
                        continue
                    par.busy = True
                    self.resident.move_to_end(r.parent)
                    wl = perturbed(par.wl, r.seed) if r.kind == "perturb" else charged(par.wl, r.seed)
                    wl_of[r.rid] = wl
                    tasks.put(("prep", _Job(r, wl, parent=par)))
                waiting = still
                # admission: prepared requests whose memory fits, on a free stream
                with lock:
                    cand = list(ready)
                for job in self._admit(cand, inflight, max_inflight):
                    with lock:
                        ready.remove(job)
                    inflight.append(job)
                    tasks.put(("launch", job))
                done = [j for j in inflight if j.bufs.get("launched") and j.event.query()]
                for j in done:
                    inflight.remove(j)
                    results.append(self._finish(j, t0))
                if not done:
                    time.sleep(0.0005)
        finally:
            stop.set()
            for th in threads:
                th.join()
            torch.cuda.synchronize()
        return results

    def close(self):
        for ent in self.resident.values():
            ent.system.close()
        self.resident.clear()
        lsw.lsw_ctx_destroy(self.ctx)


def _done(results, rid):
    return any(r.rid == rid for r in results)


def summarize(results, wall_s=None):
    lat = np.array([r.latency for r in results])
    n_sf = sum(r.n_sf for r in results)
    span = wall_s if wall_s is not None else max(r.t_done for r in results) - min(r.t_arrival for r in results)
    return {"requests": len(results), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "support_functions": int(n_sf),
            "support_functions_per_s": n_sf / span, "span_s": span}
