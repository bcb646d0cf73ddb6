"""Continuous-batching request loop over the SGF C ABI.

Requests ask either for a new factorization plus a solve ("factor") or for a
solve against a factor kept resident on the device ("solve"), each with 1-8
right-hand sides, on 3D 7-point diffusion problems of different grid sizes.
They arrive over time; an arriving request is admitted as soon as a worker
slot is free and its device-memory footprint (the plan's structural bound for
a factor, the work vectors for a solve) fits the budget next to the resident
factors and the requests in flight.  Admitted requests run concurrently, each
on its own CUDA stream from its own worker thread (the C calls release the
GIL), so their device work overlaps.  Resident factors are evicted least
recently used when memory is needed and they are idle.  The loop reports
p50/p99 latency (completion minus arrival) and solves per second.

All numerical work runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import heapq
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field

import numpy as np

import sgf_inputs as si

from . import Factor, Plan


@dataclass
class Resident:
    key: tuple
    factor: Factor
    plan: Plan
    nbytes: int
    lock: threading.Lock = field(default_factory=threading.Lock)
    users: int = 0
    coeff_req: dict = None


class Admission:
    """Host-side admission state: worker slots and a device-memory budget."""

    def __init__(self, slots: int, budget_bytes: int):
        self.slots = slots
        self.budget = budget_bytes
        self.inflight = 0
        self.reserved = 0       # bytes of requests in flight
        self.resident = 0       # bytes of resident factors

    def fits(self, need: int) -> bool:
        return self.inflight < self.slots and self.reserved + self.resident + need <= self.budget

    def take(self, need: int):
        self.inflight += 1
        self.reserved += need

    def release(self, need: int):
        self.inflight -= 1
        self.reserved -= need


class Server:
    def __init__(self, slots: int = 4, budget_bytes: int = 64 << 30, precision: str = "mixed",
                 rtol: float = 1e-10, maxit: int = 500, device: int = 0, keep_results: bool = False):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.precision = precision
        self.rtol, self.maxit = rtol, maxit
        self.adm = Admission(slots, budget_bytes)
        self.cv = threading.Condition()
        self.plans = {}
        self.resident: "OrderedDict[tuple, Resident]" = OrderedDict()
        self.keep_results = keep_results
        self.results = {}
        self.records = []
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]

    # -- sizing --------------------------------------------------------------
    def plan_for(self, edge: int) -> Plan:
        with self.cv:
            p = self.plans.get(edge)
        if p is None:
            cfg = dict(n=(edge, edge, edge), dim=3, stencil="7pt_fv_3d", dirichlet=1, leaf=8, degree=2)
            p = Plan(cfg["n"], 3, cfg["stencil"], cfg["dirichlet"], cfg["leaf"], cfg["degree"],
                     precision=self.precision)
            with self.cv:
                p = self.plans.setdefault(edge, p)
        return p

    def need_bytes(self, req) -> int:
        n = req["edge"] ** 3
        vec = 8 * n * (2 * req["nrhs"] + 6)
        if req["kind"] == "factor":
            fp64, mixed = self.plan_for(req["edge"]).footprint()
            return vec + (mixed if self.precision == "mixed" else fp64)
        return vec

    # -- resident factors -------------------------------------------------------
    def _evict_for(self, need: int):
        """Drop idle resident factors (LRU) until `need` fits; caller holds cv."""
        for key in list(self.resident.keys()):
            if self.adm.reserved + self.adm.resident + need <= self.adm.budget:
                return
            r = self.resident[key]
            if r.users == 0:
                del self.resident[key]
                self.adm.resident -= r.nbytes
                r.factor.close()

    def _pick_resident(self, req):
        """Choose a resident factor for a solve request (uniform by req['pick'])."""
        keys = [k for k in self.resident.keys()]
        if not keys:
            return None
        k = keys[min(int(req["pick"] * len(keys)), len(keys) - 1)]
        r = self.resident[k]
        r.users += 1
        self.resident.move_to_end(k)
        return r

    # -- execution --------------------------------------------------------------
    def _run(self, req, slot: int, resident):
        torch = self.torch
        stream = self.streams[slot]
        out = {}
        with torch.cuda.stream(stream):
            if req["kind"] == "factor":
                plan = self.plan_for(req["edge"])
                coeffs = torch.from_numpy(si.request_coeffs(req).ravel()).to(self.dev, non_blocking=False)
                F = Factor(plan, coeffs, stream=stream)
                resident = Resident(key=("req", req["id"]), factor=F, plan=plan,
                                    nbytes=self.need_bytes(dict(req, nrhs=0)))
                resident.coeff_req = req
                resident.users = 1
            n = resident.plan.n
            b = torch.from_numpy(si.rhs(n, req["rhs_seed"], nrhs=req["nrhs"]).reshape(req["nrhs"], n)).to(self.dev)
            with resident.lock:          # one solve at a time per factor
                x, info = resident.factor.pcg(b.reshape(-1), rtol=self.rtol, maxit=self.maxit,
                                              stream=stream, check=False)
            stream.synchronize()
            if self.keep_results:
                out["x"] = x.reshape(req["nrhs"], n).cpu().numpy()
            out.update(info)
            out["edge"] = resident.plan.n
        return out, resident

    def _worker(self, slot, job):
        req, need, resident, t_arr = job
        try:
            out, resident = self._run(req, slot, resident)
            err = None
        except Exception as e:  # a failing request is reported, the loop goes on
            out, err = {}, repr(e)
        t_done = time.perf_counter()
        with self.cv:
            self.adm.release(need)
            if resident is not None:
                resident.users -= 1
                if req["kind"] == "factor" and err is None and resident.key not in self.resident:
                    self._evict_for(resident.nbytes)
                    self.resident[resident.key] = resident
                    self.adm.resident += resident.nbytes
            self.records.append(dict(id=req["id"], kind=req["kind"], edge=req["edge"], nrhs=req["nrhs"],
                                     latency=t_done - t_arr, error=err,
                                     factor_of=resident.key[1] if resident is not None else None,
                                     iterations=out.get("iterations"), rel_residual=out.get("rel_residual")))
            if self.keep_results and "x" in out:
                self.results[req["id"]] = out["x"]
            self.cv.notify_all()

    def run(self, requests, time_scale: float = 1.0):
        """Replay `requests` (arrival_s sorted) in real time; returns the summary."""
        reqs = sorted(requests, key=lambda r: r["arrival_s"])
        pending = []          # arrived, waiting for admission (FIFO)
        threads = []
        free_slots = list(range(self.adm.slots))
        t0 = time.perf_counter()
        i = 0
        with self.cv:
            while i < len(reqs) or pending or self.adm.inflight:
                now = time.perf_counter() - t0
                while i < len(reqs) and reqs[i]["arrival_s"] * time_scale <= now:
                    pending.append((reqs[i], t0 + reqs[i]["arrival_s"] * time_scale))
                    i += 1
                # admit in arrival order while slots and memory allow
                while pending:
                    req, t_arr = pending[0]
                    if req["kind"] == "solve" and not self.resident:
                        req = dict(req, kind="factor")      # nothing resident yet
                    need = self.need_bytes(req)
                    if not self.adm.fits(need):
                        self._evict_for(need)
                        if not self.adm.fits(need):
                            break
                    if not free_slots:
                        break
                    pending.pop(0)
                    resident = self._pick_resident(req) if req["kind"] == "solve" else None
                    if req["kind"] == "solve" and resident is None:
                        req = dict(req, kind="factor")
                        need = self.need_bytes(req)
                    self.adm.take(need)
                    slot = free_slots.pop()
                    th = threading.Thread(target=self._slot_main, args=(slot, (req, need, resident, t_arr), free_slots))
                    th.start()
                    threads.append(th)
                wait = None
                if i < len(reqs):
                    wait = max(0.0, reqs[i]["arrival_s"] * time_scale - (time.perf_counter() - t0))
                self.cv.wait(timeout=wait if wait is not None else 0.05)
        for th in threads:
            th.join()
        makespan = time.perf_counter() - t0
        return self.summary(makespan)

    def _slot_main(self, slot, job, free_slots):
        self._worker(slot, job)
        with self.cv:
            free_slots.append(slot)
            self.cv.notify_all()

    def summary(self, makespan: float):
        ok = [r for r in self.records if r["error"] is None]
        lat = np.array([r["latency"] for r in ok]) * 1e3
        solves = sum(r["nrhs"] for r in ok)
        return dict(requests=len(self.records), failed=len(self.records) - len(ok),
                    p50_ms=float(np.percentile(lat, 50)) if lat.size else None,
                    p99_ms=float(np.percentile(lat, 99)) if lat.size else None,
                    mean_ms=float(lat.mean()) if lat.size else None,
                    solves_per_s=solves / makespan if makespan > 0 else None,
                    makespan_s=makespan, factors=sum(1 for r in ok if r["kind"] == "factor"),
                    max_rel_residual=max((r["rel_residual"] or 0) for r in ok) if ok else None)

    def close(self):
        for r in self.resident.values():
            r.factor.close()
        self.resident.clear()
