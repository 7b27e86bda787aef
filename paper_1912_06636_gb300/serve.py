"""Continuous-batching request loop for grid integration on one GPU.

A request is one molecule that runs ``n_iter`` SCF-like iterations on the device: each
iteration perturbs the potential, v_it = v0 (1 + 0.01 u), u ~ U(-1, 1) per point, draws a
fresh symmetric positive semi-definite density matrix P_it = X X^T / k (X ~ N(0, 1), nb x k),
and calls the library's Hamiltonian integration (Eqs. H_int_aims / H_decomp) and density
update (Eq. Density) on the request's own CUDA stream. Iteration it + 1 is issued when
iteration it has completed on the device, as in an SCF loop where the next density matrix
needs the last Hamiltonian.

Scheduling:
  * requests arrive at their arrival times (seconds after the loop starts) and wait in FIFO
    order;
  * the head of the queue is admitted when a slot is free and its estimated device memory fits
    the HBM budget (no request overtakes an earlier one, so none starves);
  * an admitted request's handle is created on a worker thread (partition, relevance and the
    uploads run on the handle's own stream from a stream-ordered pool, so creating and
    destroying handles does not stall other requests' kernels);
  * every active request keeps its grid, basis tables, H, P, v and n resident on the device
    across its iterations; requests on different streams overlap on the GPU;
  * when a request finishes, its memory is released and the next one is admitted.

All integration arithmetic runs in the library's CUDA kernels; torch only provides device
memory, streams, events and the synthetic inputs (uniform and normal draws, X X^T).
"""
from __future__ import annotations

import collections
import concurrent.futures
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import nao


@dataclass
class Request:
    rid: int
    system: object          # the fields of nao_system_desc (e.g. synth.System)
    v0: np.ndarray          # [n_points] base potential, the system's original point order
    arrival_s: float
    n_iter: int = 20
    seed: int = 0


@dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float
    started_s: float
    done_s: float
    n_points: int
    n_basis: int
    n_iter: int
    device_bytes: int
    n_electrons: np.ndarray
    flops: int = 0          # algorithmic FLOPs of all iterations (H and n, nao_grid_info)
    H: np.ndarray | None = None
    n: np.ndarray | None = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def n_basis_of(system) -> int:
    off = np.asarray(system.species_fn_offset)
    fn_l = np.asarray(system.fn_l)
    per = [int(np.sum(2 * fn_l[off[s]:off[s + 1]] + 1)) for s in range(len(off) - 1)]
    return int(sum(per[s] for s in np.asarray(system.atom_species)))


def estimate_bytes(n_points: int, nb: int, max_batch_points: int, scratch_bytes: int, p_rank: int) -> int:
    """Upper estimate of one request's device memory: the handle (points and batch tables,
    reduced-basis lists bounded by every batch holding every function, evaluation scratch, the
    split path's slices at up to three times the scratch) plus the request's H, P, v, v0, n, u and X."""
    n_batches = max(1, math.ceil(n_points / max_batch_points))
    handle = 48 * n_points + 16 * n_batches * nb + 4 * scratch_bytes + (8 << 20)
    buffers = 16 * nb * nb + 8 * nb * p_rank + 40 * n_points
    return int(handle + buffers)


@dataclass
class _Slot:
    req: Request
    grid: object = None
    stream: object = None
    bufs: dict = field(default_factory=dict)
    it: int = 0
    event: object = None
    reserved: int = 0
    admitted_s: float = 0.0
    started_s: float = 0.0
    future: object = None


class Server:
    def __init__(self, prec="split", hbm_budget_bytes: int = 150 << 30, max_active: int = 16, device: int | None = None,
                 split_slices: int | None = None, split_digits: int | None = None, capture_graph: bool = True,
                 keep_results: bool = False,
                 scratch_bytes: int = 256 << 20, p_rank: int = 16, max_batch_points: int = 200):
        import torch

        self.torch = torch
        self.prec = prec
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.opts = {"capture_graph": 1 if capture_graph else 0, "scratch_bytes": int(scratch_bytes),
                     "max_batch_points": int(max_batch_points)}
        if split_slices is not None:
            self.opts["split_slices"] = int(split_slices)
        if split_digits is not None:
            self.opts["split_digits"] = int(split_digits)
        self.keep = keep_results
        self.p_rank = int(p_rank)
        self.scratch_bytes = int(scratch_bytes)
        self.max_batch_points = int(max_batch_points)
        self.stats = {}
        # one stream per slot, reused by the requests that hold the slot (the caching allocator
        # keeps each stream's freed blocks for that stream)
        self.free_streams = collections.deque(torch.cuda.Stream(device=self.device) for _ in range(self.max_active))

    # -- per request ------------------------------------------------------------------
    def _create(self, slot: _Slot):
        torch = self.torch
        r = slot.req
        with torch.cuda.device(self.device):
            g = nao.Grid(r.system, device=self.device.index, **self.opts)
            s = slot.stream
            with torch.cuda.stream(s):
                nb, npts = g.nb, g.n_points
                b = {
                    "v0": torch.from_numpy(np.ascontiguousarray(r.v0, dtype=np.float64)).to(self.device, non_blocking=False),
                    "v": torch.empty(npts, dtype=torch.float64, device=self.device),
                    "u": torch.empty(npts, dtype=torch.float64, device=self.device),
                    "X": torch.empty((nb, self.p_rank), dtype=torch.float64, device=self.device),
                    "P": torch.empty((nb, nb), dtype=torch.float64, device=self.device),
                    "H": torch.empty((nb, nb), dtype=torch.float64, device=self.device),
                    "n": torch.empty(npts, dtype=torch.float64, device=self.device),
                    "ne": torch.zeros(r.n_iter, dtype=torch.float64, device=self.device),
                    "gen": torch.Generator(device=self.device),
                }
            s.synchronize()
        return g, b

    def _actual_bytes(self, slot: _Slot) -> int:
        torch = self.torch
        return int(nao.nao_get_info(slot.grid.h).device_bytes) + sum(
            x.numel() * x.element_size() for x in slot.bufs.values() if isinstance(x, torch.Tensor))

    def _issue(self, slot: _Slot):
        """Enqueue iteration slot.it of the request on its stream."""
        torch = self.torch
        r, b, g, s = slot.req, slot.bufs, slot.grid, slot.stream
        with torch.cuda.stream(s):
            b["gen"].manual_seed(int(r.seed) * 1_000_003 + slot.it)
            torch.rand(b["u"].shape, generator=b["gen"], dtype=torch.float64, device=self.device, out=b["u"])
            torch.mul(b["v0"], b["u"].mul_(0.02).add_(0.99), out=b["v"])
            torch.randn(b["X"].shape, generator=b["gen"], dtype=torch.float64, device=self.device, out=b["X"])
            torch.mm(b["X"], b["X"].t(), out=b["P"])
            b["P"].mul_(1.0 / self.p_rank)
            g.integrate_h(b["v"], prec=self.prec, H=b["H"], stream=s)
            g.update_density(b["P"], prec=self.prec, n=b["n"], ne=b["ne"][slot.it:slot.it + 1], stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        slot.event = ev
        slot.it += 1

    # -- the loop ----------------------------------------------------------------------
    def run(self, requests: list[Request]) -> list[Result]:
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival_s))
        waiting: collections.deque[Request] = collections.deque()
        creating: list[_Slot] = []
        active: list[_Slot] = []
        results: list[Result] = []
        used = 0
        peak_used, peak_active = 0, 0
        pool = concurrent.futures.ThreadPoolExecutor(max_workers=2)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        try:
            while pending or waiting or creating or active:
                t = now()
                while pending and pending[0].arrival_s <= t:
                    waiting.append(pending.popleft())
                # admission: FIFO head, by slot and memory
                while waiting and len(active) + len(creating) < self.max_active:
                    r = waiting[0]
                    est = estimate_bytes(len(r.v0), n_basis_of(r.system), self.max_batch_points,
                                         self.scratch_bytes, self.p_rank)
                    if used + est > self.budget and (active or creating):
                        break
                    waiting.popleft()
                    slot = _Slot(req=r, reserved=est, admitted_s=now(), stream=self.free_streams.popleft())
                    used += est
                    slot.future = pool.submit(self._create, slot)
                    creating.append(slot)
                peak_used = max(peak_used, used)
                # handles that finished creating start their first iteration
                for slot in [c for c in creating if c.future.done()]:
                    creating.remove(slot)
                    slot.grid, slot.bufs = slot.future.result()
                    slot.started_s = now()
                    active.append(slot)
                    self._issue(slot)
                    # the first call also set up the precision's device buffers: account the
                    # request's actual device memory from now on
                    actual = self._actual_bytes(slot)
                    used += actual - slot.reserved
                    slot.reserved = actual
                peak_active = max(peak_active, len(active))
                # completed iterations: next iteration, or retire the request
                progressed = False
                for slot in list(active):
                    if not slot.event.query():
                        continue
                    progressed = True
                    if slot.it < slot.req.n_iter:
                        self._issue(slot)
                        continue
                    done = now()
                    slot.grid.sync()
                    b = slot.bufs
                    with torch.cuda.stream(slot.stream):  # its work is complete: these copies do not wait
                        res = Result(rid=slot.req.rid, arrival_s=slot.req.arrival_s, admitted_s=slot.admitted_s,
                                     started_s=slot.started_s, done_s=done, n_points=slot.grid.n_points,
                                     n_basis=slot.grid.nb, n_iter=slot.req.n_iter,
                                     device_bytes=int(slot.reserved), n_electrons=b["ne"].cpu().numpy(),
                                     flops=int(slot.grid.info.flops_h + slot.grid.info.flops_n) * slot.req.n_iter)
                        if self.keep:
                            res.H = b["H"].cpu().numpy()
                            res.n = b["n"].cpu().numpy()
                    results.append(res)
                    active.remove(slot)
                    slot.grid.close()
                    slot.bufs = None
                    self.free_streams.append(slot.stream)
                    used -= slot.reserved
                if not progressed and not any(c.future.done() for c in creating):
                    time.sleep(5e-5)
        finally:
            pool.shutdown(wait=True)
            for slot in active + creating:
                if slot.grid is not None:
                    slot.grid.close()
                if slot.stream is not None:
                    self.free_streams.append(slot.stream)
        makespan = now()
        self.stats = {"makespan_s": makespan, "peak_reserved_bytes": int(peak_used), "peak_active": int(peak_active)}
        return sorted(results, key=lambda x: x.rid)


def summarize(results: list[Result], stats: dict) -> dict:
    lat = np.array([r.latency_s for r in results]) * 1e3
    pts_it = float(sum(r.n_points * r.n_iter for r in results))
    mk = stats.get("makespan_s", float("nan"))
    return {
        "requests": len(results),
        "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
        "mean_ms": float(lat.mean()) if lat.size else None,
        "makespan_s": mk,
        "requests_per_s": len(results) / mk if mk > 0 else None,
        "point_iterations_per_s": pts_it / mk if mk > 0 else None,
        "gflops_algorithmic": sum(r.flops for r in results) / mk / 1e9 if mk > 0 else None,
        "peak_active": stats.get("peak_active"),
        "peak_reserved_gb": stats.get("peak_reserved_bytes", 0) / 1e9,
    }
