"""Continuous-batching detection server.

The paper serves its detector on demand (a function-as-a-service endpoint
that takes an image and returns the feature count, §4).  Here the on-demand
loop is in-process and GPU-resident:

* the detector state (compiled kernel, ladder tables, scratch) stays on the
  device: every slot owns a ``Detector``, a CUDA stream and a device image
  buffer, created once;
* requests (host tiles of any size, uint8/uint16/float32) arrive at any time
  and queue; a request is admitted into a free slot as soon as the HBM budget
  allows its footprint (the slot's resident scratch grows to the largest tile
  it has served; the detector's fixed state, the image buffer and the
  per-image scratch are charged at the sizes the library reports);
* an admitted request's host-to-device copy and detection are enqueued
  asynchronously on its slot's stream, so requests admitted while others are
  still on the GPU overlap with them on the device (continuous batching, not
  a queue);
* completions are polled without blocking; a finished slot's result is read,
  its future fulfilled, and the slot and its memory are immediately offered to
  the next waiting request.

Each request's result is exactly the result of detecting that tile alone: a
slot's detection depends only on its own inputs and its own scratch.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Optional

import numpy as np

from . import Detector



@dataclasses.dataclass
class _Req:
    img: np.ndarray
    future: cf.Future
    t_arrive: float
    host: object = None           # pinned host bytes of img (torch uint8)
    slot: int = -1
    t_admit: float = 0.0


def image_bytes(shape, dtype) -> int:
    """Bytes of a tile's device copy."""
    H, W = shape
    return H * W * np.dtype(dtype).itemsize


def plan_admission(free, need, resident, used, budget, fixed):
    """Admission step for the request at the head of the queue.

    `free` lists the free slots, `need[k]` the bytes slot k would have to
    grow by to serve the request, `resident[k]` its resident bytes, `used`
    the bytes charged over all slots.  Returns ("admit", k) for the free slot
    needing the least growth that keeps `used` within `budget` (ties: the
    first in `free`); else ("reset", j) for the free slot with the most
    scratch grown beyond `fixed` (giving it back may make room); else
    ("wait", None) until a running detection completes."""
    for k in sorted(free, key=lambda k: need[k]):
        if used + need[k] <= budget:
            return "admit", k
    grown = [j for j in free if resident[j] > fixed]
    if grown:
        return "reset", max(grown, key=lambda j: resident[j])
    return "wait", None


class Server:
    """Slots x streams detection service with HBM-budget admission."""

    def __init__(self, n_slots=8, hbm_budget=40 << 30, device=0, **detector_params):
        import torch
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self.budget = int(hbm_budget)
        self.params = detector_params
        self.slots = []
        for _ in range(n_slots):
            self.slots.append({
                "det": Detector(device=device, **detector_params),
                "stream": torch.cuda.Stream(device=device),
                "buf": None,          # device image buffer (grows)
                "req": None,
            })
        # what every slot's detector holds, as the library allocates it
        self.fixed = self.slots[0]["det"].device_bytes()[0]
        for slot in self.slots:
            slot["resident"] = self.fixed
        self.used = sum(s["resident"] for s in self.slots)
        if self.used > self.budget:
            raise ValueError("budget smaller than the slots' fixed state")
        self.queue = collections.deque()
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.stop = False
        self.stats = {"admitted": 0, "completed": 0, "peak_in_flight": 0, "peak_bytes": self.used}
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # -------------------------------------------------------------- client
    def submit(self, img: np.ndarray) -> cf.Future:
        """Queue a host tile; returns a future of its DetectionResult.  A
        pageable (not pinned) image is first copied into pinned memory here,
        on the caller's thread, so that the server thread only enqueues
        asynchronous copies and never stalls other requests on host work."""
        t_arrive = time.perf_counter()
        fut = cf.Future()
        if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16, np.float32):
            fut.set_exception(TypeError("2-D uint8/uint16/float32 image expected"))
            return fut
        fixed_all = self.fixed * len(self.slots)
        if fixed_all + self.footprint(img.shape, img.dtype) > self.budget:
            fut.set_exception(ValueError("tile does not fit the HBM budget"))
            return fut
        host = self.torch.from_numpy(np.ascontiguousarray(img).reshape(-1).view(np.uint8))
        if not host.is_pinned():
            host = host.pin_memory()
        with self.cv:
            self.queue.append(_Req(img=img, future=fut, t_arrive=t_arrive, host=host))
            self.cv.notify()
        return fut

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()
        for s in self.slots:
            s["det"].close()

    def footprint(self, shape, dtype) -> int:
        """Device bytes a request of this size needs beyond the fixed slot
        state: the tile's device copy and the detector's per-image scratch
        (tile counters, candidate staging, prune grid), as the library
        reports them."""
        return image_bytes(shape, dtype) + self.slots[0]["det"].device_bytes(*shape)[1]

    # ----------------------------------------------------------- internals
    def _need(self, slot, req) -> int:
        want = self.fixed + self.footprint(req.img.shape, req.img.dtype)
        return max(0, want - slot["resident"])

    def _reset(self, k):
        """Give a free slot's grown scratch back (the detector's per-image
        scratch and the slot's image buffer; its fixed state stays)."""
        slot = self.slots[k]
        slot["det"].trim()
        slot["buf"] = None
        self.used -= slot["resident"] - self.fixed
        slot["resident"] = self.fixed

    def _admit(self, k, req):
        torch = self.torch
        slot = self.slots[k]
        extra = self._need(slot, req)
        slot["resident"] += extra
        self.used += extra
        img = req.img
        nbytes = img.nbytes
        if slot["buf"] is None or slot["buf"].numel() < nbytes:
            slot["buf"] = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        host = req.host
        tdtype = {np.dtype(np.uint8): torch.uint8, np.dtype(np.uint16): torch.int16,
                  np.dtype(np.float32): torch.float32}[img.dtype]
        with torch.cuda.stream(slot["stream"]):
            slot["buf"][:nbytes].copy_(host, non_blocking=True)
            dev = slot["buf"][:nbytes].view(tdtype).view(img.shape)
            slot["det"].detect(dev, slot["stream"])
        slot["host_ref"] = host
        slot["req"] = req
        req.slot = k
        req.t_admit = time.perf_counter()
        self.stats["admitted"] += 1

    def _loop(self):
        while True:
            with self.cv:
                if self.stop and not self.queue and all(s["req"] is None for s in self.slots):
                    return
                # admit in arrival order while slots and budget allow
                while self.queue:
                    req = self.queue[0]
                    free = [k for k, s in enumerate(self.slots) if s["req"] is None]
                    # prefer a slot whose resident state already fits the
                    # tile; else release the biggest grown scratch and retry
                    act, k = plan_admission(
                        free, {j: self._need(self.slots[j], req) for j in free},
                        {j: self.slots[j]["resident"] for j in free}, self.used, self.budget,
                        self.fixed)
                    if act == "wait":
                        break
                    if act == "reset":
                        self._reset(k)
                        continue
                    self.queue.popleft()
                    self._admit(k, req)
                in_flight = sum(1 for s in self.slots if s["req"] is not None)
                self.stats["peak_in_flight"] = max(self.stats["peak_in_flight"], in_flight)
                self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.used)
                if in_flight == 0:
                    self.cv.wait(timeout=0.01)
                    continue
            # poll completions without blocking the submitters
            done_any = False
            for s in self.slots:
                req = s["req"]
                if req is None or not s["det"].ready():
                    continue
                try:
                    res = s["det"].wait()
                    res.latency_ms = 1e3 * (time.perf_counter() - req.t_arrive)
                    res.queue_ms = 1e3 * (req.t_admit - req.t_arrive)
                    err = None
                except Exception as e:  # pragma: no cover - surfaced to the client
                    err = e
                with self.cv:
                    s["req"] = None
                    s["host_ref"] = None
                    self.stats["completed"] += 1
                if err is None:
                    req.future.set_result(res)
                else:
                    req.future.set_exception(err)
                done_any = True
            if not done_any:
                time.sleep(20e-6)


def poisson_arrivals(rate, duration, seed):
    """Arrival times (s) of a Poisson stream of the given rate over `duration`."""
    rng = np.random.default_rng([int(seed), int(rate)])
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append(t)


def run_open_loop(server, tiles, arrivals):
    """Submit tiles[i] at arrivals[i] (seconds from now); returns results in
    submission order and the wall time from the first arrival to the last
    completion."""
    t0 = time.perf_counter()
    futs = []
    for img, ta in zip(tiles, arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        futs.append(server.submit(img))
    res = [f.result() for f in futs]
    return res, time.perf_counter() - t0
