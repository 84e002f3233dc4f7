"""Continuous-batching eigensolver service on one GPU.

Requests (a device-resident symmetric or Hermitian matrix and the number of
lowest eigenpairs wanted) arrive over time, e.g. from the self-consistency
iterations of an electronic-structure code (Sec. 5.1), where each system is
re-submitted with a slightly changed matrix.  The server admits a waiting
request as soon as a slot (a CUDA stream) is free and the request's device
memory (workspace and outputs) fits in the HBM budget; admitted requests run
concurrently on their streams, so new work overlaps work already on the GPU.
Completion is detected with CUDA events; latency = completion - arrival.

With stage_batching the server also batches one stage across requests: each
admitted request runs its first stage (full -> band) on its slot, and the
bulge chases of every request whose first stage has finished run together
in one persistent launch on one of a few chase lanes (streams); each request
then runs its remaining stages on its slot again.  The results are
bit-identical to the one-call solve.  Merging pays little when the requests'
chases already overlap on their own streams; it pays when more problems are
ready at once than there are streams.

All numerical work happens in the library's C entry points
(gb_solve_d / gb_solve_z); this module only schedules.
"""
import collections
import time
from dataclasses import dataclass, field

import torch

from . import _lib as gb


@dataclass
class Request:
    rid: int
    A: torch.Tensor            # n x n device matrix (column-major data; symmetric / Hermitian)
    nev: int
    arrival: float             # seconds on the server clock
    nbw: int = 0
    ev: torch.Tensor = None
    Z: torch.Tensor = None
    start: float = None
    done: float = None
    status: int = None
    _ws: torch.Tensor = None
    _ready: torch.cuda.Event = None   # recorded on the submitting stream: A is written
    _end: torch.cuda.Event = None
    _front: torch.cuda.Event = None
    _phase: str = None          # stage batching: "front", "chase_wait", "chase", "back"
    _slot: int = None
    _bytes: int = 0

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def complex(self):
        return self.A.is_complex()

    def latency(self):
        return None if self.done is None else self.done - self.arrival


def request_bytes(n, nev, cplx, nbw):
    """Device bytes a request holds while admitted: workspace and outputs."""
    ws = (gb.gb_solve_workspace_bytes_z if cplx else gb.gb_solve_workspace_bytes)(n, nev, nbw)
    return ws + 8 * nev + (16 if cplx else 8) * n * nev


class EigenServer:
    def __init__(self, slots=4, hbm_budget_bytes=64 << 30, device=0, stage_batching=False, chase_lanes=4):
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.stage_batching = stage_batching
        if stage_batching:
            # chase lanes: up to chase_lanes merged chase launches in flight,
            # each on its own stream with its own problem table, so a long
            # chase does not hold back the requests that become ready after it
            self.table_bytes = gb.gb_solve_stage_table_bytes(slots)
            self.lanes = [{"stream": torch.cuda.Stream(device=self.device),
                           "table": torch.zeros(self.table_bytes, dtype=torch.uint8, device=self.device),
                           "batch": [], "end": None} for _ in range(max(1, chase_lanes))]
            self.chase_sizes = []       # requests per chase launch
        self.free = collections.deque(range(slots))
        self.budget = hbm_budget_bytes
        self.in_use = 0
        self.waiting = collections.deque()
        self.active = []
        self.finished = []
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, req, stream=None):
        """Queue a request.  `stream` is the stream whose work produces req.A
        (default: the device's current stream); the solve is ordered after
        everything already issued on it, so A may be computed on the device
        right before submit (e.g. A_{k+1} = A_k + 1e-3 E)."""
        if not req.nbw:
            req.nbw = gb.gb_solve_default_nbw(req.n)
        req._ready = torch.cuda.Event()
        req._ready.record(stream if stream is not None else torch.cuda.current_stream(self.device))
        self.waiting.append(req)

    def _admit(self):
        while self.waiting and self.free:
            req = self.waiting[0]
            need = request_bytes(req.n, req.nev, req.complex, req.nbw)
            if self.in_use + need > self.budget and self.active:
                return            # wait for memory to free up
            self.waiting.popleft()
            slot = self.free.popleft()
            st = self.streams[slot]
            with torch.cuda.stream(st):
                wsb = (gb.gb_solve_workspace_bytes_z if req.complex else gb.gb_solve_workspace_bytes)(
                    req.n, req.nev, req.nbw)
                req._ws = torch.empty(wsb, dtype=torch.uint8, device=self.device)
                req.ev = torch.empty(req.nev, dtype=torch.float64, device=self.device)
                req.Z = torch.empty((req.nev, req.n), dtype=req.A.dtype, device=self.device)
            f = gb.gb_solve_z if req.complex else gb.gb_solve_d
            # the slot stream waits for the writer of A, and A's memory is not
            # handed to another tensor before the slot stream is done with it
            st.wait_event(req._ready)
            req.A.record_stream(st)
            req.start = self.now()
            if self.stage_batching:
                req.status = gb.gb_solve_stage_front(req.complex, req.n, req.nev, req.nbw, req.A, req.n, req._ws, wsb,
                                                     st, check=False)
                req._front = torch.cuda.Event()
                req._front.record(st)
                req._phase = "front"
            else:
                req.status = f(req.n, req.nev, req.nbw, req.A, req.n, req.ev, req.Z, req.n, req._ws, wsb, st, 0,
                               check=False)
                req._end = torch.cuda.Event()
                req._end.record(st)
            req._slot, req._bytes = slot, need
            self.in_use += need
            self.active.append(req)

    def _advance(self):
        """Stage batching: start the backs of every finished chase launch,
        then merge the chases of all requests whose front is done (one kind
        of data per launch) into one launch on a free chase lane."""
        for lane in self.lanes:
            if lane["end"] is not None and lane["end"].query():
                status = gb.gb_trans_ev_query(lane["table"], 256, lane["stream"])
                for req in lane["batch"]:
                    st = self.streams[req._slot]
                    st.wait_event(lane["end"])
                    wsb = (gb.gb_solve_workspace_bytes_z if req.complex else gb.gb_solve_workspace_bytes)(
                        req.n, req.nev, req.nbw)
                    rc = gb.gb_solve_stage_back(req.complex, req.n, req.nev, req.nbw, req.ev, req.Z, req.n, req._ws,
                                                wsb, st, check=False)
                    if req.status == gb.GB_OK:
                        req.status = status if status != gb.GB_OK else rc
                    req._end = torch.cuda.Event()
                    req._end.record(st)
                    req._phase = "back"
                lane["batch"], lane["end"] = [], None
        for req in self.active:
            if req._phase == "front" and req._front.query():
                req._phase = "chase_wait"
        for lane in self.lanes:
            if lane["end"] is not None:
                continue
            ready = [r for r in self.active if r._phase == "chase_wait"]
            if not ready:
                break
            kind = ready[0].complex
            batch = [r for r in ready if r.complex == kind]
            for r in batch:                 # done already; the wait orders their writes before the chase
                lane["stream"].wait_event(r._front)
            rc = gb.gb_solve_stage_chase_batched(kind, [r.n for r in batch], [r.nev for r in batch],
                                                 [r.nbw for r in batch], [r._ws for r in batch], lane["table"],
                                                 self.table_bytes, lane["stream"], check=False)
            for r in batch:
                r._phase = "chase"
                if r.status == gb.GB_OK:
                    r.status = rc
            lane["end"] = torch.cuda.Event()
            lane["end"].record(lane["stream"])
            lane["batch"] = batch
            self.chase_sizes.append(len(batch))

    def _reap(self):
        still = []
        for req in self.active:
            if req._phase in ("front", "chase_wait", "chase"):
                still.append(req)
                continue
            if req._end.query():
                req.done = self.now()
                q = (gb.gb_solve_query_z if req.complex else gb.gb_solve_query)(
                    req._ws, req.n, req.nev, req.nbw, self.streams[req._slot])
                if req.status == gb.GB_OK:
                    req.status = q
                req._ws = None
                self.in_use -= req._bytes
                self.free.append(req._slot)
                self.finished.append(req)
            else:
                still.append(req)
        self.active = still

    def poll(self):
        if self.stage_batching:
            self._advance()
        self._reap()
        self._admit()

    def run(self, requests, idle_sleep=2e-4):
        """Serve `requests` (sorted by arrival time, seconds from now) to
        completion; returns the finished requests in completion order."""
        self.t0 = time.perf_counter()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        while pending or self.waiting or self.active:
            t = self.now()
            while pending and pending[0].arrival <= t:
                self.submit(pending.popleft())
            before = len(self.finished) + len(self.active)
            self.poll()
            if len(self.finished) + len(self.active) == before:
                time.sleep(idle_sleep)
        return self.finished


def latency_summary(finished):
    import numpy as np
    lat = np.array([r.latency() for r in finished])
    span = max(r.done for r in finished) - min(r.arrival for r in finished)
    return {"requests": len(finished), "solves_per_s": len(finished) / span,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3)}
