"""GEMMs on host-resident operands with the transfers overlapped.

``HostGemmPipeline`` keeps device copies of a fixed list of problems whose
A, B and C live in (pinned) host memory.  Each ``run()`` copies every A and
B to the device on one stream, runs the Stream-K GEMMs on a second and
copies every C back on a third, so problem i's GEMM overlaps problem i+1's
upload and problem i-1's download.  Events order each problem's steps and
keep a run from overwriting device buffers the previous run still uses.
The GEMMs are ``api.gemm`` calls; this module only schedules copies.
``run(join=False)`` leaves the current stream free, so consecutive runs
overlap too (a run's uploads start as soon as the previous run's GEMM of
the same problem has consumed its inputs); ``join()`` then makes the
current stream wait for everything enqueued.
"""
from __future__ import annotations

import torch

from . import api


class HostGemmPipeline:
    def __init__(self, problems, device=None, config=None, workspace: api.Workspace | None = None):
        """problems: list of (A, B, C) host tensors, A M x K, B K x N (any
        of the layouts ``api.gemm`` accepts), C M x N; pinned memory lets
        the copies run asynchronously."""
        self.device = torch.device(device if device is not None else torch.cuda.current_device())
        self.config = config
        # its own workspace unless given one: its GEMMs run on a stream of
        # their own
        self.ws = workspace or api.Workspace(self.device)
        self.host = list(problems)
        self.dev = []
        for (a, b, c) in self.host:
            mk = lambda t: torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=self.device)  # noqa: E731
            self.dev.append((mk(a), mk(b), mk(c)))
        self.h2d = torch.cuda.Stream(self.device)
        self.comp = torch.cuda.Stream(self.device)
        self.d2h = torch.cuda.Stream(self.device)
        n = len(self.host)
        self._in_ready = [torch.cuda.Event() for _ in range(n)]
        self._done = [None] * n        # GEMM i of the previous run finished (inputs free)
        self._out_read = [None] * n    # C i of the previous run copied back (output free)

    @property
    def bytes_in(self) -> int:
        return sum(a.numel() * a.element_size() + b.numel() * b.element_size() for a, b, _ in self.host)

    @property
    def bytes_out(self) -> int:
        return sum(c.numel() * c.element_size() for _, _, c in self.host)

    def run(self, join: bool = True):
        """Enqueue one pass over all problems after the current stream's
        work; with ``join`` the current stream then waits for the last
        download (else call ``join()`` after the last run)."""
        cur = torch.cuda.current_stream(self.device)
        for s in (self.h2d, self.comp, self.d2h):
            s.wait_stream(cur)
        done, out_read = [], []
        with torch.cuda.stream(self.h2d):
            for i, ((a, b, _), (da, db, _)) in enumerate(zip(self.host, self.dev)):
                if self._done[i] is not None:
                    self.h2d.wait_event(self._done[i])
                da.copy_(a, non_blocking=True)
                db.copy_(b, non_blocking=True)
                self._in_ready[i].record(self.h2d)
        with torch.cuda.stream(self.comp):
            for i, (da, db, dc) in enumerate(self.dev):
                self.comp.wait_event(self._in_ready[i])
                if self._out_read[i] is not None:
                    self.comp.wait_event(self._out_read[i])
                api.gemm(da, db, dc, config=self.config, workspace=self.ws)
                ev = torch.cuda.Event()
                ev.record(self.comp)
                done.append(ev)
        with torch.cuda.stream(self.d2h):
            for i, ((_, _, c), (_, _, dc)) in enumerate(zip(self.host, self.dev)):
                self.d2h.wait_event(done[i])
                c.copy_(dc, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.d2h)
                out_read.append(ev)
        self._done, self._out_read = done, out_read
        if join:
            self.join()

    def join(self):
        """The current stream waits for every upload, GEMM and download
        enqueued so far."""
        cur = torch.cuda.current_stream(self.device)
        cur.wait_stream(self.d2h)
        cur.wait_stream(self.h2d)
        cur.wait_stream(self.comp)
