"""Per-iteration log of Algorithm 1 as JSON lines.

Each step's scalar block (loss, eta, line-search halvings, iteration count,
status) is copied asynchronously into a pinned host ring after the step, so
logging adds no synchronisation to the step loop; records are written when
the ring is flushed (every `flush_every` steps and on close).  Optionally
the relative error against a reference volume is recorded too (one extra
reduction kernel and a device scalar per step).
"""
from __future__ import annotations

import json
import time

import torch

from . import native as N


class StepLog:
    def __init__(self, path: str, handle=None, geom=None, reference=None, flush_every=64):
        self.f = open(path, "a")
        self.h, self.geom, self.ref = handle, geom, reference
        self.n = flush_every
        self.ring = torch.zeros((flush_every, N.CS_NSCALARS), dtype=torch.float64).pin_memory()
        self.err = None
        if reference is not None:
            self.err = torch.zeros(flush_every, dtype=torch.float64, device=reference.device)
        self.times = [0.0] * flush_every
        self.events = [torch.cuda.Event() for _ in range(flush_every)]
        self.fill = 0

    def record(self, state, stream=None):
        """Call after a step was enqueued on `stream` for `state`."""
        s = stream if stream is not None else torch.cuda.current_stream()
        i = self.fill
        with torch.cuda.stream(s):
            self.ring[i].copy_(state.scalars, non_blocking=True)
            if self.ref is not None:
                self.h.rel_err(self.geom, state.v, self.ref, out=self.err[i:i + 1].view(()),
                               stream=s)
        self.events[i].record(s)
        self.times[i] = time.time()
        self.fill += 1
        if self.fill == self.n:
            self.flush()

    def flush(self):
        if self.fill == 0:
            return
        self.events[self.fill - 1].synchronize()
        errs = self.err[: self.fill].cpu().tolist() if self.ref is not None else None
        for i in range(self.fill):
            r = self.ring[i].tolist()
            rec = {"k": int(r[N.CS_S_K]), "loss": r[N.CS_S_LOSS], "eta": r[N.CS_S_ETA],
                   "halvings": int(r[N.CS_S_HALVINGS]), "G": r[N.CS_S_G], "Q": r[N.CS_S_Q],
                   "status": int(r[N.CS_S_STATUS]), "host_time": self.times[i]}
            if errs is not None:
                rec["rel_err"] = errs[i]
            self.f.write(json.dumps(rec) + "\n")
        self.f.flush()
        self.fill = 0

    def close(self):
        self.flush()
        self.f.close()
