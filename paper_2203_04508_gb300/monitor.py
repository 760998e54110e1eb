"""Run metrics as JSON lines: one record every `every` steps of a lattice.

A record holds the step count, the FP64 mass audit (M, the drift (M - M0) / M0 and the last
step's Eq. 18 compensation sum dM), the largest speed |v| over the fluid nodes, a flag for
non-finite populations, and the device time per step with the lattice updates per second it
gives (nodes of the whole lattice, solid ones included, per second).  Time is taken with CUDA
events on the lattice's stream around the steps alone; the audit and the speed read-out that
follow each interval are not counted.

A lattice whose populations turn non-finite gives one last record with "nan": true (its mass
audit fails with LBM_EUNSTABLE) and the run stops there.
"""
from __future__ import annotations

import json
import math
from typing import IO, List, Optional, Union

from . import _abi


class Monitor:
    """Steps `lat` and logs a record every `every` steps to `out` (a path, appended to, or an
    open text file), keeping the records in `records`."""

    def __init__(self, lat, out: Optional[Union[str, IO[str]]] = None, every: int = 100):
        if every < 1:
            raise ValueError("every >= 1")
        self.lat = lat
        self.every = int(every)
        self.out = out
        self.records: List[dict] = []
        self.steps = 0
        self.unstable = False

    def _write(self, rec: dict):
        self.records.append(rec)
        if self.out is None:
            return
        line = json.dumps(rec, allow_nan=True) + "\n"
        if isinstance(self.out, str):
            with open(self.out, "a") as fh:
                fh.write(line)
        else:
            self.out.write(line)
            self.out.flush()

    def record(self, ms_per_step: float = float("nan")) -> dict:
        """Audits the current state and logs one record (no steps taken)."""
        lat = self.lat
        rec = {"step": self.steps, "M": None, "drift": None, "dM": None, "max_speed": None, "nan": False,
               "ms_per_step": ms_per_step,
               "mlups": (lat.nx * lat.ny / (ms_per_step * 1e3)) if ms_per_step > 0 else float("nan")}
        try:
            M, M0, dM = lat.mass()
        except _abi.LbmError as e:
            if e.status != _abi.LBM_EUNSTABLE:
                raise
            rec["nan"] = True
            self.unstable = True
            self._write(rec)
            return rec
        v = lat.max_speed()
        rec.update(M=M, drift=(M - M0) / M0, dM=dM, max_speed=v, nan=not math.isfinite(v))
        self.unstable = rec["nan"]
        self._write(rec)
        return rec

    def run(self, steps: int) -> List[dict]:
        """Takes `steps` steps (fewer if the state turns non-finite), logging every `every`; the
        last interval may be shorter.  Returns the records of this call."""
        import torch
        first = len(self.records)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        left = int(steps)
        while left > 0 and not self.unstable:
            n = min(self.every, left)
            start.record(self.lat.stream)
            self.lat.step(n)
            stop.record(self.lat.stream)
            stop.synchronize()
            self.steps += n
            left -= n
            self.record(start.elapsed_time(stop) / n)
        return self.records[first:]
