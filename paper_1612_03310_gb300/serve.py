"""Continuous-batching job server for FEL design sweeps.

Jobs (grid, undulator, bunch, step count, arrival time) arrive over time.
The server keeps every admitted job's fields and particles resident on the
device and advances all of them together through one mithra batch (one
captured CUDA graph per pair of steps: the fused form, one launch per phase
for all jobs, while the jobs are small, one launch sequence per job
otherwise, mithra_batch_set_mode).  Jobs run with the library's default
launch choices (the register z-marching update and the tiled particle step,
the autotuner's choice on every grid it has timed) unless the server is given
tuning.  Admission is first come, first served while the job's device
footprint (mithra_footprint) fits the HBM budget and the batch's work per
step (cell updates plus 4 per particle push, over the jobs in it) stays
within the work budget: past the amount of work that keeps the GPU busy, a
larger batch only makes every job in it slower, so the work budget (default
1e7, a few c5 jobs, about 0.4 ms of batched step on GB300) holds the batch
near that amount while memory bounds what may wait resident (measured on
the c5 stream at 20 jobs/s for 20 s: budgets of 1e7, 4e7 and 1.5e8 finished
114, 110 and 67 jobs with p50 latencies of 3.3, 5.0 and 9.8 s, the GPU
serving 30-32 G cell updates/s in each).  The slot cap is a guard
(1024 by default).  A job that does not fit waits, later smaller jobs may go
ahead of it (first fit); a job larger than the work budget is admitted alone
into an empty batch.  Every membership change costs one graph capture at the
next tick; the batch's capture count and time are reported, and so are the
cell updates done for all jobs per second of wall time (the GPU's served
rate) beside those of the completed jobs.  Each tick advances the batch by the steps
until the next member finishes (at most tick_steps), so jobs retire exactly
at their step count; a finished job's power record is read back, its memory
freed, and its latency (arrival to completion) recorded.

Time is the wall clock (clock="wall", arrivals in seconds) or the server's
own step counter (clock="steps", arrivals in steps), the latter for
reproducible schedules in tests.

Failures stay with the jobs they hit: a job whose footprint exceeds the
whole budget is rejected on arrival; a job whose simulation cannot be
created (an allocation failure, an invalid grid) fails at admission; a job
with "cancel_at" (server time) is cancelled then, its partial power record
kept; a step that returns an error fails the jobs in the batch and the
server goes on with a fresh batch.  None of this touches the GPU beyond the
library's own error returns.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import inputs, mithra


@dataclass
class JobState:
    spec: dict
    arrival: float
    footprint: int = 0
    sim: object = None
    remaining: int = 0
    t_admit: float | None = None
    t_done: float | None = None
    power: np.ndarray | None = None
    fields: dict = field(default_factory=dict)
    status: str = "pending"  # pending, active, done, rejected, failed, cancelled
    error: str | None = None


class Server:
    def __init__(self, hbm_budget: int, max_slots: int = 1024, tick_steps: int = 64,
                 work_budget: float | None = 1.0e7,
                 precision: int = mithra.P32, tuning: dict | None = None,
                 keep_fields: tuple = (), power_plane_from_top: int = 8,
                 clock: str = "wall", sim_factory=None, batch_factory=None,
                 footprint_fn=None):
        self.budget = int(hbm_budget)
        self.max_slots = int(max_slots)
        self.tick_steps = int(tick_steps)
        self.precision = precision
        self.tuning = None if tuning is None else dict(tuning)
        self.keep_fields = tuple(keep_fields)
        self.kp_top = int(power_plane_from_top)
        self.clock = clock
        self._sim = sim_factory or mithra.Simulation
        self._batch = batch_factory or mithra.Batch
        self._fp = footprint_fn or mithra.footprint
        self.work_budget = work_budget
        self.work = 0.0        # work per step of the jobs in the batch
        self.work_done = 0.0   # cell updates done for all jobs
        self.used = 0
        self.used_peak = 0
        self.active_peak = 0
        self.capture = dict(captures=0, fused_captures=0, capture_seconds=0.0)
        self.steps_done = 0
        self.queue_depth: list[tuple[float, int]] = []

    # -- helpers --------------------------------------------------------
    @staticmethod
    def job_work(spec: dict) -> float:
        """Work of one step of a job in cell-update equivalents (a particle
        push counted as 4 cell updates, their cost ratio on GB300)."""
        g = spec["grid"]
        return float(g["nx"] * g["ny"] * g["nz"]) + 4.0 * float(spec["bunch_spec"]["n"])

    def _fits_work(self, js: JobState, n_active: int) -> bool:
        if self.work_budget is None or n_active == 0:
            return True
        return self.work + self.job_work(js.spec) <= self.work_budget

    def _now(self, t0: float) -> float:
        return (time.perf_counter() - t0) if self.clock == "wall" else float(self.steps_done)

    def _admit(self, js: JobState, batch, now: float):
        spec = js.spec
        g = dict(spec["grid"], boundary=1)
        bunch = inputs.make_bunch(spec["bunch_spec"], spec["seed"])
        sim = self._sim(g, spec["undulator"], bunch, precision=self.precision)
        try:
            if self.tuning:
                sim.set_tuning(**self.tuning)
            sim.set_power_sampling(g["nz"] - self.kp_top, spec["steps"])
            batch.add(sim)
        except Exception:
            sim.close()
            raise
        js.sim = sim
        js.remaining = spec["steps"]
        js.t_admit = now
        self.used += js.footprint
        self.work += self.job_work(spec)
        self.used_peak = max(self.used_peak, self.used)

    def _retire(self, js: JobState, batch, now: float, status: str = "done"):
        js.power = js.sim.read_power()
        for nm in self.keep_fields:
            js.fields[nm] = js.sim.copy_field(nm)
        batch.remove(js.sim)
        js.sim.close()
        js.sim = None
        js.t_done = now
        js.status = status
        self.used -= js.footprint
        self.work -= self.job_work(js.spec)

    def _drop(self, js: JobState, batch, now: float, error: str):
        """A job whose step failed: its simulation is closed, its memory freed."""
        try:
            batch.remove(js.sim)
        except Exception:
            pass
        try:
            js.sim.close()
        except Exception:
            pass
        js.sim = None
        js.t_done = now
        js.status = "failed"
        js.error = error
        self.used -= js.footprint
        self.work -= self.job_work(js.spec)

    # -- main loop ---------------------------------------------------------
    def run(self, jobs: list[dict], time_limit: float | None = None) -> dict:
        pending = deque(sorted((JobState(j, float(j.get("arrival", 0.0))) for j in jobs),
                               key=lambda s: s.arrival))
        failed: list[JobState] = []
        for js in list(pending):
            js.footprint = int(self._fp(dict(js.spec["grid"], boundary=1),
                                        js.spec["bunch_spec"]["n"], self.precision))
            if js.footprint > self.budget:
                js.status = "rejected"
                js.error = f"needs {js.footprint} B of a {self.budget} B budget"
                pending.remove(js)
                failed.append(js)
        queue: list[JobState] = []
        active: list[JobState] = []
        done: list[JobState] = []
        batch = self._batch()
        t0 = time.perf_counter()
        try:
            while pending or queue or active:
                now = self._now(t0)
                if time_limit is not None and now > time_limit:
                    break
                while pending and pending[0].arrival <= now:
                    queue.append(pending.popleft())
                for js in list(queue):  # first fit in arrival order
                    if len(active) >= self.max_slots:
                        break
                    if self.used + js.footprint <= self.budget and \
                            self._fits_work(js, len(active)):
                        queue.remove(js)
                        try:
                            self._admit(js, batch, now)
                        except mithra.MithraError as e:  # e.g. out of device memory
                            if js.sim is not None:
                                js.sim.close()
                            js.sim = None
                            js.status, js.error, js.t_done = "failed", str(e), now
                            failed.append(js)
                            continue
                        js.status = "active"
                        active.append(js)
                        self.active_peak = max(self.active_peak, len(active))
                for js in [a for a in active
                           if a.spec.get("cancel_at") is not None and a.spec["cancel_at"] <= now]:
                    self._retire(js, batch, now, status="cancelled")
                    active.remove(js)
                    failed.append(js)
                self.queue_depth.append((now, len(queue)))
                if not active:
                    if self.clock == "steps":
                        self.steps_done = int(np.ceil(pending[0].arrival)) if pending else \
                            self.steps_done
                    elif pending:
                        time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                    continue
                tick = min([self.tick_steps] + [js.remaining for js in active])
                if self.clock == "steps" and pending:
                    # stop at the next arrival so that it is admitted on time
                    tick = max(1, min(tick, int(np.ceil(pending[0].arrival)) - self.steps_done))
                if self.clock == "steps":
                    # stop at the next cancellation as well
                    cut = [int(np.ceil(a.spec["cancel_at"])) - self.steps_done for a in active
                           if a.spec.get("cancel_at") is not None]
                    if cut:
                        tick = max(1, min([tick] + cut))
                try:
                    batch.step(tick)
                    batch.sync()
                except mithra.MithraError as e:
                    # the batch's state is unknown: fail its jobs, start afresh
                    now = self._now(t0)
                    for js in active:
                        self._drop(js, batch, now, str(e))
                        failed.append(js)
                    active.clear()
                    self._add_capture_stats(batch)
                    batch.close()
                    batch = self._batch()
                    continue
                self.steps_done += tick
                now = self._now(t0)
                for js in active:
                    js.remaining -= tick
                    g = js.spec["grid"]
                    self.work_done += float(g["nx"] * g["ny"] * g["nz"]) * tick
                for js in [a for a in active if a.remaining == 0]:
                    self._retire(js, batch, now)
                    active.remove(js)
                    done.append(js)
        finally:
            for js in active:
                try:
                    batch.remove(js.sim)
                    js.sim.close()
                except Exception:
                    pass
            self._add_capture_stats(batch)
            batch.close()
        wall = time.perf_counter() - t0
        return self.stats(done, queue + active + list(pending), wall, failed)

    def _add_capture_stats(self, batch):
        st = getattr(batch, "stats", None)
        if st is None:
            return
        try:
            d = st()
        except Exception:
            return
        for k in self.capture:
            self.capture[k] += d.get(k, 0)

    def stats(self, done: list[JobState], left: list[JobState], wall: float,
              failed: list[JobState] | None = None) -> dict:
        failed = failed or []
        lat = np.array([js.t_done - js.arrival for js in done]) if done else np.array([])
        cells = sum(js.spec["grid"]["nx"] * js.spec["grid"]["ny"] * js.spec["grid"]["nz"] *
                    js.spec["steps"] for js in done)
        return dict(
            completed=len(done), unfinished=len(left), wall_s=wall,
            jobs_per_hour=3600.0 * len(done) / wall if wall > 0 else 0.0,
            p50_s=float(np.percentile(lat, 50)) if lat.size else None,
            p99_s=float(np.percentile(lat, 99)) if lat.size else None,
            cell_updates_per_s=cells / wall if wall > 0 else 0.0,
            served_cell_updates_per_s=self.work_done / wall if wall > 0 else 0.0,
            work_budget=self.work_budget,
            max_queue=max((q for _, q in self.queue_depth), default=0),
            hbm_in_use_peak=self.used_peak, hbm_budget=self.budget,
            active_peak=self.active_peak, graph_captures=self.capture["captures"],
            fused_captures=self.capture["fused_captures"],
            capture_seconds=self.capture["capture_seconds"],
            capture_ms_mean=(1e3 * self.capture["capture_seconds"] /
                             max(1, self.capture["captures"])),
            rejected=sum(js.status == "rejected" for js in failed),
            failed=sum(js.status == "failed" for js in failed),
            cancelled=sum(js.status == "cancelled" for js in failed),
            done=done, not_done=failed)
