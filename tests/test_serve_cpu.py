"""Host logic of the continuous-batching server (no GPU): admission by
footprint and slots, first fit in arrival order, ticks that stop at the next
completion, exact step counts per job, latency bookkeeping; with fake
simulations and batch."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import inputs, serve


class FakeSim:
    log = []

    def __init__(self, grid, und, bunch, precision=1):
        self.grid = grid
        self.steps = 0
        self.closed = False

    def set_tuning(self, **kw):
        pass

    def set_power_sampling(self, kp, cap):
        self.cap = cap

    def read_power(self):
        return np.zeros((self.steps, 3))

    def copy_field(self, nm):
        return np.zeros(1)

    def close(self):
        self.closed = True


class FakeBatch:
    def __init__(self):
        self.members = []
        self.ticks = []

    def add(self, s):
        assert len(self.members) < 64
        self.members.append(s)

    def remove(self, s):
        self.members.remove(s)

    def step(self, n):
        self.ticks.append((n, len(self.members)))
        for s in self.members:
            s.steps += n

    def sync(self):
        pass

    def close(self):
        pass


def make_jobs(arrivals, steps, sizes):
    rng = np.random.default_rng(0)
    jobs = []
    for k, (a, st, nx) in enumerate(zip(arrivals, steps, sizes)):
        j = inputs._job(rng, nx, 64, 1000, st, k)
        j["arrival"] = a
        jobs.append(j)
    return jobs


def run(jobs, budget, slots=8, tick=16):
    b = FakeBatch()
    srv = serve.Server(budget, max_slots=slots, tick_steps=tick, clock="steps",
                       sim_factory=FakeSim, batch_factory=lambda: b,
                       footprint_fn=lambda g, n, p: g["nx"] * 1000)
    return srv.run(jobs), b


def test_exact_steps_and_latency():
    jobs = make_jobs([0, 0, 10, 40], [50, 30, 20, 5], [32, 32, 32, 32])
    st, b = run(jobs, budget=10 ** 9)
    assert st["completed"] == 4 and st["unfinished"] == 0
    for js in st["done"]:
        assert js.power.shape[0] == js.spec["steps"]  # retired exactly at its count
        assert js.t_done - js.t_admit == js.spec["steps"]  # no queueing: never waited
    assert all(n <= 16 for n, _ in b.ticks)


def test_admission_by_footprint_first_fit():
    # budget fits one 64-job or two 32-jobs at a time
    jobs = make_jobs([0, 0, 0], [20, 20, 20], [64, 32, 32])
    st, b = run(jobs, budget=64 * 1000)
    assert st["hbm_in_use_peak"] == 64 * 1000 == st["hbm_budget"]
    done = {js.spec["jid"]: js for js in st["done"]}
    assert done[0].t_admit == 0
    assert done[1].t_admit >= done[0].t_done and done[2].t_admit >= done[0].t_done
    assert max(m for _, m in b.ticks) <= 2


def test_slot_limit():
    jobs = make_jobs([0] * 5, [10] * 5, [32] * 5)
    st, b = run(jobs, budget=10 ** 9, slots=2)
    assert max(m for _, m in b.ticks) == 2 and st["completed"] == 5


def test_oversized_job_rejected():
    # a job larger than the whole budget is rejected alone; the others run
    jobs = make_jobs([0, 0], [10, 10], [128, 32])
    st, b = run(jobs, budget=64 * 1000)
    assert st["rejected"] == 1 and st["completed"] == 1
    assert [js.spec["jid"] for js in st["done"]] == [1]
    assert st["not_done"][0].status == "rejected" and "budget" in st["not_done"][0].error


class OOMSim(FakeSim):
    """Creation fails like a device allocation failure for grids of nx 48."""

    def __init__(self, grid, und, bunch, precision=1):
        if grid["nx"] == 48:
            from paper_1612_03310_gb300 import mithra
            raise mithra.MithraError(3, "device allocation failed")
        super().__init__(grid, und, bunch, precision)


def test_allocation_failure_fails_that_job_only():
    jobs = make_jobs([0, 0, 5], [20, 20, 20], [32, 48, 32])
    b = FakeBatch()
    srv = serve.Server(10 ** 9, max_slots=8, tick_steps=16, clock="steps",
                       sim_factory=OOMSim, batch_factory=lambda: b,
                       footprint_fn=lambda g, n, p: g["nx"] * 1000)
    st = srv.run(jobs)
    assert st["completed"] == 2 and st["failed"] == 1
    bad = st["not_done"][0]
    assert bad.spec["jid"] == 1 and "allocation" in bad.error
    assert srv.used == 0                          # nothing leaked


def test_cancelled_job_keeps_its_partial_record():
    jobs = make_jobs([0, 0], [100, 40], [32, 32])
    jobs[0]["cancel_at"] = 25
    st, b = run(jobs, budget=10 ** 9)
    assert st["completed"] == 1 and st["cancelled"] == 1
    c = st["not_done"][0]
    assert c.status == "cancelled" and c.power.shape[0] == 25 and c.t_done == 25
    assert st["done"][0].power.shape[0] == 40


class FailingBatch(FakeBatch):
    """Its third step returns an error, like a device error the library reports."""

    def step(self, n):
        super().step(n)
        if len(self.ticks) == 3:
            from paper_1612_03310_gb300 import mithra
            raise mithra.MithraError(4, "CUDA error in a step")


def test_step_error_fails_the_batch_and_the_server_goes_on():
    jobs = make_jobs([0, 0, 200], [100, 100, 30], [32, 32, 32])
    made = []

    def factory():
        made.append(FailingBatch() if not made else FakeBatch())
        return made[-1]

    srv = serve.Server(10 ** 9, max_slots=8, tick_steps=16, clock="steps",
                       sim_factory=FakeSim, batch_factory=factory,
                       footprint_fn=lambda g, n, p: g["nx"] * 1000)
    st = srv.run(jobs)
    assert st["failed"] == 2 and st["completed"] == 1
    assert all("CUDA error" in js.error for js in st["not_done"])
    assert len(made) == 2 and st["done"][0].spec["jid"] == 2
    assert srv.used == 0


def test_work_budget_limits_the_batch():
    # three jobs of 32 x 32 x 64 cells and 1000 particles (69,536 work units
    # per step each): a budget of two jobs' work admits two at a time, the
    # third waits although memory would hold it; a job larger than the
    # budget runs alone
    jobs = make_jobs([0, 0, 0], [20, 20, 20], [32, 32, 32])
    w = serve.Server.job_work(jobs[0])
    assert w == 32 * 32 * 64 + 4 * 1000
    b = FakeBatch()
    srv = serve.Server(10 ** 9, max_slots=8, tick_steps=16, clock="steps", work_budget=2.5 * w,
                       sim_factory=FakeSim, batch_factory=lambda: b,
                       footprint_fn=lambda g, n, p: 1)
    st = srv.run(jobs)
    assert st["completed"] == 3
    assert max(m for _, m in b.ticks) == 2
    assert st["active_peak"] == 2
    big = make_jobs([0], [10], [64])
    b2 = FakeBatch()
    srv = serve.Server(10 ** 9, max_slots=8, tick_steps=16, clock="steps", work_budget=w,
                       sim_factory=FakeSim, batch_factory=lambda: b2,
                       footprint_fn=lambda g, n, p: 1)
    assert srv.run(big)["completed"] == 1
    # the served rate counts the cells of every job stepped, finished or not
    assert st["served_cell_updates_per_s"] > 0
