"""The multi-GPU form is replicas only (the path has no exchange step): the
host logic of bench.py's N > 1 run -- each rank its own seed, the slowest
rank's time by a MAX all-reduce, whole-job totals -- checked with two gloo
ranks on the CPU."""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    t = b.max_over_ranks(1.5 + rank, world)          # the slowest rank: 2.5
    from paper_1612_03310_gb300 import inputs
    w = inputs.workload("c1")
    bunch = b.replica_bunch(w, rank)
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()
    np.save(os.path.join(out, f"r{rank}.npy"), np.array([t, bunch["x"][0], bunch["z"][7]]))


def test_two_gloo_replicas(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    torch.multiprocessing.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2,
                                          join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 2.5
    # rank 0 runs the workload's own bunch, rank 1 another seed
    from paper_1612_03310_gb300 import inputs
    w = inputs.workload("c1")
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    assert r0[1] == P["x"][0] and r0[2] == P["z"][7]
    assert r1[1] != r0[1]


def test_replica_totals():
    b = _bench()
    v, p = b.replica_totals(4, 1000, 50, 2, 10, 0.5)
    assert v == 4 * 1000 * 10 / 0.5
    assert p == 4 * 50 * 2 * 10 / 0.5
    assert b.max_over_ranks(3.0, 1) == 3.0


def test_push_rates():
    """Deposit rates of the bench line: 8 charge and 8 current vertices per
    particle, two int32 shared atomics per charge vertex in the FP32 forms,
    over the particle step's average launch time."""
    b = _bench()
    g = dict(nx=16, ny=16, nz=16)
    r = b.push_rates({"push": (2.0, 4)}, 1000, g, "p32")      # 0.5 ms per launch
    assert r["avg_launch_ms"] == 0.5
    assert r["charge_vertex_deposits_per_s"] == 8 * 1000 / 0.5e-3
    assert r["shared_int32_atomics_per_s"] == 16 * 1000 / 0.5e-3
    assert r["l2_vector_reductions_per_s"] == 8 * 1000 / 0.5e-3
    assert r["achieved_gbs"] == b.algorithmic_bytes("push", g, 1000, "p32") / 0.5e-3 / 1e9
    assert b.push_rates({"push": (2.0, 4)}, 1000, g, "p64")["shared_int32_atomics_per_s"] is None
    assert b.push_rates({}, 1000, g, "p32") is None


def test_algorithmic_bytes_models():
    """The bench's byte models: the potential update moves every grid
    vertex's level and increment (16 B each in FP32, read and written, plus
    the 8 B lo parts of compensated levels read and written) and the 16 B
    of sources of each vertex whose sources it reads; the particle step
    100 B per particle in P32_U64 (the slot's position, state and index in
    and out, key and rank); the re-sort's slot map 16 B."""
    b = _bench()
    g = dict(nx=10, ny=12, nz=14)
    n, interior = 10 * 12 * 14, 8 * 10 * 12
    assert b.algorithmic_bytes("potential_step", g, 0, "p32") == n * 64 + interior * 16
    assert b.algorithmic_bytes("potential_step", g, 0, "p32_u64", 512) == n * 80 + 512 * 16
    assert b.algorithmic_bytes("potential_step", g, 0, "p64", 10 ** 9) == n * 128 + interior * 32
    assert b.minimum_bytes("potential_step", g, 0, "p32_c") == n * 80
    assert b.algorithmic_bytes("push", g, 7, "p32_u64") == 7 * 100
    assert b.algorithmic_bytes("push", g, 7, "p32") == 7 * 76
    assert b.algorithmic_bytes("slot_map", g, 7, "p32") == 7 * 16
