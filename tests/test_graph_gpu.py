"""Runs of four or more steps replay a captured run of four steps (CUDA
graph), in which each step's re-sort but the last runs on a side stream
beside the next step's potential update; single steps launch the kernels
one by one, the re-sort at the end of its own step.  Both give the same
state (within the order of floating-point atomic additions), from either
parity of the level ping-pong, and a change of the diagnostics or launch
choices between runs reaches the replayed steps."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

pytestmark = pytest.mark.gpu

UND = inputs.WORKLOADS["c1"]["undulator"]
FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Ax", "phi", "Jx", "rho"]


@pytest.fixture(scope="module")
def M():
    build_lib.build()
    from paper_1612_03310_gb300 import mithra
    try:
        mithra.Simulation(dict(inputs.random_grid(0, 4, 4, 4), boundary=1), None, None).close()
    except mithra.MithraError as e:
        if e.status == mithra.ENODEV:
            pytest.skip("no GB300 device")
        raise
    return mithra


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb else float(np.linalg.norm(a))


OPTICAL = dict(type="optical", gamma0=UND["gamma0"], a0=UND["K"], lambda_l=2 * UND["lambda_u"],
               polarization=(0.6, 0.8), z0_lab=0.0, offset=0.0, variance=2 * UND["lambda_u"],
               cep=0.3, direction=-1, signal="gaussian")


def pair(M, prec, seed=3, n_sub=1, und=None, boundary=1):
    g = dict(inputs.random_grid(seed, 30, 26, 40, n_sub=n_sub), boundary=boundary)
    P = inputs.random_particles(seed + 1, g, 3000, u_scale=0.3)
    und = und or dict(UND, z_ent_lab=0.0)
    return (M.Simulation(g, und, P, precision=prec), M.Simulation(g, und, P, precision=prec))


@pytest.mark.parametrize("prec_name", ["P32", "P64"])
def test_replayed_steps_equal_single_steps(M, prec_name):
    prec = getattr(M, prec_name)
    tol = 1e-12 if prec == M.P64 else 1e-5
    a, b = pair(M, prec)
    with a, b:
        a.set_power_sampling(20, 64)
        b.set_power_sampling(20, 64)
        # 1 eager step, then graph runs from the other parity, odd and even
        for n in (1, 7, 4, 5):
            a.step(n)
            for _ in range(n):
                b.step(1)
        assert a.time()[0] == b.time()[0] == 17
        for nm in FIELDS:
            assert rel_l2(a.copy_field(nm), b.copy_field(nm)) <= tol, nm
        pa, pb = a.read_power(), b.read_power()
        assert pa.shape == pb.shape == (17, 3)
        assert np.allclose(pa, pb, rtol=tol, atol=1e-30)
        qa, qb = a.copy_particles(), b.copy_particles()
        assert np.array_equal(qa["lost"], qb["lost"])


def test_settings_changed_between_runs_reach_the_replay(M):
    a, b = pair(M, M.P32, seed=7)
    with a, b:
        a.step(6)                       # captures and replays
        b.step(6)
        a.set_power_sampling(20, 100)   # must drop the captured steps
        a.set_bunch_sampling(1.0e3, 2, 10)
        a.step(6)
        assert a.read_power().shape == (6, 3)
        assert list(a.read_bunch()[:, 0]) == [8, 10, 12]
        a.set_tuning(push_variant=0)    # another particle-step form
        b.set_tuning(push_variant=0)
        a.step(5)
        for _ in range(11):
            b.step(1)
        assert a.time()[0] == b.time()[0] == 17
        for nm in ("Ex", "Bz", "rho"):
            assert rel_l2(a.copy_field(nm), b.copy_field(nm)) <= 1e-5, nm


@pytest.mark.parametrize("prec_name,n_sub,optical,boundary", [
    ("P32_C", 3, False, 1), ("P32_U64", 2, True, 2), ("P64", 3, True, 2)])
def test_replay_with_sub_steps_and_both_undulators(M, prec_name, n_sub, optical, boundary):
    # sub-cycled particle steps, the compensated levels, the optical
    # undulator's time-dependent field and both Mur orders in the replay
    prec = getattr(M, prec_name)
    tol = 1e-12 if prec == M.P64 else 1e-5
    a, b = pair(M, prec, seed=11, n_sub=n_sub, und=OPTICAL if optical else None,
                boundary=boundary)
    with a, b:
        for n in (2, 5, 6):
            a.step(n)
            for _ in range(n):
                b.step(1)
        assert a.time()[0] == b.time()[0] == 13
        for nm in FIELDS:
            assert rel_l2(a.copy_field(nm), b.copy_field(nm)) <= tol, nm
        qa, qb = a.copy_particles(), b.copy_particles()
        assert np.array_equal(qa["lost"], qb["lost"])
        for k in ("ux", "uy", "uz"):
            assert rel_l2(qa[k], qb[k]) <= tol, k


def test_profiled_steps_between_replays(M):
    """Per-kernel timing keeps every kernel of a step on the simulation's
    stream and each step's re-sort at its own end; runs replayed before and
    after it (their re-sorts beside the next update) give the state of
    single steps, and the timed scopes count one launch per step."""
    a, b = pair(M, M.P32, seed=5)
    with a, b:
        a.step(4)            # one replay
        a.profile(True)
        a.step(6)            # one by one, timed
        kt = a.kernel_times()
        a.profile(False)
        a.step(9)            # two replays and one single step
        for _ in range(19):
            b.step(1)
        assert a.time()[0] == b.time()[0] == 19
        for k in ("potential_step", "push", "scan_counts", "slot_map"):
            assert kt[k][1] == 6, (k, kt[k])
            assert kt[k][0] > 0.0, (k, kt[k])
        for nm in FIELDS:
            assert rel_l2(a.copy_field(nm), b.copy_field(nm)) <= 1e-5, nm
        qa, qb = a.copy_particles(), b.copy_particles()
        assert np.array_equal(qa["lost"], qb["lost"])
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            assert rel_l2(qa[k], qb[k]) <= 1e-5, k
