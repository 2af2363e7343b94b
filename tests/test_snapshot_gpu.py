"""Checkpoint and resume: n steps, a snapshot restored into a fresh
simulation of the same shape, n more steps equal 2n steps of one simulation
(up to the order of the floating-point current atomics), and a snapshot of
another shape is refused without changing anything."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

pytestmark = pytest.mark.gpu

UND = inputs.WORKLOADS["c1"]["undulator"]
FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Ax", "Ay", "Az", "phi", "Jx", "rho",
          "Ax_prev", "phi_prev"]


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


@pytest.mark.parametrize("prec_name", ["P64", "P32", "P32_C", "P32_U64"])
def test_restore_continues_the_run(M, prec_name):
    prec = getattr(M, prec_name)
    tol = 1e-12 if prec == M.P64 else 1e-5
    g = dict(inputs.random_grid(21, 30, 26, 40), boundary=1)
    P = inputs.random_particles(22, g, 3000, u_scale=0.3)
    und = dict(UND, z_ent_lab=0.0)
    with M.Simulation(g, und, P, precision=prec) as a, \
            M.Simulation(g, und, P, precision=prec) as b:
        a.step(7)                                   # odd: the other ping-pong parity
        snap = a.snapshot()
        a.step(6)
        b.step(2)                                   # different state, replaced below
        b.restore(snap)
        assert b.time() == (7, pytest.approx(7 * g["dt"]))
        b.step(6)
        assert a.time()[0] == b.time()[0] == 13
        for nm in FIELDS:
            assert rel_l2(b.copy_field(nm), a.copy_field(nm)) <= tol, nm
        pa, pb = a.copy_particles(), b.copy_particles()
        assert np.array_equal(pa["lost"], pb["lost"])
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            assert np.allclose(pb[k], pa[k], rtol=tol, atol=1e-30), k


def test_restore_refuses_another_shape(M):
    g1 = dict(inputs.random_grid(23, 16, 16, 24), boundary=1)
    g2 = dict(inputs.random_grid(23, 16, 16, 32), boundary=1)
    P = inputs.random_particles(24, g1, 500, u_scale=0.1)
    und = dict(UND, z_ent_lab=0.0)
    with M.Simulation(g1, und, P, precision=M.P32) as a, \
            M.Simulation(g2, und, P, precision=M.P32) as b, \
            M.Simulation(g1, und, P, precision=M.P64) as c:
        a.step(3)
        snap = a.snapshot()
        b.step(2)
        before = b.copy_field("Ax")
        for sim in (b, c):
            with pytest.raises(M.MithraError):
                sim.restore(snap)
        assert b.time()[0] == 2
        assert np.array_equal(b.copy_field("Ax"), before)
        bad = snap.copy()
        bad[0] ^= 0xff                              # not a snapshot
        with pytest.raises(M.MithraError):
            a.restore(bad)
