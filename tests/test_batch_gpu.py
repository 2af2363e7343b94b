"""The batched form: members stepped together through the captured graph
give the same results as the same simulations stepped alone, within the
parity tolerances (only the order of floating-point atomic additions may
differ), across membership changes and odd step counts."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

pytestmark = pytest.mark.gpu

UND = inputs.WORKLOADS["c1"]["undulator"]


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


def make(M, seed, shape, n, prec):
    g = dict(inputs.random_grid(seed, *shape), boundary=1)
    P = inputs.random_particles(seed + 1, g, n, u_scale=0.3)
    und = dict(UND, z_ent_lab=0.0)
    return (M.Simulation(g, und, P, precision=prec), M.Simulation(g, und, P, precision=prec))


@pytest.mark.parametrize("prec_name", ["P32", "P64"])
def test_batch_equals_alone(M, prec_name):
    prec = getattr(M, prec_name)
    tol = 1e-5 if prec_name == "P32" else 1e-11
    shapes = [(24, 20, 40), (36, 30, 44), (16, 16, 64)]
    pairs = [make(M, 100 + 7 * k, sh, 2000 + 500 * k, prec) for k, sh in enumerate(shapes)]
    with M.Batch() as b:
        for inb, _ in pairs[:2]:
            b.add(inb)
        b.step(4)            # graph path
        b.add(pairs[2][0])   # membership change: recapture
        for _, alone in pairs[:2]:
            alone.step(4)
        b.step(3)            # odd count: graph + one eager step
        for _, alone in pairs:
            alone.step(3)
        b.remove(pairs[0][0])
        pairs[0][0].step(2)  # stepped alone again after leaving
        pairs[0][1].step(2)
        b.step(2)
        for _, alone in pairs[1:]:
            alone.step(2)
        b.sync()
        assert len(b) == 2
        with pytest.raises(M.MithraError) as e:
            pairs[1][0].step(1)
        assert e.value.status == M.EBUSY
        for inb, alone in pairs:
            assert inb.time()[0] == alone.time()[0]
            for nm in ("Ax", "Ey", "Bz", "phi", "Jx", "rho"):
                assert rel_l2(inb.copy_field(nm), alone.copy_field(nm)) <= tol, nm
            pa, pb = inb.copy_particles(), alone.copy_particles()
            assert np.array_equal(pa["lost"], pb["lost"])
            assert np.abs(pa["z"] - pb["z"]).max() <= tol * 1e-2
    for inb, alone in pairs:
        inb.close()
        alone.close()


def test_seeded_members_equal_alone(M):
    # a Gaussian-beam seed and a plane-wave seed set before joining the batch
    from test_seed_gpu import beam_for, seed_for
    shapes = [(36, 30, 44), (24, 20, 40)]
    pairs = [make(M, 200 + 7 * k, sh, 1500, M.P32) for k, sh in enumerate(shapes)]
    g0 = [dict(inputs.random_grid(200 + 7 * k, *sh), boundary=1) for k, sh in enumerate(shapes)]
    seeds = [beam_for(g0[0], UND["gamma0"]), seed_for(g0[1], UND["gamma0"])]
    for (inb, alone), s in zip(pairs, seeds):
        inb.set_seed(s)
        alone.set_seed(s)
    with M.Batch() as b:
        for inb, _ in pairs:
            b.add(inb)
        b.step(25)           # the pulses reach the total-field planes at step 20
        for _, alone in pairs:
            alone.step(25)
        b.sync()
        for inb, alone in pairs:
            for nm in ("Ax", "Ay", "Ey", "Bx", "rho"):
                assert rel_l2(inb.copy_field(nm), alone.copy_field(nm)) <= 1e-5, nm
            assert np.abs(alone.copy_field("Ay")).max() > 1e-3 * 1.7e-3 * 0.1  # 0.1 A0
    for inb, alone in pairs:
        inb.close()
        alone.close()
