"""The batched form: members stepped together through the captured graph
give the same results as the same simulations stepped alone, within the
parity tolerances (only the order of floating-point atomic additions may
differ), across membership changes and odd step counts, in the fused form
(one launch per phase over a work list spanning all members) and in the
per-member form; members the fused kernels do not cover (a seed, mixed
precision forms) take the per-member form."""
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


def make(M, seed, shape, n, prec, boundary=1):
    g = dict(inputs.random_grid(seed, *shape), boundary=boundary)
    P = inputs.random_particles(seed + 1, g, n, u_scale=0.3)
    und = dict(UND, z_ent_lab=0.0)
    return (M.Simulation(g, und, P, precision=prec), M.Simulation(g, und, P, precision=prec))


@pytest.mark.parametrize("prec_name,fused,boundary", [
    ("P32", True, 1), ("P32", False, 1), ("P64", True, 1), ("P64", False, 1),
    ("P32_U64", True, 1), ("P32_C", True, 2), ("P32", True, 2)])
def test_batch_equals_alone(M, prec_name, fused, boundary):
    prec = getattr(M, prec_name)
    tol = 1e-11 if prec_name == "P64" else 1e-5
    shapes = [(24, 20, 40), (36, 30, 44), (16, 16, 64)]
    pairs = [make(M, 100 + 7 * k, sh, 2000 + 500 * k, prec, boundary)
             for k, sh in enumerate(shapes)]
    for k, (inb, alone) in enumerate(pairs):  # power recorded in and out of the batch
        kp = shapes[k][2] - 6
        inb.set_power_sampling(kp, 20)
        alone.set_power_sampling(kp, 20)
    with M.Batch() as b:
        b.set_mode(fused)
        for inb, _ in pairs[:2]:
            b.add(inb)
        b.step(4)            # graph path
        assert b.fused() == fused
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
            ra, rb = inb.read_power(), alone.read_power()
            assert ra.shape == rb.shape and ra.shape[0] > 0
            assert np.abs(ra - rb).max() <= max(tol, 1e-4 if prec_name != "P64" else 0) * \
                np.abs(rb).max()
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
        assert not b.fused()  # seeded members take the per-member form
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


def test_mixed_forms_take_the_per_member_graph(M):
    a = make(M, 300, (24, 20, 40), 1000, M.P32)
    c = make(M, 307, (20, 24, 36), 1000, M.P64)
    with M.Batch() as b:
        b.add(a[0])
        b.add(c[0])
        b.step(2)
        assert not b.fused()
        a[1].step(2)
        c[1].step(2)
        b.sync()
        for inb, alone, tol in ((a[0], a[1], 1e-5), (c[0], c[1], 1e-11)):
            assert rel_l2(inb.copy_field("Ex"), alone.copy_field("Ex")) <= tol
    for x in a + c:
        x.close()


def test_many_uneven_members_fused(M):
    # 12 members of uneven grids and particle counts in one fused batch,
    # 6 steps, each equal to its lone run
    rng = np.random.default_rng(5)
    pairs = []
    for k in range(12):
        sh = (int(rng.integers(12, 40)), int(rng.integers(12, 40)), int(rng.integers(16, 64)))
        pairs.append(make(M, 400 + 3 * k, sh, int(rng.integers(0, 3000)), M.P32_U64))
    with M.Batch() as b:
        for inb, _ in pairs:
            b.add(inb)
        b.step(6)
        assert b.fused()
        for _, alone in pairs:
            alone.step(6)
        b.sync()
        for inb, alone in pairs:
            for nm in ("Ax", "Ez", "By", "rho", "Jz"):
                assert rel_l2(inb.copy_field(nm), alone.copy_field(nm)) <= 1e-5, nm
            assert inb.time()[0] == alone.time()[0] == 6
    for inb, alone in pairs:
        inb.close()
        alone.close()
