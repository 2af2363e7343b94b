"""GPU parity of the seed field (Sec. "Seed Field", total-field/scattered-
field injection) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs
from test_parity_gpu import compare_fields, compare_particles, compare_vertices

pytestmark = pytest.mark.gpu

C0 = 299792458.0


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


def tfsf_mask(g):
    """The vertex planes k = 1 .. 4 around the injection planes k = 2, 3."""
    m = np.zeros((g["nz"], g["ny"], g["nx"]), dtype=bool)
    m[1:5] = True
    return m


def seed_for(g, gamma0, signal="gaussian", pol=(0.0, 1.0), centre=20):
    b0 = np.sqrt(1 - 1 / gamma0 ** 2)
    lam_lab = 16 * g["dz"] / (gamma0 * (1 + b0))
    tau = gamma0 * (1 - b0) * (centre * g["dt"] - 3 * g["dz"] / C0)
    return dict(a0=1e-3, lambda_l=lam_lab, polarization=pol, z0_lab=0.0, offset=C0 * tau,
                variance=0.5 * lam_lab, cep=0.4, direction=1, signal=signal)


@pytest.mark.parametrize("prec", ["P64", "P32", "P32_C"])
@pytest.mark.parametrize("signal", ["gaussian", "flat-top"])
def test_seeded_vacuum_matches_oracle(M, orc, prec, signal):
    g = dict(inputs.random_grid(61, 40, 36, 64), boundary=1)
    und = dict(gamma0=3.0, lambda_u=0.01, K=0.0, z_ent_lab=0.0, length_lab=0.0, fringe=0)
    seed = seed_for(g, 3.0, signal, pol=(0.6, 0.8))
    o = orc.OracleSim(g, und, dict(x=[], y=[], z=[], ux=[], uy=[], uz=[]))
    o.set_seed(dict(seed, gamma0=3.0))
    p = getattr(M, prec)
    with M.Simulation(g, und, None, precision=p) as sim:
        sim.set_seed(seed)
        for steps in (10, 30):
            o.step(steps)
            sim.step(steps)
            sim.sync()
            compare_fields(sim, o, 1e-10 if p == M.P64 else 1e-5,
                           names=["Ax", "Ay", "Az", "phi", "Ex", "Ey", "Bx", "By"])
            compare_vertices(sim, o, 2e-9 if p == M.P64 else 2e-4, tfsf_mask(g),
                             ["Ax", "Ay", "Ex", "Ey", "Bx", "By"])
        assert np.abs(sim.copy_field("Ay")).max() > 0  # the seed is inside


def beam_for(g, gamma0, signal="gaussian"):
    """An astigmatic Gaussian beam off the axis, waists 1.5 and 2 rest-frame
    wavelengths, polarization (0.6, 0.8), focused at the pulse's reference
    position."""
    s = seed_for(g, gamma0, signal, pol=(0.6, 0.8))
    lam_rest = 16 * g["dz"]
    xc = g.get("x0", 0.0) + 0.45 * (g["nx"] - 1) * g["dx"]
    yc = g.get("y0", 0.0) + 0.55 * (g["ny"] - 1) * g["dy"]
    return dict(s, beam="gaussian-beam", x0_lab=xc, y0_lab=yc,
                rayleigh_radius=(1.5 * lam_rest, 2.0 * lam_rest))


@pytest.mark.parametrize("prec", ["P64", "P32", "P32_C"])
@pytest.mark.parametrize("signal", ["gaussian", "neumann"])
@pytest.mark.parametrize("stencil", [0, 1])
def test_gaussian_beam_seed_vacuum_matches_oracle(M, orc, prec, signal, stencil):
    # ragged 16 x 16 column tiles (interior 38 x 34), both stencils
    g = dict(inputs.random_grid(62, 40, 36, 64, courant=0.95 if stencil == 0 else 0.5,
                                stencil=stencil), boundary=1)
    und = dict(gamma0=3.0, lambda_u=0.01, K=0.0, z_ent_lab=0.0, length_lab=0.0, fringe=0)
    seed = beam_for(g, 3.0, signal)
    o = orc.OracleSim(g, und, dict(x=[], y=[], z=[], ux=[], uy=[], uz=[]))
    o.set_seed(dict(seed, gamma0=3.0))
    p = getattr(M, prec)
    with M.Simulation(g, und, None, precision=p) as sim:
        sim.set_seed(seed)
        for steps in (10, 30):
            o.step(steps)
            sim.step(steps)
            sim.sync()
            compare_fields(sim, o, 1e-10 if p == M.P64 else 1e-5,
                           names=["Ax", "Ay", "Az", "phi", "Ex", "Ey", "Bx", "By"])
            compare_vertices(sim, o, 2e-9 if p == M.P64 else 2e-4, tfsf_mask(g),
                             ["Ax", "Ay", "Ex", "Ey", "Bx", "By"])
        Ay = sim.copy_field("Ay")
        assert np.abs(Ay).max() > 0.1 * seed["a0"] * 9.109e-31 * C0 / 1.602e-19
        # not uniform across the planes: the beam's waist is inside the grid
        col = np.abs(Ay[10]).max(axis=0)
        assert col.min() < 0.5 * col.max()


@pytest.mark.parametrize("prec", ["P64", "P32"])
@pytest.mark.parametrize("beam", ["plane-wave", "gaussian-beam"])
def test_seeded_c1_matches_oracle(M, orc, prec, beam):
    w = inputs.workload("c1")
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    # a seed at the resonant lab wavelength lambda_u (1 + K^2/2) / (2 gamma^2)
    lam_r = und["lambda_u"] * (1 + und["K"] ** 2 / 2) / (2 * 10.0 ** 2)
    seed = dict(a0=2e-4, lambda_l=lam_r, polarization=(1.0, 0.0), z0_lab=0.0,
                offset=-5e-3, variance=40 * lam_r, cep=0.0, direction=1, signal="flat-top",
                beam=beam)
    if beam == "gaussian-beam":
        # focused on the bunch axis, a waist of a third of the transverse grid
        waist = 0.33 * (g["nx"] - 1) * g["dx"]
        seed.update(x0_lab=g["x0"] + 0.5 * (g["nx"] - 1) * g["dx"],
                    y0_lab=g["y0"] + 0.5 * (g["ny"] - 1) * g["dy"], z0_lab=0.02,
                    rayleigh_radius=(waist, 1.2 * waist))
    kp = g["nz"] - 8
    o = orc.OracleSim(g, und, P)
    o.set_seed(dict(seed, gamma0=und["gamma0"]))
    p = getattr(M, prec)
    with M.Simulation(g, und, P, precision=p) as sim:
        sim.set_seed(seed)
        sim.set_power_sampling(kp, w["steps"])
        o.step(w["steps"], power_plane=kp)
        sim.step(w["steps"])
        sim.sync()
        compare_fields(sim, o, 1e-9 if p == M.P64 else 1e-4)
        rec = sim.read_power()
        po = np.array([s.p_lab for s in o.power])
        scale = np.abs(po).max()
        assert scale > 0
        assert np.abs(rec[:, 0] - po).max() <= (1e-9 if p == M.P64 else 1e-3) * scale
        compare_particles(sim, o, 1e-8 if p == M.P64 else 1e-3, 1e-9 if p == M.P64 else 1e-3)


def test_seed_argument_checks(M):
    g = dict(inputs.random_grid(0, 16, 16, 16), boundary=1)
    with M.Simulation(g, None, None) as sim:
        good = seed_for(g, 3.0)
        sim.set_seed(good)
        sim.set_seed(None)
        beam = dict(good, beam="gaussian-beam", rayleigh_radius=(1e-4, 2e-4))
        sim.set_seed(beam)
        sim.set_seed(None)
        for bad in (dict(lambda_l=0.0), dict(variance=-1.0), dict(direction=0),
                    dict(polarization=(0.0, 0.0)), dict(signal="gaussian", a0=float("nan")),
                    dict(beam="gaussian-beam"), dict(beam="gaussian-beam",
                                                     rayleigh_radius=(1e-4, -1.0)),
                    dict(beam="gaussian-beam", rayleigh_radius=(1e-4, 1e-4),
                         x0_lab=float("inf"))):
            with pytest.raises(M.MithraError) as e:
                sim.set_seed(dict(good, **bad))
            assert e.value.status == M.EINVAL
    # the optical undulator is a plane wave
    und = dict(type="optical", gamma0=3.0, a0=0.1, lambda_l=1e-6, offset=0.0, variance=1e-6,
               beam="gaussian-beam", rayleigh_radius=(1e-4, 1e-4))
    with pytest.raises(M.MithraError) as e:
        M.Simulation(g, und, None).close()
    assert e.value.status == M.EINVAL
