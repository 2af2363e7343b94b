"""Oracle pins of the optical undulator (input group UNDULATOR with
undulator-type optical, beam-type plane-wave, the signal types of the FIELD
section), against closed forms:

  - in the rest frame the field is a plane wave along z: E and B transverse,
    B = (d/c) z x E for a wave travelling along d z;
  - at a fixed rest-frame point the carrier has the Doppler-shifted period
    lambda0 / (c gamma0 (1 - d beta0)) and, on the flat top, the amplitude
    gamma0 (1 - d beta0) A0 w0 with A0 = a0 m_e c / e, w0 = 2 pi c / lambda0;
  - the Gaussian envelope's intensity falls to one half at a lab retarded
    time tau_v / 2 from its centre (tau_v is the intensity FWHM), the
    hyperbolic secant's amplitude to 1/cosh(1) at tau_v; the flat top keeps
    the full amplitude after its rise;
  - the paper's benchmark: an electron in an optical undulator with a0 = K and
    lambda0 = 2 lambda_u oscillates like one in the static undulator -- the
    same maximum |u_x| = K, and a frequency higher by (1 + beta0)/(2 beta0).
"""
import numpy as np
import pytest

from test_oracle_pic import C0, _push, golden

ME = 9.1093837015e-31
QE = 1.602176634e-19


def _optical(g0, a0, lam, direction=-1, pol=(0.0, 1.0), signal="flat-top", offset=None,
             variance=None, cep=0.0):
    return dict(type="optical", gamma0=g0, a0=a0, lambda_l=lam, polarization=pol, z0_lab=0.0,
                offset=5 * lam if offset is None else offset,
                variance=2 * lam if variance is None else variance, cep=cep,
                direction=direction, signal=signal)


@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("pol", [(0.0, 1.0), (1.0, 0.0), (0.6, 0.8)])
def test_optical_plane_wave_structure(orc, direction, pol):
    g0 = 20.0
    u = _optical(g0, 1.3, 1.0e-6, direction, pol)
    rng = np.random.default_rng(3)
    for _ in range(50):
        z = rng.uniform(-1e-4, 1e-4)
        t = rng.uniform(2e-12, 4e-12) if direction < 0 else rng.uniform(2e-12, 4e-12)
        E, B = orc.undulator_field(u, 0.0, z, t)
        scale = np.abs(E).max() + 1e-30
        assert abs(E[2]) < 1e-12 * scale and abs(B[2]) * C0 < 1e-12 * scale
        # B = (d/c) z x E, z x E = (-E_y, E_x, 0)
        np.testing.assert_allclose(B[:2] * C0, direction * np.array([-E[1], E[0]]),
                                   atol=1e-12 * scale)
        # E along the polarization
        assert abs(E[0] * pol[1] - E[1] * pol[0]) < 1e-12 * scale


@pytest.mark.parametrize("direction", [-1, 1])
def test_optical_doppler_period_and_amplitude(orc, direction):
    g0 = 8.0
    b0 = np.sqrt(1 - 1 / g0 ** 2)
    lam, a0 = 2.0e-6, 0.7
    u = _optical(g0, a0, lam, direction, (0.0, 1.0), offset=-50 * lam)  # flat top everywhere
    T = lam / (C0 * g0 * (1 - direction * b0))
    z = 3.0e-6
    ts = 1e-12 + np.linspace(0.0, T, 4001)
    Ey = np.array([orc.undulator_field(u, 0.0, z, t)[0][1] for t in ts])
    A0 = a0 * ME * C0 / QE
    w0 = 2 * np.pi * C0 / lam
    amp = g0 * (1 - direction * b0) * A0 * w0
    assert np.abs(Ey).max() == pytest.approx(amp, rel=1e-6)
    # periodic with T, and not with T / 2 (sign flips)
    e0 = orc.undulator_field(u, 0.0, z, 1.3e-12)[0][1]
    e1 = orc.undulator_field(u, 0.0, z, 1.3e-12 + T)[0][1]
    eh = orc.undulator_field(u, 0.0, z, 1.3e-12 + T / 2)[0][1]
    assert e1 == pytest.approx(e0, rel=1e-7, abs=1e-9 * amp)
    assert eh == pytest.approx(-e0, rel=1e-7, abs=1e-9 * amp)


@pytest.mark.parametrize("signal", ["gaussian", "secant-hyperbolic"])
def test_optical_envelope(orc, signal):
    # a rest frame at rest in the lab (gamma0 = 1) keeps t' = t at z = 0
    g0 = 1.0
    lam = 1.0e-6
    tv = 400 * lam / C0   # many carrier periods: the envelope varies slowly
    u0 = _optical(g0, 1.0, lam, -1, (0.0, 1.0), signal=signal, offset=0.0, variance=C0 * tv)
    u90 = dict(u0, cep=np.pi / 2)
    A0 = ME * C0 / QE
    w0 = 2 * np.pi * C0 / lam

    def envelope(t):
        a = orc.undulator_field(u0, 0.0, 0.0, t)[0][1]
        b = orc.undulator_field(u90, 0.0, 0.0, t)[0][1]
        return np.hypot(a, b) / (A0 * w0)

    assert envelope(0.0) == pytest.approx(1.0, rel=1e-5)
    if signal == "gaussian":
        assert envelope(tv / 2) ** 2 == pytest.approx(0.5, rel=1e-3)
        assert envelope(-tv / 2) ** 2 == pytest.approx(0.5, rel=1e-3)
    else:
        assert envelope(tv) == pytest.approx(1 / np.cosh(1.0), rel=1e-3)


def test_flat_top_is_flat_after_its_rise(orc):
    g0 = 1.0
    lam = 1.0e-6
    u = _optical(g0, 1.0, lam, -1, (0.0, 1.0), signal="flat-top", offset=0.0,
                 variance=50 * lam)
    u90 = dict(u, cep=np.pi / 2)
    A0 = ME * C0 / QE
    w0 = 2 * np.pi * C0 / lam
    for t in np.linspace(1e-15, 400 * lam / C0, 7):
        a = orc.undulator_field(u, 0.0, 0.0, t)[0][1]
        b = orc.undulator_field(u90, 0.0, 0.0, t)[0][1]
        assert np.hypot(a, b) == pytest.approx(A0 * w0, rel=1e-12)


def _electron(orc, und, g0, uz0, om, steps_per_period, periods, with_z=False):
    dt = 2 * np.pi / om / steps_per_period
    g = dict(nx=8, ny=8, nz=8, dx=1.0, dy=1.0, dz=1.0, x0=-3.5, y0=-3.5, z0=-3.5, dt=dt,
             n_sub=1, stencil=0, space_charge=1)
    n = 512
    E = np.zeros(3 * n)
    B = np.zeros(3 * n)
    P = dict(x=np.zeros(1), y=np.zeros(1), z=np.zeros(1), ux=np.zeros(1), uy=np.zeros(1),
             uz=np.array([uz0]))
    ux, zs = [], []
    for s in range(steps_per_period * periods):
        P, lost, _, _ = _push(orc, g, und, E, B, P, t_half=(s + 0.5) * dt, q=-1e-20)
        assert not lost.any()
        ux.append(P["ux"][0])
        zs.append(P["z"][0])
    if with_z:
        return np.array(ux), np.array(zs), dt
    return np.array(ux), dt


def _crossings(x, dt):
    """Times of the rising zero crossings of x (linear interpolation)."""
    idx = np.nonzero((x[:-1] < 0) & (x[1:] >= 0))[0]
    frac = -x[idx] / (x[idx + 1] - x[idx])
    return idx, frac, (idx + frac) * dt


def _frequency_and_drift(x, z, dt):
    """Mean angular frequency of x and the mean velocity between its first and
    last rising zero crossing (the same phase of the figure-8 motion)."""
    idx, frac, tc = _crossings(x, dt)
    zc = z[idx] + frac * (z[idx + 1] - z[idx])
    return (2 * np.pi * (len(tc) - 1) / (tc[-1] - tc[0]),
            (zc[-1] - zc[0]) / (tc[-1] - tc[0]))


def test_static_and_optical_undulators_agree(orc):
    gd = golden()
    gamma, K, lu = gd["gamma_job"], gd["undulator_parameter_job"], gd["undulator_period"]
    g0 = gamma / np.sqrt(1 + K * K / 2)
    b0 = np.sqrt(1 - 1 / g0 ** 2)
    uz0 = g0 * (np.sqrt(gamma ** 2 - 1) - b0 * gamma)
    om = 2 * np.pi / lu * g0 * b0 * C0
    spp, periods = 400, 40
    static = dict(gamma0=g0, lambda_u=lu, K=K, z_ent_lab=5 * lu, length_lab=0.0, fringe=1)
    optical = _optical(g0, K, 2 * lu, -1, (1.0, 0.0), signal="flat-top", offset=10 * lu,
                       variance=4 * lu)
    tail = slice(20 * spp, 40 * spp)
    us, zs, dt = _electron(orc, static, g0, uz0, om, spp, periods, with_z=True)
    uo, zo, _ = _electron(orc, optical, g0, uz0, om, spp, periods, with_z=True)
    assert np.abs(us[tail]).max() == pytest.approx(K, rel=1e-2)
    assert np.abs(uo[tail]).max() == pytest.approx(K, rel=1e-2)
    # the electron sees the static pattern move at -beta0 c and the optical
    # wave at -c: with its mean velocity v between crossings the frequencies
    # are k_u gamma0 (beta0 c + v) and (pi c / lambda_u) gamma0 (1 + beta0)(1 + v/c)
    fs, vs = _frequency_and_drift(us[tail], zs[tail], dt)
    fo, vo = _frequency_and_drift(uo[tail], zo[tail], dt)
    assert fs == pytest.approx(2 * np.pi / lu * g0 * (b0 * C0 + vs), rel=1e-7)
    assert fo == pytest.approx(np.pi * C0 / lu * g0 * (1 + b0) * (1 + vo / C0), rel=1e-7)
    # no mean drift in the frame of gamma0 for either, and the frequencies
    # agree to O(1/gamma0^2): the paper's equivalence
    assert abs(vs) < 1e-4 * C0 and abs(vo) < 1e-4 * C0
    assert fo / fs == pytest.approx(1.0, abs=2.0 / g0 ** 2)


@pytest.mark.parametrize("signal", ["gaussian", "secant-hyperbolic", "neumann"])
def test_pulse_field_has_no_dc(orc, signal):
    # E = -dA/dt of a vector potential that vanishes before and after the
    # pulse: its time integral at a fixed point is zero (a half-cycle envelope
    # with a cosine carrier, where a field without the envelope's derivative
    # would leave a net kick)
    lam = 1.0e-6
    tv = 0.5 * lam / C0
    u = _optical(1.0, 1.0, lam, -1, (0.0, 1.0), signal=signal, offset=0.0, variance=C0 * tv,
                 cep=np.pi / 2)
    A0 = ME * C0 / QE
    w0 = 2 * np.pi * C0 / lam
    ts = np.linspace(-20 * tv, 20 * tv, 40001)
    Ey = np.array([orc.undulator_field(u, 0.0, 0.0, t)[0][1] for t in ts])
    integral = np.trapezoid(Ey, ts)
    assert np.abs(Ey).max() > 0.1 * A0 * w0
    assert abs(integral) < 1e-6 * A0 * w0 * tv
