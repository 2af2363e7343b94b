"""Oracle pins of the Gaussian-beam seed (input group field-initialization,
type gaussian-beam).  The paper names the beam and its parameters (focus
position, direction, polarization, rayleigh-radius-parallel and
-perpendicular) but prints no formula; the oracle takes the textbook
paraxial beam, one factor per transverse axis, with the rayleigh radius read
as the 1/e radius of the field at the focus.  Pinned by:

  - the paper's own numbers: Example 2's seed (strength parameter 9.857e-7,
    wavelength 0.265187 um, radius 183.74 um) carries the 10 kW its table
    prints, Poynting flux through the focal plane integrated numerically
    from the oracle's potential;
  - the profile at the focus: exp(-xi^2/w_par^2 - eta^2/w_perp^2) with xi
    along the polarization, eta across it;
  - the wave equation: the potential, boosted into the rest frame, solves
    (lap - d_t^2/c^2) A = 0 to the paraxial error (1/(k z_R))^2; a dropped
    or doubled Gouy phase, a flipped curvature or a missing square root in
    the amplitude leave a residual a hundred times larger;
  - a very wide beam is the plane wave;
  - injected through the total-field/scattered-field planes in vacuum, the
    beam enters the total-field region and leaves the scattered-field
    region near zero (to the leak of a field that is not a solution of the
    discrete scheme).
"""
import os

import numpy as np
import pytest

from paper_1612_03310_gb300 import inputs

C0 = 299792458.0
MU0 = 1.25663706212e-6
A0_PER_A = 9.1093837015e-31 * C0 / 1.602176634e-19  # A0 / a0 = m_e c / e


def golden():
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "example2_seed.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                out[name] = float(value)
    return out


def test_example2_seed_carries_the_printed_power(orc):
    e = golden()
    lam, w0, zf = e["wavelength"], e["rayleigh_radius"], e["focus_z"]
    assert e["rayleigh_radius"] == e["seed_beam_radius"]
    assert abs(zf - e["seed_focal_point"]) < 1e-3
    # the job file's CW seed: a Gaussian envelope a million metres long
    s = dict(gamma0=1.0, a0=e["strength_parameter"], lambda_l=lam, polarization=(0.0, 1.0),
             z0_lab=zf, offset=0.700005, variance=1e6, cep=0.0, direction=1, signal="gaussian",
             beam="gaussian-beam", rayleigh_radius=(w0, w0))
    T = lam / C0
    xs = np.linspace(-4 * w0, 4 * w0, 121)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    ht = T / 1000
    hz = C0 * ht
    P = 0.0
    for m in range(16):                     # time average over one period
        t = m * T / 16
        Ay = lambda z, tt: orc.incident_potential(s, z, tt, X, Y)[..., 1]
        Ey = -(Ay(zf, t + ht) - Ay(zf, t - ht)) / (2 * ht)      # E = -dA/dt
        Bx = -(Ay(zf + hz, t) - Ay(zf - hz, t)) / (2 * hz)      # B = curl A
        P += (-Ey * Bx).sum() / MU0 * (xs[1] - xs[0]) ** 2 / 16
    assert abs(P / e["seed_power"] - 1) < 0.01, P


def _astigmatic(gamma0=1.0, direction=1, signal="flat-top"):
    lam = 1e-6
    return dict(gamma0=gamma0, a0=1e-3, lambda_l=lam, polarization=(0.6, 0.8), z0_lab=0.01,
                offset=-1.0, variance=lam, cep=0.3, direction=direction, signal=signal,
                beam="gaussian-beam", rayleigh_radius=(4 * lam, 6 * lam), x0_lab=1e-6,
                y0_lab=-2e-6)


def test_profile_at_the_focus(orc):
    s = _astigmatic()
    wp, wq = s["rayleigh_radius"]
    rng = np.random.default_rng(1)
    xi, eta = rng.uniform(-2, 2, 50) * wp, rng.uniform(-2, 2, 50) * wq
    x = s["x0_lab"] + 0.6 * xi - 0.8 * eta
    y = s["y0_lab"] + 0.8 * xi + 0.6 * eta
    t = 0.37e-15                              # zeta = 0: no curvature, no Gouy phase
    A = orc.incident_potential(s, s["z0_lab"], t, x, y)
    A00 = orc.incident_potential(s, s["z0_lab"], t, s["x0_lab"], s["y0_lab"])
    assert abs(A00[1]) > 0.1 * 1e-3 * A0_PER_A
    np.testing.assert_allclose(A / A00, np.exp(-xi ** 2 / wp ** 2 - eta ** 2 / wq ** 2)[:, None]
                               * np.ones(2), rtol=1e-12)
    # the polarization is p
    np.testing.assert_allclose(A[:, 0] * 0.8, A[:, 1] * 0.6, rtol=1e-12)


@pytest.mark.parametrize("direction", [1, -1])
def test_wave_equation_in_the_rest_frame(orc, direction):
    g0 = 2.5
    b0 = np.sqrt(1 - 1 / g0 ** 2)
    s = _astigmatic(g0, direction)
    lam, (wp, wq) = s["lambda_l"], s["rayleigh_radius"]
    zr = np.pi * wp ** 2 / lam
    rng = np.random.default_rng(2 + direction)
    n = 200
    zl = s["z0_lab"] + rng.uniform(-2, 2, n) * zr           # lab points around the focus
    tl = rng.uniform(0, 1e-12, n)
    x = s["x0_lab"] + rng.uniform(-1.5, 1.5, n) * wp
    y = s["y0_lab"] + rng.uniform(-1.5, 1.5, n) * wq
    z, t = g0 * (zl - b0 * C0 * tl), g0 * (tl - b0 * zl / C0)  # the same points, rest frame
    h = lam * g0 * (1 + direction * b0) / 100              # rest-frame wavelength / 100

    def A(dx=0.0, dy=0.0, dz=0.0, dt=0.0):
        return orc.incident_potential(s, z + dz, t + dt, x + dx, y + dy)

    def d2(**kw):                                          # fourth-order second difference
        (k, v), = kw.items()
        return (-A(**{k: 2 * v}) + 16 * A(**{k: v}) - 30 * A() + 16 * A(**{k: -v})
                - A(**{k: -2 * v})) / (12 * v * v)

    R = d2(dx=h) + d2(dy=h) + d2(dz=h) - d2(dt=h / C0) / C0 ** 2
    k = 2 * np.pi / lam
    assert np.abs(A()).max() > 0.3 * 1e-3 * A0_PER_A
    assert np.abs(R).max() <= 1e-4 * k ** 2 * 1e-3 * A0_PER_A


def test_a_wide_beam_is_the_plane_wave(orc):
    s = dict(_astigmatic(3.0, 1, "gaussian"), rayleigh_radius=(1e3, 1e3), z0_lab=0.0,
             offset=0.0, variance=1e-3)
    pw = dict(s, beam="plane-wave")
    rng = np.random.default_rng(4)
    z, t = rng.uniform(-1e-4, 1e-4, 40), rng.uniform(-1e-13, 1e-13, 40)
    x, y = rng.uniform(-1e-4, 1e-4, 40), rng.uniform(-1e-4, 1e-4, 40)
    a, b = orc.incident_potential(s, z, t, x, y), orc.incident_potential(pw, z, t, x, y)
    assert np.abs(b).max() > 0.1 * 1e-3 * A0_PER_A
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-9 * 1e-3 * A0_PER_A)


def _tfsf_run(orc, w_over_lambda, centre=80, extra=16):
    """The beam injected through the planes k = 2, 3 of a vacuum grid at
    c dt = dz; returns the potential, the incident potential at the end and
    the seed.  The pulse reaches the total-field plane at step `centre`
    (about five envelope widths after the start, so the grid starts at rest
    with the incident field still zero on the planes)."""
    nxy, nz = 64, 64
    g = dict(inputs.random_grid(0, nxy, nxy, nz, courant=1.0, stencil=0, dz_over_dx=0.5),
             z0=0.0)
    g["x0"], g["y0"] = -(nxy // 2) * g["dx"], -(nxy // 2) * g["dy"]
    gamma0 = 3.0
    b0 = np.sqrt(1 - 1 / gamma0 ** 2)
    lam_rest = 16 * g["dz"]
    lam_lab = lam_rest / (gamma0 * (1 + b0))
    tau = gamma0 * (1 - b0) * (centre * g["dt"] - 3 * g["dz"] / C0)
    seed = dict(gamma0=gamma0, a0=1e-3, lambda_l=lam_lab, polarization=(0.6, 0.8), z0_lab=0.0,
                offset=C0 * tau, variance=lam_lab, cep=0.4, direction=1, signal="gaussian",
                beam="gaussian-beam",
                rayleigh_radius=(w_over_lambda * lam_rest, 1.3 * w_over_lambda * lam_rest))
    o = orc.OracleSim(g, None, dict(x=[], y=[], z=[], ux=[], uy=[], uz=[]))
    o.set_seed(seed)
    n = centre + extra
    o.step(n)
    Z, Y, X = np.meshgrid(g["z0"] + np.arange(nz) * g["dz"], g["y0"] + np.arange(nxy) * g["dy"],
                          g["x0"] + np.arange(nxy) * g["dx"], indexing="ij")
    return o, orc.incident_potential(seed, Z, n * g["dt"], X, Y), nz


def test_beam_enters_the_total_field_region(orc):
    # Not exact as for the plane wave: the paraxial beam solves the wave
    # equation, not the discrete scheme, so the interface leaks the scheme's
    # residual of the incident field, falling with the width of the beam.
    # (The neighbours' own values in the correction, against the centre
    # vertex's value for all of them, change the result by about 1e-3 of the
    # beam only, inside this leak: that part of the correction is pinned by
    # the plane-wave tests and this bound, not beyond.)
    o, ref, nz = _tfsf_run(orc, 1.5)
    for c in range(2):
        P, f = o.potential(c), ref[..., c]
        m = np.abs(f).max()
        assert m > 0.3 * 1e-3 * A0_PER_A
        assert np.abs(P[3:nz - 1] - f[3:nz - 1]).max() <= 6e-2 * m
        assert np.abs(P[:3]).max() <= 2.5e-2 * m
        assert np.abs(P[:3, 28:36, 28:36]).max() <= 5e-3 * m
    # twice as wide: the leak at the centre falls about as 1/w^2
    o2, ref2, _ = _tfsf_run(orc, 3.0)
    m2 = np.abs(ref2[..., 1]).max()
    assert np.abs(o2.potential(1)[:3, 28:36, 28:36]).max() <= 1.5e-3 * m2
