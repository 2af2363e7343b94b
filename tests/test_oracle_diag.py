"""Oracle pins of the diagnostics (FEL-OUTPUT radiation power with
wavelengths, bunch sampling, bunching factor), against closed forms:

  - means and rms spreads of evenly spaced particles (uniform lattice);
    particles flagged lost do not count;
  - bunching factor: 1 for one phase, 0 for evenly spread phases, |2f - 1|
    for two populations half a wavelength apart, unchanged by a shift of a
    whole wavelength; the bunch generator's modulation gives b_f;
  - spectrum: a forward plane wave sampled over whole periods gives
    dW/domega = (E' T / 2)^2 A / (pi c mu0) at its frequency with
    E' = gamma0 (1 + beta0) E0, zero one bin away, and the backward factor
    gamma0 (1 - beta0); a rest-frame wave of angular frequency w sampled at a
    fixed plane appears at the lab wavelength 2 pi c / (gamma0 (1 + beta0) w).
"""
import numpy as np
import pytest

from paper_1612_03310_gb300 import inputs

C0 = 299792458.0
MU0 = 1.0 / (8.8541878128e-12 * C0 * C0)


def test_bunch_moments_of_a_lattice(orc):
    n = 1000
    L = 3.0e-3
    x = np.arange(n) * (L / n)  # uniform lattice on [0, L)
    y = -2.0 * x + 1.0e-3
    z = np.full(n, 4.0e-3)
    ux = np.linspace(-1.0, 1.0, n)
    uy = np.zeros(n)
    uz = np.full(n, 0.35)
    # lost particles anywhere must not count
    xs = np.concatenate([x, [1.0, -7.0]])
    ext = lambda a, v: np.concatenate([a, [v, v]])  # noqa: E731
    lost = np.concatenate([np.zeros(n, np.int32), np.ones(2, np.int32)])
    out = orc.bunch_stats(xs, ext(y, 5.0), ext(z, 9.0), ext(ux, 3.0), ext(uy, 3.0),
                          ext(uz, 3.0), lost, 1.0)
    mean_x = (n - 1) * L / (2 * n)
    var_x = L * L * (n * n - 1) / (12.0 * n * n)
    step_u = 2.0 / (n - 1)
    var_u = step_u * step_u * (n * n - 1) / 12.0
    np.testing.assert_allclose(out[0], mean_x, rtol=1e-13)
    np.testing.assert_allclose(out[1], 1.0e-3 - 2.0 * mean_x, rtol=1e-12)
    np.testing.assert_allclose(out[2], 4.0e-3, rtol=1e-14)
    np.testing.assert_allclose(out[3:6], [0.0, 0.0, 0.35], atol=1e-14)
    np.testing.assert_allclose(out[6], np.sqrt(var_x), rtol=1e-10)
    np.testing.assert_allclose(out[7], 2.0 * np.sqrt(var_x), rtol=1e-10)
    # constant z: no spread, up to the rounding of the one-pass variance
    # (sqrt of n eps z^2)
    assert out[8] < 1e-6 * 4.0e-3
    np.testing.assert_allclose(out[9], np.sqrt(var_u), rtol=1e-10)
    assert out[10] == 0.0 and out[11] < 1e-7
    assert out[13] == n


@pytest.mark.parametrize("f", [1.0, 0.5, 0.75, 0.1])
def test_bunching_factor_closed_forms(orc, f):
    lam = 2.1e-4
    kb = 2 * np.pi / lam
    n = 4000
    na = int(round(f * n))
    z = np.concatenate([np.full(na, 3.0e-3), np.full(n - na, 3.0e-3 + lam / 2)])
    zero = np.zeros(n)
    lost = np.zeros(n, np.int32)
    b = orc.bunch_stats(zero, zero, z, zero, zero, zero, lost, kb)[12]
    assert b == pytest.approx(abs(2 * na / n - 1), abs=1e-9)
    # a whole-wavelength shift of every particle changes nothing
    b2 = orc.bunch_stats(zero, zero, z + lam, zero, zero, zero, lost, kb)[12]
    assert b2 == pytest.approx(b, abs=1e-9)


def test_bunching_factor_even_phases_and_generator(orc):
    lam = 2.1e-4
    kb = 2 * np.pi / lam
    n = 1024
    z = 1.0e-3 + np.arange(n) * (lam / n)
    zero = np.zeros(n)
    assert orc.bunch_stats(zero, zero, z, zero, zero, zero, np.zeros(n, np.int32), kb)[12] < 1e-12
    # the c2 bunch: uniform z0 displaced by -(2 b_f / k_b) sin(k_b z0); the
    # sample mean of exp(i k_b z) matches the expectation integral over z0
    # (by quadrature) to the sampling error
    w = inputs.workload("c2")
    spec = dict(w["bunch_spec"], n=400000)
    P = inputs.make_bunch(spec, w["seed"])
    kb2, bf = spec["kb"], spec["bf"]
    z0 = np.linspace(spec["z_lo"], spec["z_hi"], 2000001)
    ph = np.exp(1j * kb2 * (z0 - (2 * bf / kb2) * np.sin(kb2 * z0)))
    expect = abs(np.trapezoid(ph, z0) / (spec["z_hi"] - spec["z_lo"]))
    lost = np.zeros(P["x"].size, np.int32)
    b = orc.bunch_stats(P["x"], P["y"], P["z"], P["ux"], P["uy"], P["uz"], lost, kb2)[12]
    assert abs(b - expect) < 3.0 / np.sqrt(P["x"].size), (b, expect)


def _plane_grid():
    return dict(nx=10, ny=8, nz=6, dx=2.0e-5, dy=3.0e-5, dz=1.0e-5, x0=0.0, y0=0.0, z0=0.0,
                dt=1.0e-14, n_sub=1, stencil=0, space_charge=1)


def _fields_at_plane(g, kp, ex, by):
    n = g["nx"] * g["ny"] * g["nz"]
    E = np.zeros(3 * n)
    B = np.zeros(3 * n)
    k, j, i = np.meshgrid(np.arange(g["nz"]), np.arange(g["ny"]), np.arange(g["nx"]),
                          indexing="ij")
    on = (k == kp).ravel()
    E[:n][on] = ex
    B[n:2 * n][on] = by
    return E, B


@pytest.mark.parametrize("direction", [1.0, -1.0])
def test_spectrum_of_a_plane_wave(orc, direction):
    g = _plane_grid()
    kp = 3
    gamma0 = 7.0
    b0 = np.sqrt(1 - 1 / gamma0 ** 2)
    lam = 3.0e-6  # lab wavelength requested
    om = orc.observed_omega([lam, lam * 40 / 41.0], gamma0)  # the line and one bin away
    dtl = gamma0 * g["dt"]
    periods = 40
    N = int(round(periods * 2 * np.pi / (om[0] * dtl)))
    dtl = periods * 2 * np.pi / (om[0] * N)  # whole periods exactly
    nv = (g["nx"] - 2) * (g["ny"] - 2)
    acc = np.zeros(2 * nv * 8)
    E0, phi = 2.5e6, 0.3
    for n in range(N):
        t = 1.0e-12 + n * dtl
        e = E0 * np.cos(om[0] * t + phi)
        E, B = _fields_at_plane(g, kp, e, direction * e / C0)
        orc.spectrum_accumulate(g, gamma0, E, B, kp, t, dtl, om, acc)
    dw = orc.spectrum_density(g, 2, acc)
    ep = gamma0 * (1 + direction * b0) * E0
    T = N * dtl
    area = nv * g["dx"] * g["dy"]
    expect = direction * (ep * T / 2) ** 2 * area / (np.pi * C0 * MU0)
    assert dw[0] == pytest.approx(expect, rel=1e-9)
    assert abs(dw[1]) < 1e-9 * abs(expect)


def test_spectrum_maps_rest_frequency_to_lab_wavelength(orc):
    # a forward rest-frame wave E_x = c B_y = E0 cos(w (t - z/c)) sampled at
    # rest times t_n at a fixed plane peaks at the Doppler-shifted lab
    # wavelength 2 pi c / (gamma0 (1 + beta0) w)
    g = _plane_grid()
    kp = 2
    zp = kp * g["dz"]
    gamma0 = 5.0
    b0 = np.sqrt(1 - 1 / gamma0 ** 2)
    w = 2 * np.pi * C0 / 4.0e-5  # rest-frame wavelength 40 um
    periods = 30
    N = 600
    dt = periods * 2 * np.pi / (w * N)
    g = dict(g, dt=dt)
    lam_lab = 2 * np.pi * C0 / (gamma0 * (1 + b0) * w)
    om = orc.observed_omega([lam_lab, lam_lab * 30 / 31.0], gamma0)
    nv = (g["nx"] - 2) * (g["ny"] - 2)
    acc = np.zeros(2 * nv * 8)
    E0 = 1.0e5
    for n in range(N):
        t = (n + 0.5) * dt
        e = E0 * np.cos(w * (t - zp / C0))
        E, B = _fields_at_plane(g, kp, e, e / C0)
        t_lab = gamma0 * (t + b0 * zp / C0)
        orc.spectrum_accumulate(g, gamma0, E, B, kp, t_lab, gamma0 * dt, om, acc)
    dw = orc.spectrum_density(g, 2, acc)
    ep = gamma0 * (1 + b0) * E0
    T = N * gamma0 * dt
    area = nv * g["dx"] * g["dy"]
    assert dw[0] == pytest.approx((ep * T / 2) ** 2 * area / (np.pi * C0 * MU0), rel=1e-9)
    assert abs(dw[1]) < 1e-9 * dw[0]
