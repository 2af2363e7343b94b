"""Pins of the oracle's particle side and diagnostics, each against something
other than the oracle's own formulas:

  - E and B from quadratic potentials equal the analytic curl/gradient (central
    differences are exact for quadratics), which fixes every index and sign of
    Sec. "Field Evaluation" (including the A_y term of B_z);
  - the trilinear gather reproduces a linear field exactly, read back through
    the Boris closed form for B = 0 (u grows by q dt E / (m c));
  - the deposit conserves charge and current exactly (partition of unity);
  - Boris invariants: |u| conserved for E = 0, the gyration angle
    2 atan(|q| B dt / (2 m gamma)) per step with the right sense of rotation;
  - a single electron in the boosted undulator oscillates with |u_x| = K, has
    no mean longitudinal drift, and radiates (Doppler-shifted to the lab) at
    lambda_u (1 + K^2/2) / (2 gamma^2); with Example 1's printed numbers that is
    the printed 3 um, and K = 1.4 at 3 cm gives the printed 0.5 T;
  - lab-frame power of a forward (backward) plane wave is gamma0^2 (1 +- beta0)^2
    times the rest-frame Poynting flux;
  - particles leaving the valid region are flagged and deposit nothing.
"""
import os

import numpy as np
import pytest

from paper_1612_03310_gb300 import inputs

C0 = 299792458.0
E_CH = 1.602176634e-19
M_E = 9.1093837015e-31
QM = -E_CH / M_E
MU0 = 1.0 / (8.8541878128e-12 * C0 * C0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "example1_table.txt")


def golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            out[parts[0]] = float(parts[1])
    return out


def _xyz(g):
    k, j, i = np.meshgrid(np.arange(g["nz"]), np.arange(g["ny"]), np.arange(g["nx"]),
                          indexing="ij")
    return g["x0"] + i * g["dx"], g["y0"] + j * g["dy"], g["z0"] + k * g["dz"]


def test_fields_exact_for_quadratic_potentials(orc):
    g = inputs.random_grid(0, 9, 10, 11)
    X, Y, Z = [a * 1.0e3 for a in _xyz(g)]  # mm, keeps magnitudes near 1
    s = 1.0e3
    # level n and n+1 potentials (quadratics) and phi^n
    Axn, Ayn, Azn = Y * Y, X * Z, X * Y + 0.5 * Z * Z
    Ax1, Ay1, Az1 = Y * Y + 0.3 * X * X, X * Z + 2.0 * X * Y, X * Y - Y * Z
    ph = X * X + Y * Z - 0.7 * Z
    lev_n = np.concatenate([a.ravel() for a in (Axn, Ayn, Azn, ph)])
    lev_1 = np.concatenate([a.ravel() for a in (Ax1, Ay1, Az1, ph)])
    E, B = orc.fields(g, lev_n, lev_1)
    n = X.size
    # analytic derivatives (d/dx in physical units = s * d/dX)
    curl_n = (s * (X - X), s * (0.0 - Y), s * (Z - 2 * Y))
    curl_1 = (s * (X - Z - X), s * (0.0 - (Y + 0.0)), s * ((Z + 2 * Y) - 2 * Y))
    # curl A^{n+1}: Bx = dAz/dy - dAy/dz = (X - Z) - X ; By = dAx/dz - dAz/dx = 0 - Y
    #               Bz = dAy/dx - dAx/dy = (Z + 2Y) - 2Y
    grad = (s * 2 * X, s * Z, s * (Y - 0.7))
    dAdt = ((Ax1 - Axn) / g["dt"], (Ay1 - Ayn) / g["dt"], (Az1 - Azn) / g["dt"])
    inner = (slice(1, -1),) * 3
    for a in range(3):
        Bexp = 0.5 * (curl_n[a] + curl_1[a])
        Eexp = -dAdt[a] - grad[a]
        Bgot = B[a * n:(a + 1) * n].reshape(X.shape)
        Egot = E[a * n:(a + 1) * n].reshape(X.shape)
        np.testing.assert_allclose(Bgot[inner], Bexp[inner], rtol=1e-10, atol=1e-9)
        np.testing.assert_allclose(Egot[inner], Eexp[inner], rtol=1e-10,
                                   atol=1e-10 * np.abs(Eexp).max())


def _push(orc, g, und, E, B, P, t_half=0.0, q=-1.0e-15):
    import ctypes as C
    L = orc.lib()
    n = g["nx"] * g["ny"] * g["nz"]
    src = np.zeros(4 * n)
    lost = np.zeros(P["x"].size, dtype=np.int32)
    arrs = [np.array(P[k], dtype=np.float64) for k in ("x", "y", "z", "ux", "uy", "uz")]
    nl = L.orc_push_deposit(C.byref(orc.make_grid(g)), C.byref(orc.make_und(und)), q, t_half,
                            orc._p(E), orc._p(B), arrs[0].size, *[orc._p(a) for a in arrs],
                            orc._p(lost), orc._p(src))
    return dict(zip(("x", "y", "z", "ux", "uy", "uz"), arrs)), lost, src, nl


NO_UND = dict(gamma0=10.0, lambda_u=0.01, K=0.0, z_ent_lab=0.0, length_lab=0.0, fringe=1)


def test_gather_linear_field_exact(orc):
    g = inputs.random_grid(0, 12, 11, 13)
    X, Y, Z = _xyz(g)
    n = X.size
    a = np.array([1.0e5, -2.0e5, 3.0e5])
    Gm = np.array([[2.0e8, -1.0e8, 0.5e8], [0.3e8, 1.0e8, -2.0e8], [-1.0e8, 0.2e8, 1.5e8]])
    E = np.concatenate([(a[c] + Gm[c, 0] * X + Gm[c, 1] * Y + Gm[c, 2] * Z).ravel()
                        for c in range(3)])
    B = np.zeros(3 * n)
    P = inputs.random_particles(4, g, 200, u_scale=0.0)
    r0 = np.stack([P["x"], P["y"], P["z"]])
    out, lost, _, _ = _push(orc, g, NO_UND, E, B, P)
    assert not lost.any()
    u = np.stack([out["ux"], out["uy"], out["uz"]])
    Erec = u * C0 / (QM * g["dt"])
    Eexp = a[:, None] + Gm @ r0
    np.testing.assert_allclose(Erec, Eexp, rtol=1e-9)


def test_deposit_conserves_charge_and_current(orc):
    g = inputs.random_grid(0, 12, 11, 13)
    n = g["nx"] * g["ny"] * g["nz"]
    P = inputs.random_particles(5, g, 300, u_scale=0.2)
    q = -3.0e-15
    out, lost, src, _ = _push(orc, g, NO_UND, np.zeros(3 * n), np.zeros(3 * n), P, q=q)
    assert not lost.any()
    V = g["dx"] * g["dy"] * g["dz"]
    np.testing.assert_allclose(src[3 * n:].sum() * V, q * P["x"].size, rtol=1e-12)
    for a, key in enumerate(("x", "y", "z")):
        flux = q * np.sum(out[key] - P[key]) / g["dt"]
        np.testing.assert_allclose(src[a * n:(a + 1) * n].sum() * V, flux, rtol=1e-10)


def test_deposit_centroids(orc):
    # CIC weights reproduce linear functions, so the first moment of one
    # particle's deposit is exact: the J deposit is centred on the mid point of
    # the step (Eq. currentIntegral: current at the time between the two
    # position samples), the rho deposit on the end position.
    g = inputs.random_grid(0, 12, 11, 13)
    n = g["nx"] * g["ny"] * g["nz"]
    X, Y, Z = _xyz(g)
    coords = (X.ravel(), Y.ravel(), Z.ravel())
    for seed in range(5):
        P = inputs.random_particles(20 + seed, g, 1, u_scale=0.6)
        out, lost, src, _ = _push(orc, g, NO_UND, np.zeros(3 * n), np.zeros(3 * n), P)
        assert not lost.any()
        rho = src[3 * n:]
        for a, key in enumerate(("x", "y", "z")):
            mid = 0.5 * (P[key][0] + out[key][0])
            J = src[a * n:(a + 1) * n]
            for b in range(3):
                cen = np.sum(J * coords[b]) / np.sum(J)
                key_b = ("x", "y", "z")[b]
                assert cen == pytest.approx(0.5 * (P[key_b][0] + out[key_b][0]), rel=1e-9,
                                            abs=1e-12)
            assert np.sum(rho * coords[a]) / np.sum(rho) == pytest.approx(out[key][0],
                                                                        rel=1e-9, abs=1e-12)
            _ = mid


def test_particle_on_vertex_deposits_there(orc):
    g = inputs.random_grid(0, 10, 10, 10)
    n = 1000
    P = dict(x=np.array([g["x0"] + 4 * g["dx"]]), y=np.array([g["y0"] + 5 * g["dy"]]),
             z=np.array([g["z0"] + 3 * g["dz"]]), ux=np.zeros(1), uy=np.zeros(1), uz=np.zeros(1))
    _, lost, src, _ = _push(orc, g, NO_UND, np.zeros(3 * n), np.zeros(3 * n), P, q=-1e-15)
    rho = src[3 * n:].reshape(10, 10, 10)
    V = g["dx"] * g["dy"] * g["dz"]
    assert rho[3, 5, 4] == pytest.approx(-1e-15 / V, rel=1e-12)
    rho[3, 5, 4] = 0.0
    assert np.abs(rho).max() < 1e-12 * 1e-15 / V


def test_boris_conserves_energy_without_E(orc):
    rng = np.random.default_rng(0)
    u = np.array([0.3, -0.8, 1.7])
    for _ in range(50):
        Bf = rng.standard_normal(3) * 2.0
        u2 = orc.boris(u, [0, 0, 0], Bf, QM, 1e-12)
        assert np.linalg.norm(u2) == pytest.approx(np.linalg.norm(u), rel=1e-14)
        u = u2


@pytest.mark.parametrize("Bz", [0.1, 3.0])
def test_boris_rotation(orc, Bz):
    u = np.array([0.5, 0.0, 0.0])
    dt = 1e-12
    gam = np.sqrt(1 + 0.25)
    u2 = orc.boris(u, [0, 0, 0], [0, 0, Bz], QM, dt)
    ang = np.arctan2(u2[1], u2[0])
    expect = 2 * np.arctan(abs(QM) * Bz * dt / (2 * gam))
    # a negative charge gyrates counter-clockwise about B (du/dt = q/(m gamma) u x B)
    assert ang == pytest.approx(expect, rel=1e-12)


def test_boris_uniform_E_linear(orc):
    u = np.array([0.1, 0.2, -0.3])
    Ef = np.array([1e6, -2e6, 3e5])
    dt = 2e-13
    for k in range(1, 6):
        u = orc.boris(u, Ef, [0, 0, 0], QM, dt)
        np.testing.assert_allclose(u, np.array([0.1, 0.2, -0.3]) + k * QM * dt * Ef / C0,
                                   rtol=1e-13)


def test_undulator_amplitude_matches_printed_field(orc):
    gd = golden()
    K, lu = gd["undulator_parameter_table"], gd["undulator_period"]
    und = dict(gamma0=50.0, lambda_u=lu, K=K, z_ent_lab=0.0, length_lab=0.0, fringe=1)
    g0 = 50.0
    zs = np.linspace(0.0, lu, 4001)
    By_lab = [orc.undulator_field(und, 0.0, zz / g0, 0.0)[1][1] / g0 for zz in zs]
    assert max(By_lab) == pytest.approx(gd["magnetic_field"], rel=1e-2)


def test_undulator_fringe_continuous(orc):
    und = dict(gamma0=20.0, lambda_u=0.02, K=1.2, z_ent_lab=0.1, length_lab=0.5, fringe=1)
    g0 = und["gamma0"]
    B0 = 2 * np.pi * M_E * C0 * und["K"] / (E_CH * und["lambda_u"])
    scaleB = g0 * B0 * np.cosh(2 * np.pi / und["lambda_u"] * 3e-4)
    scaleE = C0 * scaleB
    for edge in (und["z_ent_lab"], und["z_ent_lab"] + und["length_lab"]):
        for y in (0.0, 3e-4):
            eps = 1e-9
            lo = orc.undulator_field(und, y, (edge - eps) / g0, 0.0)
            hi = orc.undulator_field(und, y, (edge + eps) / g0, 0.0)
            np.testing.assert_allclose(lo[0], hi[0], atol=1e-5 * scaleE)
            np.testing.assert_allclose(lo[1], hi[1], atol=1e-5 * scaleB)
            # slope: one-sided differences agree
            h = 1e-6
            f = lambda zz: orc.undulator_field(und, y, zz / g0, 0.0)[1][1]  # noqa: E731
            dl = (f(edge) - f(edge - h)) / h
            dr = (f(edge + h) - f(edge)) / h
            assert dl == pytest.approx(dr, rel=2e-3, abs=1e-3)


def _single_electron(orc, gamma, K, lu, steps_per_period, periods):
    g0 = gamma / np.sqrt(1 + K * K / 2)
    b0 = np.sqrt(1 - 1 / g0 ** 2)
    # lab 4-momentum (gamma, 0, 0, gamma*beta) seen from the frame moving with b0
    uz0 = g0 * (np.sqrt(gamma ** 2 - 1) - b0 * gamma)
    om = 2 * np.pi / lu * g0 * b0 * C0
    dt = 2 * np.pi / om / steps_per_period
    g = dict(nx=8, ny=8, nz=8, dx=1.0, dy=1.0, dz=1.0, x0=-3.5, y0=-3.5, z0=-3.5, dt=dt,
             n_sub=1, stencil=0, space_charge=1)
    und = dict(gamma0=g0, lambda_u=lu, K=K, z_ent_lab=5 * lu, length_lab=0.0, fringe=1)
    n = 512
    E = np.zeros(3 * n)
    B = np.zeros(3 * n)
    P = dict(x=np.zeros(1), y=np.zeros(1), z=np.zeros(1), ux=np.zeros(1), uy=np.zeros(1),
             uz=np.array([uz0]))
    hist = []
    for s in range(steps_per_period * periods):
        P, lost, _, _ = _push(orc, g, und, E, B, P, t_half=(s + 0.5) * dt, q=-1e-20)
        assert not lost.any()
        hist.append((P["ux"][0], P["uz"][0], P["z"][0]))
    return np.array(hist), dt, g0, b0


def test_single_electron_in_undulator(orc):
    gd = golden()
    gamma, K, lu = gd["gamma_job"], gd["undulator_parameter_job"], gd["undulator_period"]
    spp = 400
    h, dt, g0, b0 = _single_electron(orc, gamma, K, lu, spp, 40)
    ux, z = h[:, 0], h[:, 2]
    tail = slice(20 * spp, 40 * spp)  # well past the entrance fringe
    assert np.abs(ux[tail]).max() == pytest.approx(K, rel=1e-2)
    assert abs(ux[tail].mean()) < 1e-2 * K
    # no mean longitudinal drift in the frame moving with gamma0 (figure-8 orbit)
    drift = (z[40 * spp - 1] - z[20 * spp - 1]) / (C0 * 20 * spp * dt)
    assert abs(drift) < 1e-3
    # oscillation frequency from zero crossings of u_x
    x = ux[tail]
    idx = np.nonzero((x[:-1] < 0) & (x[1:] >= 0))[0]
    frac = -x[idx] / (x[idx + 1] - x[idx])
    tc = (idx + frac) * dt
    period = (tc[-1] - tc[0]) / (len(tc) - 1)
    om = 2 * np.pi / period
    lam_lab = 2 * np.pi * C0 / (g0 * (1 + b0) * om)
    lam_theory = lu * (1 + K * K / 2) / (2 * gamma * gamma)
    assert lam_lab == pytest.approx(lam_theory, rel=1e-3)
    assert lam_lab == pytest.approx(gd["radiation_wavelength"], rel=1e-2)


@pytest.mark.parametrize("direction", [+1, -1])
def test_power_plane_wave_transform(orc, direction):
    g = inputs.random_grid(0, 10, 9, 8)
    n = g["nx"] * g["ny"] * g["nz"]
    E0 = 2.0e6
    E = np.zeros(3 * n)
    B = np.zeros(3 * n)
    E[:n] = E0
    B[n:2 * n] = direction * E0 / C0
    g0 = 30.0
    b0 = np.sqrt(1 - 1 / g0 ** 2)
    t = 3.0e-12
    kp = 4
    p, tl, zl = orc.radiated_power(g, g0, E, B, kp, t)
    area = (g["nx"] - 2) * (g["ny"] - 2) * g["dx"] * g["dy"]
    p_rest = direction * E0 * E0 / (MU0 * C0) * area
    factor = g0 ** 2 * (1 + direction * b0) ** 2
    assert p == pytest.approx(factor * p_rest, rel=1e-12)
    zp = g["z0"] + kp * g["dz"]
    assert tl == pytest.approx(g0 * (t + b0 * zp / C0), rel=1e-14)
    assert zl == pytest.approx(g0 * (zp + b0 * C0 * t), rel=1e-14)


def test_lost_particles(orc):
    g = inputs.random_grid(0, 10, 10, 10)
    n = 1000
    # one particle just inside the last valid cell moving out, one already out
    P = dict(x=np.array([g["x0"] + 7.9 * g["dx"], g["x0"] + 0.5 * g["dx"]]),
             y=np.array([g["y0"] + 4.5 * g["dy"]] * 2), z=np.array([g["z0"] + 4.5 * g["dz"]] * 2),
             ux=np.array([5.0, 0.0]), uy=np.zeros(2), uz=np.zeros(2))
    lost = np.zeros(2, dtype=np.int32)
    import ctypes as C
    nl0 = orc.lib().orc_mark_lost(C.byref(orc.make_grid(g)), 2, orc._p(P["x"]), orc._p(P["y"]),
                                  orc._p(P["z"]), orc._p(lost))
    assert nl0 == 1 and list(lost) == [0, 1]
    out, lost2, src, nl = _push(orc, g, NO_UND, np.zeros(3 * n), np.zeros(3 * n),
                                dict(P, x=P["x"][:1], y=P["y"][:1], z=P["z"][:1],
                                     ux=P["ux"][:1], uy=P["uy"][:1], uz=P["uz"][:1]))
    assert nl == 1 and lost2[0] == 1
    assert np.all(src == 0.0)
