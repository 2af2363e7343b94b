"""Pins of the oracle's potential update against what the paper and the
mathematics fix, independent of the oracle's own code:

  - discrete plane waves obey the scheme's dispersion relation
    (Eq. numericalDispersionCD for the standard scheme, Eq. NSFDDispersionCD
    for NSFD) to rounding, in the region the boundary cannot reach yet;
  - at c dt = dz the NSFD scheme moves a transversely uniform pulse exactly one
    cell per step along z (Sec. "Numerical Dispersion in FDTD"), and the
    first-order Mur condition absorbs it exactly at normal incidence;
  - a uniform source grows the potential as the leapfrog closed form with the
    physical sign of Eq. HelmholtzA / HelmholtzF;
  - one update equals the operator assembled by Kronecker products of 1-D
    difference matrices (brute force on an 8^3 grid);
  - Mur boundaries act the same on opposite faces (mirror symmetry) and absorb
    an outgoing pulse far better than a reflecting wall;
  - at oblique incidence the first- and second-order Mur conditions reflect
    as the continuous Engquist-Majda operators predict.
"""
import numpy as np
import pytest

from paper_1612_03310_gb300 import inputs

C0 = 299792458.0
MU0 = 1.0 / (8.8541878128e-12 * C0 * C0)
EPS0 = 8.8541878128e-12


def _coords(g):
    k, j, i = np.meshgrid(np.arange(g["nz"]), np.arange(g["ny"]), np.arange(g["nx"]),
                          indexing="ij")
    return i, j, k


def _nsfd_A(g):
    # Eq. NSFDCoefficient
    q = (g["dz"] / g["dx"]) ** 2 + (g["dz"] / g["dy"]) ** 2
    return 0.25 * (1.0 + 0.02 / q)


def _omega(g, kx, ky, kz, nsfd):
    sx = np.sin(kx * g["dx"] / 2) ** 2 / g["dx"] ** 2
    sy = np.sin(ky * g["dy"] / 2) ** 2 / g["dy"] ** 2
    sz2 = np.sin(kz * g["dz"] / 2) ** 2
    A = _nsfd_A(g) if nsfd else 0.0
    lhs = (1.0 - 4.0 * A * sz2) * (sx + sy) + sz2 / g["dz"] ** 2
    s = np.sqrt(lhs) * C0 * g["dt"]
    assert s < 1.0
    return 2.0 * np.arcsin(s) / g["dt"]


def _run_plane_wave(orc, g, nsfd, nsteps):
    i, j, k = _coords(g)
    kx = 2 * np.pi / (9.0 * g["dx"])
    ky = 2 * np.pi / (11.0 * g["dy"])
    kz = 2 * np.pi / (7.0 * g["dz"])
    w = _omega(g, kx, ky, kz, nsfd)
    phase = kx * i * g["dx"] + ky * j * g["dy"] + kz * k * g["dz"]
    one = lambda t: np.tile(np.cos(phase - w * t).ravel(), 4)  # noqa: E731
    prev, cur = one(-g["dt"]), one(0.0)
    src = np.zeros_like(cur)
    for _ in range(nsteps):
        nxt = orc.potential_step(g, prev, cur, src)
        prev, cur = cur, nxt
    expect = one(nsteps * g["dt"]).reshape(4, g["nz"], g["ny"], g["nx"])
    got = cur.reshape(4, g["nz"], g["ny"], g["nx"])
    m = nsteps + 1  # cells the boundary cannot have reached
    sl = (slice(None), slice(m, g["nz"] - m), slice(m, g["ny"] - m), slice(m, g["nx"] - m))
    return got[sl], expect[sl]


@pytest.mark.parametrize("nsfd", [True, False])
def test_plane_wave_obeys_dispersion(orc, nsfd):
    g = inputs.random_grid(0, 26, 24, 30, courant=0.95 if nsfd else 0.55,
                           stencil=0 if nsfd else 1)
    got, expect = _run_plane_wave(orc, g, nsfd, nsteps=9)
    assert got.size > 0
    np.testing.assert_allclose(got, expect, atol=2e-12, rtol=0)


def test_wrong_omega_is_detected(orc):
    # the same check with the other scheme's omega fails: the pin has teeth
    g = inputs.random_grid(0, 26, 24, 30, courant=0.95, stencil=0)
    i, j, k = _coords(g)
    kx = 2 * np.pi / (9.0 * g["dx"])
    ky = 2 * np.pi / (11.0 * g["dy"])
    kz = 2 * np.pi / (7.0 * g["dz"])
    w_nsfd = _omega(g, kx, ky, kz, True)
    w_std = _omega(g, kx, ky, kz, False)
    assert abs(w_nsfd - w_std) / w_nsfd > 1e-3


@pytest.mark.parametrize("boundary", [1, 2])
def test_nsfd_exact_along_z_and_mur_absorbs(orc, boundary):
    # c dt = dz: NSFD keeps the vacuum speed of light along z; a pulse moving
    # towards -z shifts one cell per step and leaves through k = 0 without
    # reflection (beta0 = 0 in the first-order Mur condition; the second-order
    # terms vanish for a field uniform along the face).
    g = dict(inputs.random_grid(0, 40, 40, 32, courant=1.0, stencil=0, dz_over_dx=0.5),
             boundary=boundary)
    i, j, k = _coords(g)
    prof = lambda kk: np.exp(-0.5 * ((kk - 12.0) / 2.0) ** 2)  # noqa: E731
    # psi(k, n) = f(k + n): moving to -z
    prev = np.tile(prof(k - 1.0).ravel(), 4)
    cur = np.tile(prof(k + 0.0).ravel(), 4)
    src = np.zeros_like(cur)
    nsteps = 18
    for n in range(1, nsteps + 1):
        nxt = orc.potential_step(g, prev, cur, src)
        prev, cur = cur, nxt
        got = cur.reshape(4, g["nz"], g["ny"], g["nx"])[:, :, 19:21, 19:21]
        expect = np.broadcast_to(prof(k + float(n))[:, 19:21, 19:21], got.shape)
        np.testing.assert_allclose(got, expect, atol=1e-13)


def test_uniform_source_closed_form(orc):
    # For a uniform source the scheme reduces to psi^{n+1} - 2 psi^n + psi^{n-1}
    # = (c dt)^2 S with S = mu0 J (A) or rho/eps0 (phi): psi^n = (c dt)^2 S n(n+1)/2
    # from zero initial levels, which is the leapfrog form of
    # psi(t) = c^2 S t^2 / 2, the solution of the physical Helmholtz equation.
    g = inputs.random_grid(0, 20, 20, 20, courant=0.9)
    n = g["nx"] * g["ny"] * g["nz"]
    J = np.array([3.0, -2.0, 5.0])
    rho = 7.0e-9
    src = np.concatenate([np.full(n, J[0]), np.full(n, J[1]), np.full(n, J[2]),
                          np.full(n, rho)])
    prev = np.zeros(4 * n)
    cur = np.zeros(4 * n)
    for _ in range(6):
        nxt = orc.potential_step(g, prev, cur, src)
        prev, cur = cur, nxt
    cdt2 = (C0 * g["dt"]) ** 2
    tri = 6 * 7 / 2
    got = cur.reshape(4, g["nz"], g["ny"], g["nx"])[:, 10, 10, 10]
    expect = cdt2 * tri * np.array([MU0 * J[0], MU0 * J[1], MU0 * J[2], rho / EPS0])
    np.testing.assert_allclose(got, expect, rtol=1e-12)
    assert got[3] > 0 and got[0] > 0  # physical sign


def test_space_charge_off_keeps_phi_zero(orc):
    g = inputs.random_grid(0, 10, 10, 10, space_charge=0)
    f = inputs.random_fields(3, g)
    f["prev"][3 * 1000:] = 0
    f["cur"][3 * 1000:] = 0
    nxt = orc.potential_step(g, f["prev"], f["cur"], f["src"])
    assert np.all(nxt[3 * 1000:] == 0.0)


def _second_diff(n, h):
    D = np.zeros((n, n))
    for a in range(1, n - 1):
        D[a, a - 1] = 1.0
        D[a, a] = -2.0
        D[a, a + 1] = 1.0
    return D / (h * h)


def _average_z(n, A):
    M = np.zeros((n, n))
    for a in range(1, n - 1):
        M[a, a - 1] = A
        M[a, a] = 1.0 - 2.0 * A
        M[a, a + 1] = A
    return M


@pytest.mark.parametrize("stencil", [0, 1])
def test_brute_force_operator_8cubed(orc, stencil):
    # Discrete Laplacian of Eq. updateEquation assembled from 1-D difference
    # matrices: x and y second differences of the z-weighted field
    # (Eq. NSFDtrick), plus the plain z second difference.  Index order
    # (k, j, i) with i fastest matches the host layout.
    g = inputs.random_grid(0, 8, 8, 8, stencil=stencil, courant=0.9 if stencil == 0 else 0.5)
    A = _nsfd_A(g) if stencil == 0 else 0.0
    Ix, Iy, Iz = np.eye(8), np.eye(8), np.eye(8)
    Mz = _average_z(8, A)
    L = (np.kron(Mz, np.kron(Iy, _second_diff(8, g["dx"])))
         + np.kron(Mz, np.kron(_second_diff(8, g["dy"]), Ix))
         + np.kron(_second_diff(8, g["dz"]), np.kron(Iy, Ix)))
    f = inputs.random_fields(5, g)
    n = 512
    nxt = orc.potential_step(g, f["prev"], f["cur"], f["src"])
    cdt2 = (C0 * g["dt"]) ** 2
    interior = np.zeros((8, 8, 8), bool)
    interior[1:-1, 1:-1, 1:-1] = True
    interior = interior.ravel()
    for c in range(4):
        pm = f["prev"][c * n:(c + 1) * n]
        p = f["cur"][c * n:(c + 1) * n]
        s = f["src"][c * n:(c + 1) * n] * (MU0 if c < 3 else 1.0 / EPS0)
        expect = 2 * p - pm + cdt2 * (L @ p + s)
        got = nxt[c * n:(c + 1) * n]
        np.testing.assert_allclose(got[interior], expect[interior],
                                   rtol=1e-11, atol=1e-11 * np.abs(expect).max())


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("boundary", [1, 2])
def test_mur_mirror_symmetry(orc, axis, boundary):
    g = dict(inputs.random_grid(0, 9, 10, 11), boundary=boundary)
    f = inputs.random_fields(7, g)
    shp = (4, g["nz"], g["ny"], g["nx"])
    ax = 3 - axis  # numpy axis of x/y/z in (comp, k, j, i)

    def sym(a):
        a = a.reshape(shp)
        return (0.5 * (a + np.flip(a, axis=ax))).ravel()

    prev, cur, src = sym(f["prev"]), sym(f["cur"]), sym(f["src"])
    for _ in range(4):
        nxt = orc.potential_step(g, prev, cur, src)
        prev, cur = cur, nxt
    a = cur.reshape(shp)
    np.testing.assert_allclose(a, np.flip(a, axis=ax), rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_mur_absorbs_outgoing_pulse(orc):
    # A smooth pulse, uniform in y and z, leaves through the +x face.  The
    # centre line is examined before the y and z faces can influence it (one
    # cell per step); a reflecting wall would send back a pulse of amplitude
    # ~1 there, the first-order Mur condition only a few per cent.
    g = dict(nx=40, ny=51, nz=51, dx=1.0e-4, dy=3.0e-4, dz=3.0e-4, x0=0.0, y0=0.0, z0=0.0,
             n_sub=1, stencil=1, space_charge=1)
    g["dt"] = 0.9 * g["dx"] / C0
    i, j, k = _coords(g)
    cdt = C0 * g["dt"]
    s = lambda t: np.exp(-0.5 * ((i * g["dx"] - 30 * g["dx"] - t) / (2.5 * g["dx"])) ** 2)  # noqa
    n = g["nx"] * g["ny"] * g["nz"]
    prev = np.tile(s(-cdt).ravel(), 4)
    cur = np.tile(s(0.0).ravel(), 4)
    src = np.zeros(4 * n)
    for _ in range(23):
        nxt = orc.potential_step(g, prev, cur, src)
        prev, cur = cur, nxt
    line = cur.reshape(4, g["nz"], g["ny"], g["nx"])[:, 25, 25, 20:39]
    left = np.abs(line).max()
    assert left < 0.05, left


def _oblique_reflection(orc, boundary, theta_deg, below):
    """A Gaussian wave packet (carrier 8 cells, envelope 8 cells along and 12
    across its direction) runs at theta to the normal of the k = 0 face.
    Returns the field over the original domain after the packet has met the
    face, on a grid that extends `below` planes beyond it, and the incident
    norm."""
    nx, ny, nz = 80, 40, 48
    h = 1.0e-4
    g = dict(nx=nx, ny=ny, nz=nz + below, dx=h, dy=h, dz=h, x0=0.0, y0=0.0, z0=0.0,
             dt=0.5 * h / C0, n_sub=1, stencil=1, space_charge=1, boundary=boundary)
    th = np.radians(theta_deg)
    k, j, i = np.meshgrid(np.arange(g["nz"]) - below, np.arange(ny), np.arange(nx),
                          indexing="ij")
    x, y, z = i - 20.0, j - (ny - 1) / 2.0, k - 30.0

    def packet(t):  # t: c t in cells
        s = np.sin(th) * x - np.cos(th) * z - t
        u = np.cos(th) * x + np.sin(th) * z
        return (np.exp(-(s / 8.0) ** 2 - (u / 12.0) ** 2 - (y / 12.0) ** 2)
                * np.cos(2 * np.pi * s / 8.0))

    n = g["nx"] * g["ny"] * g["nz"]
    zero = np.zeros(3 * n)
    prev = np.concatenate([packet(-0.5).ravel(), zero])
    cur = np.concatenate([packet(0.0).ravel(), zero])
    inc = np.linalg.norm(packet(0.0)[below:])
    src = np.zeros(4 * n)
    for _ in range(150):
        nxt = orc.potential_step(g, prev, cur, src)
        prev, cur = cur, nxt
    return cur[:n].reshape(g["nz"], ny, nx)[below:], inc


def test_mur_oblique_reflection_first_and_second_order(orc):
    # Reflection of a plane wave at incidence theta from the continuous
    # boundary operators (Engquist-Majda): first order
    # R1 = (1 - cos)/(1 + cos), second order R2 = R1^2 (0.172 and 0.029 at
    # 45 degrees).  The reflected field is the difference between runs on the
    # domain and on one extended 48 planes beyond the face (same boundary
    # order, so the other faces act alike in both).  A wrong sign of the
    # second-order tangential terms reflects more than the first order.
    c = np.cos(np.radians(45.0))
    r1_theory = (1 - c) / (1 + c)
    r = {}
    for b in (1, 2):
        ext, inc = _oblique_reflection(orc, b, 45.0, 48)
        dom, _ = _oblique_reflection(orc, b, 45.0, 0)
        r[b] = np.linalg.norm(dom - ext) / inc
    assert abs(r[1] - r1_theory) < 0.2 * r1_theory, r
    assert 0.5 * r1_theory ** 2 < r[2] < 1.5 * r1_theory ** 2, r
    assert r[2] < 0.3 * r[1], r
