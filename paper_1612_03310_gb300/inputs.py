"""Seeded synthetic inputs, shared by the CUDA path's tests and bench and by the
oracle.

This module holds none of the method's arithmetic.  The workloads are written
out as rest-frame numbers (cell sizes, time step, frame Lorentz factor, bunch
extent and momentum moments); how each number was chosen is recorded with the
design notes, and a CPU test re-derives them from the closed forms of the
paper's Lorentz-boost section.  A bunch is drawn from numpy's PCG64 generator
by affine maps of uniform and normal draws; the optional longitudinal density
modulation is a sinusoidal displacement of the drawn positions.
"""
from __future__ import annotations

import numpy as np

# Rest-frame workloads shaped like the paper's Example 1 (IR SASE FEL).
#   c1: 32x32x64 cells, 4096 particles, 200 steps, gamma = 10, K = 1.0,
#       lambda_u = 1.5 cm, Courant 0.95 along z, 32 steps per rest-frame period.
#   c2: 128x128x1024 cells, 2^21 particles, 5000 steps, gamma = 100, K = 1.4,
#       lambda_u = 3 cm, 100 lab periods, 50 steps per rest-frame period,
#       1e-3 density modulation at the rest-frame ponderomotive wavenumber.
#   c3: c2's physics at 256x256x2048 cells (cells halved), 2^24 particles.
WORKLOADS: dict[str, dict] = {
    "c1": dict(
        grid=dict(nx=32, ny=32, nz=64, dx=1.0e-4, dy=1.0e-4, dz=6.043149036471656e-05,
                  dt=1.9149886634733397e-13, n_sub=1, stencil=0, space_charge=1),
        undulator=dict(gamma0=8.16496580927726, lambda_u=0.015, K=1.0,
                       z_ent_lab=0.03868421052631579, length_lab=0.0, fringe=1),
        bunch=dict(n=4096, charge=1.0e-12, sigma_r=2.0e-4, trunc=3.0,
                   z_lo=0.000966903845835465, z_hi=0.002900711537506395,
                   uz_mean=0.20541217207146906, uz_sigma=0.00010208791115676327,
                   ut_sigma=0.0, bf=0.0, kb=6814.517844753226),
        steps=200, seed=1),
    "c2": dict(
        grid=dict(nx=128, ny=128, nz=1024, dx=25.0e-6, dy=25.0e-6, dz=8.887103544928604e-06,
                  dt=2.8161977202515795e-14, n_sub=1, stencil=0, space_charge=1),
        undulator=dict(gamma0=71.06690545187014, lambda_u=0.03, K=1.4,
                       z_ent_lab=0.5150526315789474, length_lab=3.0, fringe=1),
        bunch=dict(n=2097152, charge=29.5e-12, sigma_r=260.0e-6, trunc=3.0,
                   z_lo=0.0022750985075017226, z_hi=0.006825295522505168,
                   uz_mean=0.348253782693193, uz_sigma=0.00010589054240866452,
                   ut_sigma=0.0, bf=1.0e-3, kb=29766.962133610756),
        steps=5000, seed=2),
    "c3": dict(
        grid=dict(nx=256, ny=256, nz=2048, dx=12.5e-6, dy=12.5e-6, dz=4.443551772464302e-06,
                  dt=1.4080988601257897e-14, n_sub=1, stencil=0, space_charge=1),
        undulator=dict(gamma0=71.06690545187014, lambda_u=0.03, K=1.4,
                       z_ent_lab=0.5150526315789474, length_lab=3.0, fringe=1),
        bunch=dict(n=16777216, charge=29.5e-12, sigma_r=260.0e-6, trunc=3.0,
                   z_lo=0.0022750985075017226, z_hi=0.006825295522505168,
                   uz_mean=0.348253782693193, uz_sigma=0.00010589054240866452,
                   ut_sigma=0.0, bf=1.0e-3, kb=29766.962133610756),
        steps=5000, seed=3),
}


def centred_grid(grid: dict) -> dict:
    """The grid with its vertex (0,0,0) placed so that the transverse centre is
    on the undulator axis (x = y = 0) and z starts at 0."""
    g = dict(grid)
    g["x0"] = -0.5 * (g["nx"] - 1) * g["dx"]
    g["y0"] = -0.5 * (g["ny"] - 1) * g["dy"]
    g["z0"] = 0.0
    return g


def workload(name: str) -> dict:
    w = WORKLOADS[name]
    return dict(grid=centred_grid(w["grid"]), undulator=dict(w["undulator"]),
                bunch_spec=dict(w["bunch"]), steps=w["steps"], seed=w["seed"])


def _truncated_normal(rng: np.random.Generator, n: int, sigma: float, trunc: float) -> np.ndarray:
    out = rng.standard_normal(n)
    bad = np.abs(out) > trunc
    while bad.any():
        out[bad] = rng.standard_normal(int(bad.sum()))
        bad = np.abs(out) > trunc
    return sigma * out


def make_bunch(spec: dict, seed: int) -> dict:
    """Rest-frame bunch: transverse Gaussian (truncated), uniform z in
    [z_lo, z_hi] with an optional sinusoidal displacement of amplitude
    2 bf / kb, Gaussian momenta.  Returns float64 arrays and the signed
    macroparticle charge (electrons)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(spec["n"])
    x = _truncated_normal(rng, n, spec["sigma_r"], spec["trunc"])
    y = _truncated_normal(rng, n, spec["sigma_r"], spec["trunc"])
    z = spec["z_lo"] + (spec["z_hi"] - spec["z_lo"]) * rng.random(n)
    if spec.get("bf", 0.0) > 0.0:
        z = z - (2.0 * spec["bf"] / spec["kb"]) * np.sin(spec["kb"] * z)
    ux = spec.get("ut_sigma", 0.0) * rng.standard_normal(n)
    uy = spec.get("ut_sigma", 0.0) * rng.standard_normal(n)
    uz = spec["uz_mean"] + spec["uz_sigma"] * rng.standard_normal(n)
    return dict(x=x, y=y, z=z, ux=ux, uy=uy, uz=uz, q_macro=-spec["charge"] / n)


# ---------------------------------------------------------------------------
# Generic random states for parity tests (not physical bunches).

def random_grid(seed: int, nx: int, ny: int, nz: int, courant: float = 0.95,
                stencil: int = 0, n_sub: int = 1, space_charge: int = 1,
                dx: float = 1.0e-4, dz_over_dx: float = 0.6) -> dict:
    """A grid with dz = dz_over_dx * dx, dy = 0.9 dx and c dt = courant * dz."""
    dz = dz_over_dx * dx
    dy = 0.9 * dx
    c = 299792458.0
    g = dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, dt=courant * dz / c, n_sub=n_sub,
             stencil=stencil, space_charge=space_charge)
    return centred_grid(g)


def random_fields(seed: int, grid: dict, scale: float = 1.0e-6) -> dict:
    """Two potential levels and a source array with smooth-plus-noise content,
    each 4 components in the (comp, nz, ny, nx) layout, float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = grid["nx"] * grid["ny"] * grid["nz"]
    prev = scale * rng.standard_normal(4 * n)
    cur = prev + 0.1 * scale * rng.standard_normal(4 * n)
    src = np.concatenate([1.0e3 * rng.standard_normal(3 * n), 1.0e-6 * rng.standard_normal(n)])
    return dict(prev=prev, cur=cur, src=src)


def random_particles(seed: int, grid: dict, n: int, u_scale: float = 0.3,
                     margin_cells: float = 1.5) -> dict:
    """Uniform positions inside the valid particle region (cells [1, n-3]
    in each axis, kept margin_cells away from its faces), Gaussian momenta."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def axis(nv, d, r0):
        lo = r0 + (1.0 + margin_cells) * d
        hi = r0 + (nv - 2.0 - margin_cells) * d
        return lo + (hi - lo) * rng.random(n)

    x = axis(grid["nx"], grid["dx"], grid["x0"])
    y = axis(grid["ny"], grid["dy"], grid["y0"])
    z = axis(grid["nz"], grid["dz"], grid["z0"])
    u = u_scale * rng.standard_normal((3, n))
    return dict(x=x, y=y, z=z, ux=u[0].copy(), uy=u[1].copy(), uz=u[2].copy(),
                q_macro=-1.0e-15)


# ---------------------------------------------------------------------------
# Design-sweep jobs for the batched (c4) and served (c5) forms, drawn directly
# in rest-frame terms: frame Lorentz factor gamma0, undulator K, lambda_u =
# 3 cm, 50 steps per rest-frame undulator period (c dt = lambda_u / gamma0 /
# 50), dz = c dt / 0.95, dx = dy = 3 dz; the undulator fills the lab from
# z' = 0 on (no entrance inside the run); transverse Gaussian bunch of
# sigma = nx dx / 12 (cut at 3 sigma), uniform z over the central half,
# rest-frame drift u_z in [0.2, 0.4].

def _job(rng: np.random.Generator, nx: int, nz: int, n_particles: int, steps: int,
         jid: int) -> dict:
    c = 299792458.0
    lam_u = 0.03
    gamma0 = float(rng.uniform(15.0, 160.0))
    K = float(rng.uniform(0.5, 2.0))
    cdt = lam_u / gamma0 / 50.0
    dz = cdt / 0.95
    dx = 3.0 * dz
    grid = centred_grid(dict(nx=nx, ny=nx, nz=nz, dx=dx, dy=dx, dz=dz, dt=cdt / c, n_sub=1,
                             stencil=0, space_charge=1))
    und = dict(gamma0=gamma0, lambda_u=lam_u, K=K, z_ent_lab=0.0, length_lab=0.0, fringe=1)
    bunch = dict(n=int(n_particles), charge=10.0e-12, sigma_r=nx * dx / 12.0, trunc=3.0,
                 z_lo=0.25 * nz * dz, z_hi=0.75 * nz * dz,
                 uz_mean=float(rng.uniform(0.2, 0.4)), uz_sigma=1.0e-4, ut_sigma=0.0,
                 bf=1.0e-3, kb=4.0 * np.pi * gamma0 / lam_u)
    return dict(jid=jid, grid=grid, undulator=und, bunch_spec=bunch, steps=int(steps),
                seed=int(rng.integers(1 << 30)))


def batch_jobs(n_jobs: int = 64, steps: int = 1000, seed: int = 4) -> list[dict]:
    """c4: grids nx = ny in {48, 64, 80, 96, 112, 128}, nz = 4 nx, with 64-512
    particles per cell column (log-uniform)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for k in range(n_jobs):
        nx = int(rng.choice([48, 64, 80, 96, 112, 128]))
        ppc = float(np.exp(rng.uniform(np.log(64.0), np.log(512.0))))
        jobs.append(_job(rng, nx, 4 * nx, int(ppc * nx * nx), steps, k))
    return jobs


def uniform_jobs(n_jobs: int, nx: int, nz: int, n_particles: int, steps: int = 1000,
                 seed: int = 9) -> list[dict]:
    """n_jobs design-sweep jobs of one size (nx = ny, nz, n_particles) with
    the physics drawn as for c4 and c5: many small members of a batch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [_job(rng, nx, nz, n_particles, steps, k) for k in range(n_jobs)]


def serve_jobs(n_jobs: int, rate: float, seed: int = 5) -> list[dict]:
    """c5: Poisson arrivals at `rate` jobs/s; nx = ny in [32, 160], nz in
    [128, 1024] (multiples of 64), 1e3-4e6 particles (log-uniform), 500-5000
    steps.  Each job carries its arrival time in seconds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    jobs = []
    for k in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        nx = int(rng.integers(32, 161))
        nz = 64 * int(rng.integers(2, 17))
        npart = int(np.exp(rng.uniform(np.log(1.0e3), np.log(4.0e6))))
        steps = int(rng.integers(500, 5001))
        j = _job(rng, nx, nz, npart, steps, k)
        j["arrival"] = t
        jobs.append(j)
    return jobs


def describe(name: str) -> str:
    w = WORKLOADS[name]
    g = w["grid"]
    return (f"{name}: {g['nx']}x{g['ny']}x{g['nz']} cells, {w['bunch']['n']} particles, "
            f"{w['steps']} steps")


__all__ = ["WORKLOADS", "workload", "make_bunch", "random_grid", "random_fields", "uniform_jobs",
           "random_particles", "centred_grid", "describe", "batch_jobs", "serve_jobs"]
