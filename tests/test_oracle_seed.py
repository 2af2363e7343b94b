"""Oracle pins of the seed field (Sec. "Seed Field"), injected by the
total-field/scattered-field planes k = 2 (scattered) and k = 3 (total):

  - at c dt = dz the NSFD scheme moves a wave uniform in x and y exactly one
    cell per step, so in vacuum the total-field region holds the incident
    vector potential f(z_k, t_n) to rounding and the scattered-field region
    stays zero, while the lateral faces cannot reach the centre columns;
  - the injected wave is the seed itself, not its negative (the sign of the
    corrections: the scattered-field plane loses the incident part its
    total-field neighbours contribute, the total-field plane gains the part
    its scattered-field neighbours lack);
  - switching the seed off leaves the vacuum at zero.
"""
import numpy as np
import pytest

from paper_1612_03310_gb300 import inputs

C0 = 299792458.0


def _seed_grid():
    return dict(inputs.random_grid(0, 64, 64, 64, courant=1.0, stencil=0, dz_over_dx=0.5),
                z0=0.0)


CENTRE = 40  # step at which the pulse centre reaches the total-field plane


def _seed(g, signal="gaussian", pol=(0.0, 1.0), gamma0=3.0):
    b0 = np.sqrt(1 - 1 / gamma0 ** 2)
    lam_rest = 16 * g["dz"]
    lam_lab = lam_rest / (gamma0 * (1 + b0))   # a forward wave is red-shifted
    # envelope width 8 steps at a fixed point; the pulse starts 5 widths away
    tv = 0.5 * lam_lab / C0
    tau = gamma0 * (1 - b0) * (CENTRE * g["dt"] - 3 * g["dz"] / C0)
    return dict(gamma0=gamma0, a0=1e-3, lambda_l=lam_lab, polarization=pol, z0_lab=0.0,
                offset=C0 * tau, variance=C0 * tv, cep=0.4, direction=1, signal=signal)


@pytest.mark.parametrize("signal", ["gaussian", "neumann", "flat-top"])
@pytest.mark.parametrize("pol", [(0.0, 1.0), (0.6, 0.8)])
def test_seed_enters_the_total_field_region_exactly(orc, signal, pol):
    g = _seed_grid()
    seed = _seed(g, signal, pol)
    o = orc.OracleSim(g, None, dict(x=[], y=[], z=[], ux=[], uy=[], uz=[]))
    o.set_seed(seed)
    nsteps = CENTRE + 16
    o.step(nsteps)
    nz = g["nz"]
    a0m = seed["a0"] * 9.1093837015e-31 * C0 / 1.602176634e-19
    ref = np.array([orc.incident_potential(seed, g["z0"] + k * g["dz"], nsteps * g["dt"])
                    for k in range(nz)])                      # (nz, 2)
    assert np.abs(ref[3:]).max() > 0.3 * a0m                  # the pulse is inside
    for c in range(2):
        col = o.potential(c)[:, 30:34, 30:34]                 # centre columns
        tf = col[3:nz - 1]
        np.testing.assert_allclose(tf, np.broadcast_to(ref[3:nz - 1, c, None, None], tf.shape),
                                   rtol=0, atol=1e-9 * a0m)
        assert np.abs(col[:3]).max() <= 1e-9 * a0m          # scattered field: nothing
    for c in (2, 3):  # A_z and phi untouched
        assert np.abs(o.potential(c)).max() == 0.0


def test_no_seed_no_field(orc):
    g = _seed_grid()
    o = orc.OracleSim(g, None, dict(x=[], y=[], z=[], ux=[], uy=[], uz=[]))
    o.set_seed(_seed(g))
    o.set_seed(None)
    o.step(5)
    assert np.abs(o.cur).max() == 0.0
