"""The library's bunch generator (mithra_make_bunch, Sec. "Electron Bunch
Generation"), host only, against closed forms:

  - the Halton loader is the radical inverse in the prime bases (first values
    of base 5 along z: 1/5, 2/5, 3/5, 4/5; textbook);
  - the Box-Muller maps (Eq. gaussian1D, Eq. gaussian2D) give the requested
    means and spreads, and the transverse truncation at radius R gives the
    truncated 2-D Gaussian's spread sigma^2 (1 - (1 + a^2/2) e^{-a^2/2}) /
    (1 - e^{-a^2/2}), a = R / sigma, with no particle beyond R;
  - a uniform profile (Eq. uniform1D) has mean (z_lo + z_hi)/2 and spread
    (z_hi - z_lo)/sqrt(12); the displacement for a bunching factor bf gives
    |<exp(i kb z)>| = J_1(2 bf) = bf (1 - bf^2/2 + ...) (the Halton loader's
    own bunching is far below the pseudo-random one's 1/sqrt(n));
  - the split-Gaussian head and tail hold the share of the particles that a
    Gaussian of the same peak density has, half on either side;
  - the c1 and c2 workload bunches (drawn by the test inputs with numpy)
    have the same moments as the library's, where both generators mean the
    same distribution (position means, z, u_z), and each one's transverse
    spread matches its own truncation (per axis there, radial here);
  - one seed gives one bunch; bad specs are refused.
"""
import math

import numpy as np
import pytest
from scipy.special import j1

from paper_1612_03310_gb300 import build_lib, inputs


@pytest.fixture(scope="module")
def M():
    build_lib.build()
    from paper_1612_03310_gb300 import mithra
    return mithra


def _trunc2d_sigma(sigma, R):
    a2 = (R / sigma) ** 2
    e = math.exp(-a2 / 2)
    return sigma * math.sqrt((1 - (1 + a2 / 2) * e) / (1 - e))


def _trunc1d_sigma(sigma, a):
    phi = math.exp(-a * a / 2) / math.sqrt(2 * math.pi)
    return sigma * math.sqrt(1 - 2 * a * phi / math.erf(a / math.sqrt(2)))


def test_halton_radical_inverse(M):
    b = M.make_bunch(4, 1e-12, sigma_x=0, sigma_y=0, z_lo=0.0, z_hi=1.0, uz_mean=0.0)
    np.testing.assert_allclose(b["z"], [0.2, 0.4, 0.6, 0.8], rtol=0, atol=1e-15)
    assert b["q_macro"] == pytest.approx(-0.25e-12)


@pytest.mark.parametrize("sequence", ["halton", "splitmix64"])
def test_moments_and_truncation(M, sequence):
    n = 1 << 17
    sx, sy, R = 2.0e-4, 3.0e-4, 6.0e-4
    b = M.make_bunch(n, 5e-12, sigma_x=sx, sigma_y=sy, trunc_r=0.0, x0=1e-5, y0=-2e-5,
                     z_lo=1e-3, z_hi=3e-3, uz_mean=0.3, uz_sigma=1e-4, ux_sigma=2e-3,
                     uy_sigma=3e-3, sequence=sequence, seed=7)
    tol = 5.0 / math.sqrt(n)  # five standard errors
    for k, m, s in (("x", 1e-5, sx), ("y", -2e-5, sy), ("ux", 0.0, 2e-3), ("uy", 0.0, 3e-3),
                    ("uz", 0.3, 1e-4)):
        assert abs(b[k].mean() - m) <= tol * s, k
        assert abs(b[k].std() / s - 1) <= 2 * tol, k
    assert abs(b["z"].mean() - 2e-3) <= tol * 2e-3 / math.sqrt(12)
    assert abs(b["z"].std() / (2e-3 / math.sqrt(12)) - 1) <= 2 * tol
    assert b["z"].min() >= 1e-3 and b["z"].max() <= 3e-3
    # radial truncation of a round beam
    t = M.make_bunch(n, 5e-12, sigma_x=sx, sigma_y=sx, trunc_r=R, z_lo=0, z_hi=1e-3,
                     uz_mean=0.3, sequence=sequence, seed=7)
    r = np.hypot(t["x"], t["y"])
    assert r.max() <= R
    assert abs(t["x"].std() / _trunc2d_sigma(sx, R) - 1) <= 2 * tol


def test_bunching_factor(M):
    kb = 2 * math.pi / 1.0e-5
    n = 1 << 16
    for bf in (0.0, 1e-3, 0.1):
        b = M.make_bunch(n, 1e-12, sigma_x=1e-4, sigma_y=1e-4, z_lo=0.0, z_hi=200e-5,
                         uz_mean=0.3, bf=bf, kb=kb)
        got = abs(np.exp(1j * kb * b["z"]).mean())
        # z - a sin(kb z) over whole periods: J_1(kb a) (Jacobi-Anger), = bf to
        # first order with a = 2 bf / kb
        assert abs(got - j1(2 * bf)) <= 5e-4, (bf, got)
    # the pseudo-random loader: shot noise of order 1/sqrt(n)
    b = M.make_bunch(n, 1e-12, sigma_x=1e-4, sigma_y=1e-4, z_lo=0.0, z_hi=200e-5, uz_mean=0.3,
                     sequence="splitmix64", seed=3)
    assert abs(np.exp(1j * kb * b["z"]).mean()) <= 5 / math.sqrt(n)


def test_split_gaussian_head_and_tail(M):
    n = 1 << 16
    L, s = 2e-3, 1e-4
    b = M.make_bunch(n, 1e-12, sigma_x=1e-4, sigma_y=1e-4, z_lo=0.0, z_hi=L, taper_sigma=s,
                     uz_mean=0.3)
    tail = math.sqrt(2 * math.pi) * s
    out = (b["z"] < 0) | (b["z"] > L)
    assert abs(out.sum() - n * tail / (L + tail)) <= 1
    assert abs((b["z"] < 0).sum() - (b["z"] > L).sum()) <= 0.02 * out.sum()
    # each half is a half Gaussian of rms s about its edge
    assert abs(np.sqrt(np.mean(b["z"][b["z"] < 0] ** 2)) / s - 1) <= 0.05


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_workload_moments_match_the_test_inputs(M, name):
    w = inputs.workload(name)
    sp = w["bunch_spec"]
    n = min(int(sp["n"]), 1 << 17)
    ref = inputs.make_bunch(dict(sp, n=n), w["seed"])
    sig, a = sp["sigma_r"], sp["trunc"]
    b = M.make_bunch(n, sp["charge"], sigma_x=sig, sigma_y=sig, trunc_r=a * sig,
                     z_lo=sp["z_lo"], z_hi=sp["z_hi"], uz_mean=sp["uz_mean"],
                     uz_sigma=sp["uz_sigma"], bf=sp["bf"], kb=sp["kb"],
                     sequence="splitmix64", seed=w["seed"])
    tol = 5.0 / math.sqrt(n)
    L = sp["z_hi"] - sp["z_lo"]
    for k, scale in (("x", sig), ("y", sig), ("z", L), ("uz", max(sp["uz_sigma"], 1e-30))):
        assert abs(b[k].mean() - ref[k].mean()) <= 2 * tol * scale, k
    assert abs(b["z"].std() / ref["z"].std() - 1) <= 3 * tol
    if sp["uz_sigma"] > 0:
        assert abs(b["uz"].std() / ref["uz"].std() - 1) <= 3 * tol
    # transverse spread: each generator's own truncation closed form
    assert abs(b["x"].std() / _trunc2d_sigma(sig, a * sig) - 1) <= 2 * tol
    assert abs(ref["x"].std() / _trunc1d_sigma(sig, a) - 1) <= 2 * tol
    assert b["q_macro"] == pytest.approx(ref["q_macro"] * 1.0, rel=1e-12) or n != sp["n"]


def test_seed_and_errors(M):
    kw = dict(sigma_x=1e-4, sigma_y=1e-4, z_lo=0, z_hi=1e-3, uz_mean=0.3, sequence="splitmix64")
    a = M.make_bunch(1000, 1e-12, seed=1, **kw)
    b = M.make_bunch(1000, 1e-12, seed=1, **kw)
    c = M.make_bunch(1000, 1e-12, seed=2, **kw)
    assert np.array_equal(a["x"], b["x"]) and not np.array_equal(a["x"], c["x"])
    for bad in (dict(n=0), dict(z_hi=-1.0), dict(bf=1.0, kb=1.0), dict(bf=0.1),
                dict(sigma_x=-1.0)):
        args = dict(n=10, charge=1e-12, **kw)
        args.update(bad)
        nn = args.pop("n")
        with pytest.raises(M.MithraError) as e:
            M.make_bunch(nn, args.pop("charge"), **args)
        assert e.value.status == M.EINVAL
    with pytest.raises(M.MithraError):  # a truncation radius far inside the core
        M.make_bunch(100, 1e-12, trunc_r=1e-9, **dict(kw, sigma_x=1.0, sigma_y=1.0))
