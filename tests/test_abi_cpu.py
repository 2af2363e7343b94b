"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/mithra.h declares, and its host-only validation agrees with the
stability conditions the oracle derives from the paper's dispersion
relations."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def M():
    build_lib.build()
    from paper_1612_03310_gb300 import mithra
    return mithra


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mithra.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mithra_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(M):
    names = declared_symbols()
    assert len(names) >= 15
    lib = C.CDLL(M.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(M.EXPORTS) == names


def test_version(M):
    assert M.lib().mithra_version() >= 100


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("courant", [0.5, 0.9, 0.99, 1.0, 1.01, 1.3])
def test_stability_check_matches_oracle(M, orc, stencil, courant):
    g = inputs.random_grid(0, 8, 8, 8, courant=courant, stencil=stencil, dz_over_dx=0.6)
    _, unstable = orc.coefficients(g)
    st = M.check_grid(dict(g, boundary=1))
    assert (st == M.EUNSTABLE) == unstable
    assert st in (M.OK, M.EUNSTABLE)


def test_bad_grids_rejected(M):
    g = inputs.random_grid(0, 8, 8, 8)
    assert M.check_grid(dict(g, boundary=2)) == M.check_grid(dict(g, boundary=1)) == M.OK
    for bad in (dict(nx=3), dict(dx=0.0), dict(n_sub=0), dict(stencil=2), dict(boundary=0),
                dict(boundary=3)):
        assert M.check_grid({**g, "boundary": 1, **bad}) == M.EINVAL, bad
        assert M.last_error()


def test_footprint_scales(M):
    g = inputs.workload("c2")["grid"]
    b32 = M.footprint(g, 2 ** 21, M.P32)
    b64 = M.footprint(g, 2 ** 21, M.P64)
    ncell = 128 * 128 * 1024
    assert b32 > 3 * ncell * 16
    assert 1.6 < b64 / b32 < 2.0
    # compensated levels: the lo parts of both levels (4 bfloat16 per vertex)
    assert M.footprint(g, 2 ** 21, M.P32_C) == b32 + 2 * ncell * 8


def test_create_without_gpu_fails_loudly(M):
    pytest.importorskip("torch")
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = inputs.random_grid(0, 8, 8, 8)
    with pytest.raises(M.MithraError) as e:
        M.Simulation(dict(g, boundary=1), None, None)
    assert e.value.status == M.ENODEV


def test_binding_refuses_missing_library(monkeypatch):
    from paper_1612_03310_gb300 import mithra
    monkeypatch.setattr(mithra, "_lib", None)
    monkeypatch.setattr(mithra, "LIB_PATH", "/nonexistent/libmithra.so")
    with pytest.raises(mithra.MithraError):
        mithra.lib()


def test_workload_table_pinned():
    # the rest-frame literals of the workload table against the closed forms
    # of the Lorentz-boost section (gamma0 = gamma / sqrt(1 + K^2/2), the
    # boosted mean momentum and spread) and the grid recipe (c dt = rest-frame
    # period / steps per period, dz = c dt / 0.95)
    c = 299792458.0
    for name, gamma, spp in (("c1", 10.0, 32), ("c2", 100.0, 50), ("c3", 100.0, 100)):
        w = inputs.WORKLOADS[name]
        u, g, b = w["undulator"], w["grid"], w["bunch"]
        g0 = gamma / np.sqrt(1 + u["K"] ** 2 / 2)
        assert u["gamma0"] == pytest.approx(g0, rel=1e-13)
        b0 = np.sqrt(1 - 1 / g0 ** 2)
        beta = np.sqrt(1 - 1 / gamma ** 2)
        gr = gamma * g0 * (1 - beta * b0)
        assert b["uz_mean"] == pytest.approx(np.sqrt(gr * gr - 1), rel=1e-12)
        assert b["uz_sigma"] == pytest.approx(gamma * 1e-4 * g0 * (1 - beta * b0), rel=1e-12)
        cdt = u["lambda_u"] / g0 / spp
        assert g["dt"] * c == pytest.approx(cdt, rel=1e-13)
        assert g["dz"] == pytest.approx(cdt / 0.95, rel=1e-13)
        assert b["kb"] == pytest.approx(g0 * 2 * np.pi / u["lambda_u"] * (1 + b0), rel=1e-12)


def test_division_by_invariant_multiplication():
    # the cell-index decode divides by nx and nx*ny as floor(n m / 2^64) with
    # m = floor((2^64 - 1) / d) + 1 (Granlund and Montgomery); check the
    # identity on grid-sized divisors and the extreme dividends
    import random
    rng = random.Random(0)
    divs = [4, 5, 7, 8, 31, 32, 33, 127, 128, 129, 160, 256, 1000, 4096, 25600, 65536, 65537,
            131071, 2 ** 20 - 3]
    for d in divs:
        m = ((1 << 64) - 1) // d + 1
        ns = [0, 1, d - 1, d, d + 1, 2 ** 31 - 1, 2 ** 31 - 2] + [rng.randrange(2 ** 31)
                                                                   for _ in range(2000)]
        for n in ns:
            assert (n * m) >> 64 == n // d, (n, d)


def test_normalized_wavelengths():
    """Frequencies normalised to the radiation wavelength map to lab
    wavelengths lambda_r / f, both ends included."""
    from paper_1612_03310_gb300 import mithra
    lam = mithra.normalized_wavelengths(2.0e-6, 0.9, 1.1, 0.05)
    assert lam.size == 5
    assert np.allclose(2.0e-6 / lam, [0.9, 0.95, 1.0, 1.05, 1.1])


def test_boost_from_lab_reproduces_the_workloads(M):
    """The host helper mithra_boost_from_lab against the workload table's
    rest-frame numbers (themselves pinned to the Lorentz-boost closed forms
    above): the frame, the time step and cell, the beam's momentum moments and
    the bunching wavenumber; bad cases refused."""
    c = 299792458.0
    for name, gamma, spp in (("c1", 10.0, 32), ("c2", 100.0, 50), ("c3", 100.0, 100)):
        w = inputs.WORKLOADS[name]
        u, g, b = w["undulator"], w["grid"], w["bunch"]
        r = M.boost_from_lab(gamma, u["lambda_u"], u["K"], spp, 0.95, sigma_gamma_rel=1e-4)
        assert r["gamma0"] == pytest.approx(u["gamma0"], rel=1e-13)
        assert r["dt"] == pytest.approx(g["dt"], rel=1e-13)
        assert r["dz"] == pytest.approx(g["dz"], rel=1e-13)
        assert r["uz_mean"] == pytest.approx(b["uz_mean"], rel=1e-12)
        assert r["uz_sigma"] == pytest.approx(b["uz_sigma"], rel=1e-12)
        assert r["k_b"] == pytest.approx(b["kb"], rel=1e-12)
        assert r["lambda_r_lab"] == pytest.approx(
            u["lambda_u"] * (1 + u["K"] ** 2 / 2) / (2 * gamma ** 2), rel=1e-14)
        assert r["dt"] * c * spp * r["gamma0"] == pytest.approx(u["lambda_u"], rel=1e-13)
    for bad in (dict(gamma=1.0), dict(courant=1.5), dict(steps_per_period=0),
                dict(lambda_u=-0.01)):
        args = dict(gamma=10.0, lambda_u=0.015, K=1.0, steps_per_period=32, courant=0.95)
        args.update(bad)
        with pytest.raises(M.MithraError):
            M.boost_from_lab(**args)
