"""GPU parity of the diagnostics (bunch sampling, bunching factor,
frequency-resolved power) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

pytestmark = pytest.mark.gpu


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


def _c1():
    w = inputs.workload("c1")
    return w, inputs.make_bunch(w["bunch_spec"], w["seed"])


@pytest.mark.parametrize("prec", ["P64", "P32"])
def test_bunch_stats_match_oracle(M, orc, prec):
    w, P = _c1()
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    kb = w["bunch_spec"]["kb"]
    o = orc.OracleSim(g, und, P)
    p = getattr(M, prec)
    rtol = 1e-11 if p == M.P64 else 2e-6
    with M.Simulation(g, und, P, precision=p) as sim:
        for steps in (0, 40):
            o.step(steps)
            sim.step(steps)
            got = sim.bunch_stats(kb)
            ref = o.bunch_stats(kb)
            assert got[13] == ref[13] == P["x"].size
            # positions and spreads relative to the bunch size, momenta to
            # their scale, the bunching factor absolutely
            for a in range(3):
                scale = ref[6 + a] + abs(ref[a])
                assert abs(got[a] - ref[a]) <= rtol * scale, (a, got[a], ref[a])
                assert abs(got[6 + a] - ref[6 + a]) <= rtol * scale, (a, got[6 + a], ref[6 + a])
            us = max(abs(ref[5]), 1e-30)
            for a in range(3, 6):
                assert abs(got[a] - ref[a]) <= 10 * rtol * us, (a, got[a], ref[a])
                assert abs(got[6 + a] - ref[6 + a]) <= 10 * rtol * us + 1e-3 * ref[6 + a]
            assert abs(got[12] - ref[12]) <= (1e-12 if p == M.P64 else 1e-5)


@pytest.mark.parametrize("prec", ["P64", "P32"])
def test_bunch_sampling_records_match_oracle(M, orc, prec):
    """Samples every 7 steps into 5 records: the steps they were taken at
    exactly, the statistics as mithra_bunch_stats within its tolerance."""
    w, P = _c1()
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    kb = w["bunch_spec"]["kb"]
    p = getattr(M, prec)
    rtol = 1e-11 if p == M.P64 else 2e-6
    o = orc.OracleSim(g, und, P)
    with M.Simulation(g, und, P, precision=p) as sim:
        sim.step(3)
        o.step(3)
        sim.set_bunch_sampling(kb, 7, 5)
        assert sim.read_bunch().shape == (0, 15)
        sim.step(47)                     # samples due at 10, 17, ..., 45, 52
        rec = sim.read_bunch()
        assert rec.shape == (5, 15)
        assert list(rec[:, 0]) == [10, 17, 24, 31, 38]
        now = 3
        for r in rec:
            o.step(int(r[0]) - now)
            now = int(r[0])
            ref = o.bunch_stats(kb)
            got = r[1:]
            assert got[13] == ref[13]
            for a in range(3):
                scale = ref[6 + a] + abs(ref[a])
                assert abs(got[a] - ref[a]) <= rtol * scale, (a, got[a], ref[a])
            assert abs(got[12] - ref[12]) <= (1e-12 if p == M.P64 else 1e-5)
        # a fresh request restarts the records; every = 0 stops them
        sim.set_bunch_sampling(kb, 1, 4)
        sim.step(2)
        assert list(sim.read_bunch()[:, 0]) == [51, 52]
        sim.set_bunch_sampling(kb, 0, 0)
        sim.step(1)
        assert sim.read_bunch().shape == (0, 15)
        with pytest.raises(M.MithraError):
            sim.set_bunch_sampling(kb, -1, 4)


def test_bunch_stats_empty_and_errors(M):
    g = dict(inputs.random_grid(0, 8, 8, 8), boundary=1)
    with M.Simulation(g, None, None) as sim:
        assert np.all(sim.bunch_stats(1.0) == 0.0)
        with pytest.raises(M.MithraError):
            sim.bunch_stats(float("nan"))


@pytest.mark.parametrize("prec", ["P64", "P32"])
def test_spectrum_matches_oracle(M, orc, prec):
    w, P = _c1()
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    kp = g["nz"] - 8
    lam_r = und["lambda_u"] * (1 + und["K"] ** 2 / 2) / (2 * 10.0 ** 2)
    lam = lam_r * np.array([0.8, 0.9, 1.0, 1.1, 1.25, 0.5, 1.0 / 3.0])
    o = orc.OracleSim(g, und, P)
    o.set_spectrum(kp, lam)
    p = getattr(M, prec)
    with M.Simulation(g, und, P, precision=p) as sim:
        sim.set_spectrum(kp, lam)
        o.step(w["steps"])
        sim.step(w["steps"])
        got, ns = sim.read_spectrum()
        ref = o.spectrum()
        assert ns == o.spec_samples == w["steps"]
        scale = np.abs(ref).max()
        assert scale > 0
        tol = 1e-9 if p == M.P64 else 1e-3
        assert np.abs(got - ref).max() <= tol * scale, (got, ref)
        # reading does not disturb the sums; stopping frees them
        again, _ = sim.read_spectrum()
        assert np.array_equal(again, got)
        sim.set_spectrum(kp, [])
        empty, ns0 = sim.read_spectrum()
        assert empty.size == 0 and ns0 == 0


def test_spectrum_argument_checks(M):
    w, P = _c1()
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    with M.Simulation(g, und, P) as sim:
        for kp, lam in ((0, [1e-4]), (g["nz"] - 1, [1e-4]), (5, [-1e-4]), (5, [0.0]),
                        (5, np.full(65, 1e-4))):
            with pytest.raises(M.MithraError) as e:
                sim.set_spectrum(kp, lam)
            assert e.value.status == M.EINVAL
