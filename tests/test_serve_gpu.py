"""Served form on the GPU: jobs that arrive while others run are admitted
into the running batch; every job's radiated-power record and final fields
equal those of the same job run alone, within the parity tolerances.  The
jobs are small, so the batch takes the fused form (one launch per phase for
all jobs) in its automatic mode."""
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


@pytest.mark.parametrize("prec_name", ["P32", "P32_U64"])
def test_same_alone_and_in_the_mix(M, prec_name):
    from paper_1612_03310_gb300 import serve
    prec = getattr(M, prec_name)
    rng = np.random.default_rng(3)
    jobs = []
    for k, (nx, nz, n, steps, arr) in enumerate([(32, 128, 20000, 60, 0), (40, 192, 30000, 90, 0),
                                                 (24, 128, 8000, 40, 25), (48, 128, 50000, 33, 50)]):
        j = inputs._job(rng, nx, nz, n, steps, k)
        j["arrival"] = arr
        jobs.append(j)
    srv = serve.Server(hbm_budget=8 << 30, max_slots=8, tick_steps=16, clock="steps",
                       keep_fields=("Ey", "Ax", "rho"), precision=prec)
    st = srv.run(jobs)
    assert st["completed"] == 4
    assert st["fused_captures"] >= 1 and st["graph_captures"] >= st["fused_captures"]
    for js in st["done"]:
        spec = js.spec
        g = dict(spec["grid"], boundary=1)
        with M.Simulation(g, spec["undulator"], inputs.make_bunch(spec["bunch_spec"], spec["seed"]),
                          precision=prec) as alone:
            if srv.tuning:
                alone.set_tuning(**srv.tuning)
            alone.set_power_sampling(g["nz"] - 8, spec["steps"])
            alone.step(spec["steps"])
            p = alone.read_power()
            assert p.shape == js.power.shape
            scale = np.abs(p[:, 0]).max()
            assert np.abs(p[:, 0] - js.power[:, 0]).max() <= 1e-3 * scale
            for nm, v in js.fields.items():
                ref = alone.copy_field(nm)
                assert np.linalg.norm(v - ref) <= 1e-4 * np.linalg.norm(ref), nm
