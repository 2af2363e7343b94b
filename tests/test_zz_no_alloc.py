"""The allocation-free power entry point (mithra_plane_power_noalloc), for
callers that cannot call cudaMalloc (graph capture, a host framework's own
allocator, a real-time loop): called through the C ABI on device arrays the
test owns, and checked against mithra_radiated_power, the entry point that
uses the simulation's own scratch, on two calls in a row.

This file sorts last so that a run stopping at its first failure has run
every other test before it."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

pytestmark = pytest.mark.gpu

TOL = {"P64": 1e-9, "P32": 1e-3}  # the power tolerances of the parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    build_lib.build()
    from paper_1612_03310_gb300 import mithra
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch, mithra


def device_levels(torch, sim, prec_name):
    """Newest level and increment of a simulation, in the library's layout,
    as device tensors owned by the caller."""
    new = np.stack([sim.copy_field(n) for n in ("Ax", "Ay", "Az", "phi")], axis=-1)
    old = np.stack([sim.copy_field(n) for n in ("Ax_prev", "Ay_prev", "Az_prev", "phi_prev")],
                   axis=-1)
    dt = np.float64 if prec_name == "P64" else np.float32
    psi = torch.from_numpy(np.ascontiguousarray(new.astype(dt))).cuda()
    inc = torch.from_numpy(np.ascontiguousarray((new - old).astype(dt))).cuda()
    torch.cuda.synchronize()
    return psi, inc


@pytest.mark.parametrize("prec_name", ["P64", "P32"])
def test_noalloc_power_matches(env, prec_name):
    torch, M = env
    w = inputs.workload("c1")
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    prec = getattr(M, prec_name)
    kp = g["nz"] - 8
    with M.Simulation(g, und, P, precision=prec) as sim:
        for steps in (60, 25):  # two calls in a row, at different states
            sim.step(steps)
            sim.sync()
            ref, _, _ = sim.radiated_power(kp)
            psi, inc = device_levels(torch, sim, prec_name)
            got = M.plane_power_noalloc(g, und["gamma0"], prec, psi.data_ptr(), inc.data_ptr(), kp)
            assert ref != 0.0
            assert abs(got - ref) <= TOL[prec_name] * abs(ref), (got, ref)


def test_noalloc_rejects_too_many_rows(env):
    torch, M = env
    g = dict(inputs.random_grid(0, 4, 8193, 4), boundary=1)
    with pytest.raises(M.MithraError) as e:
        M.plane_power_noalloc(g, 10.0, M.P32, 16, 16, 1)
    assert e.value.status == M.EINVAL
    assert "8192" in M.last_error()
