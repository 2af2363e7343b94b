"""The allocation-free power entry point (mithra_plane_power_noalloc), for
callers that cannot call cudaMalloc (an operator inside a framework whose
caching allocator owns the device memory, a real-time loop): called through
the C ABI on device arrays the test owns, and checked against
mithra_radiated_power, the entry point that uses the simulation's own
scratch, on two calls in a row, on the legacy default stream and on a stream
the caller created, for every precision form (the compensated ones with and
without their lo parts), and for a grid with fewer rows right after one with
more, so that rows a previous call left in the shared scratch array are never
read.

This file sorts last so that a run stopping at its first failure has run
every other test before it."""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

pytestmark = pytest.mark.gpu

# the power tolerances of the parity tests: FP64 rounding order, and the FP32
# forms' bound (the test's increment is newest minus previous level formed
# from the copied-out levels, which differs from the library's stored
# increment by the rounding of a float difference)
TOL = {"P64": 1e-9, "P32": 1e-3, "P32_C": 1e-3, "P32_U64": 1e-3}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    build_lib.build()
    from paper_1612_03310_gb300 import mithra
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch, mithra


def device_levels(torch, sim, prec_name):
    """Newest level (hi part, and for the compensated forms the bfloat16 lo
    part) and increment of a simulation, in the library's layout, as device
    tensors owned by the caller."""
    new = np.stack([sim.copy_field(n) for n in ("Ax", "Ay", "Az", "phi")], axis=-1)
    old = np.stack([sim.copy_field(n) for n in ("Ax_prev", "Ay_prev", "Az_prev", "phi_prev")],
                   axis=-1)
    dt = np.float64 if prec_name == "P64" else np.float32
    hi = new.astype(dt)
    psi = torch.from_numpy(np.ascontiguousarray(hi)).cuda()
    inc = torch.from_numpy(np.ascontiguousarray((new - old).astype(dt))).cuda()
    lo = None
    if prec_name in ("P32_C", "P32_U64"):
        # copy_field returns hi + lo exactly, hi the nearest float, so the
        # remainder is the bfloat16 lo part (its conversion is exact)
        rest = torch.from_numpy(np.ascontiguousarray((new - hi).astype(np.float32)))
        lo = rest.to(torch.bfloat16).contiguous().cuda()
    torch.cuda.synchronize()
    return psi, lo, inc


def call(M, torch, g, gamma0, prec, psi, lo, inc, kp, stream=None):
    return M.plane_power_noalloc(g, gamma0, prec, psi.data_ptr(), inc.data_ptr(), kp,
                                 stream=stream, lo_newest_ptr=None if lo is None else lo.data_ptr())


@pytest.mark.parametrize("prec_name", ["P64", "P32", "P32_C", "P32_U64"])
def test_noalloc_power_matches(env, prec_name):
    torch, M = env
    w = inputs.workload("c1")
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    prec = getattr(M, prec_name)
    kp = g["nz"] - 8
    side = torch.cuda.Stream()
    with M.Simulation(g, und, P, precision=prec) as sim:
        # two calls in a row, at different states: the first on the legacy
        # default stream, the second on a stream the caller created
        for steps, stream in ((60, None), (25, side.cuda_stream)):
            sim.step(steps)
            sim.sync()
            ref, _, _ = sim.radiated_power(kp)
            psi, lo, inc = device_levels(torch, sim, prec_name)
            got = call(M, torch, g, und["gamma0"], prec, psi, lo, inc, kp, stream)
            assert ref != 0.0
            assert abs(got - ref) <= TOL[prec_name] * abs(ref), (got, ref)
            if lo is not None:
                # without the lo parts E and B lose their share: still within
                # the FP32 power bound on this workload
                hi_only = call(M, torch, g, und["gamma0"], prec, psi, None, inc, kp, stream)
                assert abs(hi_only - ref) <= TOL[prec_name] * abs(ref), (hi_only, ref)


@pytest.mark.parametrize("prec_name", ["P64", "P32"])
def test_noalloc_fewer_rows_after_more(env, prec_name):
    """A call on a grid of 40 rows, then one on a grid of 9 rows: the second
    must use only the rows it wrote (the first left 38 partial sums behind)."""
    torch, M = env
    prec = getattr(M, prec_name)
    und = inputs.workload("c1")["undulator"]
    for seed, (nx, ny, nz) in ((1, (24, 40, 12)), (2, (20, 9, 10))):
        g = dict(inputs.random_grid(seed, nx, ny, nz), boundary=1)
        f = inputs.random_fields(seed, g)
        n = nx * ny * nz
        with M.Simulation(g, und, None, precision=prec) as sim:
            for a, nm in enumerate(("Ax", "Ay", "Az", "phi")):
                sim.set_field(nm + "_prev", f["prev"][a * n:(a + 1) * n])
                sim.set_field(nm, f["cur"][a * n:(a + 1) * n])
            kp = nz // 2
            ref, _, _ = sim.radiated_power(kp)
            psi, lo, inc = device_levels(torch, sim, prec_name)
            got = call(M, torch, g, und["gamma0"], prec, psi, lo, inc, kp)
        assert ref != 0.0
        assert abs(got - ref) <= TOL[prec_name] * abs(ref), (ny, got, ref)


def test_noalloc_rejects_too_many_rows(env):
    torch, M = env
    g = dict(inputs.random_grid(0, 4, 8193, 4), boundary=1)
    with pytest.raises(M.MithraError) as e:
        M.plane_power_noalloc(g, 10.0, M.P32, 16, 16, 1)
    assert e.value.status == M.EINVAL
    assert "8192" in M.last_error()


def test_noalloc_rejects_lo_for_single_float_levels(env):
    torch, M = env
    g = dict(inputs.random_grid(0, 8, 8, 8), boundary=1)
    with pytest.raises(M.MithraError) as e:
        M.plane_power_noalloc(g, 10.0, M.P32, 16, 16, 1, lo_newest_ptr=16)
    assert e.value.status == M.EINVAL
