"""GPU parity: the CUDA path, called through the C ABI, against the FP64
oracle on the same seeded inputs.

Tolerances (relative L2 over a whole field, or per particle):
  - P64: 1e-10 for one step, 1e-9 over the c1 workload (rounding order only);
  - P32: the stated bound for FP32 state with FP64 bookkeeping, 1e-4 relative
    L2 for every field after the configured steps and 1e-3 for the radiated
    power; single steps are held to 1e-5.
Index work (the cell of every particle, the lost flags, the per-tile counts)
is compared exactly, except for particles within 1e-9 (P64) or 1e-5 (P32)
cells of a cell face, where rounding order may decide either way.
"""
import numpy as np
import pytest

from paper_1612_03310_gb300 import build_lib, inputs

pytestmark = pytest.mark.gpu

C0 = 299792458.0
FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Ax", "Ay", "Az", "phi", "Jx", "Jy", "Jz", "rho"]


@pytest.fixture(scope="module")
def M():
    build_lib.build()
    from paper_1612_03310_gb300 import mithra
    try:
        s = mithra.Simulation(dict(inputs.random_grid(0, 4, 4, 4), boundary=1), None, None)
        s.close()
    except mithra.MithraError as e:
        if e.status == mithra.ENODEV:
            pytest.skip("no GB300 device")
        raise
    return mithra


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def oracle_fields(o):
    """Fields of an OracleSim in the library's naming and (nz, ny, nx) shape."""
    g = o.g
    shp = (g["nz"], g["ny"], g["nx"])
    n = o.n_cell
    out = {}
    for a, nm in enumerate(("Ex", "Ey", "Ez")):
        out[nm] = o.E[a * n:(a + 1) * n].reshape(shp)
    for a, nm in enumerate(("Bx", "By", "Bz")):
        out[nm] = o.B[a * n:(a + 1) * n].reshape(shp)
    for a, nm in enumerate(("Ax", "Ay", "Az", "phi")):
        out[nm] = o.cur[a * n:(a + 1) * n].reshape(shp)
        out[nm + "_prev"] = o.prev[a * n:(a + 1) * n].reshape(shp)
    for a, nm in enumerate(("Jx", "Jy", "Jz", "rho")):
        out[nm] = o.src[a * n:(a + 1) * n].reshape(shp)
    return out


def set_state(sim, o, f):
    """Same potentials and sources on both sides (f from inputs.random_fields)."""
    n = o.n_cell
    o.set_potentials(f["prev"], f["cur"])
    o.set_sources(f["src"])
    for a, nm in enumerate(("Ax", "Ay", "Az", "phi")):
        sim.set_field(nm + "_prev", f["prev"][a * n:(a + 1) * n])
        sim.set_field(nm, f["cur"][a * n:(a + 1) * n])
    for a, nm in enumerate(("Jx", "Jy", "Jz", "rho")):
        sim.set_field(nm, f["src"][a * n:(a + 1) * n])


def as_f32(f):
    return {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}


def compare_fields(sim, o, tol, names=FIELDS, report=None):
    ref = oracle_fields(o)
    worst = {}
    for nm in names:
        got = sim.copy_field(nm)
        e = rel_l2(got, ref[nm])
        worst[nm] = e
    if report is not None:
        report.update(worst)
    bad = {k: v for k, v in worst.items() if v > tol}
    assert not bad, bad


def shell_mask(g, width=2):
    """Vertices within `width` of any face (the boundary vertices and the
    interior vertices their Mur updates read)."""
    k, j, i = np.meshgrid(np.arange(g["nz"]), np.arange(g["ny"]), np.arange(g["nx"]),
                          indexing="ij")
    return ((i < width) | (i >= g["nx"] - width) | (j < width) | (j >= g["ny"] - width) |
            (k < width) | (k >= g["nz"] - width))


def compare_vertices(sim, o, tol, mask, names):
    """Per-vertex check on a region: max |GPU - oracle| over the masked
    vertices, scaled by the field's largest value anywhere, so that an error
    confined to a few vertices (one boundary face, one injection plane) shows
    even where the whole-field L2 norm would hide it."""
    ref = oracle_fields(o)
    bad = {}
    for nm in names:
        r = ref[nm]
        scale = np.abs(r).max()
        if scale == 0.0:
            continue
        e = float(np.abs(sim.copy_field(nm) - r)[mask].max() / scale)
        if e > tol:
            bad[nm] = e
    assert not bad, bad


def compare_particles(sim, o, tol_cells, face_eps):
    got = sim.copy_particles()
    lost_o = o.lost.astype(bool)
    lost_g = got["lost"].astype(bool)
    assert np.array_equal(lost_o, lost_g)
    assert got["n_lost"] == int(lost_o.sum())
    keep = ~lost_o
    g = o.g
    for key, d, r0 in (("x", g["dx"], g["x0"]), ("y", g["dy"], g["y0"]), ("z", g["dz"], g["z0"])):
        a = (got[key][keep] - r0) / d
        b = (getattr(o, key)[keep] - r0) / d
        assert np.abs(a - b).max() <= tol_cells, (key, np.abs(a - b).max())
        near = np.abs(b - np.round(b)) < face_eps
        ca, cb = np.floor(a), np.floor(b)
        assert np.array_equal(ca[~near], cb[~near]), key
    for key in ("ux", "uy", "uz"):
        a = got[key][keep]
        b = getattr(o, key)[keep]
        scale = max(np.abs(b).max(), 1e-30)
        assert np.abs(a - b).max() <= tol_cells * 10 * scale + 1e-12, key


# ---------------------------------------------------------------------------
# potential update and Mur boundaries (no particles)

@pytest.mark.parametrize("prec,variant,lz", [
    ("P64", 0, 0), ("P64", 1, 0), ("P64", 1, 5), ("P64", 1, 1),
    ("P32", 0, 0), ("P32", 1, 0), ("P32", 1, 5), ("P32", 1, 1), ("P32", 2, 3),
    ("P32_C", 0, 0), ("P32_C", 2, 0), ("P32_C", 2, 5), ("P32_C", 2, 1), ("P64", 2, 7)])
@pytest.mark.parametrize("shape", [(37, 29, 45), (4, 4, 4), (33, 9, 70), (5, 41, 6), (70, 17, 9),
                                   (64, 10, 30), (32, 4, 12)])
@pytest.mark.parametrize("boundary", [1, 2])
def test_vacuum_update_parity(M, orc, prec, shape, variant, lz, boundary):
    # every form of the potential update (direct; z-marching TMA tiles with
    # several plane-chunk lengths, ragged tiles in x and y -- single-float
    # levels only; register z-marching), first- and second-order Mur with
    # random values on every boundary vertex; widths of whole 32-column
    # blocks (64, 32) beside the ragged ones, and y+ faces in the second row
    # of a block row (ny = 10) and in the first block row (ny = 4)
    nx, ny, nz = shape
    g = dict(inputs.random_grid(11, nx, ny, nz), boundary=boundary)
    f = inputs.random_fields(12, g)
    p = getattr(M, prec)
    if p != M.P64:
        f = as_f32(f)
    o = orc.OracleSim(g, None, dict(x=[], y=[], z=[], ux=[], uy=[], uz=[]))
    with M.Simulation(g, None, None, precision=p) as sim:
        sim.set_tuning(stencil_variant=variant, lz=lz)
        assert sim.tuning()["stencil_variant"] == variant
        set_state(sim, o, f)
        for steps, tol in ((1, 1e-12 if p == M.P64 else 2e-6), (14, 1e-11 if p == M.P64 else 2e-5)):
            o.step(steps)
            sim.step(steps)
            sim.sync()
            compare_fields(sim, o, tol, names=["Ax", "Ay", "Az", "phi", "Ex", "Ey", "Ez",
                                               "Bx", "By", "Bz"])
            # the boundary shell vertex by vertex (Mur faces, edges, corners)
            compare_vertices(sim, o, 20 * tol, shell_mask(g),
                             ["Ax", "Ay", "Az", "phi", "Ax_prev", "phi_prev", "Ex", "Bz"])
            ref = oracle_fields(o)
            for nm in ("Ax_prev", "phi_prev"):
                assert rel_l2(sim.copy_field(nm), ref[nm]) <= tol


# ---------------------------------------------------------------------------
# one full PIC step from random fields and particles

C1_UND = inputs.WORKLOADS["c1"]["undulator"]


@pytest.mark.parametrize("prec", ["P64", "P32", "P32_U64", "P32_C"])
@pytest.mark.parametrize("n_sub", [1, 3])
@pytest.mark.parametrize("push_variant,sparse_below", [(0, 0), (1, 0), (1, 60), (1, 1 << 30)])
def test_pic_step_parity(M, orc, prec, n_sub, push_variant, sparse_below):
    # per-particle and tiled particle kernels; n_sub = 3 lets sub-steps leave
    # the tile (gather from global memory); the 36 x 30 x 40 grid has ragged
    # tiles in every axis.  About 60 particles per tile: sparse_below = 60
    # sends part of the tiles to the per-warp path from the second step on,
    # 2^30 all of them.
    g = inputs.random_grid(21, 36, 30, 40, n_sub=n_sub)
    f = inputs.random_fields(22, g, scale=1e-9)
    P = inputs.random_particles(23, g, 6000, u_scale=0.3)
    und = dict(C1_UND, z_ent_lab=0.0)
    p = getattr(M, prec)
    if p != M.P64:
        f = as_f32(f)
    o = orc.OracleSim(g, und, P)
    with M.Simulation(dict(g, boundary=1), und, P, precision=p) as sim:
        sim.set_tuning(push_variant=push_variant, push_sparse_below=sparse_below)
        # rho^{1/2} from the initial positions agrees before anything else
        ref = oracle_fields(o)
        assert rel_l2(sim.copy_field("rho"), ref["rho"]) <= (1e-13 if p == M.P64 else 1e-6)
        set_state(sim, o, f)
        tol_f = 1e-10 if p == M.P64 else 1e-5
        tol_c = 1e-10 if p == M.P64 else 2e-5
        for steps in (1, 2):
            o.step(steps)
            sim.step(steps)
            sim.sync()
            compare_fields(sim, o, tol_f)
            compare_particles(sim, o, tol_c, 1e-9 if p == M.P64 else 1e-5)


@pytest.mark.parametrize("prec", ["P64", "P32"])
def test_lost_particles_flagged(M, orc, prec):
    g = inputs.random_grid(31, 16, 16, 16)
    # three particles heading out through x, y and z faces, one staying
    P = dict(x=np.array([g["x0"] + 12.9 * g["dx"], g["x0"] + 7.5 * g["dx"],
                         g["x0"] + 7.5 * g["dx"], g["x0"] + 7.5 * g["dx"]]),
             y=np.array([g["y0"] + 7.5 * g["dy"], g["y0"] + 1.05 * g["dy"],
                         g["y0"] + 7.5 * g["dy"], g["y0"] + 7.5 * g["dy"]]),
             z=np.array([g["z0"] + 7.5 * g["dz"], g["z0"] + 7.5 * g["dz"],
                         g["z0"] + 12.95 * g["dz"], g["z0"] + 7.5 * g["dz"]]),
             ux=np.array([5.0, 0.0, 0.0, 0.0]), uy=np.array([0.0, -5.0, 0.0, 0.0]),
             uz=np.array([0.0, 0.0, 5.0, 0.1]), q_macro=-1e-15)
    o = orc.OracleSim(g, None, P)
    with M.Simulation(dict(g, boundary=1), None, P, precision=getattr(M, prec)) as sim:
        for _ in range(3):
            o.step(1)
            sim.step(1)
        got = sim.copy_particles()
        assert list(got["lost"]) == list(o.lost) == [1, 1, 1, 0]
        assert got["n_lost"] == 3
        compare_fields(sim, o, 1e-10 if prec == "P64" else 1e-5, names=["rho", "Jx", "Jz"])


@pytest.mark.parametrize("prec", ["P64", "P32_U64"])
def test_strict_lost_policy(M, prec):
    # the three escaping particles of test_lost_particles_flagged: by default
    # they are flagged and counted; in strict mode the first synchronising
    # call after the step that loses them reports MITHRA_ELOST, the next step
    # enqueues nothing, and the state shows which particles left
    g = inputs.random_grid(31, 16, 16, 16)
    P = dict(x=np.array([g["x0"] + 12.9 * g["dx"], g["x0"] + 7.5 * g["dx"]]),
             y=np.array([g["y0"] + 7.5 * g["dy"], g["y0"] + 7.5 * g["dy"]]),
             z=np.array([g["z0"] + 7.5 * g["dz"], g["z0"] + 7.5 * g["dz"]]),
             ux=np.array([5.0, 0.0]), uy=np.array([0.0, 0.0]), uz=np.array([0.0, 0.1]),
             q_macro=-1e-15)
    with M.Simulation(dict(g, boundary=1), None, P, precision=getattr(M, prec)) as sim:
        sim.set_lost_policy(True)
        sim.step(1)
        sim.sync()  # nothing lost yet
        sim.step(2)
        with pytest.raises(M.MithraError) as e:
            sim.sync()
        assert e.value.status == M.ELOST
        assert "1 particle(s) left" in str(e.value)
        with pytest.raises(M.MithraError) as e:
            sim.step(1)
        assert e.value.status == M.ELOST
        assert sim.time()[0] == 3
        got = sim.copy_particles()  # the state is kept
        assert list(got["lost"]) == [1, 0]
        sim.set_lost_policy(False)  # back to counting only
        sim.step(1)
        sim.sync()
    with M.Simulation(dict(g, boundary=1), None, P, precision=getattr(M, prec)) as sim:
        sim.step(3)
        sim.sync()
        assert sim.copy_particles()["n_lost"] == 1


@pytest.mark.parametrize("prec", ["P64", "P32"])
def test_initially_outside_particles_are_lost(M, orc, prec):
    g = inputs.random_grid(41, 12, 12, 12)
    P = inputs.random_particles(42, g, 100)
    P["x"][:10] = g["x0"] + 0.5 * g["dx"]  # cell 0: outside the valid region
    P["z"][10:20] = g["z0"] + 11.5 * g["dz"]  # beyond the last vertex
    o = orc.OracleSim(g, None, P)
    with M.Simulation(dict(g, boundary=1), None, P, precision=getattr(M, prec)) as sim:
        got = sim.copy_particles()
        assert got["n_lost"] == o.n_lost == 20
        assert np.array_equal(got["lost"], o.lost)
        o.step(2)
        sim.step(2)
        compare_particles(sim, o, 1e-10 if prec == "P64" else 2e-5, 1e-5)


# ---------------------------------------------------------------------------
# the c1 workload end to end (200 steps), power recorded every step

@pytest.mark.parametrize("prec,push_variant,sparse_below,boundary", [
    ("P64", 1, 0, 1), ("P32", 1, 0, 1), ("P32_U64", 1, 0, 1), ("P64", 0, 0, 1), ("P32", 0, 0, 1),
    ("P32", 1, 256, 1), ("P64", 1, 256, 1), ("P64", 1, 0, 2), ("P32", 1, 0, 2),
    ("P32_C", 1, 0, 1)])
def test_workload_c1(M, orc, prec, push_variant, sparse_below, boundary):
    w = inputs.workload("c1")
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    g, und = dict(w["grid"], boundary=boundary), w["undulator"]
    kp = g["nz"] - 8
    p = getattr(M, prec)
    o = orc.OracleSim(g, und, P)
    with M.Simulation(g, und, P, precision=p) as sim:
        sim.set_tuning(push_variant=push_variant, push_sparse_below=sparse_below)
        sim.set_power_sampling(kp, w["steps"])
        o.step(w["steps"], power_plane=kp)
        sim.step(w["steps"])
        sim.sync()
        errs = {}
        compare_fields(sim, o, 1e-9 if p == M.P64 else 1e-4, report=errs)
        rec = sim.read_power()
        assert rec.shape == (w["steps"], 3)
        po = np.array([[s.p_lab, s.t_lab, s.z_lab] for s in o.power])
        scale = np.abs(po[:, 0]).max()
        assert scale > 0
        assert np.abs(rec[:, 0] - po[:, 0]).max() <= (1e-9 if p == M.P64 else 1e-3) * scale
        np.testing.assert_allclose(rec[:, 1:], po[:, 1:], rtol=1e-13)
        compare_particles(sim, o, 1e-8 if p == M.P64 else 1e-3, 1e-9 if p == M.P64 else 1e-3)
        # one-off power at the same plane equals the last record
        p1, t1, z1 = sim.radiated_power(kp)
        assert p1 == pytest.approx(rec[-1, 0], rel=1e-12, abs=1e-30)
        assert t1 == pytest.approx(rec[-1, 1], rel=1e-14)


@pytest.mark.parametrize("prec", ["P64", "P32"])
def test_workload_c2_full_size(M, orc, prec):
    # c2 at its full size (128x128x1024 cells, 2^21 particles) in the launch
    # configuration the bench times, two whole steps, every field and particle
    w = inputs.workload("c2")
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    g, und = w["grid"], w["undulator"]
    p = getattr(M, prec)
    o = orc.OracleSim(g, und, P)
    with M.Simulation(dict(g, boundary=1), und, P, precision=p) as sim:
        ref = oracle_fields(o)
        assert rel_l2(sim.copy_field("rho"), ref["rho"]) <= (1e-13 if p == M.P64 else 1e-6)
        o.step(2)
        sim.step(2)
        sim.sync()
        compare_fields(sim, o, 1e-10 if p == M.P64 else 1e-5)
        compare_particles(sim, o, 1e-10 if p == M.P64 else 2e-5, 1e-9 if p == M.P64 else 1e-5)


def test_sample_fields_match_copy(M):
    g = inputs.random_grid(51, 20, 18, 22)
    f = inputs.random_fields(52, g)
    with M.Simulation(dict(g, boundary=1), None, None, precision=M.P64) as sim:
        n = 20 * 18 * 22
        for a, nm in enumerate(("Ax", "Ay", "Az", "phi")):
            sim.set_field(nm + "_prev", f["prev"][a * n:(a + 1) * n])
            sim.set_field(nm, f["cur"][a * n:(a + 1) * n])
        sim.step(2)
        rng = np.random.default_rng(0)
        pts = np.stack([rng.integers(0, 20, 50), rng.integers(0, 18, 50),
                        rng.integers(0, 22, 50)], axis=1)
        names = ["Ex", "By", "Az", "rho", "phi"]
        s = sim.sample_fields(names, pts)
        for c, nm in enumerate(sorted(names, key=lambda x: M.FIELD_ID[x])):
            full = sim.copy_field(nm)
            np.testing.assert_array_equal(s[:, c], full[pts[:, 2], pts[:, 1], pts[:, 0]])


def test_empty_bunch_and_time(M, orc):
    g = inputs.random_grid(61, 10, 10, 10)
    with M.Simulation(dict(g, boundary=1), C1_UND, None, precision=M.P64) as sim:
        sim.step(5)
        n, t = sim.time()
        assert n == 5 and t == pytest.approx(5 * g["dt"])
        assert np.abs(sim.copy_field("Ax")).max() == 0.0


def test_torch_stream(M):
    torch = pytest.importorskip("torch")
    g = inputs.random_grid(71, 12, 12, 12)
    P = inputs.random_particles(72, g, 500)
    s = torch.cuda.Stream()
    with M.Simulation(dict(g, boundary=1), C1_UND, P, precision=M.P32,
                      stream=s.cuda_stream) as sim, \
            M.Simulation(dict(g, boundary=1), C1_UND, P, precision=M.P32) as ref:
        sim.step(3)
        ref.step(3)
        s.synchronize()
        assert rel_l2(sim.copy_field("rho"), ref.copy_field("rho")) < 1e-5


def test_autotuned_choice_matches_default(M, tmp_path, monkeypatch):
    from paper_1612_03310_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE_DIR", str(tmp_path))
    g = dict(inputs.random_grid(81, 40, 36, 48), boundary=1)
    P = inputs.random_particles(82, g, 3000)
    best = autotune.tune(g, C1_UND, P, M.P32, steps=2, warmup=1)
    st = {(c["stencil_variant"], c["lz"]) for c in autotune.stencil_candidates(g)}
    assert (best["stencil_variant"], best["lz"]) in st
    assert best["push_variant"] in (0, 1)
    with M.Simulation(g, C1_UND, P, precision=M.P32) as a, \
            M.Simulation(g, C1_UND, P, precision=M.P32) as b:
        b.set_tuning(**best)
        a.step(6)
        b.step(6)
        for nm in ("Ax", "Ez", "rho", "Jx"):
            assert rel_l2(b.copy_field(nm), a.copy_field(nm)) < 1e-5, nm


# ---------------------------------------------------------------------------
# optical undulator (plane wave along z)

def optical_c1(signal="flat-top", direction=-1, pol=(0.0, 1.0)):
    """c1's frame with the paper's equivalent optical undulator: a0 = K,
    lambda0 = 2 lambda_u, its rise two wavelengths ahead of the bunch."""
    u = inputs.WORKLOADS["c1"]["undulator"]
    lam = 2 * u["lambda_u"]
    return dict(type="optical", gamma0=u["gamma0"], a0=u["K"], lambda_l=lam, polarization=pol,
                z0_lab=0.0, offset=0.0325 + 2 * lam, variance=lam, cep=0.3,
                direction=direction, signal=signal)


@pytest.mark.parametrize("prec", ["P64", "P32"])
@pytest.mark.parametrize("signal", ["neumann", "gaussian", "secant-hyperbolic", "flat-top"])
@pytest.mark.parametrize("push_variant", [0, 1])
def test_optical_pic_step_parity(M, orc, prec, signal, push_variant):
    g = inputs.random_grid(51, 36, 30, 40, n_sub=2)
    f = inputs.random_fields(52, g, scale=1e-9)
    P = inputs.random_particles(53, g, 3000, u_scale=0.3)
    und = dict(optical_c1(signal, pol=(0.6, 0.8)), offset=0.0)
    p = getattr(M, prec)
    if p != M.P64:
        f = as_f32(f)
    o = orc.OracleSim(g, und, P)
    with M.Simulation(dict(g, boundary=1), und, P, precision=p) as sim:
        sim.set_tuning(push_variant=push_variant)
        set_state(sim, o, f)
        for steps in (1, 2):
            o.step(steps)
            sim.step(steps)
            sim.sync()
            compare_fields(sim, o, 1e-10 if p == M.P64 else 1e-5)
            compare_particles(sim, o, 1e-10 if p == M.P64 else 2e-5, 1e-9 if p == M.P64 else 1e-5)


@pytest.mark.parametrize("prec,direction", [("P64", -1), ("P32", -1), ("P64", 1)])
def test_workload_c1_optical(M, orc, prec, direction):
    w = inputs.workload("c1")
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    g, und = dict(w["grid"], boundary=1), optical_c1(direction=direction)
    kp = g["nz"] - 8
    p = getattr(M, prec)
    o = orc.OracleSim(g, und, P)
    with M.Simulation(g, und, P, precision=p) as sim:
        sim.set_power_sampling(kp, w["steps"])
        o.step(w["steps"], power_plane=kp)
        sim.step(w["steps"])
        sim.sync()
        compare_fields(sim, o, 1e-9 if p == M.P64 else 1e-4)
        rec = sim.read_power()
        po = np.array([s.p_lab for s in o.power])
        scale = np.abs(po).max()
        assert scale > 0
        assert np.abs(rec[:, 0] - po).max() <= (1e-9 if p == M.P64 else 1e-3) * scale
        compare_particles(sim, o, 1e-8 if p == M.P64 else 1e-3, 1e-9 if p == M.P64 else 1e-3)
        if direction < 0:
            # the counter-propagating laser drives the bunch: transverse
            # momenta of order a0
            got = sim.copy_particles()
            assert np.abs(got["uy"]).max() > 0.3 * und["a0"]


def test_workload_c3_first_step_sampled(M, orc):
    # c3 at its full size (256x256x2048 cells, 2^24 particles) in the launch
    # configuration the bench tunes, P32: outputs the oracle computes one by
    # one.  Before the first step rho^{1/2} is the deposit of the bunch; after
    # it, with zero potential levels -1 and 0 and J^0 = 0, phi^1 =
    # (c dt)^2 rho^{1/2} / eps0 and A^1 = 0 at interior vertices, the grid E, B
    # at t = dt/2 vanish, and every particle has made one Boris step in the
    # undulator field alone.
    from paper_1612_03310_gb300 import autotune
    w = inputs.workload("c3")
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    nz, ny, nx = g["nz"], g["ny"], g["nx"]
    rng = np.random.default_rng(9)
    pts = np.stack([rng.integers(1, nz - 1, 2000), rng.integers(1, ny - 1, 2000),
                    rng.integers(1, nx - 1, 2000)], axis=1)
    o_rho = orc.deposit_rho(g, P["q_macro"], P["x"], P["y"], P["z"])   # (nz, ny, nx)
    eps0 = 8.8541878128e-12
    cdt2 = (C0 * g["dt"]) ** 2
    with M.Simulation(g, und, P, precision=M.P32) as sim:
        autotune.apply(sim, g, und, P, M.P32)
        rho = sim.copy_field("rho")
        assert rel_l2(rho, o_rho) <= 1e-6
        sim.step(1)
        phi = sim.copy_field("phi")
        got = phi[pts[:, 0], pts[:, 1], pts[:, 2]]
        want = cdt2 * o_rho[pts[:, 0], pts[:, 1], pts[:, 2]] / eps0
        scale = np.abs(cdt2 * o_rho / eps0).max()
        assert np.abs(got - want).max() <= 1e-6 * scale
        del phi, rho
        for nm in ("Ax", "Ay", "Az"):
            assert np.abs(sim.copy_field(nm)[1:-1, 1:-1, 1:-1]).max() == 0.0
        parts = sim.copy_particles()
    # one Boris step per sampled particle in the undulator field at t = dt/2
    qm = -1.602176634e-19 / 9.1093837015e-31
    sel = np.arange(0, P["x"].size, 4096)
    for q in sel:
        u = np.array([P["ux"][q], P["uy"][q], P["uz"][q]])
        E, B = orc.undulator_field(und, P["y"][q], P["z"][q], 0.5 * g["dt"])
        u1 = orc.boris(u, E, B, qm, g["dt"])
        v = C0 * u1 / np.sqrt(1 + u1 @ u1)
        for a, key in enumerate(("ux", "uy", "uz")):
            assert parts[key][q] == pytest.approx(u1[a], rel=2e-6, abs=2e-6 * max(abs(u1[2]), 1e-30))
        for a, (key, d) in enumerate((("x", "dx"), ("y", "dy"), ("z", "dz"))):
            r1 = P[key][q] + v[a] * g["dt"]
            assert abs(parts[key][q] - r1) <= 2e-5 * g[d]


# ---------------------------------------------------------------------------
# source tiles: the particle step marks the 27 tiles around every tile that
# holds particles, and the z-marching update then skips the others' sources

def expected_marked_tiles(g, P):
    """Tiles of the 27-neighbourhoods of the tiles holding particles at P."""
    ntx, nty, ntz = -(-g["nx"] // 8), -(-g["ny"] // 8), -(-g["nz"] // 8)
    keep = P["lost"] == 0
    cell = [np.floor((P[c][keep] - g[c + "0"]) / g["d" + c] + 1e-9).astype(np.int64) // 8
            for c in ("x", "y", "z")]
    flags = np.zeros((ntz + 2, nty + 2, ntx + 2), dtype=bool)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                flags[cell[2] + 1 + dz, cell[1] + 1 + dy, cell[0] + 1 + dx] = True
    return int(flags[1:-1, 1:-1, 1:-1].sum())


@pytest.mark.parametrize("prec,push_variant,sparse_below", [
    ("P32_U64", 1, 16), ("P64", 1, 0), ("P32", 1, 1 << 30), ("P32", 0, 0)])
def test_source_tiles_marked(M, orc, prec, push_variant, sparse_below):
    w = inputs.workload("c1")
    P0 = inputs.make_bunch(w["bunch_spec"], w["seed"])
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    o = orc.OracleSim(g, und, P0)
    with M.Simulation(g, und, P0, precision=getattr(M, prec)) as sim:
        sim.set_tuning(push_variant=push_variant, push_sparse_below=sparse_below)
        # the initial deposit marks no tiles: both parities read every source
        assert sim.source_tiles()[1]
        sim.step(1)
        assert sim.source_tiles()[1]
        sim.step(2)
        P = sim.copy_particles()
        sim.step(1)
        sim.sync()
        marked, everywhere = sim.source_tiles()
        if push_variant == 0:
            assert everywhere  # the per-particle form marks no tiles
        else:
            assert not everywhere
            assert marked == expected_marked_tiles(g, P)
        # the skipped sources were zero: the fields still follow the oracle
        o.step(4)
        for _ in range(3):
            sim.step(1)
            o.step(1)
        sim.sync()
        compare_fields(sim, o, 1e-10 if prec == "P64" else 1e-4)
