"""Thin ctypes binding of the C ABI in include/mithra.h (argument marshalling
only; every step of the time loop runs in the CUDA library).

The library is loaded from ``_build/libmithra.so`` inside this package; when it
is missing the binding raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libmithra.so")

OK, EINVAL, EUNSTABLE, ENOMEM, ECUDA, ENUMERIC, ELOST, EBUSY, ENODEV = range(9)
P64, P32, P32_U64, P32_C = 0, 1, 2, 3
FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Ax", "Ay", "Az", "Jx", "Jy", "Jz", "phi", "rho",
          "Ax_prev", "Ay_prev", "Az_prev", "phi_prev"]
FIELD_ID = {name: i for i, name in enumerate(FIELDS)}

# every symbol include/mithra.h declares
EXPORTS = ["mithra_create", "mithra_step", "mithra_sync", "mithra_time", "mithra_copy_field",
           "mithra_set_field", "mithra_sample_fields", "mithra_radiated_power",
           "mithra_set_power_sampling", "mithra_read_power", "mithra_copy_particles",
           "mithra_destroy", "mithra_last_error", "mithra_check_grid", "mithra_footprint",
           "mithra_version", "mithra_profile", "mithra_kernel_times", "mithra_kernel_name",
           "mithra_source_tiles",
           "mithra_set_tuning", "mithra_get_tuning", "mithra_plane_power_noalloc",
           "mithra_batch_create", "mithra_batch_add", "mithra_batch_remove", "mithra_batch_step",
           "mithra_batch_sync", "mithra_batch_size", "mithra_batch_last_error",
           "mithra_batch_destroy", "mithra_bunch_stats", "mithra_set_spectrum",
           "mithra_read_spectrum", "mithra_set_seed", "mithra_set_bunch_sampling",
           "mithra_read_bunch", "mithra_snapshot_bytes", "mithra_snapshot", "mithra_restore",
           "mithra_boost_from_lab", "mithra_make_bunch", "mithra_set_lost_policy",
           "mithra_batch_set_mode", "mithra_batch_get_mode", "mithra_batch_stats"]


class MithraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mithra status {status}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dt", C.c_double), ("n_sub", C.c_int32), ("stencil", C.c_int32),
                ("boundary", C.c_int32), ("space_charge", C.c_int32)]


class Undulator(C.Structure):
    _fields_ = [("gamma0", C.c_double), ("lambda_u", C.c_double), ("K", C.c_double),
                ("z_ent_lab", C.c_double), ("length_lab", C.c_double), ("fringe", C.c_int32),
                ("type", C.c_int32), ("a0", C.c_double), ("lambda_l", C.c_double),
                ("pol_x", C.c_double), ("pol_y", C.c_double), ("z0_lab", C.c_double),
                ("offset", C.c_double), ("variance", C.c_double), ("cep", C.c_double),
                ("direction", C.c_int32), ("signal", C.c_int32), ("beam", C.c_int32),
                ("x0_lab", C.c_double), ("y0_lab", C.c_double), ("w_par", C.c_double),
                ("w_perp", C.c_double)]


SIGNALS = {"neumann": 0, "gaussian": 1, "secant-hyperbolic": 2, "flat-top": 3}
BEAMS = {"plane-wave": 0, "gaussian-beam": 1}


class Tuning(C.Structure):
    _fields_ = [("stencil_variant", C.c_int32), ("lz", C.c_int32), ("push_variant", C.c_int32),
                ("push_ctas_per_sm", C.c_int32), ("push_sparse_below", C.c_int32)]


class Bunch(C.Structure):
    _fields_ = [("n", C.c_int64), ("q_macro", C.c_double),
                ("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("z", C.POINTER(C.c_double)), ("ux", C.POINTER(C.c_double)),
                ("uy", C.POINTER(C.c_double)), ("uz", C.POINTER(C.c_double))]


class BunchSpec(C.Structure):
    _fields_ = [("n", C.c_int64), ("charge", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double), ("sigma_x", C.c_double), ("sigma_y", C.c_double),
                ("trunc_r", C.c_double), ("z_lo", C.c_double), ("z_hi", C.c_double),
                ("taper_sigma", C.c_double), ("ux_sigma", C.c_double), ("uy_sigma", C.c_double),
                ("uz_mean", C.c_double), ("uz_sigma", C.c_double), ("bf", C.c_double),
                ("kb", C.c_double), ("sequence", C.c_int32), ("seed", C.c_uint64)]


_lib = None


def lib():
    """Loads libmithra.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise MithraError(ENODEV, f"CUDA library missing at {LIB_PATH}: run "
                                  "__graft_entry__.build() (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    st = C.c_int
    L.mithra_create.argtypes = [C.POINTER(Grid), C.POINTER(Undulator), C.POINTER(Bunch), C.c_int,
                                vp, C.POINTER(vp)]
    L.mithra_step.argtypes = [vp, C.c_int64]
    L.mithra_sync.argtypes = [vp]
    L.mithra_time.argtypes = [vp, C.POINTER(C.c_int64), dp]
    L.mithra_copy_field.argtypes = [vp, C.c_int32, dp]
    L.mithra_set_field.argtypes = [vp, C.c_int32, dp]
    L.mithra_sample_fields.argtypes = [vp, C.c_uint32, C.POINTER(C.c_int32), C.c_int64, dp]
    L.mithra_radiated_power.argtypes = [vp, C.c_int32, dp, dp, dp]
    L.mithra_set_power_sampling.argtypes = [vp, C.c_int32, C.c_int64]
    L.mithra_read_power.argtypes = [vp, dp, C.c_int64, C.POINTER(C.c_int64)]
    L.mithra_copy_particles.argtypes = [vp, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int64)]
    L.mithra_destroy.argtypes = [vp]
    L.mithra_last_error.argtypes = [vp]
    L.mithra_last_error.restype = C.c_char_p
    L.mithra_check_grid.argtypes = [C.POINTER(Grid)]
    L.mithra_footprint.argtypes = [C.POINTER(Grid), C.c_int64, C.c_int, C.POINTER(C.c_int64)]
    L.mithra_version.restype = C.c_int32
    L.mithra_profile.argtypes = [vp, C.c_int32]
    L.mithra_kernel_times.argtypes = [vp, dp, C.POINTER(C.c_int64), C.c_int32,
                                      C.POINTER(C.c_int32)]
    L.mithra_source_tiles.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    L.mithra_kernel_name.argtypes = [C.c_int32]
    L.mithra_kernel_name.restype = C.c_char_p
    L.mithra_plane_power_noalloc.argtypes = [C.POINTER(Grid), C.c_double, C.c_int, vp, vp, vp,
                                             C.c_int32, dp, vp]
    L.mithra_batch_create.argtypes = [vp, C.POINTER(vp)]
    L.mithra_batch_add.argtypes = [vp, vp]
    L.mithra_batch_remove.argtypes = [vp, vp]
    L.mithra_batch_step.argtypes = [vp, C.c_int64]
    L.mithra_batch_sync.argtypes = [vp]
    L.mithra_batch_size.argtypes = [vp]
    L.mithra_batch_size.restype = C.c_int32
    L.mithra_batch_last_error.argtypes = [vp]
    L.mithra_batch_last_error.restype = C.c_char_p
    L.mithra_batch_destroy.argtypes = [vp]
    L.mithra_make_bunch.argtypes = [C.POINTER(BunchSpec), dp, dp, dp, dp, dp, dp, dp]
    L.mithra_set_lost_policy.argtypes = [vp, C.c_int32]
    L.mithra_batch_set_mode.argtypes = [vp, C.c_int32]
    L.mithra_batch_get_mode.argtypes = [vp, C.POINTER(C.c_int32)]
    L.mithra_batch_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), dp]
    L.mithra_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.mithra_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    for name in EXPORTS:
        if name not in ("mithra_last_error", "mithra_version", "mithra_kernel_name",
                        "mithra_batch_size", "mithra_batch_last_error"):
            getattr(L, name).restype = st
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_grid(g: dict) -> Grid:
    return Grid(int(g["nx"]), int(g["ny"]), int(g["nz"]), g["dx"], g["dy"], g["dz"],
                g.get("x0", 0.0), g.get("y0", 0.0), g.get("z0", 0.0), g["dt"],
                int(g.get("n_sub", 1)), int(g.get("stencil", 0)), int(g.get("boundary", 1)),
                int(g.get("space_charge", 1)))


class LabCase(C.Structure):
    _fields_ = [("gamma", C.c_double), ("sigma_gamma_rel", C.c_double),
                ("lambda_u", C.c_double), ("K", C.c_double),
                ("steps_per_period", C.c_int32), ("courant", C.c_double)]


class RestFrame(C.Structure):
    _fields_ = [("gamma0", C.c_double), ("beta0", C.c_double), ("dt", C.c_double),
                ("dz", C.c_double), ("uz_mean", C.c_double), ("uz_sigma", C.c_double),
                ("k_b", C.c_double), ("lambda_r_lab", C.c_double)]


def boost_from_lab(gamma: float, lambda_u: float, K: float, steps_per_period: int,
                   courant: float, sigma_gamma_rel: float = 0.0) -> dict:
    """Rest-frame numbers of a lab-frame FEL case (mithra_boost_from_lab)."""
    lab = LabCase(gamma, sigma_gamma_rel, lambda_u, K, int(steps_per_period), courant)
    out = RestFrame()
    _check(lib().mithra_boost_from_lab(C.byref(lab), C.byref(out)), None)
    return {name: getattr(out, name) for name, _ in RestFrame._fields_}


def make_bunch(n: int, charge: float, *, sigma_x: float, sigma_y: float, z_lo: float,
               z_hi: float, uz_mean: float, x0: float = 0.0, y0: float = 0.0,
               trunc_r: float = 0.0, taper_sigma: float = 0.0, ux_sigma: float = 0.0,
               uy_sigma: float = 0.0, uz_sigma: float = 0.0, bf: float = 0.0, kb: float = 0.0,
               sequence: str = "halton", seed: int = 0) -> dict:
    """Rest-frame bunch from the library's generator (mithra_make_bunch):
    arrays x, y, z, ux, uy, uz and the macroparticle charge q_macro, the
    dictionary Simulation takes."""
    spec = BunchSpec(int(n), charge, x0, y0, sigma_x, sigma_y, trunc_r, z_lo, z_hi, taper_sigma,
                     ux_sigma, uy_sigma, uz_mean, uz_sigma, bf, kb,
                     {"splitmix64": 0, "halton": 1}[sequence], int(seed))
    out = {k: np.empty(max(int(n), 1)) for k in ("x", "y", "z", "ux", "uy", "uz")}
    q = C.c_double(0.0)
    dp = C.POINTER(C.c_double)
    _check(lib().mithra_make_bunch(C.byref(spec), *[out[k].ctypes.data_as(dp) for k in
                                                     ("x", "y", "z", "ux", "uy", "uz")],
                                   C.byref(q)), None)
    out["q_macro"] = q.value
    return out


def normalized_wavelengths(lambda_r: float, f_min: float, f_max: float, df: float) -> np.ndarray:
    """Lab wavelengths for a sweep over frequencies normalised to the
    radiation wavelength lambda_r (FEL-OUTPUT minimum-/maximum-normalized-
    frequency and normalized-frequency-resolution): lambda_r / f."""
    f = np.arange(f_min, f_max + 0.5 * df, df)
    return lambda_r / f


def make_undulator(u: dict | None) -> Undulator:
    """Static: gamma0, lambda_u, K, z_ent_lab, length_lab, fringe.  Optical
    (type "optical"): gamma0, a0, lambda_l, polarization (px, py), z0_lab,
    offset, variance, cep, direction (-1 or +1), signal (a SIGNALS name);
    a seed also beam (a BEAMS name) and, for the Gaussian beam, x0_lab,
    y0_lab and rayleigh_radius (waist along, across the polarization)."""
    if u is None:
        return Undulator(1.0e3, 1.0, 0.0, 0.0, 0.0, 0)
    if u.get("type", "static") == "optical":
        px, py = u.get("polarization", (0.0, 1.0))
        wp, wq = u.get("rayleigh_radius", (0.0, 0.0))
        return Undulator(u["gamma0"], 1.0, 0.0, 0.0, 0.0, 0, 1, u["a0"], u["lambda_l"], px, py,
                         u.get("z0_lab", 0.0), u["offset"], u["variance"], u.get("cep", 0.0),
                         int(u.get("direction", -1)), SIGNALS[u.get("signal", "flat-top")],
                         BEAMS[u.get("beam", "plane-wave")], u.get("x0_lab", 0.0),
                         u.get("y0_lab", 0.0), wp, wq)
    return Undulator(u["gamma0"], u["lambda_u"], u["K"], u.get("z_ent_lab", 0.0),
                     u.get("length_lab", 0.0), int(u.get("fringe", 1)))


def _check(status: int, handle=None):
    if status != OK:
        msg = lib().mithra_last_error(handle)
        raise MithraError(status, msg.decode() if msg else "")


def check_grid(g: dict) -> int:
    """Status of mithra_check_grid (host only; no GPU needed)."""
    return lib().mithra_check_grid(C.byref(make_grid(g)))


def footprint(g: dict, n_particles: int, precision: int = P32) -> int:
    out = C.c_int64(0)
    _check(lib().mithra_footprint(C.byref(make_grid(g)), int(n_particles), int(precision),
                                  C.byref(out)))
    return int(out.value)


def plane_power_noalloc(grid: dict, gamma0: float, precision: int, psi_newest_ptr: int,
                        increment_ptr: int, k_plane: int, stream: int | None = None,
                        lo_newest_ptr: int | None = None) -> float:
    """Lab-frame power through vertex plane k_plane from device arrays the
    caller owns (device pointers as integers; lo_newest_ptr the bfloat16 lo
    parts of a compensated level, or None), with no allocation inside the
    library; see mithra_plane_power_noalloc in include/mithra.h."""
    out = C.c_double()
    _check(lib().mithra_plane_power_noalloc(C.byref(make_grid(grid)), float(gamma0), int(precision),
                                            C.c_void_p(psi_newest_ptr),
                                            C.c_void_p(lo_newest_ptr or None),
                                            C.c_void_p(increment_ptr),
                                            int(k_plane), C.byref(out), stream_arg(stream)))
    return float(out.value)


def last_error() -> str:
    m = lib().mithra_last_error(None)
    return m.decode() if m else ""


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy


def stream_arg(stream):
    """None: the library creates its own stream.  An int handle is passed
    through, except 0 (the legacy default stream in CUDA and PyTorch), which
    the C ABI spells cudaStreamLegacy because NULL means 'library-owned'."""
    if stream is None:
        return None
    return C.c_void_p(int(stream) if int(stream) != 0 else CUDA_STREAM_LEGACY)


class Simulation:
    """One simulation on the current CUDA device (see include/mithra.h)."""

    def __init__(self, grid: dict, undulator: dict | None, bunch: dict | None,
                 precision: int = P32, stream: int | None = None):
        L = lib()
        self.grid = dict(grid)
        self.precision = precision
        n = 0 if bunch is None else int(np.asarray(bunch["x"]).size)
        self.n_particles = n
        self._keep = []
        if n:
            arrs = [np.ascontiguousarray(bunch[k], dtype=np.float64)
                    for k in ("x", "y", "z", "ux", "uy", "uz")]
            self._keep = arrs
            b = Bunch(n, float(bunch.get("q_macro", 0.0)), *[_dp(a) for a in arrs])
        else:
            b = Bunch(0, 0.0, None, None, None, None, None, None)
        h = C.c_void_p()
        _check(L.mithra_create(C.byref(make_grid(grid)), C.byref(make_undulator(undulator)),
                               C.byref(b), int(precision),
                               stream_arg(stream), C.byref(h)))
        self._keep = []
        self.h = h

    # -- time loop -------------------------------------------------------
    def step(self, n: int = 1):
        _check(lib().mithra_step(self.h, int(n)), self.h)

    def sync(self):
        _check(lib().mithra_sync(self.h), self.h)

    def set_lost_policy(self, strict: bool):
        """strict: a particle lost from now on makes sync / step raise
        MithraError with status ELOST (mithra_set_lost_policy)."""
        _check(lib().mithra_set_lost_policy(self.h, 1 if strict else 0), self.h)

    def time(self):
        n = C.c_int64()
        t = C.c_double()
        _check(lib().mithra_time(self.h, C.byref(n), C.byref(t)), self.h)
        return int(n.value), float(t.value)

    # -- fields ------------------------------------------------------------
    def _shape(self):
        return (self.grid["nz"], self.grid["ny"], self.grid["nx"])

    def copy_field(self, name: str) -> np.ndarray:
        out = np.empty(self._shape(), dtype=np.float64)
        _check(lib().mithra_copy_field(self.h, FIELD_ID[name], _dp(out)), self.h)
        return out

    def set_field(self, name: str, values: np.ndarray):
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
        assert a.size == int(np.prod(self._shape()))
        _check(lib().mithra_set_field(self.h, FIELD_ID[name], _dp(a)), self.h)

    def sample_fields(self, names, ijk) -> np.ndarray:
        mask = 0
        for nm in names:
            mask |= 1 << FIELD_ID[nm]
        pts = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        m = bin(mask).count("1")
        out = np.empty((pts.shape[0], m), dtype=np.float64)
        _check(lib().mithra_sample_fields(self.h, mask, pts.ctypes.data_as(C.POINTER(C.c_int32)),
                                          pts.shape[0], _dp(out)), self.h)
        return out

    def radiated_power(self, k_plane: int):
        p, t, z = C.c_double(), C.c_double(), C.c_double()
        _check(lib().mithra_radiated_power(self.h, int(k_plane), C.byref(p), C.byref(t),
                                           C.byref(z)), self.h)
        return float(p.value), float(t.value), float(z.value)

    def set_power_sampling(self, k_plane: int, capacity: int):
        _check(lib().mithra_set_power_sampling(self.h, int(k_plane), int(capacity)), self.h)

    def read_power(self, max_records: int | None = None) -> np.ndarray:
        cnt = C.c_int64()
        _check(lib().mithra_read_power(self.h, None, 0, C.byref(cnt)), self.h)
        m = int(cnt.value) if max_records is None else min(int(cnt.value), max_records)
        out = np.zeros((max(m, 0), 3), dtype=np.float64)
        if m > 0:
            _check(lib().mithra_read_power(self.h, _dp(out), m, C.byref(cnt)), self.h)
        return out

    def set_seed(self, seed: dict | None) -> None:
        """mithra_set_seed: a seed with an optical undulator's keys (type is
        implied) plus beam ("plane-wave" or "gaussian-beam"), x0_lab, y0_lab
        and rayleigh_radius (w_par, w_perp); None switches it off."""
        if seed is None:
            _check(lib().mithra_set_seed(self.h, None), self.h)
            return
        w = make_undulator(dict(seed, type="optical", gamma0=seed.get("gamma0", 2.0)))
        _check(lib().mithra_set_seed(self.h, C.byref(w)), self.h)

    # -- diagnostics -------------------------------------------------------
    BUNCH_STATS = ("mean_x", "mean_y", "mean_z", "mean_ux", "mean_uy", "mean_uz",
                   "rms_x", "rms_y", "rms_z", "rms_ux", "rms_uy", "rms_uz", "bunching", "n")

    def bunch_stats(self, k_b: float) -> np.ndarray:
        """mithra_bunch_stats: 14 values (names in BUNCH_STATS)."""
        out = np.zeros(14)
        _check(lib().mithra_bunch_stats(self.h, C.c_double(k_b), _dp(out)), self.h)
        return out

    def set_bunch_sampling(self, k_b: float, every: int, capacity: int) -> None:
        _check(lib().mithra_set_bunch_sampling(self.h, C.c_double(k_b), int(every),
                                               int(capacity)), self.h)

    def read_bunch(self) -> np.ndarray:
        """Records (n, 15): steps completed, then the BUNCH_STATS values."""
        cnt = C.c_int64()
        _check(lib().mithra_read_bunch(self.h, None, 0, C.byref(cnt)), self.h)
        out = np.zeros((int(cnt.value), 15))
        if cnt.value:
            _check(lib().mithra_read_bunch(self.h, _dp(out), int(cnt.value), C.byref(cnt)),
                   self.h)
        return out

    def snapshot(self) -> np.ndarray:
        """The simulation's device state as bytes (mithra_snapshot)."""
        n = C.c_int64()
        _check(lib().mithra_snapshot_bytes(self.h, C.byref(n)), self.h)
        buf = np.empty(int(n.value), dtype=np.uint8)
        _check(lib().mithra_snapshot(self.h, buf.ctypes.data_as(C.c_void_p)), self.h)
        return buf

    def restore(self, snap: np.ndarray) -> None:
        """Restores a snapshot of a simulation of the same shape."""
        snap = np.ascontiguousarray(snap, dtype=np.uint8)
        _check(lib().mithra_restore(self.h, snap.ctypes.data_as(C.c_void_p)), self.h)

    def set_spectrum(self, k_plane: int, lambda_lab) -> None:
        lam = np.ascontiguousarray(lambda_lab, dtype=np.float64)
        self._spec_n = int(lam.size)
        _check(lib().mithra_set_spectrum(self.h, int(k_plane), self._spec_n,
                                         _dp(lam) if lam.size else None), self.h)

    def read_spectrum(self):
        """(dW/domega per wavelength [J s], number of samples)."""
        n = getattr(self, "_spec_n", 0)
        out = np.zeros(n)
        ns = C.c_int64()
        _check(lib().mithra_read_spectrum(self.h, _dp(out) if n else None, C.byref(ns)), self.h)
        return out, int(ns.value)

    # -- particles ---------------------------------------------------------
    def copy_particles(self) -> dict:
        n = self.n_particles
        arrs = {k: np.empty(n, dtype=np.float64) for k in ("x", "y", "z", "ux", "uy", "uz")}
        lost = np.empty(n, dtype=np.int32)
        nl = C.c_int64()
        _check(lib().mithra_copy_particles(self.h, *[_dp(arrs[k]) for k in
                                                     ("x", "y", "z", "ux", "uy", "uz")],
                                           lost.ctypes.data_as(C.POINTER(C.c_int32)),
                                           C.byref(nl)), self.h)
        arrs["lost"] = lost
        arrs["n_lost"] = int(nl.value)
        return arrs

    # -- launch choices --------------------------------------------------
    def set_tuning(self, stencil_variant: int | None = None, lz: int | None = None,
                   push_variant: int | None = None, push_ctas_per_sm: int | None = None,
                   push_sparse_below: int | None = None):
        t = self.tuning()
        for k, v in (("stencil_variant", stencil_variant), ("lz", lz),
                     ("push_variant", push_variant), ("push_ctas_per_sm", push_ctas_per_sm),
                     ("push_sparse_below", push_sparse_below)):
            if v is not None:
                t[k] = int(v)
        _check(lib().mithra_set_tuning(self.h, C.byref(Tuning(**t))), self.h)

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().mithra_get_tuning(self.h, C.byref(t)), self.h)
        return {k: int(getattr(t, k)) for k, _ in Tuning._fields_}

    # -- kernel timing ---------------------------------------------------
    def profile(self, enable: bool = True):
        _check(lib().mithra_profile(self.h, 1 if enable else 0), self.h)

    def kernel_times(self) -> dict:
        ms = np.zeros(16)
        n = np.zeros(16, dtype=np.int64)
        nk = C.c_int32()
        _check(lib().mithra_kernel_times(self.h, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64)),
                                         16, C.byref(nk)), self.h)
        out = {}
        for k in range(nk.value):
            out[lib().mithra_kernel_name(k).decode()] = (float(ms[k]), int(n[k]))
        return out

    def source_tiles(self) -> tuple[int, bool]:
        """(tiles whose sources the next potential update reads, whether it
        reads every vertex's instead)."""
        n = C.c_int64()
        e = C.c_int32()
        _check(lib().mithra_source_tiles(self.h, C.byref(n), C.byref(e)), self.h)
        return int(n.value), bool(e.value)

    def close(self):
        if getattr(self, "h", None):
            lib().mithra_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Steps several simulations together through one captured CUDA graph
    (see mithra_batch_* in include/mithra.h)."""

    def __init__(self, stream: int | None = None):
        h = C.c_void_p()
        _check(lib().mithra_batch_create(stream_arg(stream), C.byref(h)))
        self.h = h
        self.members: list[Simulation] = []

    def _check(self, st):
        if st != OK:
            m = lib().mithra_batch_last_error(self.h)
            raise MithraError(st, m.decode() if m else "")

    def add(self, sim: Simulation):
        self._check(lib().mithra_batch_add(self.h, sim.h))
        self.members.append(sim)

    def remove(self, sim: Simulation):
        self._check(lib().mithra_batch_remove(self.h, sim.h))
        self.members.remove(sim)

    def step(self, n: int = 1):
        self._check(lib().mithra_batch_step(self.h, int(n)))

    def sync(self):
        self._check(lib().mithra_batch_sync(self.h))

    def set_mode(self, fused):
        """True: one launch per phase over all members when they allow it;
        False: one launch sequence per member; "auto" (the default): fused
        for small members (mithra_batch_set_mode)."""
        mode = 2 if fused == "auto" else (1 if fused else 0)
        self._check(lib().mithra_batch_set_mode(self.h, mode))

    def stats(self) -> dict:
        """Graph captures so far, fused ones, and their host time [s]."""
        c, f, t = C.c_int64(0), C.c_int64(0), C.c_double(0.0)
        self._check(lib().mithra_batch_stats(self.h, C.byref(c), C.byref(f), C.byref(t)))
        return dict(captures=int(c.value), fused_captures=int(f.value),
                    capture_seconds=float(t.value))

    def fused(self) -> bool:
        """Whether the graph captured last is the fused form."""
        out = C.c_int32(0)
        self._check(lib().mithra_batch_get_mode(self.h, C.byref(out)))
        return bool(out.value)

    def __len__(self):
        return int(lib().mithra_batch_size(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().mithra_batch_destroy(self.h)
            self.h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
