"""Python driver of the plain FP64 CPU oracle (``orc.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
(as the checker) and by ``bench.py``'s ``cpu_baseline`` / ``--impl reference``
legs.  The product path (the CUDA library and its binding) never imports it.

The oracle runs the time step of the paper's method chapter in the paper's
order (Sec. "FDTD for Helmholtz Equation" through Sec. "Current Deposition"):

  1. potentials n+1 from n, n-1 and the sources (Eq. updateEquation, Mur ABC);
  2. E, B at t = (n+1/2) dt at the vertices (Sec. "Field Evaluation");
  3. gather + undulator field + Boris push of every particle (Eq. BorisScheme,
     Eq. fieldInterpolation, Eq. undulatorFieldRest);
  4. deposit of J^{n+1} and rho^{n+3/2} (Sec. "Current Deposition");
  5. optional radiated power through one plane, lab frame;
  6. advance the clock and rotate the levels.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")


def build(verbose: bool = False) -> str:
    """Compile ``orc.c`` into ``oracle/_build/liborc.so`` (gcc, OpenMP,
    no FMA contraction so that x86 and Arm hosts round the same way)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    src = os.path.join(_HERE, "orc.c")
    if os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "orc.h"))
    ):
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", _LIB_PATH, src, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dt", C.c_double), ("n_sub", C.c_int32), ("stencil", C.c_int32),
                ("space_charge", C.c_int32), ("boundary", C.c_int32)]


class _Und(C.Structure):
    _fields_ = [("gamma0", C.c_double), ("lambda_u", C.c_double), ("K", C.c_double),
                ("z_ent_lab", C.c_double), ("length_lab", C.c_double),
                ("fringe", C.c_int32), ("type", C.c_int32),
                ("a0", C.c_double), ("lambda_l", C.c_double), ("pol_x", C.c_double),
                ("pol_y", C.c_double), ("z0_lab", C.c_double), ("offset", C.c_double),
                ("variance", C.c_double), ("cep", C.c_double), ("direction", C.c_int32),
                ("signal", C.c_int32), ("beam", C.c_int32), ("x0_lab", C.c_double),
                ("y0_lab", C.c_double), ("w_par", C.c_double), ("w_perp", C.c_double)]


SIGNALS = {"neumann": 0, "gaussian": 1, "secant-hyperbolic": 2, "flat-top": 3}
BEAMS = {"plane-wave": 0, "gaussian-beam": 1}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        _lib.orc_coefficients.argtypes = [C.POINTER(_Grid), dp]
        _lib.orc_coefficients.restype = C.c_int
        _lib.orc_potential_step.argtypes = [C.POINTER(_Grid), dp, dp, dp, dp]
        _lib.orc_fields.argtypes = [C.POINTER(_Grid), dp, dp, dp, dp]
        _lib.orc_undulator_field.argtypes = [C.POINTER(_Und), C.c_double, C.c_double,
                                             C.c_double, dp, dp]
        _lib.orc_boris.argtypes = [dp, dp, dp, C.c_double, C.c_double]
        _lib.orc_push_deposit.argtypes = [C.POINTER(_Grid), C.POINTER(_Und), C.c_double,
                                          C.c_double, dp, dp, C.c_int64, dp, dp, dp,
                                          dp, dp, dp, ip, dp]
        _lib.orc_push_deposit.restype = C.c_int64
        _lib.orc_deposit_rho.argtypes = [C.POINTER(_Grid), C.c_double, C.c_int64, dp, dp,
                                         dp, ip, dp]
        _lib.orc_mark_lost.argtypes = [C.POINTER(_Grid), C.c_int64, dp, dp, dp, ip]
        _lib.orc_mark_lost.restype = C.c_int64
        _lib.orc_radiated_power.argtypes = [C.POINTER(_Grid), C.c_double, dp, dp, C.c_int32,
                                            C.c_double, dp, dp, dp]
        _lib.orc_constants.argtypes = [dp]
        _lib.orc_bunch_stats.argtypes = [C.c_int64, dp, dp, dp, dp, dp, dp, ip, C.c_double, dp]
        _lib.orc_spectrum_accumulate.argtypes = [C.POINTER(_Grid), C.c_double, dp, dp,
                                                 C.c_int32, C.c_double, C.c_double, C.c_int32,
                                                 dp, dp]
        _lib.orc_spectrum_density.argtypes = [C.POINTER(_Grid), C.c_int32, dp, dp]
        _lib.orc_seed_correction.argtypes = [C.POINTER(_Grid), C.POINTER(_Und), C.c_double, dp]
        _lib.orc_incident_potential.argtypes = [C.POINTER(_Und), C.c_double, C.c_double,
                                                C.c_double, C.c_double, dp]
        _lib.orc_incident_potential_many.argtypes = [C.POINTER(_Und), C.c_int64, dp, dp, dp,
                                                     dp, dp]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(C.POINTER(C.c_double))
    if a.dtype == np.int32:
        return a.ctypes.data_as(C.POINTER(C.c_int32))
    raise TypeError(a.dtype)


def constants() -> dict:
    out = np.zeros(5)
    lib().orc_constants(_p(out))
    return dict(c=out[0], e=out[1], m_e=out[2], eps0=out[3], mu0=out[4])


def make_grid(g: dict) -> _Grid:
    return _Grid(int(g["nx"]), int(g["ny"]), int(g["nz"]), g["dx"], g["dy"], g["dz"],
                 g.get("x0", 0.0), g.get("y0", 0.0), g.get("z0", 0.0), g["dt"],
                 int(g.get("n_sub", 1)), int(g.get("stencil", 0)),
                 int(g.get("space_charge", 1)), int(g.get("boundary", 1)))


def make_und(u: dict | None) -> _Und:
    """Static undulator keys: gamma0, lambda_u, K, z_ent_lab, length_lab,
    fringe.  Optical (type "optical"): gamma0, a0, lambda_l, polarization
    (px, py), z0_lab, offset, variance, cep, direction (-1 or +1), signal;
    a seed also beam ("plane-wave" or "gaussian-beam") and, for the Gaussian
    beam, x0_lab, y0_lab and rayleigh_radius (w_par, w_perp)."""
    if u is None:
        return _Und(1.0e3, 1.0, 0.0, 0.0, 0.0, 0)
    if u.get("type", "static") == "optical":
        px, py = u.get("polarization", (0.0, 1.0))
        wp, wq = u.get("rayleigh_radius", (0.0, 0.0))
        return _Und(u["gamma0"], 1.0, 0.0, 0.0, 0.0, 0, 1, u["a0"], u["lambda_l"], px, py,
                    u.get("z0_lab", 0.0), u["offset"], u["variance"], u.get("cep", 0.0),
                    int(u.get("direction", -1)), SIGNALS[u.get("signal", "flat-top")],
                    BEAMS[u.get("beam", "plane-wave")], u.get("x0_lab", 0.0),
                    u.get("y0_lab", 0.0), wp, wq)
    return _Und(u["gamma0"], u["lambda_u"], u["K"], u.get("z_ent_lab", 0.0),
                u.get("length_lab", 0.0), int(u.get("fringe", 1)))


def coefficients(g: dict):
    out = np.zeros(6)
    unstable = lib().orc_coefficients(C.byref(make_grid(g)), _p(out))
    return out, bool(unstable)


def potential_step(g: dict, prev, cur, src):
    nxt = np.zeros_like(cur)
    lib().orc_potential_step(C.byref(make_grid(g)), _p(prev), _p(cur), _p(src), _p(nxt))
    return nxt


def fields(g: dict, lev_n, lev_np1):
    n = lev_n.size // 4
    E = np.zeros(3 * n)
    B = np.zeros(3 * n)
    lib().orc_fields(C.byref(make_grid(g)), _p(lev_n), _p(lev_np1), _p(E), _p(B))
    return E, B


def deposit_rho(g: dict, q_macro: float, x, y, z) -> np.ndarray:
    """rho of particles at (x, y, z) (those outside the valid region are
    skipped), shape (nz, ny, nx)."""
    G = make_grid(g)
    xs, ys, zs = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
    lost = np.zeros(xs.size, dtype=np.int32)
    lib().orc_mark_lost(C.byref(G), xs.size, _p(xs), _p(ys), _p(zs), _p(lost))
    rho = np.zeros(int(g["nx"]) * int(g["ny"]) * int(g["nz"]))
    lib().orc_deposit_rho(C.byref(G), float(q_macro), xs.size, _p(xs), _p(ys), _p(zs), _p(lost),
                          _p(rho))
    return rho.reshape(g["nz"], g["ny"], g["nx"])


def undulator_field(u: dict, y: float, z: float, t: float):
    E = np.zeros(3)
    B = np.zeros(3)
    lib().orc_undulator_field(C.byref(make_und(u)), y, z, t, _p(E), _p(B))
    return E, B


def boris(u, E, B, qm, dtb):
    uu = np.array(u, dtype=np.float64)
    lib().orc_boris(_p(uu), _p(np.asarray(E, np.float64)), _p(np.asarray(B, np.float64)),
                    qm, dtb)
    return uu


def radiated_power(g: dict, gamma0: float, E, B, k_p: int, t: float):
    p = np.zeros(1)
    tl = np.zeros(1)
    zl = np.zeros(1)
    lib().orc_radiated_power(C.byref(make_grid(g)), gamma0, _p(E), _p(B), int(k_p), t,
                             _p(p), _p(tl), _p(zl))
    return float(p[0]), float(tl[0]), float(zl[0])


def bunch_stats(x, y, z, ux, uy, uz, lost, k_b: float) -> np.ndarray:
    """Means, rms spreads and bunching factor (orc_bunch_stats)."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z, ux, uy, uz)]
    lo = np.ascontiguousarray(lost, dtype=np.int32)
    out = np.zeros(14)
    lib().orc_bunch_stats(a[0].size, *[_p(v) for v in a], _p(lo), float(k_b), _p(out))
    return out


def spectrum_accumulate(g: dict, gamma0: float, E, B, k_p: int, t_lab: float, dt_lab: float,
                        omega, acc: np.ndarray):
    om = np.ascontiguousarray(omega, dtype=np.float64)
    lib().orc_spectrum_accumulate(C.byref(make_grid(g)), gamma0, _p(E), _p(B), int(k_p), t_lab,
                                  dt_lab, om.size, _p(om), _p(acc))


def spectrum_density(g: dict, n_freq: int, acc: np.ndarray) -> np.ndarray:
    out = np.zeros(n_freq)
    lib().orc_spectrum_density(C.byref(make_grid(g)), int(n_freq), _p(acc), _p(out))
    return out


def incident_potential(u: dict, z, t, x=0.0, y=0.0) -> np.ndarray:
    """(A_x, A_y) of a seed at rest-frame points; z, t, x, y broadcast
    together, the result has their shape plus a last axis of 2."""
    z, t, x, y = (np.array(a, dtype=np.float64, order="C")
                  for a in np.broadcast_arrays(z, t, x, y))
    out = np.zeros(z.shape + (2,))
    lib().orc_incident_potential_many(C.byref(make_und(dict(u, type="optical"))), z.size,
                                      _p(x), _p(y), _p(z), _p(t), _p(out))
    return out


def observed_omega(lambda_lab, gamma0: float) -> np.ndarray:
    """Angular frequency at which a forward lab wave of wavelength lambda_lab
    passes a plane moving with the rest frame: 2 pi c (1 - beta0) / lambda."""
    b0 = np.sqrt(1.0 - 1.0 / (gamma0 * gamma0))
    c = constants()["c"]
    return 2.0 * np.pi * c * (1.0 - b0) / np.asarray(lambda_lab, dtype=np.float64)


@dataclass
class PowerSample:
    step: int
    p_lab: float
    t_lab: float
    z_lab: float


class OracleSim:
    """FP64 state of one simulation and the step loop of the paper.

    Initial state (SASE, Sec. "Field Initialization"): potentials zero at
    levels -1 and 0, the caller's (r, u) taken as r^{1/2}, u^0, rho^{1/2}
    deposited from the initial positions, J^0 = 0.
    """

    def __init__(self, grid: dict, undulator: dict | None, bunch: dict, t0: float = 0.0):
        self.g = dict(grid)
        self.u = None if undulator is None else dict(undulator)
        self._G = make_grid(self.g)
        self._U = make_und(self.u)
        self.n_cell = int(grid["nx"]) * int(grid["ny"]) * int(grid["nz"])
        n = self.n_cell
        self.prev = np.zeros(4 * n)
        self.cur = np.zeros(4 * n)
        self.nxt = np.zeros(4 * n)
        self.src = np.zeros(4 * n)
        self.src_next = np.zeros(4 * n)
        self.E = np.zeros(3 * n)
        self.B = np.zeros(3 * n)
        self.q_macro = float(bunch.get("q_macro", 0.0))
        self.x = np.ascontiguousarray(bunch["x"], dtype=np.float64).copy()
        self.y = np.ascontiguousarray(bunch["y"], dtype=np.float64).copy()
        self.z = np.ascontiguousarray(bunch["z"], dtype=np.float64).copy()
        self.ux = np.ascontiguousarray(bunch["ux"], dtype=np.float64).copy()
        self.uy = np.ascontiguousarray(bunch["uy"], dtype=np.float64).copy()
        self.uz = np.ascontiguousarray(bunch["uz"], dtype=np.float64).copy()
        self.np = self.x.size
        self.lost = np.zeros(self.np, dtype=np.int32)
        L = lib()
        self.n_lost = int(L.orc_mark_lost(C.byref(self._G), self.np, _p(self.x), _p(self.y),
                                          _p(self.z), _p(self.lost)))
        rho = np.zeros(n)
        L.orc_deposit_rho(C.byref(self._G), self.q_macro, self.np, _p(self.x), _p(self.y),
                          _p(self.z), _p(self.lost), _p(rho))
        self.src[3 * n:] = rho
        self.t0 = float(t0)
        self.n = 0
        self.power: list[PowerSample] = []
        self.seed = None
        self.spec_plane = None
        self.spec_omega = None
        self.spec_acc = None
        self.spec_samples = 0

    def set_spectrum(self, k_plane: int, lambda_lab):
        """Running Fourier sums of the lab fields at plane k_plane, one set
        per lab wavelength, from the next step on (orc_spectrum_accumulate)."""
        g0 = self.u["gamma0"] if self.u else 1.0e3
        self.spec_plane = int(k_plane)
        self.spec_omega = observed_omega(lambda_lab, g0)
        nv = (self.g["nx"] - 2) * (self.g["ny"] - 2)
        self.spec_acc = np.zeros(self.spec_omega.size * nv * 8)
        self.spec_samples = 0

    def spectrum(self) -> np.ndarray:
        """Energy per unit observed angular frequency so far [J s]."""
        out = np.zeros(self.spec_omega.size)
        lib().orc_spectrum_density(C.byref(self._G), self.spec_omega.size, _p(self.spec_acc),
                                   _p(out))
        return out

    def set_seed(self, seed: dict | None):
        """Seed injected through the TF/SF planes (orc_seed_correction): the
        keys of an optical undulator plus beam, x0_lab, y0_lab and
        rayleigh_radius; None switches it off."""
        self.seed = None if seed is None else make_und(dict(seed, type="optical"))

    def bunch_stats(self, k_b: float) -> np.ndarray:
        return bunch_stats(self.x, self.y, self.z, self.ux, self.uy, self.uz, self.lost, k_b)

    def set_potentials(self, prev: np.ndarray, cur: np.ndarray):
        self.prev[:] = prev
        self.cur[:] = cur

    def set_sources(self, src: np.ndarray):
        self.src[:] = src

    def t_half(self) -> float:
        return self.t0 + (self.n + 0.5) * self.g["dt"]

    def step(self, nsteps: int = 1, power_plane: int | None = None):
        L = lib()
        n = self.n_cell
        for _ in range(nsteps):
            L.orc_potential_step(C.byref(self._G), _p(self.prev), _p(self.cur), _p(self.src),
                                 _p(self.nxt))
            if self.seed is not None:
                L.orc_seed_correction(C.byref(self._G), C.byref(self.seed),
                                      self.t0 + self.n * self.g["dt"], _p(self.nxt))
            L.orc_fields(C.byref(self._G), _p(self.cur), _p(self.nxt), _p(self.E), _p(self.B))
            self.src_next[:] = 0.0
            th = self.t_half()
            self.n_lost += int(L.orc_push_deposit(
                C.byref(self._G), C.byref(self._U), self.q_macro, th, _p(self.E), _p(self.B),
                self.np, _p(self.x), _p(self.y), _p(self.z), _p(self.ux), _p(self.uy),
                _p(self.uz), _p(self.lost), _p(self.src_next)))
            g0 = self.u["gamma0"] if self.u else 1.0e3
            if power_plane is not None:
                p, tl, zl = radiated_power(self.g, g0, self.E, self.B, power_plane, th)
                self.power.append(PowerSample(self.n, p, tl, zl))
            if self.spec_plane is not None:
                b0 = np.sqrt(1.0 - 1.0 / (g0 * g0))
                zp = self.g.get("z0", 0.0) + self.spec_plane * self.g["dz"]
                t_lab = g0 * (th + b0 * zp / constants()["c"])
                L.orc_spectrum_accumulate(C.byref(self._G), g0, _p(self.E), _p(self.B),
                                          self.spec_plane, t_lab, g0 * self.g["dt"],
                                          self.spec_omega.size, _p(self.spec_omega),
                                          _p(self.spec_acc))
                self.spec_samples += 1
            # rotate: (n-1, n, n+1) -> (n, n+1, scratch)
            self.prev, self.cur, self.nxt = self.cur, self.nxt, self.prev
            self.src, self.src_next = self.src_next, self.src
            self.n += 1
        _ = n

    # views in the (nz, ny, nx) host layout, per component
    def potential(self, comp: int, level: str = "cur") -> np.ndarray:
        a = self.cur if level == "cur" else self.prev
        return a[comp * self.n_cell:(comp + 1) * self.n_cell].reshape(
            self.g["nz"], self.g["ny"], self.g["nx"])

    def source(self, comp: int) -> np.ndarray:
        return self.src[comp * self.n_cell:(comp + 1) * self.n_cell].reshape(
            self.g["nz"], self.g["ny"], self.g["nx"])
