"""Writes the reference samples of the c2 workload (128x128x1024 cells, 2^21
particles) after the configured 5000 steps, computed by the FP64 oracle only.

The GPU parity test for the long run compares against these samples:
  - every field (E, B, A, phi, J, rho) on the vertex plane through the
    initial bunch centre (k = 512), rounded to float32 (the comparison
    tolerance is 1e-4, far above float32 rounding);
  - the lab-frame radiated power through plane nz - 16 at every step;
  - positions and momenta of particles 0, 512, 1024, ... (4096 of them);
  - the full FP64 L2 norm of every field;
  - at the last checkpoint, E and B on every 4th vertex along each axis
    (offset 2), float32: a uniform sample of the whole grid for the
    field L2 error.
Checkpoints at steps 1000, 2000 and 5000 are written as they are reached
(c2_reference_<step>.npz).

Usage: python tests/golden/make_c2_reference.py [out_dir]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path[:0] = [ROOT, os.path.join(ROOT, "oracle")]

import oracle  # noqa: E402
from paper_1612_03310_gb300 import inputs  # noqa: E402

FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Ax", "Ay", "Az", "phi", "Jx", "Jy", "Jz", "rho"]
PLANE_K = 512
POWER_K = 1024 - 16
CHECKPOINTS = (1000, 2000, 5000)


def fields_of(o):
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
    for a, nm in enumerate(("Jx", "Jy", "Jz", "rho")):
        out[nm] = o.src[a * n:(a + 1) * n].reshape(shp)
    return out


def main(out_dir):
    oracle.build()
    w = inputs.workload("c2")
    bunch = inputs.make_bunch(w["bunch_spec"], w["seed"])
    o = oracle.OracleSim(w["grid"], w["undulator"], bunch)
    t0 = time.time()
    done = 0
    for ck in CHECKPOINTS:
        o.step(ck - done, power_plane=POWER_K)
        done = ck
        f = fields_of(o)
        sel = slice(0, None, 512)
        sub = {}
        if ck == CHECKPOINTS[-1]:
            sub = {f"sub_{nm}": f[nm][2::4, 2::4, 2::4].astype(np.float32)
                   for nm in FIELDS[:6]}
        np.savez_compressed(
            os.path.join(out_dir, f"c2_reference_{ck}.npz"),
            steps=ck, plane_k=PLANE_K, power_k=POWER_K,
            **{f"plane_{nm}": f[nm][PLANE_K].astype(np.float32) for nm in FIELDS},
            **{f"norm_{nm}": np.linalg.norm(f[nm]) for nm in FIELDS},
            power=np.array([[s.p_lab, s.t_lab, s.z_lab] for s in o.power]),
            particle_index=np.arange(o.np)[sel],
            x=o.x[sel], y=o.y[sel], z=o.z[sel], ux=o.ux[sel], uy=o.uy[sel], uz=o.uz[sel],
            lost=o.lost[sel], n_lost=o.n_lost, **sub)
        print(f"step {ck}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else HERE)
