"""Checkpoint and resume of a load-stepping run: the iterate U, the previous
step U_n, the Dirichlet mask, tau, the load step and the raw material
constants are written to one .npz file and read back (host arrays; the
caller moves them to the device and into a handle with pfm_set_state)."""
from __future__ import annotations

import json

import numpy as np


def save(path: str, U, Un, mask, tau: float, load_step: int, material: dict, mesh) -> None:
    np.savez(path, U=np.asarray(U, dtype=np.float64), Un=np.asarray(Un, dtype=np.float64),
             mask=np.asarray(mask, dtype=np.uint8), tau=np.float64(tau), load_step=np.int64(load_step),
             material=json.dumps(material),
             mesh=np.array([mesh.nx, mesh.ny, mesh.nz, mesh.Lx, mesh.Ly, mesh.Lz], dtype=np.float64))


def load(path: str) -> dict:
    z = np.load(path, allow_pickle=False)
    m = z["mesh"]
    return dict(U=z["U"], Un=z["Un"], mask=z["mask"], tau=float(z["tau"]), load_step=int(z["load_step"]),
                material=json.loads(str(z["material"])),
                mesh=(int(m[0]), int(m[1]), int(m[2]), float(m[3]), float(m[4]), float(m[5])))
