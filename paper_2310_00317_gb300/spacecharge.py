"""Frozen space charge: lumped lenses configured from the optics (section
"Space charge": the frozen model, with enough lenses to sample the beam
envelope, transverse sizes from the Twiss module, a Gaussian transverse
distribution).

install_space_charge() computes the lattice functions along the ring on the
GPU (twiss.twiss_along), places `n_lenses` XT_SPACECHARGE rows at the row
boundaries nearest to equally spaced positions, and sizes each from the local
optics.  The lenses themselves are tracked by the library's kernel.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs as I
from . import twiss as T


def install_space_charge(table, ref, n_lenses: int, n_particles: float, eps_x: float, eps_y: float,
                         sigma_z: float = 0.0, sigma_delta: float = 0.0) -> dict:
    """Lumped frozen space-charge lenses for a beam of n_particles with
    geometric RMS emittances eps_x, eps_y, bunch length sigma_z (0: a
    coasting beam filling the ring) and momentum spread sigma_delta.  Lens k
    sits at the row boundary nearest to s_k = (k + 1/2) C / n_lenses and
    stands for C / n_lenses of ring; its sizes are
    sigma_x = sqrt(eps_x beta_x + (D_x sigma_delta)^2), sigma_y =
    sqrt(eps_y beta_y) from the lattice functions there; its peak line
    density is n_particles / (sqrt(2 pi) sigma_z), or n_particles / C when
    coasting.  Returns the new table, the boundary of every lens, and its
    beta_x, beta_y, sigma_x, sigma_y and strength per unit line density."""
    el = np.asarray(table)
    tw = T.twiss_along(el, ref)
    s = tw["s"]
    C = float(s[-1])
    if not (C > 0.0) or n_lenses < 1:
        raise ValueError("space charge needs a ring of positive length and at least one lens")
    lam0 = n_particles / (math.sqrt(2.0 * math.pi) * sigma_z) if sigma_z > 0.0 else n_particles / C
    L = C / n_lenses
    at = [int(np.argmin(np.abs(s - (k + 0.5) * L))) for k in range(n_lenses)]
    bx, by, dx = tw["betx"][at], tw["bety"][at], tw["dx"][at]
    sx = np.sqrt(eps_x * bx + (dx * sigma_delta) ** 2)
    sy = np.sqrt(eps_y * by)
    rows = []
    lens_at = {}
    for k, b in enumerate(at):
        lens_at.setdefault(b, []).append(k)
    for b in range(el.shape[0] + 1):
        for k in lens_at.get(b, []):
            rows.append(I.spacecharge(lam0, sigma_z, float(sx[k]), float(sy[k]), L))
        if b < el.shape[0]:
            rows.append(el[b])
    return dict(table=I.table(rows), boundary=np.array(at), betx=bx, bety=by, sigma_x=sx, sigma_y=sy,
                line_density=lam0, length=L, circumference=C)


def laslett_tune_shift(inst: dict, ref) -> tuple:
    """First-order incoherent tune shift of small-amplitude particles from
    the installed lenses: each acts as a thin defocusing lens of gradient
    K / (sigma_x (sigma_x + sigma_y)) in x (likewise y), K = 2 r_c lambda0 L /
    (beta0^2 gamma0^3), so dQ = sum beta K / (sigma (sigma_x + sigma_y)) /
    (4 pi) (positive numbers: the tunes move down by them)."""
    m0, q0, p0c = ref
    E0 = math.hypot(p0c, m0)
    b0, g0 = p0c / E0, E0 / m0
    rc = q0 * q0 * 2.8179403262e-15 * 0.51099895000e6 / m0
    K = 2.0 * rc * inst["line_density"] * inst["length"] / (b0 * b0 * g0 ** 3)
    sx, sy = inst["sigma_x"], inst["sigma_y"]
    dqx = float(np.sum(inst["betx"] * K / (sx * (sx + sy)))) / (4 * math.pi)
    dqy = float(np.sum(inst["bety"] * K / (sy * (sx + sy)))) / (4 * math.pi)
    return dqx, dqy
