"""Seeded synthetic inputs: droplet setups and random perturbations.

This module only builds input fields (density rho, phase field phi, velocity
u) on a lattice.  It holds none of the lattice Boltzmann arithmetic: the
coexistence densities rho_g, rho_l and the phase-field scale chi are passed in
by the caller.  Both the CUDA library's tests/benchmark and the CPU oracle's
tests draw their inputs from here.

Layout: fields are flat float64 arrays with node index n = x + nx*(y + ny*z)
(numpy C order over (z, y, x)); u is component-major ``[D, N]``.

The drop shapes stand in for the paper's droplet experiments (liquid lens,
head-on and off-centre binary collisions of immiscible drops): a gas
background at rho_g, liquid-1 drops (phi = +chi) and liquid-2 drops
(phi = -chi) at rho_l, joined by tanh profiles of width ``width`` lattice
units.  Where drops touch or overlap each node belongs to the drop whose
surface is nearest (smallest r - R).
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1710


def rng(seed: int = DEFAULT_SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def drops(shape, rho_g, rho_l, chi, drop_list, width=5.0):
    """Fields for a set of drops on a periodic box.

    shape: (nx, ny) or (nx, ny, nz).  drop_list: dicts with ``center``
    (D floats), ``R``, ``kind`` (+1 liquid 1, -1 liquid 2) and optional ``u``
    (D floats, the drop velocity).  Distances use the minimum image.
    Returns (rho[N], phi[N], u[D, N]).
    """
    D = len(shape)
    nx, ny = shape[0], shape[1]
    nz = shape[2] if D == 3 else 1
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = [x.astype(float), y.astype(float), z.astype(float)][:D]
    dims = [nx, ny, nz][:D]
    best = np.full(x.shape, np.inf)
    s_best = np.zeros(x.shape)
    kind_best = np.zeros(x.shape)
    u_best = np.zeros((D,) + x.shape)
    for d in drop_list:
        r2 = np.zeros(x.shape)
        for a in range(D):
            dd = coords[a] - float(d["center"][a])
            dd = dd - dims[a] * np.round(dd / dims[a])
            r2 += dd * dd
        r = np.sqrt(r2)
        dist = r - float(d["R"])
        s = 0.5 * (1.0 + np.tanh(2.0 * (float(d["R"]) - r) / width))
        take = dist < best
        best = np.where(take, dist, best)
        s_best = np.where(take, s, s_best)
        kind_best = np.where(take, float(d["kind"]), kind_best)
        du = d.get("u", [0.0] * D)
        for a in range(D):
            u_best[a] = np.where(take, float(du[a]) * s, u_best[a])
    rho = rho_g + (rho_l - rho_g) * s_best
    phi = kind_best * chi * s_best
    N = x.size
    return (rho.reshape(N).copy(), phi.reshape(N).copy(),
            u_best.reshape(D, N).copy())


def perturb(seed, rho, phi, u, amp_rho=1e-3, amp_phi=1e-3, amp_u=1e-3):
    """Multiplicative/additive seeded noise so that no two nodes are alike."""
    g = rng(seed)
    rho = rho * (1.0 + amp_rho * g.uniform(-1, 1, rho.shape))
    phi = phi + amp_phi * g.uniform(-1, 1, phi.shape)
    u = u + amp_u * g.uniform(-1, 1, u.shape)
    return rho, phi, u


def touching_drops_2d(nx, ny, rho_g, rho_l, chi, R=12.0, offset=20.0, width=5.0):
    """One liquid-1 and one liquid-2 drop of radius R, centres offset along x
    by ``offset`` about the box centre, at rest."""
    cx, cy = nx / 2.0, ny / 2.0
    return drops((nx, ny), rho_g, rho_l, chi,
                 [dict(center=(cx - offset / 2, cy), R=R, kind=+1),
                  dict(center=(cx + offset / 2, cy), R=R, kind=-1)], width)


def head_on_2d(seed, n, rho_g, rho_l, chi, V, R=40.0, gap=60.0, width=5.0):
    """Head-on collision in a square periodic box of edge n: liquid 1 moving
    +x at V/2, liquid 2 moving -x at V/2, centres n/2 -/+ gap, jittered by
    an integer in [-2, 2] on each axis."""
    g = rng(seed)
    j = g.integers(-2, 3, size=4)
    c = n / 2.0
    return drops((n, n), rho_g, rho_l, chi,
                 [dict(center=(c - gap + j[0], c + j[1]), R=R, kind=+1, u=(V / 2, 0.0)),
                  dict(center=(c + gap + j[2], c + j[3]), R=R, kind=-1, u=(-V / 2, 0.0))],
                 width)


def off_centre_2d(n, rho_g, rho_l, chi, V, B, R, width=5.0):
    """Off-centre binary collision in a periodic square of edge n: drops of
    radius R approach along x at +/-V/2 with centres offset along y by
    B * 2R (impact parameter B)."""
    c = n / 2.0
    gap = R + 4.0
    dy = B * 2.0 * R / 2.0
    return drops((n, n), rho_g, rho_l, chi,
                 [dict(center=(c - gap, c - dy), R=R, kind=+1, u=(V / 2, 0.0)),
                  dict(center=(c + gap, c + dy), R=R, kind=-1, u=(-V / 2, 0.0))],
                 width)


def off_centre_3d(seed, n, rho_g, rho_l, chi, V, B, R=30.0, width=5.0):
    """Off-centre binary collision in a periodic cube of edge n: drops of
    radius R approach along x at +/-V/2 with centres offset along y by
    B * 2R (impact parameter B)."""
    c = n / 2.0
    gap = R + 4.0
    dy = B * 2.0 * R / 2.0
    return drops((n, n, n), rho_g, rho_l, chi,
                 [dict(center=(c - gap, c - dy, c), R=R, kind=+1, u=(V / 2, 0.0, 0.0)),
                  dict(center=(c + gap, c + dy, c), R=R, kind=-1, u=(-V / 2, 0.0, 0.0))],
                 width)
