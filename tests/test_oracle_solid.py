"""Pins of the oracle's solid nodes (half-way bounce-back wherever a pull
reads a solid node; stencil ghosts that mirror a fluid node, the neutral
wetting of the axis walls; zero state and fields on solid nodes).

The reference for the ghost rule is the oracle's own axis walls, which are
pinned elsewhere: solid layers filling the ends of an axis of a periodic
lattice must reproduce a lattice with bounce-back walls on that axis, node
for node.  The other pins are exact invariants: a fluid at rest between
solid walls stays at rest, and bounce-back conserves the mass of each
component exactly.
"""
import numpy as np
import pytest

from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, asymmetric, base


@pytest.fixture(scope="module")
def T10(orc):
    return orc.temperature_for_ratio(A, B, RGAS, 10.0)


def drops_fields(o, shape, seed=4):
    D = len(shape)
    c = [s / 2.0 for s in shape]
    R = min(shape) / 4.0
    rho, phi, u = inputs.drops(tuple(shape), o.rho_g, o.rho_l, 5.0,
                               [dict(center=[v - 0.4 * R for v in c], R=R, kind=1, u=[0.02] * D),
                                dict(center=[v + 0.45 * R for v in c], R=0.8 * R, kind=-1, u=[-0.01] * D)],
                               width=4.0)
    return inputs.perturb(seed, rho, phi, u, 1e-3, 1e-3, 1e-3)


@pytest.mark.parametrize("lattice,shape,axes,form", [
    (0, (20, 14), (1,), 1),
    (0, (15, 12), (0, 1), 1),
    (0, (18, 11), (0,), 0),
    (1, (9, 8, 10), (0, 2), 1),
    (1, (7, 9, 8), (0, 1, 2), 1),
])
def test_solid_layers_reproduce_axis_walls(orc, T10, lattice, shape, axes, form):
    """Lattice with one solid layer at each end of the given axes (periodic
    there) against the lattice of the inner nodes with bounce-back walls on
    those axes: same state on every fluid node after 15 steps."""
    p = asymmetric(T10, force_form=form, gamma_mode=1)
    D = len(shape)
    inner = list(shape)
    outer = [s + 2 if a in axes else s for a, s in enumerate(shape)]
    bc = tuple(1 if a in axes else 0 for a in range(3))
    nz_i = inner[2] if D == 3 else 1
    nz_o = outer[2] if D == 3 else 1
    w = orc.Oracle(lattice, inner[0], inner[1], nz_i, p, bc=bc)
    rho, phi, u = drops_fields(w, inner)
    # embed the inner fields in the outer box (z, y, x order)
    grid_i = tuple(reversed(inner))
    grid_o = tuple(reversed(outer))
    sl = tuple(slice(1, -1) if (D - 1 - k) in axes else slice(None) for k in range(D))
    solid = np.ones(grid_o, np.uint8)
    solid[sl] = 0
    emb = lambda a, fill: (lambda out: (out.__setitem__(sl, a.reshape(grid_i)), out.ravel())[1])(np.full(grid_o, fill))
    rho_o, phi_o = emb(rho, 0.0), emb(phi, 0.0)
    u_o = np.stack([emb(u[a], 0.0) for a in range(D)])
    s = orc.Oracle(lattice, outer[0], outer[1], nz_o, dict(p, solid=solid.ravel()))
    fw, gw = w.init(rho, phi, u)
    fs, gs = s.init(rho_o, phi_o, u_o)
    assert w.step(fw, gw, 15) == 0
    assert s.step(fs, gs, 15) == 0
    fluid = solid.ravel() == 0
    for a_w, a_s in ((fw, fs), (gw, gs)):
        got = a_s[:, fluid]
        assert np.max(np.abs(got - a_w)) <= 1e-14 * np.abs(a_w).max()
        assert np.all(a_s[:, ~fluid] == 0.0)
    fw_, fs_ = w.fields(fw, gw), s.fields(fs, gs)
    for k in ("rho", "phi", "p"):
        assert np.max(np.abs(fs_[k][fluid] - fw_[k])) <= 1e-13 * max(np.abs(fw_[k]).max(), 1e-12), k
        assert np.all(fs_[k][~fluid] == 0.0)


def test_fluid_at_rest_between_solid_walls_stays_at_rest(orc, T10):
    p = base(T10)
    nx, ny = 12, 10
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    solid[4:6, 5:8] = 1  # and a block in the channel
    o = orc.Oracle(0, nx, ny, 1, dict(p, solid=solid.ravel()))
    rho = np.full(nx * ny, o.rho_l)
    f, g = o.init(rho, np.full(nx * ny, 5.0), np.zeros((2, nx * ny)))
    assert o.step(f, g, 50) == 0
    fl = o.fields(f, g)
    fluid = solid.ravel() == 0
    assert np.abs(fl["u"][:, fluid]).max() < 1e-14
    assert np.allclose(fl["rho"][fluid], o.rho_l, rtol=1e-14, atol=0)


@pytest.mark.parametrize("lattice,shape", [(0, (24, 20)), (1, (10, 9, 11))])
def test_bounce_back_at_solids_conserves_each_component(orc, T10, lattice, shape):
    p = asymmetric(T10)
    D = len(shape)
    g_ = np.meshgrid(*[np.arange(s) for s in reversed(shape)], indexing="ij")
    coords = list(reversed(g_))
    # an off-centre solid disc / ball and a solid wall piece
    r2 = sum((coords[a] - 0.3 * shape[a]) ** 2 for a in range(D))
    solid = ((r2 < (0.15 * min(shape)) ** 2) | (coords[1] == 0) & (coords[0] < shape[0] // 2)).astype(np.uint8)
    o = orc.Oracle(lattice, *shape, *([] if D == 3 else [1]), dict(p, solid=solid.ravel()))
    rho, phi, u = drops_fields(o, shape)
    f, g = o.init(rho, phi, u)
    fl0 = o.fields(f, g)
    assert o.step(f, g, 40) == 0
    fl = o.fields(f, g)
    fluid = solid.ravel() == 0
    assert abs(fl["rho"][fluid].sum() / fl0["rho"][fluid].sum() - 1) < 1e-13
    assert abs(fl["phi"][fluid].sum() - fl0["phi"][fluid].sum()) < 1e-12 * np.abs(fl0["phi"]).sum()
