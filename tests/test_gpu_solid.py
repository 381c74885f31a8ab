"""GPU parity of solid nodes (tel_params.solid) against the oracle's solid
nodes: half-way bounce-back at solid sources, stencil ghosts mirroring a
fluid node, zero state and fields on solid nodes.

Bars as in test_gpu_parity: FP64 <= 1e-12 after one step, <= 1e-10 after
many; one FP32 step from the same state <= 2e-5; FP32 runs <= 1e-4 on
density and phase field, mass drift <= 1e-6.
"""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from tests.cases import A, B, RGAS, asymmetric, base
from tests.test_gpu_parity import field_err, setup_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T10():
    return tel.temperature_for_ratio(A, B, RGAS, 10.0)


def mask(shape, kind=0):
    """Solid mask [z][y][x] flattened: an off-centre disc/ball, a wall piece
    along y = 0 over half the lattice, and (kind 1) isolated solid nodes and a
    convex corner, so that every ghost case (one, two and three zeroed
    components) occurs."""
    D = len(shape)
    grids = np.meshgrid(*[np.arange(s) for s in reversed(shape)], indexing="ij")
    c = list(reversed(grids))
    r2 = sum((c[a] - 0.3 * shape[a]) ** 2 for a in range(D))
    m = (r2 < (0.16 * min(shape)) ** 2) | ((c[1] == 0) & (c[0] < shape[0] // 2))
    if kind == 1:
        m |= (c[0] == shape[0] - 3) & (c[1] == shape[1] - 4)
        m |= (c[0] >= shape[0] - 6) & (c[0] <= shape[0] - 5) & (c[1] >= 2) & (c[1] <= 3)
    return m.astype(np.uint8).ravel()


def pair(orc, lattice, shape, p, bc=(0, 0, 0), kind=0, precision=tel.FP64, amp=1e-3):
    sol = mask(shape, kind)
    p = dict(p, solid=sol)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc, precision=precision, amp=amp)
    return g, o, rho, phi, u, sol


def state_err_fluid(a, b, fluid):
    fa, ga = a
    fb, gb = b
    return max(np.max(np.abs(fa[:, fluid] - fb[:, fluid]) / np.abs(fb[:, fluid])),
               np.max(np.abs(ga[:, fluid] - gb[:, fluid])) / np.abs(gb).max())


CASES = [
    (0, (24, 20), (0, 0, 0), 1, 0),
    (0, (23, 19), (1, 0, 0), 1, 1),
    (0, (70, 37), (0, 1, 0), 0, 1),
    (1, (12, 10, 11), (0, 0, 0), 1, 1),
    (1, (13, 9, 10), (0, 0, 1), 0, 0),
    (1, (37, 11, 20), (1, 0, 0), 1, 1),
]


@pytest.mark.parametrize("lattice,shape,bc,form,kind", CASES)
def test_solid_one_step_fp64(orc, T10, lattice, shape, bc, form, kind):
    p = asymmetric(T10, force_form=form)
    g, o, rho, phi, u, sol = pair(orc, lattice, shape, p, bc, kind)
    fluid = sol == 0
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    st = g.get_state()
    assert state_err_fluid(st, (fo, go), fluid) < 1e-13
    assert np.all(st[0][:, ~fluid] == 0) and np.all(st[1][:, ~fluid] == 0)
    for _ in range(2):
        g.step(1)
        assert o.step(fo, go, 1) == 0
        st = g.get_state()
        assert state_err_fluid(st, (fo, go), fluid) < 1e-12
        assert np.all(st[0][:, ~fluid] == 0) and np.all(st[1][:, ~fluid] == 0)
    a, b = g.fields(), o.fields(fo, go)
    for k in ("rho", "phi", "u", "p"):
        assert np.all(a[k][..., ~fluid] == 0), k
    e = field_err({k: v[..., fluid] for k, v in a.items()}, {k: v[..., fluid] for k, v in b.items() if k != "rc"},
                  p["chi"])
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("lattice,shape,bc,steps", [
    (0, (48, 40), (0, 0, 0), 100),
    (1, (16, 14, 12), (1, 0, 0), 30),
])
def test_solid_multi_step_fp64(orc, T10, lattice, shape, bc, steps):
    p = base(T10, nu=0.1, gamma_mode=tel.GAMMA_EXACT)
    g, o, rho, phi, u, sol = pair(orc, lattice, shape, p, bc, kind=1)
    fluid = sol == 0
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(steps)
    assert o.step(fo, go, steps) == 0
    a, b = g.fields(), o.fields(fo, go)
    e = field_err({k: v[..., fluid] for k, v in a.items()}, {k: v[..., fluid] for k, v in b.items() if k != "rc"},
                  p["chi"])
    assert max(e.values()) < 1e-10, e


@pytest.mark.parametrize("lattice,shape,bc", [(0, (33, 29), (0, 0, 0)), (1, (16, 12, 14), (0, 1, 0))])
def test_solid_fp32(orc, T10, lattice, shape, bc):
    """One FP32-shifted step from the same state against the oracle, then 60
    steps against the oracle's run, and mass conservation."""
    p = asymmetric(T10, force_form=1)
    g, o, rho, phi, u, sol = pair(orc, lattice, shape, p, bc, kind=1, precision=tel.FP32_SHIFTED, amp=1e-2)
    fluid = sol == 0
    g.init(rho, phi, u)
    g.step(2)
    f0, g0 = g.get_state()
    g.step(1)
    f1, g1 = g.get_state()
    nz = shape[2] if lattice == 1 else 1
    o1 = orc.Oracle(lattice, shape[0], shape[1], nz, dict(p, solid=sol), bc=bc)
    assert o1.step(f0, g0, 1) == 0
    ef = np.max(np.abs(f0 - f1)[:, fluid] / np.max(np.abs(f0[:, fluid]), axis=0))
    eg = np.max(np.abs(g0 - g1)) / p["chi"]
    assert max(ef, eg) < 2e-5, (ef, eg)
    q = base(T10, nu=0.1)
    g2, o2, rho, phi, u, sol = pair(orc, lattice, shape, q, bc, kind=1, precision=tel.FP32_SHIFTED)
    g2.init(rho, phi, u)
    fo, go = o2.init(rho, phi, u)
    g2.step(60)
    assert o2.step(fo, go, 60) == 0
    a, b = g2.fields(), o2.fields(fo, go)
    assert np.max(np.abs(a["rho"] - b["rho"])[fluid] / b["rho"][fluid]) < 1e-4
    assert np.max(np.abs(a["phi"] - b["phi"])) / q["chi"] < 1e-4
    assert abs(a["rho"][fluid].sum() / rho[fluid].sum() - 1) < 1e-6


def test_solid_layers_reproduce_axis_walls_gpu(T10):
    """Solid layers at both ends of y on a periodic lattice against walls on
    y: the same fluid state (FP64, node for node)."""
    p = asymmetric(T10, force_form=1)
    nx, ny = 30, 18
    w = tel.Lattice(tel.D2Q9, nx, ny, 1, p, bc=(0, 1, 0))
    sol = np.zeros((ny + 2, nx), np.uint8)
    sol[0] = sol[-1] = 1
    s = tel.Lattice(tel.D2Q9, nx, ny + 2, 1, dict(p, solid=sol.ravel()))
    from paper_1710_07486_gb300 import inputs
    rho, phi, u = inputs.drops((nx, ny), w.rho_g, w.rho_l, 5.0,
                               [dict(center=(10.0, 3.0), R=5.0, kind=1, u=(0.02, -0.01)),
                                dict(center=(20.0, 14.0), R=4.0, kind=-1)], width=4.0)
    emb = lambda a: np.concatenate([np.zeros(nx), a, np.zeros(nx)])
    w.init(rho, phi, u)
    s.init(emb(rho), emb(phi), np.stack([emb(u[0]), emb(u[1])]))
    w.step(20)
    s.step(20)
    fw, gw = w.get_state()
    fs, gs = s.get_state()
    inner = slice(nx, nx * (ny + 1))
    assert np.max(np.abs(fs[:, inner] - fw)) <= 1e-13 * np.abs(fw).max()
    assert np.max(np.abs(gs[:, inner] - gw)) <= 1e-13 * np.abs(gw).max()


def test_solid_mask_is_rejected_where_unsupported(T10):
    p = dict(base(T10), solid=np.zeros(64, np.uint8))
    with pytest.raises(tel.TelError):
        tel.Batch([(8, 8)], p)
    with pytest.raises(ValueError):
        tel.Lattice(tel.D2Q9, 8, 9, 1, p)
