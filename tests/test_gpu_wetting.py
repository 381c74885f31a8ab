"""GPU parity of the wetting walls (tel_params.wet_rho, wet_phi) against the
oracle's: at bounce-back walls and at solid nodes, FP64 and FP32-shifted,
single lattices and batches; and the physical effect on the GPU: a drop on a
wall spreads with a positive density wetting gradient and beads up with a
negative one.

Bars as in test_gpu_parity: FP64 <= 1e-12 after a few steps, <= 1e-10 after
many; one FP32 step from the same state <= 2e-5.
"""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, asymmetric, base
from tests.test_gpu_parity import field_err, setup_pair
from tests.test_gpu_solid import mask, state_err_fluid

pytestmark = pytest.mark.gpu

WET = dict(wet_rho=0.02, wet_phi=-0.15)


@pytest.fixture(scope="module")
def T10():
    return tel.temperature_for_ratio(A, B, RGAS, 10.0)


CASES = [
    # lattice, shape, bc, force form, solid mask kind (None: walls only)
    (0, (24, 20), (1, 1, 0), 1, None),
    (0, (23, 19), (1, 0, 0), 0, None),
    (0, (30, 26), (0, 1, 0), 1, 1),
    (1, (12, 10, 11), (1, 1, 1), 1, None),
    (1, (13, 9, 10), (0, 0, 1), 1, 0),
    (1, (17, 11, 12), (1, 0, 0), 0, 1),
]


@pytest.mark.parametrize("lattice,shape,bc,form,kind", CASES)
def test_wetting_fp64_against_oracle(orc, T10, lattice, shape, bc, form, kind):
    p = dict(asymmetric(T10, force_form=form), **WET)
    sol = None if kind is None else mask(shape, kind)
    if sol is not None:
        p["solid"] = sol
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc)
    fluid = np.ones(rho.size, bool) if sol is None else sol == 0
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    assert state_err_fluid(g.get_state(), (fo, go), fluid) < 1e-13
    g.step(3)
    assert o.step(fo, go, 3) == 0
    assert state_err_fluid(g.get_state(), (fo, go), fluid) < 1e-12
    a, b = g.fields(), o.fields(fo, go)
    e = field_err({k: v[..., fluid] for k, v in a.items()}, {k: v[..., fluid] for k, v in b.items() if k != "rc"},
                  p["chi"])
    assert max(e.values()) < 1e-12, e
    # the wetting gradients change the result (so the parity is not vacuous)
    n = tel.Lattice(lattice, *shape, *([] if lattice == 1 else [1]), dict(p, wet_rho=0.0, wet_phi=0.0), bc=bc)
    n.init(rho, phi, u)
    n.step(3)
    assert np.max(np.abs(n.get_state()[0] - g.get_state()[0])) > 1e-7 * np.abs(fo).max()


@pytest.mark.parametrize("lattice,shape,bc,steps", [(0, (40, 36), (1, 1, 0), 150), (1, (16, 14, 12), (0, 1, 1), 30)])
def test_wetting_multi_step_fp64(orc, T10, lattice, shape, bc, steps):
    p = dict(base(T10, nu=0.1), **WET)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(steps)
    assert o.step(fo, go, steps) == 0
    a, b = g.fields(), o.fields(fo, go)
    e = field_err(a, {k: v for k, v in b.items() if k != "rc"}, p["chi"])
    assert max(e.values()) < 1e-10, e


@pytest.mark.parametrize("lattice,shape,bc,kind", [(0, (36, 28), (1, 1, 0), None), (0, (33, 29), (1, 0, 0), 1),
                                                   (1, (16, 12, 14), (1, 1, 0), None), (1, (14, 12, 13), (0, 0, 1), 1)])
def test_wetting_fp32_one_step(orc, T10, lattice, shape, bc, kind):
    p = dict(asymmetric(T10, force_form=1), **WET)
    sol = None if kind is None else mask(shape, kind)
    if sol is not None:
        p["solid"] = sol
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc, precision=tel.FP32_SHIFTED, amp=1e-2)
    fluid = np.ones(rho.size, bool) if sol is None else sol == 0
    g.init(rho, phi, u)
    g.step(2)
    f0, g0 = g.get_state()
    g.step(1)
    f1, g1 = g.get_state()
    nz = shape[2] if lattice == 1 else 1
    o1 = orc.Oracle(lattice, shape[0], shape[1], nz, p, bc=bc)
    assert o1.step(f0, g0, 1) == 0
    ef = np.max(np.abs(f0 - f1)[:, fluid] / np.max(np.abs(f0[:, fluid]), axis=0))
    eg = np.max(np.abs(g0 - g1)) / p["chi"]
    assert max(ef, eg) < 2e-5, (ef, eg)


def test_wetting_batch_matches_single_lattices(T10):
    """Batched cases with walls and their own wetting gradients (FP64)."""
    shapes = [(40, 32), (36, 28), (52, 20)]
    ps = [dict(asymmetric(T10), bc=(1, 1, 0), wet_rho=w_r, wet_phi=w_p)
          for w_r, w_p in ((0.02, -0.1), (-0.03, 0.2), (0.0, 0.0))]
    b = tel.Batch(shapes, ps)
    singles = []
    for k, (shape, p) in enumerate(zip(shapes, ps)):
        rg, rl, _, _ = tel.coexistence(p["a"], p["b"], p["R"], p["T"])
        rho, phi, u = inputs.drops(shape, rg, rl, p["chi"],
                                   [dict(center=(shape[0] / 2, 6.0), R=7.0, kind=1, u=(0.01, 0.0))], width=4.0)
        b.init(k, rho, phi, u)
        s = tel.Lattice(tel.D2Q9, shape[0], shape[1], 1, p)
        s.init(rho, phi, u)
        singles.append(s)
    b.step(25)
    for k, s in enumerate(singles):
        s.step(25)
        got, ref = b.fields(k), s.fields()
        assert np.max(np.abs(got["rho"] - ref["rho"]) / ref["rho"]) < 1e-12, k
        assert np.max(np.abs(got["phi"] - ref["phi"])) < 1e-12 * 5.0, k


def footprint(rho, nx, ny, rmid, row):
    """Length of the liquid's contact line on a wall row: nodes above the
    mid density, with linear interpolation at the two ends."""
    r = rho.reshape(ny, nx)[row]
    inside = r > rmid
    if not inside.any():
        return 0.0
    idx = np.nonzero(inside)[0]
    lo, hi = idx[0], idx[-1]
    fl = (r[lo] - rmid) / (r[lo] - r[lo - 1]) if lo > 0 else 0.0
    fr = (r[hi] - rmid) / (r[hi] - r[hi + 1]) if hi + 1 < nx else 0.0
    return float(hi - lo + fl + fr)


def test_drop_on_a_wetting_wall_spreads_or_beads(T10):
    """A half drop of liquid 1 (R = 16) sitting on the bottom wall of a
    96 x 48 box (walls in y, periodic in x, FP64): after 2000 steps (the
    footprint has settled to 0.1 node) its contact line on the wall is
    longer with wet_rho > 0 (the wall draws density: wetting) and shorter
    with wet_rho < 0 than with the neutral wall, where the angle is 90
    degrees (footprint 2 R).  The oracle's run of the same case gives 26.2,
    31.4 and 37.4 nodes for wet_rho = -0.06, 0, 0.06 (rho_l - rho_g)."""
    nx, ny, R = 96, 48, 16.0
    p = base(T10, nu=0.1, kappa1=0.01)
    rg, rl, _, _ = tel.coexistence(p["a"], p["b"], p["R"], p["T"])
    rho, phi, u = inputs.drops((nx, ny), rg, rl, p["chi"], [dict(center=(nx / 2, -0.5), R=R, kind=1)], width=4.0)
    rmid = 0.5 * (rg + rl)
    fp = {}
    for w in (-0.06, 0.0, 0.06):
        g = tel.Lattice(tel.D2Q9, nx, ny, 1, dict(p, wet_rho=w * (rl - rg)), bc=(0, 1, 0))
        g.init(rho, phi, u)
        g.step(2000)
        a = g.fields()
        assert np.all(np.isfinite(a["rho"]))
        fp[w] = footprint(a["rho"], nx, ny, rmid, 0)
    assert fp[0.06] > fp[0.0] + 4.0 and fp[-0.06] < fp[0.0] - 4.0, fp
    assert abs(fp[0.0] - 2 * R) < 2.0, fp
