"""GPU parity of the exact per-node stabiliser (TEL_GAMMA_EXACT: the root of
the KBC entropy condition) against the oracle's exact stabiliser, and of the
FP32-shifted step on lattices with bounce-back walls.

Bars as in test_gpu_parity: FP64 <= 1e-12 after one step and <= 1e-10 after
many; one FP32 step from the same state <= 2e-5 (f relative to the node's
largest f, g to chi); FP32 runs <= 1e-4 on density and phase field.
The viscosities differ from 1/6: at beta = 1/2 every stabiliser is 2.
"""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from tests.cases import A, B, RGAS, asymmetric, base
from tests.test_gpu_parity import field_err, setup_pair, state_err

pytestmark = pytest.mark.gpu

EXACT = dict(gamma_mode=tel.GAMMA_EXACT)


@pytest.fixture(scope="module")
def T10():
    return tel.temperature_for_ratio(A, B, RGAS, 10.0)


CASES_1STEP = [
    (0, (8, 8), (0, 0, 0), 1),
    (0, (9, 11), (1, 1, 0), 1),
    (0, (70, 37), (0, 1, 0), 0),
    (1, (5, 6, 7), (1, 0, 1), 1),
    (1, (37, 11, 70), (0, 0, 0), 1),
]


@pytest.mark.parametrize("lattice,shape,bc,form", CASES_1STEP)
def test_exact_gamma_one_step_fp64(orc, T10, lattice, shape, bc, form):
    p = asymmetric(T10, force_form=form, **EXACT)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc, amp=3e-2)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    for _ in range(3):
        g.step(1)
        assert o.step(fo, go, 1) == 0
        assert state_err(g.get_state(), (fo, go)) < 1e-12
    assert g.gamma_fallbacks() == 0 and o.gamma_fallbacks() == 0


@pytest.mark.parametrize("lattice,shape,bc,steps", [
    (0, (64, 64), (0, 0, 0), 100),
    (0, (48, 40), (1, 1, 0), 100),
    (1, (16, 16, 16), (0, 0, 0), 40),
])
def test_exact_gamma_multi_step_fp64(orc, T10, lattice, shape, bc, steps):
    p = base(T10, nu=0.05, **EXACT)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(steps)
    assert o.step(fo, go, steps) == 0
    e = field_err(g.fields(), o.fields(fo, go), p["chi"])
    assert max(e.values()) < 1e-10, e


def test_exact_gamma_changes_the_update(orc, T10):
    """The exact root differs from the closed form away from equilibrium: the
    two modes give different states (so the exact path is exercised)."""
    pe = asymmetric(T10, **EXACT)
    pc = asymmetric(T10)
    ge, o, rho, phi, u = setup_pair(orc, 0, (32, 24), pe, amp=5e-2)
    gc = tel.Lattice(0, 32, 24, 1, pc)
    ge.init(rho, phi, u)
    gc.init(rho, phi, u)
    ge.step(5)
    gc.step(5)
    assert state_err(ge.get_state(), gc.get_state()) > 1e-9


@pytest.mark.parametrize("lattice,shape,bc", [
    (0, (40, 36), (0, 0, 0)),
    (0, (33, 29), (1, 1, 0)),          # FP32, walls
    (1, (16, 16, 16), (0, 0, 0)),      # vector phase A
    (1, (36, 10, 21), (1, 0, 1)),      # FP32, walls, scalar phase A
    (1, (13, 12, 11), (0, 1, 0)),
])
@pytest.mark.parametrize("mode", [tel.GAMMA_CLOSED, tel.GAMMA_EXACT, tel.GAMMA_CLOSED_F64SUM])
def test_fp32_one_step_state_parity(orc, T10, lattice, shape, bc, mode):
    """One FP32-shifted step against the oracle started from the same state,
    with each stabiliser variant (the FP64-summed closed form is the closed
    form for the oracle), periodic and walled."""
    p = asymmetric(T10, force_form=1, gamma_mode=mode)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc, precision=tel.FP32_SHIFTED, amp=1e-2)
    g.init(rho, phi, u)
    g.step(2)
    f0, g0 = g.get_state()
    g.step(1)
    f1, g1 = g.get_state()
    nz = shape[2] if lattice == 1 else 1
    o1 = orc.Oracle(lattice, shape[0], shape[1], nz, p, bc=bc)
    assert o1.step(f0, g0, 1) == 0
    ef = np.max(np.abs(f0 - f1) / np.max(np.abs(f0), axis=0))
    eg = np.max(np.abs(g0 - g1)) / p["chi"]
    assert max(ef, eg) < 2e-5, (ef, eg)
    assert g.gamma_fallbacks() == 0


@pytest.mark.parametrize("lattice,shape,bc,steps", [
    (0, (48, 40), (1, 1, 0), 100),
    (1, (16, 14, 18), (1, 0, 1), 40),
])
@pytest.mark.parametrize("mode", [tel.GAMMA_CLOSED, tel.GAMMA_EXACT])
def test_fp32_walled_runs_against_fp64_oracle(orc, T10, lattice, shape, bc, steps, mode):
    p = base(T10, nu=0.1, gamma_mode=mode)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc, precision=tel.FP32_SHIFTED)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(steps)
    assert o.step(fo, go, steps) == 0
    a, b = g.fields(), o.fields(fo, go)
    assert np.max(np.abs(a["rho"] - b["rho"]) / b["rho"]) < 1e-4
    assert np.max(np.abs(a["phi"] - b["phi"])) / p["chi"] < 1e-4
    # bounce-back conserves mass: no drift beyond FP32 rounding
    assert abs(a["rho"].sum() / rho.sum() - 1) < 1e-6
