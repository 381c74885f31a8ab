"""Carried moments (tel_params.moments = TEL_MOMENTS_CARRIED, the default
where it applies: D3Q27, FP32-shifted, periodic, nx % 32 == 0, ny % 4 == 0).
Each step adds its post-collision populations into the moments rho, phi
(Eqs. 6-8) of the nodes that the next step's pull brings them to, and the
next step's stencils read those instead of pulling the ring's populations
again.  Checked here through the C ABI:
- one step from a stepped state against the FP64 oracle (bar 2e-5, f
  relative to the node's largest f, g to chi, as the other FP32 one-step
  tests), with each stabiliser variant;
- the same after tel_set_state (the moments must be summed from the new
  state, not carried from the old one);
- multi-step runs against the oracle (1e-4 on density and phase field, the
  FP32 bar) and against the pulled moments, and the mass drift (1e-6);
- shapes where the mode does not apply run the pulled path, bit for bit.
"""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from tests.cases import A, B, RGAS, asymmetric, base
from tests.test_gpu_parity import setup_pair

pytestmark = pytest.mark.gpu

FP32 = tel.FP32_SHIFTED


@pytest.fixture(scope="module")
def T10():
    return tel.temperature_for_ratio(A, B, RGAS, 10.0)


def one_step_err(orc, p, shape, f0, g0, f1, g1):
    o = orc.Oracle(1, shape[0], shape[1], shape[2], p)
    assert o.step(f0, g0, 1) == 0
    ef = np.max(np.abs(f0 - f1) / np.max(np.abs(f0), axis=0))
    eg = np.max(np.abs(g0 - g1)) / p["chi"]
    return max(ef, eg)


@pytest.mark.parametrize("shape", [(64, 16, 12), (32, 24, 9), (64, 12, 10)])
@pytest.mark.parametrize("mode", [tel.GAMMA_CLOSED, tel.GAMMA_EXACT, tel.GAMMA_CLOSED_F64SUM])
def test_carried_one_step_against_oracle(orc, T10, shape, mode):
    """Steps 1-3 read moments from the scatter of the step before (after
    the moments kernel for step 1); the third is checked."""
    p = asymmetric(T10, force_form=1, gamma_mode=mode)
    g, o, rho, phi, u = setup_pair(orc, 1, shape, p, precision=FP32, amp=1e-2)
    g.init(rho, phi, u)
    g.step(2)
    f0, g0 = g.get_state()
    g.step(1)
    f1, g1 = g.get_state()
    e = one_step_err(orc, p, shape, f0, g0, f1, g1)
    assert e < 2e-5, e
    assert g.gamma_fallbacks() == 0


def test_carried_moments_follow_set_state(orc, T10):
    """After tel_set_state the next step takes the moments of the new state:
    a state from a different run is set mid-run and one step checked."""
    shape = (64, 16, 12)
    p = asymmetric(T10, force_form=1)
    g, o, rho, phi, u = setup_pair(orc, 1, shape, p, precision=FP32, amp=1e-2, seed=3)
    h, _, rho2, phi2, u2 = setup_pair(orc, 1, shape, p, precision=FP32, amp=1e-2, seed=4, n_drops=1)
    g.init(rho, phi, u)
    h.init(rho2, phi2, u2)
    g.step(4)
    h.step(2)
    f0, g0 = h.get_state()
    g.set_state(f0, g0)
    g.step(1)
    f1, g1 = g.get_state()
    e = one_step_err(orc, p, shape, f0, g0, f1, g1)
    assert e < 2e-5, e
    # and a second step from there (moments carried again)
    f0, g0 = f1, g1
    g.step(1)
    f1, g1 = g.get_state()
    assert one_step_err(orc, p, shape, f0, g0, f1, g1) < 2e-5


@pytest.mark.parametrize("steps", [7, 40])
def test_carried_runs_against_oracle_and_pulled(orc, T10, steps):
    """Several rotations of the three moment arrays: against the FP64 oracle
    (1e-4, the FP32 bar), against the pulled moments (the same update with
    the stencils' moments rounded differently: 1e-5), and mass drift."""
    shape = (32, 16, 16)
    p = base(T10, nu=0.1)
    g, o, rho, phi, u = setup_pair(orc, 1, shape, p, precision=FP32)
    q = tel.Lattice(tel.D3Q27, *shape, dict(p, precision=FP32, moments=tel.MOMENTS_PULLED))
    g.init(rho, phi, u)
    q.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(steps)
    q.step(steps)
    assert o.step(fo, go, steps) == 0
    a, b, c = g.fields(), o.fields(fo, go), q.fields()
    assert np.max(np.abs(a["rho"] - b["rho"]) / b["rho"]) < 1e-4
    assert np.max(np.abs(a["phi"] - b["phi"])) / p["chi"] < 1e-4
    assert np.max(np.abs(a["rho"] - c["rho"]) / c["rho"]) < 1e-5
    assert np.max(np.abs(a["phi"] - c["phi"])) / p["chi"] < 1e-5
    assert abs(a["rho"].sum() / rho.sum() - 1) < 1e-6


def test_carried_mode_elsewhere_is_the_pulled_path(T10):
    """Where the carried moments do not apply (nx % 32 != 0) both modes run
    the same kernel: identical states."""
    shape = (36, 16, 10)
    p = base(T10, nu=0.1, precision=FP32)
    rng = np.random.default_rng(2)
    rl = tel.coexistence(A, B, RGAS, T10)[1]
    rho = rl * (1.0 + 1e-2 * rng.standard_normal(int(np.prod(shape))))
    phi = 0.1 * rng.standard_normal(rho.size)
    u = 1e-3 * rng.standard_normal(3 * rho.size)
    s = []
    for m in (tel.MOMENTS_CARRIED, tel.MOMENTS_PULLED):
        lat = tel.Lattice(tel.D3Q27, *shape, dict(p, moments=m))
        lat.init(rho, phi, u)
        lat.step(5)
        s.append(lat.get_state())
    assert np.array_equal(s[0][0], s[1][0]) and np.array_equal(s[0][1], s[1][1])
