"""The van der Waals and Peng-Robinson equations of state on the CUDA path:
state and field parity with the FP64 oracle (the same bars as for Eq. 4),
FP32-shifted storage against the FP64 oracle, and flat-interface
coexistence at the common-tangent densities of each equation of state."""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from tests.cases import asymmetric, base
from tests.test_gpu_parity import field_err, setup_pair, state_err

pytestmark = pytest.mark.gpu

R = 1.0
EOS = {"vdw": dict(eos=tel.EOS_VDW, a=9.0 / 49.0, b=2.0 / 21.0, omega=0.0),
       "pr": dict(eos=tel.EOS_PR, a=2.0 / 49.0, b=2.0 / 21.0, omega=0.344)}


def eos_params(name, ratio, maker=base, **kw):
    e = EOS[name]
    T = tel.temperature_for_ratio(e["a"], e["b"], R, ratio, eos=e["eos"], omega=e["omega"])
    p = maker(T, **kw)
    p.update(a=e["a"], b=e["b"], R=R, eos=e["eos"], omega=e["omega"])
    return p


@pytest.mark.parametrize("name", ["vdw", "pr"])
@pytest.mark.parametrize("lattice,shape,bc", [(0, (70, 37), (0, 1, 0)), (1, (9, 10, 11), (1, 0, 0))])
def test_one_step_state_parity_fp64(orc, name, lattice, shape, bc):
    p = eos_params(name, 10.0, asymmetric)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(1)
    assert o.step(fo, go, 1) == 0
    assert state_err(g.get_state(), (fo, go)) < 1e-12
    e = field_err(g.fields(), o.fields(fo, go), p["chi"])
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("name", ["vdw", "pr"])
def test_multi_step_field_parity_fp64(orc, name):
    p = eos_params(name, 10.0)
    g, o, rho, phi, u = setup_pair(orc, 0, (64, 64), p)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(100)
    assert o.step(fo, go, 100) == 0
    e = field_err(g.fields(), o.fields(fo, go), p["chi"])
    assert max(e.values()) < 1e-10, e


@pytest.mark.parametrize("name", ["vdw", "pr"])
def test_fp32_shifted_against_fp64_oracle(orc, name):
    p = eos_params(name, 10.0)
    g, o, rho, phi, u = setup_pair(orc, 0, (64, 64), p, precision=tel.FP32_SHIFTED)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(100)
    o.step(fo, go, 100)
    a, b = g.fields(), o.fields(fo, go)
    assert np.max(np.abs(a["rho"] - b["rho"]) / b["rho"]) < 1e-4
    assert np.max(np.abs(a["phi"] - b["phi"])) / p["chi"] < 1e-4
    assert abs(a["rho"].sum() / rho.sum() - 1) < 1e-6


@pytest.mark.parametrize("name", ["vdw", "pr"])
def test_flat_interface_coexistence(name):
    """Liquid-gas model (lambda2 = lambda3 = kappa2 = kappa3 = 0) with a
    lattice-consistent force: a relaxed flat slab sits at the equation of
    state's common-tangent densities."""
    # van der Waals' free energy is the stiffer one at ratio 10: with the
    # weight lambda1 = 0.6 of the other two the slab goes unstable after
    # ~5000 steps (oracle and library alike); lambda1 = 0.1 relaxes.
    lam1 = 0.1 if name == "vdw" else 0.6
    p = eos_params(name, 10.0, base, lambda1=lam1, lambda2=0.0, lambda3=0.0, kappa1=0.05, kappa2=0.0, kappa3=0.0)
    lat = tel.Lattice(tel.D2Q9, 256, 4, 1, p)
    x = np.arange(256)
    s = 0.5 * (np.tanh((x - 64) / 6.0) - np.tanh((x - 192) / 6.0))
    rho = np.tile(lat.rho_g + (lat.rho_l - lat.rho_g) * s, 4)
    lat.init(rho, np.zeros_like(rho), np.zeros((2, rho.size)))
    lat.step(8000)
    f = lat.fields()
    r = f["rho"][:256]
    assert abs(r[0] / lat.rho_g - 1) < 0.02, (r[0], lat.rho_g)
    assert abs(r[128] / lat.rho_l - 1) < 0.005, (r[128], lat.rho_l)
    assert np.abs(f["u"]).max() < 1e-3
