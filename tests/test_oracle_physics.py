"""Physics pins of the oracle: a flat liquid-gas interface relaxes to the
coexistence densities of the common-tangent construction (text after Eq. 4,
Fig. 3: good agreement with the Maxwell construction)."""
import numpy as np
import pytest

from tests.cases import A, B, RGAS, base


def flat_interface(orc, ratio, form, steps=10000, nx=256, kappa1=0.05, width=12.0):
    T = orc.temperature_for_ratio(A, B, RGAS, ratio)
    # liquid-gas only: lambda2 = lambda3 = kappa2 = kappa3 = 0, phi = 0
    p = base(T, lambda2=0.0, lambda3=0.0, kappa1=kappa1, kappa2=0.0, kappa3=0.0,
             force_form=form)
    o = orc.Oracle(orc.D2Q9, nx, 1, 1, p)
    x = np.arange(nx)
    q = nx // 4
    s = 0.5 * (np.tanh((x - q) / (width / 2)) - np.tanh((x - 3 * q) / (width / 2)))
    rho = o.rho_g + (o.rho_l - o.rho_g) * s
    f, g = o.init(rho, np.zeros(nx), np.zeros((2, nx)))
    assert o.step(f, g, steps) == 0
    fl = o.fields(f, g)
    return o, fl


@pytest.mark.slow
@pytest.mark.parametrize("ratio", [3.0, 10.0])
def test_flat_interface_coexistence(orc, ratio):
    o, fl = flat_interface(orc, ratio, form=1)
    nx = len(fl["rho"])
    gas, liq = fl["rho"][0], fl["rho"][nx // 2]
    assert abs(gas / o.rho_g - 1) < 0.02
    assert abs(liq / o.rho_l - 1) < 0.005
    assert np.abs(fl["u"]).max() < 1e-3
    # the bulk thermodynamic pressure of both phases matches (p = 0 at coexistence)
    assert abs(fl["p"][0] - fl["p"][nx // 2]) < 2e-3 * o.rho_l / 3
