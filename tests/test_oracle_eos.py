"""Pins of the oracle's van der Waals and Peng-Robinson equations of state
(the alternatives the text names next to Eq. 4; textbook forms):
closed-form critical points, the pressure written out directly, the
hand-differentiated chemical potential against finite differences, the law
of corresponding states, and the Maxwell equal-area rule."""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as o

R = 1.0
VDW = (o.VDW, 9.0 / 49.0, 2.0 / 21.0, 0.0)
PR = (o.PR, 2.0 / 49.0, 2.0 / 21.0, 0.344)


def p_direct(kind, a, b, T, rho, omega):
    """The pressure as the equation of state states it."""
    if kind == o.VDW:
        return rho * R * T / (1 - b * rho) - a * rho * rho
    k = 0.37464 + 1.54226 * omega - 0.26992 * omega ** 2
    Tc = 0.07780 * a / (0.45724 * b * R)
    alpha = (1 + k * (1 - np.sqrt(T / Tc))) ** 2
    return rho * R * T / (1 - b * rho) - a * alpha * rho * rho / (1 + 2 * b * rho - b * b * rho * rho)


def test_vdw_critical_point_closed_form():
    kind, a, b, _ = VDW
    Tc, rc = o.eos_critical_point(kind, a, b, R)
    assert Tc == pytest.approx(8 * a / (27 * b * R), rel=1e-6)
    assert rc == pytest.approx(1 / (3 * b), rel=1e-5)
    assert o.eos_p(kind, a, b, R, Tc, rc) == pytest.approx(a / (27 * b * b), rel=1e-5)


def test_pr_critical_point_closed_form():
    kind, a, b, w = PR
    Tc, rc = o.eos_critical_point(kind, a, b, R, w)
    assert Tc == pytest.approx(0.07780 * a / (0.45724 * b * R), rel=1e-4)
    Zc = o.eos_p(kind, a, b, R, Tc, rc, w) / (rc * R * Tc)
    assert Zc == pytest.approx(0.3074, abs=2e-3)


@pytest.mark.parametrize("eos", [VDW, PR])
@pytest.mark.parametrize("Tr", [0.6, 0.85, 1.2])
def test_pressure_and_chemical_potential(eos, Tr):
    kind, a, b, w = eos
    Tc = o.eos_critical_point(kind, a, b, R, w)[0]
    T = Tr * Tc
    for rho in (0.01, 0.3, 1.5, 4.0, 8.0):
        assert o.eos_p(kind, a, b, R, T, rho, w) == pytest.approx(p_direct(kind, a, b, T, rho, w), rel=1e-11,
                                                                   abs=1e-13)
        h = 1e-5 * rho
        fd = (o.eos_psi(kind, a, b, R, T, rho + h, w) - o.eos_psi(kind, a, b, R, T, rho - h, w)) / (2 * h)
        assert o.eos_dpsi(kind, a, b, R, T, rho, w) == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("eos", [VDW, PR])
@pytest.mark.parametrize("ratio", [10.0, 100.0, 1000.0])
def test_coexistence_is_a_common_tangent(eos, ratio):
    kind, a, b, w = eos
    T = o.eos_temperature_for_ratio(kind, a, b, R, ratio, w)
    rg, rl, mu, p = o.eos_coexistence(kind, a, b, R, T, w)
    assert rl / rg == pytest.approx(ratio, rel=1e-6)
    rc = o.eos_critical_point(kind, a, b, R, w)[1]
    assert rg < rc < rl
    assert o.eos_p(kind, a, b, R, T, rg, w) == pytest.approx(o.eos_p(kind, a, b, R, T, rl, w), rel=1e-9)
    assert o.eos_dpsi(kind, a, b, R, T, rg, w) == pytest.approx(o.eos_dpsi(kind, a, b, R, T, rl, w), rel=1e-9,
                                                                 abs=1e-12)


def test_vdw_corresponding_states():
    """Reduced coexistence densities of van der Waals fluids depend on the
    reduced temperature only."""
    out = []
    for a, b in ((9.0 / 49.0, 2.0 / 21.0), (0.5, 0.3)):
        Tc, rc = 8 * a / (27 * b * R), 1 / (3 * b)
        rg, rl, _, _ = o.eos_coexistence(o.VDW, a, b, R, 0.8 * Tc)
        out.append((rg / rc, rl / rc))
    assert out[0][0] == pytest.approx(out[1][0], rel=1e-8)
    assert out[0][1] == pytest.approx(out[1][1], rel=1e-8)


@pytest.mark.parametrize("eos", [VDW, PR])
def test_maxwell_equal_area(eos):
    """int_{v_l}^{v_g} p dv = p_sat (v_g - v_l), v = 1/rho: the equal-area
    form of the common tangent, by quadrature of the pressure alone."""
    kind, a, b, w = eos
    T = o.eos_temperature_for_ratio(kind, a, b, R, 20.0, w)
    rg, rl, _, ps = o.eos_coexistence(kind, a, b, R, T, w)
    area, _ = integrate.quad(lambda v: p_direct(kind, a, b, T, 1.0 / v, w), 1 / rl, 1 / rg, limit=400,
                             epsabs=1e-14, epsrel=1e-12)
    assert area == pytest.approx(ps * (1 / rg - 1 / rl), rel=1e-7)
