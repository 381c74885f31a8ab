"""Pins of the oracle's thermodynamics against what the paper and textbook
thermodynamics fix: the Carnahan-Starling pressure, the critical point, the
common-tangent construction (text after Eq. 4) and the three minima of the
bulk free energy (Fig. 1 caption)."""
import numpy as np
import pytest
from scipy.integrate import quad

from tests.cases import A, B, RGAS, base


def cs_pressure(rho, T, a=A, b=B, R=RGAS):
    """Textbook Carnahan-Starling EOS, p = rho R T (1+e+e^2-e^3)/(1-e)^3 - a rho^2,
    e = b rho / 4 (a different formula from rho dPsi/drho - Psi)."""
    e = b * rho / 4.0
    return rho * R * T * (1 + e + e * e - e ** 3) / (1 - e) ** 3 - a * rho * rho


@pytest.mark.parametrize("T", [0.035, 0.05, 0.065, 0.09])
def test_peos_is_carnahan_starling(orc, T):
    for rho in np.linspace(0.01, 15.0, 57):
        p = orc.p_eos(A, B, RGAS, T, rho)
        assert p == pytest.approx(cs_pressure(rho, T), rel=1e-11, abs=1e-13)


def test_dpsi_matches_finite_difference_of_eq4(orc):
    T = 0.05
    for rho in (0.01, 0.3, 2.0, 7.5, 12.0):
        h = 1e-5 * rho
        fd = (orc.psi_tilde(A, B, RGAS, T, rho + h) - orc.psi_tilde(A, B, RGAS, T, rho - h)) / (2 * h)
        assert orc.dpsi_tilde(A, B, RGAS, T, rho) == pytest.approx(fd, rel=1e-8, abs=1e-10)


def test_critical_point():
    """CS critical point: T_c = 0.3773 a/(bR), rho_c = 0.5218/b (the paper
    prints 0.3373, read as transposed digits of 0.3773), and dp/drho =
    d2p/drho2 = 0 there."""
    from oracle import oracle as orc
    Tc, rc = orc.critical_point(A, B, RGAS)
    assert Tc * B * RGAS / A == pytest.approx(0.3773, abs=2e-4)
    assert rc * B == pytest.approx(0.5218, abs=2e-4)
    h = 1e-3
    d1 = (cs_pressure(rc + h, Tc) - cs_pressure(rc - h, Tc)) / (2 * h)
    d2 = (cs_pressure(rc + h, Tc) - 2 * cs_pressure(rc, Tc) + cs_pressure(rc - h, Tc)) / h ** 2
    assert abs(d1) < 1e-8 and abs(d2) < 1e-5
    with pytest.raises(ValueError):
        orc.coexistence(A, B, RGAS, 1.01 * Tc)


@pytest.mark.parametrize("ratio", [3.0, 10.0, 100.0, 1000.0])
def test_common_tangent_and_equal_area(orc, ratio):
    T = orc.temperature_for_ratio(A, B, RGAS, ratio)
    rg, rl, mu, pc = orc.coexistence(A, B, RGAS, T)
    assert rl / rg == pytest.approx(ratio, rel=1e-9)
    # equal pressure (textbook CS) and equal chemical potential
    assert cs_pressure(rg, T) == pytest.approx(cs_pressure(rl, T), rel=1e-9, abs=1e-15)
    assert cs_pressure(rg, T) == pytest.approx(pc, rel=1e-9, abs=1e-15)
    assert orc.dpsi_tilde(A, B, RGAS, T, rg) == pytest.approx(orc.dpsi_tilde(A, B, RGAS, T, rl), abs=1e-11)
    # Maxwell equal-area rule in the specific volume v = 1/rho:
    # int_{v_l}^{v_g} (p(v) - p_coex) dv = 0, i.e. int (p - p_c)/rho^2 drho = 0
    val, _ = quad(lambda r: (cs_pressure(r, T) - pc) / r ** 2, rg, rl, limit=400, epsabs=1e-14)
    scale, _ = quad(lambda r: abs(cs_pressure(r, T) - pc) / r ** 2, rg, rl, limit=400)
    assert abs(val) < 1e-8 * scale


def test_bulk_free_energy_minima(orc):
    """Fig. 1 caption: three minima at (rho_g, 0), (rho_l, +chi), (rho_l, -chi);
    with C and Psi_0 from the common tangent, f_B vanishes there."""
    T = orc.temperature_for_ratio(A, B, RGAS, 10.0)
    p = base(T, lambda2=0.9, lambda3=1.7)
    o = orc.Oracle(orc.D2Q9, 4, 4, 1, p)
    chi = p["chi"]
    for (r0, f0) in ((o.rho_g, 0.0), (o.rho_l, chi), (o.rho_l, -chi)):
        assert abs(o.f_bulk(r0, f0)) < 1e-12
        hr, hf = 1e-4 * r0, 1e-4 * chi
        fb = lambda r, f: o.f_bulk(r, f)
        gr = (fb(r0 + hr, f0) - fb(r0 - hr, f0)) / (2 * hr)
        gf = (fb(r0, f0 + hf) - fb(r0, f0 - hf)) / (2 * hf)
        assert abs(gr) < 1e-7 and abs(gf) < 1e-7
        Hrr = (fb(r0 + hr, f0) - 2 * fb(r0, f0) + fb(r0 - hr, f0)) / hr ** 2
        Hff = (fb(r0, f0 + hf) - 2 * fb(r0, f0) + fb(r0, f0 - hf)) / hf ** 2
        Hrf = (fb(r0 + hr, f0 + hf) - fb(r0 + hr, f0 - hf) - fb(r0 - hr, f0 + hf)
               + fb(r0 - hr, f0 - hf)) / (4 * hr * hf)
        assert Hrr > 0 and Hff > 0 and Hrr * Hff - Hrf ** 2 > 0
    # nonnegative everywhere on a grid spanning the three phases
    for r in np.linspace(0.5 * o.rho_g, 1.2 * o.rho_l, 41):
        for f in np.linspace(-1.2 * chi, 1.2 * chi, 21):
            assert o.f_bulk(r, f) >= -1e-12
