"""CPU pins of the two FP32 forms that the FP32-storage step uses where the
plain FP32 evaluation would cancel, in float32 emulation (numpy) against FP64.
No GPU is involved; the GPU parity tests check the kernel itself.

- The gas-side chemical potential of Eq. 4, rho < sqrt(rho_g rho_l), as the
  sum of two cancellation-free products: RT ln(rho/rho_g) and
  D (8RT b B - 2a), D = rho - rho_g.  The identity behind B is checked in
  exact rational arithmetic; the float32 evaluation against the oracle's
  FP64 chemical potential.
- The KBC collision (paragraph after Eq. 8) as the FP32 path forms it: FP32
  scalar products and ratio q = <ds|dh>/<dh|dh>, beta gamma = 1 - (2 beta - 1) q
  in FP64, output (1 - beta gamma) Delta + f^eq(u + F/rho) + (beta gamma -
  2 beta) Delta s on populations stored as f - w rho_ref.  Against the
  oracle's FP64 collision, the output error stays at the FP32 rounding of the
  populations, also near equilibrium, where q itself is poorly conditioned.
"""
from fractions import Fraction

import numpy as np
import pytest

from tests.cases import A, B, RGAS, asymmetric, base

f32 = np.float32


def test_gas_side_divided_difference_identity():
    """h(rho) - h(rho_g) = -b D B, h(rho) = (24 - 2 b rho)/(b rho - 4)^3,
    r = 1/(b rho - 4), q = 1/(b rho_g - 4), B = 2 r q [8 (r^2 + r q + q^2) - (r + q)]:
    exact in rational arithmetic."""
    b = Fraction(1, 5)
    rg = Fraction(7, 1000)

    def h(x):
        return (24 - 2 * b * x) / (b * x - 4) ** 3

    q = 1 / (b * rg - 4)
    for x in (Fraction(3, 1000), Fraction(7001, 1000000), Fraction(1, 10), Fraction(2, 7), Fraction(19, 4)):
        r = 1 / (b * x - 4)
        Bv = 2 * r * q * (8 * (r * r + r * q + q * q) - (r + q))
        assert h(x) - h(rg) == -b * (x - rg) * Bv


@pytest.mark.parametrize("ratio", [3.0, 10.0, 100.0, 1000.0])
def test_gas_side_float32_accuracy(orc, ratio):
    """float32 pieces (rho_g as two floats; the two products summed in
    double-float arithmetic -- FMA product errors and a TwoSum -- and rounded
    once to float32, as the kernel does) against the oracle's FP64
    (lambda1/2)(dPsi~(rho) - dPsi~(rho_g)) over [0.3 rho_g, sqrt(rho_g rho_l)]:
    within 1e-6 of the largest |mu| there (measured 1e-7 to 5e-7)."""
    T = orc.temperature_for_ratio(A, B, RGAS, ratio)
    rg, rl, _, _ = orc.coexistence(A, B, RGAS, T)
    RT, lam1h = RGAS * T, 0.3
    rho = np.geomspace(0.3 * rg, np.sqrt(rg * rl), 801).astype(f32)
    d0 = orc.dpsi_tilde(A, B, RGAS, T, rg)
    exact = np.array([lam1h * (orc.dpsi_tilde(A, B, RGAS, T, float(x)) - d0) for x in rho])
    rg_hi = f32(rg)
    rg_lo = f32(rg - float(rg_hi))
    D = (rho - rg_hi) - rg_lo
    L = np.log1p(D * f32(1.0 / rg))
    r = f32(1) / (f32(B) * rho - f32(4))
    q = f32(1.0 / (B * rg - 4.0))
    rq = r + q
    Bv = (f32(2) * q * r) * (f32(8) * (r * rq + f32(q * q)) - rq)
    c = f32(lam1h * 8 * RT * B) * Bv - f32(lam1h * 2 * A)
    def fmaf(a, b, c):
        # float32 inputs: the product is exact in float64, one rounding to float32
        return f32(np.float64(a) * np.float64(b) + np.float64(c))

    g = lam1h * RT
    g_hi = f32(g)
    g_lo = f32(g - float(g_hi))
    p1 = g_hi * L
    p2 = D * c
    e = fmaf(g_hi, L, -p1)
    e = fmaf(g_lo, L, e)
    e = e + fmaf(D, c, -p2)
    sm = p1 + p2
    bp = sm - p1
    e = e + ((p1 - (sm - bp)) + (p2 - bp))
    got = (sm + e).astype(np.float64)
    ref64 = f32(g * L.astype(np.float64) + D.astype(np.float64) * c.astype(np.float64))
    # the double-float sum rounds to the FP64 sum's float32 value, within one ulp
    assert np.max(np.abs(got - ref64) / np.maximum(np.abs(ref64), 1e-30)) <= 2.0 ** -23
    assert np.max(np.abs(got - exact)) <= 1e-6 * np.max(np.abs(exact))


def factors32(u):
    """One-dimensional factors of the entropic equilibrium, float32, [3] per axis."""
    S = np.sqrt(f32(1) + f32(3) * u * u)
    t = f32(2) - S
    return np.stack([f32(1 / 6) * t * (S - f32(2) * u) / (f32(1) + u), f32(2 / 3) * t,
                     f32(1 / 6) * t * (S + f32(2) * u) / (f32(1) - u)], axis=-1)


def collide_fp32(o, ft, F, rho_ref, beta):
    """Post-collision stored populations (f - w rho_ref) of one node, formed
    in float32 as the FP32 path does (beta gamma rounded once from the
    float32 ratio)."""
    D = o.D
    c = o.c[:, :3]
    w = o.w.astype(f32)
    rest = o.Q // 2
    wr = w * f32(rho_ref)
    rho = f32(rho_ref) + ft.sum(dtype=f32)
    j = (c[:, :D].astype(f32) * ft[:, None]).sum(axis=0, dtype=f32)
    cs2 = f32(1 / 3)
    Pi = np.zeros(6, dtype=f32)
    for a in range(D):
        Pi[a] = (c[:, a] != 0).astype(f32) @ ft + f32(rho_ref) * cs2
    for k, (a, bb) in enumerate(((0, 1), (0, 2), (1, 2))):
        if bb < D:
            Pi[3 + k] = (c[:, a] * c[:, bb]).astype(f32) @ ft
    u = np.zeros(3, dtype=f32)
    uF = np.zeros(3, dtype=f32)
    u[:D] = j / rho
    uF[:D] = u[:D] + F[:D].astype(f32) / rho
    e, eF = factors32(u), factors32(uF)
    for a in range(D, 3):
        e[a] = eF[a] = np.array([0, 1, 0], dtype=f32)
    M0, M1, M2 = e.sum(axis=1), e[:, 2] - e[:, 0], e[:, 2] + e[:, 0]
    dPi = np.zeros(6, dtype=f32)
    dPi[0] = Pi[0] - rho * M2[0] * M0[1] * M0[2]
    dPi[1] = Pi[1] - rho * M0[0] * M2[1] * M0[2]
    dPi[3] = Pi[3] - rho * M1[0] * M1[1] * M0[2]
    if D == 3:
        dPi[2] = Pi[2] - rho * M0[0] * M0[1] * M2[2]
        dPi[4] = Pi[4] - rho * M1[0] * M0[1] * M1[2]
        dPi[5] = Pi[5] - rho * M0[0] * M1[1] * M1[2]
    tr = (dPi[0] + dPi[1] + dPi[2]) / f32(D)
    ds = np.zeros(o.Q, dtype=f32)
    for i in range(o.Q):
        nz = np.flatnonzero(c[i])
        if len(nz) == 1:
            ds[i] = f32(0.5) * (dPi[nz[0]] - tr)
        elif len(nz) == 2:
            k = {(0, 1): 3, (0, 2): 4, (1, 2): 5}[tuple(nz)]
            ds[i] = f32(0.25 * c[i, nz[0]] * c[i, nz[1]]) * dPi[k]
    idx = tuple(c[:, a] + 1 for a in range(3))
    feq = rho * e[0][idx[0]] * e[1][idx[1]] * e[2][idx[2]]
    feqF = rho * eF[0][idx[0]] * eF[1][idx[1]] * eF[2][idx[2]]
    dl = ft - (feq - wr)
    dh = dl - ds
    sh = np.sum(ds * dh / feq, dtype=f32)
    hh = np.sum(dh * dh / feq, dtype=f32)
    gb = 2.0 * beta
    if hh > f32(1e-30) * rho * rho:
        gb = 1.0 - (2.0 * beta - 1.0) * float(sh / hh)
    gb = f32(gb)
    out = (f32(1) - gb) * dl + (feqF - wr) + (gb - f32(2 * beta)) * ds
    out[rest] = ft.sum(dtype=f32) - (out.sum(dtype=f32) - out[rest])
    return out


@pytest.mark.parametrize("lattice", [0, 1])
@pytest.mark.parametrize("amp", [1e-2, 1e-4, 1e-7])
def test_fp32_collision_against_fp64_oracle(orc, lattice, amp):
    """Random nodes, gas and liquid densities, |u| < 0.1, a force and
    non-equilibrium parts of relative size amp (1e-7: <dh|dh> near the FP32
    rounding of the populations).  Bar: 2e-6 of the node's largest f
    (measured up to 8.7e-7).  Planted mistakes in the emulation (the sign of
    the Delta s or Delta h term, the dropped shift, force or trace, the
    inverted ratio) give 9e-5 to 1 at amp = 1e-2."""
    T = orc.temperature_for_ratio(A, B, RGAS, 10.0)
    p = asymmetric(T) if lattice == 1 else base(T)
    o = orc.Oracle(lattice, 4, 4, 1 if lattice == 0 else 4, p)
    rho_ref = o.rho_g
    g = np.random.default_rng(7 + lattice)
    worst = 0.0
    for n in range(60):
        rho = o.rho_g * (1.0 + 0.5 * g.random()) if n % 2 else o.rho_l * (1.0 + 0.1 * g.random())
        u = g.uniform(-0.1, 0.1, 3)
        u[o.D:] = 0.0
        F = g.uniform(-1e-4, 1e-4, 3) * rho
        F[o.D:] = 0.0
        f = o.feq(rho, u) * (1.0 + amp * g.standard_normal(o.Q))
        ft = (f - o.w * rho_ref).astype(f32)
        fin = ft.astype(np.float64) + o.w * rho_ref
        post, _, _ = o.collide_f(fin, F)
        got = collide_fp32(o, ft, F, rho_ref, o.beta).astype(np.float64) + o.w * rho_ref
        worst = max(worst, np.max(np.abs(got - post)) / np.max(np.abs(fin)))
    assert worst < 2e-6, worst
