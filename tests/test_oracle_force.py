"""Pins of the oracle's lattice-consistent force (force_form 1, reading of the
force after Eq. 8) in two and three dimensions, where every term couples the
components of G = grad rho:

  F_id = c_s^2 (3/2 G - 1/2 A[G]) + div(c_s^4 G G / (4 rho)),
  A[G]_a(x) = sum_i 3 w_i c_ia (c_i . G(x - c_i)).

With mu_rho = mu_phi = 0 the oracle's force is F_id alone.  For an oblique
plane wave rho = rho0 + eps cos(k.x) on a periodic box every stencil acts on
exponentials, and the lattice weights are products of the one-dimensional
weights (1/6, 2/3, 1/6), so each stencil factorises per axis:
  sum_c w(c) e^{i k c} = (2 + cos k)/3,  sum_c w(c) c e^{i k c} = i sin(k)/3,
  sum_c w(c) c^2 e^{i k c} = cos(k)/3.
The part of F linear in eps is c_s^2 (3/2 G - 1/2 A[G]) and the part
quadratic in eps is the divergence term at rho0; both are extracted from
F(eps) and F(-eps) and compared with these closed forms, written here from
the one-dimensional sums and not from the oracle's stencil loops.
"""
import itertools

import numpy as np
import pytest

from tests.cases import A, B, RGAS, base

CS2 = 1.0 / 3.0


def s0(k):
    return (2.0 + np.cos(k)) / 3.0


def s1(k):  # sum w c e^{-ikc} = -i sin(k)/3
    return -1j * np.sin(k) / 3.0


def s2(k):
    return np.cos(k) / 3.0


def closed_forms(kvec, D, theta, rho0):
    """(G1, linear force, quadratic force) at phases theta, per unit eps."""
    k = np.asarray(kvec[:D], float)
    # G of cos(theta): grad_a = 3 sum w c_a e^{i k.c} ... = Re[e^{i theta} ghat_a]
    ghat = np.array([1j * np.sin(k[a]) * np.prod([s0(k[d]) for d in range(D) if d != a]) for a in range(D)])
    # A[G]_a = Re[e^{i theta} sum_b M_ab ghat_b], M_ab = 3 sum_i w_i c_ia c_ib e^{-i k.c_i}
    M = np.zeros((D, D), complex)
    for a in range(D):
        for b in range(D):
            if a == b:
                M[a, a] = 3.0 * s2(k[a]) * np.prod([s0(k[d]) for d in range(D) if d != a])
            else:
                M[a, b] = 3.0 * s1(k[a]) * s1(k[b]) * np.prod([s0(k[d]) for d in range(D) if d not in (a, b)])
    ph = np.exp(1j * theta)
    G1 = np.real(np.outer(ghat, ph))
    AG = np.real(np.outer(M @ ghat, ph))
    lin = CS2 * (1.5 * G1 - 0.5 * AG)
    # quadratic: T = c_s^4 G1 G1/(4 rho0) with G1_a = gam_a (-sin theta),
    # G1_a G1_b = gam_a gam_b (1 - cos 2 theta)/2; the divergence stencil on
    # e^{2 i theta} gives i sin(2 k_b) prod_{d != b} (2 + cos 2 k_d)/3
    gam = np.imag(ghat)  # ghat = i gam
    div2 = np.array([np.sin(2 * k[b]) * np.prod([s0(2 * k[d]) for d in range(D) if d != b]) for b in range(D)])
    quad = np.array([CS2 * CS2 / (4.0 * rho0) * gam[a] * np.sum(gam * div2) * 0.5 * np.sin(2 * theta)
                     for a in range(D)])
    return G1, lin, quad


@pytest.mark.parametrize("lattice,shape,kint", [
    (0, (16, 12, 1), (1, 2, 0)),
    (0, (10, 10, 1), (3, 1, 0)),
    (1, (8, 6, 10), (1, 2, 3)),
    (1, (6, 6, 6), (1, -1, 2)),
])
def test_lattice_force_on_an_oblique_plane_wave(orc, lattice, shape, kint):
    T = orc.temperature_for_ratio(A, B, RGAS, 10.0)
    o = orc.Oracle(lattice, *shape, base(T, force_form=1))
    D = o.D
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = 2 * np.pi * np.array(kint, float) / np.array([nx, ny, nz], float)
    theta = (k[0] * x + k[1] * y + k[2] * z).ravel()
    rho0, eps = 2.0, 1e-3
    zero = np.zeros(o.N)
    Fp = o.force(rho0 + eps * np.cos(theta), zero, zero, zero)[:D]
    Fm = o.force(rho0 - eps * np.cos(theta), zero, zero, zero)[:D]
    G1, lin, quad = closed_forms(k, D, theta, rho0)
    # the gradient the force uses, against its closed form
    assert np.allclose(o.gradient(np.cos(theta))[:D], G1, rtol=0, atol=1e-14)
    lin_got = (Fp - Fm) / (2 * eps)
    quad_got = (Fp + Fm) / (2 * eps * eps)
    scale = np.abs(lin).max()
    # residue: the eps^3 term of T's 1/rho, ~ eps^2 c_s^4/(4 rho0^2) ~ 1e-8
    assert np.abs(lin_got - lin).max() < 1e-7 * scale
    qs = np.abs(quad).max()
    assert qs > 1e-4 * scale
    assert np.abs(quad_got - quad).max() < 1e-5 * qs + 1e-9 * scale  # O(eps^2) residue


def test_lattice_force_cross_terms_matter(orc):
    """On an oblique wave the off-diagonal part of A[G] is not small: dropping
    it (the mistake the closed form guards against) changes the linear force
    by a visible fraction."""
    T = orc.temperature_for_ratio(A, B, RGAS, 10.0)
    k = 2 * np.pi * np.array([1, 2, 0]) / np.array([16, 12, 1])
    theta = np.array([0.3, 1.1])
    D = 2
    ghat = np.array([1j * np.sin(k[a]) * s0(k[1 - a]) for a in range(D)])
    off = 3.0 * s1(k[0]) * s1(k[1])
    assert abs(off * ghat[1]) > 0.05 * abs(ghat[0])
