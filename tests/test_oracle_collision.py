"""Pins of the oracle's single-node pieces: velocity sets, the entropic
equilibrium, the KBC split and stabiliser with exact-difference forcing
(paragraph after Eq. 8, which names the scheme), and the phase-field BGK.

Every check computes its expectation by a route of its own: moments are
summed here in numpy, the stress part Delta s is recovered here by solving the
full natural-moment linear system, and the closed forms are the textbook ones.
"""
import itertools

import numpy as np
import pytest

from tests.cases import A, B, RGAS, asymmetric

LATTICES = [(0, 2), (1, 3)]


@pytest.fixture(scope="module")
def T10(orc):
    return orc.temperature_for_ratio(A, B, RGAS, 10.0)


def make(orc, lattice, T, **kw):
    return orc.Oracle(lattice, 4, 4, 1 if lattice == 0 else 4, asymmetric(T, **kw))


def moment_matrix(c, D):
    """Rows: natural moments prod_a c_a^{e_a}, e in {0,1,2}^D."""
    rows, exps = [], []
    for e in itertools.product(range(3), repeat=D):
        rows.append(np.prod([c[:, a] ** e[a] for a in range(D)], axis=0))
        exps.append(e)
    return np.array(rows, dtype=float), exps


@pytest.mark.parametrize("lattice,D", LATTICES)
def test_velocity_set(orc, T10, lattice, D):
    o = make(orc, lattice, T10)
    c, w = o.c[:, :D].astype(float), o.w
    assert len(w) == 3 ** D and w.sum() == pytest.approx(1.0, abs=1e-15)
    I = np.eye(D)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), I / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-15)
    # fourth-order isotropy: sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    ref = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(m4, ref, atol=1e-15)
    # every velocity has its opposite; the natural moments form a basis
    for ci in c:
        assert any(np.array_equal(-ci, cj) for cj in c)
    M, _ = moment_matrix(c, D)
    assert np.linalg.matrix_rank(M) == 3 ** D


@pytest.mark.parametrize("lattice,D", LATTICES)
def test_entropic_equilibrium(orc, T10, lattice, D):
    o = make(orc, lattice, T10)
    c, w = o.c[:, :D].astype(float), o.w
    g = np.random.default_rng(3)
    assert np.allclose(o.feq(2.3, np.zeros(3)), 2.3 * w, rtol=1e-15, atol=0)
    for _ in range(20):
        rho = g.uniform(0.01, 10.0)
        u = np.zeros(3)
        u[:D] = g.uniform(-0.6, 0.6, D)
        f = o.feq(rho, u)
        assert (f > 0).all()
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(f @ c, rho * u[:D], rtol=1e-13, atol=1e-14 * rho)
        P = np.einsum("i,ia,ib->ab", f, c, c)
        S = np.sqrt(1 + 3 * u[:D] ** 2)
        for a in range(D):
            # one-dimensional entropic equilibrium: second moment rho (2 S - 1)/3
            assert P[a, a] == pytest.approx(rho * (2 * S[a] - 1) / 3, rel=1e-13)
            for b in range(D):
                if a != b:
                    assert P[a, b] == pytest.approx(rho * u[a] * u[b], rel=1e-12, abs=1e-14 * rho)
        # minimiser of H = sum f ln(f/w) under fixed rho, j: ln(f_i/w_i) is
        # affine in c_i (Lagrange multipliers of mass and momentum)
        X = np.hstack([np.ones((len(w), 1)), c])
        y = np.log(f / w)
        coef, *_ = np.linalg.lstsq(X, y, rcond=None)
        assert np.abs(X @ coef - y).max() < 1e-12


def random_population(o, D, g, rho=None, amp=0.05):
    rho = g.uniform(0.5, 5.0) if rho is None else rho
    u = np.zeros(3)
    u[:D] = g.uniform(-0.15, 0.15, D)
    f = o.feq(rho, u) * (1.0 + amp * g.uniform(-1, 1, o.Q))
    return f


@pytest.mark.parametrize("lattice,D", LATTICES)
def test_kbc_stress_part_and_conservation(orc, T10, lattice, D):
    o = make(orc, lattice, T10)
    c = o.c[:, :D].astype(float)
    M, exps = moment_matrix(c, D)
    g = np.random.default_rng(5)
    for _ in range(10):
        f = random_population(o, D, g)
        fo, ds, gamma = o.collide_f(f, np.zeros(3))
        rho = f.sum()
        u = np.zeros(3)
        u[:D] = (f @ c) / rho
        dl = f - o.feq(rho, u)
        # Delta s solved here from the natural-moment system: the deviatoric
        # second moments of Delta, every other natural moment zero
        Pi = np.einsum("i,ia,ib->ab", dl, c, c)
        tr = np.trace(Pi)
        target = np.zeros(len(exps))
        for k, e in enumerate(exps):
            if sum(e) == 2 and max(e) == 2:
                a = e.index(2)
                target[k] = Pi[a, a] - tr / D
            elif sum(e) == 2 and max(e) == 1:
                a, b = [i for i in range(D) if e[i] == 1]
                target[k] = Pi[a, b]
        ds_ref = np.linalg.solve(M, target)
        assert np.allclose(ds, ds_ref, rtol=1e-10, atol=1e-14 * rho)
        # mass and momentum are conserved by the collision without force
        assert fo.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(fo @ c, f @ c, atol=1e-14 * rho)
        # stabiliser: the post-collision deviation from equilibrium is
        # orthogonal to Delta h in the entropic scalar product
        feq = o.feq(rho, u)
        dh = dl - ds_ref
        post = fo - feq
        ip = lambda x, y: np.sum(x * y / feq)
        assert abs(ip(post, dh)) < 1e-9 * np.sqrt(ip(post, post) * ip(dh, dh)) + 1e-300
        # the non-stress part relaxes by (1 - gamma beta), the stress by (1 - 2 beta)
        assert np.allclose(post, (1 - 2 * o.beta) * ds_ref + (1 - gamma * o.beta) * dh,
                           atol=1e-13 * rho)


@pytest.mark.parametrize("lattice,D", LATTICES)
def test_kbc_limits(orc, T10, lattice, D):
    g = np.random.default_rng(7)
    # tau = 1 (nu = 1/6): beta = 1/2 gives gamma = 2 and f* = f^eq exactly
    o = make(orc, lattice, T10, nu=1.0 / 6.0)
    c = o.c[:, :D].astype(float)
    f = random_population(o, D, g)
    fo, _, gamma = o.collide_f(f, np.zeros(3))
    rho = f.sum()
    u = np.zeros(3)
    u[:D] = (f @ c) / rho
    assert gamma == 2.0
    assert np.allclose(fo, o.feq(rho, u), rtol=1e-13)
    # at equilibrium nothing changes; with Delta h = 0 the stabiliser is 2
    o = make(orc, lattice, T10)
    feq = o.feq(1.7, np.array([0.05, -0.02, 0.03]))
    fo, ds, gamma = o.collide_f(feq, np.zeros(3))
    assert np.allclose(fo, feq, rtol=1e-13, atol=1e-16)
    assert gamma == 2.0


@pytest.mark.parametrize("lattice,D", LATTICES)
def test_exact_difference_forcing(orc, T10, lattice, D):
    o = make(orc, lattice, T10)
    c = o.c[:, :D].astype(float)
    g = np.random.default_rng(9)
    for _ in range(10):
        f = random_population(o, D, g)
        F = np.zeros(3)
        F[:D] = g.uniform(-0.05, 0.05, D)
        fo, _, _ = o.collide_f(f, F)
        fo0, _, _ = o.collide_f(f, np.zeros(3))
        rho = f.sum()
        u = np.zeros(3)
        u[:D] = (f @ c) / rho
        # the forcing term is f^eq(rho, u + F/rho) - f^eq(rho, u)
        assert np.allclose(fo - fo0, o.feq(rho, u + F / rho) - o.feq(rho, u), atol=1e-15 * rho)
        assert fo.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(fo @ c - f @ c, F[:D], atol=1e-14 * rho)


@pytest.mark.parametrize("lattice,D", LATTICES)
def test_phase_field_bgk(orc, T10, lattice, D):
    o = make(orc, lattice, T10)
    p = o.params
    c = o.c[:, :D].astype(float)
    g = np.random.default_rng(11)
    for _ in range(10):
        phi, mu = g.uniform(-5, 5), g.uniform(-0.1, 0.1)
        u = np.zeros(3)
        u[:D] = g.uniform(-0.1, 0.1, D)
        ge = o.geq(phi, mu, u)
        assert ge.sum() == pytest.approx(phi, rel=1e-13, abs=1e-14)
        assert np.allclose(ge @ c, phi * u[:D], atol=1e-14)
        P = np.einsum("i,ia,ib->ab", ge, c, c)
        assert np.allclose(P, p["Gamma"] * mu * np.eye(D) + phi * np.outer(u[:D], u[:D]), atol=1e-14)
        gin = ge * (1 + 0.1 * g.uniform(-1, 1, o.Q))
        go = o.collide_g(gin, phi, mu, u)
        assert np.allclose(go, gin - (gin - ge) / p["tau_g"], atol=1e-15)
