"""Pins of the oracle's exact stabiliser (the per-node root of the entropy
condition of the KBC collision; reading of "gamma solved per node" beside the
entropic scheme named after Eq. 8).

The KBC collision f' = f - beta (2 Delta s + gamma Delta h) fixes the
relaxation of the stress part; gamma is chosen so that f' has the largest
entropy on this line, i.e. minimises H(f') = sum_i f'_i ln(f'_i/w_i).  The
checks below do not reuse the oracle's condition: H is minimised here by
scipy's bounded scalar minimiser, and the special cases are closed forms of
the collision itself (beta = 1/2, a state with no stress part).
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from tests.cases import A, B, RGAS, base

LATTICES = [0, 1]


@pytest.fixture(scope="module")
def T10(orc):
    return orc.temperature_for_ratio(A, B, RGAS, 10.0)


def oracle(orc, lattice, T, nu=0.05, mode=1):
    return orc.Oracle(lattice, 4, 4, 1 if lattice == 0 else 4,
                      base(T, nu=nu, gamma_mode=mode))


def node(o, rng, eps, rho=None):
    """A node state f = f^eq(rho, u) (1 + eps xi), xi ~ U(-1, 1)."""
    rho = rng.uniform(0.05, 9.0) if rho is None else rho
    u = np.zeros(3)
    u[:o.D] = rng.uniform(-0.15, 0.15, o.D)
    feq = o.feq(rho, u)
    return feq * (1.0 + eps * rng.uniform(-1.0, 1.0, o.Q))


def parts(o, f):
    """(feq, ds, dh) of f, with rho and u recomputed from f."""
    rho = f.sum()
    u = np.zeros(3)
    u[:o.D] = (f @ o.c[:, :o.D]) / rho
    feq = o.feq(rho, u)
    _, ds, _ = o.collide_f(f, np.zeros(3))
    return feq, ds, f - feq - ds


def H(fp, w):
    return float(np.sum(fp * np.log(fp / w)))


def admissible(f, ds, dh, beta):
    """Interval of gamma on which every f' = f - beta (2 ds + gamma dh) > 0."""
    base_ = f - 2 * beta * ds
    lo = max((base_[i] / (beta * dh[i]) for i in range(len(f)) if dh[i] < 0), default=-1e3)
    hi = min((base_[i] / (beta * dh[i]) for i in range(len(f)) if dh[i] > 0), default=1e3)
    return lo, hi


def argmin_on(fun, lo, hi, scale):
    pad = 1e-9 * (hi - lo)
    return minimize_scalar(fun, bounds=(lo + pad, hi - pad), method="bounded",
                           options=dict(xatol=1e-12 * scale))


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_gamma_minimises_the_entropy_function(orc, T10, lattice):
    o = oracle(orc, lattice, T10)
    rng = np.random.default_rng(11)
    beta = o.beta
    for eps in (0.3, 0.05):
        for _ in range(10):
            f = node(o, rng, eps)
            feq, ds, dh = parts(o, f)
            fo, _, g = o.collide_f(f, np.zeros(3))
            assert np.allclose(fo, f - beta * (2 * ds + g * dh), rtol=1e-13, atol=1e-15 * f.max())
            lo, hi = admissible(f, ds, dh, beta)
            r = argmin_on(lambda x: H(f - beta * (2 * ds + x * dh), o.w), lo, hi, max(1.0, abs(g)))
            # H is flat at its minimum: with |H| ~ 1 its argmin is fixed to
            # about sqrt(machine epsilon / H'') -- a few 1e-6 here
            assert r.x == pytest.approx(g, rel=2e-5, abs=2e-5), (eps, r.x, g)
            assert H(f - beta * (2 * ds + g * dh), o.w) <= r.fun + 1e-14 * abs(r.fun)


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_gamma_minimises_the_relative_entropy_near_equilibrium(orc, T10, lattice):
    """Close to equilibrium H itself is too flat to locate in FP64; along the
    collision line H(f') - sum_i f'_i ln(feq_i/w_i) differs from H(f') by a
    constant (f' - f is mass- and momentum-free and ln(feq_i/w_i) is affine in
    c_i, checked in test_oracle_collision), so the relative entropy
    K = sum feq [(1 + x) ln(1 + x) - x], x = f'/feq - 1, has the same argmin
    and is of order |x|^2, resolvable to rounding."""
    o = oracle(orc, lattice, T10)
    rng = np.random.default_rng(13)
    beta = o.beta

    def K(fp, feq):
        x = (fp - feq) / feq
        # (1 + x) ln(1 + x) - x; its Taylor series x^2/2 - x^3/6 + x^4/12 - x^5/20
        # where the direct form cancels
        direct = (1.0 + x) * np.log1p(x) - x
        series = x * x * (0.5 - x * (1.0 / 6.0 - x * (1.0 / 12.0 - x / 20.0)))
        return float(np.sum(feq * np.where(np.abs(x) < 1e-2, series, direct)))

    for eps in (1e-2, 1e-3, 1e-5):
        for _ in range(5):
            f = node(o, rng, eps)
            feq, ds, dh = parts(o, f)
            _, _, g = o.collide_f(f, np.zeros(3))
            lo, hi = admissible(f, ds, dh, beta)
            lo, hi = max(lo, g - 5.0), min(hi, g + 5.0)
            r = argmin_on(lambda x: K(f - beta * (2 * ds + x * dh), feq), lo, hi, max(1.0, abs(g)))
            # the rounding of f' - feq (~1e-16 of f against eps f) limits the
            # argmin to about 1e-7 + 5e-11/eps
            assert abs(r.x - g) < 1e-7 + 5e-11 / eps, (eps, r.x, g)


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_gamma_root_condition(orc, T10, lattice):
    """sum_i dh_i ln(f'_i/feq_i) vanishes at the returned gamma, to rounding."""
    o = oracle(orc, lattice, T10)
    rng = np.random.default_rng(5)
    for eps in (0.4, 1e-2, 1e-3):
        f = node(o, rng, eps)
        feq, ds, dh = parts(o, f)
        _, _, g = o.collide_f(f, np.zeros(3))
        fp = f - o.beta * (2 * ds + g * dh)
        terms = dh * np.log1p((fp - feq) / feq)
        # recomputing f' - feq here rounds at ~1e-16 of f against eps f
        assert abs(terms.sum()) <= (1e-12 + 2e-14 / eps) * np.abs(terms).sum()


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_gamma_is_two_at_beta_half(orc, T10, lattice):
    """At beta = 1/2 the collision line is f' = f - Delta s - (gamma/2) Delta h
    = f^eq + (1 - gamma/2) Delta h: at gamma = 2 it meets f^eq and every log
    term vanishes, so gamma = 2 exactly (the closed form's value too), however
    far from equilibrium."""
    o = oracle(orc, lattice, T10, nu=1.0 / 6.0)
    assert o.beta == pytest.approx(0.5, abs=1e-15)
    rng = np.random.default_rng(7)
    for eps in (0.5, 0.1, 1e-4):
        f = node(o, rng, eps)
        _, _, g = o.collide_f(f, np.zeros(3))
        assert g == pytest.approx(2.0, abs=1e-12)


def dual_vector(o, e):
    """Population vector whose natural moments vanish except prod c_a^{e_a} = 1
    (one-dimensional dual basis of {1, c, c^2} on {-1, 0, 1})."""
    def d(k, c):
        return {0: float(c == 0), 1: 0.5 * c, 2: (-1.0 if c == 0 else 0.5)}[k]
    return np.array([np.prod([d(e[a], o.c[i, a]) for a in range(o.D)]) for i in range(o.Q)])


@pytest.mark.parametrize("lattice,e", [(0, (2, 2)), (0, (2, 1)), (1, (2, 2, 0)), (1, (2, 1, 1)), (1, (2, 2, 2))])
def test_exact_gamma_without_a_stress_part(orc, T10, lattice, e):
    """A deviation from f^eq with only higher-order moments has Delta s = 0:
    the condition reads sum dh ln(1 + (1 - beta gamma) dh/feq) = 0, whose root
    is beta gamma = 1 exactly (gamma = 1/beta, the closed form's value too)."""
    o = oracle(orc, lattice, T10)
    rho, u = 3.7, np.array([0.05, -0.03, 0.02])
    feq = o.feq(rho, u)
    f = feq + 1e-2 * feq.min() * dual_vector(o, e)
    _, ds, g = o.collide_f(f, np.zeros(3))
    assert np.abs(ds).max() < 1e-15 * rho
    assert g == pytest.approx(1.0 / o.beta, rel=1e-12)


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_gamma_agrees_with_closed_form_to_second_order(orc, T10, lattice):
    """The closed form is the root of the condition expanded to second order
    in f - f^eq: the two differ by O(|f - f^eq|)."""
    oe = oracle(orc, lattice, T10, mode=1)
    oc = oracle(orc, lattice, T10, mode=0)
    rng = np.random.default_rng(3)
    xi = rng.uniform(-1.0, 1.0, oe.Q)
    feq = oe.feq(2.5, np.array([0.04, -0.07, 0.03]))
    diffs = []
    for eps in (1e-2, 1e-3, 1e-4):
        f = feq * (1.0 + eps * xi)
        ge = oe.collide_f(f, np.zeros(3))[2]
        gc = oc.collide_f(f, np.zeros(3))[2]
        diffs.append(abs(ge - gc))
    assert diffs[0] > 0
    assert 5.0 < diffs[0] / diffs[1] < 20.0 and 5.0 < diffs[1] / diffs[2] < 20.0, diffs


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_gamma_fallback_without_admissible_gamma(orc, T10, lattice):
    """No gamma keeps f' positive when a direction with Delta h_i = 0 already
    has f^eq_i + (1 - 2 beta) Delta s_i <= 0: the solver reports -1 and keeps
    gamma0 (the collision then uses the closed form and counts a fallback)."""
    o = oracle(orc, lattice, T10)
    feq = np.full(o.Q, 0.1)
    ds = np.zeros(o.Q)
    dh = np.zeros(o.Q)
    ds[0] = -1.0 / (1.0 - 2.0 * o.beta)  # A_0 = feq_0 + (1 - 2 beta) ds_0 = 0.1 - 1 < 0
    dh[1], dh[2] = 0.01, -0.01
    it, g = o.gamma_exact(feq, ds, dh, 1.7)
    assert it == -1 and g == 1.7


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_mode_collision_invariants(orc, T10, lattice):
    """With the exact stabiliser the collision still conserves mass and
    momentum, and the exact-difference forcing adds exactly F."""
    o = oracle(orc, lattice, T10)
    rng = np.random.default_rng(9)
    c = o.c[:, :o.D]
    for _ in range(10):
        f = node(o, rng, 0.2)
        F = np.zeros(3)
        F[:o.D] = rng.uniform(-0.02, 0.02, o.D)
        fo, _, _ = o.collide_f(f, F)
        assert fo.sum() == pytest.approx(f.sum(), rel=1e-14)
        assert np.allclose(fo @ c, f @ c + F[:o.D], rtol=0, atol=1e-13 * f.sum())
    assert o.gamma_fallbacks() == 0


@pytest.mark.parametrize("lattice", LATTICES)
def test_exact_gamma_one_signed_delta_h_is_rounding(orc, T10, lattice):
    """Delta h carries no mass, so a Delta h of one sign can only be rounding
    noise: the solver returns -2 (closed form kept) and it is not counted as a
    fallback."""
    o = oracle(orc, lattice, T10)
    feq = np.full(o.Q, 0.1)
    ds = np.zeros(o.Q)
    dh = np.full(o.Q, 1e-18)
    it, g = o.gamma_exact(feq, ds, dh, 1.9)
    assert it == -2 and g == 1.9
