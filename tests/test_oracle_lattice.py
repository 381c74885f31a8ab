"""Pins of the oracle's lattice-level pieces: stencils (closed forms for plane
waves), streaming and bounce-back, the chemical potentials as functional
derivatives of the discrete free energy of Eqs. 1-3 (brute force on small
grids), the force, and the conservation laws of the whole step."""
import numpy as np
import pytest

from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, asymmetric, base


@pytest.fixture(scope="module")
def T10(orc):
    return orc.temperature_for_ratio(A, B, RGAS, 10.0)


def grid(o):
    z, y, x = np.meshgrid(np.arange(o.nz), np.arange(o.ny), np.arange(o.nx), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


@pytest.mark.parametrize("lattice", [0, 1])
def test_stencils_plane_wave(orc, T10, lattice):
    n = 12
    o = orc.Oracle(lattice, n, n, 1 if lattice == 0 else n, base(T10))
    x, y, z = grid(o)
    k, l, m = 2 * np.pi * np.array([1, 2, 3]) / n
    if lattice == 0:
        m, z = 0.0, 0 * z
    psi = np.cos(k * x + l * y + m * z)
    # lattice-weight sums factor over axes: sum_c w1(c) e^{ikc} = 2/3 + cos(k)/3
    s = lambda q: 2.0 / 3 + np.cos(q) / 3
    lap_ref = 6 * (s(k) * s(l) * (s(m) if lattice == 1 else 1.0) - 1.0) * psi
    assert np.allclose(o.laplacian(psi), lap_ref, atol=1e-13)
    # gradient: 3 sum w c_a e^{i q.c}: axis a picks i sin(q_a)/3, others s(q_b)
    sn = -np.sin(k * x + l * y + m * z)
    qs = [k, l, m]
    G = o.gradient(psi)
    for a in range(o.D):
        fac = np.sin(qs[a])
        for b in range(o.D):
            if b != a:
                fac *= s(qs[b])
        assert np.allclose(G[a], fac * sn, atol=1e-13)


@pytest.mark.parametrize("lattice", [0, 1])
def test_stream_moves_and_bounces(orc, T10, lattice):
    nx, ny, nz = 5, 4, (1 if lattice == 0 else 3)
    o = orc.Oracle(lattice, nx, ny, nz, base(T10), bc=(0, 1, 0))
    N, Q = o.N, o.Q
    idx = lambda x, y, z: x + nx * (y + ny * z)
    for i in range(Q):
        cx, cy, cz = o.c[i]
        for (x, y, z) in [(0, 0, 0), (4, 3, nz - 1), (2, 1, 0)]:
            post = np.zeros((Q, N))
            post[i, idx(x, y, z)] = 1.0
            pre = o.stream(post)
            ty = y + cy
            if 0 <= ty < ny:
                dst = idx((x + cx) % nx, ty, (z + cz) % nz)
                assert pre[i, dst] == 1.0 and pre.sum() == 1.0
            else:  # beyond the wall: comes back reversed at the same node
                j = [k for k in range(Q) if (o.c[k] == -o.c[i]).all()][0]
                assert pre[j, idx(x, y, z)] == 1.0 and pre.sum() == 1.0
    g = np.random.default_rng(1)
    pre = g.uniform(size=(Q, N))
    assert np.array_equal(o.stream(o.unstream(pre)), pre)


def discrete_free_energy(o, rho, phi, p):
    """F_h = sum_x f_B + sum_x sum_i (3/2) w_i [k1 (d_i rho)^2 + k2 (d_i C1)^2
    + k3 (d_i C2)^2], written here from Eqs. 1-4: its derivative with respect
    to psi(x) is -kappa times the isotropic Laplacian, the square-gradient term
    (kappa/2)|grad psi|^2 of Eq. 3."""
    a, b, R, T = p["a"], p["b"], p["R"], p["T"]
    chi = p["chi"]
    rg, rl = o.rho_g, o.rho_l
    br = b * rho
    psi = rho * (-o.mu_coex - a * rho - 8 * R * T * (br - 6) / (br - 4) ** 2 + R * T * np.log(rho))
    c1 = 0.5 * (1 + phi / chi - (rho - rl) / (rg - rl))
    c2 = 0.5 * (1 - phi / chi - (rho - rl) / (rg - rl))
    fb = (0.5 * p["lambda1"] * (psi + o.p_coex) + 0.5 * p["lambda2"] * c1 ** 2 * (1 - c1) ** 2
          + 0.5 * p["lambda3"] * c2 ** 2 * (1 - c2) ** 2)
    shape = (o.nz, o.ny, o.nx)
    total = fb.sum()
    for i in range(o.Q):
        sh = tuple(-int(v) for v in o.c[i][::-1])
        for field, kap in ((rho, p["kappa1"]), (c1, p["kappa2"]), (c2, p["kappa3"])):
            d = np.roll(field.reshape(shape), sh, axis=(0, 1, 2)) - field.reshape(shape)
            total += 1.5 * o.w[i] * kap * (d ** 2).sum()
    return total


@pytest.mark.parametrize("lattice", [0, 1])
def test_chemical_potentials_are_functional_derivatives(orc, T10, lattice):
    n = 8 if lattice == 0 else 4
    p = asymmetric(T10)
    o = orc.Oracle(lattice, n, n, 1 if lattice == 0 else n, p)
    g = np.random.default_rng(13)
    rho = g.uniform(0.8 * o.rho_g, 1.1 * o.rho_l, o.N)
    phi = g.uniform(-p["chi"], p["chi"], o.N)
    mr, mp = o.chem_pot(rho, phi)
    for node in range(0, o.N, max(1, o.N // 16)):
        for field, mu in ((rho, mr), (phi, mp)):
            h = 1e-5 * max(1.0, abs(field[node]))
            fp = field.copy(); fp[node] += h
            fm = field.copy(); fm[node] -= h
            if field is rho:
                d = (discrete_free_energy(o, fp, phi, p) - discrete_free_energy(o, fm, phi, p)) / (2 * h)
            else:
                d = (discrete_free_energy(o, rho, fp, p) - discrete_free_energy(o, rho, fm, p)) / (2 * h)
            assert d == pytest.approx(mu[node], rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("form", [0, 1])
def test_force_reduces_to_central_differences(orc, T10, form):
    """Fields varying along x only, with mu = 0 (lambda = kappa = 0): the force
    is the ideal term alone, and each lattice sum collapses to a central
    difference along x."""
    n = 16
    p = base(T10, lambda1=0.0, lambda2=0.0, lambda3=0.0, kappa1=0.0, kappa2=0.0,
             kappa3=0.0, force_form=form)
    o = orc.Oracle(0, n, 3, 1, p)
    x, _, _ = grid(o)
    rho1 = 2.0 + 0.8 * np.sin(2 * np.pi * np.arange(n) / n) + 0.3 * np.cos(6 * np.pi * np.arange(n) / n)
    rho = rho1[x]
    phi = np.zeros(o.N)
    mr, mp = o.chem_pot(rho, phi)
    assert np.abs(mr).max() == 0 and np.abs(mp).max() == 0
    F = o.force(rho, phi, mr, mp)
    sp = lambda v, s: np.roll(v, -s)
    G = (sp(rho1, 1) - sp(rho1, -1)) / 2
    if form == 0:
        ref = G / 3
    else:
        AG = (sp(G, -1) + sp(G, 1)) / 2
        T = G * G / (36 * rho1)
        ref = (1.5 * G - 0.5 * AG) / 3 + (sp(T, 1) - sp(T, -1)) / 2
    assert np.allclose(F[0], ref[x], atol=1e-15)
    assert np.abs(F[1:]).max() < 1e-15


@pytest.mark.parametrize("lattice", [0, 1])
def test_bulk_phases_are_stationary(orc, T10, lattice):
    n = 6
    p = asymmetric(T10)
    o = orc.Oracle(lattice, n, n, 1 if lattice == 0 else n, p)
    for r0, f0 in ((o.rho_g, 0.0), (o.rho_l, p["chi"]), (o.rho_l, -p["chi"])):
        rho = np.full(o.N, r0)
        phi = np.full(o.N, f0)
        mr, mp = o.chem_pot(rho, phi)
        assert np.abs(mr).max() < 1e-13 and np.abs(mp).max() < 1e-13
        f, g = o.init(rho, phi, np.zeros((o.D, o.N)))
        assert o.step(f, g, 5) == 0
        fl = o.fields(f, g)
        assert np.allclose(fl["rho"], r0, rtol=1e-13)
        assert np.allclose(fl["phi"], f0, atol=1e-12)
        assert np.abs(fl["u"]).max() < 1e-14
        assert np.abs(fl["p"]).max() < 1e-13  # p = 0 at coexistence


def drop_case(orc, lattice, T, n, bc=(0, 0, 0), params=None, seed=3):
    p = params or asymmetric(T)
    nz = 1 if lattice == 0 else n
    o = orc.Oracle(lattice, n, n, nz, p, bc=bc)
    shape = (n, n) if lattice == 0 else (n, n, n)
    c = [n / 2.0] * len(shape)
    rho, phi, u = inputs.drops(shape, o.rho_g, o.rho_l, p["chi"],
                               [dict(center=[v - 1.5 for v in c], R=n / 4, kind=+1, u=[0.02] * len(shape)),
                                dict(center=[v + 1.7 for v in c], R=n / 5, kind=-1)], width=3.0)
    rho, phi, u = inputs.perturb(seed, rho, phi, u)
    return o, rho, phi, u


@pytest.mark.parametrize("lattice,n,bc", [(0, 16, (0, 0, 0)), (0, 16, (1, 0, 0)), (0, 12, (1, 1, 0)),
                                          (1, 8, (0, 0, 0)), (1, 8, (0, 1, 1))])
def test_mass_conservation(orc, T10, lattice, n, bc):
    o, rho, phi, u = drop_case(orc, lattice, T10, n, bc)
    f, g = o.init(rho, phi, u)
    m0, p0 = f.sum(), g.sum()
    fl = o.fields(f, g)
    assert np.allclose(fl["rho"], rho, rtol=1e-13) and np.allclose(fl["phi"], phi, atol=1e-12)
    assert np.allclose(fl["u"], u, atol=1e-14)
    assert o.step(f, g, 20) == 0
    fl = o.fields(f, g)
    assert fl["rho"].sum() == pytest.approx(m0, rel=1e-13)
    assert abs(fl["phi"].sum() - p0) < 1e-12 * np.abs(phi).sum()


@pytest.mark.parametrize("lattice,form", [(0, 0), (0, 1), (1, 1)])
def test_momentum_conserved_without_thermodynamic_force(orc, T10, lattice, form):
    """lambda = kappa = 0: mu = 0 and the force is the ideal term alone, whose
    lattice sums telescope on a periodic box, so total momentum is conserved."""
    n = 12 if lattice == 0 else 6
    p = asymmetric(T10, lambda1=0.0, lambda2=0.0, lambda3=0.0, kappa1=0.0, kappa2=0.0,
                   kappa3=0.0, force_form=form)
    o, rho, phi, u = drop_case(orc, lattice, T10, n, params=p)
    f, g = o.init(rho, phi, u)
    c = o.c[:, :o.D].astype(float)
    j0 = (c.T @ f).sum(axis=1)
    # total physical momentum = sum (j + F/2); sum F = 0 here
    for _ in range(4):
        assert o.step(f, g, 5) == 0
        j = (c.T @ f).sum(axis=1)
        assert np.allclose(j, j0, atol=1e-13 * rho.sum())


def test_translation_and_mirror_symmetry(orc, T10):
    n = 16
    o, rho, phi, u = drop_case(orc, 0, T10, n)
    f, g = o.init(rho, phi, u)
    o.step(f, g, 10)
    ref = o.fields(f, g)
    sh = lambda v: np.roll(v.reshape(n, n), (3, -5), axis=(0, 1)).ravel()
    f2, g2 = o.init(sh(rho), sh(phi), np.stack([sh(u[0]), sh(u[1])]))
    o.step(f2, g2, 10)
    tr = o.fields(f2, g2)
    assert np.array_equal(tr["rho"], sh(ref["rho"]))
    assert np.array_equal(tr["phi"], sh(ref["phi"]))
    mx = lambda v: v.reshape(n, n)[:, ::-1].ravel()
    f3, g3 = o.init(mx(rho), mx(phi), np.stack([-mx(u[0]), mx(u[1])]))
    o.step(f3, g3, 10)
    mi = o.fields(f3, g3)
    assert np.allclose(mi["rho"], mx(ref["rho"]), rtol=1e-12)
    assert np.allclose(mi["phi"], mx(ref["phi"]), atol=1e-11)
    assert np.allclose(mi["u"][0], -mx(ref["u"][0]), atol=1e-12)
    assert np.allclose(mi["u"][1], mx(ref["u"][1]), atol=1e-12)


@pytest.mark.parametrize("form", [0, 1])
def test_wall_ghosts_mirror_the_field(orc, T10, form):
    """Reading for the stencils at a bounce-back wall: the ghost node mirrors
    the first fluid node about the half-way wall.  Chemical potentials and
    force next to the wall then equal those of the mirror-doubled periodic
    field (the normal force component is odd under the mirror)."""
    n = 10
    p = asymmetric(T10, force_form=form)
    ow = orc.Oracle(0, n, n, 1, p, bc=(1, 0, 0))
    op = orc.Oracle(0, 2 * n, n, 1, p)
    rho, phi, u = drop_case(orc, 0, T10, n)[1:]
    dbl = lambda v: np.hstack([v.reshape(n, n), v.reshape(n, n)[:, ::-1]]).ravel()
    left = lambda v: v.reshape(n, 2 * n)[:, :n].ravel()
    mw = ow.chem_pot(rho, phi)
    mp_ = op.chem_pot(dbl(rho), dbl(phi))
    for a, b in zip(mw, mp_):
        assert np.allclose(a, left(b), rtol=1e-13, atol=1e-15)
    Fw = ow.force(rho, phi, *mw)
    Fp = op.force(dbl(rho), dbl(phi), *mp_)
    for a in range(2):
        assert np.allclose(Fw[a], left(Fp[a]), rtol=1e-12, atol=1e-15)


def test_bounce_back_channel_at_rest(orc, T10):
    """Uniform bulk phase between no-slip walls stays exactly at rest."""
    p = asymmetric(T10)
    o = orc.Oracle(0, 6, 9, 1, p, bc=(0, 1, 0))
    rho = np.full(o.N, o.rho_l)
    phi = np.full(o.N, -p["chi"])
    f, g = o.init(rho, phi, np.zeros((2, o.N)))
    assert o.step(f, g, 10) == 0
    fl = o.fields(f, g)
    assert np.allclose(fl["rho"], o.rho_l, rtol=1e-14) and np.abs(fl["u"]).max() < 1e-15


@pytest.mark.parametrize("lattice,n", [(0, 12), (1, 9)])
def test_update_depends_on_radius_three_only(orc, T10, lattice, n):
    """The premise of the full-size sampled parity test: one step of a node
    reads the state within 3 lattice units, so a periodic 7-wide window around
    the node reproduces the node's update exactly."""
    from tests.test_gpu_fullsize import window
    o, rho, phi, u = drop_case(orc, lattice, T10, n)
    f, g = o.init(rho, phi, u)
    o.step(f, g, 2)
    shape = (n,) * o.D
    f0, g0 = f.copy(), g.copy()
    o.step(f, g, 1)
    w = orc.Oracle(lattice, 7, 7, 1 if lattice == 0 else 7, o.params)
    rng = np.random.default_rng(2)
    for _ in range(5):
        c = [int(rng.integers(0, n)) for _ in range(o.D)]
        fw, gw = window(f0, shape, c), window(g0, shape, c)
        w.step(fw, gw, 1)
        mid = (7 ** o.D) // 2
        node = c[0] + n * (c[1] + (n * c[2] if o.D == 3 else 0))
        assert np.array_equal(fw[:, mid], f[:, node]) and np.array_equal(gw[:, mid], g[:, node])
