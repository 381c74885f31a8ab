"""Physics checks of the CUDA path against what the paper fixes:
coexistence of a flat liquid-gas interface at the common-tangent densities
(text after Eq. 4, Fig. 3) and Laplace's law for drops (2D: dp = sigma/R),
with sigma measured independently on a flat interface as the integral of the
anisotropy of the pressure tensor, sigma = int kappa1 (d rho/dx)^2 dx for the
liquid-gas model (lambda2 = lambda3 = kappa2 = kappa3 = 0)."""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, base

pytestmark = pytest.mark.gpu

KAPPA1 = 0.05


def params(ratio):
    T = tel.temperature_for_ratio(A, B, RGAS, ratio)
    return base(T, lambda2=0.0, lambda3=0.0, kappa1=KAPPA1, kappa2=0.0, kappa3=0.0, force_form=1)


def flat(ratio, steps=8000, nx=256):
    p = params(ratio)
    lat = tel.Lattice(tel.D2Q9, nx, 4, 1, p)
    x = np.arange(nx)
    q = nx // 4
    s = 0.5 * (np.tanh((x - q) / 6.0) - np.tanh((x - 3 * q) / 6.0))
    rho = np.tile(lat.rho_g + (lat.rho_l - lat.rho_g) * s, 4)
    lat.init(rho, np.zeros_like(rho), np.zeros((2, rho.size)))
    lat.step(steps)
    return lat, lat.fields()


@pytest.mark.parametrize("ratio", [3.0, 10.0])
def test_flat_interface_coexistence_gpu(ratio):
    lat, fl = flat(ratio)
    r = fl["rho"][:256]
    assert abs(r[0] / lat.rho_g - 1) < 0.02
    assert abs(r[128] / lat.rho_l - 1) < 0.005
    assert np.abs(fl["u"]).max() < 1e-3


def test_laplace_law_gpu():
    """Drops of R = 24, 32, 40 in a 160^2 box: the interface (kappa1 = 0.05)
    is ~10 nodes wide, so smaller drops have no bulk liquid at their centre.
    Laplace's law dp = sigma/R holds up to the curvature correction of a
    diffuse interface, which shrinks as R grows."""
    ratio = 10.0
    lat, fl = flat(ratio)
    r = fl["rho"][:256]
    G = (np.roll(r, -1) - np.roll(r, 1)) / 2.0
    sigma = 0.5 * np.sum(KAPPA1 * G * G)  # two interfaces in the box
    p = params(ratio)
    n = 160
    inv_r, dp = [], []
    for R in (24.0, 32.0, 40.0):
        d = tel.Lattice(tel.D2Q9, n, n, 1, p)
        rho, phi, u = inputs.drops((n, n), d.rho_g, d.rho_l, p["chi"], [dict(center=(n / 2, n / 2), R=R, kind=1)],
                                   width=8.0)
        d.init(rho, np.zeros_like(phi), u)
        d.step(10000)
        f = d.fields()
        rr = f["rho"].reshape(n, n)
        P = f["p"].reshape(n, n)
        Re = np.sqrt((rr - d.rho_g).sum() / (d.rho_l - d.rho_g) / np.pi)  # equimolar radius
        assert rr[n // 2, n // 2] > 0.95 * d.rho_l  # bulk liquid at the centre
        inv_r.append(1.0 / Re)
        dp.append(P[n // 2, n // 2] - P[0, 0])
    # dp R / sigma carries the curvature correction of a diffuse interface
    # (width ~10 nodes): it must fall monotonically towards 1 as R grows
    # (measured: 1.10, 1.05, 1.03 for R = 24, 32, 40)
    q = np.array(dp) / np.array(inv_r) / sigma
    assert dp[0] > dp[1] > dp[2] > 0
    assert q[0] > q[1] > q[2], q
    assert np.all((q > 0.95) & (q < 1.15)), q
    assert abs(q[-1] - 1.0) < 0.05, q


# ---------------------------------------------------------------------------
# Neumann triangle: a liquid-1 lens on a flat liquid-2/gas interface
# ---------------------------------------------------------------------------
def lens_params(T):
    """Three-phase parameters for which the lens relaxes to rest: density
    ratio 5, kappa1 = 0.02, kappa2 = kappa3 = 0.5, lambda2 = lambda3 =
    0.3 kappa, nu = 0.3 (the paper's kappa/lambda ratio runs away here)."""
    return base(T, kappa1=0.02, kappa2=0.5, kappa3=0.5, lambda2=0.15, lambda3=0.15, nu=0.3, Gamma=1.0,
                force_form=1)


def flat_tensions(p, steps):
    """sigma_1g, sigma_2g, sigma_12 of relaxed flat binary slabs: the
    integral of 2 f_I across an interface (two interfaces per periodic box)."""
    rg, rl = tel.coexistence(A, B, RGAS, p["T"])[:2]
    chi, Dl = p["chi"], rg - rl
    Ai = 0.5 * p["kappa1"] + (p["kappa2"] + p["kappa3"]) / (8 * Dl * Dl)
    Bi = (p["kappa2"] + p["kappa3"]) / (8 * chi * chi)
    Xi = (p["kappa3"] - p["kappa2"]) / (4 * chi * Dl)
    x = np.arange(256)
    s = 0.5 * (np.tanh((x - 64) / 3.0) - np.tanh((x - 192) / 3.0))
    out = {}
    for kind in ("1g", "2g", "12"):
        if kind == "1g":
            rho, phi = rg + (rl - rg) * s, chi * s
        elif kind == "2g":
            rho, phi = rg + (rl - rg) * s, -chi * s
        else:
            rho, phi = np.full(256, rl), chi * (2 * s - 1)
        lat = tel.Lattice(tel.D2Q9, 256, 4, 1, p)
        lat.init(np.tile(rho, 4), np.tile(phi, 4), np.zeros(2048))
        lat.step(steps)
        f = lat.fields()
        r, ph = f["rho"][:256], f["phi"][:256]
        gr = (np.roll(r, -1) - np.roll(r, 1)) / 2
        gp = (np.roll(ph, -1) - np.roll(ph, 1)) / 2
        out[kind] = 0.5 * np.sum(2 * (Ai * gr ** 2 + Bi * gp ** 2 + Xi * gr * gp))
    return out


def fit_circle(x, y):
    M = np.c_[2 * x, 2 * y, np.ones_like(x)]
    (xc, yc, c), *_ = np.linalg.lstsq(M, x * x + y * y, rcond=None)
    return xc, yc, np.sqrt(c + xc * xc + yc * yc)


def lens_angles(fields, p, nx, ny):
    """Angles of the lens's upper and lower caps with the flat liquid-2/gas
    interface at the triple point, from circles fitted to the C1 = 1/2
    contour (the middle 60% of the lens) and the far-field level of C2 = 1/2."""
    rg, rl = tel.coexistence(A, B, RGAS, p["T"])[:2]
    R = fields["rho"].reshape(ny, nx)
    PH = fields["phi"].reshape(ny, nx)
    Dl = rg - rl
    C1 = 0.5 * (1 + PH / p["chi"] - (R - rl) / Dl)
    C2 = 0.5 * (1 - PH / p["chi"] - (R - rl) / Dl)
    cols = []
    for xi in range(nx):
        col = C1[:, xi]
        inside = np.where(col > 0.5)[0]
        if len(inside) < 3:
            continue
        j0, j1 = inside.min(), inside.max()
        yb = j0 - 1 + (0.5 - col[j0 - 1]) / (col[j0] - col[j0 - 1])
        yt = j1 + (col[j1] - 0.5) / (col[j1] - col[j1 + 1])
        cols.append((xi, yb, yt))
    cols = np.array(cols)
    xs = cols[:, 0]
    xl, xr = xs.min(), xs.max()
    sel = (xs > xl + 0.2 * (xr - xl)) & (xs < xr - 0.2 * (xr - xl))
    top, bot = fit_circle(cols[sel, 0], cols[sel, 2]), fit_circle(cols[sel, 0], cols[sel, 1])
    cg = C2[:, :8].mean(axis=1)
    j1 = np.where(cg > 0.5)[0].max()
    yf = j1 + (cg[j1] - 0.5) / (cg[j1] - cg[j1 + 1])

    def angle(circ, upper):
        xc, yc, r = circ
        dx = np.sqrt(max(r * r - (yf - yc) ** 2, 0.0))
        t = np.array([-(yf - yc), dx]) / r
        if (upper and t[1] < 0) or ((not upper) and t[1] > 0):
            t = -t
        return np.degrees(np.arctan2(abs(t[1]), -t[0]))

    return angle(top, True), angle(bot, False)


def neumann_angles(s1g, s2g, s12):
    """Force balance at the triple point, sigma_2g e_x + sigma_1g (-cos a,
    sin a) + sigma_12 (-cos b, -sin b) = 0, solved for the caps' angles."""
    S = np.arccos((s2g ** 2 - s1g ** 2 - s12 ** 2) / (2 * s1g * s12))
    a = np.arctan2(s12 * np.sin(S), s1g + s12 * np.cos(S))
    return np.degrees(a), np.degrees(S - a)


def test_neumann_angles_of_a_liquid_lens_gpu():
    """A liquid-1 drop placed on the flat interface between liquid 2 and the
    gas relaxes into a lens whose two caps meet the flat interface at the
    angles the three measured interfacial tensions fix (Neumann triangle):
    within 3 degrees (the paper's agreement), with the flow at rest."""
    T = tel.temperature_for_ratio(A, B, RGAS, 5.0)
    p = lens_params(T)
    sig = flat_tensions(p, 10000)
    nx, ny = 256, 192
    lat = tel.Lattice(tel.D2Q9, nx, ny, 1, p)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    slab = 0.5 * (np.tanh((Y - 0.25 * ny) / 1.5) - np.tanh((Y - 0.75 * ny) / 1.5))
    drop = 0.5 * (1 + np.tanh((36.0 - np.hypot(X - nx / 2, Y - 0.75 * ny)) / 1.5))
    c2 = slab * (1 - drop)
    rho = lat.rho_g + (lat.rho_l - lat.rho_g) * np.clip(drop + c2, 0, 1)
    phi = p["chi"] * (drop - c2)
    lat.init(rho.ravel(), phi.ravel(), np.zeros(2 * nx * ny))
    lat.step(20000)
    f = lat.fields()
    assert np.abs(f["u"]).max() < 5e-3
    geo = lens_angles(f, p, nx, ny)
    ref = neumann_angles(sig["1g"], sig["2g"], sig["12"])
    assert abs(geo[0] - ref[0]) < 3.0 and abs(geo[1] - ref[1]) < 3.0, (geo, ref, sig)


def test_lens_state_parity_with_the_oracle_gpu(orc):
    """The lens configuration of the Neumann test, 200 steps in FP64, on the
    GPU and in the oracle: fields within 1e-10 (the full 20000-step
    relaxation takes the oracle about 20 minutes, so the angles themselves
    are measured on the GPU)."""
    T = tel.temperature_for_ratio(A, B, RGAS, 5.0)
    p = lens_params(T)
    nx, ny = 256, 192
    g = tel.Lattice(tel.D2Q9, nx, ny, 1, p)
    o = orc.Oracle(0, nx, ny, 1, p)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    slab = 0.5 * (np.tanh((Y - 0.25 * ny) / 1.5) - np.tanh((Y - 0.75 * ny) / 1.5))
    drop = 0.5 * (1 + np.tanh((36.0 - np.hypot(X - nx / 2, Y - 0.75 * ny)) / 1.5))
    c2 = slab * (1 - drop)
    rho = (o.rho_g + (o.rho_l - o.rho_g) * np.clip(drop + c2, 0, 1)).ravel()
    phi = (p["chi"] * (drop - c2)).ravel()
    u = np.zeros(2 * nx * ny)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(200)
    assert o.step(fo, go, 200) == 0
    a, b = g.fields(), o.fields(fo, go)
    assert np.max(np.abs(a["rho"] - b["rho"]) / b["rho"]) < 1e-10
    assert np.max(np.abs(a["phi"] - b["phi"])) / p["chi"] < 1e-10
    assert np.max(np.abs(a["u"] - b["u"])) < 1e-10 * max(np.abs(b["u"]).max(), 1e-3)


def test_oblique_flat_interface_d3q27_gpu():
    """A flat liquid-gas interface normal to (1, 1, 1) relaxes to the same
    coexistence densities as one normal to x (lattice-consistent force, all
    three gradient components coupled).  118^3 box: x + y + z has period 118,
    68.1 nodes along the normal, matched by a 68-node axis-aligned box."""
    p = params(10.0)
    N = 118
    L = N / np.sqrt(3.0)
    lat = tel.Lattice(tel.D3Q27, N, N, N, p)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    dn = ((x + y + z) % N).ravel() / np.sqrt(3.0)
    prof = 0.5 * (np.tanh((dn - L / 4) / 3.0) - np.tanh((dn - 3 * L / 4) / 3.0))
    lat.init(lat.rho_g + (lat.rho_l - lat.rho_g) * prof, np.zeros(N ** 3), np.zeros((3, N ** 3)))
    lat.step(3000)
    r = lat.fields(with_p=False)["rho"]
    gas_d, liq_d = r[np.argmin(dn)], r[np.argmin(np.abs(dn - L / 2))]
    a = tel.Lattice(tel.D3Q27, 68, 4, 4, p)
    xa = np.arange(68) * (L / 68)
    pa = np.tile(0.5 * (np.tanh((xa - L / 4) / 3.0) - np.tanh((xa - 3 * L / 4) / 3.0)), 16)
    a.init(a.rho_g + (a.rho_l - a.rho_g) * pa, np.zeros(68 * 16), np.zeros((3, 68 * 16)))
    a.step(3000)
    ra = a.fields(with_p=False)["rho"]
    for gas, liq in ((gas_d, liq_d), (ra[0], ra[34])):
        assert abs(gas / lat.rho_g - 1) < 0.02
        assert abs(liq / lat.rho_l - 1) < 0.005
    assert abs(gas_d / ra[0] - 1) < 5e-3 and abs(liq_d / ra[34] - 1) < 5e-4


@pytest.mark.parametrize("ratio,lam1,kap1,steps", [
    (30.0, 0.01, 0.04, 200000),
    (100.0, 0.004, 0.04, 400000),
    (300.0, 0.001, 0.03, 400000),
])
def test_high_ratio_flat_interface_gpu(ratio, lam1, kap1, steps):
    """Flat liquid-gas interfaces at density ratios 30, 100 and 300 relax to the
    Maxwell densities (gas within 2%, liquid within 0.5%) when the gas side
    of the interface is resolved: lambda1 far below the paper's 0.6 (the
    gas-side decay length sqrt(kappa1 rho_g / (lambda1/2 RT)) is 6-7 nodes
    here), kappa1 below the capillary stiffness limit kappa1 rho_l < 0.4.
    With lambda1 = 0.6 the same interfaces fail within 1000 steps or settle
    81% off in the gas (design notes, section 2b).  1024 x 4 periodic, two
    interfaces, initial tanh width 30, FP64, lattice-consistent force."""
    T = tel.temperature_for_ratio(A, B, RGAS, ratio)
    p = base(T, lambda1=lam1, lambda2=0.0, lambda3=0.0, kappa1=kap1, kappa2=0.0, kappa3=0.0, force_form=1)
    nx = 1024
    lat = tel.Lattice(tel.D2Q9, nx, 4, 1, p)
    x = np.arange(nx)
    s = 0.5 * (np.tanh((x - nx // 4) / 15.0) - np.tanh((x - 3 * nx // 4) / 15.0))
    rho = np.tile(lat.rho_g + (lat.rho_l - lat.rho_g) * s, 4)
    lat.init(rho, np.zeros_like(rho), np.zeros((2, rho.size)))
    lat.step(steps)
    f = lat.fields(with_p=False)
    r = f["rho"][:nx]
    assert abs(r[0] / lat.rho_g - 1) < 0.02, r[0] / lat.rho_g - 1
    assert abs(r[nx // 2] / lat.rho_l - 1) < 0.005, r[nx // 2] / lat.rho_l - 1
    assert np.abs(f["u"]).max() < 1e-3
