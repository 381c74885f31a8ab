"""The touching-drops configuration as configured (D2Q9 64 x 64 periodic,
FP64, 2000 steps): gas background, a liquid-1 and a liquid-2 drop of R = 12
with centres 20 apart along x, density ratio 10, zero initial velocity, equal
surface tensions.

Equal tensions: kappa2 = kappa3 = 0.5, lambda2 = lambda3 = 0.25 (the paper's
lambda = 3.125 kappa runs away in this discretisation) fix
sigma_12 = sqrt((k2 + k3)(l2 + l3))/6 in the continuum (0.114 measured on
the lattice); kappa1 = 0.0216 was set on the CPU oracle so that a relaxed
flat liquid-gas slab has the same tension.  With three equal tensions the
Neumann triangle is equilateral: every angle at a triple point is 120
degrees, the 1|2 interface is flat and each outer arc's centre lies half its
radius from it.

Checked: field parity with the oracle after all 2000 steps (<= 1e-10), the
three tensions measured on relaxed flat slabs on the GPU (equal to 5%), the
angles of both drops at the triple points from circles fitted to their outer
arcs (120 degrees within 10: after 2000 steps the drops are still merging
towards the double-bubble shape; 128 degrees on the oracle), and Laplace's
law for each drop (dp = sigma/R_arc within 15%).

Beyond the configured 2000 steps this parameter set runs away: the angles
reach 125 degrees near step 3000, then the velocity grows from 0.01 (step
3000) to 0.13 (step 4000) and the drops deform (oracle).  The same happens
with lambda = 0.3 kappa (kappa1 = 0.0183 for equal tensions) from step 3500."""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, base
from tests.test_gpu_parity import field_err
from tests.test_gpu_physics import fit_circle, flat_tensions

pytestmark = pytest.mark.gpu


def c1_params(T):
    return base(T, kappa1=0.0216, kappa2=0.5, kappa3=0.5, lambda2=0.25, lambda3=0.25, force_form=1)


def outer_arc(R, PH, lvl, x12, side):
    """Points of the rho = lvl contour of one drop away from the 1|2 line
    (side -1: the drop left of it, +1: right), by linear interpolation along
    rows and columns."""
    ny, nx = R.shape
    pts = []
    for j in range(ny):
        row = R[j]
        for i in range(nx - 1):
            a, b = row[i] - lvl, row[i + 1] - lvl
            if a * b < 0:
                x = i + a / (a - b)
                if side * (x - x12) > 3.0:
                    pts.append((x, j))
    for i in range(nx):
        col = R[:, i]
        for j in range(ny - 1):
            a, b = col[j] - lvl, col[j + 1] - lvl
            if a * b < 0 and side * (i - x12) > 3.0:
                pts.append((i, j + a / (a - b)))
    return np.array(pts, float)


def test_touching_drops_as_configured(orc):
    T = tel.temperature_for_ratio(A, B, RGAS, 10.0)
    p = c1_params(T)
    n = 64
    g = tel.Lattice(tel.D2Q9, n, n, 1, p)
    o = orc.Oracle(0, n, n, 1, p)
    rho, phi, u = inputs.touching_drops_2d(n, n, g.rho_g, g.rho_l, p["chi"])
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(2000)
    assert o.step(fo, go, 2000) == 0
    a, b = g.fields(), o.fields(fo, go)
    e = field_err(a, {k: v for k, v in b.items() if k != "rc"}, p["chi"])
    assert max(e.values()) < 1e-10, e

    s = flat_tensions(p, 8000)
    sig = np.mean(list(s.values()))
    assert max(abs(v / sig - 1) for v in s.values()) < 0.05, s

    R = a["rho"].reshape(n, n)
    PH = a["phi"].reshape(n, n)
    P = a["p"].reshape(n, n)
    lvl = 0.5 * (g.rho_g + g.rho_l)
    # the 1|2 line: phi = 0 crossings inside the liquid
    xs = []
    for j in range(n):
        for i in range(n - 1):
            if R[j, i] > lvl and R[j, i + 1] > lvl and PH[j, i] > 0 >= PH[j, i + 1]:
                xs.append(i + PH[j, i] / (PH[j, i] - PH[j, i + 1]))
    x12 = float(np.mean(xs))
    angles, dps = [], []
    for side, sgn in ((-1, 1.0), (1, -1.0)):
        pts = outer_arc(R, PH, lvl, x12, side)
        xc, yc, rc = fit_circle(pts[:, 0], pts[:, 1])
        d = -side * (x12 - xc)  # > 0: the centre lies inside the drop's part
        angles.append(np.degrees(np.arccos(-d / rc)))
        inside = P[int(round(yc)), int(round(xc))]
        dps.append((inside - P[0, 0]) * rc / s["1g" if side < 0 else "2g"])
    # still relaxing at step 2000 (the oracle: 141, 132, 130, 128 degrees
    # after 500, 1000, 1500, 2000 steps)
    assert all(abs(t - 120.0) < 10.0 for t in angles), angles
    assert all(abs(q - 1.0) < 0.15 for q in dps), dps
    print(f"C1 64^2 2000 steps: angles {angles[0]:.1f} / {angles[1]:.1f} deg, dp R/sigma {dps[0]:.3f} / "
          f"{dps[1]:.3f}, tensions {s}")
