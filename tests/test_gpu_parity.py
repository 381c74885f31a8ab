"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances: FP64 storage -- max error <= 1e-12 (relative to each field's
scale) after one step and <= 1e-10 after 100 steps, the bar of the FP64 path;
FP32-shifted storage -- <= 1e-4 relative on density and phase field and
<= 1e-6 relative drift of total mass.
Scales: rho and populations relative per element; phi relative to chi; u
relative to max(|u|_max, 1e-3).
"""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, asymmetric, base

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T10():
    return tel.temperature_for_ratio(A, B, RGAS, 10.0)


def setup_pair(orc, lattice, shape, params, bc=(0, 0, 0), seed=3, n_drops=2, amp=1e-3, precision=tel.FP64):
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) == 3 else 1
    g = tel.Lattice(lattice, nx, ny, nz, dict(params, precision=precision), bc=bc)
    o = orc.Oracle(lattice, nx, ny, nz, params, bc=bc)
    D = len(shape)
    c = [s / 2.0 for s in shape]
    R = min(shape) / 4.0
    drops = [dict(center=[v - 0.37 * R for v in c], R=R, kind=+1, u=[0.01] * D),
             dict(center=[v + 0.41 * R for v in c], R=0.8 * R, kind=-1, u=[-0.01] * D)][:n_drops]
    rho, phi, u = inputs.drops(tuple(shape), o.rho_g, o.rho_l, params["chi"], drops, width=4.0)
    rho, phi, u = inputs.perturb(seed, rho, phi, u, amp, amp, amp)
    return g, o, rho, phi, u


def field_err(a, b, chi):
    ur = max(np.abs(b["u"]).max(), 1e-3)
    return {"rho": np.max(np.abs(a["rho"] - b["rho"]) / np.abs(b["rho"])),
            "phi": np.max(np.abs(a["phi"] - b["phi"])) / chi,
            "u": np.max(np.abs(a["u"] - b["u"])) / ur,
            "p": np.max(np.abs(a["p"] - b["p"])) / max(np.abs(b["p"]).max(), 1e-6)}


def state_err(fg, fo):
    return max(np.max(np.abs(fg[0] - fo[0]) / np.maximum(np.abs(fo[0]), 1e-300)),
               np.max(np.abs(fg[1] - fo[1])) / max(np.abs(fo[1]).max(), 1e-300))


CASES_1STEP = [
    (0, (8, 8), (0, 0, 0), 1),
    (0, (8, 8), (1, 0, 0), 0),
    (0, (9, 11), (1, 1, 0), 1),
    (0, (70, 37), (0, 1, 0), 1),   # ragged: partial tile in x, partial chunk in y
    (1, (4, 4, 4), (0, 0, 0), 1),
    (1, (5, 6, 7), (1, 0, 1), 0),
    (1, (37, 11, 70), (0, 0, 0), 1),  # partial tiles in x,y; two chunks in z
]


@pytest.mark.parametrize("lattice,shape,bc,form", CASES_1STEP)
def test_one_step_state_parity_fp64(orc, T10, lattice, shape, bc, form):
    p = asymmetric(T10, force_form=form)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    assert state_err(g.get_state(), (fo, go)) < 1e-13
    g.step(1)
    assert o.step(fo, go, 1) == 0
    assert state_err(g.get_state(), (fo, go)) < 1e-12
    e = field_err(g.fields(), o.fields(fo, go), p["chi"])
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("lattice,shape,bc,steps", [
    (0, (64, 64), (0, 0, 0), 100),
    (0, (48, 40), (1, 1, 0), 100),
    (1, (16, 16, 16), (0, 0, 0), 40),
    (1, (12, 10, 70), (1, 0, 0), 10),
])
def test_multi_step_field_parity_fp64(orc, T10, lattice, shape, bc, steps):
    p = base(T10)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, bc)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(steps)
    assert o.step(fo, go, steps) == 0
    e = field_err(g.fields(), o.fields(fo, go), p["chi"])
    assert max(e.values()) < 1e-10, e


def test_touching_drops_100_steps_fp64(orc, T10):
    """64 x 64 periodic, ratio 10, liquid-1 and liquid-2 drops (R = 12) touching,
    centres 20 apart, at rest; 100 steps."""
    p = base(T10)
    g = tel.Lattice(0, 64, 64, 1, p)
    o = orc.Oracle(0, 64, 64, 1, p)
    rho, phi, u = inputs.touching_drops_2d(64, 64, o.rho_g, o.rho_l, p["chi"])
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    g.step(100)
    o.step(fo, go, 100)
    e = field_err(g.fields(), o.fields(fo, go), p["chi"])
    assert max(e.values()) < 1e-10, e


@pytest.mark.parametrize("lattice,shape", [(0, (64, 64)), (1, (16, 16, 16))])
def test_fp32_shifted_against_fp64_oracle(orc, T10, lattice, shape):
    p = base(T10)
    g, o, rho, phi, u = setup_pair(orc, lattice, shape, p, precision=tel.FP32_SHIFTED)
    g.init(rho, phi, u)
    fo, go = o.init(rho, phi, u)
    steps = 100 if lattice == 0 else 40
    g.step(steps)
    o.step(fo, go, steps)
    a, b = g.fields(), o.fields(fo, go)
    assert np.max(np.abs(a["rho"] - b["rho"]) / b["rho"]) < 1e-4
    assert np.max(np.abs(a["phi"] - b["phi"])) / p["chi"] < 1e-4
    assert abs(a["rho"].sum() / rho.sum() - 1) < 1e-6
    assert abs(a["phi"].sum() - phi.sum()) / np.abs(phi).sum() < 1e-6


@pytest.mark.parametrize("shape", [(36, 10, 21), (16, 16, 16), (37, 11, 19)])
def test_one_step_fp32_state_parity_d3q27(orc, T10, shape):
    """One FP32-shifted step against the oracle started from the same state.
    nx % 4 == 0 reads phase A as aligned four-node vectors (here with partial
    tiles in x and y and periodic seams inside a tile); nx % 4 != 0 takes the
    scalar path.  Bar: one FP32 step against FP64, 2e-5 (f relative to the
    node's largest f, g relative to chi)."""
    p = asymmetric(T10, force_form=1)
    g, o, rho, phi, u = setup_pair(orc, 1, shape, p, precision=tel.FP32_SHIFTED)
    g.init(rho, phi, u)
    g.step(2)
    f0, g0 = g.get_state()
    g.step(1)
    f1, g1 = g.get_state()
    o1 = orc.Oracle(1, shape[0], shape[1], shape[2], dict(p, rho_ref=0.0))
    assert o1.step(f0, g0, 1) == 0
    ef = np.max(np.abs(f0 - f1) / np.max(np.abs(f0), axis=0))
    eg = np.max(np.abs(g0 - g1)) / p["chi"]
    assert max(ef, eg) < 2e-5, (ef, eg)


@pytest.mark.parametrize("shape", [(36, 21), (132, 17), (64, 40), (37, 19), (38, 9)])
def test_one_step_fp32_state_parity_d2q9(orc, T10, shape):
    """As the D3Q27 case: nx % 4 == 0 reads phase A as aligned four-node
    vectors along rows of 64 (36: one partial tile with the periodic seam
    inside it; 132: two whole tiles and a partial one), nx % 4 != 0 takes the
    scalar path.  Same bar."""
    p = asymmetric(T10, force_form=1)
    g, o, rho, phi, u = setup_pair(orc, 0, shape, p, precision=tel.FP32_SHIFTED)
    g.init(rho, phi, u)
    g.step(2)
    f0, g0 = g.get_state()
    g.step(1)
    f1, g1 = g.get_state()
    o1 = orc.Oracle(0, shape[0], shape[1], 1, dict(p, rho_ref=0.0))
    assert o1.step(f0, g0, 1) == 0
    ef = np.max(np.abs(f0 - f1) / np.max(np.abs(f0), axis=0))
    eg = np.max(np.abs(g0 - g1)) / p["chi"]
    assert max(ef, eg) < 2e-5, (ef, eg)


def test_step_batches_and_checkpoint_are_bitwise(orc, T10):
    p = base(T10)
    g, o, rho, phi, u = setup_pair(orc, 0, (40, 24), p)
    g.init(rho, phi, u)
    g.step(7)
    f7, g7 = g.get_state()
    g.step(5)
    ref = g.get_state()
    h = tel.Lattice(0, 40, 24, 1, p)
    h.set_state(f7, g7)
    for _ in range(5):
        h.step(1)
    got = h.get_state()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_error_paths(T10):
    p = base(T10)
    g = tel.Lattice(0, 8, 8, 1, p)
    with pytest.raises(tel.TelError) as ei:
        g.step(1)
    assert ei.value.code == tel.TEL_ESTATE
    rho = np.full(64, g.rho_l)
    phi = np.zeros(64)
    g.init(rho, phi, np.zeros(128))
    g.step(0)
    g.sync()
    # a velocity outside the entropic equilibrium's domain is flagged, not trapped
    bad = tel.Lattice(0, 8, 8, 1, p)
    u = np.zeros(128)
    u[5] = 1.5
    with pytest.raises(tel.TelError) as ei:
        bad.init(rho, phi, u)
    assert ei.value.code == tel.TEL_EUNSTABLE
    with pytest.raises(ValueError):  # the binding checks lengths before the call
        g.init(rho[:10], phi, np.zeros(128))


def test_torch_device_buffers_and_stream(orc, T10):
    torch = pytest.importorskip("torch")
    p = base(T10)
    g, o, rho, phi, u = setup_pair(orc, 1, (8, 8, 8), p)
    s = torch.cuda.Stream()
    g.set_stream(s)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        g.init_device(dev(rho), dev(phi), dev(u.ravel()))
        g.step(3)
        out = torch.empty(g.N, dtype=torch.float64, device="cuda")
        g.fields_device(rho=out)
    s.synchronize()
    fo, go = o.init(rho, phi, u)
    o.step(fo, go, 3)
    ref = o.fields(fo, go)["rho"]
    assert np.max(np.abs(out.cpu().numpy() - ref) / ref) < 1e-12
    g.set_stream(None)
