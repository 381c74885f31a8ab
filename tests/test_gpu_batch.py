"""Batched D2Q9 lattices: many independent cases of uneven size and their own
parameters advanced by one persistent launch per step.  Each case must evolve
as a single lattice with the same parameters does, whatever tile width and
chunk length the work list uses: the per-node source is the same, but the two
kernels are separate compilations, so the compiler may contract a*b+c into
fused multiply-adds differently; the bar is therefore rounding level (FP64:
1e-12 relative after 21 steps; FP32-shifted: 1e-5 on density and phase
field, ten times under the FP32-against-oracle bar, 1e-4 on velocity and
pressure), and the FP64 cases must keep the oracle's results
(1e-10 after 20 steps)."""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, asymmetric, base

pytestmark = pytest.mark.gpu

SHAPES = [(48, 40), (100, 36), (64, 64), (33, 17), (130, 70), (16, 16)]
# every row a whole number of four-node vectors: the FP32 batch reads phase A
# as aligned vectors (one odd row, as in SHAPES, takes the scalar path)
SHAPES_VEC = [(48, 40), (100, 36), (64, 64), (36, 17), (132, 70), (16, 16)]


def case_params(k, precision, walls=False):
    ratio = (3.0, 10.0, 5.0, 10.0, 8.0, 4.0)[k % 6]
    T = tel.temperature_for_ratio(A, B, RGAS, ratio)
    p = (asymmetric if k % 2 else base)(T, precision=precision)
    if walls and k % 3 == 1:
        p["bc"] = (1, 0, 0)
    return p


def case_fields(k, shape, p):
    nx, ny = shape
    rg, rl, _, _ = tel.coexistence(p["a"], p["b"], p["R"], p["T"])
    R = min(nx, ny) / 4.0
    drops = [dict(center=(nx / 2 - 0.3 * R, ny / 2), R=R, kind=1, u=(0.01, -0.005)),
             dict(center=(nx / 2 + 0.5 * R, ny / 2 + 0.2 * R), R=0.7 * R, kind=-1, u=(-0.01, 0.0))]
    rho, phi, u = inputs.drops(shape, rg, rl, p["chi"], drops, width=4.0)
    return inputs.perturb(100 + k, rho, phi, u, 1e-3, 1e-3, 1e-3)


def run_pair(precision, steps, walls=False, tune=False, shapes=SHAPES):
    ps = [case_params(k, precision, walls) for k in range(len(shapes))]
    b = tel.Batch(shapes, ps)
    singles = []
    for k, (shape, p) in enumerate(zip(shapes, ps)):
        rho, phi, u = case_fields(k, shape, p)
        b.init(k, rho, phi, u)
        s = tel.Lattice(tel.D2Q9, shape[0], shape[1], 1, p)
        s.init(rho, phi, u)
        singles.append(s)
    done = 0
    if tune:
        done = b.tune(2)[2]
    for n in steps:
        b.step(n)
    done += sum(steps)
    for s in singles:
        s.step(done)
    return b, singles


def errs(a, b):
    return {"rho": np.max(np.abs(a["rho"] - b["rho"]) / np.abs(b["rho"])),
            "phi": np.max(np.abs(a["phi"] - b["phi"])) / 5.0,
            "u": np.max(np.abs(a["u"] - b["u"])) / max(np.abs(b["u"]).max(), 1e-3),
            "p": np.max(np.abs(a["p"] - b["p"])) / max(np.abs(b["p"]).max(), 1e-6)}


def max_rel(a, b):
    return max(errs(a, b).values())


def close_fp32(a, b, p_tol=1e-4):
    """FP32-shifted: density and phase field 1e-5 (ten times under the bar
    against the oracle), velocity and pressure (differences of nearly equal
    terms) 1e-4."""
    e = errs(a, b)
    return e["rho"] <= 1e-5 and e["phi"] <= 1e-5 and e["u"] <= 1e-4 and e["p"] <= p_tol


@pytest.mark.parametrize("precision", [tel.FP64, tel.FP32_SHIFTED])
def test_batch_matches_single_lattices(precision):
    # odd and even step counts: single launches, graph replays of step pairs
    b, singles = run_pair(precision, [3, 6, 1, 11])
    for k, s in enumerate(singles):
        got, ref = b.fields(k), s.fields()
        if precision == tel.FP64:
            assert max_rel(got, ref) <= 1e-12, (k, errs(got, ref))
        else:
            assert close_fp32(got, ref), (k, errs(got, ref))


def test_batch_with_walls_matches_single_lattices():
    b, singles = run_pair(tel.FP64, [4, 3], walls=True)
    for k, s in enumerate(singles):
        got, ref = b.fields(k), s.fields()
        assert max_rel(got, ref) <= 1e-12, (k, max_rel(got, ref))


def test_batch_after_tuning_matches_single_lattices():
    b, singles = run_pair(tel.FP32_SHIFTED, [5], tune=True)
    info = b.info()
    assert info["tile_x"] in (32, 64) and info["chunk"] in (8, 16, 32, 64)
    assert info["ncases"] == len(SHAPES) and info["nodes"] == sum(x * y for x, y in SHAPES)
    assert 0 < info["ctas"] <= info["items"]
    for k, s in enumerate(singles):
        got, ref = b.fields(k), s.fields()
        assert close_fp32(got, ref), (k, errs(got, ref))


def test_batch_vector_phase_a_matches_single_lattices():
    """FP32 batch whose rows are all whole four-node vectors: the tuner runs
    every tile width and chunk on the vector path; each case still matches
    its single lattice."""
    b, singles = run_pair(tel.FP32_SHIFTED, [4, 3], tune=True, shapes=SHAPES_VEC)
    for k, s in enumerate(singles):
        got, ref = b.fields(k), s.fields()
        assert close_fp32(got, ref), (k, errs(got, ref))


def test_batch_fp64_against_oracle(orc):
    ps = [case_params(k, tel.FP64) for k in range(3)]
    shapes = SHAPES[:3]
    b = tel.Batch(shapes, ps)
    ref = []
    for k, (shape, p) in enumerate(zip(shapes, ps)):
        rho, phi, u = case_fields(k, shape, p)
        b.init(k, rho, phi, u)
        o = orc.Oracle(0, shape[0], shape[1], 1, p)
        fo, go = o.init(rho, phi, u)
        assert o.step(fo, go, 20) == 0
        ref.append(o.fields(fo, go))
    b.step(20)
    for k in range(3):
        assert max_rel(b.fields(k), ref[k]) <= 1e-10, k


def test_batch_errors():
    p = case_params(0, tel.FP64)
    with pytest.raises(tel.TelError) as ei:
        tel.Batch([(16, 16), (16, 16)], [p, dict(p, precision=tel.FP32_SHIFTED)])
    assert ei.value.code == tel.TEL_EINVAL
    b = tel.Batch([(16, 16), (24, 8)], p)
    with pytest.raises(tel.TelError) as ei:
        b.step(1)
    assert ei.value.code == tel.TEL_ESTATE
    rg, rl, _, _ = tel.coexistence(A, B, RGAS, p["T"])
    b.init(0, np.full(256, rl), np.zeros(256), np.zeros(512))
    u = np.zeros(2 * 192)
    u[7] = 1.5  # outside the entropic equilibrium's domain: flagged, not trapped
    with pytest.raises(tel.TelError) as ei:
        b.init(1, np.full(192, rl), np.zeros(192), u)
    assert ei.value.code == tel.TEL_EUNSTABLE and "case 1" in str(ei.value)
    b.init(1, np.full(192, rl), np.zeros(192), np.zeros(384))
    b.step(2)
    b.sync()


def test_batch_full_workload_against_single_lattices():
    """The batched benchmark's full workload (256 cases, 2.5e7 nodes) after
    the tuner and two more steps: the largest, the smallest and two random
    cases against single lattices advanced by the same number of steps.
    Density ratios up to 1000 make the pressure a difference of terms some
    10^3 times its own range, so its bar is 1e-3 here; density, phase field
    and velocity keep theirs."""
    import bench
    cases = bench.workload_c4(1710, 256)
    shapes, plist, fields = bench.c4_setup(cases)
    b = tel.Batch(shapes, plist)
    for c, (rho, phi, u) in enumerate(fields):
        b.init(c, rho, phi, u)
    done = b.tune(1)[2]
    b.step(2)
    b.sync()
    sizes = [x * y for x, y in shapes]
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes)), 17, 200}
    for c in sorted(pick):
        s = tel.Lattice(tel.D2Q9, shapes[c][0], shapes[c][1], 1, plist[c])
        s.init(*fields[c])
        s.step(done + 2)
        got, ref = b.fields(c), s.fields()
        assert close_fp32(got, ref, p_tol=1e-3), (c, errs(got, ref))
