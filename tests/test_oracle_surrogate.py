"""Pins of the surrogate oracle (oracle/surrogate.py) against what fixes it
independently of its own code: scipy's periodic correlation, exact shifts,
central finite differences of every gradient, adjoint identities of pooling
and upsampling, the mass-conserving projection, and the closed-form first
Adam step."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import surrogate as so


def rng(seed=0):
    return np.random.default_rng(seed)


def test_conv_matches_scipy_periodic_correlation():
    g = rng(1)
    x = g.normal(size=(2, 6, 10, 3))
    W = g.normal(size=(9, 3, 4))
    b = g.normal(size=4)
    y = so.conv_fwd(x, W, b, relu=False)
    for bi in range(2):
        for o in range(4):
            ref = np.full((6, 10), b[o])
            for i in range(3):
                K = W[:, i, o].reshape(3, 3)  # K[dy + 1, dx + 1]
                ref += ndimage.correlate(x[bi, :, :, i], K, mode="wrap")
            assert np.allclose(y[bi, :, :, o], ref, atol=1e-12)


@pytest.mark.parametrize("dy,dx", [(-1, 0), (0, 1), (1, -1), (0, 0)])
def test_conv_with_one_tap_is_a_periodic_shift(dy, dx):
    x = rng(2).normal(size=(1, 5, 7, 2))
    W = np.zeros((9, 2, 2))
    W[3 * (dy + 1) + (dx + 1)] = np.eye(2)
    y = so.conv_fwd(x, W, np.zeros(2), relu=False)
    for h in range(5):
        for w in range(7):
            assert np.allclose(y[0, h, w], x[0, (h + dy) % 5, (w + dx) % 7])


def fd_check(f, arr, grad, n=12, eps=1e-6, seed=0, rtol=1e-6):
    """Central differences of the scalar f() at n random entries of arr."""
    g = rng(seed)
    flat = arr.reshape(-1)
    gflat = grad.reshape(-1)
    for k in g.choice(flat.size, size=min(n, flat.size), replace=False):
        v = flat[k]
        flat[k] = v + eps
        fp = f()
        flat[k] = v - eps
        fm = f()
        flat[k] = v
        num = (fp - fm) / (2 * eps)
        assert abs(num - gflat[k]) <= rtol * max(1.0, abs(num)) + 1e-8, (k, num, gflat[k])


@pytest.mark.parametrize("relu", [False, True])
def test_conv_gradients_finite_differences(relu):
    g = rng(3)
    x = g.normal(size=(2, 4, 6, 3))
    W = g.normal(size=(9, 3, 5))
    b = g.normal(size=5)
    R = g.normal(size=(2, 4, 6, 5))
    f = lambda: float((so.conv_fwd(x, W, b, relu) * R).sum())
    y = so.conv_fwd(x, W, b, relu)
    dx, dW, db = so.conv_bwd(x, W, y, R, relu)
    fd_check(f, x, dx, seed=1)
    fd_check(f, W, dW, seed=2)
    fd_check(f, b, db, seed=3)


def test_pool_and_up_adjoints_and_inverse():
    g = rng(4)
    a = g.normal(size=(2, 8, 6, 3))
    c = g.normal(size=(2, 4, 3, 3))
    assert np.isclose((so.pool_fwd(a) * c).sum(), (a * so.pool_bwd(c)).sum())
    assert np.isclose((so.up_fwd(c) * a).sum(), (c * so.up_bwd(a)).sum())
    assert np.allclose(so.pool_fwd(so.up_fwd(c)), c)


def tiny():
    ops = so.arch(2, 3, 4)
    Ws, bs = so.init_params(ops, seed=5)
    g = rng(6)
    bs = [g.normal(scale=0.1, size=b.shape) for b in bs]
    return ops, Ws, bs


def test_network_gradients_finite_differences():
    ops, Ws, bs = tiny()
    g = rng(7)
    x = g.normal(size=(2, 8, 8, so.CIN))
    T = g.normal(size=(2, 8, 8, so.NF))

    def L():
        out, _ = so.forward(ops, Ws, bs, x)
        return so.loss(out, T)[0]

    out, cache = so.forward(ops, Ws, bs, x)
    _, dout = so.loss(out, T)
    dWs, dbs, dx = so.backward(cache, Ws, dout)
    for k in (0, 4, 7, 11):
        fd_check(L, Ws[k], dWs[k], n=6, seed=k)
        fd_check(L, bs[k], dbs[k], n=3, seed=k + 20)
    fd_check(L, x, dx, n=6, seed=99)


def test_projection_conserves_mass_and_is_idempotent():
    d = rng(8).normal(size=(3, 4, 4, so.COUT))
    p = so.project(d)
    assert np.allclose(p[..., :2].sum(axis=(1, 2)), 0.0, atol=1e-12)
    assert np.allclose(p[..., 2:], d[..., 2:4])
    pad = np.concatenate([p, np.zeros(p.shape[:-1] + (so.COUT - so.NF,))], axis=-1)
    assert np.allclose(so.project(pad), p)
    x4 = rng(9).normal(size=(3, 4, 4, so.NF))
    nxt = so.advance(x4, d, [0.5, 2.0, 1.0, 1.0])
    assert np.allclose(nxt[..., :2].sum(axis=(1, 2)), x4[..., :2].sum(axis=(1, 2)))


def test_first_adam_step_moves_by_lr_times_sign():
    g = rng(10).normal(size=50)
    w = np.zeros(50)
    w1, m, v = so.adam(w, g, np.zeros(50), np.zeros(50), t=1, lr=0.01, eps=0.0)
    assert np.allclose(w1, -0.01 * np.sign(g))


def test_pack_normalises_fields():
    g = rng(11)
    rho, phi, ux, uy = (g.normal(size=(2, 4, 4)) for _ in range(4))
    x = so.pack(rho, phi, ux, uy, rho_l=2.0, chi=5.0, U=0.1)
    assert np.allclose(x[..., 0] * 2.0, rho) and np.allclose(x[..., 1] * 5.0, phi)
    assert np.allclose(x[..., 2] * 0.1, ux) and np.allclose(x[..., 3] * 0.1, uy)
    assert np.all(x[..., 4:] == 0)


def test_field_errors_definition():
    t = np.ones((1, 2, 2, 4))
    p = t.copy()
    p[..., 0] *= 1.01
    e = so.field_errors(p, t)
    assert np.isclose(e["rho"], 0.01) and e["phi"] == 0 and e["u"] == 0


def _wiring_case(seed=3, widths=(8, 8, 16), B=1, H=16, W=16):
    from tests.sur_wiring import to_bf16
    g = np.random.default_rng(seed)
    ops = so.arch(*widths)
    Ws, bs = so.init_params(ops, seed)
    Ws = [to_bf16(w) for w in Ws]
    bs = [g.normal(0.0, 0.05, size=b.shape) for b in bs]
    x = to_bf16(g.normal(size=(B, H, W, so.CIN)))
    dout = to_bf16(g.normal(size=(B, H, W, so.COUT)))
    return ops, Ws, bs, x, dout


def test_wiring_check_passes_a_correct_network():
    from tests.sur_wiring import check, oracle_records, to_bf16
    ops, Ws, bs, x, dout = _wiring_case()
    fwd, bwd = oracle_records(ops, Ws, bs, x, dout, to_bf16)
    mis = check(ops, Ws, bs, x, dout, fwd, bwd, to_bf16)
    assert len(mis) > 3 * len(Ws)
    assert max(m for _, _, m in mis) <= 1e-9, [m for m in mis if m[2] > 1e-9]


@pytest.mark.parametrize("plant", ["skip_scale", "skip_source", "relu_mask", "weight_flip", "wgrad_tap",
                                   "pool_scale"])
def test_wiring_check_catches_planted_mistakes(plant):
    """Each planted wiring mistake is flagged, at three times the pass bar
    or more (a skip scaled by 0.97 is about four BF16 ulps)."""
    from tests.sur_wiring import check, oracle_records, to_bf16
    ops, Ws, bs, x, dout = _wiring_case()
    fwd, bwd = oracle_records(ops, Ws, bs, x, dout, to_bf16, plant=plant)
    mis = check(ops, Ws, bs, x, dout, fwd, bwd, to_bf16)
    bad = [m for m in mis if m[2] > 1.0]
    assert bad and max(m[2] for m in bad) > 3.0, (plant, sorted(mis, key=lambda m: -m[2])[:3])
