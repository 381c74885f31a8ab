"""FP64 CPU oracle of the learned surrogate: a small periodic convolutional
encoder-decoder that advances the density, composition and velocity fields of
the ternary LBM k steps at a time.

TEST INFRASTRUCTURE ONLY.  Plain numpy in float64: each operation and its
gradient is written out from its definition (no blocking, no fusion), so that
the library's BF16 kernels can be checked against it.  Only the tests, the
smoke check and the benchmark's CPU leg use this module; it never imports the
library package.

The paper itself has no surrogate; this network is the learned part built on
top of the method.  Conventions (shared with the library only through this
text, not through code):

* activations are NHWC arrays ``x[b, h, w, c]`` on a periodic H x W grid;
* a 3x3 convolution is a cross-correlation with periodic wrap:
  ``y[b,h,w,o] = bias[o] + sum_t sum_i x[b,(h+dy_t)%H,(w+dx_t)%W,i] W[t,i,o]``
  with tap ``t = 3 (dy + 1) + (dx + 1)``, ``dy, dx`` in {-1, 0, 1};
* ``pool`` is the 2x2 mean, ``up`` the 2x2 nearest-neighbour copy;
* the network input has 16 channels: (rho / rho_l, phi / chi, u_x / U, u_y / U)
  and twelve zeros; of the 16 output channels the first four are the change
  of those fields over k steps, in units of ``scale[c]``;
* the head projects the density and composition changes to zero spatial mean
  per sample (the LBM conserves both components' mass exactly), so the
  prediction conserves mass by construction.
"""
from __future__ import annotations

import numpy as np

CIN = 16     # network input channels (4 fields + zero padding)
COUT = 16    # network output channels (first 4 used)
NF = 4       # fields: rho, phi, u_x, u_y


# ---------------------------------------------------------------------------
# architecture: widths (c0, c1, c2) on three resolution levels
# ---------------------------------------------------------------------------
def arch(c0=32, c1=64, c2=128):
    """The op sequence of the encoder-decoder.  Each conv entry is
    ('conv', index, cin, cout, relu); 'pool', 'up', ('save', name) and
    ('add', name) act on the running activation."""
    return [
        ("conv", 0, CIN, c0, True), ("conv", 1, c0, c0, True), ("save", "s0"), ("pool",),
        ("conv", 2, c0, c1, True), ("conv", 3, c1, c1, True), ("save", "s1"), ("pool",),
        ("conv", 4, c1, c2, True), ("conv", 5, c2, c2, True), ("conv", 6, c2, c2, True), ("up",),
        ("conv", 7, c2, c1, True), ("add", "s1"), ("conv", 8, c1, c1, True), ("up",),
        ("conv", 9, c1, c0, True), ("add", "s0"), ("conv", 10, c0, c0, True),
        ("conv", 11, c0, COUT, False),
    ]


def conv_shapes(ops):
    return [(op[2], op[3]) for op in ops if op[0] == "conv"]


# ---------------------------------------------------------------------------
# single operations and their gradients
# ---------------------------------------------------------------------------
TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shifted(x, dy, dx):
    """xs[b, h, w] = x[b, (h + dy) % H, (w + dx) % W]."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv_fwd(x, W, bias, relu):
    B, H, Wd, ci = x.shape
    co = W.shape[2]
    z = np.broadcast_to(bias, (B, H, Wd, co)).astype(np.float64).copy()
    for t, (dy, dx) in enumerate(TAPS):
        z += shifted(x, dy, dx).reshape(-1, ci).dot(W[t]).reshape(B, H, Wd, co)
    return np.maximum(z, 0.0) if relu else z


def conv_bwd(x, W, y, dy_, relu):
    """Gradients of a conv layer with respect to its input, weights and bias,
    given its output y (whose sign gives the ReLU mask) and dL/dy."""
    B, H, Wd, ci = x.shape
    co = W.shape[2]
    dz = dy_ * (y > 0) if relu else dy_
    db = dz.sum(axis=(0, 1, 2))
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    dzf = dz.reshape(-1, co)
    for t, (dy, dx_) in enumerate(TAPS):
        dW[t] = shifted(x, dy, dx_).reshape(-1, ci).T.dot(dzf)
        # x[p + d] fed y[p]: its gradient lands back at p + d
        dx += np.roll(dzf.dot(W[t].T).reshape(B, H, Wd, ci), shift=(dy, dx_), axis=(1, 2))
    return dx, dW, db


def pool_fwd(x):
    B, H, Wd, C = x.shape
    return x.reshape(B, H // 2, 2, Wd // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up_fwd(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(dy):
    B, H, Wd, C = dy.shape
    return dy.reshape(B, H // 2, 2, Wd // 2, 2, C).sum(axis=(2, 4))


# ---------------------------------------------------------------------------
# whole network
# ---------------------------------------------------------------------------
def init_params(ops, seed):
    """He-normal weights and zero biases (seeded); the last layer starts at
    zero output scale x 0.1."""
    g = np.random.default_rng(seed)
    Ws, bs = [], []
    convs = [op for op in ops if op[0] == "conv"]
    for k, (_, _, ci, co, relu) in enumerate(convs):
        std = np.sqrt(2.0 / (9 * ci)) * (1.0 if relu else 0.1)
        Ws.append(g.normal(0.0, std, size=(9, ci, co)))
        bs.append(np.zeros(co))
    return Ws, bs


def _keep(a):
    return a


def forward(ops, Ws, bs, x, rnd=None):
    """Returns the output and the cache the backward pass needs.

    ``rnd`` (default: none) is applied to every stored activation (conv,
    pool and add outputs); a test passes a rounding to a storage format to
    follow a reduced-precision implementation step by step."""
    rnd = rnd or _keep
    cache, saved = [], {}
    a = x
    for op in ops:
        if op[0] == "conv":
            _, k, ci, co, relu = op
            y = rnd(conv_fwd(a, Ws[k], bs[k], relu))
            cache.append(("conv", k, a, y, relu))
            a = y
        elif op[0] == "pool":
            cache.append(("pool",))
            a = rnd(pool_fwd(a))
        elif op[0] == "up":
            cache.append(("up",))
            a = up_fwd(a)
        elif op[0] == "save":
            cache.append(("save", op[1]))
            saved[op[1]] = a
        elif op[0] == "add":
            cache.append(("add", op[1]))
            a = rnd(a + saved[op[1]])
    return a, cache


def backward(cache, Ws, dout, rnd=None):
    """Gradients of every weight and bias from dL/d(output); ``rnd`` as in
    forward, applied to every stored activation gradient."""
    rnd = rnd or _keep
    dWs = [None] * len(Ws)
    dbs = [None] * len(Ws)
    grads_saved = {}
    d = dout
    for entry in reversed(cache):
        kind = entry[0]
        if kind == "conv":
            _, k, a_in, y, relu = entry
            d, dWs[k], dbs[k] = conv_bwd(a_in, Ws[k], y, d, relu)
            d = rnd(d)
        elif kind == "pool":
            d = rnd(pool_bwd(d))
        elif kind == "up":
            d = rnd(up_bwd(d))
        elif kind == "add":
            # y = a + s: the saved activation receives the same gradient
            grads_saved[entry[1]] = d
        elif kind == "save":
            d = rnd(d + grads_saved.pop(entry[1]))
    return dWs, dbs, d


# ---------------------------------------------------------------------------
# head, loss, optimiser, field normalisation
# ---------------------------------------------------------------------------
def project(delta):
    """delta[..., :4] with the spatial mean of channels 0 and 1 removed per
    sample (the other channels unchanged)."""
    p = delta[..., :NF].copy()
    p[..., :2] -= p[..., :2].mean(axis=(1, 2), keepdims=True)
    return p


def loss(out, target, rnd=None):
    """Mean squared error of the projected change against the target change
    (both in units of scale); returns (L, dL/d out), ``rnd`` applied to the
    latter."""
    p = project(out)
    r = p - target
    n = r.size
    L = float((r * r).sum() / n)
    g = 2.0 * r / n
    dout = np.zeros_like(out)
    dout[..., :NF] = project(np.concatenate([g, np.zeros(out.shape[:-1] + (out.shape[-1] - NF,))], axis=-1))
    return L, (rnd(dout) if rnd else dout)


def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, bias-corrected), returns new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def pack(rho, phi, ux, uy, rho_l, chi, U):
    """Fields (B, H, W) -> network input (B, H, W, 16)."""
    x = np.zeros(rho.shape + (CIN,))
    x[..., 0] = rho / rho_l
    x[..., 1] = phi / chi
    x[..., 2] = ux / U
    x[..., 3] = uy / U
    return x


def advance(x4, out, scale):
    """Next normalised fields: x + scale * project(out)."""
    return x4 + np.asarray(scale) * project(out)


def field_errors(pred, true):
    """Relative L2 errors of density, composition and velocity (normalised
    fields, last axis rho, phi, u_x, u_y)."""
    e = {}
    for name, sl in (("rho", [0]), ("phi", [1]), ("u", [2, 3])):
        num = np.sqrt(((pred[..., sl] - true[..., sl]) ** 2).sum())
        den = np.sqrt((true[..., sl] ** 2).sum())
        e[name] = float(num / den) if den > 0 else float(num)
    return e
