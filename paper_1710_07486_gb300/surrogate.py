"""Learned surrogate of the D2Q9 ternary lattice update (binding and driver).

A small periodic convolutional encoder-decoder advances the normalised
density, composition and velocity fields k lattice steps at a time.  Every
operation of training and inference runs in libternelbm's kernels
(include/ternelbm_sur.h): BF16 tensor-core convolutions with FP32
accumulation, their input and weight gradients, pooling, the
mass-conserving head, the loss and Adam.  This module only allocates device
buffers (PyTorch tensors) and issues the calls in order.

The lattice update itself produces the training snapshots (``Snapshots``),
and stays the fallback and the judge of the surrogate's error
(``Hybrid``): a surrogate step is rejected, and the lattice update runs
instead, when the per-component mass residual or the field error against a
periodic lattice check exceeds its threshold.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import Batch, TelError, lib

CIN, COUT, NF = 16, 16, 4
U_REF = 0.1  # velocity normalisation (lattice units)

SUR_SYMBOLS = ("tel_sur_conv3x3", "tel_sur_conv3x3_tc", "tel_sur_conv3x3_tc_fused", "tel_sur_flip_weights", "tel_sur_relu_bwd", "tel_sur_conv3x3_wgrad",
               "tel_sur_pool2", "tel_sur_pool2_bwd", "tel_sur_up2", "tel_sur_up2_bwd", "tel_sur_add",
               "tel_sur_pack", "tel_sur_unpack", "tel_sur_gather", "tel_sur_loss", "tel_sur_advance",
               "tel_sur_errors", "tel_sur_sums", "tel_sur_adam", "tel_sur_clip_scale", "tel_sur_adam_scaled",
               "tel_sur_zero", "tel_sur_to_bf16")


def sur_lib():
    L = lib()
    if getattr(L, "_sur_ready", False):
        return L
    vp, i, ll, f = C.c_void_p, C.c_int, C.c_longlong, C.c_float
    L.tel_sur_conv3x3.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, vp]
    L.tel_sur_conv3x3_tc.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, vp, vp]
    L.tel_sur_conv3x3_tc_fused.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, i, vp, vp, vp]
    L.tel_sur_flip_weights.argtypes = [vp, vp, i, i, vp]
    L.tel_sur_relu_bwd.argtypes = [vp, vp, vp, ll, vp]
    L.tel_sur_conv3x3_wgrad.argtypes = [vp, vp, vp, vp, i, i, i, i, i, vp]
    for n in ("tel_sur_pool2", "tel_sur_pool2_bwd", "tel_sur_up2", "tel_sur_up2_bwd"):
        getattr(L, n).argtypes = [vp, vp, i, i, i, i, vp]
    L.tel_sur_add.argtypes = [vp, vp, vp, ll, vp]
    L.tel_sur_pack.argtypes = [vp, vp, vp, vp, vp, vp, i, i, i, vp]
    L.tel_sur_unpack.argtypes = [vp, vp, vp, vp, vp, i, i, i, vp]
    L.tel_sur_gather.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i, i, i, vp]
    L.tel_sur_loss.argtypes = [vp, vp, vp, vp, vp, i, i, i, vp]
    L.tel_sur_advance.argtypes = [vp, vp, vp, vp, vp, vp, vp, i, i, i, vp]
    L.tel_sur_errors.argtypes = [vp, vp, vp, i, i, i, vp]
    L.tel_sur_sums.argtypes = [vp, vp, i, i, i, vp]
    L.tel_sur_adam.argtypes = [vp, vp, vp, vp, vp, ll, f, f, f, f, i, f, vp]
    L.tel_sur_clip_scale.argtypes = [vp, ll, f, vp, vp, vp]
    L.tel_sur_adam_scaled.argtypes = [vp, vp, vp, vp, vp, ll, f, f, f, f, i, vp, vp]
    L.tel_sur_zero.argtypes = [vp, ll, vp]
    L.tel_sur_to_bf16.argtypes = [vp, vp, ll, vp]
    for n in SUR_SYMBOLS:
        getattr(L, n).restype = C.c_int
    L._sur_ready = True
    return L


def _p(t, offset=0):
    """Device pointer of a tensor (plus an element offset), or None."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr() + offset * t.element_size())


def _ok(rc, what):
    if rc:
        raise TelError(rc, f"{what} failed")


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def layers(c0=32, c1=64, c2=128):
    """Encoder-decoder op list: ('conv', cin, cout, relu), ('pool',), ('up',),
    ('save', slot), ('add', slot).  Three levels (H, H/2, H/4)."""
    return [("conv", CIN, c0, 1), ("conv", c0, c0, 1), ("save", 0), ("pool",),
            ("conv", c0, c1, 1), ("conv", c1, c1, 1), ("save", 1), ("pool",),
            ("conv", c1, c2, 1), ("conv", c2, c2, 1), ("conv", c2, c2, 1), ("up",),
            ("conv", c2, c1, 1), ("add", 1), ("conv", c1, c1, 1), ("up",),
            ("conv", c1, c0, 1), ("add", 0), ("conv", c0, c0, 1),
            ("conv", c0, COUT, 0)]


class Net:
    """Parameters (FP32 master, BF16 working copy, Adam moments) and the
    forward/backward sequence for one batch shape (B, H, W)."""

    def __init__(self, widths=(32, 64, 128), seed=0, conv="auto"):
        """conv selects the kernel of the forward and input-gradient
        convolutions: "tc" (tcgen05, accumulator in tensor memory), "mma"
        (warp-level tensor-core kernel) or "auto" (default): tcgen05 on
        grids whose rows are whole 128-pixel segments, where its shared halo
        tile makes it the faster, the warp-level kernel elsewhere."""
        import torch
        self.torch = torch
        self.L = sur_lib()
        if conv not in ("mma", "tc", "auto"):
            raise ValueError("conv must be 'mma', 'tc' or 'auto'")
        self.conv = conv
        self.tc_err = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.ops = layers(*widths)
        self.convs = [op for op in self.ops if op[0] == "conv"]
        # flat layout: per conv W [9][cout][cin] then b [cout]
        self.woff, self.boff = [], []
        n = 0
        for _, ci, co, _ in self.convs:
            self.woff.append(n)
            n += 9 * co * ci
            self.boff.append(n)
            n += co
        self.n = n
        g = np.random.default_rng(seed)
        host = np.zeros(n, dtype=np.float32)
        for k, (_, ci, co, relu) in enumerate(self.convs):
            std = math.sqrt(2.0 / (9 * ci)) * (1.0 if relu else 0.1)
            host[self.woff[k]:self.woff[k] + 9 * co * ci] = g.normal(0.0, std, 9 * co * ci)
        dev = torch.device("cuda")
        self.w32 = torch.from_numpy(host).to(dev)
        self.w16 = torch.empty(n, dtype=torch.bfloat16, device=dev)
        self.wt16 = torch.empty(n, dtype=torch.bfloat16, device=dev)  # flipped weights (same offsets)
        self.g = torch.zeros(n, dtype=torch.float32, device=dev)
        self.m = torch.zeros(n, dtype=torch.float32, device=dev)
        self.v = torch.zeros(n, dtype=torch.float32, device=dev)
        self.t = 0
        self.sync_bf16()
        self._plans = {}

    @property
    def params(self):
        return self.n

    def conv3x3(self, x, w_off, w, bias, y, B, H, W, ci, co, relu, s):
        """One convolution with the selected kernel (weights at w[w_off:])."""
        if self.conv == "tc" or (self.conv == "auto" and W % 128 == 0):
            return self.L.tel_sur_conv3x3_tc(_p(x), _p(w, w_off), bias, _p(y), B, H, W, ci, co, relu,
                                             _p(self.tc_err), s)
        return self.L.tel_sur_conv3x3(_p(x), _p(w, w_off), bias, _p(y), B, H, W, ci, co, relu, s)

    def sync_bf16(self):
        _ok(self.L.tel_sur_to_bf16(_p(self.w32), _p(self.w16), self.n, _stream()), "to_bf16")

    def set_host_weights(self, host):
        """Replace the FP32 master weights by a host array (flat layout)."""
        self.w32.copy_(self.torch.from_numpy(np.ascontiguousarray(host, dtype=np.float32)))
        self.sync_bf16()

    def host_layers(self):
        """(W [9][cout][cin], b [cout]) per conv as float64 host arrays."""
        h = self.w32.cpu().numpy().astype(np.float64)
        out = []
        for k, (_, ci, co, _) in enumerate(self.convs):
            out.append((h[self.woff[k]:self.woff[k] + 9 * co * ci].reshape(9, co, ci),
                        h[self.boff[k]:self.boff[k] + co].copy()))
        return out

    # ------------------------------------------------------------ buffers
    def plan(self, B, H, W):
        key = (B, H, W)
        if key not in self._plans:
            self._plans[key] = _Plan(self, B, H, W)
        return self._plans[key]

    def forward(self, x16, B, H, W):
        """Network output (bf16 [B][H][W][16]) for input x16; keeps the
        activations for backward."""
        return self.plan(B, H, W).forward(x16)

    def backward(self, dout, B, H, W):
        """Accumulates the parameter gradient into self.g."""
        self.plan(B, H, W).backward(dout)

    def zero_grad(self):
        _ok(self.L.tel_sur_zero(_p(self.g), self.n, _stream()), "zero")

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8, grad_scale=1.0, clip=None):
        """One Adam step; with clip, the gradient is first scaled to a global
        norm of at most clip (computed and applied on the device)."""
        self.t += 1
        if clip is not None:
            if not hasattr(self, "_clip_work"):
                self._clip_work = self.torch.zeros(1, dtype=self.torch.float64, device="cuda")
                self._clip_scale = self.torch.ones(1, dtype=self.torch.float32, device="cuda")
            _ok(self.L.tel_sur_clip_scale(_p(self.g), self.n, float(clip), _p(self._clip_work), _p(self._clip_scale),
                                          _stream()), "clip_scale")
            _ok(self.L.tel_sur_adam_scaled(_p(self.w32), _p(self.w16), _p(self.g), _p(self.m), _p(self.v), self.n,
                                           float(lr), float(b1), float(b2), float(eps), self.t, _p(self._clip_scale),
                                           _stream()), "adam")
            return
        _ok(self.L.tel_sur_adam(_p(self.w32), _p(self.w16), _p(self.g), _p(self.m), _p(self.v), self.n,
                                float(lr), float(b1), float(b2), float(eps), self.t, float(grad_scale),
                                _stream()), "adam")


class _Plan:
    """Preallocated activations and gradients for one (B, H, W)."""

    def __init__(self, net, B, H, W):
        torch = net.torch
        self.net, self.B, self.H, self.W = net, B, H, W
        L = net.L
        dev = torch.device("cuda")
        bf = torch.bfloat16
        # forward records: (kind, ...) with the tensors each op reads/writes
        self.recs = []
        h, w, c = H, W, CIN
        saved = {}
        k = 0
        self.x_in = None
        for op in net.ops:
            if op[0] == "conv":
                _, ci, co, relu = op
                y = torch.empty((B, h, w, co), dtype=bf, device=dev)
                self.recs.append(["conv", k, ci, co, relu, h, w, None, y])
                c = co
                k += 1
            elif op[0] == "pool":
                y = torch.empty((B, h // 2, w // 2, c), dtype=bf, device=dev)
                self.recs.append(["pool", c, h, w, y])
                h, w = h // 2, w // 2
            elif op[0] == "up":
                y = torch.empty((B, 2 * h, 2 * w, c), dtype=bf, device=dev)
                self.recs.append(["up", c, 2 * h, 2 * w, y])
                h, w = 2 * h, 2 * w
            elif op[0] == "save":
                self.recs.append(["save", op[1], c, h, w])
            elif op[0] == "add":
                y = torch.empty((B, h, w, c), dtype=bf, device=dev)
                self.recs.append(["add", op[1], c, h, w, y])
        self.out = self.recs[-1][-1]
        # gradient buffers: one per record output shape, plus dz per conv
        self.dz = [torch.empty_like(r[8]) for r in self.recs if r[0] == "conv"]
        self.dx = {}
        for r in self.recs:
            if r[0] == "conv":
                self.dx[id(r)] = torch.empty((B, r[5], r[6], r[2]), dtype=bf, device=dev)
            elif r[0] == "pool":
                self.dx[id(r)] = torch.empty((B, r[2], r[3], r[1]), dtype=bf, device=dev)
            elif r[0] == "up":
                self.dx[id(r)] = torch.empty((B, r[2] // 2, r[3] // 2, r[1]), dtype=bf, device=dev)
            elif r[0] == "save":
                self.dx[id(r)] = torch.empty((B, r[3], r[4], r[2]), dtype=bf, device=dev)

    def forward(self, x16):
        net, L, B = self.net, self.net.L, self.B
        s = _stream()
        a = x16
        saved = {}
        for r in self.recs:
            kind = r[0]
            if kind == "conv":
                _, k, ci, co, relu, h, w, _, y = r
                r[7] = a
                _ok(net.conv3x3(a, net.woff[k], net.w16, _p(net.w32, net.boff[k]), y, B, h, w, ci, co, relu, s),
                    "conv3x3")
                a = y
            elif kind == "pool":
                _, c, h, w, y = r
                _ok(L.tel_sur_pool2(_p(a), _p(y), B, h, w, c, s), "pool2")
                a = y
            elif kind == "up":
                _, c, h, w, y = r
                _ok(L.tel_sur_up2(_p(a), _p(y), B, h, w, c, s), "up2")
                a = y
            elif kind == "save":
                saved[r[1]] = a
            elif kind == "add":
                _, slot, c, h, w, y = r
                _ok(L.tel_sur_add(_p(a), _p(saved[slot]), _p(y), B * h * w * c, s), "add")
                a = y
        return a

    def infer(self, x16):
        """Forward pass for inference (nothing kept for backward): on grids
        the tensor-memory halo kernel serves, an upsampling is read by the
        next convolution directly and a skip addition happens in that
        convolution's epilogue; the result equals forward()'s bit for bit."""
        net, L, B = self.net, self.net.L, self.B
        s = _stream()
        recs = self.recs

        def fusable(h, w):
            return net.conv != "mma" and w % 128 == 0 and h % 4 == 0

        a = x16
        saved = {}
        pending_up = None
        self.launches = 0  # kernels issued by this pass (one per library call below)
        i = 0
        while i < len(recs):
            r = recs[i]
            kind = r[0]
            if kind == "conv":
                _, k, ci, co, relu, h, w, _, y = r
                nxt = recs[i + 1] if i + 1 < len(recs) else None
                skip, out = None, y
                if fusable(h, w) and nxt is not None and nxt[0] == "add":
                    skip, out = saved[nxt[1]], nxt[5]
                    i += 1
                if pending_up is not None or skip is not None:
                    src = pending_up if pending_up is not None else a
                    self.launches += 1
                    _ok(L.tel_sur_conv3x3_tc_fused(_p(src), _p(net.w16, net.woff[k]), _p(net.w32, net.boff[k]),
                                                   _p(out), B, h, w, ci, co, relu, 1 if pending_up is not None else 0,
                                                   _p(skip), _p(net.tc_err), s), "conv3x3 (fused)")
                    pending_up = None
                else:
                    self.launches += 1
                    _ok(net.conv3x3(a, net.woff[k], net.w16, _p(net.w32, net.boff[k]), y, B, h, w, ci, co, relu, s),
                        "conv3x3")
                a = out
            elif kind == "pool":
                _, c, h, w, y = r
                self.launches += 1
                _ok(L.tel_sur_pool2(_p(a), _p(y), B, h, w, c, s), "pool2")
                a = y
            elif kind == "up":
                _, c, h, w, y = r
                nxt = recs[i + 1]
                if nxt[0] == "conv" and fusable(nxt[5], nxt[6]):
                    pending_up = a  # read through upsampling by the next convolution
                else:
                    self.launches += 1
                    _ok(L.tel_sur_up2(_p(a), _p(y), B, h, w, c, s), "up2")
                    a = y
            elif kind == "save":
                saved[r[1]] = a
            elif kind == "add":
                _, slot, c, h, w, y = r
                self.launches += 1
                _ok(L.tel_sur_add(_p(a), _p(saved[slot]), _p(y), B * h * w * c, s), "add")
                a = y
            i += 1
        return a

    def backward(self, dout):
        net, L, B = self.net, self.net.L, self.B
        s = _stream()
        d = dout
        gsaved = {}
        convs = [r for r in self.recs if r[0] == "conv"]
        for r in reversed(self.recs):
            kind = r[0]
            if kind == "conv":
                _, k, ci, co, relu, h, w, a_in, y = r
                dz = self.dz[k]
                if relu:
                    _ok(L.tel_sur_relu_bwd(_p(y), _p(d), _p(dz), B * h * w * co, s), "relu_bwd")
                else:
                    dz = d
                _ok(L.tel_sur_conv3x3_wgrad(_p(a_in), _p(dz), _p(net.g, net.woff[k]), _p(net.g, net.boff[k]),
                                            B, h, w, ci, co, s), "wgrad")
                if k > 0:
                    _ok(L.tel_sur_flip_weights(_p(net.w16, net.woff[k]), _p(net.wt16, net.woff[k]), ci, co, s),
                        "flip")
                    dx = self.dx[id(r)]
                    _ok(net.conv3x3(dz, net.woff[k], net.wt16, None, dx, B, h, w, co, ci, 0, s),
                        "conv3x3 (input gradient)")
                    d = dx
            elif kind == "pool":
                _, c, h, w, _ = r
                dx = self.dx[id(r)]
                _ok(L.tel_sur_pool2_bwd(_p(d), _p(dx), B, h, w, c, s), "pool2_bwd")
                d = dx
            elif kind == "up":
                _, c, h, w, _ = r
                dx = self.dx[id(r)]
                _ok(L.tel_sur_up2_bwd(_p(d), _p(dx), B, h, w, c, s), "up2_bwd")
                d = dx
            elif kind == "add":
                gsaved[r[1]] = d
            elif kind == "save":
                _, slot, c, h, w = r
                dx = self.dx[id(r)]
                _ok(L.tel_sur_add(_p(d), _p(gsaved.pop(slot)), _p(dx), B * h * w * c, s), "add (gradient)")
                d = dx
        del convs


# ---------------------------------------------------------------------------
# snapshots of the lattice update
# ---------------------------------------------------------------------------
class Snapshots:
    """Normalised fields of ``ntraj`` D2Q9 trajectories (same H x W, own
    parameters), every ``k`` steps, ``nsnap`` snapshots each, generated by
    the batched lattice update and kept on the device as FP32
    [nsnap][ntraj][H][W][4].  Trajectories whose lattice flagged an unstable
    node are marked bad and left out of training and evaluation."""

    def __init__(self, shape, params, fields, k, nsnap, tune=True):
        import torch
        L = sur_lib()
        H, W = shape
        self.H, self.W, self.k, self.nsnap = H, W, k, nsnap
        self.ntraj = n = len(params)
        dev = torch.device("cuda")
        b = Batch([(W, H)] * n, params)
        for c, (rho, phi, u) in enumerate(fields):
            b.init(c, rho, phi, u)
        if tune:
            b.tune(1)  # advances every case by the same number of steps
        N = H * W
        self.norm_host = np.array([[1.0 / coex_rho_l(p), 1.0 / p["chi"], 1.0 / U_REF] for p in params],
                                  dtype=np.float32)
        self.norm = torch.from_numpy(self.norm_host).to(dev)
        self.store = torch.empty((nsnap, n, H, W, NF), dtype=torch.float32, device=dev)
        rho = torch.empty((n, N), dtype=torch.float64, device=dev)
        phi = torch.empty((n, N), dtype=torch.float64, device=dev)
        u = torch.empty((n, 2, N), dtype=torch.float64, device=dev)
        bad = np.zeros(n, dtype=bool)
        stream = torch.cuda.Stream()
        b.set_stream(stream)
        for s in range(nsnap):
            if s:
                b.step(k)
            for c in range(n):
                b.fields_device(c, rho[c], phi[c], u[c])
            with torch.cuda.stream(stream):
                _ok(L.tel_sur_pack(_p(rho), _p(phi), _p(u), _p(self.norm), _p(self.store[s]), None, n, H, W,
                                   C.c_void_p(stream.cuda_stream)), "pack")
            bad |= np.array(b.errors()) != 0
        stream.synchronize()
        b.close()
        self.bad = bad
        self.good = np.flatnonzero(~bad)

    def pairs(self, snaps=None):
        """(src, dst) flat store indices of consecutive snapshots of good
        trajectories (store index = s * ntraj + traj)."""
        src, dst = [], []
        snaps = range(self.nsnap - 1) if snaps is None else snaps
        for s in snaps:
            for t in self.good:
                src.append(s * self.ntraj + t)
                dst.append((s + 1) * self.ntraj + t)
        return np.array(src, dtype=np.int32), np.array(dst, dtype=np.int32)

    def delta_scale(self, src, dst, sample=256, seed=0):
        """Per-field RMS of the k-step change, from a host sample of pairs."""
        g = np.random.default_rng(seed)
        idx = g.choice(len(src), size=min(sample, len(src)), replace=False)
        flat = self.store.view(-1, self.H, self.W, NF)
        a = flat[src[idx]].cpu().numpy().astype(np.float64)
        z = flat[dst[idx]].cpu().numpy().astype(np.float64)
        rms = np.sqrt(((z - a) ** 2).mean(axis=(0, 1, 2)))
        rms[2] = rms[3] = np.sqrt(0.5 * (rms[2] ** 2 + rms[3] ** 2))  # one scale: symmetries mix u_x, u_y
        return np.maximum(rms, 1e-8).astype(np.float32)


def coex_rho_l(p):
    from . import coexistence
    return coexistence(p["a"], p["b"], p["R"], p["T"])[1]


# ---------------------------------------------------------------------------
# training and inference
# ---------------------------------------------------------------------------
class Trainer:
    """Adam on the mean squared error of the projected k-step change."""

    def __init__(self, net, snaps, B=8, seed=0, scale=None, augment=True, clip=None):
        import torch
        self.net, self.snaps, self.B = net, snaps, B
        self.torch = torch
        L = net.L
        H, W = snaps.H, snaps.W
        dev = torch.device("cuda")
        self.src, self.dst = snaps.pairs()
        self.scale_host = snaps.delta_scale(self.src, self.dst) if scale is None else np.asarray(scale, np.float32)
        self.scale = torch.from_numpy(self.scale_host).to(dev)
        self.f32 = torch.empty((B, H, W, NF), dtype=torch.float32, device=dev)
        self.x16 = torch.empty((B, H, W, CIN), dtype=torch.bfloat16, device=dev)
        self.tgt = torch.empty((B, H, W, NF), dtype=torch.float32, device=dev)
        self.dout = torch.empty((B, H, W, COUT), dtype=torch.bfloat16, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.work = torch.zeros(4 * B, dtype=torch.float32, device=dev)
        self.clip = clip
        self.idx = torch.empty((3, B), dtype=torch.int32, device=dev)
        self.augment = augment and H == W
        self.rng = np.random.default_rng(seed)
        self.L = L

    def step(self, lr):
        """One training step on a random batch; returns the device loss
        tensor (read it only when needed: reading synchronises)."""
        B, H, W = self.B, self.snaps.H, self.snaps.W
        L, net = self.L, self.net
        s = _stream()
        pick = self.rng.integers(0, len(self.src), size=B)
        sym = self.rng.integers(0, 8, size=B).astype(np.int32)
        self.idx.copy_(self.torch.from_numpy(np.stack([self.src[pick], self.dst[pick], sym])), non_blocking=False)
        flat = self.snaps.store.view(-1, H, W, NF)
        _ok(L.tel_sur_gather(_p(flat), _p(self.idx[0]), _p(self.idx[1]), _p(self.idx[2]) if self.augment else None,
                             _p(self.scale), _p(self.f32), _p(self.x16), _p(self.tgt), B, H, W, s), "gather")
        out = net.forward(self.x16, B, H, W)
        _ok(L.tel_sur_zero(_p(self.loss), 1, s), "zero")
        _ok(L.tel_sur_loss(_p(out), _p(self.tgt), _p(self.dout), _p(self.loss), _p(self.work), B, H, W, s), "loss")
        net.zero_grad()
        net.backward(self.dout, B, H, W)
        net.adam(lr, clip=self.clip)
        return self.loss

    def train(self, steps, lr=1e-3, lr_min=1e-5, log_every=0):
        hist = []
        for i in range(steps):
            cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * i / max(steps, 1)))
            l = self.step(cur)
            if log_every and (i % log_every == 0 or i == steps - 1):
                hist.append((i, float(l.item())))
        return hist


class Predictor:
    """Surrogate inference for B states of H x W: advance normalised FP32
    fields by k lattice steps per call."""

    def __init__(self, net, B, H, W, scale):
        import torch
        self.net, self.B, self.H, self.W = net, B, H, W
        self.L = net.L
        dev = torch.device("cuda")
        self.scale = torch.from_numpy(np.asarray(scale, dtype=np.float32)).to(dev)
        self.x16 = torch.empty((B, H, W, CIN), dtype=torch.bfloat16, device=dev)
        self.work = torch.zeros(4 * B, dtype=torch.float32, device=dev)
        self.mass = torch.zeros(2 * B, dtype=torch.float64, device=dev)
        self.err = torch.zeros(6 * B, dtype=torch.float64, device=dev)
        self.ident = torch.from_numpy(np.arange(B, dtype=np.int32)).to(dev)
        self.torch = torch

    def load(self, f32):
        """Network input from normalised FP32 fields (via the gather kernel
        with the identity index list)."""
        _ok(self.L.tel_sur_gather(_p(f32), _p(self.ident), None, None, None, None, _p(self.x16), None, self.B,
                                  self.H, self.W, _stream()), "gather")

    def advance(self, f32, f32_next, mass=True):
        """f32_next = surrogate(f32); self.x16 must hold f32's network input
        (load() or the previous advance).  Also writes the next input."""
        plan = self.net.plan(self.B, self.H, self.W)
        out = plan.infer(self.x16)
        self.launches = plan.launches + 2  # the head's sums and the advance kernel
        if mass:
            _ok(self.L.tel_sur_zero(_p(self.mass), 4 * self.B, _stream()), "zero")  # 2B doubles = 4B floats
        _ok(self.L.tel_sur_advance(_p(f32), _p(out), _p(self.scale), _p(f32_next), _p(self.x16),
                                   _p(self.mass) if mass else None, _p(self.work), self.B, self.H, self.W,
                                   _stream()), "advance")

    def capture(self, f32, f32_next):
        """CUDA graph of one advance from f32 into f32_next (network forward,
        head, next input), replayed by replay().  Every kernel has run once
        before capture (shared-memory attributes are set on first launch)."""
        torch = self.torch
        self.advance(f32, f32_next, mass=False)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.advance(f32, f32_next, mass=False)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def errors(self, pred, ref):
        """Relative L2 errors (rho, phi, u) per sample, host array [B][3]."""
        _ok(self.L.tel_sur_zero(_p(self.err), 12 * self.B, _stream()), "zero")  # 6B doubles = 12B floats
        _ok(self.L.tel_sur_errors(_p(pred), _p(ref), _p(self.err), self.B, self.H, self.W, _stream()), "errors")
        e = self.err.cpu().numpy().reshape(self.B, 3, 2)
        return np.sqrt(e[:, :, 0] / np.maximum(e[:, :, 1], 1e-300))


class Hybrid:
    """Surrogate time stepping with the lattice update as fallback and judge.

    ``advance()`` moves B states (normalised FP32 fields [B][H][W][4]) by k
    lattice steps.  The surrogate's proposal is accepted unless
      * its mass residual |sum(next) - sum(prev)| / (H W) for density or
        composition exceeds ``mass_tol`` in any sample, or
      * on every ``check_every``-th advance, its relative L2 error against
        the lattice update from the same fields exceeds ``err_tol`` for
        density or composition in any sample;
    a rejected advance is replaced by the lattice update's result, and after
    a failed error check the remaining advances use the lattice update only,
    continuing from its own populations.
    """

    def __init__(self, net, params, H, W, k, scale, mass_tol=1e-4, err_tol=1e-2, check_every=4):
        import torch
        self.torch = torch
        self.B, self.H, self.W, self.k = len(params), H, W, k
        self.pred = Predictor(net, self.B, H, W, scale)
        self.lbm = Batch([(W, H)] * self.B, params)
        self.L = net.L
        dev = torch.device("cuda")
        self.norm_host = np.array([[1.0 / coex_rho_l(p), 1.0 / p["chi"], 1.0 / U_REF] for p in params],
                                  dtype=np.float32)
        self.norm = torch.from_numpy(self.norm_host).to(dev)
        N = H * W
        self.rho = torch.empty((self.B, N), dtype=torch.float64, device=dev)
        self.phi = torch.empty((self.B, N), dtype=torch.float64, device=dev)
        self.u = torch.empty((self.B, 2, N), dtype=torch.float64, device=dev)
        self.prop = torch.empty((self.B, H, W, NF), dtype=torch.float32, device=dev)
        self.ref = torch.empty_like(self.prop)
        self.sums = torch.zeros(2 * self.B, dtype=torch.float64, device=dev)
        self.mass_tol, self.err_tol, self.check_every = mass_tol, err_tol, check_every
        self.n = 0
        self.lbm_only = False
        self.lbm_live = False
        self.log = []
        self.failed = np.zeros(self.B, dtype=bool)

    def lattice_advance(self, f32, out, restart=True):
        """out = the lattice update's k steps from the fields f32 (restart:
        the populations restart at their equilibrium for those fields), or
        from the lattice's own populations left by its previous advance
        (restart=False, when f32 is that advance's result).  Returns a
        boolean mask of the cases whose lattice stayed stable; a flagged
        case's output is not a lattice result."""
        L, B, H, W = self.L, self.B, self.H, self.W
        if restart:
            _ok(L.tel_sur_unpack(_p(f32), _p(self.norm), _p(self.rho), _p(self.phi), _p(self.u), B, H, W,
                                 _stream()), "unpack")
            # the batch works on its own stream: the fields stay on the
            # device, and only the two stream hand-overs wait on the host
            self.torch.cuda.current_stream().synchronize()
            for c in range(B):
                self.lbm.init_device(c, self.rho[c], self.phi[c], self.u[c])
        self.lbm.step(self.k)
        for c in range(B):
            self.lbm.fields_device(c, self.rho[c], self.phi[c], self.u[c])
        ok = np.array(self.lbm.errors()) == 0  # synchronises and clears the flags
        _ok(L.tel_sur_pack(_p(self.rho), _p(self.phi), _p(self.u), _p(self.norm), _p(out), None, B, H, W,
                           _stream()), "pack")
        return ok

    def _take(self, f32, src, ok):
        """f32[c] = src[c] for the cases in ok (the others keep f32)."""
        if ok.all():
            f32.copy_(src)
        else:
            # one contiguous copy per case: no index tensor, no host upload
            for c in np.nonzero(ok)[0]:
                f32[c].copy_(src[c])

    def advance(self, f32):
        """Advance f32 in place by k steps; returns which path produced it.
        A case whose restarted lattice flags an unstable node has no judge:
        it keeps the surrogate's proposal and is marked in ``failed``."""
        B, HW = self.B, self.H * self.W
        self.n += 1
        if self.lbm_only:
            # the lattice continues from its own populations (no restart)
            ok = self.lattice_advance(f32, self.ref, restart=not self.lbm_live)
            self.lbm_live = True
            self.failed |= ~ok
            self._take(f32, self.ref, ok)
            self.log.append("lattice")
            return "lattice"
        _ok(self.L.tel_sur_sums(_p(f32), _p(self.sums), B, self.H, self.W, _stream()), "sums")
        before = self.sums.cpu().numpy().reshape(B, 2)
        self.pred.load(f32)
        self.pred.advance(f32, self.prop)
        after = self.pred.mass.cpu().numpy().reshape(B, 2)
        resid = np.abs(after - before) / HW
        path = "surrogate"
        if np.any(resid > self.mass_tol):
            ok = self.lattice_advance(f32, self.ref)
            self.failed |= ~ok
            f32.copy_(self.prop)
            self._take(f32, self.ref, ok)
            path = "lattice (mass residual)"
        elif self.check_every and self.n % self.check_every == 0:
            ok = self.lattice_advance(f32, self.ref)
            self.failed |= ~ok
            err = self.pred.errors(self.prop, self.ref)
            if np.any(err[ok, :2] > self.err_tol):
                f32.copy_(self.prop)
                self._take(f32, self.ref, ok)
                self.lbm_only = True
                self.lbm_live = bool(ok.all())  # the lattice's populations hold f32's state
                path = "lattice (error check failed)"
            else:
                f32.copy_(self.prop)
                path = "surrogate (checked)"
        else:
            f32.copy_(self.prop)
        self.log.append(path)
        return path


def _main():
    """Timing driver: python -m paper_1710_07486_gb300.surrogate
    [--batch B] [--size H] [--advances N] [--conv mma|tc] [--layers].
    Builds the 581k-parameter network with seeded weights (kernel time does
    not depend on their values), makes N advances of B states of H x H and
    prints one JSON line; --layers times every convolution shape of the
    network with both kernels instead."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--advances", type=int, default=3)
    ap.add_argument("--conv", default="auto", choices=["mma", "tc", "auto"])
    ap.add_argument("--layers", action="store_true")
    a = ap.parse_args()
    B, H = a.batch, a.size
    if a.layers:
        L = sur_lib()
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        out = []
        for ci, co, h in [(CIN, 32, H), (32, 32, H), (32, 64, H // 2), (64, 64, H // 2), (64, 128, H // 4),
                          (128, 128, H // 4), (128, 64, H // 2), (64, 32, H), (32, COUT, H)]:
            x = torch.randn((B, h, h, ci), device="cuda").to(torch.bfloat16)
            w = (torch.randn((9, co, ci), device="cuda") * 0.05).to(torch.bfloat16)
            b = torch.zeros(co, device="cuda")
            y = torch.empty((B, h, h, co), dtype=torch.bfloat16, device="cuda")
            rec = {"cin": ci, "cout": co, "hw": h}
            for name in ("mma", "tc"):
                def run():
                    if name == "tc":
                        return L.tel_sur_conv3x3_tc(_p(x), _p(w), _p(b), _p(y), B, h, h, ci, co, 1, _p(err), _stream())
                    return L.tel_sur_conv3x3(_p(x), _p(w), _p(b), _p(y), B, h, h, ci, co, 1, _stream())
                for _ in range(3):
                    _ok(run(), name)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(20):
                    run()
                e1.record()
                e1.synchronize()
                us = 1e3 * e0.elapsed_time(e1) / 20
                rec[name + "_us"] = round(us, 2)
                rec[name + "_tflops"] = round(2.0 * 9 * ci * co * B * h * h / (us * 1e-6) / 1e12, 1)
            rec["timeout"] = int(err.item())
            out.append(rec)
        print(json.dumps({"batch": B, "size": H, "layers": out}))
        return
    net = Net((32, 64, 128), seed=0, conv=a.conv)
    pr = Predictor(net, B, H, H, np.full(4, 0.01, np.float32))
    f = torch.zeros((B, H, H, NF), dtype=torch.float32, device="cuda")
    f[..., 0] = 1.0
    nxt = torch.empty_like(f)
    pr.load(f)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.advances):
        pr.advance(f, nxt, mass=False)
    e1.record()
    e1.synchronize()
    print(json.dumps({"batch": B, "size": H, "conv": a.conv, "advances": a.advances,
                      "ms_per_advance": round(e0.elapsed_time(e1) / max(a.advances, 1), 4),
                      "timeout": int(net.tc_err.item())}))


if __name__ == "__main__":
    _main()
