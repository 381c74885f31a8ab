"""Layer-by-layer ("teacher-forced") check of the surrogate network's wiring.

The whole-network comparison with the oracle cannot be tight: BF16 storage
of activations turns the network into a chaotic map of rounding decisions,
so two correct implementations differ by percents after a dozen layers.
Here every operation is instead fed the values the implementation under
test actually stored for its inputs, as the oracle's op list says they flow
(which activation enters which convolution, which saved tensor a skip adds,
which gradient reaches which buffer), and its stored output is compared with
the oracle's operation applied to those inputs.  Each comparison then sees
one rounding only, so a wiring mistake of a few percent anywhere (a wrong
skip slot, a scaled skip, a missing ReLU mask, a transposed weight, a
gradient routed to the wrong buffer) fails it.

Records (host float64 arrays, aligned with ``oracle.surrogate.arch``):
  fwd[i]: output of op i (conv, pool, up, add); None for 'save'.
  bwd[i]: dict per op --
    conv: {"dz": dL/dz, "dx": dL/dinput (None for the first conv),
           "dW": [9][cin][cout], "db": [cout]}
    pool, up, save: {"dx": gradient passed on}
    add: {}  (the gradient is shared by both operands)
"""
import numpy as np

from oracle import surrogate as so

ULP_REL = 2.0 ** -7     # one BF16 ulp at most, relative to the value: a rounding flipped by FP32 sums
FLOOR_REL = 2.0 ** -14  # absolute floor, relative to the tensor's scale (FP32 sums)
FP32_REL = 1e-4         # FP32 accumulations (weight and bias gradients), norm


def to_bf16(a):
    """Round to the nearest BF16 value, ties to even (finite inputs), through
    FP32 as the kernels store: keep the upper 16 bits of the FP32 pattern
    after adding half of the dropped range plus the kept part's lowest bit."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_misfit(got, ref):
    """Largest |got - ref| in units of the tolerance of one BF16 rounding
    of a value accumulated in FP32: <= 1 when every element agrees."""
    scale = max(float(np.abs(ref).max()), 1e-30)
    tol = ULP_REL * np.abs(ref) + FLOOR_REL * scale
    return float(np.max(np.abs(got - ref) / tol))


def rel_norm(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))


def check(ops, Ws, bs, x, dout, fwd, bwd, rnd):
    """Per-op misfits [(i, what, value)] of the records against the oracle
    operations applied to the recorded inputs.  BF16 outputs: misfit <= 1;
    FP32 weight and bias gradients: relative norm error <= FP32_REL."""
    out = []
    a, saved = x, {}
    inputs = []
    for i, op in enumerate(ops):
        kind = op[0]
        inputs.append(a)
        if kind == "conv":
            _, k, ci, co, relu = op
            out.append((i, "conv%d fwd" % k, bf16_misfit(fwd[i], rnd(so.conv_fwd(a, Ws[k], bs[k], relu)))))
            a = fwd[i]
        elif kind == "pool":
            out.append((i, "pool fwd", bf16_misfit(fwd[i], rnd(so.pool_fwd(a)))))
            a = fwd[i]
        elif kind == "up":
            out.append((i, "up fwd", bf16_misfit(fwd[i], so.up_fwd(a))))
            a = fwd[i]
        elif kind == "save":
            saved[op[1]] = a
        elif kind == "add":
            out.append((i, "add fwd", bf16_misfit(fwd[i], rnd(a + saved[op[1]]))))
            a = fwd[i]
    d, gsaved = dout, {}
    for i in reversed(range(len(ops))):
        op = ops[i]
        kind = op[0]
        r = bwd[i]
        if kind == "conv":
            _, k, ci, co, relu = op
            dz = d * (fwd[i] > 0) if relu else d
            out.append((i, "conv%d relu mask" % k, bf16_misfit(r["dz"], dz)))
            dx, dW, db = so.conv_bwd(inputs[i], Ws[k], fwd[i], d, relu)
            out.append((i, "conv%d dW" % k, rel_norm(r["dW"], dW) / FP32_REL))
            out.append((i, "conv%d db" % k, rel_norm(r["db"], db) / FP32_REL))
            if r["dx"] is not None:
                # the input gradient is computed from the stored dz
                dx_z, _, _ = so.conv_bwd(inputs[i], Ws[k], fwd[i], r["dz"], False)
                out.append((i, "conv%d dx" % k, bf16_misfit(r["dx"], rnd(dx_z))))
                d = r["dx"]
        elif kind == "pool":
            out.append((i, "pool bwd", bf16_misfit(r["dx"], rnd(so.pool_bwd(d)))))
            d = r["dx"]
        elif kind == "up":
            out.append((i, "up bwd", bf16_misfit(r["dx"], rnd(so.up_bwd(d)))))
            d = r["dx"]
        elif kind == "add":
            gsaved[op[1]] = d
        elif kind == "save":
            out.append((i, "skip gradient", bf16_misfit(r["dx"], rnd(d + gsaved.pop(op[1])))))
            d = r["dx"]
    return out


def oracle_records(ops, Ws, bs, x, dout, rnd, plant=None):
    """Records produced by the oracle's own operations with BF16 storage
    (``rnd``), walking ``ops`` as an implementation would.  ``plant`` names a
    mistake to build in, so that a test can show that ``check`` catches it:
    'skip_scale' (one skip added at 0.97), 'skip_source' (the deep skip
    saves the activation one convolution too early), 'relu_mask' (one ReLU mask dropped in the
    backward pass), 'weight_flip' (one input gradient from the untransposed
    kernel), 'wgrad_tap' (two taps of one weight gradient swapped),
    'pool_scale' (pooling adjoint without the 1/4)."""
    fwd, bwd = [None] * len(ops), [None] * len(ops)
    a, saved = x, {}
    inputs = []
    slots = [op[1] for op in ops if op[0] == "save"]
    last_save = max(i for i, op in enumerate(ops) if op[0] == "save")
    for i, op in enumerate(ops):
        kind = op[0]
        inputs.append(a)
        if kind == "conv":
            _, k, ci, co, relu = op
            fwd[i] = rnd(so.conv_fwd(a, Ws[k], bs[k], relu))
        elif kind == "pool":
            fwd[i] = rnd(so.pool_fwd(a))
        elif kind == "up":
            fwd[i] = so.up_fwd(a)
        elif kind == "save":
            saved[op[1]] = inputs[i - 1] if (plant == "skip_source" and i == last_save) else a
        elif kind == "add":
            s = saved[op[1]]
            if plant == "skip_scale" and op[1] == slots[0]:
                s = 0.97 * s
            fwd[i] = rnd(a + s)
        if fwd[i] is not None:
            a = fwd[i]
    d, gsaved = dout, {}
    first_relu = next(i for i, op in enumerate(ops) if op[0] == "conv" and op[4])
    mid_conv = [i for i, op in enumerate(ops) if op[0] == "conv"][len(Ws) // 2]
    for i in reversed(range(len(ops))):
        op = ops[i]
        kind = op[0]
        if kind == "conv":
            _, k, ci, co, relu = op
            mask = relu and not (plant == "relu_mask" and i == first_relu + 1)
            dz = rnd(d * (fwd[i] > 0)) if mask else d
            dx, dW, db = so.conv_bwd(inputs[i], Ws[k], fwd[i], dz, False)
            if plant == "weight_flip" and i == mid_conv:
                Wt = Ws[k][::-1]  # taps reversed: the flip's transpose left out
                dx, _, _ = so.conv_bwd(inputs[i], Wt, fwd[i], dz, False)
            if plant == "wgrad_tap" and i == mid_conv:
                dW = dW.copy()
                dW[[0, 1]] = dW[[1, 0]]
            r = {"dz": dz, "dW": dW, "db": db, "dx": None}
            if k > 0:
                r["dx"] = rnd(dx)
                d = r["dx"]
            bwd[i] = r
        elif kind == "pool":
            dx = so.pool_bwd(d) * (4.0 if plant == "pool_scale" else 1.0)
            bwd[i] = {"dx": rnd(dx)}
            d = bwd[i]["dx"]
        elif kind == "up":
            bwd[i] = {"dx": rnd(so.up_bwd(d))}
            d = bwd[i]["dx"]
        elif kind == "add":
            bwd[i] = {}
            gsaved[op[1]] = d
        elif kind == "save":
            bwd[i] = {"dx": rnd(d + gsaved.pop(op[1]))}
            d = bwd[i]["dx"]
    return fwd, bwd
