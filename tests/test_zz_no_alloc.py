"""tel_fields_noalloc: field extraction for callers that cannot let the
library allocate device memory (the whole device belongs to their own pool,
or their device footprint must stay fixed).  The state sits in the caller's
buffers; the library stages the result through a fixed device array.

Checked through the C ABI against tel_fields of a context holding the same
state, on two calls in a row, with the parity tolerances of the other GPU
tests (FP64 1e-12, FP32 storage 1e-4).  This file is collected last so that a
run stopping at the first failure has run everything else first.
"""
import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, base

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lattice,shape,precision,tol,with_p,bc", [
    (tel.D2Q9, (64, 48, 1), tel.FP64, 1e-12, True, (0, 0, 0)),
    (tel.D3Q27, (20, 16, 12), tel.FP32_SHIFTED, 1e-4, True, (0, 0, 0)),
    # no pressure output, bounce-back walls on one axis (the walled pull path)
    (tel.D2Q9, (40, 36, 1), tel.FP64, 1e-12, False, (0, 1, 0)),
    (tel.D3Q27, (16, 20, 12), tel.FP32_SHIFTED, 1e-4, False, (1, 0, 0)),
])
def test_fields_noalloc_matches_context(lattice, shape, precision, tol, with_p, bc):
    torch = pytest.importorskip("torch")
    T = tel.temperature_for_ratio(A, B, RGAS, 10.0)
    p = dict(base(T), precision=precision, bc=bc)
    nx, ny, nz = shape
    lat = tel.Lattice(lattice, nx, ny, nz, p)
    D = lat.D
    dims = (nx, ny) if D == 2 else (nx, ny, nz)
    c = [v / 2.0 for v in dims]
    rho, phi, u = inputs.drops(dims, lat.rho_g, lat.rho_l, p["chi"],
                               [dict(center=[v - 4 for v in c], R=min(dims) / 5, kind=1, u=[0.02] * D),
                                dict(center=[v + 4 for v in c], R=min(dims) / 6, kind=-1)], width=4.0)
    lat.init(rho, phi, u)
    w = np.array([tel_w(lattice, i) for i in range(lat.Q)])
    shift = lat.rho_g if precision == tel.FP32_SHIFTED else 0.0
    for call in range(2):
        lat.step(3 + call)
        ref = lat.fields(with_p=with_p)
        f, g = lat.get_state()
        if precision == tel.FP64:
            fd = torch.tensor(f, dtype=torch.float64, device="cuda")
            gd = torch.tensor(g, dtype=torch.float64, device="cuda")
        else:
            fd = torch.tensor(f - w[:, None] * shift, dtype=torch.float32, device="cuda")
            gd = torch.tensor(g, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        got = tel.fields_noalloc(lattice, nx, ny, nz, p, fd, gd, with_p=with_p)
        if not with_p:
            assert got["p"] is None
        for k in ("rho", "phi", "u") + (("p",) if with_p else ()):
            scale = max(np.abs(ref[k]).max(), 1e-3)
            assert np.max(np.abs(got[k] - ref[k])) / scale < tol, (call, k)


def test_fields_noalloc_rejects_lattices_beyond_the_fixed_scratch():
    T = tel.temperature_for_ratio(A, B, RGAS, 10.0)
    n = 1 + int(np.sqrt(tel.NOALLOC_MAX_NODES))
    with pytest.raises(tel.TelError) as ei:
        tel.fields_noalloc(tel.D2Q9, n, n, 1, base(T), 1, 1)
    assert ei.value.code == tel.TEL_EINVAL
    assert "scratch" in str(ei.value)


def tel_w(lattice, i):
    """Lattice weight of velocity i in the library's ordering (ABI header)."""
    c = [i % 3 - 1, (i // 3) % 3 - 1] + ([i // 9 - 1] if lattice == tel.D3Q27 else [])
    w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
    return float(np.prod([w1[v] for v in c]))


def test_fields_noalloc_reports_a_flagged_node_then_recovers():
    """A state whose density is zero everywhere makes the fields kernel raise
    its error word (non-positive density): the call returns TEL_EUNSTABLE.
    The next call clears the shared error word and succeeds."""
    torch = pytest.importorskip("torch")
    T = tel.temperature_for_ratio(A, B, RGAS, 10.0)
    p = base(T)
    nx, ny = 16, 12
    zeros = torch.zeros(9 * nx * ny, dtype=torch.float64, device="cuda")
    with pytest.raises(tel.TelError) as ei:
        tel.fields_noalloc(tel.D2Q9, nx, ny, 1, p, zeros, zeros, with_p=False)
    assert ei.value.code == tel.TEL_EUNSTABLE
    lat = tel.Lattice(tel.D2Q9, nx, ny, 1, p)
    rho, phi, u = inputs.drops((nx, ny), lat.rho_g, lat.rho_l, p["chi"],
                               [dict(center=(8.0, 6.0), R=4.0, kind=1)], width=4.0)
    lat.init(rho, phi, u)
    f, g = lat.get_state()
    fd = torch.tensor(f, dtype=torch.float64, device="cuda")
    gd = torch.tensor(g, dtype=torch.float64, device="cuda")
    got = tel.fields_noalloc(tel.D2Q9, nx, ny, 1, p, fd, gd, with_p=False)
    ref = lat.fields(with_p=False)
    assert np.max(np.abs(got["rho"] - ref["rho"])) / lat.rho_l < 1e-12
