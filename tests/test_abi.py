"""The C ABI: the library builds for sm_103a, loads, exports every entry point
that include/ternelbm.h declares, and its host-only logic (parameter
validation, common-tangent solver) behaves without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1710_07486_gb300 as tel
from tests.cases import A, B, RGAS, base

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tel_[a-z_0-9]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    L = tel.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(tel.SYMBOLS) <= names


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(tel, "_lib", None)
    monkeypatch.setattr(tel, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        tel.lib(build=False)


@pytest.mark.parametrize("ratio", [3.0, 10.0, 150.0, 1000.0])
def test_library_coexistence_matches_oracle(orc, ratio):
    T = tel.temperature_for_ratio(A, B, RGAS, ratio)
    To = orc.temperature_for_ratio(A, B, RGAS, ratio)
    assert T == pytest.approx(To, rel=1e-10)
    got = tel.coexistence(A, B, RGAS, To)
    ref = orc.coexistence(A, B, RGAS, To)
    assert got[0] == pytest.approx(ref[0], rel=1e-11)
    assert got[1] == pytest.approx(ref[1], rel=1e-12)
    assert got[2] == pytest.approx(ref[2], rel=1e-11, abs=1e-13)
    assert got[3] == pytest.approx(ref[3], rel=1e-10, abs=1e-15)


def test_invalid_parameters_rejected_before_any_device_work():
    T = tel.temperature_for_ratio(A, B, RGAS, 10.0)
    good = base(T)
    bad_cases = [
        (0, 3, 8, 1, good),                     # extent < 4
        (0, 8, 8, 2, good),                     # nz != 1 for D2Q9
        (2, 8, 8, 8, good),                     # bad lattice
        (0, 8, 8, 1, dict(good, nu=0.0)),       # tau = 1/2
        (0, 8, 8, 1, dict(good, tau_g=0.5)),
        (0, 8, 8, 1, dict(good, chi=0.0)),
        (0, 8, 8, 1, dict(good, kappa2=-1.0)),
        (0, 8, 8, 1, dict(good, T=1.0)),        # above T_c: no coexistence
        (0, 8, 8, 1, dict(good, precision=7)),
        (0, 8, 8, 1, dict(good, force_form=3)),
        (0, 8, 8, 1, dict(good, bc=(0, 2, 0))),
        (0, 8, 8, 1, dict(good, bc=(0, 1, 0), wet_rho=float("nan"))),
        (0, 8, 8, 1, dict(good, bc=(0, 1, 0), wet_phi=float("inf"))),
        (1, 32, 8, 8, dict(good, moments=2)),   # bad moments mode
    ]
    for lat, nx, ny, nz, p in bad_cases:
        with pytest.raises(tel.TelError) as ei:
            tel.Lattice(lat, nx, ny, nz, p)
        assert ei.value.code == tel.TEL_EINVAL, (lat, nx, ny, nz, p)
    with pytest.raises(tel.TelError):
        tel.coexistence(A, B, RGAS, 1.0)


def test_batch_create_validates_on_the_host():
    """Bad batch arguments are rejected before any device call."""
    T = tel.temperature_for_ratio(A, B, RGAS, 10.0)
    p = base(T)
    with pytest.raises(tel.TelError) as ei:
        tel.Batch([(16, 16), (16, 16)], [p, dict(p, precision=tel.FP32_SHIFTED)])
    assert ei.value.code == tel.TEL_EINVAL and "precision" in str(ei.value)
    with pytest.raises(tel.TelError) as ei:
        tel.Batch([(16, 16), (2, 16)], p)
    assert ei.value.code == tel.TEL_EINVAL and "case 1" in str(ei.value)
    with pytest.raises(tel.TelError) as ei:
        tel.Batch([(16, 16)], dict(p, nu=-0.1))
    assert ei.value.code == tel.TEL_EINVAL
    with pytest.raises(ValueError):
        tel.Batch([(16, 16), (16, 16)], [p])
    L = tel.lib()
    assert L.tel_batch_create(0, None, None, None, C.byref(C.c_void_p())) == tel.TEL_EINVAL


@pytest.mark.parametrize("eos,a,b,omega", [(1, 9.0 / 49.0, 2.0 / 21.0, 0.0), (2, 2.0 / 49.0, 2.0 / 21.0, 0.344)])
@pytest.mark.parametrize("ratio", [10.0, 100.0, 1000.0])
def test_library_coexistence_matches_oracle_other_eos(orc, eos, a, b, omega, ratio):
    """The library's host solver (bisection on mu + Newton) against the
    oracle's (bisection on the saturation pressure) for the van der Waals and
    Peng-Robinson equations of state."""
    T = tel.temperature_for_ratio(a, b, RGAS, ratio, eos=eos, omega=omega)
    To = orc.eos_temperature_for_ratio(eos, a, b, RGAS, ratio, omega)
    assert T == pytest.approx(To, rel=1e-10)
    got = tel.coexistence(a, b, RGAS, To, eos=eos, omega=omega)
    ref = orc.eos_coexistence(eos, a, b, RGAS, To, omega)
    assert got[0] == pytest.approx(ref[0], rel=1e-11)
    assert got[1] == pytest.approx(ref[1], rel=1e-11)
    assert got[2] == pytest.approx(ref[2], rel=1e-10, abs=1e-13)
    assert got[3] == pytest.approx(ref[3], rel=1e-9)
