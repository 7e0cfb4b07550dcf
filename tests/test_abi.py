"""CPU-side checks of the C ABI: the library loads, exports every declared
symbol, and its host-only calls (validation, coefficients, scratch sizing,
status names) behave as include/fllf.h states.  No kernel runs here."""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return pkg.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(fllf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "fllf_run" in names and "fllf_plan_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_names(lib):
    assert lib.fllf_status_str(0) == b"FLLF_OK"
    assert lib.fllf_status_str(1) == b"FLLF_EINVAL"
    assert lib.fllf_status_str(6) == b"FLLF_EBUSY"


@pytest.mark.parametrize("m,sigma,T,K", [(3.0, 0.1, 2.0, 4), (3.0, 0.2, 2.0, 8),
                                         (0.5, 0.4, 2.0, 16), (4.0, 0.05, 2.0, 64),
                                         (7.0, 30.0, 405.9, 10)])
def test_host_coefficients_match_oracle(lib, m, sigma, T, K):
    p = pkg.make_params(64, 64, 1, 4, K, m, sigma, T)
    got = np.array(pkg.fllf_coeffs(p))
    np.testing.assert_allclose(got, o.coeffs_quadrature(m, sigma, T, K), rtol=0,
                               atol=1e-12 * max(1.0, abs(m - 1) * sigma))
    p.coeff_mode = pkg.FLLF_COEFF_CLOSED_FORM
    got = np.array(pkg.fllf_coeffs(p))
    np.testing.assert_allclose(got, o.coeffs_closed_form(m, sigma, T, K), rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("field,value", [("H", 0), ("W", -3), ("C", 0), ("C", 65), ("levels", 0),
                                         ("levels", 17), ("K", 0), ("K", 65), ("sigma_r", 0.0),
                                         ("T", -1.0), ("m", float("nan")), ("precision", 3),
                                         ("coeff_mode", 2)])
def test_invalid_params_rejected(lib, field, value):
    p = pkg.make_params(32, 32, 1, 4, 4)
    setattr(p, field, value)
    assert pkg.fllf_params_validate(p) == pkg.FLLF_EINVAL
    assert pkg.fllf_plan_scratch_bytes(p) == 0
    assert lib.fllf_last_error() != b""
    with pytest.raises(pkg.FllfError) as e:
        pkg.fllf_coeffs(p)
    assert e.value.status == pkg.FLLF_EINVAL


def test_scratch_bytes_formula(lib):
    # G (float), Z (K complex) per level l >= 1, E for 1 <= l <= levels-2,
    # pitch rounded to 16 elements, each buffer 256-byte aligned.
    def expect(H, W, C, L, K, zbytes):
        total, h, w = 0, H, W
        a = lambda x: (x + 255) // 256 * 256
        for l in range(L):
            if l > 0:
                pitch = (w + 15) // 16 * 16
                g = a(4 * h * pitch * C)
                total += g + a(zbytes * K * h * pitch * C) + (g if l <= L - 2 else 0)
            h, w = (h + 1) // 2, (w + 1) // 2
        return total
    for prec, zb in (("fp32", 8), ("fp16", 4), ("bf16", 4)):
        p = pkg.make_params(2160, 3840, 3, 8, 8, precision=prec)
        assert pkg.fllf_plan_scratch_bytes(p) == expect(2160, 3840, 3, 8, 8, zb)
    p = pkg.make_params(7, 5, 1, 1, 3)
    assert pkg.fllf_plan_scratch_bytes(p) == 0


def test_null_arguments_rejected(lib):
    assert lib.fllf_plan_destroy(None) == pkg.FLLF_OK
    assert lib.fllf_run(None, None, None, None) == pkg.FLLF_EINVAL
    assert lib.fllf_poll(ctypes.c_uint64(123456789), 0) == pkg.FLLF_EINVAL


def _golden_periods():
    path = os.path.join(ROOT, "tests", "golden", "period_sigma30.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return [(float(s), int(k), float(r), float(t)) for s, k, r, t in rows]


@pytest.mark.parametrize("sigma,K,R,T_paper", _golden_periods())
def test_optimal_period_matches_paper(lib, sigma, K, R, T_paper):
    # Eq. (12) at the paper's experimental setting; it prints T = 405.9
    T = pkg.fllf_optimal_period(sigma, K, R)
    assert abs(T - T_paper) / T_paper < 2e-3


@pytest.mark.parametrize("sigma,K,R", [(30.0, 10, 256.0), (0.2, 8, 1.0), (0.1, 4, 1.0),
                                       (0.4, 16, 1.0), (15.0, 10, 256.0), (0.05, 64, 1.0)])
def test_optimal_period_matches_oracle(lib, sigma, K, R):
    T = pkg.fllf_optimal_period(sigma, K, R)
    T_ref = o.optimal_period(sigma, K, R)
    assert abs(T - T_ref) <= 1e-6 * T_ref
    # it is a minimum of E_K(T): both neighbours are no lower
    e = o.period_error(T, sigma, K, R)
    for d in (1e-3, -1e-3):
        assert o.period_error(T * (1 + d), sigma, K, R) >= e - 1e-15


def test_optimal_period_rejects_bad_arguments(lib):
    for args in ((0.0, 8, 1.0), (-1.0, 8, 1.0), (0.2, 0, 1.0), (0.2, 65, 1.0), (0.2, 8, 0.0),
                 (float("nan"), 8, 1.0), (0.2, 8, float("inf"))):
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_optimal_period(*args)
        assert e.value.status == pkg.FLLF_EINVAL


def test_fast_params_validation_and_layout(lib):
    # fast LLF (Sec. II-D): S samples held as ceil(S/2) complex planes; K, T and
    # coeff_mode are not used
    p = pkg.make_fast_params(2160, 3840, 3, 8, samples=16)
    p.K, p.T, p.coeff_mode = 0, -1.0, 7
    assert pkg.fllf_params_validate(p) == pkg.FLLF_OK
    q = pkg.make_params(2160, 3840, 3, 8, 8)
    assert pkg.fllf_plan_scratch_bytes(p) == pkg.fllf_plan_scratch_bytes(q)
    p.samples = 15   # odd: the last plane's second half is unused
    assert pkg.fllf_plan_scratch_bytes(p) == pkg.fllf_plan_scratch_bytes(q)
    for s in (0, 1, 129):
        p.samples = s
        assert pkg.fllf_params_validate(p) == pkg.FLLF_EINVAL
    p.samples = 8
    p.method = 2
    assert pkg.fllf_params_validate(p) == pkg.FLLF_EINVAL
    p.method = pkg.FLLF_METHOD_FAST
    p.sigma_r = 0.0
    assert pkg.fllf_params_validate(p) == pkg.FLLF_EINVAL
    p.sigma_r = 0.2
    with pytest.raises(pkg.FllfError) as e:
        pkg.fllf_coeffs(p)   # no Fourier coefficients
    assert e.value.status == pkg.FLLF_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of the header's structs: size and every field offset
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"fllf_params": pkg.fllf_params, "fllf_tuning": pkg.fllf_tuning,
               "fllf_server_stats": pkg.fllf_server_stats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fllf.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, key, val = line.split()
        got[(name, key)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
