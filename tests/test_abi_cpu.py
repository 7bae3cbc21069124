"""The C-ABI library on a machine without a GPU: it loads, exports every
symbol the header declares, validates arguments before touching a device,
and its planner's split and FP32 twiddle tables are exact roundings of the
FP64 values."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2006_08435_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FUSED = [16, 32, 48, 64, 80, 96, 128]


def header_functions():
    src = open(os.path.join(ROOT, "include", "fft3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fft3d_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(fft3d_lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(fft3d_lib, n), n
    assert sorted(L.exported_symbols()) == names


def test_error_strings(fft3d_lib):
    for code in range(0, -10, -1):
        s = fft3d_lib.fft3d_error_string(code).decode()
        assert s and s != "unknown error code"
    assert fft3d_lib.fft3d_error_string(-99).decode() == "unknown error code"


def _create(lib, *args):
    h = ctypes.c_void_p(1234)
    rc = lib.fft3d_plan_create(*args, ctypes.byref(h))
    return rc, h.value


@pytest.mark.parametrize("args,code", [
    ((64, 64, 64, 0, 0, -1, 0), L.FFT3D_ERR_INVALID_ARG),      # batch 0
    ((64, 64, 64, 1, 7, -1, 0), L.FFT3D_ERR_INVALID_ARG),      # precision
    ((48, 48, 48, 1, 5, -1, 0), L.FFT3D_ERR_UNSUPPORTED_PRECISION),  # FP8 at 64, 128 only
    ((64, 64, 64, 1, 0, 0, 0), L.FFT3D_ERR_INVALID_ARG),       # direction
    ((64, 64, 64, 1, 0, -1, 5), L.FFT3D_ERR_INVALID_ARG),      # norm
    ((0, 64, 64, 1, 0, -1, 0), L.FFT3D_ERR_INVALID_ARG),       # zero edge
    ((7, 7, 7, 1, 0, -1, 0), L.FFT3D_ERR_UNSUPPORTED_SIZE),    # prime 7
    ((1024, 1024, 1024, 1, 0, -1, 0), L.FFT3D_ERR_UNSUPPORTED_SIZE),  # above 512
    ((64, 128, 14, 1, 0, -1, 0), L.FFT3D_ERR_UNSUPPORTED_SIZE),  # one edge with a 7
    ((64, 128, 96, 1, 1, -1, 0), L.FFT3D_ERR_UNSUPPORTED_PRECISION),  # general path: FP32
    ((256, 256, 256, 1, 2, -1, 0), L.FFT3D_ERR_UNSUPPORTED_PRECISION),
])
def test_create_validates_before_device(fft3d_lib, args, code):
    rc, h = _create(fft3d_lib, *args)
    assert rc == code
    assert h is None


def test_create_null_out(fft3d_lib):
    assert fft3d_lib.fft3d_plan_create(64, 64, 64, 1, 0, -1, 0, None) == L.FFT3D_ERR_NULL_PTR


def test_mixed_validation(fft3d_lib):
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 3)(32, 48, 7)
    assert fft3d_lib.fft3d_plan_create_mixed(3, dims, 0, -1, 0, ctypes.byref(h)) == L.FFT3D_ERR_UNSUPPORTED_SIZE
    assert fft3d_lib.fft3d_plan_create_mixed(0, dims, 0, -1, 0, ctypes.byref(h)) == L.FFT3D_ERR_INVALID_ARG
    assert fft3d_lib.fft3d_plan_create_mixed(3, None, 0, -1, 0, ctypes.byref(h)) == L.FFT3D_ERR_NULL_PTR


def test_null_handles(fft3d_lib):
    assert fft3d_lib.fft3d_execute(None, 16, 16, None) == L.FFT3D_ERR_NULL_PTR
    assert fft3d_lib.fft3d_plan_destroy(None) == L.FFT3D_SUCCESS
    assert fft3d_lib.fft3d_get_device_status(None, None) == L.FFT3D_ERR_NULL_PTR


def test_valid_args_reach_device_check(fft3d_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    rc, _ = _create(fft3d_lib, 64, 64, 64, 1, 0, -1, 0)
    assert rc == L.FFT3D_ERR_NO_DEVICE


def _smooth(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def test_size_supported(fft3d_lib):
    """Every edge 2..512 whose prime factors are 2, 3, 5, nothing else."""
    for n in FUSED:
        assert fft3d_lib.fft3d_size_supported(n) == 1
    for n in range(-1, 1100):
        want = 2 <= n <= 512 and _smooth(n)
        assert fft3d_lib.fft3d_size_supported(n) == int(want), n


def _digit_map(lib, n):
    ns = ctypes.c_int()
    radix = (ctypes.c_int * 12)()
    pos = (ctypes.c_int * n)()
    rc = lib.fft3d_axis_digit_map(n, ctypes.byref(ns), radix, pos)
    return rc, list(radix)[:ns.value], list(pos)


@pytest.mark.parametrize("n", [2, 3, 5, 6, 12, 16, 45, 96, 100, 128, 243, 250, 256, 375, 384,
                               480, 500, 512])
def test_axis_digit_map_is_the_mixed_radix_reversal(fft3d_lib, n):
    """Bit-exact against the digit reversal written from its definition:
    output K with digits k_t (K = k_0 + R_0 (k_1 + R_1 (...))) sits at
    position sum_t k_t n / (R_0 ... R_t); a bijection; radices multiply to n
    and each has a register codelet."""
    rc, radix, pos = _digit_map(fft3d_lib, n)
    assert rc == L.FFT3D_SUCCESS
    assert int(np.prod(radix)) == n
    assert set(radix) <= {2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16}
    for K in range(n):
        digits, rem = [], K
        for r in radix:
            digits.append(rem % r)
            rem //= r
        p, span = 0, n
        for r, d in zip(radix, digits):
            span //= r
            p += d * span
        assert pos[K] == p
    assert sorted(pos) == list(range(n))


@pytest.mark.parametrize("n", [6, 16, 45, 96, 100, 128, 250, 384, 512])
@pytest.mark.parametrize("sign", [-1, 1])
def test_axis_stages_compute_the_dft(fft3d_lib, n, sign):
    """The stage algorithm the general path's kernel runs (decimation in
    frequency over the library's radices: y_k = sum_r x[j + r M] W_R^(r k)
    times W_N^(j k) to position j + k M), carried out here in FP64 NumPy,
    and read through the library's digit map, is the DFT (numpy.fft)."""
    rc, radix, pos = _digit_map(fft3d_lib, n)
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a = x.copy()
    span = n
    for R in radix:
        M = span // R
        wr = np.exp(sign * 2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
        for blk in range(n // span):
            for j in range(M):
                idx = blk * span + j + M * np.arange(R)
                y = wr.T @ a[idx]
                y *= np.exp(sign * 2j * np.pi * j * np.arange(R) / span)
                a[idx] = y
        span = M
    got = a[np.asarray(pos)]
    want = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_axis_digit_map_rejects(fft3d_lib):
    for n in (0, 1, 7, 14, 1024, 2048):
        rc, _, _ = _digit_map(fft3d_lib, max(n, 1))
        assert rc == L.FFT3D_ERR_UNSUPPORTED_SIZE
    ns = ctypes.c_int()
    assert fft3d_lib.fft3d_axis_digit_map(16, None, None, None) == L.FFT3D_ERR_NULL_PTR


@pytest.mark.parametrize("n", FUSED)
def test_twiddle_tables_are_rounded_fp64(fft3d_lib, n):
    """Each entry is the round-to-nearest FP32 of exp(-2 pi i m / n),
    m = n1*k2 mod n, with the FP64 value taken from Python's math library,
    and the split multiplies back to n with factors of at most 16."""
    buf = (ctypes.c_float * (2 * n))()
    l1, l2 = ctypes.c_int(), ctypes.c_int()
    assert fft3d_lib.fft3d_twiddle_table(n, buf, ctypes.byref(l1), ctypes.byref(l2)) == 0
    assert l1.value * l2.value == n and l1.value <= 16 and l2.value <= 16
    got = np.frombuffer(buf, dtype=np.float32).reshape(l2.value, l1.value, 2)
    for k2 in range(l2.value):
        for n1 in range(l1.value):
            a = 2 * math.pi * ((n1 * k2) % n) / n
            assert got[k2, n1, 0] == np.float32(math.cos(a))
            assert got[k2, n1, 1] == np.float32(-math.sin(a))


def _rn_bits(x: float, bits: int, min_normal_exp: int) -> float:
    """x rounded to nearest (ties to even) with `bits` significant bits and
    a subnormal quantum below 2**min_normal_exp (FP16: 11, -14; BF16: 8,
    -126), written from the definition with frexp."""
    if x == 0.0:
        return 0.0
    m, e = math.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    if e - 1 < min_normal_exp:
        q = 2.0 ** (min_normal_exp - bits + 1)
        return round(x / q) * q
    return round(m * 2.0 ** bits) * 2.0 ** (e - bits)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_tc_operand_table_is_the_twiddled_dft16(fft3d_lib, prec):
    """The tcgen05 B operands: for k1 < 4 the real 2 x 2 form of
    W_64^(n2 (k1 + 4 k2)) at the documented core-matrix positions, hi =
    rn(b) and lo = rn(b - hi) of the FP64 entry b (FP16; BF16 for split
    BF16), and hi + lo reproducing the complex matrix."""
    buf = (ctypes.c_uint16 * 8192)()
    assert fft3d_lib.fft3d_tc_operand_table(prec, buf) == 0
    raw = np.frombuffer(buf, dtype=np.uint16)
    bf16 = prec == 2
    bits, emin = (8, -126) if bf16 else (11, -14)

    def dec(u):
        if bf16:
            return float(np.array([int(u) << 16], dtype=np.uint32).view(np.float32)[0])
        return float(np.array([u], dtype=np.uint16).view(np.float16)[0])

    for k1 in range(4):
        m_rec = np.zeros((16, 16), np.complex128)
        for nn in range(32):
            for kk in range(32):
                k2, d, n2, c = nn // 2, nn % 2, kk // 2, kk % 2
                a = -2.0 * math.pi * ((n2 * (k1 + 4 * k2)) % 64) / 64.0
                wr, wi = math.cos(a), math.sin(a)
                b = (wr if d == 0 else wi) if c == 0 else (-wi if d == 0 else wr)
                off = ((nn // 8) * 4 + kk // 8) * 128 + (nn % 8) * 16 + (kk % 8) * 2
                hi = dec(raw[(0 * 4 + k1) * 1024 + off // 2])
                lo = dec(raw[(1 * 4 + k1) * 1024 + off // 2])
                assert hi == _rn_bits(b, bits, emin)
                assert lo == _rn_bits(b - hi, bits, emin)
                if c == 0:
                    if d == 0:
                        m_rec[n2, k2] += hi + lo
                    else:
                        m_rec[n2, k2] += 1j * (hi + lo)
        n2g, k2g = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
        expect = np.exp(-2j * np.pi * n2g * (k1 + 4 * k2g) / 64)
        assert np.abs(m_rec - expect).max() < (2.0 ** -15 if bf16 else 2.0 ** -20)


def test_tc_operand_table_errors(fft3d_lib):
    buf = (ctypes.c_uint16 * 8192)()
    assert fft3d_lib.fft3d_tc_operand_table(1, None) == L.FFT3D_ERR_NULL_PTR
    for bad in (0, 7, -1):
        assert fft3d_lib.fft3d_tc_operand_table(bad, buf) == L.FFT3D_ERR_INVALID_ARG


def _e4m3_values():
    """Every finite E4M3 value by code (1 sign, 4 exponent bits with bias 7,
    3 mantissa bits; exponent field 0 is subnormal, 2^-6 m / 8; the all-ones
    code is NaN, so the largest finite value is 2^8 * 1.75 = 448)."""
    vals = {}
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
        vals[code] = -v if s else v
    return vals


def _e4m3_rn(x, vals):
    """Round to nearest E4M3, ties to the even code, saturating at +-448."""
    x = max(-448.0, min(448.0, x))
    best = min(vals, key=lambda c: (abs(vals[c] - x), c & 1, c))
    return vals[best]


def test_tc_operand_table_fp8_is_the_twiddled_dft16(fft3d_lib):
    """The FP8 (E4M3) B operands: hi = rn(16 b), lo = rn(16 b - hi) of the
    FP64 entry b, at the documented byte positions, the same for the split
    and the plain FP8 kinds; hi + lo reproduces 16 times the complex matrix
    to the E4M3 resolution; the second half of the buffer is zero."""
    vals = _e4m3_values()
    for prec in (L.FFT3D_SPLIT_FP8, L.FFT3D_FP8):
        buf = (ctypes.c_uint16 * 8192)()
        assert fft3d_lib.fft3d_tc_operand_table(prec, buf) == 0
        raw = np.frombuffer(buf, dtype=np.uint8)
        assert not raw[8192:].any()
        for k1 in range(4):
            m_rec = np.zeros((16, 16), np.complex128)
            for nn in range(32):
                for kk in range(32):
                    k2, d, n2, c = nn // 2, nn % 2, kk // 2, kk % 2
                    a = -2.0 * math.pi * ((n2 * (k1 + 4 * k2)) % 64) / 64.0
                    wr, wi = math.cos(a), math.sin(a)
                    b = 16.0 * ((wr if d == 0 else wi) if c == 0 else (-wi if d == 0 else wr))
                    off = ((nn // 8) * 2 + kk // 16) * 128 + (nn % 8) * 16 + kk % 16
                    hi = vals[int(raw[(0 * 4 + k1) * 1024 + off])]
                    lo = vals[int(raw[(1 * 4 + k1) * 1024 + off])]
                    assert hi == _e4m3_rn(b, vals)
                    assert lo == _e4m3_rn(b - hi, vals)
                    if c == 0:
                        m_rec[n2, k2] += (hi + lo) if d == 0 else 1j * (hi + lo)
            n2g, k2g = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
            expect = 16.0 * np.exp(-2j * np.pi * n2g * (k1 + 4 * k2g) / 64)
            assert np.abs(m_rec - expect).max() < 2.0 ** -4


def test_tc_operand_table_bfp16_uses_the_fp16_table(fft3d_lib):
    a = (ctypes.c_uint16 * 8192)()
    b = (ctypes.c_uint16 * 8192)()
    assert fft3d_lib.fft3d_tc_operand_table(L.FFT3D_BFP16, a) == 0
    assert fft3d_lib.fft3d_tc_operand_table(L.FFT3D_SPLIT_FP16, b) == 0
    assert bytes(a) == bytes(b)


def _create_real(lib, *args):
    h = ctypes.c_void_p(1234)
    rc = lib.fft3d_real_plan_create(*args, ctypes.byref(h))
    return rc, h.value


@pytest.mark.parametrize("args,code", [
    ((64, 0, 0, -1, 0), L.FFT3D_ERR_INVALID_ARG),               # batch 0
    ((64, (1 << 24) + 1, 0, -1, 0), L.FFT3D_ERR_INVALID_ARG),   # batch too large
    ((64, 2, 7, -1, 0), L.FFT3D_ERR_INVALID_ARG),               # precision
    ((64, 2, 0, 0, 0), L.FFT3D_ERR_INVALID_ARG),                # direction
    ((64, 2, 0, 1, 5), L.FFT3D_ERR_INVALID_ARG),                # norm
    ((15, 2, 0, -1, 0), L.FFT3D_ERR_UNSUPPORTED_SIZE),          # odd edge
    ((7, 2, 0, -1, 0), L.FFT3D_ERR_UNSUPPORTED_SIZE),
    ((1024, 2, 0, -1, 0), L.FFT3D_ERR_UNSUPPORTED_SIZE),
    ((32, 2, 1, -1, 0), L.FFT3D_ERR_UNSUPPORTED_PRECISION),     # tensor cores at 64, 128 only
])
def test_real_create_validates_before_device(fft3d_lib, args, code):
    rc, h = _create_real(fft3d_lib, *args)
    assert rc == code
    assert h is None


def test_real_null_handles(fft3d_lib):
    assert fft3d_lib.fft3d_real_plan_create(64, 2, 0, -1, 0, None) == L.FFT3D_ERR_NULL_PTR
    assert fft3d_lib.fft3d_real_execute(None, 16, 16, None) == L.FFT3D_ERR_NULL_PTR
    assert fft3d_lib.fft3d_real_get_device_status(None, None) == L.FFT3D_ERR_NULL_PTR
    assert fft3d_lib.fft3d_real_plan_destroy(None) == L.FFT3D_SUCCESS


def test_real_valid_args_reach_device_check(fft3d_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    rc, h = _create_real(fft3d_lib, 64, 3, 0, -1, 0)
    assert rc == L.FFT3D_ERR_NO_DEVICE and h is None


def test_noalloc_validates_before_device(fft3d_lib):
    f = fft3d_lib.fft3d_execute_noalloc
    P = 1 << 20
    fwd, none = L.FFT3D_FORWARD, L.FFT3D_NORM_NONE
    assert f(64, 1, fwd, none, None, P, None) == L.FFT3D_ERR_NULL_PTR
    assert f(64, 1, fwd, none, P, None, None) == L.FFT3D_ERR_NULL_PTR
    assert f(64, 1, fwd, none, P + 8, P, None) == L.FFT3D_ERR_MISALIGNED  # 16-byte rule
    assert f(64, 1, fwd, none, P, P + 8, None) == L.FFT3D_ERR_MISALIGNED
    assert f(64, 1, 0, none, P, P, None) == L.FFT3D_ERR_INVALID_ARG
    assert f(64, 1, fwd, 3, P, P, None) == L.FFT3D_ERR_INVALID_ARG
    assert f(100, 1, fwd, none, P, P, None) == L.FFT3D_ERR_UNSUPPORTED_SIZE  # general path only
    assert f(64, 0, fwd, none, P, P, None) == L.FFT3D_ERR_INVALID_ARG
    for n in FUSED:
        assert f(n, L.FFT3D_NOALLOC_MAX_BATCH + 1, fwd, none, P, P, None) == \
            L.FFT3D_ERR_EXCEEDS_STATIC_SCRATCH


def test_noalloc_limit_is_reachable(fft3d_lib):
    """Every fused edge at the documented maximum batch passes the static
    scratch check (and, without a GPU, stops at the device check)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    P = 1 << 20
    for n in FUSED:
        rc = fft3d_lib.fft3d_execute_noalloc(n, L.FFT3D_NOALLOC_MAX_BATCH, L.FFT3D_FORWARD,
                                             L.FFT3D_NORM_NONE, P, P, None)
        assert rc == L.FFT3D_ERR_NO_DEVICE, (n, rc)


def _header_declarations():
    src = open(os.path.join(ROOT, "include", "fft3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for ret, name, params in re.findall(
            r"([A-Za-z_][\w \t\*]*?)\b(fft3d_[a-z0-9_]+)\s*\(([^;{()]*)\)\s*;", src, flags=re.S):
        ps = [" ".join(p.split()) for p in params.split(",")]
        ps = [] if ps == ["void"] or ps == [""] else [re.sub(r"\s*\b\w+$", "", p) for p in ps]
        out[name] = (" ".join(ret.split()), ps)
    return out


_P = ctypes.POINTER
_C_TYPES = {
    "int": {ctypes.c_int}, "size_t": {ctypes.c_size_t}, "int64_t": {ctypes.c_int64},
    "double": {ctypes.c_double}, "const char*": {ctypes.c_char_p},
    "int*": {_P(ctypes.c_int), ctypes.c_void_p}, "const int*": {_P(ctypes.c_int), ctypes.c_void_p},
    "float*": {_P(ctypes.c_float), ctypes.c_void_p}, "const float*": {_P(ctypes.c_float), ctypes.c_void_p},
    "double*": {_P(ctypes.c_double), ctypes.c_void_p},
    "const double*": {_P(ctypes.c_double), ctypes.c_void_p},
    "uint16_t*": {_P(ctypes.c_uint16), ctypes.c_void_p},
    "int64_t*": {_P(ctypes.c_int64), ctypes.c_void_p},
    "void*": {ctypes.c_void_p}, "const void*": {ctypes.c_void_p},
    "void* const*": {ctypes.c_void_p, _P(ctypes.c_void_p)},
    "const void* const*": {ctypes.c_void_p, _P(ctypes.c_void_p)},
    "fft3d_plan": {ctypes.c_void_p}, "fft3d_real_plan": {ctypes.c_void_p},
    "fft3d_plan*": {_P(ctypes.c_void_p)}, "fft3d_real_plan*": {_P(ctypes.c_void_p)},
    "fft3d_tune_timer": {ctypes.c_void_p},
}


def test_binding_signatures_match_the_header():
    """Every ctypes declaration of the binding has the header's argument
    count and, per argument and result, a ctypes type of the C type's size
    and kind (a mismatch would marshal garbage without any error)."""
    decls = _header_declarations()
    assert sorted(decls) == sorted(L._SIGS)
    for name, (res, args) in L._SIGS.items():
        cret, cparams = decls[name]
        assert len(args) == len(cparams), (name, cparams)
        assert res in _C_TYPES[cret], (name, cret, res)
        for i, (a, c) in enumerate(zip(args, cparams)):
            assert c in _C_TYPES, (name, c)
            assert a in _C_TYPES[c], (name, i, c, a)
