"""Parity of fftconv_apply (y = C x, FP32 and FP64) with the oracle."""
import numpy as np
import pytest
import torch

import fc_inputs
import oracle
from gpu_util import U32, U64, conv_bound, dev, host

pytestmark = pytest.mark.gpu

import paper_1305_3625_b300 as fc

SMALL = [1, 2, 3, 5, 8, 16, 31, 32, 33, 48]
_plans = {}


def plan(L):
    if L not in _plans:
        _plans[L] = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)
    return _plans[L]


def run_apply(L, x64):
    p = plan(L)
    y32 = torch.empty(L * L, device="cuda", dtype=torch.float32)
    y64 = torch.empty(L * L, device="cuda", dtype=torch.float64)
    x32 = dev(x64, torch.float32)
    fc.fftconv_apply_prec(p, fc.FC_F32, x32, y32)
    fc.fftconv_apply_prec(p, fc.FC_F64, dev(x64), y64)
    return host(x32).astype(np.float64), host(y32).astype(np.float64), host(y64)


def ghat_max(L):
    """max |Ghat| = Ghat(0) = sum of the (non-negative) kernel table / M^2."""
    M = fc_inputs.padded_side(L)
    return float(oracle.kernel_table(L).sum()) / M**2


@pytest.mark.parametrize("L", SMALL)
def test_apply_matches_direct_sum(L):
    rng = np.random.default_rng(100 + L)
    x = rng.standard_normal(L * L)
    x32, y32, y64 = run_apply(L, x)
    M = fc_inputs.padded_side(L)
    gm = ghat_max(L)
    ref64 = oracle.conv_direct(L, x)
    ref32 = oracle.conv_direct(L, x32)  # the FP32 path sees the rounded input
    assert np.linalg.norm(y64 - ref64) <= conv_bound(U64, M, gm, x)
    assert np.linalg.norm(y32 - ref32) <= conv_bound(U32, M, gm, x32)


@pytest.mark.parametrize("L", [64, 100, 128, 256])
def test_apply_matches_oracle_fft_route(L):
    rng = np.random.default_rng(L)
    x = rng.uniform(-1, 1, L * L)
    x32, y32, y64 = run_apply(L, x)
    M = fc_inputs.padded_side(L)
    gm = ghat_max(L)
    assert np.linalg.norm(y64 - oracle.conv_fft(L, x)) <= conv_bound(U64, M, gm, x)
    assert np.linalg.norm(y32 - oracle.conv_fft(L, x32)) <= conv_bound(U32, M, gm, x32)


@pytest.mark.parametrize("L", [1024, 2048])
def test_apply_full_size(L):
    """At the configs' sizes: the whole output against the oracle's FP64 FFT
    route, and sampled outputs against the O(L^2) direct sum."""
    p = fc_inputs.problem(L, seed=0)
    x = p["s"] - 1.0  # values in (-0.5, 0.5)
    x32, y32, y64 = run_apply(L, x)
    M = fc_inputs.padded_side(L)
    gm = ghat_max(L)
    assert np.linalg.norm(y64 - oracle.conv_fft(L, x)) <= conv_bound(U64, M, gm, x)
    assert np.linalg.norm(y32 - oracle.conv_fft(L, x32)) <= conv_bound(U32, M, gm, x32)
    rng = np.random.default_rng(7)
    pts = [(0, 0), (L - 1, L - 1), (0, L - 1), (L // 2, L // 3)] + \
          [tuple(v) for v in rng.integers(0, L, size=(12, 2))]
    for iy, ix in pts:
        # one entry may carry at most the whole l2 error
        assert abs(y64[iy * L + ix] - oracle.conv_direct_at(L, x, iy, ix)) <= conv_bound(U64, M, gm, x)
        assert abs(y32[iy * L + ix] - oracle.conv_direct_at(L, x32, iy, ix)) <= conv_bound(U32, M, gm, x32)


def test_delta_reproduces_green_row():
    L = 40
    x = np.zeros(L * L)
    x[0] = 1.0
    _, y32, y64 = run_apply(L, x)
    want = np.array([oracle.G(ix, iy) for iy in range(L) for ix in range(L)])
    assert np.max(np.abs(y64 - want)) <= 1e-13
    assert np.max(np.abs(y32 - want)) <= 2e-6


def test_apply_is_deterministic():
    L = 128
    rng = np.random.default_rng(3)
    x = rng.standard_normal(L * L)
    a = run_apply(L, x)
    b = run_apply(L, x)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_apply_rejects_wrong_dtype():
    p = plan(8)
    x = torch.zeros(64, device="cuda", dtype=torch.float32)
    y = torch.zeros(64, device="cuda", dtype=torch.float64)
    with pytest.raises(TypeError):
        fc.fftconv_apply_prec(p, fc.FC_F32, x, y)


def test_f32_only_plan_applies():
    L = 24
    p = fc.fftconv_plan_create(L, fc.FC_F32)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(L * L)
    x32 = dev(x, torch.float32)
    y32 = torch.empty_like(x32)
    fc.fftconv_apply(p, x32, y32)
    xr = host(x32).astype(np.float64)
    M = fc_inputs.padded_side(L)
    assert np.linalg.norm(host(y32) - oracle.conv_direct(L, xr)) <= conv_bound(U32, M, ghat_max(L), xr)
    # an FP32-only plan has no FP64 operator
    with pytest.raises(fc.FcError):
        fc.fftconv_apply_prec(p, fc.FC_F64, dev(x), torch.empty(L * L, device="cuda", dtype=torch.float64))
