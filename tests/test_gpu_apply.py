"""Parity of fftconv_apply (y = C x, FP32 and FP64) with the oracle."""
import numpy as np
import pytest
import torch

import fc_inputs
import oracle
from gpu_util import U32, U64, check_conv, conv_levels, conv_rel_bound, dev, direct_sum_allowance, host

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


def check(y, ref, u, M, what, ref_abs=0.0):
    check_conv(y, ref, u, M, what, ref_abs)


def fft_route_allowance(ref, M):
    """The oracle's FP64 FFT route has the FP64 error model of the kernels."""
    return U64 * conv_levels(M) * float(np.max(np.abs(ref)))


@pytest.mark.parametrize("L", SMALL)
def test_apply_matches_direct_sum(L):
    rng = np.random.default_rng(100 + L)
    x = rng.standard_normal(L * L)
    x32, y32, y64 = run_apply(L, x)
    M = fc_inputs.padded_side(L)
    check(y64, oracle.conv_direct(L, x), U64, M, f"L={L} f64", direct_sum_allowance(L, x))
    # FP32 sees the rounded input
    check(y32, oracle.conv_direct(L, x32), U32, M, f"L={L} f32", direct_sum_allowance(L, x32))


@pytest.mark.parametrize("L", [64, 100, 128, 256])
def test_apply_matches_oracle_fft_route(L):
    rng = np.random.default_rng(L)
    x = rng.uniform(-1, 1, L * L)
    x32, y32, y64 = run_apply(L, x)
    M = fc_inputs.padded_side(L)
    ref64 = oracle.conv_fft(L, x)
    check(y64, ref64, U64, M, f"L={L} f64", fft_route_allowance(ref64, M))
    check(y32, oracle.conv_fft(L, x32), U32, M, f"L={L} f32")


@pytest.mark.parametrize("L", [1024, 2048])
def test_apply_full_size(L):
    """At the configs' sizes: the whole output against the oracle's FP64 FFT
    route, and sampled outputs against the O(L^2) direct sum."""
    p = fc_inputs.problem(L, seed=0)
    x = p["s"] - 1.0  # values in (-0.5, 0.5)
    x32, y32, y64 = run_apply(L, x)
    M = fc_inputs.padded_side(L)
    ref64 = oracle.conv_fft(L, x)
    check(y64, ref64, U64, M, f"L={L} f64", fft_route_allowance(ref64, M))
    check(y32, oracle.conv_fft(L, x32), U32, M, f"L={L} f32")
    ynorm = float(np.linalg.norm(ref64))
    rng = np.random.default_rng(7)
    pts = [(0, 0), (L - 1, L - 1), (0, L - 1), (L // 2, L // 3)] + \
          [tuple(v) for v in rng.integers(0, L, size=(12, 2))]
    for iy, ix in pts:
        # one entry may carry at most the whole l2 error
        assert abs(y64[iy * L + ix] - oracle.conv_direct_at(L, x, iy, ix)) <= conv_rel_bound(U64, M) * ynorm
        assert abs(y32[iy * L + ix] - oracle.conv_direct_at(L, x32, iy, ix)) <= conv_rel_bound(U32, M) * ynorm


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
    check(host(y32).astype(np.float64), oracle.conv_direct(L, xr), U32, M, "f32-only plan")
    # an FP32-only plan has no FP64 operator
    with pytest.raises(fc.FcError):
        fc.fftconv_apply_prec(p, fc.FC_F64, dev(x), torch.empty(L * L, device="cuda", dtype=torch.float64))


@pytest.mark.parametrize("L", [3, 100, 128, 512, 1024, 2048, 4096])
def test_every_compiled_shape_matches(L):
    """Each launch shape the autotuner may pick gives the same operator (the
    radix-32 shapes from L = 2048, M = 4096, on; L = 4096 runs the M = 8192
    shapes the large instance uses)."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal(L * L)
    x32 = dev(x, torch.float32)
    xr = host(x32).astype(np.float64)
    ref32 = oracle.conv_fft(L, xr)
    M = fc_inputs.padded_side(L)
    p0 = plan(L)
    n = fc.fftconv_plan_shapes(p0, fc.FC_F32)["n_shapes"]
    for k in range(max(n)):
        shapes = tuple(min(k, n[i] - 1) for i in range(3))
        p = fc.fftconv_plan_create(L, fc.FC_F32, shapes=shapes)
        info = fc.fftconv_plan_shapes(p, fc.FC_F32)
        assert info["chosen"] == list(shapes)
        y = torch.empty_like(x32)
        fc.fftconv_apply(p, x32, y)
        check(host(y).astype(np.float64), ref32, U32, M, f"L={L} shapes {shapes} {info['radix']} {info['per_block']}")


def test_autotune_writes_cache(tmp_path, monkeypatch):
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    code = ("import paper_1305_3625_b300 as fc; p = fc.fftconv_plan_create(512, fc.FC_F32); "
            "print(fc.fftconv_plan_shapes(p, fc.FC_F32))")
    env = dict(__import__("os").environ, FC_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    lines = cache.read_text().splitlines()
    assert any("f32 M=1024 L=512 colc" in ln for ln in lines), lines
    # a second plan reads the cached choice instead of timing again
    out2 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    assert out.stdout == out2.stdout
    assert len(cache.read_text().splitlines()) == len(lines)


def test_solver_shapes_chain_tuned_and_cached(tmp_path):
    """A mixed plan's solver shapes (FC_SHAPES_SOLVE): passes A and C timed in
    the preconditioned modes, then the close candidates paired as chains of
    whole PCG iterations; the fastest pairing is the one kept and cached, and
    a second plan reads it without timing again."""
    import ast
    import re
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    code = ("import paper_1305_3625_b300 as fc; p = fc.fftconv_plan_create(512, fc.FC_F32 | fc.FC_F64); "
            "print(fc.fftconv_plan_shape_set(p, fc.FC_F32, fc.FC_SHAPES_SOLVE))")
    env = dict(__import__("os").environ, FC_TUNE_CACHE=str(cache), FC_TUNE_VERBOSE="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    chosen = ast.literal_eval(out.stdout.strip().splitlines()[-1])["chosen"]
    lines = cache.read_text().splitlines()
    cached = {}
    for ln in lines:
        key, idx = ln.rsplit("|", 1)
        cached[key.strip()] = int(idx)
    a_key = [k for k in cached if "rfwd_cg" in k]
    c_key = [k for k in cached if "rinv_cg" in k]
    assert a_key and c_key, lines
    assert cached[a_key[-1]] == chosen[0] and cached[c_key[-1]] == chosen[2]
    chain = [(int(m.group(1)), int(m.group(2)), float(m.group(3)))
             for m in re.finditer(r"PCG iteration, pass A (\d+), pass C (\d+): ([0-9.]+) us", out.stderr)]
    if chain:
        fastest = min(chain, key=lambda c: c[2])
        assert (fastest[0], fastest[1]) == (chosen[0], chosen[2]), (chain, chosen)
    out2 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    assert out2.stdout == out.stdout
    assert "PCG iteration" not in out2.stderr
    assert len(cache.read_text().splitlines()) == len(lines)
