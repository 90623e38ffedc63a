"""Large single instance, L = 4096 (padded 8192^2 FFT): the operator of every
compiled FP32 launch shape against the oracle's FFT route (normwise and
entrywise), the mixed solve against an FP64 GPU solve at the solution-error
target, its residual recomputed by the oracle, and a few quasi-static
removal steps."""
import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import U32, U64, check_conv, conv_levels, conv_max_bound, dev, host, rel2

pytestmark = pytest.mark.gpu

L = 4096
M = 8192


@pytest.fixture(scope="module")
def big():
    p = fc_inputs.problem(L, seed=0, with_t=True)
    plan = fc.fftconv_plan_create(L)
    return p, plan


@pytest.fixture(scope="module")
def field():
    """An input field and the oracle's y = C x (FP64 FFT route) for it and for
    its FP32 rounding."""
    x = fc_inputs.problem(L, seed=5)["s"] - 1.0  # values in (-0.5, 0.5)
    x32 = x.astype(np.float32).astype(np.float64)
    return x, oracle.conv_fft(L, x), x32, oracle.conv_fft(L, x32)


def test_apply_full_field(big, field):
    """The tuned plan's FP32 and FP64 operators over the whole field, and
    sampled entries of the oracle's FFT route against its direct sum of
    Eq. 1b (an independent algorithm)."""
    _, plan = big
    x, ref64, x32, ref32 = field
    y32 = torch.empty(L * L, device="cuda", dtype=torch.float32)
    y64 = torch.empty(L * L, device="cuda", dtype=torch.float64)
    fc.fftconv_apply_prec(plan, fc.FC_F32, dev(x, torch.float32), y32)
    fc.fftconv_apply_prec(plan, fc.FC_F64, dev(x), y64)
    check_conv(host(y32).astype(np.float64), ref32, U32, M, "L=4096 f32 (tuned shapes)")
    ymax = float(np.max(np.abs(ref64)))
    # the oracle's FP64 FFT route has the FP64 error model of the kernels
    check_conv(host(y64), ref64, U64, M, "L=4096 f64", U64 * conv_levels(M) * ymax)
    rng = np.random.default_rng(2)
    pts = [(0, 0), (L - 1, L - 1), (0, L - 1), (L - 1, 0)] + [tuple(v) for v in rng.integers(0, L, size=(8, 2))]
    ax = np.abs(x)
    for iy, ix in pts:
        d = oracle.conv_direct_at(L, x, iy, ix)
        # the direct sum of N products rounds like a random walk: 4 sqrt(N) u (C|x|)_i
        allow = 4.0 * L * U64 * oracle.conv_direct_at(L, ax, iy, ix)
        assert abs(ref64[iy * L + ix] - d) <= conv_max_bound(U64, M) * ymax + allow, (iy, ix)


def test_apply_every_shape(field):
    """Every FP32 launch shape compiled for M = 8192 (the tuner's candidates:
    the 1024-thread row blocks, the single-buffered column shapes, the
    TMA-staged pass C) gives the same operator, entry by entry."""
    _, _, x32, ref32 = field
    xd = dev(x32, torch.float32)
    probe = fc.fftconv_plan_create(L, fc.FC_F32, no_autotune=True)
    n = fc.fftconv_plan_shapes(probe, fc.FC_F32)["n_shapes"]
    probe.close()
    for k in range(max(n)):
        shapes = tuple(min(k, n[i] - 1) for i in range(3))
        p = fc.fftconv_plan_create(L, fc.FC_F32, shapes=shapes)
        info = fc.fftconv_plan_shapes(p, fc.FC_F32)
        y = torch.empty_like(xd)
        fc.fftconv_apply(p, xd, y)
        check_conv(host(y).astype(np.float64), ref32, U32, M,
                   f"L=4096 shapes {shapes} radix {info['radix']} per block {info['per_block']}")
        p.close()


def test_mixed_solution_error_and_oracle_residual(big):
    """The solution-error target of the mixed path at L = 4096: solved to the
    residual 3e-10 (error <= kappa * residual with kappa ~ 0.8 L ~ 3300 gives
    1e-6), it agrees with an FP64 GPU solve to 1e-12 within 1e-6 relative.
    Its residual b - (C + S) x is recomputed by the oracle's FP64 operator
    over the whole field, and on a 256^2 sub-block at a seeded corner the
    oracle's FFT-route residual is checked entry by entry against direct
    sums of Eq. 1b."""
    p, plan = big
    s, b = dev(p["s"]), dev(p["b"])
    xm = torch.zeros_like(s)
    rm = fc.cg_solve(plan, s, b, xm, rtol=3e-10, mode=fc.FC_MODE_MIXED, precond=True)
    assert rm["status"] == fc.FC_OK and rm["true_rel_resid"] <= 3e-10
    x64 = torch.zeros_like(s)
    r64 = fc.cg_solve(plan, s, b, x64, rtol=1e-12, mode=fc.FC_MODE_F64, precond=True)
    assert r64["status"] == fc.FC_OK and r64["true_rel_resid"] <= 1e-12
    xm_h, x64_h = host(xm), host(x64)
    err = rel2(xm_h, x64_h)
    print(f"L=4096 mixed vs FP64: rel err {err:.3e}; mixed {rm['iters']} iterations, "
          f"{rm['refinements']} true residuals")
    assert err <= 1e-6
    q = oracle.apply_A(L, p["s"], xm_h)
    r = p["b"] - q
    rel = float(np.linalg.norm(r) / np.linalg.norm(p["b"]))
    assert rel <= 1.01 * 3e-10, rel
    rng = np.random.default_rng(9)
    iy0, ix0 = (int(v) for v in rng.integers(0, L - 256, size=2))
    blk = (slice(iy0, iy0 + 256), slice(ix0, ix0 + 256))
    r2, b2 = r.reshape(L, L)[blk], p["b"].reshape(L, L)[blk]
    print(f"256^2 block at ({iy0}, {ix0}): relative residual {np.linalg.norm(r2) / np.linalg.norm(b2):.3e}")
    assert np.linalg.norm(r2) <= np.linalg.norm(r)
    qmax = float(np.max(np.abs(q)))
    ax = np.abs(xm_h)
    for iy, ix in [tuple(v) for v in rng.integers(0, 256, size=(12, 2))]:
        i = (iy0 + iy) * L + ix0 + ix
        r_direct = p["b"][i] - (oracle.conv_direct_at(L, xm_h, iy0 + iy, ix0 + ix) + p["s"][i] * xm_h[i])
        allow = 4.0 * L * U64 * oracle.conv_direct_at(L, ax, iy0 + iy, ix0 + ix)  # the direct sum's own rounding
        assert abs(r_direct - r[i]) <= 2 * conv_max_bound(U64, M) * qmax + allow


def test_masked_steps(big):
    p, plan = big
    s, b, t = dev(p["s"]), dev(p["b"]), dev(p["t"])
    mask = torch.ones(L * L, device="cuda", dtype=torch.uint8)
    x = torch.zeros_like(s)
    rem = torch.empty(1, device="cuda", dtype=torch.int64)
    picks = []
    for _ in range(3):
        r = fc.cg_solve(plan, s, b, x, mask=mask, rtol=1e-8, mode=fc.FC_MODE_MIXED)
        assert r["status"] == fc.FC_OK
        xh = host(x)
        mh = host(mask)
        want, _ = oracle.argmax_ratio(xh, p["t"], mh)
        fc.fc_masked_step(plan, t, mask, x, rem)
        k = int(host(rem)[0])
        assert k == want
        picks.append(k)
    assert len(set(picks)) == 3
    assert int(host(mask).sum()) == L * L - 3
