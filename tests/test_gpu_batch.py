"""Batched solves (cg_solve_batch, cg_solve_groups): nb problems of one size
per launch, each against the same problem solved alone by cg_solve with the
same launch shapes (bitwise), and against the oracle's dense solves."""
import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu

MODES = [(fc.FC_MODE_F64, False), (fc.FC_MODE_F64, True), (fc.FC_MODE_MIXED, False), (fc.FC_MODE_MIXED, True)]
_plans = {}


def plan(L):
    """Standard shapes (index 0) and the per-pass graph loop, so that a
    problem solved alone runs exactly the kernels of the batched launch."""
    if L not in _plans:
        _plans[L] = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64, shapes=(0, 0, 0), persistent=-1)
    return _plans[L]


def problems(L, nb, seed0, masked=False, b_kind="normal", broken=None):
    """nb systems; masked: problem k has a fraction broken[k] of its sites
    removed (default 0.1 each)."""
    ps = [fc_inputs.problem(L, seed=seed0 + k, b_kind=b_kind) for k in range(nb)]
    s = np.stack([p["s"] for p in ps])
    b = np.stack([p["b"] for p in ps])
    mask = None
    if masked:
        rng = np.random.default_rng(seed0)
        frac = np.full(nb, 0.1) if broken is None else np.asarray(broken)
        mask = (rng.random((nb, L * L)) >= frac[:, None]).astype(np.uint8)
    return s, b, mask


def solve_alone(L, s, b, mask, mode, precond, rtol, x0=None):
    x = dev(np.zeros(L * L) if x0 is None else x0)
    m = None if mask is None else dev(mask, torch.uint8)
    r = fc.cg_solve(plan(L), dev(s), dev(b), x, mask=m, rtol=rtol, mode=mode, precond=precond,
                    x0_zero=x0 is None, warm_resid=False)
    return host(x), r


def rtol_of(mode):
    return 1e-11 if mode == fc.FC_MODE_F64 else 1e-9


@pytest.mark.parametrize("mode,precond", MODES)
@pytest.mark.parametrize("L", [16, 33, 100])
def test_batch_equals_solves_alone(L, mode, precond):
    """Every problem of the batch: bitwise the iterate, iterations and
    refinements of the same problem solved alone (the problems converge
    after different numbers of iterations; unmasked at L = 16, masked with
    0 to 60 percent of the sites removed otherwise)."""
    nb = 5
    rtol = rtol_of(mode)
    s, b, mask = problems(L, nb, 100 * L, masked=(L != 16), broken=[0.0, 0.05, 0.2, 0.4, 0.6])
    # spread the conditioning: problem k's diagonal scaled by 4^-k
    s = s * (0.25 ** np.arange(nb))[:, None]
    x = dev(np.zeros((nb, L * L)))
    rc, rs = fc.cg_solve_batch(plan(L), dev(s), dev(b), x, mask=None if mask is None else dev(mask, torch.uint8),
                               rtol=rtol, mode=mode, precond=precond, x0_zero=True)
    assert rc == fc.FC_OK
    xb = host(x)
    iters = set()
    for k in range(nb):
        xa, ra = solve_alone(L, s[k], b[k], None if mask is None else mask[k], mode, precond, rtol)
        r = rs[k]
        assert r["status"] == ra["status"] == fc.FC_OK
        assert (r["iters"], r["refinements"], r["fp64_products"]) == (ra["iters"], ra["refinements"],
                                                                     ra["fp64_products"])
        assert r["zero_start"] == 1 and r["fp64_products"] == r["refinements"] - 1
        assert r["true_rel_resid"] == ra["true_rel_resid"] and r["true_rel_resid"] <= rtol
        assert np.array_equal(xb[k], xa)
        iters.add((r["iters"], r["refinements"]))
    assert len(iters) > 1  # the problems did not all stop together


@pytest.mark.parametrize("mode,precond", [(fc.FC_MODE_F64, False), (fc.FC_MODE_MIXED, True)])
def test_batch_matches_dense(mode, precond):
    L, nb = 12, 3
    s, b, mask = problems(L, nb, 7, masked=True)
    x = dev(np.zeros((nb, L * L)))
    rtol = 1e-12 if mode == fc.FC_MODE_F64 else 1e-10
    rc, rs = fc.cg_solve_batch(plan(L), dev(s), dev(b), x, mask=dev(mask, torch.uint8), rtol=rtol, mode=mode,
                               precond=precond, x0_zero=True)
    assert rc == fc.FC_OK
    xb = host(x)
    for k in range(nb):
        A = oracle.dense_operator(L, s[k])
        act = np.flatnonzero(mask[k])
        want = np.zeros(L * L)
        want[act] = np.linalg.solve(A[np.ix_(act, act)], b[k][act])
        assert rel2(xb[k], want) <= 100 * rtol
        assert np.all(xb[k][mask[k] == 0] == 0.0)


def test_warm_starts_zero_rhs_and_sizes():
    """Given starts (no zero start), a problem with b = 0 (finished at its
    first residual), and batch sizes that change between calls (graph
    rebuilt) on one plan."""
    L = 24
    rtol = 1e-10
    for nb in (3, 6, 1, 6):
        s, b, _ = problems(L, nb, 40 + nb)
        b[0] = 0.0
        x0 = np.random.default_rng(nb).standard_normal((nb, L * L)) * 0.1
        x0[0] = 0.0
        x = dev(x0)
        rc, rs = fc.cg_solve_batch(plan(L), dev(s), dev(b), x, rtol=rtol, mode=fc.FC_MODE_MIXED, precond=True)
        assert rc == fc.FC_OK
        xb = host(x)
        assert np.all(xb[0] == 0.0) and rs[0]["refinements"] == 1 and rs[0]["iters"] == 0
        assert rs[0]["zero_start"] == 0 and rs[0]["fp64_products"] == 1
        for k in range(1, nb):
            xa, ra = solve_alone(L, s[k], b[k], None, fc.FC_MODE_MIXED, True, rtol, x0=x0[k])
            assert np.array_equal(xb[k], xa) and rs[k]["iters"] == ra["iters"]


def test_groups_of_several_sizes():
    """cg_solve_groups runs batches of three sizes concurrently: each group's
    results are those of cg_solve_batch on the same plan."""
    sizes = {20: 4, 37: 3, 64: 5}
    groups, want = [], {}
    for L, nb in sizes.items():
        s, b, _ = problems(L, nb, 300 + L)
        x = dev(np.zeros((nb, L * L)))
        groups.append((plan(L), dev(s), dev(b), x, None))
        xw = dev(np.zeros((nb, L * L)))
        rc, rs = fc.cg_solve_batch(plan(L), dev(s), dev(b), xw, rtol=1e-9, mode=fc.FC_MODE_MIXED, precond=True,
                                   x0_zero=True)
        assert rc == fc.FC_OK
        want[L] = (host(xw), rs)
    rc, out = fc.cg_solve_groups(groups, rtol=1e-9, mode=fc.FC_MODE_MIXED, precond=True, x0_zero=True)
    assert rc == fc.FC_OK
    for (L, nb), g, rs in zip(sizes.items(), groups, out):
        assert len(rs) == nb
        assert np.array_equal(host(g[3]), want[L][0])
        assert [r["iters"] for r in rs] == [r["iters"] for r in want[L][1]]
        assert all(r["status"] == fc.FC_OK and r["true_rel_resid"] <= 1e-9 for r in rs)


def test_zero_start_equals_explicit_zero():
    """x0_zero takes P b as the first residual without a product; a start
    from an explicit zero vector computes it by the FP64 product, whose
    result is exactly P b as well (its norm summed in another order): the two
    solves agree to the tolerance with the same work."""
    L = 48
    p = fc_inputs.problem(L, seed=4, b_kind="normal")
    mask = (np.random.default_rng(1).random(L * L) >= 0.2).astype(np.uint8)
    out = []
    for x0_zero in (True, False):
        x = dev(np.zeros(L * L))
        r = fc.cg_solve(plan(L), dev(p["s"]), dev(p["b"]), x, mask=dev(mask, torch.uint8), rtol=1e-10,
                        mode=fc.FC_MODE_MIXED, precond=True, x0_zero=x0_zero, warm_resid=False)
        assert r["status"] == fc.FC_OK
        assert r["zero_start"] == int(x0_zero) and r["fp64_products"] == r["refinements"] - int(x0_zero)
        out.append((host(x), r["iters"], r["refinements"]))
    assert rel2(out[0][0], out[1][0]) <= 1e-8
    assert abs(out[0][1] - out[1][1]) <= 1 and out[0][2] == out[1][2]


def test_invalid_batches():
    L = 8
    s = dev(np.ones(2 * L * L))
    with pytest.raises(ValueError):
        fc.cg_solve_batch(plan(L), s, s, dev(np.zeros(L * L + 1)))
    with pytest.raises(fc.FcError):
        fc.cg_solve_batch(plan(L), s, s, dev(np.zeros(2 * L * L)), mode=7)
    x = dev(np.zeros(2 * L * L))
    with pytest.raises(fc.FcError):  # one plan in two groups
        fc.cg_solve_groups([(plan(L), s, s, x, None), (plan(L), s, s, x, None)])
    p64 = fc.fftconv_plan_create(L, fc.FC_F64)
    with pytest.raises(fc.FcError):  # mixed needs an FP32 side
        fc.cg_solve_batch(p64, s, s, x, mode=fc.FC_MODE_MIXED)


_oracle_x = {}


def oracle_solution(L, seed0, k, s, b, mask):
    """The oracle's FP64 CG (Listing 2) to a relative residual of 1e-13,
    cached per problem (the batched modes below share the problems)."""
    key = (L, seed0, k)
    if key not in _oracle_x:
        x, rc, _, rel = oracle.cg(L, s, b, mask=mask, rtol=1e-13)
        assert rc == 0 and rel <= 1e-13
        _oracle_x[key] = x
    return _oracle_x[key]


@pytest.mark.parametrize("mode,precond", [(fc.FC_MODE_F64, True), (fc.FC_MODE_MIXED, True),
                                          (fc.FC_MODE_MIXED, False)])
@pytest.mark.parametrize("L", [256, 512])
def test_batch_config3_sizes_against_oracle(L, mode, precond):
    """The batched workload's sizes (M = 512, 1024): three problems per batch,
    one unmasked and two with 10 and 30 percent of the sites removed, each
    bitwise the problem solved alone and within the solution-error targets
    of the oracle's solve (1e-10 FP64, 1e-6 mixed; the solver's residual
    tolerance is set below target / kappa, kappa ~ 0.8 L)."""
    nb, seed0 = 3, 5000 + L
    s, b, mask = problems(L, nb, seed0, masked=True, broken=[0.0, 0.1, 0.3])
    rtol = 1e-13 if mode == fc.FC_MODE_F64 else 2e-9
    x = dev(np.zeros((nb, L * L)))
    rc, rs = fc.cg_solve_batch(plan(L), dev(s), dev(b), x, mask=dev(mask, torch.uint8), rtol=rtol, mode=mode,
                               precond=precond, x0_zero=True)
    assert rc == fc.FC_OK
    xb = host(x)
    target = 1e-10 if mode == fc.FC_MODE_F64 else 1e-6
    for k in range(nb):
        assert rs[k]["status"] == fc.FC_OK and rs[k]["true_rel_resid"] <= rtol
        xa, ra = solve_alone(L, s[k], b[k], mask[k], mode, precond, rtol)
        assert np.array_equal(xb[k], xa) and rs[k]["iters"] == ra["iters"]
        want = oracle_solution(L, seed0, k, s[k], b[k], mask[k])
        err = rel2(xb[k], want)
        print(f"L={L} mode={mode} precond={precond} problem {k}: rel err {err:.3e}, {rs[k]['iters']} iterations")
        assert err <= target
        assert np.all(xb[k][mask[k] == 0] == 0.0)


@pytest.mark.parametrize("L", [1024, 2048])
def test_batch_server_sizes_oracle_residual(L):
    """The largest sizes the solve server batches (M = 2048, 4096): each
    problem's residual P (b - (C + S) x) recomputed by the oracle's FP64
    operator is within the tolerance, which bounds the solution error by
    |r| / lambda_min with lambda_min >= lambda_min(C) + min(s) > 1; and each
    problem is bitwise the problem solved alone."""
    nb, seed0 = 2, 7000 + L
    s, b, mask = problems(L, nb, seed0, masked=True, broken=[0.0, 0.2])
    rtol = 1e-8
    x = dev(np.zeros((nb, L * L)))
    rc, rs = fc.cg_solve_batch(plan(L), dev(s), dev(b), x, mask=dev(mask, torch.uint8), rtol=rtol,
                               mode=fc.FC_MODE_MIXED, precond=True, x0_zero=True)
    assert rc == fc.FC_OK
    xb = host(x)
    for k in range(nb):
        assert rs[k]["status"] == fc.FC_OK
        pb = np.where(mask[k] != 0, b[k], 0.0)
        r = pb - oracle.apply_A(L, s[k], xb[k], mask[k])
        rel = float(np.linalg.norm(r) / np.linalg.norm(pb))
        print(f"L={L} problem {k}: oracle residual {rel:.3e} (solver {rs[k]['true_rel_resid']:.3e})")
        assert rel <= 1.01 * rtol
        xa, ra = solve_alone(L, s[k], b[k], mask[k], fc.FC_MODE_MIXED, True, rtol)
        assert np.array_equal(xb[k], xa) and rs[k]["iters"] == ra["iters"]


@pytest.mark.parametrize("L", [100, 512])
def test_every_batched_shape_equals_alone(L):
    """The batched twin of every compiled launch shape (the batched solves'
    autotuner candidates): a batch of three problems equals the same problems
    solved alone on that shape, bitwise, and meets the tolerance by the
    oracle's residual.  (The TMA-staged pass C has no twin; a batch then runs
    the standard pass C.)"""
    probe = fc.fftconv_plan_create(L, fc.FC_F32, no_autotune=True)
    n = fc.fftconv_plan_shapes(probe, fc.FC_F32)["n_shapes"]
    probe.close()
    nb, rtol = 3, 1e-9
    s, b, mask = problems(L, nb, 900 + L, masked=True, broken=[0.0, 0.1, 0.3])
    for k in range(max(n)):
        shapes = tuple(min(k, n[i] - 1) for i in range(3))
        pl = fc.fftconv_plan_create(L, shapes=shapes, persistent=-1)
        bs = fc.fftconv_plan_batch_shapes(pl, fc.FC_F32)
        assert bs["tuned"]
        x = dev(np.zeros((nb, L * L)))
        rc, rs = fc.cg_solve_batch(pl, dev(s), dev(b), x, mask=dev(mask, torch.uint8), rtol=rtol,
                                   mode=fc.FC_MODE_MIXED, precond=True, x0_zero=True)
        assert rc == fc.FC_OK
        xb = host(x)
        for j in range(nb):
            pb = np.where(mask[j] != 0, b[j], 0.0)
            r = pb - oracle.apply_A(L, s[j], xb[j], mask[j])
            assert np.linalg.norm(r) <= 1.01 * rtol * np.linalg.norm(pb), (k, j)
            if bs["chosen"] == list(shapes):
                xa = dev(np.zeros(L * L))
                ra = fc.cg_solve(pl, dev(s[j]), dev(b[j]), xa, mask=dev(mask[j], torch.uint8), rtol=rtol,
                                 mode=fc.FC_MODE_MIXED, precond=True, x0_zero=True, warm_resid=False)
                assert np.array_equal(xb[j], host(xa)) and rs[j]["iters"] == ra["iters"], (k, j)
        pl.close()


def test_tuned_batched_shapes_equal_alone():
    """A plan's batched shapes, tuned on its first batched use, are kept for
    every later batch whatever its size; a problem solved alone on those
    shapes gives the batched result bitwise."""
    L, rtol = 512, 1e-8
    pl = fc.fftconv_plan_create(L)
    s, b, _ = problems(L, 5, 1234)
    x = dev(np.zeros((5, L * L)))
    rc, rs = fc.cg_solve_batch(pl, dev(s), dev(b), x, rtol=rtol, mode=fc.FC_MODE_MIXED, precond=True, x0_zero=True)
    assert rc == fc.FC_OK
    bs = fc.fftconv_plan_batch_shapes(pl, fc.FC_F32)
    assert bs["tuned"]
    print(f"L={L} batched shapes {bs}")
    x1 = dev(np.zeros((2, L * L)))
    rc, rs1 = fc.cg_solve_batch(pl, dev(s[:2]), dev(b[:2]), x1, rtol=rtol, mode=fc.FC_MODE_MIXED, precond=True,
                                x0_zero=True)
    assert rc == fc.FC_OK and fc.fftconv_plan_batch_shapes(pl, fc.FC_F32) == bs
    assert np.array_equal(host(x1), host(x)[:2])
    alone = fc.fftconv_plan_create(L, shapes=tuple(bs["chosen"]), persistent=-1)
    for j in range(2):
        xa = dev(np.zeros(L * L))
        fc.cg_solve(alone, dev(s[j]), dev(b[j]), xa, rtol=rtol, mode=fc.FC_MODE_MIXED, precond=True, x0_zero=True,
                    warm_resid=False)
        assert np.array_equal(host(xa), host(x)[j])
