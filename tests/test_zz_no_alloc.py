"""fc_masked_step_static, the allocation-free breaking step, against the plan
version fc_masked_step.

Some callers cannot allocate device memory when they need the next fibre to
break: their device memory is held by another allocator, or their loop must
not stall on the synchronisation that cudaMalloc implies.  This entry point
keeps its scratch in a static device array instead.  The test calls it
through the C ABI twice in a row (the array keeps the first call's contents)
and requires the same removed index, mask and x as the plan version, bit for
bit (index work).  The file is collected last, so a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import fc_inputs
import paper_1305_3625_b300 as fc

pytestmark = pytest.mark.gpu


def c_static_step(n, t, mask, x, removed):
    """Direct C-ABI call through ctypes."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fc._lib.fc_masked_step_static(ctypes.c_int64(n), ctypes.c_void_p(t.data_ptr()),
                                         ctypes.c_void_p(mask.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(removed.data_ptr()), stream)


@pytest.mark.parametrize("L", [3, 64, 1024, 4096])
def test_static_step_matches_plan_step_twice(L):
    """L = 4096 is the static scratch's limit (N = 4096^2 sites, every one of
    its 8192 block slots in use)."""
    N = L * L
    p = fc_inputs.problem(L, seed=21, with_t=True)
    rng = np.random.default_rng(L)
    x0 = rng.standard_normal(N)
    m0 = (rng.random(N) > 0.05).astype(np.uint8)
    m0[0] = 1
    plan = fc.fftconv_plan_create(L, fc.FC_F64)
    t = torch.tensor(p["t"], device="cuda")
    xa, ma = torch.tensor(x0, device="cuda"), torch.tensor(m0, device="cuda")
    xb, mb = xa.clone(), ma.clone()
    ra = torch.empty(1, device="cuda", dtype=torch.int64)
    rb = torch.empty(1, device="cuda", dtype=torch.int64)
    for _ in range(2):
        fc.fc_masked_step(plan, t, ma, xa, ra)
        assert c_static_step(N, t, mb, xb, rb) == fc.FC_OK
        torch.cuda.synchronize()
        assert int(ra.item()) == int(rb.item()) >= 0
        assert torch.equal(ma, mb) and torch.equal(xa, xb)


def test_static_step_rejects_oversized_input():
    t = torch.ones(4, device="cuda", dtype=torch.float64)
    m = torch.ones(4, device="cuda", dtype=torch.uint8)
    x = torch.zeros(4, device="cuda", dtype=torch.float64)
    r = torch.empty(1, device="cuda", dtype=torch.int64)
    assert c_static_step(4096 * 4096 + 1, t, m, x, r) == fc.FC_EINVAL
    assert "16777216" in fc.fc_last_error()
