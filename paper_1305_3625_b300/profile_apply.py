"""Run one part of the hot path on a synthetic field, for kernel profiling.

    python -m paper_1305_3625_b300.profile_apply L {f32|f64} [reps] [apply|product|removal]

Creates a plan for an L x L grid (tuned launch shapes, cached as usual) and
runs `reps` times one of:
  apply    fftconv_apply, y = C x of a uniform random field (passes k_rfwd,
           k_colc, k_rinv in the apply shapes);
  product  fftconv_cg_product, one CG product q = C p + s p with its dot
           products (the solver's shapes; pass C in its CG mode);
  removal  fc_masked_step, the breaking step argmax |x|/t on a random field
           (the removal is undone after each step, so every step scans the
           same sites).
Profilers can then capture those kernels.
"""
import sys

import torch

import paper_1305_3625_b300 as fc


def main(argv):
    L = int(argv[1])
    prec = fc.FC_F32 if argv[2] == "f32" else fc.FC_F64
    reps = int(argv[3]) if len(argv) > 3 else 2
    what = argv[4] if len(argv) > 4 else "apply"
    plan = fc.fftconv_plan_create(L, prec if what != "removal" else fc.FC_F32 | fc.FC_F64)
    dt = torch.float32 if prec == fc.FC_F32 else torch.float64
    n = L * L
    g = torch.Generator(device="cuda").manual_seed(1)
    if what == "apply":
        x = torch.rand(n, device="cuda", dtype=dt, generator=g)
        y = torch.empty_like(x)
        for _ in range(reps):
            fc.fftconv_apply_prec(plan, prec, x, y)
        shapes = fc.fftconv_plan_shape_set(plan, prec, fc.FC_SHAPES_APPLY)
    elif what == "product":
        p, r = (torch.rand(n, device="cuda", dtype=dt, generator=g) for _ in range(2))
        s = 0.5 + torch.rand(n, device="cuda", dtype=dt, generator=g)
        q = torch.empty_like(p)
        for _ in range(reps):
            fc.fftconv_cg_product(plan, prec, p, r, s, q)
        shapes = fc.fftconv_plan_shape_set(plan, prec, fc.FC_SHAPES_SOLVE)
    else:
        x = torch.randn(n, device="cuda", dtype=torch.float64, generator=g)
        t = torch.rand(n, device="cuda", dtype=torch.float64, generator=g)
        mask = torch.ones(n, device="cuda", dtype=torch.uint8)
        removed = torch.empty(1, device="cuda", dtype=torch.int64)
        x0 = x.clone()
        for _ in range(reps):
            fc.fc_masked_step(plan, t, mask, x, removed)
            mask.fill_(1)
            x.copy_(x0)
        shapes = {"removed": int(removed[0])}
    torch.cuda.synchronize()
    print("L", L, argv[2], what, shapes)


if __name__ == "__main__":
    main(sys.argv)
