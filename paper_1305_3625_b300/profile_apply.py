"""Run fftconv_apply on a synthetic field, for kernel profiling.

    python -m paper_1305_3625_b300.profile_apply L {f32|f64} [reps]

Creates a plan for an L x L grid (tuned launch shapes, cached as usual), runs
`reps` applications of C to a uniform random field and prints the shapes
used.  Profilers can then capture the three passes (k_rfwd, k_colc, k_rinv)
of those applications.
"""
import sys

import torch

import paper_1305_3625_b300 as fc


def main(argv):
    L = int(argv[1])
    prec = fc.FC_F32 if argv[2] == "f32" else fc.FC_F64
    reps = int(argv[3]) if len(argv) > 3 else 2
    plan = fc.fftconv_plan_create(L, prec)
    dt = torch.float32 if prec == fc.FC_F32 else torch.float64
    x = torch.rand(L * L, device="cuda", dtype=dt)
    y = torch.empty_like(x)
    for _ in range(reps):
        fc.fftconv_apply_prec(plan, prec, x, y)
    torch.cuda.synchronize()
    print("L", L, argv[2], "shapes", fc.fftconv_plan_shapes(plan, prec))


if __name__ == "__main__":
    main(sys.argv)
