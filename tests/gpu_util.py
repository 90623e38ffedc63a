"""Shared helpers of the -m gpu tests (device transfers, error norms, bounds)."""
import math

import numpy as np
import torch

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel2(a, b):
    """||a - b||_2 / ||b||_2."""
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def conv_levels(M):
    """Butterfly levels of the forward plus inverse padded 2D transform, plus
    the roundings of the stored spectrum and of the pointwise product."""
    return 2 * 2 * math.log2(M) + 2


def conv_rel_bound(u, M):
    """Normwise relative error allowed for y = C x through the padded M x M
    FFT round trip: ||y_hat - y||_2 <= 2 u levels ||y||_2.

    Standard FFT error analysis (Higham, Accuracy and Stability of Numerical
    Algorithms, Thm. 24.2) gives a 2-norm error growing by about u per
    radix-2 level; C is positive definite with lambda_min ~ 0.6, so the input
    and output norms are within the operator's spread and a factor 2 covers
    the constants of the radix-16 codelets and the twiddle rounding (observed
    errors are 3-22 percent of this bound for L = 1..2048)."""
    return 2.0 * u * conv_levels(M)


def conv_err(y, ref):
    return float(np.linalg.norm(y - ref)) / float(np.linalg.norm(ref))
