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


def conv_bound(u, M, ghat_max, x):
    """Error allowed for y = C x through a padded M x M FFT round trip.

    The 2D transform pair has log2(M^2) butterfly levels each way; a rounding
    of relative size u per level, plus the rounding of the stored spectrum,
    gives ||y_hat - y||_2 <= c u (2 log2(M^2) + 1) max|Ghat| ||x||_2 with a
    modest constant (Higham, Accuracy and Stability of Numerical Algorithms,
    Sec. 24.1).  c = 2 here.
    """
    levels = 2 * 2 * math.log2(M) + 1
    return 2.0 * u * levels * ghat_max * float(np.linalg.norm(x))
