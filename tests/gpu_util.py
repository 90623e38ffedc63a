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


def conv_max_bound(u, M):
    """Max-norm error allowed for y = C x, relative to max |y|:
    max_i |y_hat_i - y_i| <= u levels max_i |y_i|.

    The roundings of the FFT round trip spread over all outputs like
    independent noise of rms about u sqrt(levels) rms(y) (the normwise bound
    above adds them up); the largest of N such entries is about
    sqrt(2 ln N) of them, rms(y) <= max |y|, and
    sqrt(max(2 ln N, 1)) sqrt(levels) <= levels on every grid L <= 4096
    with M the padded side (e.g. 5.5 x 7.1 = 39 <= 50 at L = 2048).  Against max |y|
    instead of ||y||_2 the bound is about sqrt(N) times tighter per entry,
    so it fails an error confined to a few outputs (a row pair, the packed
    column 0, a tile edge) that the 2-norm bound would let through."""
    return u * conv_levels(M)


def conv_max_err(y, ref):
    return float(np.max(np.abs(y - ref))) / float(np.max(np.abs(ref)))


def direct_sum_allowance(L, x, u=U64):
    """Rounding error allowed to the oracle's direct sum of Eq. 1b itself at
    every output (naive recursive summation of N = L^2 products in FP64):
    each addition errs by at most u times the running sum, which is at most
    (C|x|)_i = sum_j G_ij |x_j| (G >= 0); N such errors of random sign add up
    to about sqrt(N) of them, and 4 sqrt(N) u (C|x|)_i covers the largest of
    the outputs.  C|x| comes from the same direct sum."""
    import oracle
    return 4.0 * math.sqrt(L * L) * u * oracle.conv_direct(L, np.abs(np.asarray(x, dtype=np.float64)))


def check_conv(y, ref, u, M, what, ref_abs=0.0):
    """Both bounds: the 2-norm one of conv_rel_bound and the max-norm one of
    conv_max_bound; ref_abs (a scalar or one value per output) is the
    reference's own rounding error, allowed on top of the max-norm bound."""
    e = conv_err(y, ref)
    bound = conv_rel_bound(u, M)
    em = conv_max_err(y, ref)
    mbound = conv_max_bound(u, M)
    ymax = float(np.max(np.abs(ref)))
    excess = float(np.max(np.abs(y - ref) - ref_abs)) / ymax
    print(f"{what}: rel err {e:.3e} (bound {bound:.3e}, {e / bound:.3f}), "
          f"max err {em:.3e} (less the reference's allowance {excess:.3e}; bound {mbound:.3e}, "
          f"{excess / mbound:.3f})")
    assert e <= bound, (what, e, bound)
    assert excess <= mbound, (what, excess, mbound)
