// The three HBM passes of one application of the coupling operator C
// (Listing 3's cpyComplex -> forward 2D FFT -> elementMult -> inverse 2D FFT
// -> cpyReal, Section 3) on the zero-padded M x M grid, with the CG vector
// work of Listing 2 fused into the first and last pass.
//
//   pass A (k_row_fwd): for each of the L data rows, form the input (plain x,
//       or the CG update x += a p, r -= a q, p = r + b p), zero-extend to M,
//       forward FFT along x, store the row of the L x M intermediate Z.
//   pass B (k_col_conv): for each of the M columns, forward FFT of the L
//       non-zero rows along y, multiply by the real kernel spectrum, inverse
//       FFT along y, keep rows [0, L) of Z.
//   pass C (k_row_inv): for each of the L rows, inverse FFT along x, keep
//       columns [0, L) (the crop of cpyReal) and apply the epilogue:
//       plain y = C x, the CG product q = P (C p + s p) with the dot products
//       p.q, r.q, q.q, or the true residual r = P (b - C x - s x).
//
// Z is row-major [L][M] complex; the spectrum is stored as its symmetric
// quarter Gq[(M/2+1)^2] (the kernel is even in each coordinate, so its
// transform is real and even in each frequency).
#pragma once

#include "fc_fft.cuh"
#include "fc_internal.h"

namespace fc {

// ------------------------------------------------------------ shapes ----

constexpr int pow2floor(int n) { return n < 2 ? 1 : 2 * pow2floor(n / 2); }

template <typename T, int M>
struct Cfg {
    static constexpr int E = Shape<T, M>::E;
    static constexpr int G = Shape<T, M>::G;
    // rows per CTA in the row passes (about 256 threads)
    static constexpr int RB = G >= 256 ? 1 : 256 / G;
    static constexpr int ROW_THREADS = RB * G;
    // columns per CTA in the column pass
    static constexpr int CB_RAW = (sizeof(T) == 4 ? 512 : 256) / G;
    static constexpr int CB_SMEM = (150 * 1024) / (seg_len(M) * (int)sizeof(cpx<T>));
    static constexpr int CB0 = CB_RAW < CB_SMEM ? CB_RAW : CB_SMEM;
    static constexpr int CB1 = CB0 < 1 ? 1 : CB0;
    static constexpr int CB = pow2floor(CB1 > M ? M : CB1);
    static constexpr int COL_THREADS = CB * G;
    static constexpr size_t ROW_SMEM = (size_t)RB * seg_len(M) * sizeof(cpx<T>);
    static constexpr size_t COL_SMEM = (size_t)CB * seg_len(M) * sizeof(cpx<T>);
};

// ------------------------------------------------------- loads/stores ---

template <typename T>
__device__ __forceinline__ cpx<T> ldc_cg(const cpx<T>* p) {
    if constexpr (sizeof(T) == 4) {
        float2 v = __ldcg(reinterpret_cast<const float2*>(p));
        return {v.x, v.y};
    } else {
        double2 v = __ldcg(reinterpret_cast<const double2*>(p));
        return {v.x, v.y};
    }
}
template <typename T>
__device__ __forceinline__ void stc(cpx<T>* p, cpx<T> v) {
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float2*>(p) = make_float2(v.x, v.y);
    else
        *reinterpret_cast<double2*>(p) = make_double2(v.x, v.y);
}

// ------------------------------------------------ block reductions -----

// Sum NV doubles over the block (fixed order: warp tree, then warp 0 over
// the warp sums).  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*scratch)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v[k] = lane < nw ? scratch[lane][k] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        }
    }
}

// Publish this block's partial sums and, in the last block to finish, add
// all blocks' partials in block order.  Returns true (in every thread of the
// last block) with the totals in tot (valid in thread 0).  Deterministic:
// the reduction order depends only on the grid and block sizes.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* part, unsigned* cnt,
                                              double (&tot)[NV]) {
    __shared__ double scratch[32][NV];
    __shared__ bool is_last;
    block_sum<NV>(v, scratch);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(size_t)blockIdx.x * NV + k] = v[k];
        __threadfence();
        unsigned prev = atomicAdd(cnt, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) acc += __ldcg(part + (size_t)b * NV + k);
        tot[k] = acc;
    }
    block_sum<NV>(tot, scratch);
    if (threadIdx.x == 0) *cnt = 0u;
    return true;
}

// ------------------------------------------------------------ pass A ----

template <typename T, int M>
__global__ void __launch_bounds__(Cfg<T, M>::ROW_THREADS) k_row_fwd(RowFwdArgs<T> a) {
    using C = cpx<T>;
    constexpr int E = Cfg<T, M>::E, G = Cfg<T, M>::G, RB = Cfg<T, M>::RB;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int t = threadIdx.x, j = t % G, c = t / G;
    const int L = a.L;
    const int iy = blockIdx.x * RB + c;
    const bool row_ok = iy < L;

    // CG scalars (read once; written only by other kernels)
    T alpha = 0, beta = 0;
    int first = 0;
    double inv_sigma = 1.0;
    if (a.mode == RF_CG) {
        first = a.st->first;
        alpha = (T)a.st->alpha;
        beta = (T)a.st->beta;
        if (a.r64) inv_sigma = 1.0 / a.st->sigma;
    }
    double sig = 0.0;
    if (a.mode == RF_XUPD) sig = a.st->sigma;  // scale of the inner run that produced d32

    C v[E];
    T acc = 0;  // partial r.r of this thread (short run, then FP64)
#pragma unroll
    for (int e = 0; e < E; ++e) {
        v[e] = C{0, 0};
        if (e < E / 2) {
            const int n = j + e * G;
            if (row_ok && n < L) {
                const size_t i = (size_t)iy * L + n;
                T val;
                if (a.mode == RF_PLAIN) {
                    val = a.x[i];
                } else if (a.mode == RF_XUPD) {
                    double xv = a.x64[i];
                    if (a.d32 && sig != 0.0) xv += sig * (double)a.d32[i];
                    if (a.mask && !a.mask[i]) xv = 0.0;
                    a.x64[i] = xv;
                    val = (T)xv;
                } else {  // RF_CG
                    T r, p;
                    if (first) {
                        if (a.r64) {
                            r = (T)(a.r64[i] * inv_sigma);
                            a.cr[i] = r;
                            a.cx[i] = 0;
                        } else {
                            r = a.cr[i];
                        }
                        p = r;
                    } else {
                        p = a.cp[i];
                        a.cx[i] = a.cx[i] + alpha * p;
                        r = a.cr[i] - alpha * a.cq[i];
                        a.cr[i] = r;
                        p = r + beta * p;
                    }
                    a.cp[i] = p;
                    acc += r * r;
                    val = p;
                }
                v[e].x = val;
            }
        }
    }
    fft_stages<T, M, false>(v, j, sm + c * seg_len(M), a.tw);
    if (row_ok) {
        C* zr = a.Z + (size_t)iy * M;
#pragma unroll
        for (int e = 0; e < E; ++e) stc(zr + j + e * G, v[e]);
    }
    if (a.mode == RF_CG) {
        double pv[1] = {(double)acc}, tot[1];
        if (grid_sum_last<1>(pv, a.part, &a.st->cntA, tot) && threadIdx.x == 0) a.st->rr = tot[0];
    }
}

// ------------------------------------------------------------ pass B ----

template <typename T, int M>
__global__ void __launch_bounds__(Cfg<T, M>::COL_THREADS) k_col_conv(ColArgs<T> a) {
    using C = cpx<T>;
    constexpr int E = Cfg<T, M>::E, G = Cfg<T, M>::G, CB = Cfg<T, M>::CB;
    constexpr int Q = M / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int t = threadIdx.x, c = t % CB, j = t / CB;
    const int L = a.L;
    const int kx = blockIdx.x * CB + c;
    const int fx = kx <= M / 2 ? kx : M - kx;

    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        v[e] = C{0, 0};
        const int n = j + e * G;
        if (e < E / 2 && n < L) v[e] = ldc_cg(a.Z + (size_t)n * M + kx);
    }
    C* seg = sm + c * seg_len(M);
    fft_stages<T, M, false>(v, j, seg, a.tw);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int ky = j + e * G;
        const int fy = ky <= M / 2 ? ky : M - ky;
        const T g = __ldg(a.Gq + (size_t)fy * Q + fx);
        v[e].x *= g;
        v[e].y *= g;
    }
    fft_stages<T, M, true>(v, j, seg, a.tw);
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
        const int n = j + e * G;
        if (n < L) stc(a.Z + (size_t)n * M + kx, v[e]);
    }
}

// ------------------------------------------------------------ pass C ----

template <typename T, int M>
__global__ void __launch_bounds__(Cfg<T, M>::ROW_THREADS) k_row_inv(RowInvArgs<T> a) {
    using C = cpx<T>;
    constexpr int E = Cfg<T, M>::E, G = Cfg<T, M>::G, RB = Cfg<T, M>::RB;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int t = threadIdx.x, j = t % G, c = t / G;
    const int L = a.L;
    const int iy = blockIdx.x * RB + c;
    const bool row_ok = iy < L;

    C v[E];
    if (row_ok) {
        const C* zr = a.Z + (size_t)iy * M;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = ldc_cg(zr + j + e * G);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = C{0, 0};
    }
    fft_stages<T, M, true>(v, j, sm + c * seg_len(M), a.tw);

    T s0 = 0, s1 = 0, s2 = 0;  // short per-thread runs, summed in FP64 below
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
        const int n = j + e * G;
        if (row_ok && n < L) {
            const size_t i = (size_t)iy * L + n;
            const T y = v[e].x;
            const bool act = a.mask == nullptr || a.mask[i] != 0;
            if (a.mode == RI_PLAIN) {
                a.y[i] = y;
            } else if (a.mode == RI_CG) {
                const T p = a.cp[i];
                const T q = act ? y + a.s[i] * p : (T)0;
                a.cq[i] = q;
                s0 += p * q;
                s1 += a.cr[i] * q;
                s2 += q * q;
            } else {  // RI_RESID (T = double)
                const double xv = a.x64[i];
                const double bv = act ? a.b64[i] : 0.0;
                const double r = act ? bv - ((double)y + a.s64[i] * xv) : 0.0;
                a.r64[i] = r;
                s0 += (T)(r * r);
                s1 += (T)(bv * bv);
            }
        }
    }
    if (a.mode == RI_CG) {
        double pv[3] = {(double)s0, (double)s1, (double)s2}, tot[3];
        if (grid_sum_last<3>(pv, a.part, &a.st->cntC, tot) && threadIdx.x == 0)
            cg_step_decide(a.st, tot[0], tot[1], tot[2], a.h_inner);
    } else if (a.mode == RI_RESID) {
        double pv[2] = {(double)s0, (double)s1}, tot[2];
        if (grid_sum_last<2>(pv, a.part, &a.st->cntC, tot) && threadIdx.x == 0)
            refine_decide(a.st, tot[0], tot[1], a.h_outer, a.h_inner);
    }
}

}  // namespace fc
