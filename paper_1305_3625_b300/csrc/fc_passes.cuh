// The three HBM passes of one application of the coupling operator C
// (Listing 4's cpyComplex -> forward 2D FFT -> elementMult -> inverse 2D FFT
// -> cpyReal, Section 3) on the zero-padded M x M grid, with the CG vector
// work of Listing 2 fused into the first and last pass.
//
// The field is real, so its row transforms are Hermitian: two rows share one
// complex FFT (x_r + i x_{r+1}) and only the half spectrum kx in [0, M/2) is
// kept, with the two real values X[0] and X[M/2] packed into slot 0 as
// X[0] + i X[M/2].  The intermediate is stored column-major, Zt[kx][iy]
// (M/2 columns of L rows), so the column pass reads contiguous columns.
//
//   pass A (k_rfwd): per pair of data rows, form the input (plain x, or the
//       CG update x += a p, r -= a q, p = r + b p), FFT the zero-padded pair,
//       split it into the two rows' half spectra, store them column-major.
//   pass B (k_colc): per column kx < M/2, forward FFT of the L non-zero rows
//       along y, multiply by the real kernel spectrum, inverse FFT, keep rows
//       [0, L).  Column 0 carries the packed pair (kx = 0, kx = M/2) and is
//       split, multiplied and re-packed in the frequency domain.
//   pass C (k_rinv): per pair of rows, rebuild the full Hermitian spectra,
//       inverse FFT both rows in one complex transform, keep columns [0, L)
//       (the crop of cpyReal) and apply the epilogue: plain y = C x, the CG
//       product q = P (C p + s p) with p.q, r.q, q.q, or the true residual
//       r = P (b - C x - s x).
//
// The kernel spectrum is stored as its (M/2+1)^2 quarter Gq (the kernel is
// even in each coordinate and symmetric in x <-> y, so Ghat is real, even in
// each frequency and Ghat[ky][kx] = Ghat[kx][ky]).
#pragma once

#include "fc_fft.cuh"
#include "fc_internal.h"

namespace fc {

// Double-buffered exchanges when PER groups' two segments fit in 160 KB.
template <typename T, int M, int PER>
__host__ __device__ constexpr bool use_db() {
    return (size_t)PER * 2 * seg_len(M) * sizeof(cpx<T>) <= 160 * 1024;
}
template <typename T, int M, int PER, bool DB = use_db<T, M, PER>()>
__host__ __device__ constexpr size_t pass_smem() {
    return (size_t)PER * (DB ? 2 : 1) * seg_len(M) * sizeof(cpx<T>);
}

// ------------------------------------------- programmatic dependencies ---
//
// The passes may be launched as programmatic dependents of the previous pass
// (graph edges of programmatic type, or the stream attribute): each block
// waits until the previous grid has completed and its writes are visible
// before any global memory access, and signals the next pass once its own
// transform is done, so that the next pass's launch overlaps this pass's
// tail (its last blocks and the grid reduction).  Signalling at block entry
// instead measured slower inside the solve graphs.  Without a programmatic
// launch both are no-ops.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_leave() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
template <typename T>
__device__ __forceinline__ cpx<T> conjc(cpx<T> a) { return {a.x, -a.y}; }

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

// The grid's partials are added by one warp alone (strided runs, one warp
// tree): lane l adds blocks l, l + 32, l + 64, ... in that order, four
// blocks' values loaded at a time so that their L2 round trips overlap.
// Totals in lane 0.  FP64 partials (NV doubles per block).
template <int NV>
__device__ __forceinline__ void warp_sum_partials(const double* part, unsigned G, double (&tot)[NV]) {
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (unsigned b0 = threadIdx.x & 31; b0 < G; b0 += 128) {
        double q[4][NV];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                q[u][k] = b0 + 32 * u < G ? __ldcg(part + (size_t)(b0 + 32 * u) * NV + k) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                if (b0 + 32 * u < G) acc[k] += q[u][k];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], off);
        tot[k] = acc[k];
    }
}

// Publish this block's partial sums and, in the last block to finish, add
// all blocks' partials in block order.  Returns true (in every thread of the
// last block) with the totals in tot (valid in thread 0).  Deterministic:
// the reduction order depends only on the grid and block sizes.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* part, unsigned* cnt, double (&tot)[NV]) {
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
    // the grid's partials are added by warp 0 alone (strided runs, one warp
    // tree); lane l adds blocks l, l + 32, l + 64, ... in that order, four
    // blocks' values loaded at a time so that their L2 round trips overlap
    if (threadIdx.x < 32) {
        __threadfence();
        warp_sum_partials<NV>(part, gridDim.x, tot);
        if (threadIdx.x == 0) *cnt = 0u;
    }
    return true;
}

// Two-float sums for the FP32 passes.  FP64 arithmetic runs at a small
// fraction of the FP32 rate on this part: a tree of FP64 adds over a block's
// partial sums cost several microseconds per pass.  The per-thread partials
// are FP32 sums of at most 16 products; they are combined across the block
// and the grid as unevaluated pairs hi + lo of floats with error-free
// transformations (Knuth's TwoSum; relative error about 2^-47 per addition,
// against 2^-53 for an FP64 add), and the totals handed to the step
// decisions are FP64.

// s + e == a + b exactly (round-to-nearest adds, never contracted).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// (hi, lo) += (h, l) in two-float arithmetic.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float h, float l) {
    float sum, err;
    two_sum(hi, h, sum, err);
    err = __fadd_rn(err, __fadd_rn(lo, l));
    hi = __fadd_rn(sum, err);
    lo = __fsub_rn(err, __fsub_rn(hi, sum));
}

// Per-thread accumulator of a pass's dot products.  FP64 passes: an FP64
// sum.  FP32 passes: Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005): each product a*b is split
// exactly into its rounded value and its rounding error (one fma), the
// rounded values are summed with TwoSum, and both kinds of error collect in
// lo.  hi + lo is as accurate as the sum taken in twice the working
// precision and rounded, plus an error of order (n u)^2 of the sum of
// |a_i b_i| (n <= 16 products per thread), so the FP32 vectors' dot products
// reach the accuracy of FP64 accumulation without FP64 arithmetic.
template <typename T>
struct Acc {
    T v = 0;
    __device__ __forceinline__ void prod(T a, T b) { v = fma(a, b, v); }
    __device__ __forceinline__ void set(T x) { v = x; }
    __device__ __forceinline__ double value() const { return (double)v; }
};
template <>
struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        float s, t;
        two_sum(hi, p, s, t);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(t, e));
    }
    __device__ __forceinline__ void set(float x) {
        hi = x;
        lo = 0.f;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Sum NV two-float values over the block (fixed order: warp tree, then warp
// 0 over the warp sums).  Result valid in thread 0.  Whole warps only.
template <int NV>
__device__ __forceinline__ void block_sum_ff(float (&hi)[NV], float (&lo)[NV], float2 (*scratch)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float h = __shfl_down_sync(0xffffffffu, hi[k], off), l = __shfl_down_sync(0xffffffffu, lo[k], off);
            ff_add(hi[k], lo[k], h, l);
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp][k] = make_float2(hi[k], lo[k]);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float2 w = lane < nw ? scratch[lane][k] : make_float2(0.f, 0.f);
            hi[k] = w.x;
            lo[k] = w.y;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float h = __shfl_down_sync(0xffffffffu, hi[k], off);
                const float l = __shfl_down_sync(0xffffffffu, lo[k], off);
                ff_add(hi[k], lo[k], h, l);
            }
        }
    }
}

// warp_sum_partials for two-float partials (NV float2 per block, the room of
// NV doubles), added in the same order with ff_add; FP64 totals in lane 0.
template <int NV>
__device__ __forceinline__ void warp_sum_partials(const float2* pf, unsigned G, double (&tot)[NV]) {
    float hi[NV], lo[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        hi[k] = 0.f;
        lo[k] = 0.f;
    }
    for (unsigned b0 = threadIdx.x & 31; b0 < G; b0 += 128) {
        float2 q[4][NV];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                q[u][k] = b0 + 32 * u < G ? __ldcg(pf + (size_t)(b0 + 32 * u) * NV + k) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                if (b0 + 32 * u < G) ff_add(hi[k], lo[k], q[u][k].x, q[u][k].y);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float h = __shfl_down_sync(0xffffffffu, hi[k], off);
            const float l = __shfl_down_sync(0xffffffffu, lo[k], off);
            ff_add(hi[k], lo[k], h, l);
        }
        tot[k] = (double)hi[k] + (double)lo[k];
    }
}

// grid_sum_last for FP32 partials (each thread's Dot2 pair): the per-block
// sums are published as two-float pairs (part holds NV float2 per block, the
// room of NV doubles) and the last block's warp 0 adds them in block order
// the same way.  tot: the FP64 totals, valid in thread 0 of the last block.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(const Acc<float> (&v)[NV], double* part, unsigned* cnt,
                                              double (&tot)[NV]) {
    __shared__ float2 scratch[32][NV];
    __shared__ bool is_last;
    float hi[NV], lo[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        hi[k] = v[k].hi;
        lo[k] = v[k].lo;
    }
    block_sum_ff<NV>(hi, lo, scratch);
    float2* pf = reinterpret_cast<float2*>(part);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) pf[(size_t)blockIdx.x * NV + k] = make_float2(hi[k], lo[k]);
        __threadfence();
        unsigned prev = atomicAdd(cnt, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    if (threadIdx.x < 32) {
        __threadfence();
        warp_sum_partials<NV>(pf, gridDim.x, tot);
        if (threadIdx.x == 0) *cnt = 0u;
    }
    return true;
}

// grid_sum_last for FP64 partials held in accumulators.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(const Acc<double> (&a)[NV], double* part, unsigned* cnt,
                                              double (&tot)[NV]) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = a[k].v;
    return grid_sum_last<NV>(v, part, cnt, tot);
}

// Publish this block's partial sums only (in the layout of grid_sum_last):
// the pass that follows adds them up (grid_total), after this grid has
// completed, so no block waits for the others.
template <int NV>
__device__ __forceinline__ void grid_publish(const Acc<float> (&v)[NV], double* part) {
    __shared__ float2 scratch[32][NV];
    float hi[NV], lo[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        hi[k] = v[k].hi;
        lo[k] = v[k].lo;
    }
    block_sum_ff<NV>(hi, lo, scratch);
    float2* pf = reinterpret_cast<float2*>(part);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) pf[(size_t)blockIdx.x * NV + k] = make_float2(hi[k], lo[k]);
}
template <int NV>
__device__ __forceinline__ void grid_publish(const Acc<double> (&a)[NV], double* part) {
    __shared__ double scratch[32][NV];
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = a[k].v;
    block_sum<NV>(v, scratch);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(size_t)blockIdx.x * NV + k] = v[k];
}

// The totals of NV sums that G blocks of an earlier pass published, added in
// the order of grid_sum_last (the same values in every block that adds
// them).  Called by one warp; totals in lane 0.
template <typename T, int NV>
__device__ __forceinline__ void warp_total(const double* part, int G, double (&tot)[NV]) {
    if constexpr (sizeof(T) == 4)
        warp_sum_partials<NV>(reinterpret_cast<const float2*>(part), (unsigned)G, tot);
    else
        warp_sum_partials<NV>(part, (unsigned)G, tot);
}

// PCG step decisions in the pass A that consumes pass C's sums: warp 0 adds
// the published partials, thread 0 evaluates the decision (pcg_zr_eval for
// RF_PCG_P, pcg_alpha_eval for RF_PCG_R) and, in the committing block,
// commits it.  Returns the coefficient (beta or alpha) in every thread and
// false when the inner run has ended (RF_PCG_P: nothing to transform).
template <typename T>
__device__ __forceinline__ bool pcg_consume(int mode, CgState* st, const double* part, int G,
                                            unsigned long long h_inner, bool commit, T& coef) {
    __shared__ double s_coef;
    __shared__ int s_go;
    if (threadIdx.x < 32) {
        const PcgView sv = pcg_view(st);  // loaded with the partials (no dependency between them)
        if (mode == RF_PCG_P) {
            double tot[2];
            warp_total<T, 2>(part, G, tot);
            if (threadIdx.x == 0) {
                const PcgZr z = pcg_zr_eval(sv, tot[0], tot[1]);
                if (commit) pcg_zr_commit(st, z, tot[0], tot[1], h_inner);
                s_coef = z.beta;
                s_go = z.d == 0;
            }
        } else {
            double tot[1];
            warp_total<T, 1>(part, G, tot);
            if (threadIdx.x == 0) {
                const PcgAlpha al = pcg_alpha_eval(sv, tot[0]);
                if (commit) pcg_alpha_commit(st, al, tot[0]);
                s_coef = al.alpha;
                s_go = 1;
            }
        }
    }
    __syncthreads();
    coef = (T)s_coef;
    return s_go != 0;
}

// --------------------------------------------------- per-element input ---

// Block-uniform scalars of a pass-A unit (the CG step of the last product,
// or the scale of the correction folded into x).
template <typename T>
struct AScal {
    int first;
    T alpha, beta, bcarry;
    double inv_sigma, sig;
};

// Pass A's inputs of one thread: elements n = j + e*G (e < E/2; the rest is
// the zero padding) of rows r0 and r0 + 1, packed as v[e] = row r0 + i row
// r0+1.  The value transformed at each element is the plain input, the CG
// update of Listing 2 (x += a p, r -= a q, p = r + b p; on the first pass of
// a run p = r, or p = r + b' p_old when the direction is kept across a
// true-residual replacement), the PCG halves (x, r update and transform r;
// p = z + b p and transform p), or the FP64 iterate with the folded-in
// correction of the last inner run (masked).  The dot products of the new r
// and p are taken by pass C, which reads both again.  Each row's operands
// are all loaded before the first is used, so a thread waits for one memory
// round trip per row instead of one per element.  vo: the problem's offset
// in the vectors (batched launches).
template <typename T, int M, int E>
__device__ __forceinline__ void pass_a_inputs(int mode, const T* __restrict__ xin, T* __restrict__ cx,
                                              T* __restrict__ cr, T* __restrict__ cp, const T* __restrict__ cq,
                                              const T* __restrict__ cz, const double* __restrict__ r64,
                                              double* __restrict__ x64, const float* __restrict__ d32,
                                              const uint8_t* __restrict__ mask, const AScal<T>& sc, int j, int r0,
                                              int L, size_t vo, cpx<T> (&v)[E]) {
    constexpr int G = M / E, H = E / 2;  // n >= M/2 >= L for e >= E/2
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cpx<T>{0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (r0 + h >= L) continue;
        const size_t b = vo + (size_t)(r0 + h) * L + j;
        bool ok[H];
#pragma unroll
        for (int e = 0; e < H; ++e) ok[e] = j + e * G < L;
        T val[H];
#pragma unroll
        for (int e = 0; e < H; ++e) val[e] = 0;
        if (mode == RF_PLAIN) {
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) val[e] = xin[b + e * G];
        } else if (mode == RF_XUPD) {
            double xv[H];
            float dv[H];
            uint8_t mv[H];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    xv[e] = x64[b + e * G];
                    dv[e] = d32 ? d32[b + e * G] : 0.f;
                    mv[e] = mask ? mask[b + e * G] : (uint8_t)1;
                }
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    double t = xv[e];
                    if (d32 && sc.sig != 0.0) t = fma(sc.sig, (double)dv[e], t);
                    if (!mv[e]) t = 0.0;
                    x64[b + e * G] = t;
                    val[e] = (T)t;
                }
        } else if (sc.first && mode != RF_PCG_P) {  // a run starts: r from the true residual (or as kept)
            if (r64) {
                double rv[H];
#pragma unroll
                for (int e = 0; e < H; ++e)
                    if (ok[e]) rv[e] = r64[b + e * G];
#pragma unroll
                for (int e = 0; e < H; ++e)
                    if (ok[e]) {
                        val[e] = (T)mul_rn(rv[e], sc.inv_sigma);
                        cr[b + e * G] = val[e];
                        cx[b + e * G] = 0;
                    }
            } else {
#pragma unroll
                for (int e = 0; e < H; ++e)
                    if (ok[e]) val[e] = cr[b + e * G];
            }
            if (mode == RF_CG) {  // p = r, or r + b' p_old when the direction is kept
                if (sc.bcarry != (T)0) {
                    T pv[H];
#pragma unroll
                    for (int e = 0; e < H; ++e)
                        if (ok[e]) pv[e] = cp[b + e * G];
#pragma unroll
                    for (int e = 0; e < H; ++e)
                        if (ok[e]) val[e] = fma(sc.bcarry, pv[e], val[e]);
                }
#pragma unroll
                for (int e = 0; e < H; ++e)
                    if (ok[e]) cp[b + e * G] = val[e];
            }
        } else if (mode == RF_PCG_P) {  // p = z + beta p
            T zv[H], pv[H];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    zv[e] = cz[b + e * G];
                    pv[e] = sc.first ? (T)0 : cp[b + e * G];
                }
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    val[e] = sc.first ? zv[e] : fma(sc.beta, pv[e], zv[e]);
                    cp[b + e * G] = val[e];
                }
        } else {  // RF_CG, RF_PCG_R: x += alpha p, r -= alpha q (and p = r + beta p)
            T pv[H], xv[H], rv[H], qv[H];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    pv[e] = cp[b + e * G];
                    xv[e] = cx[b + e * G];
                    rv[e] = cr[b + e * G];
                    qv[e] = cq[b + e * G];
                }
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    const T r = fma(-sc.alpha, qv[e], rv[e]);
                    cx[b + e * G] = fma(sc.alpha, pv[e], xv[e]);
                    cr[b + e * G] = r;
                    if (mode == RF_CG) {
                        val[e] = fma(sc.beta, pv[e], r);
                        cp[b + e * G] = val[e];
                    } else {
                        val[e] = r;
                    }
                }
        }
#pragma unroll
        for (int e = 0; e < H; ++e) {
            if (h == 0)
                v[e].x = val[e];
            else
                v[e].y = val[e];
        }
    }
}

// ------------------------------------------------------------ pass A ----

template <typename T>
__device__ __forceinline__ AScal<T> ascal_from_state(const RowFwdArgs<T>& a, const CgState* st) {
    AScal<T> sc{0, 0, 0, 0, 1.0, 0.0};
    if (a.mode == RF_CG || a.mode == RF_PCG_R || a.mode == RF_PCG_P) {
        sc.first = st->first;
        sc.alpha = (T)st->alpha;
        sc.beta = (T)st->beta;
        sc.bcarry = a.mode == RF_CG ? (T)st->beta_carry : (T)0;
        if (a.r64) sc.inv_sigma = 1.0 / st->sigma;
    } else if (a.mode == RF_XUPD) {
        sc.sig = st->sigma;  // scale of the inner run that produced d32
    }
    return sc;
}

// The transform half of a pass-A unit: FFT of the packed row pairs v, split
// into the two rows' half spectra, column-major store at offset zo.
template <typename T, int M, int E, int RB, bool DB = use_db<T, M, RB>()>
__device__ __forceinline__ void rfwd_transform(const RowFwdArgs<T>& a, cpx<T> (&v)[E], int unit, cpx<T>* sm,
                                               size_t zo) {
    using C = cpx<T>;
    constexpr int G = M / E, H = M / 2, NT = RB * G, SEG = seg_len(M);
    constexpr int GS = (DB ? 2 : 1) * SEG;  // shared elements per pair
    constexpr int NB = next_buf(M, E, DB, 0);
    const int t = threadIdx.x, j = t % G, pl = t / G;
    const int L = a.L;
    C* g0 = sm + pl * GS;
    fft_stages<T, M, E, false, DB, 0, 1, true>(v, j, g0, g0 + SEG, a.tw);
    C* wp = g0 + NB * SEG + spad(j);
#pragma unroll
    for (int e = 0; e < E; ++e) wp[pofs(e * G)] = v[e];
    __syncthreads();
    // split the pair into the two rows' half spectra, store column-major
    const int row_base = unit * 2 * RB;
    const T half = (T)0.5;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int idx = t + q * NT;
        const int r = idx % (2 * RB), kx = idx / (2 * RB);
        const int row = row_base + r;
        const C* sg = sm + (r >> 1) * GS + NB * SEG;
        C out;
        if (kx == 0) {
            const C z0 = sg[spad(0)], zh = sg[spad(H)];
            out = (r & 1) ? C{z0.y, zh.y} : C{z0.x, zh.x};
        } else {
            const C z = sg[spad(kx)], zc = sg[spad(M - kx)];
            out = (r & 1) ? C{(z.y + zc.y) * half, (zc.x - z.x) * half} : C{(z.x + zc.x) * half, (z.y - zc.y) * half};
        }
        if (row < L) stc(a.Z + zo + (size_t)kx * L + row, out);
    }
}

// One unit of pass A: RB row pairs starting at pair unit*RB, G = M/E threads
// per pair.  Leaves shared memory in use: the caller synchronises before the
// block reuses it.  vo, zo: the problem's offsets in the vectors and the
// intermediate.
// MODE >= 0: the mode fixed at compile time (the other modes' code is not
// emitted).
template <typename T, int M, int E, int RB, bool DB = use_db<T, M, RB>(), int MODE = -1>
__device__ __forceinline__ void rfwd_unit(const RowFwdArgs<T>& a, const AScal<T>& sc, int unit, cpx<T>* sm,
                                          size_t vo = 0, size_t zo = 0) {
    constexpr int G = M / E;
    const int t = threadIdx.x, j = t % G, pl = t / G;
    const int r0 = (unit * RB + pl) * 2;
    cpx<T> v[E];
    pass_a_inputs<T, M, E>(MODE >= 0 ? MODE : a.mode, a.x, a.cx, a.cr, a.cp, a.cq, a.cz, a.r64, a.x64, a.d32, a.mask,
                           sc, j, r0, a.L, vo, v);
    rfwd_transform<T, M, E, RB, DB>(a, v, unit, sm, zo);
}

// Whether a pass A takes a PCG step decision from the last pass C's
// published sums (a.npart blocks; none: the coefficients as the state holds
// them): RF_PCG_P always (beta, the stopping test), RF_PCG_R after the first
// update of a run (alpha).
template <typename T>
__device__ __forceinline__ bool pcg_decides(const RowFwdArgs<T>& a, const AScal<T>& sc) {
    return a.npart > 0 && (a.mode == RF_PCG_P || (a.mode == RF_PCG_R && !sc.first));
}

// A pass-A unit in a PCG mode that takes the step decision: each thread's
// operands (both rows) are loaded first, so that their memory round trip
// overlaps the one of the published sums; then the update with the decided
// coefficient (RF_PCG_R: x += alpha p, r -= alpha q, transform r; RF_PCG_P:
// p = z + beta p, transform p) and the transform.  Returns false, having
// written nothing, when the decision ends the run.
template <typename T, int M, int E, int RB, bool DB = use_db<T, M, RB>()>
__device__ __forceinline__ bool rfwd_unit_pcg(const RowFwdArgs<T>& a, const AScal<T>& sc, int unit, cpx<T>* sm,
                                              CgState* st, const double* part, bool commit,
                                              unsigned long long h_inner, size_t vo = 0, size_t zo = 0) {
    constexpr int G = M / E, H = E / 2;
    const int t = threadIdx.x, j = t % G, pl = t / G;
    const int L = a.L;
    const int r0 = (unit * RB + pl) * 2;
    const bool upd_r = a.mode == RF_PCG_R;
    T o0[2][H], o1[2][H], o2[2][H], o3[2][H];  // RF_PCG_R: p, x, r, q; RF_PCG_P: z, p
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const size_t b = vo + (size_t)(r0 + h) * L + j;
#pragma unroll
        for (int e = 0; e < H; ++e) {
            o0[h][e] = o1[h][e] = o2[h][e] = o3[h][e] = (T)0;
            if (r0 + h < L && j + e * G < L) {
                if (upd_r) {
                    o0[h][e] = a.cp[b + e * G];
                    o1[h][e] = a.cx[b + e * G];
                    o2[h][e] = a.cr[b + e * G];
                    o3[h][e] = a.cq[b + e * G];
                } else {
                    o0[h][e] = a.cz[b + e * G];
                    if (!sc.first) o1[h][e] = a.cp[b + e * G];
                }
            }
        }
    }
    T coef;
    if (!pcg_consume<T>(a.mode, st, part, a.npart, h_inner, commit, coef)) return false;
    cpx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cpx<T>{0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const size_t b = vo + (size_t)(r0 + h) * L + j;
#pragma unroll
        for (int e = 0; e < H; ++e) {
            if (!(r0 + h < L && j + e * G < L)) continue;
            T val;
            if (upd_r) {
                val = fma(-coef, o3[h][e], o2[h][e]);
                a.cx[b + e * G] = fma(coef, o0[h][e], o1[h][e]);
                a.cr[b + e * G] = val;
            } else {
                val = sc.first ? o0[h][e] : fma(coef, o1[h][e], o0[h][e]);
                a.cp[b + e * G] = val;
            }
            if (h == 0)
                v[e].x = val;
            else
                v[e].y = val;
        }
    }
    rfwd_transform<T, M, E, RB, DB>(a, v, unit, sm, zo);
    return true;
}

// MINB: blocks per SM the register allocation must allow; DB: double-buffered
// exchanges (default: when they fit, see use_db).
template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
__global__ void __launch_bounds__(RB*(M / E), MINB) k_rfwd(const RowFwdArgs<T> a) {
    static_assert((RB * (M / E)) % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_enter();
    if (a.mode == RF_XUPD && a.st->warm) return;  // residual already updated: no product
    if (a.mode == RF_PCG_P && a.st->idle) return;  // PCG: the run has ended
    const AScal<T> sc = ascal_from_state(a, a.st);
    rfwd_unit<T, M, E, RB, DB>(a, sc, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw));
    pdl_leave();
}

// The single-problem pass A of the PCG loop (RF_PCG_R, RF_PCG_P), which
// takes the step decision from the last pass C's published sums (pcg_decides,
// rfwd_unit_pcg).  A kernel of its own: the early loads of its operands make
// its code much larger than k_rfwd's, and k_rfwd in the plain apply then
// stalled on instruction fetch.
template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
__global__ void __launch_bounds__(RB*(M / E), MINB) k_rfwd_pcg(const RowFwdArgs<T> a) {
    static_assert((RB * (M / E)) % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_enter();
    if (a.mode == RF_PCG_P && a.st->idle) return;  // the run has ended
    const AScal<T> sc = ascal_from_state(a, a.st);
    if (pcg_decides(a, sc)) {
        if (!rfwd_unit_pcg<T, M, E, RB, DB>(a, sc, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw), a.st, a.part,
                                            blockIdx.x == 0, a.h_inner))
            return;
    } else {
        rfwd_unit<T, M, E, RB, DB>(a, sc, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw));
    }
    pdl_leave();
}

// Pass A of the plain apply y = C x (RF_PLAIN only: a kernel of its own with
// none of the other modes' code, which made the general kernel's
// instruction footprint larger).
template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
__global__ void __launch_bounds__(RB*(M / E), MINB) k_rfwd_plain(const RowFwdArgs<T> a) {
    static_assert((RB * (M / E)) % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_enter();
    const AScal<T> sc{0, 0, 0, 0, 1.0, 0.0};
    rfwd_unit<T, M, E, RB, DB, RF_PLAIN>(a, sc, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw));
    pdl_leave();
}

// The batched form: problem blockIdx.y at the strides of bb, gated.
template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
__global__ void __launch_bounds__(RB*(M / E), MINB) k_rfwd_b(const RowFwdArgs<T> a, const BatchArgs bb) {
    static_assert((RB * (M / E)) % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    CgState* const st = a.st + blockIdx.y;
    pdl_enter();
    if (bb.gate && gate_closed(st, bb.gate)) return;
    if (a.mode == RF_XUPD && st->warm) return;
    AScal<T> sc = ascal_from_state(a, st);
    // the decision first, then the unit: with many problems' blocks resident
    // the loads' latency hides behind other blocks, and the registers that
    // early loads would hold cost resident blocks (the arithmetic is the same)
    if (pcg_decides(a, sc)) {
        T coef;
        if (!pcg_consume<T>(a.mode, st, a.part + (size_t)blockIdx.y * bb.bs.part, a.npart, 0, blockIdx.x == 0, coef))
            return;
        if (a.mode == RF_PCG_P)
            sc.beta = coef;
        else
            sc.alpha = coef;
    }
    rfwd_unit<T, M, E, RB, DB>(a, sc, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw), (size_t)blockIdx.y * bb.bs.n,
                               (size_t)blockIdx.y * bb.bs.z);
    pdl_leave();
}

// ------------------------------------------------------------ pass B ----

// One unit of pass B: CB columns starting at column unit*CB, G = M/E threads
// per column (j fastest).  Unit 0 holds the packed column 0.  zo, qo: the
// problem's offsets in the intermediate and the spectrum.
// GB: the transforms' exchanges synchronise each column's threads alone
// (named barriers), so that the block's columns need not keep step.
template <typename T, int M, int E, int CB, bool DB = use_db<T, M, CB>(), bool GB = false>
__device__ __forceinline__ void colc_unit(const ColArgs<T>& a, int unit, cpx<T>* sm, size_t zo = 0, size_t qo = 0) {
    using C = cpx<T>;
    constexpr int G = M / E, H = M / 2, Q = M / 2 + 1, SEG = seg_len(M);
    constexpr int GS = (DB ? 2 : 1) * SEG;
    constexpr int NB = next_buf(M, E, DB, 0);
    const int t = threadIdx.x, j = t % G, c = t / G;
    const int L = a.L;
    const int kx = unit * CB + c;
    C* col = a.Z + zo + (size_t)kx * L;
    const T* const Gq = a.Gq + qo;

    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int n = j + e * G;
        v[e] = (e < E / 2 && n < L) ? ldc_cg(col + n) : C{0, 0};
    }
    C* g0 = sm + c * GS;
    fft_stages<T, M, E, false, DB, 0, 1, true, GB>(v, j, g0, g0 + SEG, a.tw);
    if (unit == 0) {
        // column 0 holds P = F0 + i FN (kx = 0 and kx = M/2, both real along y);
        // with the Hermitian partner P[M - ky]: W = P (g0 + gN)/2 + conj(P[M-ky]) (g0 - gN)/2
        C* seg = g0 + NB * SEG;
#pragma unroll
        for (int e = 0; e < E; ++e) seg[spad(j + e * G)] = v[e];
        __syncthreads();
        if (c == 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ky = j + e * G;
                const int fy = ky <= H ? ky : M - ky;
                const C pc = conjc(seg[spad((M - ky) & (M - 1))]);
                const T g0 = __ldg(Gq + fy), gN = __ldg(Gq + (size_t)H * Q + fy);
                const T sp = (g0 + gN) * (T)0.5, sd = (g0 - gN) * (T)0.5;
                v[e] = C{fma(v[e].x, sp, mul_rn(pc.x, sd)), fma(v[e].y, sp, mul_rn(pc.y, sd))};
            }
        } else {
            const T* gk = Gq + (size_t)kx * Q;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ky = j + e * G;
                const T g = __ldg(gk + (ky <= H ? ky : M - ky));
                v[e].x *= g;
                v[e].y *= g;
            }
        }
        __syncthreads();
    } else {
        const T* gk = Gq + (size_t)kx * Q;  // Ghat[ky][kx] = Ghat[kx][ky]: contiguous in ky
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ky = j + e * G;
            const T g = __ldg(gk + (ky <= H ? ky : M - ky));
            v[e].x *= g;
            v[e].y *= g;
        }
    }
    fft_stages<T, M, E, true, DB, NB, 1, false, GB>(v, j, g0, g0 + SEG, a.tw);
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
        const int n = j + e * G;
        if (n < L) stc(col + n, v[e]);
    }
}

template <typename T, int M, int E, int CB, int MINB = 1, bool DB = use_db<T, M, CB>(), bool GB = false>
__global__ void __launch_bounds__(CB*(M / E), MINB) k_colc(const ColArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_enter();
    if (a.gate && gate_closed(a.st, a.gate)) return;
    if (a.pcg_commit && blockIdx.x == 0 && threadIdx.x == 0) pcg_rz_commit(a.st);
    colc_unit<T, M, E, CB, DB, GB>(a, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw));
    pdl_leave();
}

template <typename T, int M, int E, int CB, int MINB = 1, bool DB = use_db<T, M, CB>(), bool GB = false>
__global__ void __launch_bounds__(CB*(M / E), MINB) k_colc_b(const ColArgs<T> a, const BatchArgs bb) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_enter();
    if ((a.gate | bb.gate) && gate_closed(a.st + blockIdx.y, a.gate | bb.gate)) return;
    if (a.pcg_commit && blockIdx.x == 0 && threadIdx.x == 0) pcg_rz_commit(a.st + blockIdx.y);
    colc_unit<T, M, E, CB, DB, GB>(a, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw), (size_t)blockIdx.y * bb.bs.z,
                                   (size_t)blockIdx.y * bb.bs.q);
    pdl_leave();
}

// ------------------------------------------------------------ pass C ----

// Pass C's outputs of one thread: elements n = j + e*G < L (e < E/2, the
// crop) of rows r0 (v[e].x) and r0 + 1 (v[e].y), through the epilogue of the
// mode: the plain output; the CG product q = P (C p + s p) with the dot
// products the CG step takes (s0..s4: p.q, r.q, q.q and, of the r and p pass
// A formed, r.r and r.p); the PCG product q with p.q (s0); the
// preconditioned residual z (s0: r.z, s1: r.r); or the FP64 true residual
// r = P (b - C x - s x) (s0: r.r, s1: (P b).(P b)).  Each
// row's operands are all loaded before the first is used.  vo: the
// problem's vector offset.
template <typename T, int M, int E>
__device__ __forceinline__ void pass_c_outputs(int mode, T* __restrict__ y, const T* __restrict__ s,
                                               const T* __restrict__ cp, const T* __restrict__ cr,
                                               T* __restrict__ cq, T* __restrict__ cz,
                                               const uint8_t* __restrict__ mask, const double* __restrict__ x64,
                                               const double* __restrict__ b64, const double* __restrict__ s64,
                                               double* __restrict__ r64, int j, int r0, int L, size_t vo,
                                               const cpx<T> (&v)[E], Acc<T>& s0, Acc<T>& s1, Acc<T>& s2,
                                               Acc<T>& s3, Acc<T>& s4) {
    constexpr int G = M / E, H = E / 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (r0 + h >= L) continue;
        const size_t b = vo + (size_t)(r0 + h) * L + j;
        bool ok[H];
        T yv[H];
        uint8_t act[H];
#pragma unroll
        for (int e = 0; e < H; ++e) {
            ok[e] = j + e * G < L;
            yv[e] = h == 0 ? v[e].x : v[e].y;
            act[e] = 1;
        }
        if (mode == RI_PLAIN) {
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) y[b + e * G] = yv[e];
            continue;
        }
        if (mask) {
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) act[e] = mask[b + e * G];
        }
        if (mode == RI_CG) {
            T pv[H], rv[H], sv[H];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    pv[e] = cp[b + e * G];
                    rv[e] = cr[b + e * G];
                    sv[e] = s[b + e * G];
                }
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    const T q = act[e] ? fma(sv[e], pv[e], yv[e]) : (T)0;
                    cq[b + e * G] = q;
                    s0.prod(pv[e], q);
                    s1.prod(rv[e], q);
                    s2.prod(q, q);
                    s3.prod(rv[e], rv[e]);
                    s4.prod(rv[e], pv[e]);
                }
        } else if (mode == RI_PQ) {
            T pv[H], sv[H];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    pv[e] = cp[b + e * G];
                    sv[e] = s[b + e * G];
                }
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    const T q = act[e] ? fma(sv[e], pv[e], yv[e]) : (T)0;
                    cq[b + e * G] = q;
                    s0.prod(pv[e], q);
                }
        } else if (mode == RI_PCG_Z) {
            T rv[H];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) rv[e] = cr[b + e * G];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    const T z = act[e] ? yv[e] : (T)0;
                    cz[b + e * G] = z;
                    s0.prod(rv[e], z);
                    s1.prod(rv[e], rv[e]);
                }
        } else {  // RI_RESID (T = double)
            double xv[H], bv[H], sv[H];
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    xv[e] = x64[b + e * G];
                    bv[e] = b64[b + e * G];
                    sv[e] = s64[b + e * G];
                }
#pragma unroll
            for (int e = 0; e < H; ++e)
                if (ok[e]) {
                    const double bb = act[e] ? bv[e] : 0.0;
                    const double r = act[e] ? bb - fma(sv[e], xv[e], (double)yv[e]) : 0.0;
                    r64[b + e * G] = r;
                    s0.prod((T)r, (T)r);
                    s1.prod((T)bb, (T)bb);
                }
        }
    }
}

// One unit of pass C: RB row pairs starting at pair unit*RB.  Adds this
// thread's partial sums to s0 .. s4.  vo, zo: the problem's offsets.
template <typename T, int M, int E, int RB, bool DB = use_db<T, M, RB>(), int MODE = -1>
__device__ __forceinline__ void rinv_unit(const RowInvArgs<T>& a, int unit, cpx<T>* sm, Acc<T>& s0, Acc<T>& s1,
                                          Acc<T>& s2, Acc<T>& s3, Acc<T>& s4, size_t vo = 0, size_t zo = 0) {
    using C = cpx<T>;
    constexpr int G = M / E, H = M / 2, NT = RB * G, SEG = seg_len(M);
    constexpr int GS = (DB ? 2 : 1) * SEG;
    constexpr int HS = H + (H >> 4) + 1;  // staging: second row of a pair at an odd bank offset
    const int t = threadIdx.x, j = t % G, pl = t / G;
    const int L = a.L;
    const int row_base = unit * 2 * RB;
    const int r0 = row_base + 2 * pl;

    // the 2*RB rows' half spectra (column-major) into the pair segments
    // (buffer 0): row 2p at st(0, kx), row 2p+1 at st(1, kx), st(h, kx) =
    // h*HS + spad(kx)
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int idx = t + q * NT;
        const int r = idx % (2 * RB), kx = idx / (2 * RB);
        const int row = row_base + r;
        const C y = row < L ? ldc_cg(a.Z + zo + (size_t)kx * L + row) : C{0, 0};
        sm[(r >> 1) * GS + (r & 1) * HS + spad(kx)] = y;
    }
    __syncthreads();
    // Hermitian extension of both rows and pair packing W = Y0 + i Y1
    C* g0 = sm + pl * GS;
    const C* h0 = g0;
    const C* h1 = g0 + HS;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = j + e * G;
        C y0, y1;
        if (k == 0) {
            y0 = C{h0[0].x, 0};
            y1 = C{h1[0].x, 0};
        } else if (k == H) {
            y0 = C{h0[0].y, 0};
            y1 = C{h1[0].y, 0};
        } else if (k < H) {
            y0 = h0[spad(k)];
            y1 = h1[spad(k)];
        } else {
            y0 = conjc(h0[spad(M - k)]);
            y1 = conjc(h1[spad(M - k)]);
        }
        v[e] = C{y0.x - y1.y, y0.y + y1.x};
    }
    if constexpr (!DB) __syncthreads();
    // with two buffers the first exchange writes buffer 1 while buffer 0 is still being read
    fft_stages<T, M, E, true, DB, DB ? 1 : 0>(v, j, g0, g0 + SEG, a.tw);
    pass_c_outputs<T, M, E>(MODE >= 0 ? MODE : a.mode, a.y, a.s, a.cp, a.cr, a.cq, a.cz, a.mask, a.x64, a.b64, a.s64,
                            a.r64, j, r0, L, vo, v, s0, s1, s2, s3, s4);
}

// Pass C's grid sums and step decisions (last block; the PCG modes only
// publish their partials for the next pass A).  warm (RI_RESID): the
// residual and its sums were updated in place, and block 0 alone hands them on.
template <typename T>
__device__ __forceinline__ void rinv_sums(const RowInvArgs<T>& a, double* part, CgState* st, const Acc<T>& s0,
                                          const Acc<T>& s1, const Acc<T>& s2, const Acc<T>& s3, const Acc<T>& s4) {
    if (a.mode == RI_CG) {
        const Acc<T> pv[5] = {s0, s1, s2, s3, s4};
        double tot[5];
        if (grid_sum_last<5>(pv, part, &st->cntC, tot) && threadIdx.x == 0)
            cg_step_decide(st, tot[0], tot[1], tot[2], tot[3], tot[4], a.h_inner);
    } else if (a.mode == RI_RESID) {
        double pv[2] = {s0.value(), s1.value()}, tot[2];
        if (grid_sum_last<2>(pv, part, &st->cntC, tot) && threadIdx.x == 0) {
            refine_decide(st, tot[0], tot[1], a.h_outer, a.h_inner);
            st->warm = 0;  // every block has read it: later cycles recompute the residual
        }
    } else if (a.mode == RI_PCG_Z) {  // the next pass A decides (pcg_step)
        const Acc<T> pv[2] = {s0, s1};
        grid_publish<2>(pv, part);
    } else if (a.mode == RI_PQ) {
        const Acc<T> pv[1] = {s0};
        grid_publish<1>(pv, part);
    }
}

template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
__global__ void __launch_bounds__(RB*(M / E), MINB) k_rinv(const RowInvArgs<T> a) {
    static_assert((RB * (M / E)) % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_enter();
    if (a.mode == RI_PQ && a.st->idle) return;  // PCG: the z pass ended the run
    Acc<T> s0, s1, s2, s3, s4;  // short per-thread runs (FP64, or Dot2 pairs in FP32)
    // warm residual: r64 and its sums (rr64, bb) are already in place, and
    // block 0 alone hands them to the decision
    const bool warm = a.mode == RI_RESID && a.st->warm;
    if (!warm) {
        rinv_unit<T, M, E, RB, DB>(a, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw), s0, s1, s2, s3, s4);
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
        s0.set((T)a.st->rr64);
        s1.set((T)a.st->bb);
    }
    pdl_leave();
    rinv_sums(a, a.part, a.st, s0, s1, s2, s3, s4);
}

// Pass C of the plain apply (RI_PLAIN only, no sums), as k_rfwd_plain.
template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
__global__ void __launch_bounds__(RB*(M / E), MINB) k_rinv_plain(const RowInvArgs<T> a) {
    static_assert((RB * (M / E)) % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_enter();
    Acc<T> s0, s1, s2, s3, s4;
    rinv_unit<T, M, E, RB, DB, RI_PLAIN>(a, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw), s0, s1, s2, s3, s4);
    pdl_leave();
}

// The batched form: problem blockIdx.y at the strides of bb, gated.
template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
__global__ void __launch_bounds__(RB*(M / E), MINB) k_rinv_b(const RowInvArgs<T> a, const BatchArgs bb) {
    static_assert((RB * (M / E)) % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    CgState* const st = a.st + blockIdx.y;
    pdl_enter();
    if (bb.gate && gate_closed(st, bb.gate)) return;
    Acc<T> s0, s1, s2, s3, s4;
    const bool warm = a.mode == RI_RESID && st->warm;
    if (!warm) {
        rinv_unit<T, M, E, RB, DB>(a, blockIdx.x, reinterpret_cast<cpx<T>*>(smraw), s0, s1, s2, s3, s4,
                                   (size_t)blockIdx.y * bb.bs.n, (size_t)blockIdx.y * bb.bs.z);
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
        s0.set((T)st->rr64);
        s1.set((T)st->bb);
    }
    pdl_leave();
    rinv_sums(a, a.part + blockIdx.y * bb.bs.part, st, s0, s1, s2, s3, s4);
}

}  // namespace fc
