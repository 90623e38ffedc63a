// Persistent inner CG loop (Listing 2) for one solve: one cooperative launch
// runs every iteration of an inner run, the three FFT passes of each product
// being phases separated by grid-wide barriers.  This replaces three kernel
// launches per iteration by three barriers.
//
// Reductions need no extra barrier: each block publishes its partial sums,
// and after the barrier every block adds all blocks' partials in block order
// itself, so every block holds bitwise the same scalars and takes the same
// step decision (alpha = r.p/p.q, |r - alpha q|^2, beta, convergence).
#pragma once

#include "fc_passes.cuh"

namespace fc {

struct PersistCtl {
    unsigned count;  // blocks arrived at the current barrier
    unsigned gen;    // barrier generation
    int err;         // 1: a barrier wait ran out (the kernel returned early)
    int pad;
};

// Grid-wide barrier of a cooperative launch (all blocks resident).  The wait
// is bounded: after `limit` polls (2^24 by default, about two seconds) it
// sets ctl->err and returns.  Returns false in every thread once an error is
// flagged.
__device__ __forceinline__ bool grid_barrier(PersistCtl* ctl, unsigned limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &ctl->gen;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->count, 0u);
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
        } else {
            unsigned polls = 0;
            while (*vgen == gen) {
                if (++polls > limit) {
                    atomicExch(&ctl->err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = *(volatile int*)&ctl->err == 0;
    }
    __syncthreads();
    return ok != 0;
}

// Sum NV values per block over the whole grid in block order (every block
// computes the same result); valid in all threads on return.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* part, double (&tot)[NV], double (*scratch)[NV],
                                             double* bcast) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) acc += __ldcg(part + (size_t)b * NV + k);
        tot[k] = acc;
    }
    block_sum<NV>(tot, scratch);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) bcast[k] = tot[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = bcast[k];
}

// Publish this block's NV partial sums in slot blockIdx.x of part: FP32
// partials (each thread's Dot2 pair) as two-float pairs (two_sum / ff_add),
// FP64 ones as doubles.  scratch: the block's shared [32][NV] doubles
// (reused as float2 pairs).
template <int NV, typename T>
__device__ __forceinline__ void publish_partials(const Acc<T> (&v)[NV], double* part, double (*scratch)[NV]) {
    if constexpr (sizeof(T) == 4) {
        float hi[NV], lo[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            hi[k] = v[k].hi;
            lo[k] = v[k].lo;
        }
        block_sum_ff<NV>(hi, lo, reinterpret_cast<float2(*)[NV]>(scratch));
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                reinterpret_cast<float2*>(part)[(size_t)blockIdx.x * NV + k] = make_float2(hi[k], lo[k]);
    } else {
        double d[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) d[k] = v[k].value();
        block_sum<NV>(d, scratch);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) part[(size_t)blockIdx.x * NV + k] = d[k];
    }
}

// The grid totals of partials published by publish_partials<NV, T>, summed
// in block order by every block (FP64 results, valid in all threads).
template <int NV, typename T>
__device__ __forceinline__ void total_partials(const double* part, double (&tot)[NV], double (*scratch)[NV],
                                               double* bcast) {
    if constexpr (sizeof(T) == 4) {
        float hi[NV], lo[NV];
        const float2* pf = reinterpret_cast<const float2*>(part);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            hi[k] = 0.f;
            lo[k] = 0.f;
            for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
                const float2 q = __ldcg(pf + (size_t)b * NV + k);
                ff_add(hi[k], lo[k], q.x, q.y);
            }
        }
        block_sum_ff<NV>(hi, lo, reinterpret_cast<float2(*)[NV]>(scratch));
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) bcast[k] = (double)hi[k] + (double)lo[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = bcast[k];
    } else {
        sum_partials<NV>(part, tot, scratch, bcast);
    }
}

template <typename T>
struct PersistArgs {
    RowFwdArgs<T> A;
    ColArgs<T> B;
    RowInvArgs<T> C;
    int nA, nB;          // units of passes A and C (row pairs / RB) and B (columns / CB)
    double* partA;       // unused (pass A takes no sums)
    double* partC;       // [gridDim][5]
    PersistCtl* ctl;
    long N;              // L*L, for the final x += alpha p
};

template <typename T, int M, int EA, int RB, int EB, int CB>
__global__ void __launch_bounds__(RB*(M / EA)) k_cg_persist(PersistArgs<T> P) {
    static_assert(RB * (M / EA) == CB * (M / EB), "phases must use the whole block");
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
    __shared__ double scratch[32][5];
    __shared__ double bcast[5];
    CgState* st = P.A.st;
    if (st->finished) return;  // the outer loop has stopped: no inner run
    const unsigned limit = st->dbg_limit ? st->dbg_limit : (1u << 24);
    // test hook: the last block never arrives, the others' waits run out
    const bool leave = st->dbg_skip == 1 && gridDim.x > 1 && blockIdx.x == gridDim.x - 1;

    // the inner-run state, kept identical in every block
    int first = st->first;
    double alpha = st->alpha, beta = st->beta;
    const double bcarry = st->beta_carry;
    const double inv_sigma = P.A.r64 ? 1.0 / st->sigma : 1.0;
    const double tol2 = st->tol2;
    int iter = st->iter, cycle_iter = st->cycle_iter;
    const int max_iter = st->max_iter, cycle_max = st->cycle_max;
    double rr = 0.0, rp = 0.0;
    int d = 0;
    bool ok = true;

    while (true) {
        // phase A: CG update + pair-packed row FFTs
        const AScal<T> sc{first, (T)alpha, (T)beta, (T)(first ? bcarry : 0.0), inv_sigma, 0.0};
        for (int u = blockIdx.x; u < P.nA; u += gridDim.x) {
            rfwd_unit<T, M, EA, RB>(P.A, sc, u, sm);
            __syncthreads();
        }
        if (leave) return;
        if (!(ok = grid_barrier(P.ctl, limit))) break;
        // phase B: column FFT x spectrum x inverse
        for (int u = blockIdx.x; u < P.nB; u += gridDim.x) {
            colc_unit<T, M, EB, CB>(P.B, u, sm);
            __syncthreads();
        }
        if (!(ok = grid_barrier(P.ctl, limit))) break;
        // phase C: inverse row FFTs, q = P (C p + s p), partial p.q, r.q, q.q,
        // r.r, r.p
        Acc<T> s0, s1, s2, s3, s4;
        for (int u = blockIdx.x; u < P.nA; u += gridDim.x) {
            rinv_unit<T, M, EA, RB>(P.C, u, sm, s0, s1, s2, s3, s4);
            __syncthreads();
        }
        {
            const Acc<T> pv[5] = {s0, s1, s2, s3, s4};
            publish_partials<5, T>(pv, P.partC, scratch);
        }
        if (!(ok = grid_barrier(P.ctl, limit))) break;
        double tot[5];
        total_partials<5, T>(P.partC, tot, scratch, bcast);
        // the step decision of cg_step_decide, taken identically in every block
        const double pq = tot[0], rq = tot[1], qq = tot[2];
        rr = tot[3];
        rp = tot[4];
        alpha = rp / pq;
        double rrn = rr - 2.0 * alpha * rq + alpha * alpha * qq;
        if (rrn < 0.0) rrn = 0.0;
        d = 0;
        if (!(pq > 0.0) || !isfinite(alpha) || !isfinite(rrn)) {
            d = 3;
            alpha = 0.0;
        } else if (rrn <= tol2) {
            d = 1;
        }
        iter += 1;
        cycle_iter += 1;
        if (d == 0 && (iter >= max_iter || cycle_iter >= cycle_max)) d = 2;
        beta = rr > 0.0 ? rrn / rr : 0.0;
        first = 0;
        if (d) break;
    }
    if (ok) {
        // last step of the run: x += alpha p (the residual is recomputed outside)
        const T a = (T)alpha;
        T* x = P.A.cx;
        const T* p = P.A.cp;
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += (long)gridDim.x * blockDim.x)
            x[i] += a * p[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rr = rr;
        st->rp = rp;
        st->alpha = alpha;
        st->beta = beta;
        st->iter = iter;
        st->cycle_iter = cycle_iter;
        st->first = 0;
        st->inner_done = ok ? d : 4;
        if (!ok) st->status = FC_ETIMEOUT;
    }
}

}  // namespace fc
