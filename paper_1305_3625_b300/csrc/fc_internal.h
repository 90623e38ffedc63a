// Internal device-side state and kernel argument blocks of the fftconv
// library.  Not part of the C ABI (include/fftconv.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fftconv.h"

namespace fc {

template <typename T>
struct cpx;

// Scalars of one solve, resident in device memory.  Each field is written by
// one thread of a pass.  A pass whose blocks all evaluate a step decision
// (the PCG passes A, see pcg_zr_eval) reads only fields that no block of it
// writes, or whose new value leads every block to the same decision.
struct CgState {
    double rr;           // r.r of the current inner residual (pass C's direct sum)
    double rp;           // r.p of the current residual and direction (pass C)
    double alpha, beta;  // CG step length and direction update of the last product
    double tol2;         // inner stop: recursive r.r <= tol2
    double sigma;        // norm of the true residual the inner run started from
    double rr64, bb;     // last true residual r.r and masked b.b (FP64)
    double rtol2;        // target: rr64 <= rtol2 * bb
    double inner_rtol2;  // mixed: inner target relative to the unit right-hand side
    double inner_goal2;  // mixed: an inner run may also stop at this fraction (squared) of
                         // the outer target (0: never)
    double beta_carry;   // direction kept across a true-residual replacement (0: restart)
    double rz, rz_prev;  // PCG: r.z of the current and of the previous iteration
    double rz_next;      // PCG: r.z just decided on, moved into rz by the next column pass
    double pshift;       // PCG: shift c of the preconditioner (C_M + c I)^-1
    int iter;            // products spent in inner loops (all cycles)
    int max_iter;
    int cycle_iter, cycle_max;
    int cycles, max_cycles;  // true-residual evaluations
    int first;               // 1: the next pass A starts a new inner run (p = r)
    int inner_done;          // 0 running, 1 converged, 2 cap reached, 3 breakdown, 4 barrier timeout
    int status;              // FC_OK, FC_ENOCONV, FC_ENANINF or FC_ETIMEOUT once finished
    int mixed;               // 1: inner runs in FP32 on the scaled residual
    int finished;
    // Warm-start residual update (a solve that follows another on the same
    // plan with the same s and b): the check kernel counts the changed
    // entries of x and flags a changed s, b or a grown active set; the update
    // kernel then sets warm, which makes the first residual passes A, B, C
    // skip their products (pass C takes rr64 and bb as given and clears warm).
    int warm;
    int warm_used;       // 1: this solve's first true residual was updated, not recomputed
    int wbad;            // the update does not apply (s or b changed, active set grew)
    unsigned wcount;     // entries of x that changed (the list holds the first kWarmMax)
    int s_check;         // 1: the warm check compares s with the last solve's (its FP32 copy is kept)
    int s_diff;          // the warm check found s changed (the FP32 copy is made anew)
    int tma_err;         // 1: a staged TMA copy never arrived (the solve ends with FC_ETIMEOUT)
    int idle;            // 1: no inner run is in progress (batched solves: the inner passes skip
                         // this problem)
    unsigned cntA, cntC;  // last-block counters of passes A and C
    double pq, rq, qq;    // grid sums of the last CG product's pass C (p.q, r.q, q.q)
    // test hooks (fc_debug_inject): 1 = the persistent kernel's last block
    // leaves before its first grid-barrier arrival, 2 = the TMA pass C issues
    // no copy for each block's first row pair; dbg_limit: polls a bounded
    // wait takes before it gives up (0: the default)
    unsigned dbg_skip, dbg_limit;
};

// Largest number of changed iterate entries the residual update takes.
constexpr int kWarmMax = 32;

// Gates of the passes of a batched solve (several problems of one size per
// launch, blockIdx.y = problem): a block returns at entry, before any work
// or reduction, when its problem's state says so.  Every block of a problem
// reads the same value: the fields are written by the last block of a pass
// only, after all blocks of that pass have arrived, or by an earlier kernel.
enum { GATE_WARM = 1, GATE_FINISHED = 2, GATE_IDLE = 4 };

__device__ __forceinline__ bool gate_closed(const CgState* st, int gate) {
    return ((gate & GATE_WARM) && st->warm) || ((gate & GATE_FINISHED) && st->finished) ||
           ((gate & GATE_IDLE) && st->idle);
}

// Per-problem strides of a batched launch (elements).  The batched kernels
// add them as index offsets (problem blockIdx.y), so a pointer argument
// keeps its meaning as a mode flag when null.  They travel in a second kernel
// parameter: widening the pass argument blocks themselves changed the
// register allocation of the single-problem kernels (spills in the
// 64-register shapes).
struct BatchStride {
    long n;     // L*L vectors (x, r, p, q, z, s, b, mask)
    long z;     // complex elements of the intermediate
    long q;     // spectrum quarter (0: one spectrum shared by all problems)
    long part;  // doubles of partial sums
};
struct BatchArgs {
    int gate;   // GATE_* bits
    BatchStride bs;
};

// Pass A modes: plain input; CG update (x, r, p) + transform p; FP64 iterate
// with the folded correction; PCG first half (x, r update, transform r);
// PCG second half (p = z + beta p, transform p).
enum { RF_PLAIN = 0, RF_CG = 1, RF_XUPD = 2, RF_PCG_R = 3, RF_PCG_P = 4 };
// Pass C modes: plain output; CG product q (five sums); FP64 true residual;
// PCG preconditioned residual z = P M^-1 r (sums r.z, r.r); PCG product q
// (sum p.q).
enum { RI_PLAIN = 0, RI_CG = 1, RI_RESID = 2, RI_PCG_Z = 3, RI_PQ = 4 };

template <typename T>
struct RowFwdArgs {
    int L, mode;
    const T* x;                  // RF_PLAIN: input field
    T *cx, *cr, *cp;             // RF_CG: CG vectors updated in place
    const T* cq;                 // RF_CG: last product
    const T* cz;                 // RF_PCG_P: preconditioned residual
    const double* r64;           // RF_CG, mixed: first pass starts from r64/sigma
    double* x64;                 // RF_XUPD: FP64 iterate (updated, then transformed)
    const float* d32;            // RF_XUPD: correction from the last inner run (or null)
    const uint8_t* mask;         // RF_XUPD: x is zeroed off the active set (null: all active)
    CgState* st;
    double* part;                // per-block partial sums (PCG: those of the last pass C)
    cpx<T>* Z;                   // L x M intermediate
    const cpx<T>* tw;            // exp(-2 pi i m/M), m < M
    int npart;                   // PCG: blocks of the pass C whose partial sums this pass adds
    unsigned long long h_inner;  // PCG, RF_PCG_P: the inner loop's conditional handle (0: none)
};

template <typename T>
struct ColArgs {
    int L;
    cpx<T>* Z;
    const T* Gq;                 // (M/2+1)^2 real spectrum quarter, 1/M^2 folded in
    const cpx<T>* tw;
    CgState* st;                 // with gate: the state whose fields may skip the pass
    int gate;                    // GATE_* bits (GATE_WARM: the residual was updated, no product)
    int pcg_commit;              // 1: block 0 moves the PCG r.z just decided on into place
};

template <typename T>
struct RowInvArgs {
    int L, mode;
    T* y;                        // RI_PLAIN output
    const T* s;                  // RI_CG: diagonal
    const T* cp;
    const T* cr;
    T* cq;                       // RI_CG: product q = P (C p + s p)
    T* cz;                       // RI_PCG_Z: preconditioned residual
                                 // (RI_PQ: q = P (C p + s p) into cq, p.q only)
    const uint8_t* mask;         // 1 = active fibre (null: all active)
    const double *x64, *b64, *s64;
    double* r64;                 // RI_RESID: r = P (b - C x - s x)
    CgState* st;
    double* part;
    unsigned long long h_outer, h_inner;  // graph conditional handles (0: none)
    const cpx<T>* Z;
    const cpx<T>* tw;
};

// Decide the CG step after the product q = A p of one iteration of Listing 2,
// from pass C's sums: p.q, r.q, q.q and r.r, r.p of the residual and
// direction pass A formed.  alpha = r.p / p.q, the exact minimiser along p
// (equal to r.r / p.q in exact CG, where r is orthogonal to the previous
// direction, and still right after a true-residual replacement); the new
// residual norm |r - alpha q|^2 = rr - 2 alpha rq + alpha^2 qq gives
// beta = |r'|^2 / |r|^2 without a second pass over the vectors.  The sums are
// Dot2-accurate (errors of order 1e-15 of sum |a_i b_i|), so the cancellation
// in |r'|^2 costs at most about 4e-15 rr / |r'|^2 of relative accuracy, far
// below what a stopping test certified by an FP64 true residual needs.
__device__ __forceinline__ void cg_step_decide(CgState* st, double pq, double rq, double qq, double rr_now,
                                               double rp_now, unsigned long long h_inner) {
    st->rr = rr_now;
    st->rp = rp_now;
    const double rr = rr_now;
    st->pq = pq;
    st->rq = rq;
    st->qq = qq;
    double alpha = rp_now / pq;
    double rrn = fma(__dmul_rn(alpha, alpha), qq, fma(-2.0 * alpha, rq, rr));  // explicit: same bits in every kernel
    if (rrn < 0.0) rrn = 0.0;
    int d = 0;
    if (!(pq > 0.0) || !isfinite(alpha) || !isfinite(rrn)) {
        d = 3;
        alpha = 0.0;
    } else if (rrn <= st->tol2) {
        d = 1;
    }
    st->iter += 1;
    st->cycle_iter += 1;
    if (d == 0 && (st->iter >= st->max_iter || st->cycle_iter >= st->cycle_max)) d = 2;
    if (st->tma_err) d = 4;  // a staged copy never arrived: end the inner run
    st->alpha = alpha;
    st->beta = rr > 0.0 ? rrn / rr : 0.0;
    st->first = 0;
    st->inner_done = d;
    st->idle = d != 0;
    if (h_inner) cudaGraphSetConditional(h_inner, d == 0 ? 1u : 0u);
}

// Preconditioned CG (Listing 2 with the Fourier preconditioner M), one
// iteration as the inner loop body runs it: x += alpha p and r -= alpha q
// (pass A; at the start of a run r from the true residual), z = M^-1 r
// (passes B, C), p = z + beta p (pass A), q = A p (passes B, C).  The two
// passes C only publish their blocks' partial sums (r.z and r.r; p.q); the
// pass A that follows each adds them up in every block, in one fixed order,
// and takes the step decision there, so no pass C waits for a last block.
// Every block evaluates the decision from the state as the pass found it
// (the eval functions below are pure functions of a snapshot of the fields
// they read); one thread commits it.  The fields a
// commit changes are either not read by the evaluation (rz moves into place
// in the next column pass, pcg_rz_commit) or change in a way that leads a
// block evaluating after the commit to the same decision (inner_done only
// goes from running to ended).

// The state fields a PCG step decision reads, loaded together at the start
// of the deciding pass.
struct PcgView {
    double rz, tol2;
    int first, inner_done, tma_err, iter, max_iter, cycle_iter, cycle_max;
};
__device__ __forceinline__ PcgView pcg_view(const CgState* st) {
    return {st->rz,   st->tol2,     st->first,      st->inner_done, st->tma_err,
            st->iter, st->max_iter, st->cycle_iter, st->cycle_max};
}

struct PcgAlpha {
    int d;  // inner_done after this step
    double alpha;
};
// After q = A p: alpha = r.z / p.q (the step of Hestenes and Stiefel with
// the preconditioner).  A breakdown (p.q not positive, alpha not finite) or
// the iteration cap ends the run after this update of x and r: the z
// decision that follows then stops the loop.
__device__ __forceinline__ PcgAlpha pcg_alpha_eval(const PcgView& st, double pq) {
    double alpha = st.rz / pq;
    int d = st.inner_done;
    if (!(pq > 0.0) || !isfinite(alpha)) {
        d = 3;
        alpha = 0.0;
    }
    if (d == 0 && (st.iter + 1 >= st.max_iter || st.cycle_iter + 1 >= st.cycle_max)) d = 2;
    if (st.tma_err) d = 4;
    return {d, alpha};
}
__device__ __forceinline__ void pcg_alpha_commit(CgState* st, const PcgAlpha& a, double pq) {
    st->pq = pq;
    st->alpha = a.alpha;
    st->iter += 1;
    st->cycle_iter += 1;
    st->inner_done = a.d;
}

struct PcgZr {
    int d;  // inner_done after this step (0: the run goes on)
    double beta;
};
// After z = M^-1 r of the updated residual: beta = r.z / r_prev.z_prev for
// the next direction, and the stopping test on r.r itself (summed directly
// from r, not from the recursion |r - alpha q|^2).
__device__ __forceinline__ PcgZr pcg_zr_eval(const PcgView& st, double rz, double rr) {
    int d = st.inner_done;
    if (d == 0) {
        if (!isfinite(rz) || !isfinite(rr))
            d = 3;
        else if (rr <= st.tol2)
            d = 1;
    }
    if (st.tma_err) d = 4;
    const double beta = (st.first || !(st.rz > 0.0)) ? 0.0 : rz / st.rz;
    return {d, beta};
}
// Sets the loop condition; once the run has ended (idle) the rest of the
// body returns at entry.
__device__ __forceinline__ void pcg_zr_commit(CgState* st, const PcgZr& z, double rz, double rr,
                                              unsigned long long h_inner) {
    st->rr = rr;
    st->beta = z.beta;
    st->rz_next = rz;
    st->inner_done = z.d;
    st->idle = z.d != 0;
    if (h_inner) cudaGraphSetConditional(h_inner, z.d == 0 ? 1u : 0u);
}
// The column pass after p = z + beta p (no block of it reads these fields).
__device__ __forceinline__ void pcg_rz_commit(CgState* st) {
    st->rz_prev = st->rz;
    st->rz = st->rz_next;
    st->first = 0;
}

// Decide the outer loop after a true residual r = P (b - A x): stop when
// |r| <= rtol |P b|, otherwise start a new inner run from it.
__device__ __forceinline__ void refine_decide(CgState* st, double rr64, double bb,
                                              unsigned long long h_outer, unsigned long long h_inner) {
    st->rr64 = rr64;
    st->bb = bb;
    st->cycles += 1;
    int go = 0;
    if (st->inner_done == 4 || st->tma_err) {
        st->status = FC_ETIMEOUT;  // a grid barrier or a staged copy wait ran out
    } else if (!isfinite(rr64) || !isfinite(bb)) {
        st->status = FC_ENANINF;
    } else if (bb == 0.0 || rr64 <= st->rtol2 * bb) {
        st->status = FC_OK;
    } else if (st->iter >= st->max_iter || st->cycles > st->max_cycles) {
        st->status = FC_ENOCONV;
    } else {
        go = 1;
    }
    if (go) {
        // Reliable update: the true residual replaces the recursive one and
        // the search direction is kept, p = r + beta' p_old with
        // beta' = |r_true|^2 / |r_i|^2 (physical units), so refinement does
        // not restart the Krylov space.  When the true residual did not drop
        // below the last recursive one (beta' >= 1: rounding floor or drift)
        // CG restarts from p = r instead.  The inner vectors are scaled by
        // 1/sigma (mixed) or 1 (FP64): in scaled units
        // beta_carry = rr64 / (sigma_old sigma_new rr_i).
        const double s_old = st->sigma;
        const double s_new = st->mixed ? sqrt(rr64) : 1.0;
        const double bphys = (st->rr > 0.0 && s_old > 0.0) ? rr64 / (s_old * s_old * st->rr) : 2.0;
        const bool carry =
            st->cycles > 1 && (st->inner_done == 1 || st->inner_done == 2) && bphys < 1.0 && s_new > 0.0;
        st->beta_carry = carry ? rr64 / (s_old * s_new * st->rr) : 0.0;
        st->first = 1;
        st->cycle_iter = 0;
        st->inner_done = 0;
        st->sigma = s_new;
        // mixed: the inner run (scaled to a unit start) stops after its
        // reduction inner_rtol, or as soon as it is a safe fraction below the
        // outer target itself, when that is reached first
        st->tol2 = st->mixed ? fmax(st->inner_rtol2, st->inner_goal2 * st->rtol2 * bb / rr64) : st->rtol2 * bb;
    }
    if (!go) st->first = 1;  // no inner run follows: the final update is a no-op
    st->finished = go ? 0 : 1;
    st->idle = go ? 0 : 1;
    if (h_outer) cudaGraphSetConditional(h_outer, (unsigned)go);
    if (h_inner) cudaGraphSetConditional(h_inner, (unsigned)go);
}

}  // namespace fc
