/*
 * fftconv.h -- C ABI of the B300 (sm_103a) FFT-convolution CG solver.
 *
 * The library solves the fibre-bundle system of Gjerden, "Making the case of
 * GPUs in courses on computational physics" (arXiv:1305.3625):
 *
 *   Eq. 1a-1b give f_i = -k_i (u_i - D) and u_i = sum_j G_ij f_j; Eq. 2 is
 *   (I + K G) f = K D.  Multiplied by K^-1 it becomes the symmetric positive
 *   definite system (C + S) x = b with S = diag(s_i), s_i = 1/k_i, b = D, and
 *   C the coupling operator (C x)_i = sum_j G(r_i - r_j) x_j over the open
 *   L x L grid, G(r) = 1/(pi r) for r > 0 and G(0) = 4 ln(1 + sqrt 2)/pi
 *   (Eq. 1c with a = 1 and (1 - nu^2)/E = 1).
 *
 *   C is applied as in Section 3 (Eq. 3, Listing 4): zero-pad x to the M x M
 *   grid (M = smallest power of two >= 2L), forward 2D FFT, multiply by the
 *   precomputed kernel spectrum, inverse 2D FFT, keep the [0, L)^2 corner.
 *   The solve is unpreconditioned conjugate gradients (Listing 2).
 *
 * Conventions for every entry point:
 *   - Fields are row-major L x L arrays, flat index i = iy*L + ix.
 *   - "device pointer" means memory of the current CUDA device (cudaMalloc,
 *     or a torch CUDA tensor).  The library never frees caller memory.
 *   - Plans and servers own their device workspaces and free them on
 *     destroy.  A plan may be used by one host thread at a time.
 *   - Every call returns an int status: FC_OK (0) or a negative FC_E* code.
 *     No call aborts the process or throws across the ABI.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef FFTCONV_H
#define FFTCONV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fc_stream_t; /* identical to cudaStream_t */

/* status codes */
#define FC_OK 0
#define FC_EINVAL (-1)   /* bad argument: size, null pointer, precision, mode  */
#define FC_ENOMEM (-2)   /* a device or pinned-host allocation failed          */
#define FC_EBUDGET (-3)  /* a request can never fit the server's memory budget */
#define FC_ENOCONV (-4)  /* CG stopped at max_iter above the tolerance         */
#define FC_ENANINF (-5)  /* NaN or Inf met in the data or the iteration        */
#define FC_ETIMEOUT (-6) /* a bounded wait ran out                              */
#define FC_ECUDA (-7)    /* a CUDA runtime call failed (see fc_last_error)     */
#define FC_ENOTFOUND (-8)/* unknown server ticket                               */

/* precision flags (bit set) */
#define FC_F32 1
#define FC_F64 2

/* Green's function of Eq. 1c (a = 1, (1 - nu^2)/E = 1) */
#define FC_GREEN_POINT 0 /* 1/(pi r) for r > 0, the exact cell integral at r = 0 */
#define FC_GREEN_CELL 1  /* the cell integral of Eq. 1c for every offset      */

/* solve modes */
#define FC_MODE_F64 0   /* plain FP64: FFTs, vectors and reductions in FP64   */
#define FC_MODE_MIXED 1 /* FP32 FFTs and vectors, FP64 reductions, FP64 true
                           residual driving iterative refinement             */

typedef struct fftconv_plan fftconv_plan;
typedef struct cg_server cg_server;

/* Launch-shape choice for the three FFT passes.  Each pass has a few compiled
 * shapes (values per thread, rows or columns per block); by default the plan
 * times them on its own size and keeps the fastest (cached in the file named
 * by FC_TUNE_CACHE, default $HOME/.cache/fftconv/tune_sm103.txt; FC_AUTOTUNE=0
 * disables the timing).  All zero = that default.  Forced shapes apply to the
 * FP32 passes of a plan that has them (FP64 compiles one shape per size). */
typedef struct cg_tune {
    int shape_rfwd;  /* 0: tuned; k > 0: compiled shape k-1 of the row pass A */
    int shape_col;   /* 0: tuned; k > 0: shape k-1 of the column pass B      */
    int shape_rinv;  /* 0: tuned; k > 0: shape k-1 of the row pass C         */
    int no_autotune; /* 1: no timing (cached choice or shape 0)             */
    int shape_pers;  /* inner CG loop: 0 tuned persistent kernel, k > 0 compiled
                        persistent kernel k-1, -1 one graph node per pass   */
    int reserved[3];
} cg_tune;

typedef struct cg_opts {
    double rtol;       /* stop when ||P(b - A x)||_2 <= rtol ||P b||_2, certified on the
                          FP64 recomputed residual                              */
    int max_iter;      /* cap on CG iterations (matrix-vector products), all cycles */
    int mode;          /* FC_MODE_F64 or FC_MODE_MIXED                           */
    int refine_every;  /* cap on inner iterations between two true residuals
                          (0: 100000)                                           */
    int max_refine;    /* cap on true-residual evaluations (0: 60)              */
    double inner_rtol; /* mixed: inner FP32 CG reduction per cycle (0: 3e-6 with
                          the preconditioner, 3e-3 without)                     */
    int x0_zero;       /* 1: start from x = 0 and ignore the input x; the first
                          true residual is then P b, taken without a product */
    int precond;       /* 1: preconditioned CG with the Fourier preconditioner
                          M^-1 = P crop (C_M + c I)^-1 pad P, C_M the padded
                          circulant of C (its spectrum, shifted), c = 0.6 x
                          the mean of s over active sites; 0: plain CG as in
                          Listing 2                                          */
    int warm_resid;    /* 0: when this solve follows a finished solve on the same
                          plan with bitwise the same s and b, an active set that
                          only shrank and at most 32 changed entries of the
                          masked x (a breaking step), the first true residual is
                          that solve's final FP64 residual updated by the exact
                          rank-K correction P'(r - A D), D = P'x - x_old, with
                          the FP64 Green's function table instead of an FP64
                          product; -1: always recompute it.  The residual that
                          certifies convergence is always a full FP64 product. */
} cg_opts;

typedef struct fc_run_result {
    int status;            /* FC_OK, or the status of the solve that stopped the run */
    int steps_done;        /* fibres removed                                     */
    long long iters;       /* CG iterations over all solves                      */
    int fp64_products;     /* FP64 true-residual products over all solves        */
    int resid_updated;     /* solves whose first residual was updated            */
    double seconds;        /* wall time of the run                               */
} fc_run_result;

typedef struct cg_result {
    int status;            /* FC_OK, FC_ENOCONV or FC_ENANINF                    */
    int iters;             /* CG iterations (products in the inner loops)        */
    int refinements;       /* true-residual evaluations (FP64 products, plus the
                              update when resid_updated is 1)                   */
    int resid_updated;     /* 1: the first true residual came from the warm-start
                              update (see cg_opts.warm_resid), not a product    */
    int zero_start;        /* 1: the first true residual was P b (x0_zero), not a
                              product                                           */
    int fp64_products;     /* FP64 operator products spent on true residuals
                              (refinements minus an updated or zero-start one)  */
    double true_rel_resid; /* ||P(b - A x)|| / ||P b|| from the last FP64 residual */
    double bnorm;          /* ||P b||                                           */
    double latency_s;      /* server: submit to completion; cg_solve: call time */
    double run_s;          /* server: admission to completion; cg_solve: call time */
} cg_result;

/* Library version string and the last CUDA error text of this thread. */
const char *fc_version(void);
const char *fc_last_error(void);

/*
 * fftconv_plan_create -- set up C for an L x L grid (Section 3: the transform
 * of G is static and computed at initialisation, Listing 4).
 *   p     out: new plan (host pointer to a handle).
 *   L     1 <= L <= 4096.  M = smallest power of two >= 2L.
 *   prec  FC_F32, FC_F64 or FC_F32|FC_F64 (the mixed solve needs both).
 *   tune  NULL or overrides.
 * Builds, on the current device: the twiddle tables, the circulant kernel
 * table, its 2D FFT in FP64 scaled by 1/M^2 (real, since G is even), kept as
 * the (M/2+1)^2 quarter in each requested precision, and all workspaces.
 * Synchronous.  Errors: FC_EINVAL (L, prec), FC_ENOMEM, FC_ECUDA, FC_ENANINF
 * (spectrum not real to 1e-12).
 */
int fftconv_plan_create(fftconv_plan **p, int L, int prec, const cg_tune *tune);

/*
 * fftconv_plan_create_green -- as fftconv_plan_create (which uses
 * FC_GREEN_POINT) with the Green's function chosen:
 *   green  FC_GREEN_POINT: G = 1/(pi r), r > 0, and the exact self term
 *          4 ln(1 + sqrt 2)/pi;
 *          FC_GREEN_CELL: G = (1/pi) * integral over the unit cell around
 *          the offset of dA/r (Eq. 1c as printed), by the closed form at r = 0
 *          and 16-, 8- or 4-point Gauss-Legendre tensor quadrature elsewhere
 *          (relative error below 1e-16).
 * Only the offset table and its spectrum differ; every call on the plan
 * (apply, cg_solve, fc_masked_step) then uses that operator.
 * Errors: as fftconv_plan_create; FC_EINVAL for another green value.
 */
int fftconv_plan_create_green(fftconv_plan **p, int L, int prec, int green, const cg_tune *tune);

/* Free a plan and its device memory (synchronises the device first). */
int fftconv_plan_destroy(fftconv_plan *p);

/* How the calls that wait for the device on this plan (cg_solve,
 * fc_fracture_run) wait: blocking = 0 spins (the default, lowest latency);
 * blocking = 1 blocks the calling thread on an event (for many host threads
 * each driving solves, as the server's slots do, so that waiting threads do
 * not compete for the host's cores).  Errors: FC_EINVAL, FC_ECUDA. */
int fftconv_plan_sync_mode(fftconv_plan *p, int blocking);

/* Query a plan: side L, padded side M, precision flags, device bytes held. */
int fftconv_plan_info(const fftconv_plan *p, int *L, int *M, int *prec, size_t *device_bytes);

/* Launch shapes of a plan for one precision (FC_F32 or FC_F64): for passes
 * A, B, C (index 0, 1, 2) the number of compiled shapes, the chosen one, and
 * its values per thread and rows-pairs / columns per block.  Host only. */
int fftconv_plan_shapes(const fftconv_plan *p, int prec, int n_shapes[3], int chosen[3], int radix[3],
                        int per_block[3]);

/* The inner CG loop of a solve in precision prec runs either as one
 * persistent cooperative kernel per inner run (chosen >= 0: which of n
 * compiled kernels, its block size and resident grid) or, when chosen is -1,
 * as one graph node per pass inside a device-side while loop.  Host only. */
int fftconv_plan_solver(const fftconv_plan *p, int prec, int *n, int *chosen, int *threads, int *grid);

/* The launch shapes of one of the plan's three uses of the passes of
 * Section 3's Fourier route, per pass: the index into the compiled-shape
 * lists that fftconv_plan_shapes counts, its radix and rows or columns per
 * block.
 *   FC_SHAPES_APPLY  fftconv_apply (timed in the plain modes at plan creation)
 *   FC_SHAPES_SOLVE  the passes inside cg_solve's graphs (FP32 passes of a
 *                    mixed plan timed again in the preconditioned solver's
 *                    modes, the vector updates and dot products of Listing 2
 *                    fused in; then the close candidates of passes A and C
 *                    timed together as chains of whole PCG iterations)
 *   FC_SHAPES_BATCH  cg_solve_batch and the calls built on it: the batched
 *                    twins (blockIdx.y = problem), FP32 ones timed in the CG
 *                    modes on the first batched use of a mixed plan and kept
 *                    for every later batch, so that a problem's result does
 *                    not depend on the size of the batch it joins
 * A plan created with forced shapes uses those everywhere (a batch keeps the
 * standard pass C where the forced one, the TMA-staged pass, has no twin).
 * *tuned (may be NULL) = 0 while the batched shapes are still to be chosen.
 * Host only.  Errors: FC_EINVAL. */
#define FC_SHAPES_APPLY 0
#define FC_SHAPES_SOLVE 1
#define FC_SHAPES_BATCH 2
int fftconv_plan_shape_set(const fftconv_plan *p, int prec, int set, int chosen[3], int radix[3], int per_block[3],
                           int *tuned);

/*
 * fftconv_apply -- y = C x (Listing 4: cpyComplex, FFT, elementMult, inverse
 * FFT, cpyReal), three kernel passes on stream.
 *   x, y  device pointers to L*L values (float for an FC_F32 apply, double
 *         for FC_F64); x and y must not overlap.
 * A plan created with FC_F32 only applies in FP32, one with FC_F64 only in
 * FP64; a plan with both applies in FP32 here (use fftconv_apply_prec).
 * Asynchronous.  Errors: FC_EINVAL, FC_ECUDA.
 */
int fftconv_apply(fftconv_plan *p, const void *x, void *y, fc_stream_t stream);

/* As fftconv_apply with the precision given explicitly (FC_F32 or FC_F64). */
int fftconv_apply_prec(fftconv_plan *p, int prec, const void *x, void *y, fc_stream_t stream);

/*
 * fftconv_cg_product -- one CG product of Listing 2 exactly as the solver's
 * passes form it (Section 3's Fourier route with the fused epilogue):
 * q = C p + s p, and the pass's grid sums of p.q, r.q and q.q, the dot
 * products the CG step takes its step length and residual norm from.
 *   p, r, s  device pointers to L*L values of the precision prec (FC_F32
 *            or FC_F64): direction, residual and diagonal; q: output.
 *   dots     host pointer to 3 doubles receiving p.q, r.q, q.q.
 * In FC_F32 every thread accumulates its products as an exact-product
 * two-float sum (Dot2) and the block and grid combine the pairs in
 * two-float arithmetic; in FC_F64 the sums are FP64.  Uses the plan's
 * intermediate and partial-sum buffers (not its solve state), so it must not
 * run concurrently with another call on the same plan.  Synchronous (waits
 * for stream).  Errors: FC_EINVAL, FC_ECUDA, FC_ENOMEM.
 */
int fftconv_cg_product(fftconv_plan *p, int prec, const void *pvec, const void *rvec, const void *s, void *q,
                       double dots[3], fc_stream_t stream);

/*
 * cg_solve -- solve P (C + S) P x = P b by CG (Listing 2), P the projection
 * on active fibres (mask), x = 0 off the active set.
 *   s     device, L*L doubles: diagonal s_i > 0 (compliance 1/k_i, Eq. 1a).
 *   b     device, L*L doubles: right-hand side (the displacement D, Eq. 2).
 *   x     device, L*L doubles: in = warm start (unless o->x0_zero), out = solution.
 *   mask  device, L*L bytes, 1 = active, or NULL (all active).
 *   o     host pointer to options (NULL: rtol 1e-10, FC_MODE_F64).
 *   r     host pointer receiving the result (may be NULL).
 * FC_MODE_F64 needs an FC_F64 plan; FC_MODE_MIXED needs FC_F32|FC_F64.
 * The whole solve is one CUDA graph launch on stream (device-side while
 * loops; no host round trip per iteration).  The call blocks the host
 * thread until the solve ends, then returns the status also stored in r.
 * The plan keeps copies of s, b, mask, x and the final FP64 residual; a
 * warm-started solve after a breaking step updates that residual instead of
 * recomputing it (cg_opts.warm_resid; the paper has no such step: it is an
 * exact rewriting of the first residual).  The plan is therefore not shared
 * by concurrent solves.
 * Errors: FC_EINVAL, FC_ECUDA; FC_ENOCONV / FC_ENANINF from the iteration
 * (x then holds the last iterate).
 */
int cg_solve(fftconv_plan *p, const double *s, const double *b, double *x, const uint8_t *mask,
             const cg_opts *o, cg_result *r, fc_stream_t stream);

/*
 * cg_solve_batch -- nb independent solves of the plan's size, each as in
 * cg_solve (Listing 2 with the same options), in one CUDA graph launch.
 * Every pass of the operator (Section 3) runs over all nb problems at once,
 * so small systems fill the GPU.  Each problem keeps its own state and step
 * decisions; a problem that has converged skips the remaining passes and the
 * loops run until the last problem finishes.  Batched launches use the
 * standard launch shape of each pass (cg_tune shapes 1, 1, 1), whatever the
 * plan's tuner chose for single solves, so problem k's result is the one
 * cg_solve gives on a plan with those shapes (and the per-pass graph loop),
 * independent of nb and of the other problems.
 *   nb    1 .. 65535 problems.
 *   s, b  device, nb*L*L doubles: problem k at offset k*L*L.
 *   x     device, nb*L*L doubles: in = starts (unless o->x0_zero), out = solutions.
 *   mask  device, nb*L*L bytes (1 = active), or NULL (all active).
 *   o     host options shared by all problems (NULL: rtol 1e-10, FC_MODE_F64).
 *         cg_opts.warm_resid does not apply (every first residual is a
 *         product, or P b with x0_zero).
 *   r     host array of nb results (may be NULL).
 * The plan owns a batch workspace (about 120 bytes per unknown and problem
 * with FC_MODE_MIXED), allocated on first use and grown to the largest nb;
 * its graph is rebuilt when nb changes.  The plan's own solve buffers are
 * not touched.  Blocks the host thread until all problems end.
 * Returns FC_OK when every problem converged, otherwise the first other
 * status; errors: FC_EINVAL, FC_ENOMEM, FC_ECUDA.
 */
int cg_solve_batch(fftconv_plan *p, int nb, const double *s, const double *b, double *x,
                   const uint8_t *mask, const cg_opts *o, cg_result *r, fc_stream_t stream);

/* One group of cg_solve_groups: nb problems on plan (layout as in
 * cg_solve_batch); r: host array of nb results or NULL. */
typedef struct cg_batch_group {
    fftconv_plan *plan;
    int nb;
    const double *s, *b;
    double *x;
    const uint8_t *mask;
    cg_result *r;
} cg_batch_group;

/*
 * cg_solve_groups -- batches of several sizes at once, in one CUDA graph
 * launch on stream: each group is a cg_solve_batch on its own plan, and the
 * graph holds each group's solve as a parallel branch (its own loops and
 * conditions), so the sizes run concurrently on the device.  The graph is
 * cached by the groups' workspaces, sizes and mode.  (Where such a graph
 * cannot be made, each group's graph runs on its plan's own stream, forked
 * from and joined to stream.)  Each group needs a distinct plan.  Blocks the
 * host thread until every group ends.
 * Returns FC_OK when every problem converged, otherwise the first other
 * status; errors: FC_EINVAL (bad group, repeated plan), FC_ENOMEM, FC_ECUDA.
 */
int cg_solve_groups(int ngroups, const cg_batch_group *groups, const cg_opts *o, fc_stream_t stream);

/*
 * fc_masked_step -- one quasi-static breaking step (Section 2: for each step
 * the displacement is set, the forces computed, and over-strained bonds
 * break).  The load is linear in D, so the first fibre to fail as D grows is
 * i* = argmax over active i of |x_i| / t_i (ties to the lowest index); it is
 * removed: mask[i*] = 0, x[i*] = 0.
 *   t        device, L*L doubles, thresholds > 0.
 *   mask     device, L*L bytes, updated in place.
 *   x        device, L*L doubles (the last solution), updated in place.
 *   removed  device pointer to one int64: receives i* (-1 if no active site).
 * Asynchronous.  Errors: FC_EINVAL, FC_ECUDA.
 */
int fc_masked_step(fftconv_plan *p, const double *t, uint8_t *mask, double *x, int64_t *removed,
                   fc_stream_t stream);

/*
 * fc_front -- front readout of a breaking run (Section 2: the front between
 * wholly broken and wholly intact material, driven across the grid by a
 * threshold gradient along y).  For every column ix of the L x L grid:
 *   first_intact[ix]  smallest iy with mask = 1 (L if the column is broken
 *                     through): the edge of the wholly broken region;
 *   damage_end[ix]    1 + largest iy with mask = 0 (0 if intact): the edge of
 *                     the wholly intact region.
 *   mask          device, L*L bytes (1 = intact).
 *   first_intact, damage_end  device, L int32 each.
 * Asynchronous.  Errors: FC_EINVAL, FC_ECUDA.
 */
int fc_front(fftconv_plan *p, const uint8_t *mask, int32_t *first_intact, int32_t *damage_end,
             fc_stream_t stream);

/*
 * fc_fracture_run -- `steps` quasi-static breaking steps (Section 2): solve
 * (cg_solve with o, warm-started from x; the first residual of every solve
 * after the first is the updated one), then remove the fibre with the
 * largest |x|/t (fc_masked_step).  Stops early when no active fibre is left
 * or a solve does not converge.
 *   s, b, t   device, L*L doubles; t the thresholds (any gradient is in t).
 *   mask, x   device, updated in place (intact set and last solution).
 *   removed   device, steps int64: index removed at each step (-1: none).
 *   ratio     device, steps doubles, or NULL: max |x|/t at each step, i.e.
 *             the inverse of the load D at which that fibre breaks (x is
 *             linear in D).
 *   res       host, may be NULL: totals of the run.
 * Blocks until the run ends (one host synchronisation per step).  Returns
 * res->status.  Errors: FC_EINVAL, FC_ECUDA, FC_ENOMEM; FC_ENOCONV /
 * FC_ENANINF from a solve.
 */
int fc_fracture_run(fftconv_plan *p, const double *s, const double *b, const double *t, uint8_t *mask,
                    double *x, int steps, const cg_opts *o, int64_t *removed, double *ratio,
                    fc_run_result *res, fc_stream_t stream);

/*
 * fc_fracture_run_batch -- nb independent breaking runs of the plan's size
 * (an ensemble of samples, Section 2's model with its own s, b, t each) in
 * lockstep: every step is one batched solve of all runs that are still going
 * (cg_solve_batch's graph, warm-started from each run's last solution) and
 * one batched removal.  After the first step each run's first true residual
 * is its last final FP64 residual updated for the one removal (r_i += x_k
 * G(r_i - r_k) on the remaining sites; cg_opts.warm_resid = -1 recomputes
 * it); the residual that certifies each solve is always an FP64 product.  A run stops when
 * no active fibre is left or its solve does not converge; from then on its
 * entries are -1 and its mask and x stay as they were.  The whole run stops
 * when every run has stopped or after `steps` steps.
 *   s, b, t   device, nb*L*L doubles (run k at offset k*L*L).
 *   mask, x   device, nb*L*L bytes / doubles, updated in place.
 *   removed   device, nb*steps int64: run k's index removed at step j at
 *             k*steps + j (-1: none).
 *   ratio     device, nb*steps doubles (same layout), or NULL: max |x|/t.
 *   res       host, nb results, or NULL (seconds: the whole call).
 * Blocks until the run ends (one host synchronisation per step).  Returns
 * FC_OK when every run ended without a failed solve, else the first failing
 * status.  Errors: FC_EINVAL, FC_ENOMEM, FC_ECUDA.
 */
int fc_fracture_run_batch(fftconv_plan *p, int nb, const double *s, const double *b, const double *t,
                          uint8_t *mask, double *x, int steps, const cg_opts *o, int64_t *removed,
                          double *ratio, fc_run_result *res, fc_stream_t stream);

/*
 * fc_masked_step_static -- the same breaking step as fc_masked_step, for
 * callers that cannot allocate device memory at the point of the call: a
 * process whose device memory is entirely reserved by another allocator (a
 * caching pool or a fixed budget), or a latency-bound loop that must not pay
 * the device-wide synchronisation that cudaMalloc/cudaFree imply.  It needs
 * no plan and allocates nothing: its scratch (the per-block winners of the
 * argmax and a counter) is a file-scope static device array of 131,328 bytes
 * that every GPU which loads the library holds until the process exits.  The
 * paper has no counterpart of this entry point.
 *   N        number of sites, 1 <= N <= 16,777,216 (= 4096^2); a larger N is
 *            rejected with FC_EINVAL and a message in fc_last_error().
 *   t, mask, x, removed  as for fc_masked_step (device pointers).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array, which keeps the
 * last call's contents (the counter is cleared on every call): calls that
 * overlap on the GPU, from several streams or threads, race.  Asynchronous.
 * Errors: FC_EINVAL, FC_ECUDA.
 */
int fc_masked_step_static(int64_t N, const double *t, uint8_t *mask, double *x, int64_t *removed,
                          fc_stream_t stream);

/* ------------------------------------------------------------- serving -- */

/* One solve request.  Host pointers: s and b (L*L doubles) are copied at
 * submit (or read when the request runs, with FC_REQ_BORROW); x (L*L
 * doubles) receives the solution before cg_poll reports done. */
typedef struct cg_request {
    int L;           /* 1..4096                                              */
    int mode;        /* FC_MODE_F64 or FC_MODE_MIXED                         */
    double rtol;     /* target relative residual (FP64 recomputed)           */
    const double *s; /* host, compliances s_i > 0                            */
    const double *b; /* host, right-hand side                                */
    double *x;       /* host, receives the solution (may be NULL)            */
    uint64_t tag;    /* caller's tag                                         */
    int precond;     /* 1: Fourier-preconditioned CG (see cg_opts.precond)   */
    int flags;       /* FC_REQ_BORROW: s and b are not copied at submit; the
                        caller keeps them valid and unchanged until cg_poll
                        reports the request done (0: copied at submit)     */
} cg_request;

#define FC_REQ_BORROW 1

/*
 * cg_server_create -- a continuous-batching solve server on the current
 * device (the paper has no serving layer; this is the many-solve workload
 * around its Listing 2 solver).
 *   mem_budget_bytes  device memory the server may hold for plans and staging.
 *   max_slots         concurrent batched solves (worker slots, each with its
 *                     own non-blocking stream), 1..256.
 *   stream            unused (each slot owns a stream).
 * A request is admitted when a slot is free and its plan fits the budget
 * (idle plans of other sizes are evicted if needed); the slot also takes the
 * queued requests of the same L, mode and preconditioning (up to 64, each
 * reserving its share of the plan's batch workspace within the budget) and
 * runs them as one cg_solve_batch launch with each request's own tolerance,
 * from x = 0.  Plans stay resident and are reused by later requests of the
 * same L; a size holds at most two plans, so a request whose size's plans
 * are both busy waits and joins the next batch.  Work of different slots overlaps on the device; each result
 * depends only on its own inputs (it equals cg_solve_batch of that request
 * alone on a plan of its size).
 */
int cg_server_create(cg_server **sv, size_t mem_budget_bytes, int max_slots, fc_stream_t stream);

/* Make plans for size L ahead of requests, so that no request waits for a
 * plan's set-up (spectrum, tables, autotuning: 20-90 ms): up to nplans idle
 * plans (at most the server's plans per size, 2 unless
 * FC_SERVER_PLANS_PER_SIZE says otherwise), each within the memory budget.
 * Blocks the calling thread while the plans are made; requests keep running.
 * Errors: FC_EINVAL, FC_EBUDGET (a plan does not fit), FC_ENOMEM, FC_ECUDA. */
int cg_server_reserve(cg_server *sv, int L, int nplans);

/* Queue a request; *ticket identifies it.  FC_EBUDGET if its plan can never
 * fit the budget, FC_EINVAL for bad arguments.  Returns at once. */
int cg_batch_submit(cg_server *sv, const cg_request *rq, uint64_t *ticket);

/* Non-blocking: *done = 1 once the request finished; then r (may be NULL)
 * receives its result (status, iterations, residual, latency) and the ticket
 * is released.  FC_ENOTFOUND for an unknown or released ticket. */
int cg_poll(cg_server *sv, uint64_t ticket, cg_result *r, int *done);

/* Memory held now and at peak, queued requests, resident plans. */
int cg_server_stats(cg_server *sv, size_t *used, size_t *peak, int *queued, int *plans);

/* Batched solves run so far, the requests they held, the largest batch. */
int cg_server_batches(cg_server *sv, long long *batches, long long *solves, int *max_batch);

/* Stop the workers (running solves finish), free plans and buffers. */
int cg_server_destroy(cg_server *sv);

/* ------------------------------------------------------------------------
 * Memory accounting, workspace guards and failure injection.  The paper has
 * no counterpart of these: they serve memory budgets and the tests of the
 * library's own error paths.
 * ---------------------------------------------------------------------- */

/* Device memory the library holds through its own allocations (plans,
 * batch workspaces, server staging, temporaries), measured at each
 * allocation and free: *live_bytes now, *peak_bytes the high-water mark
 * since the last reset, *live_allocs the live device and pinned-host
 * allocations.  reset_peak != 0 restarts the high-water mark at the live
 * value after reading it.  Any pointer may be NULL.  Host only, thread-safe. */
int fc_mem_stats(size_t *live_bytes, size_t *peak_bytes, long long *live_allocs, int reset_peak);

/* Every device buffer of a plan (and of its batch workspace) sits between
 * two 256-byte guard bands filled with a fixed byte at allocation.  This
 * checks them all on the device and sets *damaged to the number of bands
 * that no longer hold it (0: no kernel wrote outside its buffers).  Call it
 * with no work on the plan in flight; it waits for its own check only.
 * Errors: FC_EINVAL, FC_ENOMEM, FC_ECUDA. */
int fftconv_plan_check_guards(fftconv_plan *p, int *damaged);

/* Failure injection for tests.  Nothing here faults or hangs the GPU.
 *   FC_INJECT_ALLOC    (p ignored, may be NULL): value n > 0 makes the n-th
 *                      device or pinned-host allocation of the library from
 *                      now fail as if the memory were exhausted (once; the
 *                      call that made it returns FC_ENOMEM and frees what it
 *                      had allocated); 0 turns it off.  Process-wide.
 *   FC_INJECT_BARRIER  value > 0: in the plan's next solves the persistent
 *                      inner-CG kernel's last block leaves before its first
 *                      grid-barrier arrival, so the other blocks' bounded
 *                      waits, limited to `value` polls, run out and the
 *                      solve returns FC_ETIMEOUT; 0 turns it off.
 *   FC_INJECT_TMA      value > 0: in the plan's next solves and applies the
 *                      TMA-staged pass C issues no copy for each block's
 *                      first row pair, so its bounded mbarrier waits
 *                      (`value` polls) run out and a solve returns
 *                      FC_ETIMEOUT; 0 turns it off.
 * The plan hooks are written into the plan's solve state at once (a
 * synchronous copy) and copied into every later solve's state.
 * Errors: FC_EINVAL, FC_ECUDA. */
#define FC_INJECT_ALLOC 1
#define FC_INJECT_BARRIER 2
#define FC_INJECT_TMA 3
int fc_debug_inject(fftconv_plan *p, int kind, long long value);

#ifdef __cplusplus
}
#endif

#endif /* FFTCONV_H */
