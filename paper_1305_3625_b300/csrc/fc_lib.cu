// fftconv library: plans, the FFT-convolution operator and the CG solve
// behind the C ABI of include/fftconv.h.
//
// One plan holds, for one grid side L, everything the hot path touches:
// twiddle tables, the (M/2+1)^2 quarter of the kernel spectrum, the L x M
// intermediate, the CG vectors and the device-resident solve state.  A solve
// is one CUDA graph with two nested device-side while loops (outer: FP64 true
// residual and refinement; inner: CG iterations), so the host launches once
// per solve and reads one status block at the end.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <sys/stat.h>

#include <chrono>
#include <atomic>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "fc_alloc.h"
#include "fc_persist.cuh"
#include "fc_tma.cuh"
#include "fc_variants.h"

using namespace fc;

namespace {

thread_local char g_err[512] = "";

int set_cuda_err(cudaError_t e, const char* what) {
    snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
    return FC_ECUDA;
}

#define FC_CK(call)                                        \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return set_cuda_err(e_, #call); \
    } while (0)

}  // namespace

// ------------------------------------------------------------ allocations --
//
// Every device and pinned allocation of the library goes through these
// wrappers: they count the live allocations and bytes (fc_mem_stats) and honour
// the allocation-failure injection of fc_debug_inject (FC_INJECT_ALLOC), so
// that tests can fail any allocation of a set-up on the host and check that
// the error path returns FC_ENOMEM and frees what it had made.

namespace fc {

static std::atomic<long long> g_fail_countdown{0};  // n > 0: the n-th allocation from now fails
static std::mutex g_alloc_mu;
static std::unordered_map<void*, size_t> g_live;  // live allocations and their bytes
static size_t g_live_dev_bytes = 0, g_peak_dev_bytes = 0;

static bool inject_failure() {
    long long c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

static void note_alloc(void* ptr, size_t bytes, bool device) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_live[ptr] = device ? bytes : 0;
    if (device) {
        g_live_dev_bytes += bytes;
        if (g_live_dev_bytes > g_peak_dev_bytes) g_peak_dev_bytes = g_live_dev_bytes;
    }
}

static void note_free(void* ptr) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = g_live.find(ptr);
    if (it == g_live.end()) return;
    g_live_dev_bytes -= it->second;
    g_live.erase(it);
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
    if (inject_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) note_alloc(*ptr, bytes, true);
    return e;
}
cudaError_t dev_malloc_async(void** ptr, size_t bytes, cudaStream_t s) {
    if (inject_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(ptr, bytes, s);
    if (e == cudaSuccess) note_alloc(*ptr, bytes, true);
    return e;
}
cudaError_t host_malloc(void** ptr, size_t bytes) {
    if (inject_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(ptr, bytes);
    if (e == cudaSuccess) note_alloc(*ptr, bytes, false);
    return e;
}
void dev_free(void* ptr) {
    if (ptr && cudaFree(ptr) == cudaSuccess) note_free(ptr);
}
void dev_free_async(void* ptr, cudaStream_t s) {
    if (ptr && cudaFreeAsync(ptr, s) == cudaSuccess) note_free(ptr);
}
void host_free(void* ptr) {
    if (ptr && cudaFreeHost(ptr) == cudaSuccess) note_free(ptr);
}

}  // namespace fc

namespace {

// ------------------------------------------------------- utility kernels --

// exp(-2 pi i m / M) in FP64 (CUDA's sincospi) and rounded to FP32.
__global__ void k_twiddles(int M, cpx<double>* tw64, cpx<float>* tw32) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)M, &s, &c);
    if (tw64) tw64[m] = cpx<double>{c, -s};
    if (tw32) tw32[m] = cpx<float>{(float)c, (float)-s};
}

// Stage twiddle table of a (M, E) transform from the FP64 base table
// tw64[m] = exp(-2 pi i m / M): entry [e][k] (at e*NS + k) of the stage with
// span NS and radix R is tw64[e k M / (NS R)], rounded to T.
template <typename T>
__global__ void k_stage_twiddles(int M, int NS, int R, int off, const cpx<double>* tw64, cpx<T>* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NS * R) return;
    const int e = i / NS, k = i % NS;
    const cpx<double> w = tw64[(size_t)e * k * (M / (NS * R))];
    out[off + i] = cpx<T>{(T)w.x, (T)w.y};
}

// Green's function of Eq. 1c (a = 1, (1-nu^2)/E = 1): point form 1/(pi r) and
// the exact self term 4 ln(1 + sqrt 2)/pi.
__device__ double green(long dx, long dy) {
    if (dx == 0 && dy == 0) return 4.0 * log1p(sqrt(2.0)) / 3.14159265358979323846;
    return 1.0 / (3.14159265358979323846 * sqrt((double)(dx * dx + dy * dy)));
}

// Gauss-Legendre rules on [-1, 1] with 16, 8 and 4 nodes (nodes and weights
// from the host, see gauss_legendre).
struct GaussLeg {
    double x16[16], w16[16], x8[8], w8[8], x4[4], w4[4];
};

// (1/pi) times the integral of 1/r over the unit cell centred at (cx, cy) by
// the N-point tensor rule (the cell's half width 1/2 is the Jacobian of each
// coordinate).
template <int N>
__device__ double cell_quadrature(double cx, double cy, const double* xs, const double* ws) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
        const double x = cx + 0.5 * xs[i];
        double row = 0.0;
        for (int j = 0; j < N; ++j) {
            const double y = cy + 0.5 * xs[j];
            row += ws[j] * rsqrt(x * x + y * y);
        }
        acc += ws[i] * row;
    }
    return 0.25 * acc / 3.14159265358979323846;
}

// Eq. 1c's cell integral for every offset (a = 1, (1-nu^2)/E = 1): the closed
// form at r = 0, else Gauss-Legendre quadrature of the (then smooth)
// integrand.  The rule's error falls like rho^(-2n), rho ~ 4 max(|dx|, |dy|)
// the Bernstein-ellipse parameter of the nearest singularity (the origin), so
// 16 nodes for the cells next to the origin, 8 up to a distance of 31 and 4
// beyond keep it below 1e-17 relative.
__device__ double green_cell(long dx, long dy, const GaussLeg& gl) {
    if (dx == 0 && dy == 0) return green(0, 0);
    const long ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
    const long m = ax > ay ? ax : ay;
    if (m <= 2) return cell_quadrature<16>((double)ax, (double)ay, gl.x16, gl.w16);
    if (m <= 31) return cell_quadrature<8>((double)ax, (double)ay, gl.x8, gl.w8);
    return cell_quadrature<4>((double)ax, (double)ay, gl.x4, gl.w4);
}

// The Green's function on the non-negative site offsets, gt[dy * L + dx] =
// G(dx, dy) for dx, dy < L: the point form with exact self term
// (FC_GREEN_POINT) or the cell integral (FC_GREEN_CELL).
__global__ void k_green_table(int L, int kind, GaussLeg gl, double* gt) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)L * L) return;
    const long dx = (long)(idx % L), dy = (long)(idx / L);
    gt[idx] = kind == FC_GREEN_CELL ? green_cell(dx, dy, gl) : green(dx, dy);
}

// Circulant embedding on the M x M grid: index j < L is offset j, index
// j > M - L is offset j - M; indices in between are reached by no pair of
// sites and hold 0.  Values from the offset table gt (G is even in each
// coordinate).
__global__ void k_kernel_table(int L, int M, const double* gt, cpx<double>* K) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)M * M) return;
    int jy = (int)(idx / M), jx = (int)(idx % M);
    bool okx = jx < L || jx > M - L, oky = jy < L || jy > M - L;
    int ax = jx < L ? jx : M - jx, ay = jy < L ? jy : M - jy;
    K[idx] = cpx<double>{(okx && oky) ? gt[(size_t)ay * L + ax] : 0.0, 0.0};
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Keep the (M/2+1)^2 quarter of Re(FFT2(k))/M^2; track max |Im| and max |Re|
// (block maxima, one atomic per block).
__global__ void __launch_bounds__(256) k_spectrum_quarter(int M, const cpx<double>* K, double* gq64, float* gq32,
                                                          double* maxes) {
    __shared__ double smi[8], smr[8];
    const int Q = M / 2 + 1;
    const double scale = 1.0 / ((double)M * (double)M);
    double mi = 0.0, mr = 0.0;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (size_t)M * M;
         idx += (size_t)gridDim.x * blockDim.x) {
        cpx<double> z = K[idx];
        mi = fmax(mi, fabs(z.y) * scale);
        mr = fmax(mr, fabs(z.x) * scale);
        int fy = (int)(idx / M), fx = (int)(idx % M);
        if (fy < Q && fx < Q) {
            double g = z.x * scale;
            if (gq64) gq64[(size_t)fy * Q + fx] = g;
            if (gq32) gq32[(size_t)fy * Q + fx] = (float)g;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        mi = fmax(mi, __shfl_down_sync(0xffffffffu, mi, off));
        mr = fmax(mr, __shfl_down_sync(0xffffffffu, mr, off));
    }
    if ((threadIdx.x & 31) == 0) {
        smi[threadIdx.x >> 5] = mi;
        smr[threadIdx.x >> 5] = mr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mi = fmax(mi, smi[w]);
            mr = fmax(mr, smr[w]);
        }
        atomic_max_nonneg(maxes + 0, mi);
        atomic_max_nonneg(maxes + 1, mr);
    }
}

// Last step of an inner CG run: x += alpha p (the residual is recomputed).
// Problem blockIdx.y of a batch (vectors at stride N).
template <typename T>
__global__ void k_cg_final(long N, const CgState* st, T* x, const T* p) {
    st += blockIdx.y;
    x += blockIdx.y * N;
    p += blockIdx.y * N;
    if (st->first) return;
    const T alpha = (T)st->alpha;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
        x[i] += alpha * p[i];
}

// FP32 copy of the diagonal.  With a state (single-problem solves): nothing
// to do when the warm check found s bitwise unchanged since the last solve,
// whose copy is still in place.
__global__ void k_f64_to_f32(long N, const double* a, float* b, const CgState* st) {
    if (st && st->s_check && !st->s_diff) return;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// The preconditioner's shift c as a fraction of the mean of s over the active
// sites.  Measured on breaking loops (60 steps, mixed PCG to 1e-10): 0.6 took
// the iterations per solve from 9.95 to 9.32 at L = 1024, 10.35 to 9.8 at
// L = 512 and 11.1 to 10.3 at L = 128 against the plain mean (1.0); 0.2 and
// 2.0 both took more than 1.0.
constexpr double kPrecondShiftScale = 0.6;

// Shift of the Fourier preconditioner: c = kPrecondShiftScale x the mean of
// s over active sites (last block writes it).  Problem blockIdx.y of a batch (vectors at stride
// N, partial sums at stride bpart).
__global__ void __launch_bounds__(256) k_active_mean(long N, const double* s, const uint8_t* mask, double* part,
                                                     CgState* st, long bpart) {
    s += blockIdx.y * N;
    if (mask) mask += blockIdx.y * N;
    part += blockIdx.y * bpart;
    st += blockIdx.y;
    // four sites per round, all loaded before use; the count is an integer
    double sum = 0.0;
    unsigned cnt = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += 4 * stride) {
        double sv[4];
        uint8_t mv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long i = i0 + u * stride;
            sv[u] = i < N ? s[i] : 0.0;
            mv[u] = i < N ? (mask ? mask[i] : (uint8_t)1) : (uint8_t)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (mv[u]) {
                sum += sv[u];
                ++cnt;
            }
    }
    double v[2] = {sum, (double)cnt}, tot[2];
    if (grid_sum_last<2>(v, part, &st->cntA, tot) && threadIdx.x == 0)
        st->pshift = tot[1] > 0 ? kPrecondShiftScale * tot[0] / tot[1] : 1.0;
}

// The same shift from the FP32 copy of s (mixed solves): two-float sums on
// the FP32 pipe instead of FP64 adds, which run at a small fraction of the
// FP32 rate on this part (the shift only sets the preconditioner).
__global__ void __launch_bounds__(256) k_active_mean_f32(long N, const float* s, const uint8_t* mask, double* part,
                                                         CgState* st, long bpart) {
    s += blockIdx.y * N;
    if (mask) mask += blockIdx.y * N;
    part += blockIdx.y * bpart;
    st += blockIdx.y;
    Acc<float> a[2];
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += 4 * stride) {
        float sv[4];
        uint8_t mv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long i = i0 + u * stride;
            sv[u] = i < N ? s[i] : 0.f;
            mv[u] = i < N ? (mask ? mask[i] : (uint8_t)1) : (uint8_t)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (mv[u]) {
                a[0].prod(sv[u], 1.f);
                a[1].prod(1.f, 1.f);
            }
    }
    double tot[2];
    if (grid_sum_last<2>(a, part, &st->cntA, tot) && threadIdx.x == 0)
        st->pshift = tot[1] > 0 ? kPrecondShiftScale * tot[0] / tot[1] : 1.0;
}

// Spectrum quarter of the preconditioner (C_M + c I)^-1 in the scaling of
// the stored kernel spectrum: Gq = eig(C_M)/M^2, so Pq = 1/((M^2 Gq + c) M^2).
// Problem blockIdx.y of a batch writes its own spectrum (stride QQ).
template <typename T>
__global__ void k_precond_spectrum(long QQ, double MM, const double* gq64, const CgState* st, T* pq) {
    st += blockIdx.y;
    pq += blockIdx.y * QQ;
    const double c = st->pshift;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < QQ; i += (long)gridDim.x * blockDim.x)
        pq[i] = (T)(1.0 / ((MM * gq64[i] + c) * MM));
}
// The FP32 preconditioner spectrum from the FP32 kernel spectrum, in FP32
// arithmetic (an FP64 division per entry cost tens of microseconds per solve
// on this part; the preconditioner needs no more than FP32 accuracy).
__global__ void k_precond_spectrum_f32(long QQ, float MM, const float* gq32, const CgState* st, float* pq) {
    st += blockIdx.y;
    pq += blockIdx.y * QQ;
    const float c = (float)st->pshift;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < QQ; i += (long)gridDim.x * blockDim.x)
        pq[i] = 1.0f / (fmaf(MM, gq32[i], c) * MM);
}

// A solve from x = 0 needs no product for its first true residual: it is
// r = P b.  Sets x = 0 and r = P b and hands |r|^2 = |P b|^2 to the first
// refinement decision, as the warm-start update does (warm_used = 2 marks
// the zero start).  Problem blockIdx.y of a batch.
__global__ void __launch_bounds__(256) k_zero_start(long N, const double* b, const uint8_t* mask, double* x,
                                                    double* r, double* part, long bpart, CgState* st) {
    const long o = blockIdx.y * N;
    b += o, x += o, r += o;
    if (mask) mask += o;
    part += blockIdx.y * bpart;
    st += blockIdx.y;
    double v[1] = {0.0}, tot[1];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double bv = (!mask || mask[i]) ? b[i] : 0.0;
        x[i] = 0.0;
        r[i] = bv;
        v[0] += bv * bv;
    }
    if (grid_sum_last<1>(v, part, &st->cntC, tot) && threadIdx.x == 0) {
        st->rr64 = tot[0];
        st->bb = tot[0];
        st->warm = 1;
        st->warm_used = 2;
    }
}

// Residual update after one removal per problem (batched breaking runs,
// problem blockIdx.y): the previous solve's final residual r = P (b - A x)
// becomes P' (b - A P' x) = P' (r + x_k A e_k), i.e. r_i += x_k G(r_i - r_k)
// on the sites still active and 0 at the removed site k, with |r|^2 and the
// new |P' b|^2 handed to the next solve's first refinement decision (warm).
// A problem without a removal (k < 0) is left to recompute its residual.
__global__ void __launch_bounds__(256) k_warm_resid_batch(long N, int L, const double* gt, const uint8_t* mask,
                                                          const double* b64, double* r64, double* part, long bpart,
                                                          CgState* st, const long long* kidx, const double* kx) {
    const long long k = kidx[blockIdx.y];
    if (k < 0) return;  // the same in every block of the problem
    const long o = (long)blockIdx.y * N;
    mask += o, b64 += o, r64 += o;
    part += blockIdx.y * bpart;
    st += blockIdx.y;
    const double xk = kx[blockIdx.y];
    const int ky = (int)(k / L), kxx = (int)(k % L);
    double v[2] = {0.0, 0.0}, tot[2];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        double r = 0.0;
        if (mask[i]) {
            const int iy = (int)i / L, ix = (int)i - iy * L;  // L <= 4096: N < 2^31
            r = r64[i] + xk * __ldg(gt + (size_t)abs(iy - ky) * L + abs(ix - kxx));
            const double bv = b64[i];
            v[1] += bv * bv;
        }
        r64[i] = r;
        v[0] += r * r;
    }
    if (grid_sum_last<2>(v, part, &st->cntC, tot) && threadIdx.x == 0) {
        st->rr64 = tot[0];
        st->bb = tot[1];
        st->warm = 1;
        st->warm_used = 1;
    }
}

// Loop control of a batched solve (one node after the deciding pass): the
// outer loop runs while any problem is unfinished, the inner loop while any
// problem has an inner run open.  A finished problem is idle.
__global__ void __launch_bounds__(256) k_batch_ctl(int nb, const CgState* st, unsigned long long h_outer,
                                                   unsigned long long h_inner) {
    int open = 0, inner = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        open |= st[i].finished == 0;
        inner |= st[i].idle == 0;
    }
    open = __syncthreads_or(open);
    inner = __syncthreads_or(inner);
    if (threadIdx.x == 0) {
        if (h_outer) cudaGraphSetConditional(h_outer, open ? 1u : 0u);
        cudaGraphSetConditional(h_inner, inner ? 1u : 0u);
    }
}

template <typename T>
__global__ void k_fill(long N, T* a, T v) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) a[i] = v;
}

__global__ void k_fill_u8(long N, uint8_t* m, uint8_t v) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) m[i] = v;
}

// ------------------------------------------- warm-start residual update --
//
// A solve that follows another solve on the same plan, with the same s and b,
// an active set that only shrank (P' <= P) and an iterate that differs from
// the last one, x_old, in a few entries (a breaking step removes one fibre
// and zeroes its x), needs no FP64 product for its first true residual:
// with D = P' x - x_old (nonzero at the changed entries k only),
//   P' (b - A P' x) = P' (P (b - A x_old) - A D),
//   (A D)_i = sum_k D_k (G(r_i - r_k) + s_k [i = k]),
// where P (b - A x_old) is the last solve's final FP64 residual r64, still in
// the plan.  The check kernel compares the new inputs with the plan's copies
// while copying them in; the update kernel applies the rank-K correction with
// the FP64 Green's function table.  Later residuals (and the final one that
// certifies convergence) are full FP64 products.

// Copies s, b, the masked x and the mask into the plan's buffers (writing
// only entries that changed) and records: st->wbad when s or b differ bitwise
// or a site became active, st->s_diff when s differs, st->wcount changed
// entries of x with the first kWarmMax of them (flat index, x_new - x_old) in
// widx, wdx.
__global__ void __launch_bounds__(256) k_warm_check(long N, const double* __restrict__ s,
                                                    const double* __restrict__ b, const double* __restrict__ x,
                                                    const uint8_t* __restrict__ mask_in, double* __restrict__ s64,
                                                    double* __restrict__ b64, double* __restrict__ x64,
                                                    uint8_t* __restrict__ mask, CgState* st, long long* widx,
                                                    double* wdx) {
    int bad = 0, sdiff = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        // every operand of the site loaded before the first test (one round trip)
        const double sn = s[i], bn = b[i], xi = x[i], so = s64[i], bo = b64[i], xo = x64[i];
        const uint8_t mo = mask[i];
        const uint8_t mn = mask_in ? mask_in[i] : (uint8_t)1;
        if (__double_as_longlong(sn) != __double_as_longlong(so)) {
            bad = 1;
            sdiff = 1;
            s64[i] = sn;
        }
        if (__double_as_longlong(bn) != __double_as_longlong(bo)) {
            bad = 1;
            b64[i] = bn;
        }
        if (mn && !mo) bad = 1;
        if (mn != mo) mask[i] = mn;
        const double xn = mn ? xi : 0.0;
        if (__double_as_longlong(xn) != __double_as_longlong(xo)) {
            x64[i] = xn;
            const unsigned k = atomicAdd(&st->wcount, 1u);
            if (k < (unsigned)kWarmMax) {
                widx[k] = i;
                wdx[k] = xn - xo;
            }
        }
    }
    const int any_bad = __syncthreads_or(bad), any_s = __syncthreads_or(sdiff);
    if (threadIdx.x == 0) {
        if (any_bad) atomicOr(&st->wbad, 1);
        if (any_s) atomicOr(&st->s_diff, 1);
    }
}

// r64 <- P' (r64 - A D) with the recorded changes, and its sums rr64 = |r|^2,
// bb = |P' b|^2; the last block sets st->warm so that the first residual
// passes hand these to the refinement decision.  Does nothing (the passes
// then compute the residual) when the check found the update inapplicable.
__global__ void __launch_bounds__(256) k_warm_resid(long N, int L, const double* __restrict__ gt,
                                                    const uint8_t* __restrict__ mask,
                                                    const double* __restrict__ s64, const double* __restrict__ b64,
                                                    double* __restrict__ r64, double* part, CgState* st,
                                                    const long long* widx, const double* wdx) {
    __shared__ long long ki[kWarmMax];
    __shared__ int ky[kWarmMax], kx[kWarmMax];
    __shared__ double kd[kWarmMax];
    const unsigned K = st->wcount;
    if (st->wbad || K > (unsigned)kWarmMax) return;  // the same in every block
    if (threadIdx.x < K) {
        const long long i = widx[threadIdx.x];
        ki[threadIdx.x] = i;
        ky[threadIdx.x] = (int)(i / L);
        kx[threadIdx.x] = (int)(i % L);
        kd[threadIdx.x] = wdx[threadIdx.x];
    }
    __syncthreads();
    double v[2] = {0.0, 0.0}, tot[2];
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += 4 * stride) {
        uint8_t m[4];
        double r0[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // every operand of the round loaded first
            const long i = i0 + u * stride;
            m[u] = i < N ? mask[i] : (uint8_t)0;
            r0[u] = i < N ? r64[i] : 0.0;
            bv[u] = i < N ? b64[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long i = i0 + u * stride;
            if (i >= N) break;
            double r = 0.0;
            if (m[u]) {
                r = r0[u];
                if (K) {
                    const int iy = (int)i / L, ix = (int)i - iy * L;  // L <= 4096: N < 2^31
                    for (unsigned k = 0; k < K; ++k) {
                        double a = gt[(size_t)abs(iy - ky[k]) * L + abs(ix - kx[k])];
                        if (i == ki[k]) a += s64[i];
                        r = fma(-kd[k], a, r);
                    }
                }
                v[1] = fma(bv[u], bv[u], v[1]);
            }
            r64[i] = r;
            v[0] = fma(r, r, v[0]);
        }
    }
    if (grid_sum_last<2>(v, part, &st->cntC, tot) && threadIdx.x == 0) {
        st->rr64 = tot[0];
        st->bb = tot[1];
        st->warm = 1;
        st->warm_used = 1;
    }
}

struct ArgmaxCtl {
    unsigned cnt;
    int pad;
};

// One quasi-static breaking step: i* = argmax over active i of |x_i|/t_i (ties
// to the lowest index), then mask[i*] = 0 and x[i*] = 0.  The last block to
// finish reduces the per-block winners in block order.
// (value, index) order of the breaking rule: larger |x|/t first, then the
// lower index; an index of -1 marks "no active site".
// A positive double (its bits) as a float truncated to 24 significant bits,
// by integer operations; 0 outside [2^-100, 2^101) (or for a number that is
// not positive), where quotients of two such floats stay clear of the range
// in which the fast FP32 division loses its 2-ulp bound.
__device__ __forceinline__ float trunc_float(long long bits) {
    const int e = (int)(bits >> 52);  // biased exponent (a set sign bit makes it negative)
    if (e < 1023 - 100 || e > 1023 + 100) return 0.0f;
    const unsigned fb = ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((bits >> 29) & 0x7fffff);
    return __uint_as_float(fb);
}

__device__ __forceinline__ bool am_better(double ov, long long oi, double mv, long long mi) {
    return oi >= 0 && (mi < 0 || ov > mv || (ov == mv && oi < mi));
}

// The best (value, index) of a block by the breaking rule's order: warp
// shuffles, then warp 0 over the warps' winners (valid in thread 0).  The
// order is total, so the winner does not depend on the reduction order.
__device__ __forceinline__ void am_block_reduce(double& bv, long long& bi) {
    __shared__ double sv[32];
    __shared__ long long si[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, off);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (am_better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
        bv = lane < nw ? sv[lane] : -1.0;
        bi = lane < nw ? si[lane] : -1;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, off);
            const long long oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (am_better(ov, oi, bv, bi)) {
                bv = ov;
                bi = oi;
            }
        }
    }
}

// One quasi-static breaking step: i* = argmax over active i of |x_i|/t_i (ties
// to the lowest index), then mask[i*] = 0 and x[i*] = 0.  Each block reduces
// its sites; the last block to finish reduces the per-block winners.  The
// order is total, so the result does not depend on the reduction order.
// Problem blockIdx.y of a batch: fields at stride N, its result at stride
// rstride, its own winners and counter; with st, a problem whose state holds
// a status other than FC_OK (its solve failed, or it sits the step out)
// removes nothing and reports -1.
__global__ void __launch_bounds__(256) k_masked_argmax(long N, const double* t, uint8_t* mask, double* x,
                                                       int64_t* removed, double* ratio, double* pv,
                                                       long long* pi, ArgmaxCtl* ctl, long rstride = 0,
                                                       const CgState* st = nullptr, long long* kidx = nullptr,
                                                       double* kx = nullptr) {
    if (st && st[blockIdx.y].status != FC_OK) {  // the same in every block of the problem
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            removed[(long)blockIdx.y * rstride] = -1;
            if (ratio) ratio[(long)blockIdx.y * rstride] = -1.0;
            if (kidx) kidx[blockIdx.y] = -1;
        }
        return;
    }
    const long yo = (long)blockIdx.y * N;
    t += yo, mask += yo, x += yo;
    removed += (long)blockIdx.y * rstride;
    if (ratio) ratio += (long)blockIdx.y * rstride;
    pv += (long)blockIdx.y * gridDim.x;
    pi += (long)blockIdx.y * gridDim.x;
    ctl += blockIdx.y;
    __shared__ bool is_last;
    double bv = -1.0;
    long long bi = -1;
    // The exact ratio |x|/t (IEEE FP64 division) decides, but a thread first
    // ranks its sites by an FP32 estimate and divides exactly only for the
    // sites whose estimate ends within the estimate's error band of its
    // largest one (this part's FP64 unit is slow).  The estimate's operands
    // are the doubles' exponents and leading 23 mantissa bits reassembled as
    // floats by integer operations (a double-to-float conversion runs on the
    // FP64 unit), so each is within 2^-23 below its double; with a 2-ulp
    // division the estimate is within 6e-7 of the exact ratio.  The thread's
    // best site therefore ends with an estimate within 1.2e-6 of the largest
    // and is never dropped from the candidates (band 2e-6); sites with an
    // operand outside [2^-100, 2^101), and candidates beyond the four a thread
    // keeps, are divided at once.
    constexpr float kBand = 2e-6f;
    float emax = -1.0f;
    float cest[4];
    long cidx[4];
    int nc = 0;
    auto exact = [&](long i, double xa, double tv) {
        const double v = xa / tv;
        if (am_better(v, i, bv, bi)) {
            bv = v;
            bi = i;
        }
    };
    const long stride = (long)gridDim.x * blockDim.x;
    // four sites per round: their loads are issued together, one memory round
    // trip per round instead of one per site
    for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += 4 * stride) {
        uint8_t mv[4];
        double xv[4], tv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long i = i0 + u * stride;
            const bool in = i < N;
            mv[u] = in ? mask[i] : (uint8_t)0;
            xv[u] = in ? x[i] : 0.0;
            tv[u] = in ? t[i] : 1.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!mv[u]) continue;
            const long i = i0 + u * stride;
            const float xf = trunc_float(__double_as_longlong(xv[u]) & 0x7fffffffffffffffLL);
            const float tf = trunc_float(__double_as_longlong(tv[u]));
            if (!(xf > 0.0f && tf > 0.0f)) {
                exact(i, fabs(xv[u]), tv[u]);
                continue;
            }
            const float est = __fdividef(xf, tf);
            if (est > emax * (1.0f + kBand)) {  // a new leader: the old candidates fall behind
                emax = est;
                nc = 0;
            } else if (est < emax * (1.0f - kBand)) {
                continue;
            }
            if (est > emax) emax = est;
            if (nc < 4) {
                cest[nc] = est;
                cidx[nc] = i;
                ++nc;
            } else {
                exact(i, fabs(xv[u]), tv[u]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < nc && cest[c] >= emax * (1.0f - kBand)) exact(cidx[c], fabs(x[cidx[c]]), t[cidx[c]]);
    am_block_reduce(bv, bi);
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = bv;
        pi[blockIdx.x] = bi;
        __threadfence();
        is_last = atomicAdd(&ctl->cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    bv = -1.0;
    bi = -1;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        double ov = __ldcg(pv + b);
        long long oi = __ldcg(pi + b);
        if (am_better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    am_block_reduce(bv, bi);
    if (threadIdx.x == 0) {
        const long long gi = bi;
        *removed = gi;
        if (ratio) *ratio = bv;  // max |x|/t (-1 with no active site)
        if (kidx) {  // batched runs: the removal, for the next solve's residual update
            kidx[blockIdx.y] = gi;
            kx[blockIdx.y] = gi >= 0 ? x[gi] : 0.0;
        }
        if (gi >= 0) {
            mask[gi] = 0;
            x[gi] = 0.0;
        }
        ctl->cnt = 0u;
    }
}

// Front readout of a breaking run (Section 2: the front separates wholly
// broken from wholly intact material).  Column ix of the L x L grid:
// first_intact = smallest iy with mask = 1 (L when broken through),
// damage_end = 1 + largest iy with mask = 0 (0 when intact).  A block covers
// 32 columns (one per lane, so each row read is 32 contiguous bytes) and its
// 16 warps split the rows.
__global__ void __launch_bounds__(512) k_front(int L, const uint8_t* mask, int32_t* first_intact,
                                               int32_t* damage_end) {
    __shared__ int s_first[16][32], s_end[16][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ix = blockIdx.x * 32 + lane;
    int fi = L, de = 0;
    if (ix < L) {
        for (int iy = w; iy < L; iy += 16) {
            if (mask[(size_t)iy * L + ix]) {
                if (iy < fi) fi = iy;
            } else {
                de = iy + 1;
            }
        }
    }
    s_first[w][lane] = fi;
    s_end[w][lane] = de;
    __syncthreads();
    if (w == 0 && ix < L) {
        for (int k = 1; k < 16; ++k) {
            fi = min(fi, s_first[k][lane]);
            de = max(de, s_end[k][lane]);
        }
        first_intact[ix] = fi;
        damage_end[ix] = de;
    }
}
template <typename T>
bool get_variants(int M, Variants* v) {
    *v = Variants{};
    const bool f64 = sizeof(T) == 8;
    switch (M) {
        case 256: variants_256(f64, v); return true;
        case 512: variants_512(f64, v); return true;
        case 1024: variants_1024(f64, v); return true;
        case 2048: variants_2048(f64, v); return true;
        case 4096: variants_4096(f64, v); return true;
        case 8192: variants_8192(f64, v); return true;
        default: return variants_small(M, f64, v);
    }
}

int set_smem_attr(const KV& k) {
    if (k.f && k.smem > 48 * 1024)
        FC_CK(cudaFuncSetAttribute(k.f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    if (k.fp && k.smem > 48 * 1024)
        FC_CK(cudaFuncSetAttribute(k.fp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    if (k.fplain && k.smem > 48 * 1024)
        FC_CK(cudaFuncSetAttribute(k.fplain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    return FC_OK;
}

int set_smem_attrs(const Variants& v) {
    int rc = FC_OK;
    for (int k = 0; k < v.n_rfwd && !rc; ++k) rc = set_smem_attr(v.rfwd[k]);
    for (int k = 0; k < v.n_rinv && !rc; ++k) rc = set_smem_attr(v.rinv[k]);
    for (int k = 0; k < v.n_colc && !rc; ++k) rc = set_smem_attr(v.colc[k]);
    for (int k = 0; k < v.n_pers && !rc; ++k)
        if (v.pers[k].smem > 48 * 1024)
            if (cudaFuncSetAttribute(v.pers[k].f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.pers[k].smem) !=
                cudaSuccess)
                rc = set_cuda_err(cudaGetLastError(), "cudaFuncSetAttribute(persistent)");
    if (!rc) rc = set_smem_attr(v.rows_full);
    if (!rc) rc = set_smem_attr(v.cols_full);
    for (int k = 0; k < v.n_rfwd && !rc; ++k) rc = set_smem_attr(v.rfwd_b[k]);
    for (int k = 0; k < v.n_colc && !rc; ++k) rc = set_smem_attr(v.colc_b[k]);
    for (int k = 0; k < v.n_rinv && !rc; ++k) rc = set_smem_attr(v.rinv_b[k]);
    return rc;
}

constexpr int kMaxPersistGrid = 148 * 16;

int grid_1d(long n, int threads) {
    long g = (n + threads - 1) / threads;
    if (g > 148L * 16) g = 148L * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// ------------------------------------------------------------------ plan --

// A device buffer between two guard bands of kGuard bytes of kGuardByte:
// [base, base + kGuard) and [base + kGuard + bytes, base + 2 kGuard + bytes);
// the user's bytes start at base + kGuard (256-byte aligned, as cudaMalloc's).
struct GuardedAlloc {
    void* base;
    size_t bytes;
};
constexpr size_t kGuard = 256;
constexpr unsigned char kGuardByte = 0xC5;

struct PrecRes {
    bool on = false;
    Variants v;
    int sel[3] = {0, 0, 0};  // chosen shape of pass A, B, C for fftconv_apply (plain passes)
    int sel_cg[3] = {0, 0, 0};  // chosen shape of each pass inside solves (timed in the CG modes)
    int sel_b[3] = {0, 0, 0};  // chosen batched twin of pass A, B, C (indices into the same lists)
    bool tuned_b = false;      // sel_b decided (tuned on first batched use, or forced)
    bool tune_off = false;     // the plan was made without timing (no_autotune, FC_AUTOTUNE=0)
    int sel_pers = -1;       // chosen persistent inner-CG kernel (-1: graph loop)
    int pers_grid = 0;       // its cooperative grid (resident blocks)
    void* Z = nullptr;       // cpx<T>[(M/2) * L], column-major half spectra
    void* tw = nullptr;      // FP64 only: base table exp(-2 pi i m/M), m < M
    void* twst[6] = {};      // stage twiddle tables for E = 2, 4, 8, 16, 32 (index log2 E)
    void* Gq = nullptr;      // T[(M/2+1)^2]
    CUtensorMap zmap;        // FP32: Zt as floats [M/2][2L] for the TMA pass C
    bool tma_ok = false;     // zmap encoded (L even, M >= 256)
    int tma_grid = 0;        // resident blocks of the TMA pass C (its persistent grid)
    const KV& rfwd() const { return v.rfwd[sel[0]]; }
    const KV& colc() const { return v.colc[sel[1]]; }
    const KV& rinv() const { return v.rinv[sel[2]]; }
    const KV& rfwd_cg() const { return v.rfwd[sel_cg[0]]; }
    const KV& colc_cg() const { return v.colc[sel_cg[1]]; }
    const KV& rinv_cg() const { return v.rinv[sel_cg[2]]; }
    const void* tws(int E) const { return twst[tw_index(E)]; }
    // every shape this precision may launch has its stage twiddle table
    bool tables_ok(int M) const {
        auto ok = [&](int E) { return E >= M || tws(E) != nullptr; };
        for (int k = 0; k < v.n_rfwd; ++k)
            if (!ok(v.rfwd[k].E)) return false;
        for (int k = 0; k < v.n_colc; ++k)
            if (!ok(v.colc[k].E)) return false;
        for (int k = 0; k < v.n_rinv; ++k)  // pass C shapes of their own (the TMA-staged ones)
            if (!ok(v.rinv[k].E)) return false;
        for (int k = 0; k < v.n_pers; ++k)
            if (!ok(v.pers[k].EA) || !ok(v.pers[k].EB)) return false;
        return true;
    }
};

struct fftconv_plan {
    int L = 0, M = 0, prec = 0, dev = 0;
    int green = FC_GREEN_POINT;  // Green's function of Eq. 1c: point form or cell integral
    long N = 0;
    size_t bytes = 0;
    PrecRes p32, p64;
    // solve workspace (FP64 side)
    double *x64 = nullptr, *r64 = nullptr, *p64v = nullptr, *q64 = nullptr, *b64 = nullptr, *s64 = nullptr;
    uint8_t* mask = nullptr;
    // solve workspace (FP32 side, mixed mode)
    float *d32 = nullptr, *r32 = nullptr, *p32v = nullptr, *q32 = nullptr, *s32 = nullptr;
    // preconditioned CG: preconditioned residuals and preconditioner spectra
    double *z64 = nullptr, *pq64 = nullptr;
    float *z32 = nullptr, *pq32 = nullptr;
    CgState* st = nullptr;
    CgState* st_host = nullptr;  // pinned
    double* part = nullptr;
    double* partA = nullptr;  // persistent kernel: per-block partial sums
    double* partC = nullptr;
    PersistCtl* pctl = nullptr;
    double* am_v = nullptr;
    long long* am_i = nullptr;
    ArgmaxCtl* am_ctl = nullptr;
    int am_grid = 0;
    cudaGraph_t graph[4] = {};      // index mode + 2 * precond
    cudaGraphExec_t gexec[4] = {};
    // warm-start residual update: FP64 Green's function table [L][L], the
    // changed-entry list, and whether r64 is the final true residual of the
    // iterate, s, b and mask now in the plan (set after a finished solve)
    double* gtab = nullptr;
    long long* widx = nullptr;
    double* wdx = nullptr;
    bool warm_ok = false;
    bool s32_ok = false;  // s32 holds the FP32 copy of s64 (made by the last mixed solve)
    int64_t* rm_host = nullptr;  // pinned: last removed index of a fracture run
    bool blocking = false;       // waits block the host thread (event with blocking sync)
    cudaEvent_t ev_wait = nullptr;
    struct BatchWs* batch = nullptr;  // batched solves (cg_solve_batch), made on first use
    // every device buffer of the plan, each between two guard bands
    // (fftconv_plan_check_guards), and the set-up stream that fills them
    std::vector<GuardedAlloc> allocs;
    cudaStream_t setup = nullptr;
    // test hooks (fc_debug_inject): copied into each solve's state
    unsigned dbg_skip = 0, dbg_limit = 0;
};

namespace {

// Fill the two guard bands of a guarded buffer on stream s.
int fill_guards(const GuardedAlloc& a, cudaStream_t s) {
    unsigned char* b = (unsigned char*)a.base;
    FC_CK(cudaMemsetAsync(b, kGuardByte, kGuard, s));
    FC_CK(cudaMemsetAsync(b + kGuard + a.bytes, kGuardByte, kGuard, s));
    return FC_OK;
}

// A plan buffer of bytes (guarded; set-up only: the guards are filled on the
// plan's set-up stream).
int dalloc(fftconv_plan* p, void** ptr, size_t bytes) {
    void* base = nullptr;
    cudaError_t e = dev_malloc(&base, bytes + 2 * kGuard);
    if (e != cudaSuccess) {
        set_cuda_err(e, "cudaMalloc");
        return FC_ENOMEM;
    }
    p->allocs.push_back(GuardedAlloc{base, bytes});
    *ptr = (unsigned char*)base + kGuard;
    p->bytes += bytes;
    return fill_guards(p->allocs.back(), p->setup);
}

// Free one plan buffer made by dalloc.
void dfree(fftconv_plan* p, void* ptr) {
    for (size_t k = 0; k < p->allocs.size(); ++k)
        if ((unsigned char*)p->allocs[k].base + kGuard == ptr) {
            dev_free(p->allocs[k].base);
            p->bytes -= p->allocs[k].bytes;
            p->allocs.erase(p->allocs.begin() + (long)k);
            return;
        }
}

void batch_free(fftconv_plan* p);
size_t batch_bytes_of(const fftconv_plan* p);

void plan_free(fftconv_plan* p) {
    if (!p) return;
    batch_free(p);
    for (int m = 0; m < 4; ++m) {
        if (p->gexec[m]) cudaGraphExecDestroy(p->gexec[m]);
        if (p->graph[m]) cudaGraphDestroy(p->graph[m]);
    }
    for (const GuardedAlloc& a : p->allocs) dev_free(a.base);
    p->allocs.clear();
    host_free(p->st_host);
    host_free(p->rm_host);
    if (p->ev_wait) cudaEventDestroy(p->ev_wait);
    delete p;
}

template <typename T>
int launch(const void* f, int grid, int threads, size_t smem, cudaStream_t s, T& args) {
    void* kp[1] = {(void*)&args};
    FC_CK(cudaLaunchKernel(f, dim3(grid), dim3(threads), kp, smem, s));
    return FC_OK;
}

// Programmatic dependent launches between consecutive passes (FC_PDL=0 turns
// them off): the next pass's blocks are scheduled while the previous pass
// drains and wait on the device for its completion.
bool pdl_on() {
    static const bool on = [] {
        const char* e = getenv("FC_PDL");
        return !(e && !strcmp(e, "0"));
    }();
    return on;
}

// A pass launched as a programmatic dependent of the previous kernel on s
// (the passes wait for it before touching memory).
template <typename T>
int launch_dep(const void* f, int grid, int threads, size_t smem, cudaStream_t s, T& args) {
    if (!pdl_on()) return launch(f, grid, threads, smem, s, args);
    void* kp[1] = {(void*)&args};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FC_CK(cudaLaunchKernelExC(&cfg, f, kp));
    return FC_OK;
}

int row_grid(const fftconv_plan* p, const KV& k) { return ((p->L + 1) / 2 + k.per - 1) / k.per; }
int col_grid(const fftconv_plan* p, const KV& k) { return (p->M / 2) / k.per; }

// Arguments of the TMA-staged pass C for the FP32 intermediate of a plan.
RowInvTma tma_args(const fftconv_plan* p, const PrecRes& R, const RowInvArgs<float>& c) {
    RowInvTma P;
    memset(&P, 0, sizeof(P));
    P.map = R.zmap;
    P.a = c;
    P.units = (p->L + 1) / 2;
    return P;
}

// Pass C on a stream in the shape k (dep: as a programmatic dependent of the
// previous pass).
template <typename T>
int launch_rinv(fftconv_plan* p, PrecRes& R, const KV& k, RowInvArgs<T>& c, cudaStream_t s, bool dep) {
    if constexpr (sizeof(T) == 4) {
        if (k.tma) {
            if (!R.tma_ok) return FC_EINVAL;
            RowInvTma P = tma_args(p, R, c);
            return dep ? launch_dep(k.f, R.tma_grid, k.threads, k.smem, s, P)
                       : launch(k.f, R.tma_grid, k.threads, k.smem, s, P);
        }
    }
    return dep ? launch_dep(k.f, row_grid(p, k), k.threads, k.smem, s, c)
               : launch(k.f, row_grid(p, k), k.threads, k.smem, s, c);
}

// Stage twiddle tables for every value-per-thread count E that a compiled
// shape of this precision uses.
template <typename T>
int build_stage_tables(fftconv_plan* p, PrecRes& R, const cpx<double>* tw64, cudaStream_t cs) {
    int Es[8], nE = 0;
    auto addE = [&](int E) {
        if (E < 2) return;
        for (int i = 0; i < nE; ++i)
            if (Es[i] == E) return;
        Es[nE++] = E;
    };
    for (int k = 0; k < R.v.n_rfwd; ++k) addE(R.v.rfwd[k].E);
    for (int k = 0; k < R.v.n_colc; ++k) addE(R.v.colc[k].E);
    for (int k = 0; k < R.v.n_rinv; ++k) addE(R.v.rinv[k].E);  // the TMA-staged pass C has shapes of its own
    for (int k = 0; k < R.v.n_pers; ++k) {
        addE(R.v.pers[k].EA);
        addE(R.v.pers[k].EB);
    }
    addE(R.v.rows_full.E);
    addE(R.v.cols_full.E);
    const int M = p->M;
    for (int i = 0; i < nE; ++i) {
        const int E = Es[i];
        const int len = tw_len(M, E);
        const int idx = tw_index(E);
        int rc = dalloc(p, &R.twst[idx], sizeof(cpx<T>) * (size_t)(len > 2 ? len : 2));
        if (rc) return rc;
        for (int ns = E; ns < M; ns *= stage_radix(M, E, ns)) {
            const int rad = stage_radix(M, E, ns), n = ns * rad;
            k_stage_twiddles<T><<<(n + 255) / 256, 256, 0, cs>>>(M, ns, rad, tw_offset(M, E, ns), tw64,
                                                                 (cpx<T>*)R.twst[idx]);
            FC_CK(cudaGetLastError());
        }
    }
    return FC_OK;
}

}  // namespace

// ------------------------------------------------------------- autotuner --
//
// Each pass has a few compiled launch shapes (values per thread E, rows or
// columns per block).  At plan creation the tuner times every shape of each
// pass on the plan's own size (the mean of 20 programmatic launches back to
// back after 3 warm-ups, on a private stream) and keeps the fastest; choices
// are cached per (precision, M, L, pass) in a text file (FC_TUNE_CACHE,
// default $HOME/.cache/fftconv/tune_sm103.txt; keys carry the timing's
// version, "t2").  FC_AUTOTUNE=0 skips the timing.

namespace {

std::mutex g_tune_mu;
bool g_tune_loaded = false;
struct TuneEntry {
    char key[96];
    int idx;
};
TuneEntry g_tune[512];
int g_ntune = 0;

void tune_path(char* out, size_t n) {
    const char* e = getenv("FC_TUNE_CACHE");
    if (e && *e) {
        snprintf(out, n, "%s", e);
        return;
    }
    const char* h = getenv("HOME");
    snprintf(out, n, "%s/.cache/fftconv/tune_sm103.txt", h ? h : "/tmp");
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    char path[512];
    tune_path(path, sizeof(path));
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[sizeof(g_tune[0].key) - 1];  // a longer line is no entry of ours
    while (g_ntune < 512 && fgets(line, sizeof(line), f)) {
        // "<key>| <index>"; keys contain no '|'
        char* bar = strrchr(line, '|');
        if (!bar) continue;
        *bar = 0;
        int idx = -1;
        if (sscanf(bar + 1, "%d", &idx) == 1) {
            snprintf(g_tune[g_ntune].key, sizeof(g_tune[g_ntune].key), "%s", line);
            g_tune[g_ntune].idx = idx;
            ++g_ntune;
        }
    }
    fclose(f);
}

bool tune_lookup(const char* key, int* idx) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    for (int k = g_ntune - 1; k >= 0; --k)
        if (!strcmp(g_tune[k].key, key)) {
            *idx = g_tune[k].idx;
            return true;
        }
    return false;
}

void tune_store(const char* key, int idx) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    if (g_ntune < 512) {
        snprintf(g_tune[g_ntune].key, sizeof(g_tune[g_ntune].key), "%s", key);
        g_tune[g_ntune].idx = idx;
        ++g_ntune;
    }
    char path[512];
    tune_path(path, sizeof(path));
    char dir[512];
    snprintf(dir, sizeof(dir), "%s", path);
    char* slash = strrchr(dir, '/');
    if (slash) {
        *slash = 0;
        char cmd[600];
        // best effort: the cache is an optimisation only
        snprintf(cmd, sizeof(cmd), "%s", dir);
        for (char* q = cmd + 1; *q; ++q)
            if (*q == '/') {
                *q = 0;
                mkdir(cmd, 0755);
                *q = '/';
            }
        mkdir(cmd, 0755);
    }
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s| %d\n", key, idx);
    fclose(f);
}

// time one launch shape of one pass (kind 0: A, 1: B, 2: C), PLAIN mode
template <typename T>
int time_shape(fftconv_plan* p, PrecRes& R, int kind, int k, T* x, T* y, cudaStream_t s, cudaEvent_t e0,
               cudaEvent_t e1, float* ms, T* const* cgv = nullptr) {
    const KV& kv = kind == 0 ? R.v.rfwd[k] : (kind == 1 ? R.v.colc[k] : R.v.rinv[k]);
    const cpx<T>* tw = (const cpx<T>*)R.tws(kv.E);
    RowFwdArgs<T> a{};
    a.L = p->L;
    a.mode = RF_PLAIN;
    a.x = x;
    a.Z = (cpx<T>*)R.Z;
    a.tw = tw;
    ColArgs<T> b{p->L, (cpx<T>*)R.Z, (const T*)R.Gq, tw};
    RowInvArgs<T> c{};
    c.L = p->L;
    c.mode = RI_PLAIN;
    c.y = y;
    c.st = p->st;
    c.Z = (const cpx<T>*)R.Z;
    c.tw = tw;
    if (cgv) {
        // the preconditioned solver's modes: pass A's update of x and r
        // (x += a p, r -= a q) with its step decision from published sums (one
        // block's, zero: alpha = 0), pass C's product q = C p + s p with p.q
        a.mode = RF_PCG_R;
        a.cx = cgv[0];
        a.cr = cgv[1];
        a.cp = cgv[2];
        a.cq = cgv[3];
        a.st = p->st;
        a.part = p->part;
        a.npart = 1;
        c.mode = RI_PQ;
        c.cr = cgv[1];
        c.cp = cgv[2];
        c.cq = cgv[3];
        c.s = cgv[4];
        c.part = p->part;
    }
    if (kv.tma && !R.tma_ok) {  // no tensor map for this size: never chosen
        *ms = 1e30f;
        return FC_OK;
    }
    const int grid = kind == 1 ? col_grid(p, kv) : row_grid(p, kv);
    auto go = [&]() -> int {
        // programmatic launches back to back, as the passes run in an apply
        // or a solve (a shape that keeps more blocks resident overlaps the
        // next launch's start better)
        if (kind == 0)
            return launch_dep(cgv ? (kv.fp ? kv.fp : kv.f) : (kv.fplain ? kv.fplain : kv.f), grid, kv.threads,
                              kv.smem, s, a);
        if (kind == 1) return launch_dep(kv.f, grid, kv.threads, kv.smem, s, b);
        KV kc = kv;
        if (!cgv && kc.fplain) kc.f = kc.fplain;  // the apply's plain form
        return launch_rinv<T>(p, R, kc, c, s, true);
    };
    constexpr int kTimed = 20;
    int rc = FC_OK;
    for (int w = 0; w < 3 && !rc; ++w) rc = go();
    if (rc) return rc;
    FC_CK(cudaEventRecord(e0, s));
    for (int w = 0; w < kTimed && !rc; ++w) rc = go();
    if (rc) return rc;
    FC_CK(cudaEventRecord(e1, s));
    FC_CK(cudaEventSynchronize(e1));
    FC_CK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= (float)kTimed;
    return FC_OK;
}

// One preconditioned iteration (the six passes of the solve graph's loop
// body, programmatic launches) with pass A shape ia and pass C shape ic, on
// the plan's FP32 vectors and state: the mean of 8 iterations after 2.  The
// run never stops (tol2 < 0); the kernel spectrum serves both column passes.
template <typename T>
int time_pcg_chain(fftconv_plan* p, PrecRes& R, int ia, int ic, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                   float* ms) {
    const KV& ka = R.v.rfwd[ia];
    const KV& kb = R.colc_cg();
    const KV& kc = R.v.rinv[ic];
    if ((kc.tma && !R.tma_ok) || !ka.fp) {
        *ms = 1e30f;
        return FC_OK;
    }
    const long N = p->N;
    T *cx = (T*)p->d32, *cr = (T*)p->r32, *cp = (T*)p->p32v, *cq = (T*)p->q32, *cz = (T*)p->z32, *sv = (T*)p->s32;
    T* vs[5] = {cr, cp, cq, cz, sv};
    for (T* v : vs) k_fill<T><<<grid_1d(N, 256), 256, 0, s>>>(N, v, v == sv ? (T)1 : (T)0.01);
    FC_CK(cudaGetLastError());
    FC_CK(cudaMemsetAsync(cx, 0, sizeof(T) * N, s));
    CgState h{};
    h.first = 1;  // the first A skips the step (no sums yet); later iterations decide
    h.rz = 1.0;
    h.tol2 = -1.0;
    h.sigma = 1.0;
    h.max_iter = 1 << 30;
    h.cycle_max = 1 << 30;
    *p->st_host = h;
    FC_CK(cudaMemcpyAsync(p->st, p->st_host, sizeof(CgState), cudaMemcpyHostToDevice, s));
    const int npart = kc.tma ? R.tma_grid : row_grid(p, kc);
    RowFwdArgs<T> a1{};
    a1.L = p->L;
    a1.mode = RF_PCG_R;
    a1.cx = cx;
    a1.cr = cr;
    a1.cp = cp;
    a1.cq = cq;
    a1.st = p->st;
    a1.part = p->part;
    a1.npart = npart;
    a1.Z = (cpx<T>*)R.Z;
    a1.tw = (const cpx<T>*)R.tws(ka.E);
    RowFwdArgs<T> a2 = a1;
    a2.mode = RF_PCG_P;
    a2.cz = cz;
    ColArgs<T> b1{p->L, (cpx<T>*)R.Z, (const T*)R.Gq, (const cpx<T>*)R.tws(kb.E), p->st, 0};
    ColArgs<T> b2{p->L, (cpx<T>*)R.Z, (const T*)R.Gq, (const cpx<T>*)R.tws(kb.E), p->st, 0, 1};
    RowInvArgs<T> c1{};
    c1.L = p->L;
    c1.mode = RI_PCG_Z;
    c1.cr = cr;
    c1.cz = cz;
    c1.st = p->st;
    c1.part = p->part;
    c1.Z = (const cpx<T>*)R.Z;
    c1.tw = (const cpx<T>*)R.tws(kc.E);
    RowInvArgs<T> c2 = c1;
    c2.mode = RI_PQ;
    c2.s = sv;
    c2.cp = cp;
    c2.cq = cq;
    const int ga = row_grid(p, ka), gb = col_grid(p, kb);
    auto iter = [&]() -> int {
        int rc = launch_dep(ka.fp, ga, ka.threads, ka.smem, s, a1);
        if (!rc) rc = launch_dep(kb.f, gb, kb.threads, kb.smem, s, b1);
        if (!rc) rc = launch_rinv<T>(p, R, kc, c1, s, true);
        if (!rc) rc = launch_dep(ka.fp, ga, ka.threads, ka.smem, s, a2);
        if (!rc) rc = launch_dep(kb.f, gb, kb.threads, kb.smem, s, b2);
        if (!rc) rc = launch_rinv<T>(p, R, kc, c2, s, true);
        return rc;
    };
    int rc = FC_OK;
    for (int w = 0; w < 2 && !rc; ++w) rc = iter();
    if (rc) return rc;
    FC_CK(cudaEventRecord(e0, s));
    for (int w = 0; w < 8 && !rc; ++w) rc = iter();
    if (rc) return rc;
    FC_CK(cudaEventRecord(e1, s));
    FC_CK(cudaEventSynchronize(e1));
    FC_CK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= 8.0f;
    return FC_OK;
}

template <typename T>
int autotune(fftconv_plan* p, PrecRes& R, const cg_tune* tune) {
    const int n[3] = {R.v.n_rfwd, R.v.n_colc, R.v.n_rinv};
    // forced shapes select the FP32 passes of a plan that has them (FP64
    // carries one shape per size); an FP64-only plan applies them to FP64
    const bool apply = tune && (sizeof(T) == 4 || !(p->prec & FC_F32));
    const int forced[3] = {apply ? tune->shape_rfwd : 0, apply ? tune->shape_col : 0, apply ? tune->shape_rinv : 0};
    const char* env = getenv("FC_AUTOTUNE");
    const bool timing = !(tune && tune->no_autotune) && !(env && !strcmp(env, "0"));
    const char* venv = getenv("FC_TUNE_VERBOSE");
    const bool verbose = venv && strcmp(venv, "0");
    const char* names[3] = {"rfwd", "colc", "rinv"};
    bool need[3] = {false, false, false}, need_cg[3] = {false, false, false};
    char keys[3][96], keys_cg[3][96];
    for (int kind = 0; kind < 3; ++kind) {
        if (forced[kind] > 0) {
            if (forced[kind] > n[kind]) return FC_EINVAL;
            if (kind == 2 && R.v.rinv[forced[kind] - 1].tma && !R.tma_ok) return FC_EINVAL;
            R.sel[kind] = forced[kind] - 1;
            R.sel_cg[kind] = forced[kind] - 1;
            // batched solves take the same shape where it has a twin (not the TMA pass C)
            const KV& tw = kind == 0 ? R.v.rfwd_b[R.sel[kind]] : (kind == 1 ? R.v.colc_b[R.sel[kind]]
                                                                              : R.v.rinv_b[R.sel[kind]]);
            R.sel_b[kind] = tw.f ? R.sel[kind] : 0;
            continue;
        }
        R.sel[kind] = 0;
        R.sel_cg[kind] = 0;
        if (n[kind] <= 1) continue;
        snprintf(keys[kind], sizeof(keys[kind]), "t2 %s M=%d L=%d %s n=%d ", sizeof(T) == 4 ? "f32" : "f64", p->M,
                 p->L, names[kind], n[kind]);
        int idx = 0;
        if (tune_lookup(keys[kind], &idx) && idx >= 0 && idx < n[kind] && !(kind == 2 && R.v.rinv[idx].tma && !R.tma_ok))
            R.sel[kind] = idx;
        else
            need[kind] = timing;
        R.sel_cg[kind] = R.sel[kind];  // the column pass is the same in every mode
        if (kind == 1 || sizeof(T) != 4 || !(p->prec & FC_F64)) continue;  // solves: FP32 passes of mixed plans
        snprintf(keys_cg[kind], sizeof(keys_cg[kind]), "t2 f32 M=%d L=%d %s_cg n=%d ", p->M, p->L, names[kind],
                 n[kind]);
        if (tune_lookup(keys_cg[kind], &idx) && idx >= 0 && idx < n[kind] &&
            !(kind == 2 && R.v.rinv[idx].tma && !R.tma_ok))
            R.sel_cg[kind] = idx;
        else
            need_cg[kind] = timing;
    }
    if (forced[0] > 0 || forced[1] > 0 || forced[2] > 0 || n[0] <= 1) R.tuned_b = true;  // no batched tuning
    R.tune_off = !timing;
    if (!need[0] && !need[1] && !need[2] && !need_cg[0] && !need_cg[2]) return FC_OK;
    T *x = nullptr, *y = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FC_OK;
    const size_t zbytes = sizeof(cpx<T>) * (size_t)(p->M / 2) * p->L;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        dev_malloc_async((void**)&x, sizeof(T) * p->N, s) != cudaSuccess ||
        dev_malloc_async((void**)&y, sizeof(T) * p->N, s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(x, 0, sizeof(T) * p->N, s) != cudaSuccess || cudaMemsetAsync(R.Z, 0, zbytes, s) != cudaSuccess) {
        rc = set_cuda_err(cudaGetLastError(), "autotune set-up");
    }
    for (int kind = 0; kind < 3 && !rc; ++kind) {
        if (!need[kind]) continue;
        float best = 1e30f;
        int bi = 0;
        for (int k = 0; k < n[kind] && !rc; ++k) {
            float ms = 0;
            rc = time_shape<T>(p, R, kind, k, x, y, s, e0, e1, &ms);
            if (!rc && verbose) {
                const KV& kv = kind == 0 ? R.v.rfwd[k] : (kind == 1 ? R.v.colc[k] : R.v.rinv[k]);
                fprintf(stderr, "[fftconv tune] %s shape %d (E=%d, per=%d, threads=%d, smem=%zu): %.3f us\n",
                        keys[kind], k, kv.E, kv.per, kv.threads, kv.smem, ms * 1e3f);
            }
            if (!rc && ms < best) {
                best = ms;
                bi = k;
            }
        }
        if (!rc) {
            R.sel[kind] = bi;
            tune_store(keys[kind], bi);
        }
    }
    R.sel_cg[1] = R.sel[1];
    for (int kind = 0; kind < 3; kind += 2)
        if (need[kind] && !need_cg[kind] && !(sizeof(T) == 4 && (p->prec & FC_F64))) R.sel_cg[kind] = R.sel[kind];
    // inside solves passes A and C run in the CG modes (vector updates, five
    // dot products): their shapes are timed again in those modes on the
    // plan's FP32 vectors (zeroed; the plan's state, fresh, takes the steps)
    int runner[3] = {-1, -1, -1};
    for (int kind = 0; kind < 3 && !rc; ++kind) {
        if (!need_cg[kind]) continue;
        T* cgv[5] = {(T*)p->d32, (T*)p->r32, (T*)p->p32v, (T*)p->q32, (T*)p->s32};
        for (int i = 0; i < 5 && !rc; ++i)
            if (cudaMemsetAsync(cgv[i], 0, sizeof(T) * p->N, s) != cudaSuccess)
                rc = set_cuda_err(cudaGetLastError(), "autotune set-up");
        // a fresh state (first = 0: pass A decides) and zero sums; every solve
        // sets the state anew
        if (!rc && (cudaMemsetAsync(p->st, 0, sizeof(CgState), s) != cudaSuccess ||
                    cudaMemsetAsync(p->part, 0, 2 * sizeof(double), s) != cudaSuccess))
            rc = set_cuda_err(cudaGetLastError(), "autotune set-up");
        float best = 1e30f, best2 = 1e30f;
        int bi = 0, bi2 = -1;
        for (int k = 0; k < n[kind] && !rc; ++k) {
            float ms = 0;
            rc = time_shape<T>(p, R, kind, k, x, y, s, e0, e1, &ms, cgv);
            if (!rc && verbose)
                fprintf(stderr, "[fftconv tune] %s shape %d (CG mode): %.3f us\n", keys_cg[kind], k, ms * 1e3f);
            if (rc) break;
            if (ms < best) {
                best2 = best;
                bi2 = best < 1e30f ? bi : -1;
                best = ms;
                bi = k;
            } else if (ms < best2) {
                best2 = ms;
                bi2 = k;
            }
        }
        if (!rc) {
            R.sel_cg[kind] = bi;
            // a runner-up within 10 % is tried again in the iteration chain below
            runner[kind] = (bi2 >= 0 && best2 <= 1.1f * best) ? bi2 : -1;
        }
    }
    // passes A and C of a preconditioned iteration timed together: the best
    // shape of each pass alone and its close runner-up, in every pairing, as
    // chains of whole PCG iterations (programmatic launches); the passes'
    // costs in a solve include how each overlaps its neighbours.
    if constexpr (sizeof(T) == 4) {
        if (!rc && need_cg[0] && need_cg[2] && p->z32 && (runner[0] >= 0 || runner[2] >= 0)) {
            const int ca[2] = {R.sel_cg[0], runner[0]}, cc[2] = {R.sel_cg[2], runner[2]};
            float best = 1e30f;
            int ba = ca[0], bc = cc[0];
            for (int i = 0; i < 2 && !rc; ++i)
                for (int k = 0; k < 2 && !rc; ++k) {
                    if (ca[i] < 0 || cc[k] < 0) continue;
                    float ms = 0;
                    rc = time_pcg_chain<T>(p, R, ca[i], cc[k], s, e0, e1, &ms);
                    if (!rc && verbose)
                        fprintf(stderr, "[fftconv tune] f32 M=%d L=%d PCG iteration, pass A %d, pass C %d: %.3f us\n",
                                p->M, p->L, ca[i], cc[k], ms * 1e3f);
                    if (!rc && ms < best) {
                        best = ms;
                        ba = ca[i];
                        bc = cc[k];
                    }
                }
            if (!rc) {
                R.sel_cg[0] = ba;
                R.sel_cg[2] = bc;
            }
        }
    }
    for (int kind = 0; kind < 3 && !rc; kind += 2)
        if (need_cg[kind]) tune_store(keys_cg[kind], R.sel_cg[kind]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) {
        dev_free_async(x, s);
        dev_free_async(y, s);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    return rc;
}

}  // namespace

namespace {

// The batched twins of each pass, timed like the single-problem shapes
// (in the solver's modes, 2 warm-up and 5 timed launches) over nb problems at once,
// nb = min(16, 64 MB of intermediate); the fastest is kept for every batched
// solve of the plan, whatever its batch size, so that a problem's arithmetic
// does not depend on the batch it joins.  Choices are cached like the
// single-problem ones (keys "... rfwd_b ...").  Runs on the first batched use
// of a mixed plan (FP64 carries one shape); FC_AUTOTUNE=0 keeps the standard
// shapes.
template <typename T>
int autotune_batched(fftconv_plan* p, PrecRes& R) {
    if (R.tuned_b) return FC_OK;
    R.tuned_b = true;
    R.sel_b[0] = R.sel_b[1] = R.sel_b[2] = 0;
    const char* env = getenv("FC_AUTOTUNE");
    const bool timing = !R.tune_off && !(env && !strcmp(env, "0"));
    const char* venv = getenv("FC_TUNE_VERBOSE");
    const bool verbose = venv && strcmp(venv, "0");
    const KV* lists[3] = {R.v.rfwd_b, R.v.colc_b, R.v.rinv_b};
    const int n[3] = {R.v.n_rfwd, R.v.n_colc, R.v.n_rinv};
    const char* names[3] = {"rfwd_bcg", "colc_b", "rinv_bcg"};
    char keys[3][96];
    bool need[3] = {false, false, false};
    for (int kind = 0; kind < 3; ++kind) {
        if (n[kind] <= 1) continue;
        snprintf(keys[kind], sizeof(keys[kind]), "t2 %s M=%d L=%d %s n=%d ", sizeof(T) == 4 ? "f32" : "f64", p->M, p->L,
                 names[kind], n[kind]);
        int idx = 0;
        if (tune_lookup(keys[kind], &idx) && idx >= 0 && idx < n[kind] && lists[kind][idx].f)
            R.sel_b[kind] = idx;
        else
            need[kind] = timing;
    }
    if (!need[0] && !need[1] && !need[2]) return FC_OK;
    const long N = p->N, zs = (long)(p->M / 2) * p->L, ps = 3 * (long)(p->L + 1);
    long nbt = (64L << 20) / (long)(zs * sizeof(cpx<T>));
    if (nbt > 16) nbt = 16;
    if (nbt < 1) nbt = 1;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* buf = nullptr;
    // six vectors (x, r, p, q, s, output) per problem, the intermediate, the
    // states and partial sums
    const size_t bytes = sizeof(T) * 6 * (size_t)nbt * N + sizeof(cpx<T>) * (size_t)nbt * zs +
                         sizeof(CgState) * nbt + sizeof(double) * (size_t)nbt * ps;
    int rc = FC_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = set_cuda_err(cudaGetLastError(), "batched autotune set-up");
    if (!rc && dev_malloc_async(&buf, bytes, s) != cudaSuccess) {
        set_cuda_err(cudaErrorMemoryAllocation, "cudaMallocAsync(batched autotune)");
        rc = FC_ENOMEM;
    }
    if (!rc && cudaMemsetAsync(buf, 0, bytes, s) != cudaSuccess)
        rc = set_cuda_err(cudaGetLastError(), "batched autotune set-up");  // states: first = 0, alpha = 0
    T* cv[6];
    for (int i = 0; i < 6; ++i) cv[i] = (T*)buf + (size_t)i * nbt * N;
    cpx<T>* Z = (cpx<T>*)(cv[5] + nbt * N);
    CgState* st = (CgState*)(Z + nbt * zs);
    double* part = (double*)(st + nbt);
    const BatchArgs bb{0, BatchStride{N, zs, 0, ps}};
    for (int kind = 0; kind < 3 && !rc; ++kind) {
        if (!need[kind]) continue;
        float best = 1e30f;
        int bi = 0;
        for (int k = 0; k < n[kind] && !rc; ++k) {
            const KV& kv = lists[kind][k];
            if (!kv.f) continue;
            const cpx<T>* tw = (const cpx<T>*)R.tws(kv.E);
            // the modes batched solves run: pass A's update of x and r with its
            // step decision from published sums, pass C's product with p.q
            // (zeroed vectors and sums, fresh states: alpha = 0)
            RowFwdArgs<T> a{};
            a.L = p->L;
            a.mode = RF_PCG_R;
            a.cx = cv[0];
            a.cr = cv[1];
            a.cp = cv[2];
            a.cq = cv[3];
            a.st = st;
            a.part = part;
            a.npart = 1;
            a.Z = Z;
            a.tw = tw;
            ColArgs<T> b{p->L, Z, (const T*)R.Gq, tw, st, 0};
            RowInvArgs<T> c{};
            c.L = p->L;
            c.mode = RI_PQ;
            c.cr = cv[1];
            c.cp = cv[2];
            c.cq = cv[3];
            c.s = cv[4];
            c.y = cv[5];
            c.st = st;
            c.part = part;
            c.Z = Z;
            c.tw = tw;
            const int gx = kind == 1 ? col_grid(p, kv) : row_grid(p, kv);
            void* a2[2] = {kind == 0 ? (void*)&a : (kind == 1 ? (void*)&b : (void*)&c), (void*)&bb};
            auto go = [&]() -> int {
                if (cudaLaunchKernel(kv.f, dim3(gx, (unsigned)nbt), dim3(kv.threads), a2, kv.smem, s) != cudaSuccess)
                    return set_cuda_err(cudaGetLastError(), "batched autotune launch");
                return FC_OK;
            };
            float ms = 0;
            for (int w = 0; w < 2 && !rc; ++w) rc = go();
            if (!rc && cudaEventRecord(e0, s) != cudaSuccess) rc = set_cuda_err(cudaGetLastError(), "event");
            for (int w = 0; w < 5 && !rc; ++w) rc = go();
            if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = set_cuda_err(cudaGetLastError(), "event");
            if (rc) break;
            ms /= 5.0f;
            if (verbose)
                fprintf(stderr, "[fftconv tune] %s shape %d (E=%d, per=%d, threads=%d) x%ld problems: %.3f us\n",
                        keys[kind], k, kv.E, kv.per, kv.threads, nbt, ms * 1e3f);
            if (ms < best) {
                best = ms;
                bi = k;
            }
        }
        if (!rc) {
            R.sel_b[kind] = bi;
            tune_store(keys[kind], bi);
        }
    }
    if (s) {
        dev_free_async(buf, s);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" const char* fc_version(void) { return "fftconv-b300 0.1 (sm_103a)"; }
extern "C" const char* fc_last_error(void) { return g_err; }

namespace {
template <typename T>
int choose_persistent(fftconv_plan* p, PrecRes& R, T* cx, T* cr, T* cp, T* cq, T* s, int forced, bool timing,
                      bool verbose);
}  // namespace

namespace {

// cuTensorMapEncodeTiled, looked up once through the runtime's driver entry
// point (no link against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor map of the FP32 intermediate Zt, viewed as floats [M/2][2L], with
// boxes of 4 floats (the two complex values of a row pair) by up to 256
// columns, and the resident grid of the TMA pass C.  The row stride 8L bytes
// must be a multiple of 16 and a box starts at float 4u (byte 16u): L even.
// Without a map (odd L, small M, no driver entry point) that shape is never
// launched.
int setup_tma(fftconv_plan* p) {
    PrecRes& R = p->p32;
    R.tma_ok = false;
    int k = -1;
    for (int i = 0; i < R.v.n_rinv; ++i)
        if (R.v.rinv[i].tma) k = i;
    if (k < 0 || (p->L & 1) || p->M < 256) return FC_OK;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return FC_OK;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * p->L, (cuuint64_t)(p->M / 2)};
    const cuuint64_t strides[1] = {(cuuint64_t)2 * p->L * sizeof(float)};
    const cuuint32_t box[2] = {4, (cuuint32_t)tma_box_cols(p->M)};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&R.zmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, R.Z, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return FC_OK;
    int per_sm = 0, sms = 0;
    FC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, R.v.rinv[k].f, R.v.rinv[k].threads,
                                                         R.v.rinv[k].smem));
    FC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev));
    const int units = (p->L + 1) / 2;
    R.tma_grid = per_sm * sms < units ? per_sm * sms : units;
    R.tma_ok = R.tma_grid > 0;
    return FC_OK;
}

// Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1]: the roots
// of the Legendre polynomial P_n by Newton's method from the asymptotic
// guess cos(pi (i - 1/4) / (n + 1/2)), P_n and P_n' from the three-term
// recurrence, weights 2 / ((1 - x^2) P_n'(x)^2); in long double.
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        long double t = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (n + 0.5L));
        long double dp = 1.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const long double pk = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0L);
            const long double step = p1 / dp;
            t -= step;
            if (fabsl(step) < 1e-19L) break;
        }
        x[i] = (double)t;
        w[i] = (double)(2.0L / ((1.0L - t * t) * dp * dp));
    }
}

GaussLeg make_gauss_legendre() {
    GaussLeg g;
    gauss_legendre(16, g.x16, g.w16);
    gauss_legendre(8, g.x8, g.w8);
    gauss_legendre(4, g.x4, g.w4);
    return g;
}

}  // namespace

extern "C" int fftconv_plan_create(fftconv_plan** out, int L, int prec, const cg_tune* tune) {
    return fftconv_plan_create_green(out, L, prec, FC_GREEN_POINT, tune);
}

extern "C" int fftconv_plan_create_green(fftconv_plan** out, int L, int prec, int green_kind, const cg_tune* tune) {
    if (!out) return FC_EINVAL;
    *out = nullptr;
    if (L < 1 || L > 4096 || prec < 1 || prec > 3) return FC_EINVAL;
    if (green_kind != FC_GREEN_POINT && green_kind != FC_GREEN_CELL) return FC_EINVAL;
    fftconv_plan* p = new (std::nothrow) fftconv_plan();
    if (!p) return FC_ENOMEM;
    p->L = L;
    p->prec = prec;
    p->green = green_kind;
    p->M = 2;
    while (p->M < 2 * L) p->M *= 2;
    p->N = (long)L * L;
    const int M = p->M;
    const long N = p->N;
    const int Q = M / 2 + 1;
    int rc = FC_OK;
    cpx<double>* K = nullptr;
    double* maxes = nullptr;
    double* gt_tmp = nullptr;  // offset table of an FP32-only plan (kept as gtab otherwise)
    double hmax[2] = {0, 0};
    cudaStream_t cs = nullptr;  // set-up work stays off other streams (no device-wide syncs)
    cudaError_t e;
#define FC_TRY(x)                     \
    do {                              \
        rc = (x);                     \
        if (rc != FC_OK) goto fail;   \
    } while (0)
#define FC_TRYC(x)                                       \
    do {                                                 \
        e = (x);                                         \
        if (e != cudaSuccess) {                          \
            rc = set_cuda_err(e, #x);                    \
            goto fail;                                   \
        }                                                \
    } while (0)
    FC_TRYC(cudaGetDevice(&p->dev));
    FC_TRYC(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    p->setup = cs;
    // both precisions need FP64 set-up: the spectrum is built in FP64
    p->p64.on = true;
    p->p32.on = (prec & FC_F32) != 0;
    if (!get_variants<double>(M, &p->p64.v) || !get_variants<float>(M, &p->p32.v)) {
        rc = FC_EINVAL;
        goto fail;
    }
    FC_TRY(set_smem_attrs(p->p64.v));
    if (p->p32.on) FC_TRY(set_smem_attrs(p->p32.v));
    FC_TRY(dalloc(p, &p->p64.tw, sizeof(cpx<double>) * M));
    FC_TRY(dalloc(p, &p->p64.Gq, sizeof(double) * (size_t)Q * Q));
    if (p->p32.on) FC_TRY(dalloc(p, &p->p32.Gq, sizeof(float) * (size_t)Q * Q));
    // spectrum: kernel table -> unpruned FP64 2D FFT -> quarter / M^2
    e = dev_malloc_async((void**)&K, sizeof(cpx<double>) * (size_t)M * M, cs);
    if (e != cudaSuccess) {
        rc = FC_ENOMEM;
        set_cuda_err(e, "cudaMallocAsync(spectrum grid)");
        goto fail;
    }
    e = dev_malloc_async((void**)&maxes, 2 * sizeof(double), cs);
    if (e != cudaSuccess) {
        rc = FC_ENOMEM;
        set_cuda_err(e, "cudaMallocAsync(spectrum maxima)");
        goto fail;
    }
    FC_TRYC(cudaMemsetAsync(maxes, 0, 2 * sizeof(double), cs));
    k_twiddles<<<(M + 255) / 256, 256, 0, cs>>>(M, (cpx<double>*)p->p64.tw, nullptr);
    FC_TRYC(cudaGetLastError());
    FC_TRY(build_stage_tables<double>(p, p->p64, (const cpx<double>*)p->p64.tw, cs));
    if (p->p32.on) FC_TRY(build_stage_tables<float>(p, p->p32, (const cpx<double>*)p->p64.tw, cs));
    if (!p->p64.tables_ok(M) || (p->p32.on && !p->p32.tables_ok(M))) {
        snprintf(g_err, sizeof(g_err), "internal: a launch shape has no stage twiddle table (M=%d)", M);
        rc = FC_EINVAL;
        goto fail;
    }
    // Green's function on the site offsets (kept for the warm-start residual
    // update of FP64 plans), then its circulant embedding
    if (prec & FC_F64) {
        FC_TRY(dalloc(p, (void**)&p->gtab, sizeof(double) * N));
    } else {
        e = dev_malloc_async((void**)&gt_tmp, sizeof(double) * N, cs);
        if (e != cudaSuccess) {
            rc = FC_ENOMEM;
            set_cuda_err(e, "cudaMallocAsync(offset table)");
            goto fail;
        }
    }
    {
        double* gt = (prec & FC_F64) ? p->gtab : gt_tmp;
        k_green_table<<<(unsigned)((N + 255) / 256), 256, 0, cs>>>(L, p->green, make_gauss_legendre(), gt);
        FC_TRYC(cudaGetLastError());
        size_t MM = (size_t)M * M;
        k_kernel_table<<<(unsigned)((MM + 255) / 256), 256, 0, cs>>>(L, M, gt, K);
        FC_TRYC(cudaGetLastError());
        const KV& kr = p->p64.v.rows_full;
        const KV& kc = p->p64.v.cols_full;
        const void* twr = p->p64.tws(kr.E);
        const void* twc = p->p64.tws(kc.E);
        void* a1[2] = {(void*)&K, (void*)&twr};
        void* a2[2] = {(void*)&K, (void*)&twc};
        FC_TRYC(cudaLaunchKernel(kr.f, dim3((M + kr.per - 1) / kr.per), dim3(kr.threads), a1, kr.smem, cs));
        FC_TRYC(cudaLaunchKernel(kc.f, dim3(M / kc.per), dim3(kc.threads), a2, kc.smem, cs));
        k_spectrum_quarter<<<grid_1d((long)MM, 256), 256, 0, cs>>>(M, K, (double*)p->p64.Gq, (float*)p->p32.Gq,
                                                                         maxes);
        FC_TRYC(cudaGetLastError());
        FC_TRYC(cudaMemcpyAsync(hmax, maxes, sizeof(hmax), cudaMemcpyDeviceToHost, cs));
    }
    dev_free_async(K, cs);
    K = nullptr;
    dev_free_async(gt_tmp, cs);
    gt_tmp = nullptr;
    dev_free_async(maxes, cs);
    maxes = nullptr;
    FC_TRYC(cudaStreamSynchronize(cs));
    if (!(hmax[0] <= 1e-12 * hmax[1])) {
        snprintf(g_err, sizeof(g_err), "kernel spectrum not real: max|Im| %.3e, max|Re| %.3e", hmax[0], hmax[1]);
        rc = FC_ENANINF;
        goto fail;
    }
    // intermediates (half spectra, column-major) and solve workspace
    if (prec & FC_F64) FC_TRY(dalloc(p, &p->p64.Z, sizeof(cpx<double>) * (size_t)L * (M / 2)));
    if (p->p32.on) FC_TRY(dalloc(p, &p->p32.Z, sizeof(cpx<float>) * (size_t)L * (M / 2)));
    if (p->p32.on) FC_TRY(setup_tma(p));
    if (prec & FC_F64) {
        FC_TRY(dalloc(p, (void**)&p->x64, sizeof(double) * N));
        FC_TRY(dalloc(p, (void**)&p->r64, sizeof(double) * N));
        FC_TRY(dalloc(p, (void**)&p->p64v, sizeof(double) * N));
        FC_TRY(dalloc(p, (void**)&p->q64, sizeof(double) * N));
        FC_TRY(dalloc(p, (void**)&p->b64, sizeof(double) * N));
        FC_TRY(dalloc(p, (void**)&p->s64, sizeof(double) * N));
        FC_TRY(dalloc(p, (void**)&p->mask, N));
        FC_TRY(dalloc(p, (void**)&p->z64, sizeof(double) * N));
        FC_TRY(dalloc(p, (void**)&p->pq64, sizeof(double) * (size_t)Q * Q));
        FC_TRY(dalloc(p, (void**)&p->widx, sizeof(long long) * kWarmMax));
        FC_TRY(dalloc(p, (void**)&p->wdx, sizeof(double) * kWarmMax));
        if (p->p32.on) {
            FC_TRY(dalloc(p, (void**)&p->z32, sizeof(float) * N));
            FC_TRY(dalloc(p, (void**)&p->pq32, sizeof(float) * (size_t)Q * Q));
            FC_TRY(dalloc(p, (void**)&p->d32, sizeof(float) * N));
            FC_TRY(dalloc(p, (void**)&p->r32, sizeof(float) * N));
            FC_TRY(dalloc(p, (void**)&p->p32v, sizeof(float) * N));
            FC_TRY(dalloc(p, (void**)&p->q32, sizeof(float) * N));
            FC_TRY(dalloc(p, (void**)&p->s32, sizeof(float) * N));
        }
    }
    FC_TRY(dalloc(p, (void**)&p->st, sizeof(CgState)));
    FC_TRYC(cudaMemsetAsync(p->st, 0, sizeof(CgState), cs));
    {
        int g = L;  // row passes never use more blocks than rows
        FC_TRY(dalloc(p, (void**)&p->part, sizeof(double) * 3 * (size_t)(g + 1)));
        // 16 sites per thread (the FP32 estimate then skips most exact divisions)
        const long ag = (N + 4095) / 4096;
        p->am_grid = ag < 1 ? 1 : (ag > 2 * 148 ? 2 * 148 : (int)ag);
        FC_TRY(dalloc(p, (void**)&p->am_v, sizeof(double) * p->am_grid));
        FC_TRY(dalloc(p, (void**)&p->am_i, sizeof(long long) * p->am_grid));
        FC_TRY(dalloc(p, (void**)&p->am_ctl, sizeof(ArgmaxCtl)));
        FC_TRYC(cudaMemsetAsync(p->am_ctl, 0, sizeof(ArgmaxCtl), cs));
        FC_TRY(dalloc(p, (void**)&p->partA, sizeof(double) * 2 * kMaxPersistGrid));
        FC_TRY(dalloc(p, (void**)&p->partC, sizeof(double) * 5 * kMaxPersistGrid));
        FC_TRY(dalloc(p, (void**)&p->pctl, sizeof(PersistCtl)));
        FC_TRYC(cudaMemsetAsync(p->pctl, 0, sizeof(PersistCtl), cs));
    }
    if (!(prec & FC_F64)) {
        // FP32-only plan: drop the FP64 tables once the FP32 ones exist
        FC_TRYC(cudaStreamSynchronize(cs));
        dfree(p, p->p64.tw);
        dfree(p, p->p64.Gq);
        p->p64.tw = p->p64.Gq = nullptr;
        for (int i = 0; i < 6; ++i)
            if (p->p64.twst[i]) {
                dfree(p, p->p64.twst[i]);
                p->p64.twst[i] = nullptr;
            }
        p->p64.on = false;
    }
    e = host_malloc((void**)&p->st_host, sizeof(CgState));
    if (e == cudaSuccess) e = host_malloc((void**)&p->rm_host, sizeof(int64_t));
    if (e != cudaSuccess) {
        rc = FC_ENOMEM;
        set_cuda_err(e, "cudaMallocHost");
        goto fail;
    }
    FC_TRYC(cudaStreamSynchronize(cs));
    if (prec & FC_F64) {
        FC_TRY(autotune<double>(p, p->p64, tune));
        // FP64 has no batched tuning: batched solves take the single-problem
        // shapes (every FP64 shape has a batched twin), so that a problem's
        // FP64 arithmetic does not depend on the batch it joins
        for (int k = 0; k < 3; ++k) p->p64.sel_b[k] = p->p64.sel_cg[k];
        p->p64.tuned_b = true;
    }
    if (p->p32.on) FC_TRY(autotune<float>(p, p->p32, tune));
    if (prec & FC_F64) {
        const char* env = getenv("FC_AUTOTUNE");
        const bool timing = !(tune && tune->no_autotune) && !(env && !strcmp(env, "0"));
        const char* venv = getenv("FC_TUNE_VERBOSE");
        const bool verbose = venv && strcmp(venv, "0");
        const int forced = tune ? tune->shape_pers : 0;
        FC_TRY(choose_persistent<double>(p, p->p64, p->x64, p->r64, p->p64v, p->q64, p->s64, forced, timing, verbose));
        if (p->p32.on)
            FC_TRY(choose_persistent<float>(p, p->p32, p->d32, p->r32, p->p32v, p->q32, p->s32, forced, timing,
                                            verbose));
    }
    cudaStreamDestroy(cs);
    p->setup = nullptr;
    *out = p;
    return FC_OK;
fail:
    if (cs) {
        dev_free_async(K, cs);
        dev_free_async(maxes, cs);
        dev_free_async(gt_tmp, cs);
        cudaStreamSynchronize(cs);
    }
    plan_free(p);
    if (cs) cudaStreamDestroy(cs);
    return rc;
#undef FC_TRY
#undef FC_TRYC
}

extern "C" int fftconv_plan_destroy(fftconv_plan* p) {
    if (!p) return FC_EINVAL;
    cudaDeviceSynchronize();
    plan_free(p);
    return FC_OK;
}

extern "C" int fftconv_plan_info(const fftconv_plan* p, int* L, int* M, int* prec, size_t* bytes) {
    if (!p) return FC_EINVAL;
    if (L) *L = p->L;
    if (M) *M = p->M;
    if (prec) *prec = p->prec;
    if (bytes) *bytes = p->bytes + batch_bytes_of(p);
    return FC_OK;
}

extern "C" int fftconv_plan_shapes(const fftconv_plan* p, int prec, int n_shapes[3], int chosen[3], int radix[3],
                                   int per_block[3]) {
    if (!p || !n_shapes || !chosen || !radix || !per_block) return FC_EINVAL;
    const PrecRes* R = prec == FC_F32 ? (p->p32.on ? &p->p32 : nullptr) : (prec == FC_F64 && p->p64.on ? &p->p64 : nullptr);
    if (!R) return FC_EINVAL;
    const int n[3] = {R->v.n_rfwd, R->v.n_colc, R->v.n_rinv};
    const KV* k3[3] = {&R->rfwd(), &R->colc(), &R->rinv()};
    for (int i = 0; i < 3; ++i) {
        n_shapes[i] = n[i];
        chosen[i] = R->sel[i];
        radix[i] = k3[i]->E;
        per_block[i] = k3[i]->per;
    }
    return FC_OK;
}

extern "C" int fftconv_plan_shape_set(const fftconv_plan* p, int prec, int set, int chosen[3], int radix[3],
                                      int per_block[3], int* tuned) {
    if (!p || !chosen || !radix || !per_block || set < FC_SHAPES_APPLY || set > FC_SHAPES_BATCH) return FC_EINVAL;
    const PrecRes* R = prec == FC_F32 ? (p->p32.on ? &p->p32 : nullptr) : (prec == FC_F64 && p->p64.on ? &p->p64 : nullptr);
    if (!R) return FC_EINVAL;
    const int* sel = set == FC_SHAPES_APPLY ? R->sel : (set == FC_SHAPES_SOLVE ? R->sel_cg : R->sel_b);
    const KV* k3[3];
    if (set == FC_SHAPES_BATCH) {
        k3[0] = &R->v.rfwd_b[sel[0]];
        k3[1] = &R->v.colc_b[sel[1]];
        k3[2] = &R->v.rinv_b[sel[2]];
    } else {
        k3[0] = &R->v.rfwd[sel[0]];
        k3[1] = &R->v.colc[sel[1]];
        k3[2] = &R->v.rinv[sel[2]];
    }
    for (int i = 0; i < 3; ++i) {
        chosen[i] = sel[i];
        radix[i] = k3[i]->E;
        per_block[i] = k3[i]->per;
    }
    if (tuned) *tuned = set == FC_SHAPES_BATCH ? (R->tuned_b ? 1 : 0) : 1;
    return FC_OK;
}

extern "C" int fftconv_plan_solver(const fftconv_plan* p, int prec, int* n, int* chosen, int* threads, int* grid) {
    if (!p || !n || !chosen || !threads || !grid) return FC_EINVAL;
    const PrecRes* R = prec == FC_F32 ? (p->p32.on ? &p->p32 : nullptr) : (prec == FC_F64 && p->p64.on ? &p->p64 : nullptr);
    if (!R) return FC_EINVAL;
    *n = R->v.n_pers;
    *chosen = R->sel_pers;
    *threads = R->sel_pers >= 0 ? R->v.pers[R->sel_pers].threads : 0;
    *grid = R->sel_pers >= 0 ? R->pers_grid : 0;
    return FC_OK;
}

namespace {

template <typename T>
int apply_t(fftconv_plan* p, PrecRes& R, const T* x, T* y, cudaStream_t s) {
    RowFwdArgs<T> a{};
    a.L = p->L;
    a.mode = RF_PLAIN;
    a.x = x;
    a.st = p->st;
    a.part = p->part;
    const KV &ka = R.rfwd(), &kb = R.colc();
    KV kc = R.rinv();
    if (kc.fplain) kc.f = kc.fplain;  // the plain-apply forms
    a.Z = (cpx<T>*)R.Z;
    a.tw = (const cpx<T>*)R.tws(ka.E);
    int rc = launch(ka.fplain ? ka.fplain : ka.f, row_grid(p, ka), ka.threads, ka.smem, s, a);
    if (rc) return rc;
    ColArgs<T> b{p->L, (cpx<T>*)R.Z, (const T*)R.Gq, (const cpx<T>*)R.tws(kb.E)};
    rc = launch_dep(kb.f, col_grid(p, kb), kb.threads, kb.smem, s, b);
    if (rc) return rc;
    RowInvArgs<T> c{};
    c.L = p->L;
    c.mode = RI_PLAIN;
    c.y = y;
    c.st = p->st;
    c.part = p->part;
    c.Z = (const cpx<T>*)R.Z;
    c.tw = (const cpx<T>*)R.tws(kc.E);
    return launch_rinv<T>(p, R, kc, c, s, true);
}

}  // namespace

extern "C" int fftconv_apply_prec(fftconv_plan* p, int prec, const void* x, void* y, fc_stream_t stream) {
    if (!p || !x || !y) return FC_EINVAL;
    if (prec == FC_F32 && p->p32.on && p->p32.Z)
        return apply_t<float>(p, p->p32, (const float*)x, (float*)y, (cudaStream_t)stream);
    if (prec == FC_F64 && (p->prec & FC_F64))
        return apply_t<double>(p, p->p64, (const double*)x, (double*)y, (cudaStream_t)stream);
    return FC_EINVAL;
}

extern "C" int fftconv_apply(fftconv_plan* p, const void* x, void* y, fc_stream_t stream) {
    if (!p) return FC_EINVAL;
    return fftconv_apply_prec(p, (p->prec & FC_F32) ? FC_F32 : FC_F64, x, y, stream);
}

namespace {

// One CG product of Listing 2 as the solver's passes compute it: q = C p + s p
// with the pass-C sums p.q, r.q, q.q, on a state of its own.
template <typename T>
int cg_product_t(fftconv_plan* p, PrecRes& R, const T* pv, const T* rv, const T* sv, T* qv, double dots[3],
                 cudaStream_t s) {
    CgState* st = nullptr;
    if (dev_malloc_async((void**)&st, sizeof(CgState), s) != cudaSuccess) {
        set_cuda_err(cudaErrorMemoryAllocation, "cudaMallocAsync(state)");
        return FC_ENOMEM;
    }
    int rc = FC_OK;
    if (cudaMemsetAsync(st, 0, sizeof(CgState), s) != cudaSuccess) rc = set_cuda_err(cudaGetLastError(), "memset");
    const KV &ka = R.rfwd_cg(), &kb = R.colc_cg(), &kc = R.rinv_cg();
    if (!rc) {
        RowFwdArgs<T> a{};
        a.L = p->L;
        a.mode = RF_PLAIN;
        a.x = pv;
        a.st = st;
        a.part = p->part;
        a.Z = (cpx<T>*)R.Z;
        a.tw = (const cpx<T>*)R.tws(ka.E);
        rc = launch(ka.f, row_grid(p, ka), ka.threads, ka.smem, s, a);
    }
    if (!rc) {
        ColArgs<T> b{p->L, (cpx<T>*)R.Z, (const T*)R.Gq, (const cpx<T>*)R.tws(kb.E)};
        rc = launch_dep(kb.f, col_grid(p, kb), kb.threads, kb.smem, s, b);
    }
    if (!rc) {
        RowInvArgs<T> c{};
        c.L = p->L;
        c.mode = RI_CG;
        c.s = sv;
        c.cp = pv;
        c.cr = rv;
        c.cq = qv;
        c.st = st;
        c.part = p->part;
        c.Z = (const cpx<T>*)R.Z;
        c.tw = (const cpx<T>*)R.tws(kc.E);
        rc = launch_rinv<T>(p, R, kc, c, s, true);
    }
    CgState h;
    if (!rc && cudaMemcpyAsync(&h, st, sizeof(CgState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = set_cuda_err(cudaGetLastError(), "cudaMemcpyAsync(state)");
    dev_free_async(st, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = set_cuda_err(cudaGetLastError(), "cg product");
    if (!rc) {
        dots[0] = h.pq;
        dots[1] = h.rq;
        dots[2] = h.qq;
    }
    return rc;
}

}  // namespace

extern "C" int fftconv_cg_product(fftconv_plan* p, int prec, const void* pvec, const void* rvec, const void* s,
                                  void* q, double dots[3], fc_stream_t stream) {
    if (!p || !pvec || !rvec || !s || !q || !dots || !(prec == FC_F32 || prec == FC_F64)) return FC_EINVAL;
    PrecRes& R = prec == FC_F32 ? p->p32 : p->p64;
    if (!R.on) return FC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == FC_F32)
        return cg_product_t<float>(p, R, (const float*)pvec, (const float*)rvec, (const float*)s, (float*)q, dots, st);
    return cg_product_t<double>(p, R, (const double*)pvec, (const double*)rvec, (const double*)s, (double*)q, dots,
                                st);
}

// ------------------------------------------------- persistent inner CG --

namespace {

template <typename T>
PersistArgs<T> make_pargs(fftconv_plan* p, PrecRes& R, const KVP& kp, T* cx, T* cr, T* cp, T* cq, const T* s,
                          const double* r64start) {
    PersistArgs<T> P{};
    P.A.L = p->L;
    P.A.mode = RF_CG;
    P.A.cx = cx;
    P.A.cr = cr;
    P.A.cp = cp;
    P.A.cq = cq;
    P.A.r64 = r64start;
    P.A.st = p->st;
    P.A.part = p->part;
    P.A.Z = (cpx<T>*)R.Z;
    P.A.tw = (const cpx<T>*)R.tws(kp.EA);
    P.B = ColArgs<T>{p->L, (cpx<T>*)R.Z, (const T*)R.Gq, (const cpx<T>*)R.tws(kp.EB)};
    P.C.L = p->L;
    P.C.mode = RI_CG;
    P.C.s = s;
    P.C.cp = cp;
    P.C.cr = cr;
    P.C.cq = cq;
    P.C.mask = p->mask;
    P.C.st = p->st;
    P.C.part = p->part;
    P.C.Z = (const cpx<T>*)R.Z;
    P.C.tw = (const cpx<T>*)R.tws(kp.EA);
    P.nA = ((p->L + 1) / 2 + kp.RB - 1) / kp.RB;
    P.nB = (p->M / 2) / kp.CB;
    P.partA = p->partA;
    P.partC = p->partC;
    P.ctl = p->pctl;
    P.N = p->N;
    return P;
}

// Resident blocks of a persistent kernel (its cooperative grid), at most one
// per unit of work; 0 if it cannot be resident at all.
int pers_grid(fftconv_plan* p, const KVP& kp) {
    int nb = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kp.f, kp.threads, kp.smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev) != cudaSuccess) return 0;
    long g = (long)nb * sms;
    const long nA = ((p->L + 1) / 2 + kp.RB - 1) / kp.RB, nB = (p->M / 2) / kp.CB;
    const long units = nA > nB ? nA : nB;
    if (g > units) g = units;
    if (g > kMaxPersistGrid) g = kMaxPersistGrid;
    return (int)g;
}

// Time K inner iterations of each persistent variant on the plan's own size
// (r = 1, s = 1, all sites active) and keep the fastest; cached like the
// pass shapes.  forced: 0 tuned, k > 0 variant k-1, < 0 none (graph loop).
template <typename T>
int choose_persistent(fftconv_plan* p, PrecRes& R, T* cx, T* cr, T* cp, T* cq, T* s, int forced, bool timing,
                      bool verbose) {
    R.sel_pers = -1;
    const int n = R.v.n_pers;
    if (n == 0 || forced < 0) return FC_OK;
    if (forced > 0) {
        if (forced > n) return FC_OK;  // this precision has fewer kernels: graph loop
        R.sel_pers = forced - 1;
        R.pers_grid = pers_grid(p, R.v.pers[R.sel_pers]);
        if (R.pers_grid < 1) R.sel_pers = -1;
        return FC_OK;
    }
    char key[96];
    snprintf(key, sizeof(key), "%s M=%d L=%d pers n=%d ", sizeof(T) == 4 ? "f32" : "f64", p->M, p->L, n);
    int idx = -1;
    if (tune_lookup(key, &idx) && idx >= 0 && idx < n && pers_grid(p, R.v.pers[idx]) > 0) {
        R.sel_pers = idx;
        R.pers_grid = pers_grid(p, R.v.pers[idx]);
        return FC_OK;
    }
    if (!timing) {
        for (int k = 0; k < n; ++k)
            if (pers_grid(p, R.v.pers[k]) > 0) {
                R.sel_pers = k;
                R.pers_grid = pers_grid(p, R.v.pers[k]);
                return FC_OK;
            }
        return FC_OK;
    }
    const long N = p->N;
    const int K = 12;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FC_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    FC_CK(cudaEventCreate(&e0));
    FC_CK(cudaEventCreate(&e1));
    const int g1 = grid_1d(N, 256);
    k_fill<T><<<g1, 256, 0, st>>>(N, cr, (T)1);
    k_fill<T><<<g1, 256, 0, st>>>(N, cp, (T)0);
    k_fill<T><<<g1, 256, 0, st>>>(N, cq, (T)0);
    k_fill<T><<<g1, 256, 0, st>>>(N, cx, (T)0);
    k_fill<T><<<g1, 256, 0, st>>>(N, s, (T)1);
    k_fill_u8<<<g1, 256, 0, st>>>(N, p->mask, 1);
    CgState h{};
    h.first = 1;
    h.tol2 = 0.0;
    h.cycle_max = K;
    h.max_iter = 1 << 30;
    h.sigma = 1.0;
    *p->st_host = h;
    float best = 1e30f;
    int bi = -1, rc = FC_OK;
    for (int k = 0; k < n && !rc; ++k) {
        const KVP& kp = R.v.pers[k];
        const int grid = pers_grid(p, kp);
        if (grid < 1) continue;
        PersistArgs<T> P = make_pargs<T>(p, R, kp, cx, cr, cp, cq, s, nullptr);
        void* args[1] = {(void*)&P};
        float ms = 0;
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            if (cudaMemcpyAsync(p->st, p->st_host, sizeof(CgState), cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemsetAsync(p->pctl, 0, sizeof(PersistCtl), st) != cudaSuccess ||
                cudaEventRecord(e0, st) != cudaSuccess ||
                cudaLaunchCooperativeKernel(kp.f, dim3(grid), dim3(kp.threads), args, kp.smem, st) != cudaSuccess ||
                cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = set_cuda_err(cudaGetLastError(), "persistent tuning launch");
        }
        if (rc) break;
        if (verbose)
            fprintf(stderr, "[fftconv tune] %spersistent %d (EA=%d RB=%d EB=%d CB=%d threads=%d grid=%d smem=%zu): %.3f us/iter\n",
                    key, k, kp.EA, kp.RB, kp.EB, kp.CB, kp.threads, grid, kp.smem, ms * 1e3f / K);
        if (ms < best) {
            best = ms;
            bi = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc) return rc;
    if (bi >= 0) {
        R.sel_pers = bi;
        R.pers_grid = pers_grid(p, R.v.pers[bi]);
        tune_store(key, bi);
    }
    return FC_OK;
}

}  // namespace

// ------------------------------------------------------------- CG graph --

namespace {

struct GraphBuilder {
    int rc = FC_OK;
    bool pdl = false;  // programmatic edges between consecutive passes
    template <typename... A>
    cudaGraphNode_t kernel(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, const void* f, dim3 grid,
                           int threads, size_t smem, const A&... args) {
        cudaGraphNode_t n = nullptr;
        if (rc) return n;
        cudaKernelNodeParams kp{};
        kp.func = (void*)f;
        kp.gridDim = grid;
        kp.blockDim = dim3(threads);
        kp.sharedMemBytes = (unsigned)smem;
        void* args_[] = {(void*)&args...};
        kp.kernelParams = args_;
        cudaError_t e = cudaGraphAddKernelNode(&n, g, deps, ndeps, &kp);
        if (e != cudaSuccess) rc = set_cuda_err(e, "cudaGraphAddKernelNode");
        return n;
    }
    // A pass that follows another pass (a kernel node that starts with
    // pdl_enter): with pdl, a programmatic edge from the previous pass's
    // trigger port, otherwise an ordinary edge.
    template <typename... A>
    cudaGraphNode_t pass(cudaGraph_t g, cudaGraphNode_t prev, const void* f, dim3 grid, int threads, size_t smem,
                         const A&... args) {
        if (!pdl) return kernel(g, &prev, 1, f, grid, threads, smem, args...);
        cudaGraphNode_t n = kernel(g, nullptr, 0, f, grid, threads, smem, args...);
        if (rc) return n;
        cudaGraphEdgeData ed{};
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
        cudaError_t e = cudaGraphAddDependencies(g, &prev, &n, &ed, 1);
        if (e != cudaSuccess) rc = set_cuda_err(e, "cudaGraphAddDependencies(programmatic)");
        return n;
    }
    // A conditional node: WHILE (the body runs while the handle is non-zero)
    // or, with once, IF (the body runs once if it is).
    cudaGraph_t while_node(cudaGraph_t g, const cudaGraphNode_t* deps, int ndeps, cudaGraphConditionalHandle h,
                           cudaGraphNode_t* node, bool once = false) {
        if (rc) return nullptr;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = once ? cudaGraphCondTypeIf : cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaError_t e = cudaGraphAddNode(node, g, deps, nullptr, ndeps, &np);
        if (e != cudaSuccess) {
            rc = set_cuda_err(e, once ? "cudaGraphAddNode(if)" : "cudaGraphAddNode(while)");
            return nullptr;
        }
        return np.conditional.phGraph_out[0];
    }
};

// The buffers a solve graph works on: the plan's own workspace (one problem)
// or a batch workspace (nb problems of the plan's size; problem k at offset
// k * stride in every buffer and blockIdx.y = k in every pass).  Batched
// passes are gated per problem (a finished problem skips the true-residual
// passes, an idle one the inner passes), and the loops run while any
// problem needs them (k_batch_ctl).
struct SolveView {
    int nb = 1;
    bool batched = false;
    BatchStride bs{};
    double *x64 = nullptr, *r64 = nullptr, *p64v = nullptr, *q64 = nullptr, *b64 = nullptr, *s64 = nullptr;
    double *z64 = nullptr, *pq64 = nullptr;
    float *d32 = nullptr, *r32 = nullptr, *p32v = nullptr, *q32 = nullptr, *s32 = nullptr, *z32 = nullptr;
    float* pq32 = nullptr;
    uint8_t* mask = nullptr;
    void *Z32 = nullptr, *Z64 = nullptr;
    CgState* st = nullptr;
    double* part = nullptr;
    template <typename T>
    cpx<T>* Z() const {
        return (cpx<T>*)(sizeof(T) == 4 ? Z32 : Z64);
    }
    // batched launches' second argument: the inner passes skip idle
    // problems, the true-residual passes finished ones; the kernel spectrum
    // is one for all problems, the preconditioner's is per problem
    BatchArgs inner(bool shared_spectrum = false) const {
        BatchArgs b{GATE_IDLE, bs};
        if (shared_spectrum) b.bs.q = 0;
        return b;
    }
    BatchArgs outer() const {
        BatchArgs b{GATE_FINISHED, bs};
        b.bs.q = 0;
        return b;
    }
    dim3 grid(int gx) const { return dim3((unsigned)gx, (unsigned)nb); }
};

// A pass node following prev (nullptr: the first node of a body): its
// arguments, and for batched solves the batch argument bb.
template <typename A>
cudaGraphNode_t pass_node(GraphBuilder& gb, cudaGraph_t g, cudaGraphNode_t prev, const KV& k, dim3 grid,
                          const SolveView& V, const A& args, const BatchArgs& bb) {
    if (V.batched)
        return prev ? gb.pass(g, prev, k.f, grid, k.threads, k.smem, args, bb)
                    : gb.kernel(g, nullptr, 0, k.f, grid, k.threads, k.smem, args, bb);
    return prev ? gb.pass(g, prev, k.f, grid, k.threads, k.smem, args)
                : gb.kernel(g, nullptr, 0, k.f, grid, k.threads, k.smem, args);
}

SolveView plan_view(fftconv_plan* p) {
    SolveView v;
    v.x64 = p->x64, v.r64 = p->r64, v.p64v = p->p64v, v.q64 = p->q64, v.b64 = p->b64, v.s64 = p->s64;
    v.z64 = p->z64, v.pq64 = p->pq64;
    v.d32 = p->d32, v.r32 = p->r32, v.p32v = p->p32v, v.q32 = p->q32, v.s32 = p->s32, v.z32 = p->z32;
    v.pq32 = p->pq32;
    v.mask = p->mask;
    v.Z32 = p->p32.Z, v.Z64 = p->p64.Z;
    v.st = p->st, v.part = p->part;
    return v;
}

// The launch shapes of a solve graph: the tuned ones, or for batched solves
// the batched forms of the standard shapes.
const KV& rfwd_shape(const PrecRes& R, bool batched) { return batched ? R.v.rfwd_b[R.sel_b[0]] : R.rfwd_cg(); }
const KV& colc_shape(const PrecRes& R, bool batched) { return batched ? R.v.colc_b[R.sel_b[1]] : R.colc_cg(); }
const KV& rinv_shape(const PrecRes& R, bool batched) { return batched ? R.v.rinv_b[R.sel_b[2]] : R.rinv_cg(); }

// Pass C as a graph node following prev (the TMA-staged shape gets its
// tensor-map arguments).
template <typename T>
cudaGraphNode_t graph_rinv(GraphBuilder& gb, cudaGraph_t g, cudaGraphNode_t prev, fftconv_plan* p, PrecRes& R,
                           const KV& kc, const SolveView& V, const RowInvArgs<T>& c, const BatchArgs& bb) {
    if constexpr (sizeof(T) == 4) {
        if (kc.tma) {
            const RowInvTma P = tma_args(p, R, c);
            return gb.pass(g, prev, kc.f, dim3(R.tma_grid), kc.threads, kc.smem, P);
        }
    }
    return pass_node(gb, g, prev, kc, V.grid(row_grid(p, kc)), V, c, bb);
}

// After the deciding pass of a batched loop body: the loop control node.
void batch_ctl_node(GraphBuilder& gb, cudaGraph_t g, cudaGraphNode_t prev, const SolveView& V,
                    cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_inner, cudaGraphNode_t* out) {
    const int nb = V.nb;
    const CgState* cst = V.st;
    const unsigned long long ho = h_outer, hi = h_inner;
    cudaGraphNode_t n = gb.kernel(g, &prev, 1, (const void*)k_batch_ctl, dim3(1), 256, 0, nb, cst, ho, hi);
    if (out) *out = n;
}

// Inner CG loop body (Listing 2): pass A (update + row FFT), B, C (product,
// dot products, step decision).
template <typename T>
void add_inner_body(GraphBuilder& gb, cudaGraph_t body, fftconv_plan* p, PrecRes& R, const SolveView& V, T* cx,
                    T* cr, T* cp, T* cq, const T* s, const double* r64_start, cudaGraphConditionalHandle h_inner) {
    const KV &ka = rfwd_shape(R, V.batched), &kb = colc_shape(R, V.batched), &kc = rinv_shape(R, V.batched);
    RowFwdArgs<T> a{};
    a.L = p->L;
    a.mode = RF_CG;
    a.cx = cx;
    a.cr = cr;
    a.cp = cp;
    a.cq = cq;
    a.r64 = r64_start;
    a.st = V.st;
    a.part = V.part;
    a.Z = V.Z<T>();
    a.tw = (const cpx<T>*)R.tws(ka.E);
    cudaGraphNode_t nA = pass_node(gb, body, nullptr, ka, V.grid(row_grid(p, ka)), V, a, V.inner());
    ColArgs<T> b{p->L, V.Z<T>(), (const T*)R.Gq, (const cpx<T>*)R.tws(kb.E), V.st, 0};
    cudaGraphNode_t nB = pass_node(gb, body, nA, kb, V.grid(col_grid(p, kb)), V, b, V.inner(true));
    RowInvArgs<T> c{};
    c.L = p->L;
    c.mode = RI_CG;
    c.s = s;
    c.cp = cp;
    c.cr = cr;
    c.cq = cq;
    c.mask = V.mask;
    c.st = V.st;
    c.part = V.part;
    c.h_inner = V.batched ? 0 : h_inner;
    c.Z = V.Z<T>();
    c.tw = (const cpx<T>*)R.tws(kc.E);
    cudaGraphNode_t nC = graph_rinv<T>(gb, body, nB, p, R, kc, V, c, V.inner());
    if (V.batched) batch_ctl_node(gb, body, nC, V, 0, h_inner, nullptr);
}

// The inner loop body of preconditioned CG (pcg_zr_eval, pcg_alpha_eval):
// A1 (alpha from C2's p.q; x += alpha p, r -= alpha q, or at the start of a
// run r from the true residual; transform r) -> B1 with the preconditioner
// spectrum -> C1 (z = M^-1 r; publishes r.z and r.r) -> A2 (beta and the
// stopping test on r.r, the loop condition; p = z + beta p; transform p) ->
// B2 with the kernel spectrum (moves r.z into place) -> C2 (q = A p;
// publishes p.q).  Once A2 has ended the run it returns, and so do B2 and
// C2; x already holds the last update.  Batched: the loop control node
// follows A2.
template <typename T>
void add_inner_body_pcg(GraphBuilder& gb, cudaGraph_t body, fftconv_plan* p, PrecRes& R, const SolveView& V, T* cx,
                        T* cr, T* cp, T* cq, T* cz, const T* s, const T* pq, const double* r64_start,
                        cudaGraphConditionalHandle h_inner) {
    const KV &kb = colc_shape(R, V.batched), &kc = rinv_shape(R, V.batched);
    // single problem: the pass-A kernel that takes the step decision (the
    // batched twin takes it itself)
    KV ka = rfwd_shape(R, V.batched);
    if (!V.batched && ka.fp) ka.f = ka.fp;
    // blocks of pass C, whose partial sums the passes A add up
    int npart = row_grid(p, kc);
    if constexpr (sizeof(T) == 4)
        if (kc.tma) npart = R.tma_grid;
    RowFwdArgs<T> a1{};
    a1.L = p->L;
    a1.mode = RF_PCG_R;
    a1.cx = cx;
    a1.cr = cr;
    a1.cp = cp;
    a1.cq = cq;
    a1.r64 = r64_start;
    a1.st = V.st;
    a1.part = V.part;
    a1.npart = npart;
    a1.Z = V.Z<T>();
    a1.tw = (const cpx<T>*)R.tws(ka.E);
    cudaGraphNode_t n1 = pass_node(gb, body, nullptr, ka, V.grid(row_grid(p, ka)), V, a1, V.inner());
    ColArgs<T> b1{p->L, V.Z<T>(), pq, (const cpx<T>*)R.tws(kb.E), V.st, 0};
    cudaGraphNode_t n2 = pass_node(gb, body, n1, kb, V.grid(col_grid(p, kb)), V, b1, V.inner());
    RowInvArgs<T> c1{};
    c1.L = p->L;
    c1.mode = RI_PCG_Z;
    c1.cr = cr;
    c1.cz = cz;
    c1.mask = V.mask;
    c1.st = V.st;
    c1.part = V.part;
    c1.Z = V.Z<T>();
    c1.tw = (const cpx<T>*)R.tws(kc.E);
    cudaGraphNode_t n3 = graph_rinv<T>(gb, body, n2, p, R, kc, V, c1, V.inner());
    RowFwdArgs<T> a2{};
    a2.L = p->L;
    a2.mode = RF_PCG_P;
    a2.cp = cp;
    a2.cr = cr;
    a2.cz = cz;
    a2.st = V.st;
    a2.part = V.part;
    a2.npart = npart;
    a2.h_inner = V.batched ? 0 : h_inner;
    a2.Z = V.Z<T>();
    a2.tw = (const cpx<T>*)R.tws(ka.E);
    cudaGraphNode_t n4 = pass_node(gb, body, n3, ka, V.grid(row_grid(p, ka)), V, a2, V.inner());
    // the single-problem column pass returns at entry once the run has ended
    ColArgs<T> b2{p->L, V.Z<T>(), (const T*)R.Gq, (const cpx<T>*)R.tws(kb.E), V.st, V.batched ? 0 : GATE_IDLE, 1};
    cudaGraphNode_t n5;
    if (V.batched) {
        batch_ctl_node(gb, body, n4, V, 0, h_inner, &n4);
        n5 = gb.kernel(body, &n4, 1, kb.f, V.grid(col_grid(p, kb)), kb.threads, kb.smem, b2, V.inner(true));
    } else {
        n5 = pass_node(gb, body, n4, kb, V.grid(col_grid(p, kb)), V, b2, V.inner(true));
    }
    RowInvArgs<T> c2{};
    c2.L = p->L;
    c2.mode = RI_PQ;
    c2.s = s;
    c2.cp = cp;
    c2.cq = cq;
    c2.mask = V.mask;
    c2.st = V.st;
    c2.part = V.part;
    c2.Z = V.Z<T>();
    c2.tw = (const cpx<T>*)R.tws(kc.E);
    graph_rinv<T>(gb, body, n5, p, R, kc, V, c2, V.inner());
}

// Add one solve (prologue, outer loop) to graph g as a branch with no
// dependencies: its own conditional handles, its own buffers V.
int add_solve_nodes(fftconv_plan* p, const SolveView& V, int mode, bool precond, bool pdl, cudaGraph_t g) {
    GraphBuilder gb;
    gb.pdl = pdl;
    cudaGraphConditionalHandle h_outer = 0, h_inner = 0;
    cudaGraphNode_t nPro = nullptr, nOuter = nullptr;
    const long N = p->N;
    const bool mixed = mode == FC_MODE_MIXED;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h_outer, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return set_cuda_err(e, "cudaGraphConditionalHandleCreate");
    int ndeps = 0;
    if (mixed) {
        // FP32 copy of the diagonal for the inner products (all problems)
        const double* sa = V.s64;
        float* sb = V.s32;
        const long NA = N * V.nb;
        const CgState* sst = V.batched ? nullptr : V.st;  // batches always convert
        nPro = gb.kernel(g, nullptr, 0, (const void*)k_f64_to_f32, dim3(grid_1d(NA, 256)), 256, 0, NA, sa, sb, sst);
        ndeps = 1;
    }
    if (precond) {
        // preconditioner shift c = 0.6 x mean active s, then its spectrum quarter
        const double* sa = V.s64;
        const uint8_t* mk = V.mask;
        double* pt = V.part;
        CgState* cst = V.st;
        const long bpart = V.bs.part;
        int gm = grid_1d(N, 256);
        if (gm > 512) gm = 512;
        if (gm > 3 * (p->L + 1) / 2) gm = 3 * (p->L + 1) / 2;  // the partial-sum buffer holds 3 (L+1) doubles
        cudaGraphNode_t nm;
        if (mixed) {  // from the FP32 copy of s the prologue has just made
            const float* s32 = V.s32;
            nm = gb.kernel(g, &nPro, 1, (const void*)k_active_mean_f32, V.grid(gm), 256, 0, N, s32, mk, pt, cst,
                           bpart);
        } else {
            nm = gb.kernel(g, ndeps ? &nPro : nullptr, ndeps, (const void*)k_active_mean, V.grid(gm), 256, 0, N, sa,
                           mk, pt, cst, bpart);
        }
        const long QQ = (long)(p->M / 2 + 1) * (p->M / 2 + 1);
        const double MM = (double)p->M * (double)p->M;
        const double* g64 = (const double*)p->p64.Gq;
        const CgState* ccst = V.st;
        if (mixed) {
            float* pq = V.pq32;
            const float MMf = (float)MM;  // M^2 <= 2^26: exact
            const float* g32 = (const float*)p->p32.Gq;
            nPro = gb.kernel(g, &nm, 1, (const void*)k_precond_spectrum_f32, V.grid(grid_1d(QQ, 256)), 256, 0, QQ,
                             MMf, g32, ccst, pq);
        } else {
            double* pq = V.pq64;
            nPro = gb.kernel(g, &nm, 1, (const void*)k_precond_spectrum<double>, V.grid(grid_1d(QQ, 256)), 256, 0,
                             QQ, MM, g64, ccst, pq);
        }
        ndeps = 1;
    }
    cudaGraph_t outer = gb.while_node(g, ndeps ? &nPro : nullptr, ndeps, h_outer, &nOuter);
    if (!gb.rc) {
        e = cudaGraphConditionalHandleCreate(&h_inner, outer, 0, 0);
        if (e != cudaSuccess) gb.rc = set_cuda_err(e, "cudaGraphConditionalHandleCreate(inner)");
    }
    if (!gb.rc) {
        const KV &ka = rfwd_shape(p->p64, V.batched), &kb = colc_shape(p->p64, V.batched),
                 &kc = rinv_shape(p->p64, V.batched);
        RowFwdArgs<double> a{};
        a.L = p->L;
        a.mode = RF_XUPD;
        a.x64 = V.x64;
        a.d32 = mixed ? V.d32 : nullptr;
        a.mask = V.mask;
        a.st = V.st;
        a.part = V.part;
        a.Z = V.Z<double>();
        a.tw = (const cpx<double>*)p->p64.tws(ka.E);
        // the mask is applied to x in the same pass (x = 0 off the active set)
        cudaGraphNode_t nA = pass_node(gb, outer, nullptr, ka, V.grid(row_grid(p, ka)), V, a, V.outer());
        ColArgs<double> b{p->L, V.Z<double>(), (const double*)p->p64.Gq, (const cpx<double>*)p->p64.tws(kb.E), V.st,
                          GATE_WARM};
        cudaGraphNode_t nB = pass_node(gb, outer, nA, kb, V.grid(col_grid(p, kb)), V, b, V.outer());
        RowInvArgs<double> c{};
        c.L = p->L;
        c.mode = RI_RESID;
        c.mask = V.mask;
        c.x64 = V.x64;
        c.b64 = V.b64;
        c.s64 = V.s64;
        c.r64 = V.r64;
        c.st = V.st;
        c.part = V.part;
        c.h_outer = V.batched ? 0 : h_outer;
        c.h_inner = V.batched ? 0 : h_inner;
        c.Z = V.Z<double>();
        c.tw = (const cpx<double>*)p->p64.tws(kc.E);
        cudaGraphNode_t nC = pass_node(gb, outer, nB, kc, V.grid(row_grid(p, kc)), V, c, V.outer());
        if (V.batched) batch_ctl_node(gb, outer, nC, V, h_outer, h_inner, &nC);
        cudaGraphNode_t nInner = nullptr;
        cudaGraph_t inner = gb.while_node(outer, &nC, 1, h_inner, &nInner);
        if (!gb.rc) {
            if (mixed && precond)
                add_inner_body_pcg<float>(gb, inner, p, p->p32, V, V.d32, V.r32, V.p32v, V.q32, V.z32, V.s32, V.pq32,
                                          V.r64, h_inner);
            else if (precond)
                add_inner_body_pcg<double>(gb, inner, p, p->p64, V, V.x64, V.r64, V.p64v, V.q64, V.z64, V.s64,
                                           V.pq64, nullptr, h_inner);
            else if (mixed)
                add_inner_body<float>(gb, inner, p, p->p32, V, V.d32, V.r32, V.p32v, V.q32, V.s32, V.r64, h_inner);
            else
                add_inner_body<double>(gb, inner, p, p->p64, V, V.x64, V.r64, V.p64v, V.q64, V.s64, nullptr,
                                       h_inner);
        }
        const CgState* cst = V.st;
        if (precond) {
            // the residual half updates x before each stopping test: nothing left to apply
        } else if (mixed) {
            float* fx = V.d32;
            const float* fp = V.p32v;
            gb.kernel(outer, &nInner, 1, (const void*)k_cg_final<float>, V.grid(grid_1d(N, 256)), 256, 0, N, cst, fx,
                      fp);
        } else {
            double* fx = V.x64;
            const double* fp = V.p64v;
            gb.kernel(outer, &nInner, 1, (const void*)k_cg_final<double>, V.grid(grid_1d(N, 256)), 256, 0, N, cst,
                      fx, fp);
        }
    }
    return gb.rc;
}

// Build the solve graph for one mode on the buffers of V:
//   [prologue] -> while(outer) { A64 (fold correction, mask, FFT x) -> B64 ->
//                                C64 (true residual, decide) ->
//                                while(inner) { A -> B -> C } -> final }
// (batched: a loop control node after C64 and after each inner body).
int build_graph_with(fftconv_plan* p, const SolveView& V, int mode, bool precond, bool pdl, cudaGraph_t* gout,
                     cudaGraphExec_t* eout) {
    cudaGraph_t g = nullptr;
    FC_CK(cudaGraphCreate(&g, 0));
    int rc = add_solve_nodes(p, V, mode, precond, pdl, g);
    if (rc) {
        cudaGraphDestroy(g);
        return rc;
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return set_cuda_err(e, "cudaGraphInstantiate");
    }
    *gout = g;
    *eout = ex;
    return FC_OK;
}

// The solve graph with programmatic edges between passes where the driver
// accepts them inside the conditional bodies, else with ordinary edges.
int build_graph_view(fftconv_plan* p, const SolveView& V, int mode, bool precond, cudaGraph_t* g,
                     cudaGraphExec_t* ex) {
    if (pdl_on() && build_graph_with(p, V, mode, precond, true, g, ex) == FC_OK) return FC_OK;
    return build_graph_with(p, V, mode, precond, false, g, ex);
}

int build_graph(fftconv_plan* p, int mode, bool precond) {
    const int gi = mode + 2 * precond;
    return build_graph_view(p, plan_view(p), mode, precond, &p->graph[gi], &p->gexec[gi]);
}

}  // namespace

namespace {

// FP64 true residual r = P (b - A x) after folding the last correction into
// x, with the refinement decision (passes A, B, C in RESID mode).
int launch_resid_chain(fftconv_plan* p, bool mixed, cudaStream_t st) {
    const KV &ka = p->p64.rfwd(), &kb = p->p64.colc(), &kc = p->p64.rinv();
    RowFwdArgs<double> a{};
    a.L = p->L;
    a.mode = RF_XUPD;
    a.x64 = p->x64;
    a.d32 = mixed ? p->d32 : nullptr;
    a.mask = p->mask;
    a.st = p->st;
    a.part = p->part;
    a.Z = (cpx<double>*)p->p64.Z;
    a.tw = (const cpx<double>*)p->p64.tws(ka.E);
    int rc = launch(ka.f, row_grid(p, ka), ka.threads, ka.smem, st, a);
    if (rc) return rc;
    ColArgs<double> b{p->L, (cpx<double>*)p->p64.Z, (const double*)p->p64.Gq, (const cpx<double>*)p->p64.tws(kb.E),
                      p->st, GATE_WARM};
    rc = launch(kb.f, col_grid(p, kb), kb.threads, kb.smem, st, b);
    if (rc) return rc;
    RowInvArgs<double> c{};
    c.L = p->L;
    c.mode = RI_RESID;
    c.mask = p->mask;
    c.x64 = p->x64;
    c.b64 = p->b64;
    c.s64 = p->s64;
    c.r64 = p->r64;
    c.st = p->st;
    c.part = p->part;
    c.Z = (const cpx<double>*)p->p64.Z;
    c.tw = (const cpx<double>*)p->p64.tws(kc.E);
    return launch(kc.f, row_grid(p, kc), kc.threads, kc.smem, st, c);
}

// One inner CG run as a cooperative launch of the persistent kernel (it
// returns at once when the outer loop has finished).
int launch_persistent(fftconv_plan* p, bool mixed, cudaStream_t st) {
    PrecRes& R = mixed ? p->p32 : p->p64;
    const KVP& kp = R.v.pers[R.sel_pers];
    if (mixed) {
        PersistArgs<float> pa = make_pargs<float>(p, R, kp, p->d32, p->r32, p->p32v, p->q32, p->s32, p->r64);
        void* args[1] = {(void*)&pa};
        FC_CK(cudaLaunchCooperativeKernel(kp.f, dim3(R.pers_grid), dim3(kp.threads), args, kp.smem, st));
    } else {
        PersistArgs<double> pa = make_pargs<double>(p, R, kp, p->x64, p->r64, p->p64v, p->q64, p->s64, nullptr);
        void* args[1] = {(void*)&pa};
        FC_CK(cudaLaunchCooperativeKernel(kp.f, dim3(R.pers_grid), dim3(kp.threads), args, kp.smem, st));
    }
    return FC_OK;
}

}  // namespace

// Wait until the work queued on st is done: spinning (the default, lowest
// latency) or, after fftconv_plan_sync_mode(p, 1), blocking the thread.
static cudaError_t wait_stream(fftconv_plan* p, cudaStream_t st) {
    if (!p->blocking) return cudaStreamSynchronize(st);
    cudaError_t e = cudaEventRecord(p->ev_wait, st);
    return e != cudaSuccess ? e : cudaEventSynchronize(p->ev_wait);
}

extern "C" int fftconv_plan_sync_mode(fftconv_plan* p, int blocking) {
    if (!p || (blocking != 0 && blocking != 1)) return FC_EINVAL;
    if (blocking && !p->ev_wait)
        FC_CK(cudaEventCreateWithFlags(&p->ev_wait, cudaEventBlockingSync | cudaEventDisableTiming));
    p->blocking = blocking != 0;
    return FC_OK;
}

namespace {

// Blocks of k_zero_start for one problem (its partial sums fit the plan's
// 3 (L+1) doubles).
int zero_start_grid(const fftconv_plan* p) {
    int g = grid_1d(p->N, 256);
    if (g > 3 * (p->L + 1)) g = 3 * (p->L + 1);
    return g;
}

// The counts of a finished solve's state.
void fill_result(const CgState& f, cg_result* r) {
    r->status = f.status;
    r->iters = f.iter;
    r->refinements = f.cycles;
    r->resid_updated = f.warm_used == 1;
    r->zero_start = f.warm_used == 2;
    r->fp64_products = f.cycles - (f.warm_used != 0 ? 1 : 0);
    r->true_rel_resid = f.bb > 0 ? sqrt(f.rr64 / f.bb) : 0.0;
    r->bnorm = sqrt(f.bb);
}

// Initial state of a solve with options o.
int init_state(const cg_opts* o, CgState* h) {
    *h = CgState{};
    h->rtol2 = o->rtol * o->rtol;
    // default inner reduction per refinement cycle: the preconditioned FP32
    // solve stays accurate to a few 1e-6 (3e-6 spent one FP64 product per
    // breaking step where 1e-5 spent 1.08, at the same iteration count), plain
    // FP32 CG drifts beyond about 3e-3
    const double irt = o->inner_rtol > 0 ? o->inner_rtol : (o->precond ? 3e-6 : 3e-3);
    h->inner_rtol2 = irt * irt;
    {
        // the fraction of the outer target at which an inner run may stop
        // early (FC_INNER_GOAL, default 0.85; 0 turns it off)
        static const double goal = [] {
            const char* e = getenv("FC_INNER_GOAL");
            const double v = e ? atof(e) : 0.85;
            return v > 0.0 && v < 1.0 ? v : 0.0;
        }();
        h->inner_goal2 = goal * goal;
    }
    h->max_iter = o->max_iter > 0 ? o->max_iter : 1000000;
    h->cycle_max = o->refine_every > 0 ? o->refine_every : 100000;
    h->max_cycles = o->max_refine > 0 ? o->max_refine : 60;
    h->mixed = o->mode == FC_MODE_MIXED;
    h->sigma = 0.0;
    h->first = 1;
    return FC_OK;
}

}  // namespace

extern "C" int cg_solve(fftconv_plan* p, const double* s, const double* b, double* x, const uint8_t* mask,
                        const cg_opts* o, cg_result* r, fc_stream_t stream) {
    if (!p || !s || !b || !x) return FC_EINVAL;
    cg_opts def{};
    def.rtol = 1e-10;
    def.mode = FC_MODE_F64;
    if (!o) o = &def;
    const int mode = o->mode;
    if (mode != FC_MODE_F64 && mode != FC_MODE_MIXED) return FC_EINVAL;
    if (!(p->prec & FC_F64)) return FC_EINVAL;
    if (mode == FC_MODE_MIXED && !(p->prec & FC_F32)) return FC_EINVAL;
    if (!(o->rtol >= 0.0)) return FC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const long N = p->N;
    const bool mixed = mode == FC_MODE_MIXED;
    const auto t_call = std::chrono::steady_clock::now();
    const bool precond = o->precond != 0;
    const int gi = mode + 2 * (precond ? 1 : 0);
    // the persistent inner kernel runs plain CG; preconditioned CG uses the graph loop
    const bool persistent = !precond && (mixed ? p->p32.sel_pers : p->p64.sel_pers) >= 0;
    if (!persistent && !p->gexec[gi]) {
        int rc = build_graph(p, mode, precond);
        if (rc) return rc;
    }
    CgState h;
    init_state(o, &h);
    h.dbg_skip = p->dbg_skip;
    h.dbg_limit = p->dbg_limit;
    // inputs into the plan's buffers (the graph is built on them); after a
    // finished solve, through the check that may replace the first FP64
    // residual product by the update from the last residual (and that finds
    // whether the FP32 copy of s is still valid)
    const bool try_warm = p->warm_ok && !o->x0_zero && o->warm_resid == 0;
    // the FP32 copy of s may be kept only if the last solve made it (a mixed
    // one) and the check finds s unchanged
    h.s_check = try_warm && p->s32_ok ? 1 : 0;
    p->s32_ok = false;
    *p->st_host = h;
    FC_CK(cudaMemcpyAsync(p->st, p->st_host, sizeof(CgState), cudaMemcpyHostToDevice, st));
    p->warm_ok = false;  // the buffers change from here on
    if (try_warm) {
        k_warm_check<<<grid_1d(N, 256), 256, 0, st>>>(N, s, b, x, mask, p->s64, p->b64, p->x64, p->mask, p->st,
                                                       p->widx, p->wdx);
        FC_CK(cudaGetLastError());
        // two blocks per SM, each thread four sites per round: the FP64 block
        // reductions of many small blocks had cost as much as the update itself
        int g = grid_1d(N, 256);
        if (g > 2 * 148) g = 2 * 148;
        if (g > p->L + 1) g = p->L + 1;  // the partial-sum buffer holds 3 (L+1) doubles
        k_warm_resid<<<g, 256, 0, st>>>(N, p->L, p->gtab, p->mask, p->s64, p->b64, p->r64, p->part, p->st, p->widx,
                                        p->wdx);
        FC_CK(cudaGetLastError());
    } else {
        FC_CK(cudaMemcpyAsync(p->s64, s, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        FC_CK(cudaMemcpyAsync(p->b64, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        if (!o->x0_zero) FC_CK(cudaMemcpyAsync(p->x64, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        if (mask) {
            FC_CK(cudaMemcpyAsync(p->mask, mask, N, cudaMemcpyDeviceToDevice, st));
        } else {
            k_fill_u8<<<grid_1d(N, 256), 256, 0, st>>>(N, p->mask, 1);
            FC_CK(cudaGetLastError());
        }
        if (o->x0_zero) {
            // x = 0: the first true residual is P b, no product
            k_zero_start<<<zero_start_grid(p), 256, 0, st>>>(N, p->b64, p->mask, p->x64, p->r64, p->part, 0,
                                                             p->st);
            FC_CK(cudaGetLastError());
        }
    }
    if (persistent) {
        // Host-driven refinement loop: per cycle the FP64 true residual
        // (3 passes, device-side decision) and one cooperative launch that
        // runs the whole inner CG run; one status read per cycle.
        FC_CK(cudaMemsetAsync(p->pctl, 0, sizeof(PersistCtl), st));
        if (mixed) {
            k_f64_to_f32<<<grid_1d(N, 256), 256, 0, st>>>(N, p->s64, p->s32, p->st);
            FC_CK(cudaGetLastError());
        }
        for (int cyc = 0; cyc <= h.max_cycles + 1; ++cyc) {
            int rc = launch_resid_chain(p, mixed, st);
            if (!rc) rc = launch_persistent(p, mixed, st);
            if (rc) return rc;
            FC_CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(CgState), cudaMemcpyDeviceToHost, st));
            FC_CK(wait_stream(p, st));
            if (p->st_host->finished) break;
        }
    } else {
        FC_CK(cudaGraphLaunch(p->gexec[gi], st));
    }
    FC_CK(cudaMemcpyAsync(x, p->x64, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    FC_CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    FC_CK(wait_stream(p, st));
    const CgState& f = *p->st_host;
    // r64 is the true residual of the final x64 whenever the refinement
    // decision finished the solve
    p->warm_ok = f.finished && (f.status == FC_OK || f.status == FC_ENOCONV);
    p->s32_ok = mixed;  // every mixed solve converts s (or keeps a valid copy)
    if (r) {
        fill_result(f, r);
        r->latency_s = r->run_s =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_call).count();
    }
    return f.status;
}

// ------------------------------------------------------ batched solves --
//
// cg_solve_batch: nb independent systems of the plan's size in one graph
// launch.  Every pass runs over all problems at once (blockIdx.y = problem),
// so small systems fill the GPU that one of them alone leaves idle.  Each
// problem keeps its own state and decisions; a problem that converged skips
// the remaining passes, and the loops run until the last problem is done.
// The arithmetic of each problem is that of cg_solve with the same launch
// shapes (the thread-load pass C in place of the TMA-staged one).

struct BatchWs {
    int cap = 0;          // problems the buffers hold
    bool has64 = false;   // FP64 inner vectors (FP64-mode batches) allocated
    bool has32 = false;   // FP32 inner vectors (mixed batches) allocated
    SolveView v;
    CgState* st_host = nullptr;  // pinned, st_cap states
    int st_cap = 0;
    // instantiated solve graphs by (mode index, problems launched), least
    // recently used evicted
    struct Graph {
        int gi = -1, nb = 0;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        unsigned long long used = 0;
    };
    static constexpr int kGraphs = 16;
    Graph graphs[kGraphs];
    unsigned long long tick = 0;
    cudaStream_t stream = nullptr;  // own stream: groups of cg_solve_groups run concurrently
    cudaEvent_t ev = nullptr;
    size_t bytes = 0;
    std::vector<GuardedAlloc> blocks;  // each between two guard bands
    // batched breaking steps: per-problem argmax winners and counters
    double* am_v = nullptr;
    long long* am_i = nullptr;
    ArgmaxCtl* am_ctl = nullptr;
    long long* rm_idx = nullptr;  // per problem: the site removed last and its x before removal
    double* rm_x = nullptr;
    int am_cap = 0;
    unsigned long long gen = 0;  // unique per allocation of the buffers (keys of combined graphs)
};

namespace {

void batch_graphs_free(BatchWs* w) {
    for (auto& g : w->graphs) {
        if (g.ex) cudaGraphExecDestroy(g.ex);
        if (g.g) cudaGraphDestroy(g.g);
        g = BatchWs::Graph{};
    }
}

// Buffers back to the stream-ordered pool on st (every earlier batch on this
// workspace has finished: the calls wait for their batches).
void batch_buffers_free(BatchWs* w, cudaStream_t st) {
    batch_graphs_free(w);
    for (const GuardedAlloc& a : w->blocks) dev_free_async(a.base, st);
    w->blocks.clear();
    w->v = SolveView{};
    w->cap = 0;
    w->has64 = w->has32 = false;
    w->bytes = 0;
    w->am_v = nullptr;
    w->am_i = nullptr;
    w->am_ctl = nullptr;
    w->rm_idx = nullptr;
    w->rm_x = nullptr;
    w->am_cap = 0;
}

size_t batch_bytes_of(const fftconv_plan* p) { return p->batch ? p->batch->bytes : 0; }

void batch_free(fftconv_plan* p) {
    BatchWs* w = p->batch;
    if (!w) return;
    batch_buffers_free(w, w->stream);
    cudaStreamSynchronize(w->stream);
    host_free(w->st_host);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->stream) cudaStreamDestroy(w->stream);
    delete w;
    p->batch = nullptr;
}

template <typename P>
int balloc(BatchWs* w, P** ptr, size_t bytes, cudaStream_t st) {
    void* q = nullptr;
    cudaError_t e = dev_malloc_async(&q, bytes + 2 * kGuard, st);
    if (e != cudaSuccess) {
        set_cuda_err(e, "cudaMallocAsync(batch)");
        return FC_ENOMEM;
    }
    w->blocks.push_back(GuardedAlloc{q, bytes});
    w->bytes += bytes;
    *ptr = (P*)((unsigned char*)q + kGuard);
    return fill_guards(w->blocks.back(), st);
}

// Problems a padded batch of nb launches: the next of 1, 2, 3, 4, 6, 8, 12,
// 16, 24, 32, 48, 64, ... (at most 1.5 nb), so that the server's batches of
// varying size reuse a few instantiated graphs.
int batch_bucket(int nb) {
    int b = 1;
    while (b < nb) b = (b & (b - 1)) ? (b / 3) * 4 : (b >= 2 ? b + b / 2 : b + 1);
    return b;
}

// Buffers for nb problems in the given mode on stream st (grown, never
// shrunk; stream-ordered, so growing stalls no other stream; the graphs are
// rebuilt after a re-allocation).
int batch_reserve(fftconv_plan* p, int nb, bool mixed, cudaStream_t st) {
    if (mixed && p->p32.on && !p->p32.tuned_b) {
        const int rc = autotune_batched<float>(p, p->p32);
        if (rc) return rc;
    }
    if (!p->batch) {
        p->batch = new (std::nothrow) BatchWs();
        if (!p->batch) return FC_ENOMEM;
        FC_CK(cudaStreamCreateWithFlags(&p->batch->stream, cudaStreamNonBlocking));
        FC_CK(cudaEventCreateWithFlags(&p->batch->ev, cudaEventDisableTiming));
    }
    BatchWs* w = p->batch;
    if (w->st_cap < nb) {
        const int n = nb > 64 ? nb : 64;
        host_free(w->st_host);
        w->st_host = nullptr;
        w->st_cap = 0;
        if (host_malloc((void**)&w->st_host, sizeof(CgState) * n) != cudaSuccess) {
            set_cuda_err(cudaErrorMemoryAllocation, "cudaMallocHost(batch states)");
            return FC_ENOMEM;
        }
        w->st_cap = n;
    }
    const bool need64 = !mixed, need32 = mixed;
    if (w->cap >= nb && (!need64 || w->has64) && (!need32 || w->has32)) return FC_OK;
    const int cap = nb > w->cap ? nb : w->cap;
    const bool h64 = w->has64 || need64, h32 = w->has32 || need32;
    batch_buffers_free(w, st);
    const long N = p->N, Q = p->M / 2 + 1, QQ = Q * Q;
    const long zs = (long)(p->M / 2) * p->L;
    const long ps = 3 * (long)(p->L + 1);
    const size_t n = (size_t)cap;
    SolveView& v = w->v;
    v.nb = cap;
    v.batched = true;
    v.bs = BatchStride{N, zs, QQ, ps};
    int rc = FC_OK;
    auto A = [&](auto** ptr, size_t bytes) {
        if (!rc) rc = balloc(w, ptr, bytes, st);
    };
    A(&v.x64, 8 * n * N);
    A(&v.r64, 8 * n * N);
    A(&v.b64, 8 * n * N);
    A(&v.s64, 8 * n * N);
    A(&v.mask, n * N);
    A(&v.Z64, 16 * n * zs);
    A(&v.st, sizeof(CgState) * n);
    A(&v.part, 8 * n * ps);
    if (h64) {
        A(&v.p64v, 8 * n * N);
        A(&v.q64, 8 * n * N);
        A(&v.z64, 8 * n * N);
        A(&v.pq64, 8 * n * QQ);
    }
    if (h32) {
        A(&v.d32, 4 * n * N);
        A(&v.r32, 4 * n * N);
        A(&v.p32v, 4 * n * N);
        A(&v.q32, 4 * n * N);
        A(&v.s32, 4 * n * N);
        A(&v.z32, 4 * n * N);
        A(&v.pq32, 4 * n * QQ);
        A(&v.Z32, 8 * n * zs);
    }
    if (!rc && cudaMemsetAsync(v.st, 0, sizeof(CgState) * n, st) != cudaSuccess)
        rc = set_cuda_err(cudaGetLastError(), "cudaMemsetAsync(batch states)");
    if (rc) {
        batch_buffers_free(w, st);
        return rc;
    }
    static std::atomic<unsigned long long> next_gen{1};
    w->cap = cap;
    w->has64 = h64;
    w->has32 = h32;
    w->gen = next_gen++;
    return FC_OK;
}

// The instantiated solve graph for (mode index gi, nbg problems), built on
// first use.
int batch_graph(fftconv_plan* p, int gi, int nbg, cudaGraphExec_t* ex) {
    BatchWs* w = p->batch;
    BatchWs::Graph* slot = nullptr;
    for (auto& g : w->graphs)
        if (g.ex && g.gi == gi && g.nb == nbg) slot = &g;
    if (!slot) {
        for (auto& g : w->graphs)
            if (!slot || !g.ex || (slot->ex && g.used < slot->used)) slot = &g;
        if (slot->ex) cudaGraphExecDestroy(slot->ex);
        if (slot->g) cudaGraphDestroy(slot->g);
        *slot = BatchWs::Graph{};
        SolveView V = w->v;
        V.nb = nbg;
        int rc = build_graph_view(p, V, gi & 1, (gi & 2) != 0, &slot->g, &slot->ex);
        if (rc) return rc;
        slot->gi = gi;
        slot->nb = nbg;
    }
    slot->used = ++w->tick;
    *ex = slot->ex;
    return FC_OK;
}

int batch_stage_in(fftconv_plan* p, int nb, int nbg, const double* s, const double* b, const double* x,
                   const uint8_t* mask, const cg_opts* o, cudaStream_t st, const double* rtols);
int batch_stage_out(fftconv_plan* p, int nb, double* x, cudaStream_t st);

// Queue one batch on stream st: inputs in, the solve graph, x and the
// states out.  The caller waits on st and then reads the states.  pad: the
// graph runs a bucket of problems (batch_bucket), the ones past nb finished
// from the start (their blocks return at entry).
int batch_enqueue(fftconv_plan* p, int nb, const double* s, const double* b, double* x, const uint8_t* mask,
                  const cg_opts* o, cudaStream_t st, const double* rtols = nullptr, bool pad = false) {
    const int mode = o->mode;
    const bool mixed = mode == FC_MODE_MIXED, precond = o->precond != 0;
    const int nbg = pad ? batch_bucket(nb) : nb;
    int rc = batch_reserve(p, nbg, mixed, st);
    if (rc) return rc;
    cudaGraphExec_t ex = nullptr;
    rc = batch_graph(p, mode + 2 * (precond ? 1 : 0), nbg, &ex);
    if (rc) return rc;
    rc = batch_stage_in(p, nb, nbg, s, b, x, mask, o, st, rtols);
    if (rc) return rc;
    FC_CK(cudaGraphLaunch(ex, st));
    return batch_stage_out(p, nb, x, st);
}

// A batch's inputs into the workspace on st: states (the problems past nb
// finished from the start), s, b, the mask, and x or the zero start.
int batch_stage_in(fftconv_plan* p, int nb, int nbg, const double* s, const double* b, const double* x,
                   const uint8_t* mask, const cg_opts* o, cudaStream_t st, const double* rtols) {
    BatchWs* w = p->batch;
    const SolveView& v = w->v;
    const long N = p->N;
    const size_t nN = (size_t)nb * N;
    CgState h;
    init_state(o, &h);
    for (int k = 0; k < nbg; ++k) {
        w->st_host[k] = h;
        if (rtols && k < nb) w->st_host[k].rtol2 = rtols[k] * rtols[k];
        if (k >= nb) {  // padding: nothing to do
            w->st_host[k].finished = 1;
            w->st_host[k].idle = 1;
            w->st_host[k].status = FC_OK;
        }
    }
    FC_CK(cudaMemcpyAsync(v.st, w->st_host, sizeof(CgState) * nbg, cudaMemcpyHostToDevice, st));
    FC_CK(cudaMemcpyAsync(v.s64, s, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    FC_CK(cudaMemcpyAsync(v.b64, b, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    if (mask) {
        FC_CK(cudaMemcpyAsync(v.mask, mask, nN, cudaMemcpyDeviceToDevice, st));
    } else {
        k_fill_u8<<<grid_1d((long)nN, 256), 256, 0, st>>>((long)nN, v.mask, 1);
        FC_CK(cudaGetLastError());
    }
    if (o->x0_zero) {
        k_zero_start<<<dim3(zero_start_grid(p), nb), 256, 0, st>>>(N, v.b64, v.mask, v.x64, v.r64, v.part,
                                                                   v.bs.part, v.st);
        FC_CK(cudaGetLastError());
    } else {
        FC_CK(cudaMemcpyAsync(v.x64, x, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    }
    return FC_OK;
}

// A finished batch's solutions and states out of the workspace on st.
int batch_stage_out(fftconv_plan* p, int nb, double* x, cudaStream_t st) {
    BatchWs* w = p->batch;
    FC_CK(cudaMemcpyAsync(x, w->v.x64, sizeof(double) * (size_t)nb * p->N, cudaMemcpyDeviceToDevice, st));
    FC_CK(cudaMemcpyAsync(w->st_host, w->v.st, sizeof(CgState) * nb, cudaMemcpyDeviceToHost, st));
    return FC_OK;
}

int batch_check(const fftconv_plan* p, int nb, const double* s, const double* b, double* x, const cg_opts* o) {
    if (!p || nb < 1 || nb > 65535 || !s || !b || !x || !o) return FC_EINVAL;
    if (o->mode != FC_MODE_F64 && o->mode != FC_MODE_MIXED) return FC_EINVAL;
    if (!(p->prec & FC_F64)) return FC_EINVAL;
    if (o->mode == FC_MODE_MIXED && !(p->prec & FC_F32)) return FC_EINVAL;
    if (!(o->rtol >= 0.0)) return FC_EINVAL;
    return FC_OK;
}

// Results of a finished batch; returns the first status that is not FC_OK.
int batch_results(fftconv_plan* p, int nb, cg_result* r, double seconds) {
    int status = FC_OK;
    for (int k = 0; k < nb; ++k) {
        const CgState& f = p->batch->st_host[k];
        if (status == FC_OK && f.status != FC_OK) status = f.status;
        if (r) {
            fill_result(f, r + k);
            r[k].latency_s = r[k].run_s = seconds;
        }
    }
    return status;
}

}  // namespace

extern "C" int cg_solve_batch(fftconv_plan* p, int nb, const double* s, const double* b, double* x,
                              const uint8_t* mask, const cg_opts* o, cg_result* r, fc_stream_t stream) {
    cg_opts def{};
    def.rtol = 1e-10;
    def.mode = FC_MODE_F64;
    if (!o) o = &def;
    int rc = batch_check(p, nb, s, b, x, o);
    if (rc) return rc;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    rc = batch_enqueue(p, nb, s, b, x, mask, o, st);
    if (rc) return rc;
    FC_CK(wait_stream(p, st));
    return batch_results(p, nb, r,
                         std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
}

// The solve server's entry (fc_server.cu): cg_solve_batch with a tolerance
// per problem (host array of nb values).
int fc_batch_solve_rtols(fftconv_plan* p, int nb, const double* s, const double* b, double* x, const cg_opts* o,
                         const double* rtols, cg_result* r, cudaStream_t st) {
    int rc = batch_check(p, nb, s, b, x, o);
    if (rc) return rc;
    for (int k = 0; k < nb; ++k)
        if (!(rtols[k] >= 0.0)) return FC_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    rc = batch_enqueue(p, nb, s, b, x, nullptr, o, st, rtols, true);
    if (rc) return rc;
    FC_CK(wait_stream(p, st));
    return batch_results(p, nb, r,
                         std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
}

namespace {

// One graph holding every group's batched solve as a parallel branch (one
// launch for all sizes), cached by the groups' workspace generations (unique
// per allocation, so a graph never outlives the buffers it names in use),
// batch sizes and mode; least recently used of four evicted.
struct GroupsGraph {
    std::vector<unsigned long long> gens;
    std::vector<int> nbs;
    int gi = -1;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    unsigned long long used = 0;
};
std::mutex g_groups_mu;
GroupsGraph g_groups[4];
unsigned long long g_groups_tick = 0;

// The combined graph for these groups (call with g_groups_mu held).
int groups_graph(int ngroups, const cg_batch_group* g, int mode, bool precond, cudaGraphExec_t* ex) {
    const int gi = mode + 2 * (precond ? 1 : 0);
    std::vector<unsigned long long> gens;
    std::vector<int> nbs;
    for (int i = 0; i < ngroups; ++i) {
        gens.push_back(g[i].plan->batch->gen);
        nbs.push_back(g[i].nb);
    }
    GroupsGraph* slot = nullptr;
    for (auto& c : g_groups)
        if (c.ex && c.gi == gi && c.gens == gens && c.nbs == nbs) slot = &c;
    if (!slot) {
        for (auto& c : g_groups)
            if (!slot || !c.ex || (slot->ex && c.used < slot->used)) slot = &c;
        if (slot->ex) cudaGraphExecDestroy(slot->ex);
        if (slot->g) cudaGraphDestroy(slot->g);
        *slot = GroupsGraph{};
        int rc = FC_ECUDA;
        for (int pdl = pdl_on() ? 1 : 0; pdl >= 0 && rc != FC_OK; --pdl) {
            cudaGraph_t gr = nullptr;
            FC_CK(cudaGraphCreate(&gr, 0));
            rc = FC_OK;
            for (int i = 0; i < ngroups && rc == FC_OK; ++i) {
                SolveView V = g[i].plan->batch->v;
                V.nb = g[i].nb;
                rc = add_solve_nodes(g[i].plan, V, mode, precond, pdl != 0, gr);
            }
            cudaGraphExec_t e = nullptr;
            if (rc == FC_OK && cudaGraphInstantiate(&e, gr, 0) != cudaSuccess)
                rc = set_cuda_err(cudaGetLastError(), "cudaGraphInstantiate(groups)");
            if (rc == FC_OK) {
                slot->g = gr;
                slot->ex = e;
            } else {
                cudaGraphDestroy(gr);
            }
        }
        if (rc) return rc;
        slot->gens = gens;
        slot->nbs = nbs;
        slot->gi = gi;
    }
    slot->used = ++g_groups_tick;
    *ex = slot->ex;
    return FC_OK;
}

}  // namespace

extern "C" int cg_solve_groups(int ngroups, const cg_batch_group* g, const cg_opts* o, fc_stream_t stream) {
    if (ngroups < 1 || !g) return FC_EINVAL;
    cg_opts def{};
    def.rtol = 1e-10;
    def.mode = FC_MODE_F64;
    if (!o) o = &def;
    for (int i = 0; i < ngroups; ++i) {
        int rc = batch_check(g[i].plan, g[i].nb, g[i].s, g[i].b, g[i].x, o);
        if (rc) return rc;
        for (int j = 0; j < i; ++j)
            if (g[j].plan == g[i].plan) return FC_EINVAL;  // one workspace per plan
    }
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    // fork: every group on its plan's own stream after the caller's work
    for (int i = 0; i < ngroups; ++i) {
        int rc = batch_reserve(g[i].plan, g[i].nb, o->mode == FC_MODE_MIXED, st);
        if (rc) return rc;
    }
    {
        // one graph for all groups: inputs in, one launch, outputs out, all on st
        std::unique_lock<std::mutex> lk(g_groups_mu);
        cudaGraphExec_t ex = nullptr;
        if (groups_graph(ngroups, g, o->mode, o->precond != 0, &ex) == FC_OK) {
            int rc = FC_OK;
            for (int i = 0; i < ngroups && rc == FC_OK; ++i)
                rc = batch_stage_in(g[i].plan, g[i].nb, g[i].nb, g[i].s, g[i].b, g[i].x, g[i].mask, o, st, nullptr);
            if (rc == FC_OK && cudaGraphLaunch(ex, st) != cudaSuccess)
                rc = set_cuda_err(cudaGetLastError(), "cudaGraphLaunch(groups)");
            lk.unlock();
            for (int i = 0; i < ngroups && rc == FC_OK; ++i) rc = batch_stage_out(g[i].plan, g[i].nb, g[i].x, st);
            FC_CK(wait_stream(g[0].plan, st));
            if (rc) return rc;
            const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            int status = FC_OK;
            for (int i = 0; i < ngroups; ++i) {
                const int si = batch_results(g[i].plan, g[i].nb, g[i].r, secs);
                if (status == FC_OK) status = si;
            }
            return status;
        }
    }
    // no combined graph could be made: each group's graph on its plan's
    // stream, forked from and joined to st
    cudaEvent_t fork = g[0].plan->batch->ev;
    FC_CK(cudaEventRecord(fork, st));
    for (int i = 0; i < ngroups; ++i) {
        BatchWs* w = g[i].plan->batch;
        FC_CK(cudaStreamWaitEvent(w->stream, fork, 0));
    }
    int rc = FC_OK;
    for (int i = 0; i < ngroups && rc == FC_OK; ++i) {
        BatchWs* w = g[i].plan->batch;
        rc = batch_enqueue(g[i].plan, g[i].nb, g[i].s, g[i].b, g[i].x, g[i].mask, o, w->stream);
    }
    // join (also after a failed enqueue: no group's work outlives the call)
    for (int i = 0; i < ngroups; ++i) {
        BatchWs* w = g[i].plan->batch;
        if (cudaEventRecord(w->ev, w->stream) != cudaSuccess || cudaStreamWaitEvent(st, w->ev, 0) != cudaSuccess)
            cudaStreamSynchronize(w->stream);
    }
    FC_CK(wait_stream(g[0].plan, st));
    if (rc) return rc;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int status = FC_OK;
    for (int i = 0; i < ngroups; ++i) {
        const int si = batch_results(g[i].plan, g[i].nb, g[i].r, secs);
        if (status == FC_OK) status = si;
    }
    return status;
}

// fc_fracture_run_batch: nb independent breaking runs of the plan's size in
// lockstep.  The fields stay in the batch workspace for the whole run; each
// step is one batched solve (warm-started from the last solution, first
// residual by product) and one batched removal.
extern "C" int fc_fracture_run_batch(fftconv_plan* p, int nb, const double* s, const double* b, const double* t,
                                     uint8_t* mask, double* x, int steps, const cg_opts* o, int64_t* removed,
                                     double* ratio, fc_run_result* res, fc_stream_t stream) {
    if (!t || !mask || !removed || steps < 0) return FC_EINVAL;
    cg_opts def{};
    def.rtol = 1e-10;
    def.mode = FC_MODE_F64;
    if (!o) o = &def;
    int rc = batch_check(p, nb, s, b, x, o);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const bool mixed = o->mode == FC_MODE_MIXED, precond = o->precond != 0;
    rc = batch_reserve(p, nb, mixed, st);
    if (rc) return rc;
    BatchWs* w = p->batch;
    if (w->am_cap < nb) {
        rc = balloc(w, &w->am_v, sizeof(double) * (size_t)nb * p->am_grid, st);
        if (!rc) rc = balloc(w, &w->am_i, sizeof(long long) * (size_t)nb * p->am_grid, st);
        if (!rc) rc = balloc(w, &w->am_ctl, sizeof(ArgmaxCtl) * (size_t)nb, st);
        if (!rc) rc = balloc(w, &w->rm_idx, sizeof(long long) * (size_t)nb, st);
        if (!rc) rc = balloc(w, &w->rm_x, sizeof(double) * (size_t)nb, st);
        if (rc) return rc;
        FC_CK(cudaMemsetAsync(w->am_ctl, 0, sizeof(ArgmaxCtl) * (size_t)nb, st));
        w->am_cap = nb;
    }
    cudaGraphExec_t ex = nullptr;
    rc = batch_graph(p, o->mode + 2 * (precond ? 1 : 0), nb, &ex);
    if (rc) return rc;
    const SolveView& v = w->v;
    const long N = p->N;
    const size_t nN = (size_t)nb * N;
    FC_CK(cudaMemcpyAsync(v.s64, s, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    FC_CK(cudaMemcpyAsync(v.b64, b, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    FC_CK(cudaMemcpyAsync(v.x64, x, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st));
    FC_CK(cudaMemcpyAsync(v.mask, mask, nN, cudaMemcpyDeviceToDevice, st));
    std::vector<fc_run_result> acc((size_t)nb);
    std::vector<int> alive((size_t)nb, 1);
    for (auto& a : acc) a.status = FC_OK;
    CgState h;
    init_state(o, &h);
    // after the first step each solve's first residual is updated from the
    // last one (the removal is the only change), unless turned off
    const bool warm = o->warm_resid == 0 && p->gtab != nullptr;
    int64_t* rm_host = nullptr;
    if (host_malloc((void**)&rm_host, sizeof(int64_t) * (size_t)nb) != cudaSuccess) {
        set_cuda_err(cudaErrorMemoryAllocation, "cudaMallocHost(removed indices)");
        return FC_ENOMEM;
    }
    int step = 0;
    for (; step < steps && rc == FC_OK; ++step) {
        for (int k = 0; k < nb; ++k) {
            w->st_host[k] = h;
            if (!alive[k]) {  // nothing left to solve: the problem sits out (and removes nothing)
                w->st_host[k].finished = 1;
                w->st_host[k].idle = 1;
                w->st_host[k].status = FC_ENOCONV;
            }
        }
        if (cudaMemcpyAsync(v.st, w->st_host, sizeof(CgState) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = set_cuda_err(cudaGetLastError(), "fc_fracture_run_batch(states)");
            break;
        }
        if (step > 0 && warm) {
            // the first residual of this solve from the last one and the removal
            int gw = grid_1d(N, 256);
            if (gw > p->L + 1) gw = p->L + 1;  // two partial sums per block in 3 (L+1) doubles per problem
            k_warm_resid_batch<<<dim3(gw, nb), 256, 0, st>>>(N, p->L, p->gtab, v.mask, v.b64, v.r64, v.part,
                                                             v.bs.part, v.st, w->rm_idx, w->rm_x);
            if (cudaGetLastError() != cudaSuccess) {
                rc = set_cuda_err(cudaGetLastError(), "k_warm_resid_batch");
                break;
            }
        }
        if (cudaGraphLaunch(ex, st) != cudaSuccess ||
            cudaMemcpyAsync(w->st_host, v.st, sizeof(CgState) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            rc = set_cuda_err(cudaGetLastError(), "fc_fracture_run_batch(solve)");
            break;
        }
        k_masked_argmax<<<dim3(p->am_grid, nb), 256, 0, st>>>(N, t, v.mask, v.x64, removed + step,
                                                              ratio ? ratio + step : nullptr, w->am_v, w->am_i,
                                                              w->am_ctl, steps, v.st, w->rm_idx, w->rm_x);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy2DAsync(rm_host, sizeof(int64_t), removed + step, sizeof(int64_t) * steps, sizeof(int64_t), nb,
                              cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            wait_stream(p, st) != cudaSuccess) {
            rc = set_cuda_err(cudaGetLastError(), "fc_fracture_run_batch(step)");
            break;
        }
        int any = 0;
        for (int k = 0; k < nb; ++k) {
            if (!alive[k]) continue;
            const CgState& f = w->st_host[k];
            cg_result r{};
            fill_result(f, &r);
            acc[k].iters += r.iters;
            acc[k].fp64_products += r.fp64_products;
            acc[k].resid_updated += r.resid_updated;
            if (f.status != FC_OK) {
                acc[k].status = f.status;
                alive[k] = 0;
            } else if (rm_host[k] < 0) {
                alive[k] = 0;  // no active fibre left
            } else {
                acc[k].steps_done = step + 1;
            }
            any |= alive[k];
        }
        if (!any) {
            ++step;
            break;
        }
    }
    // steps not run: nothing removed (index -1, ratio -1)
    if (rc == FC_OK && step < steps) {
        const std::vector<int64_t> none((size_t)(steps - step), -1);
        const std::vector<double> noratio((size_t)(steps - step), -1.0);
        for (int k = 0; k < nb && rc == FC_OK; ++k) {
            if (cudaMemcpyAsync(removed + (size_t)k * steps + step, none.data(), sizeof(int64_t) * (steps - step),
                                cudaMemcpyHostToDevice, st) != cudaSuccess ||
                (ratio && cudaMemcpyAsync(ratio + (size_t)k * steps + step, noratio.data(),
                                          sizeof(double) * (steps - step), cudaMemcpyHostToDevice, st) != cudaSuccess))
                rc = set_cuda_err(cudaGetLastError(), "fc_fracture_run_batch(tail)");
        }
        if (rc == FC_OK && cudaStreamSynchronize(st) != cudaSuccess)
            rc = set_cuda_err(cudaGetLastError(), "fc_fracture_run_batch(tail)");
    }
    if (rc == FC_OK) {
        if (cudaMemcpyAsync(x, v.x64, sizeof(double) * nN, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(mask, v.mask, nN, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            wait_stream(p, st) != cudaSuccess)
            rc = set_cuda_err(cudaGetLastError(), "fc_fracture_run_batch(results)");
    }
    host_free(rm_host);
    if (rc) return rc;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int status = FC_OK;
    for (int k = 0; k < nb; ++k) {
        acc[k].seconds = secs;
        if (res) res[k] = acc[k];
        if (status == FC_OK && acc[k].status != FC_OK) status = acc[k].status;
    }
    return status;
}

extern "C" int fc_masked_step(fftconv_plan* p, const double* t, uint8_t* mask, double* x, int64_t* removed,
                              fc_stream_t stream) {
    if (!p || !t || !mask || !x || !removed) return FC_EINVAL;
    k_masked_argmax<<<p->am_grid, 256, 0, (cudaStream_t)stream>>>(p->N, t, mask, x, removed, nullptr, p->am_v,
                                                                   p->am_i, p->am_ctl);
    FC_CK(cudaGetLastError());
    return FC_OK;
}

extern "C" int fc_front(fftconv_plan* p, const uint8_t* mask, int32_t* first_intact, int32_t* damage_end,
                        fc_stream_t stream) {
    if (!p || !mask || !first_intact || !damage_end) return FC_EINVAL;
    k_front<<<(p->L + 31) / 32, 512, 0, (cudaStream_t)stream>>>(p->L, mask, first_intact, damage_end);
    FC_CK(cudaGetLastError());
    return FC_OK;
}

extern "C" int fc_fracture_run(fftconv_plan* p, const double* s, const double* b, const double* t, uint8_t* mask,
                               double* x, int steps, const cg_opts* o, int64_t* removed, double* ratio,
                               fc_run_result* res, fc_stream_t stream) {
    if (!p || !s || !b || !t || !mask || !x || !removed || steps < 0) return FC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    fc_run_result acc{};
    acc.status = FC_OK;
    for (int k = 0; k < steps; ++k) {
        cg_result r{};
        const int rc = cg_solve(p, s, b, x, mask, o, &r, stream);  // returns with the stream drained
        if (rc == FC_EINVAL || rc == FC_ECUDA || rc == FC_ENOMEM) return rc;
        acc.iters += r.iters;
        acc.fp64_products += r.fp64_products;
        acc.resid_updated += r.resid_updated;
        if (rc != FC_OK) {
            acc.status = rc;
            break;
        }
        k_masked_argmax<<<p->am_grid, 256, 0, st>>>(p->N, t, mask, x, removed + k, ratio ? ratio + k : nullptr,
                                                    p->am_v, p->am_i, p->am_ctl);
        FC_CK(cudaGetLastError());
        FC_CK(cudaMemcpyAsync(p->rm_host, removed + k, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        FC_CK(wait_stream(p, st));
        if (*p->rm_host < 0) break;  // no active fibre left
        acc.steps_done = k + 1;
    }
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = acc;
    return acc.status;
}

// ------------------------------------------- allocation-free masked step --
//
// fc_masked_step_static: the breaking step for callers that cannot allocate
// device memory at the point of the call.  Its scratch (per-block winners of
// the argmax and the last-block counter) lives in the file-scope array below
// instead of a plan; every GPU that loads the library holds these 131,328
// bytes until the process exits.

namespace {
constexpr int kStaticMaxBlocks = 8192;  // one block per 2048 sites
constexpr long long kStaticMaxN = (long long)kStaticMaxBlocks * 2048;  // 16,777,216 = 4096^2
constexpr size_t kStaticCtlBytes = 256;
constexpr size_t kStaticScratchBytes =
    kStaticCtlBytes + (size_t)kStaticMaxBlocks * (sizeof(double) + sizeof(long long));
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

extern "C" int fc_masked_step_static(int64_t N, const double* t, uint8_t* mask, double* x, int64_t* removed,
                                     fc_stream_t stream) {
    if (N < 1 || N > kStaticMaxN) {
        snprintf(g_err, sizeof(g_err),
                 "fc_masked_step_static: N = %lld is outside [1, %lld], the largest size its static scratch "
                 "(%d block results) can hold",
                 (long long)N, kStaticMaxN, kStaticMaxBlocks);
        return FC_EINVAL;
    }
    if (!t || !mask || !x || !removed) return FC_EINVAL;
    int dev = 0;
    FC_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return FC_EINVAL;
    void* base = nullptr;
    {
        // set-up once per device, with that device current: the array's device
        // address (in host code its name is only a stand-in)
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess) return set_cuda_err(e, "cudaGetSymbolAddress(g_static_scratch)");
            g_static_ptr[dev] = ptr;
        }
        base = g_static_ptr[dev];
    }
    ArgmaxCtl* ctl = reinterpret_cast<ArgmaxCtl*>(base);
    double* pv = reinterpret_cast<double*>(static_cast<char*>(base) + kStaticCtlBytes);
    long long* pi = reinterpret_cast<long long*>(static_cast<char*>(base) + kStaticCtlBytes +
                                                 (size_t)kStaticMaxBlocks * sizeof(double));
    const int grid = (int)((N + 2047) / 2048);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the counter must start at 0
    FC_CK(cudaMemsetAsync(ctl, 0, sizeof(ArgmaxCtl), s));
    k_masked_argmax<<<grid, 256, 0, s>>>((long)N, t, mask, x, removed, nullptr, pv, pi, ctl);
    FC_CK(cudaGetLastError());
    return FC_OK;
}

// ------------------------------------------------ memory and test hooks --

extern "C" int fc_mem_stats(size_t* live_bytes, size_t* peak_bytes, long long* live_allocs, int reset_peak) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (live_bytes) *live_bytes = g_live_dev_bytes;
    if (peak_bytes) *peak_bytes = g_peak_dev_bytes;
    if (live_allocs) *live_allocs = (long long)g_live.size();
    if (reset_peak) g_peak_dev_bytes = g_live_dev_bytes;
    return FC_OK;
}

extern "C" int fc_debug_inject(fftconv_plan* p, int kind, long long value) {
    if (value < 0) return FC_EINVAL;
    switch (kind) {
        case FC_INJECT_ALLOC:
            g_fail_countdown.store(value);
            return FC_OK;
        case FC_INJECT_BARRIER:
        case FC_INJECT_TMA:
            if (!p || value > 0xffffffffLL) return FC_EINVAL;
            p->dbg_skip = value ? (kind == FC_INJECT_BARRIER ? 1u : 2u) : 0u;
            p->dbg_limit = (unsigned)value;
            {
                // the plan's state now as well (applies read it; solves copy it in)
                const unsigned v[2] = {p->dbg_skip, p->dbg_limit};
                static_assert(offsetof(CgState, dbg_limit) == offsetof(CgState, dbg_skip) + sizeof(unsigned),
                              "adjacent hook fields");
                FC_CK(cudaMemcpy((char*)p->st + offsetof(CgState, dbg_skip), v, sizeof(v), cudaMemcpyHostToDevice));
            }
            return FC_OK;
        default:
            return FC_EINVAL;
    }
}

namespace {

// Guard bands of a plan's buffers: block b checks band b (kGuard bytes, one
// per thread) and counts it once if any byte differs from kGuardByte.
__global__ void __launch_bounds__(256) k_check_guards(const unsigned char* const* bands, unsigned* damaged) {
    const unsigned char* g = bands[blockIdx.x];
    const int bad = g[threadIdx.x] != kGuardByte;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicAdd(damaged, 1u);
}

}  // namespace

extern "C" int fftconv_plan_check_guards(fftconv_plan* p, int* damaged) {
    if (!p || !damaged) return FC_EINVAL;
    *damaged = 0;
    std::vector<const unsigned char*> bands;
    auto add = [&](const GuardedAlloc& a) {
        const unsigned char* b = (const unsigned char*)a.base;
        bands.push_back(b);
        bands.push_back(b + kGuard + a.bytes);
    };
    for (const GuardedAlloc& a : p->allocs) add(a);
    if (p->batch)
        for (const GuardedAlloc& a : p->batch->blocks) add(a);
    if (bands.empty()) return FC_OK;
    static_assert(kGuard == 256, "one thread per guard byte");
    cudaStream_t s = nullptr;
    void* dev = nullptr;
    const size_t pbytes = sizeof(void*) * bands.size();
    FC_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int rc = FC_OK;
    unsigned h = 0;
    if (dev_malloc_async(&dev, pbytes + sizeof(unsigned), s) != cudaSuccess) {
        set_cuda_err(cudaErrorMemoryAllocation, "cudaMallocAsync(guard list)");
        rc = FC_ENOMEM;
    } else {
        unsigned* cnt = (unsigned*)((unsigned char*)dev + pbytes);
        if (cudaMemcpyAsync(dev, bands.data(), pbytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(cnt, 0, sizeof(unsigned), s) != cudaSuccess)
            rc = set_cuda_err(cudaGetLastError(), "guard check set-up");
        if (!rc) {
            k_check_guards<<<(unsigned)bands.size(), 256, 0, s>>>((const unsigned char* const*)dev, cnt);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&h, cnt, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
                rc = set_cuda_err(cudaGetLastError(), "guard check");
        }
        dev_free_async(dev, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = set_cuda_err(cudaGetLastError(), "guard check");
    cudaStreamDestroy(s);
    if (!rc) *damaged = (int)h;
    return rc;
}
