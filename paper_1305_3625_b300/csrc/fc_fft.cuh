// Register-resident Stockham FFT building blocks for sm_103a.
//
// One transform of length M (a power of two, 2..8192) is held by G = M/E
// threads, each owning E complex values in registers.  Thread j owns the
// elements j + e*G (e = 0..E-1) both on input and on output, so a warp of
// consecutive j touches consecutive addresses of a row in global memory.
// Each radix-E Stockham stage (twiddle, E-point DFT in registers) is followed
// by one exchange through shared memory; a trailing stage of smaller radix
// R = M / E^k runs entirely in registers (E/R butterflies per thread).
//
// Forward transform: X[k] = sum_n x[n] exp(-2 pi i nk/M); the inverse uses
// exp(+2 pi i nk/M) and is unnormalised (the 1/M^2 of the 2D round trip is
// folded into the stored kernel spectrum).  This is the Fourier
// diagonalisation of the coupling operator of Eq. 3 (Section 3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace fc {

template <typename T>
struct __align__(2 * sizeof(T)) cpx {
    T x, y;
};

// Products whose rounding the compiler may not change: every multiply-add
// of the pass kernels is written as an explicit fma of a rounded product,
// so that two kernels built from the same arithmetic (a pass and its batched
// twin, whatever their register pressure) round identically.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> w) {
    return {fma(a.x, w.x, -mul_rn(a.y, w.y)), fma(a.x, w.y, mul_rn(a.y, w.x))};
}
// a * conj(w)
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> w) {
    return {fma(a.x, w.x, mul_rn(a.y, w.y)), fma(a.y, w.x, -mul_rn(a.x, w.y))};
}

// Read-only (L1-cached) load of one complex value.
template <typename T>
__device__ __forceinline__ cpx<T> ldg_c(const cpx<T>* p) {
    if constexpr (sizeof(T) == 4) {
        float2 v = __ldg(reinterpret_cast<const float2*>(p));
        return {v.x, v.y};
    } else {
        double2 v = __ldg(reinterpret_cast<const double2*>(p));
        return {v.x, v.y};
    }
}

// cos(pi q / 16), q = 0..8 (exact mathematical constants); the angles
// 2 pi Q / 32 of the radix-32 rotations are multiples of pi / 16.
constexpr double kCosPi16[9] = {1.0,
                                0.980785280403230449126182236134239037,
                                0.923879532511286756128183189396788287,
                                0.831469612302545237078788377617905757,
                                0.707106781186547524400844362104849039,
                                0.555570233019602224742830813948532874,
                                0.382683432365089771728459984030398867,
                                0.195090322016128267848284868477022241,
                                0.0};
// cos and sin of 2 pi Q / 32 for Q in [0, 16).
__host__ __device__ constexpr double cos32(int Q) { return Q <= 8 ? kCosPi16[Q] : -kCosPi16[16 - Q]; }
__host__ __device__ constexpr double sin32(int Q) { return Q <= 8 ? kCosPi16[8 - Q] : kCosPi16[Q - 8]; }

// Multiply by exp(-/+ 2 pi i Q/32) (forward / inverse), Q in [0, 16).
template <int Q, bool INV, typename T>
__device__ __forceinline__ cpx<T> rot32(cpx<T> a) {
    if constexpr (Q == 0) {
        return a;
    } else if constexpr (Q == 8) {
        return INV ? cpx<T>{-a.y, a.x} : cpx<T>{a.y, -a.x};
    } else if constexpr (Q == 4 || Q == 12) {
        constexpr T h = (T)kCosPi16[4];
        // (1 -/+ i) h  for Q = 4, (-1 -/+ i) h for Q = 12
        if constexpr (Q == 4)
            return INV ? cpx<T>{mul_rn(a.x - a.y, h), mul_rn(a.x + a.y, h)}
                       : cpx<T>{mul_rn(a.x + a.y, h), mul_rn(a.y - a.x, h)};
        else
            return INV ? cpx<T>{-mul_rn(a.x + a.y, h), mul_rn(a.x - a.y, h)}
                       : cpx<T>{mul_rn(a.y - a.x, h), -mul_rn(a.x + a.y, h)};
    } else {
        constexpr T c = (T)cos32(Q);
        constexpr T s = INV ? (T)sin32(Q) : -(T)sin32(Q);
        return {fma(a.x, c, -mul_rn(a.y, s)), fma(a.x, s, mul_rn(a.y, c))};
    }
}

// The butterfly of a radix-2 level with a constant rotation folded in:
// lo = a + w b, hi = a - w b, w = exp(-/+ 2 pi i Q/32).  A generic rotation
// is applied as c (b.x - t b.y, b.y + t b.x) with t = s/c (or its
// cotangent form when |s| > |c|), so that the scale c enters the two sums
// as fused multiply-adds: 6 operations per butterfly instead of 8.
template <int Q, bool INV, typename T>
__device__ __forceinline__ void bfly(cpx<T> a, cpx<T> b, cpx<T>& lo, cpx<T>& hi) {
    if constexpr (Q == 0) {
        lo = a + b;
        hi = a - b;
    } else if constexpr (Q == 8) {
        const cpx<T> wb = INV ? cpx<T>{-b.y, b.x} : cpx<T>{b.y, -b.x};
        lo = a + wb;
        hi = a - wb;
    } else if constexpr (Q == 4 || Q == 12) {
        // w b = h (u, v) with w = (+/-1 +/- i) h
        constexpr T h = (T)kCosPi16[4];
        T u, v;
        if constexpr (Q == 4) {
            u = INV ? b.x - b.y : b.x + b.y;
            v = INV ? b.x + b.y : b.y - b.x;
        } else {
            u = INV ? -(b.x + b.y) : b.y - b.x;
            v = INV ? b.x - b.y : -(b.x + b.y);
        }
        lo = cpx<T>{fma(h, u, a.x), fma(h, v, a.y)};
        hi = cpx<T>{fma(-h, u, a.x), fma(-h, v, a.y)};
    } else {
        constexpr double cd = cos32(Q), sd = INV ? sin32(Q) : -sin32(Q);
        if constexpr (cd * cd >= sd * sd) {  // w b = c (b.x - t b.y, b.y + t b.x)
            constexpr T c = (T)cd, t = (T)(sd / cd);
            const T u = fma(-t, b.y, b.x), v = fma(t, b.x, b.y);
            lo = cpx<T>{fma(c, u, a.x), fma(c, v, a.y)};
            hi = cpx<T>{fma(-c, u, a.x), fma(-c, v, a.y)};
        } else {  // w b = s (k b.x - b.y, b.x + k b.y), k = c/s
            constexpr T sc = (T)sd, k = (T)(cd / sd);
            const T u = fma(k, b.x, -b.y), v = fma(k, b.y, b.x);
            lo = cpx<T>{fma(sc, u, a.x), fma(sc, v, a.y)};
            hi = cpx<T>{fma(-sc, u, a.x), fma(-sc, v, a.y)};
        }
    }
}

template <int R, bool INV, typename T, int... K>
__device__ __forceinline__ void bfly_level(const cpx<T>* e, const cpx<T>* o, cpx<T>* v,
                                           std::integer_sequence<int, K...>) {
    (bfly<K * 32 / R, INV>(e[K], o[K], v[K], v[K + R / 2]), ...);
}

template <int R, bool INV, typename T, int... K>
__device__ __forceinline__ void rotate_consts(cpx<T>* o, std::integer_sequence<int, K...>) {
    ((o[K] = rot32<K * 32 / R, INV>(o[K])), ...);
}

// In-register R-point DFT (R = 1, 2, 4, 8, 16, 32), natural order in and
// out, by recursive radix-2 decimation in time.
template <int R, bool INV, typename T>
struct Dft {
    static __device__ __forceinline__ void run(cpx<T> (&v)[R]) {
        cpx<T> e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        Dft<R / 2, INV, T>::run(e);
        Dft<R / 2, INV, T>::run(o);
        bfly_level<R, INV, T>(e, o, v, std::make_integer_sequence<int, R / 2>{});
    }
};
template <bool INV, typename T>
struct Dft<1, INV, T> {
    static __device__ __forceinline__ void run(cpx<T> (&)[1]) {}
};
template <bool INV, typename T>
struct Dft<2, INV, T> {
    static __device__ __forceinline__ void run(cpx<T> (&v)[2]) {
        cpx<T> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    }
};

// R-point DFT of a sequence whose upper half is zero (v[n] = 0 for
// n >= R/2, the zero padding): X[2m] is the R/2-point DFT of x and
// X[2m+1] that of x[n] exp(-/+ 2 pi i n/R), so no additions of zeros.
template <int R, bool INV, typename T>
struct DftZeroHalf {
    static __device__ __forceinline__ void run(cpx<T> (&v)[R]) {
        if constexpr (R == 1) {
            return;
        } else {
            cpx<T> a[R / 2], b[R / 2];
#pragma unroll
            for (int n = 0; n < R / 2; ++n) a[n] = b[n] = v[n];
            rotate_consts<R, INV, T>(b, std::make_integer_sequence<int, R / 2>{});
            Dft<R / 2, INV, T>::run(a);
            Dft<R / 2, INV, T>::run(b);
#pragma unroll
            for (int m = 0; m < R / 2; ++m) {
                v[2 * m] = a[m];
                v[2 * m + 1] = b[m];
            }
        }
    }
};

// Shared-memory index with one padding slot every 2^P elements (P = 4; 5 in
// the exchanges of radix-32 stages); it spreads the radix-E "expand" writes
// (stride E) over the banks.  For every access pattern of the stages below,
// spad(base + c) = spad(base) + c + (c >> P) with c a compile-time multiple
// of the stride (checked exhaustively for all M <= 8192, E in {2,4,8,16}
// with P = 4 and E = 32, M >= 1024 with P = 5), so addresses are a base plus
// immediates.  seg_len(M) covers both paddings.
template <int P = 4>
__host__ __device__ __forceinline__ constexpr int spad(int i) { return i + (i >> P); }
__host__ __device__ constexpr int seg_len(int M) { return M + (M >> 4) + 2; }
template <int P = 4>
__host__ __device__ constexpr int pofs(int c) { return c + (c >> P); }
__host__ __device__ constexpr int pad_shift(int E) { return E >= 32 ? 5 : 4; }

// Stage structure of a length-M transform with E values per thread: stages
// NS = 1, E, E^2, ... of radix E, the last one of radix M/NS if smaller.
__host__ __device__ constexpr int stage_radix(int M, int E, int NS) { return NS * E <= M ? E : M / NS; }
__host__ __device__ constexpr int n_exchanges(int M, int E) {
    int n = 0;
    for (int ns = 1; ns * E < M; ns *= E) ++n;
    return n;
}
// Stage twiddle table: for each stage with NS > 1 a block of R x NS entries,
// entry [e][k] = exp(-2 pi i e k / (NS R)) (R the stage radix), so that the
// threads of a warp (consecutive k) read consecutive entries; the offset of
// stage NS's block, and the whole table's length.
__host__ __device__ constexpr int tw_offset(int M, int E, int NS) {
    int off = 0;
    for (int ns = E; ns < NS && ns < M; ns *= stage_radix(M, E, ns)) off += ns * stage_radix(M, E, ns);
    return off;
}
__host__ __device__ constexpr int tw_len(int M, int E) { return tw_offset(M, E, M); }
// Slot of E's table among a plan's tables (log2 E for E = 2 .. 32).
__host__ __device__ constexpr int tw_index(int E) {
    return E == 2 ? 1 : E == 4 ? 2 : E == 8 ? 3 : E == 16 ? 4 : E == 32 ? 5 : 0;
}

// Load the R-1 twiddles e = 1..R-1 of column k of a stage block (entry
// [e][k] at blk[e*NS + k]): one coalesced load per e across the warp.
template <typename T, int R, int NS>
__device__ __forceinline__ void load_twiddles(const cpx<T>* __restrict__ blk, int k, cpx<T> (&w)[R]) {
#pragma unroll
    for (int e = 1; e < R; ++e) w[e] = ldg_c(blk + e * NS + k);
}

// Stockham transform of one length-M sequence held by G = M/E threads as
// v[e] = x[j + e*G] (thread j of its group); on return v[e] = X[j + e*G].
// sm0/sm1: this group's two shared segments (seg_len(M) elements each).
// With DB the exchanges alternate between them (starting with BUF) and need
// one barrier each; without DB only sm0 is used and each exchange ends with
// a second barrier.  tws: the stage twiddle table of (M, E).  ZH: the
// upper half of the sequence is zero (x[n] = 0 for n >= M/2, so v[e] = 0 for
// e >= E/2: the zero padding), which the first stage skips.  GB: the
// exchanges synchronise each group alone (exchange_sync).  All threads of
// the block call this together.
// The barrier of an exchange.  GB: each group of G threads (whole warps,
// consecutive in the block: group threadIdx.x / G, at most 15 groups) waits
// only for itself on its own named barrier, 1 + group; otherwise the block.
template <int G, bool GB>
__device__ __forceinline__ void exchange_sync() {
    if constexpr (GB) {
        static_assert(G % 32 == 0, "group barriers need whole warps");
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / G)), "n"(G) : "memory");
    } else {
        __syncthreads();
    }
}

template <typename T, int M, int E, bool INV, bool DB, int BUF = 0, int NS = 1, bool ZH = false, bool GB = false>
__device__ __forceinline__ void fft_stages(cpx<T> (&v)[E], int j, cpx<T>* sm0, cpx<T>* sm1,
                                           const cpx<T>* __restrict__ tws) {
    constexpr int G = M / E;
    if constexpr (NS * E <= M) {
        const int k = j & (NS - 1);
        if constexpr (NS > 1) {
            cpx<T> w[E];
            load_twiddles<T, E, NS>(tws + tw_offset(M, E, NS), k, w);
#pragma unroll
            for (int e = 1; e < E; ++e) v[e] = INV ? cmulc(v[e], w[e]) : cmul(v[e], w[e]);
        }
        if constexpr (ZH && NS == 1)
            DftZeroHalf<E, INV, T>::run(v);
        else
            Dft<E, INV, T>::run(v);
        if constexpr (NS * E < M) {
            cpx<T>* sm = (DB && BUF) ? sm1 : sm0;
            constexpr int P = pad_shift(E);
            cpx<T>* wp = sm + spad<P>((j / NS) * NS * E + k);
#pragma unroll
            for (int e = 0; e < E; ++e) wp[pofs<P>(e * NS)] = v[e];
            exchange_sync<G, GB>();
            const cpx<T>* rp = sm + spad<P>(j);
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = rp[pofs<P>(e * G)];
            if constexpr (!DB) exchange_sync<G, GB>();
            fft_stages<T, M, E, INV, DB, DB ? 1 - BUF : 0, NS * E, false, GB>(v, j, sm0, sm1, tws);
        }
    } else {
        constexpr int R = M / NS;  // 2 <= R < E, last stage
        constexpr int B = E / R;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int jj = j + b * G;
            cpx<T> u[R], w[R];
            load_twiddles<T, R, NS>(tws + tw_offset(M, E, NS), jj, w);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                u[r] = v[b + r * B];
                if (r > 0) u[r] = INV ? cmulc(u[r], w[r]) : cmul(u[r], w[r]);
            }
            Dft<R, INV, T>::run(u);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * B] = u[r];
        }
    }
}

// Buffer a caller may write right after fft_stages<..., DB, BUF> returns
// (the one the next exchange would use).
__host__ __device__ constexpr int next_buf(int M, int E, bool DB, int BUF) {
    return DB ? (BUF + n_exchanges(M, E)) % 2 : 0;
}

}  // namespace fc
