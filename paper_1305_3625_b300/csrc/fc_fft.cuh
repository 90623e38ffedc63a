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

template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> w) {
    return {a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x};
}
// a * conj(w)
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> w) {
    return {a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y};
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

// cos and sin of 2 pi q / 16, q = 0..7 (exact mathematical constants).
constexpr double kCos16[8] = {1.0,
                              0.92387953251128675612818318939678829,
                              0.70710678118654752440084436210484904,
                              0.38268343236508977172845998403039887,
                              0.0,
                              -0.38268343236508977172845998403039887,
                              -0.70710678118654752440084436210484904,
                              -0.92387953251128675612818318939678829};
constexpr double kSin16[8] = {0.0,
                              0.38268343236508977172845998403039887,
                              0.70710678118654752440084436210484904,
                              0.92387953251128675612818318939678829,
                              1.0,
                              0.92387953251128675612818318939678829,
                              0.70710678118654752440084436210484904,
                              0.38268343236508977172845998403039887};

// Multiply by exp(-/+ 2 pi i Q/16) (forward / inverse), Q in [0, 8).
template <int Q, bool INV, typename T>
__device__ __forceinline__ cpx<T> rot16(cpx<T> a) {
    if constexpr (Q == 0) {
        return a;
    } else if constexpr (Q == 4) {
        return INV ? cpx<T>{-a.y, a.x} : cpx<T>{a.y, -a.x};
    } else if constexpr (Q == 2 || Q == 6) {
        constexpr T h = (T)kCos16[2];
        // (1 -/+ i) h  for Q = 2, (-1 -/+ i) h for Q = 6
        if constexpr (Q == 2)
            return INV ? cpx<T>{(a.x - a.y) * h, (a.x + a.y) * h} : cpx<T>{(a.x + a.y) * h, (a.y - a.x) * h};
        else
            return INV ? cpx<T>{-(a.x + a.y) * h, (a.x - a.y) * h} : cpx<T>{(a.y - a.x) * h, -(a.x + a.y) * h};
    } else {
        constexpr T c = (T)kCos16[Q];
        constexpr T s = INV ? (T)kSin16[Q] : -(T)kSin16[Q];
        return {a.x * c - a.y * s, a.x * s + a.y * c};
    }
}

template <int R, bool INV, typename T, int... K>
__device__ __forceinline__ void twiddle_consts(cpx<T>* o, std::integer_sequence<int, K...>) {
    ((o[K] = rot16<K * 16 / R, INV>(o[K])), ...);
}

// In-register R-point DFT (R = 1, 2, 4, 8, 16), natural order in and out,
// by recursive radix-2 decimation in time.
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
        twiddle_consts<R, INV, T>(o, std::make_integer_sequence<int, R / 2>{});
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            v[k] = e[k] + o[k];
            v[k + R / 2] = e[k] - o[k];
        }
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

// Shared-memory index with one padding slot every 16 elements; it spreads the
// radix-16 "expand" writes (stride 16) over the banks.  For every access
// pattern of the stages below, spad(base + c) = spad(base) + c + (c >> 4)
// with c a compile-time multiple of the stride (checked exhaustively for all
// M <= 8192, E in {2,4,8,16}), so addresses are a base plus immediates.
__host__ __device__ __forceinline__ constexpr int spad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int seg_len(int M) { return M + (M >> 4) + 2; }
__host__ __device__ constexpr int pofs(int c) { return c + (c >> 4); }

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
// a second barrier.  tws: the stage twiddle table of (M, E).  All threads of
// the block call this together.
template <typename T, int M, int E, bool INV, bool DB, int BUF = 0, int NS = 1>
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
        Dft<E, INV, T>::run(v);
        if constexpr (NS * E < M) {
            cpx<T>* sm = (DB && BUF) ? sm1 : sm0;
            cpx<T>* wp = sm + spad((j / NS) * NS * E + k);
#pragma unroll
            for (int e = 0; e < E; ++e) wp[pofs(e * NS)] = v[e];
            __syncthreads();
            const cpx<T>* rp = sm + spad(j);
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = rp[pofs(e * G)];
            if constexpr (!DB) __syncthreads();
            fft_stages<T, M, E, INV, DB, DB ? 1 - BUF : 0, NS * E>(v, j, sm0, sm1, tws);
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
