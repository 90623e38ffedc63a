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
// radix-16 "expand" writes (stride 16) over the banks.
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int seg_len(int M) { return M + (M >> 4) + 2; }

constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// Stockham transform of one length-M sequence held by G = M/E threads as
// v[e] = x[j + e*G] (thread j of its group); on return v[e] = X[j + e*G].
// sm is this group's shared segment (seg_len(M) elements); tw[m] =
// exp(-2 pi i m / M).  All threads of the block call this together (it uses
// __syncthreads between the exchanges).
template <typename T, int M, int E, bool INV, int NS = 1>
__device__ __forceinline__ void fft_stages(cpx<T> (&v)[E], int j, cpx<T>* sm, const cpx<T>* __restrict__ tw) {
    constexpr int G = M / E;
    if constexpr (NS * E <= M) {
        const int k = j & (NS - 1);
        if constexpr (NS > 1) {
            constexpr int step = M / (NS * E);
#pragma unroll
            for (int e = 1; e < E; ++e) {
                cpx<T> w = ldg_c(tw + e * k * step);
                v[e] = INV ? cmulc(v[e], w) : cmul(v[e], w);
            }
        }
        Dft<E, INV, T>::run(v);
        if constexpr (NS * E < M) {
            const int idxD = (j / NS) * NS * E + k;
#pragma unroll
            for (int e = 0; e < E; ++e) sm[spad(idxD + e * NS)] = v[e];
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = sm[spad(j + e * G)];
            __syncthreads();
            fft_stages<T, M, E, INV, NS * E>(v, j, sm, tw);
        }
    } else {
        constexpr int R = M / NS;  // 2 <= R < E, last stage
        constexpr int B = E / R;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int jj = j + b * G;
            cpx<T> u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                u[r] = v[b + r * B];
                if (r > 0) {
                    cpx<T> w = ldg_c(tw + r * jj);
                    u[r] = INV ? cmulc(u[r], w) : cmul(u[r], w);
                }
            }
            Dft<R, INV, T>::run(u);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * B] = u[r];
        }
    }
}

}  // namespace fc
