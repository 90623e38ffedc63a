// Template machinery that instantiates the pass kernels of one padded size
// and records their launch shapes (included by the fc_var_*.cu units only).
#pragma once

#include "fc_persist.cuh"
#include "fc_tma.cuh"
#include "fc_variants.h"

namespace fc {

// Unpruned forward FFT of every row of an M x M grid (spectrum set-up only).
template <int M, int E, int RB>
__global__ void __launch_bounds__(RB*(M / E)) k_rows_full(cpx<double>* K, const cpx<double>* tw) {
    using C = cpx<double>;
    constexpr int G = M / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int j = threadIdx.x % G, c = threadIdx.x / G, row = blockIdx.x * RB + c;
    const bool ok = row < M;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = ok ? K[(size_t)row * M + j + e * G] : C{0, 0};
    fft_stages<double, M, E, false, false, 0>(v, j, sm + c * seg_len(M), sm + c * seg_len(M), tw);
    if (ok)
#pragma unroll
        for (int e = 0; e < E; ++e) K[(size_t)row * M + j + e * G] = v[e];
}

// Unpruned forward FFT of every column of an M x M grid.
template <int M, int E, int CB>
__global__ void __launch_bounds__(CB*(M / E)) k_cols_full(cpx<double>* K, const cpx<double>* tw) {
    using C = cpx<double>;
    constexpr int G = M / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int c = threadIdx.x % CB, j = threadIdx.x / CB, col = blockIdx.x * CB + c;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = K[(size_t)(j + e * G) * M + col];
    fft_stages<double, M, E, false, false, 0>(v, j, sm + c * seg_len(M), sm + c * seg_len(M), tw);
#pragma unroll
    for (int e = 0; e < E; ++e) K[(size_t)(j + e * G) * M + col] = v[e];
}

constexpr int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T, int M, int E, int RB, int MINB = 1, bool DB = use_db<T, M, RB>()>
void add_row(Variants& v) {
    if constexpr (RB * (M / E) <= 1024 && pass_smem<T, M, RB, DB>() <= 200 * 1024) {
        KV f{(const void*)k_rfwd<T, M, E, RB, MINB, DB>, RB * (M / E), RB, E, pass_smem<T, M, RB, DB>()};
        f.fp = (const void*)k_rfwd_pcg<T, M, E, RB, MINB, DB>;
        f.fplain = (const void*)k_rfwd_plain<T, M, E, RB, MINB, DB>;
        KV i{(const void*)k_rinv<T, M, E, RB, MINB, DB>, RB * (M / E), RB, E, pass_smem<T, M, RB, DB>()};
        i.fplain = (const void*)k_rinv_plain<T, M, E, RB, MINB, DB>;
        for (int k = 0; k < v.n_rfwd; ++k)
            if (v.rfwd[k].f == f.f) return;
        if (v.n_rfwd >= Variants::kMax || v.n_rinv >= Variants::kMax) return;
        // the batched twins (same arithmetic, blockIdx.y = problem) at the same index
        v.rfwd_b[v.n_rfwd] = KV{(const void*)k_rfwd_b<T, M, E, RB, MINB, DB>, f.threads, RB, E, f.smem};
        v.rinv_b[v.n_rinv] = KV{(const void*)k_rinv_b<T, M, E, RB, MINB, DB>, i.threads, RB, E, i.smem};
        v.rfwd[v.n_rfwd++] = f;
        v.rinv[v.n_rinv++] = i;
    }
}

// TMA-staged pass C (FP32): one row pair per loop iteration, M/E threads.
template <int M, int E = 16>
void add_rinv_tma(Variants& v) {
    // whole warps per block (the block reductions shuffle across full warps)
    if constexpr (M / E >= 32 && tma_smem_bytes(M) <= 200 * 1024) {
        // no batched twin: rinv_b at this index stays empty
        if (v.n_rinv < Variants::kMax) {
            KV k{(const void*)k_rinv_tma<M, E>, M / E, 1, E, tma_smem_bytes(M), 1};
            k.fplain = (const void*)k_rinv_tma<M, E, RI_PLAIN>;
            v.rinv[v.n_rinv++] = k;
        }
    }
}

template <typename T, int M, int E, int CB, int MINB = 1, bool DB = use_db<T, M, CB>(), bool GB = false>
void add_col(Variants& v) {
    if constexpr (CB * (M / E) <= 1024 && pass_smem<T, M, CB, DB>() <= 200 * 1024 &&
                  (!GB || ((M / E) % 32 == 0 && CB > 1 && CB <= 15))) {
        KV c{(const void*)k_colc<T, M, E, CB, MINB, DB, GB>, CB * (M / E), CB, E, pass_smem<T, M, CB, DB>()};
        for (int k = 0; k < v.n_colc; ++k)
            if (v.colc[k].f == c.f) return;
        if (v.n_colc >= Variants::kMax) return;
        v.colc_b[v.n_colc] = KV{(const void*)k_colc_b<T, M, E, CB, MINB, DB, GB>, c.threads, CB, E, c.smem};
        v.colc[v.n_colc++] = c;
    }
}

template <typename T, int M, int EA, int EB, int NT>
void add_pers(Variants& v) {
    constexpr int GA = EA <= M ? M / EA : 1, GB = EB <= M ? M / EB : 1;
    constexpr int RB = NT / GA, CB = NT / GB;
    constexpr size_t SA = pass_smem<T, M, (RB > 0 ? RB : 1)>(), SB = pass_smem<T, M, (CB > 0 ? CB : 1)>();
    constexpr size_t SM = SA > SB ? SA : SB;
    if constexpr (M >= 64 && EA <= M && EB <= M && RB >= 1 && CB >= 1 && RB * GA == NT && CB * GB == NT &&
                  CB <= M / 2 && NT <= 1024 && NT % 32 == 0 && SM <= 200 * 1024) {
        if (v.n_pers < 6)
            v.pers[v.n_pers++] = KVP{(const void*)k_cg_persist<T, M, EA, RB, EB, CB>, NT, EA, RB, EB, CB, SM};
    }
}

// Launch shapes compiled for each (precision, M).  FP32 sizes from 256 up
// carry seven to twelve shapes per pass for the autotuner: E = 32, 16, 8 or 4 with
// one or more rows or columns per block, single-buffered 64-register shapes
// (more resident blocks), 1024-thread row blocks, and the TMA-staged pass C.
// FP64 (ALU-bound on this part) carries one or two: radix 8 and radix 16.
template <typename T, int M>
void make_variants(Variants& v) {
    constexpr int H = M / 2;
    if constexpr (sizeof(T) == 4) {
        if constexpr (M <= 16) {
            add_row<T, M, M, 64>(v);
            add_col<T, M, M, clampi(64, 1, H)>(v);
        } else if constexpr (M <= 128) {
            constexpr int G = M / 16;
            add_row<T, M, 16, clampi(128 / G, 1, 128)>(v);
            add_col<T, M, 16, clampi(256 / G, 1, H)>(v);
        } else {
            constexpr int G16 = M / 16, G8 = M / 8, G4 = M / 4;
            add_row<T, M, 16, clampi(256 / G16, 1, 64)>(v);
            add_row<T, M, 16, clampi(512 / G16, 1, 64)>(v);
            add_row<T, M, 8, clampi(256 / G8, 1, 64)>(v);
            add_row<T, M, 8, clampi(512 / G8, 1, 64)>(v);
            add_row<T, M, 4, clampi(512 / G4, 1, 64)>(v);
            add_col<T, M, 16, clampi(128 / G16, 1, H)>(v);
            add_col<T, M, 16, clampi(256 / G16, 1, H)>(v);
            add_col<T, M, 8, clampi(256 / G8, 1, H)>(v);
            add_col<T, M, 8, clampi(512 / G8, 1, H)>(v);
            add_col<T, M, 4, clampi(512 / G4, 1, H)>(v);
            // single-buffered, at most 64 registers: more resident blocks
            // (a one-wave grid where the default shapes need 1.15 waves)
            constexpr int C1 = clampi(128 / G16, 1, H), C2 = clampi(256 / G16, 1, H);
            constexpr int R1 = clampi(128 / G16, 1, 64), R2 = clampi(256 / G16, 1, 64);
            add_col<T, M, 16, C1, clampi(65536 / (C1 * G16 * 64), 1, 16), false>(v);
            add_col<T, M, 16, C2, clampi(65536 / (C2 * G16 * 64), 1, 16), false>(v);
            // the same with a 72-register cap (fewer spills, one block fewer per SM)
            constexpr int MB72 = clampi(65536 / (C1 * G16 * 72), 1, 16);
            if constexpr (MB72 > 1) add_col<T, M, 16, C1, MB72, false>(v);
            add_row<T, M, 16, R1, clampi(65536 / (R1 * G16 * 64), 1, 16), false>(v);
            add_row<T, M, 16, R2, clampi(65536 / (R2 * G16 * 64), 1, 16), false>(v);
            // 1024-thread row blocks: more rows per block make the column-major
            // intermediate's row segments longer (full 32-byte sectors at M = 8192)
            add_row<T, M, 16, clampi(1024 / G16, 1, 64), 1, false>(v);
            if constexpr (M >= 4096) {
                // radix-32 stages: one exchange fewer per transform at M = 8192
                // (32^2 x 8; below M = 4096 they timed no faster than radix 16)
                constexpr int G32 = M / 32;
                add_row<T, M, 32, clampi(256 / G32, 1, 64)>(v);
                add_row<T, M, 32, clampi(512 / G32, 1, 64)>(v);
                add_col<T, M, 32, clampi(256 / G32, 1, H)>(v);
                add_col<T, M, 32, clampi(256 / G32, 1, H), 2>(v);
                add_col<T, M, 32, clampi(512 / G32, 1, H)>(v);
                // the same with each column's exchanges on its own named barrier
                add_col<T, M, 32, clampi(512 / G32, 1, H), 1, use_db<T, M, clampi(512 / G32, 1, H)>(), true>(v);
            }
            add_rinv_tma<M>(v);
            if constexpr (M >= 4096) add_rinv_tma<M, 32>(v);
        }
        add_pers<T, M, 16, 16, (M * M / 32 < 256 ? M * M / 32 : 256)>(v);
        add_pers<T, M, 16, 8, 256>(v);
        add_pers<T, M, 8, 8, 256>(v);
        add_pers<T, M, 16, 16, 512>(v);
        add_pers<T, M, 8, 8, 512>(v);
        add_pers<T, M, 8, 8, 1024>(v);
    } else {
        constexpr int E = M <= 8 ? M : (M <= 2048 ? 8 : 16);
        constexpr int G = M / E;
        constexpr int RB = M <= 8 ? 64 : clampi(256 / G, 1, 128);
        constexpr int CB = clampi(256 / G, 1, H);
        add_row<T, M, E, RB>(v);
        add_col<T, M, E, CB>(v);
        if constexpr (M >= 256 && M <= 2048) {
            // radix 16: one twiddled stage fewer than radix 8 below M = 4096
            constexpr int G16 = M / 16;
            add_row<T, M, 16, clampi(256 / G16, 1, 128)>(v);
            add_col<T, M, 16, clampi(256 / G16, 1, H)>(v);
        }
        constexpr int CBF = clampi(256 / G, 1, M);
        v.rows_full = KV{(const void*)k_rows_full<M, E, RB>, RB * G, RB, E, (size_t)RB * seg_len(M) * sizeof(cpx<double>)};
        v.cols_full = KV{(const void*)k_cols_full<M, E, CBF>, CBF * G, CBF, E, (size_t)CBF * seg_len(M) * sizeof(cpx<double>)};
        add_pers<T, M, E, E, (M / E) * 4 <= 256 ? (M / E) * 4 : (M / E)>(v);
        add_pers<T, M, E, E, 256>(v);
    }
}

}  // namespace fc
