// Compiled launch shapes of the FFT passes (the autotuner's candidates).
// The kernels of each padded size M are instantiated in a translation unit
// of their own (fc_var_*.cu), so that the sizes compile in parallel; this
// header holds the tables those units fill in.
#pragma once

#include <stddef.h>

namespace fc {

// One compiled launch shape of a pass: E values per thread (stage radix) and
// `per` row pairs (passes A, C) or columns (pass B) per block.
struct KV {
    const void* f = nullptr;
    int threads = 0, per = 0, E = 0;
    size_t smem = 0;
    int tma = 0;  // 1: TMA-staged persistent pass C (k_rinv_tma; needs the plan's tensor map)
    const void* fp = nullptr;  // pass A: the same shape's PCG step-deciding kernel (k_rfwd_pcg)
    const void* fplain = nullptr;  // passes A, C: the same shape's plain-apply kernel (k_rfwd_plain, k_rinv_plain)
};

// One compiled persistent inner-CG kernel: pass A/C shape (EA, RB) and
// pass B shape (EB, CB) with the same block size.
struct KVP {
    const void* f = nullptr;
    int threads = 0, EA = 0, RB = 0, EB = 0, CB = 0;
    size_t smem = 0;
};

struct Variants {
    static constexpr int kMax = 16;  // compiled shapes per pass and size (at most)
    KV rfwd[kMax], colc[kMax], rinv[kMax];
    int n_rfwd = 0, n_colc = 0, n_rinv = 0;
    KVP pers[6];
    int n_pers = 0;
    KV rows_full, cols_full;  // FP64 only: spectrum set-up
    // the batched twins (blockIdx.y = problem, the same arithmetic per problem)
    // of rfwd[k], colc[k], rinv[k]; an entry with f == nullptr has none (the
    // TMA-staged pass C)
    KV rfwd_b[kMax], colc_b[kMax], rinv_b[kMax];
};

// Fill v with the compiled shapes of size M in FP32 (f64 = false) or FP64;
// false for a size that has none.  One definition per padded size, each in
// its own translation unit.
bool variants_small(int M, bool f64, Variants* v);  // M = 2 .. 128
void variants_256(bool f64, Variants* v);
void variants_512(bool f64, Variants* v);
void variants_1024(bool f64, Variants* v);
void variants_2048(bool f64, Variants* v);
void variants_4096(bool f64, Variants* v);
void variants_8192(bool f64, Variants* v);

}  // namespace fc
