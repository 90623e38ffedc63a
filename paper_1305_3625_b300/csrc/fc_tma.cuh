// Pass C (inverse row FFT + crop + epilogue) with its input staged by the
// Tensor Memory Accelerator.
//
// The pass reads the column-major half spectra Zt[kx][row]: for one row pair
// that is 16 bytes per column kx, a strided gather that the thread-issued
// loads of k_rinv wait on (the dominant stall at large L).  Here one thread
// per block describes the pair's rows as 2D tensor boxes (4 floats = the two
// rows' complex values, by up to 256 columns) and the TMA unit copies them
// into shared memory while the block transforms the previous pair: a
// persistent loop over row pairs with two staging buffers, each signalled by
// its own mbarrier (expected transaction bytes).  A buffer, once its staged
// values are in registers, serves as the exchange buffer of that pair's FFT.
// All waits are bounded; a wait that runs out sets tma_err in the solve state
// (the step decisions then end the solve with FC_ETIMEOUT) and the block stops
// transforming, waits (bounded) for its copies in flight and still joins the
// grid reduction.
#pragma once

#include <cuda.h>

#include "fc_passes.cuh"

namespace fc {

// ------------------------------------------------------------ PTX helpers --

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Order this thread's earlier shared-memory accesses (generic proxy) before
// later accesses of the async proxy (TMA writes, mbarrier transactions).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; gives up after
// `limit` polls (2^20 by default; each try_wait may itself suspend the
// thread briefly: well over the microseconds a staged copy takes, well under
// a second) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 2D tiled TMA load of one box into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- pass C --

// Arguments of the TMA pass C: the ordinary pass-C arguments, the number of
// row pairs, and the tensor map of Zt viewed as floats [M/2][2L] (box: 4
// floats x BK columns).
struct RowInvTma {  // CUtensorMap carries its own (64-byte or wider) alignment
    CUtensorMap map;
    RowInvArgs<float> a;
    int units;
};

// Bytes of one staging buffer: the larger of the pair's two half spectra
// (M/2 columns x 16 bytes) and the FFT's exchange segment, 128-byte aligned.
__host__ __device__ constexpr size_t tma_buf_bytes(int M) {
    const size_t stage = (size_t)(M / 2) * 16, seg = (size_t)seg_len(M) * sizeof(cpx<float>);
    const size_t b = stage > seg ? stage : seg;
    return (b + 127) / 128 * 128;
}
// Two staging buffers.  (A third buffer for double-buffered exchanges, one
// barrier per exchange, measured slower at M = 8192: the shared-memory
// carve-out it takes leaves too little L1 for the twiddle tables.)
__host__ __device__ constexpr size_t tma_smem_bytes(int M) { return 2 * tma_buf_bytes(M) + 128; }
__host__ __device__ constexpr int tma_box_cols(int M) { return M / 2 < 256 ? M / 2 : 256; }

// MODE >= 0: the pass-C mode fixed at compile time (RI_PLAIN: the plain
// apply's form, without the other modes' epilogues and sums).
template <int M, int E, int MODE = -1>
__global__ void __launch_bounds__(M / E) k_rinv_tma(const __grid_constant__ RowInvTma P) {
    using C = cpx<float>;
    constexpr int G = M / E, H = M / 2, BK = tma_box_cols(M), NBOX = H / BK;
    constexpr unsigned UNIT_BYTES = (unsigned)H * 16u;
    constexpr size_t BUF = tma_buf_bytes(M);
    static_assert(H % BK == 0 && (BK * 16) % 128 == 0, "TMA boxes must tile the pair's columns");
    static_assert(G % 32 == 0, "the block reductions need whole warps");
    extern __shared__ __align__(16) unsigned char smraw[];  // aligned to 128 bytes below
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_ok;
    const RowInvArgs<float>& a = P.a;
    // 128-byte aligned staging buffers (TMA destinations)
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 127) & ~(uintptr_t)127);
    C* buf[2] = {reinterpret_cast<C*>(base), reinterpret_cast<C*>(base + BUF)};
    const int j = threadIdx.x;
    const int L = a.L;
    pdl_enter();
    if (a.mode == RI_PQ && a.st->idle) return;  // PCG: the z pass ended the run (no copy issued yet)
    const unsigned limit = a.st->dbg_limit ? a.st->dbg_limit : (1u << 20);
    // test hook: no copy for the block's first row pair, its waits run out
    const bool skip_first = a.st->dbg_skip == 2;
    if (j == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    auto issue = [&](int unit, int b) {
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[b], UNIT_BYTES);
#pragma unroll 1
        for (int k = 0; k < NBOX; ++k)
            tma_load_2d(reinterpret_cast<unsigned char*>(buf[b]) + (size_t)k * BK * 16, &P.map, 4 * unit, k * BK,
                        &bar[b]);
    };
    Acc<float> s0, s1, s2, s3, s4;
    unsigned ph0 = 0, ph1 = 0;
    bool pending[2] = {false, false};
    int u = blockIdx.x;
    if (j == 0 && u < P.units && !skip_first) issue(u, 0);
    pending[0] = u < P.units;
    bool ok = true;
    for (int it = 0; u < P.units; ++it, u += gridDim.x) {
        const int cur = it & 1;
        const int nu = u + gridDim.x;
        if (j == 0 && nu < P.units) issue(nu, cur ^ 1);
        pending[cur ^ 1] = nu < P.units;
        unsigned& ph = cur ? ph1 : ph0;
        if (j == 0) s_ok = mbar_wait_bounded(&bar[cur], ph, limit);
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        mbar_wait_bounded(&bar[cur], ph, limit);  // completes at once; acquires the staged data in this thread
        ph ^= 1u;
        pending[cur] = false;
        const C* stg = buf[cur];
        // Hermitian extension of both rows and pair packing W = Y0 + i Y1
        // (stg[2 kx + h] = row h's value at column kx; slot 0 packs X[0] + i X[M/2])
        C v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = j + e * G;
            C y0, y1;
            if (k == 0) {
                y0 = C{stg[0].x, 0.f};
                y1 = C{stg[1].x, 0.f};
            } else if (k == H) {
                y0 = C{stg[0].y, 0.f};
                y1 = C{stg[1].y, 0.f};
            } else if (k < H) {
                const float4 q = *reinterpret_cast<const float4*>(stg + 2 * k);
                y0 = C{q.x, q.y};
                y1 = C{q.z, q.w};
            } else {
                const float4 q = *reinterpret_cast<const float4*>(stg + 2 * (M - k));
                y0 = C{q.x, -q.y};
                y1 = C{q.z, -q.w};
            }
            v[e] = C{y0.x - y1.y, y0.y + y1.x};
        }
        __syncthreads();  // staged values consumed: the buffer becomes the exchange buffer
        fft_stages<float, M, E, true, false, 0>(v, j, buf[cur], buf[cur], a.tw);
        pass_c_outputs<float, M, E>(MODE >= 0 ? MODE : a.mode, a.y, a.s, a.cp, a.cr, a.cq, a.cz, a.mask, a.x64, a.b64,
                                    a.s64, a.r64, j,
                                    2 * u, L, 0, v, s0, s1, s2, s3, s4);
        __syncthreads();  // exchanges done: the buffer may receive the copy issued next
    }
    if (!ok && j == 0) {
        // a staged copy never arrived: flag it (the step decisions then stop
        // the solve with FC_ETIMEOUT) and let the copies in flight land
        // (bounded) before the block's shared memory is released
        atomicExch(&a.st->tma_err, 1);
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait_bounded(&bar[b], b ? ph1 : ph0, limit);
    }
    pdl_leave();  // every block still joins the grid reduction below
    if constexpr (MODE != RI_PLAIN) rinv_sums(a, a.part, a.st, s0, s1, s2, s3, s4);
}

}  // namespace fc
