// Depth sweeps with the lateral transforms as DFT-matrix products on the fifth-generation tensor
// cores (tcgen05: single-thread MMAs with shared-memory operands and TMEM accumulators), a precision
// variant of the split-step depth step (Examples section), for nx = 16 R with R = 8, 16, 32, 64.
//
// Four-step factorisation, N = 16 R: an item's points x[R n1 + n2] form X[n1][n2] (16 x R) and
//   forward  Y = F16 X,  Y'[k1][n2] = Y[k1][n2] w^(k1 n2),  Z = Y' F_R,  Z[k1][k2] = x^[k1 + 16 k2],
//   inverse  Y'' = Z conj(F_R),  Y'''[k1][n2] = Y''[k1][n2] w^-(k1 n2),  X' = conj(F16) Y''',
// w = exp(-2 pi i / N); the 1/N sits in the phase-shift table (natural frequency order).  Every
// product is one real GEMM with the data as the M = 128-row operand and the real form of the DFT
// matrix as the N operand: a complex row vector enters as its interleaved (re, im) values and the
// constant matrix [[Fr, -Fi], [Fi, Fr]] (interleaved the same way) gives the interleaved (re, im)
// outputs.  Operands are split as x = hi + lo in 16 bits and every product takes the three terms
// hi hi + hi lo + lo hi:
//   BF16: hi = bf16(x), lo = bf16(x - hi), all three terms in one FP32 accumulator;
//   FP16: hi = fp16(x), lo = fp16((x - hi) 2^11), hi hi in one accumulator and the two scaled cross
//         terms in a second one, added as acc0 + 2^-11 acc1; each item is brought to a largest
//         component in [1/2, 1) by an exact power-of-two scale before each depth step (FP16's exponent
//         range) and scaled back after it.
// A row of an operand holds [hi | lo] along K, so the three terms are three K ranges of the same
// two tiles (A hi x B hi, A hi x B lo, A lo x B hi).  The inverse products use the forward matrices
// through conj(M conj(F)) = conj(conj(M) F): the operand is written conjugated and the accumulator
// read back conjugated, so only F16 and F_R are kept in shared memory.
//
// A CTA runs ITEMS (shot, frequency) items through the whole depth loop (16 at R = 8, else 8).  The
// left products (16-point, contraction over n1) take rows (item, n2), ITEMS R rows in 128-row tiles;
// the right products (R-point, contraction over n2) take rows (item, k1), ITEMS 16 rows.  Each group
// of 128 threads (one at R <= 32, two at R = 64) owns one TMEM lane per thread: thread r of a group
// owns row r of its left tiles -- the wavefield lives in those registers between depth steps -- and
// row r of the right tiles (at R = 64 the two groups split the right product's columns).  The
// passage between the two row layouts goes through the shared-memory operand tiles.  One thread
// issues the MMAs of a stage and commits them to an mbarrier that every thread waits on (bounded:
// a wait that runs out sets the error flag, the CTA stops and writes NaN to its outputs).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lsm_async.cuh"
#include "lsm_fft.cuh"
#include "lsm_internal.h"
#include "lsm_tc.cuh"
#include "lsm_umma.cuh"

namespace lsm {

// tcgen05 transform precisions (numbering continues TcPrecision)
enum Tc5Precision { PREC_FP16X3_TC5 = 4, PREC_BF16X3_TC5 = 5 };

// Widths with a tcgen05 transform: N = 16 R, R = 8 .. 64 (the right product's N = 2 R must be a
// multiple of 16 for M = 128, and a CTA's right operand rows must fill 128-row tiles).
constexpr bool tc5_width(int n) { return n == 128 || n == 256 || n == 512 || n == 1024; }

template <int N>
struct Tc5Shape {
    static_assert(tc5_width(N), "tcgen05 transforms: nx = 128, 256, 512 or 1024");
    static constexpr int R = N / 16;
    static constexpr int ITEMS = R == 8 ? 16 : 8;     // items per CTA
    static constexpr int GROUPS = R == 64 ? 2 : 1;    // 128-thread groups
    static constexpr int THREADS = 128 * GROUPS;
    static constexpr int LT = ITEMS * R / 128;        // left tiles (128 rows (item, n2) each)
    static constexpr int LTT = LT / GROUPS;           // left tiles per thread
    static constexpr int RT = ITEMS * 16 / 128;       // right tiles (128 rows (item, k1) each)
    static constexpr int RCOLS = 2 * R / GROUPS;      // right-product columns per thread
    static constexpr int RCH = RCOLS >= 32 ? 32 : RCOLS;  // columns per TMEM load of the right product
    static constexpr int KB_R = (4 * R + 63) / 64;    // 64-element K blocks of a right operand row
    static constexpr int LTILE = 128 * 128;           // bytes of a left tile (K = 64: hi 32 | lo 32)
    static constexpr int RTILE = KB_R * 128 * 128;    // bytes of a right tile (K = 4 R: hi 2R | lo 2R)
    // shared memory (bytes from the 1024-aligned base): the constant B operands of the left product
    // (32 rows x 64 K) and of the right product (2 R rows x 4 R K), the A operand (the left tiles or
    // the right tiles; the adjoint's four image rows use it between depth steps), the twiddles in both
    // index orders, then the staged phase-shift and split-step rows of the CTA's frequencies: per
    // frequency slot one Phi row and one D row
    static constexpr int OFF_BLF = 0;
    static constexpr int OFF_BRF = OFF_BLF + 32 * 128;
    static constexpr int BRF_BYTES = KB_R * 2 * R * 128;
    static constexpr int OFF_A = (OFF_BRF + BRF_BYTES + 1023) / 1024 * 1024;
    static constexpr int A_BYTES = LT * LTILE > RT * RTILE ? LT * LTILE : RT * RTILE;
    static constexpr int OFF_TW = OFF_A + A_BYTES;             // w^(k1 n2) as [k1][n2] float2
    static constexpr int OFF_TWT = OFF_TW + 16 * R * 8;        // the same as [n2][k1]
    static constexpr int OFF_STG = OFF_TWT + 16 * R * 8;       // [wslots][Phi row, D row]
    static constexpr int SLOT_BYTES = 2 * N * 8;
    static_assert(OFF_A % 1024 == 0, "operand tiles are 1024-byte aligned");
    static_assert(4 * N * 4 <= A_BYTES, "the adjoint's image rows fit the operand buffer");
    // TMEM columns: left accumulators [tile][acc][32], right accumulators [tile][acc][2R]; at R = 64
    // both sets take the same columns (an accumulator is read out before the next product is issued)
    static constexpr uint32_t TM_L = 0;
    static constexpr uint32_t TM_R = R == 64 ? 0 : (uint32_t)(64 * LT);
    static constexpr uint32_t TM_NEED = R == 64 ? (uint32_t)(64 * LT) : (uint32_t)(64 * LT + 4 * R * RT);
    static constexpr uint32_t TM_COLS = TM_NEED <= 32 ? 32 : TM_NEED <= 64 ? 64 : TM_NEED <= 128 ? 128 : 256;
    static_assert(TM_NEED <= 256 && 4 * R * RT <= 256, "accumulators fit 256 TMEM columns");
    static constexpr int MIN_BLOCKS = R == 64 ? 1 : 2;
};

template <int PREC>
struct Tc5Split {
    static constexpr bool FP16 = PREC == PREC_FP16X3_TC5;
    // packed 16-bit pair (lo half = first value) of hi parts and of lo parts of (x0, x1)
    static __device__ __forceinline__ void split(float x0, float x1, uint32_t& hi, uint32_t& lo) {
        const float2 x = make_float2(x0, x1);
        if constexpr (FP16) {
            const __half2 h = __floats2half2_rn(x0, x1);
            const float2 hf = __half22float2(h);
            // (x - hi) 2^11 as one paired multiply and one paired fused multiply-add
            const float2 r = __ffma2_rn(hf, make_float2(-2048.f, -2048.f), __fmul2_rn(x, make_float2(2048.f, 2048.f)));
            const __half2 l = __floats2half2_rn(r.x, r.y);
            hi = *reinterpret_cast<const uint32_t*>(&h);
            lo = *reinterpret_cast<const uint32_t*>(&l);
        } else {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            const float2 r = __ffma2_rn(__bfloat1622float2(h), make_float2(-1.f, -1.f), x);
            const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
            hi = *reinterpret_cast<const uint32_t*>(&h);
            lo = *reinterpret_cast<const uint32_t*>(&l);
        }
    }
    static __device__ __forceinline__ uint16_t hi16(float x) {
        if constexpr (FP16) {
            const __half h = __float2half_rn(x);
            return *reinterpret_cast<const uint16_t*>(&h);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            return *reinterpret_cast<const uint16_t*>(&h);
        }
    }
    static __device__ __forceinline__ float hi_value(float x) {
        if constexpr (FP16) return __half2float(__float2half_rn(x));
        else return __bfloat162float(__float2bfloat16_rn(x));
    }
    static __device__ __forceinline__ uint16_t lo16(float x) {
        const float r = x - hi_value(x);
        if constexpr (FP16) {
            const __half h = __float2half_rn(r * 2048.f);
            return *reinterpret_cast<const uint16_t*>(&h);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(r);
            return *reinterpret_cast<const uint16_t*>(&h);
        }
    }
};

// Constant B operand of one complex product with a DFT matrix G[n][k] = exp(sgn 2 pi i n k / L)
// (contraction over n, output k), in the real interleaved form: row c = 2 k + o (o = 0 re, 1 im) of
// nrows = 2 L rows; K element 2 n + q (q = 0 re, 1 im) of the hi part, and kper + 2 n + q of the lo
// part.  K runs in blocks of 64 elements, block b at base + b * nrows * 128.
template <int PREC>
__device__ void tc5_build_dft(unsigned char* base, int L, int sgn, int kper) {
    using SP = Tc5Split<PREC>;
    const int nrows = 2 * L;
    const int kk = 2 * L;  // K elements of each part (hi, lo)
    for (int idx = threadIdx.x; idx < nrows * kk; idx += blockDim.x) {
        const int c = idx / kk, k = idx % kk;
        const int kf = c >> 1, o = c & 1, n = k >> 1, q = k & 1;
        float sn, cs;
        sincospif((float)sgn * 2.0f * (float)((n * kf) % L) / (float)L, &sn, &cs);
        // (Gr + i Gi)(xr + i xi): re = Gr xr - Gi xi, im = Gi xr + Gr xi
        const float b = o == 0 ? (q == 0 ? cs : -sn) : (q == 0 ? sn : cs);
        const int khi = k, klo = kper + k;
        *reinterpret_cast<uint16_t*>(base + (khi / 64) * nrows * 128 + umma::sw128_offset(c, khi % 64)) = SP::hi16(b);
        *reinterpret_cast<uint16_t*>(base + (klo / 64) * nrows * 128 + umma::sw128_offset(c, klo % 64)) = SP::lo16(b);
    }
}

// Issue the three split products of one stage: D (+)= A[k ranges] B[k ranges]; A and B are K-major
// 128B-swizzled operands whose K axis is [hi (kper) | lo (kper)] in blocks of 64; kper a multiple of 16.
template <int PREC>
__device__ __forceinline__ void tc5_issue(uint32_t d0, uint32_t d1, uint32_t a_base, int a_rows, uint32_t b_base,
                                          int b_rows, int kper, uint32_t idesc) {
    constexpr bool FP16 = PREC == PREC_FP16X3_TC5;
    auto kaddr = [](uint32_t base, int rows, int k) { return base + (uint32_t)((k / 64) * rows * 128 + (k % 64) * 2); };
    const int steps = kper / 16;
    // hi x hi
    for (int s = 0; s < steps; ++s)
        umma::mma_f16(d0, umma::desc_sw128(kaddr(a_base, a_rows, 16 * s)), umma::desc_sw128(kaddr(b_base, b_rows, 16 * s)),
                      idesc, s > 0);
    // hi x lo, lo x hi (FP16: second accumulator, scaled by 2^11)
    const uint32_t dx = FP16 ? d1 : d0;
    for (int s = 0; s < steps; ++s)
        umma::mma_f16(dx, umma::desc_sw128(kaddr(a_base, a_rows, 16 * s)),
                      umma::desc_sw128(kaddr(b_base, b_rows, kper + 16 * s)), idesc, FP16 ? s > 0 : true);
    for (int s = 0; s < steps; ++s)
        umma::mma_f16(dx, umma::desc_sw128(kaddr(a_base, a_rows, kper + 16 * s)),
                      umma::desc_sw128(kaddr(b_base, b_rows, 16 * s)), idesc, true);
}

// Dynamic shared memory of a CTA whose items span `wslots` frequencies; wslots = 0: the Phi and D
// rows are read from global memory (L2) instead of being staged.
template <int N>
constexpr size_t tc5_smem_bytes(int wslots) {
    return (size_t)Tc5Shape<N>::OFF_STG + (size_t)wslots * Tc5Shape<N>::SLOT_BYTES + 1024;
}

// acc0 + 2^-11 acc1 over C columns (FP16's two accumulators), as paired FMAs
template <int C>
__device__ __forceinline__ void tc5_combine(float (&y)[C], const float (&y2)[C]) {
#pragma unroll
    for (int i = 0; i < C; i += 2) {
        const float2 v = __ffma2_rn(make_float2(y2[i], y2[i + 1]), make_float2(1.f / 2048.f, 1.f / 2048.f),
                                    make_float2(y[i], y[i + 1]));
        y[i] = v.x;
        y[i + 1] = v.y;
    }
}

// C consecutive accumulator columns of this thread's lane (C = 16 or 32)
template <int C>
__device__ __forceinline__ void tc5_ld(uint32_t taddr, float (&v)[C]) {
    static_assert(C == 16 || C == 32, "TMEM loads of 16 or 32 columns");
    if constexpr (C == 32) umma::tmem_ld32(taddr, v);
    else umma::tmem_ld16(taddr, v);
}

// the accumulator columns [col, col + C) of this lane, FP16's two accumulators combined
template <int C, bool FP16>
__device__ __forceinline__ void tc5_read(uint32_t taddr, uint32_t acc1_offset, float (&v)[C]) {
    tc5_ld<C>(taddr, v);
    if constexpr (FP16) {
        float v2[C];
        tc5_ld<C>(taddr + acc1_offset, v2);
        tc5_combine<C>(v, v2);
    }
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }

template <int N, int PREC, int MODE>
__global__ void __launch_bounds__(Tc5Shape<N>::THREADS, Tc5Shape<N>::MIN_BLOCKS) tc5_sweep_kernel(const SweepArgs a) {
    using S = Tc5Shape<N>;
    using SP = Tc5Split<PREC>;
    constexpr bool FP16 = SP::FP16;
    constexpr int R = S::R, ITEMS = S::ITEMS, LT = S::LT, LTT = S::LTT, RT = S::RT;
    constexpr int RCOLS = S::RCOLS, RCH = S::RCH;
    extern __shared__ unsigned char tc5_smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float wmax[S::THREADS / 32][LTT];  // R = 64: each warp's maxima (an item spans two warps)
    unsigned char* base = tc5_smem_raw + ((1024u - (umma::smem_u32(tc5_smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = umma::smem_u32(base);
    float2* TW = reinterpret_cast<float2*>(base + S::OFF_TW);    // [k1][n2]
    float2* TWT = reinterpret_cast<float2*>(base + S::OFF_TWT);  // [n2][k1]
    unsigned char* stg = base + S::OFF_STG;
    unsigned char* Abuf = base + S::OFF_A;
    float* img = reinterpret_cast<float*>(Abuf);                 // [4][N], between depth steps only

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = tid >> 7;  // 128-thread group
    const int r = tid & 127;   // this thread's TMEM lane: row r of the tiles
    const int nitems = a.nshots * a.nw;
    const int shot0 = a.shot0_dev ? __ldg(a.shot0_dev) : a.shot0;
    const int nz = a.nz;
    const bool staged = a.wslots > 0;
    // frequencies of the CTA's items (frequency-major item order): slots w_first .. w_last
    const int w_first = min((int)blockIdx.x * ITEMS, nitems - 1) / a.nshots;
    const int w_last = (min(((int)blockIdx.x + 1) * ITEMS, nitems) - 1) / a.nshots;
    const int nslots = w_last - w_first + 1;  // <= a.wslots when staged

    // ---- set-up: constants, barrier, TMEM
    tc5_build_dft<PREC>(base + S::OFF_BLF, 16, -1, 32);
    tc5_build_dft<PREC>(base + S::OFF_BRF, R, -1, 2 * R);
    for (int idx = tid; idx < 16 * R; idx += S::THREADS) {
        const int k1 = idx / R, nn = idx % R;
        float sn, cs;
        sincospif(-2.0f * (float)((k1 * nn) % N) / (float)N, &sn, &cs);
        TW[idx] = make_float2(cs, sn);
        TWT[nn * 16 + k1] = make_float2(cs, sn);
    }
    umma::fence_smem_to_async();
    if (tid == 0) umma::mbar_init(&bar, 1);
    if (warp == 0) umma::tmem_alloc(&tslot, S::TM_COLS);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    uint32_t phase = 0;
    bool alive = true;

    // this thread's rows of the left tiles: slot i is row r of tile grp LTT + i, i.e. column n2 of
    // the CTA's item (128 tile + r) / R
    const int n2 = r % R;
    int itemL[LTT], iwL[LTT], shotL[LTT];
    bool okL[LTT];
#pragma unroll
    for (int i = 0; i < LTT; ++i) {
        itemL[i] = blockIdx.x * ITEMS + (128 * (grp * LTT + i) + r) / R;
        okL[i] = itemL[i] < nitems;
        iwL[i] = okL[i] ? itemL[i] / a.nshots : w_first;
        shotL[i] = okL[i] ? shot0 + (itemL[i] - iwL[i] * a.nshots) : shot0;
    }
    // rows of the right tiles: row r of tile sigma is (item (128 sigma + r) / 16, k1 = r % 16); this
    // thread reads the complex columns kb .. kb + RCOLS / 2 of it
    const int k1R = r % 16;
    const int kb = grp * (R / S::GROUPS);
    int iwR[RT];
#pragma unroll
    for (int sg = 0; sg < RT; ++sg) {
        const int item = blockIdx.x * ITEMS + (128 * sg + r) / 16;
        iwR[sg] = item < nitems ? item / a.nshots : w_first;
    }

    // the wavefield: u[i][n1] = x[R n1 + n2] of the item of left slot i
    float2 u[LTT][16];

    // staging of the Phi (which = 0) or D (which = 1) rows of depth `row` for the CTA's frequencies,
    // one cp.async group (nothing when the rows are read from global memory)
    auto stage_rows = [&](int row, int which) {
        if (!staged) return;
        constexpr int CH = N * 8 / 16;  // 16-byte chunks per row
        for (int c = tid; c < nslots * CH; c += S::THREADS) {
            const int sl = c / CH, ch = c - sl * CH;
            const float2* src = (which ? a.dss : a.phi) + ((size_t)(w_first + sl) * nz + row) * N + 2 * ch;
            cp_async16(stg + sl * S::SLOT_BYTES + which * (N * 8) + ch * 16, src);
        }
        cp_async_commit();
    };
    // the Phi and D rows of depth j at frequency iw
    auto phi_s = [&](int iw, int j) -> const float2* {
        if (staged) return reinterpret_cast<const float2*>(stg + (iw - w_first) * S::SLOT_BYTES);
        return a.phi + ((size_t)iw * nz + j) * N;
    };
    auto dss_s = [&](int iw, int j) -> const float2* {
        if (staged) return reinterpret_cast<const float2*>(stg + (iw - w_first) * S::SLOT_BYTES + N * 8);
        return a.dss + ((size_t)iw * nz + j) * N;
    };
    auto srow = [&](int i, int jz) -> float2* {
        const int slot = shotL[i] % a.ring;
        return a.S + (((size_t)slot * a.nw + iwL[i]) * nz + jz) * (size_t)N;
    };
    // the source-wavefield rows of depth jz of all the CTA's items into L2, one 128-byte line at a time
    auto prefetch_srows = [&](int jz) {
        constexpr int LINES = N * 8 / 128;
        if (jz < 0 || jz >= nz) return;
        for (int l = tid; l < ITEMS * LINES; l += S::THREADS) {
            const int item = blockIdx.x * ITEMS + l / LINES;
            if (item < nitems) {
                const int iw = item / a.nshots;
                const int slot = (shot0 + item - iw * a.nshots) % a.ring;
                const unsigned char* row =
                    reinterpret_cast<const unsigned char*>(a.S + (((size_t)slot * a.nw + iw) * nz + jz) * (size_t)N);
                prefetch_l2(row + (l % LINES) * 128);
            }
        }
    };

    // wait for the MMAs of a stage; every thread agrees on the outcome
    // (the phase advances only when every thread saw it complete, so that after a failure every
    // thread still names the pending phase)
    auto stage_wait = [&]() -> bool {
        const bool ok = umma::mbar_wait(&bar, phase);
        umma::fence_after_sync();
        const bool all = __syncthreads_and(ok) != 0;
        if (all) phase ^= 1u;
        return all;
    };
    // operand writes visible to the tensor core, then one thread issues a stage's products
    auto issue_left = [&]() {
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            constexpr uint32_t IDESC_L = umma::idesc_f16(!FP16, 128, 32);
#pragma unroll
            for (int tau = 0; tau < LT; ++tau)
                tc5_issue<PREC>(tmem + S::TM_L + tau * 64, tmem + S::TM_L + tau * 64 + 32,
                                sbase + S::OFF_A + tau * S::LTILE, 128, sbase + S::OFF_BLF, 32, 32, IDESC_L);
            umma::mma_commit(&bar);
        }
    };
    auto issue_right = [&]() {
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            constexpr uint32_t IDESC_R = umma::idesc_f16(!FP16, 128, 2 * R);
#pragma unroll
            for (int sg = 0; sg < RT; ++sg)
                tc5_issue<PREC>(tmem + S::TM_R + sg * 4 * R, tmem + S::TM_R + sg * 4 * R + 2 * R,
                                sbase + S::OFF_A + sg * S::RTILE, 128, sbase + S::OFF_BRF, 2 * R, 2 * R, IDESC_R);
            umma::mma_commit(&bar);
        }
    };
    // 32-bit (re, im) pair / 16-byte chunk of K elements at element e of row rr of the tile at `tile`
    auto kput32 = [](unsigned char* tile, int rr, int e, uint32_t v) {
        *reinterpret_cast<uint32_t*>(tile + (e / 64) * (128 * 128) + umma::sw128_offset(rr, e % 64)) = v;
    };
    auto kput128 = [](unsigned char* tile, int rr, int e, uint4 v) {
        *reinterpret_cast<uint4*>(tile + (e / 64) * (128 * 128) + umma::sw128_offset(rr, e % 64)) = v;
    };

    // One depth step on u: F^-1 (phi . F u) (conj(phi) when conj_phi) with the Phi row of depth j.
    // Staging: the D row d_row (>= 0) is requested after the first barrier and the Phi row phi_next
    // (>= 0) of the next step once this step's Phi row has been read; every staged row has landed and
    // is visible to all threads when the step returns.
    auto transform_step = [&](bool conj_phi, int j, int d_row, int phi_next) -> bool {
        // FP16: per-item power-of-two scale (an item is R consecutive rows of a left tile: R lanes of
        // a warp up to R = 32, two warps at R = 64)
        int ex[LTT];
#pragma unroll
        for (int i = 0; i < LTT; ++i) ex[i] = 0;
        if constexpr (FP16) {
            float mx[LTT];
#pragma unroll
            for (int i = 0; i < LTT; ++i) {
                mx[i] = 0.f;
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) mx[i] = fmaxf(mx[i], fmaxf(fabsf(u[i][n1].x), fabsf(u[i][n1].y)));
#pragma unroll
                for (int o = (R < 32 ? R : 32) / 2; o > 0; o >>= 1)
                    mx[i] = fmaxf(mx[i], __shfl_xor_sync(0xffffffffu, mx[i], o));
            }
            if constexpr (R == 64) {
                if (lane == 0) {
#pragma unroll
                    for (int i = 0; i < LTT; ++i) wmax[warp][i] = mx[i];
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < LTT; ++i) mx[i] = fmaxf(mx[i], wmax[warp ^ 1][i]);
            }
#pragma unroll
            for (int i = 0; i < LTT; ++i) {
                if (mx[i] > 0.f && mx[i] <= 3.0e38f) frexpf(mx[i], &ex[i]);
                ex[i] = max(-100, min(ex[i], 100));
                const float down = ldexpf(1.f, -ex[i]);
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) u[i][n1] = __fmul2_rn(u[i][n1], make_float2(down, down));
            }
        }
        // (1) left operand tiles: row r, K = [hi: (re, im) of n1 = 0..15 | lo: same]
#pragma unroll
        for (int i = 0; i < LTT; ++i) {
            unsigned char* tile = Abuf + (grp * LTT + i) * S::LTILE;
#pragma unroll
            for (int c = 0; c < 4; ++c) {  // chunk c: n1 = 4c .. 4c+3
                uint32_t h[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) SP::split(u[i][4 * c + q].x, u[i][4 * c + q].y, h[q], l[q]);
                kput128(tile, r, 8 * c, make_uint4(h[0], h[1], h[2], h[3]));
                kput128(tile, r, 32 + 8 * c, make_uint4(l[0], l[1], l[2], l[3]));
            }
        }
        issue_left();
        if (d_row >= 0) stage_rows(d_row, 1);
        if (!stage_wait()) return false;
        // (2) Y[k1][n2] of this thread's left rows -> twiddle -> right operand rows (item, k1),
        // K = 2 n2 + q
#pragma unroll
        for (int i = 0; i < LTT; ++i) {
            const int tau = grp * LTT + i;
            float y[32];
            tc5_read<32, FP16>(tmem + lane_base + S::TM_L + tau * 64, 32, y);
            const int item_local = (128 * tau + r) / R;
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const float2 v = cmul(make_float2(y[2 * k1], y[2 * k1 + 1]), TW[k1 * R + n2]);
                uint32_t h, l;
                SP::split(v.x, v.y, h, l);
                const int rho = item_local * 16 + k1;
                unsigned char* tile = Abuf + (RT == 1 ? 0 : (rho >> 7)) * S::RTILE;
                kput32(tile, rho & 127, 2 * n2, h);
                kput32(tile, rho & 127, 2 * R + 2 * n2, l);
            }
        }
        cp_async_wait_all();  // this step's Phi row (requested a step earlier) has landed
        issue_right();
        if (!stage_wait()) return false;
        // (3) Z[k1][k2] (row r of each right tile, columns kb ..) -> phase shift -> right operand of
        // the inverse (conjugated), same rows
#pragma unroll
        for (int sg = 0; sg < RT; ++sg) {
            const float2* prow = phi_s(iwR[sg], j);
            unsigned char* tile = Abuf + sg * S::RTILE;
#pragma unroll
            for (int h0 = 0; h0 < RCOLS / RCH; ++h0) {
                float z[RCH];
                tc5_read<RCH, FP16>(tmem + lane_base + S::TM_R + sg * 4 * R + 2 * kb + h0 * RCH, 2 * R, z);
#pragma unroll
                for (int c = 0; c < RCH / 8; ++c) {  // chunk: 4 complex columns
                    const int k20 = kb + h0 * (RCH / 2) + 4 * c;
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 p = prow[k1R + 16 * (k20 + q)];
                        const float2 zz = make_float2(z[2 * (4 * c + q)], z[2 * (4 * c + q) + 1]);
                        const float2 v = conj_phi ? cmulc(zz, p) : cmul(zz, p);
                        SP::split(v.x, -v.y, h[q], l[q]);  // conjugated: the inverse runs on F_R
                    }
                    kput128(tile, r, 2 * k20, make_uint4(h[0], h[1], h[2], h[3]));
                    kput128(tile, r, 2 * R + 2 * k20, make_uint4(l[0], l[1], l[2], l[3]));
                }
            }
        }
        issue_right();
        if (phi_next >= 0) stage_rows(phi_next, 0);  // this step's Phi row has been read
        if (!stage_wait()) return false;
        // (4) the accumulator holds conj(Y2) for Y2 = Z conj(F_R) (rows (item, k1), columns n2); the
        // inverse left product takes conj(Y2 w^-(k1 n2)) = conj(Y2) w^(k1 n2), rows (item, n2), K = 2 k1 + q
#pragma unroll
        for (int sg = 0; sg < RT; ++sg) {
            const int item_local = (128 * sg + r) / 16;
#pragma unroll
            for (int h0 = 0; h0 < RCOLS / RCH; ++h0) {
                float y[RCH];
                tc5_read<RCH, FP16>(tmem + lane_base + S::TM_R + sg * 4 * R + 2 * kb + h0 * RCH, 2 * R, y);
#pragma unroll
                for (int q = 0; q < RCH / 2; ++q) {
                    const int nn = kb + h0 * (RCH / 2) + q;
                    const float2 v = cmul(make_float2(y[2 * q], y[2 * q + 1]), TWT[nn * 16 + k1R]);
                    uint32_t h, l;
                    SP::split(v.x, v.y, h, l);
                    const int rho = item_local * R + nn;
                    unsigned char* tile = Abuf + (LT == 1 ? 0 : (rho >> 7)) * S::LTILE;
                    kput32(tile, rho & 127, 2 * k1R, h);
                    kput32(tile, rho & 127, 32 + 2 * k1R, l);
                }
            }
        }
        issue_left();
        if (!stage_wait()) return false;
        // (5) x'[R n1 + n2] = conj(accumulator) of this thread's left rows back into the registers
#pragma unroll
        for (int i = 0; i < LTT; ++i) {
            float x[32];
            tc5_read<32, FP16>(tmem + lane_base + S::TM_L + (grp * LTT + i) * 64, 32, x);
            const float up = FP16 ? ldexpf(1.f, ex[i]) : 1.f;
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) u[i][n1] = make_float2(x[2 * n1] * up, -x[2 * n1 + 1] * up);
        }
        cp_async_wait_all();  // the rows staged during this step have landed
        umma::fence_before_sync();
        __syncthreads();  // TMEM reads done before the next MMAs; staged rows visible to every thread
        return true;
    };

    auto mul_d = [&](bool conj, int j) {
#pragma unroll
        for (int i = 0; i < LTT; ++i) {
            const float2* drow = dss_s(iwL[i], j);
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                const float2 dd = drow[R * n1 + n2];
                u[i][n1] = conj ? cmulc(u[i][n1], dd) : cmul(u[i][n1], dd);
            }
        }
    };

    if constexpr (MODE == MODE_SOURCE) {
        // step j (0 .. nz-2) propagates S_j to S_{j+1} with the rows of depth j
#pragma unroll
        for (int i = 0; i < LTT; ++i) {
            const int xs = okL[i] ? __ldg(a.src_ix + shotL[i]) : -1;
            const float2 w = okL[i] ? __ldg(a.wavelet + iwL[i]) : make_float2(0.f, 0.f);
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) u[i][n1] = (R * n1 + n2 == xs) ? w : make_float2(0.f, 0.f);
        }
        if (nz > 1) stage_rows(0, 0);
        cp_async_wait_all();
        __syncthreads();
        for (int jz = 0; jz < nz; ++jz) {
#pragma unroll
            for (int i = 0; i < LTT; ++i)
                if (okL[i]) {
                    float2* row = srow(i, jz);
#pragma unroll
                    for (int n1 = 0; n1 < 16; ++n1)
                        __stcs(row + R * n1 + n2, alive ? u[i][n1] : make_float2(NAN, NAN));
                }
            if (jz + 1 < nz && alive) {
                alive = transform_step(false, jz, jz, jz + 2 < nz ? jz + 1 : -1);
                mul_d(false, jz);
            }
        }
    } else if constexpr (MODE == MODE_ADJOINT) {
        // step j (0 .. nz-2): image term of depth j, then R_{j+1} = P_j^H R_j with the rows of depth j
        // (receivers at every column: the tensor-core variants take no receiver list)
#pragma unroll
        for (int i = 0; i < LTT; ++i) {
            const float2* drow = a.din + ((size_t)(shotL[i] - shot0) * a.nw + iwL[i]) * a.nrec;
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) u[i][n1] = okL[i] ? __ldcs(drow + R * n1 + n2) : make_float2(0.f, 0.f);
        }
        if (nz > 1) {
            stage_rows(0, 0);
            stage_rows(0, 1);
        }
        cp_async_wait_all();
        __syncthreads();
        float* part = a.part + (size_t)blockIdx.x * nz * N;
        // image row slot of this warp: four slots, each covering every column once
        const int islot = R == 64 ? warp >> 1 : warp;
        for (int jz = 0; jz < nz; ++jz) {
            float c[16];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) c[n1] = 0.f;
#pragma unroll
            for (int i = 0; i < LTT; ++i)
                if (okL[i]) {
                    const float2* row = srow(i, jz);
#pragma unroll
                    for (int n1 = 0; n1 < 16; ++n1) {
                        const float2 s = __ldcs(row + R * n1 + n2);
                        c[n1] += fmaf(s.x, u[i][n1].x, s.y * u[i][n1].y);
                    }
                }
            prefetch_srows(jz + 1);
            // below R = 32 a warp holds 32 / R items: lanes of equal n2 are summed first
#pragma unroll
            for (int off = R; off < 32; off <<= 1) {
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) c[n1] += __shfl_xor_sync(0xffffffffu, c[n1], off);
            }
            if (R >= 32 || lane < R) {
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) img[islot * N + R * n1 + n2] = alive ? c[n1] : NAN;
            }
            __syncthreads();
            {
                const float4* rows4 = reinterpret_cast<const float4*>(img);
                float4* prow = reinterpret_cast<float4*>(part + (size_t)jz * N);
                for (int x4 = tid; x4 < N / 4; x4 += S::THREADS) {
                    float4 acc = rows4[x4];
#pragma unroll
                    for (int w2 = 1; w2 < 4; ++w2) {
                        const float4 v4 = rows4[w2 * (N / 4) + x4];
                        acc.x += v4.x;
                        acc.y += v4.y;
                        acc.z += v4.z;
                        acc.w += v4.w;
                    }
                    prow[x4] = acc;
                }
            }
            __syncthreads();  // the image rows (in the operand buffer) are read before it is rewritten
            if (jz + 1 < nz && alive) {
                mul_d(true, jz);
                // the next step's D row is requested once this one has been applied
                alive = transform_step(true, jz, jz + 2 < nz ? jz + 1 : -1, jz + 2 < nz ? jz + 1 : -1);
            }
        }
    } else {  // MODE_FORWARD
        // U_j = P_j U_{j+1} + S_j m_j from the deepest row up; step k = nz-2-j uses the rows of depth j
#pragma unroll
        for (int i = 0; i < LTT; ++i)
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) u[i][n1] = make_float2(0.f, 0.f);
        if (nz > 1) stage_rows(nz - 2, 0);
        cp_async_wait_all();
        __syncthreads();
        for (int jz = nz - 1; jz >= 0; --jz) {
            prefetch_srows(jz);
            if (jz + 1 < nz && alive) {
                alive = transform_step(false, jz, jz, jz >= 1 ? jz - 1 : -1);
                mul_d(false, jz);
            }
            const float* mrow = a.m + (size_t)jz * N;
#pragma unroll
            for (int i = 0; i < LTT; ++i)
                if (okL[i]) {
                    const float2* row = srow(i, jz);
#pragma unroll
                    for (int n1 = 0; n1 < 16; ++n1) {
                        const float2 s = __ldcs(row + R * n1 + n2);
                        const float mm = __ldg(mrow + R * n1 + n2);
                        u[i][n1].x = fmaf(s.x, mm, u[i][n1].x);
                        u[i][n1].y = fmaf(s.y, mm, u[i][n1].y);
                    }
                }
        }
#pragma unroll
        for (int i = 0; i < LTT; ++i)
            if (okL[i]) {
                float2* orow = a.dout + ((size_t)(shotL[i] - shot0) * a.nw + iwL[i]) * a.nrec;
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) orow[R * n1 + n2] = alive ? u[i][n1] : make_float2(NAN, NAN);
            }
    }

    // ---- tear-down: a stage that ran out of time may still have MMAs in flight; wait for them
    // (bounded) before the columns are freed, and record the failure
    cp_async_wait_all();
    if (!alive) {
        if (tid == 0 && a.dev_err) atomicExch(a.dev_err, 1);
        umma::mbar_wait(&bar, phase);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, S::TM_COLS);
}

}  // namespace lsm
