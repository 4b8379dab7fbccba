// Lateral transforms as DFT-matrix products on the tensor cores (precision variants of the split-step
// depth step, Examples section).  For N = 16 R2 (R2 = 8, 16, ..., 64), one item's N points are the
// 16 x R2 matrix X[n1][n2] = u[R2 n1 + n2] and the forward DFT is the four-step product
//   Z = (F16 X . W) F_R2,  Z[k1][k2] = U[k1 + 16 k2],  W[k1][n2] = exp(-2 pi i k1 n2 / N),
// F_R the R-point DFT matrix; the inverse is X = conj(F16) ((Z conj(F_R2)) . conj(W)) (the 1/N
// sits in the phase-shift table).  Each product is a complex GEMM done as real mma.sync.m16n8k16
// products with FP32 accumulation, and every FP32 operand x is split as x = hi + lo in a 16-bit
// format:
//   PREC_BF16X3: hi = bf16(x), lo = bf16(x - hi); a b ~ ah bh + ah bl + al bh;
//   PREC_FP16X3: hi = fp16(x), lo = fp16((x - hi) 2^11); the two lo terms accumulate separately
//                and are scaled back by 2^-11 (keeps lo out of the fp16 subnormal range); each
//                item is block-scaled by a power of two per depth step (FP16's exponent range);
//   PREC_BF16X1: hi only (one product; shows the error of a plain bf16 transform).
// One warp holds one (shot, w) item for the whole depth loop, in the mma accumulator layout: lane
// (g = lane / 4, c = lane % 4) holds, for n-tile j and element e, row g + 8 (e / 2) and column
// 8 j + 2 c + (e % 2) of the 16 x R2 matrix.  Step-1 products read their data operand from a
// per-warp shared buffer; step-3 products take it straight from the previous accumulators.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lsm_fft.cuh"
#include "lsm_internal.h"

namespace lsm {

enum TcPrecision { PREC_FP32 = 0, PREC_BF16X3 = 1, PREC_FP16X3 = 2, PREC_BF16X1 = 3 };

template <int N>
struct TcShape {
    static_assert(N % 16 == 0 && N >= 16 && N <= 1024, "tensor-core transforms for nx = 16 R2 <= 1024");
    static constexpr int R2 = N / 16;
    static constexpr int NT = (R2 + 7) / 8;       // n-tiles (8 columns each)
    static constexpr bool PAD = R2 % 8 != 0;      // columns R2 .. 8 NT - 1 are zero padding
    static constexpr int KS = (R2 + 15) / 16;     // k-steps (16) of the right product
    static constexpr int LD = 8 * NT + 4;         // row stride of the per-warp buffer (see tc_phys)
    static constexpr int BUF = 16 * LD;           // float2 per warp
    // constant fragments: left A (F16) [6 variants][32 lanes][4 x b32]; right B (F_R2) [KS][NT][6][32][2]
    static constexpr int A_WORDS = 6 * 32 * 4;
    static constexpr int B_WORDS = KS * NT * 6 * 32 * 2;
};

// variants of a constant complex matrix: 0 re hi, 1 im hi, 2 -im hi, 3 re lo, 4 im lo, 5 -im lo
template <int PREC>
__device__ __forceinline__ void split_pack(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    if constexpr (PREC == PREC_FP16X3) {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn((x0 - hf.x) * 2048.f, (x1 - hf.y) * 2048.f);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (PREC == PREC_FP16X3) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// accumulators of one complex 16 x 8 tile; FP16X3 keeps a second set for the scaled lo terms
template <int PREC>
struct CTile {
    float re[4], im[4];
    float re2[4], im2[4];  // used by FP16X3 only
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int e = 0; e < 4; ++e) re[e] = im[e] = 0.f;
        if constexpr (PREC == PREC_FP16X3) {
#pragma unroll
            for (int e = 0; e < 4; ++e) re2[e] = im2[e] = 0.f;
        }
    }
    __device__ __forceinline__ float2 get(int e) const {
        if constexpr (PREC == PREC_FP16X3)
            return make_float2(fmaf(re2[e], 1.f / 2048.f, re[e]), fmaf(im2[e], 1.f / 2048.f, im[e]));
        else
            return make_float2(re[e], im[e]);
    }
};

// C += sum of two real products into each of C.re and C.im, as split fragments (index 0 hi, 1 lo):
//   C.re += A1 B1 + A2 B2,  C.im += A3 B3 + A4 B4,
// each real product as hi hi (+ hi lo + lo hi; for FP16X3 the cross terms go to re2/im2, which hold
// them scaled by 2^11).  A complex product takes (A1, B1, A2, B2, A3, B3, A4, B4) =
// (Ar, Br, -Ai, Bi, Ar, Bi, Ai, Br).
template <int PREC>
__device__ __forceinline__ void cross_terms(float (&cr)[4], float (&ci)[4], const uint32_t (&A1)[2][4],
                                            const uint32_t (&B1)[2][2], const uint32_t (&A2)[2][4],
                                            const uint32_t (&B2)[2][2], const uint32_t (&A3)[2][4],
                                            const uint32_t (&B3)[2][2], const uint32_t (&A4)[2][4],
                                            const uint32_t (&B4)[2][2]) {
    mma16816<PREC>(cr, A1[0], B1[1][0], B1[1][1]);
    mma16816<PREC>(cr, A2[0], B2[1][0], B2[1][1]);
    mma16816<PREC>(ci, A3[0], B3[1][0], B3[1][1]);
    mma16816<PREC>(ci, A4[0], B4[1][0], B4[1][1]);
    mma16816<PREC>(cr, A1[1], B1[0][0], B1[0][1]);
    mma16816<PREC>(cr, A2[1], B2[0][0], B2[0][1]);
    mma16816<PREC>(ci, A3[1], B3[0][0], B3[0][1]);
    mma16816<PREC>(ci, A4[1], B4[0][0], B4[0][1]);
}

template <int PREC>
__device__ __forceinline__ void cgemm4(CTile<PREC>& C, const uint32_t (&A1)[2][4], const uint32_t (&B1)[2][2],
                                       const uint32_t (&A2)[2][4], const uint32_t (&B2)[2][2],
                                       const uint32_t (&A3)[2][4], const uint32_t (&B3)[2][2],
                                       const uint32_t (&A4)[2][4], const uint32_t (&B4)[2][2]) {
    mma16816<PREC>(C.re, A1[0], B1[0][0], B1[0][1]);
    mma16816<PREC>(C.re, A2[0], B2[0][0], B2[0][1]);
    mma16816<PREC>(C.im, A3[0], B3[0][0], B3[0][1]);
    mma16816<PREC>(C.im, A4[0], B4[0][0], B4[0][1]);
    if constexpr (PREC == PREC_FP16X3) {
        cross_terms<PREC>(C.re2, C.im2, A1, B1, A2, B2, A3, B3, A4, B4);
    } else if constexpr (PREC == PREC_BF16X3) {
        cross_terms<PREC>(C.re, C.im, A1, B1, A2, B2, A3, B3, A4, B4);
    }
}

// Build the constant fragments of F16 (left operand A) and F_R2 (right operand B) in shared memory.
// conj variants are obtained by swapping the "im" and "-im" variants at use.
template <int N, int PREC>
__device__ void tc_build_constants(uint32_t* Afr, uint32_t* Bfr) {
    using S = TcShape<N>;
    // A: lane l, word w (elements 2w, 2w + 1): row g + 8 ((w) & 1), col 2 tig + 8 (w >> 1) + {0, 1}
    for (int idx = threadIdx.x; idx < 32 * 4; idx += blockDim.x) {
        const int l = idx >> 2, w = idx & 3;
        const int g = l >> 2, tig = l & 3;
        const int row = g + 8 * (w & 1);
        const int col = 2 * tig + 8 * (w >> 1);
        float re[2], im[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float sn, cs;
            sincospif(-2.0f * (float)((row * (col + q)) % 16) / 16.f, &sn, &cs);
            re[q] = cs;
            im[q] = sn;
        }
        uint32_t h, lo;
        split_pack<PREC>(re[0], re[1], h, lo);
        Afr[(0 * 32 + l) * 4 + w] = h;
        Afr[(3 * 32 + l) * 4 + w] = lo;
        split_pack<PREC>(im[0], im[1], h, lo);
        Afr[(1 * 32 + l) * 4 + w] = h;
        Afr[(4 * 32 + l) * 4 + w] = lo;
        split_pack<PREC>(-im[0], -im[1], h, lo);
        Afr[(2 * 32 + l) * 4 + w] = h;
        Afr[(5 * 32 + l) * 4 + w] = lo;
    }
    // B: (kk, jj), lane l, word w: k = 16 kk + 2 tig + 8 w + {0, 1}, n = 8 jj + g; zero beyond R2
    for (int idx = threadIdx.x; idx < S::KS * S::NT * 32 * 2; idx += blockDim.x) {
        const int w = idx & 1;
        const int l = (idx >> 1) & 31;
        const int tile = idx >> 6;  // kk * NT + jj
        const int kk = tile / S::NT, jj = tile % S::NT;
        const int g = l >> 2, tig = l & 3;
        const int n = 8 * jj + g;
        float re[2], im[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = 16 * kk + 2 * tig + 8 * w + q;
            if (k < S::R2 && n < S::R2) {  // zero rows and columns beyond R2 keep the padding zero
                float sn, cs;
                sincospif(-2.0f * (float)((k * n) % S::R2) / (float)S::R2, &sn, &cs);
                re[q] = cs;
                im[q] = sn;
            } else {
                re[q] = im[q] = 0.f;
            }
        }
        uint32_t h, lo;
        const int base = tile * 6 * 32 * 2;
        split_pack<PREC>(re[0], re[1], h, lo);
        Bfr[base + (0 * 32 + l) * 2 + w] = h;
        Bfr[base + (3 * 32 + l) * 2 + w] = lo;
        split_pack<PREC>(im[0], im[1], h, lo);
        Bfr[base + (1 * 32 + l) * 2 + w] = h;
        Bfr[base + (4 * 32 + l) * 2 + w] = lo;
        split_pack<PREC>(-im[0], -im[1], h, lo);
        Bfr[base + (2 * 32 + l) * 2 + w] = h;
        Bfr[base + (5 * 32 + l) * 2 + w] = lo;
    }
}

template <int N>
struct TcItem {
    float2 x[TcShape<N>::NT][4];  // the item, accumulator layout
};

// Position of matrix element (row, col) in the per-warp buffer: row stride LD = R2 + 4 and the
// column's low three bits XORed with s(row) = (row & 1) | (row & 4), found by exhaustive search over
// linear XOR maps so that both the accumulator-layout writes (rows g, columns 2 c) and the
// operand-layout reads (rows 2 c, columns g) of a half-warp touch 16 different 8-byte bank pairs.
// The XOR stays inside each group of 8 columns, so every element a lane touches is one of two
// per-lane bases plus a compile-time offset.
template <int N>
__device__ __forceinline__ int tc_phys(int row, int col) {
    return row * TcShape<N>::LD + (col ^ ((row & 1) | (row & 4)));
}

// left product: out = F16 . M (CONJ: conj(F16)), M read from the per-warp buffer (tc_phys layout)
template <int N, int PREC, bool CONJ>
__device__ __forceinline__ void tc_left(TcItem<N>& out, const float2* buf, const uint32_t* Afr, int lane) {
    using S = TcShape<N>;
    const int g = lane >> 2, tig = lane & 3;
    // operand element (row 2 tig + 8 w + q, column 8 j + g) = buf[lb_q + 8 w LD + 8 j]
    const int lb0 = tc_phys<N>(2 * tig, g), lb1 = tc_phys<N>(2 * tig + 1, g);
    uint32_t Ar[2][4], Ai[2][4], An[2][4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        Ar[0][w] = Afr[(0 * 32 + lane) * 4 + w];
        Ar[1][w] = Afr[(3 * 32 + lane) * 4 + w];
        Ai[0][w] = Afr[((CONJ ? 2 : 1) * 32 + lane) * 4 + w];
        Ai[1][w] = Afr[((CONJ ? 5 : 4) * 32 + lane) * 4 + w];
        An[0][w] = Afr[((CONJ ? 1 : 2) * 32 + lane) * 4 + w];
        An[1][w] = Afr[((CONJ ? 4 : 5) * 32 + lane) * 4 + w];
    }
#pragma unroll
    for (int j = 0; j < S::NT; ++j) {
        // B element (k = 2 tig + 8 w + q, n = 8 j + g) = M[k][8 j + g]
        uint32_t Br[2][2], Bi[2][2];
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            const float2 v0 = buf[lb0 + 8 * w * S::LD + 8 * j];
            const float2 v1 = buf[lb1 + 8 * w * S::LD + 8 * j];
            split_pack<PREC>(v0.x, v1.x, Br[0][w], Br[1][w]);
            split_pack<PREC>(v0.y, v1.y, Bi[0][w], Bi[1][w]);
        }
        CTile<PREC> C;
        C.zero();
        cgemm4<PREC>(C, Ar, Br, An, Bi, Ar, Bi, Ai, Br);
#pragma unroll
        for (int e = 0; e < 4; ++e) out.x[j][e] = C.get(e);
    }
}

// right product: out = M . F_R2 (CONJ: conj(F_R2)), M in accumulator layout (chained as operand A:
// A word w of k-step kk holds elements 2 (w % 2) + {0, 1} of accumulator tile 2 kk + w / 2).
template <int N, int PREC, bool CONJ>
__device__ __forceinline__ void tc_right(TcItem<N>& out, const TcItem<N>& in, const uint32_t* Bfr, int lane) {
    using S = TcShape<N>;
#pragma unroll
    for (int jj = 0; jj < S::NT; ++jj) {
        CTile<PREC> C;
        C.zero();
#pragma unroll
        for (int kk = 0; kk < S::KS; ++kk) {
            uint32_t Ar[2][4], Ai[2][4], An[2][4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int tile = 2 * kk + (w >> 1);
                const int e0 = 2 * (w & 1);
                float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
                if (tile < S::NT) {
                    v0 = in.x[tile < S::NT ? tile : 0][e0];
                    v1 = in.x[tile < S::NT ? tile : 0][e0 + 1];
                }
                split_pack<PREC>(v0.x, v1.x, Ar[0][w], Ar[1][w]);
                split_pack<PREC>(v0.y, v1.y, Ai[0][w], Ai[1][w]);
                split_pack<PREC>(-v0.y, -v1.y, An[0][w], An[1][w]);
            }
            const uint32_t* base = Bfr + (kk * S::NT + jj) * 6 * 32 * 2;
            uint32_t Br[2][2], Bi[2][2];
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                Br[0][w] = base[(0 * 32 + lane) * 2 + w];
                Br[1][w] = base[(3 * 32 + lane) * 2 + w];
                Bi[0][w] = base[((CONJ ? 2 : 1) * 32 + lane) * 2 + w];
                Bi[1][w] = base[((CONJ ? 5 : 4) * 32 + lane) * 2 + w];
            }
            cgemm4<PREC>(C, Ar, Br, An, Bi, Ar, Bi, Ai, Br);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) out.x[jj][e] = C.get(e);
    }
}

// write the item (accumulator layout, matrix rows x columns) to the per-warp buffer (tc_phys layout)
template <int N>
__device__ __forceinline__ void tc_store(const TcItem<N>& it, float2* buf, int lane) {
    using S = TcShape<N>;
    const int g = lane >> 2, tig = lane & 3;
    // accumulator element (row g + 8 h, column 8 j + 2 tig + e0) = buf[sb_e0 + 8 h LD + 8 j]
    const int sb0 = tc_phys<N>(g, 2 * tig), sb1 = tc_phys<N>(g, 2 * tig + 1);
#pragma unroll
    for (int j = 0; j < S::NT; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) buf[((e & 1) ? sb1 : sb0) + 8 * (e >> 1) * S::LD + 8 * j] = it.x[j][e];
}

// whether element (j, e) of a lane is a real column of the 16 x R2 matrix (not zero padding)
template <int N>
__device__ __forceinline__ bool tc_valid(int lane, int j, int e) {
    return !TcShape<N>::PAD || 8 * j + 2 * (lane & 3) + (e & 1) < TcShape<N>::R2;
}
// column index (natural position for the matrix rows n1, columns n2) of element (j, e); real
// columns only
template <int N>
__device__ __forceinline__ int tc_xpos(int lane, int j, int e) {
    const int g = lane >> 2, tig = lane & 3;
    return TcShape<N>::R2 * (g + 8 * (e >> 1)) + 8 * j + 2 * tig + (e & 1);
}
// frequency index of element (j, e) of Z (rows k1, columns k2)
template <int N>
__device__ __forceinline__ int tc_kpos(int lane, int j, int e) {
    const int g = lane >> 2, tig = lane & 3;
    return (g + 8 * (e >> 1)) + 16 * (8 * j + 2 * tig + (e & 1));
}

// u <- F^-1 (phi . F u) with phi (already divided by N, natural frequency order) or conj(phi)
template <int N, int PREC, bool CONJ_PHI>
__device__ __forceinline__ void tc_phase_step(TcItem<N>& u, float2* buf, const uint32_t* Afr, const uint32_t* Bfr,
                                              const float2* tws, const float2* __restrict__ phi, int lane) {
    using S = TcShape<N>;
    // FP16 has a 5-bit exponent: the item is brought to a largest component in [1/2, 1) by an exact
    // power-of-two scale before the split and scaled back after the step (the products are linear),
    // so wavefields of any magnitude stay inside the FP16 normal range at every stage (at most
    // 16 R2 after the two forward factors).  BF16 keeps the FP32 exponent range and needs no scale.
    int ex = 0;
    if constexpr (PREC == PREC_FP16X3) {
        float mx = 0.f;
#pragma unroll
        for (int j = 0; j < S::NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fmaxf(fabsf(u.x[j][e].x), fabsf(u.x[j][e].y)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (mx > 0.f && mx <= 3.0e38f) frexpf(mx, &ex);
        ex = max(-100, min(ex, 100));  // both 2^ex and 2^-ex stay normal FP32 numbers
        const float down = ldexpf(1.f, -ex);
#pragma unroll
        for (int j = 0; j < S::NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) u.x[j][e] = make_float2(u.x[j][e].x * down, u.x[j][e].y * down);
    }
    TcItem<N> y;
    __syncwarp();
    tc_store<N>(u, buf, lane);
    __syncwarp();
    tc_left<N, PREC, false>(y, buf, Afr, lane);
#pragma unroll
    for (int j = 0; j < S::NT; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) y.x[j][e] = cmul(y.x[j][e], tws[(j * 4 + e) * 32 + lane]);
    TcItem<N> z;
    tc_right<N, PREC, false>(z, y, Bfr, lane);
#pragma unroll
    for (int j = 0; j < S::NT; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 p = tc_valid<N>(lane, j, e) ? __ldg(phi + tc_kpos<N>(lane, j, e)) : make_float2(0.f, 0.f);
            z.x[j][e] = CONJ_PHI ? cmulc(z.x[j][e], p) : cmul(z.x[j][e], p);
        }
    tc_right<N, PREC, true>(y, z, Bfr, lane);
#pragma unroll
    for (int j = 0; j < S::NT; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) y.x[j][e] = cmulc(y.x[j][e], tws[(j * 4 + e) * 32 + lane]);
    __syncwarp();
    tc_store<N>(y, buf, lane);
    __syncwarp();
    tc_left<N, PREC, true>(u, buf, Afr, lane);
    if constexpr (PREC == PREC_FP16X3) {
        const float up = ldexpf(1.f, ex);
#pragma unroll
        for (int j = 0; j < S::NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) u.x[j][e] = make_float2(u.x[j][e].x * up, u.x[j][e].y * up);
    }
}

template <int N>
constexpr size_t tc_smem_bytes(int warps, bool adjoint) {
    using S = TcShape<N>;
    return (size_t)(S::A_WORDS + S::B_WORDS) * 4 + (size_t)S::NT * 4 * 32 * sizeof(float2) +
           (size_t)warps * S::BUF * sizeof(float2) + (adjoint ? (size_t)2 * warps * N * sizeof(float) : 0);
}

// Depth sweeps with the tensor-core transforms; same modes, inputs and outputs as sweep_kernel,
// one item per warp, coefficients read straight from the tables (Phi in natural frequency order).
template <int N, int PREC, int MODE>
// Up to 7 warps per block and two blocks per SM (at most 146 registers a thread): the 2,048 items of a
// 512-wide window of 16 shots x 128 frequencies then run in a single wave on 152 SMs.  Above N = 512
// an item takes more registers and one block per SM leaves a thread up to 255.
__global__ void __launch_bounds__(224, N > 512 ? 1 : 2) tc_sweep_kernel(const SweepArgs a) {
    using S = TcShape<N>;
    constexpr int NT = S::NT;
    extern __shared__ float4 smem_f4[];
    uint32_t* Afr = reinterpret_cast<uint32_t*>(smem_f4);
    uint32_t* Bfr = Afr + S::A_WORDS;
    float2* tws = reinterpret_cast<float2*>(Bfr + S::B_WORDS);  // twiddles W, [element][lane]
    float2* bufs = tws + NT * 4 * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float* img = reinterpret_cast<float*>(bufs + nwarps * S::BUF);  // [2][nwarps][N]
    float2* buf = bufs + warp * S::BUF;
    const int nitems = a.nshots * a.nw;
    const int item = blockIdx.x * nwarps + warp;
    const bool ok = item < nitems;
    const int iw = ok ? item / a.nshots : 0;
    const int ishot = ok ? item - iw * a.nshots : 0;
    const int shot = (a.shot0_dev ? __ldg(a.shot0_dev) : a.shot0) + ishot;
    const int slot = shot % a.ring;
    const int nz = a.nz;

    tc_build_constants<N, PREC>(Afr, Bfr);
    // W[k1][n2] for element (j, e) of lane l: k1 = g + 8 (e / 2), n2 = 8 j + 2 c + (e % 2)
    for (int idx = threadIdx.x; idx < NT * 4 * 32; idx += blockDim.x) {
        const int l = idx & 31, je = idx >> 5, j = je >> 2, e = je & 3;
        const int k1 = (l >> 2) + 8 * (e >> 1), n2 = 8 * j + 2 * (l & 3) + (e & 1);
        float sn, cs;
        sincospif(-2.0f * (float)((k1 * n2) % N) / (float)N, &sn, &cs);
        tws[idx] = make_float2(cs, sn);
    }
    __syncthreads();

    const float2* phi_w = a.phi + (size_t)iw * nz * N;
    const float2* dss_w = a.dss + (size_t)iw * nz * N;
    float2* Sitem = a.S + ((size_t)slot * a.nw + iw) * (size_t)nz * N;
    TcItem<N> u;

    auto load_nat = [&](TcItem<N>& v, const float2* row) {
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                v.x[j][e] = ok && tc_valid<N>(lane, j, e) ? __ldcs(row + tc_xpos<N>(lane, j, e))
                                                          : make_float2(0.f, 0.f);
    };
    auto mul_d = [&](TcItem<N>& v, const float2* drow, bool conj) {
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (tc_valid<N>(lane, j, e)) {
                    const float2 dd = __ldg(drow + tc_xpos<N>(lane, j, e));
                    v.x[j][e] = conj ? cmulc(v.x[j][e], dd) : cmul(v.x[j][e], dd);
                }
            }
    };

    if constexpr (MODE == MODE_SOURCE) {
        const int xs = ok ? __ldg(a.src_ix + shot) : -1;
        const float2 w = ok ? __ldg(a.wavelet + iw) : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                u.x[j][e] = tc_valid<N>(lane, j, e) && tc_xpos<N>(lane, j, e) == xs ? w : make_float2(0.f, 0.f);
        for (int jz = 0; jz < nz; ++jz) {
            if (ok) {
                float2* row = Sitem + (size_t)jz * N;
#pragma unroll
                for (int j = 0; j < NT; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (tc_valid<N>(lane, j, e)) __stcs(row + tc_xpos<N>(lane, j, e), u.x[j][e]);
            }
            if (jz + 1 < nz) {
                tc_phase_step<N, PREC, false>(u, buf, Afr, Bfr, tws, phi_w + (size_t)jz * N, lane);
                mul_d(u, dss_w + (size_t)jz * N, false);
            }
        }
    } else if constexpr (MODE == MODE_ADJOINT) {
        // receivers at every column (the tensor-core variant takes no receiver list)
        load_nat(u, a.din + ((size_t)ishot * a.nw + iw) * a.nrec);
        float* part = a.part + (size_t)blockIdx.x * nz * N;
        for (int jz = 0; jz < nz; ++jz) {
            TcItem<N> s;
            load_nat(s, Sitem + (size_t)jz * N);
            float* slab = img + ((size_t)(jz & 1) * nwarps + warp) * N;
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (tc_valid<N>(lane, j, e))
                        slab[tc_xpos<N>(lane, j, e)] = fmaf(s.x[j][e].x, u.x[j][e].x, s.x[j][e].y * u.x[j][e].y);
            __syncthreads();
            {
                // the block's partial row: the warps' rows summed in warp order, four columns a thread
                const float4* rows = reinterpret_cast<const float4*>(img + (size_t)(jz & 1) * nwarps * N);
                float4* prow = reinterpret_cast<float4*>(part + (size_t)jz * N);
                for (int x4 = threadIdx.x; x4 < N / 4; x4 += blockDim.x) {
                    float4 acc = rows[x4];
                    for (int w2 = 1; w2 < nwarps; ++w2) {
                        const float4 u4 = rows[w2 * (N / 4) + x4];
                        acc.x += u4.x; acc.y += u4.y; acc.z += u4.z; acc.w += u4.w;
                    }
                    prow[x4] = acc;
                }
            }
            if (jz + 1 < nz) {
                mul_d(u, dss_w + (size_t)jz * N, true);
                tc_phase_step<N, PREC, true>(u, buf, Afr, Bfr, tws, phi_w + (size_t)jz * N, lane);
            }
        }
    } else {  // MODE_FORWARD
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) u.x[j][e] = make_float2(0.f, 0.f);
        for (int jz = nz - 1; jz >= 0; --jz) {
            if (jz + 1 < nz) {
                tc_phase_step<N, PREC, false>(u, buf, Afr, Bfr, tws, phi_w + (size_t)jz * N, lane);
                mul_d(u, dss_w + (size_t)jz * N, false);
            }
            TcItem<N> s;
            load_nat(s, Sitem + (size_t)jz * N);
            const float* mrow = a.m + (size_t)jz * N;
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float mm = tc_valid<N>(lane, j, e) ? __ldg(mrow + tc_xpos<N>(lane, j, e)) : 0.f;
                    u.x[j][e].x = fmaf(s.x[j][e].x, mm, u.x[j][e].x);
                    u.x[j][e].y = fmaf(s.x[j][e].y, mm, u.x[j][e].y);
                }
        }
        if (ok) {
            float2* orow = a.dout + ((size_t)ishot * a.nw + iw) * a.nrec;
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (tc_valid<N>(lane, j, e)) orow[tc_xpos<N>(lane, j, e)] = u.x[j][e];
        }
    }
}

}  // namespace lsm
