// Register-resident lateral FFT for the split-step depth step (Examples section: shot-profile
// split-step Fourier operator).  One transform of N complex points is held by T = N / V threads,
// V points per thread.  The forward transform is a decimation-in-frequency mixed-radix FFT whose
// output stays in digit-reversed order; the inverse runs the same stages backwards with
// conjugated twiddles, takes that order as input and returns natural order.  So one depth step
// F^-1 (Phi . F u) needs no reordering pass, and the inverse's output layout (thread t holds
// x = t + T r, r < V) is the forward's input layout, so consecutive depth steps chain in
// registers.  Stages exchange data through a padded shared-memory buffer per transform.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace lsm {

// ------------------------------------------------------------------ complex helpers

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// ------------------------------------------------------------------ compile-time trigonometry
// cos / sin of 2 pi num / den for the butterfly constants, from their Taylor series evaluated
// in double at compile time (argument reduced to [-pi, pi]; 20 terms leave < 1e-16 error).

constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double series_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 20; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double series_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 20; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
constexpr double turn_angle(int num, int den) {
    int k = ((num % den) + den) % den;
    if (2 * k > den) k -= den;
    return 2.0 * kPi * k / den;
}

// v * exp(-2 pi i K / L) (forward) or v * exp(+2 pi i K / L) (inverse)
template <int L, int K, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v) {
    constexpr int k = ((K % L) + L) % L;
    if constexpr (k == 0) {
        return v;
    } else if constexpr (2 * k == L) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * k == L) {  // forward: * (-i)
        return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else if constexpr (4 * k == 3 * L) {  // forward: * (+i)
        return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    } else {
        constexpr float c = (float)series_cos(turn_angle(k, L));
        constexpr float s = INV ? (float)series_sin(turn_angle(k, L)) : -(float)series_sin(turn_angle(k, L));
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

// ------------------------------------------------------------------ in-register radix-R DFT
// In natural order in and out; INV selects the +i sign (unnormalised inverse).

// Odd prime R (3, 5, 7): direct DFT using the symmetry of its constants.  With a_n = x_n + x_{R-n}
// and b_n = x_n - x_{R-n} (n = 1 .. (R-1)/2), re_k = x_0 + sum a_n cos(2 pi n k / R) and
// im_k = sum b_n sin(2 pi n k / R); the forward DFT is y_k = re_k - i im_k, y_{R-k} = re_k + i im_k
// (the inverse swaps the two).
template <int R, int K, int NN>
struct OddConst {
    static constexpr float c = (float)series_cos(turn_angle(NN * K, R));
    static constexpr float s = (float)series_sin(turn_angle(NN * K, R));
};

template <int R, bool INV, int K, int... Ns>
__device__ __forceinline__ void odd_output(float2* y, float2 x0, const float2* a, const float2* b,
                                           std::integer_sequence<int, Ns...>) {
    float2 re = x0, im = make_float2(0.f, 0.f);
    ((re.x = fmaf(a[Ns + 1].x, OddConst<R, K, Ns + 1>::c, re.x),
      re.y = fmaf(a[Ns + 1].y, OddConst<R, K, Ns + 1>::c, re.y),
      im.x = fmaf(b[Ns + 1].x, OddConst<R, K, Ns + 1>::s, im.x),
      im.y = fmaf(b[Ns + 1].y, OddConst<R, K, Ns + 1>::s, im.y)), ...);
    const float2 mi = make_float2(im.y, -im.x);  // -i * im
    y[K] = INV ? csub(re, mi) : cadd(re, mi);
    y[R - K] = INV ? cadd(re, mi) : csub(re, mi);
}

template <int R, bool INV, int... Ks>
__device__ __forceinline__ void odd_dft(float2* v, std::integer_sequence<int, Ks...>) {
    constexpr int H = (R - 1) / 2;
    float2 a[H + 1], b[H + 1], y[R];
    float2 y0 = v[0];
#pragma unroll
    for (int n = 1; n <= H; ++n) {
        a[n] = cadd(v[n], v[R - n]);
        b[n] = csub(v[n], v[R - n]);
        y0 = cadd(y0, a[n]);
    }
    y[0] = y0;
    (odd_output<R, INV, Ks + 1>(y, v[0], a, b, std::make_integer_sequence<int, H>{}), ...);
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = y[k];
}

// Power-of-two R: split-radix decimation in time (Yavne's split of the radix-2 and radix-4 steps, in
// the form of Duhamel and Hollmann).  The DFT X of L points is assembled from E, the DFT of the even
// points, and O1, O3, the DFTs of the points 1 and 3 mod 4: with a = W^k O1[k], b = W^3k O3[k]
// (W = exp(-2 pi i / L), conjugated for the inverse) and k < L/4,
//   X[k] = E[k] + (a + b),          X[k + L/2] = E[k] - (a + b),
//   X[k + L/4] = E[k + L/4] - i (a - b),   X[k + 3L/4] = E[k + L/4] + i (a - b)   (+i / -i for the
// inverse).  Against radix-2 passes it needs fewer non-trivial twiddles (26 instead of 34 for 32
// points, 8 instead of 10 for 16) at the same number of additions.  All indices are compile-time, so
// the recursion unrolls into straight-line code over registers, with the output in natural order.
// Sums and differences use the paired FP32 instructions of sm_100-class GPUs (one instruction for
// both components); a - b is formed exactly as fma(b, -1, a).
template <int L, bool INV, int K>
__device__ __forceinline__ void sr_combine(const float2* e, const float2* o1, const float2* o3, float2* out) {
    const float2 a = twiddle_const<L, K, INV>(o1[K]);
    const float2 b = twiddle_const<L, 3 * K, INV>(o3[K]);
    const float2 s = __fadd2_rn(a, b);
    const float2 d = __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b
    const float2 jd = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);  // +i d / -i d
    out[K] = __fadd2_rn(e[K], s);
    out[K + L / 2] = __ffma2_rn(s, make_float2(-1.f, -1.f), e[K]);
    out[K + L / 4] = __fadd2_rn(e[K + L / 4], jd);
    out[K + 3 * L / 4] = __ffma2_rn(jd, make_float2(-1.f, -1.f), e[K + L / 4]);
}

template <int L, bool INV, int... Ks>
__device__ __forceinline__ void sr_combine_all(const float2* e, const float2* o1, const float2* o3, float2* out,
                                               std::integer_sequence<int, Ks...>) {
    (sr_combine<L, INV, Ks>(e, o1, o3, out), ...);
}

// DFT of the L points v[OFF + STRIDE n] (n < L) into out[0 .. L), natural order
template <int L, int OFF, int STRIDE, bool INV>
__device__ __forceinline__ void sr_dft(const float2* v, float2* out) {
    if constexpr (L == 1) {
        out[0] = v[OFF];
    } else if constexpr (L == 2) {
        out[0] = __fadd2_rn(v[OFF], v[OFF + STRIDE]);
        out[1] = __ffma2_rn(v[OFF + STRIDE], make_float2(-1.f, -1.f), v[OFF]);
    } else {
        float2 e[L / 2], o1[L / 4], o3[L / 4];
        sr_dft<L / 2, OFF, 2 * STRIDE, INV>(v, e);
        sr_dft<L / 4, OFF + STRIDE, 4 * STRIDE, INV>(v, o1);
        sr_dft<L / 4, OFF + 3 * STRIDE, 4 * STRIDE, INV>(v, o3);
        sr_combine_all<L, INV>(e, o1, o3, out, std::make_integer_sequence<int, L / 4>{});
    }
}

template <int R, bool INV>
__device__ __forceinline__ void small_dft(float2* v) {
    if constexpr (R == 3 || R == 5 || R == 7) {
        odd_dft<R, INV>(v, std::make_integer_sequence<int, (R - 1) / 2>{});
    } else if constexpr (R > 1) {
        static_assert((R & (R - 1)) == 0, "power-of-two or odd prime radix");
        float2 t[R];
        sr_dft<R, 0, 1, INV>(v, t);
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = t[k];
    }
}

// ------------------------------------------------------------------ stage plan
// Stage s works on blocks of length L(s) = N / (R(0)...R(s-1)); each block is split into R(s)
// interleaved sub-sequences of length M(s) = L(s) / R(s).  Butterfly beta = t + T i (i < NB(s))
// takes block b = beta / M, offset n1 = beta % M, inputs b L + n1 + M n2 (n2 < R), and writes
// output k2, twiddled by exp(-2 pi i n1 k2 / L), to position b L + k2 M + n1.  Radices: for a
// power-of-two N, R(s) = min(V, L(s)); for N = q 2^a with q in {3, 5, 7}, the first stage has
// radix q and the others min(power-of-two part of V, L(s)).  Every radix divides V.  So thread t
// holds input x = t + T (r / R0) + M0 (r % R0) in register r (x = t + T r when R0 = V), and after
// the last stage (M = 1) register r = i R_last + k2 holds position (t + T i) R_last + k2; the
// position's mixed-radix digits, read in reverse, give the frequency index.

constexpr int odd_part(int n) {
    while (n > 1 && n % 2 == 0) n /= 2;
    return n;
}

template <int N, int V>
struct Plan {
    static constexpr int Q = odd_part(N);
    static_assert(Q == 1 || Q == 3 || Q == 5 || Q == 7, "N = 2^a times 1, 3, 5 or 7");
    static_assert(N % V == 0 && V % Q == 0 && V / Q >= 2 && V >= 2, "V points per thread");
    static constexpr int T = N / V;
    static_assert(T <= 32 && (T & (T - 1)) == 0, "a power-of-two number of threads, one warp at most");
    static constexpr int VP2 = V / odd_part(V);  // power-of-two part of V
    static constexpr int R(int s) {
        int len = N;
        for (int i = 0; i < s; ++i) len /= R(i);
        if (s == 0) return Q > 1 ? Q : (len < V ? len : V);
        return len < VP2 ? len : VP2;
    }
    static constexpr int L(int s) {
        int len = N;
        for (int i = 0; i < s; ++i) len /= R(i);
        return len;
    }
    static constexpr int M(int s) { return L(s) / R(s); }
    static constexpr int NB(int s) { return V / R(s); }
    static constexpr int count_stages() {
        int s = 0;
        while (L(s) > 1) ++s;
        return s;
    }
    static constexpr int NS = count_stages();
    static constexpr int RLAST = R(NS - 1);
    static constexpr int R0 = R(0);
    static constexpr int M0 = M(0);
    // twiddles live in registers for power-of-two plans and in a shared table otherwise
    static constexpr bool TW_SMEM = Q > 1;
    static constexpr int tw_offset(int s) {
        int off = 0;
        for (int i = 0; i < s; ++i)
            if (M(i) > 1) off += NB(i) * (R(i) - 1);
        return off;
    }
    static constexpr int NTW = (!TW_SMEM && tw_offset(NS) > 0) ? tw_offset(NS) : 1;
    // shared twiddle table: exp(-2 pi i e / L(s)) for e < L(s), per stage with M(s) > 1
    static constexpr int tab_offset(int s) {
        int off = 0;
        for (int i = 0; i < s; ++i)
            if (M(i) > 1) off += L(i);
        return off;
    }
    static constexpr int TAB = TW_SMEM ? tab_offset(NS) : 0;
    // padded shared-memory index: one float2 of padding every 16 removes bank conflicts of the
    // strided stage exchanges
    static __device__ __forceinline__ int phys(int a) { return a + (a >> 4); }
    static constexpr int BUF = N + N / 16;
    // natural-order column held in register r of thread t
    static __host__ __device__ constexpr int xpos(int t, int r) { return t + T * (r / R0) + M0 * (r % R0); }
    // frequency index held at final position pos
    static __host__ __device__ constexpr int freq_of_position(int pos) {
        int k = 0, weight = 1;
        for (int s = 0; s < NS; ++s) {
            const int digit = (pos / M(s)) % R(s);
            k += digit * weight;
            weight *= R(s);
        }
        return k;
    }
    // final position of register r of thread t
    static __host__ __device__ constexpr int position_of(int t, int r) {
        return (t + T * (r / RLAST)) * RLAST + (r % RLAST);
    }
};

// Pair plan: N = 512 at V = 16 points per thread, T = 32 threads (one warp) per transform.  It has
// the stages of the 32-point plan, 512 = 32 x 16, but the two lanes t and t ^ 16 share each 32-point
// first-stage DFT: with p = t mod 16 and h = t / 16, lane t holds x = p + 16 (2 r + h) = t + 32 r,
// the even (h = 0) or odd (h = 1) points of column p's 32-point DFT, runs the 16-point DFT of its
// half, and the lanes exchange half their outputs with one shuffle per value for the final radix-2
// step, X[k] = E[k] + w^k O[k] and X[k + 16] = E[k] - w^k O[k] (w = exp(-2 pi i / 32)): lane h
// produces k in [8h, 8h + 8) and k + 16.  Twice the threads per transform of the 32-point plan
// without a third stage, so a window of few items fills twice the warps per SM.
template <int N, int V>
constexpr bool pair_plan() { return N == 512 && V == 16; }

template <>
struct Plan<512, 16> {
    static constexpr int N = 512, V = 16, Q = 1, T = 32, VP2 = 16;
    static constexpr int R(int s) { return s == 0 ? 32 : 16; }
    static constexpr int L(int s) { return s == 0 ? 512 : 16; }
    static constexpr int M(int s) { return s == 0 ? 16 : 1; }
    static constexpr int NB(int) { return 1; }
    static constexpr int NS = 2, RLAST = 16, R0 = 32, M0 = 16;
    static constexpr bool TW_SMEM = false;
    static constexpr int NTW = 16, TAB = 0;
    static __device__ __forceinline__ int phys(int a) { return a + (a >> 4); }
    static constexpr int BUF = N + N / 16;
    static __host__ __device__ constexpr int xpos(int t, int r) { return t + T * r; }
    // first-stage output (32-point DFT index k2) held in register i of lane t after the exchange
    static __host__ __device__ constexpr int k2_of(int t, int i) { return (i & 7) + 8 * (t >> 4) + 16 * (i >> 3); }
    // position 16 k2 + k1 holds frequency k2 + 32 k1
    static __host__ __device__ constexpr int freq_of_position(int pos) { return (pos / 16) % 32 + 32 * (pos % 16); }
    // lane t holds the last-stage block of positions 16 t .. 16 t + 15 (register r = k1)
    static __host__ __device__ constexpr int position_of(int t, int r) { return 16 * t + r; }
};

template <int N, int V>
struct Twiddles {
    using P = Plan<N, V>;
    float2 w[P::NTW];
    const float2* table;  // shared table (TW_SMEM plans)
    int t;
    // twiddle exp(-2 pi i n1 k2 / L(S)) of butterfly i of this thread, k2 >= 1 (plan quantities are
    // bound to constexpr locals so that register indices fold at compile time)
    template <int S>
    __device__ __forceinline__ float2 at(int i, int k2) const {
        constexpr int M = P::M(S), L = P::L(S), R = P::R(S);
        if constexpr (P::TW_SMEM) {
            constexpr int TOFF = P::tab_offset(S);
            const int n1 = (t + P::T * i) % M;
            return table[TOFF + (n1 * k2) % L];
        } else {
            constexpr int OFF = P::tw_offset(S);
            return w[OFF + i * (R - 1) + (k2 - 1)];
        }
    }
};

template <int N, int V, int S>
__device__ __forceinline__ void init_twiddles_stage(Twiddles<N, V>& tw, int t, float2* table) {
    using P = Plan<N, V>;
    constexpr int M = P::M(S), L = P::L(S), R = P::R(S), NB = P::NB(S);
    if constexpr (M > 1) {
        if constexpr (P::TW_SMEM) {
            constexpr int TOFF = P::tab_offset(S);
            for (int e = threadIdx.x; e < L; e += blockDim.x) {
                float sn, cs;
                sincospif(-2.0f * (float)e / (float)L, &sn, &cs);
                table[TOFF + e] = make_float2(cs, sn);
            }
        } else {
            constexpr int OFF = P::tw_offset(S);
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int n1 = (t + P::T * i) % M;
#pragma unroll
                for (int k2 = 1; k2 < R; ++k2) {
                    const int e = (n1 * k2) % L;
                    float sn, cs;
                    sincospif(-2.0f * (float)e / (float)L, &sn, &cs);
                    tw.w[OFF + i * (R - 1) + (k2 - 1)] = make_float2(cs, sn);
                }
            }
        }
    }
    if constexpr (S + 1 < P::NS) init_twiddles_stage<N, V, S + 1>(tw, t, table);
}

// Registers: every thread computes its own twiddles.  Shared table (mixed-radix plans): the whole
// block fills it, so every thread must call this and the block must synchronise before first use.
template <int N, int V>
__device__ __forceinline__ void init_twiddles(Twiddles<N, V>& tw, int t, float2* table = nullptr) {
    tw.t = t;
    tw.table = table;
    if constexpr (pair_plan<N, V>()) {
        // first-stage twiddle exp(-2 pi i p k2 / 512) of each output register
        const int p = t & 15;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = (p * Plan<N, V>::k2_of(t, i)) % 512;
            float sn, cs;
            sincospif(-2.0f * (float)e / 512.0f, &sn, &cs);
            tw.w[i] = make_float2(cs, sn);
        }
    } else {
        init_twiddles_stage<N, V, 0>(tw, t, table);
    }
}

// ------------------------------------------------------------------ exchanges

template <int N, int V, int S>
__device__ __forceinline__ void store_outputs(const float2 (&v)[V], float2* buf, int t) {
    using P = Plan<N, V>;
    constexpr int R = P::R(S), L = P::L(S), M = P::M(S);
#pragma unroll
    for (int i = 0; i < P::NB(S); ++i) {
        const int beta = t + P::T * i;
        const int base = (beta / M) * L + (beta % M);
#pragma unroll
        for (int k2 = 0; k2 < R; ++k2) buf[P::phys(base + k2 * M)] = v[i * R + k2];
    }
}

template <int N, int V, int S>
__device__ __forceinline__ void load_outputs(float2 (&v)[V], const float2* buf, int t) {
    using P = Plan<N, V>;
    constexpr int R = P::R(S), L = P::L(S), M = P::M(S);
#pragma unroll
    for (int i = 0; i < P::NB(S); ++i) {
        const int beta = t + P::T * i;
        const int base = (beta / M) * L + (beta % M);
#pragma unroll
        for (int k2 = 0; k2 < R; ++k2) v[i * R + k2] = buf[P::phys(base + k2 * M)];
    }
}

// input positions of stage S are the output positions of stage S-1 with a different grouping
template <int N, int V, int S>
__device__ __forceinline__ void load_inputs(float2 (&v)[V], const float2* buf, int t) {
    using P = Plan<N, V>;
    constexpr int R = P::R(S), L = P::L(S), M = P::M(S);
#pragma unroll
    for (int i = 0; i < P::NB(S); ++i) {
        const int beta = t + P::T * i;
        const int base = (beta / M) * L + (beta % M);
#pragma unroll
        for (int n2 = 0; n2 < R; ++n2) v[i * R + n2] = buf[P::phys(base + n2 * M)];
    }
}

template <int N, int V, int S>
__device__ __forceinline__ void store_inputs(const float2 (&v)[V], float2* buf, int t) {
    using P = Plan<N, V>;
    constexpr int R = P::R(S), L = P::L(S), M = P::M(S);
#pragma unroll
    for (int i = 0; i < P::NB(S); ++i) {
        const int beta = t + P::T * i;
        const int base = (beta / M) * L + (beta % M);
#pragma unroll
        for (int n2 = 0; n2 < R; ++n2) buf[P::phys(base + n2 * M)] = v[i * R + n2];
    }
}

// ------------------------------------------------------------------ transforms

template <int N, int V, int S>
__device__ __forceinline__ void forward_stages(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t) {
    using P = Plan<N, V>;
    constexpr int R = P::R(S);
#pragma unroll
    for (int i = 0; i < P::NB(S); ++i) {
        small_dft<R, false>(&v[i * R]);
        if constexpr (P::M(S) > 1) {
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2)
                v[i * R + k2] = cmul(v[i * R + k2], tw.template at<S>(i, k2));
        }
    }
    if constexpr (S + 1 < P::NS) {
        __syncwarp();
        store_outputs<N, V, S>(v, buf, t);
        __syncwarp();
        load_inputs<N, V, S + 1>(v, buf, t);
        forward_stages<N, V, S + 1>(v, tw, buf, t);
    }
}

template <int N, int V, int S>
__device__ __forceinline__ void inverse_stages(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t) {
    using P = Plan<N, V>;
    constexpr int R = P::R(S);
#pragma unroll
    for (int i = 0; i < P::NB(S); ++i) {
        if constexpr (P::M(S) > 1) {
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2)
                v[i * R + k2] = cmulc(v[i * R + k2], tw.template at<S>(i, k2));
        }
        small_dft<R, true>(&v[i * R]);
    }
    if constexpr (S > 0) {
        __syncwarp();
        store_inputs<N, V, S>(v, buf, t);
        __syncwarp();
        load_outputs<N, V, S - 1>(v, buf, t);
        inverse_stages<N, V, S - 1>(v, tw, buf, t);
    }
}

// Unnormalised forward DFT; natural layout in (x = t + T r), digit-reversed layout out.
template <int N, int V>
__device__ __forceinline__ void fft_forward(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t) {
    forward_stages<N, V, 0>(v, tw, buf, t);
}

// Unnormalised inverse DFT; digit-reversed layout in, natural layout out.
template <int N, int V>
__device__ __forceinline__ void fft_inverse(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t) {
    inverse_stages<N, V, Plan<N, V>::NS - 1>(v, tw, buf, t);
}

// One phase-shift step in the transform domain for two-stage plans, F^-1 (phi . F v): forward
// first stage in registers, then, per last-stage butterfly, forward last stage -> multiply by phi
// (or conj(phi)) -> inverse last stage in place in the exchange buffer, then the inverse first stage
// in registers.  Equivalent to fft_forward, a pointwise multiply in the digit-reversed register
// order, and fft_inverse.  phi is indexed like the register layout: phi[r * T + t] multiplies
// register r of thread t.  UNROLL runs a thread's last-stage butterflies side by side (more
// independent work while its own registers are parked in shared memory; source and forward sweeps
// at nx = 512: 0.87 -> 0.83 and 0.83 -> 0.80 ms); without it they run as a runtime loop whose code
// exists once, which the adjoint sweep, holding the next source-wavefield row in registers as well,
// measured faster (0.855 against 0.866 ms).  mid() runs once the first stage's outputs are stored.
template <int N, int V, bool CONJ, bool UNROLL, class Mid>
__device__ __forceinline__ void phase_shift_two_stage(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t,
                                                      const float2* phi, Mid&& mid) {
    using P = Plan<N, V>;
    static_assert(P::NS == 2, "two-stage plans only");
    constexpr int R0 = P::R(0), R1 = P::R(1), M1 = P::M(1), L1 = P::L(1), T = P::T;
    static_assert(M1 == 1 && R0 == V, "one first-stage butterfly per thread, unit-stride last stage");
    small_dft<R0, false>(v);
#pragma unroll
    for (int k2 = 1; k2 < R0; ++k2) v[k2] = cmul(v[k2], tw.template at<0>(0, k2));
    __syncwarp();
    store_outputs<N, V, 0>(v, buf, t);
    __syncwarp();
    mid();  // the caller's work for while the thread's registers are parked (e.g. loads to issue)
    auto last_stage_block = [&](int i) {
        float2* blk = buf + (t + T * i) * L1;  // last-stage block, unit stride
        const int a0 = (t + T * i) * L1;
        float2 u[R1];
#pragma unroll
        for (int n2 = 0; n2 < R1; ++n2) u[n2] = blk[P::phys(a0 + n2) - a0];
        small_dft<R1, false>(u);
#pragma unroll
        for (int k2 = 0; k2 < R1; ++k2) {
            const float2 ph = phi[(i * R1 + k2) * T + t];
            u[k2] = CONJ ? cmulc(u[k2], ph) : cmul(u[k2], ph);
        }
        small_dft<R1, true>(u);
#pragma unroll
        for (int n2 = 0; n2 < R1; ++n2) blk[P::phys(a0 + n2) - a0] = u[n2];
    };
    if constexpr (UNROLL) {
#pragma unroll
        for (int i = 0; i < P::NB(1); ++i) last_stage_block(i);
    } else {
#pragma unroll 1
        for (int i = 0; i < P::NB(1); ++i) last_stage_block(i);
    }
    __syncwarp();
    load_outputs<N, V, 0>(v, buf, t);
#pragma unroll
    for (int k2 = 1; k2 < R0; ++k2) v[k2] = cmulc(v[k2], tw.template at<0>(0, k2));
    small_dft<R0, true>(v);
}


// ------------------------------------------------------------------ pair plan step

// w^J (forward, w = exp(-2 pi i / 32)) or its conjugate, and the same times w^8 = -i (or +i)
template <int J, bool INV>
struct PairConst {
    static constexpr float c = (float)series_cos(turn_angle(J, 32));
    static constexpr float s = INV ? (float)series_sin(turn_angle(J, 32)) : -(float)series_sin(turn_angle(J, 32));
    // w^(J + 8) = w^J * (-i) forward, conj: * (+i)
    static constexpr float c8 = INV ? -s : s;
    static constexpr float s8 = INV ? c : -c;
};

__device__ __forceinline__ float2 shfl_pair(float2 v) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 16), __shfl_xor_sync(0xffffffffu, v.y, 16));
}

// final radix-2 step of the forward 32-point DFT for output pair J: in, lane h holds E (h = 0) or
// O (h = 1) at registers J and J + 8; out, register J holds X[J + 8h] and register J + 8 holds
// X[J + 8h + 16]
template <int J>
__device__ __forceinline__ void pair_forward_radix2(float2 (&v)[16], bool h) {
    const float2 keep = v[J], give = v[J + 8];
    const float2 recv = shfl_pair(h ? keep : give);  // lane 0 gets O[J], lane 1 gets E[J + 8]
    const float2 e = h ? recv : keep;                // E[J + 8h]
    const float2 o = h ? give : recv;                // O[J + 8h]
    using C = PairConst<J, false>;
    const float2 w = h ? make_float2(C::c8, C::s8) : make_float2(C::c, C::s);
    const float2 tw = cmul(o, w);
    v[J] = __fadd2_rn(e, tw);
    v[J + 8] = __ffma2_rn(tw, make_float2(-1.f, -1.f), e);
}

// first radix-2 step of the inverse 32-point DFT for pair J (the forward step undone): in, registers
// J and J + 8 hold Y[J + 8h] and Y[J + 8h + 16]; out, lane 0 holds e[k] = Y[k] + Y[k + 16] and lane 1
// o[k] = (Y[k] - Y[k + 16]) conj(w)^k at registers J (k = J) and J + 8 (k = J + 8)
template <int J>
__device__ __forceinline__ void pair_inverse_radix2(float2 (&v)[16], bool h) {
    const float2 lo = v[J], hi = v[J + 8];
    const float2 e = __fadd2_rn(lo, hi);
    using C = PairConst<J, true>;
    const float2 w = h ? make_float2(C::c8, C::s8) : make_float2(C::c, C::s);
    const float2 o = cmul(__ffma2_rn(hi, make_float2(-1.f, -1.f), lo), w);
    const float2 recv = shfl_pair(h ? e : o);  // lane 0 gets e[J + 8], lane 1 gets o[J]
    v[J] = h ? recv : e;
    v[J + 8] = h ? o : recv;
}

template <int... Js>
__device__ __forceinline__ void pair_forward_radix2_all(float2 (&v)[16], bool h, std::integer_sequence<int, Js...>) {
    (pair_forward_radix2<Js>(v, h), ...);
}
template <int... Js>
__device__ __forceinline__ void pair_inverse_radix2_all(float2 (&v)[16], bool h, std::integer_sequence<int, Js...>) {
    (pair_inverse_radix2<Js>(v, h), ...);
}

// One phase-shift step F^-1 (phi . F v) of the pair plan (N = 512, 16 points per thread): the
// forward first stage (16-point DFT, radix-2 exchange across the lane pair, twiddles) into the
// exchange buffer, mid(), then the lane's last-stage block (positions 16 t .. 16 t + 15: 16-point
// DFT, phi or conj(phi), inverse 16-point DFT) in place, then the inverse first stage back into the
// natural layout.  phi[r * 32 + t] multiplies register r of lane t's block.
template <bool CONJ, class Mid>
__device__ __forceinline__ void phase_shift_pair(float2 (&v)[16], const Twiddles<512, 16>& tw, float2* buf, int t,
                                                 const float2* phi, Mid&& mid) {
    using P = Plan<512, 16>;
    const bool h = t >= 16;
    const int p = t & 15;
    small_dft<16, false>(v);
    pair_forward_radix2_all(v, h, std::make_integer_sequence<int, 8>{});
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = cmul(v[i], tw.w[i]);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) buf[P::phys(16 * P::k2_of(t, i) + p)] = v[i];
    __syncwarp();
    mid();
    {
        float2 u[16];
        const int a0 = 16 * t;
#pragma unroll
        for (int n = 0; n < 16; ++n) u[n] = buf[P::phys(a0 + n)];
        small_dft<16, false>(u);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float2 ph = phi[k * 32 + t];
            u[k] = CONJ ? cmulc(u[k], ph) : cmul(u[k], ph);
        }
        small_dft<16, true>(u);
#pragma unroll
        for (int n = 0; n < 16; ++n) buf[P::phys(a0 + n)] = u[n];
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = cmulc(buf[P::phys(16 * P::k2_of(t, i) + p)], tw.w[i]);
    pair_inverse_radix2_all(v, h, std::make_integer_sequence<int, 8>{});
    small_dft<16, true>(v);
}

}  // namespace lsm
