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
// Radix-2 decimation-in-frequency passes (natural in, bit-reversed out) followed by a
// compile-time renaming to natural order.  INV selects the +i sign (unnormalised inverse).

// The sum and difference use the paired-FP32 instructions of sm_100-class GPUs (one instruction
// for both components); a - b is formed exactly as fma(b, -1, a).
template <bool INV, int H, int K>
__device__ __forceinline__ void r2_butterfly(float2* v) {
    const float2 a = v[K], b = v[K + H];
    v[K] = __fadd2_rn(a, b);
    v[K + H] = twiddle_const<2 * H, K, INV>(__ffma2_rn(b, make_float2(-1.f, -1.f), a));
}

template <int R, bool INV, int H, int... Ks>
__device__ __forceinline__ void r2_pass(float2* v, std::integer_sequence<int, Ks...>) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * H) {
        (r2_butterfly<INV, H, Ks>(v + blk), ...);
    }
}

template <int R, bool INV, int H>
__device__ __forceinline__ void r2_passes(float2* v) {
    r2_pass<R, INV, H>(v, std::make_integer_sequence<int, H>{});
    if constexpr (H > 1) r2_passes<R, INV, H / 2>(v);
}

constexpr int bit_reverse(int k, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) {
        r = (r << 1) | (k & 1);
        k >>= 1;
    }
    return r;
}

template <int R, bool INV>
__device__ __forceinline__ void small_dft(float2* v) {
    if constexpr (R > 1) {
        r2_passes<R, INV, R / 2>(v);
        float2 t[R];
#pragma unroll
        for (int k = 0; k < R; ++k) t[k] = v[bit_reverse(k, R)];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = t[k];
    }
}

// ------------------------------------------------------------------ stage plan
// Stage s works on blocks of length L(s) = N / (R(0)...R(s-1)); each block is split into R(s)
// interleaved sub-sequences of length M(s) = L(s) / R(s).  Butterfly beta = t + T i (i < NB(s))
// takes block b = beta / M, offset n1 = beta % M, inputs b L + n1 + M n2 (n2 < R), and writes
// output k2, twiddled by exp(-2 pi i n1 k2 / L), to position b L + k2 M + n1.  Radices are
// greedy: R(s) = min(V, L(s)).  After the last stage (M = 1) thread t's register
// r = i R_last + k2 holds position (t + T i) R_last + k2; the position's mixed-radix digits,
// read in reverse, give the frequency index.

template <int N, int V>
struct Plan {
    static_assert((N & (N - 1)) == 0 && (V & (V - 1)) == 0, "powers of two");
    static_assert(N >= V && V >= 2, "V points per thread");
    static constexpr int T = N / V;
    static_assert(T <= 32, "one transform per warp at most");
    static constexpr int L(int s) {
        int len = N;
        for (int i = 0; i < s; ++i) len /= (len < V ? len : V);
        return len;
    }
    static constexpr int R(int s) { return L(s) < V ? L(s) : V; }
    static constexpr int M(int s) { return L(s) / R(s); }
    static constexpr int NB(int s) { return V / R(s); }
    static constexpr int count_stages() {
        int s = 0;
        while (L(s) > 1) ++s;
        return s;
    }
    static constexpr int NS = count_stages();
    static constexpr int RLAST = R(NS - 1);
    // registers of precomputed twiddles: stages with M > 1
    static constexpr int tw_offset(int s) {
        int off = 0;
        for (int i = 0; i < s; ++i)
            if (M(i) > 1) off += NB(i) * (R(i) - 1);
        return off;
    }
    static constexpr int NTW = tw_offset(NS) > 0 ? tw_offset(NS) : 1;
    // padded shared-memory index: one float2 of padding every 16 removes bank conflicts of the
    // strided stage exchanges
    static __device__ __forceinline__ int phys(int a) { return a + (a >> 4); }
    static constexpr int BUF = N + N / 16;
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

template <int N, int V>
struct Twiddles {
    float2 w[Plan<N, V>::NTW];
};

template <int N, int V>
__device__ __forceinline__ void init_twiddles(Twiddles<N, V>& tw, int t) {
    using P = Plan<N, V>;
#pragma unroll
    for (int s = 0; s < P::NS; ++s) {
        if (P::M(s) > 1) {
#pragma unroll
            for (int i = 0; i < P::NB(s); ++i) {
                const int beta = t + P::T * i;
                const int n1 = beta % P::M(s);
#pragma unroll
                for (int k2 = 1; k2 < P::R(s); ++k2) {
                    const int e = (n1 * k2) % P::L(s);
                    float sn, cs;
                    sincospif(-2.0f * (float)e / (float)P::L(s), &sn, &cs);
                    tw.w[P::tw_offset(s) + i * (P::R(s) - 1) + (k2 - 1)] = make_float2(cs, sn);
                }
            }
        }
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
                v[i * R + k2] = cmul(v[i * R + k2], tw.w[P::tw_offset(S) + i * (R - 1) + (k2 - 1)]);
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
                v[i * R + k2] = cmulc(v[i * R + k2], tw.w[P::tw_offset(S) + i * (R - 1) + (k2 - 1)]);
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
// first stage in registers, then, per last-stage butterfly (a runtime loop, so its code exists
// once), forward last stage -> multiply by phi (or conj(phi)) -> inverse last stage in place in
// the exchange buffer, then the inverse first stage in registers.  Equivalent to fft_forward, a
// pointwise multiply in the digit-reversed register order, and fft_inverse; the smaller code
// footprint keeps more of the depth loop in the instruction cache.  phi is indexed like the
// register layout: phi[r * T + t] multiplies register r of thread t.
template <int N, int V, bool CONJ>
__device__ __forceinline__ void phase_shift_two_stage(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t,
                                                      const float2* phi) {
    using P = Plan<N, V>;
    static_assert(P::NS == 2, "two-stage plans only");
    constexpr int R0 = P::R(0), R1 = P::R(1), M1 = P::M(1), L1 = P::L(1), T = P::T;
    static_assert(M1 == 1 && R0 == V, "one first-stage butterfly per thread, unit-stride last stage");
    small_dft<R0, false>(v);
#pragma unroll
    for (int k2 = 1; k2 < R0; ++k2) v[k2] = cmul(v[k2], tw.w[P::tw_offset(0) + (k2 - 1)]);
    __syncwarp();
    store_outputs<N, V, 0>(v, buf, t);
    __syncwarp();
#pragma unroll 1
    for (int i = 0; i < P::NB(1); ++i) {
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
    }
    __syncwarp();
    load_outputs<N, V, 0>(v, buf, t);
#pragma unroll
    for (int k2 = 1; k2 < R0; ++k2) v[k2] = cmulc(v[k2], tw.w[P::tw_offset(0) + (k2 - 1)]);
    small_dft<R0, true>(v);
}

}  // namespace lsm
