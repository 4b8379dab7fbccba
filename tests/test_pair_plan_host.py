"""Host check of the pair plan's index maps (the second FFT tile at nx = 512, 16 points per lane,
one warp per transform), before and beside its GPU parity tests.

The lane-level steps of the device transform are replayed in numpy with the same index maps:
lane t = p + 16 h holds x = t + 32 r; each lane's 16-point DFT; the radix-2 step across lanes t and
t ^ 16 (lane h producing outputs k = j + 8h and k + 16 of column p's 32-point DFT); the stage
twiddle exp(-2 pi i p k2 / 512); the store to position 16 k2 + p; the lane's 16-point block DFT.  The
result must be numpy's FFT at frequency k2 + 32 k1 of position 16 k2 + k1, and the inverse steps must
return the input (times 512).
"""

import numpy as np

N, T, V = 512, 32, 16


def xpos(t, r):
    return t + T * r


def k2_of(t, i):
    return (i & 7) + 8 * (t >> 4) + 16 * (i >> 3)


def freq_of_position(pos):
    return (pos // 16) % 32 + 32 * (pos % 16)


def position_of(t, r):
    return 16 * t + r


def dft(v, inv=False):
    n = len(v)
    k = np.arange(n)
    sign = 1.0 if inv else -1.0
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n) @ v


def forward_pair(u):
    regs = np.array([[u[xpos(t, r)] for r in range(V)] for t in range(T)])
    regs = np.array([dft(regs[t]) for t in range(T)])           # h = 0: E[k], h = 1: O[k]
    out = np.zeros_like(regs)
    w = np.exp(-2j * np.pi / 32)
    for t in range(T):
        h, partner = t >> 4, t ^ 16
        for j in range(8):
            keep, give = regs[t, j], regs[t, j + 8]
            recv = regs[partner, j] if h == 0 else regs[partner, j + 8]   # the partner's send
            e = recv if h else keep
            o = give if h else recv
            tw = o * w ** (j + 8 * h)
            out[t, j], out[t, j + 8] = e + tw, e - tw
    buf = np.zeros(N, dtype=complex)
    for t in range(T):
        p = t & 15
        for i in range(V):
            buf[16 * k2_of(t, i) + p] = out[t, i] * np.exp(-2j * np.pi * p * k2_of(t, i) / N)
    blocks = np.array([dft(buf[16 * t:16 * t + 16]) for t in range(T)])  # register r = k1 of lane t
    return blocks


def inverse_pair(blocks):
    buf = np.zeros(N, dtype=complex)
    for t in range(T):
        buf[16 * t:16 * t + 16] = dft(blocks[t], inv=True)
    regs = np.zeros((T, V), dtype=complex)
    for t in range(T):
        p = t & 15
        for i in range(V):
            regs[t, i] = buf[16 * k2_of(t, i) + p] * np.exp(2j * np.pi * p * k2_of(t, i) / N)
    wc = np.exp(2j * np.pi / 32)
    e_o = np.zeros_like(regs)
    for t in range(T):
        h = t >> 4
        for j in range(8):
            lo, hi = regs[t, j], regs[t, j + 8]
            e_o[t, j], e_o[t, j + 8] = lo + hi, (lo - hi) * wc ** (j + 8 * h)   # (e, o) of k = j + 8h
    v = np.zeros_like(regs)
    for t in range(T):
        h, partner = t >> 4, t ^ 16
        for j in range(8):
            e, o = e_o[t, j], e_o[t, j + 8]
            pe, po = e_o[partner, j], e_o[partner, j + 8]
            recv = po if h else pe          # the partner sends e (h = 1) or o (h = 0): lane 0 gets e[j + 8], lane 1 o[j]
            v[t, j] = recv if h else e
            v[t, j + 8] = o if h else recv
    v = np.array([dft(v[t], inv=True) for t in range(T)])
    u = np.zeros(N, dtype=complex)
    for t in range(T):
        for r in range(V):
            u[xpos(t, r)] = v[t, r]
    return u


def test_index_maps_cover_every_point_once():
    assert sorted(xpos(t, r) for t in range(T) for r in range(V)) == list(range(N))
    assert sorted(16 * k2_of(t, i) + (t & 15) for t in range(T) for i in range(V)) == list(range(N))
    assert sorted(freq_of_position(position_of(t, r)) for t in range(T) for r in range(V)) == list(range(N))


def test_forward_matches_numpy_fft_in_digit_order():
    rng = np.random.default_rng(3)
    u = rng.normal(size=N) + 1j * rng.normal(size=N)
    blocks = forward_pair(u)
    ref = np.fft.fft(u)
    got = np.zeros(N, dtype=complex)
    for t in range(T):
        for r in range(V):
            got[freq_of_position(position_of(t, r))] = blocks[t, r]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_inverse_undoes_forward():
    rng = np.random.default_rng(4)
    u = rng.normal(size=N) + 1j * rng.normal(size=N)
    back = inverse_pair(forward_pair(u)) / N
    np.testing.assert_allclose(back, u, rtol=0, atol=1e-10 * np.abs(u).max())
