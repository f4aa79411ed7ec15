"""The decomposition behind the library's own r2c transform, modelled on the
CPU and checked against numpy's FFT (no GPU):

* the radix schedules of the x / y passes (radix 8, radix 4 for blocks of 16,
  12 and 4, radix 3 for a block of 3) and of the z FFTs (also radix 4 for
  blocks of 32), with the
  decimation-in-frequency twiddles W_S^{nk} and the digit-reversed output
  positions the kernels write back in natural order;
* a real z row d read as N/2 complex values d[2n] + i d[2n+1], transformed
  along y, x and z, and split per pair of rows (kx, ky), (-kx, -ky) into the
  r2c transform: D[l] = (C[l] + conj C'[M-l]) / 2 - (i/2) W_N^l (C[l] - conj C'[M-l]);
* the enumeration of the N^2/2 + 2 row pairs, each row visited once.

The GPU tests (test_gpu_own_fft.py) check the kernels themselves."""
import numpy as np
import pytest


def radix_axis(S):
    return 3 if S == 3 else (4 if S in (4, 12, 16) else 8)


def radix_z(S):
    return 4 if S == 32 else radix_axis(S)


def dif_freq(S, mul, p, radix):
    if S == 1:
        return 0
    R = radix(S)
    Q = S // R
    return (p // Q) * mul + dif_freq(Q, mul * R, p % Q, radix)


def dif_fft(x, radix):
    """In-place radix-R decimation in frequency over blocks of S = L, L/R1, ...
    (the kernels' steps), then outputs read back from their digit-reversed
    positions."""
    L = len(x)
    buf = np.array(x, dtype=complex)
    S = L
    while True:
        R = radix(S)
        Q = S // R
        for beta in range(L // R):
            base = (beta // Q) * S + beta % Q
            n = beta % Q
            idx = base + Q * np.arange(R)
            V = np.fft.fft(buf[idx])                      # the R-point DFT of the step
            if Q > 1:
                V = V * np.exp(-2j * np.pi * n * np.arange(R) / S)   # W_S^{nk}
            buf[idx] = V
        if Q == 1:
            break
        S = Q
    out = np.empty(L, complex)
    for p in range(L):
        out[dif_freq(L, 1, p, radix)] = buf[p]
    return out


@pytest.mark.parametrize("L", [64, 128, 192, 256, 512, 1024, 2048])
def test_axis_schedule_is_the_dft(L):
    x = np.random.default_rng(L).standard_normal(L) + 1j * np.random.default_rng(L + 1).standard_normal(L)
    np.testing.assert_allclose(dif_fft(x, radix_axis), np.fft.fft(x), rtol=0, atol=1e-10 * np.sqrt(L))


@pytest.mark.parametrize("M", [64, 96, 128, 256, 512, 1024])
def test_z_schedule_is_the_dft(M):
    # also the row slots: position p at p ^ ((p >> 2) & 15), a bijection on
    # [0, M] below M + 16 (below M + 2 for powers of two)
    slots = [p ^ ((p >> 2) & 15) for p in range(M + 1)]
    assert len(set(slots)) == M + 1 and max(slots) < (M + 2 if (M & (M - 1)) == 0 else M + 16)
    x = np.random.default_rng(M).standard_normal(M) + 1j * np.random.default_rng(M + 7).standard_normal(M)
    np.testing.assert_allclose(dif_fft(x, radix_z), np.fft.fft(x), rtol=0, atol=1e-10 * np.sqrt(M))


def pair_rows(p, N):
    M = N // 2
    if p < (M - 1) * N:
        return 1 + p // N, p % N
    q = p - (M - 1) * N
    return (0, q) if q <= M else (M, q - (M + 1))


def split2(u, v, w):
    """2 D[l] from u = C[l], v = C'[M-l] and w = W_N^l."""
    return (u + np.conj(v)) - 1j * w * (u - np.conj(v))


@pytest.mark.parametrize("N", [8, 16, 24, 32])
def test_packed_rows_and_pair_split_give_rfftn(N):
    M = N // 2
    d = np.random.default_rng(N).standard_normal((N, N, N))
    c = d[:, :, 0::2] + 1j * d[:, :, 1::2]                       # z pairs as complex
    C = np.fft.fft(np.fft.fft(c, axis=1), axis=0)                 # the y pass, then the x pass
    W = np.exp(-2j * np.pi * np.arange(N) / N)
    D = np.zeros((N, N, M + 1), complex)
    seen = np.zeros((N, N), int)
    for p in range((M - 1) * N + 2 * (M + 1)):
        i, j = pair_rows(p, N)
        pi, pj = (N - i) % N, (N - j) % N
        A = dif_fft(C[i, j], radix_z) if M >= 4 else np.fft.fft(C[i, j])
        B = dif_fft(C[pi, pj], radix_z) if M >= 4 else np.fft.fft(C[pi, pj])
        for l in range(M + 1):
            la, lb = l % M, (M - l) % M
            D[i, j, l] = split2(A[la], B[lb], W[l]) / 2
            D[pi, pj, l] = split2(B[la], A[lb], W[l]) / 2
        seen[i, j] += 1
        if (pi, pj) != (i, j):
            seen[pi, pj] += 1
    assert (seen == 1).all()                                      # every row of the half grid once
    np.testing.assert_allclose(D, np.fft.rfftn(d), rtol=0, atol=1e-9 * N ** 1.5)
