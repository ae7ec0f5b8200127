"""The sine-transform identities the CUDA kernels rely on, checked in numpy against the
DST-I matrix itself (no GPU; independent of the oracle, whose sine transforms are
scipy's).

For x_1..x_{N-1} (complex), X_k = sum_j x_j sin(pi j k / N):
* half length: with y_j = sin(pi j/N)(x_j + x_{N-j}) + (x_j - x_{N-j})/2 (x_0 = x_N = 0)
  and Y = FFT_N(y):  X_{2q} = (i/2)(Y_q - Y_{N-q}),
  X_{2q+1} = Y_0/2 + sum_{p=1..q} (Y_p + Y_{N-p})/2;
* odd extension: Y = FFT_{2N}(0, x_1..x_{N-1}, 0, -x_{N-1}..-x_1) gives X_k = (i/2) Y_k.
The kernels take the odd-output prefix sum in chunks per thread plus a pass over the
chunk totals; the chunked form is checked too.
"""
import numpy as np
import pytest


def _dst1(x):
    N = x.shape[-1] + 1
    j = np.arange(1, N)
    return x @ np.sin(np.pi * np.outer(j, j) / N)


def _half_length(x, chunks=1):
    N = x.shape[-1] + 1
    xf = np.zeros(x.shape[:-1] + (N + 1,), dtype=complex)
    xf[..., 1:N] = x
    j = np.arange(N)
    y = np.sin(np.pi * j / N) * (xf[..., j] + xf[..., N - j]) + 0.5 * (xf[..., j] - xf[..., N - j])
    Y = np.fft.fft(y)
    q = np.arange(N // 2)
    Ym = Y[..., (N - q) % N]
    even = 0.5j * (Y[..., q] - Ym)            # X_{2q}, q >= 1
    R = 0.5 * (Y[..., q] + Ym)
    R[..., 0] *= 0.5                           # Y_0 / 2
    # prefix sum in `chunks` contiguous chunks, then the chunk totals
    parts = np.split(R, chunks, axis=-1)
    local = [np.cumsum(p, axis=-1) for p in parts]
    offs = np.cumsum([np.zeros(R.shape[:-1])] + [l[..., -1] for l in local[:-1]], axis=0)
    odd = np.concatenate([l + o[..., None] for l, o in zip(local, offs)], axis=-1)
    X = np.zeros(x.shape[:-1] + (N,), dtype=complex)
    X[..., 2 * q[1:]] = even[..., 1:]
    X[..., 2 * q + 1] = odd
    return X[..., 1:]


def _odd_extension(x):
    N = x.shape[-1] + 1
    y = np.zeros(x.shape[:-1] + (2 * N,), dtype=complex)
    y[..., 1:N] = x
    y[..., N + 1:] = -x[..., ::-1]
    return 0.5j * np.fft.fft(y)[..., 1:N]


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128, 256, 512])
def test_half_length_dst_equals_the_matrix_product(N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((3, N - 1)) + 1j * rng.standard_normal((3, N - 1))
    ref = _dst1(x)
    for chunks in (1, 2, min(N // 2, 16)):
        got = _half_length(x, chunks)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), chunks


@pytest.mark.parametrize("N", [2, 4, 8, 64])
def test_odd_extension_dst_equals_the_matrix_product(N):
    rng = np.random.default_rng(N + 1)
    x = rng.standard_normal((2, N - 1)) + 1j * rng.standard_normal((2, N - 1))
    ref = _dst1(x)
    assert np.abs(_odd_extension(x) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_orthonormal_dst_is_its_own_inverse():
    N = 32
    x = np.random.default_rng(7).standard_normal(N - 1) + 0j
    s = np.sqrt(2.0 / N)
    assert np.abs(s * _half_length(s * _half_length(x)) - x).max() <= 1e-13
