"""The exact Gram matrix kernel of the isometry-centre move (tcgen05 tensor
cores, bf16 digit products with exact FP32 sums and 64-bit integer
accumulation) against its definition computed here with integer arithmetic.

Definition: X = M as a real m x 2n matrix (Re, Im interleaved); column c is
rounded to the integer N_c = rint(X_c 2^(23 - E_c)), max |X_c| < 2^E_c; the
integer Gram matrix N^T N is converted to double and scaled back by
2^(E_a + E_b - 46); Re G_ij = Xhat_2i.Xhat_2j + Xhat_2i+1.Xhat_2j+1,
Im G_ij = Xhat_2i.Xhat_2j+1 - Xhat_2i+1.Xhat_2j.  The kernel must reproduce
this bit for bit (the same integers, the same final roundings), and stay
within 2^-22 (relative to max |G|) of the plain complex128 M^H M."""
import numpy as np
import pytest

import paper_2511_05719_gb300 as P

torch = pytest.importorskip("torch")


def reference(M):
    m, n = M.shape
    X = np.empty((m, 2 * n), dtype=np.float32)
    X[:, 0::2] = M.real
    X[:, 1::2] = M.imag
    amax = np.max(np.abs(X), axis=0)
    E = np.zeros(2 * n, dtype=np.int64)
    nz = amax > 0
    E[nz] = np.frexp(amax[nz])[1]
    N = np.rint(np.ldexp(X.astype(np.float64), (23 - E)[None, :])).astype(np.int64)
    GX = N.T @ N                                   # exact: |N| <= 2^23, m <= 2^16 rows
    scale = np.ldexp(1.0, (E[:, None] + E[None, :] - 46))
    F = GX.astype(np.float64) * scale
    xx, yy = F[0::2, 0::2], F[1::2, 1::2]
    xy, yx = F[0::2, 1::2], F[1::2, 0::2]
    return (xx + yy) + 1j * (xy - yx)


def sample(m, n, seed, zero_col=False, spread=6.0):
    rng = np.random.default_rng(seed)
    col_scale = 10.0 ** rng.uniform(-spread, 0, size=n)
    M = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) * col_scale[None, :]
    M[rng.random((m, n)) < 0.1] *= 1e-4            # mixed magnitudes inside a column
    if zero_col:
        M[:, n // 2] = 0
    return M.astype(np.complex64)


@pytest.mark.gpu
@pytest.mark.parametrize("m,n", [(1, 1), (37, 5), (300, 64), (1000, 100), (5000, 256), (4200, 130),
                                 (64, 512), (20000, 32)])
def test_gram_exact_bitwise(m, n):
    M = sample(m, n, 1000 * m + n, zero_col=n > 2)
    G = P.gram_exact(torch.from_numpy(M).cuda()).cpu().numpy()
    want = reference(M)
    assert np.array_equal(G.view(np.float64), want.view(np.float64))
    plain = M.astype(np.complex128).conj().T @ M.astype(np.complex128)
    assert np.max(np.abs(G - plain)) <= 2.0 ** -22 * np.max(np.abs(plain))


@pytest.mark.gpu
def test_gram_exact_two_calls_and_hermitian():
    M1, M2 = sample(777, 48, 1), sample(3000, 200, 2)
    for M in (M1, M2, M1):
        G = P.gram_exact(torch.from_numpy(M).cuda()).cpu().numpy()
        assert np.array_equal(G, G.conj().T)
        assert np.array_equal(G.view(np.float64), reference(M).view(np.float64))


def test_reference_pins_the_definition():
    """The integer reference equals the plain complex128 Gram matrix when
    every entry already fits 23 bits below its column maximum."""
    rng = np.random.default_rng(7)
    ints = rng.integers(-2 ** 20, 2 ** 20, size=(50, 6)) + 1j * rng.integers(-2 ** 20, 2 ** 20, size=(50, 6))
    M = (ints * 2.0 ** -30).astype(np.complex64)
    plain = M.astype(np.complex128).conj().T @ M.astype(np.complex128)
    assert np.allclose(reference(M), plain, rtol=0, atol=1e-15 * np.max(np.abs(plain)))
