"""The split-BF16 arithmetic of the tensor-core far field (reading c23), emulated on the CPU:
BF16 round-to-nearest-even of float32 values (8 significant bits: error <= 2^-8 of the
magnitude), the hi + lo split (error <= 2^-16), and a 2-D DFT evaluated as
three-term split products (hi*hi + lo*hi + hi*lo) against the FP64 transform. These pin the
representation bound and the error level that the GPU tolerance (1e-3) is derived from."""
import numpy as np


def bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = bf16(x)
    lo = bf16(x - hi)
    return hi, lo


def test_bf16_rounding_is_nearest_even():
    # values exactly representable stay put; halfway cases go to the even neighbour
    assert bf16(np.float32(1.0)) == 1.0
    one_ulp = np.float32(2.0 ** -7)                       # bf16 spacing at 1
    assert bf16(np.float32(1.0) + one_ulp / 2) == 1.0     # tie -> even (1.0)
    assert bf16(np.float32(1.0) + 3 * one_ulp / 2) == np.float32(1.0) + 2 * one_ulp
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32)
    # 8 significant bits: the rounding error is at most 2^-8 of the magnitude
    assert np.all(np.abs(bf16(x) - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-7))


def test_hi_lo_split_represents_to_two_to_minus_16():
    x = (np.random.default_rng(1).standard_normal(20000) * 10.0 ** np.random.default_rng(2).uniform(-6, 6, 20000)
         ).astype(np.float32)
    hi, lo = split(x)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(x) * (1 + 1e-6))
    assert np.sqrt(np.mean((err / np.abs(x)) ** 2)) < 2.0 ** -17   # typical error well inside the bound


def _dft_split(X, inverse=False):
    """F X F^T with F = exp(-+2 pi i m c / N), every real product as the three split terms."""
    N = X.shape[0]
    m = np.arange(N)
    ang = 2 * np.pi * ((np.outer(m, m) % N) / N)
    Fr, Fi = np.cos(ang), (np.sin(ang) if inverse else -np.sin(ang))
    Frh, Frl = split(Fr)
    Fih, Fil = split(Fi)

    def prod(Ah, Al, B):
        Bh, Bl = split(B)
        f = lambda a, b: a.astype(np.float64) @ b.astype(np.float64)
        return f(Ah, Bh) + f(Al, Bh) + f(Ah, Bl)

    def pass_(Zr, Zi):   # D = F Z^T (rows of Z contracted), as the kernel's passes
        Dr = prod(Frh, Frl, Zr.T) - prod(Fih, Fil, Zi.T)
        Di = prod(Frh, Frl, Zi.T) + prod(Fih, Fil, Zr.T)
        return Dr.astype(np.float32), Di.astype(np.float32)

    D1r, D1i = pass_(X.real.astype(np.float32), X.imag.astype(np.float32))
    D2r, D2i = pass_(D1r, D1i)
    return D2r.astype(np.float64) + 1j * D2i.astype(np.float64)


def test_split_dft_matches_fp64_transform_to_about_1e_5():
    rng = np.random.default_rng(3)
    for N in (32, 64, 128):
        X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
        ref = np.fft.fft2(X.astype(np.complex128))
        got = _dft_split(X)
        e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert e < 2e-5, (N, e)
        # the inverse direction (conjugate matrix) as well
        back = _dft_split(ref.astype(np.complex64), inverse=True) / (N * N)
        assert np.linalg.norm(back - X) / np.linalg.norm(X) < 2e-5


def test_dropping_a_split_term_is_visible():
    # with only hi*hi the transform is off by about the BF16 rounding (1e-3): the three terms matter
    rng = np.random.default_rng(4)
    N = 64
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    m = np.arange(N)
    F = np.exp(-2j * np.pi * (np.outer(m, m) % N) / N)
    Fh = bf16(F.real) + 1j * bf16(F.imag)
    Xh = bf16(X.real) + 1j * bf16(X.imag)
    one_term = Fh @ Xh @ Fh.T
    ref = np.fft.fft2(X.astype(np.complex128))
    assert np.linalg.norm(one_term - ref) / np.linalg.norm(ref) > 1e-3
