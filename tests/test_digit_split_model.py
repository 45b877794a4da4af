"""The exact digit split behind the tensor-core stochastic operators, checked
on the CPU in integer arithmetic (no GPU, no library code).

The claim: for sources with components in {0, +-1}, cutting every component
x of gamma5 X (per source, timeslice and block of 4096 complex rows) to
m = trunc(x 2^(55 - e)) with |x| < 2^e, splitting m into five signed 11-bit
digits and summing digit products over at most 8192 real columns keeps
every partial sum an integer below 2^24 (so FP32 accumulation is exact), and
the digit sums recombined with weights 2^(e - 55 + 11(4 - s)) give O_ij(t)
of Eq. stoop up to the truncation (below 2^(e-55) per component) and FP64
rounding.
"""

import numpy as np

import oracle
from paper_1405_4524_gb300 import inputs

BLOCK = 4096  # complex rows per exponent block (8192 real columns)


def digit_model(eta, X):
    n, T = eta.shape[0], eta.shape[1]
    K = int(np.prod(eta.shape[2:]))
    e_ = eta.reshape(n, T, K)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), K // 12)
    y = X.reshape(n, T, K) * g5
    O = np.zeros((T, n, n), dtype=np.complex128)
    worst = 0
    for t in range(T):
        # real form: columns (Re, Im) interleaved; A = eta, B_re = (yr, yi), B_im = (yi, -yr)
        A = np.stack([e_[:, t].real, e_[:, t].imag], axis=-1).reshape(n, 2 * K).astype(np.int64)
        assert np.all(np.isin(A, (-1, 0, 1)))
        acc_re = np.zeros((n, n))
        acc_im = np.zeros((n, n))
        for b0 in range(0, K, BLOCK):
            yb = y[:, t, b0:b0 + BLOCK]
            mx = np.maximum(np.abs(yb.real).max(axis=1), np.abs(yb.imag).max(axis=1))
            e = np.where(mx > 0, np.frexp(mx)[1], 0)  # |x| < 2^e
            scale = np.ldexp(1.0, 55 - e)[:, None]
            mr = np.trunc(yb.real * scale).astype(np.int64)  # exact: |m| < 2^55
            mi = np.trunc(yb.imag * scale).astype(np.int64)
            Ab = A[:, 2 * b0:2 * (b0 + yb.shape[1])]
            for s in range(5):
                def dig(m):
                    d = (np.abs(m) >> (11 * (4 - s))) & 2047
                    return np.where(m < 0, -d, d)
                dr, di = dig(mr), dig(mi)
                Bre = np.stack([dr, di], axis=-1).reshape(n, -1)
                Bim = np.stack([di, -dr], axis=-1).reshape(n, -1)
                Dre = Ab @ Bre.T  # exact integer sums over <= 8192 columns
                Dim = Ab @ Bim.T
                worst = max(worst, int(np.abs(Dre).max()), int(np.abs(Dim).max()))
                w = np.ldexp(1.0, e - 55 + 11 * (4 - s))[None, :]
                acc_re += Dre * w
                acc_im += Dim * w
        O[t] = acc_re + 1j * acc_im
    return O, worst


def test_digit_split_is_exact_to_the_stated_bound():
    dims = (4, 4, 4, 6)  # 768 complex rows per slice: blocks cover whole slices
    n = 5
    eta = inputs.make_z4(dims, n, 8101)
    rng = np.random.default_rng(8102)
    X = inputs.make_gaussian_spinors(dims, n, 8103) * np.exp(rng.uniform(-8, 8, (n, dims[3])))[
        :, :, None, None, None, None, None]
    O, worst = digit_model(eta, X)
    assert worst < 2 ** 24  # every FP32 partial sum of the products is an exact integer
    want = oracle.stochastic_operator(eta, X)
    # truncation: below 2^(e-55) per component, at most 2*K components per element
    K = 12 * 4 * 4 * 4
    bound = np.zeros_like(want.real)
    for t in range(dims[3]):
        m = np.max(np.abs(X[:, t].reshape(n, -1).view(np.float64)), axis=1)
        bound[t] = 2 * K * np.ldexp(1.0, np.frexp(m)[1] - 55)[None, :] * 2
    err = np.maximum(np.abs(O.real - want.real), np.abs(O.imag - want.imag))
    assert np.all(err <= bound + 1e-13 * np.abs(want).max())
    assert np.max(np.abs(O - want)) <= 1e-13 * np.max(np.abs(want))


def test_digit_split_two_blocks_and_dilution():
    """A slice of 6144 rows (two exponent blocks, the second partial) and
    time-diluted sources (zeros off the source timeslice)."""
    dims = (8, 8, 8, 2)
    n = 3
    eta = inputs.make_z4(dims, n, 8201, [0, 1, 0])
    X = inputs.make_gaussian_spinors(dims, n, 8202)
    X[1, 1, :4] *= 1e-6  # a block whose rows span six decades
    O, worst = digit_model(eta, X)
    assert worst < 2 ** 24
    want = oracle.stochastic_operator(eta, X)
    assert np.max(np.abs(O - want)) <= 1e-13 * np.max(np.abs(want))
