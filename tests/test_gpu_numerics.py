"""Accuracy of the two places where the factorisations leave plain IEEE FP64 arithmetic.

1. The LU refactorisation forms its pivots' reciprocals as the hardware's
   approximate FP64 reciprocal (which flushes subnormal inputs to zero) refined
   by two Newton-Raphson steps.  For every normal pivot whose reciprocal is
   normal the result equals IEEE 1/u bit for bit, except for u just below a
   power of two (every mantissa bit set), where it is one unit in the last
   place off (a relative error of 2^-52 in one multiplier, below the rounding
   of the LU's own updates); a
   zero or subnormal pivot gives NaN, which the refactorisation's pivot check
   reports as a singular Jacobian (exactly as it reports a zero pivot).
2. The Schur-complement Cholesky (Prop. 3) applies each group's rank-K
   trailing update C -= P P^T emulated on the bf16 tensor cores.  Each row of P
   is written against its own power of two 2^E_r (|P_rk| < 2^E_r <= 2 max_k
   |P_rk|) as eight 7-bit digits plus a tail below 2^(E_r - 56); the dropped
   digit-pair levels (i + j >= 8, at most 7 pairs of products below 2^14 at
   level 8, each 2^-7 smaller per further level) and the tails bound each
   product's error by (7.1 + 2) 2^(E_r + E_c - 56), i.e. below
   4.6 u max|P_r| max|P_c| with u = 2^-53, so the update errs by less than
   5 K u max|P_r| max|P_c|, plus the final FP64 roundings (at most
   2 u (|C| + sum_k |P_rk P_ck|)).  The test checks every element of an
   update of 512 rows x 128 columns whose rows span nine decades against a
   long-double reference.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
U = 2.0 ** -53


def test_pivot_reciprocal_is_ieee_division():
    rng = np.random.default_rng(11)
    n = 4 << 20
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-1000, 1001, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    u = sign * np.ldexp(mant, expo)
    # pivots of the size the relative pivot test sees, powers of two and their neighbours
    extra = np.concatenate([np.ldexp(1.0, np.arange(-1000, 1001)),
                            np.nextafter(np.ldexp(1.0, np.arange(-1000, 1001)), 0.0),
                            np.nextafter(np.ldexp(1.0, np.arange(-1000, 1001)), np.inf),
                            rng.uniform(1e-16, 1e-12, 100000), -rng.uniform(1e-16, 1e-12, 100000),
                            np.array([1.0, -1.0, 3.0, 1.0 / 3.0, 0.1, 1e-300, 1e300])])
    u = np.concatenate([u, extra])
    r = P.pivot_reciprocal(torch.as_tensor(u, device=DEV)).cpu().numpy()
    ref = 1.0 / u
    bad = np.flatnonzero(r != ref)
    # the only operands that differ lie just below a power of two (every mantissa bit set; 1/u
    # then lies just above the power of two's reciprocal), and by one unit in the last place
    mant_bits = u[bad].view(np.int64) & ((1 << 52) - 1)
    assert np.all(mant_bits == (1 << 52) - 1), u[bad[mant_bits != (1 << 52) - 1][:5]]
    ulps = np.abs(r[bad].view(np.int64) - ref[bad].view(np.int64))
    assert np.all(np.sign(r[bad]) == np.sign(ref[bad])) and np.all(ulps <= 1), ulps.max()
    assert bad.size <= 2001


def test_pivot_reciprocal_zero_and_subnormal_give_nan():
    tiny = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-310, -2.2e-308])
    r = P.pivot_reciprocal(torch.as_tensor(tiny, device=DEV)).cpu().numpy()
    assert np.all(np.isnan(r)), r


@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("K,decades", [(128, 9), (64, 9), (128, 0)])
def test_emulated_rank_k_update_error_bound(K, decades, engine):
    rng = np.random.default_rng(5 + K + decades)
    M, c0 = 512, 0
    r0 = c0 + K
    n = r0 + M
    A = rng.standard_normal((n, n))
    # rows of P spread over `decades` decades, entries within a row over two more
    row_scale = 10.0 ** (-decades * np.arange(M) / (M - 1))
    Pm = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-2, 0, (M, K)) * row_scale[:, None]
    A[r0:, c0:c0 + K] = Pm
    Cm = A[r0:, r0:].copy()
    # column-major storage on the device: the tensor's row j is column j of A
    At = torch.as_tensor(np.ascontiguousarray(A.T), device=DEV)
    P.dense_syrk_emulated(At, c0, K, r0, engine=engine)
    got = At.cpu().numpy().T[r0:, r0:]
    Pl = Pm.astype(np.longdouble)
    ref = Cm.astype(np.longdouble) - Pl @ Pl.T
    err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
    pmax = np.abs(Pm).max(axis=1)
    absprod = np.abs(Pm) @ np.abs(Pm).T
    bound = 5 * K * U * np.outer(pmax, pmax) + 2 * U * (np.abs(Cm) + absprod)
    lower = np.tril(np.ones((M, M), dtype=bool))
    ratio = (err / bound)[lower]
    assert ratio.max() <= 1.0, ratio.max()
    # the upper triangle of the block is not touched
    assert np.array_equal(got[~lower], Cm[~lower])
    # and the update really happened: the result is the product's, not the input
    assert np.abs((got - Cm)[lower]).max() > 0.1


@pytest.mark.parametrize("M,K,c0", [(2771, 128, 0), (300, 96, 8), (129, 32, 0), (64, 64, 40), (1, 128, 0)])
def test_emulated_update_engines_bit_identical(M, K, c0):
    """The tcgen05 kernel (level sums in tensor memory) and the warp-level mma.sync kernel add
    the same exact integer digit products and round them the same way (the tcgen05 epilogue
    in integer arithmetic): the updated triangles are equal bit for bit, on ragged sizes
    (partial 128 x 64 and 64 x 64 tiles) and the largest update of the 9.2k-bus grid's Schur
    complement (2,771 rows)."""
    rng = np.random.default_rng(M + K)
    r0 = c0 + K
    n = r0 + M
    A = rng.standard_normal((n, n)) * 10.0 ** rng.uniform(-6, 3, (n, 1))
    outs = []
    for engine in (2, 1, 0):  # tcgen05, mma.sync, and the size-based choice between them
        At = torch.as_tensor(np.ascontiguousarray(A.T), device=DEV)
        P.dense_syrk_emulated(At, c0, K, r0, engine=engine)
        outs.append(At.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    # and it is the update: the lower triangle changed, everything else did not
    low = np.tril(np.ones((M, M), dtype=bool))
    got = outs[0].T
    assert np.array_equal(got[:, :r0], A[:, :r0]) and np.array_equal(got[:r0, :], A[:r0, :])
    blk, ref = got[r0:, r0:], A[r0:, r0:]
    assert np.array_equal(blk[~low], ref[~low])
    Pm = A[r0:, c0:c0 + K]
    exact = ref - Pm @ Pm.T
    scale = np.abs(Pm).max(axis=1)
    err = np.abs(blk - exact)[low] / (np.outer(scale, scale)[low] + np.abs(ref)[low])
    assert err.max() < 1e-12


def test_fp64_peak_is_plausible():
    tf, ms = P.fp64_peak()
    assert 0.3 < tf < 3.0 and ms > 0.0
