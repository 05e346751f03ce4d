"""The FP64 step's integer moment arithmetic, run on the host (no GPU).

The LBM_F64 step kernels form each node's moments (the density deviation, the
momentum and the pair sums and differences of the TRT collision, Sect. 2) as
exact fixed-point sums, rounded once to double.  lbm_exact_moments_host runs
the same routine on the host; these tests hold it to exact rational
arithmetic, with the lattice velocities taken from the oracle's D3Q19 table.
"""
from fractions import Fraction

import numpy as np
import pytest

import paper_1410_0412_gb300 as lbm
from oracle.d3q19 import C, INV, W


def exact_moments(d):
    """[22] exact rationals: drho, j, sa_1..9, da_1..9 of one node's 19 PDFs."""
    f = [Fraction(float(v)) for v in d]
    drho = sum(f, Fraction(0))
    j = [sum((int(C[i][a]) * f[i] for i in range(19)), Fraction(0)) for a in range(3)]
    sa = [f[2 * k - 1] + f[2 * k] for k in range(1, 10)]
    da = [f[2 * k - 1] - f[2 * k] for k in range(1, 10)]
    return [drho] + j + sa + da


def biased_exponents(d):
    return (np.asarray(d, dtype=np.float64).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)


def test_pair_layout_matches_the_direction_table():
    # the routine pairs directions 2k-1 and 2k and sums j with the sign pattern
    # of the first directions (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1)
    # (1,0,-1) (0,1,1) (0,1,-1); the oracle's table must agree
    for k in range(1, 10):
        assert INV[2 * k - 1] == 2 * k
    firsts = [tuple(int(x) for x in C[2 * k - 1]) for k in range(1, 10)]
    assert firsts == [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1),
                      (0, 1, -1)]


def test_moments_equal_the_correctly_rounded_exact_sums():
    # PDFs near w_i rho (all within 5 binades of the largest): every output is
    # the exact sum rounded once, bit for bit
    rng = np.random.default_rng(3)
    n = 1500
    rho = rng.uniform(0.5, 1.5, size=(n, 1))
    d = np.asarray(W)[None, :] * rho * (1.0 + rng.uniform(-0.03, 0.03, size=(n, 19)))
    got = lbm.lbm_exact_moments_host(d)
    for k in range(n):
        assert np.all(biased_exponents(d[k]) >= biased_exponents(d[k]).max() - 5)
        want = [float(x) for x in exact_moments(d[k])]
        assert got[k].tolist() == want, k


def test_deviation_form_mixed_scales_stays_within_the_truncation_bound():
    # shifted PDFs f - w rho0: signs and exponents spread over ten decades; a
    # PDF more than 5 binades below the largest loses bits under 2^-57 of it
    rng = np.random.default_rng(4)
    n = 800
    d = rng.choice([-1.0, 1.0], size=(n, 19)) * 10.0 ** rng.uniform(-12, -2, size=(n, 19))
    got = lbm.lbm_exact_moments_host(d)
    for k in range(n):
        emax = int(biased_exponents(d[k]).max())
        lsb = Fraction(2) ** (emax - 1080)
        for out, x in zip(got[k], exact_moments(d[k])):
            # at most 19 truncations of one lsb each, then one rounding
            bound = 19 * lsb + Fraction(abs(out)) * Fraction(2) ** -53
            assert abs(Fraction(out) - x) <= bound


def test_exact_cancellation_and_zero():
    # opposite PDFs that cancel exactly give exact zeros (an IEEE sum in the
    # wrong order need not); an all-zero node gives zeros
    d = np.zeros((2, 19))
    d[0, 1], d[0, 2] = 0.1, 0.1
    d[0, 0] = 1.0 / 3.0
    got = lbm.lbm_exact_moments_host(d)
    assert got[0, 1] == 0.0 and got[0, 13] == 0.0  # jx and da_1
    assert got[0, 4] == float(Fraction(0.1) + Fraction(0.1))
    assert np.all(got[1] == 0.0)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 1e307])
def test_nonfinite_or_huge_pdf_marks_the_node(bad):
    d = np.tile(np.asarray(W, dtype=np.float64), (3, 1))
    d[1, 7] = bad
    got = lbm.lbm_exact_moments_host(d)
    assert np.isnan(got[1, 0])
    assert np.isfinite(got[0]).all() and np.isfinite(got[2]).all()


def test_rejects_bad_shapes():
    with pytest.raises(ValueError):
        lbm.lbm_exact_moments_host(np.zeros((4, 18)))


def test_property_exact_or_within_bound():
    """Property test over arbitrary finite PDFs (hypothesis, where installed): every output is
    within 19 truncations of 2^(emax-1080) plus one rounding of the exact rational sum, and
    exactly the rounded sum when no PDF lies more than 5 binades below the largest."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=300, deadline=None)
    @hyp.given(st.lists(st.floats(min_value=-1e6, max_value=1e6, allow_nan=False, allow_infinity=False,
                                  allow_subnormal=False), min_size=19, max_size=19))
    def check(vals):
        d = np.asarray(vals, dtype=np.float64)[None, :]
        got = lbm.lbm_exact_moments_host(d)[0]
        e = biased_exponents(d[0])
        emax = max(int(e.max()), 64)
        exact = exact_moments(d[0])
        within5 = bool(np.all((e == 0) | (e >= emax - 5)))
        lsb = Fraction(2) ** (emax - 1080)
        for out, x in zip(got, exact):
            if within5:
                assert out == float(x)
            else:
                assert abs(Fraction(out) - x) <= 19 * lsb + Fraction(abs(out)) * Fraction(2) ** -53

    check()
