"""The FP64 step's fixed-point pair update, run on the host (no GPU).

The TRT collision (Sect. 2) updates each opposite pair (a, b = inv a) from
its even and odd parts: p_a,b = e +- o with e = K0 + (c_a.u)(c_a.T) +
qp (d_a + d_b) and o = qm (d_a - d_b) + c_a.O (K0, T, O halved for the face
diagonals).  The LBM_F64 step kernels evaluate this in 64-bit fixed point;
lbm_fx_pairs_host runs the same routine on the host.  These tests hold it to
exact rational arithmetic of that formula, with the lattice velocities from
the oracle's D3Q19 table: every value within 8 units of the pair scale plus
half an ulp of its rounding.  They also check which nodes the routine refuses
(the kernels then take the FP64 update).
"""
from fractions import Fraction

import numpy as np
import pytest

import paper_1410_0412_gb300 as lbm
from oracle.d3q19 import C, W


def _exact_pairs(d, t, qm, qp):
    f = [Fraction(float(v)) for v in d]
    u = [Fraction(float(v)) for v in t[0:3]]
    K0 = Fraction(float(t[3]))
    T = [Fraction(float(v)) for v in t[4:7]]
    O = [Fraction(float(v)) for v in t[7:10]]
    qm, qp = Fraction(qm), Fraction(qp)
    out = [None] * 19
    for k in range(1, 10):
        a, b = 2 * k - 1, 2 * k
        c = [int(x) for x in C[a]]
        h = Fraction(1) if k <= 3 else Fraction(1, 2)
        cu = sum(c[i] * u[i] for i in range(3))
        ct = sum(c[i] * T[i] for i in range(3))
        co = sum(c[i] * O[i] for i in range(3))
        e = h * K0 + h * cu * ct + qp * (f[a] + f[b])
        o = qm * (f[a] - f[b]) + h * co
        out[a], out[b] = e + o, e - o
    return out


def _ulp(x):
    return np.spacing(abs(x))


def _nodes(n, seed, shifted):
    rng = np.random.default_rng(seed)
    w = np.asarray(W, dtype=np.float64)
    rho = 1 + 0.02 * (rng.random(n) - 0.5)
    u = 0.2 * (rng.random((n, 3)) - 0.5)
    cu = u @ np.asarray(C, dtype=np.float64).T
    feq = w * rho[:, None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u * u).sum(1)[:, None])
    d = feq * (1 + 0.05 * (rng.random((n, 19)) - 0.5))
    if shifted:
        d = d - w * 1.0
    B = 2.0 ** (np.floor(np.log2(np.abs(d).max(1))))
    terms = np.empty((n, 10))
    terms[:, 0:3] = u
    terms[:, 3] = (rng.random(n) - 0.5) * 0.9 * B
    terms[:, 4:10] = (rng.random((n, 6)) - 0.5) * 0.45 * B[:, None]
    return d, terms


@pytest.mark.parametrize("lp1", [True, False])
@pytest.mark.parametrize("shifted", [False, True])
def test_fx_pairs_within_bound_of_exact_rationals(lp1, shifted):
    d, terms = _nodes(300, 7 + shifted + 2 * lp1, shifted)
    qm = -1.0 / 14.0
    qp = 0.0 if lp1 else 0.125
    out, ok = lbm.lbm_fx_pairs_host(d, terms, qm, qp, lp1)
    assert ok.all()
    for n in range(len(d)):
        ex = _exact_pairs(d[n], terms[n], qm, qp)
        unit = Fraction(2) ** (int(out[n, 0]) - 1080)
        for i in range(1, 19):
            err = abs(Fraction(float(out[n, i])) - ex[i])
            assert err <= 8 * unit + Fraction(float(_ulp(out[n, i]))) / 2, (n, i, float(err))


def test_fx_pairs_is_as_tight_as_a_quarter_ulp_at_rest_scale():
    # PDFs near w_i rho (full storage, l+ = 1): the fixed-point error stays
    # below a quarter ulp of the smallest PDFs (the diagonals, ~1/36) before
    # the final rounding, so each value is within 3/4 ulp of the exact result
    rng = np.random.default_rng(3)
    n = 300
    w = np.asarray(W, dtype=np.float64)
    rho = 1 + 0.02 * (rng.random(n) - 0.5)
    u = 0.04 * (rng.random((n, 3)) - 0.5)
    cu = u @ np.asarray(C, dtype=np.float64).T
    d = w * rho[:, None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u * u).sum(1)[:, None])
    d = d * (1 + 1e-3 * (rng.random((n, 19)) - 0.5))
    uu = (u * u).sum(1)
    terms = np.column_stack([u, rho / 18 * (1 - 1.5 * uu), (rho / 4)[:, None] * u, (rho / 6 * 8 / 7)[:, None] * u])
    out, ok = lbm.lbm_fx_pairs_host(d, terms, -1.0 / 14.0, 0.0, True)
    assert ok.all()
    for n in range(len(d)):
        ex = _exact_pairs(d[n], terms[n], -1.0 / 14.0, 0.0)
        for i in range(1, 19):
            err = abs(Fraction(float(out[n, i])) - ex[i])
            assert err <= Fraction(3, 4) * Fraction(float(_ulp(float(ex[i])))), (n, i)


@pytest.mark.parametrize("lp1", [True, False])
@pytest.mark.parametrize("shifted", [False, True])
def test_fx_pairs_short_conversions_give_the_same_bits(lp1, shifted):
    # the kernels convert positive values in a common range with shorter
    # routines (moments: positive PDFs within 5 binades of the largest;
    # outputs: 2^32 <= v < 2^63); they must give the general routines' bits
    d, terms = _nodes(2000, 20 + shifted + 2 * lp1, shifted)
    qp = 0.0 if lp1 else 0.125
    fast, ok1 = lbm.lbm_fx_pairs_host(d, terms, -1.0 / 14.0, qp, lp1)
    gen, ok2 = lbm.lbm_fx_pairs_host(d, terms, -1.0 / 14.0, qp, lp1, general=True)
    assert ok1.all() and ok2.all()
    assert np.array_equal(fast.view(np.uint64), gen.view(np.uint64))


def test_fx_pairs_refuses_values_outside_its_range():
    d, terms = _nodes(6, 11, False)
    B = 2.0 ** np.floor(np.log2(np.abs(d).max(1)))
    bad = terms.copy()
    bad[0, 0] = 0.25            # |u_x| = 1/4
    bad[1, 2] = -0.3            # |u_z| > 1/4
    bad[2, 3] = 0.5 * B[2]      # K0 = B/2
    bad[3, 5] = 0.25 * B[3]     # T_y = B/4
    bad[4, 9] = -0.3 * B[4]     # O_z < -B/4
    bad[5, 4] = np.nan          # NaN
    _, ok = lbm.lbm_fx_pairs_host(d, bad, -1.0 / 14.0, 0.0, True)
    assert not ok.any()
    d2 = d.copy()
    d2[0, 3] = np.inf           # a non-finite PDF
    _, ok = lbm.lbm_fx_pairs_host(d2, terms, -1.0 / 14.0, 0.0, True)
    assert not ok[0] and ok[1:].all()


def test_fx_pairs_argument_checks():
    d, terms = _nodes(2, 1, False)
    for qm, qp, lp1 in ((0.5, 0.0, True), (-0.1, 0.1, True), (0.1, -0.5, False)):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_fx_pairs_host(d, terms, qm, qp, lp1)
