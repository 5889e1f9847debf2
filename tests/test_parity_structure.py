"""The parity-class structure the folded kernels rely on, checked on the CPU
against the oracle's own atoms, weights, tables (Alg. 2) and projections.

For a weighting function symmetric about the area's centre in both directions
and atoms that are even or odd in each direction (the DCT-II and the
sequency-ordered Walsh rows), the weighted inner product of atoms of different
parity classes (p mod 2, q mod 2) vanishes, so the table of eq. (16) splits
into four class blocks; eq. (12) and the class blocks can then be evaluated on
one quadrant of the area from the folded signal
X_ab = x + (-1)^a x(M-1-m, n) + (-1)^b x(m, N-1-n) + (-1)^(a+b) x(M-1-m, N-1-n).
None of this is in the paper; the library detects it per plan, and these tests
pin the identities it uses to the oracle, independently of the CUDA kernels.
"""
import numpy as np
import pytest

import oracle as O
from paper_2204_14194_gb300 import workloads as W


def _pattern(M, N, shift=0):
    sup = np.ones((M, N), dtype=np.uint8)
    sup[M // 4:3 * M // 4, N // 4 + shift:3 * N // 4 + shift] = 0
    if shift == 0:
        for (r, c) in ((1, 2), (2, N - 4)):
            for rr, cc in ((r, c), (M - 2 - r, c), (r, N - 2 - c), (M - 2 - r, N - 2 - c)):
                sup[rr:rr + 2, cc:cc + 2] = 0
    return sup


def _classes(K, M, N):
    MN = M * N
    kk = np.arange(K) % MN
    return 2 * ((kk // N) & 1) + ((kk % N) & 1)


def _fold(x, a, b):
    M, N = x.shape
    xm, xn, xmn = x[::-1, :], x[:, ::-1], x[::-1, ::-1]
    f = x + (-1) ** a * xm + (-1) ** b * xn + (-1) ** (a + b) * xmn
    return f[:M // 2, :N // 2]


@pytest.mark.parametrize("M,N,basis", [(16, 16, "dct_wht"), (16, 8, "dct_wht"), (16, 16, "dct"), (8, 16, "wht")])
def test_cross_class_table_entries_vanish(M, N, basis):
    phi = O.dictionary(basis, M, N)
    K = phi.shape[0]
    w = O.weights(M, N, 0.8, _pattern(M, N))
    assert (w == w[::-1, :]).all() and (w == w[:, ::-1]).all()
    Cm, D = O.fase_tables(phi, w)
    cls = _classes(K, M, N)
    diag = np.sqrt(np.outer(np.diag(Cm), np.diag(Cm)))
    cross = cls[:, None] != cls[None, :]
    assert np.abs(Cm[cross]).max() <= 1e-12 * diag.max()
    # the same classes are not empty of overlap (the blocks carry the table)
    assert np.abs(Cm[~cross & ~np.eye(K, dtype=bool)]).max() > 1e-3 * diag.max()


def test_a_shifted_pattern_breaks_the_classes():
    M = N = 16
    phi = O.dictionary("dct_wht", M, N)
    w = O.weights(M, N, 0.8, _pattern(M, N, shift=1))
    Cm, _ = O.fase_tables(phi, w)
    cls = _classes(phi.shape[0], M, N)
    cross = cls[:, None] != cls[None, :]
    assert np.abs(Cm[cross]).max() > 1e-3 * np.abs(np.diag(Cm)).max()


@pytest.mark.parametrize("M,N,basis", [(16, 16, "dct_wht"), (8, 16, "dct")])
def test_folded_projections_table_rows_and_diagonal(M, N, basis):
    phi = O.dictionary(basis, M, N)
    K = phi.shape[0]
    sup = _pattern(M, N)
    w = O.weights(M, N, 0.8, sup)
    Cm, _ = O.fase_tables(phi, w)
    cls = _classes(K, M, N)
    s = W.patch(max(M, N), 77)[:M, :N]
    # eq. (12): R_k = <s, phi_k>_w from the oracle's projection state (p_k C_kk)
    ps = O.projection_state(phi, w, np.where(sup > 0, s, 0.0))
    R = ps.p * ps.ckk
    x = w * np.where(sup > 0, s, 0.0)
    for k in range(K):
        a, b = cls[k] >> 1, cls[k] & 1
        q = phi[k][:M // 2, :N // 2]
        # projections from the folded signal of the atom's class
        assert abs(np.sum(q * _fold(x, a, b)) - R[k]) <= 1e-9 * (1 + abs(R[k]))
        # diagonal and compact row entries: four times the quadrant sums
        assert abs(4 * np.sum(w[:M // 2, :N // 2] * q * q) - Cm[k, k]) <= 1e-12 * Cm[k, k]
    for u in range(0, K, 7):
        same = np.nonzero(cls == cls[u])[0]
        qu = w[:M // 2, :N // 2] * phi[u][:M // 2, :N // 2]
        row = np.array([4 * np.sum(qu * phi[k][:M // 2, :N // 2]) for k in same])
        np.testing.assert_allclose(row, Cm[same, u], rtol=0, atol=1e-12 * np.abs(np.diag(Cm)).max())
