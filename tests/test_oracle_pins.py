"""Pins for the FP64 CPU oracle: each test ties it to something other than itself.

Citations are to Seiler & Kaup, arXiv 2204.14194.  What pins what:
  eq. (5)          exact decay values at integer distances, symmetries
  dictionaries     DCT atoms == scipy's inverse orthonormal DCT of impulses;
                   WHT atoms == Hadamard rows picked by the Gray-code /
                   bit-reversal sequency permutation (a different construction)
  duplicates       DCT_{L/2} is a square wave, so it coincides with WAL_{L/2}
  eq. (6) == (7)   brute-force argmin e_k equals argmax p_k^2 C_kk, and
                   e_k = E - p_k^2 C_kk holds numerically
  Alg. 1 == Alg. 3 the paper's equivalence claim, and the R recurrence of
                   eq. (15) equals the scalar products of SE's own residual
  single atom      closed form c_nu = gamma (1-gamma)^(nu-1) a, exact model
  three atoms      closed-form selection order, coefficients and tie margin
  energy           E drops by gamma (2-gamma) R_u^2 / C_uu per iteration
  w == 1, gamma=1  orthonormal case reduces to the best I-term approximation
                   from scipy's DCT / an independent fast WHT
  Table I          operation counts reproduce Fig. 3's plotted data
"""
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import oracle as O
from paper_2204_14194_gb300 import opcount
from paper_2204_14194_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------ eq. 4-5
def test_weights_integer_distances_and_masking():
    M = N = 9                      # odd: the centre pixel (4, 4) has distance 0
    sup = np.ones((M, N), dtype=np.uint8)
    sup[2, 7] = 0
    w = O.weights(M, N, 0.8, sup)
    assert w[4, 4] == 1.0
    for j in range(1, 5):          # on the axes the distance is the integer j
        for (m, n) in ((4, 4 + j), (4, 4 - j), (4 + j, 4), (4 - j, 4)):
            assert w[m, n] == pytest.approx(0.8 ** j, rel=1e-15)
    assert w[4 + 3, 4 + 4] == pytest.approx(0.8 ** 5, rel=1e-15)   # 3-4-5 triangle
    assert w[2, 7] == 0.0
    # even size: the centre lies between pixels, distance sqrt(0.5) from the four middle ones
    w2 = O.weights(32, 32, 0.8, np.ones((32, 32), np.uint8))
    for (m, n) in ((15, 15), (15, 16), (16, 15), (16, 16)):
        assert w2[m, n] == pytest.approx(0.8 ** math.sqrt(0.5), rel=1e-15)
    np.testing.assert_array_equal(w2, w2[::-1, :])
    np.testing.assert_array_equal(w2, w2[:, ::-1])
    np.testing.assert_array_equal(w2, w2.T)
    assert np.all(O.weights(32, 32, 1.0, np.ones((32, 32), np.uint8)) == 1.0)


# ------------------------------------------------------------ dictionaries
@pytest.mark.parametrize("M,N", [(4, 4), (8, 16), (32, 32)])
def test_dct_atoms_are_scipy_inverse_dct_of_impulses(M, N):
    phi = O.dict_dct(M, N)
    for k in [0, 1, N, N + 1, M * N // 2 + 3, M * N - 1]:
        p, q = divmod(k, N)
        e = np.zeros((M, N))
        e[p, q] = 1.0
        np.testing.assert_allclose(phi[k], scipy.fft.idctn(e, norm="ortho"), atol=1e-14)


def _sequency_hadamard(L):
    """Walsh functions in sequency order from the Gray-code/bit-reversal rule."""
    H = scipy.linalg.hadamard(L).astype(np.float64)
    bits = int(math.log2(L))
    out = np.empty_like(H)
    for p in range(L):
        g = p ^ (p >> 1)
        rev = int(format(g, f"0{bits}b")[::-1], 2)
        out[p] = H[rev]
    return out


@pytest.mark.parametrize("M,N", [(4, 4), (8, 16), (32, 32), (64, 64)])
def test_wht_atoms_match_gray_code_sequency_construction(M, N):
    phi = O.dict_wht(M, N).reshape(M * N, M * N)
    ref = np.kron(_sequency_hadamard(M), _sequency_hadamard(N)) / math.sqrt(M * N)
    np.testing.assert_array_equal(phi, ref)
    np.testing.assert_allclose(phi @ phi.T, np.eye(M * N), atol=1e-13)


def test_duplicate_atoms_of_dct_union_wht():
    # DCT_{L/2}[m] = sqrt(2/L) cos(pi (2m+1)/4) = +-1/sqrt(L) with signs + - - + ...,
    # which is the Walsh function of sequency L/2; DC coincides too.
    for L in (4, 16, 32):
        phi = O.dict_dct_wht(L, L)
        dup = O.find_duplicates(phi)
        h, MN = L // 2, L * L
        expect = {MN + 0, MN + h, MN + h * L, MN + h * L + h}
        assert set(np.nonzero(dup)[0].tolist()) == expect
    g = W.gaussian_dictionary(64, 8, 8, 5)
    assert O.find_duplicates(g).sum() == 0


# ------------------------------------------------------------- eq. 6 == 7
def _tiny_cases():
    cases = []
    for L, seed in ((4, 11), (8, 12)):
        phi = O.dict_dct_wht(L, L)
        sup = W.centred_support(L, L)
        cases.append((phi, sup, W.patch(L, seed), O.find_duplicates(phi)))
    phi = W.gaussian_dictionary(64, 8, 8, 13)
    sup = W.rect_support(8, 8, _rng(14))
    cases.append((phi, sup, W.patch(8, 15), O.find_duplicates(phi)))
    return cases


def test_bruteforce_distance_equals_score_selection():
    for phi, sup, s, dup in _tiny_cases():
        w = O.weights(*sup.shape, 0.8, sup)
        I = 30
        a = O.se_original(phi, w, s, 0.5, I, dup)
        b = O.se_original(phi, w, s, 0.5, I, dup, brute_force=True)
        ok = np.cumprod(a.margin > 1e-9).astype(bool)      # compare up to a near-tie
        assert ok[:10].all()
        np.testing.assert_array_equal(a.u[ok], b.u[ok])
        np.testing.assert_allclose(b.c[ok], a.c[ok], rtol=1e-12, atol=0)


def test_distance_identity_e_equals_E_minus_score():
    for phi, sup, s, dup in _tiny_cases():
        w = O.weights(*sup.shape, 0.8, sup)
        for I in (0, 3, 11):
            r = O.se_original(phi, w, s, 0.5, max(I, 1), dup).r if I else np.where(sup > 0, s, 0.0)
            st = O.projection_state(phi, w, r)
            E = float(np.sum(w * r * r))
            np.testing.assert_allclose(st.e, E - st.p ** 2 * st.ckk, rtol=1e-12, atol=1e-12 * E)
            np.testing.assert_allclose(st.score, st.p ** 2 * st.ckk, rtol=1e-15)


# -------------------------------------------------------- Alg. 1 == Alg. 3
def test_fase_equals_se_on_config1():
    c = W.config1()
    phi = O.dict_dct_wht(32, 32)
    dup = O.find_duplicates(phi)
    w = O.weights(32, 32, c.rho_hat, c.support)
    a = O.se_original(phi, w, c.samples[0], c.gamma, c.iterations, dup)
    Cm, D = O.fase_tables(phi, w)
    f = O.fase(phi, w, Cm, D, c.samples[0], c.gamma, c.iterations, dup)
    assert a.margin.min() > 1e-9
    np.testing.assert_array_equal(a.u, f.u)
    np.testing.assert_allclose(f.c, a.c, rtol=1e-11)
    np.testing.assert_allclose(f.out, a.out, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("case", range(3))
def test_R_recurrence_equals_scalar_products_of_residual(case):
    phi, sup, s, dup = _tiny_cases()[case]
    w = O.weights(*sup.shape, 0.8, sup)
    Cm, D = O.fase_tables(phi, w)
    for I in (1, 5, 20):
        a = O.se_original(phi, w, s, 0.5, I, dup)
        f = O.fase(phi, w, Cm, D, s, 0.5, I, dup)
        if a.margin.min() > 1e-9:
            np.testing.assert_array_equal(a.u, f.u)
        st = O.projection_state(phi, w, a.r)
        R_explicit = st.p * st.ckk                      # eq. (11) from SE's residual
        scale = np.max(np.abs(R_explicit))
        np.testing.assert_allclose(f.R, R_explicit, rtol=0, atol=1e-11 * scale)


def test_tables_symmetric_and_D():
    phi, sup, s, dup = _tiny_cases()[1]
    w = O.weights(*sup.shape, 0.8, sup)
    Cm, D = O.fase_tables(phi, w)
    A = phi.reshape(phi.shape[0], -1)
    np.testing.assert_allclose(Cm, (A * w.ravel()) @ A.T, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(Cm, Cm.T)
    np.testing.assert_allclose(D, 1.0 / np.sqrt(np.diag(Cm)), rtol=1e-15)


# ------------------------------------------------------ closed-form single atom
@pytest.mark.parametrize("basis,j", [("dct_wht", 33), ("dct_wht", 1024 + 70), ("gauss", 17)])
def test_single_atom_closed_form(basis, j):
    L = 32 if basis == "dct_wht" else 8
    phi = O.dict_dct_wht(L, L) if basis == "dct_wht" else W.gaussian_dictionary(64, 8, 8, 21)
    dup = O.find_duplicates(phi)
    assert not dup[j]
    sup = W.centred_support(L, L)
    w = O.weights(L, L, 0.8, sup)
    a, gamma, I = 37.5, 0.5, 30      # (1-gamma)^I stays far above FP64 rounding of s
    s = a * phi[j]
    r = O.se_original(phi, w, s, gamma, I, dup)
    assert np.all(r.u == j)
    nu = np.arange(1, I + 1)
    np.testing.assert_allclose(r.c, gamma * (1 - gamma) ** (nu - 1) * a, rtol=1e-11)
    np.testing.assert_allclose(r.g, a * (1 - (1 - gamma) ** I) * phi[j], rtol=1e-11, atol=1e-12)


def test_three_atom_sequence_and_tie_margin_closed_form():
    """With w == 1 and orthonormal atoms, C = I, so the projection of eq. (3) is the atom's
    amplitude in the residual.  Eq. (8) multiplies the selected amplitude by (1 - gamma), so
    the selected sequence, the coefficients and the gap (s1 - s2) / s1 between the two best
    eq. (7) scores (the tie margin) follow in closed form.  The largest amplitude sits at
    the highest index, so the score scan has to move the old best into second place."""
    M = N = 8
    phi = O.dict_dct(M, N)
    w = O.weights(M, N, 0.8, np.ones((M, N), dtype=np.uint8), rho=np.ones((M, N)))
    idx, amp = [40, 7, 23], [5.0, -3.0, 2.0]
    s = sum(a * phi[k] for k, a in zip(idx, amp))
    gamma, I = 0.5, 7
    r = O.se_original(phi, w, s, gamma, I)
    cur = dict(zip(idx, amp))
    for nu in range(I):
        order = sorted(cur, key=lambda k: -cur[k] ** 2)
        s1, s2 = cur[order[0]] ** 2, cur[order[1]] ** 2
        assert s1 - s2 > 1e-3 * s1                      # no near-tie in this schedule
        assert r.u[nu] == order[0]
        assert r.c[nu] == pytest.approx(gamma * cur[order[0]], rel=1e-12)
        assert r.margin[nu] == pytest.approx((s1 - s2) / s1, rel=1e-9)
        cur[order[0]] *= 1.0 - gamma


# ------------------------------------------------------------------ energy
def test_energy_drop_per_iteration():
    for phi, sup, s, dup in _tiny_cases() + [(O.dict_dct_wht(32, 32), W.centred_support(32, 32),
                                              W.patch(32, 3), None)]:
        if dup is None:
            dup = O.find_duplicates(phi)
        w = O.weights(*sup.shape, 0.8, sup)
        gamma, I = 0.5, 40
        r = O.se_original(phi, w, s, gamma, I, dup)
        ckk = O.projection_state(phi, w, np.zeros_like(w)).ckk
        E0 = float(np.sum(w * np.where(sup > 0, s, 0.0) ** 2))
        E = np.concatenate([[E0], r.energy])
        p_u = r.c / gamma
        drop = gamma * (2 - gamma) * p_u ** 2 * ckk[r.u]        # = gamma(2-gamma) R_u^2 / C_uu
        np.testing.assert_allclose(E[:-1] - E[1:], drop, rtol=1e-9, atol=1e-12 * E0)
        assert np.all(np.diff(E) <= 1e-12 * E0)


# ------------------------------------------- orthonormal special case (w == 1)
@pytest.mark.parametrize("basis", ["dct", "wht"])
def test_unweighted_orthonormal_is_best_I_term(basis):
    L, I = 16, 40
    s = W.patch(L, 77)
    sup = np.ones((L, L), dtype=np.uint8)
    w = O.weights(L, L, 1.0, sup)
    phi = O.dict_dct(L, L) if basis == "dct" else O.dict_wht(L, L)
    if basis == "dct":
        coef = scipy.fft.dctn(s, norm="ortho").ravel()
        synth = lambda c: scipy.fft.idctn(c.reshape(L, L), norm="ortho")
    else:
        Hs = _sequency_hadamard(L) / math.sqrt(L)
        coef = (Hs @ s @ Hs.T).ravel()
        synth = lambda c: Hs.T @ c.reshape(L, L) @ Hs
    r = O.se_original(phi, w, s, 1.0, I)
    order = np.argsort(-np.abs(coef), kind="stable")[:I]
    np.testing.assert_array_equal(r.u, order)
    np.testing.assert_allclose(r.c, coef[order], rtol=1e-11)
    kept = np.zeros_like(coef)
    kept[order] = coef[order]
    np.testing.assert_allclose(r.g, synth(kept), atol=1e-10)


# ---------------------------------------------------------------- homogeneity
def test_homogeneity_power_of_two_is_bitwise():
    phi, sup, s, dup = _tiny_cases()[1]
    w = O.weights(*sup.shape, 0.8, sup)
    a = O.se_original(phi, w, s, 0.5, 25, dup)
    b = O.se_original(phi, w, 4.0 * s, 0.5, 25, dup)
    np.testing.assert_array_equal(a.u, b.u)
    np.testing.assert_array_equal(4.0 * a.c, b.c)


# --------------------------------------------------------------- edge cases
def test_empty_support_and_zero_signal():
    phi = O.dict_dct_wht(8, 8)
    dup = O.find_duplicates(phi)
    sup0 = np.zeros((8, 8), dtype=np.uint8)
    r = O.se_original(phi, O.weights(8, 8, 0.8, sup0), np.ones((8, 8)), 0.5, 3, dup)
    assert r.status == -5
    sup = W.centred_support(8, 8)
    r = O.se_original(phi, O.weights(8, 8, 0.8, sup), np.zeros((8, 8)), 0.5, 5, dup)
    assert r.status == 0 and np.all(r.u == 0) and np.all(r.c == 0.0)
    # values on B are never read
    s = W.patch(8, 3)
    s_nan = s.copy()
    s_nan[sup == 0] = np.nan
    w = O.weights(8, 8, 0.8, sup)
    a = O.se_original(phi, w, s, 0.5, 10, dup)
    b = O.se_original(phi, w, s_nan, 0.5, 10, dup)
    np.testing.assert_array_equal(a.u, b.u)
    np.testing.assert_array_equal(a.out[sup == 0], b.out[sup == 0])


def test_batch_matches_single_block():
    phi = O.dict_dct_wht(8, 8)
    dup = O.find_duplicates(phi)
    sup = W.centred_support(8, 8)
    w = O.weights(8, 8, 0.8, sup)
    s = np.stack([W.patch(8, 100 + i) for i in range(5)])
    out, u, c, rc = O.se_original_batch(phi, w, s, 0.5, 12, dup, nthreads=2)
    assert rc == 0
    for b in range(5):
        one = O.se_original(phi, w, s[b], 0.5, 12, dup)
        np.testing.assert_array_equal(u[b], one.u)
        np.testing.assert_array_equal(c[b], one.c)
        np.testing.assert_array_equal(out[b], one.out)
    Cm, D = O.fase_tables(phi, w)
    out2, u2, c2, rc2 = O.fase_batch(phi, w, Cm, D, s, 0.5, 12, dup, nthreads=2)
    assert rc2 == 0
    np.testing.assert_array_equal(u2, u)


# ------------------------------------------------------------ Table I / Fig. 3
def test_table1_counts_reproduce_fig3():
    rows = []
    with open(os.path.join(GOLDEN, "fig3_operation_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                curve, I, v = line.split()
                rows.append((curve, int(I), float(v)))
    assert len(rows) == 25
    for curve, I, v in rows:
        if curve == "SE":
            ops = opcount.total(opcount.se_ops(64, 64, 4096, I))
        elif curve == "FASE":
            ops = opcount.total(opcount.fase_ops(64, 64, 4096, I))
        else:
            ops = opcount.total(opcount.table_ops(64, 64, 4096))
        assert math.log10(ops) == pytest.approx(v, abs=6e-7), (curve, I)


@pytest.mark.parametrize("M,N,K", [(32, 32, 2048), (64, 64, 4096), (16, 16, 512)])
def test_per_iteration_count_is_the_slope_of_table1(M, N, K):
    """The benchmark's per-iteration operation count is the I-slope of Table I's FaSE row
    (which the Fig. 3 data pins); the parity-class count applies it to one class of K/4
    atoms plus one comparison per class."""
    slope = opcount.total(opcount.fase_ops(M, N, K, 101)) - opcount.total(opcount.fase_ops(M, N, K, 100))
    assert opcount.fase_iteration_ops(M, N, K) == slope
    q = opcount.total(opcount.fase_ops(M, N, K // 4, 2)) - opcount.total(opcount.fase_ops(M, N, K // 4, 1))
    assert opcount.fase_iteration_ops_classes(M, N, K) == q + 4
    # the iteration kernels' own share: Table I's per-iteration count without the
    # model accumulate (one multiply and one add per area pixel, eq. 9)
    model = opcount.total(opcount.fase_ops(M, N, K, 101)) - opcount.total(opcount.fase_ops(M, N, K, 100)) \
        - (opcount.total(opcount.fase_ops(1, 1, K, 101)) - opcount.total(opcount.fase_ops(1, 1, K, 100)))
    assert model == 2 * (M * N - 1)
    assert opcount.fase_select_update_ops(M, N, K) == 5 * K + 1
    assert opcount.fase_select_update_ops(M, N, K, classes=4) == 5 * (K // 4) + 4 + 1


# ------------------------------------------------------------- 3-D blocks
# The paper names the extension to video (three-dimensional areas) in its
# conclusion; the method runs unchanged on the flattened area, only the
# weighting function and the dictionaries gain a third coordinate.
@pytest.mark.parametrize("M,N,T", [(4, 6, 3), (8, 8, 4)])
def test_dct3_atoms_are_scipy_inverse_dct_of_impulses(M, N, T):
    phi = O.dictionary3("dct", M, N, T)
    V = M * N * T
    for k in [0, 1, N, M * N, M * N + N + 1, V // 2 + 3, V - 1]:
        r, rest = divmod(k, M * N)
        p, q = divmod(rest, N)
        e = np.zeros((T, M, N))
        e[r, p, q] = 1.0
        np.testing.assert_allclose(phi[k], scipy.fft.idctn(e, norm="ortho"), atol=1e-14)


def test_wht3_atoms_are_kronecker_products_of_sequency_rows():
    M, N, T = 4, 8, 2
    phi = O.dictionary3("wht", M, N, T).reshape(M * N * T, M * N * T)
    ref = np.kron(np.kron(_sequency_hadamard(T), _sequency_hadamard(M)), _sequency_hadamard(N))
    np.testing.assert_array_equal(phi, ref / math.sqrt(M * N * T))
    u = O.dictionary3("dct_wht", M, N, T)
    np.testing.assert_array_equal(u[M * N * T:], O.dictionary3("wht", M, N, T))


def test_weights3_integer_distances_and_masking():
    rho = 0.8
    sup = np.ones((5, 5, 5), dtype=np.uint8)
    sup[4, 4, 4] = 0
    w = O.weights3(5, 5, 5, rho, sup)
    assert w[2, 2, 2] == 1.0                                  # centre
    assert w[2, 2, 4] == pytest.approx(rho ** 2, rel=1e-15)   # axis
    assert w[3, 4, 4] == pytest.approx(rho ** 3, rel=1e-15)   # (1, 2, 2): distance 3
    assert w[4, 4, 4] == 0.0
    # T = 1 is the 2-D weighting and dictionary
    s2 = W.centred_support(8, 8)
    np.testing.assert_array_equal(O.weights3(8, 8, 1, rho, s2[None]), O.weights(8, 8, rho, s2)[None])
    np.testing.assert_array_equal(O.dictionary3("dct_wht", 8, 8, 1)[:, 0], O.dict_dct_wht(8, 8))


@pytest.mark.parametrize("basis,j", [("dct", 37), ("dct_wht", 300)])
def test_single_atom_closed_form_3d(basis, j):
    M, N, T = 8, 8, 4
    phi = O.flat(O.dictionary3(basis, M, N, T))
    dup = O.find_duplicates(phi)
    assert not dup[j]
    w = O.flat(O.weights3(M, N, T, 0.8, W.centred_support3(M, N, T)))
    a, gamma, I = 21.0, 0.5, 30
    r = O.se_original(phi, w, a * phi[j], gamma, I, dup)
    assert np.all(r.u == j)
    nu = np.arange(1, I + 1)
    np.testing.assert_allclose(r.c, gamma * (1 - gamma) ** (nu - 1) * a, rtol=1e-11)
    np.testing.assert_allclose(r.g, a * (1 - (1 - gamma) ** I) * phi[j], rtol=1e-11, atol=1e-12)


def test_fase_equals_se_on_a_video_block():
    M, N, T, I = 8, 8, 4, 40
    phi = O.flat(O.dictionary3("dct_wht", M, N, T))
    dup = O.find_duplicates(phi)
    w = O.flat(O.weights3(M, N, T, 0.8, W.centred_support3(M, N, T)))
    s = O.flat(W.video_block(M, N, T, 5))
    a = O.se_original(phi, w, s, 0.5, I, dup)
    Cm, D = O.fase_tables(phi, w)
    f = O.fase(phi, w, Cm, D, s, 0.5, I, dup)
    t = int(np.argmax(a.margin <= 1e-9)) if np.any(a.margin <= 1e-9) else I
    assert t >= 10
    np.testing.assert_array_equal(a.u[:t], f.u[:t])
    np.testing.assert_allclose(f.c[:t], a.c[:t], rtol=1e-10)
    # the energy drops monotonically, as in 2-D
    assert np.all(np.diff(a.energy) <= 1e-9 * a.energy[0])



# ---------------------------------------------------------- complex atoms
# The paper states SE and FaSE for complex-valued atoms (conjugated scalar
# products, Hermitian C); DFT and binarised DFT atoms are its complex examples.
@pytest.mark.parametrize("M,N", [(4, 4), (8, 6)])
def test_dft_atoms_give_numpy_fft2(M, N):
    phi = O.dict_complex("dft", M, N)
    x = np.random.default_rng(M * N).standard_normal((M, N)) + 1j * np.random.default_rng(7).standard_normal((M, N))
    R = np.einsum("kmn,mn->k", phi.conj(), x)          # sum x conj(phi_k)
    np.testing.assert_allclose(R, np.fft.fft2(x).ravel() / math.sqrt(M * N), atol=1e-12)
    G = np.einsum("kmn,lmn->kl", phi.conj(), phi)
    np.testing.assert_allclose(G, np.eye(M * N), atol=1e-13)


def test_binarised_dft_atoms_by_exact_phase():
    from fractions import Fraction
    M, N = 4, 6
    phi = O.dict_complex("bdft", M, N)
    s = 1.0 / math.sqrt(2 * M * N)
    for k in range(M * N):
        mu, eta = divmod(k, N)
        for m in range(M):
            for n in range(N):
                f = (Fraction(mu * m, M) + Fraction(eta * n, N)) % 1
                re = s if (f <= Fraction(1, 4) or f >= Fraction(3, 4)) else -s
                im = s if f <= Fraction(1, 2) else -s
                assert phi[k, m, n] == re + 1j * im, (k, m, n)
    u = O.dict_complex("dft_bdft", M, N)
    np.testing.assert_array_equal(u[M * N:], phi)


def test_complex_duplicates_match_brute_force():
    M = N = 8
    phi = O.dict_complex("dft_bdft", M, N).reshape(2 * M * N, M * N)
    nrm = np.linalg.norm(phi, axis=1)
    G = np.abs(phi.conj() @ phi.T)
    ref = np.zeros(len(phi), dtype=np.uint8)
    for j in range(1, len(phi)):
        ref[j] = np.any(G[:j, j] >= (1 - 1e-12) * nrm[:j] * nrm[j])
    ex = O.find_duplicates_c(phi.reshape(-1, M, N))
    np.testing.assert_array_equal(ex, ref)
    assert ex[M * N] == 1          # the binarised DC atom is (1 + j) times the DFT DC atom


@pytest.mark.parametrize("a", [37.5, 12.0 - 20.0j])
def test_complex_single_atom_closed_form(a):
    L, j, gamma, I = 16, 37, 0.5, 30
    phi = O.dict_complex("dft", L, L)
    w = O.weights(L, L, 0.8, W.centred_support(L, L))
    r = O.se_original_c(phi, w, a * phi[j], gamma, I)
    assert np.all(r.u == j)
    nu = np.arange(1, I + 1)
    np.testing.assert_allclose(r.c, gamma * (1 - gamma) ** (nu - 1) * a, rtol=1e-11)
    loss = w == 0
    np.testing.assert_allclose(r.out[loss], a * (1 - (1 - gamma) ** I) * phi[j][loss], rtol=1e-11, atol=1e-12)


def test_complex_unweighted_is_best_I_term_of_fft2():
    L, I = 8, 20
    rng = np.random.default_rng(3)
    s = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    w = np.ones((L, L))
    r = O.se_original_c(O.dict_complex("dft", L, L), w, s, 1.0, I)
    coef = np.fft.fft2(s).ravel() / L
    order = np.argsort(-np.abs(coef), kind="stable")[:I]
    np.testing.assert_array_equal(r.u, order)
    np.testing.assert_allclose(r.c, coef[order], rtol=1e-11)


def test_complex_fase_equals_se_and_energy_drops():
    L, I = 8, 40
    phi = O.dict_complex("dft_bdft", L, L)
    dup = O.find_duplicates_c(phi)
    w = O.weights(L, L, 0.8, W.centred_support(L, L))
    s = W.patch(L, 11)
    a = O.se_original_c(phi, w, s, 0.5, I, dup)
    f = O.fase_c(phi, w, s, 0.5, I, dup)
    t = int(np.argmax(a.margin <= 1e-9)) if np.any(a.margin <= 1e-9) else I
    assert t >= 10
    np.testing.assert_array_equal(a.u[:t], f.u[:t])
    np.testing.assert_allclose(f.c[:t], a.c[:t], rtol=1e-10)
    assert np.all(np.diff(a.energy) <= 1e-9 * a.energy[0])
