/*
 * se_oracle.c -- plain FP64 CPU oracle for Selective Extrapolation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with
 * the CUDA library: it builds its own weighting function and its own DCT /
 * WHT atoms, and it implements the method from the paper's equations with
 * straightforward loops in double precision, so that a reader can check each
 * step against the paper by eye.
 *
 * Contents (Seiler & Kaup, "A Fast Algorithm for Selective Signal
 * Extrapolation with Arbitrary Basis Functions"):
 *   or_weights            eq. (4)-(5)   weighting function w = rho on A, 0 on B
 *   or_dict_dct/wht       Sec. I        example dictionaries (normalisation and
 *                                       ordering are this oracle's reading)
 *   or_weights3, or_dict_*3             the same for M x N x T (video) blocks,
 *                                       the 3-D extension the paper names in
 *                                       its conclusion
 *   or_dict_dft/bdft, or_*_c            complex-valued atoms (DFT, binarised
 *                                       DFT) and Alg. 1-3 with conjugates,
 *                                       the paper's general case
 *   or_find_duplicates                  collinear atoms (reading: only the
 *                                       lowest index of a collinear group
 *                                       may be selected)
 *   or_projection_state   eq. (3),(6),(7) p_k, C_kk, e_k for one residual
 *   or_se_original        Alg. 1        the original SE, eqs. (2)-(10)
 *   or_fase_tables        Alg. 2        tables C_(k,l), D_k, eqs. (16)-(17)
 *   or_fase               Alg. 3        Fast SE, eqs. (12), (18)-(20)
 *   or_*_batch                          loops over blocks (OpenMP over blocks
 *                                       only; the per-block arithmetic is the
 *                                       single-block function unchanged)
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - ties in the argmax go to the smallest index k;
 *   - an atom whose weighted energy C_kk is <= 1e-14 * max_j C_jj cannot be
 *     selected (its projection would divide by ~0);
 *   - an atom collinear (over the whole area L) with an atom of lower index
 *     cannot be selected;
 *   - if every admissible score is 0 the smallest admissible k is taken with
 *     coefficient 0; the loop always runs exactly I iterations;
 *   - the residual starts as s on A and 0 on B, so whatever B holds is never
 *     read (w is 0 there, eq. 4, so this changes no scalar product).
 *
 * Array layouts: an area is M x N row-major (m = row).  A dictionary is
 * atom-major: phi[k * MN + m * N + n].  C is K x K row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXCLUDE_REL 1e-14
#define OR_COLLINEAR_REL 1e-12

/* ---------------------------------------------------------------- eq. 4-5 */

/* w[m,n] = rho_hat ^ sqrt((m-(M-1)/2)^2 + (n-(N-1)/2)^2) on A, 0 on B.
 * If rho is non-NULL it replaces the isotropic decay of eq. (5). */
void or_weights(int M, int N, double rho_hat, const uint8_t *support,
                const double *rho, double *w)
{
    for (int m = 0; m < M; ++m) {
        for (int n = 0; n < N; ++n) {
            double dm = m - (M - 1) / 2.0;
            double dn = n - (N - 1) / 2.0;
            double r = rho ? rho[m * N + n] : pow(rho_hat, sqrt(dm * dm + dn * dn));
            w[m * N + n] = support[m * N + n] ? r : 0.0;
        }
    }
}

/* ------------------------------------------------------------ dictionaries */

/* 2-D orthonormal DCT-II atom (p, q) at (m, n); k = p * N + q. */
void or_dict_dct(int M, int N, double *phi)
{
    const double pi = 3.14159265358979323846;
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < N; ++q) {
            double ap = p == 0 ? sqrt(1.0 / M) : sqrt(2.0 / M);
            double aq = q == 0 ? sqrt(1.0 / N) : sqrt(2.0 / N);
            double *a = phi + (size_t)(p * N + q) * M * N;
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < N; ++n)
                    a[m * N + n] = ap * aq * cos(pi * (2 * m + 1) * p / (2.0 * M))
                                           * cos(pi * (2 * n + 1) * q / (2.0 * N));
        }
}

/* Rows of the natural-order Hadamard matrix of size L (a power of two):
 * H[i][j] = (-1)^popcount(i & j).  The Walsh function of sequency p is the
 * Hadamard row with exactly p sign changes; it is found by counting. */
static void walsh_rows(int L, double *W /* L x L, row p = sequency p */)
{
    for (int i = 0; i < L; ++i) {
        int changes = 0;
        int prev = 1;
        for (int j = 0; j < L; ++j) {
            int bits = i & j, par = 0;
            while (bits) { par ^= bits & 1; bits >>= 1; }
            int v = par ? -1 : 1;
            if (j > 0 && v != prev) ++changes;
            prev = v;
        }
        for (int j = 0; j < L; ++j) {
            int bits = i & j, par = 0;
            while (bits) { par ^= bits & 1; bits >>= 1; }
            W[changes * L + j] = par ? -1.0 : 1.0;
        }
    }
}

/* 2-D WHT atom (p, q) = wal_p[m] * wal_q[n] / sqrt(MN), sequency order;
 * k = p * N + q.  M and N must be powers of two.  Returns 0 on success. */
int or_dict_wht(int M, int N, double *phi)
{
    if (M <= 0 || N <= 0 || (M & (M - 1)) || (N & (N - 1))) return -1;
    double *wm = malloc(sizeof(double) * M * M);
    double *wn = malloc(sizeof(double) * N * N);
    if (!wm || !wn) { free(wm); free(wn); return -2; }
    walsh_rows(M, wm);
    walsh_rows(N, wn);
    double s = 1.0 / sqrt((double)M * N);
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < N; ++q) {
            double *a = phi + (size_t)(p * N + q) * M * N;
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < N; ++n)
                    a[m * N + n] = wm[p * M + m] * wn[q * N + n] * s;
        }
    free(wm);
    free(wn);
    return 0;
}

/* DCT atoms at k in [0, MN), WHT atoms at k in [MN, 2MN). */
int or_dict_dct_wht(int M, int N, double *phi)
{
    or_dict_dct(M, N, phi);
    return or_dict_wht(M, N, phi + (size_t)M * N * M * N);
}

/* ------------------------------------------------ 3-D areas (video blocks) */
/* The method itself does not depend on the dimension of the area (Sec. II
 * works on any set of sample positions); for an M x N x T block the samples
 * are stored frame-major, index (t * M + m) * N + n, and the functions of
 * Alg. 1-3 below run unchanged on the flattened area.  Only the weighting
 * function and the example dictionaries need the third coordinate. */

/* eq. (5) with the distance to the centre of the M x N x T block. */
void or_weights3(int M, int N, int T, double rho_hat, const uint8_t *support, const double *rho,
                 double *w)
{
    for (int t = 0; t < T; ++t)
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < N; ++n) {
                const size_t i = ((size_t)t * M + m) * N + n;
                double dt = t - (T - 1) / 2.0, dm = m - (M - 1) / 2.0, dn = n - (N - 1) / 2.0;
                double r = rho ? rho[i] : pow(rho_hat, sqrt(dt * dt + dm * dm + dn * dn));
                w[i] = support[i] ? r : 0.0;
            }
}

/* 3-D orthonormal DCT-II atom (r, p, q) at (t, m, n); k = (r * M + p) * N + q. */
void or_dict_dct3(int M, int N, int T, double *phi)
{
    const double pi = 3.14159265358979323846;
    const size_t V = (size_t)M * N * T;
    for (int r = 0; r < T; ++r)
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < N; ++q) {
                double ar = r == 0 ? sqrt(1.0 / T) : sqrt(2.0 / T);
                double ap = p == 0 ? sqrt(1.0 / M) : sqrt(2.0 / M);
                double aq = q == 0 ? sqrt(1.0 / N) : sqrt(2.0 / N);
                double *a = phi + ((size_t)r * M * N + (size_t)p * N + q) * V;
                for (int t = 0; t < T; ++t)
                    for (int m = 0; m < M; ++m)
                        for (int n = 0; n < N; ++n)
                            a[((size_t)t * M + m) * N + n] =
                                ar * ap * aq * cos(pi * (2 * t + 1) * r / (2.0 * T)) *
                                cos(pi * (2 * m + 1) * p / (2.0 * M)) * cos(pi * (2 * n + 1) * q / (2.0 * N));
            }
}

/* 3-D WHT atom (r, p, q) = wal_r[t] wal_p[m] wal_q[n] / sqrt(MNT), sequency
 * order, k = (r * M + p) * N + q; M, N, T powers of two.  Returns 0 on success. */
int or_dict_wht3(int M, int N, int T, double *phi)
{
    if (M <= 0 || N <= 0 || T <= 0 || (M & (M - 1)) || (N & (N - 1)) || (T & (T - 1))) return -1;
    double *wm = malloc(sizeof(double) * M * M);
    double *wn = malloc(sizeof(double) * N * N);
    double *wt = malloc(sizeof(double) * T * T);
    if (!wm || !wn || !wt) { free(wm); free(wn); free(wt); return -2; }
    walsh_rows(M, wm);
    walsh_rows(N, wn);
    walsh_rows(T, wt);
    const size_t V = (size_t)M * N * T;
    double s = 1.0 / sqrt((double)V);
    for (int r = 0; r < T; ++r)
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < N; ++q) {
                double *a = phi + ((size_t)r * M * N + (size_t)p * N + q) * V;
                for (int t = 0; t < T; ++t)
                    for (int m = 0; m < M; ++m)
                        for (int n = 0; n < N; ++n)
                            a[((size_t)t * M + m) * N + n] = wt[r * T + t] * wm[p * M + m] * wn[q * N + n] * s;
            }
    free(wm);
    free(wn);
    free(wt);
    return 0;
}

/* 3-D DCT atoms at k in [0, MNT), 3-D WHT atoms at k in [MNT, 2MNT). */
int or_dict_dct_wht3(int M, int N, int T, double *phi)
{
    or_dict_dct3(M, N, T, phi);
    return or_dict_wht3(M, N, T, phi + (size_t)M * N * T * M * N * T);
}

/* excluded[j] = 1 if atom j is collinear over L with an atom i < j:
 * |<phi_i, phi_j>| >= (1 - 1e-12) * |phi_i| * |phi_j|.  For such a pair the
 * unit-norm atoms differ (up to sign) by at most sqrt(2e-12) < 1.5e-6 in l2,
 * so a pair whose normalised magnitudes differ by more than 1e-5 at one of
 * the first pixels cannot be collinear and is skipped before the full
 * inner product. */
void or_find_duplicates(int K, int MN, const double *phi, uint8_t *excluded)
{
    double *nrm = malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int p = 0; p < MN; ++p) s += phi[(size_t)k * MN + p] * phi[(size_t)k * MN + p];
        nrm[k] = sqrt(s);
        excluded[k] = 0;
    }
    int probe = MN < 4 ? MN : 4;
    for (int j = 1; j < K; ++j) {
        for (int i = 0; i < j && !excluded[j]; ++i) {
            if (excluded[i] || nrm[i] == 0.0 || nrm[j] == 0.0) continue;
            int maybe = 1;
            for (int p = 0; p < probe; ++p) {
                double a = fabs(phi[(size_t)i * MN + p]) / nrm[i];
                double b = fabs(phi[(size_t)j * MN + p]) / nrm[j];
                if (fabs(a - b) > 1e-5) { maybe = 0; break; }
            }
            if (!maybe) continue;
            double d = 0.0;
            for (int p = 0; p < MN; ++p) d += phi[(size_t)i * MN + p] * phi[(size_t)j * MN + p];
            if (fabs(d) >= (1.0 - OR_COLLINEAR_REL) * nrm[i] * nrm[j]) excluded[j] = 1;
        }
    }
    free(nrm);
}

/* ------------------------------------------------------------ eq. 3, 6, 7 */

/* For residual r: num_k = sum r phi_k w, den_k = sum phi_k w phi_k = C_kk,
 * p_k = num_k / den_k (eq. 3), e_k = sum w (r - p_k phi_k)^2 (eq. 6) and
 * score_k = p_k^2 C_kk (eq. 7).  Any output pointer may be NULL. */
void or_projection_state(int MN, int K, const double *phi, const double *w,
                         const double *r, double *p, double *ckk, double *e,
                         double *score)
{
    for (int k = 0; k < K; ++k) {
        const double *a = phi + (size_t)k * MN;
        double num = 0.0, den = 0.0;
        for (int i = 0; i < MN; ++i) {
            num += r[i] * a[i] * w[i];
            den += a[i] * w[i] * a[i];
        }
        double pk = den > 0.0 ? num / den : 0.0;
        if (p) p[k] = pk;
        if (ckk) ckk[k] = den;
        if (score) score[k] = pk * pk * den;
        if (e) {
            double ek = 0.0;
            for (int i = 0; i < MN; ++i) {
                double d = r[i] - pk * a[i];
                ek += d * d * w[i];
            }
            e[k] = ek;
        }
    }
}

/* Which atoms may be selected: not collinear with a lower index, and with
 * C_kk above 1e-14 of the largest C_jj.  Returns the admissible count. */
static int admissible(int K, const double *ckk, const uint8_t *dup, uint8_t *ok)
{
    double mx = 0.0;
    for (int k = 0; k < K; ++k) if (ckk[k] > mx) mx = ckk[k];
    int n = 0;
    for (int k = 0; k < K; ++k) {
        ok[k] = (!dup || !dup[k]) && ckk[k] > OR_EXCLUDE_REL * mx && mx > 0.0;
        n += ok[k];
    }
    return n;
}

/* ------------------------------------------------------------------ Alg. 1 */

/* Original Selective Extrapolation for one block.
 *   s        M x N samples (values on B are never read)
 *   w        M x N weighting function (eq. 4), 0 exactly on B
 *   phi      K atoms, atom-major
 *   dup      K flags from or_find_duplicates (NULL: none)
 *   selector 0: u = argmax p_k^2 C_kk (eq. 7);  1: u = argmin e_k (eq. 6),
 *            evaluated literally from the residual (brute force)
 * Outputs (each may be NULL except out):
 *   out      M x N: s on A, model g on B (final replacement step)
 *   g_full   M x N: the model g over all of L (eq. 1)
 *   r_final  M x N: the final residual r^(I)
 *   u_log, c_log   selected index u and coefficient c of each iteration
 *   e_log    weighted residual energy E = sum w r^2 after each iteration
 *   margin_log  (s1 - s2) / s1 over the two best admissible scores
 * Returns 0, or -5 if no atom is admissible (empty support). */
int or_se_original(int M, int N, int K, const double *phi, const double *w,
                   const uint8_t *dup, const double *s, double gamma, int I,
                   int selector, double *out, double *g_full, double *r_final,
                   int32_t *u_log, double *c_log, double *e_log,
                   double *margin_log)
{
    const int MN = M * N;
    double *r = malloc(sizeof(double) * MN);
    double *g = calloc(MN, sizeof(double));
    double *p = malloc(sizeof(double) * K);
    double *ckk = malloc(sizeof(double) * K);
    double *e = malloc(sizeof(double) * K);
    double *sc = malloc(sizeof(double) * K);
    uint8_t *ok = malloc(K);
    int rc = 0;

    /* eq. (2): r^(0) = s (on A; B is masked by w = 0 and never read) */
    for (int i = 0; i < MN; ++i) r[i] = w[i] > 0.0 ? s[i] : 0.0;

    or_projection_state(MN, K, phi, w, r, NULL, ckk, NULL, NULL);
    if (admissible(K, ckk, dup, ok) == 0) { rc = -5; goto done; }

    for (int nu = 1; nu <= I; ++nu) {
        /* eq. (3) for every k; eq. (6) only for the brute-force selector */
        or_projection_state(MN, K, phi, w, r, p, NULL, selector ? e : NULL, sc);

        int u = -1;
        double best = 0.0;
        for (int k = 0; k < K; ++k) {
            if (!ok[k]) continue;
            double v = selector ? -e[k] : sc[k];    /* argmin e == argmax -e */
            if (u < 0 || v > best) { best = v; u = k; }
        }
        if (margin_log) {
            /* margin over the eq. (7) scores, whichever selector was used */
            double s1 = -1.0, s2 = -1.0;
            for (int k = 0; k < K; ++k) {
                if (!ok[k]) continue;
                if (sc[k] > s1) { s2 = s1; s1 = sc[k]; }
                else if (sc[k] > s2) s2 = sc[k];
            }
            margin_log[nu - 1] = s1 > 0.0 ? (s1 - (s2 < 0.0 ? 0.0 : s2)) / s1 : 0.0;
        }

        /* eq. (8): fast orthogonality deficiency compensation */
        double c = gamma * p[u];

        /* eqs. (9)-(10): model and residual update */
        const double *a = phi + (size_t)u * MN;
        for (int i = 0; i < MN; ++i) {
            g[i] += c * a[i];
            r[i] -= c * a[i];
        }
        if (u_log) u_log[nu - 1] = u;
        if (c_log) c_log[nu - 1] = c;
        if (e_log) {
            double E = 0.0;
            for (int i = 0; i < MN; ++i) E += w[i] * r[i] * r[i];
            e_log[nu - 1] = E;
        }
    }

done:
    /* replacement of B by the model */
    for (int i = 0; i < MN; ++i) out[i] = w[i] > 0.0 ? s[i] : g[i];
    if (g_full) memcpy(g_full, g, sizeof(double) * MN);
    if (r_final) memcpy(r_final, r, sizeof(double) * MN);
    free(r); free(g); free(p); free(ckk); free(e); free(sc); free(ok);
    return rc;
}

/* ------------------------------------------------------------------ Alg. 2 */

/* C_(k,l) = sum phi_k w phi_l for l >= k, mirrored (eq. 16);
 * D_k = 1 / sqrt(C_kk) (eq. 17). */
void or_fase_tables(int M, int N, int K, const double *phi, const double *w,
                    double *C, double *D)
{
    const int MN = M * N;
    for (int k = 0; k < K; ++k) {
        const double *a = phi + (size_t)k * MN;
        for (int l = k; l < K; ++l) {
            const double *b = phi + (size_t)l * MN;
            double acc = 0.0;
            for (int i = 0; i < MN; ++i) acc += a[i] * w[i] * b[i];
            C[(size_t)k * K + l] = acc;
            C[(size_t)l * K + k] = acc;
        }
        D[k] = C[(size_t)k * K + k] > 0.0 ? 1.0 / sqrt(C[(size_t)k * K + k]) : 0.0;
    }
}

/* ------------------------------------------------------------------ Alg. 3 */

/* Fast Selective Extrapolation for one block, given the tables of Alg. 2.
 * Same argument meaning as or_se_original; R_final (K, may be NULL)
 * receives the running scalar products R_k^(I). */
int or_fase(int M, int N, int K, const double *phi, const double *w,
            const double *C, const double *D, const uint8_t *dup,
            const double *s, double gamma, int I, double *out, double *g_full,
            double *R_final, int32_t *u_log, double *c_log)
{
    const int MN = M * N;
    double *R = malloc(sizeof(double) * K);
    double *g = calloc(MN, sizeof(double));
    double *ckk = malloc(sizeof(double) * K);
    uint8_t *ok = malloc(K);
    int rc = 0;

    for (int k = 0; k < K; ++k) ckk[k] = C[(size_t)k * K + k];
    if (admissible(K, ckk, dup, ok) == 0) { rc = -5; goto done; }

    /* eq. (12): R_k^(0) = sum s phi_k w */
    for (int k = 0; k < K; ++k) {
        const double *a = phi + (size_t)k * MN;
        double acc = 0.0;
        for (int i = 0; i < MN; ++i) acc += (w[i] > 0.0 ? s[i] : 0.0) * a[i] * w[i];
        R[k] = acc;
    }

    for (int nu = 1; nu <= I; ++nu) {
        /* eq. (18): u = argmax |R_k| D_k */
        int u = -1;
        double best = 0.0;
        for (int k = 0; k < K; ++k) {
            if (!ok[k]) continue;
            double v = fabs(R[k]) * D[k];
            if (u < 0 || v > best) { best = v; u = k; }
        }
        /* eq. (19): c = gamma R_u D_u^2 */
        double c = gamma * R[u] * D[u] * D[u];
        /* eq. (9): model update */
        const double *a = phi + (size_t)u * MN;
        for (int i = 0; i < MN; ++i) g[i] += c * a[i];
        /* eq. (20): R_k -= c C_(k,u) */
        for (int k = 0; k < K; ++k) R[k] -= c * C[(size_t)k * K + u];
        if (u_log) u_log[nu - 1] = u;
        if (c_log) c_log[nu - 1] = c;
    }

done:
    for (int i = 0; i < MN; ++i) out[i] = w[i] > 0.0 ? s[i] : g[i];
    if (g_full) memcpy(g_full, g, sizeof(double) * MN);
    if (R_final) memcpy(R_final, R, sizeof(double) * K);
    free(R); free(g); free(ckk); free(ok);
    return rc;
}

/* ----------------------------------------------------------------- batches */

/* Original SE over B blocks.  Block b uses samples s + b*MN, weights
 * w + (w_stride ? b*MN : 0) and iteration count iters[b] (or I if iters is
 * NULL); logs (u, c, tie margin) are [B, I] row-major with stride I.  nthreads <= 0
 * lets OpenMP decide.  Returns the first non-zero block status, else 0. */
int or_se_original_batch(int B, int M, int N, int K, const double *phi,
                         const double *w, int w_stride, const uint8_t *dup,
                         const double *s, double gamma, int I,
                         const int32_t *iters, double *out, int32_t *u_log,
                         double *c_log, double *margin_log, int nthreads)
{
    const int MN = M * N;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b) {
        int Ib = iters ? iters[b] : I;
        int rc = or_se_original(M, N, K, phi, w + (w_stride ? (size_t)b * MN : 0), dup,
                                s + (size_t)b * MN, gamma, Ib, 0, out + (size_t)b * MN,
                                NULL, NULL, u_log ? u_log + (size_t)b * I : NULL,
                                c_log ? c_log + (size_t)b * I : NULL, NULL,
                                margin_log ? margin_log + (size_t)b * I : NULL);
        if (rc) {
#ifdef _OPENMP
#pragma omp critical
#endif
            if (!status) status = rc;
        }
    }
    return status;
}

/* Fast SE over B blocks that share one weighting pattern and its tables. */
int or_fase_batch(int B, int M, int N, int K, const double *phi, const double *w,
                  const double *C, const double *D, const uint8_t *dup,
                  const double *s, double gamma, int I, double *out,
                  int32_t *u_log, double *c_log, int nthreads)
{
    const int MN = M * N;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b) {
        int rc = or_fase(M, N, K, phi, w, C, D, dup, s + (size_t)b * MN, gamma, I,
                         out + (size_t)b * MN, NULL, NULL,
                         u_log ? u_log + (size_t)b * I : NULL,
                         c_log ? c_log + (size_t)b * I : NULL);
        if (rc) {
#ifdef _OPENMP
#pragma omp critical
#endif
            if (!status) status = rc;
        }
    }
    return status;
}

/* ----------------------------------------------- complex-valued atoms */
/* The paper states SE and FaSE for complex-valued signals and atoms (Sec. II
 * and III): the scalar products use the conjugated atom, the selection takes
 * |R_k| D_k, the coefficient is complex and C is Hermitian.  Complex arrays
 * are kept as separate real and imaginary planes ("_re", "_im").  Signals in
 * the tests are real images or, for the closed-form pin, a complex atom. */

/* 2-D DFT atom (mu, eta): exp(j 2 pi (mu m / M + eta n / N)) / sqrt(MN),
 * k = mu * N + eta.  The phase is reduced exactly in integers,
 * theta = 2 pi a / (MN) with a = (mu m N + eta n M) mod MN. */
void or_dict_dft(int M, int N, double *re, double *im)
{
    const double pi = 3.14159265358979323846;
    const long L = (long)M * N;
    const double s = 1.0 / sqrt((double)L);
    for (int mu = 0; mu < M; ++mu)
        for (int eta = 0; eta < N; ++eta) {
            const size_t k = (size_t)mu * N + eta;
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < N; ++n) {
                    long a = ((long)mu * m * N + (long)eta * n * M) % L;
                    re[k * L + (size_t)m * N + n] = s * cos(2.0 * pi * a / L);
                    im[k * L + (size_t)m * N + n] = s * sin(2.0 * pi * a / L);
                }
        }
}

/* Binarised DFT atom (reading of "a binarized version of DFT functions"):
 * sgn(cos theta) + j sgn(sin theta) with sgn(0) = +1, decided exactly on the
 * integer phase a of or_dict_dft (cos >= 0 iff 4a <= L or 4a >= 3L;
 * sin >= 0 iff 2a <= L), scaled to unit norm by 1 / sqrt(2 MN). */
void or_dict_bdft(int M, int N, double *re, double *im)
{
    const long L = (long)M * N;
    const double s = 1.0 / sqrt(2.0 * (double)L);
    for (int mu = 0; mu < M; ++mu)
        for (int eta = 0; eta < N; ++eta) {
            const size_t k = (size_t)mu * N + eta;
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < N; ++n) {
                    long a = ((long)mu * m * N + (long)eta * n * M) % L;
                    re[k * L + (size_t)m * N + n] = (4 * a <= L || 4 * a >= 3 * L) ? s : -s;
                    im[k * L + (size_t)m * N + n] = (2 * a <= L) ? s : -s;
                }
        }
}

/* DFT atoms at k in [0, MN), binarised DFT atoms at k in [MN, 2MN). */
void or_dict_dft_bdft(int M, int N, double *re, double *im)
{
    const size_t V = (size_t)M * N;
    or_dict_dft(M, N, re, im);
    or_dict_bdft(M, N, re + V * V, im + V * V);
}

/* Complex collinearity: excluded[j] = 1 if |<phi_i, phi_j>| >= (1 - 1e-12)
 * |phi_i| |phi_j| for some i < j, with <a, b> = sum conj(a) b (plain double
 * loop over all pairs; the complex dictionaries of the tests are small). */
void or_find_duplicates_c(int K, int MN, const double *re, const double *im, uint8_t *excluded)
{
    double *nrm = malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int p = 0; p < MN; ++p) {
            const size_t i = (size_t)k * MN + p;
            s += re[i] * re[i] + im[i] * im[i];
        }
        nrm[k] = sqrt(s);
        excluded[k] = 0;
    }
    for (int j = 1; j < K; ++j) {
        if (nrm[j] == 0.0) continue;
        for (int i = 0; i < j && !excluded[j]; ++i) {
            if (nrm[i] == 0.0) continue;
            double dr = 0.0, di = 0.0;
            for (int p = 0; p < MN; ++p) {
                const size_t a = (size_t)i * MN + p, b = (size_t)j * MN + p;
                dr += re[a] * re[b] + im[a] * im[b];
                di += re[a] * im[b] - im[a] * re[b];
            }
            if (sqrt(dr * dr + di * di) >= (1.0 - OR_COLLINEAR_REL) * nrm[i] * nrm[j]) excluded[j] = 1;
        }
    }
    free(nrm);
}

/* Alg. 1 with complex atoms (eqs. 2-10 with conjugates).  s is complex
 * (s_im may be NULL for a real signal).  out_re/out_im: s on A, g on B;
 * u_log, c_re/c_im (complex coefficient), margin_log as in or_se_original.
 * Returns 0, or -5 if no atom is admissible. */
int or_se_original_c(int M, int N, int K, const double *re, const double *im, const double *w,
                     const uint8_t *dup, const double *s_re, const double *s_im, double gamma, int I,
                     double *out_re, double *out_im, int32_t *u_log, double *c_re, double *c_im,
                     double *e_log, double *margin_log)
{
    const int MN = M * N;
    double *rr = malloc(sizeof(double) * MN), *ri = malloc(sizeof(double) * MN);
    double *gr = calloc(MN, sizeof(double)), *gi = calloc(MN, sizeof(double));
    double *ckk = malloc(sizeof(double) * K), *pr = malloc(sizeof(double) * K), *pi_ = malloc(sizeof(double) * K);
    double *sc = malloc(sizeof(double) * K);
    uint8_t *ok = malloc(K);
    int rc = 0;

    /* eq. (2): r^(0) = s on A (B never read) */
    for (int i = 0; i < MN; ++i) {
        rr[i] = w[i] > 0.0 ? s_re[i] : 0.0;
        ri[i] = w[i] > 0.0 && s_im ? s_im[i] : 0.0;
    }
    /* denominator of eq. (3): sum conj(phi_k) w phi_k */
    for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int i = 0; i < MN; ++i) {
            const size_t a = (size_t)k * MN + i;
            acc += (re[a] * re[a] + im[a] * im[a]) * w[i];
        }
        ckk[k] = acc;
    }
    if (admissible(K, ckk, dup, ok) == 0) { rc = -5; goto done; }

    for (int nu = 1; nu <= I; ++nu) {
        /* eq. (3): p_k = sum r conj(phi_k) w / C_kk; eq. (7): score |p_k|^2 C_kk */
        for (int k = 0; k < K; ++k) {
            double nr = 0.0, ni = 0.0;
            for (int i = 0; i < MN; ++i) {
                const size_t a = (size_t)k * MN + i;
                /* r * conj(phi) = (rr + j ri)(pr - j pi) */
                nr += (rr[i] * re[a] + ri[i] * im[a]) * w[i];
                ni += (ri[i] * re[a] - rr[i] * im[a]) * w[i];
            }
            pr[k] = ckk[k] > 0.0 ? nr / ckk[k] : 0.0;
            pi_[k] = ckk[k] > 0.0 ? ni / ckk[k] : 0.0;
            sc[k] = (pr[k] * pr[k] + pi_[k] * pi_[k]) * ckk[k];
        }
        int u = -1;
        double best = 0.0;
        for (int k = 0; k < K; ++k) {
            if (!ok[k]) continue;
            if (u < 0 || sc[k] > best) { best = sc[k]; u = k; }
        }
        if (margin_log) {
            double s1 = -1.0, s2 = -1.0;
            for (int k = 0; k < K; ++k) {
                if (!ok[k]) continue;
                if (sc[k] > s1) { s2 = s1; s1 = sc[k]; }
                else if (sc[k] > s2) s2 = sc[k];
            }
            margin_log[nu - 1] = s1 > 0.0 ? (s1 - (s2 < 0.0 ? 0.0 : s2)) / s1 : 0.0;
        }
        /* eq. (8) */
        const double cr = gamma * pr[u], ci = gamma * pi_[u];
        /* eqs. (9)-(10): g += c phi_u, r -= c phi_u */
        for (int i = 0; i < MN; ++i) {
            const size_t a = (size_t)u * MN + i;
            const double vr = cr * re[a] - ci * im[a], vi = cr * im[a] + ci * re[a];
            gr[i] += vr; gi[i] += vi;
            rr[i] -= vr; ri[i] -= vi;
        }
        if (u_log) u_log[nu - 1] = u;
        if (c_re) c_re[nu - 1] = cr;
        if (c_im) c_im[nu - 1] = ci;
        if (e_log) {
            double E = 0.0;
            for (int i = 0; i < MN; ++i) E += w[i] * (rr[i] * rr[i] + ri[i] * ri[i]);
            e_log[nu - 1] = E;
        }
    }
done:
    for (int i = 0; i < MN; ++i) {
        out_re[i] = w[i] > 0.0 ? s_re[i] : gr[i];
        if (out_im) out_im[i] = w[i] > 0.0 ? (s_im ? s_im[i] : 0.0) : gi[i];
    }
    free(rr); free(ri); free(gr); free(gi); free(ckk); free(pr); free(pi_); free(sc); free(ok);
    return rc;
}

/* Alg. 2 + 3 with complex atoms: C_(k,l) = sum conj(phi_k) w phi_l (Hermitian),
 * R_k^(0) = sum s conj(phi_k) w, u = argmax |R_k| D_k, c = gamma R_u D_u^2,
 * R_k -= c C_(k,u).  Outputs as or_se_original_c (no energy / margins). */
int or_fase_c(int M, int N, int K, const double *re, const double *im, const double *w,
              const uint8_t *dup, const double *s_re, const double *s_im, double gamma, int I,
              double *out_re, double *out_im, int32_t *u_log, double *c_re, double *c_im)
{
    const int MN = M * N;
    double *Cr = malloc(sizeof(double) * K * K), *Ci = malloc(sizeof(double) * K * K);
    double *Rr = malloc(sizeof(double) * K), *Ri = malloc(sizeof(double) * K);
    double *D = malloc(sizeof(double) * K), *ckk = malloc(sizeof(double) * K);
    double *gr = calloc(MN, sizeof(double)), *gi = calloc(MN, sizeof(double));
    uint8_t *ok = malloc(K);
    int rc = 0;
    /* Alg. 2: eq. (16) on the upper triangle, Hermitian mirror; eq. (17) */
    for (int k = 0; k < K; ++k)
        for (int l = k; l < K; ++l) {
            double ar = 0.0, ai = 0.0;
            for (int i = 0; i < MN; ++i) {
                const size_t a = (size_t)k * MN + i, b = (size_t)l * MN + i;
                ar += (re[a] * re[b] + im[a] * im[b]) * w[i];
                ai += (re[a] * im[b] - im[a] * re[b]) * w[i];
            }
            Cr[(size_t)k * K + l] = ar; Ci[(size_t)k * K + l] = ai;
            Cr[(size_t)l * K + k] = ar; Ci[(size_t)l * K + k] = -ai;
        }
    for (int k = 0; k < K; ++k) {
        ckk[k] = Cr[(size_t)k * K + k];
        D[k] = ckk[k] > 0.0 ? 1.0 / sqrt(ckk[k]) : 0.0;
    }
    if (admissible(K, ckk, dup, ok) == 0) { rc = -5; goto done; }
    /* eq. (12) */
    for (int k = 0; k < K; ++k) {
        double ar = 0.0, ai = 0.0;
        for (int i = 0; i < MN; ++i) {
            if (!(w[i] > 0.0)) continue;
            const size_t a = (size_t)k * MN + i;
            const double sr = s_re[i], si = s_im ? s_im[i] : 0.0;
            ar += (sr * re[a] + si * im[a]) * w[i];
            ai += (si * re[a] - sr * im[a]) * w[i];
        }
        Rr[k] = ar; Ri[k] = ai;
    }
    for (int nu = 1; nu <= I; ++nu) {
        int u = -1;
        double best = 0.0;
        for (int k = 0; k < K; ++k) {   /* eq. (18) */
            if (!ok[k]) continue;
            double v = sqrt(Rr[k] * Rr[k] + Ri[k] * Ri[k]) * D[k];
            if (u < 0 || v > best) { best = v; u = k; }
        }
        const double cr = gamma * Rr[u] * D[u] * D[u], ci = gamma * Ri[u] * D[u] * D[u];   /* eq. (19) */
        for (int i = 0; i < MN; ++i) {   /* eq. (9) */
            const size_t a = (size_t)u * MN + i;
            gr[i] += cr * re[a] - ci * im[a];
            gi[i] += cr * im[a] + ci * re[a];
        }
        for (int k = 0; k < K; ++k) {    /* eq. (20): R_k -= c C_(k,u) */
            const double xr = Cr[(size_t)k * K + u], xi = Ci[(size_t)k * K + u];
            Rr[k] -= cr * xr - ci * xi;
            Ri[k] -= cr * xi + ci * xr;
        }
        if (u_log) u_log[nu - 1] = u;
        if (c_re) c_re[nu - 1] = cr;
        if (c_im) c_im[nu - 1] = ci;
    }
done:
    for (int i = 0; i < MN; ++i) {
        out_re[i] = w[i] > 0.0 ? s_re[i] : gr[i];
        if (out_im) out_im[i] = w[i] > 0.0 ? (s_im ? s_im[i] : 0.0) : gi[i];
    }
    free(Cr); free(Ci); free(Rr); free(Ri); free(D); free(ckk); free(gr); free(gi); free(ok);
    return rc;
}

/* Complex Alg. 1 over B real-valued blocks (one pattern or per-block w). */
int or_se_original_c_batch(int B, int M, int N, int K, const double *re, const double *im,
                           const double *w, int w_stride, const uint8_t *dup, const double *s,
                           double gamma, int I, double *out_re, int32_t *u_log, double *c_re,
                           double *c_im, double *margin_log, int nthreads)
{
    const int MN = M * N;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b) {
        int rc = or_se_original_c(M, N, K, re, im, w + (w_stride ? (size_t)b * MN : 0), dup,
                                  s + (size_t)b * MN, NULL, gamma, I, out_re + (size_t)b * MN, NULL,
                                  u_log ? u_log + (size_t)b * I : NULL, c_re ? c_re + (size_t)b * I : NULL,
                                  c_im ? c_im + (size_t)b * I : NULL, NULL,
                                  margin_log ? margin_log + (size_t)b * I : NULL);
        if (rc) {
#ifdef _OPENMP
#pragma omp critical
#endif
            if (!status) status = rc;
        }
    }
    return status;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
