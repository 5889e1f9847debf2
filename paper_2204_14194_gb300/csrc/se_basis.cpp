// se_basis.cpp -- host-side construction of the method's inputs for a plan:
// the dictionaries named by se_basis, the weighting function of eqs. (4)-(5)
// and the collinear-duplicate flags that make ties go to the smallest index.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <random>
#include <vector>

#include "se_host.h"

namespace se {

// 2-D orthonormal DCT-II, atom (p, q) at index p*N + q (separable product of
// the 1-D DCT-II rows with the sqrt(1/L) / sqrt(2/L) normalisation).
void dct_rows(int L, std::vector<double> &T)
{
    const double pi = 3.14159265358979323846;
    T.assign(static_cast<size_t>(L) * L, 0.0);
    for (int p = 0; p < L; ++p) {
        const double a = std::sqrt((p == 0 ? 1.0 : 2.0) / L);
        for (int m = 0; m < L; ++m) T[static_cast<size_t>(p) * L + m] = a * std::cos(pi * (2 * m + 1) * p / (2.0 * L));
    }
}

// Walsh functions in sequency order: wal_p(m) = (-1)^(sum_i r_i(p) m_i) with
// r_i(p) the bits of the Gray code of p taken in reverse order, so that
// wal_p has exactly p sign changes.
void walsh_seq_rows(int L, std::vector<double> &T)
{
    int bits = 0;
    while ((1 << bits) < L) ++bits;
    T.assign(static_cast<size_t>(L) * L, 0.0);
    for (int p = 0; p < L; ++p) {
        const unsigned g = static_cast<unsigned>(p ^ (p >> 1));
        unsigned rev = 0;
        for (int i = 0; i < bits; ++i)
            if (g & (1u << i)) rev |= 1u << (bits - 1 - i);
        for (int m = 0; m < L; ++m) {
            const int par = __builtin_popcount(rev & static_cast<unsigned>(m)) & 1;
            T[static_cast<size_t>(p) * L + m] = par ? -1.0 : 1.0;
        }
    }
}

// Atoms that are products of 1-D rows: atom (r, p, q) at k = (r M + p) N + q
// holds tt_r[t] tm_p[m] tn_q[n] * scale at pixel (t M + m) N + n (frame-major;
// T = 1 is the 2-D case).
static void separable(int M, int N, int T, const std::vector<double> &Tm, const std::vector<double> &Tn,
                      const std::vector<double> &Tt, double scale, double *phi)
{
    const size_t V = static_cast<size_t>(M) * N * T;
    for (int r = 0; r < T; ++r)
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < N; ++q) {
                double *a = phi + (static_cast<size_t>(r) * M * N + static_cast<size_t>(p) * N + q) * V;
                for (int t = 0; t < T; ++t)
                    for (int m = 0; m < M; ++m) {
                        const double vm = Tt[static_cast<size_t>(r) * T + t] * Tm[static_cast<size_t>(p) * M + m] * scale;
                        for (int n = 0; n < N; ++n)
                            a[(static_cast<size_t>(t) * M + m) * N + n] = vm * Tn[static_cast<size_t>(q) * N + n];
                    }
            }
}

bool build_dictionary(int M, int N, int T, int basis, int K, const double *numeric,
                      std::vector<double> &phi, std::string *why)
{
    const size_t MN = static_cast<size_t>(M) * N * T;   // samples of the (flattened) area
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    switch (basis) {
    case 1:   // DCT
    case 2:   // WHT
    case 3: { // DCT u WHT
        const size_t expect = basis == 3 ? 2 * MN : MN;
        if (static_cast<size_t>(K) != expect) {
            *why = "K does not match the basis cardinality (" + std::to_string(expect) + ")";
            return false;
        }
        if (basis != 1 && (!pow2(M) || !pow2(N) || !pow2(T))) {
            *why = "the WHT needs power-of-two M, N (and T)";
            return false;
        }
        phi.assign(static_cast<size_t>(K) * MN, 0.0);
        std::vector<double> Tm, Tn, Tt;
        if (basis == 1 || basis == 3) {
            dct_rows(M, Tm);
            dct_rows(N, Tn);
            dct_rows(T, Tt);
            separable(M, N, T, Tm, Tn, Tt, 1.0, phi.data());
        }
        if (basis == 2 || basis == 3) {
            walsh_seq_rows(M, Tm);
            walsh_seq_rows(N, Tn);
            walsh_seq_rows(T, Tt);
            separable(M, N, T, Tm, Tn, Tt, 1.0 / std::sqrt(static_cast<double>(MN)),
                      phi.data() + (basis == 3 ? MN * MN : 0));
        }
        return true;
    }
    case 4:
        if (K < 1 || !numeric) {
            *why = "NUMERIC needs K >= 1 and a dictionary";
            return false;
        }
        phi.assign(numeric, numeric + static_cast<size_t>(K) * MN);
        for (double v : phi)
            if (!std::isfinite(v)) {
                *why = "the dictionary holds a non-finite value";
                return false;
            }
        return true;
    default:
        *why = "unknown basis";
        return false;
    }
}

// An atom that is collinear (over the whole area) with an atom of lower
// index can never win the argmax under smallest-index tie-breaking, so it is
// flagged inadmissible.  Candidates are found by sorting the atoms on
// |<a_k, z>| / |a_k| for a fixed pseudo-random vector z: collinear unit atoms
// differ by at most sqrt(2e-12) in l2, so their keys differ by at most
// 1.5e-6 |z|; only neighbours within 1e-5 |z| get the exact cosine test.
void find_collinear(int K, int MN, const double *phi, std::vector<uint8_t> &dup)
{
    dup.assign(K, 0);
    std::vector<double> z(MN), nrm(K), key(K);
    std::mt19937_64 gen(0x5e1ec7ull);
    std::normal_distribution<double> nd(0.0, 1.0);
    double zn = 0.0;
    for (int i = 0; i < MN; ++i) { z[i] = nd(gen); zn += z[i] * z[i]; }
    zn = std::sqrt(zn);
    for (int k = 0; k < K; ++k) {
        const double *a = phi + static_cast<size_t>(k) * MN;
        double s = 0.0, d = 0.0;
        for (int i = 0; i < MN; ++i) { s += a[i] * a[i]; d += a[i] * z[i]; }
        nrm[k] = std::sqrt(s);
        key[k] = nrm[k] > 0.0 ? std::fabs(d) / nrm[k] : -1.0;
    }
    std::vector<int> ord(K);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return key[x] < key[y]; });
    const double win = 1e-5 * zn;
    for (int i = 0; i < K; ++i) {
        const int ki = ord[i];
        if (nrm[ki] == 0.0) continue;
        for (int j = i + 1; j < K && key[ord[j]] - key[ki] <= win; ++j) {
            const int kj = ord[j];
            if (nrm[kj] == 0.0) continue;
            const double *a = phi + static_cast<size_t>(ki) * MN;
            const double *b = phi + static_cast<size_t>(kj) * MN;
            double d = 0.0;
            for (int t = 0; t < MN; ++t) d += a[t] * b[t];
            if (std::fabs(d) >= (1.0 - 1e-12) * nrm[ki] * nrm[kj]) dup[std::max(ki, kj)] = 1;
        }
    }
}

// eq. (4)-(5): w = rho on A (rho_hat ^ distance to the area centre unless a
// rho map is given), 0 on B; an M x N x T area is frame-major and its
// distance has a temporal term (T = 1: the 2-D weighting).
void weighting(int M, int N, int T, double rho_hat, const double *rho, const uint8_t *support,
               std::vector<double> &w)
{
    w.assign(static_cast<size_t>(M) * N * T, 0.0);
    for (int t = 0; t < T; ++t)
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < N; ++n) {
                const size_t i = (static_cast<size_t>(t) * M + m) * N + n;
                if (!support[i]) continue;
                if (rho) {
                    w[i] = rho[i];
                } else {
                    const double dt = t - 0.5 * (T - 1), dm = m - 0.5 * (M - 1), dn = n - 0.5 * (N - 1);
                    w[i] = std::pow(rho_hat, std::sqrt(dt * dt + dm * dm + dn * dn));
                }
            }
}

}  // namespace se
