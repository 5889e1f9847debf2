"""The oracle's pins reject an oracle with a planted mistake.

Each mutant below is one plausible slip in ``oracle/se_oracle.c``, such as a
dropped term, a flipped sign, a wrong index or a wrong normalisation.  The test
copies the C source into a temporary directory and applies the slip there.  It
builds the copy with the oracle's own compiler flags and runs the CPU pin tests
against it in a child process.  Every mutant must make at least one pin fail.
The unchanged source, built the same way, must pass every pin.  The committed
oracle is never modified.

A mutant names the equation or algorithm step it breaks.  Mutants that cannot
change a result are not listed.  Two examples:
  - reading C(u,k) for C(k,u) in eq. (20): the table is symmetric;
  - transposing a sequency-ordered Walsh matrix: the matrix is symmetric.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_parity_structure.py"]

# (name, exact text in se_oracle.c -- must occur once, replacement)
MUTANTS = [
    # eq. (5): distance measured from the wrong centre
    ("w_centre", "double dm = m - (M - 1) / 2.0;", "double dm = m - M / 2.0;"),
    # eq. (4): w not zeroed on the loss area B
    ("w_mask", "w[m * N + n] = support[m * N + n] ? r : 0.0;", "w[m * N + n] = r;"),
    # DCT atoms: DC row not scaled by sqrt(1/M)
    ("dct_norm", "double ap = p == 0 ? sqrt(1.0 / M) : sqrt(2.0 / M);\n            double aq",
     "double ap = sqrt(2.0 / M);\n            double aq"),
    # DCT atoms: half-sample shift dropped
    ("dct_phase", "a[m * N + n] = ap * aq * cos(pi * (2 * m + 1) * p / (2.0 * M))",
     "a[m * N + n] = ap * aq * cos(pi * (2 * m) * p / (2.0 * M))"),
    # WHT atoms: sequency miscounted
    ("wht_sequency", "if (j > 0 && v != prev) ++changes;", "if (j > 1 && v != prev) ++changes;"),
    # WHT atoms: 1/MN instead of 1/sqrt(MN)
    ("wht_norm", "double s = 1.0 / sqrt((double)M * N);", "double s = 1.0 / ((double)M * N);"),
    # collinear atoms: the higher index kept instead of the lower
    ("dup_keeps_high",
     "if (fabs(d) >= (1.0 - OR_COLLINEAR_REL) * nrm[i] * nrm[j]) excluded[j] = 1;",
     "if (fabs(d) >= (1.0 - OR_COLLINEAR_REL) * nrm[i] * nrm[j]) excluded[i] = 1;"),
    # eq. (3): denominator without the weighting function
    ("p_den_unweighted", "den += a[i] * w[i] * a[i];", "den += a[i] * a[i];"),
    # eq. (6): residual energy without w
    ("e_unweighted", "ek += d * d * w[i];", "ek += d * d;"),
    # eq. (7): score without C_kk
    ("score_no_ckk", "if (score) score[k] = pk * pk * den;", "if (score) score[k] = pk * pk;"),
    # eq. (7): tie goes to the largest index
    ("alg1_tie_high", "double v = selector ? -e[k] : sc[k];    /* argmin e == argmax -e */\n"
     "            if (u < 0 || v > best)",
     "double v = selector ? -e[k] : sc[k];    /* argmin e == argmax -e */\n"
     "            if (u < 0 || v >= best)"),
    # eq. (8): orthogonality deficiency factor dropped
    ("alg1_no_gamma", "double c = gamma * p[u];", "double c = p[u];"),
    # eq. (10): residual updated with the wrong sign
    ("alg1_residual_sign", "r[i] -= c * a[i];", "r[i] += c * a[i];"),
    # eq. (9): model update uses gamma instead of the coefficient
    ("alg1_model", "g[i] += c * a[i];\n            r[i]", "g[i] += gamma * a[i];\n            r[i]"),
    # replacement: A overwritten by the model too
    ("alg1_replace", "/* replacement of B by the model */\n"
     "    for (int i = 0; i < MN; ++i) out[i] = w[i] > 0.0 ? s[i] : g[i];",
     "/* replacement of B by the model */\n"
     "    for (int i = 0; i < MN; ++i) out[i] = g[i];"),
    # tie margin: second-best score not tracked
    ("margin_second", "if (sc[k] > s1) { s2 = s1; s1 = sc[k]; }\n"
     "                else if (sc[k] > s2) s2 = sc[k];\n            }\n"
     "            margin_log[nu - 1] = s1 > 0.0 ? (s1 - (s2 < 0.0 ? 0.0 : s2)) / s1 : 0.0;\n        }\n\n"
     "        /* eq. (8)",
     "if (sc[k] > s1) { s1 = sc[k]; }\n"
     "                else if (sc[k] > s2) s2 = sc[k];\n            }\n"
     "            margin_log[nu - 1] = s1 > 0.0 ? (s1 - (s2 < 0.0 ? 0.0 : s2)) / s1 : 0.0;\n        }\n\n"
     "        /* eq. (8)"),
    # eq. (16): table without the weighting function
    ("alg2_C_unweighted", "acc += a[i] * w[i] * b[i];", "acc += a[i] * b[i];"),
    # eq. (17): D = 1 / C_kk instead of 1 / sqrt(C_kk)
    ("alg2_D", "D[k] = C[(size_t)k * K + k] > 0.0 ? 1.0 / sqrt(C[(size_t)k * K + k]) : 0.0;",
     "D[k] = C[(size_t)k * K + k] > 0.0 ? 1.0 / C[(size_t)k * K + k] : 0.0;"),
    # eq. (12): initial projections without w
    ("alg3_R0_unweighted", "acc += (w[i] > 0.0 ? s[i] : 0.0) * a[i] * w[i];",
     "acc += (w[i] > 0.0 ? s[i] : 0.0) * a[i];"),
    # eq. (18): selection by |R_k| without D_k
    ("alg3_select_no_D", "double v = fabs(R[k]) * D[k];", "double v = fabs(R[k]);"),
    # eq. (19): one factor D_u instead of D_u^2
    ("alg3_coef_D", "double c = gamma * R[u] * D[u] * D[u];", "double c = gamma * R[u] * D[u];"),
    # eq. (20): wrong column of C
    ("alg3_update_column", "R[k] -= c * C[(size_t)k * K + u];", "R[k] -= c * C[(size_t)k * K + k];"),
    # batch driver: every block reads the samples of block 0
    ("batch_se_samples", "s + (size_t)b * MN, gamma, Ib", "s, gamma, Ib"),
    ("batch_fase_samples", "s + (size_t)b * MN, gamma, I,\n                         out",
     "s, gamma, I,\n                         out"),
    # 3-D eq. (5): distance in t from the wrong centre
    ("w3_centre", "double dt = t - (T - 1) / 2.0", "double dt = t - T / 2.0"),
    # 3-D DCT: half-sample shift dropped in t
    ("dct3_phase", "cos(pi * (2 * t + 1) * r / (2.0 * T))", "cos(pi * (2 * t) * r / (2.0 * T))"),
    # 3-D WHT: normalised over one frame instead of the whole block
    ("wht3_norm", "double s = 1.0 / sqrt((double)V);", "double s = 1.0 / sqrt((double)M * N);"),
    # complex DFT atoms conjugated
    ("dft_conjugate", "im[k * L + (size_t)m * N + n] = s * sin(2.0 * pi * a / L);",
     "im[k * L + (size_t)m * N + n] = -s * sin(2.0 * pi * a / L);"),
    # binarised DFT: sgn(0) = -1 for the sine
    ("bdft_sign_zero", "im[k * L + (size_t)m * N + n] = (2 * a <= L) ? s : -s;",
     "im[k * L + (size_t)m * N + n] = (2 * a < L) ? s : -s;"),
    # complex duplicates: imaginary part of <phi_i, phi_j> dropped
    ("dup_c_real_only", "di += re[a] * im[b] - im[a] * re[b];", "di += 0.0;"),
    # complex eq. (3): atom not conjugated in the imaginary part
    ("se_c_conjugate", "ni += (ri[i] * re[a] - rr[i] * im[a]) * w[i];",
     "ni += (ri[i] * re[a] + rr[i] * im[a]) * w[i];"),
    # complex eq. (9)-(10): wrong sign in the complex product c * phi_u
    ("se_c_product", "const double vr = cr * re[a] - ci * im[a]", "const double vr = cr * re[a] + ci * im[a]"),
    # complex eq. (16): table mirrored without the conjugate
    ("fase_c_hermitian", "Ci[(size_t)l * K + k] = -ai;", "Ci[(size_t)l * K + k] = ai;"),
    # complex eq. (20): wrong sign in the complex product c * C(k,u)
    ("fase_c_update", "Ri[k] -= cr * xi + ci * xr;", "Ri[k] -= cr * xi - ci * xr;"),
    # complex eq. (12): atom not conjugated
    ("fase_c_R0_conjugate", "ai += (si * re[a] - sr * im[a]) * w[i];",
     "ai += (si * re[a] + sr * im[a]) * w[i];"),
    # complex eq. (17): 1 / C_kk instead of 1 / sqrt(C_kk)
    ("fase_c_D", "D[k] = ckk[k] > 0.0 ? 1.0 / sqrt(ckk[k]) : 0.0;", "D[k] = ckk[k] > 0.0 ? 1.0 / ckk[k] : 0.0;"),
    # complex eq. (18): |R_k| from the real part only
    ("fase_c_select_real", "double v = sqrt(Rr[k] * Rr[k] + Ri[k] * Ri[k]) * D[k];",
     "double v = sqrt(Rr[k] * Rr[k]) * D[k];"),
    # complex eq. (3): denominator from the real part of the atom only
    ("se_c_ckk_real", "acc += (re[a] * re[a] + im[a] * im[a]) * w[i];", "acc += (re[a] * re[a]) * w[i];"),
    # 3-D eq. (4): w not zeroed on the loss area
    ("w3_mask", "w[i] = support[i] ? r : 0.0;", "w[i] = r;"),
    # 3-D DCT: DC row in t not scaled by sqrt(1/T)
    ("dct3_norm", "double ar = r == 0 ? sqrt(1.0 / T) : sqrt(2.0 / T);", "double ar = sqrt(2.0 / T);"),
    # admissible atoms: zero-energy atoms not excluded
    ("admissible_energy", "ok[k] = (!dup || !dup[k]) && ckk[k] > OR_EXCLUDE_REL * mx && mx > 0.0;",
     "ok[k] = (!dup || !dup[k]);"),
    # admissible atoms: duplicate flags ignored
    ("admissible_dup", "ok[k] = (!dup || !dup[k]) && ckk[k] > OR_EXCLUDE_REL * mx && mx > 0.0;",
     "ok[k] = ckk[k] > OR_EXCLUDE_REL * mx && mx > 0.0;"),
    # eq. (6) selector: argmax e_k instead of argmin
    ("bruteforce_argmax", "double v = selector ? -e[k] : sc[k];", "double v = selector ? e[k] : sc[k];"),
    # eq. (2): initial residual reads the samples on B
    ("alg1_r0_reads_B", "for (int i = 0; i < MN; ++i) r[i] = w[i] > 0.0 ? s[i] : 0.0;",
     "for (int i = 0; i < MN; ++i) r[i] = s[i];"),
    # weighted residual energy without w
    ("alg1_energy_unweighted", "E += w[i] * r[i] * r[i];", "E += r[i] * r[i];"),
]

_CHILD = (
    "import sys, oracle, pytest\n"
    "oracle.use_library(sys.argv[1])\n"
    "sys.exit(pytest.main(['-x', '-q', '-m', 'not gpu', '-p', 'no:cacheprovider',]"
    " + sys.argv[2:]))\n"
)


def _source() -> str:
    with open(os.path.join(ROOT, "oracle", "se_oracle.c")) as f:
        return f.read()


def _run_pins(src_text: str, tag: str, tmp: str) -> subprocess.CompletedProcess:
    src = os.path.join(tmp, f"{tag}.c")
    lib = os.path.join(tmp, f"lib{tag}.so")
    with open(src, "w") as f:
        f.write(src_text)
    oracle.build(force=True, src=src, out=lib)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-c", _CHILD, lib] + PINS, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_every_mutant_text_occurs_once():
    src = _source()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


def test_pins_reject_every_planted_mistake(tmp_path):
    src = _source()
    jobs = [("unchanged", src)] + [(name, src.replace(old, new)) for name, old, new in MUTANTS]
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as pool:
        results = dict(zip([j[0] for j in jobs],
                           pool.map(lambda j: _run_pins(j[1], j[0], str(tmp_path)), jobs)))
    control = results.pop("unchanged")
    assert control.returncode == 0, control.stdout[-3000:] + control.stderr[-2000:]
    # pytest exits with 1 when a test failed; anything else (a crash, a
    # collection error) would not show that a pin caught the mistake
    survivors = [n for n, r in results.items() if r.returncode == 0]
    other = {n: r.returncode for n, r in results.items() if r.returncode not in (0, 1)}
    assert not survivors, f"mutants no pin rejects: {survivors}"
    assert not other, f"mutants that did not end in a failed pin: {other}"
