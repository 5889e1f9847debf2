"""FP64 CPU oracle for Selective Extrapolation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never loads it and shares
no code with it.  The arithmetic lives in ``se_oracle.c`` (plain C loops in
double precision, one function per equation / algorithm of the paper); this
file only compiles it with gcc and marshals numpy arrays through ctypes.

Functions (citations are to Seiler & Kaup, arXiv 2204.14194):
  weights             eq. (4)-(5)
  dict_dct / dict_wht / dict_dct_wht   example dictionaries (Sec. I, Fig. 1)
  find_duplicates     collinear atoms, lowest index kept (tie-break reading)
  projection_state    eq. (3), (6), (7) for one residual
  se_original         Alg. 1 (eqs. 2-10) for one block
  fase_tables         Alg. 2 (eqs. 16-17)
  fase                Alg. 3 (eqs. 12, 18-20) for one block
  se_original_batch / fase_batch   the same over many blocks (OpenMP over blocks)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "se_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libse_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False, src: str = _SRC, out: str = _OUT) -> str:
    """Compile ``src`` (default ``se_oracle.c``) into the shared library ``out``
    (default ``oracle/_build/libse_oracle.so``) with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-fopenmp", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(C.CDLL(build()))
        return _lib


def use_library(path: str) -> None:
    """Route every function of this module through the shared library at
    ``path`` (a build of a modified copy of ``se_oracle.c``).  The pin tests use
    it to check that they reject an oracle with a planted mistake."""
    global _lib
    with _lock:
        _lib = _configure(C.CDLL(os.path.abspath(path)))


def _configure(lib):
    vp = C.c_void_p
    ip = C.c_int
    dbl = C.c_double
    lib.or_weights.argtypes = [ip, ip, dbl, _u8, vp, _dp]
    lib.or_dict_dct.argtypes = [ip, ip, _dp]
    lib.or_dict_wht.argtypes = [ip, ip, _dp]
    lib.or_dict_wht.restype = ip
    lib.or_dict_dct_wht.argtypes = [ip, ip, _dp]
    lib.or_dict_dct_wht.restype = ip
    lib.or_weights3.argtypes = [ip, ip, ip, dbl, _u8, vp, _dp]
    lib.or_dict_dct3.argtypes = [ip, ip, ip, _dp]
    lib.or_dict_wht3.argtypes = [ip, ip, ip, _dp]
    lib.or_dict_wht3.restype = ip
    lib.or_dict_dct_wht3.argtypes = [ip, ip, ip, _dp]
    lib.or_dict_dct_wht3.restype = ip
    lib.or_find_duplicates.argtypes = [ip, ip, _dp, _u8]
    lib.or_dict_dft.argtypes = [ip, ip, _dp, _dp]
    lib.or_dict_bdft.argtypes = [ip, ip, _dp, _dp]
    lib.or_dict_dft_bdft.argtypes = [ip, ip, _dp, _dp]
    lib.or_find_duplicates_c.argtypes = [ip, ip, _dp, _dp, _u8]
    lib.or_se_original_c.argtypes = [ip, ip, ip, _dp, _dp, _dp, vp, _dp, vp, dbl, ip,
                                     _dp, vp, vp, vp, vp, vp, vp]
    lib.or_se_original_c.restype = ip
    lib.or_fase_c.argtypes = [ip, ip, ip, _dp, _dp, _dp, vp, _dp, vp, dbl, ip, _dp, vp, vp, vp, vp]
    lib.or_fase_c.restype = ip
    lib.or_se_original_c_batch.argtypes = [ip, ip, ip, ip, _dp, _dp, _dp, ip, vp, _dp, dbl, ip,
                                           _dp, vp, vp, vp, vp, ip]
    lib.or_se_original_c_batch.restype = ip
    lib.or_projection_state.argtypes = [ip, ip, _dp, _dp, _dp, vp, vp, vp, vp]
    lib.or_se_original.argtypes = [ip, ip, ip, _dp, _dp, vp, _dp, dbl, ip, ip,
                                   _dp, vp, vp, vp, vp, vp, vp]
    lib.or_se_original.restype = ip
    lib.or_fase_tables.argtypes = [ip, ip, ip, _dp, _dp, _dp, _dp]
    lib.or_fase.argtypes = [ip, ip, ip, _dp, _dp, _dp, _dp, vp, _dp, dbl, ip,
                            _dp, vp, vp, vp, vp]
    lib.or_fase.restype = ip
    lib.or_se_original_batch.argtypes = [ip, ip, ip, ip, _dp, _dp, ip, vp, _dp, dbl,
                                         ip, vp, _dp, vp, vp, vp, ip]
    lib.or_se_original_batch.restype = ip
    lib.or_fase_batch.argtypes = [ip, ip, ip, ip, _dp, _dp, _dp, _dp, vp, _dp, dbl,
                                  ip, _dp, vp, vp, ip]
    lib.or_fase_batch.restype = ip
    lib.or_max_threads.restype = ip
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def weights(M: int, N: int, rho_hat: float, support: np.ndarray,
            rho: Optional[np.ndarray] = None) -> np.ndarray:
    """Weighting function w of eq. (4) with the isotropic decay of eq. (5)."""
    w = np.empty((M, N))
    sup = np.ascontiguousarray(support, dtype=np.uint8)
    rr = None if rho is None else _f64(rho)
    _load().or_weights(M, N, float(rho_hat), sup, _ptr(rr), w)
    return w


def dict_dct(M: int, N: int) -> np.ndarray:
    phi = np.empty((M * N, M, N))
    _load().or_dict_dct(M, N, phi)
    return phi


def dict_wht(M: int, N: int) -> np.ndarray:
    phi = np.empty((M * N, M, N))
    if _load().or_dict_wht(M, N, phi) != 0:
        raise ValueError("WHT needs power-of-two M and N")
    return phi


def dict_dct_wht(M: int, N: int) -> np.ndarray:
    phi = np.empty((2 * M * N, M, N))
    if _load().or_dict_dct_wht(M, N, phi) != 0:
        raise ValueError("WHT needs power-of-two M and N")
    return phi


def dictionary(basis: str, M: int, N: int, numeric: Optional[np.ndarray] = None) -> np.ndarray:
    if basis == "dct":
        return dict_dct(M, N)
    if basis == "wht":
        return dict_wht(M, N)
    if basis == "dct_wht":
        return dict_dct_wht(M, N)
    if basis == "numeric":
        return _f64(numeric)
    raise ValueError(basis)


def weights3(M: int, N: int, T: int, rho_hat: float, support: np.ndarray,
             rho: Optional[np.ndarray] = None) -> np.ndarray:
    """eq. (4)-(5) for an M x N x T block (frame-major [T][M][N])."""
    w = np.empty((T, M, N))
    sup = np.ascontiguousarray(support, dtype=np.uint8)
    rr = None if rho is None else _f64(rho)
    _load().or_weights3(M, N, T, float(rho_hat), sup, _ptr(rr), w)
    return w


def dictionary3(basis: str, M: int, N: int, T: int) -> np.ndarray:
    """3-D DCT / WHT / DCT u WHT atoms, shape (K, T, M, N), k = (r M + p) N + q."""
    V = M * N * T
    K = 2 * V if basis == "dct_wht" else V
    phi = np.empty((K, T, M, N))
    lib = _load()
    if basis == "dct":
        lib.or_dict_dct3(M, N, T, phi)
        return phi
    fn = {"wht": lib.or_dict_wht3, "dct_wht": lib.or_dict_dct_wht3}[basis]
    if fn(M, N, T, phi) != 0:
        raise ValueError("WHT needs power-of-two M, N and T")
    return phi


def flat(a: np.ndarray) -> np.ndarray:
    """A 3-D block (or stack of atoms / blocks) as the 2-D area (T M) x N that
    Alg. 1-3 run on unchanged (frame-major flattening)."""
    a = np.ascontiguousarray(a)
    return a.reshape(a.shape[:-3] + (a.shape[-3] * a.shape[-2], a.shape[-1]))


def find_duplicates(phi: np.ndarray) -> np.ndarray:
    K = phi.shape[0]
    MN = int(np.prod(phi.shape[1:]))
    ex = np.zeros(K, dtype=np.uint8)
    _load().or_find_duplicates(K, MN, _f64(phi), ex)
    return ex


@dataclass
class ProjState:
    p: np.ndarray
    ckk: np.ndarray
    e: np.ndarray
    score: np.ndarray


def projection_state(phi: np.ndarray, w: np.ndarray, r: np.ndarray) -> ProjState:
    """p_k (eq. 3), C_kk, e_k (eq. 6) and p_k^2 C_kk (eq. 7) for residual r."""
    K = phi.shape[0]
    MN = int(np.prod(phi.shape[1:]))
    out = [np.empty(K) for _ in range(4)]
    _load().or_projection_state(MN, K, _f64(phi), _f64(w), _f64(r), *[_ptr(o) for o in out])
    return ProjState(*out)


@dataclass
class SEResult:
    out: np.ndarray
    g: np.ndarray
    u: np.ndarray
    c: np.ndarray
    r: Optional[np.ndarray] = None
    energy: Optional[np.ndarray] = None
    margin: Optional[np.ndarray] = None
    R: Optional[np.ndarray] = None
    status: int = 0


def se_original(phi: np.ndarray, w: np.ndarray, s: np.ndarray, gamma: float, I: int,
                dup: Optional[np.ndarray] = None, brute_force: bool = False) -> SEResult:
    """Alg. 1 for one block; ``brute_force`` selects by eq. (6) instead of eq. (7)."""
    K = phi.shape[0]
    M, N = w.shape
    out, g, r = np.empty((M, N)), np.empty((M, N)), np.empty((M, N))
    u = np.empty(I, dtype=np.int32)
    c, e, mg = np.empty(I), np.empty(I), np.empty(I)
    d = None if dup is None else np.ascontiguousarray(dup, dtype=np.uint8)
    rc = _load().or_se_original(M, N, K, _f64(phi), _f64(w), _ptr(d), _f64(s), float(gamma),
                                int(I), int(brute_force), out, _ptr(g), _ptr(r), _ptr(u),
                                _ptr(c), _ptr(e), _ptr(mg))
    return SEResult(out, g, u, c, r=r, energy=e, margin=mg, status=rc)


def fase_tables(phi: np.ndarray, w: np.ndarray):
    """Alg. 2: the K x K table C (eq. 16) and D (eq. 17)."""
    K = phi.shape[0]
    M, N = w.shape
    Cm = np.empty((K, K))
    D = np.empty(K)
    _load().or_fase_tables(M, N, K, _f64(phi), _f64(w), Cm, D)
    return Cm, D


def fase(phi: np.ndarray, w: np.ndarray, Cm: np.ndarray, D: np.ndarray, s: np.ndarray,
         gamma: float, I: int, dup: Optional[np.ndarray] = None) -> SEResult:
    """Alg. 3 for one block given the tables of Alg. 2."""
    K = phi.shape[0]
    M, N = w.shape
    out, g = np.empty((M, N)), np.empty((M, N))
    R = np.empty(K)
    u = np.empty(I, dtype=np.int32)
    c = np.empty(I)
    d = None if dup is None else np.ascontiguousarray(dup, dtype=np.uint8)
    rc = _load().or_fase(M, N, K, _f64(phi), _f64(w), _f64(Cm), _f64(D), _ptr(d), _f64(s),
                         float(gamma), int(I), out, _ptr(g), _ptr(R), _ptr(u), _ptr(c))
    return SEResult(out, g, u, c, R=R, status=rc)


def se_original_batch(phi: np.ndarray, w: np.ndarray, s: np.ndarray, gamma: float, I: int,
                      dup: Optional[np.ndarray] = None, iters: Optional[np.ndarray] = None,
                      nthreads: int = 0, margins: bool = False):
    """Alg. 1 over blocks ``s[B, M, N]``; ``w`` is one pattern [M, N] or per block [B, M, N].

    Returns (out [B, M, N], u [B, I], c [B, I], status), plus the tie margins
    [B, I] when ``margins``.  With per-block iteration counts, log entries
    past a block's count are left as -1 / NaN.
    """
    K = phi.shape[0]
    B, M, N = s.shape
    out = np.empty((B, M, N))
    u = np.full((B, I), -1, dtype=np.int32)
    c = np.full((B, I), np.nan)
    mg = np.full((B, I), np.nan) if margins else None
    d = None if dup is None else np.ascontiguousarray(dup, dtype=np.uint8)
    it = None if iters is None else np.ascontiguousarray(iters, dtype=np.int32)
    rc = _load().or_se_original_batch(B, M, N, K, _f64(phi), _f64(w), int(w.ndim == 3), _ptr(d),
                                      _f64(s), float(gamma), int(I), _ptr(it), out, _ptr(u),
                                      _ptr(c), _ptr(mg), int(nthreads))
    if margins:
        return out, u, c, mg, rc
    return out, u, c, rc


def fase_batch(phi, w, Cm, D, s, gamma, I, dup=None, nthreads: int = 0):
    """Alg. 3 over blocks that share one pattern.  Returns (out, u, c, status)."""
    K = phi.shape[0]
    B, M, N = s.shape
    out = np.empty((B, M, N))
    u = np.empty((B, I), dtype=np.int32)
    c = np.empty((B, I))
    d = None if dup is None else np.ascontiguousarray(dup, dtype=np.uint8)
    rc = _load().or_fase_batch(B, M, N, K, _f64(phi), _f64(w), _f64(Cm), _f64(D), _ptr(d),
                               _f64(s), float(gamma), int(I), out, _ptr(u), _ptr(c), int(nthreads))
    return out, u, c, rc


def max_threads() -> int:
    return int(_load().or_max_threads())


# ------------------------------------------------------------ complex atoms
def dict_complex(basis: str, M: int, N: int) -> np.ndarray:
    """DFT / binarised DFT / their union as complex128 atoms (K, M, N)."""
    V = M * N
    K = 2 * V if basis == "dft_bdft" else V
    re, im = np.empty((K, M, N)), np.empty((K, M, N))
    fn = {"dft": _load().or_dict_dft, "bdft": _load().or_dict_bdft, "dft_bdft": _load().or_dict_dft_bdft}[basis]
    fn(M, N, re, im)
    return re + 1j * im


def _planes(phi: np.ndarray):
    return np.ascontiguousarray(phi.real, dtype=np.float64), np.ascontiguousarray(phi.imag, dtype=np.float64)


def find_duplicates_c(phi: np.ndarray) -> np.ndarray:
    K = phi.shape[0]
    MN = int(np.prod(phi.shape[1:]))
    re, im = _planes(phi)
    ex = np.zeros(K, dtype=np.uint8)
    _load().or_find_duplicates_c(K, MN, re, im, ex)
    return ex


def se_original_c(phi: np.ndarray, w: np.ndarray, s: np.ndarray, gamma: float, I: int,
                  dup: Optional[np.ndarray] = None) -> SEResult:
    """Complex Alg. 1 for one block; ``s`` real or complex.  ``out`` and ``g`` are complex."""
    K = phi.shape[0]
    M, N = w.shape
    re, im = _planes(phi)
    s = np.asarray(s)
    s_re, s_im = np.ascontiguousarray(s.real, dtype=np.float64), np.ascontiguousarray(np.imag(s), dtype=np.float64)
    o_re, o_im = np.empty((M, N)), np.empty((M, N))
    u = np.empty(I, dtype=np.int32)
    cr, ci, e, mg = np.empty(I), np.empty(I), np.empty(I), np.empty(I)
    d = None if dup is None else np.ascontiguousarray(dup, dtype=np.uint8)
    rc = _load().or_se_original_c(M, N, K, re, im, _f64(w), _ptr(d), s_re, _ptr(s_im), float(gamma), int(I),
                                  o_re, _ptr(o_im), _ptr(u), _ptr(cr), _ptr(ci), _ptr(e), _ptr(mg))
    out = o_re + 1j * o_im
    g = np.where(np.asarray(w) > 0, np.nan, out)
    return SEResult(out, g, u, cr + 1j * ci, energy=e, margin=mg, status=rc)


def fase_c(phi: np.ndarray, w: np.ndarray, s: np.ndarray, gamma: float, I: int,
           dup: Optional[np.ndarray] = None) -> SEResult:
    """Complex Alg. 2 + 3 for one block (tables built inside)."""
    K = phi.shape[0]
    M, N = w.shape
    re, im = _planes(phi)
    s = np.asarray(s)
    s_re, s_im = np.ascontiguousarray(s.real, dtype=np.float64), np.ascontiguousarray(np.imag(s), dtype=np.float64)
    o_re, o_im = np.empty((M, N)), np.empty((M, N))
    u = np.empty(I, dtype=np.int32)
    cr, ci = np.empty(I), np.empty(I)
    d = None if dup is None else np.ascontiguousarray(dup, dtype=np.uint8)
    rc = _load().or_fase_c(M, N, K, re, im, _f64(w), _ptr(d), s_re, _ptr(s_im), float(gamma), int(I),
                           o_re, _ptr(o_im), _ptr(u), _ptr(cr), _ptr(ci))
    return SEResult(o_re + 1j * o_im, None, u, cr + 1j * ci, status=rc)


def se_original_c_batch(phi: np.ndarray, w: np.ndarray, s: np.ndarray, gamma: float, I: int,
                        dup: Optional[np.ndarray] = None, nthreads: int = 0, margins: bool = False):
    """Complex Alg. 1 over real blocks ``s[B, M, N]``; returns (Re out, u, complex c, status[, margins])."""
    K = phi.shape[0]
    B, M, N = s.shape
    re, im = _planes(phi)
    out = np.empty((B, M, N))
    u = np.full((B, I), -1, dtype=np.int32)
    cr, ci = np.full((B, I), np.nan), np.full((B, I), np.nan)
    mg = np.full((B, I), np.nan) if margins else None
    d = None if dup is None else np.ascontiguousarray(dup, dtype=np.uint8)
    rc = _load().or_se_original_c_batch(B, M, N, K, re, im, _f64(w), int(w.ndim == 3), _ptr(d), _f64(s),
                                        float(gamma), int(I), out, _ptr(u), _ptr(cr), _ptr(ci), _ptr(mg),
                                        int(nthreads))
    if margins:
        return out, u, cr + 1j * ci, mg, rc
    return out, u, cr + 1j * ci, rc

