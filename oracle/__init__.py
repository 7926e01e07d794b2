"""FP64 CPU oracle for the layered-media FMM -- TEST INFRASTRUCTURE ONLY.

A plain restatement, in C (``lmfmm_oracle.c``), of Cho & Huang, arXiv:1902.08250:
direct summation of the middle-layer three-layer Green's function with adaptive
Gauss-Kronrod Sommerfeld quadrature on a deformed contour (Sec. 2.1, Sec. 4.2,
Sec. 5), and a plain FMM following Algorithm 1.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package; the library in ``paper_1902_08250_gb300`` never does.

Parity status of each function is recorded in its docstring; none is
"parity unpinned" -- every function is checked in ``tests/test_oracle_*.py``
against closed forms, library routines, brute force or numbers the paper
prints.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lmfmm_oracle.c")
_LIB = os.path.join(_HERE, "liblmfmm_oracle.so")

TERMS = {"tt": 1, "bb": 2, "tb": 3, "bt": 4}
MASK_ALL = 0b1111


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


def _declare(L):
    sig = {
        "orc_sroot": (None, [_P, _D, _P]),
        "orc_sigma_paper_solve": (None, [_P, _D, _D, _D, _D, _P]),
        "orc_sigma_paper_closed": (None, [_P, _D, _D, _D, _D, _P]),
        "orc_sigma2t_safe": (None, [_P, _D, _D, _D, _D, _P]),
        "orc_sigma_layer2": (None, [_P, _D, _D, _D, _D, _P]),
        "orc_spectral_refl": (None, [_P, _D, _D, _D, _D, _D, _D, _P]),
        "orc_spectral_refl_solve": (None, [_P, _D, _D, _D, _D, _D, _D, _P]),
        "orc_set_tolerance": (None, [_D, _D]),
        "orc_set_boundaries": (None, [_I, _D, _I, _D]),
        "orc_cross_field": (_I, [_D, _D, _D, _D, _D, _D, _D, _D, _I, _I, _P]),
        "orc_cross_direct": (_I, [_D, _D, _D, _D, _I64, _P, _P, _I64, _P, _P, _I, _P, _I64, _P, _I, _P]),
        "orc_gk15_pow": (None, [_I, _D, _D, _P]),
        "orc_sommerfeld_free": (_I, [_D, _D, _D, _I, _P]),
        "orc_dirichlet": (_I, [_D, _D, _D, _D, _D, _I, _P]),
        "orc_g2t_paper": (_I, [_D, _D, _D, _D, _D, _D, _D, _D, _I, _P]),
        "orc_green_refl": (_I, [_D, _D, _D, _D, _D, _D, _D, _D, _I, _I, _P]),
        "orc_green_term": (_I, [_D, _D, _D, _D, _I, _D, _D, _D, _D, _P]),
        "orc_direct_apply": (_I, [_D, _D, _D, _D, _I64, _P, _P, _I, _P, _I64, _P, _I, _I, _P]),
        "orc_direct_apply_deriv": (_I, [_D, _D, _D, _D, _I64, _P, _P, _I, _P, _I64, _P, _I, _I, _P]),
        "orc_green_refl_deriv": (_I, [_D, _D, _D, _D, _D, _D, _D, _D, _I, _I, _P]),
        "orc_green_free_grad": (None, [_D, _D, _D, _P]),
        "orc_tree_build": (_I, [_I64, _P, _P, _D, _I, _P, _P, _P]),
        "orc_vlist": (_I64, [_I, _I, _I64, _P]),
        "orc_adaptive_tree": (_I64, [_I64, _P, _P, _D, _I, _I, _I64, _P, _P, _P, _P]),
        "orc_adaptive_lists": (_I64, [_I64, _P, _P, _D, _I, _I, _I, _I64, _P]),
        "orc_ulist": (_I64, [_I, _I, _I64, _P]),
        "orc_m2l_image_table": (_I, [_D, _D, _D, _D, _I, _D, _D, _I, _P]),
        "orc_m2l_free_table": (None, [_D, _D, _D, _I, _P]),
        "orc_fmm_apply": (_I, [_D, _D, _D, _D, _I64, _P, _P, _I, _I, _I, _P, _P]),
        "orc_s2m": (None, [_I64, _P, _P, _P, _D, _D, _D, _I, _P]),
        "orc_l2t": (None, [_I64, _P, _P, _P, _D, _D, _D, _I, _P]),
        "orc_shift": (None, [_P, _D, _D, _D, _I, _P]),
        "orc_besj": (_D, [_I, _D]),
        "orc_green_free": (None, [_D, _D, _P]),
        "orc_psi_e4": (_I, [_D, _D, _D, _D, _I, _D, _D, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cplx_in(z):
    z = complex(z)
    return np.array([z.real, z.imag])


def set_tolerance(atol=1e-15, rtol=1e-13):
    lib().orc_set_tolerance(atol, rtol)


BC = {"transmission": 0, "dirichlet": 1, "neumann": 2, "impedance": 3}


def set_boundaries(top="transmission", top_alpha=0.0, bottom="transmission", bottom_alpha=0.0):
    """Kinds of the middle layer's interfaces (y = 0 top, y = -d bottom) for every later
    oracle call: transmission (the outer wave number k1 / k3), or a wall -- Dirichlet
    (R = -1), Neumann (R = +1), impedance (R = (s2 + i k2 alpha)/(s2 - i k2 alpha))."""
    lib().orc_set_boundaries(BC[top], float(top_alpha), BC[bottom], float(bottom_alpha))


# --- branch and densities ---------------------------------------------------
def sroot(lam, k):
    """s = sqrt(lam^2 - k^2) on the Re s >= 0 sheet (Eq. (Green); reading G1)."""
    o = np.zeros(2)
    lib().orc_sroot(_ptr(_cplx_in(lam)), k, _ptr(o))
    return complex(o[0], o[1])


def _vec_call(fn, n, lam, *args):
    o = np.zeros(2 * n)
    fn(_ptr(_cplx_in(lam)), *args, _ptr(o))
    return o[0::2] + 1j * o[1::2]


def sigma_paper_solve(lam, k1, k2, k3, d):
    """(sigma1, sigma2t, sigma2b, sigma3) from the paper's 4x4 system (Example 4)."""
    return _vec_call(lib().orc_sigma_paper_solve, 4, lam, k1, k2, k3, d)


def sigma_paper_closed(lam, k1, k2, k3, d):
    """The paper's printed closed forms (Example 4), literally."""
    return _vec_call(lib().orc_sigma_paper_closed, 4, lam, k1, k2, k3, d)


def sigma2t_safe(lam, k1, k2, k3, d):
    """sigma_2^t with numerator and denominator divided by e^{d s2}."""
    return _vec_call(lib().orc_sigma2t_safe, 1, lam, k1, k2, k3, d)[0]


def sigma_layer2(lam, k1, k2, k3, d):
    """(sigma_tt, sigma_bb, sigma_tb) for a middle-layer source (reading R1)."""
    return _vec_call(lib().orc_sigma_layer2, 3, lam, k1, k2, k3, d)


def spectral_refl(lam, k1, k2, k3, d, y, y0):
    """Reflected spectral field g_r^(lam; y, y0) from the closed-form densities."""
    return _vec_call(lib().orc_spectral_refl, 1, lam, k1, k2, k3, d, y, y0)[0]


def spectral_refl_solve(lam, k1, k2, k3, d, y, y0):
    """Reflected spectral field from a direct solve of the interface conditions."""
    return _vec_call(lib().orc_spectral_refl_solve, 1, lam, k1, k2, k3, d, y, y0)[0]


def gk15_pow(n, a, b):
    o = np.zeros(2)
    lib().orc_gk15_pow(n, a, b, _ptr(o))
    return o[0], o[1]


# --- Sommerfeld integrals -----------------------------------------------------
NORTH, EAST, AUTO = 0, 1, -1


def _green_out(fn, *args):
    o = np.zeros(2)
    st = fn(*args, _ptr(o))
    if st != 0:
        raise RuntimeError("oracle quadrature did not converge")
    return complex(o[0], o[1])


def sommerfeld_free(k, X, Y, tail):
    """(1/4pi) Int e^{i lam X} e^{-s|Y|}/s d lam on the first contour (Example 1)."""
    return _green_out(lib().orc_sommerfeld_free, k, X, Y, tail)


def dirichlet(k, x, y, x0, y0, tail):
    """Dirichlet half-space scattered field, sigma = -1 (Example 2)."""
    return _green_out(lib().orc_dirichlet, k, x, y, x0, y0, tail)


def g2t_paper(k1, k2, k3, d, x, y, x0, y0, tail):
    """The paper's g_2^t for a top-layer source (Example 4), literal densities."""
    return _green_out(lib().orc_g2t_paper, k1, k2, k3, d, x, y, x0, y0, tail)


def green_refl(k1, k2, k3, d, x, y, x0, y0, mask=MASK_ALL, tailmode=AUTO):
    """Reflected part G_r of the middle-layer Green's function (selected terms)."""
    return _green_out(lib().orc_green_refl, k1, k2, k3, d, x, y, x0, y0, mask, tailmode)


DX, DY, DD = 1, 2, 3


def green_refl_deriv(k1, k2, k3, d, x, y, x0, y0, deriv, mask=MASK_ALL):
    """d/dx or d/dy (target coordinates, deriv = DX, DY) or d/dd (deriv = DD) of G_r,
    by the chain rule inside the Sommerfeld integrand."""
    return _green_out(lib().orc_green_refl_deriv, k1, k2, k3, d, x, y, x0, y0, mask, deriv)


def green_free_grad(k, dx, dy):
    """Target gradient of (i/4) H0^(1)(k r) at offset (dx, dy): (i/4)(-k) H1^(1)(k r) (dx, dy)/r."""
    o = np.zeros(4)
    lib().orc_green_free_grad(k, dx, dy, _ptr(o))
    return complex(o[0], o[1]), complex(o[2], o[3])


def green_term(k1, k2, k3, d, term, x, y, x0, y0):
    """One image term G_m (term in 1..4 = tt, bb, tb, bt)."""
    return _green_out(lib().orc_green_term, k1, k2, k3, d, term, x, y, x0, y0)


def green_free(k, r):
    o = np.zeros(2)
    lib().orc_green_free(k, r, _ptr(o))
    return complex(o[0], o[1])


def besj(n, x):
    return lib().orc_besj(n, x)


# --- direct summation -----------------------------------------------------------
def direct_apply(medium, x, y, q, targets=None, refl_mask=MASK_ALL, nthreads=0):
    """u_i = sum_{j!=i} q_j (i/4)H0(k2 r_ij) + sum_j q_j G_r(x_i, x_j)  (Eq. (direct_sum)).

    q: complex array [nvec, n] (or [n]); returns [nvec, ntargets] (or [ntargets]).
    """
    k1, k2, k3, d = medium
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    q = np.asarray(q)
    one = q.ndim == 1
    q2 = _c(q.reshape(1, -1) if one else q, np.complex128)
    n = x.size
    nvec = q2.shape[0]
    if targets is None:
        tg = None
        nt = n
    else:
        tg = _c(targets, np.int64)
        nt = tg.size
    u = np.zeros((nvec, nt), np.complex128)
    st = lib().orc_direct_apply(k1, k2, k3, d, n, _ptr(x), _ptr(y), nvec, _ptr(q2), nt,
                                _ptr(tg) if tg is not None else None, refl_mask, nthreads, _ptr(u))
    if st != 0:
        raise RuntimeError("oracle quadrature did not converge")
    return u[0] if one else u


def direct_apply_deriv(medium, x, y, q, deriv, targets=None, nthreads=0):
    """Derivative of the direct sum at the targets: d u_i/dx_i or d u_i/dy_i with the
    sources fixed (deriv = DX, DY), or d u_i/dd (deriv = DD).  Layout as direct_apply."""
    k1, k2, k3, d = medium
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    q = np.asarray(q)
    one = q.ndim == 1
    q2 = _c(q.reshape(1, -1) if one else q, np.complex128)
    n = x.size
    nvec = q2.shape[0]
    tg = None if targets is None else _c(targets, np.int64)
    nt = n if tg is None else tg.size
    u = np.zeros((nvec, nt), np.complex128)
    st = lib().orc_direct_apply_deriv(k1, k2, k3, d, n, _ptr(x), _ptr(y), nvec, _ptr(q2), nt,
                                      _ptr(tg) if tg is not None else None, deriv, nthreads, _ptr(u))
    if st != 0:
        raise RuntimeError("oracle quadrature did not converge")
    return u[0] if one else u


# --- tree and lists ----------------------------------------------------------------
def tree_build(x, y, d, L):
    """Uniform strip-forest quadtree (Algorithm 1 step 1; reading G11).

    Returns (x_origin, R, perm, leaf_start)."""
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    n = x.size
    mn, mx = x.min(), x.max()
    R = int(np.floor(mx / d) - np.floor(mn / d)) + 1
    nleaf = R << (2 * L)
    hdr = np.zeros(2)
    perm = np.zeros(n, np.int64)
    ls = np.zeros(nleaf + 1, np.int64)
    lib().orc_tree_build(n, _ptr(x), _ptr(y), d, L, _ptr(hdr), _ptr(perm), _ptr(ls))
    return hdr[0], int(hdr[1]), perm, ls


def vlist(R, level):
    """V (interaction) list at a level: rows of (target box, term, source box)."""
    n = lib().orc_vlist(R, level, 0, None)
    out = np.zeros((max(n, 1), 3), np.int64)
    lib().orc_vlist(R, level, n, _ptr(out))
    return out[:n]


def ulist(R, L):
    """U (direct interaction) list at the leaf level: (target leaf, term, source leaf)."""
    n = lib().orc_ulist(R, L, 0, None)
    out = np.zeros((max(n, 1), 3), np.int64)
    lib().orc_ulist(R, L, n, _ptr(out))
    return out[:n]


# --- expansions and translations ---------------------------------------------------
def m2l_image_table(medium, term, dx, h, P):
    """Layered M2L matrix A_pq (Lemma M2L; reading G2), p, q in -P..P."""
    k1, k2, k3, d = medium
    np_ = 2 * P + 1
    out = np.zeros((np_, np_), np.complex128)
    st = lib().orc_m2l_image_table(k1, k2, k3, d, term, dx, h, P, _ptr(out))
    if st != 0:
        raise RuntimeError("oracle quadrature did not converge")
    return out


def m2l_free_table(k, cx_, cy_, P):
    np_ = 2 * P + 1
    out = np.zeros((np_, np_), np.complex128)
    lib().orc_m2l_free_table(k, cx_, cy_, P, _ptr(out))
    return out


def s2m(x, y, q, centre, k, P):
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    q = _c(q, np.complex128)
    out = np.zeros(2 * P + 1, np.complex128)
    lib().orc_s2m(x.size, _ptr(x), _ptr(y), _ptr(q), centre[0], centre[1], k, P, _ptr(out))
    return out


def l2t(x, y, Lc, centre, k, P):
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    Lc = _c(Lc, np.complex128)
    out = np.zeros(x.size, np.complex128)
    lib().orc_l2t(x.size, _ptr(x), _ptr(y), _ptr(Lc), centre[0], centre[1], k, P, _ptr(out))
    return out


def shift(coef, sx, sy, k, P):
    """M2M (shift = child - parent) or L2L (shift = parent - child) translation."""
    c = _c(coef, np.complex128)
    out = np.zeros(2 * P + 1, np.complex128)
    lib().orc_shift(_ptr(c), sx, sy, k, P, _ptr(out))
    return out


def fmm_apply(medium, x, y, q, L, P):
    """Plain FMM (Algorithm 1) at depth L and order P. q: [nvec, n] or [n]."""
    k1, k2, k3, d = medium
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    q = np.asarray(q)
    one = q.ndim == 1
    q2 = _c(q.reshape(1, -1) if one else q, np.complex128)
    u = np.zeros_like(q2)
    st = lib().orc_fmm_apply(k1, k2, k3, d, x.size, _ptr(x), _ptr(y), L, P, q2.shape[0], _ptr(q2),
                             _ptr(u))
    if st != 0:
        raise RuntimeError("oracle quadrature did not converge")
    return u[0] if one else u


def psi_e4(medium, p, X, Y):
    """Evanescent part of the three-layer local basis Psi_p (Sec. 5, Fig. order3layer)."""
    k1, k2, k3, d = medium
    return _green_out(lib().orc_psi_e4, k1, k2, k3, d, p, X, Y)


# --- cross-layer operator (Example 4 as printed: layer-1 sources, layer-2 targets) ---
G2T, G2B, G1 = 1, 2, 4


def cross_field(medium, x, y, x0, y0, which=G2T | G2B, dy=False):
    """The printed Example 4 fields for a source (x0, y0 > 0) in layer 1: g_2^t, g_2^b (target
    in layer 2) or g_1^s (target in layer 1), selected by the bits of `which`; dy=True gives
    the target y-derivative."""
    k1, k2, k3, d = medium
    return _green_out(lib().orc_cross_field, k1, k2, k3, d, x, y, x0, y0, which, int(dy))


def cross_direct(medium, xs, ys, xt, yt, q, targets=None, nthreads=0):
    """u_i = sum_j q_j (g_2^t + g_2^b)(x_i, x_j), sources in layer 1, targets in layer 2.
    q: [nvec, ns] or [ns]; returns [nvec, ntargets] (or [ntargets])."""
    k1, k2, k3, d = medium
    xs, ys, xt, yt = (_c(a, np.float64) for a in (xs, ys, xt, yt))
    q = np.asarray(q)
    one = q.ndim == 1
    q2 = _c(q.reshape(1, -1) if one else q, np.complex128)
    tg = None if targets is None else _c(targets, np.int64)
    nt = xt.size if tg is None else tg.size
    u = np.zeros((q2.shape[0], nt), np.complex128)
    st = lib().orc_cross_direct(k1, k2, k3, d, xs.size, _ptr(xs), _ptr(ys), xt.size, _ptr(xt), _ptr(yt),
                                q2.shape[0], _ptr(q2), nt, _ptr(tg) if tg is not None else None, nthreads,
                                _ptr(u))
    if st != 0:
        raise RuntimeError("oracle quadrature did not converge")
    return u[0] if one else u


# --- adaptive tree (Algorithm 1 step 1) ------------------------------------------
def adaptive_tree(x, y, d, s, Lmax):
    """Adaptive strip-forest tree: a box with more than s points below level Lmax is split.
    Returns (hdr = (x_origin, R), boxes [nbox, 4] = (level, col, row, leaf), perm, pstart)."""
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    cap = 1024
    while True:
        hdr = np.zeros(2)
        boxes = np.zeros((cap, 4), np.int64)
        perm = np.zeros(x.size, np.int64)
        pstart = np.zeros(cap + 1, np.int64)
        nb = lib().orc_adaptive_tree(x.size, _ptr(x), _ptr(y), d, s, Lmax, cap, _ptr(hdr), _ptr(boxes),
                                     _ptr(perm), _ptr(pstart))
        if nb >= 0:
            return (hdr[0], int(hdr[1])), boxes[:nb].copy(), perm, pstart[:nb + 1].copy()
        cap *= 4


def adaptive_lists(x, y, d, s, Lmax, which):
    """V (which = 0) or U (which = 1) rows (target box, term, source box) of the adaptive tree,
    by dual traversal from every pair of roots; sorted."""
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    cnt = lib().orc_adaptive_lists(x.size, _ptr(x), _ptr(y), d, s, Lmax, which, 0, None)
    out = np.zeros((max(cnt, 1), 3), np.int64)
    lib().orc_adaptive_lists(x.size, _ptr(x), _ptr(y), d, s, Lmax, which, cnt, _ptr(out))
    return out[:cnt]
