"""FP64 CPU oracle for the Q2X moments -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2107_10942_gb300``)
never imports it and shares no code with it.

The oracle computes each coefficient from its definition, Eq. (bas4): the
integral of density x R_n^{-m}(y - c) (double layer: density x n.grad R_n^{-m})
over the element by collapsed Gauss-Legendre quadrature (Sec. 4.2.1), with
R_n^m from Eq. (bas1)-(bas2) in Cartesian form -- never from the paper's
recursions.  The numerical work lives in ``q2x_oracle.c`` (plain C99 +
OpenMP); this module builds it with gcc and wraps it with ctypes.

Packing of the (p+1)^2 real outputs: index k = n*n + n + m holds Re F_n^m for
m >= 0 and Im F_n^{|m|} for m < 0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

NORM_COEFF = 0
NORM_MOMENT = 1
KIND = {"segment": 0, "triangle": 1, "tetra": 2}
NVERT = {0: 2, 1: 3, 2: 4}
PMAX = 40


def build(force: bool = False) -> str:
    """Compile q2x_oracle.c into _build/liboracle.so (gcc, C99 + OpenMP)."""
    src = os.path.join(_HERE, "q2x_oracle.c")
    hdr = os.path.join(_HERE, "harmonics_body.h")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            L.oracle_gauss_legendre.argtypes = [i, p, p]
            L.oracle_rnm.argtypes = [d, d, d, i, p, p]
            L.oracle_snm.argtypes = [d, d, d, i, p, p]
            L.oracle_moments.argtypes = [i, i, i, i, i, i, i64, p, i64, p, p, i64, p, p, p, p, i]
            L.oracle_moments_cs.argtypes = [i, i, i, i, i, i64, p, p, i64, p, p, p, p, p, i]
            L.oracle_farfield.argtypes = [i, p, p, i64, p, p, p]
            L.oracle_potential.argtypes = [i, i, i, i64, p, i64, p, p, i64, i64, i64, p, p, i]
            L.oracle_max_threads.argtypes = []
            for f in (L.oracle_gauss_legendre, L.oracle_rnm, L.oracle_snm, L.oracle_moments,
                      L.oracle_moments_cs, L.oracle_farfield, L.oracle_potential, L.oracle_max_threads):
                f.restype = ctypes.c_int
            _LIB = L
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def gauss_legendre(k: int):
    """k-point Gauss-Legendre nodes and weights on [0, 1]."""
    x = np.zeros(k)
    w = np.zeros(k)
    if lib().oracle_gauss_legendre(k, _ptr(x), _ptr(w)):
        raise ValueError("bad k")
    return x, w


def rnm(xyz, p: int) -> np.ndarray:
    """Complex R_n^m(x,y,z) of Eq. (bas1), packed k = n*n+n+m over -n..n."""
    np_ = (p + 1) ** 2
    re = np.zeros(np_)
    im = np.zeros(np_)
    if lib().oracle_rnm(float(xyz[0]), float(xyz[1]), float(xyz[2]), p, _ptr(re), _ptr(im)):
        raise ValueError("bad p")
    return re + 1j * im


def snm(xyz, p: int) -> np.ndarray:
    """Complex S_n^m(x,y,z) of Eq. (bas1), packed k = n*n+n+m over -n..n."""
    np_ = (p + 1) ** 2
    re = np.zeros(np_)
    im = np.zeros(np_)
    if lib().oracle_snm(float(xyz[0]), float(xyz[1]), float(xyz[2]), p, _ptr(re), _ptr(im)):
        raise ValueError("bad p")
    return re + 1j * im


def moments(kind, vxyz, idx, sigma, p, leaf_off=None, leaf_c=None, leaf_p=None,
            layer=0, density=0, norm=NORM_COEFF, nq=0, nthreads=0) -> np.ndarray:
    """Leaf (or per-element) Q2X coefficients by quadrature.

    kind: "segment" | "triangle" | "tetra" (or 0/1/2); vxyz: (3, n_vert) float64;
    idx: (nv, n_elem) int32; sigma: (n_elem,) for constant density, (n_vert,) for
    linear; leaf_off: (n_leaves+1,) int64 or None (one expansion per element);
    leaf_c: (3, n_leaves) centres (per element when leaf_off is None).
    Returns (n_leaves, (p+1)^2) float64."""
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    vxyz = _f64(vxyz)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    sigma = _f64(sigma)
    n_vert = vxyz.shape[1]
    n_elem = idx.shape[1]
    if leaf_off is None:
        n_leaves = n_elem
        lo = None
    else:
        lo = np.ascontiguousarray(leaf_off, dtype=np.int64)
        n_leaves = lo.shape[0] - 1
    lc = _f64(leaf_c)
    assert lc.shape == (3, n_leaves)
    lp = None if leaf_p is None else np.ascontiguousarray(leaf_p, dtype=np.int32)
    out = np.zeros((n_leaves, (p + 1) ** 2))
    rc = lib().oracle_moments(k, layer, density, norm, p, nq, n_vert, _ptr(vxyz), n_elem,
                              _ptr(idx), _ptr(sigma), n_leaves, _ptr(lo), _ptr(lc), _ptr(lp),
                              _ptr(out), nthreads)
    if rc:
        raise ValueError("oracle_moments failed: %d" % rc)
    return out


def moments_cs(kind, vre, vim, idx, sigma, elem_c, p, density=0, norm=NORM_COEFF, nq=0,
               nthreads=0) -> np.ndarray:
    """Per-element single-layer moments at complex vertices vre + i*vim
    (complex-step derivatives).  Returns complex (n_elem, (p+1)^2)."""
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    vre = _f64(vre)
    vim = _f64(vim)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    sigma = _f64(sigma)
    ec = _f64(elem_c)
    n_elem = idx.shape[1]
    ore = np.zeros((n_elem, (p + 1) ** 2))
    oim = np.zeros((n_elem, (p + 1) ** 2))
    rc = lib().oracle_moments_cs(k, density, norm, p, nq, vre.shape[1], _ptr(vre), _ptr(vim),
                                 n_elem, _ptr(idx), _ptr(sigma), _ptr(ec), _ptr(ore), _ptr(oim),
                                 nthreads)
    if rc:
        raise ValueError("oracle_moments_cs failed: %d" % rc)
    return ore + 1j * oim


def potential(kind, vxyz, idx, sigma, tgt, e0=0, e1=None, density=0, nq=12, nthreads=0) -> np.ndarray:
    """Single-layer potential (1/4pi) sum_e int_e sigma / |r - y| of the
    elements [e0, e1) at targets tgt (N, 3), by collapsed Gauss product rules
    with nq nodes per direction (for targets well separated from the
    elements; near targets need ``oracle.nearfield``)."""
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    vxyz = _f64(vxyz)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    sigma = _f64(sigma)
    tgt = _f64(np.atleast_2d(tgt))
    n_elem = idx.shape[1]
    e1 = n_elem if e1 is None else int(e1)
    out = np.zeros(tgt.shape[0])
    rc = lib().oracle_potential(k, int(density), int(nq), vxyz.shape[1], _ptr(vxyz), n_elem, _ptr(idx),
                                _ptr(sigma), int(e0), e1, tgt.shape[0], _ptr(tgt), _ptr(out), nthreads)
    if rc:
        raise ValueError("oracle_potential failed: %d" % rc)
    return out


def farfield(coef, c, pts, p) -> np.ndarray:
    """Series sum_{n<=p} sum_m F_n^m S_n^m(r - c) at pts (N,3) for packed
    COEFF-normalised coefficients; returns (real part, imaginary part)."""
    coef = _f64(coef)
    c = _f64(c)
    pts = _f64(np.atleast_2d(pts))
    out = np.zeros(pts.shape[0])
    oim = np.zeros(pts.shape[0])
    if lib().oracle_farfield(p, _ptr(coef), _ptr(c), pts.shape[0], _ptr(pts), _ptr(out), _ptr(oim)):
        raise ValueError("bad p")
    return out, oim


# ---------------------------------------------------------------- translation

def unpack_complex(coef, p):
    """Packed real rows (..., (p+1)^2) -> complex F_n^m for every m in -n..n
    (same index k = n*n+n+m), using F_n^{-m} = (-1)^m conj(F_n^m), Eq. (bas2.1)."""
    coef = np.asarray(coef, dtype=np.float64)
    F = np.zeros(coef.shape, dtype=np.complex128)
    for n in range(p + 1):
        k0 = n * n + n
        F[..., k0] = coef[..., k0]
        for m in range(1, n + 1):
            v = coef[..., k0 + m] + 1j * coef[..., k0 - m]
            F[..., k0 + m] = v
            F[..., k0 - m] = (-1) ** m * np.conj(v)
    return F


def pack_complex(F, p):
    """Complex F_n^m (all m) -> packed real rows (Re at m >= 0, Im F^{|m|} at m < 0)."""
    out = np.zeros(F.shape, dtype=np.float64)
    for n in range(p + 1):
        k0 = n * n + n
        out[..., k0] = F[..., k0].real
        for m in range(1, n + 1):
            out[..., k0 + m] = F[..., k0 + m].real
            out[..., k0 - m] = F[..., k0 + m].imag
    return out


def translate(coef, src_c, dst_c, p, norm=NORM_COEFF):
    """Expansion coefficients about dst_c from those about src_c, one row per
    expansion (coef (N, (p+1)^2) packed, src_c and dst_c (3, N)), exact for
    every degree n <= p.

    With x = y - src_c and t = src_c - dst_c, the Taylor series of R_n^m in
    (xi, eta, z) and the derivative rules of Eq. (bas5) give the finite sum
        R_n^m(x + t) = sum_{k=0..n} sum_{l=-k..k} R_k^l(t) R_{n-k}^{m-l}(x),
    so, term by term in Eq. (bas4):
        MOMENT: M_n^m(dst) = sum_{k,l} R_k^l(t) M_{n-k}^{m-l}(src)
        COEFF : F_n^m(dst) = sum_{k,l} (-1)^k R_k^l(t) F_{n-k}^{m+l}(src)
    (the double-layer coefficients translate the same way: n.grad commutes
    with the shift).  Plain loops over (n, m, k, l), vectorised over rows."""
    coef = np.atleast_2d(np.asarray(coef, dtype=np.float64))
    src_c = np.asarray(src_c, dtype=np.float64).reshape(3, -1)
    dst_c = np.asarray(dst_c, dtype=np.float64).reshape(3, -1)
    N = coef.shape[0]
    F = unpack_complex(coef, p)
    R = np.stack([rnm(src_c[:, i] - dst_c[:, i], p) for i in range(N)])  # (N, (p+1)^2)
    G = np.zeros_like(F)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            acc = np.zeros(N, dtype=np.complex128)
            for k in range(n + 1):
                nn = n - k
                sk = (-1) ** k if norm == NORM_COEFF else 1
                for l in range(-k, k + 1):
                    mm = m + l if norm == NORM_COEFF else m - l
                    if abs(mm) > nn:
                        continue
                    acc += sk * R[:, k * k + k + l] * F[:, nn * nn + nn + mm]
            G[:, n * n + n + m] = acc
    return pack_complex(G, p)
