"""FP64 CPU oracle of the multilayer shallow-water LBM step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY. This package checks the CUDA path; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import it. It shares no code with the product package.

Parameters are plain dicts (the same data the CUDA binding receives):
    n, lattice (1 = D1Q3, 2 = D2Q9), nx, ny, tau,
    gamma[n]  (gamma_{i,i+1}), S[i][k-1] (S_{ik}, i = 0..n-1, k = 1..n-i),
    mu[n], beta[n], nw, mw, hstar, and optionally a sinusoidal substrate
    sub_amp, sub_kx, sub_ky (z_0 = sub_amp cos 2 pi (kx x / nx + ky y / ny))
    and the wetting potential's kind: wet_kind 0 (the power law with
    exponents nw, mw) or 1 (exponential, decay rate kappa).
Arrays are float64 numpy arrays in the layouts documented in oracle.h.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ORC_MAXN = 8
_lib = None


class orc_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("gamma", ctypes.c_double * ORC_MAXN),
        ("S", (ctypes.c_double * ORC_MAXN) * ORC_MAXN),
        ("mu", ctypes.c_double * ORC_MAXN),
        ("beta", ctypes.c_double * ORC_MAXN),
        ("nw", ctypes.c_int),
        ("mw", ctypes.c_int),
        ("hstar", ctypes.c_double),
        ("sub_amp", ctypes.c_double),
        ("sub_kx", ctypes.c_int),
        ("sub_ky", ctypes.c_int),
        ("wet_kind", ctypes.c_int),
        ("kappa", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(orc_params)
        sig = {
            "orc_phi": (ctypes.c_double, [P, ctypes.c_int, ctypes.c_double]),
            "orc_dphi": (ctypes.c_double, [P, ctypes.c_int, ctypes.c_double]),
            "orc_spreading_from_tensions": (None, [P, _D]),
            "orc_Q": (ctypes.c_int, [P]),
            "orc_build_D": (None, [P, _D, _D]),
            "orc_friction": (ctypes.c_int, [P, _D, _D, _D, _D, _D]),
            "orc_pressures": (None, [P, _D, _D, _D, _D, _D, _D, _D]),
            "orc_pressures_sub": (None, [P, _D, _D, _D, _D, ctypes.c_double, _D, _D, _D]),
            "orc_substrate": (ctypes.c_double, [P, ctypes.c_long, ctypes.c_long]),
            "orc_equilibrium": (None, [P, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _D]),
            "orc_init": (None, [P, _D, _D]),
            "orc_moments": (None, [P, _D, _D, _D, _D]),
            "orc_step": (ctypes.c_int, [P, _D, _D]),
            "orc_run": (ctypes.c_int, [P, _D, ctypes.c_long]),
            "orc_set_threads": (None, [ctypes.c_int]),
            "orc_max_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def make_params(p: dict) -> orc_params:
    s = orc_params()
    n = int(p["n"])
    if not 1 <= n <= ORC_MAXN:
        raise ValueError("n out of range")
    s.n = n
    s.lattice = int(p.get("lattice", 2))
    s.nx = int(p.get("nx", 1))
    s.ny = int(p.get("ny", 1))
    s.tau = float(p.get("tau", 1.0))
    for i in range(n):
        s.gamma[i] = float(p["gamma"][i])
        s.mu[i] = float(p["mu"][i])
        s.beta[i] = float(p["beta"][i])
    S = p.get("S")
    if S is not None:
        for i in range(n):
            for k in range(1, n - i + 1):
                s.S[i][k - 1] = float(S[i][k - 1])
    s.nw = int(p["nw"])
    s.mw = int(p["mw"])
    s.hstar = float(p["hstar"])
    s.sub_amp = float(p.get("sub_amp", 0.0))
    s.wet_kind = int(p.get("wet_kind", 0))
    s.kappa = float(p.get("kappa", 0.0))
    s.sub_kx = int(p.get("sub_kx", 0))
    s.sub_ky = int(p.get("sub_ky", 0))
    return s


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _vec(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


def Q(p):
    return 3 if int(p.get("lattice", 2)) == 1 else 9


def lattice(p):
    """(cx, cy, w) of the lattice as numpy arrays (oracle's own tables)."""
    s = make_params(p)
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    lib()  # ensure loaded
    fn = _lib.orc_lattice
    fn.restype = None
    fn.argtypes = [ctypes.POINTER(orc_params), ctypes.POINTER(ctypes.c_int),
                   ctypes.POINTER(ctypes.c_int), _D]
    fn(ctypes.byref(s), cx, cy, w)
    q = Q(p)
    return (np.array(cx[:q]), np.array(cy[:q]), np.array(w[:q]))


def phi(p, k, h):
    s = make_params(p)
    return lib().orc_phi(ctypes.byref(s), int(k), float(h))


def dphi(p, k, h):
    s = make_params(p)
    return lib().orc_dphi(ctypes.byref(s), int(k), float(h))


def spreading_from_tensions(p, gamma_full):
    """Returns (S as list of rows, gamma_{i,i+1} list) from the (n+2)^2 table."""
    s = make_params(dict(p, S=None))
    g = _vec(gamma_full)
    n = s.n
    assert g.size == (n + 2) ** 2
    lib().orc_spreading_from_tensions(ctypes.byref(s), _ptr(g))
    S = [[s.S[i][k - 1] for k in range(1, n - i + 1)] for i in range(n)]
    gam = [s.gamma[i] for i in range(n)]
    return S, gam


def build_D(p, h):
    s = make_params(p)
    h = _vec(h, s.n)
    D = np.zeros((3 * s.n, 3 * s.n))
    lib().orc_build_D(ctypes.byref(s), _ptr(h), _ptr(D))
    return D


def friction(p, h, Jx, Jy=None):
    s = make_params(p)
    n = s.n
    h = _vec(h, n)
    Jx = _vec(Jx, n)
    Jy = _vec(np.zeros(n) if Jy is None else Jy, n)
    Rx = np.zeros(n)
    Ry = np.zeros(n)
    rc = lib().orc_friction(ctypes.byref(s), _ptr(h), _ptr(Jx), _ptr(Jy),
                            _ptr(Rx), _ptr(Ry))
    if rc != 0:
        raise FloatingPointError("singular boundary-condition matrix")
    return Rx, Ry


def pressures_sub(p, h, gzx, gzy, lz, g0sq):
    s = make_params(p)
    n = s.n
    args = [_vec(a, n) for a in (h, gzx, gzy, lz)]
    La, Pi, pp = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_pressures_sub(ctypes.byref(s), *[_ptr(a) for a in args], float(g0sq), _ptr(La),
                            _ptr(Pi), _ptr(pp))
    return La, Pi, pp


def substrate(p):
    """z_0 on the lattice, [ny][nx]."""
    s = make_params(p)
    return np.array([[lib().orc_substrate(ctypes.byref(s), x, y) for x in range(s.nx)]
                     for y in range(s.ny)])


def pressures(p, h, gzx, gzy, lz):
    s = make_params(p)
    n = s.n
    args = [_vec(a, n) for a in (h, gzx, gzy, lz)]
    La = np.zeros(n)
    Pi = np.zeros(n)
    pp = np.zeros(n)
    lib().orc_pressures(ctypes.byref(s), *[_ptr(a) for a in args], _ptr(La),
                        _ptr(Pi), _ptr(pp))
    return La, Pi, pp


def equilibrium(p, h, Ux, Uy=0.0):
    s = make_params(p)
    feq = np.zeros(9)
    lib().orc_equilibrium(ctypes.byref(s), float(h), float(Ux), float(Uy),
                          _ptr(feq))
    return feq[: Q(p)]


def f_shape(p):
    return (int(p["n"]), Q(p), int(p.get("ny", 1)), int(p.get("nx", 1)))


def init(p, h0):
    s = make_params(p)
    h0 = _vec(h0, s.n * s.nx * s.ny)
    f = np.zeros(f_shape(p))
    lib().orc_init(ctypes.byref(s), _ptr(h0), _ptr(f))
    return f


def moments(p, f):
    s = make_params(p)
    f = np.ascontiguousarray(f, dtype=np.float64)
    shp = (s.n, s.ny, s.nx)
    h = np.zeros(shp)
    Jx = np.zeros(shp)
    Jy = np.zeros(shp)
    lib().orc_moments(ctypes.byref(s), _ptr(f), _ptr(h), _ptr(Jx), _ptr(Jy))
    return h, Jx, Jy


def step(p, f):
    s = make_params(p)
    fin = np.ascontiguousarray(f, dtype=np.float64)
    assert fin.shape == f_shape(p)
    fout = np.zeros_like(fin)
    rc = lib().orc_step(ctypes.byref(s), _ptr(fin), _ptr(fout))
    if rc != 0:
        raise FloatingPointError("oracle step failed")
    return fout


def run(p, f, nsteps):
    s = make_params(p)
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    assert g.shape == f_shape(p)
    rc = lib().orc_run(ctypes.byref(s), _ptr(g), int(nsteps))
    if rc != 0:
        raise FloatingPointError("oracle run failed")
    return g


def heights(p, f):
    return moments(p, f)[0]


def set_threads(n):
    """Threads of the oracle's per-cell loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def max_threads():
    return int(lib().orc_max_threads())
