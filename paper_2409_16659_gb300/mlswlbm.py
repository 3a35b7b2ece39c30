"""Thin ctypes binding of the C ABI in include/mlswlbm.h (same names).

Argument marshalling only: every step of the solver runs in the CUDA library
libmlswlbm.so. Loading fails loudly if the library is missing; there is no
CPU path.

Parameter dicts (also accepted by the oracle) use the keys
    n, lattice (1 = D1Q3, 2 = D2Q9), nx, ny, tau, gamma[n], S[i][k-1],
    mu[n], beta[n], nw, mw, hstar (and optional flags, a sinusoidal
    substrate sub_amp, sub_kx, sub_ky, and the wetting potential's kind
    wet_kind 0 = power law, 1 = exponential with decay rate kappa).
Host arrays are numpy float32 (or anything numpy can view as such);
device arrays are torch CUDA tensors (float32, contiguous). PyTorch is used
only for device memory and streams.
"""
import ctypes
import os

import numpy as np

MLSW_MAX_LAYERS = 5
MLSW_D1Q3 = 1
MLSW_D2Q9 = 2
MLSW_FLAG_SKIP_STABILITY_CHECK = 1
MLSW_FLAG_NO_PERSISTENT = 2
MLSW_BATCH_TILE8 = 1
MLSW_BATCH_AUTOTUNE = 2

MLSW_OK = 0
MLSW_ERR_ARG = -1
MLSW_ERR_NOMEM = -2
MLSW_ERR_CUDA = -3
MLSW_ERR_NONFINITE = -4
MLSW_ERR_UNSTABLE = -5
MLSW_ERR_TIMEOUT = -6
MLSW_ERR_UNSUPPORTED = -7

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmlswlbm.so")


class mlsw_params(ctypes.Structure):
    _fields_ = [
        ("n_layers", ctypes.c_int),
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("gamma", ctypes.c_double * MLSW_MAX_LAYERS),
        ("spread", (ctypes.c_double * MLSW_MAX_LAYERS) * MLSW_MAX_LAYERS),
        ("mu", ctypes.c_double * MLSW_MAX_LAYERS),
        ("beta", ctypes.c_double * MLSW_MAX_LAYERS),
        ("wet_n", ctypes.c_int),
        ("wet_m", ctypes.c_int),
        ("hstar", ctypes.c_double),
        ("flags", ctypes.c_int),
        ("sub_amp", ctypes.c_double),
        ("sub_kx", ctypes.c_int),
        ("sub_ky", ctypes.c_int),
        ("wet_kind", ctypes.c_int),
        ("wet_kappa", ctypes.c_double),
    ]


class MlswError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, mlswlbm_strerror(code), code))


_lib = None
_P = ctypes.POINTER(mlsw_params)
_H = ctypes.c_void_p
_F = ctypes.POINTER(ctypes.c_float)
_D = ctypes.POINTER(ctypes.c_double)

EXPORTS = {
    "mlswlbm_spreading_from_tensions": (ctypes.c_int, [ctypes.c_int, _D, _P]),
    "mlswlbm_check_params": (ctypes.c_int, [_P]),
    "mlswlbm_create": (ctypes.c_int, [_P, _F, ctypes.c_void_p, ctypes.POINTER(_H)]),
    "mlswlbm_step": (ctypes.c_int, [_H, ctypes.c_long]),
    "mlswlbm_get_heights": (ctypes.c_int, [_H, _F]),
    "mlswlbm_get_heights_device": (ctypes.c_int, [_H, ctypes.c_void_p]),
    "mlswlbm_set_heights_device": (ctypes.c_int, [_H, ctypes.c_void_p]),
    "mlswlbm_set_heights": (ctypes.c_int, [_H, _F]),
    "mlswlbm_get_state": (ctypes.c_int, [_H, _F]),
    "mlswlbm_set_state": (ctypes.c_int, [_H, _F]),
    "mlswlbm_save_state": (ctypes.c_int, [_H, _F, _F]),
    "mlswlbm_load_state": (ctypes.c_int, [_H, _F, _F]),
    "mlswlbm_get_diagnostics": (ctypes.c_int, [_H, _D, _D, _D]),
    "mlswlbm_status": (ctypes.c_int, [_H]),
    "mlswlbm_get_free_energy": (ctypes.c_int, [_H, _D]),
    "mlswlbm_get_spectrum": (ctypes.c_int, [_H, ctypes.c_int, _D]),
    "mlswlbm_get_radial_profile": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int, _D,
                                                  ctypes.POINTER(ctypes.c_longlong)]),
    "mlswlbm_fit_cap_angle": (ctypes.c_int, [_D, _D, ctypes.c_int, ctypes.c_double, _D, _D]),
    "mlswlbm_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint, ctypes.c_void_p]),
    "mlswlbm_step_until": (ctypes.c_int, [_H, ctypes.c_long, ctypes.c_long, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_long), _D]),
    "mlswlbm_set_stream": (ctypes.c_int, [_H, ctypes.c_void_p]),
    "mlswlbm_debug_bounds_violations": (ctypes.c_int, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "mlswlbm_launch_count": (ctypes.c_long, [_H]),
    "mlswlbm_destroy": (None, [_H]),
    "mlswlbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mlswlbm_diagnostics_noalloc": (ctypes.c_int, [_P, ctypes.c_void_p, _F,
                                                   ctypes.c_void_p, ctypes.c_void_p]),
    "mlswlbm_friction_eval": (ctypes.c_int, [_P, ctypes.c_long, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "mlswlbm_batch_create": (ctypes.c_int, [ctypes.c_int, _P, ctypes.POINTER(_F), ctypes.c_int,
                                            ctypes.c_void_p, ctypes.POINTER(_H)]),
    "mlswlbm_batch_step": (ctypes.c_int, [_H, ctypes.c_long]),
    "mlswlbm_batch_get_heights": (ctypes.c_int, [_H, ctypes.c_int, _F]),
    "mlswlbm_batch_get_heights_device": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p]),
    "mlswlbm_batch_set_heights_device": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p]),
    "mlswlbm_batch_get_heights_device_many": (ctypes.c_int, [_H, ctypes.c_int,
                                                             ctypes.POINTER(ctypes.c_int),
                                                             ctypes.c_void_p]),
    "mlswlbm_batch_set_heights_device_many": (ctypes.c_int, [_H, ctypes.c_int,
                                                             ctypes.POINTER(ctypes.c_int),
                                                             ctypes.c_void_p]),
    "mlswlbm_batch_select": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mlswlbm_batch_modes": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), _D]),
    "mlswlbm_batch_status": (ctypes.c_int, [_H]),
    "mlswlbm_batch_tile_rows": (ctypes.c_int, [_H, ctypes.c_int]),
    "mlswlbm_batch_launch_count": (ctypes.c_long, [_H]),
    "mlswlbm_batch_groups": (ctypes.c_int, [_H]),
    "mlswlbm_batch_destroy": (None, [_H]),
}


def lib():
    """Loads libmlswlbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmlswlbm.so is not built; run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc, where):
    if rc != MLSW_OK:
        raise MlswError(rc, where)


def mlswlbm_strerror(code):
    return lib().mlswlbm_strerror(int(code)).decode()


def make_params(p):
    """dict -> mlsw_params (marshalling only)."""
    s = mlsw_params()
    n = int(p["n"])
    if not 1 <= n <= MLSW_MAX_LAYERS:
        raise ValueError("n must be in 1..%d" % MLSW_MAX_LAYERS)
    s.n_layers = n
    s.lattice = int(p.get("lattice", MLSW_D2Q9))
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
                s.spread[i][k - 1] = float(S[i][k - 1])
    s.wet_n = int(p["nw"])
    s.wet_m = int(p["mw"])
    s.hstar = float(p["hstar"])
    s.flags = int(p.get("flags", 0))
    s.sub_amp = float(p.get("sub_amp", 0.0))
    s.sub_kx = int(p.get("sub_kx", 0))
    s.sub_ky = int(p.get("sub_ky", 0))
    s.wet_kind = int(p.get("wet_kind", 0))
    s.wet_kappa = float(p.get("kappa", 0.0))
    return s


def _host_f32(a, size=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if size is not None and a.size != size:
        raise ValueError("expected %d floats, got %d" % (size, a.size))
    return a


def _fptr(a):
    return a.ctypes.data_as(_F)


def _dev_ptr(t, numel=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d elements, got %d" % (numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def mlswlbm_spreading_from_tensions(n, gamma_full, p=None):
    """Returns (S rows, gamma list) for the (n+2)^2 tension table."""
    s = make_params(p) if p is not None else mlsw_params()
    g = np.ascontiguousarray(gamma_full, dtype=np.float64)
    if g.size != (n + 2) ** 2:
        raise ValueError("tension table must have (n+2)^2 entries")
    _check(lib().mlswlbm_spreading_from_tensions(int(n), g.ctypes.data_as(_D),
                                                 ctypes.byref(s)),
           "mlswlbm_spreading_from_tensions")
    S = [[s.spread[i][k - 1] for k in range(1, n - i + 1)] for i in range(n)]
    return S, [s.gamma[i] for i in range(n)]


def mlswlbm_check_params(p):
    s = make_params(p)
    return lib().mlswlbm_check_params(ctypes.byref(s))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)  # torch.cuda.Stream


class Solver:
    """Owns one mlsw_handle. Methods map 1:1 to the C entry points."""

    def __init__(self, p, h_init, stream=None):
        self.p = dict(p)
        self.n = int(p["n"])
        self.nx = int(p.get("nx", 1))
        self.ny = int(p.get("ny", 1))
        self.Q = 3 if int(p.get("lattice", 2)) == MLSW_D1Q3 else 9
        self.ncell = self.nx * self.ny
        self._params = make_params(p)
        h = _host_f32(h_init, self.n * self.ncell)
        self._h = _H()
        _check(lib().mlswlbm_create(ctypes.byref(self._params), _fptr(h),
                                    _stream_ptr(stream), ctypes.byref(self._h)),
               "mlswlbm_create")

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if self._h:
            lib().mlswlbm_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- entry points --------------------------------------------------------
    def step(self, nsteps=1):
        _check(lib().mlswlbm_step(self._h, int(nsteps)), "mlswlbm_step")

    def get_heights(self, out=None):
        shape = (self.n, self.ny, self.nx)
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        rc = lib().mlswlbm_get_heights(self._h, _fptr(_checked_out(out, self.n * self.ncell)))
        _check(rc, "mlswlbm_get_heights")
        return out

    def get_heights_device(self, dev_out):
        _check(lib().mlswlbm_get_heights_device(self._h, _dev_ptr(dev_out, self.n * self.ncell)),
               "mlswlbm_get_heights_device")
        return dev_out

    def set_heights_device(self, dev_in):
        _check(lib().mlswlbm_set_heights_device(self._h, _dev_ptr(dev_in, self.n * self.ncell)),
               "mlswlbm_set_heights_device")

    def set_heights(self, h):
        a = _host_f32(h, self.n * self.ncell)
        _check(lib().mlswlbm_set_heights(self._h, _fptr(a)), "mlswlbm_set_heights")

    def free_energy(self):
        F = ctypes.c_double()
        _check(lib().mlswlbm_get_free_energy(self._h, ctypes.byref(F)), "mlswlbm_get_free_energy")
        return F.value

    def spectrum(self, nbins=None):
        """mlswlbm_get_spectrum: radially averaged power spectrum of every
        layer, array [n][nbins] (default nbins = min(nx, ny) // 2, or nx // 2
        for D1Q3)."""
        nx, ny = self.nx, self.ny
        if nbins is None:
            nbins = max(1, (min(nx, ny) if ny > 1 else nx) // 2)
        out = np.empty((self.n, int(nbins)), dtype=np.float64)
        _check(lib().mlswlbm_get_spectrum(self._h, int(nbins), out.ctypes.data_as(_D)),
               "mlswlbm_get_spectrum")
        return out

    def radial_profile(self, centre, nbins):
        """mlswlbm_get_radial_profile: ring means of the interfaces z_0..z_n
        around centre = (cx, cy), array [n + 1][nbins], and the cells per
        ring [nbins]."""
        out = np.empty((self.n + 1, int(nbins)), dtype=np.float64)
        cnt = np.empty(int(nbins), dtype=np.int64)
        _check(lib().mlswlbm_get_radial_profile(
            self._h, float(centre[0]), float(centre[1]), int(nbins), out.ctypes.data_as(_D),
            cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))), "mlswlbm_get_radial_profile")
        return out, cnt

    def step_until(self, max_steps, check_every, ke_threshold):
        """Steps until the kinetic energy drops below ke_threshold; returns
        (steps taken, last kinetic energy)."""
        done, ke = ctypes.c_long(), ctypes.c_double()
        _check(lib().mlswlbm_step_until(self._h, int(max_steps), int(check_every),
                                        float(ke_threshold), ctypes.byref(done), ctypes.byref(ke)),
               "mlswlbm_step_until")
        return done.value, ke.value

    def get_state(self, out=None):
        shape = (self.n, self.Q, self.ny, self.nx)
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        _check(lib().mlswlbm_get_state(self._h, _fptr(_checked_out(out, out.size))),
               "mlswlbm_get_state")
        return out

    def set_state(self, f):
        a = _host_f32(f, self.n * self.Q * self.ncell)
        _check(lib().mlswlbm_set_state(self._h, _fptr(a)), "mlswlbm_set_state")

    def save_state(self):
        """(H, g): the internal representation (bit-exact checkpoint)."""
        H = np.empty(self.n, dtype=np.float32)
        g = np.empty((self.n, self.Q, self.ny, self.nx), dtype=np.float32)
        _check(lib().mlswlbm_save_state(self._h, _fptr(H), _fptr(g)), "mlswlbm_save_state")
        return H, g

    def load_state(self, H, g):
        Ha = _host_f32(H, self.n)
        ga = _host_f32(g, self.n * self.Q * self.ncell)
        _check(lib().mlswlbm_load_state(self._h, _fptr(Ha), _fptr(ga)), "mlswlbm_load_state")

    def get_diagnostics(self):
        mass = (ctypes.c_double * self.n)()
        ke = ctypes.c_double()
        hmin = ctypes.c_double()
        rc = lib().mlswlbm_get_diagnostics(self._h, mass, ctypes.byref(ke), ctypes.byref(hmin))
        _check(rc, "mlswlbm_get_diagnostics")
        return np.array(mass[:]), ke.value, hmin.value

    def status(self):
        return lib().mlswlbm_status(self._h)

    def set_stream(self, stream):
        _check(lib().mlswlbm_set_stream(self._h, _stream_ptr(stream)), "mlswlbm_set_stream")

    def launch_count(self):
        return int(lib().mlswlbm_launch_count(self._h))


def _checked_out(out, size):
    if not (isinstance(out, np.ndarray) and out.dtype == np.float32
            and out.flags["C_CONTIGUOUS"] and out.size == size):
        raise ValueError("output must be a contiguous float32 array of %d elements" % size)
    return out


def mlswlbm_create(p, h_init, stream=None):
    return Solver(p, h_init, stream)


def mlswlbm_step(s, nsteps=1):
    s.step(nsteps)


def mlswlbm_get_heights(s, out=None):
    return s.get_heights(out)


def mlswlbm_set_heights(s, h):
    s.set_heights(h)


def mlswlbm_get_state(s, out=None):
    return s.get_state(out)


def mlswlbm_set_state(s, f):
    s.set_state(f)


def mlswlbm_save_state(s):
    return s.save_state()


def mlswlbm_load_state(s, H, g):
    s.load_state(H, g)


def mlswlbm_get_diagnostics(s):
    return s.get_diagnostics()


def mlswlbm_status(s):
    return s.status()


def mlswlbm_destroy(s):
    s.close()


def mlswlbm_friction_eval(p, h, Jx, Jy=None, Rx=None, Ry=None, stream=None):
    """Device tensors [n, ncell]; returns (Rx, Ry)."""
    import torch
    s = make_params(p)
    n = int(p["n"])
    ncell = h.numel() // n
    if Rx is None:
        Rx = torch.empty_like(h)
    if Jy is not None and Ry is None:
        Ry = torch.empty_like(h)
    rc = lib().mlswlbm_friction_eval(
        ctypes.byref(s), ncell, _dev_ptr(h, n * ncell), _dev_ptr(Jx, n * ncell),
        _dev_ptr(Jy, n * ncell) if Jy is not None else None, _dev_ptr(Rx, n * ncell),
        _dev_ptr(Ry, n * ncell) if Ry is not None else None,
        _stream_ptr(stream if stream is not None else torch.cuda.current_stream()))
    _check(rc, "mlswlbm_friction_eval")
    return Rx, Ry


def mlswlbm_diagnostics_noalloc(p, f, out, H=None, stream=None):
    """Diagnostics of a caller-owned device population array, allocating
    nothing: f is a float32 CUDA tensor of n*Q*nx*ny elements, out a float64
    CUDA tensor of n + 2 elements (mass per layer, kinetic energy, min h);
    H (n floats) when f holds the shifted rest planes of save_state."""
    import torch
    s = make_params(p)
    n = int(p["n"])
    q = 3 if int(p.get("lattice", 2)) == MLSW_D1Q3 else 9
    numel = n * q * int(p.get("nx", 1)) * int(p.get("ny", 1))
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.is_contiguous() and out.numel() == n + 2):
        raise ValueError("out must be a contiguous float64 CUDA tensor of n + 2 elements")
    Ha = None if H is None else _host_f32(H, n)
    rc = lib().mlswlbm_diagnostics_noalloc(
        ctypes.byref(s), _dev_ptr(f, numel), None if Ha is None else _fptr(Ha),
        ctypes.c_void_p(out.data_ptr()),
        _stream_ptr(stream if stream is not None else torch.cuda.current_stream()))
    _check(rc, "mlswlbm_diagnostics_noalloc")
    return out


class Batch:
    """Many independent D2Q9 lattices stepped together (mlswlbm_batch_*).

    params: list of parameter dicts; heights: list of [n][ny][nx] arrays;
    flags: MLSW_BATCH_TILE8 / MLSW_BATCH_AUTOTUNE; stream as for Solver.
    """

    def __init__(self, params, heights, flags=0, stream=None):
        if len(params) != len(heights) or not params:
            raise ValueError("need one heights array per parameter set")
        self.count = len(params)
        arr = (mlsw_params * self.count)()
        self._h = []
        for j, p in enumerate(params):
            arr[j] = make_params(p)
            n, ny, nx = int(p["n"]), int(p.get("ny", 1)), int(p.get("nx", 1))
            self._h.append(_host_f32(heights[j], n * nx * ny))
        self.shapes = [(int(p["n"]), int(p.get("ny", 1)), int(p.get("nx", 1))) for p in params]
        ptrs = (_F * self.count)(*[_fptr(a) for a in self._h])
        h = _H()
        _check(lib().mlswlbm_batch_create(self.count, arr, ptrs, int(flags),
                                          _stream_ptr(stream), ctypes.byref(h)),
               "mlswlbm_batch_create")
        self._b = h
        self._h = None  # copied by the library

    def step(self, nsteps=1):
        _check(lib().mlswlbm_batch_step(self._b, int(nsteps)), "mlswlbm_batch_step")

    def get_heights(self, index, out=None):
        if out is None:
            out = np.empty(self.shapes[index], dtype=np.float32)
        rc = lib().mlswlbm_batch_get_heights(self._b, int(index),
                                             _fptr(_checked_out(out, int(np.prod(self.shapes[index])))))
        _check(rc, "mlswlbm_batch_get_heights")
        return out

    def get_heights_device(self, index, out):
        """mlswlbm_batch_get_heights_device: out is a float32 CUDA tensor of
        the instance's [n][ny][nx] heights (asynchronous)."""
        _check(lib().mlswlbm_batch_get_heights_device(
            self._b, int(index), _dev_ptr(out, int(np.prod(self.shapes[index])))),
            "mlswlbm_batch_get_heights_device")
        return out

    def set_heights_device(self, index, h):
        """mlswlbm_batch_set_heights_device: restarts the instance at rest
        from the float32 CUDA tensor h (asynchronous)."""
        _check(lib().mlswlbm_batch_set_heights_device(
            self._b, int(index), _dev_ptr(h, int(np.prod(self.shapes[index])))),
            "mlswlbm_batch_set_heights_device")

    def _many(self, indices, t):
        idx = np.ascontiguousarray([int(i) for i in indices], dtype=np.int32)
        if idx.size and (idx.min() < 0 or idx.max() >= len(self.shapes)):
            raise ValueError("instance index out of range")
        elems = sum(int(np.prod(self.shapes[i])) for i in idx)
        return idx, _dev_ptr(t, elems)

    def get_heights_device_many(self, indices, out):
        """mlswlbm_batch_get_heights_device_many: out is a float32 CUDA tensor
        holding the listed instances' heights one after another
        (asynchronous)."""
        idx, ptr = self._many(indices, out)
        _check(lib().mlswlbm_batch_get_heights_device_many(
            self._b, int(idx.size), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ptr),
            "mlswlbm_batch_get_heights_device_many")
        return out

    def set_heights_device_many(self, indices, h):
        """mlswlbm_batch_set_heights_device_many: restarts the listed
        instances at rest from the float32 CUDA tensor h, their heights one
        after another (asynchronous)."""
        idx, ptr = self._many(indices, h)
        _check(lib().mlswlbm_batch_set_heights_device_many(
            self._b, int(idx.size), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ptr),
            "mlswlbm_batch_set_heights_device_many")

    def select(self, indices):
        """mlswlbm_batch_select: only these instances advance in later steps;
        the others keep their states."""
        idx = np.ascontiguousarray(sorted(int(i) for i in indices), dtype=np.int32)
        _check(lib().mlswlbm_batch_select(self._b, int(idx.size),
                                          idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
               "mlswlbm_batch_select")

    def modes(self, kx, ky):
        """Complex hhat_i(q) of every layer (rows) of every instance: an array
        [count][MLSW_MAX_LAYERS], zero beyond each instance's n."""
        kx = np.ascontiguousarray(kx, dtype=np.int32)
        ky = np.ascontiguousarray(ky, dtype=np.int32)
        if kx.size != self.count or ky.size != self.count:
            raise ValueError("one mode per instance")
        out = np.zeros(2 * MLSW_MAX_LAYERS * self.count, dtype=np.float64)
        ip = ctypes.POINTER(ctypes.c_int)
        _check(lib().mlswlbm_batch_modes(self._b, kx.ctypes.data_as(ip), ky.ctypes.data_as(ip),
                                         out.ctypes.data_as(_D)), "mlswlbm_batch_modes")
        o = out.reshape(self.count, MLSW_MAX_LAYERS, 2)
        return o[..., 0] + 1j * o[..., 1]

    def status(self):
        return lib().mlswlbm_batch_status(self._b)

    def tile_rows(self, index):
        return lib().mlswlbm_batch_tile_rows(self._b, int(index))

    def launch_count(self):
        return lib().mlswlbm_batch_launch_count(self._b)

    def groups(self):
        return lib().mlswlbm_batch_groups(self._b)

    def close(self):
        if getattr(self, "_b", None):
            lib().mlswlbm_batch_destroy(self._b)
            self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlswlbm_debug_bounds_violations():
    """Accesses out of range counted by a bounds-checked build since the last
    call (the counters are cleared), or None for a release build."""
    n = ctypes.c_ulonglong(0)
    rc = lib().mlswlbm_debug_bounds_violations(ctypes.byref(n))
    if rc == MLSW_ERR_UNSUPPORTED:
        return None
    _check(rc, "mlswlbm_debug_bounds_violations")
    return int(n.value)


def selftest_bounded_wait(arrive, limit=256, stream=None):
    """mlswlbm_selftest_bounded_wait: MLSW_OK or MLSW_ERR_TIMEOUT."""
    return lib().mlswlbm_selftest_bounded_wait(int(bool(arrive)), int(limit), _stream_ptr(stream))


def fit_cap_angle(profile, area, base):
    """mlswlbm_fit_cap_angle: (theta in degrees, E) of the arc fit to a
    radial profile with ring areas `area` above the level `base`."""
    prof = np.ascontiguousarray(profile, dtype=np.float64)
    ar = np.ascontiguousarray(area, dtype=np.float64)
    if ar.size != prof.size:
        raise ValueError("one area per ring")
    th, e = ctypes.c_double(), ctypes.c_double()
    _check(lib().mlswlbm_fit_cap_angle(prof.ctypes.data_as(_D), ar.ctypes.data_as(_D),
                                       int(prof.size), float(base), ctypes.byref(th),
                                       ctypes.byref(e)), "mlswlbm_fit_cap_angle")
    return th.value, e.value


EXPORTS_UNET = {
    "mlswlbm_unet_param_count": (ctypes.c_long, []),
    "mlswlbm_unet_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, _D, ctypes.c_ulonglong, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "mlswlbm_unet_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int]),
    "mlswlbm_unet_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int, ctypes.c_double, _D]),
    "mlswlbm_unet_status": (ctypes.c_int, [ctypes.c_void_p]),
    "mlswlbm_unet_set_params": (ctypes.c_int, [ctypes.c_void_p, _F, ctypes.c_long]),
    "mlswlbm_unet_get_params": (ctypes.c_int, [ctypes.c_void_p, _F, ctypes.c_long]),
    "mlswlbm_unet_debug": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_long]),
    "mlswlbm_unet_destroy": (None, [ctypes.c_void_p]),
    "mlswlbm_max_abs_diff": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p]),
}


EXPORTS.update(EXPORTS_UNET)  # bound by lib() with the others


def max_abs_diff(a, b, out=None, stream=None):
    """mlswlbm_max_abs_diff: per item (first dimension) the largest
    |a - b| of two float32 contiguous CUDA tensors of one shape, a NaN or
    infinite difference as +inf. Returns out (a float32 CUDA tensor of the
    item count), enqueued on `stream` (default: torch's current stream)."""
    import torch
    for t in (a, b):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous()):
            raise ValueError("float32 contiguous CUDA tensors expected")
    if tuple(a.shape) != tuple(b.shape) or a.dim() < 1 or a.numel() == 0:
        raise ValueError("a and b must have one non-empty shape")
    count = int(a.shape[0])
    if out is None:
        out = torch.empty(count, dtype=torch.float32, device=a.device)
    elif not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
              and out.numel() == count):
        raise ValueError("out: float32 contiguous CUDA tensor of the item count")
    st = torch.cuda.current_stream() if stream is None else stream
    _check(lib().mlswlbm_max_abs_diff(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                      count, int(a.numel() // count),
                                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(st)),
           "mlswlbm_max_abs_diff")
    return out


UNET_TENSORS = ("X0", "A0", "S0", "P1", "A1", "S1", "P2", "A2", "S2", "P3", "A3", "S3",
                "U2", "B2", "D2", "U1", "B1", "D1", "U0", "B0", "D0", "YG")
UNET_CHANNELS = (16, 32, 32, 32, 64, 64, 64, 128, 128, 128, 256, 256,
                 256, 128, 128, 128, 64, 64, 64, 32, 32, 16)
UNET_LEVELS = (0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0, 0)


class UNet:
    """mlswlbm_unet_*: the U-Net surrogate of 64 LBM steps on tcgen05.
    Device arrays are torch CUDA tensors of float32 [batch][n][ny][nx]."""

    def __init__(self, n, nx, ny, max_batch, extra=(), seed=0, in_scale=20.0, out_scale=100.0,
                 stream=None):
        self.n, self.nx, self.ny, self.max_batch = int(n), int(nx), int(ny), int(max_batch)
        self.in_scale, self.out_scale = float(in_scale), float(out_scale)
        self.extra = [float(v) for v in extra]
        ex = (ctypes.c_double * max(1, len(self.extra)))(*self.extra)
        self._u = ctypes.c_void_p()
        _check(lib().mlswlbm_unet_create(self.n, self.nx, self.ny, self.max_batch,
                                         len(self.extra), ex, int(seed), self.in_scale,
                                         self.out_scale, _stream_ptr(stream),
                                         ctypes.byref(self._u)), "mlswlbm_unet_create")

    def close(self):
        if self._u:
            lib().mlswlbm_unet_destroy(self._u)
            self._u = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def param_count():
        return int(lib().mlswlbm_unet_param_count())

    def _batch(self, t):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous()):
            raise ValueError("float32 contiguous CUDA tensor expected")
        if tuple(t.shape[1:]) != (self.n, self.ny, self.nx) or not 1 <= t.shape[0] <= self.max_batch:
            raise ValueError("shape [batch][n][ny][nx] expected")
        return int(t.shape[0])

    def predict(self, h, out):
        b = self._batch(h)
        if tuple(out.shape) != tuple(h.shape):
            raise ValueError("out must match h")
        self._batch(out)
        _check(lib().mlswlbm_unet_predict(self._u, ctypes.c_void_p(h.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), b),
               "mlswlbm_unet_predict")
        return out

    def train_step(self, h, target, lr):
        b = self._batch(h)
        if tuple(target.shape) != tuple(h.shape):
            raise ValueError("target must match h")
        loss = ctypes.c_double()
        _check(lib().mlswlbm_unet_train_step(self._u, ctypes.c_void_p(h.data_ptr()),
                                             ctypes.c_void_p(target.data_ptr()), b, float(lr),
                                             ctypes.byref(loss)), "mlswlbm_unet_train_step")
        return loss.value

    def status(self):
        return int(lib().mlswlbm_unet_status(self._u))

    def get_params(self):
        out = np.empty(self.param_count(), dtype=np.float32)
        _check(lib().mlswlbm_unet_get_params(self._u, _fptr(out), out.size),
               "mlswlbm_unet_get_params")
        return out

    def set_params(self, w):
        a = np.ascontiguousarray(w, dtype=np.float32)
        _check(lib().mlswlbm_unet_set_params(self._u, _fptr(a), a.size),
               "mlswlbm_unet_set_params")

    def _tensor_shape(self, name):
        i = UNET_TENSORS.index(name)
        lev = UNET_LEVELS[i]
        return i, (self.max_batch, (self.ny >> lev) + 2, (self.nx >> lev) + 2, UNET_CHANNELS[i])

    def tensor(self, name, grad=False):
        """An activation (or its gradient) of the last pass as float32
        [max_batch][h + 2][w + 2][C], halo ring included."""
        i, shape = self._tensor_shape(name)
        out = np.empty(shape, dtype=np.uint16)
        _check(lib().mlswlbm_unet_debug(self._u, 1 if grad else 0, i, out.ctypes.data, out.nbytes),
               "mlswlbm_unet_debug")
        return (out.astype(np.uint32) << 16).view(np.float32)

    def skip_grad(self, level):
        name = ("S0", "S1", "S2")[level]
        _, shape = self._tensor_shape(name)
        out = np.empty(shape, dtype=np.uint16)
        _check(lib().mlswlbm_unet_debug(self._u, 4, int(level), out.ctypes.data, out.nbytes),
               "mlswlbm_unet_debug")
        return (out.astype(np.uint32) << 16).view(np.float32)

    def param_grads(self):
        out = np.empty(self.param_count(), dtype=np.float32)
        _check(lib().mlswlbm_unet_debug(self._u, 2, 0, out.ctypes.data, out.nbytes),
               "mlswlbm_unet_debug")
        return out

    def output(self):
        out = np.empty((self.max_batch, self.n, self.ny, self.nx), dtype=np.float32)
        _check(lib().mlswlbm_unet_debug(self._u, 3, 0, out.ctypes.data, out.nbytes),
               "mlswlbm_unet_debug")
        return out
