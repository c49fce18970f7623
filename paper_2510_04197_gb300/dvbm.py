"""Thin ctypes binding of libdvbm (include/dvbm.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only converts
Python/torch arguments into the C ABI's plain pointers and sizes.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if libdvbm.so
is missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libdvbm.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EUNSTABLE", "ETIMEOUT", "ESTATE"]
D2Q25_SPLIT_II, D2Q16_SPLIT_I = 0, 1
FP64, FP32DEV = 0, 1
PERIODIC, ZEROGRAD, WALL, EXTERNAL = 0, 1, 2, 3
XLO, XHI, YLO, YHI = 0, 1, 2, 3


class DVBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class BC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u_wall", ctypes.c_double * 2), ("T_wall", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("R", ctypes.c_double),
                ("T_ref", ctypes.c_double), ("rho0", ctypes.c_double), ("T0", ctypes.c_double),
                ("beta", ctypes.c_double), ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("check_every", ctypes.c_int), ("timeout_s", ctypes.c_double)]


# exported symbol -> (restype, argtypes)
_VP, _DP, _CI, _CD = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "dvbm_default_opts": (_CI, [ctypes.POINTER(Opts)]),
    "dvbm_create": (_CI, [ctypes.POINTER(_VP), _CI, _CI, _CI, _CD, _CD, _CD, ctypes.POINTER(BC), _CI,
                          ctypes.POINTER(Opts), _VP]),
    "dvbm_init": (_CI, [_VP, _VP, _VP, _VP, _VP, _CI]),
    "dvbm_step": (_CI, [_VP, _CI]),
    "dvbm_moments": (_CI, [_VP, _VP, _VP, _VP, _VP, _CI]),
    "dvbm_totals": (_CI, [_VP, _DP]),
    "dvbm_state_bytes": (ctypes.c_size_t, [_VP]),
    "dvbm_get_state": (_CI, [_VP, _VP, ctypes.c_size_t, _CI]),
    "dvbm_set_state": (_CI, [_VP, _VP, ctypes.c_size_t, _CI]),
    "dvbm_dt": (_CD, [_VP]),
    "dvbm_steps_taken": (ctypes.c_longlong, [_VP]),
    "dvbm_last_error": (ctypes.c_char_p, [_VP]),
    "dvbm_destroy": (None, [_VP]),
    "dvbm_record": (_CI, [_VP, _CI]),
    "dvbm_adjoint": (_CI, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _DP]),
    "dvbm_adjoint_begin": (_CI, [_VP, _VP, _VP]),
    "dvbm_adjoint_advance": (_CI, [_VP, ctypes.POINTER(_CI)]),
    "dvbm_adjoint_halo_pack": (_CI, [_VP, _VP, _VP]),
    "dvbm_adjoint_halo_unpack": (_CI, [_VP, _VP, _VP]),
    "dvbm_adjoint_finish": (_CI, [_VP, _VP, _VP, _VP, _VP, _DP]),
    "dvbm_halo_bytes": (ctypes.c_size_t, [_VP]),
    "dvbm_halo_pack": (_CI, [_VP, _VP, _VP]),
    "dvbm_halo_unpack": (_CI, [_VP, _VP, _VP]),
    "dvbm_set_dt": (_CI, [_VP, _CD]),
    "dvbm_cfl_dt_noalloc": (_CI, [_VP, _VP, _VP, _VP, ctypes.c_longlong, _CD, _CD, _CD, _CD, _VP, _DP]),
}

_lib = None


def lib():
    """Load libdvbm.so (built in-tree by paper_2510_04197_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is missing: build it with paper_2510_04197_gb300.build.build()")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != OK:
        msg = lib().dvbm_last_error(ctx).decode(errors="replace")
        raise DVBMError(status, msg)


def default_opts(**kw) -> Opts:
    o = Opts()
    _check(lib().dvbm_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def make_bcs(bcs: Optional[Sequence] = None):
    """bcs: None (all periodic) or 4 entries (xlo, xhi, ylo, yhi) each an int kind
    or a tuple (WALL, (ux_w, uy_w), T_w)."""
    arr = (BC * 4)()
    for s in range(4):
        b = PERIODIC if bcs is None else bcs[s]
        if isinstance(b, (tuple, list)):
            arr[s].kind = int(b[0])
            arr[s].u_wall[0], arr[s].u_wall[1] = float(b[1][0]), float(b[1][1])
            arr[s].T_wall = float(b[2])
        else:
            arr[s].kind = int(b)
            arr[s].T_wall = 1.0
    return arr


def _ptr(t):
    """Device pointer of a contiguous tensor, or None."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("halo buffers must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libdvbm needs a CUDA device; there is no CPU fallback")
    return torch


class Simulation:
    """A DVBM context on the current CUDA device and torch's current stream."""

    def __init__(self, Nx: int, Ny: int, Pr: float, gamma: float, mu: float, bcs=None,
                 storage: int = FP64, stream=None, lattice: int = D2Q25_SPLIT_II, **opts):
        torch = _torch()
        self.Nx, self.Ny, self.storage = int(Nx), int(Ny), int(storage)
        self.lattice = int(lattice)
        self.npop = 32 if self.lattice == D2Q16_SPLIT_I else 50
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._opts = default_opts(**opts)
        self._bcs = make_bcs(bcs)
        h = ctypes.c_void_p()
        st = lib().dvbm_create(ctypes.byref(h), self.lattice, self.Nx, self.Ny, float(Pr), float(gamma),
                               float(mu), self._bcs, self.storage, ctypes.byref(self._opts),
                               ctypes.c_void_p(self.stream.cuda_stream))
        _check(st, None)
        self._h = h

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().dvbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- helpers
    def _field(self, a):
        torch = _torch()
        t = torch.as_tensor(a, dtype=torch.float64, device=self.device).contiguous()
        if tuple(t.shape) != (self.Ny, self.Nx):
            raise ValueError(f"field must have shape ({self.Ny}, {self.Nx})")
        return t

    # -- API
    def init(self, rho, ux, uy, T):
        """Equilibrium initial conditions from (rho, ux, uy, T) fields [Ny, Nx]."""
        f = [self._field(a) for a in (rho, ux, uy, T)]
        _check(lib().dvbm_init(self._h, *[ctypes.c_void_p(t.data_ptr()) for t in f], 1), self._h)
        return self

    def init_host(self, rho, ux, uy, T):
        """Same, from host numpy arrays (the library copies them)."""
        f = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, T)]
        for a in f:
            if a.shape != (self.Ny, self.Nx):
                raise ValueError("bad field shape")
        _check(lib().dvbm_init(self._h, *[a.ctypes.data_as(ctypes.c_void_p) for a in f], 0), self._h)
        return self

    def step(self, n: int = 1):
        _check(lib().dvbm_step(self._h, int(n)), self._h)
        return self

    def moments(self):
        """dict of device float64 tensors rho, ux, uy, T of shape [Ny, Nx]."""
        torch = _torch()
        out = {k: torch.empty((self.Ny, self.Nx), dtype=torch.float64, device=self.device)
               for k in ("rho", "ux", "uy", "T")}
        _check(lib().dvbm_moments(self._h, *[ctypes.c_void_p(out[k].data_ptr()) for k in ("rho", "ux", "uy", "T")],
                                  1), self._h)
        return out

    def moments_host(self):
        out = {k: np.empty((self.Ny, self.Nx)) for k in ("rho", "ux", "uy", "T")}
        _check(lib().dvbm_moments(self._h, *[out[k].ctypes.data_as(ctypes.c_void_p) for k in ("rho", "ux", "uy", "T")],
                                  0), self._h)
        return out

    def totals(self):
        out = (ctypes.c_double * 4)()
        _check(lib().dvbm_totals(self._h, out), self._h)
        return tuple(out)

    @property
    def state_bytes(self) -> int:
        return int(lib().dvbm_state_bytes(self._h))

    def get_state(self):
        """Device uint8 tensor holding the packed state (populations + step counter)."""
        torch = _torch()
        buf = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
        _check(lib().dvbm_get_state(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel(), 1), self._h)
        return buf

    def set_state(self, buf):
        _check(lib().dvbm_set_state(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel(), 1), self._h)
        return self

    def populations(self, buf=None):
        """View of a packed state as [npop, Ny, Nx] (float64 or float32 deviations)."""
        torch = _torch()
        buf = self.get_state() if buf is None else buf
        dt = torch.float64 if self.storage == FP64 else torch.float32
        return buf[:-8].view(dt).view(self.npop, self.Ny, self.Nx)

    def record(self, every: int):
        """Keep checkpoints every `every` steps of the next init + step run."""
        _check(lib().dvbm_record(self._h, int(every)), self._h)
        return self

    def adjoint(self, dL_drho=None, dL_dT=None):
        """Gradients of a loss of the final (rho, T) fields with respect to the
        initial fields and (mu, Pr, gamma), by the hand-written adjoint."""
        torch = _torch()
        args = []
        keep = []
        for a in (dL_drho, dL_dT):
            if a is None:
                args.append(None)
            else:
                t = self._field(a)
                keep.append(t)
                args.append(ctypes.c_void_p(t.data_ptr()))
        out = {k: torch.empty((self.Ny, self.Nx), dtype=torch.float64, device=self.device)
               for k in ("rho0", "ux0", "uy0", "T0")}
        gp = (ctypes.c_double * 3)()
        _check(lib().dvbm_adjoint(self._h, args[0], args[1], *[ctypes.c_void_p(out[k].data_ptr())
                                                             for k in ("rho0", "ux0", "uy0", "T0")], gp), self._h)
        out["mu"], out["Pr"], out["gamma"] = gp[0], gp[1], gp[2]
        return out

    # -- stepwise adjoint (a band of a decomposed grid; the drivers in slab.py)
    def adjoint_begin(self, dL_drho=None, dL_dT=None):
        """lambda^N of the backward pass from dL/drho, dL/dT of the band's
        current state; its halo rows are exchanged next."""
        args, self._adj_keep = [], []
        for a in (dL_drho, dL_dT):
            if a is None:
                args.append(None)
            else:
                t = self._field(a)
                self._adj_keep.append(t)  # read by stream-ordered kernels
                args.append(ctypes.c_void_p(t.data_ptr()))
        _check(lib().dvbm_adjoint_begin(self._h, args[0], args[1]), self._h)
        return self

    def adjoint_advance(self) -> int:
        """One action of the backward pass; returns what the neighbouring
        bands exchange next: 1 (segment state rows), 2 (adjoint state rows),
        3 (branch-code rows of the step just recomputed), or 0 when the pass
        is complete."""
        h = _CI(0)
        _check(lib().dvbm_adjoint_advance(self._h, ctypes.byref(h)), self._h)
        return int(h.value)

    def adjoint_halo_pack(self, lo=None, hi=None):
        _check(lib().dvbm_adjoint_halo_pack(self._h, _ptr(lo), _ptr(hi)), self._h)
        return self

    def adjoint_halo_unpack(self, lo=None, hi=None):
        _check(lib().dvbm_adjoint_halo_unpack(self._h, _ptr(lo), _ptr(hi)), self._h)
        return self

    def adjoint_finish(self):
        """Gradients of the band's initial fields and the band's share of
        dL/d(mu, Pr, gamma)."""
        torch = _torch()
        out = {k: torch.empty((self.Ny, self.Nx), dtype=torch.float64, device=self.device)
               for k in ("rho0", "ux0", "uy0", "T0")}
        gp = (ctypes.c_double * 3)()
        _check(lib().dvbm_adjoint_finish(self._h, *[ctypes.c_void_p(out[k].data_ptr())
                                                    for k in ("rho0", "ux0", "uy0", "T0")], gp), self._h)
        self._adj_keep = []
        out["mu"], out["Pr"], out["gamma"] = gp[0], gp[1], gp[2]
        return out

    def adjoint_stepwise(self, dL_drho=None, dL_dT=None):
        """The stepwise pass on a context that needs no neighbours (a whole
        periodic grid): the same results as a one-band decomposition."""
        self.adjoint_begin(dL_drho, dL_dT)
        while self.adjoint_advance():
            pass
        return self.adjoint_finish()

    # -- slabs of a grid decomposed along y (EXTERNAL y sides)
    @property
    def halo_bytes(self) -> int:
        return int(lib().dvbm_halo_bytes(self._h))

    def halo_buffer(self):
        """An empty device buffer for one side's halo rows, [npop, 2, Nx]."""
        torch = _torch()
        dt = torch.float64 if self.storage == FP64 else torch.float32
        return torch.empty((self.npop, 2, self.Nx), dtype=dt, device=self.device)

    def halo_pack(self, lo=None, hi=None):
        """Copy the band's two lowest rows into lo and two highest into hi."""
        _check(lib().dvbm_halo_pack(self._h, _ptr(lo), _ptr(hi)), self._h)
        return self

    def halo_unpack(self, lo=None, hi=None):
        """Fill the ghost rows below (lo) and above (hi) the band."""
        _check(lib().dvbm_halo_unpack(self._h, _ptr(lo), _ptr(hi)), self._h)
        return self

    def set_dt(self, dt: float):
        _check(lib().dvbm_set_dt(self._h, float(dt)), self._h)
        return self

    @property
    def dt(self) -> float:
        return float(lib().dvbm_dt(self._h))

    @property
    def steps(self) -> int:
        return int(lib().dvbm_steps_taken(self._h))


def abi_velocities(R: float = 1.0, T_ref: float = 1.0, lattice: int = D2Q25_SPLIT_II):
    """Discrete velocities (vx, vy) of the ABI population order c = n p + q.
    D2Q25: node order 0, +a, -a, +b, -b with a = sqrt(5 - sqrt 10), b = sqrt(5 + sqrt 10);
    D2Q16: +a, -a, +b, -b with a = sqrt(3 - sqrt 6), b = sqrt(3 + sqrt 6)."""
    if lattice == D2Q16_SPLIT_I:
        a, b = np.sqrt(3 - np.sqrt(6)), np.sqrt(3 + np.sqrt(6))
        xi = np.array([a, -a, b, -b]) * np.sqrt(R * T_ref)
    else:
        a, b = np.sqrt(5 - np.sqrt(10)), np.sqrt(5 + np.sqrt(10))
        xi = np.array([0.0, a, -a, b, -b]) * np.sqrt(R * T_ref)
    n = len(xi)
    return np.repeat(xi, n), np.tile(xi, n)
