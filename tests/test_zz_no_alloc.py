"""The allocation-free time-step entry point, dvbm_cfl_dt_noalloc.

Some callers cannot allocate device memory (during CUDA graph capture, inside
a framework that owns the device memory budget, or where cudaMalloc would
synchronise the device).  This entry point computes the CFL time step with
scratch space in a fixed device array inside the library instead of an
allocation.  The test checks, on two calls in a row, that it returns the same
dt as the existing path (dvbm_init followed by dvbm_dt) for the same fields,
and that it rejects sizes above its published maximum.  It lives in its own
file, collected last, so a failure here cannot hide another test's result.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _fields(N, seed):
    from paper_2510_04197_gb300 import inputs
    F = inputs.multimode(N, seed=seed, rms_Ma=0.5)
    return [torch.tensor(a, device="cuda") for a in (F.rho, F.ux, F.uy, F.T)]


def test_noalloc_dt_matches_dvbm_init_twice():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    L = dvbm.lib()
    stream = torch.cuda.current_stream()
    for call, (N, seed) in enumerate([(256, 0), (192, 1)]):
        f = _fields(N, seed)
        sim = dvbm.Simulation(N, N, 0.71, 1.4, 1e-3, cfl=0.05)
        sim.init(*f)
        ref = sim.dt
        sim.close()
        out = ctypes.c_double(-1.0)
        st = L.dvbm_cfl_dt_noalloc(*[ctypes.c_void_p(t.data_ptr()) for t in f], N * N, 1.4, 1.0, 0.05, 1.0 / N,
                                   ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
        assert st == dvbm.OK, (call, st)
        assert math.isclose(out.value, ref, rel_tol=1e-15, abs_tol=0.0), (call, out.value, ref)


def test_noalloc_rejects_sizes_beyond_maximum():
    from paper_2510_04197_gb300 import dvbm
    L = dvbm.lib()
    f = _fields(64, 2)
    out = ctypes.c_double(0.0)
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in f]
    big = 67108864 + 1  # DVBM_NOALLOC_MAX_CELLS + 1
    assert L.dvbm_cfl_dt_noalloc(*ptrs, big, 1.4, 1.0, 0.05, 1.0, None, ctypes.byref(out)) == dvbm.EINVAL
    assert L.dvbm_cfl_dt_noalloc(*ptrs, 0, 1.4, 1.0, 0.05, 1.0, None, ctypes.byref(out)) == dvbm.EINVAL
