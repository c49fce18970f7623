"""The allocation-free time-step entry point, dvbm_cfl_dt_noalloc.

Some callers cannot allocate device memory: code inside a framework whose
caching allocator owns the device memory budget, or loops where cudaMalloc
would synchronise the device.  This entry point computes the CFL time step with
scratch space in a fixed device array inside the library instead of an
allocation.  The test checks, on two calls in a row, that it returns the same
dt as the existing path (dvbm_init followed by dvbm_dt) for the same fields,
that a repeated call leaves the device's free memory unchanged, and that it
rejects sizes above its published maximum and fields with an invalid cell.  It lives in its own
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


def test_noalloc_leaves_device_memory_unchanged_and_rejects_bad_cells():
    from paper_2510_04197_gb300 import dvbm
    L = dvbm.lib()
    f = _fields(128, 3)
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in f]
    out = ctypes.c_double(0.0)
    assert L.dvbm_cfl_dt_noalloc(*ptrs, 128 * 128, 1.4, 1.0, 0.05, 1.0 / 128, None, ctypes.byref(out)) == dvbm.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert L.dvbm_cfl_dt_noalloc(*ptrs, 128 * 128, 1.4, 1.0, 0.05, 1.0 / 128, None, ctypes.byref(out)) == dvbm.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    bad = [t.clone() for t in f]
    bad[0][5, 7] = -1.0  # rho <= 0 in one cell
    out2 = ctypes.c_double(-1.0)
    st = L.dvbm_cfl_dt_noalloc(*[ctypes.c_void_p(t.data_ptr()) for t in bad], 128 * 128, 1.4, 1.0, 0.05, 1.0 / 128,
                               None, ctypes.byref(out2))
    assert st == dvbm.EINVAL and out2.value == -1.0
