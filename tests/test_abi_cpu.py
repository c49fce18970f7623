"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/dvbm.h declares, and rejects invalid arguments
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2510_04197_gb300 import build, dvbm
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    return dvbm


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dvbm_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    names = declared_functions()
    assert "dvbm_step" in names and "dvbm_create" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding's signature table covers the same set
    assert names == set(L.SIGNATURES), names ^ set(L.SIGNATURES)


def test_default_opts_are_paper_defaults(L):
    o = L.default_opts()
    assert (o.R, o.T_ref, o.beta, o.cfl, o.dt) == (1.0, 1.0, 1.2, 0.01, 0.0)  # Sec. III.A.3
    assert L.lib().dvbm_default_opts(None) == L.EINVAL


@pytest.mark.parametrize("args,frag", [
    (dict(Pr=0.0), "Pr"), (dict(Pr=-1.0), "Pr"), (dict(gamma=1.0), "gamma"), (dict(gamma=2.5), "gamma"),
    (dict(mu=0.0), "mu"), (dict(Nx=3), "grid"), (dict(Ny=2), "grid"), (dict(storage=7), "storage"),
    (dict(lattice=3), "lattice"), (dict(bcs=[0, 1, 0, 0]), "paired"), (dict(beta=0.5), "beta"),
    (dict(bcs=[0, 0, 5, 5]), "kind"), (dict(bcs=[3, 3, 0, 0]), "external"), (dict(bcs=[3, 1, 0, 0]), "external"),
    (dict(bcs=[0, 0, 3, 0]), "paired"),
])
def test_create_rejects_invalid_arguments(L, args, frag):
    a = dict(lattice=0, Nx=16, Ny=16, Pr=0.71, gamma=1.4, mu=1e-3, bcs=None, storage=0, beta=1.2)
    a.update(args)
    o = L.default_opts(beta=a["beta"])
    h = ctypes.c_void_p()
    st = L.lib().dvbm_create(ctypes.byref(h), a["lattice"], a["Nx"], a["Ny"], a["Pr"], a["gamma"], a["mu"],
                             L.make_bcs(a["bcs"]), a["storage"], ctypes.byref(o), None)
    assert st == L.EINVAL
    assert not h.value
    assert frag in L.lib().dvbm_last_error(None).decode()


def test_null_context_calls_fail_cleanly(L):
    lib = L.lib()
    assert lib.dvbm_step(None, 1) == L.EINVAL
    assert lib.dvbm_init(None, None, None, None, None, 1) == L.EINVAL
    assert lib.dvbm_moments(None, None, None, None, None, 1) == L.EINVAL
    assert lib.dvbm_state_bytes(None) == 0
    assert lib.dvbm_dt(None) == 0.0
    assert lib.dvbm_halo_bytes(None) == 0
    assert lib.dvbm_halo_pack(None, None, None) == L.EINVAL
    assert lib.dvbm_halo_unpack(None, None, None) == L.EINVAL
    assert lib.dvbm_set_dt(None, 1e-3) == L.EINVAL
    lib.dvbm_destroy(None)
    st = lib.dvbm_create(None, 0, 16, 16, 0.71, 1.4, 1e-3, None, 0, None, None)
    assert st == L.EINVAL


def test_create_without_a_usable_device_reports_ecuda(L):
    """Valid arguments on a host with no usable CUDA device: dvbm_create
    returns ECUDA (not an allocation failure), leaves *out NULL and says why."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p(1)
    st = L.lib().dvbm_create(ctypes.byref(h), 0, 16, 16, 0.71, 1.4, 1e-3, None, 0, None, None)
    assert st == L.ECUDA, st
    assert not h.value
    assert b"no usable CUDA device" in L.lib().dvbm_last_error(None)
