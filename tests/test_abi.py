"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/cmc.h declares (no GPU needed: no device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cmc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1206_5878_gb300 import _build
    return _build.build()


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for must in ("cmc_init", "cmc_step", "cmc_energy", "cmc_lagrange_radii", "cmc_get_state",
                 "cmc_set_state", "cmc_destroy", "cmc_last_error", "cmc_set_stream",
                 "cmc_rng_philox", "cmc_sort_radius", "cmc_potential", "cmc_timestep",
                 "cmc_relax", "cmc_orbit", "cmc_energy_correction"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(libpath):
    from paper_1206_5878_gb300 import _native
    assert set(_native.SIGNATURES) == set(declared_functions())
    lib = _native.load()
    assert lib.cmc_kernels_per_step(None) == 0
    assert lib.cmc_last_error(None) == b""


def test_config_defaults(libpath):
    import math

    import paper_1206_5878_gb300 as g
    c = g.config()
    assert (c.precision, c.bin_size, c.max_trials, c.energy_correction) == (0, 20, 1000, 1)
    assert c.theta_max == math.pi / 2 and c.gamma == 0.1


def test_init_rejects_bad_arguments_without_a_gpu(libpath):
    """Argument checks run before any CUDA call."""
    from paper_1206_5878_gb300 import _native
    lib = _native.load()
    ctx = ctypes.c_void_p()
    st = lib.cmc_init(ctypes.byref(ctx), None, 0, None, None, None, None, None, None, None, 0,
                      None)
    assert st == _native.CMC_EINVAL and not ctx.value
    assert b"bad arguments" in lib.cmc_last_error(None)


def test_release_build_has_no_debug_checks(libpath):
    """The release library reports no failed device index checks (its
    checks are compiled out); the debug build is a separate library."""
    from paper_1206_5878_gb300 import _build, _native
    lib = _native.load()
    assert lib.cmc_is_debug_build() == 0
    site = ctypes.c_uint32(7)
    assert lib.cmc_debug_check(ctypes.byref(site)) == 0 and site.value == 0
    assert lib.cmc_debug_check(None) == _native.CMC_EINVAL
    assert _build.LIB_DEBUG != _build.LIB


def test_stellar_evolution_timestep_is_the_oracles(libpath):
    """cmc_tse is host arithmetic: Eq. 11 as the oracle writes it, to the
    bit, +inf without mass loss."""
    import math

    import oracle
    lib = ctypes.CDLL(libpath)
    lib.cmc_tse.restype = ctypes.c_double
    lib.cmc_tse.argtypes = [ctypes.c_double] * 3
    for M, T, dm in ((0.83, 0.02, 3e-5), (1.0, 17.3, 0.25), (5e4, 1e-3, 7.0)):
        assert lib.cmc_tse(M, T, dm) == oracle.tse(M, T, dm)
    assert lib.cmc_tse(1.0, 1.0, 0.0) == math.inf
    assert lib.cmc_tse(1.0, 1.0, -1.0) == math.inf
