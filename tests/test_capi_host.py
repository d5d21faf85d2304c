"""Host-side checks of the C-ABI library (no GPU needed).

The library must build, load and export every function include/reg.h
declares; argument validation that happens before any CUDA call is checked
here on the CPU.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, 'include')):
        if fn.endswith('.h'):
            text = open(os.path.join(ROOT, 'include', fn)).read()
            text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
            names += re.findall(r'^\s*(?:const\s+)?\w+\s*\*?\s*(reg_\w+)\s*\(', text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope='module')
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_03630_gb300 import reg
    return reg.lib()


def test_header_declares_the_calls_of_the_path():
    names = declared_functions()
    for n in ('reg_create', 'reg_set_images', 'reg_gradient', 'reg_hessian_matvec',
              'reg_precond_apply', 'reg_solve', 'reg_destroy'):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    out = ctypes.c_void_p()
    cases = [(2, 8, 8, 4, 1e-2, 2, 0),        # grid too small
             (8, 8, 8, 0, 1e-2, 2, 0),        # nt < 1
             (8, 8, 8, 65, 1e-2, 2, 0),       # nt > 64
             (8, 8, 8, 4, 0.0, 2, 0),         # beta <= 0
             (8, 8, 8, 4, -1.0, 2, 0),
             (8, 8, 8, 4, 1e-2, 7, 0),        # unknown operator
             (2048, 1024, 1024, 4, 1e-2, 2, 0)]   # more than 2^30 points
    for args in cases:
        s = lib.reg_create(*args, ctypes.byref(out))
        assert s == 1, (args, s)                 # REG_EINVAL
        assert out.value is None
        assert lib.reg_last_error(None)


def test_status_strings_and_default_options(lib):
    from paper_1608_03630_gb300 import reg
    assert lib.reg_status_string(0) == b'REG_OK'
    assert lib.reg_status_string(7) == b'REG_EMAXITER'
    o = reg.Registration.default_opts()
    assert o.gtol == 1e-2 and o.max_gn == 50 and o.max_pcg == 500
    assert o.armijo_c == 1e-4 and o.armijo_shrink == 0.5
    # two-level preconditioner: off unless coarse_factor is set; inner PCG
    # to 0.2 relative, at most 12 iterations; the fine nt on the coarse grid
    assert o.coarse_factor == 0 and o.coarse_tol == 0.2 and o.coarse_max == 12
    assert o.coarse_nt == 0 and o.use_graph == 2


def test_null_context_is_rejected(lib):
    assert lib.reg_destroy(None) == 0
    assert lib.reg_set_stream(None, None) == 1
    assert lib.reg_hessian_matvec(None, None, None) == 1
    assert lib.reg_solve(None, None, None, None) == 1
    assert lib.reg_set_staging(None, 1) == 1
    assert lib.reg_unet_set_mma(None, 1) == 1
    assert lib.reg_set_coarse_tile(None, 2, 8) == 1
    assert lib.reg_get_coarse_tile(None, None, None) == 1


def test_dependent_launch_switch(lib):
    """The process-wide launch switch takes 0 or 1 and touches no GPU."""
    assert lib.reg_set_dependent_launch(2) == 1
    assert lib.reg_set_dependent_launch(-1) == 1
    assert lib.reg_set_dependent_launch(0) == 0
    assert lib.reg_set_dependent_launch(1) == 0


def test_fault_injection_arguments(lib):
    """Arming and disarming the host-side injection touches no GPU."""
    assert lib.reg_debug_inject(5, 0) == 1
    assert lib.reg_debug_inject(-1, 0) == 1
    assert lib.reg_debug_inject(1, -1) == 1
    assert lib.reg_debug_inject(4, 1) == 1      # the wait test fires on the next launch only
    for what in (1, 2, 3):
        assert lib.reg_debug_inject(what, 2) == 0
    assert lib.reg_debug_inject(4, 0) == 0
    assert lib.reg_debug_inject(0, 0) == 0


def test_unet_and_resample_reject_bad_arguments_before_touching_the_gpu(lib):
    out = ctypes.c_void_p()
    ch = (ctypes.c_int * 4)(16, 32, 64, 128)
    cases = [(64, 0, ch, 2, 3),      # no levels
             (64, 7, ch, 2, 3),      # too many levels
             (60, 4, ch, 2, 3),      # R not divisible by 2^(L-1)
             (4, 1, ch, 2, 3),       # R < 8
             (64, 4, None, 2, 3),    # no channel list
             (64, 4, ch, 0, 3),      # cin < 1
             (64, 4, ch, 2, 200),    # cout > 128
             (256, 4, ch, 2, 3)]     # R^3 above the GEMM grid limit
    for R, L, c, ci, co in cases:
        s = lib.reg_unet_create(R, L, ctypes.cast(c, ctypes.c_void_p) if c else None, ci, co,
                                ctypes.byref(out))
        assert s == 1, (R, L, ci, co, s)
        assert out.value is None
    bad = (ctypes.c_int * 4)(16, 0, 64, 128)
    assert lib.reg_unet_create(64, 4, ctypes.cast(bad, ctypes.c_void_p), 2, 3,
                               ctypes.byref(out)) == 1
    n = (ctypes.c_int * 3)(8, 8, 8)
    z = (ctypes.c_int * 3)(8, 0, 8)
    p = ctypes.c_void_p(16)
    assert lib.reg_spectral_resample(None, n, 1, p, p, None) == 1
    assert lib.reg_spectral_resample(n, z, 1, p, p, None) == 1
    assert lib.reg_spectral_resample(n, n, 0, p, p, None) == 1
    assert lib.reg_spectral_resample(n, n, 1, None, p, None) == 1
