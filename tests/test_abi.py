"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and exports
every entry point that include/fr.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fr_create", "fr_set_mesh", "fr_update_mesh", "fr_residual", "fr_jvp",
                 "fr_precond_build", "fr_precond_apply", "fr_gmres", "fr_bdf2_step",
                 "fr_ptc_solve", "fr_destroy", "fr_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1903_06304_gb300 import fr
    lib = fr.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1903_06304_gb300 import fr
    assert set(declared_functions()) <= set(fr._SIGS)


def test_default_config_is_the_papers():
    from paper_1903_06304_gb300 import fr
    c = fr._Config()
    fr.load().fr_default_config(ctypes.byref(c))
    assert c.gamma == 1.4 and c.prandtl == 0.72
    assert c.dtau0 == 0.01 and c.dtau_min == 0.01 and c.dtau_max == 1e20 and c.r_ser == 2.0
    assert c.restart == 30 and c.tol_res == 1e-6 and c.dtau_unsteady == 1e20 and c.lag == 2


def test_bad_config_rejected_without_gpu():
    from paper_1903_06304_gb300 import fr
    lib = fr.load()
    c = fr._Config()
    lib.fr_default_config(ctypes.byref(c))
    c.p = 7
    h = ctypes.c_void_p()
    assert lib.fr_create(ctypes.byref(c), ctypes.byref(h)) == -1
    # every enumerated option is validated before any device call
    for field, bad in (("orthog", 2), ("krylov_arith", 2), ("apply_accum", 5), ("block_mode", -1)):
        lib.fr_default_config(ctypes.byref(c))
        setattr(c, field, bad)
        assert lib.fr_create(ctypes.byref(c), ctypes.byref(h)) == -1, field
    lib.fr_default_config(ctypes.byref(c))
    assert c.krylov_arith == 0 and c.orthog == 0


def test_oracle_and_library_share_no_code():
    """The oracle imports nothing of the CUDA path and vice versa."""
    import glob
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        src = open(f).read()
        assert "paper_1903_06304_gb300.fr" not in src and "libfr" not in src
        assert "import fr\n" not in src
    for f in glob.glob(os.path.join(ROOT, "paper_1903_06304_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            assert "import oracle" not in src and "from oracle" not in src


def test_bad_batch_rejected_without_gpu():
    """fr_batch_create validates the cases and the restart length before any GPU work."""
    from paper_1903_06304_gb300 import fr
    lib = fr.load()
    c = fr._Config()
    lib.fr_default_config(ctypes.byref(c))
    h = ctypes.c_void_p()
    good = fr._Case(2, 4, 4, 0.1, 0.0, 1.0)
    bad = [fr._Case(0, 4, 4, 0.1, 0.0, 1.0), fr._Case(2, 1, 4, 0.1, 0.0, 1.0),
           fr._Case(2, 4, 4, 0.0, 0.0, 1.0), fr._Case(5, 4, 4, 0.1, 10.0, 1.0)]
    for b in bad:
        arr = (fr._Case * 2)(good, b)
        assert lib.fr_batch_create(ctypes.byref(c), ctypes.cast(arr, ctypes.c_void_p), 2,
                                   ctypes.byref(h)) == -1
        assert not h.value
    c.restart = 200   # the batched Arnoldi keeps at most 128 vectors on the device
    arr = (fr._Case * 1)(good)
    assert lib.fr_batch_create(ctypes.byref(c), ctypes.cast(arr, ctypes.c_void_p), 1,
                               ctypes.byref(h)) == -1
