"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function that include/jagp.h declares."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for f in sorted(os.listdir(HEADER_DIR)):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(HEADER_DIR, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs the CUDA toolkit to build")
def test_library_exports_every_declared_symbol():
    import paper_2002_07401_gb300 as pg
    path = pg._build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert {"jagp_create", "jagp_eval", "vmc_sweep", "local_energy"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_bad_args_without_gpu():
    """Argument validation happens on the host before any CUDA call."""
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("needs the CUDA toolkit to build")
    import paper_2002_07401_gb300 as pg
    L = pg.lib()
    assert L.jagp_status_string(0) == b"ok"
    assert L.jagp_status_string(1) == b"invalid argument"
    # null handle / bad sizes are rejected on the host
    assert L.jagp_state_bytes(None, 4) == 0
    assert L.jagp_eval(None, None, 1, None, None, None, None) == 1
    assert L.vmc_sweep(None, None, None, 1, 1, 0, 0, None, None, None) == 1
    assert L.local_energy(None, None, None, 1, None, None, None) == 1
    h = ctypes.c_void_p()
    assert L.jagp_create(ctypes.byref(h), None, None) == 1
    # tuning calls reject a null handle or tuning before touching CUDA
    t = pg._Tuning()
    assert L.jagp_set_tuning(None, ctypes.byref(t)) == 1
    assert L.jagp_autotune(None, None, 1, ctypes.byref(t), None) == 1
    # the per-handle error text needs a handle
    assert L.jagp_last_error(None, None, 0) == 1
    # reblocking checks its sizes on the host
    assert L.jagp_reblock_levels(257) == 8 and L.jagp_reblock_levels(1) == 0
    assert L.jagp_reblock(None, 10, 1, None, None, None, None) == 1
    # the SR step checks its arguments on the host
    assert L.jagp_sr_workspace_bytes(0, 5) == 0 and L.jagp_sr_workspace_bytes(10, 5) > 0
    assert L.jagp_sr_step(None, 5, None, 10, 5, 1e-3, 1.0, 10, 1e-10, None, None, None, None, None, None) == 1
    assert L.jagp_logpsi_derivs(None, None, None, 1, None, None, 1, None) == 1
    # lattice-regularised DMC: a handle, sizes and the estimator's p are checked on the host
    assert L.jagp_lrdmc_workspace_bytes(None, 4) == 0
    assert L.jagp_lrdmc_project(None, None, None, 4, 0, 0, 0.2, 0.0, 0.1, 0.0, 10, None, None, None, None, None,
                                None) == 1
    assert L.jagp_lrdmc_branch(None, None, 4, 0, None, None, None, None, None, None) == 1
    assert L.jagp_lrdmc_energy(None, None, 4, 0, None, None) == 1


def test_oracle_and_product_share_no_code():
    """Neither side imports or includes the other."""
    pkg = os.path.join(ROOT, "paper_2002_07401_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|include)\s+[\"<]?([a-z_]+)", txt), f
    txt = open(os.path.join(ROOT, "oracle", "jagp_oracle.c")).read()
    assert "#include \"" not in txt
