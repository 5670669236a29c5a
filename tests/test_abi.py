"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/elder.h declares; the oracle library is separate from it."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*)\s+(elder_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1906_01632_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert {"elder_create", "elder_step", "elder_solve", "elder_moments", "elder_grad"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (elder_\w+)", out))
    assert declared <= exported


def test_python_binding_names_match_abi():
    from paper_1906_01632_gb300 import elder as E
    for name in _declared():
        if name in ("elder_last_error", "elder_sizes"):
            continue
        assert hasattr(E, name), name


def test_oracle_and_cuda_path_share_nothing():
    """No source of the CUDA path mentions the oracle and vice versa."""
    csrc = os.path.join(ROOT, "paper_1906_01632_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "elder_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1906_01632_gb300", txt, re.M), f
            assert not re.search(r'#include\s*[<"].*elder\.h', txt), f


def test_config_default_without_gpu():
    """elder_config_default is pure host code."""
    from paper_1906_01632_gb300 import elder as E
    cfg = E.elder_config_default(32, 32, 8)
    assert (cfg.nx, cfg.ny, cfg.nz) == (32, 32, 8)
    assert cfg.Lx == 600.0 and cfg.Lz == 150.0 and cfg.rho1 == 1200.0
    assert cfg.Dm == 3.565e-6
    assert (cfg.smoother, cfg.ilu_beta, cfg.omega_ilu) == (E.ELDER_SMOOTH_ZLINE, 0.0, 1.0)
    with pytest.raises(AttributeError):
        E.elder_config_default(4, 4, 2, no_such_field=1)


@pytest.mark.parametrize("bad", [
    dict(nx=6),                       # top square edges off the nodes (bc_mode 0)
    dict(nz=129),                     # z-line smoother: lines of at most 129 nodes
    dict(smoother=7), dict(precision=5), dict(omega_line=0.0), dict(omega=-1.0),
    dict(max_samples=0), dict(nu1=0), dict(bc_mode=9), dict(mu=0.0),
    dict(smoother=2, omega_ilu=0.0), dict(smoother=2, ilu_beta=float("nan")),
])
def test_create_rejects_invalid_config_before_touching_a_device(bad):
    """elder_create validates the configuration on the host and returns
    ELDER_EINVAL with a message before any CUDA call (this runs without a
    GPU)."""
    import ctypes
    from paper_1906_01632_gb300 import elder as E
    grid = {k: bad.pop(k) for k in ("nx", "nz") if k in bad}
    cfg = E.elder_config_default(grid.get("nx", 8), 8, grid.get("nz", 4), **bad)
    h = ctypes.c_void_p()
    rc = E.lib().elder_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == E.ELDER_EINVAL and not h.value
    assert E.lib().elder_last_error(None)
