"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/pm.h declares.  No GPU needed."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1608_00802_gb300 import build
    return build.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "pm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pm_create", "pm_deposit", "pm_forces", "pm_step", "pm_energy", "pm_power_spectrum"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(pm_[a-z0-9_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1608_00802_gb300 import pm
    assert sorted(pm.EXPORTS) == _declared()
    lib = pm.load_library(libpath)
    for n in _declared():
        assert hasattr(lib, n)


def test_config_layout_matches_header(libpath):
    """The ctypes struct has the C layout: defaults written by the library
    land in the right fields."""
    from paper_1608_00802_gb300 import pm
    cfg = pm.pm_config()
    pm.load_library(libpath).pm_config_default(cfg)
    assert (cfg.precision, cfg.quantum, cfg.force_mode, cfg.lap, cfg.cosmological) == (0, 1, 0, 0, 1)
    assert (cfg.omega_m, cfg.omega_l, cfg.h, cfg.m22) == (0.3, 0.7, 0.7, 2.5)
    assert (cfg.rho_floor, cfg.rho_fp64) == (1e-6, 1e-2)


def test_library_hbar_over_m_matches_oracle(libpath):
    from oracle import pm_oracle as O
    from paper_1608_00802_gb300 import pm
    lib = pm.load_library(libpath)
    for m22, h in [(2.5, 0.7), (1.0, 0.7), (10.0, 0.68)]:
        cfg = pm.pm_config()
        lib.pm_config_default(cfg)
        cfg.m22, cfg.h = m22, h
        assert lib.pm_hbar_over_m(cfg) == pytest.approx(O.hbar_over_m(m22, h), rel=1e-14)


def test_invalid_configuration_rejected_without_gpu(libpath):
    from paper_1608_00802_gb300 import pm
    lib = pm.load_library(libpath)
    cfg = pm.pm_config()
    lib.pm_config_default(cfg)
    cfg.n_part, cfg.n_mesh, cfg.box = 10, 7, 1.0      # odd mesh
    assert lib.pm_arena_bytes(cfg) == 0
    assert b"n_mesh" in lib.pm_last_error(None)
