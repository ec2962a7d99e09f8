"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU needed)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\*?\s*(lb_\w+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300 import lbac
    return lbac


def test_header_declares_entry_points():
    names = _declared()
    for n in ("lb_create", "lb_step", "lb_set_source", "lb_record_receivers", "lb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    raw = lib.raw()
    missing = [n for n in sorted(_declared()) if not hasattr(raw, n)]
    assert not missing, missing


def test_config_default_and_footprint_without_gpu(lib):
    cfg = lib.lb_config_default()
    assert cfg.lattice == 5 and cfg.tau == 0.5 and cfg.storage == lib.LB_F32
    cfg.nx, cfg.ny = 4096, 4096
    b = lib.lb_footprint(cfg, 0, 0, 0)
    # two population buffers + eta^2 + the 1-byte medium index and its 256-entry table
    assert b == 2 * 5 * 4096 * 4096 * 4 + 4096 * 4096 * 4 + 4096 * 4096 + 1024


def test_create_rejects_bad_config_without_touching_gpu(lib):
    import numpy as np
    c = np.ones((8, 8), np.float32)
    cfg = lib.lb_config_default()
    cfg.nx, cfg.ny = 8, 8
    cfg.c_map = c.ctypes.data_as(lib.ctypes.POINTER(lib.ctypes.c_float))
    cfg.tau = 0.3          # below 1/2: rejected by validation before any CUDA call
    with pytest.raises(lib.LBError) as e:
        lib.lb_create(cfg)
    assert e.value.status == lib.LB_EINVAL
    assert "tau" in lib.lb_last_error(None)
