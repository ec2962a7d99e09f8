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


def _cfg(lib, c, **kw):
    cfg = lib.lb_config_default()
    cfg.nx, cfg.ny = c.shape[1], c.shape[0]
    cfg.c_map = c.ctypes.data_as(lib.ctypes.POINTER(lib.ctypes.c_float))
    for k, v in kw.items():
        if k == "s":
            for i, x in enumerate(v):
                cfg.s[i] = x
        elif k == "w_ref":
            for i, x in enumerate(v):
                cfg.w_ref[i] = x
        else:
            setattr(cfg, k, v)
    return cfg


# Each configuration is refused by the validation that runs before any CUDA call, with
# LB_EINVAL and a message naming the offending field.
BAD = [
    (dict(lattice=6), "lattice"),
    (dict(lattice=5, nz=4), "nz"),
    (dict(lattice=7, collision=1, s=[1.0] * 7), "BGK"),
    (dict(lattice=7, time_block=4), "D3Q7"),
    (dict(storage=7), "storage"),
    (dict(storage=3, step_kernel=2), "LB_F64"),
    (dict(boundary=5), "boundary"),
    (dict(nx=0), "grid"),
    (dict(collision=1, s=[1.0, 1.0, 1.0, 2.5, 1.0]), "MRT rate"),
    (dict(lattice=9, w_ref=(0.5, 0.2, 0.2)), "w_ref"),
    (dict(sponge_width=4, sponge_sigma_max=1.5), "sponge"),
    (dict(n_patches=5), "n_patches"),
    (dict(time_block=3), "time_block"),
    (dict(time_block=4, storage=2), "FP32"),
    (dict(lattice=9, time_block=4, storage=1), "FP32"),
    (dict(step_kernel=9), "step_kernel"),
    (dict(streaming=2), "streaming"),
    (dict(streaming=1, storage=2), "LB_STREAM_AA"),
    (dict(streaming=1, time_block=4), "LB_STREAM_AA"),
    (dict(streaming=1, step_kernel=2), "LB_STREAM_AA"),
    (dict(streaming=1, lattice=7), "LB_STREAM_AA"),
]


@pytest.mark.parametrize("kw,word", BAD)
def test_create_refuses_invalid_configs_without_gpu(lib, kw, word):
    import numpy as np
    c = np.ones((8, 8), np.float32)
    cfg = _cfg(lib, c, **kw)
    with pytest.raises(lib.LBError) as e:
        lib.lb_create(cfg)
    assert e.value.status == lib.LB_EINVAL
    assert word in lib.lb_last_error(None)


def test_create_refuses_fp64_with_a_patch_without_gpu(lib):
    import numpy as np
    c = np.ones((32, 32), np.float32)
    p = (lib.lb_patch * 1)(lib.lb_patch(8, 8, 8, 8, 2, 0))
    cfg = _cfg(lib, c, storage=3)
    cfg.patches = lib.ctypes.cast(p, lib.ctypes.POINTER(lib.lb_patch))
    cfg.n_patches = 1
    with pytest.raises(lib.LBError) as e:
        lib.lb_create(cfg)
    assert e.value.status == lib.LB_EINVAL and "LB_F64" in lib.lb_last_error(None)


def test_footprint_of_fp64_storage_without_gpu(lib):
    cfg = lib.lb_config_default()
    cfg.nx, cfg.ny, cfg.storage = 256, 128, 3
    plane = 256 * 128
    # FP64 populations (two buffers), the FP32 eta^2 and medium index, the FP64 eta^2 and
    # coefficient table
    expect = 2 * 5 * plane * 8 + plane * 4 + plane + 1024 + plane * 8 + 256
    assert lib.lb_footprint(cfg, 0, 0, 0) == expect


def test_footprint_of_in_place_streaming_without_gpu(lib):
    # LB_STREAM_AA keeps one population buffer: the footprint drops by exactly one buffer
    for lattice, storage, eb in ((5, 0, 4), (9, 0, 4), (5, 1, 2), (9, 1, 2)):
        cfg = lib.lb_config_default()
        cfg.nx, cfg.ny, cfg.lattice, cfg.storage = 1000, 700, lattice, storage
        two = lib.lb_footprint(cfg, 100, 8, 0)
        cfg.streaming = lib.LB_STREAM_AA
        one = lib.lb_footprint(cfg, 100, 8, 0)
        assert two - one == lattice * 700 * 1024 * eb   # pitch 1024 (multiple of 32)


def test_create_refuses_in_place_streaming_with_a_patch_without_gpu(lib):
    import numpy as np
    c = np.ones((32, 32), np.float32)
    p = (lib.lb_patch * 1)(lib.lb_patch(8, 8, 8, 8, 2, 0))
    cfg = _cfg(lib, c, streaming=1)
    cfg.patches = lib.ctypes.cast(p, lib.ctypes.POINTER(lib.lb_patch))
    cfg.n_patches = 1
    with pytest.raises(lib.LBError) as e:
        lib.lb_create(cfg)
    assert e.value.status == lib.LB_EINVAL and "LB_STREAM_AA" in lib.lb_last_error(None)
