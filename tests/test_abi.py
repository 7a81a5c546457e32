"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol include/atari_gpu.h declares, and its host-side logic
(defaults, footprint, argument validation) works without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1907_08467_gb300 import env as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            syms |= set(re.findall(r"ATARI_API\s+[^;(]*?\b(atari_\w+)\s*\(", txt))
    return syms


@pytest.fixture(scope="module")
def lib():
    return E.load_library()


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert set(E.EXPORTS) == syms


def test_default_config_and_footprint(lib):
    c = E._Config()
    lib.atari_default_config(C.byref(c))
    assert (c.frameskip, c.n_cache, c.startup_frames, c.max_noops, c.log_cap) == (4, 30, 64, 30, 4096)
    f1 = lib.atari_env_footprint(1000, 8, C.byref(c))
    f2 = lib.atari_env_footprint(2000, 8, C.byref(c))
    assert f2 > f1 > 0
    per_env = (f2 - f1) / 1000
    # state 256 + log 2*4096*4 + frames 2*33600 + stack ring 28224 + small fields
    assert 120_000 < per_env < 140_000


def _create(lib, roms, sizes, n_envs=2, cfg=None):
    c = cfg or E.make_config()
    buf = [C.create_string_buffer(r, len(r)) for r in roms]
    rp = (C.c_void_p * len(roms))(*[C.cast(b, C.c_void_p) for b in buf])
    sz = (C.c_size_t * len(roms))(*sizes)
    meta = (E._Meta * len(roms))(*[E._Meta(0x80, 0x81) for _ in roms])
    er = (C.c_int32 * n_envs)(*([0] * n_envs))
    luma = (C.c_uint8 * 128)()
    out = C.c_void_p()
    rc = lib.atari_env_create(rp, sz, meta, len(roms), er, None, n_envs, C.byref(c), luma, C.byref(out))
    return rc, out


def test_rejects_bad_rom_size_before_touching_the_device(lib):
    rc, out = _create(lib, [b"\0" * 3000], [3000])
    assert rc == -22 and not out.value
    assert b"size" in lib.atari_last_error()


def test_rejects_bad_config(lib):
    rom = b"\xea" * 4096
    for field, val in (("frameskip", 1), ("n_cache", 0), ("output_mode", 7), ("log_cap", 10), ("form", 9)):
        c = E.make_config()
        setattr(c, field, val)
        rc, _ = _create(lib, [rom], [4096], cfg=c)
        assert rc == -22, field


def test_null_env_calls_fail_cleanly(lib):
    assert lib.atari_env_step(None, None, None, None, None, None) == -22
    assert lib.atari_env_reset(None, None, None) == -22
    lib.atari_env_destroy(None)


def test_no_device_reports_cuda_error_instead_of_crashing(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, out = _create(lib, [b"\xea" * 4096], [4096])
    assert rc in (-5, -12) and not out.value
