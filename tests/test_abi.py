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
    assert c.idle_skip == 1 and E.make_config().idle_skip == 1
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
    for field, val in (("frameskip", 1), ("n_cache", 0), ("output_mode", 7), ("log_cap", 10), ("form", 9),
                       ("idle_skip", 2)):
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


def test_server_footprint_and_host_validation(lib):
    """Serving: footprint = env footprint + per-tick buffers for each tick in
    flight; create refuses a plain-form config and a budget below one env
    slot before touching the device."""
    from paper_1907_08467_gb300 import server as S
    c = E.make_config(form=E.FORM_BATCHED)
    s2 = S.server_config(inflight=2)
    s3 = S.server_config(inflight=3)
    f = lambda slots, tick, sc: lib.atari_server_footprint(slots, tick, 32, C.byref(c), C.byref(sc))
    env_per = lib.atari_env_footprint(2000, 32, C.byref(c)) - lib.atari_env_footprint(1000, 32, C.byref(c))
    assert f(2000, 0, s2) - f(1000, 0, s2) == env_per
    tick_per = (f(1000, 2000, s2) - f(1000, 1000, s2)) / 1000 / 2
    assert 4 * 7056 <= tick_per < 4 * 7056 + 64      # packed stack + actions/rewards/dones/work list
    assert f(1000, 1000, s3) > f(1000, 1000, s2)
    roms = [bytes(4096)]
    buf = [C.create_string_buffer(r, len(r)) for r in roms]
    rp = (C.c_void_p * 1)(*[C.cast(b, C.c_void_p) for b in buf])
    sz = (C.c_size_t * 1)(4096)
    meta = (E._Meta * 1)(E._Meta(0x80, 0x81))
    luma = (C.c_uint8 * 128)()
    out = C.c_void_p()
    small = S.server_config(budget_bytes=100 << 10)   # below the cartridge images plus one slot
    assert lib.atari_server_create(rp, sz, meta, 1, C.byref(c), luma, C.byref(small), C.byref(out)) == -12
    assert b"budget" in lib.atari_last_error()
    plain = E.make_config(form=E.FORM_PLAIN)
    assert lib.atari_server_create(rp, sz, meta, 1, C.byref(plain), luma, C.byref(s2), C.byref(out)) == -22
    bad = S.server_config(inflight=9)
    assert lib.atari_server_create(rp, sz, meta, 1, C.byref(c), luma, C.byref(bad), C.byref(out)) == -22
    assert not out.value


def test_server_binding_marshals_to_the_library():
    """AtariServer passes cartridges, luma table and limits through the C ABI:
    a budget below one env slot comes back as the library's ENOMEM."""
    from paper_1907_08467_gb300 import synth
    from paper_1907_08467_gb300.server import AtariServer, ServerError
    w = synth.workload(3, n_envs=32)
    with pytest.raises(ServerError) as e:
        AtariServer.from_roms(w.roms[:3], budget_bytes=100 << 10, sticky=True)
    assert e.value.rc == -12 and "budget" in str(e.value)
