"""Thin Python binding of the serving loop (include/atari_server.h).

Argument marshalling only: the request loop, admission, tick packing and
every kernel run inside the CUDA library (its launcher and completer threads
are native).  ctypes releases the GIL around each call, so Python client
threads step their sessions concurrently.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

EAGAIN, EBUSY, ESESSION = -11, -16, -3
STACK = (4, 84, 84)


class _ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("max_slots", C.c_int), ("max_tick_envs", C.c_int),
                ("max_session_envs", C.c_int), ("inflight", C.c_int), ("idle_timeout_ms", C.c_int)]


class _RequestInfo(C.Structure):
    _fields_ = [("submit_ns", C.c_int64), ("launch_ns", C.c_int64), ("done_ns", C.c_int64), ("tick_envs", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("ticks", C.c_uint64), ("requests", C.c_uint64), ("env_steps", C.c_uint64),
                ("sessions_admitted", C.c_uint64), ("launches", C.c_uint64), ("budget_bytes", C.c_uint64), ("bytes_in_use", C.c_uint64),
                ("fixed_bytes", C.c_uint64), ("per_env_bytes", C.c_uint64), ("capacity", C.c_int),
                ("free_slots", C.c_int), ("queued_sessions", C.c_int), ("pending_requests", C.c_int),
                ("overlapped_ticks", C.c_uint64)]


class _LoadgenConfig(C.Structure):
    _fields_ = [("n_clients", C.c_int), ("seconds", C.c_double), ("think_mean_ms", C.c_double),
                ("min_envs", C.c_int), ("max_envs", C.c_int), ("session_steps_mean", C.c_double),
                ("seed", C.c_uint64), ("want_obs", C.c_int)]


class _LoadgenResult(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("env_steps", C.c_uint64), ("frames", C.c_uint64),
                ("sessions", C.c_uint64), ("seconds", C.c_double), ("frames_per_s", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double), ("mean_ms", C.c_double),
                ("admit_p50_ms", C.c_double), ("admit_p99_ms", C.c_double), ("ticks", C.c_uint64),
                ("mean_tick_envs", C.c_double), ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64)]


def declare(L):
    """Argument and result types of the serving entry points."""
    from .env import _Config
    P = C.c_void_p
    L.atari_server_default_config.argtypes = [C.POINTER(_ServerConfig)]
    L.atari_server_default_config.restype = None
    L.atari_server_footprint.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(_Config), C.POINTER(_ServerConfig)]
    L.atari_server_footprint.restype = C.c_size_t
    L.atari_server_create.argtypes = [P, P, P, C.c_int, C.POINTER(_Config), P, C.POINTER(_ServerConfig),
                                      C.POINTER(P)]
    L.atari_server_open.argtypes = [P, C.c_int, C.c_int, C.c_uint32, C.c_int, C.POINTER(C.c_int)]
    L.atari_server_step.argtypes = [P, C.c_int, P, P, P, P, C.POINTER(_RequestInfo)]
    L.atari_server_close.argtypes = [P, C.c_int]
    L.atari_server_get_stats.argtypes = [P, C.POINTER(_Stats)]
    L.atari_server_destroy.argtypes = [P]
    L.atari_server_destroy.restype = None
    L.atari_server_loadgen.argtypes = [P, C.POINTER(_LoadgenConfig), C.POINTER(_LoadgenResult)]
    for n in ("atari_server_create", "atari_server_open", "atari_server_step", "atari_server_close",
              "atari_server_get_stats", "atari_server_loadgen"):
        getattr(L, n).restype = C.c_int


class ServerError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__(f"atari_server error {rc}: {msg}")
        self.rc = rc


def _addr(a):
    """Host address of a numpy array or a (pinned) CPU torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return C.c_void_p(a.ctypes.data)
    assert a.device.type == "cpu" and a.is_contiguous()
    return C.c_void_p(a.data_ptr())


def server_config(budget_bytes=40 << 30, max_slots=0, max_tick_envs=0, max_session_envs=2048, inflight=2,
                  idle_timeout_ms=0) -> _ServerConfig:
    return _ServerConfig(budget_bytes, max_slots, max_tick_envs, max_session_envs, inflight, idle_timeout_ms)


class Session:
    """n envs of one cartridge served by an AtariServer; env j keyed key_base + j."""

    def __init__(self, server, sid, rom, n, key_base):
        self.server, self.sid, self.rom, self.n, self.key_base = server, sid, rom, n, key_base
        self.last_info = None

    def step(self, actions, obs=None, rewards=None, dones=None, want_obs=True):
        """One step; outputs go to the given host buffers (numpy or pinned
        torch) or to new numpy arrays.  Returns (obs, rewards, dones)."""
        a = np.ascontiguousarray(actions, dtype=np.uint8) if isinstance(actions, (list, tuple, np.ndarray)) \
            else actions
        if obs is None and want_obs:
            obs = np.empty((self.n,) + STACK, np.uint8)
        if rewards is None:
            rewards = np.empty(self.n, np.int32)
        if dones is None:
            dones = np.empty(self.n, np.uint8)
        info = _RequestInfo()
        S = self.server
        rc = S.lib.atari_server_step(S.h, self.sid, _addr(a), _addr(obs), _addr(rewards), _addr(dones),
                                     C.byref(info))
        S._check(rc)
        self.last_info = info
        return obs, rewards, dones

    def close(self):
        if self.sid is not None:
            self.server._check(self.server.lib.atari_server_close(self.server.h, self.sid))
            self.sid = None


class AtariServer:
    """Serving loop over one GPU: sessions of envs, continuous batching of
    their step requests, admission by a device-memory budget."""

    def __init__(self, roms, meta, *, luma, budget_bytes=40 << 30, max_slots=0, max_tick_envs=0,
                 max_session_envs=2048, inflight=2, idle_timeout_ms=0, **cfg):
        from .env import FORM_BATCHED, OUT_STACK, _Meta, load_library, make_config
        cfg.setdefault("form", FORM_BATCHED)
        cfg.setdefault("output_mode", OUT_STACK)
        self.lib = load_library()
        self.cfg = make_config(**cfg)
        self.scfg = server_config(budget_bytes, max_slots, max_tick_envs, max_session_envs, inflight,
                                  idle_timeout_ms)
        self._roms = [C.create_string_buffer(bytes(r), len(r)) for r in roms]
        rp = (C.c_void_p * len(roms))(*[C.cast(b, C.c_void_p) for b in self._roms])
        sz = (C.c_size_t * len(roms))(*[len(r) for r in roms])
        mt = (_Meta * len(roms))(*[_Meta(s, g) for s, g in meta])
        lu = np.frombuffer(bytes(luma), dtype=np.uint8) if isinstance(luma, (bytes, bytearray)) \
            else np.ascontiguousarray(luma, dtype=np.uint8)
        assert lu.size == 128, "luma table has 128 entries"
        h = C.c_void_p()
        self.h = None
        rc = self.lib.atari_server_create(rp, sz, mt, len(roms), C.byref(self.cfg), C.c_void_p(lu.ctypes.data),
                                          C.byref(self.scfg), C.byref(h))
        self._check(rc)
        self.h = h

    @classmethod
    def from_roms(cls, roms, **kw):
        from .synth import luma_table
        return cls([r.data for r in roms], [(r.score_addr, r.gameover_addr) for r in roms], luma=luma_table(), **kw)

    def _check(self, rc):
        if rc != 0:
            raise ServerError(rc, self.lib.atari_last_error().decode())

    def open(self, rom, n, key_base, timeout_ms=-1) -> Session:
        sid = C.c_int(-1)
        self._check(self.lib.atari_server_open(self.h, rom, n, key_base, timeout_ms, C.byref(sid)))
        return Session(self, sid.value, rom, n, key_base)

    def stats(self) -> dict:
        s = _Stats()
        self._check(self.lib.atari_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def loadgen(self, n_clients=64, seconds=60.0, think_mean_ms=2.0, min_envs=1, max_envs=2048,
                session_steps_mean=100.0, seed=1, want_obs=True) -> dict:
        c = _LoadgenConfig(n_clients, seconds, think_mean_ms, min_envs, max_envs, session_steps_mean, seed,
                           int(want_obs))
        r = _LoadgenResult()
        self._check(self.lib.atari_server_loadgen(self.h, C.byref(c), C.byref(r)))
        return {k: getattr(r, k) for k, _ in _LoadgenResult._fields_}

    def close(self):
        if self.h:
            self.lib.atari_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(slots, tick_envs, n_roms, budget_bytes=40 << 30, inflight=2, **cfg) -> int:
    """Device bytes a server holds for `slots` env slots and `tick_envs` envs per tick."""
    from .env import FORM_BATCHED, OUT_STACK, load_library, make_config
    cfg.setdefault("form", FORM_BATCHED)
    cfg.setdefault("output_mode", OUT_STACK)
    L = load_library()
    c = make_config(**cfg)
    s = server_config(budget_bytes, inflight=inflight)
    return int(L.atari_server_footprint(slots, tick_envs, n_roms, C.byref(c), C.byref(s)))
