"""Thin Python binding of the C ABI in include/atari_gpu.h.

Argument marshalling only: every step of the emulation runs in the CUDA
library.  PyTorch provides device memory and streams; tensors are passed to
the library as raw pointers.  If the CUDA library cannot be built or loaded,
constructing an env raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

OUT_PALETTE, OUT_STACK = 0, 1
FORM_PLAIN, FORM_BATCHED = 0, 1
ST_ILLEGAL, ST_FRAME_CAP, ST_LOG_OVERFLOW, ST_BAD_ACTION, ST_STALL = 1, 2, 4, 8, 16
STATE_BYTES = 256

_lock = threading.Lock()
_lib = None


class _Config(C.Structure):
    _fields_ = [("frameskip", C.c_int), ("sticky", C.c_int), ("n_cache", C.c_int),
                ("startup_frames", C.c_int), ("max_noops", C.c_int), ("output_mode", C.c_int),
                ("form", C.c_int), ("log_cap", C.c_int), ("envs_per_block", C.c_int),
                ("envs_per_warp", C.c_int), ("raster_warps_per_frame", C.c_int), ("seed", C.c_uint64),
                ("tia_warps", C.c_int), ("grouping", C.c_int), ("dispatch", C.c_int),
                ("idle_skip", C.c_int)]


class _Meta(C.Structure):
    _fields_ = [("score_addr", C.c_uint8), ("gameover_addr", C.c_uint8)]


EXPORTS = ["atari_default_config", "atari_env_create", "atari_env_reset", "atari_env_step",
           "atari_env_step_host", "atari_env_status", "atari_env_get_state", "atari_env_set_state",
           "atari_env_get_frames", "atari_env_get_cache", "atari_env_counters", "atari_env_info",
           "atari_env_footprint", "atari_env_destroy", "atari_last_error", "atari_env_profile",
           "atari_env_profile_read", "atari_env_launch_shape", "atari_step_noalloc", "atari_env_policy",
           "atari_env_rollout", "atari_env_rollout_ex", "atari_nstep_returns", "atari_vtrace",
           "atari_server_default_config", "atari_server_footprint", "atari_server_create",
           "atari_server_open", "atari_server_step", "atari_server_close", "atari_server_get_stats",
           "atari_server_destroy", "atari_server_loadgen"]
PROF_SLOTS = 8
PROF_NAMES = ["interpreter", "rasteriser", "preprocess", "fused_raster_preprocess", "copy", "policy", "regroup", "s7"]


def load_library(path: str | None = None):
    """Build (if stale) and load libatari_gpu.so; declare every exported symbol."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        L = C.CDLL(path or _build.build())
        P = C.c_void_p
        L.atari_default_config.argtypes = [C.POINTER(_Config)]
        L.atari_default_config.restype = None
        L.atari_env_create.argtypes = [P, P, P, C.c_int, P, P, C.c_int, C.POINTER(_Config), P, C.POINTER(P)]
        L.atari_env_reset.argtypes = [P, P, P]
        L.atari_env_step.argtypes = [P, P, P, P, P, P]
        L.atari_env_step_host.argtypes = [P, P, P, P, P, P]
        L.atari_env_status.argtypes = [P, P, P]
        L.atari_env_get_state.argtypes = [P, P, P]
        L.atari_env_set_state.argtypes = [P, P, P]
        L.atari_env_get_frames.argtypes = [P, P, P]
        L.atari_env_get_cache.argtypes = [P, P, P]
        L.atari_env_counters.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), P]
        L.atari_env_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
        L.atari_env_footprint.argtypes = [C.c_int, C.c_int, C.POINTER(_Config)]
        L.atari_env_footprint.restype = C.c_size_t
        L.atari_env_destroy.argtypes = [P]
        L.atari_env_destroy.restype = None
        L.atari_last_error.restype = C.c_char_p
        L.atari_env_profile.argtypes = [P, C.c_int]
        L.atari_env_profile_read.argtypes = [P, P, P]
        L.atari_env_launch_shape.argtypes = [P, P, P, P, P, P, P]
        L.atari_step_noalloc.argtypes = [P, C.c_size_t, _Meta, P, P, C.c_int, P, P, P, P, C.c_int, C.c_int,
                                         C.c_int, C.c_uint64, P]
        L.atari_step_noalloc.restype = C.c_int
        L.atari_env_policy.argtypes = [P, P, P, P, P, P]
        L.atari_env_rollout.argtypes = [P, P, C.c_int, P, P, P, P, P, P, C.c_int, C.c_int, P]
        L.atari_env_rollout_ex.argtypes = [P, P, C.c_int, P, P, P, P, P, P, P, P, C.c_int, C.c_int, P]
        L.atari_nstep_returns.argtypes = [P, P, C.c_int, C.c_int, P, C.c_int, C.c_int, C.c_float, P, P]
        L.atari_vtrace.argtypes = [P, P, P, C.c_int, C.c_int, P, P, C.c_int, C.c_int, C.c_float, C.c_float,
                                   C.c_float, P, P, P]
        from . import server as _srv
        _srv.declare(L)
        for name in ("atari_env_create", "atari_env_reset", "atari_env_step", "atari_env_step_host",
                     "atari_env_status", "atari_env_get_state", "atari_env_set_state",
                     "atari_env_get_frames", "atari_env_get_cache", "atari_env_counters", "atari_env_info",
                     "atari_env_profile", "atari_env_profile_read", "atari_env_launch_shape",
                     "atari_env_policy", "atari_env_rollout", "atari_env_rollout_ex", "atari_nstep_returns",
                     "atari_vtrace"):
            getattr(L, name).restype = C.c_int
        if path is None:
            _lib = L
        return L


class AtariError(RuntimeError):
    pass


def _check(rc: int):
    if rc != 0:
        raise AtariError(f"atari_gpu error {rc}: {load_library().atari_last_error().decode()}")


def make_config(frameskip=4, sticky=False, n_cache=30, startup_frames=64, max_noops=30,
                output_mode=OUT_STACK, form=FORM_PLAIN, log_cap=4096, envs_per_block=0, envs_per_warp=0,
                raster_warps_per_frame=0, seed=1, tia_warps=0, grouping=0, dispatch=0, idle_skip=1) -> _Config:
    return _Config(frameskip, int(sticky), n_cache, startup_frames, max_noops, output_mode, form,
                   log_cap, envs_per_block, envs_per_warp, raster_warps_per_frame, seed, tia_warps, grouping,
                   dispatch, int(idle_skip))


def footprint(n_envs: int, n_roms: int, **cfg) -> int:
    """Device bytes an env of this configuration holds (admission control)."""
    c = make_config(**cfg)
    return int(load_library().atari_env_footprint(n_envs, n_roms, C.byref(c)))


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class AtariEnv:
    """A batch of emulated consoles resident on one GPU.

    roms: list of cartridge images (bytes); meta: list of (score_addr,
    gameover_addr); env_rom: cartridge index per env (ROM-major order keeps
    warps on one cartridge).
    """

    def __init__(self, roms, meta, env_rom, *, luma=None, env_key=None, device=None, **cfg):
        import torch
        self._torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.lib = load_library()
        self.cfg = make_config(**cfg)
        self.n = len(env_rom)
        self.n_roms = len(roms)
        self.output_mode = self.cfg.output_mode
        self._rom_bufs = [C.create_string_buffer(bytes(r), len(r)) for r in roms]
        rp = (C.c_void_p * len(roms))(*[C.cast(b, C.c_void_p) for b in self._rom_bufs])
        sizes = (C.c_size_t * len(roms))(*[len(r) for r in roms])
        metas = (_Meta * len(roms))(*[_Meta(int(s), int(g)) for s, g in meta])
        er = np.ascontiguousarray(env_rom, dtype=np.int32)
        ek = None if env_key is None else np.ascontiguousarray(env_key, dtype=np.uint32)
        lt = None if luma is None else np.frombuffer(bytes(luma), dtype=np.uint8).copy()
        out = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.atari_env_create(
                rp, sizes, metas, len(roms), er.ctypes.data_as(C.c_void_p),
                ek.ctypes.data_as(C.c_void_p) if ek is not None else None, self.n,
                C.byref(self.cfg), lt.ctypes.data_as(C.c_void_p) if lt is not None else None, C.byref(out)))
        self.h = out

    @classmethod
    def from_workload(cls, w, **kw):
        from .synth import luma_table
        cfg = dict(frameskip=w.frameskip, sticky=w.sticky, output_mode=w.output_mode, seed=w.seed)
        cfg.update(kw)
        return cls([r.data for r in w.roms], [(r.score_addr, r.gameover_addr) for r in w.roms], w.env_rom,
                   luma=luma_table(), **cfg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.atari_env_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def obs_shape(self):
        return (self.n, 210, 160) if self.output_mode == OUT_PALETTE else (self.n, 4, 84, 84)

    def alloc_outputs(self):
        t = self._torch
        return (t.empty(self.obs_shape(), dtype=t.uint8, device=self.device),
                t.empty(self.n, dtype=t.int32, device=self.device),
                t.empty(self.n, dtype=t.uint8, device=self.device))

    def step(self, actions, obs=None, rewards=None, dones=None, stream=None):
        """Device step: actions is a uint8 CUDA tensor [n]; returns (obs, rewards, dones)."""
        t = self._torch
        assert actions.dtype == t.uint8 and actions.is_cuda and actions.numel() == self.n and actions.is_contiguous()
        if obs is None and rewards is None and dones is None:
            obs, rewards, dones = self.alloc_outputs()
        _check(self.lib.atari_env_step(self.h, _ptr(actions), _ptr(obs), _ptr(rewards), _ptr(dones),
                                       _stream(stream)))
        return obs, rewards, dones

    def step_host(self, actions, obs=None, rewards=None, dones=None, stream=None):
        """Host step: numpy (or pinned torch CPU) buffers in and out; synchronous."""
        def hp(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                return a.ctypes.data_as(C.c_void_p)
            return C.c_void_p(a.data_ptr())
        a = actions if not isinstance(actions, np.ndarray) else np.ascontiguousarray(actions, dtype=np.uint8)
        if obs is None and rewards is None and dones is None:
            obs = np.empty(self.obs_shape(), np.uint8)
            rewards = np.empty(self.n, np.int32)
            dones = np.empty(self.n, np.uint8)
        _check(self.lib.atari_env_step_host(self.h, hp(a), hp(obs), hp(rewards), hp(dones), _stream(stream)))
        return obs, rewards, dones

    def reset(self, mask=None, stream=None):
        _check(self.lib.atari_env_reset(self.h, _ptr(mask), _stream(stream)))

    def state(self, stream=None):
        t = self._torch
        out = t.empty((self.n, STATE_BYTES), dtype=t.uint8, device=self.device)
        _check(self.lib.atari_env_get_state(self.h, _ptr(out), _stream(stream)))
        return out

    def set_state(self, st, stream=None):
        assert st.dtype == self._torch.uint8 and st.is_cuda and st.numel() == self.n * STATE_BYTES
        _check(self.lib.atari_env_set_state(self.h, _ptr(st.contiguous()), _stream(stream)))

    def frames(self, stream=None):
        t = self._torch
        out = t.empty((self.n, 2, 210, 160), dtype=t.uint8, device=self.device)
        _check(self.lib.atari_env_get_frames(self.h, _ptr(out), _stream(stream)))
        return out

    def cache(self, stream=None):
        t = self._torch
        out = t.empty((self.n_roms, self.cfg.n_cache, STATE_BYTES), dtype=t.uint8, device=self.device)
        _check(self.lib.atari_env_get_cache(self.h, _ptr(out), _stream(stream)))
        return out

    def status(self, stream=None):
        t = self._torch
        out = t.empty(self.n, dtype=t.int32, device=self.device)
        _check(self.lib.atari_env_status(self.h, _ptr(out), _stream(stream)))
        return out

    def counters(self, stream=None):
        """(6502 instructions executed, TIA writes logged, lockstep issue rounds
        summed over envs) of the last step; timer-wait iterations retired at
        once are not counted as executed."""
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(self.lib.atari_env_counters(self.h, C.byref(a), C.byref(b), C.byref(c), _stream(stream)))
        return a.value, b.value, c.value

    def profile(self, enable: bool = True):
        """Record CUDA events around every kernel launch of step()."""
        _check(self.lib.atari_env_profile(self.h, int(enable)))

    def profile_read(self):
        """{kernel: (total ms, launches)} since the last read (synchronises)."""
        ms = (C.c_double * PROF_SLOTS)()
        ln = (C.c_uint64 * PROF_SLOTS)()
        _check(self.lib.atari_env_profile_read(self.h, ms, ln))
        return {PROF_NAMES[k]: (ms[k], ln[k]) for k in range(PROF_SLOTS) if ln[k]}

    def policy(self, obs, weights, actions=None, logits=None, stream=None):
        """Linear softmax policy on the stack (see atari_env_policy); returns actions."""
        t = self._torch
        if actions is None:
            actions = t.empty(self.n, dtype=t.uint8, device=self.device)
        _check(self.lib.atari_env_policy(self.h, _ptr(obs), _ptr(weights), _ptr(actions), _ptr(logits),
                                         _stream(stream)))
        return actions

    def rollout(self, weights, n_steps, obs, actions, rewards, dones, ring_planes, ring_rewards, ring_start=0,
                stream=None):
        """n_steps of policy -> step -> ring append, all on the device."""
        _check(self.lib.atari_env_rollout(self.h, _ptr(weights), n_steps, _ptr(obs), _ptr(actions), _ptr(rewards),
                                          _ptr(dones), _ptr(ring_planes), _ptr(ring_rewards),
                                          ring_planes.shape[0], ring_start, _stream(stream)))

    def rollout_ex(self, weights, n_steps, obs, actions, rewards, dones, ring_planes, ring_rewards, ring_dones=None,
                   ring_mu=None, ring_start=0, stream=None):
        """As rollout(), also keeping each step's dones and the behaviour
        probability of each sampled action in the ring."""
        _check(self.lib.atari_env_rollout_ex(self.h, _ptr(weights), n_steps, _ptr(obs), _ptr(actions),
                                             _ptr(rewards), _ptr(dones), _ptr(ring_planes), _ptr(ring_rewards),
                                             _ptr(ring_dones), _ptr(ring_mu), ring_planes.shape[0], ring_start,
                                             _stream(stream)))

    def launch_shape(self):
        """(envs per warp, envs per block, warps per frame, interpreter grid,
        tia_warps: 2 with paired TIA warps, else 1, grouping: 1 env order, 2 bank-aware, + 4 with the
        compact opcode switch)."""
        v = [C.c_int() for _ in range(6)]
        _check(self.lib.atari_env_launch_shape(self.h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def info(self):
        n, b = C.c_int(), C.c_size_t()
        _check(self.lib.atari_env_info(self.h, C.byref(n), C.byref(b)))
        return n.value, b.value


def nstep_returns(rewards, dones, values, T, gamma, ring_start=0, out=None, stream=None):
    """Bootstrapped N-step returns [T][n] over a device ring (atari_nstep_returns).
    rewards, dones: [ring_depth][n]; values: [T + 1][n]."""
    import torch
    n = rewards.shape[1]
    if out is None:
        out = torch.empty((T, n), dtype=torch.float32, device=rewards.device)
    _check(load_library().atari_nstep_returns(_ptr(rewards), _ptr(dones), rewards.shape[0], ring_start,
                                              _ptr(values), T, n, C.c_float(gamma), _ptr(out), _stream(stream)))
    return out


def vtrace(rewards, dones, mu, values, pi, T, gamma, rho_bar=1.0, c_bar=1.0, ring_start=0, stream=None):
    """V-trace targets and advantages [T][n] over a device ring (atari_vtrace).
    rewards, dones, mu: [ring_depth][n]; values: [T + 1][n]; pi: [T][n]."""
    import torch
    n = rewards.shape[1]
    vs = torch.empty((T, n), dtype=torch.float32, device=rewards.device)
    adv = torch.empty((T, n), dtype=torch.float32, device=rewards.device)
    _check(load_library().atari_vtrace(_ptr(rewards), _ptr(dones), _ptr(mu), rewards.shape[0], ring_start,
                                       _ptr(values), _ptr(pi), T, n, C.c_float(gamma), C.c_float(rho_bar),
                                       C.c_float(c_bar), _ptr(vs), _ptr(adv), _stream(stream)))
    return vs, adv
