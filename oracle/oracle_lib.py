"""ctypes binding of the C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
STATE_BYTES = 256

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
             os.path.getmtime(os.path.join(HERE, "oracle.h"))))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC,
                               "-lpthread", "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Config(C.Structure):
    _fields_ = [("frameskip", C.c_int), ("sticky", C.c_int), ("n_cache", C.c_int),
                ("startup_frames", C.c_int), ("max_noops", C.c_int), ("output_mode", C.c_int),
                ("seed", C.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, U8P = C.c_void_p, C.POINTER(C.c_uint8)
            L.orc_machine_new.restype = P
            L.orc_machine_new.argtypes = [C.c_char_p, C.c_size_t]
            L.orc_machine_free.argtypes = [P]
            L.orc_machine_step.argtypes = [P]
            L.orc_machine_run_frame.argtypes = [P, P]
            L.orc_machine_set_action.argtypes = [P, C.c_int]
            L.orc_machine_get_state.argtypes = [P, P]
            L.orc_machine_set_state.argtypes = [P, P]
            L.orc_machine_cycles.restype = C.c_uint64
            L.orc_machine_cycles.argtypes = [P]
            L.orc_machine_peek.restype = C.c_uint8
            L.orc_machine_peek.argtypes = [P, C.c_uint16]
            L.orc_machine_last_vsync.argtypes = [P, C.POINTER(C.c_uint64)]
            L.orc_machine_tia_writes.restype = C.c_uint32
            L.orc_machine_tia_writes.argtypes = [P]
            L.orc_alu_adc.restype = C.c_uint32
            L.orc_alu_adc.argtypes = [C.c_uint8, C.c_uint8, C.c_uint8]
            L.orc_alu_sbc.restype = C.c_uint32
            L.orc_alu_sbc.argtypes = [C.c_uint8, C.c_uint8, C.c_uint8]
            L.orc_base_cycles.argtypes = [C.c_uint8]
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_envs_create.restype = P
            L.orc_envs_create.argtypes = [P, P, P, P, C.c_int, P, P, C.c_int, C.POINTER(_Config), P]
            L.orc_envs_free.argtypes = [P]
            L.orc_envs_step.argtypes = [P, P, P, P, P, C.c_int]
            L.orc_envs_get_state.argtypes = [P, P]
            L.orc_envs_set_state.argtypes = [P, P]
            L.orc_envs_get_frames.argtypes = [P, P]
            L.orc_envs_get_cache.argtypes = [P, P]
            L.orc_envs_reset.argtypes = [P, P]
            L.orc_envs_instructions.restype = C.c_uint64
            L.orc_envs_instructions.argtypes = [P]
            L.orc_preprocess.argtypes = [P, P, P, P]
            L.orc_exp_own.argtypes = [C.c_float]
            L.orc_exp_own.restype = C.c_float
            L.orc_policy_logits.argtypes = [P, P, P]
            L.orc_policy_sample.argtypes = [P, C.c_uint32]
            L.orc_envs_policy.argtypes = [P, P, P, P, P, C.c_int]
            L.orc_policy_prob.argtypes = [P, C.c_int]
            L.orc_policy_prob.restype = C.c_float
            L.orc_envs_policy_mu.argtypes = [C.c_int, P, P, P]
            L.orc_nstep_returns.argtypes = [C.c_int, C.c_int, P, P, P, C.c_double, P]
            L.orc_vtrace.argtypes = [C.c_int, C.c_int, P, P, P, P, P, C.c_double, C.c_double, C.c_double, P, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def alu_adc(a, b, p):
    return lib().orc_alu_adc(a, b, p)


def alu_sbc(a, b, p):
    return lib().orc_alu_sbc(a, b, p)


def base_cycles(op):
    return lib().orc_base_cycles(op)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(v) for v in o]


def exp_own(x: float) -> float:
    return lib().orc_exp_own(x)


def policy_logits(stack: np.ndarray, w_bf16: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(stack, dtype=np.uint8).reshape(-1)
    w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
    out = np.zeros(18, dtype=np.float32)
    lib().orc_policy_logits(_ptr(x), _ptr(w), _ptr(out))
    return out


def policy_sample(logits: np.ndarray, u: int) -> int:
    l = np.ascontiguousarray(logits, dtype=np.float32)
    return lib().orc_policy_sample(_ptr(l), u)


def policy_prob(logits: np.ndarray, a: int) -> float:
    l = np.ascontiguousarray(logits, dtype=np.float32)
    return lib().orc_policy_prob(_ptr(l), int(a))


def policy_mu(logits: np.ndarray, actions: np.ndarray) -> np.ndarray:
    """Behaviour probability of each env's sampled action, fp32 [n]."""
    l = np.ascontiguousarray(logits, dtype=np.float32).reshape(-1, 18)
    a = np.ascontiguousarray(actions, dtype=np.uint8)
    mu = np.zeros(l.shape[0], dtype=np.float32)
    lib().orc_envs_policy_mu(l.shape[0], _ptr(l), _ptr(a), _ptr(mu))
    return mu


def _rollout_args(rewards, dones, values):
    r = np.ascontiguousarray(rewards, dtype=np.float32)
    d = np.ascontiguousarray(dones, dtype=np.uint8)
    v = np.ascontiguousarray(values, dtype=np.float32)
    T, n = r.shape
    assert d.shape == (T, n) and v.shape == (T + 1, n)
    return r, d, v, T, n


def nstep_returns(rewards, dones, values, gamma: float) -> np.ndarray:
    """Bootstrapped N-step returns [T][n] (float64) of a time-major rollout."""
    r, d, v, T, n = _rollout_args(rewards, dones, values)
    out = np.zeros((T, n), dtype=np.float64)
    lib().orc_nstep_returns(T, n, _ptr(r), _ptr(d), _ptr(v), gamma, _ptr(out))
    return out


def vtrace(rewards, dones, values, pi, mu, gamma: float, rho_bar: float, c_bar: float):
    """V-trace targets and policy-gradient advantages [T][n] (float64)."""
    r, d, v, T, n = _rollout_args(rewards, dones, values)
    p = np.ascontiguousarray(pi, dtype=np.float32)
    m = np.ascontiguousarray(mu, dtype=np.float32)
    assert p.shape == (T, n) and m.shape == (T, n)
    vs = np.zeros((T, n), dtype=np.float64)
    adv = np.zeros((T, n), dtype=np.float64)
    lib().orc_vtrace(T, n, _ptr(r), _ptr(d), _ptr(v), _ptr(p), _ptr(m), gamma, rho_bar, c_bar, _ptr(vs), _ptr(adv))
    return vs, adv


def preprocess(f3: np.ndarray, f4: np.ndarray, luma: bytes) -> np.ndarray:
    f3 = np.ascontiguousarray(f3, dtype=np.uint8)
    f4 = np.ascontiguousarray(f4, dtype=np.uint8)
    lt = np.frombuffer(bytes(luma), dtype=np.uint8).copy()
    out = np.zeros((84, 84), dtype=np.uint8)
    lib().orc_preprocess(_ptr(f3), _ptr(f4), _ptr(lt), _ptr(out))
    return out


class OracleMachine:
    """One console for hand-assembled programs and definition tests."""

    def __init__(self, rom: bytes):
        self._rom = C.create_string_buffer(bytes(rom), len(rom))
        self.h = lib().orc_machine_new(self._rom, len(rom))
        if not self.h:
            raise ValueError("bad ROM size")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_machine_free(self.h)
            self.h = None

    def step(self) -> int:
        return lib().orc_machine_step(self.h)

    def run_frame(self, render: bool = False):
        fb = np.zeros((210, 160), dtype=np.uint8) if render else None
        lines = lib().orc_machine_run_frame(self.h, _ptr(fb) if render else None)
        return (lines, fb) if render else lines

    def set_action(self, a: int):
        lib().orc_machine_set_action(self.h, a)

    def state(self) -> np.ndarray:
        o = np.zeros(STATE_BYTES, dtype=np.uint8)
        lib().orc_machine_get_state(self.h, _ptr(o))
        return o

    def set_state(self, s: np.ndarray):
        s = np.ascontiguousarray(s, dtype=np.uint8)
        lib().orc_machine_set_state(self.h, _ptr(s))

    @property
    def cycles(self) -> int:
        return lib().orc_machine_cycles(self.h)

    def peek(self, addr: int) -> int:
        return lib().orc_machine_peek(self.h, addr)

    def ram(self) -> np.ndarray:
        return self.state()[0x80:0x100].copy()

    def last_vsync(self):
        c = C.c_uint64(0)
        ok = lib().orc_machine_last_vsync(self.h, C.byref(c))
        return c.value if ok else None

    @property
    def tia_writes(self) -> int:
        return lib().orc_machine_tia_writes(self.h)


class OracleEnvs:
    """A batch of independent environments stepped by the oracle."""

    def __init__(self, roms, score_addr, gameover_addr, env_rom, *, frameskip=4, sticky=False,
                 n_cache=30, startup_frames=64, max_noops=30, output_mode=1, seed=1, luma=None,
                 env_key=None):
        self.n_envs = len(env_rom)
        self.output_mode = output_mode
        self.frameskip = frameskip
        self._roms = [C.create_string_buffer(bytes(r), len(r)) for r in roms]
        rp = (C.c_void_p * len(roms))(*[C.cast(b, C.c_void_p) for b in self._roms])
        sizes = (C.c_size_t * len(roms))(*[len(r) for r in roms])
        sa = np.asarray(score_addr, dtype=np.uint8)
        ga = np.asarray(gameover_addr, dtype=np.uint8)
        er = np.asarray(env_rom, dtype=np.int32)
        ek = None if env_key is None else np.asarray(env_key, dtype=np.uint32)
        cfg = _Config(frameskip, int(sticky), n_cache, startup_frames, max_noops, output_mode, seed)
        lt = np.frombuffer(bytes(luma), dtype=np.uint8).copy() if luma is not None else None
        self.n_roms, self.n_cache = len(roms), n_cache
        self.h = lib().orc_envs_create(rp, sizes, _ptr(sa), _ptr(ga), len(roms), _ptr(er),
                                       _ptr(ek) if ek is not None else None, self.n_envs,
                                       C.byref(cfg), _ptr(lt) if lt is not None else None)
        if not self.h:
            raise ValueError("oracle rejected the configuration")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_envs_free(self.h)
            self.h = None

    def step(self, actions, n_threads: int = 1):
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        n = self.n_envs
        obs = np.zeros((n, 210, 160) if self.output_mode == 0 else (n, 4, 84, 84), dtype=np.uint8)
        rew = np.zeros(n, dtype=np.int32)
        done = np.zeros(n, dtype=np.uint8)
        lib().orc_envs_step(self.h, _ptr(a), _ptr(obs), _ptr(rew), _ptr(done), n_threads)
        return obs, rew, done

    def state(self) -> np.ndarray:
        o = np.zeros((self.n_envs, STATE_BYTES), dtype=np.uint8)
        lib().orc_envs_get_state(self.h, _ptr(o))
        return o

    def set_state(self, st: np.ndarray):
        st = np.ascontiguousarray(st, dtype=np.uint8)
        assert st.shape == (self.n_envs, STATE_BYTES)
        lib().orc_envs_set_state(self.h, _ptr(st))

    def frames(self) -> np.ndarray:
        o = np.zeros((self.n_envs, 2, 210, 160), dtype=np.uint8)
        lib().orc_envs_get_frames(self.h, _ptr(o))
        return o

    def cache(self) -> np.ndarray:
        o = np.zeros((self.n_roms, self.n_cache, STATE_BYTES), dtype=np.uint8)
        lib().orc_envs_get_cache(self.h, _ptr(o))
        return o

    def reset(self, mask=None):
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        lib().orc_envs_reset(self.h, _ptr(m) if m is not None else None)

    def policy(self, obs, w_bf16, n_threads: int = 1):
        """Actions (and logits) of the linear softmax policy for every env."""
        o = np.ascontiguousarray(obs, dtype=np.uint8)
        w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
        act = np.zeros(self.n_envs, dtype=np.uint8)
        logits = np.zeros((self.n_envs, 18), dtype=np.float32)
        lib().orc_envs_policy(self.h, _ptr(o), _ptr(w), _ptr(act), _ptr(logits), n_threads)
        return act, logits

    def instructions(self) -> int:
        return lib().orc_envs_instructions(self.h)
