"""Shared-start inputs for the divergence study (paper Section 4, Fig. 3:
every emulator starts from one initial state and the frame rate is followed
as the emulators' paths drift apart).

Byte surgery on canonical 256-byte states only: each env's machine part
(CPU, RIOT, TIA, RAM: bytes 0x00-0x5F and 0x80-0xFF) is replaced by one
start state of its cartridge, chosen by `entry`; its own env fields (episode,
step, env key, status, cartridge) are kept, the last applied action is
cleared and the score baseline is set to the new state's score byte, exactly
what a reset from that entry leaves.  No emulation arithmetic lives here;
each side applies it to the start states of its own cache.
"""
from __future__ import annotations

import numpy as np


def shared_start_states(states: np.ndarray, cache: np.ndarray, env_rom, score_addr, entry: int = 0) -> np.ndarray:
    """states [n][256], cache [n_roms][n_cache][256] -> new states [n][256]."""
    st = np.array(states, dtype=np.uint8, copy=True)
    env_rom = np.asarray(env_rom, dtype=np.int64)
    src = np.asarray(cache, dtype=np.uint8)[env_rom, entry]
    st[:, 0x00:0x60] = src[:, 0x00:0x60]
    st[:, 0x80:0x100] = src[:, 0x80:0x100]
    st[:, 0x70] = 0
    score = np.asarray(score_addr, dtype=np.int64)[env_rom]
    st[:, 0x71] = src[np.arange(len(st)), 0x80 + (score & 0x7F)]
    return st
