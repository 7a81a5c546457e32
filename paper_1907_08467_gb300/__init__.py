"""Batched Atari 2600 emulation on one GB300 GPU.

A from-scratch, GB300-native implementation of the emulation path of
"Accelerating Reinforcement Learning through GPU Atari Emulation" (CuLE):
a 6507+RIOT interpreter kernel that logs TIA writes, a TIA replay kernel
rendering 160x210 frames, fused luma/max/84x84/frame-stack preprocessing and
on-device reset from cached start states, behind the C ABI in
include/atari_gpu.h.  `env.AtariEnv` is the Python binding; `synth` holds the
seeded input generators.
"""
__all__ = ["env", "synth", "build"]


def __getattr__(name):
    if name == "AtariEnv":
        from .env import AtariEnv
        return AtariEnv
    raise AttributeError(name)
