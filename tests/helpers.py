"""Shared helpers for tests: hand-assembled test cartridges."""
from paper_1907_08467_gb300.synth.asm6502 import Assembler

JAM = ".byte $02"   # an undocumented opcode: halts the CPU (end of a test program)


def rom(src: str, size: int = 4096, symbols=None, start: str = "Start") -> bytes:
    """Assemble `src` at $F000 into a 4 KB cartridge whose reset vector is `start`."""
    text = "        .org $F000\n" + src + f"\n        .org $FFFA\n        .word {start}, {start}, {start}\n"
    return Assembler(symbols).assemble(text, org=0xF000, size=4096)


def run_to_jam(m, limit=100000):
    """Step a machine until it halts on the JAM opcode; returns instructions run."""
    for i in range(limit):
        if m.step() < 0:
            return i
    raise AssertionError("program did not halt")
