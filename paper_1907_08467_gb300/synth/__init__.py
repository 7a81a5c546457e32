"""Seeded synthetic inputs: a tiny 6502 assembler, cartridge generators,
the luma table of the stated color model, and action streams.  Input
generation only; no emulation arithmetic lives here."""
from .asm6502 import assemble, Assembler, OPCODES, SYMBOLS  # noqa: F401
from .roms import (Rom, Workload, workload, actions, luma_table, rom_playfield,  # noqa: F401
                   rom_sprite, rom_banked)
from .fuzz import fuzz_rom  # noqa: F401,E402
from .policy import policy_weights  # noqa: F401,E402
from .shared_start import shared_start_states  # noqa: F401,E402
