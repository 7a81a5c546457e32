"""Seeded random-program cartridges for differential testing.

Input generator only.  Each cartridge keeps a fixed frame skeleton (VSYNC,
VBLANK, 192 visible and 30 overscan lines, each line started by WSYNC) and
fills every line with a random block of legal instructions drawn from the
whole documented instruction set: ALU and decimal arithmetic, every
addressing mode, read-modify-write on RAM and on TIA strobe registers, TIA
and RIOT reads and writes, balanced stack operations, short branches and a
subroutine call.  Optionally the blocks also use the stable undocumented
opcodes (read-modify-write plus accumulator operations on RAM and on TIA
strobes, SAX, LAX, ANC, ALR, SBX, SBC $EB and the NOPs of one to three
bytes), and optionally one line holds an opcode that halts the CPU.  Random stores stay in RAM $80-$EF and the frame counter and
game-over byte live at $F1 / $F2, which only the skeleton writes.
"""
from __future__ import annotations

import random

from .asm6502 import Assembler
from .roms import Rom

# TIA write registers a random block may touch (never VSYNC / WSYNC / RSYNC,
# which drive the frame skeleton).
TIA_W = [0x01, 0x04, 0x05, 0x06, 0x07, 0x08, 0x09, 0x0A, 0x0B, 0x0C, 0x0D, 0x0E, 0x0F, 0x10, 0x11,
         0x12, 0x13, 0x14, 0x15, 0x19, 0x1B, 0x1C, 0x1D, 0x1E, 0x1F, 0x20, 0x21, 0x22, 0x23, 0x24,
         0x25, 0x26, 0x27, 0x28, 0x29, 0x2A, 0x2B, 0x2C, 0x2D, 0x3F]
TIA_STROBES = [0x10, 0x11, 0x12, 0x13, 0x14, 0x2A, 0x2B, 0x2C, 0x1B, 0x1C]
RIOT_R = [0x280, 0x281, 0x282, 0x283, 0x284, 0x285, 0x28C, 0x2A4]
RIOT_W = [0x281, 0x283, 0x294, 0x295, 0x296, 0x297, 0x280]


def _undoc(rng: random.Random, emit, ram: int):
    """One stable undocumented instruction (worst-case cycles counted)."""
    r = rng.random()
    if r < 0.30:
        emit(f"{rng.choice(['SLO', 'RLA', 'SRE', 'RRA', 'DCP', 'ISC'])} ${ram:02X}", 5)
    elif r < 0.40:
        emit(f"{rng.choice(['SLO', 'DCP', 'ISC'])} ${rng.choice(TIA_STROBES):02X}", 5)
    elif r < 0.48:
        emit("TXA", 2); emit("AND #$6F", 2); emit("TAX", 2)
        emit(f"{rng.choice(['SLO', 'RLA', 'SRE', 'RRA', 'DCP', 'ISC'])} $80,X", 6)
    elif r < 0.56:
        emit(f"SAX ${rng.choice([ram, rng.choice(TIA_W)]):02X}", 3)
    elif r < 0.66:
        emit(f"LAX ${rng.choice([ram, rng.randrange(16)]):02X}", 3)
    elif r < 0.72:
        emit(f"LAX (${0xE0 + 2 * rng.randrange(4):02X}),Y", 6)
    elif r < 0.84:
        emit(f"{rng.choice(['ANC', 'ALR', 'SBX'])} #${rng.randrange(256):02X}", 2)
    elif r < 0.88:
        emit(f".byte $EB, ${rng.randrange(256):02X}", 2)
    elif r < 0.92:
        emit(f".byte ${rng.choice([0x1A, 0x3A, 0x5A, 0x7A, 0xDA, 0xFA]):02X}", 2)
    elif r < 0.95:
        emit(f".byte ${rng.choice([0x80, 0x82, 0x89, 0xC2, 0xE2]):02X}, ${rng.randrange(256):02X}", 2)
    elif r < 0.98:
        emit(f".byte ${rng.choice([0x04, 0x44, 0x64, 0x14, 0x34]):02X}, ${ram:02X}", 4)
    else:
        emit(f".byte $0C, ${ram:02X}, $00", 4)


def _block(rng: random.Random, budget: int, tag: str, undoc: bool = False) -> str:
    """Random straight-line code of at most `budget` cycles (worst case)."""
    out, used, k = [], 0, 0

    def emit(text, cyc):
        nonlocal used
        out.append(text)
        used += cyc

    while used < budget - 8:
        k += 1
        if undoc and rng.random() < 0.25:
            _undoc(rng, emit, 0x80 + rng.randrange(0x70))
            continue
        r = rng.random()
        ram = 0x80 + rng.randrange(0x70)          # leave $F0-$FF to the stack
        if r < 0.16:
            op = rng.choice(["ADC", "SBC", "AND", "ORA", "EOR", "CMP", "LDA", "LDX", "LDY", "CPX", "CPY"])
            emit(f"{op} #${rng.randrange(256):02X}", 2)
        elif r < 0.30:
            op = rng.choice(["ADC", "SBC", "AND", "ORA", "EOR", "CMP", "LDA", "STA", "BIT"])
            emit(f"{op} ${ram:02X}", 3)
        elif r < 0.36:
            op = rng.choice(["ADC", "SBC", "LDA", "CMP", "EOR"])
            emit(f"{op}.w ${ram:04X}", 4)
        elif r < 0.44:
            op = rng.choice(["INC", "DEC", "ASL", "LSR", "ROL", "ROR"])
            emit(f"{op} ${ram:02X}", 5)
        elif r < 0.50:
            op = rng.choice(["ASL", "LSR", "ROL", "ROR"])
            emit(f"{op} A", 2)
        elif r < 0.58:
            emit(rng.choice(["CLC", "SEC", "SED", "CLD", "CLV", "TAX", "TAY", "TXA", "TYA", "INX", "INY",
                             "DEX", "DEY", "NOP", "TSX"]), 2)
        elif r < 0.64:
            reg = rng.choice(TIA_W)
            emit(f"{rng.choice(['STA', 'STX', 'STY'])} ${reg:02X}", 3)
        elif r < 0.67:
            emit(f"{rng.choice(['INC', 'DEC', 'ASL'])} ${rng.choice(TIA_STROBES):02X}", 5)
        elif r < 0.72:
            emit(f"{rng.choice(['LDA', 'LDX', 'LDY', 'BIT'])} ${rng.randrange(16):02X}", 3)
        elif r < 0.76:
            emit(f"LDA ${rng.choice(RIOT_R):04X}", 4)
        elif r < 0.78:
            emit(f"STA ${rng.choice(RIOT_W):04X}", 4)
        elif r < 0.82:
            # indexed with the index masked into RAM for stores
            emit("TXA", 2); emit("AND #$6F", 2); emit("TAX", 2)
            emit(f"{rng.choice(['STA', 'LDA', 'ADC', 'INC', 'ROL'])} $80,X", 6)
        elif r < 0.86:
            emit(f"{rng.choice(['LDA', 'LDX', 'CMP', 'EOR'])} $F{rng.randrange(16):X}{rng.randrange(256):02X},Y", 5)
        elif r < 0.89:
            emit(f"LDA (${0xE0 + 2 * rng.randrange(4):02X},X)", 6)
        elif r < 0.92:
            emit(f"{rng.choice(['LDA', 'ADC', 'SBC', 'CMP'])} (${0xE0 + 2 * rng.randrange(4):02X}),Y", 6)
        elif r < 0.95:
            if rng.random() < 0.5:
                emit("PHA", 3); emit(rng.choice(["LDA #$00", "LDA #$FF", "SEC"]), 2); emit("PLA", 4)
            else:
                emit("PHP", 3); emit(rng.choice(["SED", "CLC", "CLV"]), 2); emit("PLP", 4)
        elif r < 0.98:
            lab = f"{tag}_{k}"
            emit(f"{rng.choice(['BNE', 'BEQ', 'BCC', 'BCS', 'BPL', 'BMI', 'BVC', 'BVS'])} {lab}", 4)
            emit("NOP", 2)
            out.append(f"{lab}:")
        else:
            emit("JSR Sub", 12)
    return "\n".join("        " + s if not s.endswith(":") else s for s in out) + "\n"


def fuzz_rom(seed: int, jam: bool = False, lines: int = 24, undoc: bool = False) -> Rom:
    """A cartridge whose frames are made of random blocks (see module doc).
    `lines` visible lines get random blocks (the rest of the 192 are plain);
    `undoc` mixes the stable undocumented opcodes into every block."""
    rng = random.Random(0xF000 + seed)
    src = """
        .org $F000
Reset:  SEI
        CLD
        LDX #$FF
        TXS
        LDX #7
PtrLp:  LDA PtrInit,X
        STA $E0,X
        DEX
        BPL PtrLp
        STA WSYNC
Main:   LDA #2
        STA VSYNC
        STA VBLANK
        STA WSYNC
        STA WSYNC
        STA WSYNC
        LDA #0
        STA VSYNC
        CLD
"""
    for v in range(4):
        src += _block(rng, 60, f"v{v}", undoc) + "        STA WSYNC\n"
    src += """
        LDX #32
VbW:    STA WSYNC
        DEX
        BNE VbW
        STA WSYNC
        LDA #0
        STA VBLANK
"""
    jam_line = rng.randrange(lines) if jam else -1
    jam_at = 100 + rng.randrange(20)      # frame-counter value that halts the CPU
    for ln in range(lines):
        if ln == jam_line:
            src += f"        LDA $F1\n        CMP #{jam_at}\n        BNE NoJam\n        .byte $02\nNoJam:\n"
        src += _block(rng, 62, f"l{ln}", undoc) + "        STA WSYNC\n"
    src += f"""
        LDX #{192 - lines}
VisW:   STA WSYNC
        DEX
        BNE VisW
        LDA #2
        STA VBLANK
"""
    for o in range(3):
        src += _block(rng, 60, f"o{o}", undoc) + "        STA WSYNC\n"
    src += """
        INC $F1
        LDA $F1
        CMP #$%02X
        BCC NotOver
        LDA #1
        STA $F2
        LDA #0
        STA $F1
NotOver:
        LDX #26
OsW:    STA WSYNC
        DEX
        BNE OsW
        STA WSYNC
        JMP Main
Sub:    LDA $90
        EOR #$5A
        RTS
        .align 256
PtrInit: .word $0090, $00A0, Table, $0085
Table:  .byte %s
        .org $FFFA
        .word Reset, Reset, Reset
""" % (rng.randrange(130, 250), ", ".join(f"${rng.randrange(256):02X}" for _ in range(64)))
    data = Assembler().assemble(src, org=0xF000, size=4096)
    return Rom(f"fuzz-{seed}{'-jam' if jam else ''}{'-undoc' if undoc else ''}", data, 0x83, 0xF2,
               {"family": "fuzz"})
