"""Seeded synthetic cartridges and workloads.

Input generator only.  The paper measures on the 57-game ALE suite; those ROMs
are not available, so every workload here is a family of seeded synthetic
programs with the structure of an Atari 2600 game loop: a 262-line NTSC frame
(3 VSYNC + 37 VBLANK + 192 visible + 30 overscan lines), joystick and fire
reads, a RAM score byte (the reward), a RAM game-over byte, and, depending on
the family, player / missile / ball sprites, collision reads, RIOT-timer
waits, and F8 / F6 bank switching.

Nothing here executes 6502 code.  Expected values that depend on execution
come from the oracle only; the few closed-form facts the generator knows
(for example the frame at which the game-over byte is set) are returned in
the ROM's metadata so tests can check the oracle against them.
"""

from __future__ import annotations

import hashlib
import random
from dataclasses import dataclass, field

from .asm6502 import Assembler

# RAM map shared by all generated programs (zero page $80-$FF).
FC = 0x82        # 16-bit frame counter
PHASE = 0x84
TMP = 0x85
PAT = 0x86       # 16-byte pattern table $86-$95
P0Y, P1Y, M0Y, M1Y, BLY = 0x96, 0x97, 0x98, 0x99, 0x9A
P0X, P1X, M0X, M1X, BLX = 0x9B, 0x9C, 0x9D, 0x9E, 0x9F
VEL = 0xA0       # autonomous velocity of P1
LFSR = 0xA2      # 16-bit Galois LFSR (config-3 family)
TMP2 = 0xA4
SCORE_SLOTS = [(0x80, 0x81), (0xD0, 0xD1), (0xE0, 0xE1)]

# Joystick nibbles (SWCHA high nibble, active low: bit7 R, bit6 L, bit5 D, bit4 U)
# reachable with the 18 ALE actions.
VALID_NIBBLES = [0xF0, 0xE0, 0xD0, 0xB0, 0x70, 0x60, 0xA0, 0x50, 0x90]


@dataclass
class Rom:
    name: str
    data: bytes
    score_addr: int
    gameover_addr: int
    info: dict = field(default_factory=dict)

    @property
    def sha256(self) -> str:
        return hashlib.sha256(self.data).hexdigest()


def _equates(score, gameover):
    return {"SCORE": score, "GAMEOVER": gameover, "FC": FC, "PHASE": PHASE, "TMP": TMP,
            "PAT": PAT, "P0Y": P0Y, "P1Y": P1Y, "M0Y": M0Y, "M1Y": M1Y, "BLY": BLY,
            "P0X": P0X, "P1X": P1X, "M0X": M0X, "M1X": M1X, "BLX": BLX, "VEL": VEL,
            "LFSR": LFSR, "TMP2": TMP2}


def _hexb(vals):
    return ", ".join(f"${v & 0xFF:02X}" for v in vals)


# ---------------------------------------------------------------- building blocks

def _init_block(rng: random.Random, sprites: bool) -> str:
    pat = [rng.randrange(256) for _ in range(16)]
    s = f"""
Reset:  SEI
        CLD
        LDX #$FF
        TXS
        LDX #15
InitLp: LDA InitPat,X
        STA PAT,X
        DEX
        BPL InitLp
        LDA #${rng.randrange(256):02X}
        STA PHASE
        LDA #${rng.randrange(1, 256):02X}
        STA LFSR
        LDA #${rng.randrange(256):02X}
        STA LFSR+1
"""
    if sprites:
        vals = [rng.randrange(10, 170) for _ in range(5)] + [rng.randrange(8, 100) for _ in range(5)]
        for addr, v in zip(["P0Y", "P1Y", "M0Y", "M1Y", "BLY", "P0X", "P1X", "M0X", "M1X", "BLX"], vals):
            s += f"        LDA #{v}\n        STA {addr}\n"
        s += f"        LDA #${rng.choice([1, 2, 0xFF, 0xFE]):02X}\n        STA VEL\n"
        s += f"        LDA #${rng.choice([0, 1, 2, 3, 4, 6]) | (rng.randrange(4) << 4):02X}\n        STA NUSIZ0\n"
        s += f"        LDA #${rng.choice([0, 1, 3, 5, 7]) | (rng.randrange(4) << 4):02X}\n        STA NUSIZ1\n"
        s += f"        LDA #${rng.randrange(256) & 0xFE:02X}\n        STA COLUP0\n"
        s += f"        LDA #${rng.randrange(256) & 0xFE:02X}\n        STA COLUP1\n"
        ctrl = rng.choice([0x00, 0x01, 0x10, 0x11, 0x21, 0x31, 0x02, 0x04, 0x05, 0x13])
        s += f"        LDA #${ctrl:02X}\n        STA CTRLPF\n"
        s += f"        LDA #${rng.choice([0, 8]):02X}\n        STA REFP1\n"
        s += f"        LDA #${rng.choice([0, 1]):02X}\n        STA VDELP0\n"
        s += f"        LDA #${rng.choice([0, 1]):02X}\n        STA VDELBL\n"
    return s, pat


def _vsync_top() -> str:
    # Entered at cycle 0 of a line (after WSYNC); the VSYNC rise ends the frame.
    return """
Main:   LDA #2
        STA VSYNC
        STA VBLANK
        STA WSYNC
        STA WSYNC
        STA WSYNC
        LDA #0
        STA VSYNC
"""


def _chunk_joy_pf(rng) -> list[str]:
    """VBLANK logic for the playfield family; each chunk fits in one line."""
    a = """
        LDA SWCHA
        ASL
        BCS NoRight
        INC PHASE
NoRight: ASL
        BCS NoLeft
        DEC PHASE
NoLeft: STA TMP
        STA WSYNC
"""
    b = """
        LDA PHASE
        AND #15
        TAX
        LDA TMP
        ASL
        BCS NoDown
        ROL PAT,X
NoDown: ASL
        BCS NoUp
        LSR PAT,X
NoUp:   STA WSYNC
"""
    c = """
        LDA INPT4
        BMI NoFire
        LDA FC
        AND #15
        TAX
        LDA PAT,X
        EOR #$FF
        STA PAT,X
NoFire: STA WSYNC
"""
    cond = rng.choice(VALID_NIBBLES)
    d = f"""
        LDA SWCHA
        AND #$F0
        CMP #${cond:02X}
        BNE NoScore
        INC SCORE
NoScore: STA WSYNC
"""
    return [a, b, c, d], cond


def _chunk_gameover(limit: int) -> str:
    return f"""
        INC FC
        BNE FcHi
        INC FC+1
FcHi:   LDA FC
        CMP #<{limit}
        LDA FC+1
        SBC #>{limit}
        BCC NotOver
        LDA #1
        STA GAMEOVER
NotOver: STA WSYNC
"""


def _wait_lines(n: int, label: str) -> str:
    assert n >= 1
    return f"""
        LDX #{n}
{label}: STA WSYNC
        DEX
        BNE {label}
"""


def _visible_pf(rng) -> str:
    return """
        STA WSYNC
        LDA #0
        STA VBLANK
        LDY #0
Vis:    TYA
        CLC
        ADC PHASE
        AND #15
        TAX
        LDA ColTab,X
        STA COLUBK
        LDA PAT,X
        STA PF1
        EOR PHASE
        STA PF2
        AND #$F0
        STA PF0
        LDA PfTab,X
        STA COLUPF
        INY
        CPY #192
        STA WSYNC
        BNE Vis
"""


def _tables(rng, pat, sprites: bool) -> str:
    s = "        .align 256\n"
    s += "ColTab: .byte " + _hexb([rng.randrange(256) for _ in range(16)]) + "\n"
    s += "PfTab:  .byte " + _hexb([rng.randrange(256) for _ in range(16)]) + "\n"
    s += "InitPat: .byte " + _hexb(pat) + "\n"
    if sprites:
        s += "Spr0:   .byte " + _hexb([rng.randrange(256) for _ in range(16)]) + "\n"
        s += "Spr1:   .byte " + _hexb([rng.randrange(256) for _ in range(16)]) + "\n"
    return s


def _vectors(reset_label="Reset") -> str:
    return f"""
        .org $FFFA
        .word {reset_label}, {reset_label}, {reset_label}
"""


# ---------------------------------------------------------------- config-1 family

def rom_playfield(seed: int) -> Rom:
    """4 KB playfield/background program (the tiny plain-method workload)."""
    rng = random.Random(0x1000 + seed)
    score, gameover = SCORE_SLOTS[seed % 3]
    limit = rng.randrange(100, 401)
    init, pat = _init_block(rng, sprites=False)
    chunks, cond = _chunk_joy_pf(rng)
    src = "        .org $F000\n" + init + "        STA WSYNC\n" + _vsync_top()
    for c in chunks:                      # lines L0+3 .. L0+6
        src += c
    src += _wait_lines(36 - len(chunks), "VblWait")   # -> start of L0+39
    src += _visible_pf(rng)                            # L0+40 .. L0+231, ends at L0+232
    src += """
        LDA #2
        STA VBLANK
"""
    src += _chunk_gameover(limit)                      # L0+232
    src += _wait_lines(29, "OsWait")                   # -> L0+262
    src += "        JMP Main\n"
    src += _tables(rng, pat, sprites=False)
    src += _vectors()
    data = Assembler(_equates(score, gameover)).assemble(src, org=0xF000, size=4096)
    return Rom(f"playfield-{seed}", data, score, gameover,
               {"family": "playfield", "gameover_frame_counter": limit, "score_nibble": cond})


# ---------------------------------------------------------------- config-2 family

def _posobj_sub() -> str:
    # Coarse/fine horizontal positioning: A = x, X = object (0 P0 .. 4 BL).
    return """
PosObj: STA WSYNC
        SEC
PosDiv: SBC #15
        BCS PosDiv
        EOR #7
        ASL
        ASL
        ASL
        ASL
        STA HMP0,X
        STA RESP0,X
        RTS
"""


def _sprite_logic(rng, cond) -> list[str]:
    """VBLANK logic chunks of the sprite family (each one line)."""
    a = """
        LDA SWCHA
        ASL
        BCS SNoR
        INC P0X
SNoR:   ASL
        BCS SNoL
        DEC P0X
SNoL:   ASL
        BCS SNoD
        INC P0Y
SNoD:   ASL
        BCS SNoU
        DEC P0Y
SNoU:   STA WSYNC
"""
    b = """
        LDA P1Y
        CLC
        ADC VEL
        STA P1Y
        LDA P1X
        SEC
        SBC VEL
        STA P1X
        LDA INPT4
        BMI SNoF
        LDA P0Y
        STA M0Y
        LDA P0X
        STA M0X
SNoF:   STA WSYNC
"""
    c = f"""
        INC M1Y
        DEC BLX
        INC BLY
        INC BLY
        LDA SWCHA
        AND #$F0
        CMP #${cond:02X}
        BNE SNoSc
        INC PHASE
SNoSc:  STA WSYNC
"""
    # Clamp x positions to [0, 100) so PosObj (its divide loop plus the call
    # overhead) stays within one scanline per object; split in
    # two chunks (three objects, then two) so each fits in a scanline.
    def clamp(hi, lo, tag):
        return f"""
        LDX #{hi}
Clamp{tag}: LDA P0X,X
        CMP #100
        BCC ClampOk{tag}
        AND #$3F
        STA P0X,X
ClampOk{tag}: DEX
        CPX #{lo - 1 if lo > 0 else 255}
        BNE Clamp{tag}
        STA WSYNC
"""
    return [a, b, c, clamp(4, 2, "A"), clamp(1, 0, "B")]


def _sprite_positioning() -> str:
    # Five positioning lines, then HMOVE right after WSYNC, then HMCLR.
    s = ""
    for i, v in enumerate(["P0X", "P1X", "M0X", "M1X", "BLX"]):
        s += f"        LDA {v}\n        LDX #{i}\n        JSR PosObj\n"
    s += """
        STA WSYNC
        STA HMOVE
        LDA #0
        STA HMCLR
        STA WSYNC
"""
    return s  # consumes 7 lines (5 PosObj WSYNCs + 2)


def _visible_sprite(rng) -> str:
    # Two-line kernel: even lines P0 + ball + playfield, odd lines P1 + missiles.
    return """
        STA WSYNC
        LDA #0
        STA VBLANK
        LDY #0
SVis:   TYA
        SEC
        SBC P0Y
        CMP #16
        BCC SD0
        LDA #0
        BEQ SS0
SD0:    TAX
        LDA Spr0,X
SS0:    STA GRP0
        TYA
        SEC
        SBC BLY
        CMP #8
        LDA #0
        ROL
        EOR #1
        ASL
        STA ENABL
        TYA
        LSR
        LSR
        AND #15
        TAX
        LDA PAT,X
        STA PF1
        INY
        STA WSYNC
        TYA
        SEC
        SBC P1Y
        CMP #16
        BCC SD1
        LDA #0
        BEQ SS1
SD1:    TAX
        LDA Spr1,X
SS1:    STA GRP1
        TYA
        SEC
        SBC M0Y
        CMP #6
        LDA #0
        ROL
        EOR #1
        ASL
        STA ENAM0
        TYA
        SEC
        SBC M1Y
        CMP #4
        LDA #0
        ROL
        EOR #1
        ASL
        STA ENAM1
        INY
        CPY #192
        STA WSYNC
        BNE SVis
        LDA #0
        STA GRP0
        STA GRP1
        STA ENAM0
        STA ENAM1
        STA ENABL
"""


def _collision_score() -> str:
    # One overscan line: collisions drive the score, then clear the latches.
    return """
        LDA CXPPMM
        BPL NoPP
        INC SCORE
NoPP:   BIT CXM0P
        BVC NoM0P
        INC SCORE
NoM0P:  BIT CXP0FB
        BPL NoP0F
        INC SCORE
NoP0F:  STA CXCLR
        STA WSYNC
"""


def rom_sprite(seed: int) -> Rom:
    """4 KB program with players, missiles, ball, HMOVE and collision-driven score."""
    rng = random.Random(0x2000 + seed)
    score, gameover = SCORE_SLOTS[seed % 3]
    limit = rng.randrange(100, 401)
    init, pat = _init_block(rng, sprites=True)
    cond = rng.choice(VALID_NIBBLES)
    src = "        .org $F000\n" + init + "        STA WSYNC\n" + _vsync_top()
    chunks = _sprite_logic(rng, cond)
    for c in chunks:                                   # L0+3 .. L0+6
        src += c
    src += _sprite_positioning()                       # 7 lines -> L0+14
    src += _wait_lines(36 - len(chunks) - 7, "SVblW")  # -> L0+39
    src += _visible_sprite(rng)                        # L0+40 .. L0+231 -> L0+232
    src += """
        LDA #2
        STA VBLANK
"""
    src += _collision_score()                          # L0+232
    src += _chunk_gameover(limit)                      # L0+233
    src += _wait_lines(28, "SOsW")                     # -> L0+262
    src += "        JMP Main\n"
    src += _posobj_sub()
    src += _tables(rng, pat, sprites=True)
    src += _vectors()
    data = Assembler(_equates(score, gameover)).assemble(src, org=0xF000, size=4096)
    return Rom(f"sprite-{seed}", data, score, gameover,
               {"family": "sprite", "gameover_frame_counter": limit})


# ---------------------------------------------------------------- config-3 family

def _lfsr_gameover(threshold: int = 44) -> str:
    # Galois LFSR step mixed with the joystick; game over when below threshold
    # (after frame 128 so the start-state cache never holds a finished game).
    return f"""
        LDA SWCHA
        AND #$F0
        EOR LFSR
        STA LFSR
        LSR LFSR+1
        ROR LFSR
        BCC LfNoTap
        LDA LFSR+1
        EOR #$B4
        STA LFSR+1
LfNoTap: INC FC
        BNE LfHi
        INC FC+1
LfHi:   LDA FC+1
        BNE LfChk
        LDA FC
        BPL LfDone
LfChk:  LDA LFSR+1
        BNE LfDone
        LDA LFSR
        CMP #{threshold}
        BCS LfDone
        LDA #1
        STA GAMEOVER
LfDone:
"""


def rom_banked(seed: int, scheme: str) -> Rom:
    """Batching family: 4 KB, F8 (8 KB), F6 (16 KB) or F4 (32 KB) with code in
    every bank.

    Bank 0 holds reset and the frame loop with RIOT-timer VBLANK and overscan
    waits.  The game logic runs in the last bank and the visible kernel in
    bank 1 (4 KB carts keep everything in one bank).  Banks are entered
    through stubs at $FFC0 + 6 j, identical in every bank: touch hotspot j,
    then JMP to bank j's entry ($F000 for j >= 1, $F800 for bank 0).  F4's
    hotspots start at $FFF4, so its stubs sit lower, at $FF80 + 6 j.
    """
    rng = random.Random(0x3000 + seed)
    nbanks = {"4k": 1, "f8": 2, "f6": 4, "f4": 8}[scheme]
    hot0 = {"4k": None, "f8": 0x1FF8, "f6": 0x1FF6, "f4": 0x1FF4}[scheme]
    stub_base = 0xFF80 if scheme == "f4" else 0xFFC0
    score, gameover = SCORE_SLOTS[seed % 3]
    sprites = rng.random() < 0.5
    init, pat = _init_block(rng, sprites=sprites)
    cond = rng.choice(VALID_NIBBLES)
    eq = _equates(score, gameover)
    kern_bank = 1 % nbanks
    logic_bank = nbanks - 1
    visible = _visible_sprite(rng) if sprites else _visible_pf(rng)
    if sprites:
        chunks = _sprite_logic(rng, cond)
    else:
        chunks, _ = _chunk_joy_pf(rng)
    logic = "".join(c.replace("STA WSYNC", "") for c in chunks)
    if sprites:
        logic += _sprite_positioning()

    def go(bank):
        return f"        JMP Stub{bank}\n" if nbanks > 1 else {0: "        JMP Entry0\n",
                                                              "L": "        JMP EntryL\n",
                                                              "K": "        JMP EntryK\n"}[bank]

    frame = "        .org $F000\n" + init + "        STA WSYNC\n" + _vsync_top() + """
        LDA #43
        STA TIM64T
        LDA #1
        STA TMP2
""" + (go(logic_bank) if nbanks > 1 else go("L"))
    cont = """
        .org $F800
Entry0: LDA TMP2
        CMP #1
        BEQ AfterLogic
        LDA #2
        STA VBLANK
        LDA #34
        STA TIM64T
""" + (_collision_score().replace("STA WSYNC", "") if sprites else "") + _lfsr_gameover() + """
OsWait: LDA INTIM
        BNE OsWait
        STA WSYNC
        JMP Main
AfterLogic:
        LDA #2
        STA TMP2
VbWait: LDA INTIM
        BNE VbWait
""" + (go(kern_bank) if nbanks > 1 else go("K"))
    tables = _tables(rng, pat, sprites)

    def stubs():
        s = f"        .org ${stub_base:04X}\n"
        for j in range(nbanks):
            s += f"Stub{j}: BIT ${hot0 + j:04X}\n        JMP ${0xF800 if j == 0 else 0xF000:04X}\n"
        s += f"ResetStub: BIT ${hot0:04X}\n        JMP Reset\n"
        return s

    images = []
    if nbanks == 1:
        src = frame + "EntryL:\n" + logic + go(0) + "EntryK:\n" + visible + go(0)
        if sprites:
            src += _posobj_sub()
        src += cont + tables + _vectors()
        img = Assembler(eq).assemble(src, org=0xF000, size=4096)
        images.append(img)
    else:
        for b in range(nbanks):
            if b == 0:
                src = frame + cont
            elif b == logic_bank:
                src = "        .org $F000\nLogicEntry:\n" + logic + go(0) + (_posobj_sub() if sprites else "")
            elif b == kern_bank:
                src = "        .org $F000\nKernEntry:\n" + visible + go(0)
            else:
                src = "        .org $F000\nSpare: JMP Stub0\n"
            src += tables + stubs() + _vectors("ResetStub")
            syms = dict(eq)
            if b != 0:
                syms["Reset"] = 0xF000
            img = Assembler(syms).assemble(src, org=0xF000, size=4096)
            images.append(img)
    data = b"".join(images)
    return Rom(f"banked-{scheme}-{seed}", data, score, gameover,
               {"family": "banked", "scheme": scheme, "sprites": sprites})


# ---------------------------------------------------------------- workloads

def luma_table() -> bytes:
    """128-entry luma table of the console's color indices (index = value >> 1).

    Stated YIQ model: hue h = i >> 3, lum l = i & 7; Y = 0.075 + 0.125 l;
    hue 0 is gray (I = Q = 0); hue h >= 1 has chroma 0.25 at angle
    33 deg + (h - 1) * 360/15 deg.  RGB from the FCC YIQ matrix, clamped to
    [0, 1] and rounded to 8 bits, then luma = (299 R + 587 G + 114 B + 500) // 1000.
    """
    import math
    out = bytearray(128)
    for i in range(128):
        h, l = i >> 3, i & 7
        y = 0.075 + 0.125 * l
        if h == 0:
            ii = qq = 0.0
        else:
            th = math.radians(33.0 + (h - 1) * 24.0)
            ii, qq = 0.25 * math.cos(th), 0.25 * math.sin(th)
        rgb = (y + 0.956 * ii + 0.621 * qq, y - 0.272 * ii - 0.647 * qq, y - 1.106 * ii + 1.703 * qq)
        r, g, b = (int(round(255.0 * min(1.0, max(0.0, c)))) for c in rgb)
        out[i] = (299 * r + 587 * g + 114 * b + 500) // 1000
    return bytes(out)


@dataclass
class Workload:
    name: str
    roms: list
    env_rom: list          # ROM index of each env, ROM-major
    n_envs: int
    steps: int
    frameskip: int = 4
    sticky: bool = False
    output_mode: int = 1   # 0 = palette frame of the last frame, 1 = 84x84x4 luma stack
    seed: int = 1


def workload(config: int, n_envs: int | None = None, steps: int | None = None) -> Workload:
    """The five synthetic workloads (sizes overridable for smaller test cases)."""
    if config == 1:
        roms = [rom_playfield(1)]
        n = n_envs or 16
        return Workload("playfield-4k x16", roms, [0] * n, n, steps or 250, output_mode=0, seed=1)
    if config == 2:
        roms = [rom_sprite(s) for s in range(1, 9)]
        n = n_envs or 4096
        return Workload("sprite-4k x8 roms, 4096 envs", roms, _rom_major(n, len(roms)), n, steps or 2000, seed=2)
    if config == 3:
        schemes = ["4k"] * 12 + ["f8"] * 10 + ["f6"] * 10
        roms = [rom_banked(s + 1, schemes[s]) for s in range(32)]
        n = n_envs or 32768
        return Workload("banked 4k/f8/f6 x32 roms, 32768 envs, sticky", roms, _rom_major(n, len(roms)), n,
                        steps or 1000, sticky=True, seed=3)
    if config == 5:
        roms = [rom_sprite(s) for s in range(1, 17)]
        n = n_envs or 16384
        return Workload("sprite-4k x16 roms, 16384 envs, policy", roms, _rom_major(n, len(roms)), n,
                        steps or 10000, seed=5)
    raise ValueError(config)


def _rom_major(n: int, r: int) -> list:
    return [min(r - 1, (i * r) // n) for i in range(n)]


def actions(seed: int, steps: int, n_envs: int, n_actions: int = 18):
    """Uniform random actions, [steps, n_envs] uint8, from a seeded counter-based stream."""
    import numpy as np
    g = np.random.Generator(np.random.Philox(key=seed))
    return g.integers(0, n_actions, size=(steps, n_envs), dtype=np.uint8)
