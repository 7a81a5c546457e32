"""Tiny two-pass assembler for the documented NMOS 6502 instruction set.

Input generator only: it turns assembly text into cartridge bytes.  It holds
no emulation arithmetic (nothing here executes an instruction), so both the
CPU oracle and the CUDA path may consume what it produces.

Syntax (one statement per line, ';' starts a comment):

    name = expr            equate (evaluated immediately, must be known)
    label:                 label at the current address
    .org expr              set the location counter
    .byte e1, e2, ...      emit bytes
    .word e1, e2, ...      emit little-endian 16-bit words
    .fill n, value         emit n copies of value
    .align n[, value]      pad to a multiple of n
    MNE                    implied / accumulator ("ASL" or "ASL A")
    MNE #expr              immediate
    MNE expr               zero page if the value is known and < $100 and the
                           opcode has a zero-page form, else absolute
    MNE expr,X / expr,Y    indexed (zero page or absolute as above)
    MNE (expr,X)           indexed indirect
    MNE (expr),Y           indirect indexed
    JMP (expr)             indirect
    Bxx expr               relative branch
    MNE.w ...              force the absolute form

Expressions are Python expressions over numbers ($hex, %bin, decimal), labels,
equates, '<' (low byte) and '>' (high byte) prefixes.
"""

from __future__ import annotations

import re

# Documented NMOS 6502 opcode map: mnemonic -> {mode: opcode}.
# Modes: imp acc imm zp zpx zpy abs abx aby ind izx izy rel
OPCODES = {
    "ADC": {"imm": 0x69, "zp": 0x65, "zpx": 0x75, "abs": 0x6D, "abx": 0x7D, "aby": 0x79, "izx": 0x61, "izy": 0x71},
    "AND": {"imm": 0x29, "zp": 0x25, "zpx": 0x35, "abs": 0x2D, "abx": 0x3D, "aby": 0x39, "izx": 0x21, "izy": 0x31},
    "ASL": {"acc": 0x0A, "zp": 0x06, "zpx": 0x16, "abs": 0x0E, "abx": 0x1E},
    "BCC": {"rel": 0x90}, "BCS": {"rel": 0xB0}, "BEQ": {"rel": 0xF0}, "BMI": {"rel": 0x30},
    "BNE": {"rel": 0xD0}, "BPL": {"rel": 0x10}, "BVC": {"rel": 0x50}, "BVS": {"rel": 0x70},
    "BIT": {"zp": 0x24, "abs": 0x2C},
    "BRK": {"imp": 0x00},
    "CLC": {"imp": 0x18}, "CLD": {"imp": 0xD8}, "CLI": {"imp": 0x58}, "CLV": {"imp": 0xB8},
    "CMP": {"imm": 0xC9, "zp": 0xC5, "zpx": 0xD5, "abs": 0xCD, "abx": 0xDD, "aby": 0xD9, "izx": 0xC1, "izy": 0xD1},
    "CPX": {"imm": 0xE0, "zp": 0xE4, "abs": 0xEC},
    "CPY": {"imm": 0xC0, "zp": 0xC4, "abs": 0xCC},
    "DEC": {"zp": 0xC6, "zpx": 0xD6, "abs": 0xCE, "abx": 0xDE},
    "DEX": {"imp": 0xCA}, "DEY": {"imp": 0x88},
    "EOR": {"imm": 0x49, "zp": 0x45, "zpx": 0x55, "abs": 0x4D, "abx": 0x5D, "aby": 0x59, "izx": 0x41, "izy": 0x51},
    "INC": {"zp": 0xE6, "zpx": 0xF6, "abs": 0xEE, "abx": 0xFE},
    "INX": {"imp": 0xE8}, "INY": {"imp": 0xC8},
    "JMP": {"abs": 0x4C, "ind": 0x6C},
    "JSR": {"abs": 0x20},
    "LDA": {"imm": 0xA9, "zp": 0xA5, "zpx": 0xB5, "abs": 0xAD, "abx": 0xBD, "aby": 0xB9, "izx": 0xA1, "izy": 0xB1},
    "LDX": {"imm": 0xA2, "zp": 0xA6, "zpy": 0xB6, "abs": 0xAE, "aby": 0xBE},
    "LDY": {"imm": 0xA0, "zp": 0xA4, "zpx": 0xB4, "abs": 0xAC, "abx": 0xBC},
    "LSR": {"acc": 0x4A, "zp": 0x46, "zpx": 0x56, "abs": 0x4E, "abx": 0x5E},
    "NOP": {"imp": 0xEA},
    "ORA": {"imm": 0x09, "zp": 0x05, "zpx": 0x15, "abs": 0x0D, "abx": 0x1D, "aby": 0x19, "izx": 0x01, "izy": 0x11},
    "PHA": {"imp": 0x48}, "PHP": {"imp": 0x08}, "PLA": {"imp": 0x68}, "PLP": {"imp": 0x28},
    "ROL": {"acc": 0x2A, "zp": 0x26, "zpx": 0x36, "abs": 0x2E, "abx": 0x3E},
    "ROR": {"acc": 0x6A, "zp": 0x66, "zpx": 0x76, "abs": 0x6E, "abx": 0x7E},
    "RTI": {"imp": 0x40}, "RTS": {"imp": 0x60},
    "SBC": {"imm": 0xE9, "zp": 0xE5, "zpx": 0xF5, "abs": 0xED, "abx": 0xFD, "aby": 0xF9, "izx": 0xE1, "izy": 0xF1},
    "SEC": {"imp": 0x38}, "SED": {"imp": 0xF8}, "SEI": {"imp": 0x78},
    "STA": {"zp": 0x85, "zpx": 0x95, "abs": 0x8D, "abx": 0x9D, "aby": 0x99, "izx": 0x81, "izy": 0x91},
    "STX": {"zp": 0x86, "zpy": 0x96, "abs": 0x8E},
    "STY": {"zp": 0x84, "zpx": 0x94, "abs": 0x8C},
    "TAX": {"imp": 0xAA}, "TAY": {"imp": 0xA8}, "TSX": {"imp": 0xBA}, "TXA": {"imp": 0x8A},
    "TXS": {"imp": 0x9A}, "TYA": {"imp": 0x98},
}

# Stable undocumented NMOS operations (for cartridges and tests that use
# them); the assembler accepts these mnemonics as well.
UNDOC_OPCODES = {
    "SLO": {"zp": 0x07, "zpx": 0x17, "abs": 0x0F, "abx": 0x1F, "aby": 0x1B, "izx": 0x03, "izy": 0x13},
    "RLA": {"zp": 0x27, "zpx": 0x37, "abs": 0x2F, "abx": 0x3F, "aby": 0x3B, "izx": 0x23, "izy": 0x33},
    "SRE": {"zp": 0x47, "zpx": 0x57, "abs": 0x4F, "abx": 0x5F, "aby": 0x5B, "izx": 0x43, "izy": 0x53},
    "RRA": {"zp": 0x67, "zpx": 0x77, "abs": 0x6F, "abx": 0x7F, "aby": 0x7B, "izx": 0x63, "izy": 0x73},
    "DCP": {"zp": 0xC7, "zpx": 0xD7, "abs": 0xCF, "abx": 0xDF, "aby": 0xDB, "izx": 0xC3, "izy": 0xD3},
    "ISC": {"zp": 0xE7, "zpx": 0xF7, "abs": 0xEF, "abx": 0xFF, "aby": 0xFB, "izx": 0xE3, "izy": 0xF3},
    "SAX": {"zp": 0x87, "zpy": 0x97, "abs": 0x8F, "izx": 0x83},
    "LAX": {"zp": 0xA7, "zpy": 0xB7, "abs": 0xAF, "aby": 0xBF, "izx": 0xA3, "izy": 0xB3},
    "ANC": {"imm": 0x0B}, "ALR": {"imm": 0x4B}, "SBX": {"imm": 0xCB},
}
ALL_OPCODES = {**OPCODES, **UNDOC_OPCODES}

MODE_SIZE = {"imp": 1, "acc": 1, "imm": 2, "zp": 2, "zpx": 2, "zpy": 2, "abs": 3, "abx": 3,
             "aby": 3, "ind": 3, "izx": 2, "izy": 2, "rel": 2}

# Standard register names of the console (write and read views of the TIA, RIOT).
SYMBOLS = {
    "VSYNC": 0x00, "VBLANK": 0x01, "WSYNC": 0x02, "RSYNC": 0x03, "NUSIZ0": 0x04, "NUSIZ1": 0x05,
    "COLUP0": 0x06, "COLUP1": 0x07, "COLUPF": 0x08, "COLUBK": 0x09, "CTRLPF": 0x0A, "REFP0": 0x0B,
    "REFP1": 0x0C, "PF0": 0x0D, "PF1": 0x0E, "PF2": 0x0F, "RESP0": 0x10, "RESP1": 0x11,
    "RESM0": 0x12, "RESM1": 0x13, "RESBL": 0x14, "AUDC0": 0x15, "AUDC1": 0x16, "AUDF0": 0x17,
    "AUDF1": 0x18, "AUDV0": 0x19, "AUDV1": 0x1A, "GRP0": 0x1B, "GRP1": 0x1C, "ENAM0": 0x1D,
    "ENAM1": 0x1E, "ENABL": 0x1F, "HMP0": 0x20, "HMP1": 0x21, "HMM0": 0x22, "HMM1": 0x23,
    "HMBL": 0x24, "VDELP0": 0x25, "VDELP1": 0x26, "VDELBL": 0x27, "RESMP0": 0x28, "RESMP1": 0x29,
    "HMOVE": 0x2A, "HMCLR": 0x2B, "CXCLR": 0x2C,
    "CXM0P": 0x00, "CXM1P": 0x01, "CXP0FB": 0x02, "CXP1FB": 0x03, "CXM0FB": 0x04, "CXM1FB": 0x05,
    "CXBLPF": 0x06, "CXPPMM": 0x07, "INPT0": 0x08, "INPT1": 0x09, "INPT2": 0x0A, "INPT3": 0x0B,
    "INPT4": 0x0C, "INPT5": 0x0D,
    "SWCHA": 0x280, "SWACNT": 0x281, "SWCHB": 0x282, "SWBCNT": 0x283, "INTIM": 0x284,
    "TIMINT": 0x285, "TIM1T": 0x294, "TIM8T": 0x295, "TIM64T": 0x296, "T1024T": 0x297,
}


class AsmError(Exception):
    pass


_num_re = re.compile(r"\$([0-9A-Fa-f]+)|%([01]+)")


def _py_expr(text: str) -> str:
    text = _num_re.sub(lambda m: str(int(m.group(1), 16)) if m.group(1) else str(int(m.group(2), 2)), text)
    text = text.strip()
    if text.startswith("<"):
        return "((" + text[1:] + ") & 255)"
    if text.startswith(">"):
        return "(((" + text[1:] + ") >> 8) & 255)"
    return text


class Assembler:
    """Two passes: pass 1 fixes every statement's size, pass 2 emits bytes."""

    def __init__(self, symbols: dict | None = None):
        self.symbols = dict(SYMBOLS)
        if symbols:
            self.symbols.update(symbols)

    def _eval(self, expr: str, env: dict, strict: bool):
        try:
            return int(eval(_py_expr(expr), {"__builtins__": {}}, env))
        except NameError:
            if strict:
                raise AsmError(f"undefined symbol in '{expr}'")
            return None

    def _parse_operand(self, mne: str, opnd: str, env: dict, strict: bool, force_abs: bool):
        modes = ALL_OPCODES[mne]
        o = opnd.strip()
        if o == "" or o.upper() == "A":
            if "acc" in modes:
                return "acc", None
            if "imp" in modes and o == "":
                return "imp", None
            raise AsmError(f"{mne}: operand required")
        if "rel" in modes:
            return "rel", self._eval(o, env, strict)
        if o.startswith("#"):
            return "imm", self._eval(o[1:], env, strict)
        m = re.fullmatch(r"\((.+),\s*[xX]\s*\)", o)
        if m:
            return "izx", self._eval(m.group(1), env, strict)
        m = re.fullmatch(r"\((.+)\)\s*,\s*[yY]", o)
        if m:
            return "izy", self._eval(m.group(1), env, strict)
        m = re.fullmatch(r"\((.+)\)", o)
        if m and "ind" in modes:
            return "ind", self._eval(m.group(1), env, strict)
        idx = None
        m = re.fullmatch(r"(.+),\s*([xXyY])", o)
        if m:
            o, idx = m.group(1), m.group(2).upper()
        v = self._eval(o, env, strict)
        zp_mode = {None: "zp", "X": "zpx", "Y": "zpy"}[idx]
        abs_mode = {None: "abs", "X": "abx", "Y": "aby"}[idx]
        if (not force_abs) and v is not None and 0 <= v < 0x100 and zp_mode in modes:
            return zp_mode, v
        if abs_mode not in modes:
            raise AsmError(f"{mne}: no {abs_mode} form for '{opnd}'")
        return abs_mode, v

    def assemble(self, text: str, org: int = 0xF000, size: int = 4096, fill: int = 0xFF):
        """Assemble `text` into a `size`-byte image whose first byte is at `org`."""
        lines = []
        for raw in text.splitlines():
            line = raw.split(";", 1)[0].rstrip()
            if line.strip():
                lines.append(line)
        labels: dict = {}
        modes1: dict = {}
        for pass_no in (1, 2):
            strict = pass_no == 2
            env = dict(self.symbols)
            env.update(labels)
            pc = org
            image = bytearray([fill] * size)
            for li, line in enumerate(lines):
                s = line.strip()
                m = re.match(r"^([A-Za-z_][A-Za-z0-9_]*):\s*(.*)$", s)
                if m:
                    labels[m.group(1)] = pc
                    env[m.group(1)] = pc
                    s = m.group(2).strip()
                    if not s:
                        continue
                m = re.match(r"^([A-Za-z_][A-Za-z0-9_]*)\s*=\s*(.+)$", s)
                if m:
                    v = self._eval(m.group(2), env, True)
                    self.symbols[m.group(1)] = v
                    env[m.group(1)] = v
                    continue
                if s.startswith("."):
                    d, _, rest = s.partition(" ")
                    d = d.lower()
                    args = [a for a in rest.split(",")] if rest.strip() else []
                    if d == ".org":
                        pc = self._eval(rest, env, True)
                    elif d in (".byte", ".word"):
                        w = 1 if d == ".byte" else 2
                        for a in args:
                            v = self._eval(a, env, strict) or 0
                            for i in range(w):
                                self._emit(image, org, size, pc + i, (v >> (8 * i)) & 0xFF, strict)
                            pc += w
                    elif d == ".fill":
                        n = self._eval(args[0], env, True)
                        v = self._eval(args[1], env, True) if len(args) > 1 else 0
                        for i in range(n):
                            self._emit(image, org, size, pc + i, v & 0xFF, strict)
                        pc += n
                    elif d == ".align":
                        n = self._eval(args[0], env, True)
                        v = self._eval(args[1], env, True) if len(args) > 1 else 0
                        while pc % n:
                            self._emit(image, org, size, pc, v & 0xFF, strict)
                            pc += 1
                    else:
                        raise AsmError(f"unknown directive {d}")
                    continue
                parts = s.split(None, 1)
                mne = parts[0].upper()
                force_abs = mne.endswith(".W")
                if force_abs:
                    mne = mne[:-2]
                if mne not in ALL_OPCODES:
                    raise AsmError(f"unknown mnemonic '{mne}' in '{line}'")
                if pass_no == 2 and modes1.get(li) in ("abs", "abx", "aby"):
                    force_abs = True  # keep the size chosen in pass 1 (forward reference)
                mode, v = self._parse_operand(mne, parts[1] if len(parts) > 1 else "", env, strict, force_abs)
                if pass_no == 1:
                    modes1[li] = mode
                op = ALL_OPCODES[mne][mode]
                n = MODE_SIZE[mode]
                self._emit(image, org, size, pc, op, strict)
                if mode == "rel":
                    if strict:
                        off = v - (pc + 2)
                        if not -128 <= off <= 127:
                            raise AsmError(f"branch out of range in '{line}'")
                        self._emit(image, org, size, pc + 1, off & 0xFF, strict)
                elif n >= 2:
                    val = v if v is not None else 0
                    if strict and mode in ("imm", "zp", "zpx", "zpy", "izx", "izy") and not 0 <= val < 0x100:
                        raise AsmError(f"operand out of byte range in '{line}'")
                    self._emit(image, org, size, pc + 1, val & 0xFF, strict)
                    if n == 3:
                        self._emit(image, org, size, pc + 2, (val >> 8) & 0xFF, strict)
                pc += n
        self.labels = labels
        return bytes(image)

    @staticmethod
    def _emit(image, org, size, addr, byte, strict):
        off = addr - org
        if not 0 <= off < size:
            if strict:
                raise AsmError(f"address ${addr:04X} outside image")
            return
        image[off] = byte


def assemble(text: str, org: int = 0xF000, size: int = 4096, symbols: dict | None = None, fill: int = 0xFF):
    a = Assembler(symbols)
    img = a.assemble(text, org=org, size=size, fill=fill)
    return img, a.labels
