/*
 * CPU oracle -- TEST INFRASTRUCTURE (see oracle.h).  Plain C, single-threaded
 * per environment, no code shared with the CUDA path.
 *
 * Paper passages followed:
 *   - Section 3 (CuLE): one emulated console per environment; CPU state and
 *     the 128-byte RAM per console; the TIA renders a 160x210 frame; only the
 *     last two frames of a four-frame skip are rendered because the agent
 *     sees their pixelwise maximum; reset copies one of 30 cached start
 *     states built from 64 start-up frames plus up to 30 random no-op frames.
 *   - Section 1 footnote on raw frames: every emulated frame counts, frame
 *     skip 4.
 *   - Section 4 (memory discussion): four stacked 84x84 frames per env.
 *
 * The machine behaviour is the public definition of the console, with these
 * readings where the paper is silent:
 *   R1  a frame ends when a VSYNC write takes D1 from 0 to 1 (the writing
 *       instruction completes), or at the first instruction boundary 400
 *       lines after the frame's first line (status FRAME_CAP).
 *   R2  the 210-row window starts 31 lines after the frame's first line;
 *       columns are color clocks 68..227 of a 228-clock line.
 *   R3  an instruction starting at cycle k0 and lasting n cycles makes its
 *       data access at kA = k0 + n - 1 (read-modify-write: read at kA-2,
 *       old value written at kA-1, new value at kA); opcode, operand and
 *       indirect-pointer fetches happen at k0.  A TIA write takes effect at
 *       color clock 3(t+1) for an access at cycle t; a collision read at t
 *       sees pixels at clocks < 3t.
 *   R4  RESPx at beam column b puts the player at (b+5) mod 160, RESMx/RESBL
 *       at (b+4) mod 160; during HBLANK at 3 / 2.
 *   R5  HMOVE moves all five objects immediately by the signed high nibble
 *       of HMxx (positive = left); an HMOVE whose effect clock is in HBLANK
 *       blanks columns 0..7 of that line.
 *   R6  collisions latch only at visible, unblanked pixels.
 *   R7  pixel value = COLUxx & 0xFE.
 *   R8  playfield priority (CTRLPF D2) wins over score mode (CTRLPF D1).
 *   R9  undriven TIA read bits are 0; INPT0..3 read 0; INPT5 reads 0x80.
 *   R10 RIOT timer: written value v, interval I = 2^s at cycle w; read at
 *       cycle c, n = c - (w + 1): n < (v+1) I gives v - floor(n / I), else
 *       (0xFF - (n - (v+1) I)) & 0xFF with the TIMINT flag (bit 7) set.
 *   R11 power-on: registers and RAM 0, SP = 0xFD, P = 0x24, bank 0, PC from
 *       the reset vector, timer 0 with interval 1024 written at cycle 0.
 *   R12 the stable undocumented opcodes of the NMOS part execute per their
 *       published descriptions (see UNDOC below); the other 21 opcodes halt
 *       the CPU (JAM, status ILLEGAL); the env is done at the end of every
 *       step it ends halted, which also sets ILLEGAL.
 *   R13 decimal mode follows the NMOS behaviour described by B. Clark
 *       ("Decimal Mode", 6502.org): A and C by nibble adjustment, N and V
 *       from the intermediate result of ADC, Z (and all SBC flags) binary.
 *   R16 a cartridge hotspot access switches the bank first; a read returns
 *       the byte of the new bank.
 *   R17-R21 env semantics: see orc_envs_step.
 *   RESMPx: while D1 is set the missile is hidden; when D1 goes 1 -> 0 the
 *       missile is placed at the player's position + 4 * (player scale).
 *   Score mode colors playfield pixels (not the ball) with COLUP0 on the
 *       left half and COLUP1 on the right half; within the playfield/ball
 *       tier a playfield pixel is chosen before a ball pixel.
 *   INPT4 reads 0x00 while fire is pressed; with VBLANK D6 set, a press is
 *       latched until a VBLANK write clears D6.
 *   Policy (inference-path loop, Section 4's inference-only measurements with
 *       a DNN picking actions on the device): a linear softmax over the
 *       84x84x4 stack with bf16 weights and fp32 accumulation; the fp32
 *       reduction order is fixed (441 chunks of 64 sequential fmaf, partials
 *       reduced pairwise s[i] += s[i + h] for h = 256, 128, ..., 1 over 512
 *       zero-padded slots), exp is Cody-Waite reduction plus a degree-7
 *       Taylor polynomial, and the action is the smallest j whose running
 *       sum exceeds u * total, u = (x >> 8) 2^-24 for the env's Philox word
 *       x (the last action with nonzero weight if rounding leaves none).
 *   Learner-side targets over a rollout (Appendix, "A2C" and "V-trace"): the
 *       bootstrapped N-step return of the A2C cost and the V-trace target of
 *       its sum definition with truncated importance weights, in double
 *       precision; a done inside the rollout ends the return (the discount
 *       after a done step is 0), which the paper does not discuss.
 */
#include "oracle.h"
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ machine */

enum { OBJ_P0 = 1, OBJ_P1 = 2, OBJ_M0 = 4, OBJ_M1 = 8, OBJ_BL = 16, OBJ_PF = 32 };
#define NO_LINE (~(uint64_t)0)
#define LINE_CLOCKS 228
#define LINE_CYCLES 76
#define WINDOW_Y0 31
#define FRAME_CAP_LINES 400

struct orc_machine {
    /* CPU */
    uint8_t a, x, y, sp, p, jam;
    uint16_t pc;
    uint64_t k;            /* CPU cycles since power-on */
    uint64_t instret;
    /* cartridge */
    const uint8_t *rom;
    uint32_t rom_size;
    int scheme;            /* 0: 2K/4K, 1: F8, 2: F6, 3: F4 */
    uint8_t bank;
    /* RIOT */
    uint8_t ram[128];
    uint64_t tim_cw;
    uint8_t tim_v, tim_shift;
    uint8_t swcha_out, swacnt, swchb_out, swbcnt;
    uint8_t joy;           /* SWCHA input pins (active low) */
    uint8_t fire;          /* 1 while the P0 button is pressed */
    uint8_t inpt4_latch;
    /* TIA */
    uint8_t vsync, vblank, nusiz[2], colup[2], colupf, colubk, ctrlpf, refp[2];
    uint8_t pf0, pf1, pf2, enam[2], enabl_new, enabl_old;
    uint8_t grp_new[2], grp_old[2], vdelp[2], vdelbl, resmp[2];
    uint8_t hm[5];         /* HMP0 HMP1 HMM0 HMM1 HMBL */
    uint8_t pos[5];        /* P0 P1 M0 M1 BL */
    uint16_t cx;
    uint64_t bar_line;
    uint64_t tia_clock;    /* every color clock < tia_clock has been evaluated */
    /* frame bookkeeping */
    uint64_t frame_line;   /* first line of the current frame */
    uint32_t frame_no;
    uint8_t *fb;           /* 210x160 target while rendering, else NULL */
    /* per-instruction events */
    int wsync, vs_rise;
    uint64_t vs_rise_t, last_vsync_t;
    int have_vsync;
    uint32_t tia_writes;
    uint32_t status;
};

/* ---- opcode table: documented NMOS 6502, plus the stable undocumented opcodes ---- */
enum {
    M_IMP, M_ACC, M_IMM, M_ZP, M_ZPX, M_ZPY, M_ABS, M_ABX, M_ABY, M_IND, M_IZX, M_IZY, M_REL
};
enum {
    O_ADC = 1, O_AND, O_ASL, O_BCC, O_BCS, O_BEQ, O_BIT, O_BMI, O_BNE, O_BPL, O_BRK, O_BVC, O_BVS,
    O_CLC, O_CLD, O_CLI, O_CLV, O_CMP, O_CPX, O_CPY, O_DEC, O_DEX, O_DEY, O_EOR, O_INC, O_INX,
    O_INY, O_JMP, O_JSR, O_LDA, O_LDX, O_LDY, O_LSR, O_NOP, O_ORA, O_PHA, O_PHP, O_PLA, O_PLP,
    O_ROL, O_ROR, O_RTI, O_RTS, O_SBC, O_SEC, O_SED, O_SEI, O_STA, O_STX, O_STY, O_TAX, O_TAY,
    O_TSX, O_TXA, O_TXS, O_TYA,
    /* undocumented NMOS operations with a stable, published behaviour */
    O_SLO, O_RLA, O_SRE, O_RRA, O_SAX, O_LAX, O_DCP, O_ISC, O_ANC, O_ALR, O_SBX
};
typedef struct { uint8_t op, mode, cycles; } opinfo;
static const uint8_t MODE_LEN[13] = {1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 2, 2, 2};

/* (opcode, operation, mode, documented base cycles) */
static const uint8_t DOC[151][4] = {
    {0x69,O_ADC,M_IMM,2},{0x65,O_ADC,M_ZP,3},{0x75,O_ADC,M_ZPX,4},{0x6D,O_ADC,M_ABS,4},
    {0x7D,O_ADC,M_ABX,4},{0x79,O_ADC,M_ABY,4},{0x61,O_ADC,M_IZX,6},{0x71,O_ADC,M_IZY,5},
    {0x29,O_AND,M_IMM,2},{0x25,O_AND,M_ZP,3},{0x35,O_AND,M_ZPX,4},{0x2D,O_AND,M_ABS,4},
    {0x3D,O_AND,M_ABX,4},{0x39,O_AND,M_ABY,4},{0x21,O_AND,M_IZX,6},{0x31,O_AND,M_IZY,5},
    {0x0A,O_ASL,M_ACC,2},{0x06,O_ASL,M_ZP,5},{0x16,O_ASL,M_ZPX,6},{0x0E,O_ASL,M_ABS,6},
    {0x1E,O_ASL,M_ABX,7},
    {0x90,O_BCC,M_REL,2},{0xB0,O_BCS,M_REL,2},{0xF0,O_BEQ,M_REL,2},{0x30,O_BMI,M_REL,2},
    {0xD0,O_BNE,M_REL,2},{0x10,O_BPL,M_REL,2},{0x50,O_BVC,M_REL,2},{0x70,O_BVS,M_REL,2},
    {0x24,O_BIT,M_ZP,3},{0x2C,O_BIT,M_ABS,4},
    {0x00,O_BRK,M_IMP,7},
    {0x18,O_CLC,M_IMP,2},{0xD8,O_CLD,M_IMP,2},{0x58,O_CLI,M_IMP,2},{0xB8,O_CLV,M_IMP,2},
    {0xC9,O_CMP,M_IMM,2},{0xC5,O_CMP,M_ZP,3},{0xD5,O_CMP,M_ZPX,4},{0xCD,O_CMP,M_ABS,4},
    {0xDD,O_CMP,M_ABX,4},{0xD9,O_CMP,M_ABY,4},{0xC1,O_CMP,M_IZX,6},{0xD1,O_CMP,M_IZY,5},
    {0xE0,O_CPX,M_IMM,2},{0xE4,O_CPX,M_ZP,3},{0xEC,O_CPX,M_ABS,4},
    {0xC0,O_CPY,M_IMM,2},{0xC4,O_CPY,M_ZP,3},{0xCC,O_CPY,M_ABS,4},
    {0xC6,O_DEC,M_ZP,5},{0xD6,O_DEC,M_ZPX,6},{0xCE,O_DEC,M_ABS,6},{0xDE,O_DEC,M_ABX,7},
    {0xCA,O_DEX,M_IMP,2},{0x88,O_DEY,M_IMP,2},
    {0x49,O_EOR,M_IMM,2},{0x45,O_EOR,M_ZP,3},{0x55,O_EOR,M_ZPX,4},{0x4D,O_EOR,M_ABS,4},
    {0x5D,O_EOR,M_ABX,4},{0x59,O_EOR,M_ABY,4},{0x41,O_EOR,M_IZX,6},{0x51,O_EOR,M_IZY,5},
    {0xE6,O_INC,M_ZP,5},{0xF6,O_INC,M_ZPX,6},{0xEE,O_INC,M_ABS,6},{0xFE,O_INC,M_ABX,7},
    {0xE8,O_INX,M_IMP,2},{0xC8,O_INY,M_IMP,2},
    {0x4C,O_JMP,M_ABS,3},{0x6C,O_JMP,M_IND,5},
    {0x20,O_JSR,M_ABS,6},
    {0xA9,O_LDA,M_IMM,2},{0xA5,O_LDA,M_ZP,3},{0xB5,O_LDA,M_ZPX,4},{0xAD,O_LDA,M_ABS,4},
    {0xBD,O_LDA,M_ABX,4},{0xB9,O_LDA,M_ABY,4},{0xA1,O_LDA,M_IZX,6},{0xB1,O_LDA,M_IZY,5},
    {0xA2,O_LDX,M_IMM,2},{0xA6,O_LDX,M_ZP,3},{0xB6,O_LDX,M_ZPY,4},{0xAE,O_LDX,M_ABS,4},
    {0xBE,O_LDX,M_ABY,4},
    {0xA0,O_LDY,M_IMM,2},{0xA4,O_LDY,M_ZP,3},{0xB4,O_LDY,M_ZPX,4},{0xAC,O_LDY,M_ABS,4},
    {0xBC,O_LDY,M_ABX,4},
    {0x4A,O_LSR,M_ACC,2},{0x46,O_LSR,M_ZP,5},{0x56,O_LSR,M_ZPX,6},{0x4E,O_LSR,M_ABS,6},
    {0x5E,O_LSR,M_ABX,7},
    {0xEA,O_NOP,M_IMP,2},
    {0x09,O_ORA,M_IMM,2},{0x05,O_ORA,M_ZP,3},{0x15,O_ORA,M_ZPX,4},{0x0D,O_ORA,M_ABS,4},
    {0x1D,O_ORA,M_ABX,4},{0x19,O_ORA,M_ABY,4},{0x01,O_ORA,M_IZX,6},{0x11,O_ORA,M_IZY,5},
    {0x48,O_PHA,M_IMP,3},{0x08,O_PHP,M_IMP,3},{0x68,O_PLA,M_IMP,4},{0x28,O_PLP,M_IMP,4},
    {0x2A,O_ROL,M_ACC,2},{0x26,O_ROL,M_ZP,5},{0x36,O_ROL,M_ZPX,6},{0x2E,O_ROL,M_ABS,6},
    {0x3E,O_ROL,M_ABX,7},
    {0x6A,O_ROR,M_ACC,2},{0x66,O_ROR,M_ZP,5},{0x76,O_ROR,M_ZPX,6},{0x6E,O_ROR,M_ABS,6},
    {0x7E,O_ROR,M_ABX,7},
    {0x40,O_RTI,M_IMP,6},{0x60,O_RTS,M_IMP,6},
    {0xE9,O_SBC,M_IMM,2},{0xE5,O_SBC,M_ZP,3},{0xF5,O_SBC,M_ZPX,4},{0xED,O_SBC,M_ABS,4},
    {0xFD,O_SBC,M_ABX,4},{0xF9,O_SBC,M_ABY,4},{0xE1,O_SBC,M_IZX,6},{0xF1,O_SBC,M_IZY,5},
    {0x38,O_SEC,M_IMP,2},{0xF8,O_SED,M_IMP,2},{0x78,O_SEI,M_IMP,2},
    {0x85,O_STA,M_ZP,3},{0x95,O_STA,M_ZPX,4},{0x8D,O_STA,M_ABS,4},{0x9D,O_STA,M_ABX,5},
    {0x99,O_STA,M_ABY,5},{0x81,O_STA,M_IZX,6},{0x91,O_STA,M_IZY,6},
    {0x86,O_STX,M_ZP,3},{0x96,O_STX,M_ZPY,4},{0x8E,O_STX,M_ABS,4},
    {0x84,O_STY,M_ZP,3},{0x94,O_STY,M_ZPX,4},{0x8C,O_STY,M_ABS,4},
    {0xAA,O_TAX,M_IMP,2},{0xA8,O_TAY,M_IMP,2},{0xBA,O_TSX,M_IMP,2},{0x8A,O_TXA,M_IMP,2},
    {0x9A,O_TXS,M_IMP,2},{0x98,O_TYA,M_IMP,2},
};
/* The stable undocumented opcodes of the NMOS part (opcode, operation, mode,
 * base cycles), per the published descriptions of its undocumented
 * instructions: a read-modify-write of memory followed by an accumulator
 * operation (SLO = ASL + ORA, RLA = ROL + AND, SRE = LSR + EOR, RRA = ROR +
 * ADC, DCP = DEC + CMP, ISC = INC + SBC; always the long cycle count), SAX
 * (store A AND X), LAX (load A and X), ANC (AND, carry = bit 7), ALR (AND
 * then LSR), SBX (X = (A AND X) - operand, flags as CMP), SBC $EB, and the
 * NOPs of one to three bytes (those with a memory operand read it).  The
 * remaining 21 opcodes (12 that halt the part, and ANE, LXA, SHA, SHX, SHY,
 * TAS, LAS, ARR, whose results depend on the chip or, for ARR, on a decimal
 * mode that is not described consistently) stay unmodelled: they halt. */
static const uint8_t UNDOC[84][4] = {
    {0x07,O_SLO,M_ZP,5},{0x17,O_SLO,M_ZPX,6},{0x0F,O_SLO,M_ABS,6},{0x1F,O_SLO,M_ABX,7},
    {0x1B,O_SLO,M_ABY,7},{0x03,O_SLO,M_IZX,8},{0x13,O_SLO,M_IZY,8},
    {0x27,O_RLA,M_ZP,5},{0x37,O_RLA,M_ZPX,6},{0x2F,O_RLA,M_ABS,6},{0x3F,O_RLA,M_ABX,7},
    {0x3B,O_RLA,M_ABY,7},{0x23,O_RLA,M_IZX,8},{0x33,O_RLA,M_IZY,8},
    {0x47,O_SRE,M_ZP,5},{0x57,O_SRE,M_ZPX,6},{0x4F,O_SRE,M_ABS,6},{0x5F,O_SRE,M_ABX,7},
    {0x5B,O_SRE,M_ABY,7},{0x43,O_SRE,M_IZX,8},{0x53,O_SRE,M_IZY,8},
    {0x67,O_RRA,M_ZP,5},{0x77,O_RRA,M_ZPX,6},{0x6F,O_RRA,M_ABS,6},{0x7F,O_RRA,M_ABX,7},
    {0x7B,O_RRA,M_ABY,7},{0x63,O_RRA,M_IZX,8},{0x73,O_RRA,M_IZY,8},
    {0xC7,O_DCP,M_ZP,5},{0xD7,O_DCP,M_ZPX,6},{0xCF,O_DCP,M_ABS,6},{0xDF,O_DCP,M_ABX,7},
    {0xDB,O_DCP,M_ABY,7},{0xC3,O_DCP,M_IZX,8},{0xD3,O_DCP,M_IZY,8},
    {0xE7,O_ISC,M_ZP,5},{0xF7,O_ISC,M_ZPX,6},{0xEF,O_ISC,M_ABS,6},{0xFF,O_ISC,M_ABX,7},
    {0xFB,O_ISC,M_ABY,7},{0xE3,O_ISC,M_IZX,8},{0xF3,O_ISC,M_IZY,8},
    {0x87,O_SAX,M_ZP,3},{0x97,O_SAX,M_ZPY,4},{0x8F,O_SAX,M_ABS,4},{0x83,O_SAX,M_IZX,6},
    {0xA7,O_LAX,M_ZP,3},{0xB7,O_LAX,M_ZPY,4},{0xAF,O_LAX,M_ABS,4},{0xBF,O_LAX,M_ABY,4},
    {0xA3,O_LAX,M_IZX,6},{0xB3,O_LAX,M_IZY,5},
    {0x0B,O_ANC,M_IMM,2},{0x2B,O_ANC,M_IMM,2},{0x4B,O_ALR,M_IMM,2},{0xCB,O_SBX,M_IMM,2},
    {0xEB,O_SBC,M_IMM,2},
    {0x1A,O_NOP,M_IMP,2},{0x3A,O_NOP,M_IMP,2},{0x5A,O_NOP,M_IMP,2},{0x7A,O_NOP,M_IMP,2},
    {0xDA,O_NOP,M_IMP,2},{0xFA,O_NOP,M_IMP,2},
    {0x80,O_NOP,M_IMM,2},{0x82,O_NOP,M_IMM,2},{0x89,O_NOP,M_IMM,2},{0xC2,O_NOP,M_IMM,2},
    {0xE2,O_NOP,M_IMM,2},
    {0x04,O_NOP,M_ZP,3},{0x44,O_NOP,M_ZP,3},{0x64,O_NOP,M_ZP,3},
    {0x14,O_NOP,M_ZPX,4},{0x34,O_NOP,M_ZPX,4},{0x54,O_NOP,M_ZPX,4},{0x74,O_NOP,M_ZPX,4},
    {0xD4,O_NOP,M_ZPX,4},{0xF4,O_NOP,M_ZPX,4},
    {0x0C,O_NOP,M_ABS,4},
    {0x1C,O_NOP,M_ABX,4},{0x3C,O_NOP,M_ABX,4},{0x5C,O_NOP,M_ABX,4},{0x7C,O_NOP,M_ABX,4},
    {0xDC,O_NOP,M_ABX,4},{0xFC,O_NOP,M_ABX,4},
};
static opinfo OPS[256];
static pthread_once_t ops_once = PTHREAD_ONCE_INIT;
static void build_ops(void) {
    memset(OPS, 0, sizeof OPS);
    for (int i = 0; i < 151; i++) {
        OPS[DOC[i][0]].op = DOC[i][1];
        OPS[DOC[i][0]].mode = DOC[i][2];
        OPS[DOC[i][0]].cycles = DOC[i][3];
    }
    for (int i = 0; i < 84; i++) {
        OPS[UNDOC[i][0]].op = UNDOC[i][1];
        OPS[UNDOC[i][0]].mode = UNDOC[i][2];
        OPS[UNDOC[i][0]].cycles = UNDOC[i][3];
    }
}
int orc_base_cycles(uint8_t opcode) {
    pthread_once(&ops_once, build_ops);
    return OPS[opcode].cycles;
}

/* ---- flags ---- */
#define F_C 0x01
#define F_Z 0x02
#define F_I 0x04
#define F_D 0x08
#define F_B 0x10
#define F_U 0x20
#define F_V 0x40
#define F_N 0x80

static uint8_t set_nz(uint8_t p, uint8_t v) {
    p &= (uint8_t)~(F_N | F_Z);
    if (v == 0) p |= F_Z;
    if (v & 0x80) p |= F_N;
    return p;
}

/* ADC: binary per the two's-complement definition; decimal per Clark's NMOS
 * description (A and C from nibble adjustment; N, V from the intermediate;
 * Z from the binary sum). */
uint32_t orc_alu_adc(uint8_t a, uint8_t b, uint8_t p) {
    unsigned c = p & F_C;
    unsigned bin = (unsigned)a + b + c;
    uint8_t np = p & (uint8_t)~(F_N | F_V | F_Z | F_C);
    if ((bin & 0xFF) == 0) np |= F_Z;
    if (!(p & F_D)) {
        uint8_t r = (uint8_t)bin;
        if (bin > 0xFF) np |= F_C;
        if (~(a ^ b) & (a ^ r) & 0x80) np |= F_V;
        if (r & 0x80) np |= F_N;
        return r | ((uint32_t)np << 8);
    }
    int al = (a & 0x0F) + (b & 0x0F) + (int)c;
    if (al >= 0x0A) al = ((al + 0x06) & 0x0F) + 0x10;
    int s = (a & 0xF0) + (b & 0xF0) + al;                       /* unsigned intermediate */
    int ss = (int)(int8_t)(a & 0xF0) + (int)(int8_t)(b & 0xF0) + al; /* signed intermediate */
    if (ss & 0x80) np |= F_N;
    if (ss < -128 || ss > 127) np |= F_V;
    if (s >= 0xA0) s += 0x60;
    if (s >= 0x100) np |= F_C;
    return (uint8_t)s | ((uint32_t)np << 8);
}

/* SBC: binary is ADC of the complement; decimal per Clark's NMOS description
 * (accumulator by nibble adjustment, every flag from the binary operation). */
uint32_t orc_alu_sbc(uint8_t a, uint8_t b, uint8_t p) {
    uint32_t binres = orc_alu_adc(a, (uint8_t)~b, (uint8_t)(p & ~F_D));
    if (!(p & F_D)) return binres;
    uint8_t np = (uint8_t)((binres >> 8) | F_D);
    int c = p & F_C;
    int al = (a & 0x0F) - (b & 0x0F) + c - 1;
    if (al < 0) al = ((al - 0x06) & 0x0F) - 0x10;
    int s = (a & 0xF0) - (b & 0xF0) + al;
    if (s < 0) s -= 0x60;
    return (uint8_t)s | ((uint32_t)np << 8);
}

/* ---- TIA: per-pixel object evaluation ---- */
static int pf_on(const orc_machine *m, unsigned col) {
    unsigned b = (col < 80) ? col / 4 : (col - 80) / 4;      /* 0..19 within a half */
    if (col >= 80 && (m->ctrlpf & 1)) b = 19 - b;            /* mirrored right half */
    if (b < 4) return (m->pf0 >> (4 + b)) & 1;
    if (b < 12) return (m->pf1 >> (7 - (b - 4))) & 1;
    return (m->pf2 >> (b - 12)) & 1;
}

static const uint8_t COPY_MASK[8] = {1, 3, 5, 7, 9, 1, 13, 1}; /* bit j: copy at 16*j, j = 0, 1, 2, 4 */
static int copy_offsets(uint8_t nus, int *offs) {
    int n = 0;
    unsigned mask = COPY_MASK[nus & 7];
    if (mask & 1) offs[n++] = 0;
    if (mask & 2) offs[n++] = 16;
    if (mask & 4) offs[n++] = 32;
    if (mask & 8) offs[n++] = 64;
    return n;
}

static int player_on(const orc_machine *m, int i, unsigned col) {
    uint8_t g = m->vdelp[i] & 1 ? m->grp_old[i] : m->grp_new[i];
    if (!g) return 0;
    int scale = (m->nusiz[i] & 7) == 5 ? 2 : (m->nusiz[i] & 7) == 7 ? 4 : 1;
    unsigned d = (col + 160 - m->pos[i]) % 160;
    int offs[4];
    int n = copy_offsets(m->nusiz[i], offs);
    for (int c = 0; c < n; c++) {
        int e = (int)d - offs[c];
        if (e >= 0 && e < 8 * scale) {
            int bit = e / scale;                               /* 0 = leftmost */
            int sh = (m->refp[i] & 8) ? bit : 7 - bit;
            if ((g >> sh) & 1) return 1;
        }
    }
    return 0;
}

static int missile_on(const orc_machine *m, int i, unsigned col) {
    if (!(m->enam[i] & 2) || (m->resmp[i] & 2)) return 0;
    int w = 1 << ((m->nusiz[i] >> 4) & 3);
    unsigned d = (col + 160 - m->pos[2 + i]) % 160;
    int offs[4];
    int n = copy_offsets(m->nusiz[i], offs);
    for (int c = 0; c < n; c++) {
        int e = (int)d - offs[c];
        if (e >= 0 && e < w) return 1;
    }
    return 0;
}

static int ball_on(const orc_machine *m, unsigned col) {
    uint8_t en = (m->vdelbl & 1) ? m->enabl_old : m->enabl_new;
    if (!(en & 2)) return 0;
    int w = 1 << ((m->ctrlpf >> 4) & 3);
    unsigned d = (col + 160 - m->pos[4]) % 160;
    return (int)d < w;
}

static unsigned objects_at(const orc_machine *m, unsigned col) {
    unsigned o = 0;
    if (player_on(m, 0, col)) o |= OBJ_P0;
    if (player_on(m, 1, col)) o |= OBJ_P1;
    if (missile_on(m, 0, col)) o |= OBJ_M0;
    if (missile_on(m, 1, col)) o |= OBJ_M1;
    if (ball_on(m, col)) o |= OBJ_BL;
    if (pf_on(m, col)) o |= OBJ_PF;
    return o;
}

/* 15 collision latches: bit 2r+1 = D7 and bit 2r = D6 of read register r. */
static uint16_t collisions_of(unsigned o) {
#define BOTH(a, b) (((o & (a)) && (o & (b))) ? 1u : 0u)
    uint16_t c = 0;
    c |= (uint16_t)(BOTH(OBJ_M0, OBJ_P1) << 1 | BOTH(OBJ_M0, OBJ_P0) << 0);
    c |= (uint16_t)(BOTH(OBJ_M1, OBJ_P0) << 3 | BOTH(OBJ_M1, OBJ_P1) << 2);
    c |= (uint16_t)(BOTH(OBJ_P0, OBJ_PF) << 5 | BOTH(OBJ_P0, OBJ_BL) << 4);
    c |= (uint16_t)(BOTH(OBJ_P1, OBJ_PF) << 7 | BOTH(OBJ_P1, OBJ_BL) << 6);
    c |= (uint16_t)(BOTH(OBJ_M0, OBJ_PF) << 9 | BOTH(OBJ_M0, OBJ_BL) << 8);
    c |= (uint16_t)(BOTH(OBJ_M1, OBJ_PF) << 11 | BOTH(OBJ_M1, OBJ_BL) << 10);
    c |= (uint16_t)(BOTH(OBJ_BL, OBJ_PF) << 13);
    c |= (uint16_t)(BOTH(OBJ_P0, OBJ_P1) << 15 | BOTH(OBJ_M0, OBJ_M1) << 14);
#undef BOTH
    return c;
}

static uint8_t color_of(const orc_machine *m, unsigned o, unsigned col) {
    int p0 = (o & (OBJ_P0 | OBJ_M0)) != 0;
    int p1 = (o & (OBJ_P1 | OBJ_M1)) != 0;
    int pf = (o & OBJ_PF) != 0, bl = (o & OBJ_BL) != 0;
    uint8_t c;
    if (m->ctrlpf & 4) {                     /* playfield priority; score mode ignored */
        if (pf || bl) c = m->colupf;
        else if (p0) c = m->colup[0];
        else if (p1) c = m->colup[1];
        else c = m->colubk;
    } else {
        if (p0) c = m->colup[0];
        else if (p1) c = m->colup[1];
        else if (pf) c = (m->ctrlpf & 2) ? m->colup[col < 80 ? 0 : 1] : m->colupf;
        else if (bl) c = m->colupf;
        else c = m->colubk;
    }
    return c & 0xFE;
}

/* Evaluate every color clock in [tia_clock, upto). */
static void tia_advance(orc_machine *m, uint64_t upto) {
    for (uint64_t c = m->tia_clock; c < upto; c++) {
        uint64_t line = c / LINE_CLOCKS;
        unsigned x = (unsigned)(c % LINE_CLOCKS);
        if (x < 68) continue;                          /* horizontal blank */
        unsigned col = x - 68;
        uint8_t px = 0;
        int blank = (m->vblank & 2) || (line == m->bar_line && col < 8);
        if (!blank) {
            unsigned o = objects_at(m, col);
            m->cx |= collisions_of(o);
            px = color_of(m, o, col);
        }
        if (m->fb && line >= m->frame_line + WINDOW_Y0 && line < m->frame_line + WINDOW_Y0 + ORC_FRAME_H)
            m->fb[(line - m->frame_line - WINDOW_Y0) * ORC_FRAME_W + col] = px;
    }
    if (upto > m->tia_clock) m->tia_clock = upto;
}

static uint8_t reset_pos(uint64_t effect_clock, int is_player) {
    unsigned x = (unsigned)(effect_clock % LINE_CLOCKS);
    if (x < 68) return is_player ? 3 : 2;
    return (uint8_t)((x - 68 + (is_player ? 5 : 4)) % 160);
}

static void tia_write(orc_machine *m, unsigned reg, uint8_t v, uint64_t t) {
    uint64_t eff = 3 * (t + 1);
    tia_advance(m, eff);
    m->tia_writes++;
    switch (reg) {
    case 0x00:
        if (!(m->vsync & 2) && (v & 2)) { m->vs_rise = 1; m->vs_rise_t = t; }
        m->vsync = v; break;
    case 0x01:
        m->vblank = v;
        if (!(v & 0x40)) m->inpt4_latch = 0;
        else if (m->fire) m->inpt4_latch = 1;
        break;
    case 0x02: m->wsync = 1; break;
    case 0x03: break;                                  /* RSYNC: not modelled */
    case 0x04: m->nusiz[0] = v; break;
    case 0x05: m->nusiz[1] = v; break;
    case 0x06: m->colup[0] = v; break;
    case 0x07: m->colup[1] = v; break;
    case 0x08: m->colupf = v; break;
    case 0x09: m->colubk = v; break;
    case 0x0A: m->ctrlpf = v; break;
    case 0x0B: m->refp[0] = v; break;
    case 0x0C: m->refp[1] = v; break;
    case 0x0D: m->pf0 = v; break;
    case 0x0E: m->pf1 = v; break;
    case 0x0F: m->pf2 = v; break;
    case 0x10: m->pos[0] = reset_pos(eff, 1); break;
    case 0x11: m->pos[1] = reset_pos(eff, 1); break;
    case 0x12: m->pos[2] = reset_pos(eff, 0); break;
    case 0x13: m->pos[3] = reset_pos(eff, 0); break;
    case 0x14: m->pos[4] = reset_pos(eff, 0); break;
    case 0x1B: m->grp_new[0] = v; m->grp_old[1] = m->grp_new[1]; break;
    case 0x1C: m->grp_new[1] = v; m->grp_old[0] = m->grp_new[0]; m->enabl_old = m->enabl_new; break;
    case 0x1D: m->enam[0] = v; break;
    case 0x1E: m->enam[1] = v; break;
    case 0x1F: m->enabl_new = v; break;
    case 0x20: case 0x21: case 0x22: case 0x23: case 0x24: m->hm[reg - 0x20] = v; break;
    case 0x25: m->vdelp[0] = v; break;
    case 0x26: m->vdelp[1] = v; break;
    case 0x27: m->vdelbl = v; break;
    case 0x28: case 0x29: {
        int i = reg - 0x28;
        if ((m->resmp[i] & 2) && !(v & 2)) {
            int scale = (m->nusiz[i] & 7) == 5 ? 2 : (m->nusiz[i] & 7) == 7 ? 4 : 1;
            m->pos[2 + i] = (uint8_t)((m->pos[i] + 4 * scale) % 160);
        }
        m->resmp[i] = v;
        break;
    }
    case 0x2A:
        for (int i = 0; i < 5; i++) {
            int s = (m->hm[i] >> 4) & 0xF;
            if (s >= 8) s -= 16;
            m->pos[i] = (uint8_t)(((int)m->pos[i] - s + 160) % 160);
        }
        if (eff % LINE_CLOCKS < 68) m->bar_line = eff / LINE_CLOCKS;
        break;
    case 0x2B: memset(m->hm, 0, sizeof m->hm); break;
    case 0x2C: m->cx = 0; break;
    default: break;                                    /* audio, 0x2D-0x3F */
    }
}

static uint8_t tia_read(orc_machine *m, unsigned reg, uint64_t t) {
    if (reg < 8) {
        tia_advance(m, 3 * t);
        return (uint8_t)((((m->cx >> (2 * reg + 1)) & 1) << 7) | (((m->cx >> (2 * reg)) & 1) << 6));
    }
    if (reg == 0x0C) return (m->fire || m->inpt4_latch) ? 0x00 : 0x80;
    if (reg == 0x0D) return 0x80;
    return 0x00;
}

/* ---- RIOT ---- */
static uint8_t riot_read(orc_machine *m, uint16_t addr, uint64_t t) {
    if (!(addr & 0x04)) {
        switch (addr & 3) {
        case 0: return (uint8_t)((m->swcha_out & m->swacnt) | (m->joy & ~m->swacnt));
        case 1: return m->swacnt;
        case 2: return (uint8_t)((m->swchb_out & m->swbcnt) | (0x0B & ~m->swbcnt));
        default: return m->swbcnt;
        }
    }
    uint64_t n = t - (m->tim_cw + 1);
    uint64_t span = ((uint64_t)m->tim_v + 1) << m->tim_shift;
    if (addr & 1) return n >= span ? 0x80 : 0x00;      /* TIMINT */
    if (n < span) return (uint8_t)(m->tim_v - (n >> m->tim_shift));
    return (uint8_t)((0xFF - (n - span)) & 0xFF);
}

static void riot_write(orc_machine *m, uint16_t addr, uint8_t v, uint64_t t) {
    if (!(addr & 0x04)) {
        switch (addr & 3) {
        case 0: m->swcha_out = v; break;
        case 1: m->swacnt = v; break;
        case 2: m->swchb_out = v; break;
        default: m->swbcnt = v; break;
        }
        return;
    }
    if (addr & 0x10) {
        static const uint8_t SH[4] = {0, 3, 6, 10};
        m->tim_v = v;
        m->tim_shift = SH[addr & 3];
        m->tim_cw = t;
    }
}

/* ---- cartridge ---- */
static void cart_hotspot(orc_machine *m, uint16_t off) {
    if (m->scheme == 1 && (off == 0xFF8 || off == 0xFF9)) m->bank = (uint8_t)(off - 0xFF8);
    if (m->scheme == 2 && off >= 0xFF6 && off <= 0xFF9) m->bank = (uint8_t)(off - 0xFF6);
    if (m->scheme == 3 && off >= 0xFF4 && off <= 0xFFB) m->bank = (uint8_t)(off - 0xFF4);
}
static uint8_t cart_byte(const orc_machine *m, uint16_t off) {
    if (m->rom_size == 2048) return m->rom[off & 0x7FF];
    return m->rom[(uint32_t)m->bank * 4096u + off];
}

/* ---- bus (13-bit address) ---- */
static uint8_t bus_read(orc_machine *m, uint16_t addr, uint64_t t) {
    addr &= 0x1FFF;
    if (addr & 0x1000) { cart_hotspot(m, addr & 0xFFF); return cart_byte(m, addr & 0xFFF); }
    if (!(addr & 0x80)) return tia_read(m, addr & 0x0F, t);
    if (!(addr & 0x200)) return m->ram[addr & 0x7F];
    return riot_read(m, addr, t);
}
static void bus_write(orc_machine *m, uint16_t addr, uint8_t v, uint64_t t) {
    addr &= 0x1FFF;
    if (addr & 0x1000) { cart_hotspot(m, addr & 0xFFF); return; }
    if (!(addr & 0x80)) { tia_write(m, addr & 0x3F, v, t); return; }
    if (!(addr & 0x200)) { m->ram[addr & 0x7F] = v; return; }
    riot_write(m, addr, v, t);
}

static void push(orc_machine *m, uint8_t v, uint64_t t) { bus_write(m, (uint16_t)(0x100 | m->sp), v, t); m->sp--; }
static uint8_t pull(orc_machine *m, uint64_t t) { m->sp++; return bus_read(m, (uint16_t)(0x100 | m->sp), t); }

static uint8_t compare(uint8_t p, uint8_t r, uint8_t v) {
    p = set_nz(p, (uint8_t)(r - v));
    if (r >= v) p |= F_C; else p &= (uint8_t)~F_C;
    return p;
}

static int is_read_op(int op) {
    switch (op) {
    case O_LDA: case O_LDX: case O_LDY: case O_ADC: case O_SBC: case O_AND: case O_ORA:
    case O_EOR: case O_CMP: case O_CPX: case O_CPY: case O_BIT: case O_LAX: case O_NOP: return 1;
    default: return 0;
    }
}

/* Execute one instruction.  Returns the cycles it took, or -1 when jammed. */
static int cpu_exec(orc_machine *m) {
    if (m->jam) return -1;
    uint64_t k0 = m->k;
    m->wsync = 0;
    m->vs_rise = 0;
    uint16_t pc = m->pc;
    uint8_t opc = bus_read(m, pc, k0);
    opinfo oi = OPS[opc];
    if (!oi.cycles) { m->jam = 1; m->status |= ORC_ST_ILLEGAL; return -1; }
    int len = MODE_LEN[oi.mode];
    uint8_t b1 = len >= 2 ? bus_read(m, (uint16_t)(pc + 1), k0) : 0;
    uint8_t b2 = len >= 3 ? bus_read(m, (uint16_t)(pc + 2), k0) : 0;
    m->pc = (uint16_t)(pc + len);
    int n = oi.cycles;
    uint16_t ea = 0;
    int cross = 0;
    switch (oi.mode) {
    case M_ZP: ea = b1; break;
    case M_ZPX: ea = (uint8_t)(b1 + m->x); break;
    case M_ZPY: ea = (uint8_t)(b1 + m->y); break;
    case M_ABS: ea = (uint16_t)(b1 | b2 << 8); break;
    case M_ABX: { uint16_t b = (uint16_t)(b1 | b2 << 8); ea = (uint16_t)(b + m->x); cross = (b ^ ea) >> 8 != 0; break; }
    case M_ABY: { uint16_t b = (uint16_t)(b1 | b2 << 8); ea = (uint16_t)(b + m->y); cross = (b ^ ea) >> 8 != 0; break; }
    case M_IZX: {
        uint8_t zp = (uint8_t)(b1 + m->x);
        ea = (uint16_t)(bus_read(m, zp, k0) | bus_read(m, (uint8_t)(zp + 1), k0) << 8);
        break;
    }
    case M_IZY: {
        uint16_t b = (uint16_t)(bus_read(m, b1, k0) | bus_read(m, (uint8_t)(b1 + 1), k0) << 8);
        ea = (uint16_t)(b + m->y);
        cross = (b ^ ea) >> 8 != 0;
        break;
    }
    case M_IND: {
        uint16_t ptr = (uint16_t)(b1 | b2 << 8);
        uint16_t hi = (uint16_t)((ptr & 0xFF00) | ((ptr + 1) & 0x00FF)); /* page-wrap bug */
        ea = (uint16_t)(bus_read(m, ptr, k0) | bus_read(m, hi, k0) << 8);
        break;
    }
    case M_REL: ea = (uint16_t)(m->pc + (int8_t)b1); break;
    default: break;
    }
    if (cross && is_read_op(oi.op)) n++;

    /* branches: cycle count depends on the outcome; no data access */
    int take = -1;
    switch (oi.op) {
    case O_BCC: take = !(m->p & F_C); break;
    case O_BCS: take = !!(m->p & F_C); break;
    case O_BEQ: take = !!(m->p & F_Z); break;
    case O_BNE: take = !(m->p & F_Z); break;
    case O_BMI: take = !!(m->p & F_N); break;
    case O_BPL: take = !(m->p & F_N); break;
    case O_BVC: take = !(m->p & F_V); break;
    case O_BVS: take = !!(m->p & F_V); break;
    default: break;
    }
    if (take >= 0) {
        if (take) {
            n += 1;
            if ((m->pc ^ ea) & 0xFF00) n += 1;
            m->pc = ea;
        }
        m->k = k0 + (uint64_t)n;
        m->instret++;
        return n;
    }

    uint64_t kA = k0 + (uint64_t)n - 1;
    uint8_t v;
    switch (oi.op) {
    case O_LDA: m->a = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->p = set_nz(m->p, m->a); break;
    case O_LDX: m->x = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->p = set_nz(m->p, m->x); break;
    case O_LDY: m->y = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->p = set_nz(m->p, m->y); break;
    case O_STA: bus_write(m, ea, m->a, kA); break;
    case O_STX: bus_write(m, ea, m->x, kA); break;
    case O_STY: bus_write(m, ea, m->y, kA); break;
    case O_ADC: case O_SBC: {
        v = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA);
        uint32_t r = oi.op == O_ADC ? orc_alu_adc(m->a, v, m->p) : orc_alu_sbc(m->a, v, m->p);
        m->a = (uint8_t)r;
        m->p = (uint8_t)((r >> 8) | F_U);
        break;
    }
    case O_AND: v = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->a &= v; m->p = set_nz(m->p, m->a); break;
    case O_ORA: v = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->a |= v; m->p = set_nz(m->p, m->a); break;
    case O_EOR: v = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->a ^= v; m->p = set_nz(m->p, m->a); break;
    case O_CMP: v = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->p = compare(m->p, m->a, v); break;
    case O_CPX: v = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->p = compare(m->p, m->x, v); break;
    case O_CPY: v = oi.mode == M_IMM ? b1 : bus_read(m, ea, kA); m->p = compare(m->p, m->y, v); break;
    case O_BIT:
        v = bus_read(m, ea, kA);
        m->p &= (uint8_t)~(F_N | F_V | F_Z);
        m->p |= v & (F_N | F_V);
        if (!(m->a & v)) m->p |= F_Z;
        break;
    case O_ASL: case O_LSR: case O_ROL: case O_ROR: case O_INC: case O_DEC: {
        int acc = oi.mode == M_ACC;
        uint8_t old = acc ? m->a : bus_read(m, ea, kA - 2);
        uint8_t r;
        uint8_t c = m->p & F_C;
        switch (oi.op) {
        case O_ASL: r = (uint8_t)(old << 1); c = old >> 7; break;
        case O_LSR: r = old >> 1; c = old & 1; break;
        case O_ROL: r = (uint8_t)(old << 1 | (m->p & F_C)); c = old >> 7; break;
        case O_ROR: r = (uint8_t)(old >> 1 | (m->p & F_C) << 7); c = old & 1; break;
        case O_INC: r = (uint8_t)(old + 1); break;
        default: r = (uint8_t)(old - 1); break;
        }
        if (oi.op != O_INC && oi.op != O_DEC) m->p = (uint8_t)((m->p & ~F_C) | c);
        m->p = set_nz(m->p, r);
        if (acc) m->a = r;
        else { bus_write(m, ea, old, kA - 1); bus_write(m, ea, r, kA); }
        break;
    }
    case O_SLO: case O_RLA: case O_SRE: case O_RRA: case O_DCP: case O_ISC: {
        /* read-modify-write of memory (old value written back first, as the
         * documented RMW instructions do), then the accumulator operation */
        uint8_t old = bus_read(m, ea, kA - 2), r;
        uint8_t c = m->p & F_C;
        switch (oi.op) {
        case O_SLO: r = (uint8_t)(old << 1); c = old >> 7; break;
        case O_RLA: r = (uint8_t)(old << 1 | (m->p & F_C)); c = old >> 7; break;
        case O_SRE: r = old >> 1; c = old & 1; break;
        case O_RRA: r = (uint8_t)(old >> 1 | (m->p & F_C) << 7); c = old & 1; break;
        case O_DCP: r = (uint8_t)(old - 1); break;
        default: r = (uint8_t)(old + 1); break;
        }
        bus_write(m, ea, old, kA - 1);
        bus_write(m, ea, r, kA);
        switch (oi.op) {
        case O_SLO: m->a |= r; m->p = set_nz((uint8_t)((m->p & ~F_C) | c), m->a); break;
        case O_RLA: m->a &= r; m->p = set_nz((uint8_t)((m->p & ~F_C) | c), m->a); break;
        case O_SRE: m->a ^= r; m->p = set_nz((uint8_t)((m->p & ~F_C) | c), m->a); break;
        case O_RRA: {
            uint32_t s2 = orc_alu_adc(m->a, r, (uint8_t)((m->p & ~F_C) | c));
            m->a = (uint8_t)s2;
            m->p = (uint8_t)((s2 >> 8) | F_U);
            break;
        }
        case O_DCP: m->p = compare(m->p, m->a, r); break;
        default: {
            uint32_t s2 = orc_alu_sbc(m->a, r, m->p);
            m->a = (uint8_t)s2;
            m->p = (uint8_t)((s2 >> 8) | F_U);
            break;
        }
        }
        break;
    }
    case O_SAX: bus_write(m, ea, m->a & m->x, kA); break;
    case O_LAX: m->a = m->x = bus_read(m, ea, kA); m->p = set_nz(m->p, m->a); break;
    case O_ANC: m->a &= b1; m->p = set_nz(m->p, m->a); m->p = (uint8_t)((m->p & ~F_C) | (m->a >> 7)); break;
    case O_ALR:
        m->a &= b1;
        m->p = (uint8_t)((m->p & ~F_C) | (m->a & 1));
        m->a >>= 1;
        m->p = set_nz(m->p, m->a);
        break;
    case O_SBX: {
        uint8_t ax = m->a & m->x;
        m->p = (uint8_t)((m->p & ~F_C) | (ax >= b1 ? F_C : 0));
        m->x = (uint8_t)(ax - b1);
        m->p = set_nz(m->p, m->x);
        break;
    }
    case O_NOP:
        if (oi.mode != M_IMP && oi.mode != M_IMM) (void)bus_read(m, ea, kA);  /* the operand read */
        break;
    case O_INX: m->x++; m->p = set_nz(m->p, m->x); break;
    case O_INY: m->y++; m->p = set_nz(m->p, m->y); break;
    case O_DEX: m->x--; m->p = set_nz(m->p, m->x); break;
    case O_DEY: m->y--; m->p = set_nz(m->p, m->y); break;
    case O_TAX: m->x = m->a; m->p = set_nz(m->p, m->x); break;
    case O_TAY: m->y = m->a; m->p = set_nz(m->p, m->y); break;
    case O_TXA: m->a = m->x; m->p = set_nz(m->p, m->a); break;
    case O_TYA: m->a = m->y; m->p = set_nz(m->p, m->a); break;
    case O_TSX: m->x = m->sp; m->p = set_nz(m->p, m->x); break;
    case O_TXS: m->sp = m->x; break;
    case O_CLC: m->p &= (uint8_t)~F_C; break;
    case O_SEC: m->p |= F_C; break;
    case O_CLI: m->p &= (uint8_t)~F_I; break;
    case O_SEI: m->p |= F_I; break;
    case O_CLV: m->p &= (uint8_t)~F_V; break;
    case O_CLD: m->p &= (uint8_t)~F_D; break;
    case O_SED: m->p |= F_D; break;
    case O_PHA: push(m, m->a, kA); break;
    case O_PHP: push(m, m->p | F_B | F_U, kA); break;
    case O_PLA: m->a = pull(m, kA); m->p = set_nz(m->p, m->a); break;
    case O_PLP: m->p = (uint8_t)((pull(m, kA) & ~F_B) | F_U); break;
    case O_JMP: m->pc = ea; break;
    case O_JSR: {
        uint16_t ret = (uint16_t)(pc + 2);
        push(m, (uint8_t)(ret >> 8), kA);
        push(m, (uint8_t)ret, kA);
        m->pc = ea;
        break;
    }
    case O_RTS: {
        uint8_t lo = pull(m, kA), hi = pull(m, kA);
        m->pc = (uint16_t)((lo | hi << 8) + 1);
        break;
    }
    case O_RTI: {
        m->p = (uint8_t)((pull(m, kA) & ~F_B) | F_U);
        uint8_t lo = pull(m, kA), hi = pull(m, kA);
        m->pc = (uint16_t)(lo | hi << 8);
        break;
    }
    case O_BRK: {
        uint16_t ret = (uint16_t)(pc + 2);
        push(m, (uint8_t)(ret >> 8), kA);
        push(m, (uint8_t)ret, kA);
        push(m, m->p | F_B | F_U, kA);
        m->p |= F_I;
        m->pc = (uint16_t)(bus_read(m, 0x1FFE, kA) | bus_read(m, 0x1FFF, kA) << 8);
        break;
    }
    default: break;
    }
    m->k = k0 + (uint64_t)n;
    if (m->wsync) m->k = ((m->k + LINE_CYCLES - 1) / LINE_CYCLES) * LINE_CYCLES;
    m->instret++;
    return (int)(m->k - k0);
}

static void power_on(orc_machine *m) {
    const uint8_t *rom = m->rom;
    uint32_t sz = m->rom_size;
    int scheme = m->scheme;
    memset(m, 0, sizeof *m);
    m->rom = rom;
    m->rom_size = sz;
    m->scheme = scheme;
    m->sp = 0xFD;
    m->p = 0x24;
    m->tim_shift = 10;
    m->bar_line = NO_LINE;
    m->joy = 0xFF;
    m->pc = (uint16_t)(cart_byte(m, 0xFFC) | cart_byte(m, 0xFFD) << 8);
}

static int scheme_of(size_t size) {
    if (size == 2048 || size == 4096) return 0;
    if (size == 8192) return 1;
    if (size == 16384) return 2;
    if (size == 32768) return 3;
    return -1;
}

orc_machine *orc_machine_new(const uint8_t *rom, size_t rom_size) {
    int sc = scheme_of(rom_size);
    if (sc < 0) return NULL;
    pthread_once(&ops_once, build_ops);
    orc_machine *m = (orc_machine *)calloc(1, sizeof *m);
    m->rom = rom;
    m->rom_size = (uint32_t)rom_size;
    m->scheme = sc;
    power_on(m);
    return m;
}
void orc_machine_free(orc_machine *m) { free(m); }
int orc_machine_step(orc_machine *m) {
    int n = cpu_exec(m);
    if (m->vs_rise) { m->last_vsync_t = m->vs_rise_t; m->have_vsync = 1; }
    return n;
}

/* Map one of the 18 ALE actions onto the joystick pins and fire button. */
static void apply_action(orc_machine *m, int a) {
    static const uint8_t DIRS[18] = {      /* bit0 up, bit1 right, bit2 left, bit3 down */
        0, 0, 1, 2, 4, 8, 3, 5, 10, 12, 1, 2, 4, 8, 3, 5, 10, 12};
    uint8_t d = DIRS[a];
    uint8_t joy = 0xFF;
    if (d & 2) joy &= (uint8_t)~0x80;
    if (d & 4) joy &= (uint8_t)~0x40;
    if (d & 8) joy &= (uint8_t)~0x20;
    if (d & 1) joy &= (uint8_t)~0x10;
    m->joy = joy;
    m->fire = (a == 1 || a >= 10);
    if (m->fire && (m->vblank & 0x40)) m->inpt4_latch = 1;
}
void orc_machine_set_action(orc_machine *m, int action) { apply_action(m, action); }

/* Run one frame (R1).  fb, if given, receives the 210x160 window (R2). */
static int run_frame(orc_machine *m, uint8_t *fb) {
    uint64_t L0 = m->frame_line, next;
    m->fb = fb;
    if (fb) memset(fb, 0, ORC_FRAME_H * ORC_FRAME_W);
    for (;;) {
        if (m->jam) { next = m->k / LINE_CYCLES; break; }
        cpu_exec(m);
        if (m->jam) { next = m->k / LINE_CYCLES; break; }
        if (m->vs_rise) {
            m->last_vsync_t = m->vs_rise_t;
            m->have_vsync = 1;
            next = m->vs_rise_t / LINE_CYCLES;
            break;
        }
        if (m->k >= (L0 + FRAME_CAP_LINES) * LINE_CYCLES) {
            m->status |= ORC_ST_FRAME_CAP;
            next = m->k / LINE_CYCLES;
            break;
        }
    }
    tia_advance(m, 3 * m->k);
    if (fb) {
        for (int r = 0; r < ORC_FRAME_H; r++)
            if (L0 + WINDOW_Y0 + (uint64_t)r >= next) memset(fb + r * ORC_FRAME_W, 0, ORC_FRAME_W);
    }
    m->fb = NULL;
    m->frame_line = next;
    m->frame_no++;
    return (int)(next - L0);
}
int orc_machine_run_frame(orc_machine *m, uint8_t *fb) { return run_frame(m, fb); }
uint64_t orc_machine_cycles(const orc_machine *m) { return m->k; }
int orc_machine_last_vsync(const orc_machine *m, uint64_t *cycle) { *cycle = m->last_vsync_t; return m->have_vsync; }
uint32_t orc_machine_tia_writes(const orc_machine *m) { return m->tia_writes; }
uint8_t orc_machine_peek(orc_machine *m, uint16_t addr) {
    addr &= 0x1FFF;
    if (addr & 0x1000) return cart_byte(m, addr & 0xFFF);
    if ((addr & 0x280) == 0x080) return m->ram[addr & 0x7F];
    return 0;
}

/* ---- canonical 256-byte state ---- */
static void put16(uint8_t *o, uint16_t v) { o[0] = (uint8_t)v; o[1] = (uint8_t)(v >> 8); }
static void put32(uint8_t *o, uint32_t v) { for (int i = 0; i < 4; i++) o[i] = (uint8_t)(v >> (8 * i)); }
static void put64(uint8_t *o, uint64_t v) { for (int i = 0; i < 8; i++) o[i] = (uint8_t)(v >> (8 * i)); }
static uint16_t get16(const uint8_t *o) { return (uint16_t)(o[0] | o[1] << 8); }
static uint32_t get32(const uint8_t *o) { return (uint32_t)o[0] | (uint32_t)o[1] << 8 | (uint32_t)o[2] << 16 | (uint32_t)o[3] << 24; }
static uint64_t get64(const uint8_t *o) { uint64_t v = 0; for (int i = 7; i >= 0; i--) v = v << 8 | o[i]; return v; }

static void pack_machine(const orc_machine *m, uint8_t *o) {
    o[0x00] = m->a; o[0x01] = m->x; o[0x02] = m->y; o[0x03] = m->sp; o[0x04] = m->p;
    o[0x05] = m->bank; put16(o + 0x06, m->pc);
    put64(o + 0x08, m->k);
    put64(o + 0x10, m->tim_cw);
    o[0x18] = m->tim_v; o[0x19] = m->tim_shift; o[0x1A] = m->swcha_out; o[0x1B] = m->swacnt;
    o[0x1C] = m->swchb_out; o[0x1D] = m->swbcnt; o[0x1E] = m->jam; o[0x1F] = m->inpt4_latch;
    o[0x20] = m->vsync; o[0x21] = m->vblank; o[0x22] = m->nusiz[0]; o[0x23] = m->nusiz[1];
    o[0x24] = m->colup[0]; o[0x25] = m->colup[1]; o[0x26] = m->colupf; o[0x27] = m->colubk;
    o[0x28] = m->ctrlpf; o[0x29] = m->refp[0]; o[0x2A] = m->refp[1]; o[0x2B] = m->pf0;
    o[0x2C] = m->pf1; o[0x2D] = m->pf2; o[0x2E] = m->enam[0]; o[0x2F] = m->enam[1];
    o[0x30] = m->enabl_new; o[0x31] = m->enabl_old; o[0x32] = m->grp_new[0]; o[0x33] = m->grp_old[0];
    o[0x34] = m->grp_new[1]; o[0x35] = m->grp_old[1]; o[0x36] = m->vdelp[0]; o[0x37] = m->vdelp[1];
    o[0x38] = m->vdelbl; o[0x39] = m->resmp[0]; o[0x3A] = m->resmp[1];
    for (int i = 0; i < 5; i++) { o[0x3B + i] = m->hm[i]; o[0x40 + i] = m->pos[i]; }
    o[0x45] = 0;
    put16(o + 0x46, m->cx);
    put64(o + 0x48, m->bar_line);
    put64(o + 0x50, m->frame_line);
    put32(o + 0x58, m->frame_no);
    put32(o + 0x5C, 0);
    memcpy(o + 0x80, m->ram, 128);
}

static void unpack_machine(orc_machine *m, const uint8_t *o) {
    m->a = o[0x00]; m->x = o[0x01]; m->y = o[0x02]; m->sp = o[0x03]; m->p = o[0x04];
    /* the cartridge latches only its own bank bits: one for F8, two for F6, three for F4 */
    m->bank = (uint8_t)(o[0x05] & (m->scheme == 3 ? 7u : m->scheme == 2 ? 3u : m->scheme == 1 ? 1u : 0u));
    m->pc = get16(o + 0x06);
    m->k = get64(o + 0x08);
    m->tim_cw = get64(o + 0x10);
    m->tim_v = o[0x18]; m->tim_shift = o[0x19]; m->swcha_out = o[0x1A]; m->swacnt = o[0x1B];
    m->swchb_out = o[0x1C]; m->swbcnt = o[0x1D]; m->jam = o[0x1E]; m->inpt4_latch = o[0x1F];
    m->vsync = o[0x20]; m->vblank = o[0x21]; m->nusiz[0] = o[0x22]; m->nusiz[1] = o[0x23];
    m->colup[0] = o[0x24]; m->colup[1] = o[0x25]; m->colupf = o[0x26]; m->colubk = o[0x27];
    m->ctrlpf = o[0x28]; m->refp[0] = o[0x29]; m->refp[1] = o[0x2A]; m->pf0 = o[0x2B];
    m->pf1 = o[0x2C]; m->pf2 = o[0x2D]; m->enam[0] = o[0x2E]; m->enam[1] = o[0x2F];
    m->enabl_new = o[0x30]; m->enabl_old = o[0x31]; m->grp_new[0] = o[0x32]; m->grp_old[0] = o[0x33];
    m->grp_new[1] = o[0x34]; m->grp_old[1] = o[0x35]; m->vdelp[0] = o[0x36]; m->vdelp[1] = o[0x37];
    m->vdelbl = o[0x38]; m->resmp[0] = o[0x39]; m->resmp[1] = o[0x3A];
    for (int i = 0; i < 5; i++) { m->hm[i] = o[0x3B + i]; m->pos[i] = o[0x40 + i]; }
    m->cx = get16(o + 0x46);
    m->bar_line = get64(o + 0x48);
    m->frame_line = get64(o + 0x50);
    m->frame_no = (uint32_t)(o[0x58] | o[0x59] << 8 | o[0x5A] << 16 | (uint32_t)o[0x5B] << 24);
    memcpy(m->ram, o + 0x80, 128);
    m->tia_clock = 3 * m->k;
}

void orc_machine_get_state(const orc_machine *m, uint8_t *out) {
    memset(out, 0, ORC_STATE_BYTES);
    pack_machine(m, out);
}
void orc_machine_set_state(orc_machine *m, const uint8_t *in) { unpack_machine(m, in); }

/* ------------------------------------------------------------------ Philox */

/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw (SC'11):
 * ten rounds of two 32x32->64 multiplies, the key bumped by the Weyl
 * constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    uint32_t ctr[4] = {a, b, c, d}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}
static uint32_t mulhi(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * n) >> 32); }

#define PURPOSE_STICKY 1u
#define PURPOSE_RESET 2u
#define PURPOSE_CACHE 3u
#define PURPOSE_POLICY 4u

/* ------------------------------------------------------------------ preprocessing */

/* Exact integer area resampling 210x160 -> 84x84 (weights in 1/84 pixel
 * units), round half up, of the per-pixel maximum of the two frames' lumas. */
void orc_preprocess(const uint8_t *f3, const uint8_t *f4, const uint8_t *luma, uint8_t *out) {
    for (int i = 0; i < ORC_OBS; i++) {
        int ylo = (210 * i) / 84, yhi = (210 * i + 210 + 83) / 84;
        for (int j = 0; j < ORC_OBS; j++) {
            int xlo = (160 * j) / 84, xhi = (160 * j + 160 + 83) / 84;
            int64_t s = 0;
            for (int y = ylo; y < yhi && y < 210; y++) {
                int a0 = 84 * y > 210 * i ? 84 * y : 210 * i;
                int a1 = 84 * y + 84 < 210 * i + 210 ? 84 * y + 84 : 210 * i + 210;
                int wy = a1 - a0;
                if (wy <= 0) continue;
                for (int x = xlo; x < xhi && x < 160; x++) {
                    int b0 = 84 * x > 160 * j ? 84 * x : 160 * j;
                    int b1 = 84 * x + 84 < 160 * j + 160 ? 84 * x + 84 : 160 * j + 160;
                    int wx = b1 - b0;
                    if (wx <= 0) continue;
                    uint8_t l3 = luma[f3[y * 160 + x] >> 1], l4 = luma[f4[y * 160 + x] >> 1];
                    s += (int64_t)wy * wx * (l3 > l4 ? l3 : l4);
                }
            }
            out[i * ORC_OBS + j] = (uint8_t)((s + 16800) / 33600);
        }
    }
}

/* ------------------------------------------------------------------ environments */

typedef struct {
    orc_machine m;
    uint32_t episode, step_no, env_key, status;
    uint8_t last_action, score_prev;
    int rom;
    uint64_t instret;      /* instructions retired by this env (all episodes) */
    uint8_t fb[2][ORC_FRAME_H * ORC_FRAME_W];
    uint8_t stack[4][ORC_OBS * ORC_OBS];
} orc_env;

struct orc_envs {
    int n_roms, n_envs;
    orc_config cfg;
    uint8_t luma[128];
    uint8_t **roms;
    size_t *rom_sizes;
    uint8_t *score_addr, *gameover_addr;
    orc_machine *cache;    /* [n_roms][n_cache] */
    orc_env *env;
};

/* Start states of ROM r (Section 3, reset strategy): from power-on, run the
 * start-up frames and then n_k = mulhi(philox(seed, r, k, purpose 3, 0),
 * max_noops + 1) further no-op frames; state k is the machine after those
 * frames.  The machine is deterministic, so one run from power-on with a
 * snapshot after every frame >= startup_frames gives every k. */
static void build_cache(orc_envs *e, int r) {
    int nmax = e->cfg.max_noops;
    orc_machine *snap = (orc_machine *)calloc((size_t)nmax + 1, sizeof *snap);
    orc_machine m;
    memset(&m, 0, sizeof m);
    m.rom = e->roms[r];
    m.rom_size = (uint32_t)e->rom_sizes[r];
    m.scheme = scheme_of(e->rom_sizes[r]);
    power_on(&m);
    for (int f = 0; f < e->cfg.startup_frames + nmax; f++) {
        if (f >= e->cfg.startup_frames) snap[f - e->cfg.startup_frames] = m;
        apply_action(&m, 0);
        run_frame(&m, NULL);
    }
    snap[nmax] = m;
    for (int k = 0; k < e->cfg.n_cache; k++) {
        uint32_t extra = mulhi(philox_word(e->cfg.seed, (uint32_t)r, (uint32_t)k, PURPOSE_CACHE << 8, 0),
                               (uint32_t)nmax + 1);
        e->cache[r * e->cfg.n_cache + k] = snap[extra];
    }
    free(snap);
}

typedef struct { orc_envs *e; int lo, hi; } cache_job;
static void *cache_worker(void *p) {
    cache_job *j = (cache_job *)p;
    for (int r = j->lo; r < j->hi; r++) build_cache(j->e, r);
    return NULL;
}
static void build_all_caches(orc_envs *e) {
    int nt = e->n_roms < 16 ? e->n_roms : 16;
    pthread_t th[16];
    cache_job jobs[16];
    for (int t = 0; t < nt; t++) {
        jobs[t] = (cache_job){e, e->n_roms * t / nt, e->n_roms * (t + 1) / nt};
        pthread_create(&th[t], NULL, cache_worker, &jobs[t]);
    }
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

/* Copy cached start state number mulhi(philox(seed, env_key, 0, purpose 2, episode), n_cache). */
static void reset_env(orc_envs *e, orc_env *v) {
    uint32_t idx = mulhi(philox_word(e->cfg.seed, v->env_key, 0, PURPOSE_RESET << 8, v->episode),
                         (uint32_t)e->cfg.n_cache);
    v->m = e->cache[v->rom * e->cfg.n_cache + (int)idx];
    v->m.status = 0;
    v->last_action = 0;
    v->score_prev = v->m.ram[e->score_addr[v->rom] & 0x7F];
    memset(v->stack, 0, sizeof v->stack);
}

orc_envs *orc_envs_create(const uint8_t *const *roms, const size_t *rom_sizes,
                          const uint8_t *score_addr, const uint8_t *gameover_addr, int n_roms,
                          const int32_t *env_rom, const uint32_t *env_key, int n_envs,
                          const orc_config *cfg, const uint8_t *luma) {
    if (n_roms <= 0 || n_envs < 0 || cfg->frameskip < 2 || cfg->n_cache < 1 || cfg->max_noops < 0 ||
        cfg->startup_frames < 0)
        return NULL;
    for (int r = 0; r < n_roms; r++)
        if (scheme_of(rom_sizes[r]) < 0) return NULL;
    for (int i = 0; i < n_envs; i++)
        if (env_rom[i] < 0 || env_rom[i] >= n_roms) return NULL;
    pthread_once(&ops_once, build_ops);
    orc_envs *e = (orc_envs *)calloc(1, sizeof *e);
    e->n_roms = n_roms;
    e->n_envs = n_envs;
    e->cfg = *cfg;
    if (luma) memcpy(e->luma, luma, 128);
    e->roms = (uint8_t **)calloc((size_t)n_roms, sizeof *e->roms);
    e->rom_sizes = (size_t *)calloc((size_t)n_roms, sizeof *e->rom_sizes);
    e->score_addr = (uint8_t *)calloc((size_t)n_roms, 1);
    e->gameover_addr = (uint8_t *)calloc((size_t)n_roms, 1);
    for (int r = 0; r < n_roms; r++) {
        e->roms[r] = (uint8_t *)malloc(rom_sizes[r]);
        memcpy(e->roms[r], roms[r], rom_sizes[r]);
        e->rom_sizes[r] = rom_sizes[r];
        e->score_addr[r] = score_addr[r];
        e->gameover_addr[r] = gameover_addr[r];
    }
    e->cache = (orc_machine *)calloc((size_t)n_roms * (size_t)cfg->n_cache, sizeof *e->cache);
    build_all_caches(e);
    e->env = (orc_env *)calloc((size_t)(n_envs ? n_envs : 1), sizeof *e->env);
    for (int i = 0; i < n_envs; i++) {
        orc_env *v = &e->env[i];
        v->rom = env_rom[i];
        v->env_key = env_key ? env_key[i] : (uint32_t)i;
        v->episode = 0;
        reset_env(e, v);
    }
    return e;
}

void orc_envs_free(orc_envs *e) {
    if (!e) return;
    for (int r = 0; r < e->n_roms; r++) free(e->roms[r]);
    free(e->roms); free(e->rom_sizes); free(e->score_addr); free(e->gameover_addr);
    free(e->cache); free(e->env); free(e);
}

void orc_envs_reset(orc_envs *e, const uint8_t *mask) {
    for (int i = 0; i < e->n_envs; i++) {
        if (mask && !mask[i]) continue;
        e->env[i].episode++;
        reset_env(e, &e->env[i]);
    }
}

/* One env step (R17-R21): F frames with the action (sticky repeats drawn per
 * frame), reward = sum of per-frame int8 deltas of the score byte, the last
 * two frames rendered, done read after frame F, observation emitted, then a
 * reset from the cache when done. */
static void step_env(orc_envs *e, int i, uint8_t action, uint8_t *obs, int32_t *reward, uint8_t *done) {
    orc_env *v = &e->env[i];
    int F = e->cfg.frameskip;
    if (action >= 18) { v->status |= ORC_ST_BAD_ACTION; action = 0; }
    int32_t r = 0;
    uint8_t score_a = e->score_addr[v->rom] & 0x7F, over_a = e->gameover_addr[v->rom] & 0x7F;
    uint64_t retired0 = v->m.instret;
    for (int f = 1; f <= F; f++) {
        uint8_t a = action;
        if (e->cfg.sticky) {
            uint32_t u = philox_word(e->cfg.seed, v->env_key, v->step_no, (uint32_t)f | PURPOSE_STICKY << 8, v->episode);
            if (u < 0x40000000u) a = v->last_action;
        }
        v->last_action = a;
        apply_action(&v->m, a);
        uint8_t *fb = f >= F - 1 ? v->fb[f - (F - 1)] : NULL;
        run_frame(&v->m, fb);
        uint8_t s = v->m.ram[score_a];
        r += (int8_t)(uint8_t)(s - v->score_prev);
        v->score_prev = s;
    }
    v->status |= v->m.status;
    if (v->m.jam) v->status |= ORC_ST_ILLEGAL;   /* done because the CPU is halted */
    v->instret += v->m.instret - retired0;
    int d = v->m.ram[over_a] != 0 || v->m.jam;
    if (e->cfg.output_mode == 0) {
        memcpy(obs, v->fb[1], ORC_FRAME_H * ORC_FRAME_W);
    } else {
        memmove(v->stack[0], v->stack[1], 3 * ORC_OBS * ORC_OBS);
        orc_preprocess(v->fb[0], v->fb[1], e->luma, v->stack[3]);
        memcpy(obs, v->stack, sizeof v->stack);
    }
    *reward = r;
    *done = (uint8_t)d;
    v->step_no++;
    if (d) {
        v->episode++;
        reset_env(e, v);
    }
}

typedef struct {
    orc_envs *e;
    const uint8_t *actions;
    uint8_t *obs;
    int32_t *rewards;
    uint8_t *dones;
    int lo, hi;
} step_job;

static void *step_worker(void *p) {
    step_job *j = (step_job *)p;
    size_t ob = j->e->cfg.output_mode == 0 ? ORC_FRAME_H * ORC_FRAME_W : 4 * ORC_OBS * ORC_OBS;
    for (int i = j->lo; i < j->hi; i++)
        step_env(j->e, i, j->actions[i], j->obs + ob * (size_t)i, j->rewards + i, j->dones + i);
    return NULL;
}

int orc_envs_step(orc_envs *e, const uint8_t *actions, uint8_t *obs, int32_t *rewards,
                  uint8_t *dones, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > e->n_envs) n_threads = e->n_envs ? e->n_envs : 1;
    step_job jobs[256];
    pthread_t th[256];
    if (n_threads > 256) n_threads = 256;
    for (int t = 0; t < n_threads; t++) {
        jobs[t] = (step_job){e, actions, obs, rewards, dones,
                             (int)((int64_t)e->n_envs * t / n_threads),
                             (int)((int64_t)e->n_envs * (t + 1) / n_threads)};
    }
    if (n_threads == 1) { step_worker(&jobs[0]); return 0; }
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, step_worker, &jobs[t]);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    return 0;
}

/* Inverse of orc_envs_get_state for the machine and env fields; each env
 * keeps its cartridge (the state's cartridge field is not read). */
void orc_envs_set_state(orc_envs *e, const uint8_t *in) {
    for (int i = 0; i < e->n_envs; i++) {
        orc_env *v = &e->env[i];
        const uint8_t *o = in + (size_t)ORC_STATE_BYTES * i;
        unpack_machine(&v->m, o);
        v->episode = get32(o + 0x60);
        v->step_no = get32(o + 0x64);
        v->env_key = get32(o + 0x68);
        v->status = get32(o + 0x6C);
        v->last_action = o[0x70];
        v->score_prev = o[0x71];
    }
}

void orc_envs_get_state(const orc_envs *e, uint8_t *out) {
    for (int i = 0; i < e->n_envs; i++) {
        const orc_env *v = &e->env[i];
        uint8_t *o = out + (size_t)ORC_STATE_BYTES * i;
        memset(o, 0, ORC_STATE_BYTES);
        pack_machine(&v->m, o);
        put32(o + 0x60, v->episode);
        put32(o + 0x64, v->step_no);
        put32(o + 0x68, v->env_key);
        put32(o + 0x6C, v->status);
        o[0x70] = v->last_action;
        o[0x71] = v->score_prev;
        put16(o + 0x72, (uint16_t)v->rom);
    }
}

void orc_envs_get_frames(const orc_envs *e, uint8_t *out) {
    for (int i = 0; i < e->n_envs; i++) memcpy(out + (size_t)i * sizeof e->env[i].fb, e->env[i].fb, sizeof e->env[i].fb);
}

void orc_envs_get_cache(const orc_envs *e, uint8_t *out) {
    for (int i = 0; i < e->n_roms * e->cfg.n_cache; i++) {
        memset(out + (size_t)i * ORC_STATE_BYTES, 0, ORC_STATE_BYTES);
        pack_machine(&e->cache[i], out + (size_t)i * ORC_STATE_BYTES);
    }
}

uint64_t orc_envs_instructions(const orc_envs *e) {
    uint64_t s = 0;
    for (int i = 0; i < e->n_envs; i++) s += e->env[i].instret;
    return s;
}

/* ------------------------------------------------------------------ policy */

/* exp(x) for x <= 0 (and small positive x): x = k ln2 + r with the two-part
 * Cody-Waite constant (C1 = 355/512 exactly representable, C2 the
 * remainder), exp(r) by the degree-7 Taylor polynomial in Horner form with
 * fused multiply-adds, scaled by 2^k through the exponent field.  Results
 * below the normal range are flushed to 0. */
float orc_exp_own(float x) {
    if (x < -87.0f) return 0.0f;
    float kf = rintf(x * 1.44269504088896341f);
    float r = fmaf(-kf, 0.693359375f, x);
    r = fmaf(-kf, -2.12194440e-4f, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int k = (int)kf;
    if (k < -126) return 0.0f;
    union { uint32_t u; float f; } sc;
    sc.u = (uint32_t)(k + 127) << 23;
    return p * sc.f;
}

static float bf16_to_f32(uint16_t b) {
    union { uint32_t u; float f; } v;
    v.u = (uint32_t)b << 16;
    return v.f;
}

void orc_policy_logits(const uint8_t *x, const uint16_t *w, float *logits) {
    static __thread float part[512][ORC_POLICY_A];
    for (int c = 0; c < 512; c++) {
        for (int j = 0; j < ORC_POLICY_A; j++) part[c][j] = 0.0f;
        if (c >= ORC_POLICY_K / 64) continue;
        for (int q = 0; q < 64; q++) {
            int k = c * 64 + q;
            float xv = (float)x[k];
            for (int j = 0; j < ORC_POLICY_A; j++)
                part[c][j] = fmaf(xv, bf16_to_f32(w[(size_t)k * ORC_POLICY_A + j]), part[c][j]);
        }
    }
    for (int h = 256; h >= 1; h >>= 1)
        for (int i = 0; i < h; i++)
            for (int j = 0; j < ORC_POLICY_A; j++) part[i][j] = part[i][j] + part[i + h][j];
    for (int j = 0; j < ORC_POLICY_A; j++) logits[j] = part[0][j];
}

int orc_policy_sample(const float *l, uint32_t u) {
    float m = l[0];
    for (int j = 1; j < ORC_POLICY_A; j++) if (l[j] > m) m = l[j];
    float e[ORC_POLICY_A], tot = 0.0f;
    for (int j = 0; j < ORC_POLICY_A; j++) { e[j] = orc_exp_own(l[j] - m); tot = tot + e[j]; }
    /* u as an exact 24-bit fraction in [0, 1); when rounding leaves every
     * running sum at or below the threshold, the last action with nonzero
     * weight is taken */
    float thr = ((float)(u >> 8) * 5.9604644775390625e-08f) * tot;
    float c = 0.0f;
    int last = 0;
    for (int j = 0; j < ORC_POLICY_A; j++) {
        c = c + e[j];
        if (e[j] > 0.0f) last = j;
        if (c > thr) return j;
    }
    return last;
}

typedef struct {
    const orc_envs *e;
    const uint8_t *obs;
    const uint16_t *w;
    uint8_t *act;
    float *logits;
    int lo, hi;
} policy_job;

static void *policy_worker(void *p) {
    policy_job *j = (policy_job *)p;
    for (int i = j->lo; i < j->hi; i++) {
        const orc_env *v = &j->e->env[i];
        float l[ORC_POLICY_A];
        orc_policy_logits(j->obs + (size_t)i * ORC_POLICY_K, j->w, l);
        uint32_t u = philox_word(j->e->cfg.seed, v->env_key, v->step_no, PURPOSE_POLICY << 8, v->episode);
        j->act[i] = (uint8_t)orc_policy_sample(l, u);
        if (j->logits) memcpy(j->logits + (size_t)i * ORC_POLICY_A, l, sizeof l);
    }
    return NULL;
}

void orc_envs_policy(const orc_envs *e, const uint8_t *obs, const uint16_t *w, uint8_t *actions, float *logits,
                     int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 64) n_threads = 64;
    if (n_threads > e->n_envs) n_threads = e->n_envs ? e->n_envs : 1;
    policy_job jobs[64];
    pthread_t th[64];
    for (int t = 0; t < n_threads; t++)
        jobs[t] = (policy_job){e, obs, w, actions, logits, (int)((int64_t)e->n_envs * t / n_threads),
                               (int)((int64_t)e->n_envs * (t + 1) / n_threads)};
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, policy_worker, &jobs[t]);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
}

/* Behaviour probability mu(a|s) of the sampled action (the quantity a
 * training buffer keeps for V-trace, Appendix "V-trace"): the action's
 * softmax weight over the total, the weights and total formed exactly as in
 * orc_policy_sample, fp32 division. */
float orc_policy_prob(const float *l, int a) {
    float m = l[0];
    for (int j = 1; j < ORC_POLICY_A; j++) if (l[j] > m) m = l[j];
    float e[ORC_POLICY_A], tot = 0.0f;
    for (int j = 0; j < ORC_POLICY_A; j++) { e[j] = orc_exp_own(l[j] - m); tot = tot + e[j]; }
    return e[a] / tot;
}

void orc_envs_policy_mu(int n, const float *logits, const uint8_t *actions, float *mu) {
    for (int i = 0; i < n; i++) mu[i] = orc_policy_prob(logits + (size_t)i * ORC_POLICY_A, actions[i]);
}

/* ------------------------------------------------------------------ learner-side targets
 * Appendix, "A2C" and "V-trace": over a rollout of T steps of n envs,
 * time-major arrays ([T][n]; values [T+1][n], row T the bootstrap value of
 * the state after the last step), in double precision, each target written
 * out as its sum definition.  Reading (the paper does not treat episode
 * ends inside a rollout): a done at step t ends the return there, i.e. the
 * discount after step t is gamma_t = gamma * (1 - done_t). */

/* Bootstrapped N-step return of Eq. costPi:
 *   R_t = sum_{i=0}^{k-1} gamma^i r_{t+i} + gamma^k V(s_{t+k}),  k = T - t,
 * with the sum cut after the first done at or after t (no bootstrap then). */
void orc_nstep_returns(int T, int n, const float *rewards, const uint8_t *dones, const float *values,
                       double gamma, double *returns) {
    for (int e = 0; e < n; e++) {
        for (int t = 0; t < T; t++) {
            double sum = 0.0, disc = 1.0;
            int ended = 0;
            for (int u = t; u < T; u++) {
                sum += disc * (double)rewards[(size_t)u * n + e];
                if (dones[(size_t)u * n + e]) { ended = 1; break; }
                disc *= gamma;
            }
            if (!ended) sum += disc * (double)values[(size_t)T * n + e];
            returns[(size_t)t * n + e] = sum;
        }
    }
}

/* V-trace target of Eq. target.off with the truncated importance weights of
 * Eqs. rho and c:
 *   v_t = V(s_t) + sum_{u=t}^{T-1} ( prod_{i=t}^{u-1} gamma_i c_i ) delta_u,
 *   delta_u = rho_u ( r_u + gamma_u V(s_{u+1}) - V(s_u) ),
 *   rho_u = min(rho_bar, pi_u / mu_u),  c_u = min(c_bar, pi_u / mu_u),
 * (gamma_i in place of the constant gamma per the reading above), and the
 * policy-gradient advantage of the paper's actor update,
 *   A_t = rho_t ( r_t + gamma_t v_{t+1} - V(s_t) ),  v_T = V(s_T).
 * pi and mu are the target and behaviour probabilities of the actions taken. */
void orc_vtrace(int T, int n, const float *rewards, const uint8_t *dones, const float *values, const float *pi,
                const float *mu, double gamma, double rho_bar, double c_bar, double *vs, double *pg_adv) {
    for (int e = 0; e < n; e++) {
        for (int t = 0; t < T; t++) {
            double v = (double)values[(size_t)t * n + e], coef = 1.0;
            for (int u = t; u < T; u++) {
                const size_t k = (size_t)u * n + e;
                const double g = dones[k] ? 0.0 : gamma;
                const double ratio = (double)pi[k] / (double)mu[k];
                const double rho = ratio < rho_bar ? ratio : rho_bar;
                const double c = ratio < c_bar ? ratio : c_bar;
                const double delta = rho * ((double)rewards[k] + g * (double)values[k + n] - (double)values[k]);
                v += coef * delta;
                coef *= g * c;
            }
            vs[(size_t)t * n + e] = v;
        }
        for (int t = 0; t < T; t++) {
            const size_t k = (size_t)t * n + e;
            const double g = dones[k] ? 0.0 : gamma;
            const double ratio = (double)pi[k] / (double)mu[k];
            const double rho = ratio < rho_bar ? ratio : rho_bar;
            const double vnext = t + 1 < T ? vs[k + n] : (double)values[(size_t)T * n + e];
            pg_adv[k] = rho * ((double)rewards[k] + g * vnext - (double)values[k]);
        }
    }
}
