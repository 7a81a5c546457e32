// Device-side console: MOS 6507 interpreter, RIOT, TIA register file with
// lazy bitmask collision evaluation, and the per-frame TIA-write log.
//
// Paper, Section 3 (CuLE): the Atari CPU kernel executes the game code,
// keeps CPU state and the 128-byte RAM per emulator, and does not render: it
// copies TIA writes into a per-env buffer in device memory, which a second
// kernel replays into frames.  Here each log record carries the color clock
// at which the write takes effect, so the replay is exact.  The CPU kernel
// must still answer collision-register reads mid-frame, so collisions are
// evaluated here, lazily: only when a collision-relevant register is about
// to change or a collision register is read, over the span of color clocks
// since the last evaluation, with 160-bit object masks per scanline segment.
//
// Machine readings (effect clocks, positions, HMOVE bar, timer) follow the
// library's stated model: a write at CPU cycle t takes effect at color clock
// 3(t+1); a collision read at t sees clocks < 3t; an instruction of n cycles
// starting at k0 makes its data access at k0+n-1 (read-modify-write: read at
// -2, old value written at -1, new value at the last cycle); fetches and
// indirect pointer reads happen at k0.
#pragma once
#include <cstdint>

namespace atari {

// ---------------------------------------------------------------- state layout
// Canonical 256-byte per-env state (little-endian), identical to the layout
// documented in include/atari_gpu.h.
namespace S {
constexpr int A = 0x00, X = 0x01, Y = 0x02, SP = 0x03, P = 0x04, BANK = 0x05, PC = 0x06;
constexpr int CYCLES = 0x08, TIM_CW = 0x10, TIM_V = 0x18, TIM_SHIFT = 0x19, SWCHA_OUT = 0x1A,
              SWACNT = 0x1B, SWCHB_OUT = 0x1C, SWBCNT = 0x1D, JAM = 0x1E, INPT4_LATCH = 0x1F;
constexpr int TIA = 0x20;  // 0x20..0x3F registers, 0x40..0x44 positions
constexpr int POS = 0x40, CX = 0x46, BAR_LINE = 0x48, FRAME_LINE = 0x50, FRAME_NO = 0x58;
constexpr int EPISODE = 0x60, STEP = 0x64, ENV_KEY = 0x68, STATUS = 0x6C, LAST_ACTION = 0x70,
              SCORE_PREV = 0x71, ROM = 0x72, RAM = 0x80;
constexpr int MACHINE_END = 0x60;  // bytes [0, 0x60) and [0x80, 0x100) are machine state
}  // namespace S

constexpr uint32_t ST_ILLEGAL = 1u, ST_FRAME_CAP = 2u, ST_LOG_OVERFLOW = 4u, ST_BAD_ACTION = 8u, ST_STALL = 16u;
constexpr uint64_t NO_LINE = ~0ull;
constexpr int WINDOW_Y0 = 31, FRAME_H = 210, FRAME_W = 160, CAP_LINES = 400;

// Decode word: op | mode << 8 | cycles << 12 (4 bits) | read-penalty << 16
enum Mode : uint32_t { IMP, ACC, IMM, ZP, ZPX, ZPY, ABS, ABX, ABY, IND, IZX, IZY, REL };
enum Op : uint32_t {
  O_JAM = 0, O_ADC, O_AND, O_ASL, O_BCC, O_BCS, O_BEQ, O_BIT, O_BMI, O_BNE, O_BPL, O_BRK, O_BVC,
  O_BVS, O_CLC, O_CLD, O_CLI, O_CLV, O_CMP, O_CPX, O_CPY, O_DEC, O_DEX, O_DEY, O_EOR, O_INC,
  O_INX, O_INY, O_JMP, O_JSR, O_LDA, O_LDX, O_LDY, O_LSR, O_NOP, O_ORA, O_PHA, O_PHP, O_PLA,
  O_PLP, O_ROL, O_ROR, O_RTI, O_RTS, O_SBC, O_SEC, O_SED, O_SEI, O_STA, O_STX, O_STY, O_TAX,
  O_TAY, O_TSX, O_TXA, O_TXS, O_TYA,
  // undocumented NMOS operations with a stable published behaviour
  O_SLO, O_RLA, O_SRE, O_RRA, O_SAX, O_LAX, O_DCP, O_ISC, O_ANC, O_ALR, O_SBX
};

// TIA write registers that change what collides, and those the replay needs.
constexpr uint64_t COLL_REGS =
    (1ull << 0x01) | (1ull << 0x04) | (1ull << 0x05) | (1ull << 0x0A) | (1ull << 0x0B) | (1ull << 0x0C) |
    (1ull << 0x0D) | (1ull << 0x0E) | (1ull << 0x0F) | (0x1Full << 0x10) | (0x1Full << 0x1B) |
    (0x1Full << 0x25) | (1ull << 0x2A);
constexpr uint64_t LOG_REGS = COLL_REGS | (0xFull << 0x06) | (0x1Full << 0x20) | (1ull << 0x2B);

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds; each round multiplies counter words 0 and 2 by the
// two round constants, mixes the high halves with words 1, 3 and the key,
// and the key advances by the golden-ratio Weyl increments between rounds.
__host__ __device__ inline uint32_t philox_x0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint64_t m0 = (uint64_t)c0 * 0xD2511F53u;
    uint64_t m1 = (uint64_t)c2 * 0xCD9E8D57u;
    uint32_t y0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0;
    uint32_t y2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)m1;
    c3 = (uint32_t)m0;
    c0 = y0;
    c2 = y2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c0;
}
__host__ __device__ inline uint32_t scale32(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * n) >> 32); }
constexpr uint32_t PURPOSE_STICKY = 1, PURPOSE_RESET = 2, PURPOSE_CACHE = 3;

// ---------------------------------------------------------------- 160-bit masks
struct M160 {
  uint32_t w0, w1, w2, w3, w4;
};
__device__ __forceinline__ uint32_t spread2(uint32_t b) {  // bit i -> bits 2i, 2i+1
  uint32_t x = b & 0xFF;
  x = (x | (x << 4)) & 0x0F0Fu;
  x = (x | (x << 2)) & 0x3333u;
  x = (x | (x << 1)) & 0x5555u;
  return x * 3u;
}
__device__ __forceinline__ uint32_t spread4(uint32_t b) {  // bit i -> bits 4i..4i+3
  uint32_t x = b & 0xFF;
  x = (x | (x << 12)) & 0x000F000Fu;
  x = (x | (x << 6)) & 0x03030303u;
  x = (x | (x << 3)) & 0x11111111u;
  return x * 15u;
}
// Rotate a 160-bit mask so that pixel p moves to pixel (p + s) mod 160.
__device__ __forceinline__ M160 rot160(M160 a, uint32_t s) {
  uint32_t q = s >> 5, r = s & 31;
  // whole-word rotation by q (0..4) via three conditional fixed rotations
  if (q & 1) { uint32_t t = a.w4; a.w4 = a.w3; a.w3 = a.w2; a.w2 = a.w1; a.w1 = a.w0; a.w0 = t; }
  if (q & 2) { uint32_t t0 = a.w3, t1 = a.w4; a.w4 = a.w2; a.w3 = a.w1; a.w2 = a.w0; a.w1 = t1; a.w0 = t0; }
  if (q & 4) { uint32_t t0 = a.w1, t1 = a.w2, t2 = a.w3, t3 = a.w4; a.w4 = a.w0; a.w0 = t0; a.w1 = t1; a.w2 = t2; a.w3 = t3; }
  if (r) {
    M160 b;
    b.w0 = __funnelshift_l(a.w4, a.w0, r);
    b.w1 = __funnelshift_l(a.w0, a.w1, r);
    b.w2 = __funnelshift_l(a.w1, a.w2, r);
    b.w3 = __funnelshift_l(a.w2, a.w3, r);
    b.w4 = __funnelshift_l(a.w3, a.w4, r);
    return b;
  }
  return a;
}
__device__ __forceinline__ uint32_t range_word(int w, uint32_t lo, uint32_t hi) {
  int a = (int)lo - 32 * w, b = (int)hi - 32 * w;
  a = a < 0 ? 0 : (a > 32 ? 32 : a);
  b = b < 0 ? 0 : (b > 32 ? 32 : b);
  if (b <= a) return 0u;
  uint32_t hiMask = b == 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
  uint32_t loMask = a == 32 ? 0xFFFFFFFFu : ((1u << a) - 1u);
  return hiMask & ~loMask;
}

// copies: bit0 offset 0, bit1 +16, bit2 +32, bit3 +64
__device__ __forceinline__ uint32_t copy_bits(uint32_t nusiz) {
  switch (nusiz & 7) {
    case 1: return 3; case 2: return 5; case 3: return 7; case 4: return 9; case 6: return 13;
    default: return 1;
  }
}
// Pixel pattern of a player with pixel i (left to right) at bit i.
__device__ __forceinline__ uint32_t player_bits(uint32_t grp, uint32_t refp) {
  return (refp & 8) ? (grp & 0xFF) : (__brev(grp & 0xFF) >> 24);
}
// Masks of the objects at pixel 0 (before the move to their position): the
// widest (three copies, or a 32-pixel quad-size player) spans words 0..2, so
// words 3 and 4 are always zero.
__device__ __forceinline__ M160 player_base(uint32_t grp, uint32_t refp, uint32_t nusiz) {
  uint32_t g = player_bits(grp, refp);
  M160 m{0, 0, 0, 0, 0};
  uint32_t mode = nusiz & 7;
  if (mode == 5) m.w0 = spread2(g);
  else if (mode == 7) m.w0 = spread4(g);
  else {
    uint32_t c = copy_bits(nusiz);
    m.w0 = ((c & 1) ? g : 0u) | ((c & 2) ? (g << 16) : 0u);
    m.w1 = (c & 4) ? g : 0u;
    m.w2 = (c & 8) ? g : 0u;
  }
  return m;
}
__device__ __forceinline__ M160 missile_base(uint32_t nusiz) {
  uint32_t w = 1u << ((nusiz >> 4) & 3);
  uint32_t base = (1u << w) - 1u;
  M160 m{0, 0, 0, 0, 0};
  uint32_t c = ((nusiz & 7) == 5 || (nusiz & 7) == 7) ? 1u : copy_bits(nusiz);
  m.w0 = ((c & 1) ? base : 0u) | ((c & 2) ? (base << 16) : 0u);
  m.w1 = (c & 4) ? base : 0u;
  m.w2 = (c & 8) ? base : 0u;
  return m;
}
__device__ __forceinline__ M160 ball_base(uint32_t ctrlpf) {
  uint32_t w = 1u << ((ctrlpf >> 4) & 3);
  return M160{(1u << w) - 1u, 0, 0, 0, 0};
}
__device__ __forceinline__ M160 player_mask(uint32_t grp, uint32_t refp, uint32_t nusiz, uint32_t pos) {
  return rot160(player_base(grp, refp, nusiz), pos);
}
__device__ __forceinline__ M160 missile_mask(uint32_t nusiz, uint32_t pos) {
  return rot160(missile_base(nusiz), pos);
}
__device__ __forceinline__ M160 ball_mask(uint32_t ctrlpf, uint32_t pos) {
  return rot160(ball_base(ctrlpf), pos);
}
// 20 playfield bits of a half, bit b = 4-pixel block b from the left.
__device__ __forceinline__ uint32_t pf20(uint32_t pf0, uint32_t pf1, uint32_t pf2) {
  return ((pf0 >> 4) & 0xF) | ((__brev(pf1 & 0xFF) >> 24) << 4) | ((pf2 & 0xFF) << 12);
}
__device__ __forceinline__ M160 pf_mask(uint32_t pf0, uint32_t pf1, uint32_t pf2, uint32_t ctrlpf) {
  uint32_t l = pf20(pf0, pf1, pf2);
  uint32_t r = (ctrlpf & 1) ? (__brev(l) >> 12) : l;
  M160 m;
  m.w0 = spread4(l & 0xFF);
  m.w1 = spread4((l >> 8) & 0xFF);
  m.w2 = spread4((l >> 16) & 0xF) | (spread4(r & 0xF) << 16);
  m.w3 = spread4((r >> 4) & 0xFF);
  m.w4 = spread4((r >> 12) & 0xFF);
  return m;
}
__device__ __forceinline__ bool meet(const M160 &a, const M160 &b, const M160 &r) {
  return ((a.w0 & b.w0 & r.w0) | (a.w1 & b.w1 & r.w1) | (a.w2 & b.w2 & r.w2) | (a.w3 & b.w3 & r.w3) |
          (a.w4 & b.w4 & r.w4)) != 0u;
}

// ---------------------------------------------------------------- memory policies
// Plain form: RAM bytes live in the env's canonical state in global memory and
// the ROM image is read from global memory.
struct GlobalMem {
  uint8_t *ram;          // 128 bytes
  const uint8_t *rom;    // this env's image, banks of 4096 (2K images stored mirrored)
  __device__ __forceinline__ uint32_t ram_rd(uint32_t a) const { return ram[a]; }
  __device__ __forceinline__ void ram_wr(uint32_t a, uint32_t v) const { ram[a] = (uint8_t)v; }
  __device__ __forceinline__ uint32_t rom_rd(uint32_t off) const { return __ldg(rom + off); }
};
// Batched form: RAM in shared memory, one 32-bit word per byte, interleaved
// by thread (word addr * stride + lane) so a warp's accesses never conflict;
// the ROM image of the block's cartridge staged in shared memory.
struct SharedMem {
  uint32_t *ram;         // &smem_ram[threadIdx.x]
  uint32_t stride;       // threads per block
  const uint8_t *rom;    // shared-memory ROM image
  __device__ __forceinline__ uint32_t ram_rd(uint32_t a) const { return ram[a * stride]; }
  __device__ __forceinline__ void ram_wr(uint32_t a, uint32_t v) const { ram[a * stride] = v & 0xFF; }
  __device__ __forceinline__ uint32_t rom_rd(uint32_t off) const { return rom[off]; }
};

struct LogSink {
  uint32_t *rec;   // log records of this frame, or nullptr when not rendering
  uint32_t n, cap;
};

// ---------------------------------------------------------------- the console
template <class Mem>
struct Console {
  // CPU
  uint32_t A, X, Y, SP, P, PC, bank, jam;
  // time: CPU cycles since the first line of the current frame, and that line
  uint32_t kf;
  uint64_t L0;
  // RIOT
  uint64_t tim_cw;
  uint32_t tim_v, tim_shift, swcha_out, swacnt, swchb_out, swbcnt;
  uint32_t joy, fire, inpt4_latch;
  // TIA registers
  uint32_t vsync, vblank, nusiz0, nusiz1, colup0, colup1, colupf, colubk, ctrlpf, refp0, refp1;
  uint32_t pf0, pf1, pf2, enam0, enam1, enabl_new, enabl_old, grp0_new, grp0_old, grp1_new, grp1_old;
  uint32_t vdelp0, vdelp1, vdelbl, resmp0, resmp1, hmp0, hmp1, hmm0, hmm1, hmbl;
  uint32_t pos_p0, pos_p1, pos_m0, pos_m1, pos_bl;
  uint32_t cx;
  uint64_t bar_line;
  uint32_t ceval;      // collisions accounted for every color clock < ceval (frame-relative)
  uint32_t frame_no;
  uint32_t status;
  uint32_t instret;
  // per-instruction events
  uint32_t wsync, vs_rise, vs_rise_kf;
  uint32_t scheme;     // 0 plain, 1 F8, 2 F6
  Mem mem;
  const uint32_t *dec; // 256-entry decode table
  LogSink log;

  // ---- canonical state I/O (machine part) ----
  __device__ void load(const uint8_t *s) {
    // the cartridge latches only its own bank bits (F8 one, F6 two); scheme is set before load
    A = s[S::A]; X = s[S::X]; Y = s[S::Y]; SP = s[S::SP]; P = s[S::P];
    bank = s[S::BANK] & (scheme == 3 ? 7u : scheme == 2 ? 3u : scheme == 1 ? 1u : 0u);
    PC = s[S::PC] | (uint32_t)s[S::PC + 1] << 8;
    uint64_t k = ld64(s + S::CYCLES);
    tim_cw = ld64(s + S::TIM_CW);
    tim_v = s[S::TIM_V]; tim_shift = s[S::TIM_SHIFT]; swcha_out = s[S::SWCHA_OUT]; swacnt = s[S::SWACNT];
    swchb_out = s[S::SWCHB_OUT]; swbcnt = s[S::SWBCNT]; jam = s[S::JAM]; inpt4_latch = s[S::INPT4_LATCH];
    const uint8_t *t = s + S::TIA;
    vsync = t[0]; vblank = t[1]; nusiz0 = t[2]; nusiz1 = t[3]; colup0 = t[4]; colup1 = t[5]; colupf = t[6];
    colubk = t[7]; ctrlpf = t[8]; refp0 = t[9]; refp1 = t[10]; pf0 = t[11]; pf1 = t[12]; pf2 = t[13];
    enam0 = t[14]; enam1 = t[15]; enabl_new = t[16]; enabl_old = t[17]; grp0_new = t[18]; grp0_old = t[19];
    grp1_new = t[20]; grp1_old = t[21]; vdelp0 = t[22]; vdelp1 = t[23]; vdelbl = t[24]; resmp0 = t[25];
    resmp1 = t[26]; hmp0 = t[27]; hmp1 = t[28]; hmm0 = t[29]; hmm1 = t[30]; hmbl = t[31];
    pos_p0 = s[S::POS]; pos_p1 = s[S::POS + 1]; pos_m0 = s[S::POS + 2]; pos_m1 = s[S::POS + 3]; pos_bl = s[S::POS + 4];
    cx = s[S::CX] | (uint32_t)s[S::CX + 1] << 8;
    bar_line = ld64(s + S::BAR_LINE);
    L0 = ld64(s + S::FRAME_LINE);
    frame_no = ld32(s + S::FRAME_NO);
    kf = (uint32_t)(k - 76ull * L0);
    ceval = 3u * kf;
    status = 0;
    instret = 0;
    joy = 0xFF; fire = 0;
  }
  __device__ void store(uint8_t *s) const {
    s[S::A] = A; s[S::X] = X; s[S::Y] = Y; s[S::SP] = SP; s[S::P] = P; s[S::BANK] = bank;
    s[S::PC] = PC & 0xFF; s[S::PC + 1] = PC >> 8;
    st64(s + S::CYCLES, 76ull * L0 + kf);
    st64(s + S::TIM_CW, tim_cw);
    s[S::TIM_V] = tim_v; s[S::TIM_SHIFT] = tim_shift; s[S::SWCHA_OUT] = swcha_out; s[S::SWACNT] = swacnt;
    s[S::SWCHB_OUT] = swchb_out; s[S::SWBCNT] = swbcnt; s[S::JAM] = jam; s[S::INPT4_LATCH] = inpt4_latch;
    uint8_t *t = s + S::TIA;
    t[0] = vsync; t[1] = vblank; t[2] = nusiz0; t[3] = nusiz1; t[4] = colup0; t[5] = colup1; t[6] = colupf;
    t[7] = colubk; t[8] = ctrlpf; t[9] = refp0; t[10] = refp1; t[11] = pf0; t[12] = pf1; t[13] = pf2;
    t[14] = enam0; t[15] = enam1; t[16] = enabl_new; t[17] = enabl_old; t[18] = grp0_new; t[19] = grp0_old;
    t[20] = grp1_new; t[21] = grp1_old; t[22] = vdelp0; t[23] = vdelp1; t[24] = vdelbl; t[25] = resmp0;
    t[26] = resmp1; t[27] = hmp0; t[28] = hmp1; t[29] = hmm0; t[30] = hmm1; t[31] = hmbl;
    s[S::POS] = pos_p0; s[S::POS + 1] = pos_p1; s[S::POS + 2] = pos_m0; s[S::POS + 3] = pos_m1; s[S::POS + 4] = pos_bl;
    s[0x45] = 0;
    s[S::CX] = cx & 0xFF; s[S::CX + 1] = cx >> 8;
    st64(s + S::BAR_LINE, bar_line);
    st64(s + S::FRAME_LINE, L0);
    st32(s + S::FRAME_NO, frame_no);
    st32(s + 0x5C, 0);
  }
  // Render-state snapshot for the replay: bytes 0x20..0x5F of the canonical layout.
  __device__ void snapshot(uint8_t *o) const {
    uint8_t tmp[64];
    // reuse store's field order for the TIA block
    tmp[0] = vsync; tmp[1] = vblank; tmp[2] = nusiz0; tmp[3] = nusiz1; tmp[4] = colup0; tmp[5] = colup1;
    tmp[6] = colupf; tmp[7] = colubk; tmp[8] = ctrlpf; tmp[9] = refp0; tmp[10] = refp1; tmp[11] = pf0;
    tmp[12] = pf1; tmp[13] = pf2; tmp[14] = enam0; tmp[15] = enam1; tmp[16] = enabl_new; tmp[17] = enabl_old;
    tmp[18] = grp0_new; tmp[19] = grp0_old; tmp[20] = grp1_new; tmp[21] = grp1_old; tmp[22] = vdelp0;
    tmp[23] = vdelp1; tmp[24] = vdelbl; tmp[25] = resmp0; tmp[26] = resmp1; tmp[27] = hmp0; tmp[28] = hmp1;
    tmp[29] = hmm0; tmp[30] = hmm1; tmp[31] = hmbl; tmp[32] = pos_p0; tmp[33] = pos_p1; tmp[34] = pos_m0;
    tmp[35] = pos_m1; tmp[36] = pos_bl; tmp[37] = 0; tmp[38] = 0; tmp[39] = 0;
    uint64_t bl = bar_line;
    for (int i = 0; i < 8; i++) tmp[40 + i] = (uint8_t)(bl >> (8 * i));
    for (int i = 0; i < 8; i++) tmp[48 + i] = (uint8_t)(L0 >> (8 * i));
    for (int i = 56; i < 64; i++) tmp[i] = 0;
    uint4 *dst = reinterpret_cast<uint4 *>(o);
    const uint4 *src = reinterpret_cast<const uint4 *>(tmp);
#pragma unroll
    for (int i = 0; i < 4; i++) dst[i] = src[i];
  }

  static __device__ __forceinline__ uint64_t ld64(const uint8_t *p) {
    uint64_t v = 0;
#pragma unroll
    for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
    return v;
  }
  static __device__ __forceinline__ uint32_t ld32(const uint8_t *p) {
    return p[0] | (uint32_t)p[1] << 8 | (uint32_t)p[2] << 16 | (uint32_t)p[3] << 24;
  }
  static __device__ __forceinline__ void st64(uint8_t *p, uint64_t v) {
#pragma unroll
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
  }
  static __device__ __forceinline__ void st32(uint8_t *p, uint32_t v) {
#pragma unroll
    for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
  }

  // ---- inputs: the 18 actions of the agent interface on the P0 joystick ----
  __device__ void apply_action(uint32_t a) {
    // directions per action: up 1, right 2, left 4, down 8
    uint32_t d;
    switch (a) {
      case 2: case 10: d = 1; break;
      case 3: case 11: d = 2; break;
      case 4: case 12: d = 4; break;
      case 5: case 13: d = 8; break;
      case 6: case 14: d = 3; break;
      case 7: case 15: d = 5; break;
      case 8: case 16: d = 10; break;
      case 9: case 17: d = 12; break;
      default: d = 0; break;
    }
    joy = 0xFFu & ~(((d & 2) ? 0x80u : 0u) | ((d & 4) ? 0x40u : 0u) | ((d & 8) ? 0x20u : 0u) | ((d & 1) ? 0x10u : 0u));
    fire = (a == 1 || a >= 10) ? 1u : 0u;
    if (fire && (vblank & 0x40)) inpt4_latch = 1;
  }

  // ---- collisions ----
  __device__ __forceinline__ uint32_t live_objects() const {
    uint32_t g0 = (vdelp0 & 1) ? grp0_old : grp0_new;
    uint32_t g1 = (vdelp1 & 1) ? grp1_old : grp1_new;
    uint32_t eb = (vdelbl & 1) ? enabl_old : enabl_new;
    uint32_t l = 0;
    if (g0) l |= 1;
    if (g1) l |= 2;
    if ((enam0 & 2) && !(resmp0 & 2)) l |= 4;
    if ((enam1 & 2) && !(resmp1 & 2)) l |= 8;
    if (eb & 2) l |= 16;
    if ((pf0 & 0xF0) | pf1 | pf2) l |= 32;
    return l;
  }
  // Latch collisions among live objects on visible columns [lo, hi).
  __device__ void collide_cols(uint32_t live, uint32_t lo, uint32_t hi) {
    M160 r{range_word(0, lo, hi), range_word(1, lo, hi), range_word(2, lo, hi), range_word(3, lo, hi), range_word(4, lo, hi)};
    M160 z{0, 0, 0, 0, 0};
    M160 p0 = (live & 1) ? player_mask((vdelp0 & 1) ? grp0_old : grp0_new, refp0, nusiz0, pos_p0) : z;
    M160 p1 = (live & 2) ? player_mask((vdelp1 & 1) ? grp1_old : grp1_new, refp1, nusiz1, pos_p1) : z;
    M160 m0 = (live & 4) ? missile_mask(nusiz0, pos_m0) : z;
    M160 m1 = (live & 8) ? missile_mask(nusiz1, pos_m1) : z;
    M160 b = (live & 16) ? ball_mask(ctrlpf, pos_bl) : z;
    M160 f = (live & 32) ? pf_mask(pf0, pf1, pf2, ctrlpf) : z;
    uint32_t c = 0;
    c |= (uint32_t)meet(m0, p1, r) << 1 | (uint32_t)meet(m0, p0, r) << 0;
    c |= (uint32_t)meet(m1, p0, r) << 3 | (uint32_t)meet(m1, p1, r) << 2;
    c |= (uint32_t)meet(p0, f, r) << 5 | (uint32_t)meet(p0, b, r) << 4;
    c |= (uint32_t)meet(p1, f, r) << 7 | (uint32_t)meet(p1, b, r) << 6;
    c |= (uint32_t)meet(m0, f, r) << 9 | (uint32_t)meet(m0, b, r) << 8;
    c |= (uint32_t)meet(m1, f, r) << 11 | (uint32_t)meet(m1, b, r) << 10;
    c |= (uint32_t)meet(b, f, r) << 13;
    c |= (uint32_t)meet(p0, p1, r) << 15 | (uint32_t)meet(m0, m1, r) << 14;
    cx |= c;
  }
  // Segment [x0, x1) of color clocks on frame-relative line `line`.
  __device__ __forceinline__ void collide_segment(uint32_t live, uint32_t line, uint32_t x0, uint32_t x1) {
    if (x1 <= 68) return;
    uint32_t lo = x0 > 68 ? x0 - 68 : 0, hi = x1 - 68;
    if (L0 + line == bar_line && lo < 8) lo = 8;
    if (lo < hi) collide_cols(live, lo, hi);
  }
  // Account collisions for every color clock in [ceval, upto).
  __device__ void cx_eval(uint32_t upto) {
    uint32_t from = ceval;
    if (upto <= from) return;
    ceval = upto;
    if (vblank & 2) return;
    uint32_t live = live_objects();
    if (__popc(live) < 2) return;
    uint32_t la = from / 228u, xa = from - la * 228u;
    uint32_t lb = upto / 228u, xb = upto - lb * 228u;
    if (la == lb) {
      collide_segment(live, la, xa, xb);
    } else {
      collide_segment(live, la, xa, 228);
      if (lb > la + 1) collide_segment(live, la + 1, 0, 228);  // state is constant: one full line stands for all
      if (xb) collide_segment(live, lb, 0, xb);
    }
  }

  // ---- TIA ----
  __device__ __forceinline__ static uint32_t res_pos(uint32_t eff, uint32_t add, uint32_t hblank_pos) {
    uint32_t x = eff % 228u;
    if (x < 68) return hblank_pos;
    uint32_t p = x - 68 + add;
    return p >= 160 ? p - 160 : p;
  }
  __device__ __forceinline__ static uint32_t hm_move(uint32_t pos, uint32_t hm) {
    int s = (int)((hm >> 4) & 0xF);
    if (s >= 8) s -= 16;
    int p = (int)pos - s;
    if (p < 0) p += 160;
    if (p >= 160) p -= 160;
    return (uint32_t)p;
  }
  __device__ void tia_write(uint32_t reg, uint32_t v, uint32_t t) {
    uint32_t eff = 3u * (t + 1u);
    if ((COLL_REGS >> reg) & 1ull) cx_eval(eff);
    if (log.rec && ((LOG_REGS >> reg) & 1ull)) {
      if (log.n < log.cap) log.rec[log.n] = eff << 14 | reg << 8 | v;
      else status |= ST_LOG_OVERFLOW;
      log.n++;
    }
    switch (reg) {
      case 0x00:
        if (!(vsync & 2) && (v & 2)) { vs_rise = 1; vs_rise_kf = t; }
        vsync = v; break;
      case 0x01:
        vblank = v;
        if (!(v & 0x40)) inpt4_latch = 0;
        else if (fire) inpt4_latch = 1;
        break;
      case 0x02: wsync = 1; break;
      case 0x04: nusiz0 = v; break;
      case 0x05: nusiz1 = v; break;
      case 0x06: colup0 = v; break;
      case 0x07: colup1 = v; break;
      case 0x08: colupf = v; break;
      case 0x09: colubk = v; break;
      case 0x0A: ctrlpf = v; break;
      case 0x0B: refp0 = v; break;
      case 0x0C: refp1 = v; break;
      case 0x0D: pf0 = v; break;
      case 0x0E: pf1 = v; break;
      case 0x0F: pf2 = v; break;
      case 0x10: pos_p0 = res_pos(eff, 5, 3); break;
      case 0x11: pos_p1 = res_pos(eff, 5, 3); break;
      case 0x12: pos_m0 = res_pos(eff, 4, 2); break;
      case 0x13: pos_m1 = res_pos(eff, 4, 2); break;
      case 0x14: pos_bl = res_pos(eff, 4, 2); break;
      case 0x1B: grp0_new = v; grp1_old = grp1_new; break;
      case 0x1C: grp1_new = v; grp0_old = grp0_new; enabl_old = enabl_new; break;
      case 0x1D: enam0 = v; break;
      case 0x1E: enam1 = v; break;
      case 0x1F: enabl_new = v; break;
      case 0x20: hmp0 = v; break;
      case 0x21: hmp1 = v; break;
      case 0x22: hmm0 = v; break;
      case 0x23: hmm1 = v; break;
      case 0x24: hmbl = v; break;
      case 0x25: vdelp0 = v; break;
      case 0x26: vdelp1 = v; break;
      case 0x27: vdelbl = v; break;
      case 0x28:
        if ((resmp0 & 2) && !(v & 2)) {
          uint32_t sc = (nusiz0 & 7) == 5 ? 8u : (nusiz0 & 7) == 7 ? 16u : 4u;
          pos_m0 = (pos_p0 + sc) % 160u;
        }
        resmp0 = v; break;
      case 0x29:
        if ((resmp1 & 2) && !(v & 2)) {
          uint32_t sc = (nusiz1 & 7) == 5 ? 8u : (nusiz1 & 7) == 7 ? 16u : 4u;
          pos_m1 = (pos_p1 + sc) % 160u;
        }
        resmp1 = v; break;
      case 0x2A:
        pos_p0 = hm_move(pos_p0, hmp0); pos_p1 = hm_move(pos_p1, hmp1);
        pos_m0 = hm_move(pos_m0, hmm0); pos_m1 = hm_move(pos_m1, hmm1); pos_bl = hm_move(pos_bl, hmbl);
        if (eff % 228u < 68u) bar_line = L0 + eff / 228u;
        break;
      case 0x2B: hmp0 = hmp1 = hmm0 = hmm1 = hmbl = 0; break;
      case 0x2C:
        if (eff > ceval) ceval = eff;
        cx = 0;
        break;
      default: break;  // RSYNC, audio, unused addresses
    }
  }
  __device__ uint32_t tia_read(uint32_t reg, uint32_t t) {
    if (reg < 8) {
      cx_eval(3u * t);
      return (((cx >> (2 * reg + 1)) & 1u) << 7) | (((cx >> (2 * reg)) & 1u) << 6);
    }
    if (reg == 0x0C) return (fire || inpt4_latch) ? 0x00u : 0x80u;
    if (reg == 0x0D) return 0x80u;
    return 0;
  }

  // ---- RIOT ----
  __device__ uint32_t riot_read(uint32_t addr, uint32_t t) {
    if (!(addr & 4)) {
      switch (addr & 3) {
        case 0: return ((swcha_out & swacnt) | (joy & ~swacnt)) & 0xFF;
        case 1: return swacnt;
        case 2: return ((swchb_out & swbcnt) | (0x0Bu & ~swbcnt)) & 0xFF;
        default: return swbcnt;
      }
    }
    uint64_t now = 76ull * L0 + t;
    uint64_t n = now - (tim_cw + 1);
    uint64_t span = (uint64_t)(tim_v + 1) << tim_shift;
    if (addr & 1) return n >= span ? 0x80u : 0u;
    if (n < span) return tim_v - (uint32_t)(n >> tim_shift);
    return (uint32_t)(0xFFull - (n - span)) & 0xFF;
  }
  __device__ void riot_write(uint32_t addr, uint32_t v, uint32_t t) {
    if (!(addr & 4)) {
      switch (addr & 3) {
        case 0: swcha_out = v; break;
        case 1: swacnt = v; break;
        case 2: swchb_out = v; break;
        default: swbcnt = v; break;
      }
      return;
    }
    if (addr & 0x10) {
      tim_v = v;
      uint32_t sel = addr & 3;
      tim_shift = sel == 0 ? 0 : sel == 1 ? 3 : sel == 2 ? 6 : 10;
      tim_cw = 76ull * L0 + t;
    }
  }

  // ---- cartridge and bus ----
  __device__ __forceinline__ void hotspot(uint32_t off) {
    if (scheme == 1) { if (off == 0xFF8 || off == 0xFF9) bank = off - 0xFF8; }
    else if (scheme == 2) { if (off >= 0xFF6 && off <= 0xFF9) bank = off - 0xFF6; }
    else if (scheme == 3) { if (off >= 0xFF4 && off <= 0xFFB) bank = off - 0xFF4; }
  }
  __device__ __forceinline__ uint32_t rd(uint32_t addr, uint32_t t) {
    addr &= 0x1FFF;
    if (addr & 0x1000) {
      uint32_t off = addr & 0xFFF;
      if (scheme) hotspot(off);
      return mem.rom_rd(bank * 4096u + off);
    }
    if (!(addr & 0x80)) return tia_read(addr & 0x0F, t);
    if (!(addr & 0x200)) return mem.ram_rd(addr & 0x7F);
    return riot_read(addr, t);
  }
  __device__ __forceinline__ void wr(uint32_t addr, uint32_t v, uint32_t t) {
    addr &= 0x1FFF;
    if (addr & 0x1000) { if (scheme) hotspot(addr & 0xFFF); return; }
    if (!(addr & 0x80)) { tia_write(addr & 0x3F, v, t); return; }
    if (!(addr & 0x200)) { mem.ram_wr(addr & 0x7F, v); return; }
    riot_write(addr, v, t);
  }

  // ---- flags ----
  __device__ __forceinline__ void nz(uint32_t v) { P = (P & ~0x82u) | (v & 0x80u) | ((v & 0xFF) ? 0u : 2u); }

  __device__ __forceinline__ void adc(uint32_t v) {
    uint32_t c = P & 1u;
    if (!(P & 0x08)) {
      uint32_t s = A + v + c;
      uint32_t r = s & 0xFF;
      uint32_t ov = (~(A ^ v) & (A ^ r)) & 0x80u;
      P = (P & ~0xC3u) | (s > 0xFF ? 1u : 0u) | (ov ? 0x40u : 0u) | (r & 0x80u) | (r ? 0u : 2u);
      A = r;
      return;
    }
    // decimal mode (NMOS): low nibble adjust, N/V from the signed intermediate,
    // high adjust and carry on the unsigned one, Z from the binary sum
    uint32_t zb = (A + v + c) & 0xFF;
    int lo = (int)(A & 0x0F) + (int)(v & 0x0F) + (int)c;
    if (lo > 9) lo = ((lo + 6) & 0x0F) + 0x10;
    int hs = (int)(int8_t)(uint8_t)(A & 0xF0) + (int)(int8_t)(uint8_t)(v & 0xF0) + lo;
    int hu = (int)(A & 0xF0) + (int)(v & 0xF0) + lo;
    uint32_t np = P & ~0xC3u;
    if (hs & 0x80) np |= 0x80;
    if (hs > 127 || hs < -128) np |= 0x40;
    if (hu >= 0xA0) hu += 0x60;
    if (hu > 0xFF) np |= 1;
    if (!zb) np |= 2;
    P = np;
    A = (uint32_t)hu & 0xFF;
  }
  __device__ __forceinline__ void sbc(uint32_t v) {
    uint32_t c = P & 1u;
    uint32_t nv = v ^ 0xFF;
    uint32_t s = A + nv + c;  // binary difference and flags (also the decimal flags)
    uint32_t r = s & 0xFF;
    uint32_t ov = (~(A ^ nv) & (A ^ r)) & 0x80u;
    uint32_t np = (P & ~0xC3u) | (s > 0xFF ? 1u : 0u) | (ov ? 0x40u : 0u) | (r & 0x80u) | (r ? 0u : 2u);
    if (P & 0x08) {
      int lo = (int)(A & 0x0F) - (int)(v & 0x0F) + (int)c - 1;
      if (lo < 0) lo = ((lo - 6) & 0x0F) - 0x10;
      int hi = (int)(A & 0xF0) - (int)(v & 0xF0) + lo;
      if (hi < 0) hi -= 0x60;
      r = (uint32_t)hi & 0xFF;
    }
    P = np;
    A = r;
  }
  __device__ __forceinline__ void cmp(uint32_t reg, uint32_t v) {
    uint32_t d = (reg - v) & 0xFF;
    P = (P & ~0x83u) | (reg >= v ? 1u : 0u) | (d & 0x80u) | (d ? 0u : 2u);
  }
  __device__ __forceinline__ void push(uint32_t v, uint32_t t) { wr(0x100u | SP, v, t); SP = (SP - 1) & 0xFF; }
  __device__ __forceinline__ uint32_t pull(uint32_t t) { SP = (SP + 1) & 0xFF; return rd(0x100u | SP, t); }

  // ---- one instruction ----
  __device__ void exec() {
    const uint32_t k0 = kf;
    wsync = 0;
    vs_rise = 0;
    const uint32_t pc = PC;
    const uint32_t opcode = rd(pc, k0);
    const uint32_t d = dec[opcode];
    const uint32_t op = d & 0xFF, mode = (d >> 8) & 0xF;
    uint32_t n = (d >> 12) & 15;
    if (op == O_JAM) { jam = 1; status |= ST_ILLEGAL; return; }
    uint32_t b1 = 0, b2 = 0, ea = 0, cross = 0;
    switch (mode) {
      case IMP: case ACC: PC = (pc + 1) & 0xFFFF; break;
      case IMM: b1 = rd(pc + 1, k0); PC = (pc + 2) & 0xFFFF; break;
      case ZP: b1 = rd(pc + 1, k0); ea = b1; PC = (pc + 2) & 0xFFFF; break;
      case ZPX: b1 = rd(pc + 1, k0); ea = (b1 + X) & 0xFF; PC = (pc + 2) & 0xFFFF; break;
      case ZPY: b1 = rd(pc + 1, k0); ea = (b1 + Y) & 0xFF; PC = (pc + 2) & 0xFFFF; break;
      case ABS: b1 = rd(pc + 1, k0); b2 = rd(pc + 2, k0); ea = b1 | b2 << 8; PC = (pc + 3) & 0xFFFF; break;
      case ABX: { b1 = rd(pc + 1, k0); b2 = rd(pc + 2, k0); uint32_t b = b1 | b2 << 8; ea = (b + X) & 0xFFFF;
                  cross = (b ^ ea) >> 8; PC = (pc + 3) & 0xFFFF; break; }
      case ABY: { b1 = rd(pc + 1, k0); b2 = rd(pc + 2, k0); uint32_t b = b1 | b2 << 8; ea = (b + Y) & 0xFFFF;
                  cross = (b ^ ea) >> 8; PC = (pc + 3) & 0xFFFF; break; }
      case IND: { b1 = rd(pc + 1, k0); b2 = rd(pc + 2, k0); uint32_t p = b1 | b2 << 8;
                  uint32_t lo = rd(p, k0), hi = rd((p & 0xFF00) | ((p + 1) & 0xFF), k0);
                  ea = lo | hi << 8; PC = (pc + 3) & 0xFFFF; break; }
      case IZX: { b1 = rd(pc + 1, k0); uint32_t z = (b1 + X) & 0xFF;
                  uint32_t lo = rd(z, k0), hi = rd((z + 1) & 0xFF, k0); ea = lo | hi << 8; PC = (pc + 2) & 0xFFFF; break; }
      case IZY: { b1 = rd(pc + 1, k0); uint32_t lo = rd(b1, k0), hi = rd((b1 + 1) & 0xFF, k0);
                  uint32_t b = lo | hi << 8; ea = (b + Y) & 0xFFFF; cross = (b ^ ea) >> 8; PC = (pc + 2) & 0xFFFF; break; }
      case REL: b1 = rd(pc + 1, k0); PC = (pc + 2) & 0xFFFF; ea = (PC + (uint32_t)(int32_t)(int8_t)(uint8_t)b1) & 0xFFFF; break;
    }
    if (cross && ((d >> 16) & 1)) n++;
    instret++;
    if (mode == REL) {
      uint32_t take;
      switch (op) {
        case O_BCC: take = !(P & 0x01); break;
        case O_BCS: take = P & 0x01; break;
        case O_BNE: take = !(P & 0x02); break;
        case O_BEQ: take = P & 0x02; break;
        case O_BVC: take = !(P & 0x40); break;
        case O_BVS: take = P & 0x40; break;
        case O_BPL: take = !(P & 0x80); break;
        default: take = P & 0x80; break;  // BMI
      }
      if (take) {
        n += ((PC ^ ea) & 0xFF00) ? 2u : 1u;
        PC = ea;
      }
      kf = k0 + n;
      return;
    }
    const uint32_t kA = k0 + n - 1;
    switch (op) {
      case O_LDA: A = mode == IMM ? b1 : rd(ea, kA); nz(A); break;
      case O_LDX: X = mode == IMM ? b1 : rd(ea, kA); nz(X); break;
      case O_LDY: Y = mode == IMM ? b1 : rd(ea, kA); nz(Y); break;
      case O_STA: wr(ea, A, kA); break;
      case O_STX: wr(ea, X, kA); break;
      case O_STY: wr(ea, Y, kA); break;
      case O_ADC: adc(mode == IMM ? b1 : rd(ea, kA)); break;
      case O_SBC: sbc(mode == IMM ? b1 : rd(ea, kA)); break;
      case O_AND: A &= mode == IMM ? b1 : rd(ea, kA); nz(A); break;
      case O_ORA: A |= mode == IMM ? b1 : rd(ea, kA); nz(A); break;
      case O_EOR: A ^= mode == IMM ? b1 : rd(ea, kA); nz(A); break;
      case O_CMP: cmp(A, mode == IMM ? b1 : rd(ea, kA)); break;
      case O_CPX: cmp(X, mode == IMM ? b1 : rd(ea, kA)); break;
      case O_CPY: cmp(Y, mode == IMM ? b1 : rd(ea, kA)); break;
      case O_BIT: { uint32_t v = rd(ea, kA); P = (P & ~0xC2u) | (v & 0xC0u) | ((A & v) ? 0u : 2u); break; }
      case O_ASL: case O_LSR: case O_ROL: case O_ROR: case O_INC: case O_DEC: {
        uint32_t old = mode == ACC ? A : rd(ea, kA - 2);
        uint32_t r, c = P & 1u;
        switch (op) {
          case O_ASL: r = (old << 1) & 0xFF; c = old >> 7; break;
          case O_LSR: r = old >> 1; c = old & 1; break;
          case O_ROL: r = ((old << 1) | (P & 1u)) & 0xFF; c = old >> 7; break;
          case O_ROR: r = (old >> 1) | ((P & 1u) << 7); c = old & 1; break;
          case O_INC: r = (old + 1) & 0xFF; break;
          default: r = (old - 1) & 0xFF; break;
        }
        P = (P & ~1u) | c;
        nz(r);
        if (mode == ACC) A = r;
        else { wr(ea, old, kA - 1); wr(ea, r, kA); }
        break;
      }
      case O_SLO: case O_RLA: case O_SRE: case O_RRA: case O_DCP: case O_ISC: {
        // read-modify-write of memory (both writes), then the accumulator operation
        const uint32_t old = rd(ea, kA - 2);
        uint32_t r, c = P & 1u;
        switch (op) {
          case O_SLO: r = (old << 1) & 0xFF; c = old >> 7; break;
          case O_RLA: r = ((old << 1) | (P & 1u)) & 0xFF; c = old >> 7; break;
          case O_SRE: r = old >> 1; c = old & 1; break;
          case O_RRA: r = (old >> 1) | ((P & 1u) << 7); c = old & 1; break;
          case O_DCP: r = (old - 1) & 0xFF; break;
          default: r = (old + 1) & 0xFF; break;
        }
        wr(ea, old, kA - 1);
        wr(ea, r, kA);
        switch (op) {
          case O_SLO: A |= r; P = (P & ~1u) | c; nz(A); break;
          case O_RLA: A &= r; P = (P & ~1u) | c; nz(A); break;
          case O_SRE: A ^= r; P = (P & ~1u) | c; nz(A); break;
          case O_RRA: P = (P & ~1u) | c; adc(r); break;
          case O_DCP: cmp(A, r); break;
          default: sbc(r); break;
        }
        break;
      }
      case O_SAX: wr(ea, A & X, kA); break;
      case O_LAX: A = rd(ea, kA); X = A; nz(A); break;
      case O_ANC: A &= b1; nz(A); P = (P & ~1u) | (A >> 7); break;
      case O_ALR: A &= b1; P = (P & ~1u) | (A & 1u); A >>= 1; nz(A); break;
      case O_SBX: { const uint32_t ax = A & X; P = (P & ~1u) | (ax >= b1 ? 1u : 0u); X = (ax - b1) & 0xFF; nz(X); break; }
      case O_NOP: if (mode != IMP && mode != IMM) (void)rd(ea, kA); break;  // the operand read
      case O_INX: X = (X + 1) & 0xFF; nz(X); break;
      case O_INY: Y = (Y + 1) & 0xFF; nz(Y); break;
      case O_DEX: X = (X - 1) & 0xFF; nz(X); break;
      case O_DEY: Y = (Y - 1) & 0xFF; nz(Y); break;
      case O_TAX: X = A; nz(X); break;
      case O_TAY: Y = A; nz(Y); break;
      case O_TXA: A = X; nz(A); break;
      case O_TYA: A = Y; nz(A); break;
      case O_TSX: X = SP; nz(X); break;
      case O_TXS: SP = X; break;
      case O_CLC: P &= ~0x01u; break;
      case O_SEC: P |= 0x01u; break;
      case O_CLI: P &= ~0x04u; break;
      case O_SEI: P |= 0x04u; break;
      case O_CLV: P &= ~0x40u; break;
      case O_CLD: P &= ~0x08u; break;
      case O_SED: P |= 0x08u; break;
      case O_PHA: push(A, kA); break;
      case O_PHP: push(P | 0x30u, kA); break;
      case O_PLA: A = pull(kA); nz(A); break;
      case O_PLP: P = (pull(kA) & ~0x10u) | 0x20u; break;
      case O_JMP: PC = ea; break;
      case O_JSR: { uint32_t ret = (pc + 2) & 0xFFFF; push(ret >> 8, kA); push(ret & 0xFF, kA); PC = ea; break; }
      case O_RTS: { uint32_t lo = pull(kA); uint32_t hi = pull(kA); PC = ((lo | hi << 8) + 1) & 0xFFFF; break; }
      case O_RTI: { P = (pull(kA) & ~0x10u) | 0x20u; uint32_t lo = pull(kA); uint32_t hi = pull(kA); PC = lo | hi << 8; break; }
      case O_BRK: {
        uint32_t ret = (pc + 2) & 0xFFFF;
        push(ret >> 8, kA); push(ret & 0xFF, kA); push(P | 0x30u, kA);
        P |= 0x04u;
        uint32_t lo = rd(0x1FFE, kA), hi = rd(0x1FFF, kA);
        PC = lo | hi << 8;
        break;
      }
      default: break;
    }
    uint32_t k = k0 + n;
    if (wsync) k = ((k + 75u) / 76u) * 76u;
    kf = k;
  }

  // ---- one frame: until the VSYNC rise, the line cap, or a halted CPU ----
  // Returns the number of lines in the frame.
  __device__ uint32_t run_frame() {
    uint32_t next_rel;
    for (;;) {
      if (jam) { next_rel = kf / 76u; break; }
      exec();
      if (jam) { next_rel = kf / 76u; break; }
      if (vs_rise) { next_rel = vs_rise_kf / 76u; break; }
      if (kf >= 76u * CAP_LINES) { status |= ST_FRAME_CAP; next_rel = kf / 76u; break; }
    }
    cx_eval(3u * kf);
    L0 += next_rel;
    kf -= 76u * next_rel;
    ceval -= 228u * next_rel;
    frame_no++;
    return next_rel;
  }
};

}  // namespace atari
