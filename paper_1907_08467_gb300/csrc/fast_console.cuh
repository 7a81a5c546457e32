// Console for the batched form, laid out for the issue rate of sm_103a.
//
// Same machine and canonical state as Console in device_machine.cuh:
//   - the hot loop is a single switch on the opcode byte; every case has its
//     addressing mode and cycle count folded in;
//   - CPU registers (flags split, N and Z kept as the last result byte),
//     the cycle counter and the bank in registers;
//   - RAM (bytes), the TIA register file (bytes) and the I/O state
//     (collision cursor and latches, RIOT timer and ports, inputs, log
//     cursor, frame base line) in shared memory, one block per env with odd
//     word strides, so lanes reading the same field never bank-conflict and
//     every access is a base pointer plus an offset;
//   - the block's cartridge staged in shared memory as bytes (16 KB for an
//     F6 cartridge); an instruction's bytes are fetched as two aligned words
//     joined by one funnel shift.
// Instructions the hot switch does not take (BRK, RTI, JMP (ind), undocumented
// opcodes, stack or pointer bytes outside RAM, fetches outside the cartridge
// or next to a bank hotspot) run the general decoder out of line.
#pragma once
#include <cstdint>

#include "device_machine.cuh"

namespace atari {

enum TiaSlot : uint32_t {
  T_VSYNC = 0, T_VBLANK, T_NUSIZ0, T_NUSIZ1, T_COLUP0, T_COLUP1, T_COLUPF, T_COLUBK, T_CTRLPF, T_REFP0,
  T_REFP1, T_PF0, T_PF1, T_PF2, T_ENAM0, T_ENAM1, T_ENABL_N, T_ENABL_O, T_GRP0_N, T_GRP0_O, T_GRP1_N,
  T_GRP1_O, T_VDELP0, T_VDELP1, T_VDELBL, T_RESMP0, T_RESMP1, T_HMP0, T_HMP1, T_HMM0, T_HMM1, T_HMBL,
  T_P0, T_P1, T_M0, T_M1, T_BL
};
// I/O state words (shared memory, interleaved by env)
enum IoWord : uint32_t {
  IO_CEVAL = 0, IO_CX, IO_L0LO, IO_L0HI, IO_BARLO, IO_BARHI, IO_TCWLO, IO_TCWHI, IO_TV, IO_TSH, IO_PORTS,
  IO_JOY, IO_FIRE, IO_LATCH, IO_LOGLO, IO_LOGHI, IO_LOGN, IO_LOGCAP, IO_STATUS,
  IO_BANDN,      // next quarter-frame band whose start snapshot is due (1..3), 4: none
  IO_BSLO, IO_BSHI,  // where this frame's band snapshots go (3 x 64 bytes)
  IO_QHEAD, IO_QTAIL, IO_ACK,  // split form: TIA event queue cursors and the TIA side's acknowledgements
  IO_WORDS
};
constexpr uint32_t IO_WSYNC = 1u, IO_VSYNC_RISE = 2u;


// Per-env blocks of shared memory, env-major, with strides chosen so that a
// warp's lanes touching the same field hit 32 different banks: RAM 128 bytes
// padded to 132 (33 words), I/O state IO_WORDS words, TIA file 44 bytes (11
// words).  Every access is the lane's base plus a constant or one add.  Bytes
// rather than one word per RAM byte keep a 64-env work item small enough for
// four blocks per SM.
constexpr uint32_t RAM_BYTES = 132, IO_STRIDE = IO_WORDS, TIA_STRIDE = 44;
static_assert(IO_STRIDE % 2 == 1 && (TIA_STRIDE / 4) % 2 == 1 && (RAM_BYTES / 4) % 2 == 1 && RAM_BYTES % 4 == 0,
              "odd word strides");
constexpr uint32_t ENV_SMEM = RAM_BYTES + 4 * IO_STRIDE + TIA_STRIDE;
// bytes per cartridge in the batched form's device copy (up to eight 4 KB banks, F4)
constexpr uint32_t ROMB_SLOT = 32768;

// Shared-memory views of one env's TIA file and I/O state.  The pointers
// reach the out-of-line I/O functions as plain pointers; the assumption lets
// the compiler address them as shared memory there too.
struct IoCtx {
  uint8_t *tia;
  uint32_t *io;
  __device__ __forceinline__ uint8_t *t() const { __builtin_assume(__isShared(tia)); return tia; }
  __device__ __forceinline__ uint32_t *w() const { __builtin_assume(__isShared(io)); return io; }
  __device__ __forceinline__ uint32_t T(uint32_t s) const { return t()[s]; }
  __device__ __forceinline__ void Tset(uint32_t s, uint32_t v) const { t()[s] = (uint8_t)v; }
  __device__ __forceinline__ uint32_t G(uint32_t i) const { return w()[i]; }
  __device__ __forceinline__ void Sset(uint32_t i, uint32_t v) const { w()[i] = v; }
  __device__ __forceinline__ uint64_t G64(uint32_t i) const { return (uint64_t)w()[i] | (uint64_t)w()[i + 1] << 32; }
  __device__ __forceinline__ void S64(uint32_t i, uint64_t v) const {
    w()[i] = (uint32_t)v;
    w()[i + 1] = (uint32_t)(v >> 32);
  }
};

// ---------------------------------------------------------------- collisions (cold)
__device__ __noinline__ uint32_t fc_collide_cols(IoCtx c, uint32_t live, uint32_t lo, uint32_t hi) {
  M160 r{range_word(0, lo, hi), range_word(1, lo, hi), range_word(2, lo, hi), range_word(3, lo, hi),
         range_word(4, lo, hi)};
  M160 z{0, 0, 0, 0, 0};
  const uint32_t nus0 = c.T(T_NUSIZ0), nus1 = c.T(T_NUSIZ1), ctrl = c.T(T_CTRLPF);
  M160 p0 = (live & 1) ? player_mask((c.T(T_VDELP0) & 1) ? c.T(T_GRP0_O) : c.T(T_GRP0_N), c.T(T_REFP0), nus0,
                                     c.T(T_P0))
                       : z;
  M160 p1 = (live & 2) ? player_mask((c.T(T_VDELP1) & 1) ? c.T(T_GRP1_O) : c.T(T_GRP1_N), c.T(T_REFP1), nus1,
                                     c.T(T_P1))
                       : z;
  M160 m0 = (live & 4) ? missile_mask(nus0, c.T(T_M0)) : z;
  M160 m1 = (live & 8) ? missile_mask(nus1, c.T(T_M1)) : z;
  M160 b = (live & 16) ? ball_mask(ctrl, c.T(T_BL)) : z;
  M160 f = (live & 32) ? pf_mask(c.T(T_PF0), c.T(T_PF1), c.T(T_PF2), ctrl) : z;
  uint32_t x = 0;
  x |= (uint32_t)meet(m0, p1, r) << 1 | (uint32_t)meet(m0, p0, r) << 0;
  x |= (uint32_t)meet(m1, p0, r) << 3 | (uint32_t)meet(m1, p1, r) << 2;
  x |= (uint32_t)meet(p0, f, r) << 5 | (uint32_t)meet(p0, b, r) << 4;
  x |= (uint32_t)meet(p1, f, r) << 7 | (uint32_t)meet(p1, b, r) << 6;
  x |= (uint32_t)meet(m0, f, r) << 9 | (uint32_t)meet(m0, b, r) << 8;
  x |= (uint32_t)meet(m1, f, r) << 11 | (uint32_t)meet(m1, b, r) << 10;
  x |= (uint32_t)meet(b, f, r) << 13;
  x |= (uint32_t)meet(p0, p1, r) << 15 | (uint32_t)meet(m0, m1, r) << 14;
  return x;
}

__device__ __forceinline__ uint32_t fc_live(IoCtx c) {
  const uint32_t g0 = (c.T(T_VDELP0) & 1) ? c.T(T_GRP0_O) : c.T(T_GRP0_N);
  const uint32_t g1 = (c.T(T_VDELP1) & 1) ? c.T(T_GRP1_O) : c.T(T_GRP1_N);
  const uint32_t eb = (c.T(T_VDELBL) & 1) ? c.T(T_ENABL_O) : c.T(T_ENABL_N);
  return (g0 ? 1u : 0u) | (g1 ? 2u : 0u) | (((c.T(T_ENAM0) & 2) && !(c.T(T_RESMP0) & 2)) ? 4u : 0u) |
         (((c.T(T_ENAM1) & 2) && !(c.T(T_RESMP1) & 2)) ? 8u : 0u) | ((eb & 2) ? 16u : 0u) |
         (((c.T(T_PF0) & 0xF0) | c.T(T_PF1) | c.T(T_PF2)) ? 32u : 0u);
}

// Account collisions for every color clock in [ceval, upto) (frame-relative).
__device__ __forceinline__ void fc_cx_eval(IoCtx c, uint32_t upto) {
  const uint32_t from = c.G(IO_CEVAL);
  if (upto <= from) return;
  c.Sset(IO_CEVAL, upto);
  if (c.T(T_VBLANK) & 2) return;
  const uint32_t la = from / 228u, xa = from - la * 228u;
  const uint32_t lb = upto / 228u, xb = upto - lb * 228u;
  if (la == lb && xb <= 68) return;  // the span lies in one line's horizontal blank
  const uint32_t live = fc_live(c);
  if (__popc(live) < 2) return;
  const uint64_t L0 = c.G64(IO_L0LO), bar = c.G64(IO_BARLO);
  uint32_t x = 0;
  auto seg = [&](uint32_t line, uint32_t x0, uint32_t x1) {
    if (x1 <= 68) return;
    uint32_t lo = x0 > 68 ? x0 - 68 : 0, hi = x1 - 68;
    if (L0 + line == bar && lo < 8) lo = 8;
    if (lo < hi) x |= fc_collide_cols(c, live, lo, hi);
  };
  if (la == lb) {
    seg(la, xa, xb);
  } else {
    seg(la, xa, 228);
    if (lb > la + 1) seg(la + 1, 0, 228);
    if (xb) seg(lb, 0, xb);
  }
  c.Sset(IO_CX, c.G(IO_CX) | x);
}

// ---------------------------------------------------------------- I/O (cold)
__device__ __forceinline__ uint32_t fc_res_pos(uint32_t eff, uint32_t add, uint32_t hb) {
  const uint32_t x = eff % 228u;
  if (x < 68) return hb;
  const uint32_t p = x - 68 + add;
  return p >= 160 ? p - 160 : p;
}
__device__ __forceinline__ uint32_t fc_hm_move(uint32_t pos, uint32_t hm) {
  int s = (int)((hm >> 4) & 0xF);
  if (s >= 8) s -= 16;
  int p = (int)pos - s;
  p += p < 0 ? 160 : 0;
  p -= p >= 160 ? 160 : 0;
  return (uint32_t)p;
}

// Read a TIA or RIOT address (13-bit, neither RAM nor cartridge) at cycle t.
// Read a RIOT address (ports, timer) at absolute CPU cycle `now`.
__device__ __forceinline__ uint32_t fc_riot_read(IoCtx c, uint32_t a, uint64_t now) {
  const uint32_t ports = c.G(IO_PORTS);
  if (!(a & 4)) {
    const uint32_t sh = 8 * (a & 2);             // SWCHA/SWACNT in bytes 0/1, SWCHB/SWBCNT in 2/3
    const uint32_t out = (ports >> sh) & 0xFF, ddr = (ports >> (sh + 8)) & 0xFF;
    if (a & 1) return ddr;
    const uint32_t pins = (a & 2) ? 0x0Bu : c.G(IO_JOY);
    return ((out & ddr) | (pins & ~ddr)) & 0xFF;
  }
  const uint64_t n = now - (c.G64(IO_TCWLO) + 1);
  const uint32_t tv = c.G(IO_TV), sh = c.G(IO_TSH);
  const uint64_t span = (uint64_t)(tv + 1) << sh;
  if (a & 1) return n >= span ? 0x80u : 0u;
  if (n < span) return tv - (uint32_t)(n >> sh);
  return (uint32_t)(0xFFull - (n - span)) & 0xFF;
}
// Collision-latch byte of TIA read register reg (0..7) from the CX word.
__device__ __forceinline__ uint32_t fc_cx_byte(uint32_t cx, uint32_t reg) {
  return (((cx >> (2 * reg + 1)) & 1u) << 7) | (((cx >> (2 * reg)) & 1u) << 6);
}
// Read a TIA or RIOT address (13-bit, neither RAM nor cartridge) at cycle t.
__device__ __noinline__ uint32_t fc_io_read(IoCtx c, uint32_t a, uint32_t t) {
  if (!(a & 0x80)) {
    const uint32_t reg = a & 0x0F;
    if (reg < 8) {
      fc_cx_eval(c, 3u * t);
      return fc_cx_byte(c.G(IO_CX), reg);
    }
    if (reg == 0x0C) return (c.G(IO_FIRE) || c.G(IO_LATCH)) ? 0x00u : 0x80u;
    if (reg == 0x0D) return 0x80u;
    return 0;
  }
  return fc_riot_read(c, a, 76ull * c.G64(IO_L0LO) + t);
}

// 64-byte render snapshot: TIA file (canonical bytes 0x20..0x44), HMOVE bar
// line, frame base line; word 14 = the number of log records before it.
__device__ __forceinline__ void fc_snapshot(IoCtx c, uint8_t *o, uint32_t nrec) {
  uint32_t v[16];
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    uint32_t x = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (q * 4 + b < 37) x |= c.T(q * 4 + b) << (8 * b);
    v[q] = x;
  }
  v[9] &= 0xFFu;
  v[10] = c.G(IO_BARLO); v[11] = c.G(IO_BARHI);
  v[12] = c.G(IO_L0LO); v[13] = c.G(IO_L0HI);
  v[14] = nrec; v[15] = 0;
  uint4 *d = reinterpret_cast<uint4 *>(o);
#pragma unroll
  for (int q = 0; q < 4; ++q) d[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// First color clock of quarter-frame band q (rows 210 q / 4 of the window).
__device__ __forceinline__ uint32_t fc_band_clk(uint32_t q) { return 228u * (WINDOW_Y0 + (FRAME_H * q) / 4u); }

// Snapshot the render state at the start of every band due by clock eff: the
// state after all records of earlier clocks, so the rasteriser's warps start
// their bands there instead of replaying the frame from its first record.
__device__ __noinline__ void fc_band_snap(IoCtx c, uint32_t eff) {
  uint32_t bn = c.G(IO_BANDN);
  uint8_t *base = reinterpret_cast<uint8_t *>((uint64_t)c.G(IO_BSLO) | (uint64_t)c.G(IO_BSHI) << 32);
  const uint32_t nrec = c.G(IO_LOGN);
  while (bn < 4 && eff >= fc_band_clk(bn)) {
    fc_snapshot(c, base + (bn - 1) * 64, nrec);
    ++bn;
  }
  c.Sset(IO_BANDN, bn);
}

// Log the frame's TIA writes to p (cap records; p null: no log); bands:
// where the three quarter-frame start snapshots go, or null for none.
__device__ __forceinline__ void fc_set_log(IoCtx c, uint32_t *p, uint32_t cap, uint8_t *bands) {
  c.Sset(IO_LOGLO, (uint32_t)(uint64_t)p);
  c.Sset(IO_LOGHI, (uint32_t)((uint64_t)p >> 32));
  c.Sset(IO_LOGN, 0);
  c.Sset(IO_LOGCAP, cap);
  c.Sset(IO_BANDN, bands ? 1u : 4u);
  c.Sset(IO_BSLO, (uint32_t)(uint64_t)bands);
  c.Sset(IO_BSHI, (uint32_t)((uint64_t)bands >> 32));
}

// Append one TIA write record (effect clock, register, value) to the log of
// a rendered frame.
__device__ __forceinline__ void fc_log(IoCtx c, uint32_t eff, uint32_t reg, uint32_t v) {
  const uint32_t lo = c.G(IO_LOGLO), hi = c.G(IO_LOGHI);
  if (lo | hi) {
    if (c.G(IO_BANDN) < 4 && eff >= fc_band_clk(c.G(IO_BANDN))) fc_band_snap(c, eff);
    uint32_t *lp = reinterpret_cast<uint32_t *>((uint64_t)lo | (uint64_t)hi << 32);
    const uint32_t nrec = c.G(IO_LOGN);
    if (nrec < c.G(IO_LOGCAP)) lp[nrec] = eff << 14 | reg << 8 | v;
    else c.Sset(IO_STATUS, c.G(IO_STATUS) | ST_LOG_OVERFLOW);
    c.Sset(IO_LOGN, nrec + 1);
  }
}

// TIA registers whose writes only set a colour or a motion register: logged,
// no collision or timing effect (COLUP0, COLUP1, COLUPF, COLUBK, HMP0..HMBL).
constexpr uint64_t FAST_TIA_REGS = (0xFull << 0x06) | (0x1Full << 0x20);

// Write a RIOT address at absolute CPU cycle `now`.
__device__ __forceinline__ void fc_riot_write(IoCtx c, uint32_t a, uint32_t v, uint64_t now) {
  if (!(a & 4)) {
    const uint32_t sh = 8 * (a & 3);
    c.Sset(IO_PORTS, (c.G(IO_PORTS) & ~(0xFFu << sh)) | (v & 0xFF) << sh);
  } else if (a & 0x10) {
    const uint32_t sel = a & 3;
    c.Sset(IO_TV, v & 0xFF);
    c.Sset(IO_TSH, sel == 0 ? 0 : sel == 1 ? 3 : sel == 2 ? 6 : 10);
    c.S64(IO_TCWLO, now);
  }
}
// The TIA part of a write (register reg at cycle t): collisions up to the
// write, log record, register update.  cpu_latch: this thread also keeps the
// fire-button latch (the split form keeps it on the CPU side).
__device__ __forceinline__ uint32_t fc_tia_write(IoCtx c, uint32_t reg, uint32_t v, uint32_t t, bool cpu_latch) {
  const uint32_t eff = 3u * (t + 1u);
  if ((COLL_REGS >> reg) & 1ull) fc_cx_eval(c, eff);
  if ((LOG_REGS >> reg) & 1ull) fc_log(c, eff, reg, v);
  uint32_t flags = 0;
  switch (reg) {
    case 0x00:
      if (!(c.T(T_VSYNC) & 2) && (v & 2)) flags |= IO_VSYNC_RISE;
      c.Tset(T_VSYNC, v);
      break;
    case 0x01:
      c.Tset(T_VBLANK, v);
      if (cpu_latch) {
        if (!(v & 0x40)) c.Sset(IO_LATCH, 0);
        else if (c.G(IO_FIRE)) c.Sset(IO_LATCH, 1);
      }
      break;
    case 0x02: flags |= IO_WSYNC; break;
    case 0x04: case 0x05: case 0x06: case 0x07: case 0x08: case 0x09: case 0x0A: case 0x0B: case 0x0C:
    case 0x0D: case 0x0E: case 0x0F:
      c.Tset(reg - 2, v); break;                 // NUSIZ0 .. PF2 are slots 2 .. 13
    case 0x10: c.Tset(T_P0, fc_res_pos(eff, 5, 3)); break;
    case 0x11: c.Tset(T_P1, fc_res_pos(eff, 5, 3)); break;
    case 0x12: c.Tset(T_M0, fc_res_pos(eff, 4, 2)); break;
    case 0x13: c.Tset(T_M1, fc_res_pos(eff, 4, 2)); break;
    case 0x14: c.Tset(T_BL, fc_res_pos(eff, 4, 2)); break;
    case 0x1B: c.Tset(T_GRP1_O, c.T(T_GRP1_N)); c.Tset(T_GRP0_N, v); break;
    case 0x1C:
      c.Tset(T_GRP0_O, c.T(T_GRP0_N)); c.Tset(T_ENABL_O, c.T(T_ENABL_N)); c.Tset(T_GRP1_N, v); break;
    case 0x1D: c.Tset(T_ENAM0, v); break;
    case 0x1E: c.Tset(T_ENAM1, v); break;
    case 0x1F: c.Tset(T_ENABL_N, v); break;
    case 0x20: case 0x21: case 0x22: case 0x23: case 0x24: c.Tset(T_HMP0 + (reg - 0x20), v); break;
    case 0x25: c.Tset(T_VDELP0, v); break;
    case 0x26: c.Tset(T_VDELP1, v); break;
    case 0x27: c.Tset(T_VDELBL, v); break;
    case 0x28: case 0x29: {
      const uint32_t i = reg - 0x28;
      if ((c.T(T_RESMP0 + i) & 2) && !(v & 2)) {
        const uint32_t nus = c.T(T_NUSIZ0 + i);
        const uint32_t sc = (nus & 7) == 5 ? 8u : (nus & 7) == 7 ? 16u : 4u;
        c.Tset(T_M0 + i, (c.T(T_P0 + i) + sc) % 160u);
      }
      c.Tset(T_RESMP0 + i, v);
      break;
    }
    case 0x2A:
      for (uint32_t o = 0; o < 5; ++o) c.Tset(T_P0 + o, fc_hm_move(c.T(T_P0 + o), c.T(T_HMP0 + o)));
      if (eff % 228u < 68u) c.S64(IO_BARLO, c.G64(IO_L0LO) + eff / 228u);
      break;
    case 0x2B:
      for (uint32_t o = 0; o < 5; ++o) c.Tset(T_HMP0 + o, 0);
      break;
    case 0x2C:
      if (eff > c.G(IO_CEVAL)) c.Sset(IO_CEVAL, eff);
      c.Sset(IO_CX, 0);
      break;
    default: break;  // RSYNC, audio, unused addresses
  }
  return flags;
}
// Write a TIA or RIOT address at cycle t; returns IO_WSYNC / IO_VSYNC_RISE.
__device__ __noinline__ uint32_t fc_io_write(IoCtx c, uint32_t a, uint32_t v, uint32_t t) {
  if (a & 0x80) {
    fc_riot_write(c, a, v, 76ull * c.G64(IO_L0LO) + t);
    return 0;
  }
  return fc_tia_write(c, a & 0x3F, v, t, true);
}

// End of a frame: collisions up to the current cycle, then rebase to the next frame.
__device__ __noinline__ void fc_frame_end(IoCtx c, uint32_t kf, uint32_t next_rel) {
  fc_cx_eval(c, 3u * kf);
  c.S64(IO_L0LO, c.G64(IO_L0LO) + next_rel);
  c.Sset(IO_CEVAL, c.G(IO_CEVAL) - 228u * next_rel);
}

// ---------------------------------------------------------------- split form
// In the split form a block's warps come in pairs: a CPU warp runs the 6507
// and RIOT and pushes every TIA write into a per-env queue in shared memory;
// the paired TIA warp (same lane, same env) applies the writes, logs them and
// evaluates collisions.  The CPU keeps its own copies of VSYNC, VBLANK, the
// fire latch and the frame base line; it waits for the TIA side only when it
// reads a collision register and at the end of the step.  Events (32 bits):
//   write       0b00 | cycle:16 | register:6 | value:8
//   frame end   0b01 | cycle of the end:16 | lines to the next frame:14
//   control     0b10 | kind:2 | argument   (begin/end of a logged frame,
//               collision sync up to a cycle, end of the step)
constexpr uint32_t QLEN = 32;             // queue entries per env (a power of two)
constexpr uint32_t QSTRIDE = QLEN + 1;    // shared-memory words per env queue (odd)
constexpr uint32_t EV_WRITE = 0u, EV_FRAME_END = 1u << 30, EV_CTRL = 2u << 30;
constexpr uint32_t EV_BEGIN_LOG = EV_CTRL, EV_END_LOG = EV_CTRL | 1u << 28, EV_SYNC = EV_CTRL | 2u << 28,
                   EV_STEP_END = EV_CTRL | 3u << 28;
// A wait between an env's CPU and TIA warps gives up after WAIT_NS of the
// GPU's global timer and the env is declared stalled.  The longest legitimate
// wait is about one frame of the slowest lane of the partner warp (a few
// milliseconds), so the limit is far above it and still short.
constexpr uint64_t WAIT_NS = 200000000ull;  // 200 ms
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// registers whose writes reach the TIA side (WSYNC, RSYNC, audio and unused
// addresses change nothing there)
constexpr uint64_t SPLIT_PUSH_REGS = LOG_REGS | COLL_REGS | 1ull | (1ull << 0x2C);

// ---------------------------------------------------------------- the console
// Split form, CPU side: bounded waits on the TIA side's cursors in this env's
// I/O block.  Wait until the queue has room behind `qtail` (returns the last
// head read: still full means the wait ran out), or until `n` events are
// acknowledged (false means the wait ran out).
__device__ __noinline__ uint32_t fc_q_wait_room(uint32_t *iow, uint32_t qtail) {
  __builtin_assume(__isShared(iow));
  const volatile uint32_t *h = iow + IO_QHEAD;
  uint32_t head = *h;
  if (qtail - head < QLEN) return head;
  const uint64_t t0 = global_ns();
  while (qtail - head >= QLEN && global_ns() - t0 < WAIT_NS) {
    __nanosleep(32);
    head = *h;
  }
  return head;
}
__device__ __noinline__ bool fc_q_wait_ack(uint32_t *iow, uint32_t n) {
  __builtin_assume(__isShared(iow));
  const volatile uint32_t *a = iow + IO_ACK;
  if ((int32_t)(*a - n) >= 0) return true;
  const uint64_t t0 = global_ns();
  while ((int32_t)(*a - n) < 0) {
    if (global_ns() - t0 >= WAIT_NS) return false;
    __nanosleep(32);
  }
  return true;
}

// Split form, CPU side: read a TIA or RIOT address (13-bit, neither RAM nor
// cartridge) at cycle t, out of line so that the many read sites of the
// opcode switch stay small.  A collision-latch read first pushes a sync event
// at queue position qtail (waiting, bounded, for room behind the TIA side's
// cursor qhead_seen) and waits until the TIA side has acknowledged nreq + 1
// sync events, i.e. has evaluated collisions up to cycle t.  Returns the
// value in bits 0-7; bit 8 when the sync event was pushed (the caller counts
// it, and the queue is then empty), bit 9 when a wait ran out (the caller
// halts the env).  `broken` (an earlier wait ran out) skips the sync and
// returns the latches as they stand.
constexpr uint32_t SIO_PUSHED = 0x100u, SIO_STALL = 0x200u;
__device__ __noinline__ uint32_t fc_split_io_read(IoCtx c, uint32_t *q, uint32_t qtail, uint32_t qhead_seen,
                                                  uint32_t nreq, uint32_t broken, uint32_t a, uint32_t t,
                                                  uint64_t l0) {
  if (a & 0x80) return fc_riot_read(c, a, 76ull * l0 + t);
  const uint32_t reg = a & 0x0F;
  if (reg == 0x0C) return (c.G(IO_FIRE) || c.G(IO_LATCH)) ? 0x00u : 0x80u;
  if (reg == 0x0D) return 0x80u;
  if (reg >= 8) return 0;
  volatile uint32_t *vw = reinterpret_cast<volatile uint32_t *>(c.w());
  if (broken) return fc_cx_byte(vw[IO_CX], reg);
  if (qtail - qhead_seen >= QLEN) {
    qhead_seen = fc_q_wait_room(c.w(), qtail);
    if (qtail - qhead_seen >= QLEN) return SIO_STALL | fc_cx_byte(vw[IO_CX], reg);
  }
  __builtin_assume(__isShared(q));
  reinterpret_cast<volatile uint32_t *>(q)[qtail & (QLEN - 1)] = EV_SYNC | (t & 0xFFFFu);
  __threadfence_block();
  vw[IO_QTAIL] = qtail + 1;
  if (!fc_q_wait_ack(c.w(), nreq + 1)) return SIO_PUSHED | SIO_STALL | fc_cx_byte(vw[IO_CX], reg);
  __threadfence_block();
  return SIO_PUSHED | fc_cx_byte(vw[IO_CX], reg);
}

// COMPACT: the hot opcode switch keeps only the common addressing forms
// (implied, accumulator, immediate, zero page and absolute reads, writes and
// branches, indexed loads and stores); the indirect forms, BIT, stack
// pushes and pulls and indexed or absolute read-modify-writes go to the
// general decoder.  A smaller hot loop for the instruction cache; the
// results are the same either way.
template <bool SPLIT, bool COMPACT = false> struct FastConsoleT;
template <bool SPLIT, bool COMPACT> __device__ __forceinline__ void fc_exec_general(FastConsoleT<SPLIT, COMPACT> *self);

template <bool SPLIT, bool COMPACT>
struct FastConsoleT {
  const uint8_t *rom8;     // staged cartridge bytes (banks of 4096, then 16 bytes of padding)
  const uint8_t *dec_op;   // general decoder: opcode -> operation | penalty << 7, then mode | cycles << 4
  uint8_t *ram;            // this env's RAM block (shared memory, 4-byte aligned)
  IoCtx io;
  uint32_t A, X, Y, SP, PC, fc, fv, fn, fz, fdi;  // fdi holds the D (0x08) and I (0x04) bits
  uint32_t bank, jam, scheme;
  uint32_t kf;             // CPU cycles since the first line of the frame
  uint32_t pend;           // I/O flags of the current instruction
  uint32_t vs_kf;          // cycle of a VSYNC rise in this frame, ~0 if none
  uint32_t status, instret, frame_no;
  uint32_t rounds;         // lockstep issue rounds of this env's warp in the step (the same on every lane)
  uint32_t wmask;          // lanes of this warp running envs (lockstep issue)
  uint32_t idle;           // retire RIOT-timer wait-loop iterations at once
  // split form: this env's TIA event queue and the CPU side's copies
  uint32_t *q;
  uint32_t qtail, qhead_seen, nreq, vsync_c, vblank_c, broken;  // qhead_seen: the TIA side's cursor as last read
  uint64_t l0c;

  __device__ __forceinline__ uint32_t P() const {
    return (fn & 0x80) | fv | 0x20 | fdi | ((fz & 0xFF) ? 0u : 2u) | fc;
  }
  __device__ __forceinline__ void setP(uint32_t p) {
    fn = p & 0x80; fv = p & 0x40; fdi = p & 0x0C; fz = (p & 2) ? 0u : 1u; fc = p & 1;
  }

  // ---- canonical state I/O ----
  __device__ void load(const uint8_t *s) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(s);
    const uint32_t w0 = w[0], w1 = w[1];
    A = w0 & 0xFF; X = (w0 >> 8) & 0xFF; Y = (w0 >> 16) & 0xFF; SP = w0 >> 24;
    setP(w1 & 0xFF); PC = w1 >> 16;
    bank = (w1 >> 8) & (scheme == 3 ? 7u : scheme == 2 ? 3u : scheme == 1 ? 1u : 0u);  // scheme is set before load
    const uint64_t k = (uint64_t)w[2] | (uint64_t)w[3] << 32;
    io.Sset(IO_TCWLO, w[4]); io.Sset(IO_TCWHI, w[5]);
    const uint32_t w6 = w[6], w7 = w[7];
    io.Sset(IO_TV, w6 & 0xFF); io.Sset(IO_TSH, (w6 >> 8) & 0xFF);
    io.Sset(IO_PORTS, (w6 >> 16) | ((w7 & 0xFFFF) << 16));
    jam = (w7 >> 16) & 0xFF;
    io.Sset(IO_LATCH, w7 >> 24);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const uint32_t v = w[8 + q];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (q * 4 + b < 37) io.Tset(q * 4 + b, v >> (8 * b));
    }
    io.Sset(IO_CX, w[17] >> 16);
    io.Sset(IO_BARLO, w[18]); io.Sset(IO_BARHI, w[19]);
    io.Sset(IO_L0LO, w[20]); io.Sset(IO_L0HI, w[21]);
    frame_no = w[22];
    const uint64_t L0 = (uint64_t)w[20] | (uint64_t)w[21] << 32;
    kf = (uint32_t)(k - 76ull * L0);
    io.Sset(IO_CEVAL, 3u * kf);
    io.Sset(IO_JOY, 0xFF); io.Sset(IO_FIRE, 0);
    io.Sset(IO_LOGLO, 0); io.Sset(IO_LOGHI, 0); io.Sset(IO_LOGN, 0); io.Sset(IO_LOGCAP, 0);
    io.Sset(IO_STATUS, 0);
    const uint4 *r4 = reinterpret_cast<const uint4 *>(s + S::RAM);
    uint32_t *r32 = reinterpret_cast<uint32_t *>(ram);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 v = r4[q];
      r32[4 * q] = v.x; r32[4 * q + 1] = v.y; r32[4 * q + 2] = v.z; r32[4 * q + 3] = v.w;
    }
    status = 0; instret = 0; rounds = 0; pend = 0; vs_kf = ~0u;
    if constexpr (SPLIT) {
      vsync_c = io.T(T_VSYNC);
      vblank_c = io.T(T_VBLANK);
      l0c = L0;
      qtail = qhead_seen = nreq = broken = 0;
      io.Sset(IO_QHEAD, 0); io.Sset(IO_QTAIL, 0); io.Sset(IO_ACK, 0);
    }
  }
  __device__ void store(uint8_t *s) const {
    uint32_t *w = reinterpret_cast<uint32_t *>(s);
    const uint64_t L0 = io.G64(IO_L0LO);
    w[0] = A | X << 8 | Y << 16 | SP << 24;
    w[1] = P() | bank << 8 | PC << 16;
    const uint64_t k = 76ull * L0 + kf;
    w[2] = (uint32_t)k; w[3] = (uint32_t)(k >> 32);
    w[4] = io.G(IO_TCWLO); w[5] = io.G(IO_TCWHI);
    const uint32_t ports = io.G(IO_PORTS);
    w[6] = io.G(IO_TV) | io.G(IO_TSH) << 8 | (ports & 0xFFFF) << 16;
    w[7] = (ports >> 16) | jam << 16 | io.G(IO_LATCH) << 24;
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (q * 4 + b < 37) v |= io.T(q * 4 + b) << (8 * b);
      if (q == 9) v = (v & 0xFFFFu) | io.G(IO_CX) << 16;
      w[8 + q] = v;
    }
    w[18] = io.G(IO_BARLO); w[19] = io.G(IO_BARHI);
    w[20] = (uint32_t)L0; w[21] = (uint32_t)(L0 >> 32);
    w[22] = frame_no; w[23] = 0;
    uint4 *r4 = reinterpret_cast<uint4 *>(s + S::RAM);
    const uint32_t *r32 = reinterpret_cast<const uint32_t *>(ram);
#pragma unroll
    for (int q = 0; q < 8; ++q) r4[q] = make_uint4(r32[4 * q], r32[4 * q + 1], r32[4 * q + 2], r32[4 * q + 3]);
  }
  __device__ void snapshot(uint8_t *o) const { fc_snapshot(io, o, 0); }
  __device__ void set_log(uint32_t *p, uint32_t cap, uint8_t *bands) { fc_set_log(io, p, cap, bands); }
  // Band starts the frame never reached take its final state.
  __device__ void finish_bands() {
    if (io.G(IO_BANDN) < 4) fc_band_snap(io, ~0u);
  }
  __device__ uint32_t log_count() const { return io.G(IO_LOGN); }
  __device__ uint32_t all_status() const { return status | io.G(IO_STATUS); }

  __device__ void apply_action(uint32_t a) {
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
    io.Sset(IO_JOY, 0xFFu & ~(((d & 2) ? 0x80u : 0u) | ((d & 4) ? 0x40u : 0u) | ((d & 8) ? 0x20u : 0u) |
                              ((d & 1) ? 0x10u : 0u)));
    const uint32_t fire = (a == 1 || a >= 10) ? 1u : 0u;
    io.Sset(IO_FIRE, fire);
    const uint32_t vb = SPLIT ? vblank_c : io.T(T_VBLANK);
    if (fire && (vb & 0x40)) io.Sset(IO_LATCH, 1);
  }

  // Cartridge bytes i .. i+3 of the stage, byte i lowest (i + 3 may run into
  // the padding after the last bank).
  __device__ __forceinline__ uint32_t fetch4(uint32_t i) const {
    const uint32_t *r32 = reinterpret_cast<const uint32_t *>(rom8);
    const uint32_t q = i >> 2;
    return __funnelshift_r(r32[q], r32[q + 1], (i & 3u) * 8u);
  }

  // ---- bus ----
  __device__ __forceinline__ void hotspot(uint32_t off) {
    if (scheme == 1) { if (off == 0xFF8 || off == 0xFF9) bank = off - 0xFF8; }
    else if (scheme == 2) { if (off >= 0xFF6 && off <= 0xFF9) bank = off - 0xFF6; }
    else if (scheme == 3) { if (off >= 0xFF4 && off <= 0xFFB) bank = off - 0xFF4; }
  }
  __device__ __forceinline__ void note_vsync(uint32_t t) {
    if (vs_kf == ~0u) vs_kf = t;
  }
  // ---- split form: the queue to the TIA side ----
  __device__ __forceinline__ volatile uint32_t *vio(uint32_t i) const {
    return reinterpret_cast<volatile uint32_t *>(io.w() + i);
  }
  __device__ __forceinline__ void stall() {
    broken = 1;
    status |= ST_STALL;
    jam = 1;
  }
  // Append an event (waits, bounded, while the queue is full).  The TIA
  // side's cursor is reread only when the queue looks full; the waits run out
  // of line so that each inlined push stays small.
  __device__ __forceinline__ void push(uint32_t ev) {
    if (broken) return;
    if (qtail - qhead_seen >= QLEN) {
      qhead_seen = fc_q_wait_room(io.w(), qtail);
      if (qtail - qhead_seen >= QLEN) { stall(); return; }
    }
    reinterpret_cast<volatile uint32_t *>(q)[qtail & (QLEN - 1)] = ev;
    __threadfence_block();
    ++qtail;
    *vio(IO_QTAIL) = qtail;
  }
  // Wait (bounded) until the TIA side has acknowledged n events.
  __device__ __forceinline__ void wait_ack(uint32_t n) {
    if (broken) return;
    if (!fc_q_wait_ack(io.w(), n)) { stall(); return; }
    __threadfence_block();
  }
  // TIA write in the split form: WSYNC, the VSYNC rise and the VBLANK latch
  // effects here, the register itself on the TIA side.
  __device__ __forceinline__ void tia_out(uint32_t reg, uint32_t v, uint32_t t) {
    if (reg == 0x02) { pend |= IO_WSYNC; return; }
    if (reg == 0x00) {
      if (!(vsync_c & 2) && (v & 2)) { pend |= IO_VSYNC_RISE; note_vsync(t); }
      vsync_c = v;
    } else if (reg == 0x01) {
      vblank_c = v;
      if (!(v & 0x40)) io.Sset(IO_LATCH, 0);
      else if (io.G(IO_FIRE)) io.Sset(IO_LATCH, 1);
    }
    if ((SPLIT_PUSH_REGS >> reg) & 1ull) push(EV_WRITE | t << 14 | reg << 8 | v);
  }
  // Read / write a TIA or RIOT address at cycle t.
  __device__ __forceinline__ uint32_t io_read(uint32_t a, uint32_t t) {
    if constexpr (!SPLIT) {
      return fc_io_read(io, a, t);
    } else {
      const uint32_t r = fc_split_io_read(io, q, qtail, qhead_seen, nreq, broken, a, t, l0c);
      if (r & SIO_PUSHED) { ++qtail; ++nreq; qhead_seen = qtail; }
      if (r & SIO_STALL) stall();
      return r & 0xFFu;
    }
  }
  __device__ __forceinline__ void io_write(uint32_t a, uint32_t v, uint32_t t) {
    if constexpr (!SPLIT) {
      const uint32_t f = fc_io_write(io, a, v, t);
      pend |= f;
      if (f & IO_VSYNC_RISE) note_vsync(t);
    } else {
      if (a & 0x80) fc_riot_write(io, a, v, 76ull * l0c + t);
      else tia_out(a & 0x3F, v, t);
    }
  }
  __device__ __forceinline__ void frame_end_out(uint32_t next_rel) {
    if constexpr (!SPLIT) {
      fc_frame_end(io, kf, next_rel);
    } else {
      push(EV_FRAME_END | kf << 14 | next_rel);
      l0c += next_rel;
    }
  }

  // zero-page access: RAM for $80-$FF, TIA below
  __device__ __forceinline__ uint32_t rdz(uint32_t z, uint32_t t) {
    return (z & 0x80) ? ram[z & 0x7F] : io_read(z, t);
  }
  __device__ __forceinline__ void wrz(uint32_t z, uint32_t v, uint32_t t) {
    if (z & 0x80) ram[z & 0x7F] = v & 0xFF;
    else io_write(z, v & 0xFF, t);
  }
  __device__ __forceinline__ uint32_t rd(uint32_t addr, uint32_t t) {
    const uint32_t a = addr & 0x1FFF;
    if ((a & 0x1280) == 0x0080) return ram[a & 0x7F];
    if (a & 0x1000) {
      const uint32_t off = a & 0xFFF;
      if (scheme) hotspot(off);
      return rom8[bank * 4096u + off];
    }
    return io_read(a, t);
  }
  __device__ __forceinline__ void wr(uint32_t addr, uint32_t v, uint32_t t) {
    const uint32_t a = addr & 0x1FFF;
    if ((a & 0x1280) == 0x0080) { ram[a & 0x7F] = v & 0xFF; return; }
    if (a & 0x1000) { if (scheme) hotspot(a & 0xFFF); return; }
    io_write(a, v & 0xFF, t);
  }

  // Store instructions write through here (one inlined copy): RAM, cartridge
  // hotspots, WSYNC and the colour / motion registers inline, every other
  // TIA or RIOT address through the out-of-line writer.
  __device__ __forceinline__ void bus_store(uint32_t addr, uint32_t v, uint32_t t) {
    const uint32_t a = addr & 0x1FFF;
    if ((a & 0x1280) == 0x0080) { ram[a & 0x7F] = v & 0xFF; return; }
    if (a & 0x1000) { if (scheme) hotspot(a & 0xFFF); return; }
    if (!(a & 0x80)) {
      const uint32_t reg = a & 0x3F;
      if constexpr (SPLIT) {
        tia_out(reg, v & 0xFF, t);
        return;
      }
      if (reg == 0x02) { pend |= IO_WSYNC; return; }
      if ((FAST_TIA_REGS >> reg) & 1ull) {
        fc_log(io, 3u * (t + 1u), reg, v & 0xFF);
        io.Tset(reg < 0x20 ? reg - 2 : reg - 5, v & 0xFF);
        return;
      }
    }
    io_write(a, v & 0xFF, t);
  }

  // ---- ALU ----
  __device__ __forceinline__ void adc(uint32_t v) {
    const uint32_t c = fc;
    if (!(fdi & 0x08)) {
      const uint32_t s = A + v + c;
      const uint32_t r = s & 0xFF;
      fv = ((~(A ^ v) & (A ^ r)) & 0x80u) >> 1;
      fc = s >> 8;
      fn = fz = r;
      A = r;
      return;
    }
    const uint32_t zb = (A + v + c) & 0xFF;
    int lo = (int)(A & 0x0F) + (int)(v & 0x0F) + (int)c;
    if (lo > 9) lo = ((lo + 6) & 0x0F) + 0x10;
    const int hs = (int)(int8_t)(uint8_t)(A & 0xF0) + (int)(int8_t)(uint8_t)(v & 0xF0) + lo;
    int hu = (int)(A & 0xF0) + (int)(v & 0xF0) + lo;
    fn = (uint32_t)hs & 0x80;
    fv = (hs > 127 || hs < -128) ? 0x40u : 0u;
    if (hu >= 0xA0) hu += 0x60;
    fc = hu > 0xFF ? 1u : 0u;
    fz = zb;
    A = (uint32_t)hu & 0xFF;
  }
  __device__ __forceinline__ void sbc(uint32_t v) {
    const uint32_t c = fc;
    const uint32_t nv = v ^ 0xFF;
    const uint32_t s = A + nv + c;
    uint32_t r = s & 0xFF;
    fv = ((~(A ^ nv) & (A ^ r)) & 0x80u) >> 1;
    fc = s >> 8;
    fn = fz = r;
    if (fdi & 0x08) {
      int lo = (int)(A & 0x0F) - (int)(v & 0x0F) + (int)c - 1;
      if (lo < 0) lo = ((lo - 6) & 0x0F) - 0x10;
      int hi = (int)(A & 0xF0) - (int)(v & 0xF0) + lo;
      if (hi < 0) hi -= 0x60;
      r = (uint32_t)hi & 0xFF;
    }
    A = r;
  }
  __device__ __forceinline__ void cmp(uint32_t reg, uint32_t v) {
    fc = reg >= v ? 1u : 0u;
    fn = fz = (reg - v) & 0xFF;
  }
  __device__ __forceinline__ uint32_t asl(uint32_t v) { fc = v >> 7; const uint32_t r = (v << 1) & 0xFF; fn = fz = r; return r; }
  __device__ __forceinline__ uint32_t lsr(uint32_t v) { fc = v & 1; const uint32_t r = v >> 1; fn = fz = r; return r; }
  __device__ __forceinline__ uint32_t rol(uint32_t v) { const uint32_t r = ((v << 1) | fc) & 0xFF; fc = v >> 7; fn = fz = r; return r; }
  __device__ __forceinline__ uint32_t ror(uint32_t v) { const uint32_t r = (v >> 1) | (fc << 7); fc = v & 1; fn = fz = r; return r; }
  __device__ __forceinline__ uint32_t inc(uint32_t v) { const uint32_t r = (v + 1) & 0xFF; fn = fz = r; return r; }
  __device__ __forceinline__ uint32_t dec(uint32_t v) { const uint32_t r = (v - 1) & 0xFF; fn = fz = r; return r; }

  // ---- RIOT-timer wait loops ----
  // LDA INTIM at pc with BNE back to pc right after it: an iteration that
  // reads a nonzero timer value changes nothing but the cycle count (A and the
  // N, Z flags are overwritten by the read that exits), and the read has no
  // side effect.  With the timer counting in intervals of 2^sh >= 8 cycles, at
  // least the loop's period (7 cycles, 8 when the branch crosses a page), the
  // first read at or after the cycle where INTIM reaches 0 reads 0.  So the
  // iterations before that read retire at once: the cycle count advances
  // exactly as if they ran, and the returned cycle is where the exiting LDA
  // starts.  They are not counted in instret, which counts the instructions
  // the issue rounds execute.  Anything else (no such loop, a faster
  // timer, the timer already at 0 or past it, a frame that would reach the
  // line cap) returns k0 unchanged.
  __device__ __forceinline__ uint32_t idle_forward(uint32_t w, uint32_t pc, uint32_t k0) {
    const uint32_t a = (w >> 8) & 0xFFFF;
    if ((a & 0x1285u) != 0x0284u || (w >> 24) != 0xD0u) return k0;  // INTIM (any mirror), then BNE
    const uint32_t off = pc & 0xFFF;
    if (off > 0xFFBu || rom8[bank * 4096u + off + 4] != 0xFBu) return k0;  // BNE offset -5: back to pc
    const uint32_t sh = io.G(IO_TSH);
    if (sh < 3) return k0;
    const uint64_t l0 = SPLIT ? l0c : io.G64(IO_L0LO);
    const uint64_t n0 = 76ull * l0 + k0 + 3 - (io.G64(IO_TCWLO) + 1);  // the read's cycle, as the timer counts it
    const uint64_t zero = (uint64_t)io.G(IO_TV) << sh;                 // first cycle reading 0
    if (n0 >= zero) return k0;
    const uint32_t period = (((pc + 5) ^ pc) & 0xFF00) ? 8u : 7u;
    const uint64_t it = (zero - n0 + period - 1) / period;
    const uint64_t k1 = k0 + it * period;
    if (k1 + 6 >= 76ull * CAP_LINES) return k0;
    return (uint32_t)k1;
  }

  // ---- one instruction, hot form ----
  // Returns false (with nothing changed) for the cases the general decoder
  // takes.  Each case sets the cycle count n and the next PC; the tail
  // applies the WSYNC stall.
  // w = cartridge bytes PC .. PC+3 of the current bank (fetch4).
  __device__ __forceinline__ bool exec(uint32_t w) {
    const uint32_t pc = PC;
    const uint32_t off = pc & 0xFFF;
    // no hot fetch may touch a hotspot: F8/F6 hotspots start at $FF6, F4's at $FF4
    if (!(pc & 0x1000) || off > (scheme == 3 ? 0xFF1u : scheme ? 0xFF3u : 0xFFCu)) return false;
    const uint32_t k0 = kf;
    const uint32_t b1 = (w >> 8) & 0xFF;
    const uint32_t a16 = (w >> 8) & 0xFFFF;
    uint32_t n;
    uint32_t sa = ~0u, sv = 0, stc = 0;  // pending store: address (~0: none), value, cycle
    pend = 0;
#define ZPX_ ((b1 + X) & 0xFF)
#define ZPY_ ((b1 + Y) & 0xFF)
#define ABX_ ((a16 + X) & 0xFFFF)
#define ABY_ ((a16 + Y) & 0xFFFF)
#define XPG(base, ea) ((((base) ^ (ea)) >> 8) & 1u)
#define NZ(v) (fn = fz = (v))
#define COLD_ if constexpr (COMPACT) return false;
// read instructions: imm, zp, zp,X, abs, abs,X, abs,Y, (zp,X), (zp),Y
#define RD_OPS(OPI, OPZ, OPZX, OPA, OPAX, OPAY, OPIX, OPIY, BODY)                                          \
  case OPI: { const uint32_t v = b1; BODY; n = 2; PC = pc + 2; break; }                                      \
  case OPZ: { const uint32_t v = rdz(b1, k0 + 2); BODY; n = 3; PC = pc + 2; break; }                          \
  case OPZX: { const uint32_t v = rdz(ZPX_, k0 + 3); BODY; n = 4; PC = pc + 2; break; }                       \
  case OPA: { const uint32_t ka = (OPA == 0xAD && idle) ? idle_forward(w, pc, k0) : k0;                     \
              const uint32_t v = rd(a16, ka + 3); BODY; n = 4 + (ka - k0); PC = pc + 3; break; }             \
  case OPAX: { const uint32_t ea = ABX_; n = 4 + XPG(a16, ea); const uint32_t v = rd(ea, k0 + n - 1); BODY;   \
               PC = pc + 3; break; }                                                                          \
  case OPAY: { const uint32_t ea = ABY_; n = 4 + XPG(a16, ea); const uint32_t v = rd(ea, k0 + n - 1); BODY;   \
               PC = pc + 3; break; }                                                                          \
  case OPIX: { COLD_ const uint32_t z = ZPX_; if (!(z & 0x80) || z == 0xFF) return false;                   \
               const uint32_t ea = ram[z & 0x7F] | ram[(z + 1) & 0x7F] << 8;                      \
               const uint32_t v = rd(ea, k0 + 5); BODY; n = 6; PC = pc + 2; break; }                           \
  case OPIY: { COLD_ if (!(b1 & 0x80) || b1 == 0xFF) return false;                                           \
               const uint32_t base = ram[b1 & 0x7F] | ram[(b1 + 1) & 0x7F] << 8;                  \
               const uint32_t ea = (base + Y) & 0xFFFF; n = 5 + XPG(base, ea);                                \
               const uint32_t v = rd(ea, k0 + n - 1); BODY; PC = pc + 2; break; }
// read-modify-write: acc, zp, zp,X, abs, abs,X.  The memory forms take RAM
// here (where the old-value write is invisible); a TIA, RIOT or cartridge
// address goes to the general decoder, which models both writes.
#define RMW_MEM_OPS(OPZ, OPZX, OPA, OPAX, FN)                                                                \
  case OPZ: { if (!(b1 & 0x80)) return false;                                                                 \
              ram[b1 & 0x7F] = FN(ram[b1 & 0x7F]); n = 5; PC = pc + 2; break; }                              \
  case OPZX: { COLD_ const uint32_t z = ZPX_; if (!(z & 0x80)) return false;                                 \
               ram[z & 0x7F] = FN(ram[z & 0x7F]); n = 6; PC = pc + 2; break; }                                \
  case OPA: { COLD_ if ((a16 & 0x1280) != 0x0080) return false;                                              \
              ram[a16 & 0x7F] = FN(ram[a16 & 0x7F]); n = 6; PC = pc + 3; break; }                            \
  case OPAX: { COLD_ const uint32_t ea = ABX_; if ((ea & 0x1280) != 0x0080) return false;                   \
               ram[ea & 0x7F] = FN(ram[ea & 0x7F]); n = 7; PC = pc + 3; break; }
#define RMW_OPS(OPACC, OPZ, OPZX, OPA, OPAX, FN)                                                             \
  case OPACC: { A = FN(A); n = 2; PC = pc + 1; break; }                                                       \
  RMW_MEM_OPS(OPZ, OPZX, OPA, OPAX, FN)
// memory-only read-modify-write (INC, DEC): zp, zp,X, abs, abs,X
#define RMWM_OPS(OPZ, OPZX, OPA, OPAX, FN) RMW_MEM_OPS(OPZ, OPZX, OPA, OPAX, FN)
#define BR(OPC, COND)                                                                                          \
  case OPC: {                                                                                                 \
    const uint32_t nx = (pc + 2) & 0xFFFF;                                                                    \
    n = 2; PC = nx;                                                                                           \
    if (COND) { const uint32_t tg = (nx + (uint32_t)(int32_t)(int8_t)(uint8_t)b1) & 0xFFFF;                   \
                n += ((nx ^ tg) & 0xFF00) ? 2u : 1u; PC = tg; }                                               \
    break; }
#define IMPL(OPC, BODY) case OPC: { BODY; n = 2; PC = pc + 1; break; }
    switch (w & 0xFF) {
      RD_OPS(0xA9, 0xA5, 0xB5, 0xAD, 0xBD, 0xB9, 0xA1, 0xB1, { A = v; NZ(A); })            // LDA
      RD_OPS(0x69, 0x65, 0x75, 0x6D, 0x7D, 0x79, 0x61, 0x71, { adc(v); })                  // ADC
      RD_OPS(0xE9, 0xE5, 0xF5, 0xED, 0xFD, 0xF9, 0xE1, 0xF1, { sbc(v); })                  // SBC
      RD_OPS(0x29, 0x25, 0x35, 0x2D, 0x3D, 0x39, 0x21, 0x31, { A &= v; NZ(A); })           // AND
      RD_OPS(0x09, 0x05, 0x15, 0x0D, 0x1D, 0x19, 0x01, 0x11, { A |= v; NZ(A); })           // ORA
      RD_OPS(0x49, 0x45, 0x55, 0x4D, 0x5D, 0x59, 0x41, 0x51, { A ^= v; NZ(A); })           // EOR
      RD_OPS(0xC9, 0xC5, 0xD5, 0xCD, 0xDD, 0xD9, 0xC1, 0xD1, { cmp(A, v); })               // CMP
      // LDX: imm, zp, zp,Y, abs, abs,Y
      case 0xA2: X = b1; NZ(X); n = 2; PC = pc + 2; break;
      case 0xA6: X = rdz(b1, k0 + 2); NZ(X); n = 3; PC = pc + 2; break;
      case 0xB6: X = rdz(ZPY_, k0 + 3); NZ(X); n = 4; PC = pc + 2; break;
      case 0xAE: X = rd(a16, k0 + 3); NZ(X); n = 4; PC = pc + 3; break;
      case 0xBE: { const uint32_t ea = ABY_; n = 4 + XPG(a16, ea); X = rd(ea, k0 + n - 1); NZ(X); PC = pc + 3; break; }
      // LDY: imm, zp, zp,X, abs, abs,X
      case 0xA0: Y = b1; NZ(Y); n = 2; PC = pc + 2; break;
      case 0xA4: Y = rdz(b1, k0 + 2); NZ(Y); n = 3; PC = pc + 2; break;
      case 0xB4: Y = rdz(ZPX_, k0 + 3); NZ(Y); n = 4; PC = pc + 2; break;
      case 0xAC: Y = rd(a16, k0 + 3); NZ(Y); n = 4; PC = pc + 3; break;
      case 0xBC: { const uint32_t ea = ABX_; n = 4 + XPG(a16, ea); Y = rd(ea, k0 + n - 1); NZ(Y); PC = pc + 3; break; }
      // CPX, CPY: imm, zp, abs
      case 0xE0: cmp(X, b1); n = 2; PC = pc + 2; break;
      case 0xE4: cmp(X, rdz(b1, k0 + 2)); n = 3; PC = pc + 2; break;
      case 0xEC: cmp(X, rd(a16, k0 + 3)); n = 4; PC = pc + 3; break;
      case 0xC0: cmp(Y, b1); n = 2; PC = pc + 2; break;
      case 0xC4: cmp(Y, rdz(b1, k0 + 2)); n = 3; PC = pc + 2; break;
      case 0xCC: cmp(Y, rd(a16, k0 + 3)); n = 4; PC = pc + 3; break;
      // BIT: zp, abs
      case 0x24: { COLD_ const uint32_t v = rdz(b1, k0 + 2); fn = v; fv = v & 0x40; fz = A & v; n = 3; PC = pc + 2; break; }
      case 0x2C: { COLD_ const uint32_t v = rd(a16, k0 + 3); fn = v; fv = v & 0x40; fz = A & v; n = 4; PC = pc + 3; break; }
      // stores
      case 0x85: sa = b1; sv = A; stc = k0 + 2; n = 3; PC = pc + 2; break;
      case 0x95: sa = ZPX_; sv = A; stc = k0 + 3; n = 4; PC = pc + 2; break;
      case 0x8D: sa = a16; sv = A; stc = k0 + 3; n = 4; PC = pc + 3; break;
      case 0x9D: sa = ABX_; sv = A; stc = k0 + 4; n = 5; PC = pc + 3; break;
      case 0x99: sa = ABY_; sv = A; stc = k0 + 4; n = 5; PC = pc + 3; break;
      case 0x81: { COLD_ const uint32_t z = ZPX_; if (!(z & 0x80) || z == 0xFF) return false;
                   sa = ram[z & 0x7F] | ram[(z + 1) & 0x7F] << 8; sv = A; stc = k0 + 5; n = 6; PC = pc + 2; break; }
      case 0x91: { COLD_ if (!(b1 & 0x80) || b1 == 0xFF) return false;
                   const uint32_t base = ram[b1 & 0x7F] | ram[(b1 + 1) & 0x7F] << 8;
                   sa = (base + Y) & 0xFFFF; sv = A; stc = k0 + 5; n = 6; PC = pc + 2; break; }
      case 0x86: sa = b1; sv = X; stc = k0 + 2; n = 3; PC = pc + 2; break;
      case 0x96: sa = ZPY_; sv = X; stc = k0 + 3; n = 4; PC = pc + 2; break;
      case 0x8E: sa = a16; sv = X; stc = k0 + 3; n = 4; PC = pc + 3; break;
      case 0x84: sa = b1; sv = Y; stc = k0 + 2; n = 3; PC = pc + 2; break;
      case 0x94: sa = ZPX_; sv = Y; stc = k0 + 3; n = 4; PC = pc + 2; break;
      case 0x8C: sa = a16; sv = Y; stc = k0 + 3; n = 4; PC = pc + 3; break;
      RMW_OPS(0x0A, 0x06, 0x16, 0x0E, 0x1E, asl)
      RMW_OPS(0x4A, 0x46, 0x56, 0x4E, 0x5E, lsr)
      RMW_OPS(0x2A, 0x26, 0x36, 0x2E, 0x3E, rol)
      RMW_OPS(0x6A, 0x66, 0x76, 0x6E, 0x7E, ror)
      RMWM_OPS(0xE6, 0xF6, 0xEE, 0xFE, inc)
      RMWM_OPS(0xC6, 0xD6, 0xCE, 0xDE, dec)
      BR(0x10, !(fn & 0x80))
      BR(0x30, (fn & 0x80))
      BR(0x50, !fv)
      BR(0x70, fv)
      BR(0x90, !fc)
      BR(0xB0, fc)
      BR(0xD0, (fz & 0xFF))
      BR(0xF0, !(fz & 0xFF))
      IMPL(0xE8, { X = (X + 1) & 0xFF; NZ(X); })
      IMPL(0xC8, { Y = (Y + 1) & 0xFF; NZ(Y); })
      IMPL(0xCA, { X = (X - 1) & 0xFF; NZ(X); })
      IMPL(0x88, { Y = (Y - 1) & 0xFF; NZ(Y); })
      IMPL(0xAA, { X = A; NZ(X); })
      IMPL(0xA8, { Y = A; NZ(Y); })
      IMPL(0x8A, { A = X; NZ(A); })
      IMPL(0x98, { A = Y; NZ(A); })
      IMPL(0xBA, { X = SP; NZ(X); })
      IMPL(0x9A, { SP = X; })
      IMPL(0x18, { fc = 0; })
      IMPL(0x38, { fc = 1; })
      IMPL(0x58, { fdi &= ~0x04u; })
      IMPL(0x78, { fdi |= 0x04u; })
      IMPL(0xB8, { fv = 0; })
      IMPL(0xD8, { fdi &= ~0x08u; })
      IMPL(0xF8, { fdi |= 0x08u; })
      IMPL(0xEA, {})
      case 0x48: COLD_ if (!(SP & 0x80)) return false; ram[SP & 0x7F] = A; SP = (SP - 1) & 0xFF; n = 3; PC = pc + 1; break;
      case 0x08: COLD_ if (!(SP & 0x80)) return false; ram[SP & 0x7F] = P() | 0x10u; SP = (SP - 1) & 0xFF; n = 3; PC = pc + 1; break;
      case 0x68: { COLD_ const uint32_t s1 = (SP + 1) & 0xFF; if (!(s1 & 0x80)) return false;
                   SP = s1; A = ram[s1 & 0x7F]; NZ(A); n = 4; PC = pc + 1; break; }
      case 0x28: { COLD_ const uint32_t s1 = (SP + 1) & 0xFF; if (!(s1 & 0x80)) return false;
                   SP = s1; setP(ram[s1 & 0x7F]); n = 4; PC = pc + 1; break; }
      case 0x4C: PC = a16; n = 3; break;
      case 0x20: { if (SP < 0x81) return false;
                   const uint32_t ret = (pc + 2) & 0xFFFF;
                   ram[SP & 0x7F] = ret >> 8; ram[(SP - 1) & 0x7F] = ret & 0xFF;
                   SP = (SP - 2) & 0xFF; PC = a16; n = 6; break; }
      case 0x60: { const uint32_t s1 = (SP + 1) & 0xFF, s2 = (SP + 2) & 0xFF;
                   if (!(s1 & 0x80) || !(s2 & 0x80)) return false;
                   PC = ((ram[s1 & 0x7F] | ram[s2 & 0x7F] << 8) + 1) & 0xFFFF; SP = s2; n = 6; break; }
      default: return false;  // BRK, RTI, JMP (ind), undocumented
    }
#undef ZPX_
#undef ZPY_
#undef ABX_
#undef ABY_
#undef XPG
#undef NZ
#undef COLD_
#undef RD_OPS
#undef RMW_MEM_OPS
#undef RMW_OPS
#undef RMWM_OPS
#undef BR
#undef IMPL
    if (sa != ~0u) bus_store(sa, sv, stc);
    PC &= 0xFFFF;
    uint32_t k = k0 + n;
    if (pend & IO_WSYNC) k = ((k + 75u) / 76u) * 76u;
    kf = k;
    instret++;
    return true;
  }

  // ---- one instruction, general form (every case; run out of line) ----
  __device__ void exec_general() {
    const uint32_t k0 = kf;
    pend = 0;
    const uint32_t pc = PC;
    const uint32_t opcode = rd(pc, k0);
    const uint32_t opb = dec_op[opcode];
    const uint32_t op = opb & 0x7F;
    const uint32_t info = dec_op[256 + opcode];
    const uint32_t mode = info & 0xF;
    uint32_t n = info >> 4;
    if (op == O_JAM) { jam = 1; status |= ST_ILLEGAL; return; }
    uint32_t b1 = 0, b2 = 0, ea = 0, cross = 0;
    if (mode >= IMM) b1 = rd(pc + 1, k0);
    if (mode >= ABS && mode <= IND) b2 = rd(pc + 2, k0);
    switch (mode) {
      case IMP: case ACC: PC = (pc + 1) & 0xFFFF; break;
      case IMM: PC = (pc + 2) & 0xFFFF; break;
      case ZP: ea = b1; PC = (pc + 2) & 0xFFFF; break;
      case ZPX: ea = (b1 + X) & 0xFF; PC = (pc + 2) & 0xFFFF; break;
      case ZPY: ea = (b1 + Y) & 0xFF; PC = (pc + 2) & 0xFFFF; break;
      case ABS: ea = b1 | b2 << 8; PC = (pc + 3) & 0xFFFF; break;
      case ABX: { const uint32_t b = b1 | b2 << 8; ea = (b + X) & 0xFFFF; cross = (b ^ ea) >> 8; PC = (pc + 3) & 0xFFFF; break; }
      case ABY: { const uint32_t b = b1 | b2 << 8; ea = (b + Y) & 0xFFFF; cross = (b ^ ea) >> 8; PC = (pc + 3) & 0xFFFF; break; }
      case IND: { const uint32_t p = b1 | b2 << 8;
                  const uint32_t lo = rd(p, k0), hi = rd((p & 0xFF00) | ((p + 1) & 0xFF), k0);
                  ea = lo | hi << 8; PC = (pc + 3) & 0xFFFF; break; }
      case IZX: { const uint32_t z = (b1 + X) & 0xFF; const uint32_t lo = rd(z, k0), hi = rd((z + 1) & 0xFF, k0);
                  ea = lo | hi << 8; PC = (pc + 2) & 0xFFFF; break; }
      case IZY: { const uint32_t lo = rd(b1, k0), hi = rd((b1 + 1) & 0xFF, k0); const uint32_t b = lo | hi << 8;
                  ea = (b + Y) & 0xFFFF; cross = (b ^ ea) >> 8; PC = (pc + 2) & 0xFFFF; break; }
      default: PC = (pc + 2) & 0xFFFF; ea = (PC + (uint32_t)(int32_t)(int8_t)(uint8_t)b1) & 0xFFFF; break;
    }
    if (cross && (opb >> 7)) n++;
    instret++;
    if (mode == REL) {
      uint32_t take;
      switch (op) {
        case O_BCC: take = fc ^ 1u; break;
        case O_BCS: take = fc; break;
        case O_BNE: take = (fz & 0xFF) ? 1u : 0u; break;
        case O_BEQ: take = (fz & 0xFF) ? 0u : 1u; break;
        case O_BVC: take = fv ? 0u : 1u; break;
        case O_BVS: take = fv ? 1u : 0u; break;
        case O_BPL: take = (fn & 0x80) ? 0u : 1u; break;
        default: take = (fn & 0x80) ? 1u : 0u; break;
      }
      if (take) { n += ((PC ^ ea) & 0xFF00) ? 2u : 1u; PC = ea; }
      kf = k0 + n;
      return;
    }
    const uint32_t kA = k0 + n - 1;
    switch (op) {
      case O_LDA: A = mode == IMM ? b1 : rd(ea, kA); fn = fz = A; break;
      case O_LDX: X = mode == IMM ? b1 : rd(ea, kA); fn = fz = X; break;
      case O_LDY: Y = mode == IMM ? b1 : rd(ea, kA); fn = fz = Y; break;
      case O_STA: wr(ea, A, kA); break;
      case O_STX: wr(ea, X, kA); break;
      case O_STY: wr(ea, Y, kA); break;
      case O_ADC: adc(mode == IMM ? b1 : rd(ea, kA)); break;
      case O_SBC: sbc(mode == IMM ? b1 : rd(ea, kA)); break;
      case O_AND: A &= mode == IMM ? b1 : rd(ea, kA); fn = fz = A; break;
      case O_ORA: A |= mode == IMM ? b1 : rd(ea, kA); fn = fz = A; break;
      case O_EOR: A ^= mode == IMM ? b1 : rd(ea, kA); fn = fz = A; break;
      case O_CMP: cmp(A, mode == IMM ? b1 : rd(ea, kA)); break;
      case O_CPX: cmp(X, mode == IMM ? b1 : rd(ea, kA)); break;
      case O_CPY: cmp(Y, mode == IMM ? b1 : rd(ea, kA)); break;
      case O_BIT: { const uint32_t v = rd(ea, kA); fn = v; fv = v & 0x40; fz = A & v; break; }
      case O_ASL: case O_LSR: case O_ROL: case O_ROR: case O_INC: case O_DEC: {
        const uint32_t old = mode == ACC ? A : rd(ea, kA - 2);
        uint32_t r;
        switch (op) {
          case O_ASL: r = asl(old); break;
          case O_LSR: r = lsr(old); break;
          case O_ROL: r = rol(old); break;
          case O_ROR: r = ror(old); break;
          case O_INC: r = inc(old); break;
          default: r = dec(old); break;
        }
        if (mode == ACC) A = r;
        else { wr(ea, old, kA - 1); wr(ea, r, kA); }
        break;
      }
      case O_SLO: case O_RLA: case O_SRE: case O_RRA: case O_DCP: case O_ISC: {
        // read-modify-write of memory (both writes), then the accumulator operation
        const uint32_t old = rd(ea, kA - 2);
        uint32_t r, c = fc;
        switch (op) {
          case O_SLO: r = (old << 1) & 0xFF; c = old >> 7; break;
          case O_RLA: r = ((old << 1) | fc) & 0xFF; c = old >> 7; break;
          case O_SRE: r = old >> 1; c = old & 1; break;
          case O_RRA: r = (old >> 1) | (fc << 7); c = old & 1; break;
          case O_DCP: r = (old - 1) & 0xFF; break;
          default: r = (old + 1) & 0xFF; break;
        }
        wr(ea, old, kA - 1);
        wr(ea, r, kA);
        switch (op) {
          case O_SLO: A |= r; fc = c; fn = fz = A; break;
          case O_RLA: A &= r; fc = c; fn = fz = A; break;
          case O_SRE: A ^= r; fc = c; fn = fz = A; break;
          case O_RRA: fc = c; adc(r); break;
          case O_DCP: cmp(A, r); break;
          default: sbc(r); break;
        }
        break;
      }
      case O_SAX: wr(ea, A & X, kA); break;
      case O_LAX: A = rd(ea, kA); X = A; fn = fz = A; break;
      case O_ANC: A &= b1; fn = fz = A; fc = A >> 7; break;
      case O_ALR: A &= b1; fc = A & 1u; A >>= 1; fn = fz = A; break;
      case O_SBX: { const uint32_t ax = A & X; fc = ax >= b1 ? 1u : 0u; X = (ax - b1) & 0xFF; fn = fz = X; break; }
      case O_NOP: if (mode != IMP && mode != IMM) (void)rd(ea, kA); break;  // the operand read
      case O_INX: X = (X + 1) & 0xFF; fn = fz = X; break;
      case O_INY: Y = (Y + 1) & 0xFF; fn = fz = Y; break;
      case O_DEX: X = (X - 1) & 0xFF; fn = fz = X; break;
      case O_DEY: Y = (Y - 1) & 0xFF; fn = fz = Y; break;
      case O_TAX: X = A; fn = fz = X; break;
      case O_TAY: Y = A; fn = fz = Y; break;
      case O_TXA: A = X; fn = fz = A; break;
      case O_TYA: A = Y; fn = fz = A; break;
      case O_TSX: X = SP; fn = fz = X; break;
      case O_TXS: SP = X; break;
      case O_CLC: fc = 0; break;
      case O_SEC: fc = 1; break;
      case O_CLI: fdi &= ~0x04u; break;
      case O_SEI: fdi |= 0x04u; break;
      case O_CLV: fv = 0; break;
      case O_CLD: fdi &= ~0x08u; break;
      case O_SED: fdi |= 0x08u; break;
      case O_PHA: wr(0x100u | SP, A, kA); SP = (SP - 1) & 0xFF; break;
      case O_PHP: wr(0x100u | SP, P() | 0x10u, kA); SP = (SP - 1) & 0xFF; break;
      case O_PLA: SP = (SP + 1) & 0xFF; A = rd(0x100u | SP, kA); fn = fz = A; break;
      case O_PLP: SP = (SP + 1) & 0xFF; setP(rd(0x100u | SP, kA)); break;
      case O_JMP: PC = ea; break;
      case O_JSR: {
        const uint32_t ret = (pc + 2) & 0xFFFF;
        wr(0x100u | SP, ret >> 8, kA); SP = (SP - 1) & 0xFF;
        wr(0x100u | SP, ret & 0xFF, kA); SP = (SP - 1) & 0xFF;
        PC = ea;
        break;
      }
      case O_RTS: {
        SP = (SP + 1) & 0xFF; const uint32_t lo = rd(0x100u | SP, kA);
        SP = (SP + 1) & 0xFF; const uint32_t hi = rd(0x100u | SP, kA);
        PC = ((lo | hi << 8) + 1) & 0xFFFF;
        break;
      }
      case O_RTI: {
        SP = (SP + 1) & 0xFF; setP(rd(0x100u | SP, kA));
        SP = (SP + 1) & 0xFF; const uint32_t lo = rd(0x100u | SP, kA);
        SP = (SP + 1) & 0xFF; const uint32_t hi = rd(0x100u | SP, kA);
        PC = lo | hi << 8;
        break;
      }
      case O_BRK: {
        const uint32_t ret = (pc + 2) & 0xFFFF;
        wr(0x100u | SP, ret >> 8, kA); SP = (SP - 1) & 0xFF;
        wr(0x100u | SP, ret & 0xFF, kA); SP = (SP - 1) & 0xFF;
        wr(0x100u | SP, P() | 0x10u, kA); SP = (SP - 1) & 0xFF;
        fdi |= 0x04u;
        const uint32_t lo = rd(0x1FFE, kA), hi = rd(0x1FFF, kA);
        PC = lo | hi << 8;
        break;
      }
      default: break;
    }
    uint32_t k = k0 + n;
    if (pend & IO_WSYNC) k = ((k + 75u) / 76u) * 76u;
    kf = k;
  }

  // One frame.  Lanes of a warp issue in program order of the laggard: each
  // round the lane with the smallest emulated cycle count leads, and every
  // lane whose PC equals the leader's executes its instruction with it.  Lanes
  // that ran a shorter path wait at the join point until the laggard reaches
  // it, so the warp reconverges on code rather than on time (lanes a few
  // cycles apart after a page-crossing or a different branch path still run
  // together), and the executing lanes take one case of the opcode switch.
  // One warp reduction elects the leader: the minimum of (cycle << 16 | PC)
  // over the active lanes gives its PC directly (ties in the cycle go to the
  // smaller PC), and all-ones means no lane is active.  The cycle saturates
  // below 0xFFFF, so the key always names a lane's actual PC.  The leader
  // always advances (every instruction takes at least 2 cycles, and a frame
  // ends after at most 400 lines), so the loop ends.
  __device__ __forceinline__ uint32_t run_frame() {
    uint32_t next_rel = 0;
    vs_kf = ~0u;
    bool active = !jam;
    if (jam) next_rel = kf / 76u;
    for (;;) {
      // next instruction word, fetched before the election so the two latencies overlap
      // (bank < banks of the staged cartridge, so the index stays in the stage)
      const uint32_t w = fetch4(bank * 4096u + (PC & 0xFFFu));
      const uint32_t key = active ? (min(kf, 0xFFFEu) << 16 | (PC & 0xFFFFu)) : 0xFFFFFFFFu;
      const uint32_t lead = __reduce_min_sync(wmask, key);
      if (lead == 0xFFFFFFFFu) break;
      ++rounds;
      if (active && PC == (lead & 0xFFFFu)) {
        if (!exec(w)) fc_exec_general<SPLIT, COMPACT>(this);
        if (jam | (vs_kf != ~0u) | (kf >= 76u * CAP_LINES)) {
          if (jam) next_rel = kf / 76u;
          else if (vs_kf != ~0u) next_rel = vs_kf / 76u;
          else { status |= ST_FRAME_CAP; next_rel = kf / 76u; }
          active = false;
        }
      }
    }
    frame_end_out(next_rel);
    kf -= 76u * next_rel;
    frame_no++;
    return next_rel;
  }
};

using FastConsole = FastConsoleT<false, false>;

// Out-of-line general instruction on a copy of the console.  Only the CPU
// and timing state comes back: the caller's pointers into shared memory are
// never reloaded from the copy, so they keep their shared address space.
template <bool SPLIT, bool COMPACT>
__device__ __noinline__ void fc_exec_general_impl(FastConsoleT<SPLIT, COMPACT> *c) { c->exec_general(); }
template <bool SPLIT, bool COMPACT>
__device__ __forceinline__ void fc_exec_general(FastConsoleT<SPLIT, COMPACT> *self) {
  FastConsoleT<SPLIT, COMPACT> tmp = *self;
  fc_exec_general_impl<SPLIT, COMPACT>(&tmp);
  self->A = tmp.A; self->X = tmp.X; self->Y = tmp.Y; self->SP = tmp.SP; self->PC = tmp.PC;
  self->fc = tmp.fc; self->fv = tmp.fv; self->fn = tmp.fn; self->fz = tmp.fz; self->fdi = tmp.fdi;
  self->bank = tmp.bank; self->jam = tmp.jam; self->kf = tmp.kf; self->pend = tmp.pend; self->vs_kf = tmp.vs_kf;
  self->status = tmp.status; self->instret = tmp.instret; self->frame_no = tmp.frame_no;
  if constexpr (SPLIT) {
    self->qtail = tmp.qtail; self->qhead_seen = tmp.qhead_seen; self->nreq = tmp.nreq; self->vsync_c = tmp.vsync_c; self->vblank_c = tmp.vblank_c;
    self->broken = tmp.broken; self->l0c = tmp.l0c;
  }
}

}  // namespace atari
