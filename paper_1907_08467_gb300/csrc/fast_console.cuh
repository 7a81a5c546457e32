// Register-resident console for the batched form.
//
// Same machine and the same canonical state as Console in
// device_machine.cuh, laid out for speed on sm_103a:
//   - CPU registers, split flags (N and Z kept as the last result byte),
//     cycle counter, RIOT state and the collision-liveness shadows of the
//     TIA in registers;
//   - RAM in shared memory, one 32-bit word per byte, interleaved by env
//     (word = addr * E + env) so a warp's RAM accesses never bank-conflict;
//   - the 37-byte TIA register file in shared memory (byte per register,
//     interleaved the same way), read only on cold paths;
//   - the block's cartridge staged in shared memory as one word per byte
//     offset: bytes off, off+1, off+2 and the addressing mode / cycle count
//     of the opcode at off, so an instruction is fetched with one load.
// Collision-mask evaluation and RIOT/TIA reads are out of line (cold paths).
#pragma once
#include <cstdint>

#include "device_machine.cuh"

namespace atari {

constexpr uint32_t TIA_BYTES = 40;  // shared-memory bytes per env for the TIA file (37 used)
enum TiaSlot : uint32_t {
  T_VSYNC = 0, T_VBLANK, T_NUSIZ0, T_NUSIZ1, T_COLUP0, T_COLUP1, T_COLUPF, T_COLUBK, T_CTRLPF, T_REFP0,
  T_REFP1, T_PF0, T_PF1, T_PF2, T_ENAM0, T_ENAM1, T_ENABL_N, T_ENABL_O, T_GRP0_N, T_GRP0_O, T_GRP1_N,
  T_GRP1_O, T_VDELP0, T_VDELP1, T_VDELBL, T_RESMP0, T_RESMP1, T_HMP0, T_HMP1, T_HMM0, T_HMM1, T_HMBL,
  T_P0, T_P1, T_M0, T_M1, T_BL
};

// Staged-ROM word: byte0 | byte1 << 8 | byte2 << 16 | mode << 24 | cycles << 28 (bit 31: penalty)
__host__ __device__ constexpr uint32_t romw_mode(uint32_t w) { return (w >> 24) & 0xF; }
__host__ __device__ constexpr uint32_t romw_cycles(uint32_t w) { return (w >> 28) & 7; }

// ---------------------------------------------------------------- cold paths
// Collision bits among live objects over visible columns [lo, hi) of one line.
__device__ __noinline__ uint32_t fc_collide_cols(const uint8_t *tia, uint32_t E, uint32_t live, uint32_t lo,
                                                 uint32_t hi) {
  auto R = [&](uint32_t s) { return (uint32_t)tia[s * E]; };
  M160 r{range_word(0, lo, hi), range_word(1, lo, hi), range_word(2, lo, hi), range_word(3, lo, hi),
         range_word(4, lo, hi)};
  M160 z{0, 0, 0, 0, 0};
  const uint32_t nus0 = R(T_NUSIZ0), nus1 = R(T_NUSIZ1), ctrl = R(T_CTRLPF);
  M160 p0 = (live & 1) ? player_mask((R(T_VDELP0) & 1) ? R(T_GRP0_O) : R(T_GRP0_N), R(T_REFP0), nus0, R(T_P0)) : z;
  M160 p1 = (live & 2) ? player_mask((R(T_VDELP1) & 1) ? R(T_GRP1_O) : R(T_GRP1_N), R(T_REFP1), nus1, R(T_P1)) : z;
  M160 m0 = (live & 4) ? missile_mask(nus0, R(T_M0)) : z;
  M160 m1 = (live & 8) ? missile_mask(nus1, R(T_M1)) : z;
  M160 b = (live & 16) ? ball_mask(ctrl, R(T_BL)) : z;
  M160 f = (live & 32) ? pf_mask(R(T_PF0), R(T_PF1), R(T_PF2), ctrl) : z;
  uint32_t c = 0;
  c |= (uint32_t)meet(m0, p1, r) << 1 | (uint32_t)meet(m0, p0, r) << 0;
  c |= (uint32_t)meet(m1, p0, r) << 3 | (uint32_t)meet(m1, p1, r) << 2;
  c |= (uint32_t)meet(p0, f, r) << 5 | (uint32_t)meet(p0, b, r) << 4;
  c |= (uint32_t)meet(p1, f, r) << 7 | (uint32_t)meet(p1, b, r) << 6;
  c |= (uint32_t)meet(m0, f, r) << 9 | (uint32_t)meet(m0, b, r) << 8;
  c |= (uint32_t)meet(m1, f, r) << 11 | (uint32_t)meet(m1, b, r) << 10;
  c |= (uint32_t)meet(b, f, r) << 13;
  c |= (uint32_t)meet(p0, p1, r) << 15 | (uint32_t)meet(m0, m1, r) << 14;
  return c;
}

// Collisions over the color clocks [from, upto) (frame-relative), state constant.
__device__ __noinline__ uint32_t fc_collide_span(const uint8_t *tia, uint32_t E, uint32_t live, uint32_t from,
                                                 uint32_t upto, uint64_t L0, uint64_t bar) {
  uint32_t la = from / 228u, xa = from - la * 228u;
  uint32_t lb = upto / 228u, xb = upto - lb * 228u;
  uint32_t c = 0;
  auto seg = [&](uint32_t line, uint32_t x0, uint32_t x1) {
    if (x1 <= 68) return;
    uint32_t lo = x0 > 68 ? x0 - 68 : 0, hi = x1 - 68;
    if (L0 + line == bar && lo < 8) lo = 8;
    if (lo < hi) c |= fc_collide_cols(tia, E, live, lo, hi);
  };
  if (la == lb) {
    seg(la, xa, xb);
  } else {
    seg(la, xa, 228);
    if (lb > la + 1) seg(la + 1, 0, 228);
    if (xb) seg(lb, 0, xb);
  }
  return c;
}

__device__ __noinline__ uint32_t fc_riot_read(uint32_t addr, uint64_t now, uint32_t ports, uint32_t joy,
                                              uint64_t tim_cw, uint32_t tim_v, uint32_t tim_shift) {
  const uint32_t swcha_out = ports & 0xFF, swacnt = (ports >> 8) & 0xFF, swchb_out = (ports >> 16) & 0xFF,
                 swbcnt = ports >> 24;
  if (!(addr & 4)) {
    switch (addr & 3) {
      case 0: return ((swcha_out & swacnt) | (joy & ~swacnt)) & 0xFF;
      case 1: return swacnt;
      case 2: return ((swchb_out & swbcnt) | (0x0Bu & ~swbcnt)) & 0xFF;
      default: return swbcnt;
    }
  }
  uint64_t n = now - (tim_cw + 1);
  uint64_t span = (uint64_t)(tim_v + 1) << tim_shift;
  if (addr & 1) return n >= span ? 0x80u : 0u;
  if (n < span) return tim_v - (uint32_t)(n >> tim_shift);
  return (uint32_t)(0xFFull - (n - span)) & 0xFF;
}

// ---------------------------------------------------------------- the console
struct FastConsole;
__device__ __forceinline__ void fc_exec_general(FastConsole *self);

struct FastConsole {
  // shared-memory views
  const uint32_t *romw;    // staged cartridge words (banks of 4096)
  const uint8_t *dec_op;   // opcode -> operation
  uint32_t *ram;           // &ram_block[env], stride E words
  uint8_t *tia;            // &tia_block[env], stride E bytes
  uint32_t E;
  // CPU
  uint32_t A, X, Y, SP, PC, fc, fv, fn, fz, fdi;  // fdi holds the D (0x08) and I (0x04) bits
  uint32_t bank, jam, scheme;
  uint32_t kf;             // CPU cycles since the first line of the frame
  uint64_t L0;             // first line of the frame
  // RIOT
  uint64_t tim_cw;
  uint32_t tim_v, tim_shift, ports, joy, fire, latch;
  // TIA shadows used by the collision-liveness test
  uint32_t vsync, vblank, g0n, g0o, g1n, g1o, ebn, ebo, vd, en, rm, pf0, pf1, pf2;
  uint32_t cx, ceval;
  uint64_t bar;
  uint32_t frame_no, status, instret;
  uint32_t wsync, vs_rise, vs_kf;
  uint32_t *logp;
  uint32_t logn, logcap;

  __device__ __forceinline__ uint32_t T(uint32_t s) const { return tia[s * E]; }
  __device__ __forceinline__ void Tset(uint32_t s, uint32_t v) { tia[s * E] = (uint8_t)v; }
  __device__ __forceinline__ uint32_t P() const {
    return (fn & 0x80) | fv | 0x20 | fdi | ((fz & 0xFF) ? 0u : 2u) | fc;
  }
  __device__ __forceinline__ void setP(uint32_t p) {
    fn = p & 0x80; fv = p & 0x40; fdi = p & 0x0C; fz = (p & 2) ? 0u : 1u; fc = p & 1;
  }

  // ---- canonical state I/O ----
  __device__ void load(const uint8_t *s) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(s);
    uint32_t w0 = w[0], w1 = w[1];
    A = w0 & 0xFF; X = (w0 >> 8) & 0xFF; Y = (w0 >> 16) & 0xFF; SP = w0 >> 24;
    setP(w1 & 0xFF); bank = (w1 >> 8) & 0xFF; PC = w1 >> 16;
    uint64_t k = (uint64_t)w[2] | (uint64_t)w[3] << 32;
    tim_cw = (uint64_t)w[4] | (uint64_t)w[5] << 32;
    uint32_t w6 = w[6], w7 = w[7];
    tim_v = w6 & 0xFF; tim_shift = (w6 >> 8) & 0xFF;
    ports = (w6 >> 16) | ((w7 & 0xFFFF) << 16);     // SWCHA out, SWACNT, SWCHB out, SWBCNT
    jam = (w7 >> 16) & 0xFF; latch = w7 >> 24;
#pragma unroll
    for (int q = 0; q < 10; ++q) {                 // bytes 0x20..0x47 -> TIA file (37 bytes used)
      uint32_t v = w[8 + q];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (q * 4 + b < 37) tia[(q * 4 + b) * E] = (uint8_t)(v >> (8 * b));
    }
    cx = w[17] >> 16;
    bar = (uint64_t)w[18] | (uint64_t)w[19] << 32;
    L0 = (uint64_t)w[20] | (uint64_t)w[21] << 32;
    frame_no = w[22];
    kf = (uint32_t)(k - 76ull * L0);
    ceval = 3u * kf;
    vsync = T(T_VSYNC); vblank = T(T_VBLANK);
    g0n = T(T_GRP0_N); g0o = T(T_GRP0_O); g1n = T(T_GRP1_N); g1o = T(T_GRP1_O);
    ebn = T(T_ENABL_N); ebo = T(T_ENABL_O);
    vd = (T(T_VDELP0) & 1) | (T(T_VDELP1) & 1) << 1 | (T(T_VDELBL) & 1) << 2;
    en = (T(T_ENAM0) >> 1 & 1) | (T(T_ENAM1) & 2);
    rm = (T(T_RESMP0) >> 1 & 1) | (T(T_RESMP1) & 2);
    pf0 = T(T_PF0); pf1 = T(T_PF1); pf2 = T(T_PF2);
    const uint4 *r4 = reinterpret_cast<const uint4 *>(s + S::RAM);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      uint4 v = r4[q];
      uint32_t ws[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int b = 0; b < 16; ++b) ram[(q * 16 + b) * E] = (ws[b >> 2] >> (8 * (b & 3))) & 0xFF;
    }
    status = 0;
    instret = 0;
    joy = 0xFF;
    fire = 0;
    logp = nullptr;
  }
  __device__ void store(uint8_t *s) const {
    uint32_t *w = reinterpret_cast<uint32_t *>(s);
    w[0] = A | X << 8 | Y << 16 | SP << 24;
    w[1] = P() | bank << 8 | PC << 16;
    uint64_t k = 76ull * L0 + kf;
    w[2] = (uint32_t)k; w[3] = (uint32_t)(k >> 32);
    w[4] = (uint32_t)tim_cw; w[5] = (uint32_t)(tim_cw >> 32);
    w[6] = tim_v | tim_shift << 8 | (ports & 0xFFFF) << 16;
    w[7] = (ports >> 16) | jam << 16 | latch << 24;
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (q * 4 + b < 37) v |= (uint32_t)tia[(q * 4 + b) * E] << (8 * b);
      if (q == 9) v = (v & 0xFFFFu) | cx << 16;   // 0x46: collision latches (0x45 is zero)
      w[8 + q] = v;
    }
    w[18] = (uint32_t)bar; w[19] = (uint32_t)(bar >> 32);
    w[20] = (uint32_t)L0; w[21] = (uint32_t)(L0 >> 32);
    w[22] = frame_no; w[23] = 0;
    uint4 *r4 = reinterpret_cast<uint4 *>(s + S::RAM);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      uint32_t ws[4];
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) v |= (ram[(q * 16 + k2 * 4 + b) * E] & 0xFF) << (8 * b);
        ws[k2] = v;
      }
      r4[q] = make_uint4(ws[0], ws[1], ws[2], ws[3]);
    }
  }
  // Render-state snapshot (canonical bytes 0x20..0x5F) for the replay.
  __device__ void snapshot(uint8_t *o) const {
    uint32_t v[16];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      uint32_t x = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (q * 4 + b < 37) x |= (uint32_t)tia[(q * 4 + b) * E] << (8 * b);
      v[q] = x;
    }
    v[9] &= 0xFFu;
    v[10] = (uint32_t)bar; v[11] = (uint32_t)(bar >> 32);
    v[12] = (uint32_t)L0; v[13] = (uint32_t)(L0 >> 32);
    v[14] = 0; v[15] = 0;
    uint4 *d = reinterpret_cast<uint4 *>(o);
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }

  __device__ __forceinline__ void apply_action(uint32_t a) {
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
    if (fire && (vblank & 0x40)) latch = 1;
  }

  // ---- collisions ----
  __device__ __forceinline__ uint32_t live() const {
    uint32_t g0 = (vd & 1) ? g0o : g0n, g1 = (vd & 2) ? g1o : g1n, eb = (vd & 4) ? ebo : ebn;
    return (g0 ? 1u : 0u) | (g1 ? 2u : 0u) | ((en & ~rm) & 3u) << 2 | (eb & 2u) << 3 |
           (((pf0 & 0xF0) | pf1 | pf2) ? 32u : 0u);
  }
  __device__ __forceinline__ void cx_eval(uint32_t upto) {
    uint32_t from = ceval;
    if (upto <= from) return;
    ceval = upto;
    if (vblank & 2) return;
    uint32_t l = live();
    if (__popc(l) < 2) return;
    cx |= fc_collide_span(tia, E, l, from, upto, L0, bar);
  }

  // ---- TIA ----
  __device__ __forceinline__ static uint32_t res_pos(uint32_t eff, uint32_t add, uint32_t hb) {
    uint32_t x = eff % 228u;
    if (x < 68) return hb;
    uint32_t p = x - 68 + add;
    return p >= 160 ? p - 160 : p;
  }
  __device__ __forceinline__ static uint32_t hm_move(uint32_t pos, uint32_t hm) {
    int s = (int)((hm >> 4) & 0xF);
    if (s >= 8) s -= 16;
    int p = (int)pos - s;
    p += p < 0 ? 160 : 0;
    p -= p >= 160 ? 160 : 0;
    return (uint32_t)p;
  }
  __device__ void tia_write(uint32_t reg, uint32_t v, uint32_t t) {
    const uint32_t eff = 3u * (t + 1u);
    if ((COLL_REGS >> reg) & 1ull) cx_eval(eff);
    if (logp && ((LOG_REGS >> reg) & 1ull)) {
      if (logn < logcap) logp[logn] = eff << 14 | reg << 8 | v;
      else status |= ST_LOG_OVERFLOW;
      logn++;
    }
    switch (reg) {
      case 0x00:
        if (!(vsync & 2) && (v & 2)) { vs_rise = 1; vs_kf = t; }
        vsync = v; Tset(T_VSYNC, v); break;
      case 0x01:
        vblank = v; Tset(T_VBLANK, v);
        if (!(v & 0x40)) latch = 0;
        else if (fire) latch = 1;
        break;
      case 0x02: wsync = 1; break;
      case 0x04: case 0x05: case 0x06: case 0x07: case 0x08: case 0x09: case 0x0A: case 0x0B: case 0x0C:
        Tset(reg - 2, v); break;                    // NUSIZ0 .. REFP1 are slots 2 .. 10
      case 0x0D: pf0 = v; Tset(T_PF0, v); break;
      case 0x0E: pf1 = v; Tset(T_PF1, v); break;
      case 0x0F: pf2 = v; Tset(T_PF2, v); break;
      case 0x10: Tset(T_P0, res_pos(eff, 5, 3)); break;
      case 0x11: Tset(T_P1, res_pos(eff, 5, 3)); break;
      case 0x12: Tset(T_M0, res_pos(eff, 4, 2)); break;
      case 0x13: Tset(T_M1, res_pos(eff, 4, 2)); break;
      case 0x14: Tset(T_BL, res_pos(eff, 4, 2)); break;
      case 0x1B: g0n = v; g1o = g1n; Tset(T_GRP0_N, v); Tset(T_GRP1_O, g1o); break;
      case 0x1C: g1n = v; g0o = g0n; ebo = ebn; Tset(T_GRP1_N, v); Tset(T_GRP0_O, g0o); Tset(T_ENABL_O, ebo); break;
      case 0x1D: en = (en & ~1u) | (v >> 1 & 1); Tset(T_ENAM0, v); break;
      case 0x1E: en = (en & ~2u) | (v & 2); Tset(T_ENAM1, v); break;
      case 0x1F: ebn = v; Tset(T_ENABL_N, v); break;
      case 0x20: case 0x21: case 0x22: case 0x23: case 0x24: Tset(T_HMP0 + (reg - 0x20), v); break;
      case 0x25: vd = (vd & ~1u) | (v & 1); Tset(T_VDELP0, v); break;
      case 0x26: vd = (vd & ~2u) | (v & 1) << 1; Tset(T_VDELP1, v); break;
      case 0x27: vd = (vd & ~4u) | (v & 1) << 2; Tset(T_VDELBL, v); break;
      case 0x28: case 0x29: {
        const uint32_t i = reg - 0x28;
        const uint32_t old = T(T_RESMP0 + i);
        if ((old & 2) && !(v & 2)) {
          uint32_t nus = T(T_NUSIZ0 + i);
          uint32_t sc = (nus & 7) == 5 ? 8u : (nus & 7) == 7 ? 16u : 4u;
          Tset(T_M0 + i, (T(T_P0 + i) + sc) % 160u);
        }
        Tset(T_RESMP0 + i, v);
        rm = (rm & ~(1u << i)) | ((v >> 1) & 1) << i;
        break;
      }
      case 0x2A:
#pragma unroll
        for (uint32_t o = 0; o < 5; ++o) Tset(T_P0 + o, hm_move(T(T_P0 + o), T(T_HMP0 + o)));
        if (eff % 228u < 68u) bar = L0 + eff / 228u;
        break;
      case 0x2B:
#pragma unroll
        for (uint32_t o = 0; o < 5; ++o) Tset(T_HMP0 + o, 0);
        break;
      case 0x2C:
        if (eff > ceval) ceval = eff;
        cx = 0;
        break;
      default: break;
    }
  }
  __device__ __forceinline__ uint32_t tia_read(uint32_t reg, uint32_t t) {
    if (reg < 8) {
      cx_eval(3u * t);
      return (((cx >> (2 * reg + 1)) & 1u) << 7) | (((cx >> (2 * reg)) & 1u) << 6);
    }
    if (reg == 0x0C) return (fire || latch) ? 0x00u : 0x80u;
    if (reg == 0x0D) return 0x80u;
    return 0;
  }
  __device__ __forceinline__ void riot_write(uint32_t addr, uint32_t v, uint32_t t) {
    if (!(addr & 4)) {
      const uint32_t sh = 8 * (addr & 3);
      ports = (ports & ~(0xFFu << sh)) | (v & 0xFF) << sh;
      return;
    }
    if (addr & 0x10) {
      tim_v = v;
      const uint32_t sel = addr & 3;
      tim_shift = sel == 0 ? 0 : sel == 1 ? 3 : sel == 2 ? 6 : 10;
      tim_cw = 76ull * L0 + t;
    }
  }

  // ---- bus ----
  __device__ __forceinline__ void hotspot(uint32_t off) {
    if (scheme == 1) { if (off == 0xFF8 || off == 0xFF9) bank = off - 0xFF8; }
    else if (scheme == 2) { if (off >= 0xFF6 && off <= 0xFF9) bank = off - 0xFF6; }
  }
  __device__ uint32_t rd_slow(uint32_t addr, uint32_t t) {
    if (addr & 0x1000) {
      const uint32_t off = addr & 0xFFF;
      if (scheme) hotspot(off);
      return romw[bank * 4096u + off] & 0xFF;
    }
    if (!(addr & 0x80)) return tia_read(addr & 0x0F, t);
    if (!(addr & 0x200)) return ram[(addr & 0x7F) * E];
    return fc_riot_read(addr, 76ull * L0 + t, ports, joy, tim_cw, tim_v, tim_shift);
  }
  __device__ __forceinline__ uint32_t rd(uint32_t addr, uint32_t t) {
    addr &= 0x1FFF;
    if ((addr & 0x1280) == 0x0080) return ram[(addr & 0x7F) * E];
    return rd_slow(addr, t);
  }
  __device__ __forceinline__ void wr(uint32_t addr, uint32_t v, uint32_t t) {
    addr &= 0x1FFF;
    if ((addr & 0x1280) == 0x0080) { ram[(addr & 0x7F) * E] = v & 0xFF; return; }
    if (addr & 0x1000) { if (scheme) hotspot(addr & 0xFFF); return; }
    if (!(addr & 0x80)) { tia_write(addr & 0x3F, v & 0xFF, t); return; }
    riot_write(addr, v, t);
  }
  __device__ __forceinline__ void push(uint32_t v, uint32_t t) { wr(0x100u | SP, v, t); SP = (SP - 1) & 0xFF; }
  __device__ __forceinline__ uint32_t pull(uint32_t t) { SP = (SP + 1) & 0xFF; return rd(0x100u | SP, t); }

  // ---- ALU ----
  __device__ __forceinline__ void adc(uint32_t v) {
    const uint32_t c = fc;
    if (!(fdi & 0x08)) {
      uint32_t s = A + v + c;
      uint32_t r = s & 0xFF;
      fv = ((~(A ^ v) & (A ^ r)) & 0x80u) >> 1;
      fc = s >> 8;
      fn = fz = r;
      A = r;
      return;
    }
    uint32_t zb = (A + v + c) & 0xFF;
    int lo = (int)(A & 0x0F) + (int)(v & 0x0F) + (int)c;
    if (lo > 9) lo = ((lo + 6) & 0x0F) + 0x10;
    int hs = (int)(int8_t)(uint8_t)(A & 0xF0) + (int)(int8_t)(uint8_t)(v & 0xF0) + lo;
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


  // ---- single bus sites of the hot path ----
  __device__ __forceinline__ uint32_t bus_read(uint32_t ea, uint32_t t) {
    const uint32_t a = ea & 0x1FFF;
    if ((a & 0x1280) == 0x0080) return ram[(a & 0x7F) * E];
    if (a & 0x1000) {
      const uint32_t off = a & 0xFFF;
      if (scheme) hotspot(off);
      return romw[bank * 4096u + off] & 0xFF;
    }
    if (!(a & 0x80)) return tia_read(a & 0x0F, t);
    return fc_riot_read(a, 76ull * L0 + t, ports, joy, tim_cw, tim_v, tim_shift);
  }
  __device__ __forceinline__ void bus_write(uint32_t ea, uint32_t v, uint32_t t) {
    const uint32_t a = ea & 0x1FFF;
    if ((a & 0x1280) == 0x0080) { ram[(a & 0x7F) * E] = v & 0xFF; return; }
    if (a & 0x1000) { if (scheme) hotspot(a & 0xFFF); return; }
    if (!(a & 0x80)) { tia_write(a & 0x3F, v & 0xFF, t); return; }
    riot_write(a, v, t);
  }

  // ---- one instruction, hot form ----
  // Handles every instruction whose fetch comes from the cartridge away from
  // hotspots, except BRK, RTI, JMP (ind), stack accesses outside RAM and
  // indirect pointers outside RAM; those run exec_general out of line on a
  // copy of the register state.  One bus-read and one bus-write site.
  __device__ __forceinline__ bool exec() {
    const uint32_t k0 = kf;
    const uint32_t pc = PC;
    const uint32_t off = pc & 0xFFF;
    if (!(pc & 0x1000) || off > (scheme ? 0xFF3u : 0xFFDu)) return false;
    const uint32_t w = romw[bank * 4096u + off];
    const uint32_t op = dec_op[w & 0xFF];
    const uint32_t mode = romw_mode(w);
    uint32_t n = romw_cycles(w);
    const uint32_t b1 = (w >> 8) & 0xFF, b2 = (w >> 16) & 0xFF;
    if (op == O_JAM || op == O_BRK || op == O_RTI || mode == IND) return false;
    uint32_t ea = 0, cross = 0, len = 2;
    switch (mode) {
      case IMP: case ACC: len = 1; break;
      case IMM: break;
      case ZP: ea = b1; break;
      case ZPX: ea = (b1 + X) & 0xFF; break;
      case ZPY: ea = (b1 + Y) & 0xFF; break;
      case ABS: ea = b1 | b2 << 8; len = 3; break;
      case ABX: { uint32_t b = b1 | b2 << 8; ea = (b + X) & 0xFFFF; cross = (b ^ ea) >> 8; len = 3; break; }
      case ABY: { uint32_t b = b1 | b2 << 8; ea = (b + Y) & 0xFFFF; cross = (b ^ ea) >> 8; len = 3; break; }
      case IZX: {
        const uint32_t z = (b1 + X) & 0xFF;
        if (!(z & 0x80) || z == 0xFF) return false;            // pointer bytes outside RAM
        ea = ram[(z & 0x7F) * E] | ram[((z + 1) & 0x7F) * E] << 8;
        break;
      }
      case IZY: {
        if (!(b1 & 0x80) || b1 == 0xFF) return false;
        const uint32_t b = ram[(b1 & 0x7F) * E] | ram[((b1 + 1) & 0x7F) * E] << 8;
        ea = (b + Y) & 0xFFFF;
        cross = (b ^ ea) >> 8;
        break;
      }
      default: break;  // REL
    }
    const uint32_t next = (pc + len) & 0xFFFF;
    if (cross && (w >> 31)) n++;
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
      PC = next;
      if (take) {
        const uint32_t tgt = (next + (uint32_t)(int32_t)(int8_t)(uint8_t)b1) & 0xFFFF;
        n += ((next ^ tgt) & 0xFF00) ? 2u : 1u;
        PC = tgt;
      }
      kf = k0 + n;
      instret++;
      return true;
    }
    // stack and flow: RAM stack only
    switch (op) {
      case O_PHA: case O_PHP:
        if (!(SP & 0x80)) return false;
        ram[(SP & 0x7F) * E] = op == O_PHA ? A : (P() | 0x10u);
        SP = (SP - 1) & 0xFF;
        PC = next; kf = k0 + n; instret++;
        return true;
      case O_PLA: case O_PLP: {
        const uint32_t sp1 = (SP + 1) & 0xFF;
        if (!(sp1 & 0x80)) return false;
        SP = sp1;
        const uint32_t v = ram[(sp1 & 0x7F) * E];
        if (op == O_PLA) { A = v; fn = fz = v; } else setP(v);
        PC = next; kf = k0 + n; instret++;
        return true;
      }
      case O_JSR: {
        if (SP < 0x81) return false;
        const uint32_t ret = (pc + 2) & 0xFFFF;
        ram[(SP & 0x7F) * E] = ret >> 8;
        ram[((SP - 1) & 0x7F) * E] = ret & 0xFF;
        SP = (SP - 2) & 0xFF;
        PC = ea; kf = k0 + n; instret++;
        return true;
      }
      case O_RTS: {
        const uint32_t s1 = (SP + 1) & 0xFF, s2 = (SP + 2) & 0xFF;
        if (!(s1 & 0x80) || !(s2 & 0x80)) return false;
        const uint32_t lo = ram[(s1 & 0x7F) * E], hi = ram[(s2 & 0x7F) * E];
        SP = s2;
        PC = ((lo | hi << 8) + 1) & 0xFFFF; kf = k0 + n; instret++;
        return true;
      }
      case O_JMP: PC = ea; kf = k0 + n; instret++; return true;
      default: break;
    }
    const uint32_t kA = k0 + n - 1;
    const bool rmw = op == O_ASL || op == O_LSR || op == O_ROL || op == O_ROR || op == O_INC || op == O_DEC;
    const bool store = op == O_STA || op == O_STX || op == O_STY;
    wsync = 0;
    vs_rise = 0;
    // the single read site: operand of read instructions and read-modify-write
    uint32_t v = 0;
    if (mode == IMM) v = b1;
    else if (mode == ACC) v = A;
    else if (!store && mode != IMP) v = bus_read(ea, rmw ? kA - 2 : kA);
    uint32_t r = v;
    switch (op) {
      case O_LDA: A = v; fn = fz = v; break;
      case O_LDX: X = v; fn = fz = v; break;
      case O_LDY: Y = v; fn = fz = v; break;
      case O_STA: r = A; break;
      case O_STX: r = X; break;
      case O_STY: r = Y; break;
      case O_ADC: adc(v); break;
      case O_SBC: sbc(v); break;
      case O_AND: A &= v; fn = fz = A; break;
      case O_ORA: A |= v; fn = fz = A; break;
      case O_EOR: A ^= v; fn = fz = A; break;
      case O_CMP: cmp(A, v); break;
      case O_CPX: cmp(X, v); break;
      case O_CPY: cmp(Y, v); break;
      case O_BIT: fn = v; fv = v & 0x40; fz = A & v; break;
      case O_ASL: r = (v << 1) & 0xFF; fc = v >> 7; fn = fz = r; break;
      case O_LSR: r = v >> 1; fc = v & 1; fn = fz = r; break;
      case O_ROL: r = ((v << 1) | fc) & 0xFF; fc = v >> 7; fn = fz = r; break;
      case O_ROR: r = (v >> 1) | (fc << 7); fc = v & 1; fn = fz = r; break;
      case O_INC: r = (v + 1) & 0xFF; fn = fz = r; break;
      case O_DEC: r = (v - 1) & 0xFF; fn = fz = r; break;
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
      default: break;  // NOP
    }
    if (rmw && mode == ACC) A = r;
    // the single write site: stores, and the two writes of read-modify-write
    if (store || (rmw && mode != ACC)) {
#pragma unroll 1
      for (uint32_t wi = store ? 1u : 0u; wi < 2; ++wi) bus_write(ea, wi ? r : v, kA - 1 + wi);
    }
    PC = next;
    uint32_t k = k0 + n;
    if (wsync) k = ((k + 75u) / 76u) * 76u;
    kf = k;
    instret++;
    return true;
  }

  // ---- one instruction, general form (every case; used out of line) ----
  __device__ __forceinline__ void exec_general() {
    const uint32_t k0 = kf;
    wsync = 0;
    vs_rise = 0;
    const uint32_t pc = PC;
    const uint32_t off = pc & 0xFFF;
    uint32_t w;
    if ((pc & 0x1000) && off <= (scheme ? 0xFF3u : 0xFFDu)) {
      w = romw[bank * 4096u + off];
    } else {
      // fetch byte by byte through the bus (code outside the cartridge or next to hotspots)
      const uint32_t op0 = rd(pc, k0);
      const uint32_t info = romw_info_of(op0);
      const uint32_t mode = info & 0xF;
      const uint32_t b1 = (mode >= IMM) ? rd(pc + 1, k0) : 0u;
      const uint32_t b2 = (mode >= ABS && mode <= IND) ? rd(pc + 2, k0) : 0u;
      w = op0 | b1 << 8 | b2 << 16 | info << 24;
    }
    const uint32_t op = dec_op[w & 0xFF];
    const uint32_t mode = romw_mode(w);
    uint32_t n = romw_cycles(w);
    if (op == O_JAM) { jam = 1; status |= ST_ILLEGAL; return; }
    const uint32_t b1 = (w >> 8) & 0xFF, b2 = (w >> 16) & 0xFF;
    uint32_t ea = 0, cross = 0;
    switch (mode) {
      case IMP: case ACC: PC = (pc + 1) & 0xFFFF; break;
      case IMM: PC = (pc + 2) & 0xFFFF; break;
      case ZP: ea = b1; PC = (pc + 2) & 0xFFFF; break;
      case ZPX: ea = (b1 + X) & 0xFF; PC = (pc + 2) & 0xFFFF; break;
      case ZPY: ea = (b1 + Y) & 0xFF; PC = (pc + 2) & 0xFFFF; break;
      case ABS: ea = b1 | b2 << 8; PC = (pc + 3) & 0xFFFF; break;
      case ABX: { uint32_t b = b1 | b2 << 8; ea = (b + X) & 0xFFFF; cross = (b ^ ea) >> 8; PC = (pc + 3) & 0xFFFF; break; }
      case ABY: { uint32_t b = b1 | b2 << 8; ea = (b + Y) & 0xFFFF; cross = (b ^ ea) >> 8; PC = (pc + 3) & 0xFFFF; break; }
      case IND: { uint32_t p = b1 | b2 << 8;
                  uint32_t lo = rd(p, k0), hi = rd((p & 0xFF00) | ((p + 1) & 0xFF), k0);
                  ea = lo | hi << 8; PC = (pc + 3) & 0xFFFF; break; }
      case IZX: { uint32_t z = (b1 + X) & 0xFF; uint32_t lo = rd(z, k0), hi = rd((z + 1) & 0xFF, k0);
                  ea = lo | hi << 8; PC = (pc + 2) & 0xFFFF; break; }
      case IZY: { uint32_t lo = rd(b1, k0), hi = rd((b1 + 1) & 0xFF, k0); uint32_t b = lo | hi << 8;
                  ea = (b + Y) & 0xFFFF; cross = (b ^ ea) >> 8; PC = (pc + 2) & 0xFFFF; break; }
      default: PC = (pc + 2) & 0xFFFF; ea = (PC + (uint32_t)(int32_t)(int8_t)(uint8_t)b1) & 0xFFFF; break;  // REL
    }
    if (cross && (w >> 31)) n++;
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
      if (take) {
        n += ((PC ^ ea) & 0xFF00) ? 2u : 1u;
        PC = ea;
      }
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
      case O_BIT: { uint32_t v = rd(ea, kA); fn = v; fv = v & 0x40; fz = A & v; break; }
      case O_ASL: case O_LSR: case O_ROL: case O_ROR: case O_INC: case O_DEC: {
        const uint32_t old = mode == ACC ? A : rd(ea, kA - 2);
        uint32_t r;
        switch (op) {
          case O_ASL: r = (old << 1) & 0xFF; fc = old >> 7; break;
          case O_LSR: r = old >> 1; fc = old & 1; break;
          case O_ROL: r = ((old << 1) | fc) & 0xFF; fc = old >> 7; break;
          case O_ROR: r = (old >> 1) | (fc << 7); fc = old & 1; break;
          case O_INC: r = (old + 1) & 0xFF; break;
          default: r = (old - 1) & 0xFF; break;
        }
        fn = fz = r;
        if (mode == ACC) A = r;
        else { wr(ea, old, kA - 1); wr(ea, r, kA); }
        break;
      }
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
      case O_PHA: push(A, kA); break;
      case O_PHP: push(P() | 0x10u, kA); break;
      case O_PLA: A = pull(kA); fn = fz = A; break;
      case O_PLP: setP(pull(kA)); break;
      case O_JMP: PC = ea; break;
      case O_JSR: { uint32_t ret = (pc + 2) & 0xFFFF; push(ret >> 8, kA); push(ret & 0xFF, kA); PC = ea; break; }
      case O_RTS: { uint32_t lo = pull(kA); uint32_t hi = pull(kA); PC = ((lo | hi << 8) + 1) & 0xFFFF; break; }
      case O_RTI: { setP(pull(kA)); uint32_t lo = pull(kA); uint32_t hi = pull(kA); PC = lo | hi << 8; break; }
      case O_BRK: {
        uint32_t ret = (pc + 2) & 0xFFFF;
        push(ret >> 8, kA); push(ret & 0xFF, kA); push(P() | 0x10u, kA);
        fdi |= 0x04u;
        uint32_t lo = rd(0x1FFE, kA), hi = rd(0x1FFF, kA);
        PC = lo | hi << 8;
        break;
      }
      default: break;  // NOP
    }
    uint32_t k = k0 + n;
    if (wsync) k = ((k + 75u) / 76u) * 76u;
    kf = k;
  }
  // mode/cycles/penalty of an opcode for the byte-wise fetch path
  __device__ __forceinline__ uint32_t romw_info_of(uint32_t opcode) const { return dec_op[256 + opcode]; }

  __device__ __forceinline__ uint32_t run_frame() {
    uint32_t next_rel;
    vs_rise = 0;
    for (;;) {
      if (jam) { next_rel = kf / 76u; break; }
      if (!exec()) fc_exec_general(this);
      if (jam) { next_rel = kf / 76u; break; }
      if (vs_rise) { next_rel = vs_kf / 76u; break; }
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

// Out-of-line general instruction: runs on a copy of the register state (the
// caller's console stays in registers; only this rare path touches memory).
__device__ __noinline__ void fc_exec_general_impl(FastConsole *c) { c->exec_general(); }
__device__ __forceinline__ void fc_exec_general(FastConsole *self) {
  FastConsole tmp = *self;
  fc_exec_general_impl(&tmp);
  *self = tmp;
}

}  // namespace atari
