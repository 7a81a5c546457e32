// TIA replay (rasteriser) and preprocessing kernels' device helpers.
//
// Paper, Section 3: the TIA kernel replays the per-env buffer of TIA writes
// into the TIA registers and renders the 160x210 frame into global memory;
// rendering one game with several threads (screen rows are independent) is
// named there as future work and is done here.  Here one warp renders one frame: every lane holds the same
// register file, the log records are fetched 32 at a time and broadcast by
// shuffle, and lane l renders columns l, l+32, ..., l+128 of each row.
#pragma once
#include <cstdint>
#include "device_machine.cuh"

namespace atari {

struct RenderRegs {
  uint32_t vblank, nusiz0, nusiz1, ctrlpf, refp0, refp1;
  uint32_t pf0, pf1, pf2, enam0, enam1, enabl_new, enabl_old, grp0_new, grp0_old, grp1_new, grp1_old;
  uint32_t vdelp0, vdelp1, vdelbl, resmp0, resmp1, hmp0, hmp1, hmm0, hmm1, hmbl;
  uint32_t p0, p1, m0, m1, bl;
  uint32_t bar;  // frame-relative line of the HMOVE bar, or ~0u
  // The four colour registers as the bytes of one word, in the order of the
  // colour classes below: 0 COLUBK, 1 COLUP0, 2 COLUP1, 3 COLUPF.
  uint32_t pal;
  // Per lane, one nibble per column lane + 32k (bit 4k): v_* = the object
  // covers the column (players, missiles and ball with their enables,
  // playfield); sel = nibble k holds the colour class of the column after
  // the priority rules; cw, c4 = the five pixel colours (bytes 0..3 of cw,
  // byte 0 of c4), zero while blanked.  Rebuilt for what `dirty` names
  // before the next pixel is drawn.
  uint32_t vp0, vp1, vm0, vm1, vbl, vpf, sel, cw, c4;
  uint32_t dirty;  // 1 P0, 2 P1, 4 M0, 8 M1, 16 BL, 32 PF, 64 priority or score mode, 128 colours or blanking

  // from a 64-byte snapshot (canonical bytes 0x20..0x5F)
  __device__ void load(const uint8_t *t) {
    vblank = t[1]; nusiz0 = t[2]; nusiz1 = t[3];
    pal = (uint32_t)t[7] | (uint32_t)t[4] << 8 | (uint32_t)t[5] << 16 | (uint32_t)t[6] << 24;
    ctrlpf = t[8]; refp0 = t[9]; refp1 = t[10]; pf0 = t[11]; pf1 = t[12]; pf2 = t[13]; enam0 = t[14];
    enam1 = t[15]; enabl_new = t[16]; enabl_old = t[17]; grp0_new = t[18]; grp0_old = t[19]; grp1_new = t[20];
    grp1_old = t[21]; vdelp0 = t[22]; vdelp1 = t[23]; vdelbl = t[24]; resmp0 = t[25]; resmp1 = t[26];
    hmp0 = t[27]; hmp1 = t[28]; hmm0 = t[29]; hmm1 = t[30]; hmbl = t[31];
    p0 = t[32]; p1 = t[33]; m0 = t[34]; m1 = t[35]; bl = t[36];
    uint64_t b = 0, l0 = 0;
    for (int i = 7; i >= 0; --i) { b = (b << 8) | t[40 + i]; l0 = (l0 << 8) | t[48 + i]; }
    bar = (b != NO_LINE && b >= l0 && b - l0 < 1024) ? (uint32_t)(b - l0) : ~0u;
    dirty = 255;
  }

  static __device__ __forceinline__ uint32_t res_pos(uint32_t eff, uint32_t add, uint32_t hb) {
    uint32_t x = eff % 228u;
    if (x < 68) return hb;
    uint32_t p = x - 68 + add;
    return p >= 160 ? p - 160 : p;
  }
  static __device__ __forceinline__ uint32_t move(uint32_t pos, uint32_t hm) {
    int s = (int)((hm >> 4) & 0xF);
    if (s >= 8) s -= 16;
    int p = (int)pos - s;
    p += p < 0 ? 160 : 0;
    p -= p >= 160 ? 160 : 0;
    return (uint32_t)p;
  }
  // Apply a logged write (effect clock eff, frame-relative).  An object is
  // marked stale only when something its coverage is built from changes.
  __device__ void apply(uint32_t reg, uint32_t v, uint32_t eff) {
    switch (reg) {
      case 0x01: dirty |= (vblank ^ v) & 2 ? 128 : 0; vblank = v; break;
      case 0x04: dirty |= v != nusiz0 ? 1 | 4 : 0; nusiz0 = v; break;
      case 0x05: dirty |= v != nusiz1 ? 2 | 8 : 0; nusiz1 = v; break;
      case 0x06: pal = (pal & 0xFFFF00FFu) | v << 8; dirty |= 128; break;
      case 0x07: pal = (pal & 0xFF00FFFFu) | v << 16; dirty |= 128; break;
      case 0x08: pal = (pal & 0x00FFFFFFu) | v << 24; dirty |= 128; break;
      case 0x09: pal = (pal & 0xFFFFFF00u) | v; dirty |= 128; break;
      case 0x0A:
        dirty |= ((ctrlpf ^ v) & 0x30 ? 16 : 0) | ((ctrlpf ^ v) & 1 ? 32 : 0) | ((ctrlpf ^ v) & 6 ? 64 : 0);
        ctrlpf = v; break;
      case 0x0B: dirty |= (refp0 ^ v) & 8 ? 1 : 0; refp0 = v; break;
      case 0x0C: dirty |= (refp1 ^ v) & 8 ? 2 : 0; refp1 = v; break;
      case 0x0D: dirty |= (pf0 ^ v) & 0xF0 ? 32 : 0; pf0 = v; break;
      case 0x0E: dirty |= v != pf1 ? 32 : 0; pf1 = v; break;
      case 0x0F: dirty |= v != pf2 ? 32 : 0; pf2 = v; break;
      case 0x10: { const uint32_t x = res_pos(eff, 5, 3); dirty |= x != p0 ? 1 : 0; p0 = x; break; }
      case 0x11: { const uint32_t x = res_pos(eff, 5, 3); dirty |= x != p1 ? 2 : 0; p1 = x; break; }
      case 0x12: { const uint32_t x = res_pos(eff, 4, 2); dirty |= x != m0 ? 4 : 0; m0 = x; break; }
      case 0x13: { const uint32_t x = res_pos(eff, 4, 2); dirty |= x != m1 ? 8 : 0; m1 = x; break; }
      case 0x14: { const uint32_t x = res_pos(eff, 4, 2); dirty |= x != bl ? 16 : 0; bl = x; break; }
      // GRP0 sets P0's new graphic and copies P1's new graphic to its old one
      // (shown when the vertical delay is on); GRP1 likewise, and the ball's
      // enable to its delayed copy.
      case 0x1B:
        dirty |= (!(vdelp0 & 1) && v != grp0_new ? 1 : 0) | ((vdelp1 & 1) && grp1_old != grp1_new ? 2 : 0);
        grp0_new = v; grp1_old = grp1_new; break;
      case 0x1C:
        dirty |= (!(vdelp1 & 1) && v != grp1_new ? 2 : 0) | ((vdelp0 & 1) && grp0_old != grp0_new ? 1 : 0) |
                 ((vdelbl & 1) && ((enabl_old ^ enabl_new) & 2) ? 16 : 0);
        grp1_new = v; grp0_old = grp0_new; enabl_old = enabl_new; break;
      case 0x1D: dirty |= (enam0 ^ v) & 2 ? 4 : 0; enam0 = v; break;
      case 0x1E: dirty |= (enam1 ^ v) & 2 ? 8 : 0; enam1 = v; break;
      case 0x1F: dirty |= !(vdelbl & 1) && ((enabl_new ^ v) & 2) ? 16 : 0; enabl_new = v; break;
      case 0x20: hmp0 = v; break;
      case 0x21: hmp1 = v; break;
      case 0x22: hmm0 = v; break;
      case 0x23: hmm1 = v; break;
      case 0x24: hmbl = v; break;
      case 0x25: dirty |= (vdelp0 ^ v) & 1 ? 1 : 0; vdelp0 = v; break;
      case 0x26: dirty |= (vdelp1 ^ v) & 1 ? 2 : 0; vdelp1 = v; break;
      case 0x27: dirty |= (vdelbl ^ v) & 1 ? 16 : 0; vdelbl = v; break;
      case 0x28:
        if ((resmp0 & 2) && !(v & 2)) m0 = (p0 + ((nusiz0 & 7) == 5 ? 8u : (nusiz0 & 7) == 7 ? 16u : 4u)) % 160u;
        resmp0 = v; dirty |= 4; break;
      case 0x29:
        if ((resmp1 & 2) && !(v & 2)) m1 = (p1 + ((nusiz1 & 7) == 5 ? 8u : (nusiz1 & 7) == 7 ? 16u : 4u)) % 160u;
        resmp1 = v; dirty |= 8; break;
      case 0x2A:
        p0 = move(p0, hmp0); p1 = move(p1, hmp1); m0 = move(m0, hmm0); m1 = move(m1, hmm1); bl = move(bl, hmbl);
        if (eff % 228u < 68u) bar = eff / 228u;
        dirty |= 1 | 2 | 4 | 8 | 16;
        break;
      case 0x2B: hmp0 = hmp1 = hmm0 = hmm1 = hmbl = 0; break;
      default: break;
    }
  }

  // Coverage nibbles of an object whose unmoved mask is u (words 3, 4 zero)
  // placed at pos: column x = lane + 32k shows mask pixel d = (x - pos) mod
  // 160, and with d0 = (lane - pos) mod 160 = 32 q + r that pixel is bit r
  // of word (q + k) mod 5.  So the five nibbles are bit r of words 0..2,
  // rotated right by q nibbles within five.
  static __device__ __forceinline__ uint32_t cover(const M160 &u, uint32_t pos, uint32_t lane) {
    int d = (int)lane - (int)pos;
    d += d < 0 ? 160 : 0;
    const uint32_t q4 = ((uint32_t)d >> 5) * 4u, r = (uint32_t)d & 31u;
    const uint32_t b = ((u.w0 >> r) & 1u) | ((u.w1 >> r) & 1u) << 4 | ((u.w2 >> r) & 1u) << 8;
    return ((b >> q4) | (b << (20u - q4))) & 0x11111u;
  }
  // Playfield nibbles: column x lies in 4-pixel block x >> 2 = (lane >> 2) +
  // 8k of the 40 blocks, the left half's 20 then the right half's (repeated,
  // or mirrored when CTRLPF bit 0 is set).
  static __device__ __forceinline__ uint32_t pf_cover(uint32_t pf0, uint32_t pf1, uint32_t pf2, uint32_t ctrlpf,
                                                      uint32_t lane) {
    const uint32_t l = pf20(pf0, pf1, pf2);
    const uint32_t rh = (ctrlpf & 1) ? (__brev(l) >> 12) : l;
    const uint64_t g = ((uint64_t)l | (uint64_t)rh << 20) >> (lane >> 2);
    const uint32_t lo = (uint32_t)g;
    return (lo & 1u) | (lo >> 4 & 0x10u) | (lo >> 8 & 0x100u) | (lo >> 12 & 0x1000u) | ((uint32_t)(g >> 16) & 0x10000u);
  }
  __device__ __forceinline__ void refresh(uint32_t lane) {
    if (dirty & 127) refresh_classes(lane);
    cw = (vblank & 2) ? 0u : __byte_perm(pal, 0, sel) & 0xFEFEFEFEu;
    c4 = (vblank & 2) ? 0u : __byte_perm(pal, 0, sel >> 16) & 0xFEu;
    dirty = 0;
  }
  __device__ __forceinline__ void refresh_classes(uint32_t lane) {
    if (dirty & 1) {
      const uint32_t g = (vdelp0 & 1) ? grp0_old : grp0_new;
      vp0 = (g & 0xFF) ? cover(player_base(g, refp0, nusiz0), p0, lane) : 0u;
    }
    if (dirty & 2) {
      const uint32_t g = (vdelp1 & 1) ? grp1_old : grp1_new;
      vp1 = (g & 0xFF) ? cover(player_base(g, refp1, nusiz1), p1, lane) : 0u;
    }
    if (dirty & 4) vm0 = ((enam0 & 2) && !(resmp0 & 2)) ? cover(missile_base(nusiz0), m0, lane) : 0u;
    if (dirty & 8) vm1 = ((enam1 & 2) && !(resmp1 & 2)) ? cover(missile_base(nusiz1), m1, lane) : 0u;
    if (dirty & 16) vbl = ((((vdelbl & 1) ? enabl_old : enabl_new) & 2)) ? cover(ball_base(ctrlpf), bl, lane) : 0u;
    if (dirty & 32) vpf = pf_cover(pf0, pf1, pf2, ctrlpf, lane);
    // Colour class of each column, all five at once on the nibble planes.
    // Normal priority: player 0 and missile 0, then player 1 and missile 1,
    // then playfield (in score mode coloured as player 0 left of column 80
    // and player 1 right of it), then ball, then background.  Playfield
    // priority (CTRLPF bit 2): playfield and ball first (score mode off).
    const uint32_t a = vp0 | vm0, bb = vp1 | vm1, fl = vpf | vbl;
    uint32_t c0, c1;  // class bit 0 (classes 1, 3) and bit 1 (classes 2, 3)
    if (ctrlpf & 4) {
      c0 = fl | (a & ~fl);
      c1 = fl | (bb & ~a & ~fl);
    } else if (ctrlpf & 2) {
      const uint32_t right = 0x11000u | (lane >= 16u ? 0x100u : 0u);  // columns >= 80
      const uint32_t pf = vpf & ~a & ~bb, ball = vbl & ~vpf & ~a & ~bb;
      c0 = a | (pf & ~right) | ball;
      c1 = (bb & ~a) | (pf & right) | ball;
    } else {
      const uint32_t o = fl & ~a & ~bb;
      c0 = a | o;
      c1 = (bb & ~a) | o;
    }
    sel = c0 | c1 << 1;
  }
  // Rebuild the stale coverage if any lane of the warp is about to draw
  // (draws = this lane has a pixel to draw before the next register write).
  // Every lane applies the same writes, so `dirty` is the same in all lanes
  // and the rebuild runs once for the whole warp.
  __device__ __forceinline__ void prepare(bool draws, uint32_t lane) {
    if (dirty != 0 && __any_sync(0xFFFFFFFFu, draws)) refresh(lane);
  }
  // Pixels k0..4 of the lane on a line, drawn from one register state (no
  // write lands between them); the stores before k0 are skipped.
  __device__ __forceinline__ void row_from(uint32_t k0, uint32_t lane, uint8_t *row) const {
    if (k0 == 0) row[lane] = (uint8_t)cw;
    if (k0 <= 1) row[lane + 32] = (uint8_t)(cw >> 8);
    if (k0 <= 2) row[lane + 64] = (uint8_t)(cw >> 16);
    if (k0 <= 3) row[lane + 96] = (uint8_t)(cw >> 24);
    if (k0 <= 4) row[lane + 128] = (uint8_t)c4;
  }
  // Pixel of column lane + 32k (the lane's own column); prepare() has run
  // since the last write.
  __device__ __forceinline__ uint32_t pixel_k(uint32_t k) const { return __byte_perm(cw, c4, k); }
  // The HMOVE bar blanks columns 0..7 of its line.
  __device__ __forceinline__ void hmove_bar(uint32_t lane, uint32_t line, uint8_t *row) const {
    if (line == bar && lane < 8) row[lane] = 0;
  }
};

// Render one frame with one warp.  recs: log records; row_buf: 160 bytes of
// shared memory private to this warp; out: 210x160 frame.
__device__ inline void render_frame_warp(RenderRegs &R, const uint32_t *recs, uint32_t n_rec, uint32_t n_lines,
                                         uint8_t *row_buf, uint8_t *out) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t ri = 0, base = 0;
  uint32_t chunk = lane < n_rec ? recs[lane] : 0xFFFFFFFFu;
  for (uint32_t r = 0; r < (uint32_t)FRAME_H; ++r) {
    const uint32_t line = WINDOW_Y0 + r;
    if (line >= n_lines) {
#pragma unroll
      for (int k = 0; k < 5; ++k) row_buf[lane + 32 * k] = 0;
    } else {
      const uint32_t cl = 228u * line, end = cl + 228u;
      uint32_t k = 0;
      while (ri < n_rec) {
        if (ri - base >= 32) {
          base += 32;
          chunk = base + lane < n_rec ? recs[base + lane] : 0xFFFFFFFFu;
        }
        const uint32_t rec = __shfl_sync(0xFFFFFFFFu, chunk, ri - base);
        const uint32_t c = rec >> 14;
        if (c >= end) break;
        R.prepare(k < 5 && cl + 68u + lane + 32u * k < c, lane);
        while (k < 5 && cl + 68u + lane + 32u * k < c) {
          row_buf[lane + 32 * k] = (uint8_t)R.pixel_k(k);
          ++k;
        }
        R.apply((rec >> 8) & 0x3F, rec & 0xFF, c);
        ++ri;
      }
      R.prepare(k < 5, lane);
      R.row_from(k, lane, row_buf);
      R.hmove_bar(lane, line, row_buf);
    }
    __syncwarp();
    const uint32_t *src = reinterpret_cast<const uint32_t *>(row_buf);
    uint32_t *dst = reinterpret_cast<uint32_t *>(out + r * FRAME_W);
    dst[lane] = src[lane];
    if (lane < 8) dst[32 + lane] = src[32 + lane];
    __syncwarp();
  }
}

// Exact integer area weights (units of 1/84 source pixel) of the 210x160 ->
// 84x84 resampling.  Output row i covers source rows [2.5 i, 2.5 i + 2.5):
// three rows with weights (84, 84, 42) for even i, (42, 84, 84) for odd i.
// Output column j covers [160 j / 84, 160 (j + 1) / 84): up to three columns.
__device__ __forceinline__ void col_weights(uint32_t j, uint32_t &x0, uint32_t &w0, uint32_t &w1, uint32_t &w2) {
  uint32_t a = 160u * j, b = a + 160u;
  x0 = a / 84u;
  uint32_t e0 = 84u * x0 + 84u;
  w0 = (e0 < b ? e0 : b) - a;
  uint32_t e1 = e0 + 84u;
  uint32_t s1 = e0;
  w1 = s1 < b ? ((e1 < b ? e1 : b) - s1) : 0u;
  w2 = 160u - w0 - w1;
}

}  // namespace atari
