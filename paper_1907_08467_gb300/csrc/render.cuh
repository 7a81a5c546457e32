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
  uint32_t vblank, nusiz0, nusiz1, colup0, colup1, colupf, colubk, ctrlpf, refp0, refp1;
  uint32_t pf0, pf1, pf2, enam0, enam1, enabl_new, enabl_old, grp0_new, grp0_old, grp1_new, grp1_old;
  uint32_t vdelp0, vdelp1, vdelbl, resmp0, resmp1, hmp0, hmp1, hmm0, hmm1, hmbl;
  uint32_t p0, p1, m0, m1, bl;
  uint32_t bar;  // frame-relative line of the HMOVE bar, or ~0u
  // Per lane: bit k of v_* = the object covers column lane + 32k (players,
  // missiles and ball with their enables, playfield).  Rebuilt from the
  // objects' 160-bit masks for the objects in `dirty` before the next pixel.
  uint32_t vp0, vp1, vm0, vm1, vbl, vpf;
  uint32_t dirty;  // 1 P0, 2 P1, 4 M0, 8 M1, 16 BL, 32 PF

  // from a 64-byte snapshot (canonical bytes 0x20..0x5F)
  __device__ void load(const uint8_t *t) {
    vblank = t[1]; nusiz0 = t[2]; nusiz1 = t[3]; colup0 = t[4]; colup1 = t[5]; colupf = t[6]; colubk = t[7];
    ctrlpf = t[8]; refp0 = t[9]; refp1 = t[10]; pf0 = t[11]; pf1 = t[12]; pf2 = t[13]; enam0 = t[14];
    enam1 = t[15]; enabl_new = t[16]; enabl_old = t[17]; grp0_new = t[18]; grp0_old = t[19]; grp1_new = t[20];
    grp1_old = t[21]; vdelp0 = t[22]; vdelp1 = t[23]; vdelbl = t[24]; resmp0 = t[25]; resmp1 = t[26];
    hmp0 = t[27]; hmp1 = t[28]; hmm0 = t[29]; hmm1 = t[30]; hmbl = t[31];
    p0 = t[32]; p1 = t[33]; m0 = t[34]; m1 = t[35]; bl = t[36];
    uint64_t b = 0, l0 = 0;
    for (int i = 7; i >= 0; --i) { b = (b << 8) | t[40 + i]; l0 = (l0 << 8) | t[48 + i]; }
    bar = (b != NO_LINE && b >= l0 && b - l0 < 1024) ? (uint32_t)(b - l0) : ~0u;
    dirty = 63;
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
  // Apply a logged write (effect clock eff, frame-relative).
  __device__ void apply(uint32_t reg, uint32_t v, uint32_t eff) {
    switch (reg) {
      case 0x01: vblank = v; break;
      case 0x04: nusiz0 = v; dirty |= 1 | 4; break;
      case 0x05: nusiz1 = v; dirty |= 2 | 8; break;
      case 0x06: colup0 = v; break;
      case 0x07: colup1 = v; break;
      case 0x08: colupf = v; break;
      case 0x09: colubk = v; break;
      case 0x0A: ctrlpf = v; dirty |= 16 | 32; break;
      case 0x0B: refp0 = v; dirty |= 1; break;
      case 0x0C: refp1 = v; dirty |= 2; break;
      case 0x0D: pf0 = v; dirty |= 32; break;
      case 0x0E: pf1 = v; dirty |= 32; break;
      case 0x0F: pf2 = v; dirty |= 32; break;
      case 0x10: p0 = res_pos(eff, 5, 3); dirty |= 1; break;
      case 0x11: p1 = res_pos(eff, 5, 3); dirty |= 2; break;
      case 0x12: m0 = res_pos(eff, 4, 2); dirty |= 4; break;
      case 0x13: m1 = res_pos(eff, 4, 2); dirty |= 8; break;
      case 0x14: bl = res_pos(eff, 4, 2); dirty |= 16; break;
      case 0x1B: grp0_new = v; grp1_old = grp1_new; dirty |= 1 | 2; break;
      case 0x1C: grp1_new = v; grp0_old = grp0_new; enabl_old = enabl_new; dirty |= 1 | 2 | 16; break;
      case 0x1D: enam0 = v; dirty |= 4; break;
      case 0x1E: enam1 = v; dirty |= 8; break;
      case 0x1F: enabl_new = v; dirty |= 16; break;
      case 0x20: hmp0 = v; break;
      case 0x21: hmp1 = v; break;
      case 0x22: hmm0 = v; break;
      case 0x23: hmm1 = v; break;
      case 0x24: hmbl = v; break;
      case 0x25: vdelp0 = v; dirty |= 1; break;
      case 0x26: vdelp1 = v; dirty |= 2; break;
      case 0x27: vdelbl = v; dirty |= 16; break;
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

  static __device__ __forceinline__ uint32_t lane_bits(const M160 &m, uint32_t lane) {
    return ((m.w0 >> lane) & 1u) | ((m.w1 >> lane) & 1u) << 1 | ((m.w2 >> lane) & 1u) << 2 |
           ((m.w3 >> lane) & 1u) << 3 | ((m.w4 >> lane) & 1u) << 4;
  }
  __device__ __forceinline__ void refresh(uint32_t lane) {
    if (dirty & 1) {
      const uint32_t g = (vdelp0 & 1) ? grp0_old : grp0_new;
      vp0 = g ? lane_bits(player_mask(g, refp0, nusiz0, p0), lane) : 0u;
    }
    if (dirty & 2) {
      const uint32_t g = (vdelp1 & 1) ? grp1_old : grp1_new;
      vp1 = g ? lane_bits(player_mask(g, refp1, nusiz1, p1), lane) : 0u;
    }
    if (dirty & 4) vm0 = ((enam0 & 2) && !(resmp0 & 2)) ? lane_bits(missile_mask(nusiz0, m0), lane) : 0u;
    if (dirty & 8) vm1 = ((enam1 & 2) && !(resmp1 & 2)) ? lane_bits(missile_mask(nusiz1, m1), lane) : 0u;
    if (dirty & 16) vbl = ((((vdelbl & 1) ? enabl_old : enabl_new) & 2)) ? lane_bits(ball_mask(ctrlpf, bl), lane) : 0u;
    if (dirty & 32) vpf = lane_bits(pf_mask(pf0, pf1, pf2, ctrlpf), lane);
    dirty = 0;
  }
  // Rebuild the stale coverage bits if any lane of the warp is about to draw
  // (draws = this lane has a pixel to draw before the next register write).
  // Every lane applies the same writes, so `dirty` is the same in all lanes
  // and the rebuild runs once for the whole warp.
  __device__ __forceinline__ void prepare(bool draws, uint32_t lane) {
    if (__any_sync(0xFFFFFFFFu, draws && dirty != 0)) refresh(lane);
  }
  // All five pixels of the lane on a line drawn from one register state
  // (no write lands between them): pixel_k for k = 0..4 with the blanking
  // and priority tests taken once.
  __device__ __forceinline__ void row5(uint32_t lane, uint32_t line, uint8_t *row) const {
    if (vblank & 2) {
#pragma unroll
      for (int k = 0; k < 5; ++k) row[lane + 32 * k] = 0;
      return;
    }
    const uint32_t a = vp0 | vm0, b = vp1 | vm1, f = vpf, l = vbl;
    uint32_t c[5];
    if (ctrlpf & 4) {
#pragma unroll
      for (int k = 0; k < 5; ++k)
        c[k] = (((f | l) >> k) & 1u) ? colupf : ((a >> k) & 1u) ? colup0 : ((b >> k) & 1u) ? colup1 : colubk;
    } else {
      const uint32_t pl = (ctrlpf & 2) ? colup0 : colupf, pr = (ctrlpf & 2) ? colup1 : colupf;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const bool half = k >= 3 || (k == 2 && lane >= 16u);  // column lane + 32k >= 80
        c[k] = ((a >> k) & 1u) ? colup0 : ((b >> k) & 1u) ? colup1 : ((f >> k) & 1u) ? (half ? pr : pl)
             : ((l >> k) & 1u) ? colupf : colubk;
      }
    }
    if (line == bar && lane < 8) c[0] = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) row[lane + 32 * k] = (uint8_t)(c[k] & 0xFE);
  }
  // Pixel of column lane + 32k on a frame-relative line (the lane's own column);
  // prepare() has run since the last write.
  __device__ __forceinline__ uint32_t pixel_k(uint32_t k, uint32_t lane, uint32_t line) const {
    if ((vblank & 2) || (k == 0 && line == bar && lane < 8)) return 0;
    const bool P0 = (vp0 >> k) & 1u, P1 = (vp1 >> k) & 1u, M0 = (vm0 >> k) & 1u, M1 = (vm1 >> k) & 1u;
    const bool BL = (vbl >> k) & 1u, PF = (vpf >> k) & 1u;
    const bool half = lane + 32u * k >= 80u;
    uint32_t c;
    if (ctrlpf & 4) {
      c = (PF || BL) ? colupf : (P0 || M0) ? colup0 : (P1 || M1) ? colup1 : colubk;
    } else {
      c = (P0 || M0) ? colup0 : (P1 || M1) ? colup1
          : PF ? ((ctrlpf & 2) ? (half ? colup1 : colup0) : colupf)
          : BL ? colupf : colubk;
    }
    return c & 0xFE;
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
          row_buf[lane + 32 * k] = (uint8_t)R.pixel_k(k, lane, line);
          ++k;
        }
        R.apply((rec >> 8) & 0x3F, rec & 0xFF, c);
        ++ri;
      }
      R.prepare(k < 5, lane);
      if (__all_sync(0xFFFFFFFFu, k == 0)) R.row5(lane, line, row_buf);
      else
        for (; k < 5; ++k) row_buf[lane + 32 * k] = (uint8_t)R.pixel_k(k, lane, line);
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
