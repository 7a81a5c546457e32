// Batched form: persistent ROM-grouped interpreter and fused replay +
// preprocessing.
//
// Interpreter: envs are grouped by cartridge into work items of E envs
// (E = warps per block x envs per warp; a warp may run fewer than 32 envs,
// which trades SIMT width for more independent instruction streams when the
// batch is small).  Each block takes work items from an atomic queue, stages
// the item's cartridge in shared memory when it differs from the one it
// holds, and runs every env of the item for the whole step.
//
// Fused replay + preprocessing (the paper's TIA kernel with the rows of a
// frame spread over several warps, followed by the agent's preprocessing):
// one block per env renders frames F-1 and F into shared memory, takes the
// pixelwise maximum of their lumas, resamples to 84x84 and pushes the plane
// into the env's stack; frames never reach HBM.
#pragma once
#include <cstdint>

#include "device_machine.cuh"
#include "fast_console.cuh"
#include "render.cuh"

namespace atari {

struct BatchArgs {
  uint8_t *state;
  const uint8_t *cache;
  const uint8_t *romb;       // [n_roms][ROMB_SLOT] cartridge bytes, banks of 4096
  const uint32_t *info;      // per ROM: scheme | score << 8 | gameover << 16 | banks << 24
  const uint8_t *dec_op;     // 512 bytes: op per opcode, then mode/cycles/penalty per opcode
  const uint8_t *actions;
  int32_t *rew_int;
  uint8_t *done_int;
  int32_t *rew_out;
  uint8_t *done_out;
  uint32_t *log;
  uint8_t *snap;
  uint8_t *bsnap;            // null, or [n][2][3][64] quarter-frame band start snapshots
  uint32_t *meta;
  uint32_t *counters;
  const int32_t *grp_rom, *grp_start, *grp_count, *perm;
  const int32_t *opos;       // null, or the packed action/output position of each work-list entry
  int *queue;
  int n_groups, lanes, E, rom_stage;  // rom_stage: bytes staged per block (largest cartridge)
  int frameskip, sticky, n_cache, log_cap, first_slot;
  int tia_off;               // split form test mode: the TIA side takes no events
  int idle;                  // retire RIOT-timer wait-loop iterations at once
  uint64_t seed;
};

__device__ __forceinline__ void fast_reset_from_cache(uint8_t *st, const uint8_t *cache, uint32_t score,
                                                      uint32_t rom, uint32_t n_cache, uint64_t seed,
                                                      uint32_t env_key, uint32_t episode) {
  uint32_t idx = scale32(philox_x0(seed, env_key, 0u, PURPOSE_RESET << 8, episode), n_cache);
  const uint8_t *src = cache + ((size_t)rom * n_cache + idx) * 256;
  const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
  uint4 *d4 = reinterpret_cast<uint4 *>(st);
#pragma unroll
  for (int i = 0; i < 6; ++i) d4[i] = s4[i];
#pragma unroll
  for (int i = 8; i < 16; ++i) d4[i] = s4[i];
  st[S::LAST_ACTION] = 0;
  st[S::SCORE_PREV] = src[S::RAM + score];
  *reinterpret_cast<uint32_t *>(st + S::EPISODE) = episode;
}

// Env slot i; o = where its action is read and its reward and done written.
// Split form: logged-frame setup, frame records and the log count happen on
// the TIA side, in queue order; the step ends once the TIA side has caught up.
template <bool SPLIT, bool COMPACT>
__device__ __forceinline__ void fast_step_env(FastConsoleT<SPLIT, COMPACT> &m, uint8_t *st, int i, int o, const BatchArgs &a,
                                              uint32_t rom, uint32_t score, uint32_t gameover) {
  const uint32_t *ew = reinterpret_cast<const uint32_t *>(st + S::EPISODE);
  uint32_t episode = ew[0], step_no = ew[1], env_key = ew[2], env_status = ew[3];
  uint32_t last = st[S::LAST_ACTION];
  uint32_t score_prev = st[S::SCORE_PREV];
  uint32_t action = a.actions[o];
  if (action >= 18) { env_status |= ST_BAD_ACTION; action = 0; }
  int32_t reward = 0;
  uint32_t log_total = 0;
  const int F = a.frameskip;
  for (int f = 1; f <= F; ++f) {
    uint32_t act = action;
    if (a.sticky) {
      uint32_t u = philox_x0(a.seed, env_key, step_no, (uint32_t)f | PURPOSE_STICKY << 8, episode);
      if (u < 0x40000000u) act = last;
    }
    last = act;
    m.apply_action(act);
    const int slot = f - (F - 1);
    const bool logging = slot >= a.first_slot;
    if constexpr (SPLIT) {
      if (logging) m.push(EV_BEGIN_LOG | (uint32_t)slot);
      m.run_frame();
      if (logging) m.push(EV_END_LOG | (uint32_t)slot);
    } else {
      if (logging) {
        m.snapshot(a.snap + ((size_t)i * 2 + slot) * 64);
        m.set_log(a.log + ((size_t)i * 2 + slot) * a.log_cap, (uint32_t)a.log_cap,
                  a.bsnap ? a.bsnap + ((size_t)i * 2 + slot) * 3 * 64 : nullptr);
      } else {
        m.set_log(nullptr, 0, nullptr);
      }
      const uint32_t lines = m.run_frame();
      if (logging) {
        m.finish_bands();
        uint32_t *mt = a.meta + ((size_t)i * 2 + slot) * 2;
        const uint32_t nrec = m.log_count();
        mt[0] = nrec;
        mt[1] = lines;
        log_total += nrec;
      }
    }
    const uint32_t s = m.ram[score];
    reward += (int32_t)(int8_t)(uint8_t)(s - score_prev);
    score_prev = s;
  }
  if constexpr (SPLIT) {
    m.push(EV_STEP_END);
    m.wait_ack(m.nreq + 1);
  }
  env_status |= m.all_status();
  if (m.jam) env_status |= ST_ILLEGAL;
  const uint32_t done = (m.ram[gameover] != 0 || m.jam) ? 1u : 0u;
  a.rew_int[i] = reward;
  a.done_int[i] = (uint8_t)done;
  if (a.rew_out) a.rew_out[o] = reward;
  if (a.done_out) a.done_out[o] = (uint8_t)done;
  if (a.counters) {
    a.counters[3 * i] = m.instret;
    a.counters[3 * i + 2] = m.rounds;
    if constexpr (!SPLIT) a.counters[3 * i + 1] = log_total;
  }
  uint32_t *ewo = reinterpret_cast<uint32_t *>(st + S::EPISODE);
  ewo[1] = step_no + 1;
  ewo[3] = env_status;
  if (done) {
    fast_reset_from_cache(st, a.cache, score, rom, (uint32_t)a.n_cache, a.seed, env_key, episode + 1);
  } else {
    m.store(st);
    st[S::LAST_ACTION] = (uint8_t)last;
    st[S::SCORE_PREV] = (uint8_t)score_prev;
  }
}

// TIA side of the split form for env slot i: applies the CPU side's events in
// order until the end of the step.  Every wait is bounded; running out sets
// ST_STALL and ends the loop.
__device__ void tia_worker(IoCtx c, const uint32_t *q, int i, const BatchArgs &a) {
  if (a.tia_off) return;
  volatile uint32_t *vw = reinterpret_cast<volatile uint32_t *>(c.w());
  const volatile uint32_t *vq = reinterpret_cast<const volatile uint32_t *>(q);
  uint32_t head = 0, ack = 0, lines = 0, log_total = 0;
  uint64_t idle_since = 0;  // global-timer time the queue was first seen empty (0: not idle)
  for (;;) {
    if (head == vw[IO_QTAIL]) {
      const uint64_t now = global_ns();
      if (!idle_since) idle_since = now;
      else if (now - idle_since >= WAIT_NS) {
        c.Sset(IO_STATUS, c.G(IO_STATUS) | ST_STALL);
        break;
      }
      __nanosleep(128);  // an idle TIA lane polls gently: the CPU warps share the SM's memory pipe
      continue;
    }
    idle_since = 0;
    __threadfence_block();
    const uint32_t ev = vq[head & (QLEN - 1)];
    vw[IO_QHEAD] = ++head;
    const uint32_t kind = ev >> 30;
    if (kind == 0) {
      fc_tia_write(c, (ev >> 8) & 0x3F, ev & 0xFF, (ev >> 14) & 0xFFFF, false);
    } else if (kind == 1) {
      lines = ev & 0x3FFF;
      fc_frame_end(c, (ev >> 14) & 0xFFFF, lines);
    } else {
      const uint32_t sub = (ev >> 28) & 3, slot = ev & 1;
      if (sub == 0) {
        fc_snapshot(c, a.snap + ((size_t)i * 2 + slot) * 64, 0);
        fc_set_log(c, a.log + ((size_t)i * 2 + slot) * a.log_cap, (uint32_t)a.log_cap,
                   a.bsnap ? a.bsnap + ((size_t)i * 2 + slot) * 3 * 64 : nullptr);
      } else if (sub == 1) {
        if (c.G(IO_BANDN) < 4) fc_band_snap(c, ~0u);
        const uint32_t nrec = c.G(IO_LOGN);
        uint32_t *mt = a.meta + ((size_t)i * 2 + slot) * 2;
        mt[0] = nrec;
        mt[1] = lines;
        log_total += nrec;
        fc_set_log(c, nullptr, 0, nullptr);
      } else if (sub == 2) {
        fc_cx_eval(c, 3u * (ev & 0xFFFFu));
        __threadfence_block();
        vw[IO_ACK] = ++ack;
      } else {
        if (a.counters) a.counters[3 * i + 1] = log_total;
        __threadfence_block();
        vw[IO_ACK] = ++ack;
        break;
      }
    }
  }
}

template <bool COMPACT>
__global__ void __launch_bounds__(128) k_interp_batched(BatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t *rom8 = smem;                                  // rom_stage bytes, then 16 of padding
  uint8_t *dec_op = smem + (size_t)a.rom_stage + 16;
  uint8_t *ram = dec_op + 512;
  uint32_t *iow = reinterpret_cast<uint32_t *>(ram + RAM_BYTES * a.E);
  uint8_t *tia = reinterpret_cast<uint8_t *>(iow + IO_STRIDE * a.E);
  __shared__ int s_group;
  for (int t = threadIdx.x; t < 512; t += blockDim.x) dec_op[t] = a.dec_op[t];
  int cur_rom = -1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();  // everyone is done with the previous item (ROM words, s_group)
    if (threadIdx.x == 0) s_group = atomicAdd(a.queue, 1);
    __syncthreads();
    const int g = s_group;
    if (g >= a.n_groups) break;
    const int rom = a.grp_rom[g];
    if (rom != cur_rom) {
      const uint32_t banks = a.info[rom] >> 24;
      const uint4 *src = reinterpret_cast<const uint4 *>(a.romb + (size_t)rom * ROMB_SLOT);
      uint4 *dst = reinterpret_cast<uint4 *>(rom8);
      for (uint32_t q = threadIdx.x; q < banks * 256u; q += blockDim.x) dst[q] = src[q];
      if (threadIdx.x == 0) dst[banks * 256u] = make_uint4(0, 0, 0, 0);
      cur_rom = rom;
      __syncthreads();
    }
    const int jj = warp * a.lanes + lane;
    const bool runs = lane < a.lanes && jj < a.grp_count[g];
    const uint32_t wmask = __ballot_sync(0xFFFFFFFFu, runs);
    if (runs) {
      const int j = jj;
      {
        const int p = a.grp_start[g] + j;
        const int i = a.perm[p];
        const int o = a.opos ? a.opos[p] : i;
        uint8_t *st = a.state + (size_t)i * 256;
        const uint32_t inf = a.info[rom];
        FastConsoleT<false, COMPACT> m;
        m.rom8 = rom8;
        m.dec_op = dec_op;
        m.ram = ram + RAM_BYTES * j;
        m.io = IoCtx{tia + TIA_STRIDE * j, iow + IO_STRIDE * j};
        m.scheme = inf & 0xFF;
        m.wmask = wmask;
        m.idle = (uint32_t)a.idle;
        m.load(st);
        fast_step_env(m, st, i, o, a, (uint32_t)rom, (inf >> 8) & 0x7F, (inf >> 16) & 0x7F);
      }
    }
  }
}

// Split form: blockDim = 2 W warps; warps [0, W) run the CPUs of the work
// item's envs, warp W + w the TIA side of CPU warp w's envs (lane for lane).
// Shared memory: cartridge stage, decoder table, per-env RAM, I/O words, TIA
// file, then the per-env event queues.
template <bool COMPACT>
__global__ void __launch_bounds__(256, 2) k_interp_split(BatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t *rom8 = smem;
  uint8_t *dec_op = smem + (size_t)a.rom_stage + 16;
  uint8_t *ram = dec_op + 512;
  uint32_t *iow = reinterpret_cast<uint32_t *>(ram + RAM_BYTES * a.E);
  uint8_t *tia = reinterpret_cast<uint8_t *>(iow + IO_STRIDE * a.E);
  uint32_t *qs = reinterpret_cast<uint32_t *>(tia + TIA_STRIDE * a.E);
  __shared__ int s_group;
  for (int t = threadIdx.x; t < 512; t += blockDim.x) dec_op[t] = a.dec_op[t];
  int cur_rom = -1;
  const int W = a.E / a.lanes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool cpu = warp < W;
  const int cw = cpu ? warp : warp - W;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_group = atomicAdd(a.queue, 1);
    __syncthreads();
    const int g = s_group;
    if (g >= a.n_groups) break;
    const int rom = a.grp_rom[g];
    if (rom != cur_rom) {
      const uint32_t banks = a.info[rom] >> 24;
      const uint4 *src = reinterpret_cast<const uint4 *>(a.romb + (size_t)rom * ROMB_SLOT);
      uint4 *dst = reinterpret_cast<uint4 *>(rom8);
      for (uint32_t q = threadIdx.x; q < banks * 256u; q += blockDim.x) dst[q] = src[q];
      if (threadIdx.x == 0) dst[banks * 256u] = make_uint4(0, 0, 0, 0);
      cur_rom = rom;
      __syncthreads();
    }
    const int jj = cw * a.lanes + lane;
    const bool runs = lane < a.lanes && jj < a.grp_count[g];
    const uint32_t wmask = __ballot_sync(0xFFFFFFFFu, runs);
    const int p = a.grp_start[g] + jj;
    const int i = runs ? a.perm[p] : 0;
    const int o = runs ? (a.opos ? a.opos[p] : i) : 0;
    uint8_t *st = a.state + (size_t)i * 256;
    const uint32_t inf = a.info[rom];
    const IoCtx io{tia + TIA_STRIDE * jj, iow + IO_STRIDE * jj};
    uint32_t *q = qs + QSTRIDE * jj;
    FastConsoleT<true, COMPACT> m;
    if (cpu && runs) {
      m.rom8 = rom8;
      m.dec_op = dec_op;
      m.ram = ram + RAM_BYTES * jj;
      m.io = io;
      m.q = q;
      m.scheme = inf & 0xFF;
      m.wmask = wmask;
      m.idle = (uint32_t)a.idle;
      m.load(st);
    }
    __syncthreads();  // the envs' state is in shared memory before the TIA side starts
    if (runs) {
      if (cpu) fast_step_env<true, COMPACT>(m, st, i, o, a, (uint32_t)rom, (inf >> 8) & 0x7F, (inf >> 16) & 0x7F);
      else tia_worker(io, q, i, a);
    }
  }
}

// Bank-aware grouping: within each cartridge's run [seg[r], seg[r+1]) of the
// env list, envs are ordered by the bank their canonical state holds at the
// start of the step (byte 5, reduced to the cartridge's bank bits), stable in
// env order, so the lanes of a warp start the step in one bank.  A counting
// sort with up to eight keys (F4); one block of 256 threads per cartridge.
// Cartridges with one bank keep the list as it is.
__global__ void __launch_bounds__(256) k_group_by_bank(const uint8_t *state, const int32_t *perm_in,
                                                        const int32_t *seg, const uint32_t *info, int32_t *perm_out) {
  constexpr uint32_t KEYS = 8;
  const int r = blockIdx.x;
  const int a = seg[r], b = seg[r + 1];
  const uint32_t banks = info[r] >> 24;
  if (banks <= 1) {
    for (int p = a + (int)threadIdx.x; p < b; p += blockDim.x) perm_out[p] = perm_in[p];
    return;
  }
  const uint32_t mask = banks - 1;  // 1 for F8, 3 for F6, 7 for F4
  __shared__ int cnt[KEYS], base[KEYS], wcnt[8][KEYS];
  if (threadIdx.x < KEYS) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int p = a + (int)threadIdx.x; p < b; p += blockDim.x)
    atomicAdd(&cnt[state[(size_t)perm_in[p] * 256 + 5] & mask], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = a;
    for (uint32_t v = 0; v < KEYS; ++v) { base[v] = s; s += cnt[v]; }
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p0 = a; p0 < b; p0 += blockDim.x) {
    const int p = p0 + (int)threadIdx.x;
    const bool valid = p < b;
    const int env = valid ? perm_in[p] : 0;
    const uint32_t bk = valid ? (state[(size_t)env * 256 + 5] & mask) : 0u;
    uint32_t rank = 0;
#pragma unroll
    for (uint32_t v = 0; v < KEYS; ++v) {
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, valid && bk == v);
      if (lane == 0) wcnt[warp][v] = __popc(m);
      if (valid && bk == v) rank = __popc(m & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (valid) {
      int off = 0;
      for (uint32_t w2 = 0; w2 < warp; ++w2) off += wcnt[w2][bk];
      perm_out[base[bk] + off + (int)rank] = env;
    }
    __syncthreads();
    if (threadIdx.x < KEYS) {
      int t = 0;
      for (int w2 = 0; w2 < 8; ++w2) t += wcnt[w2][threadIdx.x];
      base[threadIdx.x] += t;
    }
    __syncthreads();
  }
}

// Render rows [r0, r1) of one frame with one warp into a shared-memory frame.
// R holds the render state after records [0, ri0); records from ri0 on that
// take effect before the band's first row are applied first.
__device__ inline void render_rows_warp(RenderRegs &R, const uint32_t *recs, uint32_t n_rec, uint32_t n_lines,
                                        uint32_t r0, uint32_t r1, uint8_t *frame, uint32_t ri0) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t ri = ri0, base = ri0;
  uint32_t chunk = base + lane < n_rec ? recs[base + lane] : 0xFFFFFFFFu;
  // records that take effect before the band's first row: apply only
  const uint32_t start_clk = 228u * (WINDOW_Y0 + r0);
  while (ri < n_rec) {
    if (ri - base >= 32) {
      base += 32;
      chunk = base + lane < n_rec ? recs[base + lane] : 0xFFFFFFFFu;
    }
    const uint32_t rec = __shfl_sync(0xFFFFFFFFu, chunk, ri - base);
    const uint32_t c = rec >> 14;
    if (c >= start_clk) break;
    R.apply((rec >> 8) & 0x3F, rec & 0xFF, c);
    ++ri;
  }
  for (uint32_t r = r0; r < r1; ++r) {
    uint8_t *row = frame + r * FRAME_W;
    const uint32_t line = WINDOW_Y0 + r;
    if (line >= n_lines) {
#pragma unroll
      for (int k = 0; k < 5; ++k) row[lane + 32 * k] = 0;
      continue;
    }
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
        row[lane + 32 * k] = (uint8_t)R.pixel_k(k);
        ++k;
      }
      R.apply((rec >> 8) & 0x3F, rec & 0xFF, c);
      ++ri;
    }
    R.prepare(k < 5, lane);
    R.row_from(k, lane, row);
    R.hmove_bar(lane, line, row);
  }
}

// One block per env: warps [0, W) render frame F-1, warps [W, 2W) frame F,
// each warp a band of rows; then luma max, 84x84 area resampling, stack push.
__global__ void __launch_bounds__(256, 3) k_raster_preprocess(const uint32_t *log, const uint8_t *snap, const uint8_t *bsnap,
                                                           const uint32_t *meta,
                                                           const uint8_t *luma_g, uint8_t *ring, uint8_t *head,
                                                           const uint8_t *done, uint8_t *obs, int n, int log_cap,
                                                           int warps_per_frame, const int32_t *perm,
                                                           const int32_t *opos, int base) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint8_t *fa = sm;                        // frame F-1, later the luma maximum
  uint8_t *fb = sm + FRAME_H * FRAME_W;    // frame F
  uint8_t *luma = fb + FRAME_H * FRAME_W;
  uint8_t *plane = luma + 128;
  // block b (counted from base) serves env slot perm[b] and writes its stack
  // at position opos[b]
  const int blk = base + (int)blockIdx.x;
  if (blk >= n) return;
  const int i = perm ? perm[blk] : blk;
  const int o = opos ? opos[blk] : i;
  const int warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < 128; t += blockDim.x) luma[t] = luma_g[t];
  if (warp < 2 * warps_per_frame) {
    const int slot = warp / warps_per_frame, band = warp % warps_per_frame;
    const uint32_t r0 = (uint32_t)(FRAME_H * band / warps_per_frame);
    const uint32_t r1 = (uint32_t)(FRAME_H * (band + 1) / warps_per_frame);
    const size_t fs = (size_t)i * 2 + slot;
    const uint32_t *mt = meta + fs * 2;
    const uint32_t n_rec = mt[0] < (uint32_t)log_cap ? mt[0] : (uint32_t)log_cap;
    // a band starting at a quarter of the frame starts from the interpreter's
    // snapshot there; the first band from the frame's start
    const uint32_t q = (uint32_t)(band * 4 / warps_per_frame);
    RenderRegs R;
    uint32_t ri0 = 0;
    if (bsnap && q > 0 && (band * 4) % warps_per_frame == 0) {
      const uint8_t *bs = bsnap + (fs * 3 + q - 1) * 64;
      R.load(bs);
      ri0 = reinterpret_cast<const uint32_t *>(bs)[14];
      ri0 = ri0 < n_rec ? ri0 : n_rec;
    } else {
      R.load(snap + fs * 64);
    }
    render_rows_warp(R, log + fs * log_cap, n_rec, mt[1], r0, r1, slot ? fb : fa, ri0);
  }
  __syncthreads();
  {
    uint32_t *a4 = reinterpret_cast<uint32_t *>(fa);
    const uint32_t *b4 = reinterpret_cast<const uint32_t *>(fb);
    for (int q = threadIdx.x; q < FRAME_H * FRAME_W / 4; q += blockDim.x) {
      uint32_t x = a4[q], y = b4[q], r = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t la = luma[((x >> (8 * k)) & 0xFF) >> 1], lb = luma[((y >> (8 * k)) & 0xFF) >> 1];
        r |= (la > lb ? la : lb) << (8 * k);
      }
      a4[q] = r;
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 84 * 84; o += blockDim.x) {
    uint32_t oi = o / 84, oj = o % 84;
    uint32_t y0 = (5u * oi) >> 1;
    uint32_t wy0 = (oi & 1) ? 42u : 84u, wy1 = 84u, wy2 = (oi & 1) ? 84u : 42u;
    uint32_t x0, wx0, wx1, wx2;
    col_weights(oj, x0, wx0, wx1, wx2);
    const uint8_t *r0 = fa + y0 * FRAME_W + x0;
    const uint8_t *r1 = r0 + FRAME_W;
    const uint8_t *r2 = r1 + FRAME_W;
    uint32_t rs0 = wx0 * r0[0] + wx1 * r0[1] + (wx2 ? wx2 * r0[2] : 0u);
    uint32_t rs1 = wx0 * r1[0] + wx1 * r1[1] + (wx2 ? wx2 * r1[2] : 0u);
    uint32_t rs2 = wx0 * r2[0] + wx1 * r2[1] + (wx2 ? wx2 * r2[2] : 0u);
    plane[o] = (uint8_t)((wy0 * rs0 + wy1 * rs1 + wy2 * rs2 + 16800u) / 33600u);
  }
  __syncthreads();
  const uint32_t h = head[i];
  uint8_t *rg = ring + (size_t)i * 4 * 7056;
  const uint32_t *pl32 = reinterpret_cast<const uint32_t *>(plane);
  if (obs) {
    uint8_t *ob = obs + (size_t)o * 4 * 7056;
    for (int s = 0; s < 3; ++s) {
      const uint4 *src = reinterpret_cast<const uint4 *>(rg + ((h + 1 + s) & 3) * 7056);
      uint4 *dst = reinterpret_cast<uint4 *>(ob + s * 7056);
      for (int q = threadIdx.x; q < 7056 / 16; q += blockDim.x) dst[q] = src[q];
    }
    const uint4 *p16 = reinterpret_cast<const uint4 *>(plane);
    uint4 *dst = reinterpret_cast<uint4 *>(ob + 3 * 7056);
    for (int q = threadIdx.x; q < 7056 / 16; q += blockDim.x) dst[q] = p16[q];
  }
  __syncthreads();
  if (done[i]) {
    uint4 *z = reinterpret_cast<uint4 *>(rg);
    for (int q = threadIdx.x; q < 4 * 7056 / 16; q += blockDim.x) z[q] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) head[i] = 0;
  } else {
    uint32_t *dst = reinterpret_cast<uint32_t *>(rg + h * 7056);
    for (int q = threadIdx.x; q < 7056 / 4; q += blockDim.x) dst[q] = pl32[q];
    if (threadIdx.x == 0) head[i] = (uint8_t)((h + 1) & 3);
  }
}

}  // namespace atari
