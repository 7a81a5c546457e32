// Batched Atari 2600 emulation on GB300 (sm_103a): kernels and the C ABI.
//
// Paper, Section 3 (CuLE): an Atari CPU kernel (one thread per emulator) and
// a TIA kernel (renders from the CPU kernel's buffer of TIA writes), frames
// rendered only where the agent needs them, reset from a cache of start
// states.  The step here is: interpreter (all F frames, logging the writes of
// frames F-1 and F) -> rasteriser -> preprocessing (luma, max of the two
// frames, exact 84x84 area resampling, 4-frame stack); finished episodes are
// reset inside the interpreter's epilogue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/atari_gpu.h"
#include "env_internal.h"
#include "device_machine.cuh"
#include "render.cuh"
#include "batched.cuh"
#include "policy.cuh"
#include "learner.cuh"

using namespace atari;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}
#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e__ = (expr);                                                            \
    if (e__ != cudaSuccess)                                                              \
      return fail(ATARI_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__));     \
  } while (0)

// ------------------------------------------------------------------ decode table
// The NMOS 6502 opcode matrix (row = high nibble, column = low nibble): the
// documented opcodes and the 84 undocumented ones with a stable published
// behaviour; empty cells (the 12 halting opcodes and ANE, LXA, SHA, SHX, SHY,
// TAS, LAS, ARR) halt the CPU.
const char *const OPMAP[256] = {
    "BRK imp", "ORA izx", 0, "SLO izx", "NOP zp", "ORA zp", "ASL zp", "SLO zp", "PHP imp", "ORA imm", "ASL acc", "ANC imm", "NOP abs", "ORA abs", "ASL abs", "SLO abs",
    "BPL rel", "ORA izy", 0, "SLO izy", "NOP zpx", "ORA zpx", "ASL zpx", "SLO zpx", "CLC imp", "ORA aby", "NOP imp", "SLO aby", "NOP abx", "ORA abx", "ASL abx", "SLO abx",
    "JSR abs", "AND izx", 0, "RLA izx", "BIT zp", "AND zp", "ROL zp", "RLA zp", "PLP imp", "AND imm", "ROL acc", "ANC imm", "BIT abs", "AND abs", "ROL abs", "RLA abs",
    "BMI rel", "AND izy", 0, "RLA izy", "NOP zpx", "AND zpx", "ROL zpx", "RLA zpx", "SEC imp", "AND aby", "NOP imp", "RLA aby", "NOP abx", "AND abx", "ROL abx", "RLA abx",
    "RTI imp", "EOR izx", 0, "SRE izx", "NOP zp", "EOR zp", "LSR zp", "SRE zp", "PHA imp", "EOR imm", "LSR acc", "ALR imm", "JMP abs", "EOR abs", "LSR abs", "SRE abs",
    "BVC rel", "EOR izy", 0, "SRE izy", "NOP zpx", "EOR zpx", "LSR zpx", "SRE zpx", "CLI imp", "EOR aby", "NOP imp", "SRE aby", "NOP abx", "EOR abx", "LSR abx", "SRE abx",
    "RTS imp", "ADC izx", 0, "RRA izx", "NOP zp", "ADC zp", "ROR zp", "RRA zp", "PLA imp", "ADC imm", "ROR acc", 0, "JMP ind", "ADC abs", "ROR abs", "RRA abs",
    "BVS rel", "ADC izy", 0, "RRA izy", "NOP zpx", "ADC zpx", "ROR zpx", "RRA zpx", "SEI imp", "ADC aby", "NOP imp", "RRA aby", "NOP abx", "ADC abx", "ROR abx", "RRA abx",
    "NOP imm", "STA izx", "NOP imm", "SAX izx", "STY zp", "STA zp", "STX zp", "SAX zp", "DEY imp", "NOP imm", "TXA imp", 0, "STY abs", "STA abs", "STX abs", "SAX abs",
    "BCC rel", "STA izy", 0, 0, "STY zpx", "STA zpx", "STX zpy", "SAX zpy", "TYA imp", "STA aby", "TXS imp", 0, 0, "STA abx", 0, 0,
    "LDY imm", "LDA izx", "LDX imm", "LAX izx", "LDY zp", "LDA zp", "LDX zp", "LAX zp", "TAY imp", "LDA imm", "TAX imp", 0, "LDY abs", "LDA abs", "LDX abs", "LAX abs",
    "BCS rel", "LDA izy", 0, "LAX izy", "LDY zpx", "LDA zpx", "LDX zpy", "LAX zpy", "CLV imp", "LDA aby", "TSX imp", 0, "LDY abx", "LDA abx", "LDX aby", "LAX aby",
    "CPY imm", "CMP izx", "NOP imm", "DCP izx", "CPY zp", "CMP zp", "DEC zp", "DCP zp", "INY imp", "CMP imm", "DEX imp", "SBX imm", "CPY abs", "CMP abs", "DEC abs", "DCP abs",
    "BNE rel", "CMP izy", 0, "DCP izy", "NOP zpx", "CMP zpx", "DEC zpx", "DCP zpx", "CLD imp", "CMP aby", "NOP imp", "DCP aby", "NOP abx", "CMP abx", "DEC abx", "DCP abx",
    "CPX imm", "SBC izx", "NOP imm", "ISC izx", "CPX zp", "SBC zp", "INC zp", "ISC zp", "INX imp", "SBC imm", "NOP imp", "SBC imm", "CPX abs", "SBC abs", "INC abs", "ISC abs",
    "BEQ rel", "SBC izy", 0, "ISC izy", "NOP zpx", "SBC zpx", "INC zpx", "ISC zpx", "SED imp", "SBC aby", "NOP imp", "ISC aby", "NOP abx", "SBC abx", "INC abx", "ISC abx",
};

const char *const MNEMONICS[] = {"JAM", "ADC", "AND", "ASL", "BCC", "BCS", "BEQ", "BIT", "BMI", "BNE", "BPL",
                                 "BRK", "BVC", "BVS", "CLC", "CLD", "CLI", "CLV", "CMP", "CPX", "CPY", "DEC",
                                 "DEX", "DEY", "EOR", "INC", "INX", "INY", "JMP", "JSR", "LDA", "LDX", "LDY",
                                 "LSR", "NOP", "ORA", "PHA", "PHP", "PLA", "PLP", "ROL", "ROR", "RTI", "RTS",
                                 "SBC", "SEC", "SED", "SEI", "STA", "STX", "STY", "TAX", "TAY", "TSX", "TXA",
                                 "TXS", "TYA", "SLO", "RLA", "SRE", "RRA", "SAX", "LAX", "DCP", "ISC", "ANC",
                                 "ALR", "SBX"};
const char *const MODES[] = {"imp", "acc", "imm", "zp", "zpx", "zpy", "abs", "abx", "aby", "ind", "izx", "izy", "rel"};

// Cycle counts from the documented timing rules of each instruction class.
uint32_t cycles_for(uint32_t op, uint32_t mode, bool &penalty) {
  penalty = false;
  switch (op) {
    case O_BRK: return 7;
    case O_JSR: case O_RTS: case O_RTI: return 6;
    case O_PHA: case O_PHP: return 3;
    case O_PLA: case O_PLP: return 4;
    case O_JMP: return mode == ABS ? 3 : 5;
    default: break;
  }
  if (mode == REL || mode == IMP) return 2;
  if (op == O_SLO || op == O_RLA || op == O_SRE || op == O_RRA || op == O_DCP || op == O_ISC) {
    switch (mode) {  // undocumented read-modify-write: always the long count
      case ZP: return 5; case ZPX: case ABS: return 6; case ABX: case ABY: return 7; default: return 8;  // izx, izy
    }
  }
  if (op == O_STA || op == O_STX || op == O_STY || op == O_SAX) {
    switch (mode) {
      case ZP: return 3; case ZPX: case ZPY: case ABS: return 4;
      case ABX: case ABY: return 5; default: return 6;  // izx, izy
    }
  }
  if (op == O_ASL || op == O_LSR || op == O_ROL || op == O_ROR || op == O_INC || op == O_DEC) {
    switch (mode) {
      case ACC: return 2; case ZP: return 5; case ZPX: case ABS: return 6; default: return 7;  // abx
    }
  }
  penalty = mode == ABX || mode == ABY || mode == IZY;
  switch (mode) {
    case IMM: return 2; case ZP: return 3; case ZPX: case ZPY: case ABS: case ABX: case ABY: return 4;
    case IZX: return 6; default: return 5;  // izy
  }
}

// t[256] <- per opcode: operation | mode << 8 | base cycles << 12 (4 bits) |
// page-cross penalty << 16; 0 for the opcodes that halt the CPU.
void fill_decode_table(uint32_t *t) {
  for (int o = 0; o < 256; ++o) {
    t[o] = 0;
    if (!OPMAP[o]) continue;
    char mn[4] = {OPMAP[o][0], OPMAP[o][1], OPMAP[o][2], 0};
    const char *md = OPMAP[o] + 4;
    uint32_t op = 0, mode = 0;
    for (uint32_t i = 0; i < sizeof(MNEMONICS) / sizeof(*MNEMONICS); ++i)
      if (!strcmp(MNEMONICS[i], mn)) op = i;
    for (uint32_t i = 0; i < sizeof(MODES) / sizeof(*MODES); ++i)
      if (!strcmp(MODES[i], md)) mode = i;
    bool pen;
    uint32_t cyc = cycles_for(op, mode, pen);
    t[o] = op | mode << 8 | cyc << 12 | (pen ? 1u : 0u) << 16;
  }
}

std::vector<uint32_t> build_decode_table() {
  std::vector<uint32_t> t(256, 0u);
  fill_decode_table(t.data());
  return t;
}

// The batched console's decode bytes: per opcode, operation | page-cross
// penalty << 7, then mode | cycles << 4.
std::vector<uint8_t> build_dec_op(const std::vector<uint32_t> &dec) {
  std::vector<uint8_t> d(512, 0);
  for (int o = 0; o < 256; ++o) {
    const uint32_t t = dec[o];
    d[o] = (uint8_t)((t & 0x7F) | ((t >> 16) & 1u) << 7);
    d[256 + o] = (uint8_t)(((t >> 8) & 0xFu) | ((t >> 12) & 0xFu) << 4);
  }
  return d;
}

int scheme_of(size_t sz);

// Cartridge info word: scheme | score RAM index << 8 | game-over RAM index
// << 16 | 4 KB banks << 24 (a 2 KB image counts as one bank).
uint32_t rom_info_word(size_t rom_size, const atari_rom_meta &meta) {
  return (uint32_t)scheme_of(rom_size) | (uint32_t)(meta.score_addr & 0x7F) << 8 |
         (uint32_t)(meta.gameover_addr & 0x7F) << 16 | (uint32_t)(rom_size <= 4096 ? 1u : rom_size / 4096) << 24;
}

// ------------------------------------------------------------------ kernels
constexpr int ROM_SLOT = 32768;  // bytes reserved per cartridge image on the device (the largest, F4)

struct RomInfo {
  uint32_t scheme, score, gameover;
};

__device__ __forceinline__ RomInfo rom_info(const uint32_t *info, uint32_t r) {
  uint32_t v = info[r];
  return RomInfo{v & 0xFF, (v >> 8) & 0x7F, (v >> 16) & 0x7F};
}

// Copy a cached start state into an env's canonical state and re-key the
// env fields (Section 3, reset strategy: a finished emulator takes a randomly
// chosen cached start state in place of its terminal state).
__device__ void reset_from_cache(uint8_t *st, const uint8_t *cache, const uint32_t *info, uint32_t rom,
                                 uint32_t n_cache, uint64_t seed, uint32_t env_key, uint32_t episode) {
  uint32_t idx = scale32(philox_x0(seed, env_key, 0u, PURPOSE_RESET << 8, episode), n_cache);
  const uint8_t *src = cache + ((size_t)rom * n_cache + idx) * 256;
  const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
  uint4 *d4 = reinterpret_cast<uint4 *>(st);
#pragma unroll
  for (int i = 0; i < 6; ++i) d4[i] = s4[i];     // 0x00..0x5F
#pragma unroll
  for (int i = 8; i < 16; ++i) d4[i] = s4[i];    // 0x80..0xFF
  RomInfo ri = rom_info(info, rom);
  st[S::LAST_ACTION] = 0;
  st[S::SCORE_PREV] = src[S::RAM + ri.score];
  Console<GlobalMem>::st32(st + S::EPISODE, episode);
}

// One block per ROM: from power-on, run the start-up frames, then keep a
// snapshot after each of the next max_noops + 1 frames.  Lane 0 runs the
// batched form's console (RAM, I/O state and the staged cartridge in shared
// memory), which steps the same machine as the plain console and is far
// faster than it for one sequential trajectory; the block stages the
// cartridge.  rom_stage = bytes of the largest cartridge.
__global__ void __launch_bounds__(128) k_cache_run(uint8_t *work, uint8_t *snaps, const uint8_t *roms,
                                                    const uint32_t *info, const uint8_t *dec_op_g, int rom_stage,
                                                    int startup, int max_noops) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t *rom8 = smem;                                   // rom_stage bytes, then 16 of padding
  uint8_t *dec_op = smem + (size_t)rom_stage + 16;
  uint8_t *ram = dec_op + 512;
  uint32_t *iow = reinterpret_cast<uint32_t *>(ram + RAM_BYTES);
  uint8_t *tia = reinterpret_cast<uint8_t *>(iow + IO_STRIDE);
  const int r = blockIdx.x;
  const uint32_t inf = info[r];
  const uint32_t banks = inf >> 24;
  const uint4 *src = reinterpret_cast<const uint4 *>(roms + (size_t)r * ROM_SLOT);
  uint4 *dst = reinterpret_cast<uint4 *>(rom8);
  for (uint32_t q = threadIdx.x; q < banks * 256u; q += blockDim.x) dst[q] = src[q];
  if (threadIdx.x == 0) dst[banks * 256u] = make_uint4(0, 0, 0, 0);
  for (int t = threadIdx.x; t < 512; t += blockDim.x) dec_op[t] = dec_op_g[t];
  __syncthreads();
  if (threadIdx.x != 0) return;
  uint8_t *st = work + (size_t)r * 256;
  FastConsoleT<false, false> m;
  m.rom8 = rom8;
  m.dec_op = dec_op;
  m.ram = ram;
  m.io = IoCtx{tia, iow};
  m.scheme = inf & 0xFF;
  m.wmask = 1u;
  m.idle = 1u;
  m.load(st);
  m.set_log(nullptr, 0, nullptr);
  for (int f = 0; f < startup; ++f) {
    m.apply_action(0);
    m.run_frame();
  }
  for (int j = 0; j <= max_noops; ++j) {
    m.store(st);
    const uint4 *s4 = reinterpret_cast<const uint4 *>(st);
    uint4 *d4 = reinterpret_cast<uint4 *>(snaps + ((size_t)r * (max_noops + 1) + j) * 256);
    for (int q = 0; q < 16; ++q) d4[q] = s4[q];
    if (j < max_noops) {
      m.apply_action(0);
      m.run_frame();
    }
  }
}

__global__ void k_cache_pick(uint8_t *cache, const uint8_t *snaps, int n_roms, int n_cache, int max_noops,
                             uint64_t seed) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_roms * n_cache) return;
  int r = t / n_cache, k = t % n_cache;
  uint32_t n = scale32(philox_x0(seed, (uint32_t)r, (uint32_t)k, PURPOSE_CACHE << 8, 0u), (uint32_t)max_noops + 1);
  const uint4 *src = reinterpret_cast<const uint4 *>(snaps + ((size_t)r * (max_noops + 1) + n) * 256);
  uint4 *dst = reinterpret_cast<uint4 *>(cache + (size_t)t * 256);
  for (int i = 0; i < 16; ++i) dst[i] = src[i];
}

// Initial reset (episode 0, fresh env fields) or a forced reset of masked envs.
__global__ void k_reset(uint8_t *state, const uint8_t *cache, const uint32_t *info, const int32_t *env_rom,
                        const uint32_t *env_key, const uint8_t *mask, uint8_t *ring, uint8_t *head, int n,
                        int n_cache, uint64_t seed, int initial) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mask && !mask[i]) return;
  uint8_t *st = state + (size_t)i * 256;
  uint32_t rom = (uint32_t)env_rom[i];
  uint32_t episode;
  if (initial) {
    for (int b = 0x60; b < 0x80; ++b) st[b] = 0;
    Console<GlobalMem>::st32(st + S::ENV_KEY, env_key[i]);
    st[S::ROM] = rom & 0xFF;
    st[S::ROM + 1] = rom >> 8;
    episode = 0;
  } else {
    episode = Console<GlobalMem>::ld32(st + S::EPISODE) + 1;
  }
  reset_from_cache(st, cache, info, rom, (uint32_t)n_cache, seed, Console<GlobalMem>::ld32(st + S::ENV_KEY), episode);
  if (ring) {
    uint4 z{0, 0, 0, 0};
    uint4 *p = reinterpret_cast<uint4 *>(ring + (size_t)i * 4 * 7056);
    for (int q = 0; q < 4 * 7056 / 16; ++q) p[q] = z;
    head[i] = 0;
  }
}

struct StepArgs {
  uint8_t *state;
  const uint8_t *cache;
  const uint8_t *roms;
  const uint32_t *info;
  const uint32_t *dec;
  const uint8_t *actions;
  int32_t *rew_int;
  uint8_t *done_int;
  int32_t *rew_out;
  uint8_t *done_out;
  uint32_t *log;
  uint8_t *snap;
  uint32_t *meta;
  uint32_t *counters;
  int n, frameskip, sticky, n_cache, log_cap, first_slot;
  uint64_t seed;
};

// The per-env step body shared by the interpreter kernels.
template <class Mem>
__device__ void step_env(Console<Mem> &m, uint8_t *st, int i, const StepArgs &a, RomInfo ri) {
  uint32_t action = a.actions[i];
  uint32_t env_status = Console<Mem>::ld32(st + S::STATUS);
  if (action >= 18) { env_status |= ST_BAD_ACTION; action = 0; }
  const uint32_t env_key = Console<Mem>::ld32(st + S::ENV_KEY);
  const uint32_t step_no = Console<Mem>::ld32(st + S::STEP);
  uint32_t episode = Console<Mem>::ld32(st + S::EPISODE);
  uint32_t last = st[S::LAST_ACTION];
  uint32_t score_prev = st[S::SCORE_PREV];
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
    if (logging) {
      m.snapshot(a.snap + ((size_t)i * 2 + slot) * 64);
      m.log.rec = a.log + ((size_t)i * 2 + slot) * a.log_cap;
      m.log.n = 0;
      m.log.cap = (uint32_t)a.log_cap;
    } else {
      m.log.rec = nullptr;
    }
    uint32_t lines = m.run_frame();
    if (logging) {
      uint32_t *mt = a.meta + ((size_t)i * 2 + slot) * 2;
      mt[0] = m.log.n;
      mt[1] = lines;
      log_total += m.log.n;
    }
    uint32_t s = m.mem.ram_rd(ri.score);
    reward += (int32_t)(int8_t)(uint8_t)(s - score_prev);
    score_prev = s;
  }
  env_status |= m.status;
  if (m.jam) env_status |= ST_ILLEGAL;  // done because the CPU is halted
  const uint32_t done = (m.mem.ram_rd(ri.gameover) != 0 || m.jam) ? 1u : 0u;
  a.rew_int[i] = reward;
  a.done_int[i] = (uint8_t)done;
  if (a.rew_out) a.rew_out[i] = reward;
  if (a.done_out) a.done_out[i] = (uint8_t)done;
  if (a.counters) {
    a.counters[3 * i] = m.instret;
    a.counters[3 * i + 1] = log_total;
    a.counters[3 * i + 2] = 0;  // one thread per env: no lockstep issue rounds
  }
  Console<Mem>::st32(st + S::STATUS, env_status);
  Console<Mem>::st32(st + S::STEP, step_no + 1);
  if (done) {
    reset_from_cache(st, a.cache, a.info, Console<Mem>::ld32(st + S::ROM) & 0xFFFF, (uint32_t)a.n_cache, a.seed,
                     env_key, episode + 1);
  } else {
    st[S::LAST_ACTION] = (uint8_t)last;
    st[S::SCORE_PREV] = (uint8_t)score_prev;
  }
}

// Plain form: one thread per env, state, RAM and ROM in global memory.
__global__ void __launch_bounds__(128) k_interp_plain(StepArgs a) {
  __shared__ uint32_t dec[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) dec[t] = a.dec[t];
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  uint8_t *st = a.state + (size_t)i * 256;
  uint32_t rom = st[S::ROM] | (uint32_t)st[S::ROM + 1] << 8;
  RomInfo ri = rom_info(a.info, rom);
  Console<GlobalMem> m;
  m.mem.ram = st + S::RAM;
  m.mem.rom = a.roms + (size_t)rom * ROM_SLOT;
  m.dec = dec;
  m.scheme = ri.scheme;
  m.load(st);
  step_env(m, st, i, a, ri);
  // machine part written before a possible reset overwrote it: store first
  // when not done; reset_from_cache already wrote the whole machine part
  if (!a.done_int[i]) m.store(st);
}

// Rasteriser: one warp per (env, slot) frame; frame (i, slot) goes to
// out + i * env_stride + (slot - first_slot) * 33600.
__global__ void __launch_bounds__(128) k_raster(const uint32_t *log, const uint8_t *snap, const uint32_t *meta,
                                                uint8_t *out, size_t env_stride, int n, int first_slot, int log_cap) {
  __shared__ __align__(16) uint8_t rows[4][160];
  const int warp = threadIdx.x >> 5;
  const int slots = 2 - first_slot;
  const long long w = (long long)blockIdx.x * 4 + warp;
  if (w >= (long long)n * slots) return;
  const int i = (int)(w / slots), slot = first_slot + (int)(w % slots);
  const size_t fs = (size_t)i * 2 + slot;
  RenderRegs R;
  R.load(snap + fs * 64);
  const uint32_t *mt = meta + fs * 2;
  uint32_t n_rec = mt[0] < (uint32_t)log_cap ? mt[0] : (uint32_t)log_cap;
  render_frame_warp(R, log + fs * log_cap, n_rec, mt[1], rows[warp],
                    out + (size_t)i * env_stride + (size_t)(slot - first_slot) * (FRAME_H * FRAME_W));
}

// Preprocessing: one block per env.  Luma of both frames, pixelwise maximum,
// exact integer area resampling to 84x84 (round half up), push into the
// env's 4-plane ring and write the ordered stack (oldest first) to obs.
__global__ void __launch_bounds__(256) k_preprocess(const uint8_t *frames, const uint8_t *luma_g, uint8_t *ring,
                                                    uint8_t *head, const uint8_t *done, uint8_t *obs, int n) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint8_t *mx = sm;                    // 210*160 luma maximum
  uint8_t *luma = sm + FRAME_H * FRAME_W;
  uint8_t *plane = luma + 128;         // 84*84 new plane
  const int i = blockIdx.x;
  if (i >= n) return;
  for (int t = threadIdx.x; t < 128; t += blockDim.x) luma[t] = luma_g[t];
  __syncthreads();
  const uint4 *f3 = reinterpret_cast<const uint4 *>(frames + (size_t)i * 2 * FRAME_H * FRAME_W);
  const uint4 *f4 = f3 + FRAME_H * FRAME_W / 16;
  for (int q = threadIdx.x; q < FRAME_H * FRAME_W / 16; q += blockDim.x) {
    uint4 a = f3[q], b = f4[q];
    const uint8_t *pa = reinterpret_cast<const uint8_t *>(&a);
    const uint8_t *pb = reinterpret_cast<const uint8_t *>(&b);
    uint4 r;
    uint8_t *pr = reinterpret_cast<uint8_t *>(&r);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      uint8_t la = luma[pa[k] >> 1], lb = luma[pb[k] >> 1];
      pr[k] = la > lb ? la : lb;
    }
    reinterpret_cast<uint4 *>(mx)[q] = r;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 84 * 84; o += blockDim.x) {
    uint32_t oi = o / 84, oj = o % 84;
    uint32_t y0 = (5u * oi) >> 1;
    uint32_t wy0 = (oi & 1) ? 42u : 84u, wy1 = 84u, wy2 = (oi & 1) ? 84u : 42u;
    uint32_t x0, wx0, wx1, wx2;
    col_weights(oj, x0, wx0, wx1, wx2);
    uint32_t s = 0;
    const uint8_t *r0 = mx + y0 * FRAME_W + x0;
    uint32_t rs0 = wx0 * r0[0] + wx1 * r0[1] + (wx2 ? wx2 * r0[2] : 0u);
    const uint8_t *r1 = r0 + FRAME_W;
    uint32_t rs1 = wx0 * r1[0] + wx1 * r1[1] + (wx2 ? wx2 * r1[2] : 0u);
    const uint8_t *r2 = r1 + FRAME_W;
    uint32_t rs2 = wx0 * r2[0] + wx1 * r2[1] + (wx2 ? wx2 * r2[2] : 0u);
    s = wy0 * rs0 + wy1 * rs1 + wy2 * rs2;
    plane[o] = (uint8_t)((s + 16800u) / 33600u);
  }
  __syncthreads();
  const uint32_t h = head[i];
  uint8_t *rg = ring + (size_t)i * 4 * 7056;
  uint8_t *ob = obs ? obs + (size_t)i * 4 * 7056 : nullptr;
  const uint32_t *pl32 = reinterpret_cast<const uint32_t *>(plane);
  // obs slots 0..2 are the ring's planes h, h+1, h+2 (oldest first) -- the
  // plane at h is the oldest and is about to be overwritten by the new one
  if (ob) {
    for (int s = 0; s < 3; ++s) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(rg + ((h + 1 + s) & 3) * 7056);
      uint32_t *dst = reinterpret_cast<uint32_t *>(ob + s * 7056);
      for (int q = threadIdx.x; q < 7056 / 4; q += blockDim.x) dst[q] = src[q];
    }
    uint32_t *dst = reinterpret_cast<uint32_t *>(ob + 3 * 7056);
    for (int q = threadIdx.x; q < 7056 / 4; q += blockDim.x) dst[q] = pl32[q];
  }
  __syncthreads();
  if (done[i]) {
    uint32_t *z = reinterpret_cast<uint32_t *>(rg);
    for (int q = threadIdx.x; q < 4 * 7056 / 4; q += blockDim.x) z[q] = 0;
    if (threadIdx.x == 0) head[i] = 0;
  } else {
    uint32_t *dst = reinterpret_cast<uint32_t *>(rg + h * 7056);
    for (int q = threadIdx.x; q < 7056 / 4; q += blockDim.x) dst[q] = pl32[q];
    if (threadIdx.x == 0) head[i] = (uint8_t)((h + 1) & 3);
  }
}

__global__ void k_status(const uint8_t *state, uint32_t *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = Console<GlobalMem>::ld32(state + (size_t)i * 256 + S::STATUS);
}

template <class T>
int dalloc(T **p, size_t bytes, size_t &total) {
  if (bytes == 0) { *p = nullptr; return 0; }
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) return fail(ATARI_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  total += bytes;
  return 0;
}

}  // namespace

// ------------------------------------------------------------------ env object
// Chunks of envs in the overlapped host-buffer step (batched stack output).
constexpr int HOST_CHUNKS = 8;

struct atari_env {
  int device = 0;
  int n = 0, n_roms = 0;
  atari_config cfg{};
  size_t bytes = 0;
  uint8_t *d_roms = nullptr;
  uint32_t *d_info = nullptr;
  uint32_t *d_dec = nullptr;
  int32_t *d_env_rom = nullptr;
  uint32_t *d_env_key = nullptr;
  uint8_t *d_state = nullptr;
  uint8_t *d_cache = nullptr;
  uint32_t *d_log = nullptr;
  uint8_t *d_snap = nullptr;
  uint8_t *d_bsnap = nullptr;   // batched stack form: [n][2][3][64] band start snapshots
  uint32_t *d_meta = nullptr;
  uint8_t *d_frames = nullptr;
  uint8_t *d_ring = nullptr;
  uint8_t *d_head = nullptr;
  uint8_t *d_luma = nullptr;
  int32_t *d_rew = nullptr;
  uint8_t *d_done = nullptr;
  uint32_t *d_ctr = nullptr;
  uint8_t *d_act = nullptr;   // staging for atari_env_step_host
  uint8_t *d_obs_tmp = nullptr;
  // batched form
  uint8_t *d_romb = nullptr;        // [n_roms][ROMB_SLOT] cartridge bytes for the batched stage
  uint8_t *d_dec_op = nullptr;      // 512 bytes
  int32_t *d_grp = nullptr;         // rom, start, count per work item (3 * n_groups) then perm (n)
  int32_t *d_seg = nullptr;         // first env-list position of each cartridge (n_roms + 1)
  int32_t *d_perm_dyn = nullptr;    // bank-aware grouping: the env list re-sorted at every step
  int grouping = 1;                 // 1 env order, 2 bank-aware
  bool banked = false;              // some cartridge has more than one bank
  int *d_queue = nullptr;
  int n_groups = 0, lanes = 32, warps = 4, wpf = 4, grid = 0, rom_stage = 4096, max_blocks = 1;
  bool split = false;   // paired CPU / TIA warps (k_interp_split)
  bool compact = false; // the interpreter with the compact hot opcode switch
  std::vector<int32_t> h_env_rom;
  std::vector<uint32_t> h_banks;
  cudaStream_t cap_stream = nullptr;
  // atari_env_step_host, batched stack output: the stacks come back on two
  // streams of their own, one chunk of envs at a time, while the next chunk
  // renders
  cudaStream_t copy_stream[2] = {};
  cudaEvent_t copy_ev[HOST_CHUNKS + 1] = {};
  struct GraphEntry { const void *k[4]; cudaGraphExec_t exec; };
  std::vector<GraphEntry> graphs;
  // profiling: (slot, start, end) event triples of the launches since the last read
  bool profiling = false;
  struct Rec { int slot; cudaEvent_t a, b; };
  std::vector<Rec> prof;
  std::vector<cudaEvent_t> pool;
};

namespace {

int scheme_of(size_t sz) {
  if (sz == 2048 || sz == 4096) return 0;
  if (sz == 8192) return 1;
  if (sz == 16384) return 2;
  if (sz == 32768) return 3;
  return -1;
}

size_t obs_bytes(const atari_config &c) { return c.output_mode == ATARI_OUT_PALETTE ? 210 * 160 : 4 * 7056; }

int validate(const atari_config &c) {
  if (c.frameskip < 2 || c.frameskip > 16) return fail(ATARI_EINVAL, "frameskip must be in 2..16");
  if (c.n_cache < 1 || c.n_cache > 64) return fail(ATARI_EINVAL, "n_cache must be in 1..64");
  if (c.startup_frames < 0 || c.startup_frames > 100000) return fail(ATARI_EINVAL, "bad startup_frames");
  if (c.max_noops < 0 || c.max_noops > 1000) return fail(ATARI_EINVAL, "bad max_noops");
  if (c.output_mode != ATARI_OUT_PALETTE && c.output_mode != ATARI_OUT_STACK)
    return fail(ATARI_EINVAL, "bad output_mode");
  if (c.form != ATARI_FORM_PLAIN && c.form != ATARI_FORM_BATCHED) return fail(ATARI_EINVAL, "bad form");
  if (c.log_cap < 256 || c.log_cap > (1 << 20)) return fail(ATARI_EINVAL, "log_cap must be in 256..2^20");
  if (c.sticky != 0 && c.sticky != 1) return fail(ATARI_EINVAL, "sticky must be 0 or 1");
  if (c.envs_per_block < 0 || c.envs_per_block > 128 || c.envs_per_warp < 0 || c.envs_per_warp > 32 ||
      c.raster_warps_per_frame < 0 || c.raster_warps_per_frame > 4 || c.tia_warps < 0 || c.tia_warps > 3 ||
      c.grouping < 0 || c.grouping > 2 || c.dispatch < 0 || c.dispatch > 2 || c.idle_skip < 0 || c.idle_skip > 1)
    return fail(ATARI_EINVAL, "envs_per_block must be 0..128, envs_per_warp 0..32, raster_warps_per_frame 0..4, "
                              "tia_warps 0..3, grouping 0..2, dispatch 0..2, idle_skip 0..1");
  return 0;
}

}  // namespace


namespace {

// Envs grouped by cartridge into work items of E envs (ascending env index
// within a cartridge); uploads rom/start/count per item and the permutation.
int build_groups(atari_env *E, int lanes, int warps, bool split) {
  const int per = lanes * warps;
  std::vector<int32_t> rom, start, count, perm;
  perm.reserve(E->n);
  for (int r = 0; r < E->n_roms; ++r) {
    int first = (int)perm.size();
    for (int i = 0; i < E->n; ++i)
      if (E->h_env_rom[i] == r) perm.push_back(i);
    for (int s = first; s < (int)perm.size(); s += per) {
      rom.push_back(r);
      start.push_back(s);
      count.push_back(std::min(per, (int)perm.size() - s));
    }
  }
  const int ng = (int)rom.size();
  if (E->d_seg) {
    std::vector<int32_t> seg(E->n_roms + 1, 0);
    for (int r = 0, p = 0; r < E->n_roms; ++r) {
      seg[r] = p;
      for (int i = 0; i < E->n; ++i) p += E->h_env_rom[i] == r ? 1 : 0;
      seg[r + 1] = p;
    }
    CUDA_TRY(cudaMemcpy(E->d_seg, seg.data(), seg.size() * 4, cudaMemcpyHostToDevice));
  }
  std::vector<int32_t> blob;
  blob.insert(blob.end(), rom.begin(), rom.end());
  blob.insert(blob.end(), start.begin(), start.end());
  blob.insert(blob.end(), count.begin(), count.end());
  blob.insert(blob.end(), perm.begin(), perm.end());
  if (E->d_grp) cudaFree(E->d_grp);
  E->d_grp = nullptr;
  size_t dummy = 0;
  if (int rc = dalloc(&E->d_grp, std::max<size_t>(blob.size(), 1) * 4, dummy)) return rc;
  CUDA_TRY(cudaMemcpy(E->d_grp, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice));
  E->n_groups = ng;
  E->lanes = lanes;
  E->warps = warps;
  E->split = split;
  const size_t smem = (size_t)E->rom_stage + 16 + 512 + (size_t)lanes * warps * (ENV_SMEM + (split ? 4 * QSTRIDE : 0));
  int per_sm = 0;
  if (split) {
    CUDA_TRY(cudaFuncSetAttribute(k_interp_split<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaFuncSetAttribute(k_interp_split<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interp_split<false>, 2 * warps * 32, smem));
  } else {
    CUDA_TRY(cudaFuncSetAttribute(k_interp_batched<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaFuncSetAttribute(k_interp_batched<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interp_batched<false>, warps * 32, smem));
  }
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device));
  E->max_blocks = std::max(1, per_sm) * sms;
  E->grid = std::max(1, std::min(ng, E->max_blocks));
  for (auto &g : E->graphs) cudaGraphExecDestroy(g.exec);
  E->graphs.clear();
  return 0;
}

BatchArgs batch_args(atari_env *E, const uint8_t *d_actions, int32_t *d_rewards, uint8_t *d_dones) {
  const atari_config &c = E->cfg;
  BatchArgs a;
  a.state = E->d_state;
  a.cache = E->d_cache;
  a.romb = E->d_romb;
  a.info = E->d_info;
  a.dec_op = E->d_dec_op;
  a.actions = d_actions;
  a.rew_int = E->d_rew;
  a.done_int = E->d_done;
  a.rew_out = d_rewards;
  a.done_out = d_dones;
  a.log = E->d_log;
  a.snap = E->d_snap;
  a.bsnap = E->d_bsnap;
  a.meta = E->d_meta;
  a.counters = E->d_ctr;
  a.grp_rom = E->d_grp;
  a.grp_start = E->d_grp + E->n_groups;
  a.grp_count = E->d_grp + 2 * E->n_groups;
  a.perm = E->grouping == 2 ? E->d_perm_dyn : E->d_grp + 3 * E->n_groups;
  a.opos = nullptr;
  a.queue = E->d_queue;
  a.n_groups = E->n_groups;
  a.lanes = E->lanes;
  a.E = E->lanes * E->warps;
  a.rom_stage = E->rom_stage;
  a.frameskip = c.frameskip;
  a.sticky = c.sticky;
  a.n_cache = c.n_cache;
  a.log_cap = c.log_cap;
  a.first_slot = c.output_mode == ATARI_OUT_PALETTE ? 1 : 0;
  a.seed = c.seed;
  a.tia_off = c.tia_warps == 3 ? 1 : 0;
  a.idle = c.idle_skip;
  return a;
}

size_t interp_smem(const atari_env *E) {
  return (size_t)E->rom_stage + 16 + 512 + (size_t)E->lanes * E->warps * (ENV_SMEM + (E->split ? 4 * QSTRIDE : 0));
}
// The batched interpreter in the env's current form and shape.
void launch_interp(atari_env *E, const BatchArgs &a, int grid, cudaStream_t s) {
  const unsigned th = (E->split ? 2 : 1) * E->warps * 32;
  if (E->split) {
    if (E->compact) k_interp_split<true><<<grid, th, interp_smem(E), s>>>(a);
    else k_interp_split<false><<<grid, th, interp_smem(E), s>>>(a);
  } else {
    if (E->compact) k_interp_batched<true><<<grid, th, interp_smem(E), s>>>(a);
    else k_interp_batched<false><<<grid, th, interp_smem(E), s>>>(a);
  }
}

size_t fused_smem() { return 2 * 210 * 160 + 128 + 7056; }

// Bank-aware grouping: the env list of this step, re-sorted by bank within
// each cartridge from the states as they stand.
void launch_regroup(atari_env *E, cudaStream_t s) {
  k_group_by_bank<<<E->n_roms, 256, 0, s>>>(E->d_state, E->d_grp + 3 * E->n_groups, E->d_seg, E->d_info,
                                             E->d_perm_dyn);
}

struct ProfScope;  // defined below
int setup_batched(atari_env *E, const std::vector<uint8_t> &img, const std::vector<uint32_t> &dec);

}  // namespace
namespace {
cudaEvent_t take_event(atari_env *E) {
  if (!E->pool.empty()) {
    cudaEvent_t e = E->pool.back();
    E->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// RAII bracket: records start/end events around one launch when profiling.
struct ProfScope {
  atari_env *E;
  int slot;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(atari_env *E_, int slot_, cudaStream_t s_) : E(E_), slot(slot_), s(s_) {
    if (E->profiling) {
      a = take_event(E);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = take_event(E);
      cudaEventRecord(b, s);
      E->prof.push_back({slot, a, b});
    }
  }
};
}  // namespace

extern "C" {

void atari_default_config(atari_config *c) {
  if (!c) return;
  memset(c, 0, sizeof *c);
  c->frameskip = 4;
  c->sticky = 0;
  c->n_cache = 30;
  c->startup_frames = 64;
  c->max_noops = 30;
  c->output_mode = ATARI_OUT_STACK;
  c->form = ATARI_FORM_PLAIN;
  c->log_cap = 4096;
  c->envs_per_block = 0;
  c->envs_per_warp = 0;
  c->raster_warps_per_frame = 0;
  c->idle_skip = 1;
  c->seed = 1;
}

const char *atari_last_error(void) { return g_err.c_str(); }

size_t atari_env_footprint(int n_envs, int n_roms, const atari_config *cfg) {
  if (!cfg || n_envs < 0 || n_roms < 0) return 0;
  size_t n = (size_t)n_envs;
  size_t b = 0;
  b += (size_t)n_roms * ROM_SLOT + (size_t)n_roms * 4 + 1024 + 512;  // images, info, decode word and byte tables
  b += n * (4 + 4 + 256);                                 // env_rom, env_key, state
  b += (size_t)n_roms * cfg->n_cache * 256;               // cache
  b += n * 2 * (size_t)cfg->log_cap * 4;                  // log
  b += n * 2 * 64 + n * 2 * 2 * 4;                        // snapshots, meta
  if (cfg->form == ATARI_FORM_PLAIN) b += n * 2 * 210 * 160;   // frames (plain form only)
  else b += (size_t)n_roms * ROMB_SLOT + n * 8 + 64 + (size_t)(n_roms + 1) * 4;  // stage bytes, work items, regrouping
  if (cfg->output_mode == ATARI_OUT_STACK) b += n * 4 * 7056 + n;
  if (cfg->output_mode == ATARI_OUT_STACK && cfg->form == ATARI_FORM_BATCHED) b += n * 2 * 3 * 64;  // band snapshots
  b += n * (4 + 1 + 12 + 1);                              // rewards, dones, counters, action staging
  return b;
}

int atari_env_create(const uint8_t *const *roms, const size_t *rom_sizes, const atari_rom_meta *meta, int n_roms,
                     const int32_t *env_rom, const uint32_t *env_key, int n_envs, const atari_config *cfg,
                     const uint8_t *luma, atari_env **out) {
  g_err.clear();
  if (!out) return fail(ATARI_EINVAL, "out is NULL");
  *out = nullptr;
  if (!roms || !rom_sizes || !meta || n_roms <= 0 || n_roms > 65535) return fail(ATARI_EINVAL, "bad ROM list");
  if (n_envs < 0 || (n_envs > 0 && !env_rom)) return fail(ATARI_EINVAL, "bad env list");
  if (!cfg) return fail(ATARI_EINVAL, "cfg is NULL");
  if (int e = validate(*cfg)) return e;
  if (cfg->output_mode == ATARI_OUT_STACK && !luma) return fail(ATARI_EINVAL, "luma table required for stack output");
  for (int r = 0; r < n_roms; ++r) {
    if (!roms[r] || scheme_of(rom_sizes[r]) < 0)
      return fail(ATARI_EINVAL, "ROM " + std::to_string(r) + ": size must be 2048, 4096, 8192, 16384 or 32768");
    if (meta[r].score_addr < 0x80 || meta[r].gameover_addr < 0x80)
      return fail(ATARI_EINVAL, "ROM " + std::to_string(r) + ": score/game-over addresses must be in $80-$FF");
  }
  for (int i = 0; i < n_envs; ++i)
    if (env_rom[i] < 0 || env_rom[i] >= n_roms) return fail(ATARI_EINVAL, "env_rom out of range");

  atari_env *E = new atari_env();
  E->n = n_envs;
  E->n_roms = n_roms;
  E->cfg = *cfg;
  cudaGetDevice(&E->device);
  auto bail = [&](int code) {
    atari_env_destroy(E);
    return code;
  };
  size_t &T = E->bytes;
  const size_t n = (size_t)n_envs;
  const atari_config &c = E->cfg;
  int rc = 0;
  if ((rc = dalloc(&E->d_roms, (size_t)n_roms * ROM_SLOT, T)) || (rc = dalloc(&E->d_info, (size_t)n_roms * 4, T)) ||
      (rc = dalloc(&E->d_dec, 1024, T)) || (rc = dalloc(&E->d_env_rom, n * 4, T)) ||
      (rc = dalloc(&E->d_env_key, n * 4, T)) || (rc = dalloc(&E->d_state, n * 256, T)) ||
      (rc = dalloc(&E->d_cache, (size_t)n_roms * c.n_cache * 256, T)) ||
      (rc = dalloc(&E->d_log, n * 2 * (size_t)c.log_cap * 4, T)) || (rc = dalloc(&E->d_snap, n * 2 * 64, T)) ||
      (rc = dalloc(&E->d_meta, n * 2 * 2 * 4, T)) ||
      (c.form == ATARI_FORM_PLAIN && (rc = dalloc(&E->d_frames, n * 2 * 210 * 160, T))) ||
      (rc = dalloc(&E->d_rew, n * 4, T)) || (rc = dalloc(&E->d_done, n, T)) || (rc = dalloc(&E->d_ctr, n * 12, T)) ||
      (rc = dalloc(&E->d_act, n, T)) || (rc = dalloc(&E->d_luma, 128, T)) || (rc = dalloc(&E->d_dec_op, 512, T)))
    return bail(rc);
  if (c.output_mode == ATARI_OUT_STACK) {
    if ((rc = dalloc(&E->d_ring, n * 4 * 7056, T)) || (rc = dalloc(&E->d_head, n, T))) return bail(rc);
    if (c.form == ATARI_FORM_BATCHED && (rc = dalloc(&E->d_bsnap, n * 2 * 3 * 64, T))) return bail(rc);
  }
  // render inputs start zeroed (a step that failed to write them still renders defined values)
  if (n && (cudaMemset(E->d_snap, 0, n * 2 * 64) != cudaSuccess || cudaMemset(E->d_meta, 0, n * 2 * 2 * 4) != cudaSuccess ||
            (E->d_bsnap && cudaMemset(E->d_bsnap, 0, n * 2 * 3 * 64) != cudaSuccess)))
    return bail(fail(ATARI_ECUDA, "zeroing render buffers failed"));

  // cartridges: 2K images mirrored to 4K, each in a 16 KB slot
  std::vector<uint8_t> img((size_t)n_roms * ROM_SLOT, 0);
  std::vector<uint32_t> info(n_roms);
  std::vector<uint8_t> power((size_t)n_roms * 256, 0);
  for (int r = 0; r < n_roms; ++r) {
    uint8_t *dst = img.data() + (size_t)r * ROM_SLOT;
    if (rom_sizes[r] == 2048) {
      memcpy(dst, roms[r], 2048);
      memcpy(dst + 2048, roms[r], 2048);
    } else {
      memcpy(dst, roms[r], rom_sizes[r]);
    }
    info[r] = rom_info_word(rom_sizes[r], meta[r]);
    // power-on state: registers and RAM zero, SP $FD, P $24, PC from the reset
    // vector of bank 0, timer 0 with interval 1024 written at cycle 0
    uint8_t *p = power.data() + (size_t)r * 256;
    p[S::SP] = 0xFD;
    p[S::P] = 0x24;
    p[S::PC] = dst[0xFFC];
    p[S::PC + 1] = dst[0xFFD];
    p[S::TIM_SHIFT] = 10;
    for (int b = 0; b < 8; ++b) p[S::BAR_LINE + b] = 0xFF;
  }
  std::vector<uint32_t> dec = build_decode_table();
  E->h_env_rom.assign(env_rom, env_rom + n);
  E->h_banks.resize(n_roms);
  for (int r = 0; r < n_roms; ++r) E->h_banks[r] = rom_sizes[r] <= 4096 ? 1u : (uint32_t)(rom_sizes[r] / 4096);
  std::vector<uint32_t> keys(n);
  for (size_t i = 0; i < n; ++i) keys[i] = env_key ? env_key[i] : (uint32_t)i;

  auto up = [&](void *d, const void *h, size_t b) -> int {
    if (!b) return 0;
    cudaError_t e = cudaMemcpy(d, h, b, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? 0 : fail(ATARI_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
  };
  const std::vector<uint8_t> dec_op = build_dec_op(dec);
  if ((rc = up(E->d_roms, img.data(), img.size())) || (rc = up(E->d_info, info.data(), info.size() * 4)) ||
      (rc = up(E->d_dec, dec.data(), 1024)) || (rc = up(E->d_dec_op, dec_op.data(), 512)) || (rc = up(E->d_env_rom, env_rom, n * 4)) ||
      (rc = up(E->d_env_key, keys.data(), n * 4)))
    return bail(rc);
  if (luma && (rc = up(E->d_luma, luma, 128))) return bail(rc);

  // start-state cache (Section 3): run each ROM from power-on on the device
  uint8_t *d_work = nullptr, *d_snaps = nullptr;
  size_t scratch = 0;
  if ((rc = dalloc(&d_work, (size_t)n_roms * 256, scratch)) ||
      (rc = dalloc(&d_snaps, (size_t)n_roms * (c.max_noops + 1) * 256, scratch))) {
    cudaFree(d_work);
    return bail(rc);
  }
  rc = up(d_work, power.data(), power.size());
  if (!rc) {
    uint32_t max_banks = 1;
    for (int r = 0; r < n_roms; ++r) max_banks = std::max(max_banks, E->h_banks[r]);
    const int stage = (int)max_banks * 4096;
    const size_t cache_smem = (size_t)stage + 16 + 512 + RAM_BYTES + 4 * IO_STRIDE + TIA_STRIDE;
    k_cache_run<<<n_roms, 128, cache_smem>>>(d_work, d_snaps, E->d_roms, E->d_info, E->d_dec_op, stage,
                                           c.startup_frames, c.max_noops);
    int tot = n_roms * c.n_cache;
    k_cache_pick<<<(tot + 127) / 128, 128>>>(E->d_cache, d_snaps, n_roms, c.n_cache, c.max_noops, c.seed);
    if (n_envs > 0)
      k_reset<<<(n_envs + 127) / 128, 128>>>(E->d_state, E->d_cache, E->d_info, E->d_env_rom, E->d_env_key, nullptr,
                                             E->d_ring, E->d_head, n_envs, c.n_cache, c.seed, 1);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail(ATARI_ECUDA, std::string("cache build: ") + cudaGetErrorString(e));
  }
  cudaFree(d_work);
  cudaFree(d_snaps);
  if (rc) return bail(rc);
  if (c.form == ATARI_FORM_BATCHED) {
    if ((rc = setup_batched(E, img, dec))) return bail(rc);
  }
  *out = E;
  return 0;
}

void atari_env_destroy(atari_env *E) {
  if (!E) return;
  void *ptrs[] = {E->d_roms, E->d_info, E->d_dec, E->d_env_rom, E->d_env_key, E->d_state, E->d_cache, E->d_log,
                  E->d_snap, E->d_bsnap, E->d_meta, E->d_frames, E->d_ring, E->d_head, E->d_luma, E->d_rew, E->d_done,
                  E->d_ctr, E->d_act, E->d_obs_tmp, E->d_romb, E->d_dec_op, E->d_grp, E->d_queue, E->d_seg,
                  E->d_perm_dyn};
  for (auto &g : E->graphs) cudaGraphExecDestroy(g.exec);
  if (E->cap_stream) cudaStreamDestroy(E->cap_stream);
  for (auto cs : E->copy_stream)
    if (cs) cudaStreamDestroy(cs);
  for (auto e : E->copy_ev)
    if (e) cudaEventDestroy(e);
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (auto &r : E->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : E->pool) cudaEventDestroy(e);
  delete E;
}

int atari_env_reset(atari_env *E, const uint8_t *d_mask, atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  k_reset<<<(E->n + 127) / 128, 128, 0, s>>>(E->d_state, E->d_cache, E->d_info, E->d_env_rom, E->d_env_key, d_mask,
                                             E->d_ring, E->d_head, E->n, E->cfg.n_cache, E->cfg.seed, 0);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // extern "C"

namespace {

int step_plain(atari_env *E, const uint8_t *d_actions, uint8_t *d_obs, int32_t *d_rewards, uint8_t *d_dones,
               cudaStream_t s) {
  const atari_config &c = E->cfg;
  StepArgs a;
  a.state = E->d_state;
  a.cache = E->d_cache;
  a.roms = E->d_roms;
  a.info = E->d_info;
  a.dec = E->d_dec;
  a.actions = d_actions;
  a.rew_int = E->d_rew;
  a.done_int = E->d_done;
  a.rew_out = d_rewards;
  a.done_out = d_dones;
  a.log = E->d_log;
  a.snap = E->d_snap;
  a.meta = E->d_meta;
  a.counters = E->d_ctr;
  a.n = E->n;
  a.frameskip = c.frameskip;
  a.sticky = c.sticky;
  a.n_cache = c.n_cache;
  a.log_cap = c.log_cap;
  a.first_slot = 0;
  a.seed = c.seed;
  {
    ProfScope p(E, ATARI_PROF_INTERP, s);
    k_interp_plain<<<(E->n + 127) / 128, 128, 0, s>>>(a);
  }
  CUDA_TRY(cudaGetLastError());
  long long warps = (long long)E->n * 2;
  {
    ProfScope p(E, ATARI_PROF_RASTER, s);
    k_raster<<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(E->d_log, E->d_snap, E->d_meta, E->d_frames,
                                                          (size_t)2 * 210 * 160, E->n, 0, c.log_cap);
  }
  CUDA_TRY(cudaGetLastError());
  if (c.output_mode == ATARI_OUT_STACK) {
    size_t smem = 210 * 160 + 128 + 7056;
    {
      ProfScope p(E, ATARI_PROF_PREPROC, s);
      k_preprocess<<<E->n, 256, smem, s>>>(E->d_frames, E->d_luma, E->d_ring, E->d_head, E->d_done, d_obs, E->n);
    }
    CUDA_TRY(cudaGetLastError());
  } else if (d_obs) {
    ProfScope p(E, ATARI_PROF_COPY, s);
    CUDA_TRY(cudaMemcpy2DAsync(d_obs, 210 * 160, E->d_frames + 210 * 160, 2 * 210 * 160, 210 * 160, E->n,
                               cudaMemcpyDeviceToDevice, s));
  }
  return 0;
}


// Batched form: reset the work queue, persistent interpreter, then the fused
// replay + preprocessing (stack output) or the replay of frame F straight
// into the observation (palette output).
int launch_batched(atari_env *E, const uint8_t *d_actions, uint8_t *d_obs, int32_t *d_rewards, uint8_t *d_dones,
                   cudaStream_t s) {
  const atari_config &c = E->cfg;
  BatchArgs a = batch_args(E, d_actions, d_rewards, d_dones);
  if (E->grouping == 2) {
    ProfScope p(E, ATARI_PROF_GROUP, s);
    launch_regroup(E, s);
  }
  CUDA_TRY(cudaMemsetAsync(E->d_queue, 0, sizeof(int), s));
  {
    ProfScope p(E, ATARI_PROF_INTERP, s);
    launch_interp(E, a, E->grid, s);
  }
  CUDA_TRY(cudaGetLastError());
  if (c.output_mode == ATARI_OUT_STACK) {
    ProfScope p(E, ATARI_PROF_FUSED, s);
    k_raster_preprocess<<<E->n, 64 * E->wpf, fused_smem(), s>>>(E->d_log, E->d_snap, E->d_bsnap, E->d_meta, E->d_luma, E->d_ring,
                                                                E->d_head, E->d_done, d_obs, E->n, c.log_cap, E->wpf, nullptr, nullptr, 0);
  } else if (d_obs) {
    ProfScope p(E, ATARI_PROF_RASTER, s);
    k_raster<<<(unsigned)((E->n + 3) / 4), 128, 0, s>>>(E->d_log, E->d_snap, E->d_meta, d_obs, (size_t)210 * 160,
                                                         E->n, 1, c.log_cap);
  }
  CUDA_TRY(cudaGetLastError());
  return 0;
}

int step_batched(atari_env *E, const uint8_t *d_actions, uint8_t *d_obs, int32_t *d_rewards, uint8_t *d_dones,
                 cudaStream_t s) {
  if (E->profiling) return launch_batched(E, d_actions, d_obs, d_rewards, d_dones, s);
  const void *key[4] = {d_actions, d_obs, d_rewards, d_dones};
  cudaGraphExec_t exec = nullptr;
  for (auto &g : E->graphs)
    if (!memcmp(g.k, key, sizeof key)) exec = g.exec;
  if (!exec) {
    if (E->graphs.size() >= 4) {
      cudaGraphExecDestroy(E->graphs.front().exec);
      E->graphs.erase(E->graphs.begin());
    }
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_batched(E, d_actions, d_obs, d_rewards, d_dones, E->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(E->cap_stream, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (ce != cudaSuccess) return fail(ATARI_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(ATARI_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    atari_env::GraphEntry ge;
    memcpy(ge.k, key, sizeof key);
    ge.exec = exec;
    E->graphs.push_back(ge);
  }
  CUDA_TRY(cudaGraphLaunch(exec, s));
  return 0;
}


// Time the batched interpreter on a copy of the current state and keep the
// fastest (envs per warp, warps per block); then the fastest number of warps
// per frame in the fused replay.  Every configuration computes the same
// results; only speed differs.  The state, stack ring and heads are restored.
int autotune(atari_env *E) {
  const size_t n = (size_t)E->n;
  uint8_t *st_bak = nullptr, *ring_bak = nullptr, *head_bak = nullptr;
  size_t dummy = 0;
  if (int rc = dalloc(&st_bak, n * 256, dummy)) return rc;
  CUDA_TRY(cudaMemcpy(st_bak, E->d_state, n * 256, cudaMemcpyDeviceToDevice));
  std::vector<uint8_t> acts(n);
  uint32_t x = 0x9E3779B9u;
  for (auto &v : acts) { x ^= x << 13; x ^= x >> 17; x ^= x << 5; v = (uint8_t)(x % 18u); }
  CUDA_TRY(cudaMemcpy(E->d_act, acts.data(), n, cudaMemcpyHostToDevice));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // (envs per warp, CPU warps per block, paired TIA warps)
  const int cand[][3] = {{32, 4, 0}, {32, 2, 0}, {32, 1, 0}, {16, 4, 0}, {16, 2, 0}, {16, 1, 0}, {8, 4, 0},
                         {8, 2, 0},  {8, 1, 0},  {4, 4, 0},  {4, 2, 0},  {4, 1, 0},  {2, 4, 0},  {2, 2, 0},
                         {1, 4, 0},  {32, 4, 1}, {32, 2, 1}, {32, 1, 1}, {16, 4, 1}, {16, 2, 1}, {16, 1, 1},
                         {8, 4, 1},  {8, 2, 1},  {8, 1, 1}};
  // shapes within 3 % of the fastest count as equal; the first of them in
  // candidate order (the widest warps) is taken, so the choice is stable
  // from run to run
  std::vector<std::pair<float, int>> timed;
  bool was_prof = E->profiling;
  E->profiling = false;
  for (int ci = 0; ci < (int)(sizeof cand / sizeof cand[0]); ++ci) {
    const auto &c = cand[ci];
    if ((size_t)c[0] * c[1] > 4 * n && c[0] * c[1] > 32) continue;  // far more slots than envs
    if ((E->cfg.tia_warps == 1 && c[2]) || (E->cfg.tia_warps >= 2 && !c[2])) continue;
    if (int rc = build_groups(E, c[0], c[1], c[2] != 0)) { cudaFree(st_bak); return rc; }
    BatchArgs a = batch_args(E, E->d_act, nullptr, nullptr);
    float t = 0;
    for (int rep = 0; rep < 2; ++rep) {
      CUDA_TRY(cudaMemcpy(E->d_state, st_bak, n * 256, cudaMemcpyDeviceToDevice));
      CUDA_TRY(cudaMemset(E->d_queue, 0, sizeof(int)));
      cudaEventRecord(e0);
      launch_interp(E, a, E->grid, nullptr);
      cudaEventRecord(e1);
      CUDA_TRY(cudaEventSynchronize(e1));
      CUDA_TRY(cudaGetLastError());
      cudaEventElapsedTime(&t, e0, e1);
    }
    timed.push_back({t, ci});
  }
  float best = 1e30f;
  for (auto &p : timed) best = std::min(best, p.first);
  int bl = 32, bw = 4, bs = E->cfg.tia_warps >= 2 ? 1 : 0;
  for (auto &p : timed)
    if (p.first <= 1.03f * best) { bl = cand[p.second][0]; bw = cand[p.second][1]; bs = cand[p.second][2]; break; }
  int rc = build_groups(E, bl, bw, bs != 0);
  // ROM-to-warp grouping on the chosen shape: env order, or bank-aware
  // (the regrouping kernel's time counted with the interpreter's); the
  // bank-aware order must be 3 % faster to be taken
  E->grouping = E->cfg.grouping ? E->cfg.grouping : 1;
  if (!rc && E->cfg.grouping == 0 && E->banked) {
    float tg[3] = {0, 0, 0};
    for (int g = 1; g <= 2 && !rc; ++g) {
      E->grouping = g;
      BatchArgs a = batch_args(E, E->d_act, nullptr, nullptr);
      for (int rep = 0; rep < 2; ++rep) {
        if (cudaMemcpy(E->d_state, st_bak, n * 256, cudaMemcpyDeviceToDevice) != cudaSuccess ||
            cudaMemset(E->d_queue, 0, sizeof(int)) != cudaSuccess) {
          rc = fail(ATARI_ECUDA, "autotune: state restore failed");
          break;
        }
        cudaEventRecord(e0);
        if (g == 2) launch_regroup(E, nullptr);
        launch_interp(E, a, E->grid, nullptr);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&tg[g], e0, e1);
      }
    }
    E->grouping = tg[2] < 0.97f * tg[1] ? 2 : 1;
  }
  // opcode dispatch on the chosen shape and grouping: the full hot switch, or
  // the compact one (rare forms through the general decoder); the compact
  // switch must be 3 % faster to be taken
  E->compact = E->cfg.dispatch == 2;
  if (!rc && E->cfg.dispatch == 0) {
    float td[2] = {0, 0};
    for (int cmp = 0; cmp <= 1 && !rc; ++cmp) {
      E->compact = cmp != 0;
      BatchArgs a = batch_args(E, E->d_act, nullptr, nullptr);
      for (int rep = 0; rep < 2; ++rep) {
        if (cudaMemcpy(E->d_state, st_bak, n * 256, cudaMemcpyDeviceToDevice) != cudaSuccess ||
            cudaMemset(E->d_queue, 0, sizeof(int)) != cudaSuccess) {
          rc = fail(ATARI_ECUDA, "autotune: state restore failed");
          break;
        }
        cudaEventRecord(e0);
        if (E->grouping == 2) launch_regroup(E, nullptr);
        launch_interp(E, a, E->grid, nullptr);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&td[cmp], e0, e1);
      }
    }
    E->compact = td[1] < 0.97f * td[0];
  }
  if (!rc && E->cfg.output_mode == ATARI_OUT_STACK) {
    if (!(rc = dalloc(&ring_bak, n * 4 * 7056, dummy)) && !(rc = dalloc(&head_bak, n, dummy))) {
      cudaMemcpy(ring_bak, E->d_ring, n * 4 * 7056, cudaMemcpyDeviceToDevice);
      cudaMemcpy(head_bak, E->d_head, n, cudaMemcpyDeviceToDevice);
      float fb = 1e30f;
      for (int wpf : {4, 2, 1}) {  // a later (smaller) split must be 3 % faster to be taken
        float t = 0;
        for (int rep = 0; rep < 2; ++rep) {
          cudaEventRecord(e0);
          k_raster_preprocess<<<E->n, 64 * wpf, fused_smem()>>>(E->d_log, E->d_snap, E->d_bsnap, E->d_meta, E->d_luma, E->d_ring,
                                                               E->d_head, E->d_done, nullptr, E->n, E->cfg.log_cap, wpf, nullptr, nullptr, 0);
          cudaEventRecord(e1);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&t, e0, e1);
        }
        if (t < 0.97f * fb) { fb = t; E->wpf = wpf; }
      }
      cudaMemcpy(E->d_ring, ring_bak, n * 4 * 7056, cudaMemcpyDeviceToDevice);
      cudaMemcpy(E->d_head, head_bak, n, cudaMemcpyDeviceToDevice);
    }
  }
  CUDA_TRY(cudaMemcpy(E->d_state, st_bak, n * 256, cudaMemcpyDeviceToDevice));
  cudaError_t ce = cudaDeviceSynchronize();
  cudaFree(st_bak);
  if (ring_bak) cudaFree(ring_bak);
  if (head_bak) cudaFree(head_bak);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  E->profiling = was_prof;
  if (rc) return rc;
  if (ce != cudaSuccess) return fail(ATARI_ECUDA, std::string("autotune: ") + cudaGetErrorString(ce));
  return 0;
}

int setup_batched(atari_env *E, const std::vector<uint8_t> &img, const std::vector<uint32_t> &dec) {
  const int R = E->n_roms;
  std::vector<uint8_t> bytes((size_t)R * ROMB_SLOT, 0u);
  (void)dec;  // the decode bytes were uploaded at create for the start-state cache
  uint32_t max_banks = 1;
  for (int r = 0; r < R; ++r) {
    const uint32_t banks = E->h_banks[r];
    max_banks = std::max(max_banks, banks);
    memcpy(bytes.data() + (size_t)r * ROMB_SLOT, img.data() + (size_t)r * ROM_SLOT, (size_t)banks * 4096);
  }
  E->rom_stage = (int)max_banks * 4096;
  E->banked = max_banks > 1;
  size_t &T = E->bytes;
  if (int rc = dalloc(&E->d_seg, (size_t)(R + 1) * 4, T)) return rc;
  if (int rc = dalloc(&E->d_perm_dyn, std::max<size_t>((size_t)E->n, 1) * 4, T)) return rc;
  if (int rc = dalloc(&E->d_romb, bytes.size(), T)) return rc;
  if (int rc = dalloc(&E->d_queue, 64, T)) return rc;
  CUDA_TRY(cudaMemcpy(E->d_romb, bytes.data(), bytes.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking));
  CUDA_TRY(cudaFuncSetAttribute(k_raster_preprocess, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem()));
  const atari_config &c = E->cfg;
  if (c.envs_per_block > 0 && c.envs_per_warp > 0) {
    int L = std::min(32, c.envs_per_warp), W = std::max(1, std::min(4, c.envs_per_block / L));
    E->wpf = c.raster_warps_per_frame > 0 ? c.raster_warps_per_frame : 4;
    E->grouping = c.grouping ? c.grouping : 1;
    E->compact = c.dispatch == 2;
    return build_groups(E, L, W, c.tia_warps >= 2);
  }
  E->grouping = c.grouping ? c.grouping : 1;
  E->compact = c.dispatch == 2;
  if (E->n == 0) return build_groups(E, 32, 4, c.tia_warps >= 2);
  return autotune(E);
}
}  // namespace

extern "C" {

int atari_env_step(atari_env *E, const uint8_t *d_actions, uint8_t *d_obs, int32_t *d_rewards, uint8_t *d_dones,
                   atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->n == 0) return 0;
  if (!d_actions) return fail(ATARI_EINVAL, "d_actions is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (E->cfg.form == ATARI_FORM_BATCHED) return step_batched(E, d_actions, d_obs, d_rewards, d_dones, s);
  return step_plain(E, d_actions, d_obs, d_rewards, d_dones, s);
}

namespace {
// Host-buffer step of the batched form with stack output: the interpreter,
// then the fused kernel in chunks of envs on the step stream; each chunk's
// stacks are copied out while the next chunk renders, and rewards and dones
// as soon as the interpreter is done.  Each chunk's copy is split in halves
// over two copy streams: one device-to-host copy per stream moves about 40 %
// of what two concurrent ones do.  Results are those of atari_env_step
// (every env's fused work is independent of the others').
int step_host_overlapped(atari_env *E, uint8_t *obs, int32_t *rewards, uint8_t *dones, cudaStream_t s) {
  const atari_config &c = E->cfg;
  const size_t ob = obs_bytes(c);
  const int n = E->n;
  if (!E->copy_stream[0]) {
    for (auto &cs : E->copy_stream) CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    for (auto &e : E->copy_ev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaStream_t *cs = E->copy_stream;
  BatchArgs a = batch_args(E, E->d_act, nullptr, nullptr);
  if (E->grouping == 2) {
    ProfScope p(E, ATARI_PROF_GROUP, s);
    launch_regroup(E, s);
  }
  CUDA_TRY(cudaMemsetAsync(E->d_queue, 0, sizeof(int), s));
  {
    ProfScope p(E, ATARI_PROF_INTERP, s);
    launch_interp(E, a, E->grid, s);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventRecord(E->copy_ev[0], s));
  CUDA_TRY(cudaStreamWaitEvent(cs[0], E->copy_ev[0], 0));
  if (rewards) CUDA_TRY(cudaMemcpyAsync(rewards, E->d_rew, (size_t)n * 4, cudaMemcpyDeviceToHost, cs[0]));
  if (dones) CUDA_TRY(cudaMemcpyAsync(dones, E->d_done, (size_t)n, cudaMemcpyDeviceToHost, cs[0]));
  // chunks of at least 1024 envs (a few waves of the fused kernel each)
  const int chunks = n >= 1024 * HOST_CHUNKS ? HOST_CHUNKS : n >= 4096 ? 4 : 1;
  for (int k = 0; k < chunks; ++k) {
    const int b0 = (int)((int64_t)n * k / chunks), b1 = (int)((int64_t)n * (k + 1) / chunks);
    {
      ProfScope p(E, ATARI_PROF_FUSED, s);
      k_raster_preprocess<<<b1 - b0, 64 * E->wpf, fused_smem(), s>>>(
          E->d_log, E->d_snap, E->d_bsnap, E->d_meta, E->d_luma, E->d_ring, E->d_head, E->d_done, E->d_obs_tmp, n,
          c.log_cap, E->wpf, nullptr, nullptr, b0);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(E->copy_ev[k + 1], s));
    const size_t lo = (size_t)b0 * ob, mid = (size_t)(b0 + (b1 - b0) / 2) * ob, hi = (size_t)b1 * ob;
    for (int h = 0; h < 2; ++h) {
      const size_t x0 = h ? mid : lo, x1 = h ? hi : mid;
      CUDA_TRY(cudaStreamWaitEvent(cs[h], E->copy_ev[k + 1], 0));
      if (x1 > x0) CUDA_TRY(cudaMemcpyAsync(obs + x0, E->d_obs_tmp + x0, x1 - x0, cudaMemcpyDeviceToHost, cs[h]));
    }
  }
  CUDA_TRY(cudaStreamSynchronize(cs[0]));
  CUDA_TRY(cudaStreamSynchronize(cs[1]));
  CUDA_TRY(cudaStreamSynchronize(s));
  return 0;
}
}  // namespace

int atari_env_step_host(atari_env *E, const uint8_t *actions, uint8_t *obs, int32_t *rewards, uint8_t *dones,
                        atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->n == 0) return 0;
  if (!actions) return fail(ATARI_EINVAL, "actions is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ob = obs_bytes(E->cfg);
  if (obs && !E->d_obs_tmp) {
    size_t dummy = 0;
    if (int rc = dalloc(&E->d_obs_tmp, (size_t)E->n * ob, dummy)) return rc;
    E->bytes += dummy;
  }
  CUDA_TRY(cudaMemcpyAsync(E->d_act, actions, E->n, cudaMemcpyHostToDevice, s));
  if (obs && E->cfg.form == ATARI_FORM_BATCHED && E->cfg.output_mode == ATARI_OUT_STACK)
    return step_host_overlapped(E, obs, rewards, dones, s);
  if (int rc = atari_env_step(E, E->d_act, obs ? E->d_obs_tmp : nullptr, nullptr, nullptr, stream)) return rc;
  if (obs) CUDA_TRY(cudaMemcpyAsync(obs, E->d_obs_tmp, (size_t)E->n * ob, cudaMemcpyDeviceToHost, s));
  if (rewards) CUDA_TRY(cudaMemcpyAsync(rewards, E->d_rew, (size_t)E->n * 4, cudaMemcpyDeviceToHost, s));
  if (dones) CUDA_TRY(cudaMemcpyAsync(dones, E->d_done, (size_t)E->n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return 0;
}

int atari_env_status(atari_env *E, uint32_t *d_status, atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->n == 0) return 0;
  if (!d_status) return fail(ATARI_EINVAL, "d_status is NULL");
  k_status<<<(E->n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(E->d_state, d_status, E->n);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

int atari_env_get_state(atari_env *E, void *d_dst, atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->n == 0) return 0;
  if (!d_dst) return fail(ATARI_EINVAL, "d_dst is NULL");
  CUDA_TRY(cudaMemcpyAsync(d_dst, E->d_state, (size_t)E->n * 256, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return 0;
}

int atari_env_set_state(atari_env *E, const void *d_src, atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->n == 0) return 0;
  if (!d_src) return fail(ATARI_EINVAL, "d_src is NULL");
  CUDA_TRY(cudaMemcpyAsync(E->d_state, d_src, (size_t)E->n * 256, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return 0;
}

int atari_env_get_frames(atari_env *E, uint8_t *d_dst, atari_stream stream) {
  g_err.clear();
  if (!E || !d_dst) return fail(ATARI_EINVAL, "bad argument");
  if (E->cfg.form != ATARI_FORM_PLAIN) return fail(ATARI_EINVAL, "frames are materialised by the plain form only");
  CUDA_TRY(cudaMemcpyAsync(d_dst, E->d_frames, (size_t)E->n * 2 * 210 * 160, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  return 0;
}

int atari_env_get_cache(atari_env *E, void *d_dst, atari_stream stream) {
  g_err.clear();
  if (!E || !d_dst) return fail(ATARI_EINVAL, "bad argument");
  CUDA_TRY(cudaMemcpyAsync(d_dst, E->d_cache, (size_t)E->n_roms * E->cfg.n_cache * 256, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  return 0;
}

int atari_env_counters(atari_env *E, uint64_t *instructions, uint64_t *log_records, uint64_t *lane_rounds,
                       atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  std::vector<uint32_t> h((size_t)E->n * 3);
  if (E->n) {
    CUDA_TRY(cudaMemcpyAsync(h.data(), E->d_ctr, h.size() * 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  }
  uint64_t a = 0, b = 0, c = 0;
  for (int i = 0; i < E->n; ++i) { a += h[3 * i]; b += h[3 * i + 1]; c += h[3 * i + 2]; }
  if (instructions) *instructions = a;
  if (log_records) *log_records = b;
  if (lane_rounds) *lane_rounds = c;
  return 0;
}

int atari_env_policy(atari_env *E, const uint8_t *d_obs, const uint16_t *d_weights, uint8_t *d_actions,
                     float *d_logits, atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->cfg.output_mode != ATARI_OUT_STACK) return fail(ATARI_EINVAL, "the policy reads the 84x84x4 stack output");
  if (E->n == 0) return 0;
  if (!d_obs || !d_weights || !d_actions) return fail(ATARI_EINVAL, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  {
    ProfScope p(E, ATARI_PROF_POLICY, s);
    k_policy<<<(E->n + POLICY_TPB - 1) / POLICY_TPB, POLICY_TPB, 0, s>>>(d_obs, d_weights, E->d_state, d_actions,
                                                                      d_logits, nullptr, E->n, E->cfg.seed);
  }
  CUDA_TRY(cudaGetLastError());
  return 0;
}

int atari_env_rollout_ex(atari_env *E, const uint16_t *d_weights, int n_steps, uint8_t *d_obs, uint8_t *d_actions,
                         int32_t *d_rewards, uint8_t *d_dones, uint8_t *d_ring_planes, float *d_ring_rewards,
                         uint8_t *d_ring_dones, float *d_ring_mu, int ring_depth, int ring_start,
                         atari_stream stream) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (E->cfg.output_mode != ATARI_OUT_STACK) return fail(ATARI_EINVAL, "the rollout loop needs stack output");
  if (n_steps < 0 || ring_depth < 1 || ring_start < 0) return fail(ATARI_EINVAL, "bad n_steps / ring arguments");
  if (E->n == 0 || n_steps == 0) return 0;
  if (!d_weights || !d_obs || !d_actions || !d_rewards || !d_dones || !d_ring_planes || !d_ring_rewards)
    return fail(ATARI_EINVAL, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  for (int t = 0; t < n_steps; ++t) {
    const int slot = (int)(((long long)ring_start + t) % ring_depth);
    {
      ProfScope p(E, ATARI_PROF_POLICY, s);
      k_policy<<<(E->n + POLICY_TPB - 1) / POLICY_TPB, POLICY_TPB, 0, s>>>(
          d_obs, d_weights, E->d_state, d_actions, nullptr, d_ring_mu ? d_ring_mu + (size_t)slot * E->n : nullptr,
          E->n, E->cfg.seed);
    }
    CUDA_TRY(cudaGetLastError());
    if (int rc = atari_env_step(E, d_actions, d_obs, d_rewards, d_dones, stream)) return rc;
    {
      ProfScope p(E, ATARI_PROF_COPY, s);
      k_ring_append<<<E->n, 128, 0, s>>>(d_obs, d_rewards, d_dones, d_ring_planes, d_ring_rewards, d_ring_dones,
                                        E->n, slot);
    }
    CUDA_TRY(cudaGetLastError());
  }
  return 0;
}

int atari_env_rollout(atari_env *E, const uint16_t *d_weights, int n_steps, uint8_t *d_obs, uint8_t *d_actions,
                      int32_t *d_rewards, uint8_t *d_dones, uint8_t *d_ring_planes, float *d_ring_rewards,
                      int ring_depth, int ring_start, atari_stream stream) {
  return atari_env_rollout_ex(E, d_weights, n_steps, d_obs, d_actions, d_rewards, d_dones, d_ring_planes,
                              d_ring_rewards, nullptr, nullptr, ring_depth, ring_start, stream);
}

static int check_rollout_args(const void *rew, const void *done, int depth, int start, const void *values, int T,
                              int n, float gamma) {
  if (n < 0 || T < 1 || depth < T || start < 0) return fail(ATARI_EINVAL, "need n >= 0, 1 <= T <= ring_depth, ring_start >= 0");
  if (!(gamma >= 0.0f && gamma <= 1.0f)) return fail(ATARI_EINVAL, "gamma must be in [0, 1]");
  if (n > 0 && (!rew || !done || !values)) return fail(ATARI_EINVAL, "NULL buffer");
  return 0;
}

int atari_nstep_returns(const float *d_rewards, const uint8_t *d_dones, int ring_depth, int ring_start,
                        const float *d_values, int T, int n, float gamma, float *d_returns, atari_stream stream) {
  g_err.clear();
  if (int rc = check_rollout_args(d_rewards, d_dones, ring_depth, ring_start, d_values, T, n, gamma)) return rc;
  if (n == 0) return 0;
  if (!d_returns) return fail(ATARI_EINVAL, "NULL buffer");
  k_nstep_returns<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_rewards, d_dones, ring_depth,
                                                                     ring_start % ring_depth, d_values, T, n, gamma,
                                                                     d_returns);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

int atari_vtrace(const float *d_rewards, const uint8_t *d_dones, const float *d_mu, int ring_depth, int ring_start,
                 const float *d_values, const float *d_pi, int T, int n, float gamma, float rho_bar, float c_bar,
                 float *d_vs, float *d_pg_adv, atari_stream stream) {
  g_err.clear();
  if (int rc = check_rollout_args(d_rewards, d_dones, ring_depth, ring_start, d_values, T, n, gamma)) return rc;
  if (!(c_bar >= 0.0f && rho_bar >= c_bar)) return fail(ATARI_EINVAL, "need rho_bar >= c_bar >= 0");
  if (n == 0) return 0;
  if (!d_mu || !d_pi || !d_vs || !d_pg_adv) return fail(ATARI_EINVAL, "NULL buffer");
  k_vtrace<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_rewards, d_dones, d_mu, ring_depth,
                                                              ring_start % ring_depth, d_values, d_pi, T, n, gamma,
                                                              rho_bar, c_bar, d_vs, d_pg_adv);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

int atari_env_profile(atari_env *E, int enable) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  E->profiling = enable != 0;
  return 0;
}

int atari_env_profile_read(atari_env *E, double *ms, uint64_t *launches) {
  g_err.clear();
  if (!E || !ms || !launches) return fail(ATARI_EINVAL, "bad argument");
  for (int k = 0; k < ATARI_PROF_SLOTS; ++k) { ms[k] = 0; launches[k] = 0; }
  for (auto &r : E->prof) {
    CUDA_TRY(cudaEventSynchronize(r.b));
    float t = 0;
    CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.slot] += t;
    launches[r.slot] += 1;
    E->pool.push_back(r.a);
    E->pool.push_back(r.b);
  }
  E->prof.clear();
  return 0;
}

int atari_env_launch_shape(atari_env *E, int *envs_per_warp, int *envs_per_block, int *raster_warps_per_frame,
                           int *grid, int *tia_warps, int *grouping) {
  g_err.clear();
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  const bool b = E->cfg.form == ATARI_FORM_BATCHED;
  if (envs_per_warp) *envs_per_warp = b ? E->lanes : 32;
  if (envs_per_block) *envs_per_block = b ? E->lanes * E->warps : 128;
  if (raster_warps_per_frame) *raster_warps_per_frame = b ? E->wpf : 1;
  if (grid) *grid = b ? E->grid : (E->n + 127) / 128;
  if (tia_warps) *tia_warps = (b && E->split) ? 2 : 1;
  if (grouping) *grouping = b ? (E->grouping | (E->compact ? 4 : 0)) : 1;
  return 0;
}

int atari_env_info(atari_env *E, int *n_envs, size_t *device_bytes) {
  if (!E) return fail(ATARI_EINVAL, "env is NULL");
  if (n_envs) *n_envs = E->n;
  if (device_bytes) *device_bytes = E->bytes;
  return 0;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free step
// For callers that cannot allocate device memory: code that runs under a
// framework whose allocator owns every device buffer, or inside a region of
// a fixed device-memory budget.  They pass their own state, start-state,
// action and output buffers; everything else the step needs lives in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
namespace {
constexpr int NA_MAX_ENVS = 64;
constexpr int NA_LOG_CAP = 4096;
constexpr size_t NA_ROM = 0;                                            // one cartridge, banks of 4 KB
constexpr size_t NA_DEC = NA_ROM + ROM_SLOT;                            // 256-entry decode table
constexpr size_t NA_INFO = NA_DEC + 1024;                               // cartridge info word
constexpr size_t NA_REW = NA_INFO + 256;                                // rewards (internal copy)
constexpr size_t NA_DONE = NA_REW + 4 * NA_MAX_ENVS;                    // dones (internal copy)
constexpr size_t NA_CTR = NA_DONE + 256;                                // counters
constexpr size_t NA_META = NA_CTR + 12 * NA_MAX_ENVS;                   // per frame: records, lines
constexpr size_t NA_SNAP = NA_META + 16 * NA_MAX_ENVS;                  // per frame: 64-byte snapshot
constexpr size_t NA_LOG = NA_SNAP + 128 * NA_MAX_ENVS;                  // per frame: TIA-write log
constexpr size_t NA_BYTES = NA_LOG + (size_t)NA_MAX_ENVS * 2 * NA_LOG_CAP * 4;
static __device__ __align__(256) uint8_t g_noalloc_scratch[NA_BYTES];

std::mutex g_na_mu;
void *g_na_addr[64] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side name of the array is not a device address).
int noalloc_scratch(uint8_t **out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(ATARI_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(ATARI_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_na_addr[dev] = p;
  }
  *out = static_cast<uint8_t *>(g_na_addr[dev]);
  return 0;
}

// Every env of this variant belongs to the one staged cartridge.
__global__ void __launch_bounds__(128) k_interp_noalloc(StepArgs a) {
  __shared__ uint32_t dec[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) dec[t] = a.dec[t];
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  uint8_t *st = a.state + (size_t)i * 256;
  st[S::ROM] = 0;
  st[S::ROM + 1] = 0;
  RomInfo ri = rom_info(a.info, 0);
  Console<GlobalMem> m;
  m.mem.ram = st + S::RAM;
  m.mem.rom = a.roms;
  m.dec = dec;
  m.scheme = ri.scheme;
  m.load(st);
  step_env(m, st, i, a, ri);
  if (!a.done_int[i]) m.store(st);
}
}  // namespace

extern "C" int atari_step_noalloc(const uint8_t *rom, size_t rom_size, atari_rom_meta meta, uint8_t *d_state,
                                  const uint8_t *d_cache, int n_cache, const uint8_t *d_actions, uint8_t *d_frame,
                                  int32_t *d_rewards, uint8_t *d_dones, int n_envs, int frameskip, int sticky,
                                  uint64_t seed, atari_stream stream) {
  g_err.clear();
  if (n_envs < 0 || n_envs > NA_MAX_ENVS)
    return fail(ATARI_EINVAL, "atari_step_noalloc: n_envs must be in 0.." + std::to_string(NA_MAX_ENVS) +
                                  " (the fixed scratch array holds at most that many envs)");
  const int sc = scheme_of(rom_size);
  if (!rom || sc < 0) return fail(ATARI_EINVAL, "atari_step_noalloc: ROM size must be 2048, 4096, 8192, 16384 or 32768");
  if (meta.score_addr < 0x80 || meta.gameover_addr < 0x80)
    return fail(ATARI_EINVAL, "atari_step_noalloc: score/game-over addresses must be in $80-$FF");
  if (n_cache < 1 || n_cache > 64) return fail(ATARI_EINVAL, "atari_step_noalloc: n_cache must be in 1..64");
  if (frameskip < 2 || frameskip > 16) return fail(ATARI_EINVAL, "atari_step_noalloc: frameskip must be in 2..16");
  if (sticky != 0 && sticky != 1) return fail(ATARI_EINVAL, "atari_step_noalloc: sticky must be 0 or 1");
  if (n_envs == 0) return 0;
  if (!d_state || !d_cache || !d_actions) return fail(ATARI_EINVAL, "atari_step_noalloc: NULL buffer");
  uint8_t *scr = nullptr;
  if (int rc = noalloc_scratch(&scr)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // cartridge image (2K mirrored), decode table and info word, from host
  // arrays that need no allocation
  static uint8_t img[ROM_SLOT];
  static uint32_t dec[256];
  static uint32_t info[64];
  std::lock_guard<std::mutex> lk(g_na_mu);
  memset(img, 0, sizeof img);
  if (rom_size == 2048) {
    memcpy(img, rom, 2048);
    memcpy(img + 2048, rom, 2048);
  } else {
    memcpy(img, rom, rom_size);
  }
  fill_decode_table(dec);
  memset(info, 0, sizeof info);
  info[0] = rom_info_word(rom_size, meta);
  CUDA_TRY(cudaMemcpyAsync(scr + NA_ROM, img, sizeof img, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(scr + NA_DEC, dec, sizeof dec, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(scr + NA_INFO, info, sizeof info, cudaMemcpyHostToDevice, s));
  // the previous call's frame records must not leak into this one
  CUDA_TRY(cudaMemsetAsync(scr + NA_META, 0, NA_LOG - NA_META, s));
  StepArgs a;
  a.state = d_state;
  a.cache = d_cache;
  a.roms = scr + NA_ROM;
  a.info = reinterpret_cast<const uint32_t *>(scr + NA_INFO);
  a.dec = reinterpret_cast<const uint32_t *>(scr + NA_DEC);
  a.actions = d_actions;
  a.rew_int = reinterpret_cast<int32_t *>(scr + NA_REW);
  a.done_int = scr + NA_DONE;
  a.rew_out = d_rewards;
  a.done_out = d_dones;
  a.log = reinterpret_cast<uint32_t *>(scr + NA_LOG);
  a.snap = scr + NA_SNAP;
  a.meta = reinterpret_cast<uint32_t *>(scr + NA_META);
  a.counters = reinterpret_cast<uint32_t *>(scr + NA_CTR);
  a.n = n_envs;
  a.frameskip = frameskip;
  a.sticky = sticky;
  a.n_cache = n_cache;
  a.log_cap = NA_LOG_CAP;
  a.first_slot = 1;
  a.seed = seed;
  k_interp_noalloc<<<(n_envs + 127) / 128, 128, 0, s>>>(a);
  CUDA_TRY(cudaGetLastError());
  if (d_frame) {
    k_raster<<<(unsigned)((n_envs + 3) / 4), 128, 0, s>>>(a.log, a.snap, a.meta, d_frame, (size_t)210 * 160, n_envs, 1,
                                                          NA_LOG_CAP);
    CUDA_TRY(cudaGetLastError());
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Serving ticks: the env is a pool of slots; each tick steps the slots of the
// sessions whose requests it carries (see env_internal.h).

namespace {

// Slots that start a new session: env fields cleared, key and cartridge set,
// episode 0 from the start-state cache, empty stack.  One block per slot.
__global__ void k_serve_init(uint8_t *state, const uint8_t *cache, const uint32_t *info, int32_t *env_rom,
                             uint32_t *env_key, uint8_t *ring, uint8_t *head, const int32_t *init, int n_init,
                             int n_cache, uint64_t seed) {
  const int k = blockIdx.x;
  if (k >= n_init) return;
  const int slot = init[k];
  const uint32_t rom = (uint32_t)init[n_init + k];
  const uint32_t key = (uint32_t)init[2 * n_init + k];
  if (threadIdx.x == 0) {
    uint8_t *st = state + (size_t)slot * 256;
    for (int b = 0x60; b < 0x80; ++b) st[b] = 0;
    Console<GlobalMem>::st32(st + S::ENV_KEY, key);
    st[S::ROM] = rom & 0xFF;
    st[S::ROM + 1] = rom >> 8;
    reset_from_cache(st, cache, info, rom, (uint32_t)n_cache, seed, key, 0u);
    env_rom[slot] = (int32_t)rom;
    env_key[slot] = key;
    head[slot] = 0;
  }
  uint4 *p = reinterpret_cast<uint4 *>(ring + (size_t)slot * 4 * 7056);
  for (int q = threadIdx.x; q < 4 * 7056 / 16; q += blockDim.x) p[q] = make_uint4(0, 0, 0, 0);
}

}  // namespace

namespace atari_internal {

int env_slots(const atari_env *E) { return E ? E->n : 0; }
int env_device(const atari_env *E) { return E ? E->device : 0; }
int env_n_roms(const atari_env *E) { return E ? E->n_roms : 0; }
int env_frameskip(const atari_env *E) { return E ? E->cfg.frameskip : 0; }
void env_shape(const atari_env *E, int *lanes, int *warps) {
  *lanes = E->lanes;
  *warps = E->warps;
}
int set_error(int code, const std::string &msg) { return fail(code, msg); }

int serve_tick(atari_env *E, const ServeTick &t, cudaStream_t s) {
  if (!E || E->cfg.form != ATARI_FORM_BATCHED || E->cfg.output_mode != ATARI_OUT_STACK)
    return fail(ATARI_EINVAL, "serving needs a batched env with stack output");
  if (t.n_active <= 0) return 0;
  const atari_config &c = E->cfg;
  if (t.n_init > 0) {
    k_serve_init<<<t.n_init, 128, 0, s>>>(E->d_state, E->d_cache, E->d_info, E->d_env_rom, E->d_env_key, E->d_ring,
                                          E->d_head, t.d_init, t.n_init, c.n_cache, c.seed);
    CUDA_TRY(cudaGetLastError());
  }
  BatchArgs a = batch_args(E, t.d_actions, t.d_rew, t.d_done);
  a.grp_rom = t.d_blob;
  a.grp_start = t.d_blob + t.n_groups;
  a.grp_count = t.d_blob + 2 * t.n_groups;
  a.perm = t.d_blob + 3 * t.n_groups;
  a.opos = a.perm + t.n_active;
  a.queue = t.d_queue;
  a.n_groups = t.n_groups;
  CUDA_TRY(cudaMemsetAsync(t.d_queue, 0, sizeof(int), s));
  const int grid = std::max(1, std::min(t.n_groups, E->max_blocks));
  launch_interp(E, a, grid, s);
  CUDA_TRY(cudaGetLastError());
  k_raster_preprocess<<<t.n_active, 64 * E->wpf, fused_smem(), s>>>(E->d_log, E->d_snap, E->d_bsnap, E->d_meta, E->d_luma,
                                                                   E->d_ring, E->d_head, E->d_done, t.d_obs,
                                                                   t.n_active, c.log_cap, E->wpf, a.perm, a.opos, 0);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace atari_internal
