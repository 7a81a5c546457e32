/*
 * atari_gpu.h -- C ABI of the batched Atari 2600 emulator for GB300 (sm_103a).
 *
 * The library steps thousands of independent consoles (MOS 6507 CPU, TIA
 * video/collision chip, RIOT 6532 RAM/timer/ports, 2-32 KB cartridges with
 * F8, F6 and F4 bank switching) in lockstep on one GPU.  It is the data-parallel
 * emulation path of "Accelerating Reinforcement Learning through GPU Atari
 * Emulation" (CuLE), Section 3: a CPU-interpreter kernel that logs TIA
 * register writes to a per-env buffer in device memory, a TIA kernel that
 * replays that buffer into 160x210 frames, only the last two frames of a
 * four-frame skip rendered (their pixelwise maximum is the agent's input),
 * and episode reset by copying one of 30 cached random start states.
 *
 * Conventions for every entry point:
 *   - Return 0 on success or a negative code (ATARI_E*).  Nothing throws
 *     across the ABI.  atari_last_error() gives a thread-local message for
 *     the last failing call on the calling thread.
 *   - Pointers named d_* are DEVICE pointers on the device current when the
 *     env was created; every other pointer is a host pointer.
 *   - Device work is enqueued on the caller's stream (NULL = legacy default
 *     stream).  atari_env_step does not synchronise the host.
 *   - Per-env machine faults never fail a call: they set bits of the env's
 *     status word (ATARI_ST_*), readable with atari_env_status.
 *   - Ownership: the library owns all machine state, logs, frames, the start
 *     state cache and its copies of the ROMs (ROM bytes are copied at create,
 *     the caller may free them).  The caller owns action and output buffers.
 */
#ifndef ATARI_GPU_H
#define ATARI_GPU_H
#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ATARI_API __attribute__((visibility("default")))
#else
#define ATARI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct atari_env atari_env;   /* opaque, library-owned */
typedef void *atari_stream;           /* a cudaStream_t */

/* error codes */
#define ATARI_OK 0
#define ATARI_EINVAL (-22)   /* bad argument, ROM size or configuration */
#define ATARI_ENOMEM (-12)   /* device or host allocation failed */
#define ATARI_ECUDA (-5)     /* a CUDA runtime call failed (message has the CUDA error) */

/* per-env status bits (sticky for the life of the env) */
#define ATARI_ST_ILLEGAL 1u       /* undocumented opcode: CPU halted, env done at step end */
#define ATARI_ST_FRAME_CAP 2u     /* a frame ran 400 lines without a VSYNC rise */
#define ATARI_ST_LOG_OVERFLOW 4u  /* a rendered frame wrote more TIA registers than log_cap */
#define ATARI_ST_BAD_ACTION 8u    /* an action >= 18 was taken as NOOP */
#define ATARI_ST_STALL 16u        /* a bounded wait between an env's CPU and TIA warps ran out (tia_warps 2); the env halts */

/* output modes */
#define ATARI_OUT_PALETTE 0  /* d_obs = uint8 [n][210][160] palette values (COLU & 0xFE) of frame F */
#define ATARI_OUT_STACK 1    /* d_obs = uint8 [n][4][84][84] luma stack, slot 3 newest */

/* execution forms */
#define ATARI_FORM_PLAIN 0      /* one launch per kernel per step, state/RAM/ROM in global memory */
#define ATARI_FORM_BATCHED 1    /* ROM-grouped persistent interpreter (RAM/ROM in shared memory),
                                   fused rasterise+preprocess, whole step captured in a CUDA graph */

/* RAM addresses ($80-$FF) of a cartridge's score byte (reward = per-frame
 * int8 delta, summed over the step) and game-over byte (done when nonzero). */
typedef struct {
    uint8_t score_addr;
    uint8_t gameover_addr;
} atari_rom_meta;

typedef struct {
    int frameskip;        /* frames per step F, 2..16 (paper: 4); frames F-1 and F are rendered */
    int sticky;           /* 1: each frame repeats the previous frame's action with p = 1/4 */
    int n_cache;          /* cached start states per ROM, 1..64 (paper: 30) */
    int startup_frames;   /* no-op frames from power-on before the first cached state (paper: 64) */
    int max_noops;        /* extra random no-op frames, 0..max_noops (paper: up to 30) */
    int output_mode;      /* ATARI_OUT_* */
    int form;             /* ATARI_FORM_* */
    int log_cap;          /* TIA-write log entries per rendered frame (>= 256; default 4096) */
    int envs_per_block;   /* batched form: envs per interpreter block, <= 128 (0 = autotune) */
    int envs_per_warp;    /* batched form: envs per warp, 1..32 (0 = autotune); fewer than 32 trades
                             SIMT width for more independent instruction streams on small batches */
    int raster_warps_per_frame; /* batched form: warps rendering one frame, 1..4 (0 = autotune) */
    uint64_t seed;        /* Philox4x32-10 key for start states, resets and sticky draws */
    int tia_warps;        /* batched form: 1 = each warp runs its envs' CPU and TIA; 2 = a TIA warp per
                             CPU warp takes the TIA writes, logging and collisions off the CPU's
                             path; 0 = autotune; 3 = as 2 with the TIA side switched off, to test the
                             bounded waits (every env ends its steps with ATARI_ST_STALL) */
    int grouping;         /* batched form, how envs of one cartridge are ordered into warps: 1 = env order;
                             2 = bank-aware: re-sorted at every step by the bank their state holds at the
                             step's start (stable in env order), so a warp's lanes start in one bank of an
                             banked cartridge; 0 = autotune */
    int dispatch;         /* batched form, the interpreter's hot opcode switch: 1 = every common opcode inline;
                             2 = compact (indirect forms, BIT, stack pushes and pulls, indexed and absolute
                             read-modify-writes through the general decoder: a smaller hot loop); 0 = autotune */
    int idle_skip;        /* batched form: 1 = a RIOT-timer wait loop (LDA INTIM at PC, BNE back to PC) retires
                             the iterations that read a nonzero timer value at once (cycles and instruction
                             counts advanced exactly; same results), 0 = every iteration runs.  Default 1;
                             the plain form runs every iteration */
} atari_config;

/* Fill *cfg with the paper's defaults: F = 4, no sticky actions, 30 cached
 * states, 64 start-up frames, up to 30 no-ops, stack output, plain form,
 * log_cap 4096, autotuned launch shapes, timer-wait skipping on, seed 1. */
ATARI_API void atari_default_config(atari_config *cfg);

/*
 * Create n_envs environments.  roms[r] (host) holds rom_sizes[r] bytes:
 * 2048 or 4096 (plain, 2K mirrored), 8192 (F8), 16384 (F6) or 32768 (F4); other sizes
 * return ATARI_EINVAL.  env_rom[i] (host, n_envs) picks env i's cartridge;
 * env_key[i] (host, may be NULL = i) keys env i's random streams, so a
 * subset of envs created with the same keys reproduces the same run.
 * luma (host, 128 bytes) maps palette index (value >> 1) to luma; required
 * for ATARI_OUT_STACK, ignored otherwise.  Builds the start-state cache on
 * the device (Section 3, reset strategy) and resets every env to
 * cache[rom][mulhi32(philox(seed, env_key, 0, 2 << 8, 0), n_cache)].
 * Synchronous.  On success *out receives the env.
 */
ATARI_API int atari_env_create(const uint8_t *const *roms, const size_t *rom_sizes, const atari_rom_meta *meta,
                     int n_roms, const int32_t *env_rom, const uint32_t *env_key, int n_envs,
                     const atari_config *cfg, const uint8_t *luma, atari_env **out);

/*
 * Force a reset of the envs whose d_mask byte is nonzero (d_mask NULL: all):
 * episode += 1, state <- cached start state, frame stack zeroed.
 * Paper, Section 3 (reset strategy): at the end of an episode an emulator
 * copies a randomly chosen cached start state into its terminal state, in
 * place of running 64 start-up frames and up to 30 random no-op frames.  The
 * cached state is cache[rom][mulhi32(philox(seed, env_key, 0, 2 << 8,
 * episode), n_cache)] with the incremented episode.  d_mask (device, n bytes)
 * is read on `stream`; NULL env returns ATARI_EINVAL.
 */
ATARI_API int atari_env_reset(atari_env *env, const uint8_t *d_mask, atari_stream stream);

/*
 * One step of every env.  Paper, Section 1 (the inference path: environments
 * take an action set and return the next observable states and rewards),
 * Section 1 footnote (frame skip 4, every emulated frame counted) and
 * Section 3 (only the last two frames of the four are rendered; the agent's
 * input is their pixelwise maximum; finished episodes restart from the
 * cache of start states).
 * d_actions[i] (device, uint8, ALE action 0..17) is
 * applied for F frames (sticky repeats drawn per frame when enabled).
 * Writes d_obs (layout per output_mode), d_rewards[i] (int32: sum over the F
 * frames of the int8 change of the score byte) and d_dones[i] (uint8: the
 * game-over byte is nonzero after frame F, or the CPU halted).  Envs that are
 * done are reset on the device after their observation is written; the
 * observation returned is the terminal one.  Any output pointer may be NULL
 * to skip that output.
 */
ATARI_API int atari_env_step(atari_env *env, const uint8_t *d_actions, uint8_t *d_obs, int32_t *d_rewards,
                   uint8_t *d_dones, atari_stream stream);

/*
 * Same step with host buffers (the host round trip of Section 1's inference
 * path, for callers whose agent runs on the host): copies actions host->device, steps, and
 * copies obs / rewards / dones device->host, then returns with every copy
 * complete.  Host pointers may be pageable or pinned (pinned lets the copies
 * overlap the rendering); NULL skips.  In the batched form with stack output
 * the env renders in chunks of envs on `stream` and copies each chunk's
 * stacks back on a stream of its own while the next chunk renders; results
 * are the same as atari_env_step's.  Other forms copy on `stream`.
 */
ATARI_API int atari_env_step_host(atari_env *env, const uint8_t *actions, uint8_t *obs, int32_t *rewards,
                        uint8_t *dones, atari_stream stream);

/*
 * Inference-path policy (paper Section 4, inference-only measurements: a
 * network picks actions on the GPU next to the emulator).  A linear softmax
 * over the stack: logits[j] = sum_k obs[k] * W[k][j] for k = plane * 7056 +
 * row * 84 + column, d_weights (device) = bf16 bit patterns [28224][18],
 * fp32 accumulation in a fixed order (441 chunks of 64 sequential fused
 * multiply-adds; chunk partials reduced by s[i] += s[i + h], h = 256 .. 1,
 * over 512 zero-padded slots), softmax weights exp(l - max) by Cody-Waite
 * reduction and a degree-7 polynomial, action = smallest j whose running
 * weight sum exceeds u * total, u = 24-bit fraction of the env's Philox word
 * (seed; env key, step, 4 << 8, episode).  d_obs (device) = [n][4][84][84]
 * (stack output mode required); d_actions (device, n) receives the actions,
 * d_logits (device, n * 18 floats, may be NULL) the logits.
 */
ATARI_API int atari_env_policy(atari_env *env, const uint8_t *d_obs, const uint16_t *d_weights, uint8_t *d_actions,
                               float *d_logits, atari_stream stream);

/*
 * The inference-path loop, entirely on the device: n_steps iterations of
 * policy(d_obs) -> d_actions, atari_env_step(d_actions) -> d_obs, d_rewards,
 * d_dones, then the newest plane of every env's stack and its reward (as
 * float) appended to ring slot (ring_start + t) mod ring_depth of
 * d_ring_planes (device, [ring_depth][n][84*84]) and d_ring_rewards
 * (device, [ring_depth][n]).  No host synchronisation.
 */
ATARI_API int atari_env_rollout(atari_env *env, const uint16_t *d_weights, int n_steps, uint8_t *d_obs,
                                uint8_t *d_actions, int32_t *d_rewards, uint8_t *d_dones, uint8_t *d_ring_planes,
                                float *d_ring_rewards, int ring_depth, int ring_start, atari_stream stream);

/*
 * The inference-path loop with the training buffer V-trace needs (paper
 * Appendix, "V-trace": the behaviour probabilities mu(a|s) are stored with
 * the experiences).  As atari_env_rollout, and also: d_ring_dones (device,
 * uint8 [ring_depth][n], may be NULL) receives each step's dones, d_ring_mu
 * (device, float [ring_depth][n], may be NULL) the probability the policy
 * gave the action it sampled (its softmax weight over the total, fp32), in
 * the same ring slot as the step's plane and reward.
 */
ATARI_API int atari_env_rollout_ex(atari_env *env, const uint16_t *d_weights, int n_steps, uint8_t *d_obs,
                                   uint8_t *d_actions, int32_t *d_rewards, uint8_t *d_dones, uint8_t *d_ring_planes,
                                   float *d_ring_rewards, uint8_t *d_ring_dones, float *d_ring_mu, int ring_depth,
                                   int ring_start, atari_stream stream);

/*
 * Learner-side targets over a rollout held in a device ring (paper Appendix,
 * "A2C": the bootstrapped N-step return R_t = sum_{i<k} gamma^i r_{t+i} +
 * gamma^k V(s_{t+k}); "V-trace": the target v_t of the sum definition with
 * truncated importance weights rho_t = min(rho_bar, pi_t / mu_t) and c_t =
 * min(c_bar, pi_t / mu_t), computed by the paper's recursive form
 * v_t = V_t + delta_t + gamma c_t (v_{t+1} - V_{t+1}), and the actor's
 * advantage rho_t (r_t + gamma v_{t+1} - V_t)).
 *
 * Step t (0 <= t < T) of the rollout is ring slot (ring_start + t) mod
 * ring_depth of d_rewards (float [ring_depth][n]), d_dones (uint8, same
 * shape) and d_mu (float, same shape: behaviour probabilities, > 0), as
 * atari_env_rollout_ex writes them.  d_values (float [T + 1][n]) holds
 * V(s_0) .. V(s_T), row T the bootstrap value of the state after the last
 * step; d_pi (float [T][n]) the target policy's probabilities of the actions
 * taken.  Outputs (float [T][n], time-major): d_returns; d_vs (targets) and
 * d_pg_adv (advantages).  All buffers are device memory owned by the caller.
 * Reading where the paper is silent: a done at step t ends the return there
 * (the discount after step t is 0, no bootstrap across an episode end).
 * fp32, one rounding per operation in the order above, so results are
 * within a few units of fp32 rounding of the exact values, not bit-equal to
 * a double computation.  ATARI_EINVAL for T < 1, T > ring_depth,
 * ring_start < 0, gamma outside [0, 1], rho_bar < c_bar or c_bar < 0, or a
 * NULL buffer with n > 0.  Enqueued on `stream`.
 */
ATARI_API int atari_nstep_returns(const float *d_rewards, const uint8_t *d_dones, int ring_depth, int ring_start,
                                  const float *d_values, int T, int n, float gamma, float *d_returns,
                                  atari_stream stream);
ATARI_API int atari_vtrace(const float *d_rewards, const uint8_t *d_dones, const float *d_mu, int ring_depth,
                           int ring_start, const float *d_values, const float *d_pi, int T, int n, float gamma,
                           float rho_bar, float c_bar, float *d_vs, float *d_pg_adv, atari_stream stream);

/* d_status (device, uint32 [n]) <- per-env status bits (ATARI_ST_*), on
 * `stream`.  The paper is silent on machine faults; here they never fail a
 * call: an undocumented opcode halts that env's CPU (done at step end), a
 * frame longer than 400 lines ends at the cap, a log overflow truncates that
 * frame's rendering, an out-of-range action runs as NOOP, and a split-form
 * wait that runs out halts the env.  Each sets its bit for the life of the
 * env.  NULL env or d_status returns ATARI_EINVAL. */
ATARI_API int atari_env_status(atari_env *env, uint32_t *d_status, atari_stream stream);

/*
 * Canonical per-env state, 256 bytes per env, little-endian (layout in the
 * table below).  get copies n*256 bytes to d_dst; set loads them from d_src
 * (both device buffers owned by the caller, copied on `stream`).  The paper
 * keeps each console's CPU state and its 128 bytes of RAM in device memory
 * (Section 3) but defines no save/restore; this layout is the library's
 * own.  A saved state restores a run exactly: the random streams are keyed
 * by fields inside it.  A bank byte with bits the cartridge does not latch
 * is reduced to the cartridge's bits when the state is next stepped.  NULL
 * env or buffer returns ATARI_EINVAL.
 *
 *   0x00 A  0x01 X  0x02 Y  0x03 SP  0x04 P (bit 5 set, B clear)  0x05 bank
 *   0x06 u16 PC   0x08 u64 CPU cycle   0x10 u64 RIOT timer write cycle
 *   0x18 timer value  0x19 timer shift (0,3,6,10)  0x1A SWCHA out  0x1B SWACNT
 *   0x1C SWCHB out  0x1D SWBCNT  0x1E jam  0x1F INPT4 latch
 *   0x20..0x3F TIA: VSYNC VBLANK NUSIZ0 NUSIZ1 COLUP0 COLUP1 COLUPF COLUBK
 *        CTRLPF REFP0 REFP1 PF0 PF1 PF2 ENAM0 ENAM1 ENABL(new) ENABL(old)
 *        GRP0(new) GRP0(old) GRP1(new) GRP1(old) VDELP0 VDELP1 VDELBL
 *        RESMP0 RESMP1 HMP0 HMP1 HMM0 HMM1 HMBL
 *   0x40..0x44 positions P0 P1 M0 M1 BL (0..159)   0x46 u16 collision latches
 *        (bit 2r+1 = D7, bit 2r = D6 of read register r)
 *   0x48 u64 HMOVE-bar line (all ones: none)   0x50 u64 first line of frame
 *   0x58 u32 frames since power-on
 *   0x60 u32 episode  0x64 u32 step  0x68 u32 env key  0x6C u32 status
 *   0x70 last applied action  0x71 score baseline  0x72 u16 ROM index
 *   0x80..0xFF the 128 bytes of RAM
 */
ATARI_API int atari_env_get_state(atari_env *env, void *d_dst, atari_stream stream);
ATARI_API int atari_env_set_state(atari_env *env, const void *d_src, atari_stream stream);

/* d_dst <- the two rendered frames of the last step, uint8 [n][2][210][160]
 * (frames F-1 and F, palette values).  Available in the plain form only
 * (the batched form never materialises frames); ATARI_EINVAL otherwise. */
ATARI_API int atari_env_get_frames(atari_env *env, uint8_t *d_dst, atari_stream stream);

/* d_dst <- the start-state cache, [n_roms][n_cache][256] canonical states
 * (the cache of random initial states of Section 3's reset strategy).
 * Device buffer owned by the caller, copied on `stream`. */
ATARI_API int atari_env_get_cache(atari_env *env, void *d_dst, atari_stream stream);

/* Counters of the last step: 6502 instructions executed (sum over envs; the
 * iterations of a RIOT-timer wait loop that the batched form retires at once,
 * see idle_skip, are not counted), TIA
 * log records written, and lockstep issue rounds summed over the envs (each
 * env counts the rounds its warp issued, so instructions / lane_rounds is
 * the fraction of a warp's lanes that execute per round: the emulated-
 * instruction SIMT efficiency the paper's divergence discussion in Section 4
 * is about; 0 in the plain form, which has no lockstep issue).  Host
 * pointers, any may be NULL; synchronises `stream`. */
ATARI_API int atari_env_counters(atari_env *env, uint64_t *instructions, uint64_t *log_records,
                                 uint64_t *lane_rounds, atari_stream stream);

/*
 * Per-kernel device timing.  With profiling enabled, every kernel launch of
 * atari_env_step is bracketed by CUDA events recorded on the step's stream.
 * atari_env_profile_read waits for the recorded work, then returns for each
 * kernel slot the summed milliseconds and the launch count since the last
 * read, and clears them.  ms and launches are host arrays of ATARI_PROF_SLOTS.
 */
#define ATARI_PROF_SLOTS 8
#define ATARI_PROF_INTERP 0     /* 6507+RIOT interpreter (all frames of a step) */
#define ATARI_PROF_RASTER 1     /* TIA replay into frames */
#define ATARI_PROF_PREPROC 2    /* luma / max / 84x84 / stack */
#define ATARI_PROF_FUSED 3      /* fused replay + preprocessing (batched form) */
#define ATARI_PROF_COPY 4       /* output copies, rollout-ring appends */
#define ATARI_PROF_POLICY 5     /* linear softmax policy */
#define ATARI_PROF_GROUP 6      /* bank-aware regrouping of the env list (batched form, grouping 2) */
ATARI_API int atari_env_profile(atari_env *env, int enable);
ATARI_API int atari_env_profile_read(atari_env *env, double *ms, uint64_t *launches);

/* Launch shape in use (batched form: the autotuned or configured values;
 * plain form: 32 envs per warp, 128 per block, 1 warp per frame, and the
 * grid of the interpreter launch).  tia_warps: 2 when paired TIA warps run
 * the envs' TIA side, else 1.  grouping: 1 env order, 2 bank-aware (see
 * atari_config; the plain form reports 1), plus 4 when the compact opcode
 * switch is in use.  Host pointers; any may be NULL.
 * The paper runs one emulator per thread with no grouping (Section 3); the
 * shape is this library's own tuning and changes speed only, never results. */
ATARI_API int atari_env_launch_shape(atari_env *env, int *envs_per_warp, int *envs_per_block,
                                     int *raster_warps_per_frame, int *grid, int *tia_warps, int *grouping);

/* Number of envs, and the bytes of device memory the env holds. */
ATARI_API int atari_env_info(atari_env *env, int *n_envs, size_t *device_bytes);

/* Device bytes atari_env_create would allocate for this configuration
 * (used for admission against a memory budget; Section 4 discusses the
 * device-memory cost per environment of frames and emulator state). */
ATARI_API size_t atari_env_footprint(int n_envs, int n_roms, const atari_config *cfg);

/* Free every device and host allocation of the env (library-owned state,
 * logs, cache, ROM copies, captured graphs).  The paper defines no teardown;
 * the caller must not use the env afterwards, and work still queued on a
 * stream that uses it must have finished.  Safe on NULL. */
ATARI_API void atari_env_destroy(atari_env *env);

/*
 * Allocation-free step, for callers that cannot allocate device memory (a
 * framework whose allocator owns every device buffer, or a fixed device
 * memory budget): it calls no cudaMalloc/cudaFree.  The paper has no
 * counterpart; it is a variant of the plain-form step above.
 *
 * Steps n_envs <= 64 envs of ONE cartridge (rom, host, rom_size bytes; meta
 * gives its score and game-over RAM addresses).  d_state (device, n*256
 * canonical states, in/out) is advanced one step of `frameskip` frames with
 * d_actions (device, n bytes); every state's ROM index field is set to 0.
 * d_cache (device, n_cache*256) holds the cartridge's start states (e.g. from
 * atari_env_get_cache); finished envs are reset from it as in
 * atari_env_step.  d_frame (device, n*210*160, may be NULL) receives frame F
 * (palette values), d_rewards / d_dones (device, may be NULL) the rewards and
 * dones.  Results equal atari_env_step of a plain-form env with palette
 * output and log_cap 4096 on the same states and actions: the scratch log
 * holds 4096 TIA writes per rendered frame, so a frame with more writes is
 * truncated and its env flagged ATARI_ST_LOG_OVERFLOW, as in such an env.
 *
 * Its scratch (the cartridge image, TIA-write logs and frame records) is one
 * fixed array of about 2.1 MB inside the library, held by every GPU that
 * loads the library until the process exits.  n_envs above 64 returns
 * ATARI_EINVAL.  The first call on a device looks up that array's device
 * address; make that first call before any stream capture.  Every call
 * shares the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.
 */
ATARI_API int atari_step_noalloc(const uint8_t *rom, size_t rom_size, atari_rom_meta meta, uint8_t *d_state,
                                 const uint8_t *d_cache, int n_cache, const uint8_t *d_actions, uint8_t *d_frame,
                                 int32_t *d_rewards, uint8_t *d_dones, int n_envs, int frameskip, int sticky,
                                 uint64_t seed, atari_stream stream);

/* Thread-local message describing the last failing call on this thread ("" if
 * none).  Owned by the library; valid until the next call on the same
 * thread.  The paper defines no error reporting; every entry point returns
 * a negative ATARI_E* code and sets this message instead of throwing. */
ATARI_API const char *atari_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
