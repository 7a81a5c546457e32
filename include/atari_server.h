/*
 * atari_server.h -- C ABI of the serving loop over the batched emulator.
 *
 * Many clients step their own sessions (n envs of one cartridge each) through
 * one GPU.  All machine state stays resident in device memory.  New sessions
 * are admitted while the device bytes they need fit a stated budget.  This
 * follows the paper's memory-limit discussion in Section 4 (frames and state
 * grow linearly with the env count).  Step requests that arrive while earlier
 * ticks run on the GPU go into the next tick: continuous batching with up to
 * `inflight` ticks on the device at once, each on its own stream.  A tick
 * packs the requests' envs cartridge by cartridge into one persistent
 * interpreter launch.  The fused rasterise + preprocess kernel follows, then
 * each request's outputs are copied back to it.
 *
 * Determinism: env j of a session is keyed key_base + j for every random
 * draw (sticky actions, reset choices).  A session's results therefore depend
 * only on its cartridge, its keys, its actions and the server's ROM list and
 * configuration.  They are bit-identical whether it runs alone or beside other
 * sessions, and equal to an atari_env created with the same ROM list and
 * env_key[j] = key_base + j.
 *
 * Conventions are those of atari_gpu.h (0 or a negative ATARI_E* code,
 * atari_last_error() for the message; all pointers here are host pointers).
 * Threads: open/step/close/get_stats may be called from any number of client
 * threads at once.  Only one step of a given session may be outstanding at a
 * time; a second one gets ATARI_EBUSY.
 */
#ifndef ATARI_SERVER_H
#define ATARI_SERVER_H
#include "atari_gpu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct atari_server atari_server;   /* opaque, library-owned */

#define ATARI_EAGAIN (-11)    /* a session was not admitted within the timeout (it is withdrawn) */
#define ATARI_EBUSY (-16)     /* the session already has a step in flight, or close during a step */
#define ATARI_ESESSION (-3)   /* no such open session (never opened, closed, or reclaimed as idle) */

typedef struct {
    uint64_t budget_bytes;  /* device bytes the server may hold in all (default 40 GB) */
    int max_slots;          /* upper bound on resident envs; 0 = as many as the budget allows */
    int max_tick_envs;      /* envs one tick may carry; 0 = every slot */
    int max_session_envs;   /* largest session accepted; 0 = 2048 */
    int inflight;           /* ticks in flight at once, 1..4; 0 = 2 */
    int idle_timeout_ms;    /* admitted sessions idle this long are closed; 0 = never */
} atari_server_config;

typedef struct {
    int64_t submit_ns;      /* steady-clock time the request was queued */
    int64_t launch_ns;      /* ... taken into a tick */
    int64_t done_ns;        /* ... its outputs were in the caller's buffers */
    int tick_envs;          /* envs carried by that tick */
} atari_request_info;

typedef struct {
    uint64_t ticks, requests, env_steps, sessions_admitted;
    uint64_t launches;      /* kernels launched by the ticks so far */
    uint64_t budget_bytes, bytes_in_use, fixed_bytes, per_env_bytes;
    int capacity;           /* env slots allocated on the device */
    int free_slots, queued_sessions, pending_requests;
    uint64_t overlapped_ticks;  /* ticks whose device work began before an earlier tick's had ended
                                   (CUDA events on the ticks' streams): continuous batching overlapping
                                   on the GPU, not only queued on the host */
} atari_server_stats;

ATARI_API void atari_server_default_config(atari_server_config *c);

/* Device bytes a server of this configuration holds for `slots` env slots
 * and `tick_envs` envs per tick (cartridges, cache, slots, tick buffers). */
ATARI_API size_t atari_server_footprint(int slots, int tick_envs, int n_roms, const atari_config *cfg,
                                        const atari_server_config *scfg);

/* Create a server on the current device.  cfg must select ATARI_FORM_BATCHED
 * and ATARI_OUT_STACK; the luma table is required.  The slot count is
 * the largest that fits budget_bytes, capped by max_slots.  The tick buffers
 * are sized for max_tick_envs.  Everything is allocated here, and nothing on
 * the device is allocated per request.  A cfg without an envs_per_warp /
 * envs_per_block choice gets 32 envs per warp, 128 per block.  Returns
 * ATARI_ENOMEM when not even one env fits the budget. */
ATARI_API int atari_server_create(const uint8_t *const *roms, const size_t *rom_sizes, const atari_rom_meta *meta,
                                  int n_roms, const atari_config *cfg, const uint8_t *luma,
                                  const atari_server_config *scfg, atari_server **out);

/* Open a session of n_envs envs (1..max_session_envs) of cartridge `rom`,
 * keyed key_base + j.  Admission is FIFO: a session waits while any earlier
 * queued session waits or while it does not fit (free slots and budget).
 * Blocks up to timeout_ms (negative: no limit).  On timeout the session is
 * withdrawn and ATARI_EAGAIN returned.  A session larger than the whole
 * budget gets ATARI_ENOMEM at once.  Its envs start from a cached start state
 * (episode 0) with their first step. */
ATARI_API int atari_server_open(atari_server *S, int rom, int n_envs, uint32_t key_base, int timeout_ms,
                                int *session);

/* One step of every env of the session: actions[n_envs] in, obs[n_envs][4][84][84]
 * (may be NULL), rewards[n_envs] and dones[n_envs] out.  Blocks until the
 * outputs are in place.  Page-locked output buffers are written by the copy
 * engine directly; pageable ones are filled after the tick completes.
 * info (may be NULL) receives the request's timestamps. */
ATARI_API int atari_server_step(atari_server *S, int session, const uint8_t *actions, uint8_t *obs,
                                int32_t *rewards, uint8_t *dones, atari_request_info *info);

/* Close a session and free its slots, admitting queued sessions. */
ATARI_API int atari_server_close(atari_server *S, int session);

ATARI_API int atari_server_get_stats(atari_server *S, atari_server_stats *out);

/* Stop the server threads and free everything.  No client call may be in
 * progress. */
ATARI_API void atari_server_destroy(atari_server *S);

/* Closed-loop load generator run inside the library, with one native
 * thread per client.  Each client repeats the following until `seconds`
 * have passed:
 *   1. open a session of U{min_envs..max_envs} envs on U{0..n_roms-1};
 *   2. step it a geometric number of times (mean session_steps_mean), with
 *      uniform random actions and an Exp(think_mean_ms) pause after each
 *      reply;
 *   3. close it.
 * Results: request latency percentiles (submit to outputs in place),
 * admission waits and aggregate emulated frames per second. */
typedef struct {
    int n_clients;
    double seconds;
    double think_mean_ms;
    int min_envs, max_envs;
    double session_steps_mean;
    uint64_t seed;
    int want_obs;           /* 1: every request takes its 84x84x4 stacks back to host memory */
} atari_loadgen_config;

typedef struct {
    uint64_t requests, env_steps, frames, sessions;
    double seconds, frames_per_s;
    double p50_ms, p99_ms, max_ms, mean_ms;
    double admit_p50_ms, admit_p99_ms;
    uint64_t ticks;
    double mean_tick_envs;
    uint64_t h2d_bytes, d2h_bytes;   /* request payload bytes moved (actions in; stacks, rewards, dones out) */
} atari_loadgen_result;

ATARI_API int atari_server_loadgen(atari_server *S, const atari_loadgen_config *c, atari_loadgen_result *out);

#ifdef __cplusplus
}
#endif
#endif
