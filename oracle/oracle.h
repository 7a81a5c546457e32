/*
 * CPU oracle for the batched Atari 2600 emulation path -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  The product (CUDA) path never calls it and
 * shares no code, header, table or helper with it.
 *
 * What it computes: the exact, definitional emulation the paper's CuLE system
 * performs (Section 3, "CUDA Learning Environment"): one console per
 * environment, each step a frame-skipped run of the machine, the last two
 * frames rendered, a pixelwise maximum over them (Section 3, second
 * advantage of the two-kernel split), rewards and dones, and reset from a
 * cache of random start states (Section 3, reset strategy: 64 start-up frames
 * plus up to 30 random no-op frames, 30 cached states).
 *
 * The machine itself (6507, TIA, RIOT, cartridges) is not specified by the
 * paper; the oracle follows the public machine definition with the readings
 * stated in oracle.c's header comment.  It takes the slowest faithful route:
 * instruction by instruction with cycle accounting, and the TIA advanced one
 * color clock at a time, every pixel and collision computed from the live
 * registers (no log, no replay).
 */
#ifndef ATARI_ORACLE_H
#define ATARI_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_STATE_BYTES 256
#define ORC_FRAME_H 210
#define ORC_FRAME_W 160
#define ORC_OBS 84

/* status bits (sticky per env) */
#define ORC_ST_ILLEGAL 1u     /* CPU met an undocumented opcode and halted (JAM) */
#define ORC_ST_FRAME_CAP 2u   /* a frame ran 400 lines without a VSYNC rise */
#define ORC_ST_BAD_ACTION 8u  /* an action >= 18 was taken as NOOP */

typedef struct orc_machine orc_machine;
typedef struct orc_envs orc_envs;

/* ---- machine-level hooks (hand-assembled programs, definition tests) ---- */
orc_machine *orc_machine_new(const uint8_t *rom, size_t rom_size); /* NULL on bad size */
void orc_machine_free(orc_machine *m);
int orc_machine_step(orc_machine *m);            /* one instruction; returns cycles (incl. WSYNC stall) or -1 if jammed */
int orc_machine_run_frame(orc_machine *m, uint8_t *fb /* 210*160 or NULL */); /* returns lines in frame */
void orc_machine_set_action(orc_machine *m, int action);
void orc_machine_get_state(const orc_machine *m, uint8_t *out256);
void orc_machine_set_state(orc_machine *m, const uint8_t *in256);
uint64_t orc_machine_cycles(const orc_machine *m);
uint8_t orc_machine_peek(orc_machine *m, uint16_t addr);       /* side-effect-free view of RAM/ROM */
int orc_machine_last_vsync(const orc_machine *m, uint64_t *cycle); /* cycle of last VSYNC rise */
uint32_t orc_machine_tia_writes(const orc_machine *m);         /* count of TIA register writes */

/* ---- arithmetic hooks used by the exhaustive ADC/SBC test ---- */
/* p: processor flags in (C bit 0, D bit 3); returns (a' | p' << 8) */
uint32_t orc_alu_adc(uint8_t a, uint8_t b, uint8_t p);
uint32_t orc_alu_sbc(uint8_t a, uint8_t b, uint8_t p);
/* documented base cycle count of an opcode (0 for undocumented) */
int orc_base_cycles(uint8_t opcode);

/* ---- Philox4x32-10 (Salmon et al., SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- environments ---- */
typedef struct {
    int frameskip;       /* >= 2; frames F-1 and F are rendered */
    int sticky;          /* 1: repeat the previous action with p = 1/4 per frame */
    int n_cache;         /* cached start states per ROM (30) */
    int startup_frames;  /* 64 */
    int max_noops;       /* 30 */
    int output_mode;     /* 0: palette frame of frame F (210x160); 1: 84x84x4 luma stack */
    uint64_t seed;
} orc_config;

orc_envs *orc_envs_create(const uint8_t *const *roms, const size_t *rom_sizes,
                          const uint8_t *score_addr, const uint8_t *gameover_addr, int n_roms,
                          const int32_t *env_rom, const uint32_t *env_key /* NULL: index */,
                          int n_envs, const orc_config *cfg, const uint8_t *luma128);
void orc_envs_free(orc_envs *e);
/* One step of every env.  obs: mode 0 -> n*210*160, mode 1 -> n*4*84*84. */
int orc_envs_step(orc_envs *e, const uint8_t *actions, uint8_t *obs, int32_t *rewards,
                  uint8_t *dones, int n_threads);
void orc_envs_get_state(const orc_envs *e, uint8_t *out /* n*256 */);
void orc_envs_set_state(orc_envs *e, const uint8_t *in /* n*256 */);
void orc_envs_get_frames(const orc_envs *e, uint8_t *out /* n*2*210*160: frames F-1, F */);
void orc_envs_get_cache(const orc_envs *e, uint8_t *out /* n_roms*n_cache*256 */);
void orc_envs_reset(orc_envs *e, const uint8_t *mask /* NULL: all */);
uint64_t orc_envs_instructions(const orc_envs *e); /* 6502 instructions retired (all envs) */

/* ---- inference-path policy (linear softmax on the 84x84x4 stack) ---- */
#define ORC_POLICY_K 28224
#define ORC_POLICY_A 18
/* exp by Cody-Waite range reduction and a degree-7 polynomial, fp32, fmaf */
float orc_exp_own(float x);
/* logits of one stack: canonical order (441 chunks of 64 sequential fmaf,
 * chunk partials reduced by a strided-halving tree over 512 slots) */
void orc_policy_logits(const uint8_t *stack, const uint16_t *w_bf16, float *logits18);
/* action from logits and a 32-bit uniform word x: smallest j with
 * cumsum(exp_own(l - max)) > ((x >> 8) 2^-24) * sum, else the last j with
 * nonzero weight */
int orc_policy_sample(const float *logits18, uint32_t u);
/* for every env: logits from obs (n x 28224), draw from the env's Philox
 * stream (env key, step, 4 << 8, episode), action out */
void orc_envs_policy(const orc_envs *e, const uint8_t *obs, const uint16_t *w_bf16, uint8_t *actions,
                     float *logits, int n_threads);

/* behaviour probability of action a under the softmax of logits18 (fp32,
 * weights and total as in orc_policy_sample) */
float orc_policy_prob(const float *logits18, int a);
/* mu[i] = orc_policy_prob(logits[i], actions[i]) for n envs */
void orc_envs_policy_mu(int n, const float *logits, const uint8_t *actions, float *mu);

/* ---- learner-side targets over a rollout (Appendix: A2C, V-trace) ----
 * Time-major [T][n] arrays; values [T+1][n] (row T: bootstrap value);
 * double-precision outputs [T][n]; a done at step t ends the return there. */
void orc_nstep_returns(int T, int n, const float *rewards, const uint8_t *dones, const float *values,
                       double gamma, double *returns);
void orc_vtrace(int T, int n, const float *rewards, const uint8_t *dones, const float *values, const float *pi,
                const float *mu, double gamma, double rho_bar, double c_bar, double *vs, double *pg_adv);

/* ---- preprocessing of one env-step (exposed for the downsample pins) ---- */
void orc_preprocess(const uint8_t *f3, const uint8_t *f4, const uint8_t *luma128,
                    uint8_t *out84x84);

#ifdef __cplusplus
}
#endif
#endif
