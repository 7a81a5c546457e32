// Library-internal interface between the emulator's translation unit
// (atari_gpu.cu: kernels, env state) and the serving loop (server.cu).  Not
// exported from the shared library.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/atari_gpu.h"

namespace atari_internal {

// One serving tick on an env used as a pool of slots (batched form, stack
// output).  Device arrays, all written by the host for this tick:
//   d_blob = grp_rom[n_groups], grp_start[n_groups], grp_count[n_groups],
//            perm[n_active] (slot per work-list entry),
//            opos[n_active] (packed output position per work-list entry);
//   d_init = slots[n_init], roms[n_init], keys[n_init]: slots that start a new
//            session, set to episode 0 from the start-state cache first.
// Packed buffers are indexed by output position: d_actions[n_active],
// d_obs[n_active][4][84][84] (may be null), d_rew[n_active], d_done[n_active].
// d_queue is the tick's own work-item counter (zeroed here).
struct ServeTick {
  const int32_t *d_blob = nullptr;
  int n_groups = 0, n_active = 0;
  const int32_t *d_init = nullptr;
  int n_init = 0;
  const uint8_t *d_actions = nullptr;
  uint8_t *d_obs = nullptr;
  int32_t *d_rew = nullptr;
  uint8_t *d_done = nullptr;
  int *d_queue = nullptr;
};

int env_slots(const atari_env *E);
int env_device(const atari_env *E);
int env_n_roms(const atari_env *E);
int env_frameskip(const atari_env *E);
void env_shape(const atari_env *E, int *lanes, int *warps);
// Enqueue the tick on stream s (no host synchronisation).
int serve_tick(atari_env *E, const ServeTick &t, cudaStream_t s);
// Record an error message for atari_last_error() on the calling thread.
int set_error(int code, const std::string &msg);

}  // namespace atari_internal
