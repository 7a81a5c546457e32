// Host scheduling core of the serving loop: sessions, admission by a device
// memory budget, the FIFO of pending step requests and the packing of the
// requests taken by one tick into a ROM-grouped work list.  Plain C++17 with
// no CUDA dependency; the server (server.cu) wraps it with a mutex and runs
// each planned tick on the GPU.
//
// A session is n envs of one cartridge, keyed key_base + j (j < n) for the
// env-local random streams (sticky actions, reset draws), so a session's
// results depend only on its cartridge, its keys and its actions: never on
// which slots it holds or on what else runs in the same tick.
#pragma once
#include <cstddef>
#include <cstdint>
#include <deque>
#include <vector>

namespace atari_serve {

struct SchedConfig {
  uint64_t budget_bytes = 0;   // admission budget for everything the server holds on the device
  uint64_t fixed_bytes = 0;    // part of the budget taken whatever is admitted (cartridges, cache, tick buffers)
  uint64_t per_env_bytes = 0;  // device bytes one resident env holds
  int capacity = 0;            // env slots allocated on the device
  int max_tick_envs = 0;       // envs one tick may carry
  int max_session_envs = 0;    // largest session accepted
  int n_roms = 0;
  int lanes = 32, warps = 4;   // work item = up to lanes * warps envs of one cartridge
  int64_t idle_timeout_ns = 0; // admitted sessions idle this long are closed (0: never)
};

enum SessionState { SESSION_QUEUED = 0, SESSION_ADMITTED = 1, SESSION_CLOSED = 2 };

struct Request {
  int sid = -1;
  const uint8_t *actions = nullptr;  // host, n bytes
  uint8_t *obs = nullptr;            // host outputs; obs may be null
  int32_t *rew = nullptr;
  uint8_t *done = nullptr;
  int64_t t_submit = 0, t_launch = 0, t_done = 0;
  int n = 0;
  int out_offset = 0;                // first packed output position in its tick
  int tick_envs = 0;                 // envs carried by that tick
  int status = 0;
  bool launched = false, finished = false;
};

struct Session {
  int rom = 0, n = 0;
  uint32_t key_base = 0;
  SessionState state = SESSION_QUEUED;
  std::vector<int32_t> slots;
  bool needs_init = false, busy = false;
  int64_t last = 0;
};

// One tick: the requests it carries and everything the device needs for it.
// blob = grp_rom[n_groups], grp_start[n_groups], grp_count[n_groups],
//        perm[n_active] (slot of each work-list position),
//        opos[n_active] (packed output position of each work-list position).
// init = slots[n_init], roms[n_init], keys[n_init]: envs stepped for the first
// time, which start from a cached state (episode 0) before the step.
struct TickPlan {
  std::vector<Request *> reqs;
  std::vector<int32_t> blob;
  std::vector<int32_t> init;
  std::vector<uint8_t> actions;  // packed, by output position
  int n_groups = 0, n_active = 0, n_init = 0;
  void clear() {
    reqs.clear();
    blob.clear();
    init.clear();
    actions.clear();
    n_groups = n_active = n_init = 0;
  }
};

// error codes shared with the C ABI
constexpr int E_INVAL = -22, E_NOMEM = -12, E_BUSY = -16, E_NOSESSION = -3;

class Scheduler {
 public:
  explicit Scheduler(const SchedConfig &c);
  const SchedConfig &config() const { return cfg_; }

  // New session; returns its id (>= 0) or a negative error.  It is admitted
  // at once when nothing is queued ahead of it and it fits the budget and
  // the free slots; otherwise it waits in FIFO order.
  int open(int rom, int n, uint32_t key_base, int64_t now);
  SessionState state(int sid) const;
  const Session *session(int sid) const;
  // Close a session (admitted or queued): frees its slots, then admits queued
  // sessions in FIFO order while the head fits.  E_BUSY while a request of it
  // is in flight.
  int close(int sid, int64_t now);
  // Queue a step request of an admitted, idle session.
  int enqueue(Request *r, int64_t now);
  // Take back a request not yet planned into a tick.
  bool withdraw(Request *r);
  // Plan the next tick from the pending FIFO (up to max_tick_envs envs, at
  // least one request); false when nothing is pending.
  bool plan_tick(TickPlan &t, int64_t now);
  // After the tick's results are delivered: its sessions take requests again.
  void finish_tick(const TickPlan &t, int64_t now);
  // Close admitted, idle sessions whose last activity is older than the
  // idle timeout; returns their ids.
  std::vector<int> reclaim_idle(int64_t now);

  uint64_t bytes_in_use() const { return cfg_.fixed_bytes + (uint64_t)used_envs_ * cfg_.per_env_bytes; }
  int free_slots() const { return (int)free_.size(); }
  int queued_sessions() const { return (int)admit_q_.size(); }
  int pending_requests() const { return (int)pending_.size(); }
  uint64_t admitted_total() const { return admitted_total_; }

 private:
  bool fits(int n) const;
  void admit(int sid, int64_t now);
  void admit_queued(int64_t now);

  SchedConfig cfg_;
  std::vector<Session> sessions_;
  std::vector<int32_t> free_;     // free slots, popped from the back
  std::deque<int> admit_q_;       // queued session ids, FIFO
  std::deque<Request *> pending_; // step requests, FIFO
  int used_envs_ = 0;
  uint64_t admitted_total_ = 0;
};

}  // namespace atari_serve
