// Serving loop over the batched emulator: continuous batching of per-session
// step requests with admission by a device-memory budget (include/atari_server.h).
//
// Threads:
//   clients    atari_server_open / step / close: queue work, wait on cv_cli;
//   launcher   takes the pending FIFO into a tick whenever a tick context
//              is free: packs the work list (serve_sched.cpp), one H2D copy,
//              the tick's kernels and the D2H copies on the context's stream;
//   completer  waits for launched ticks in order, hands rewards/dones (and
//              pageable stacks) to their requests, frees the context.
// With `inflight` contexts, up to that many ticks overlap on the device
// (different streams, disjoint sessions).  A session has at most one request
// in flight, and its next request is only queued after the previous reply
// was delivered, i.e. after that tick's stream work completed.  So ticks
// never race on a slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "../../include/atari_server.h"
#include "env_internal.h"
#include "serve_sched.h"

using atari_internal::set_error;
using namespace atari_serve;

namespace {

constexpr size_t STACK_BYTES = 4 * 7056;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-tick input buffer layout (host pinned and device alike):
// blob ints (3 * groups + 2 * envs), init ints (3 * envs), actions (envs).
struct InLayout {
  size_t blob_off, init_off, act_off, bytes;
  InLayout(int tick_envs, int n_roms) {
    const size_t T = (size_t)tick_envs, R = (size_t)n_roms;
    blob_off = 0;
    init_off = align_up(4 * (3 * (T + R) + 2 * T), 256);
    act_off = init_off + align_up(4 * 3 * T, 256);
    bytes = act_off + align_up(T, 256);
  }
};

size_t tick_device_bytes(int tick_envs, int n_roms) {
  InLayout L(tick_envs, n_roms);
  const size_t T = (size_t)tick_envs;
  return L.bytes + align_up(T * STACK_BYTES, 256) + align_up(5 * T, 256) + 256;
}

#define SRV_CUDA(expr, code_on_fail)                                                             \
  do {                                                                                           \
    cudaError_t e__ = (expr);                                                                    \
    if (e__ != cudaSuccess) return set_error(code_on_fail, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
  } while (0)

struct TickCtx {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t t_begin = nullptr, t_end = nullptr;  // timing events around the tick's device work
  uint8_t *h_in = nullptr, *h_out = nullptr;   // pinned
  uint8_t *d_in = nullptr, *d_obs = nullptr, *d_out = nullptr;
  int *d_queue = nullptr;
  TickPlan plan;
  std::vector<Request *> pageable;             // requests whose stacks are copied after completion
};

}  // namespace

struct atari_server {
  atari_env *env = nullptr;
  int device = 0, n_roms = 0, tick_cap = 0, inflight = 2;
  std::unique_ptr<Scheduler> sched;
  std::vector<TickCtx> ctx;
  std::mutex mu;
  std::condition_variable cv_srv, cv_done, cv_cli;
  std::deque<int> free_ctx, launched;
  std::thread launcher, completer;
  bool stop = false, stop_completer = false;
  int fatal = 0;
  std::string fatal_msg;
  uint64_t ticks = 0, requests = 0, env_steps = 0, launches = 0;
  uint64_t tick_env_sum = 0;
  // device overlap of ticks: times (ms after t_ref) of the tick ends seen so far
  cudaEvent_t t_ref = nullptr;
  double last_end_ms = -1.0;
  uint64_t overlapped_ticks = 0;
};

namespace {

void fail_all_locked(atari_server *S, int code, const std::string &msg) {
  if (!S->fatal) {
    S->fatal = code;
    S->fatal_msg = msg;
  }
  S->cv_cli.notify_all();
  S->cv_srv.notify_all();
  S->cv_done.notify_all();
}

// Enqueue one planned tick on its context's stream.
int launch_tick(atari_server *S, TickCtx &c) {
  const TickPlan &p = c.plan;
  InLayout L(S->tick_cap, S->n_roms);
  std::memcpy(c.h_in + L.blob_off, p.blob.data(), p.blob.size() * 4);
  std::memcpy(c.h_in + L.init_off, p.init.data(), p.init.size() * 4);
  std::memcpy(c.h_in + L.act_off, p.actions.data(), p.actions.size());
  const size_t in_bytes = L.act_off + (size_t)p.n_active;
  SRV_CUDA(cudaEventRecord(c.t_begin, c.stream), ATARI_ECUDA);
  SRV_CUDA(cudaMemcpyAsync(c.d_in, c.h_in, in_bytes, cudaMemcpyHostToDevice, c.stream), ATARI_ECUDA);
  atari_internal::ServeTick t;
  t.d_blob = reinterpret_cast<const int32_t *>(c.d_in + L.blob_off);
  t.n_groups = p.n_groups;
  t.n_active = p.n_active;
  t.d_init = reinterpret_cast<const int32_t *>(c.d_in + L.init_off);
  t.n_init = p.n_init;
  t.d_actions = c.d_in + L.act_off;
  t.d_obs = c.d_obs;
  t.d_rew = reinterpret_cast<int32_t *>(c.d_out);
  t.d_done = c.d_out + 4 * (size_t)p.n_active;
  t.d_queue = c.d_queue;
  if (int rc = atari_internal::serve_tick(S->env, t, c.stream)) return rc;
  SRV_CUDA(cudaMemcpyAsync(c.h_out, c.d_out, 5 * (size_t)p.n_active, cudaMemcpyDeviceToHost, c.stream), ATARI_ECUDA);
  c.pageable.clear();
  for (Request *r : p.reqs) {
    if (!r->obs) continue;
    cudaPointerAttributes pa{};
    const bool pinned = cudaPointerGetAttributes(&pa, r->obs) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();  // an unregistered pointer may leave an error behind on older runtimes
    if (pinned) {
      SRV_CUDA(cudaMemcpyAsync(r->obs, c.d_obs + (size_t)r->out_offset * STACK_BYTES, (size_t)r->n * STACK_BYTES,
                               cudaMemcpyDeviceToHost, c.stream),
               ATARI_ECUDA);
    } else {
      c.pageable.push_back(r);
    }
  }
  SRV_CUDA(cudaEventRecord(c.t_end, c.stream), ATARI_ECUDA);
  SRV_CUDA(cudaEventRecord(c.done, c.stream), ATARI_ECUDA);
  return 0;
}

void launcher_main(atari_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  int64_t last_reclaim = now_ns();
  while (!S->stop && !S->fatal) {
    const int64_t now = now_ns();
    if (S->sched->config().idle_timeout_ns > 0 && now - last_reclaim > 20'000'000) {
      if (!S->sched->reclaim_idle(now).empty()) S->cv_cli.notify_all();
      last_reclaim = now;
    }
    if (S->free_ctx.empty() || S->sched->pending_requests() == 0) {
      S->cv_srv.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    const int k = S->free_ctx.front();
    S->free_ctx.pop_front();
    TickCtx &c = S->ctx[(size_t)k];
    S->sched->plan_tick(c.plan, now);
    lk.unlock();
    const int rc = launch_tick(S, c);
    const std::string msg = rc ? std::string(atari_last_error()) : std::string();
    lk.lock();
    if (rc) {
      // the planned requests are failed by the completer once the stream drains
      fail_all_locked(S, rc, "serving tick launch: " + msg);
    }
    S->launched.push_back(k);
    S->cv_done.notify_one();
  }
}

void completer_main(atari_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_done.wait(lk, [&] { return !S->launched.empty() || S->stop_completer; });
    if (S->launched.empty()) break;  // launcher joined and nothing left in flight
    const int k = S->launched.front();
    TickCtx &c = S->ctx[(size_t)k];
    lk.unlock();
    int status = 0;
    std::string msg;
    cudaError_t e = cudaEventSynchronize(c.done);
    if (e != cudaSuccess) {
      status = ATARI_ECUDA;
      msg = std::string("serving tick: ") + cudaGetErrorString(e);
    }
    const TickPlan &p = c.plan;
    // where the tick ran on the device, in ms after the server's reference event
    float t_b = 0.0f, t_e = 0.0f;
    const bool timed = !status && cudaEventElapsedTime(&t_b, S->t_ref, c.t_begin) == cudaSuccess &&
                       cudaEventElapsedTime(&t_e, S->t_ref, c.t_end) == cudaSuccess;
    if (!status) {
      const int32_t *rew = reinterpret_cast<const int32_t *>(c.h_out);
      const uint8_t *done = c.h_out + 4 * (size_t)p.n_active;
      for (Request *r : p.reqs) {
        std::memcpy(r->rew, rew + r->out_offset, (size_t)r->n * 4);
        std::memcpy(r->done, done + r->out_offset, (size_t)r->n);
      }
      for (Request *r : c.pageable) {
        e = cudaMemcpy(r->obs, c.d_obs + (size_t)r->out_offset * STACK_BYTES, (size_t)r->n * STACK_BYTES,
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
          status = ATARI_ECUDA;
          msg = std::string("serving tick copy: ") + cudaGetErrorString(e);
          break;
        }
      }
    }
    const int64_t t = now_ns();
    lk.lock();
    S->launched.pop_front();
    if (status) fail_all_locked(S, status, msg);
    const int st = status ? status : S->fatal;
    for (Request *r : p.reqs) {
      r->status = st;
      r->t_done = t;
      r->finished = true;
    }
    S->sched->finish_tick(p, t);
    if (timed) {
      // ticks complete in launch order: this one overlapped an earlier one on
      // the device when it began before the latest earlier end
      if (S->last_end_ms >= 0.0 && (double)t_b < S->last_end_ms) S->overlapped_ticks++;
      S->last_end_ms = std::max(S->last_end_ms, (double)t_e);
    }
    S->ticks++;
    S->launches += 2 + (p.n_init > 0 ? 1 : 0);
    S->requests += p.reqs.size();
    S->env_steps += (uint64_t)p.n_active;
    S->tick_env_sum += (uint64_t)p.n_active;
    S->free_ctx.push_back(k);
    S->cv_cli.notify_all();
    S->cv_srv.notify_one();
  }
}

void free_server(atari_server *S) {
  for (TickCtx &c : S->ctx) {
    if (c.stream) cudaStreamSynchronize(c.stream);
    if (c.done) cudaEventDestroy(c.done);
    if (c.t_begin) cudaEventDestroy(c.t_begin);
    if (c.t_end) cudaEventDestroy(c.t_end);
    if (c.stream) cudaStreamDestroy(c.stream);
    if (c.h_in) cudaFreeHost(c.h_in);
    if (c.h_out) cudaFreeHost(c.h_out);
    if (c.d_in) cudaFree(c.d_in);
    if (c.d_obs) cudaFree(c.d_obs);
    if (c.d_out) cudaFree(c.d_out);
    if (c.d_queue) cudaFree(c.d_queue);
  }
  if (S->t_ref) cudaEventDestroy(S->t_ref);
  if (S->env) atari_env_destroy(S->env);
  delete S;
}

uint64_t per_env_bytes(int n_roms, const atari_config *cfg) {
  return (uint64_t)(atari_env_footprint(1, n_roms, cfg) - atari_env_footprint(0, n_roms, cfg));
}

atari_server_config resolved(const atari_server_config *in) {
  atari_server_config c;
  atari_server_default_config(&c);
  if (in) c = *in;
  if (c.max_session_envs <= 0) c.max_session_envs = 2048;
  if (c.inflight <= 0) c.inflight = 2;
  return c;
}

}  // namespace

extern "C" {

void atari_server_default_config(atari_server_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->budget_bytes = 40ull << 30;
  c->max_session_envs = 2048;
  c->inflight = 2;
}

size_t atari_server_footprint(int slots, int tick_envs, int n_roms, const atari_config *cfg,
                              const atari_server_config *scfg) {
  if (!cfg || slots < 0 || tick_envs < 0 || n_roms < 0) return 0;
  const atari_server_config c = resolved(scfg);
  return atari_env_footprint(slots, n_roms, cfg) + (size_t)c.inflight * tick_device_bytes(tick_envs, n_roms);
}

int atari_server_create(const uint8_t *const *roms, const size_t *rom_sizes, const atari_rom_meta *meta, int n_roms,
                        const atari_config *cfg, const uint8_t *luma, const atari_server_config *scfg,
                        atari_server **out) {
  if (!out) return set_error(ATARI_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return set_error(ATARI_EINVAL, "cfg is NULL");
  if (cfg->form != ATARI_FORM_BATCHED || cfg->output_mode != ATARI_OUT_STACK)
    return set_error(ATARI_EINVAL, "the server needs form ATARI_FORM_BATCHED and output ATARI_OUT_STACK");
  if (n_roms <= 0 || n_roms > 65535) return set_error(ATARI_EINVAL, "bad ROM list");
  const atari_server_config sc = resolved(scfg);
  if (sc.inflight < 1 || sc.inflight > 4) return set_error(ATARI_EINVAL, "inflight must be 1..4");
  if (sc.max_slots < 0 || sc.max_tick_envs < 0 || sc.idle_timeout_ms < 0)
    return set_error(ATARI_EINVAL, "negative server limit");
  // largest slot count whose footprint (tick buffers sized for as many envs
  // as slots, unless capped) fits the budget
  auto fits = [&](int s) {
    const int t = sc.max_tick_envs > 0 ? std::min(sc.max_tick_envs, s) : s;
    return atari_server_footprint(s, t, n_roms, cfg, &sc) <= sc.budget_bytes;
  };
  int hi = sc.max_slots > 0 ? sc.max_slots : (1 << 24), lo = 0;
  if (fits(hi)) lo = hi;
  while (lo < hi) {
    const int mid = lo + (hi - lo + 1) / 2;
    if (fits(mid)) lo = mid;
    else hi = mid - 1;
  }
  const int slots = lo;
  if (slots < 1) return set_error(ATARI_ENOMEM, "the budget does not hold one env slot");
  const int tick_cap = sc.max_tick_envs > 0 ? std::min(sc.max_tick_envs, slots) : slots;

  atari_config ec = *cfg;
  if (ec.envs_per_warp <= 0 || ec.envs_per_block <= 0) {
    ec.envs_per_warp = 32;
    ec.envs_per_block = 128;
  }
  std::vector<int32_t> env_rom((size_t)slots, 0);
  std::vector<uint32_t> env_key((size_t)slots);
  for (int s = 0; s < slots; ++s) env_key[(size_t)s] = (uint32_t)s;
  auto *S = new atari_server();
  if (int rc = atari_env_create(roms, rom_sizes, meta, n_roms, env_rom.data(), env_key.data(), slots, &ec, luma,
                                &S->env)) {
    delete S;
    return rc;
  }
  S->device = atari_internal::env_device(S->env);
  S->n_roms = n_roms;
  S->tick_cap = tick_cap;
  S->inflight = sc.inflight;
  SchedConfig k;
  k.budget_bytes = sc.budget_bytes;
  k.per_env_bytes = per_env_bytes(n_roms, cfg);
  k.fixed_bytes = atari_server_footprint(slots, tick_cap, n_roms, cfg, &sc) - (uint64_t)slots * k.per_env_bytes;
  k.capacity = slots;
  k.max_tick_envs = tick_cap;
  k.max_session_envs = std::min(sc.max_session_envs, tick_cap);
  k.n_roms = n_roms;
  atari_internal::env_shape(S->env, &k.lanes, &k.warps);
  k.idle_timeout_ns = (int64_t)sc.idle_timeout_ms * 1000000;
  S->sched.reset(new Scheduler(k));
  InLayout L(tick_cap, n_roms);
  S->ctx.resize((size_t)sc.inflight);
  for (int i = 0; i < sc.inflight; ++i) {
    TickCtx &c = S->ctx[(size_t)i];
    cudaError_t e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming | cudaEventBlockingSync);
    if (e == cudaSuccess) e = cudaEventCreate(&c.t_begin);
    if (e == cudaSuccess) e = cudaEventCreate(&c.t_end);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c.h_in, L.bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c.h_out, align_up(5 * (size_t)tick_cap, 256), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_in, L.bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c.d_obs, align_up((size_t)tick_cap * STACK_BYTES, 256));
    if (e == cudaSuccess) e = cudaMalloc(&c.d_out, align_up(5 * (size_t)tick_cap, 256));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c.d_queue, 256);
    if (e != cudaSuccess) {
      const int code = (e == cudaErrorMemoryAllocation) ? ATARI_ENOMEM : ATARI_ECUDA;
      free_server(S);
      return set_error(code, std::string("server tick buffers: ") + cudaGetErrorString(e));
    }
    S->free_ctx.push_back(i);
  }
  {
    cudaError_t e = cudaEventCreate(&S->t_ref);
    if (e == cudaSuccess) e = cudaEventRecord(S->t_ref, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(S->t_ref);
    if (e != cudaSuccess) {
      free_server(S);
      return set_error(ATARI_ECUDA, std::string("server timing event: ") + cudaGetErrorString(e));
    }
  }
  S->launcher = std::thread(launcher_main, S);
  S->completer = std::thread(completer_main, S);
  *out = S;
  return 0;
}

int atari_server_open(atari_server *S, int rom, int n_envs, uint32_t key_base, int timeout_ms, int *session) {
  if (!S || !session) return set_error(ATARI_EINVAL, "server or session pointer is NULL");
  *session = -1;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->fatal) return set_error(S->fatal, S->fatal_msg);
  const int sid = S->sched->open(rom, n_envs, key_base, now_ns());
  if (sid < 0)
    return set_error(sid, sid == ATARI_ENOMEM ? "session larger than the device budget"
                                              : "bad cartridge index or session size");
  auto admitted = [&] { return S->sched->state(sid) != SESSION_QUEUED || S->fatal || S->stop; };
  if (timeout_ms < 0) {
    S->cv_cli.wait(lk, admitted);
  } else if (!S->cv_cli.wait_for(lk, std::chrono::milliseconds(timeout_ms), admitted)) {
    S->sched->close(sid, now_ns());
    return set_error(ATARI_EAGAIN, "session not admitted within the timeout");
  }
  if (S->fatal) return set_error(S->fatal, S->fatal_msg);
  if (S->sched->state(sid) != SESSION_ADMITTED) return set_error(ATARI_ESESSION, "server stopping");
  *session = sid;
  return 0;
}

int atari_server_step(atari_server *S, int session, const uint8_t *actions, uint8_t *obs, int32_t *rewards,
                      uint8_t *dones, atari_request_info *info) {
  if (!S || !actions || !rewards || !dones) return set_error(ATARI_EINVAL, "NULL argument");
  Request r;
  r.sid = session;
  r.actions = actions;
  r.obs = obs;
  r.rew = rewards;
  r.done = dones;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->fatal) return set_error(S->fatal, S->fatal_msg);
  if (int rc = S->sched->enqueue(&r, now_ns()))
    return set_error(rc, rc == ATARI_EBUSY ? "session already has a step in flight" : "no such open session");
  S->cv_srv.notify_one();
  S->cv_cli.wait(lk, [&] { return r.finished || (S->fatal && !r.launched) || (S->stop && !r.launched); });
  if (!r.finished) {  // failed or stopping before it was taken into a tick
    S->sched->withdraw(&r);
    return set_error(S->fatal ? S->fatal : ATARI_ESESSION, S->fatal ? S->fatal_msg : "server stopping");
  }
  if (info) {
    info->submit_ns = r.t_submit;
    info->launch_ns = r.t_launch;
    info->done_ns = r.t_done;
    info->tick_envs = r.tick_envs;
  }
  if (r.status) return set_error(r.status, S->fatal_msg);
  return 0;
}

int atari_server_close(atari_server *S, int session) {
  if (!S) return set_error(ATARI_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  const int rc = S->sched->close(session, now_ns());
  if (rc) return set_error(rc, rc == ATARI_EBUSY ? "session has a step in flight" : "no such open session");
  S->cv_cli.notify_all();
  return 0;
}

int atari_server_get_stats(atari_server *S, atari_server_stats *out) {
  if (!S || !out) return set_error(ATARI_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  const SchedConfig &k = S->sched->config();
  std::memset(out, 0, sizeof *out);
  out->ticks = S->ticks;
  out->requests = S->requests;
  out->env_steps = S->env_steps;
  out->sessions_admitted = S->sched->admitted_total();
  out->launches = S->launches;
  out->budget_bytes = k.budget_bytes;
  out->bytes_in_use = S->sched->bytes_in_use();
  out->fixed_bytes = k.fixed_bytes;
  out->per_env_bytes = k.per_env_bytes;
  out->capacity = k.capacity;
  out->free_slots = S->sched->free_slots();
  out->queued_sessions = S->sched->queued_sessions();
  out->pending_requests = S->sched->pending_requests();
  out->overlapped_ticks = S->overlapped_ticks;
  return 0;
}

void atari_server_destroy(atari_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_srv.notify_all();
    S->cv_done.notify_all();
    S->cv_cli.notify_all();
  }
  if (S->launcher.joinable()) S->launcher.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop_completer = true;
    S->cv_done.notify_all();
  }
  if (S->completer.joinable()) S->completer.join();
  free_server(S);
}

// ---------------------------------------------------------------------------
// Closed-loop load generator.

int atari_server_loadgen(atari_server *S, const atari_loadgen_config *c, atari_loadgen_result *out) {
  if (!S || !c || !out) return set_error(ATARI_EINVAL, "NULL argument");
  if (c->n_clients < 1 || c->n_clients > 1024 || c->seconds <= 0 || c->min_envs < 1 || c->max_envs < c->min_envs ||
      c->session_steps_mean < 1 || c->think_mean_ms < 0)
    return set_error(ATARI_EINVAL, "bad load generator configuration");
  std::memset(out, 0, sizeof *out);
  atari_server_stats s0;
  atari_server_get_stats(S, &s0);
  const int64_t t0 = now_ns();
  const int64_t deadline = t0 + (int64_t)(c->seconds * 1e9);
  std::atomic<uint32_t> next_key{1};
  std::atomic<int> err{0};
  struct ClientOut {
    std::vector<float> lat_ms, admit_ms;
    uint64_t env_steps = 0, sessions = 0, h2d = 0, d2h = 0;
  };
  std::vector<ClientOut> res((size_t)c->n_clients);
  const int n_roms = S->n_roms;
  auto client = [&](int id) {
    cudaSetDevice(S->device);
    ClientOut &o = res[(size_t)id];
    std::mt19937_64 rng(c->seed * 0x9E3779B97F4A7C15ull + (uint64_t)id);
    std::uniform_int_distribution<int> pick_rom(0, n_roms - 1), pick_n(c->min_envs, c->max_envs), pick_a(0, 17);
    std::geometric_distribution<int> pick_len(1.0 / c->session_steps_mean);
    std::exponential_distribution<double> think(c->think_mean_ms > 0 ? 1.0 / c->think_mean_ms : 1.0);
    const size_t cap = (size_t)c->max_envs;
    uint8_t *act = nullptr, *obs = nullptr, *done = nullptr;
    int32_t *rew = nullptr;
    cudaError_t e = cudaHostAlloc((void **)&act, cap, cudaHostAllocDefault);
    if (e == cudaSuccess && c->want_obs) e = cudaHostAlloc((void **)&obs, cap * STACK_BYTES, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&rew, cap * 4, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&done, cap, cudaHostAllocDefault);
    if (e != cudaSuccess) err = ATARI_ENOMEM;
    while (!err && now_ns() < deadline) {
      const int rom = pick_rom(rng), n = pick_n(rng);
      const int steps = 1 + pick_len(rng);
      const uint32_t key = next_key.fetch_add(1) * 2048u;
      int sid = -1;
      const int64_t ta = now_ns();
      int rc = atari_server_open(S, rom, n, key, -1, &sid);
      if (rc) {
        err = rc;
        break;
      }
      o.admit_ms.push_back((float)((now_ns() - ta) / 1e6));
      o.sessions++;
      for (int s = 0; s < steps && now_ns() < deadline; ++s) {
        for (int j = 0; j < n; ++j) act[j] = (uint8_t)pick_a(rng);
        atari_request_info info;
        rc = atari_server_step(S, sid, act, obs, rew, done, &info);
        if (rc) {
          err = rc;
          break;
        }
        o.lat_ms.push_back((float)((info.done_ns - info.submit_ns) / 1e6));
        o.env_steps += (uint64_t)n;
        o.h2d += (uint64_t)n;
        o.d2h += (uint64_t)n * (5 + (c->want_obs ? STACK_BYTES : 0));
        if (c->think_mean_ms > 0) std::this_thread::sleep_for(std::chrono::duration<double, std::milli>(think(rng)));
      }
      atari_server_close(S, sid);
    }
    if (act) cudaFreeHost(act);
    if (obs) cudaFreeHost(obs);
    if (rew) cudaFreeHost(rew);
    if (done) cudaFreeHost(done);
  };
  std::vector<std::thread> th;
  for (int i = 0; i < c->n_clients; ++i) th.emplace_back(client, i);
  for (auto &t : th) t.join();
  const double secs = (now_ns() - t0) / 1e9;
  if (err) return set_error(err, std::string("load generator: ") + atari_last_error());
  std::vector<float> lat, adm;
  for (auto &o : res) {
    lat.insert(lat.end(), o.lat_ms.begin(), o.lat_ms.end());
    adm.insert(adm.end(), o.admit_ms.begin(), o.admit_ms.end());
    out->env_steps += o.env_steps;
    out->sessions += o.sessions;
    out->h2d_bytes += o.h2d;
    out->d2h_bytes += o.d2h;
  }
  auto pct = [](std::vector<float> &v, double q) -> double {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t k = (size_t)std::min<double>((double)v.size() - 1, std::round(q * ((double)v.size() - 1)));
    return v[k];
  };
  out->requests = lat.size();
  out->seconds = secs;
  atari_server_stats s1;
  atari_server_get_stats(S, &s1);
  out->frames = out->env_steps * (uint64_t)atari_internal::env_frameskip(S->env);
  out->frames_per_s = (double)out->frames / secs;
  double sum = 0.0;
  for (float v : lat) sum += v;
  out->mean_ms = lat.empty() ? 0.0 : sum / (double)lat.size();
  out->p50_ms = pct(lat, 0.50);
  out->p99_ms = pct(lat, 0.99);
  out->max_ms = lat.empty() ? 0.0 : lat.back();
  out->admit_p50_ms = pct(adm, 0.50);
  out->admit_p99_ms = pct(adm, 0.99);
  out->ticks = s1.ticks - s0.ticks;
  out->mean_tick_envs = out->ticks ? (double)(s1.env_steps - s0.env_steps) / (double)out->ticks : 0.0;
  return 0;
}

}  // extern "C"
