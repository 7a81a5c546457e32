// Host scheduling core of the serving loop (see serve_sched.h).
#include "serve_sched.h"

#include <algorithm>

namespace atari_serve {

Scheduler::Scheduler(const SchedConfig &c) : cfg_(c) {
  free_.reserve((size_t)c.capacity);
  for (int s = c.capacity - 1; s >= 0; --s) free_.push_back(s);  // pop order: ascending slots
}

bool Scheduler::fits(int n) const {
  return n <= (int)free_.size() && bytes_in_use() + (uint64_t)n * cfg_.per_env_bytes <= cfg_.budget_bytes;
}

void Scheduler::admit(int sid, int64_t now) {
  Session &s = sessions_[(size_t)sid];
  s.slots.resize((size_t)s.n);
  for (int j = 0; j < s.n; ++j) {
    s.slots[(size_t)j] = free_.back();
    free_.pop_back();
  }
  used_envs_ += s.n;
  s.state = SESSION_ADMITTED;
  s.needs_init = true;
  s.last = now;
  ++admitted_total_;
}

void Scheduler::admit_queued(int64_t now) {
  while (!admit_q_.empty()) {
    const int sid = admit_q_.front();
    if (sessions_[(size_t)sid].state != SESSION_QUEUED) {  // closed while queued
      admit_q_.pop_front();
      continue;
    }
    if (!fits(sessions_[(size_t)sid].n)) break;  // strict FIFO: nothing overtakes the head
    admit_q_.pop_front();
    admit(sid, now);
  }
}

int Scheduler::open(int rom, int n, uint32_t key_base, int64_t now) {
  if (rom < 0 || rom >= cfg_.n_roms || n < 1 || n > cfg_.max_session_envs || n > cfg_.capacity) return E_INVAL;
  if (cfg_.fixed_bytes + (uint64_t)n * cfg_.per_env_bytes > cfg_.budget_bytes) return E_NOMEM;  // never fits
  Session s;
  s.rom = rom;
  s.n = n;
  s.key_base = key_base;
  s.state = SESSION_QUEUED;
  s.last = now;
  sessions_.push_back(std::move(s));
  const int sid = (int)sessions_.size() - 1;
  if (admit_q_.empty() && fits(n)) admit(sid, now);
  else admit_q_.push_back(sid);
  return sid;
}

SessionState Scheduler::state(int sid) const {
  if (sid < 0 || sid >= (int)sessions_.size()) return SESSION_CLOSED;
  return sessions_[(size_t)sid].state;
}

const Session *Scheduler::session(int sid) const {
  if (sid < 0 || sid >= (int)sessions_.size()) return nullptr;
  return &sessions_[(size_t)sid];
}

int Scheduler::close(int sid, int64_t now) {
  if (sid < 0 || sid >= (int)sessions_.size()) return E_NOSESSION;
  Session &s = sessions_[(size_t)sid];
  if (s.state == SESSION_CLOSED) return E_NOSESSION;
  if (s.busy) return E_BUSY;
  if (s.state == SESSION_ADMITTED) {
    for (int32_t slot : s.slots) free_.push_back(slot);
    used_envs_ -= s.n;
    s.slots.clear();
    s.slots.shrink_to_fit();
  }
  s.state = SESSION_CLOSED;
  admit_queued(now);
  return 0;
}

int Scheduler::enqueue(Request *r, int64_t now) {
  if (!r || r->sid < 0 || r->sid >= (int)sessions_.size()) return E_NOSESSION;
  Session &s = sessions_[(size_t)r->sid];
  if (s.state != SESSION_ADMITTED) return E_NOSESSION;
  if (s.busy) return E_BUSY;
  s.busy = true;
  s.last = now;
  r->n = s.n;
  r->t_submit = now;
  r->launched = r->finished = false;
  r->status = 0;
  pending_.push_back(r);
  return 0;
}

bool Scheduler::withdraw(Request *r) {
  auto it = std::find(pending_.begin(), pending_.end(), r);
  if (it == pending_.end()) return false;
  pending_.erase(it);
  sessions_[(size_t)r->sid].busy = false;
  return true;
}

bool Scheduler::plan_tick(TickPlan &t, int64_t now) {
  t.clear();
  if (pending_.empty()) return false;
  int total = 0;
  while (!pending_.empty()) {
    Request *r = pending_.front();
    if (!t.reqs.empty() && total + r->n > cfg_.max_tick_envs) break;
    pending_.pop_front();
    r->out_offset = total;
    r->launched = true;
    r->t_launch = now;
    total += r->n;
    t.reqs.push_back(r);
  }
  t.n_active = total;
  for (Request *r : t.reqs) r->tick_envs = total;
  // work list: cartridge by cartridge, requests in FIFO order within one,
  // cut into items of at most lanes * warps envs
  const int per = std::max(1, cfg_.lanes * cfg_.warps);
  std::vector<int32_t> g_rom, g_start, g_count, perm, opos;
  perm.reserve((size_t)total);
  opos.reserve((size_t)total);
  std::vector<std::vector<int>> by_rom((size_t)cfg_.n_roms);
  for (int q = 0; q < (int)t.reqs.size(); ++q) by_rom[(size_t)sessions_[(size_t)t.reqs[(size_t)q]->sid].rom].push_back(q);
  for (int rom = 0; rom < cfg_.n_roms; ++rom) {
    const int first = (int)perm.size();
    for (int q : by_rom[(size_t)rom]) {
      const Request *r = t.reqs[(size_t)q];
      const Session &s = sessions_[(size_t)r->sid];
      for (int j = 0; j < s.n; ++j) {
        perm.push_back(s.slots[(size_t)j]);
        opos.push_back(r->out_offset + j);
      }
    }
    for (int st = first; st < (int)perm.size(); st += per) {
      g_rom.push_back(rom);
      g_start.push_back(st);
      g_count.push_back(std::min(per, (int)perm.size() - st));
    }
  }
  t.n_groups = (int)g_rom.size();
  t.blob.reserve((size_t)3 * t.n_groups + 2 * (size_t)total);
  t.blob.insert(t.blob.end(), g_rom.begin(), g_rom.end());
  t.blob.insert(t.blob.end(), g_start.begin(), g_start.end());
  t.blob.insert(t.blob.end(), g_count.begin(), g_count.end());
  t.blob.insert(t.blob.end(), perm.begin(), perm.end());
  t.blob.insert(t.blob.end(), opos.begin(), opos.end());
  // first steps of newly admitted sessions start from a cached state
  std::vector<int32_t> i_slot, i_rom, i_key;
  for (Request *r : t.reqs) {
    Session &s = sessions_[(size_t)r->sid];
    if (!s.needs_init) continue;
    s.needs_init = false;
    for (int j = 0; j < s.n; ++j) {
      i_slot.push_back(s.slots[(size_t)j]);
      i_rom.push_back(s.rom);
      i_key.push_back((int32_t)(s.key_base + (uint32_t)j));
    }
  }
  t.n_init = (int)i_slot.size();
  t.init.insert(t.init.end(), i_slot.begin(), i_slot.end());
  t.init.insert(t.init.end(), i_rom.begin(), i_rom.end());
  t.init.insert(t.init.end(), i_key.begin(), i_key.end());
  t.actions.resize((size_t)total);
  for (Request *r : t.reqs) std::copy(r->actions, r->actions + r->n, t.actions.begin() + r->out_offset);
  return true;
}

void Scheduler::finish_tick(const TickPlan &t, int64_t now) {
  for (Request *r : t.reqs) {
    Session &s = sessions_[(size_t)r->sid];
    s.busy = false;
    s.last = now;
  }
}

std::vector<int> Scheduler::reclaim_idle(int64_t now) {
  std::vector<int> out;
  if (cfg_.idle_timeout_ns <= 0) return out;
  for (int sid = 0; sid < (int)sessions_.size(); ++sid) {
    const Session &s = sessions_[(size_t)sid];
    if (s.state == SESSION_ADMITTED && !s.busy && now - s.last > cfg_.idle_timeout_ns) {
      close(sid, now);
      out.push_back(sid);
    }
  }
  return out;
}

}  // namespace atari_serve
