// Host checks of the serving loop's scheduling core (no GPU): admission by
// budget and free slots in FIFO order, the packing of a tick's requests into
// a cartridge-grouped work list, busy rules, idle reclaim, and slot
// accounting over long random open/step/close sequences.  Prints "ok" and
// exits 0, or names the first failed check and exits 1.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <set>
#include <vector>

#include "serve_sched.h"

using namespace atari_serve;

static int g_fail = 0;
#define CHECK(c)                                                      \
  do {                                                                \
    if (!(c)) {                                                       \
      std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #c);        \
      std::exit(1);                                                   \
    }                                                                 \
  } while (0)

static SchedConfig base(int capacity, int budget_envs) {
  SchedConfig c;
  c.per_env_bytes = 1000;
  c.fixed_bytes = 5000;
  c.budget_bytes = c.fixed_bytes + (uint64_t)budget_envs * c.per_env_bytes;
  c.capacity = capacity;
  c.max_tick_envs = capacity;
  c.max_session_envs = capacity;
  c.n_roms = 3;
  c.lanes = 4;
  c.warps = 2;
  return c;
}

static void admission_fifo() {
  Scheduler s(base(100, 100));
  const int a = s.open(0, 60, 0, 0);
  CHECK(a >= 0 && s.state(a) == SESSION_ADMITTED);
  const int b = s.open(1, 50, 100, 0);
  CHECK(b >= 0 && s.state(b) == SESSION_QUEUED);   // 40 slots free
  const int c = s.open(2, 10, 200, 0);
  CHECK(c >= 0 && s.state(c) == SESSION_QUEUED);   // fits, but FIFO: never overtakes b
  CHECK(s.queued_sessions() == 2);
  CHECK(s.close(a, 1) == 0);
  CHECK(s.state(b) == SESSION_ADMITTED && s.state(c) == SESSION_ADMITTED);
  CHECK(s.free_slots() == 40);
  CHECK(s.bytes_in_use() == 5000 + 60 * 1000);
  // a queued session can be withdrawn (open timed out)
  const int d = s.open(0, 45, 300, 2);
  CHECK(s.state(d) == SESSION_QUEUED);
  CHECK(s.close(d, 3) == 0 && s.state(d) == SESSION_CLOSED);
  CHECK(s.close(d, 3) == E_NOSESSION);
  const int e = s.open(0, 40, 400, 4);
  CHECK(s.state(e) == SESSION_ADMITTED && s.free_slots() == 0);
}

static void budget_binds_before_slots() {
  Scheduler s(base(100, 70));        // 100 slots but budget for 70 envs
  const int a = s.open(0, 60, 0, 0);
  CHECK(s.state(a) == SESSION_ADMITTED);
  const int b = s.open(0, 20, 0, 0);
  CHECK(s.state(b) == SESSION_QUEUED && s.free_slots() == 40);
  CHECK(s.open(0, 71, 0, 0) == E_NOMEM);   // larger than the whole budget
  CHECK(s.open(3, 1, 0, 0) == E_INVAL);    // no such cartridge
  CHECK(s.open(0, 0, 0, 0) == E_INVAL);
  CHECK(s.open(0, 101, 0, 0) == E_INVAL);
  CHECK(s.close(a, 1) == 0 && s.state(b) == SESSION_ADMITTED);
}

struct Sim {
  Scheduler s;
  std::map<int, std::vector<uint8_t>> acts;
  explicit Sim(const SchedConfig &c) : s(c) {}
};

// Every invariant of one planned tick.
static void check_tick(const Scheduler &s, const TickPlan &t, const SchedConfig &c,
                       const std::set<int> &first_step) {
  int total = 0;
  for (const Request *r : t.reqs) {
    CHECK(r->out_offset == total && r->launched && r->tick_envs == t.n_active);
    total += r->n;
  }
  CHECK(total == t.n_active);
  CHECK(t.reqs.size() == 1 || t.n_active <= c.max_tick_envs);
  const int G = t.n_groups, N = t.n_active;
  CHECK((int)t.blob.size() == 3 * G + 2 * N);
  const int32_t *rom = t.blob.data(), *st = rom + G, *cnt = st + G, *perm = cnt + G, *opos = perm + N;
  // groups tile [0, N) in order, ascending cartridge, at most lanes * warps each
  int at = 0;
  for (int g = 0; g < G; ++g) {
    CHECK(st[g] == at && cnt[g] >= 1 && cnt[g] <= c.lanes * c.warps);
    if (g) CHECK(rom[g] >= rom[g - 1]);
    at += cnt[g];
  }
  CHECK(at == N);
  // (slot -> request env) mapping: perm/opos agree with the sessions
  std::vector<int> seen_out((size_t)N, 0);
  std::map<int32_t, int> slot_seen;
  std::map<int, const Request *> by_off;
  for (const Request *r : t.reqs) by_off[r->out_offset] = r;
  for (int g = 0; g < G; ++g)
    for (int p = st[g]; p < st[g] + cnt[g]; ++p) {
      CHECK(opos[p] >= 0 && opos[p] < N);
      seen_out[(size_t)opos[p]]++;
      auto it = by_off.upper_bound(opos[p]);
      --it;
      const Request *r = it->second;
      const int j = opos[p] - r->out_offset;
      CHECK(j >= 0 && j < r->n);
      const Session *ss = s.session(r->sid);
      CHECK(ss && ss->rom == rom[g]);
      CHECK(ss->slots[(size_t)j] == perm[p]);
      CHECK(++slot_seen[perm[p]] == 1);
      CHECK(t.actions[(size_t)opos[p]] == r->actions[j]);
    }
  for (int v : seen_out) CHECK(v == 1);
  // init entries: exactly the sessions stepped for the first time
  int n_init = 0;
  for (const Request *r : t.reqs)
    if (first_step.count(r->sid)) {
      const Session *ss = s.session(r->sid);
      for (int j = 0; j < r->n; ++j) {
        bool found = false;
        for (int k = 0; k < t.n_init; ++k)
          if (t.init[(size_t)k] == ss->slots[(size_t)j]) {
            CHECK(t.init[(size_t)(t.n_init + k)] == ss->rom);
            CHECK((uint32_t)t.init[(size_t)(2 * t.n_init + k)] == ss->key_base + (uint32_t)j);
            found = true;
          }
        CHECK(found);
      }
      n_init += r->n;
    }
  CHECK(n_init == t.n_init);
}

static void random_traffic(uint64_t seed, int max_tick) {
  SchedConfig c = base(500, 450);
  c.max_tick_envs = max_tick;
  c.max_session_envs = std::min(120, max_tick);
  Scheduler s(c);
  std::mt19937_64 rng(seed);
  std::vector<int> open_ids;
  std::set<int> stepped;
  std::map<int, std::vector<uint8_t>> acts;
  std::vector<Request *> live;
  int64_t now = 0;
  for (int it = 0; it < 3000; ++it) {
    now += 10;
    const int op = (int)(rng() % 10);
    if (op < 2) {
      const int sid = s.open((int)(rng() % 3), 1 + (int)(rng() % c.max_session_envs), (uint32_t)(rng() % 100000) * 128, now);
      CHECK(sid >= 0);
      open_ids.push_back(sid);
    } else if (op < 3 && !open_ids.empty()) {
      const int k = (int)(rng() % open_ids.size());
      const int sid = open_ids[(size_t)k];
      const int rc = s.close(sid, now);
      const Session *ss = s.session(sid);
      if (rc == E_BUSY) CHECK(ss->busy);
      else {
        CHECK(rc == 0);
        open_ids.erase(open_ids.begin() + k);
      }
    } else if (op < 7 && !open_ids.empty()) {
      const int sid = open_ids[rng() % open_ids.size()];
      const Session *ss = s.session(sid);
      auto *r = new Request();
      r->sid = sid;
      auto &a = acts[sid];
      a.resize((size_t)ss->n);
      for (auto &x : a) x = (uint8_t)(rng() % 18);
      r->actions = a.data();
      const int rc = s.enqueue(r, now);
      if (ss->state != SESSION_ADMITTED) CHECK(rc == E_NOSESSION);
      else if (ss->busy && rc == E_BUSY) {
      } else CHECK(rc == 0);
      if (rc) delete r;
      else live.push_back(r);
    } else {
      TickPlan t;
      std::set<int> first;
      for (Request *r : live)
        if (!r->launched && s.session(r->sid)->needs_init) first.insert(r->sid);
      if (s.plan_tick(t, now)) {
        std::set<int> in_tick;
        for (Request *r : t.reqs) in_tick.insert(r->sid);
        std::set<int> first_here;
        for (int sid : first) if (in_tick.count(sid)) first_here.insert(sid);
        check_tick(s, t, c, first_here);
        s.finish_tick(t, now);
        for (Request *r : t.reqs) {
          live.erase(std::find(live.begin(), live.end(), r));
          delete r;
        }
      }
    }
    // slot accounting: admitted sessions' slots and the free list partition all slots
    std::set<int32_t> all;
    int used = 0;
    for (int sid : open_ids) {
      const Session *ss = s.session(sid);
      if (ss->state != SESSION_ADMITTED) continue;
      used += ss->n;
      for (int32_t x : ss->slots) CHECK(all.insert(x).second);
    }
    CHECK(used + s.free_slots() == c.capacity);
    CHECK(s.bytes_in_use() <= c.budget_bytes);
    CHECK(s.bytes_in_use() == c.fixed_bytes + (uint64_t)used * c.per_env_bytes);
  }
  for (Request *r : live) delete r;
}

static void busy_and_reclaim() {
  SchedConfig c = base(50, 50);
  c.idle_timeout_ns = 100;
  Scheduler s(c);
  const int a = s.open(0, 10, 0, 0), b = s.open(1, 10, 1000, 0);
  Request ra, rb, rb2;
  std::vector<uint8_t> acts(10, 3);
  ra.sid = a;
  ra.actions = acts.data();
  rb.sid = b;
  rb.actions = acts.data();
  rb2 = rb;
  CHECK(s.enqueue(&ra, 50) == 0);
  CHECK(s.enqueue(&rb, 50) == 0);
  CHECK(s.enqueue(&rb2, 50) == E_BUSY);
  CHECK(s.close(a, 60) == E_BUSY);
  CHECK(s.withdraw(&rb));
  CHECK(!s.withdraw(&rb));
  TickPlan t;
  CHECK(s.plan_tick(t, 70) && t.reqs.size() == 1 && t.n_init == 10);
  // a busy session is never reclaimed, an idle one is
  auto gone = s.reclaim_idle(1000);
  CHECK(gone.size() == 1 && gone[0] == b && s.state(b) == SESSION_CLOSED);
  CHECK(s.state(a) == SESSION_ADMITTED);
  s.finish_tick(t, 1000);
  CHECK(s.reclaim_idle(1050).empty());
  gone = s.reclaim_idle(1101);
  CHECK(gone.size() == 1 && gone[0] == a);
  CHECK(s.free_slots() == 50);
  // the second step of a session carries no init entries
  const int d = s.open(2, 5, 7, 2000);
  Request r1;
  r1.sid = d;
  r1.actions = acts.data();
  CHECK(s.enqueue(&r1, 2000) == 0 && s.plan_tick(t, 2000) && t.n_init == 5);
  s.finish_tick(t, 2001);
  CHECK(s.enqueue(&r1, 2002) == 0 && s.plan_tick(t, 2002) && t.n_init == 0);
  CHECK(!s.plan_tick(t, 2003));
}

static void tick_cap_splits() {
  SchedConfig c = base(300, 300);
  c.max_tick_envs = 100;
  c.max_session_envs = 100;
  Scheduler s(c);
  std::vector<uint8_t> acts(100, 1);
  std::vector<Request> rs(4);
  const int n[4] = {60, 30, 20, 100};
  for (int i = 0; i < 4; ++i) {
    rs[(size_t)i].sid = s.open(i % 3, n[i], (uint32_t)i * 1000, 0);
    rs[(size_t)i].actions = acts.data();
    CHECK(s.enqueue(&rs[(size_t)i], 1) == 0);
  }
  TickPlan t;
  CHECK(s.plan_tick(t, 2) && t.n_active == 90 && t.reqs.size() == 2);   // 60 + 30; 20 more would pass 100
  CHECK(s.plan_tick(t, 3) && t.n_active == 20);                           // FIFO: the 100 does not fit after 20
  CHECK(s.plan_tick(t, 4) && t.n_active == 100);
  CHECK(!s.plan_tick(t, 5));
}

int main() {
  admission_fifo();
  budget_binds_before_slots();
  busy_and_reclaim();
  tick_cap_splits();
  for (uint64_t seed = 1; seed <= 6; ++seed) random_traffic(seed, seed % 2 ? 500 : 150);
  (void)g_fail;
  std::printf("ok\n");
  return 0;
}
