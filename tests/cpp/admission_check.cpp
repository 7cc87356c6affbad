// Host-only checks of the serving loop's admission policy (mg_admission.h).
// Exits non-zero with a message on the first failed check.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <vector>

#include "mg_admission.h"

using namespace mg::admission;

#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      std::fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c); \
      std::exit(1);                                                \
    }                                                              \
  } while (0)

static Key key(int n, int bc = 0) {
  Key k;
  k.n = n;
  k.bc = bc;
  k.dx = 1.0 / n;
  return k;
}

static int fake[1000];  // addresses stand in for contexts

static void* created(Pool& p, const Decision& d, int tag) {
  CHECK(d.act == Act::CREATE);
  p.set_ctx(d.id, &fake[tag]);
  return &fake[tag];
}

int main() {
  {  // a released hierarchy is reused by the next request of its key
    Pool p(1000);
    Decision d = p.admit(key(32), 100);
    void* c = created(p, d, 1);
    CHECK(p.resident_bytes() == 100);
    Decision again = p.admit(key(32), 100);  // the only one is busy: a second is created
    CHECK(again.act == Act::CREATE);
    p.set_ctx(again.id, &fake[2]);
    p.release(c);
    Decision u = p.admit(key(32), 100);
    CHECK(u.act == Act::USE && u.ctx == c);
    Decision other = p.admit(key(32, 1), 100);  // another rule: another key
    CHECK(other.act == Act::CREATE);
    CHECK(p.created() == 3 && p.resident_bytes() == 300);
  }
  {  // busy hierarchies hold their room; idle ones are evicted, oldest first
    Pool p(250);
    void* a = created(p, p.admit(key(64), 100), 1);
    void* b = created(p, p.admit(key(128), 100), 2);
    CHECK(p.admit(key(256), 100).act == Act::WAIT);
    CHECK(p.resident_bytes() == 200);
    p.release(b);
    p.release(a);  // a is now the more recently used
    Decision d = p.admit(key(256), 100);
    CHECK(d.act == Act::CREATE && d.evict.size() == 1 && d.evict[0] == b);
    CHECK(p.resident_bytes() == 200 && p.peak_bytes() == 200 && p.evictions() == 1);
    p.set_ctx(d.id, &fake[3]);
    Decision e = p.admit(key(256, 2), 240);  // needs both idle... only a is idle
    CHECK(e.act == Act::WAIT);
    p.release(&fake[3]);
    Decision f = p.admit(key(256, 2), 240);
    CHECK(f.act == Act::CREATE && f.evict.size() == 2);
    CHECK(f.evict[0] == a && f.evict[1] == &fake[3]);
    CHECK(p.resident_bytes() == 240 && p.evictions() == 3);
  }
  {  // larger than the whole budget: never
    Pool p(100);
    CHECK(p.admit(key(512), 101).act == Act::NEVER);
    CHECK(p.resident_bytes() == 0 && p.created() == 0);
  }
  {  // a failed creation gives its bytes back
    Pool p(100);
    Decision d = p.admit(key(32), 60);
    p.drop(d.id);
    CHECK(p.resident_bytes() == 0 && p.created() == 0 && p.residents().empty());
    CHECK(p.admit(key(64), 100).act == Act::CREATE);
  }
  {  // a later request passes a waiting head at most max_bypass times
    Pool p(150);
    void* big = created(p, p.admit(key(128), 100), 1);  // running
    std::vector<Key> q = {key(256), key(16), key(16), key(16)};
    std::vector<size_t> need = {120, 10, 10, 10};
    int bypassed = 0, tag = 100;
    auto attempt = [&](size_t i) {
      Decision d = p.admit(q[i], need[i]);
      if (d.act == Act::CREATE) {
        p.set_ctx(d.id, &fake[tag++]);
        return true;
      }
      return d.act == Act::USE;
    };
    auto take = [&](int i) {  // the server removes what it picked from the queue
      if (i >= 0) {
        q.erase(q.begin() + i);
        need.erase(need.begin() + i);
      }
      return i;
    };
    CHECK(take(pick(q.size(), bypassed, 2, attempt)) == 1 && bypassed == 1);
    CHECK(take(pick(q.size(), bypassed, 2, attempt)) == 1 && bypassed == 2);
    CHECK(pick(q.size(), bypassed, 2, attempt) == -1);  // the head's turn now
    CHECK(q.size() == 2);
    p.release(big);
    p.release(&fake[101]);
    CHECK(take(pick(q.size(), bypassed, 2, attempt)) == 0 && bypassed == 0);
    CHECK(q.size() == 1 && q[0].n == 16);
    CHECK(p.resident_bytes() <= 150);
  }
  {  // random traffic: the budget and the pool's books always hold
    std::mt19937 rng(7);
    const size_t budget = 1000;
    Pool p(budget);
    std::vector<void*> busy;
    std::set<void*> gone;
    int next = 1;
    for (int step = 0; step < 20000; ++step) {
      if (!busy.empty() && (rng() % 3 == 0)) {
        const size_t i = rng() % busy.size();
        p.release(busy[i]);
        busy.erase(busy.begin() + (long)i);
      } else {
        const int n = 16 << (rng() % 4);
        const size_t need = (size_t)(n / 16) * (n / 16) * 15;  // 15, 60, 240, 960
        Decision d = p.admit(key(n, (int)(rng() % 3)), need);
        for (void* c : d.evict) {
          CHECK(!gone.count(c));
          for (void* b : busy) CHECK(b != c);  // never a busy one
          gone.insert(c);
        }
        if (d.act == Act::CREATE) {
          void* c = &fake[next % 1000];
          fake[next % 1000] = next;
          ++next;
          if (gone.count(c)) gone.erase(c);  // address reused by the fake allocator
          p.set_ctx(d.id, c);
          busy.push_back(c);
        } else if (d.act == Act::USE) {
          CHECK(!gone.count(d.ctx));
          busy.push_back(d.ctx);
        }
      }
      size_t sum = 0;
      for (const Resident& r : p.residents()) sum += r.bytes;
      CHECK(sum == p.resident_bytes());
      CHECK(p.resident_bytes() <= budget && p.peak_bytes() <= budget);
    }
    CHECK(p.evictions() > 0);
  }
  std::printf("admission checks passed\n");
  return 0;
}
