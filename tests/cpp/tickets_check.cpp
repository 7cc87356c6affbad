// Host-only checks of the serving loop's ticket book (mg_tickets.h): several
// threads polling and waiting on one ticket, every record freed exactly once
// and never read after it is freed.  Exits non-zero on the first failed check.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <thread>
#include <vector>

#include "mg_tickets.h"

#define CHECK(c)                                                                    \
  do {                                                                              \
    if (!(c)) {                                                                     \
      std::fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c);   \
      std::exit(1);                                                                 \
    }                                                                               \
  } while (0)

using mg::tickets::Book;
using mg::tickets::Got;

static std::atomic<int> g_alive{0};
static std::atomic<int> g_freed{0};

struct Rec {
  bool done = false;
  int waiters = 0;
  bool retired = false;
  int value = 0;
  int magic = 0x5eed;
  Rec() { ++g_alive; }
  ~Rec() {
    CHECK(magic == 0x5eed);  // freed twice, or never a record
    magic = 0;
    --g_alive;
    ++g_freed;
  }
};

struct Server {
  std::mutex mu;
  std::condition_variable cv;
  Book<Rec> book;
};

static void finish(Server& S, Rec* r, int value) {
  std::lock_guard<std::mutex> lk(S.mu);
  r->value = value;
  r->done = true;
  S.cv.notify_all();
}

int main() {
  {  // poll: pending, then done once, then unknown
    Server S;
    Rec* r = new Rec;
    S.book.add(1, r);
    int seen = -1;
    {
      std::lock_guard<std::mutex> lk(S.mu);
      CHECK(S.book.poll(1, [&](const Rec& x) { seen = x.done; }) == Got::PENDING);
      CHECK(seen == 0);
    }
    finish(S, r, 7);
    std::lock_guard<std::mutex> lk(S.mu);
    CHECK(S.book.poll(1, [&](const Rec& x) { seen = x.value; }) == Got::DONE);
    CHECK(seen == 7);
    CHECK(S.book.poll(1, [&](const Rec&) {}) == Got::UNKNOWN);
    CHECK(S.book.live() == 0 && g_alive == 0);
  }
  {  // a wait that times out keeps the ticket
    Server S;
    S.book.add(2, new Rec);
    std::unique_lock<std::mutex> lk(S.mu);
    CHECK(S.book.wait(2, lk, S.cv, 0.01, [](const Rec&) {}) == Got::PENDING);
    CHECK(S.book.live() == 1);
    S.book.clear();
    CHECK(g_alive == 0);
  }
  // Many rounds of: W threads waiting on one ticket, P threads polling it,
  // one thread finishing it.  Every waiter gets the value; the record is
  // freed exactly once; later calls see an unknown ticket.
  for (int round = 0; round < 300; ++round) {
    Server S;
    Rec* r = new Rec;
    const long long t = 100 + round;
    S.book.add(t, r);
    const int W = 2 + round % 3, P = round % 2;
    std::atomic<int> got_done{0}, got_value{0}, got_unknown{0};
    std::atomic<int> started{0};
    std::vector<std::thread> th;
    for (int w = 0; w < W; ++w)
      th.emplace_back([&] {
        std::unique_lock<std::mutex> lk(S.mu);
        ++started;
        int v = -1;
        const Got g = S.book.wait(t, lk, S.cv, 10.0, [&](const Rec& x) { v = x.value; });
        if (g == Got::DONE) {
          ++got_done;
          if (v == 42) ++got_value;
        } else if (g == Got::UNKNOWN) {
          ++got_unknown;  // it arrived after a poll retired the ticket
        }
      });
    for (int q = 0; q < P; ++q)
      th.emplace_back([&] {
        for (int k = 0; k < 1000; ++k) {
          std::lock_guard<std::mutex> lk(S.mu);
          int v = -1;
          const Got g = S.book.poll(t, [&](const Rec& x) { v = x.value; });
          if (g == Got::DONE) {
            CHECK(v == 42);
            ++got_done;
            break;
          }
          if (g == Got::UNKNOWN) break;
        }
      });
    while (started < W) std::this_thread::yield();
    std::this_thread::sleep_for(std::chrono::microseconds(50 * (round % 4)));
    finish(S, r, 42);
    for (std::thread& x : th) x.join();
    // every waiter was inside wait() before the finish, so none sees an
    // unknown ticket and each receives the value
    CHECK(got_unknown == 0 && got_value == W);
    CHECK(g_alive == 0);  // freed, once (the destructor checks the once)
    std::lock_guard<std::mutex> lk(S.mu);
    CHECK(S.book.poll(t, [](const Rec&) {}) == Got::UNKNOWN);
  }
  {  // waiters that all started before the finish all receive the result
    Server S;
    Rec* r = new Rec;
    S.book.add(9, r);
    std::atomic<int> ok{0}, started{0};
    std::vector<std::thread> th;
    for (int w = 0; w < 4; ++w)
      th.emplace_back([&] {
        std::unique_lock<std::mutex> lk(S.mu);
        ++started;
        int v = -1;
        if (S.book.wait(9, lk, S.cv, 10.0, [&](const Rec& x) { v = x.value; }) == Got::DONE &&
            v == 5)
          ++ok;
      });
    while (started < 4) std::this_thread::yield();
    {
      // every waiter is inside wait() once it released the mutex
      std::lock_guard<std::mutex> lk(S.mu);
      CHECK(r->waiters == 4);
    }
    finish(S, r, 5);
    for (std::thread& x : th) x.join();
    CHECK(ok == 4 && g_alive == 0);
  }
  std::printf("ticket checks passed (%d records freed)\n", g_freed.load());
  return 0;
}
