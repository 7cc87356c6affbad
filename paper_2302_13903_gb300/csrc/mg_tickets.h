// mg_tickets.h -- the serving loop's ticket book: which requests a caller can
// still poll or wait on, and when a finished request's record may be freed.
// Host-only, so that its thread safety is tested without a GPU.
//
// A request record R carries three fields the book uses:
//   bool done;     set (under the caller's mutex) when the result is final
//   int waiters;   threads blocked in wait() on it
//   bool retired;  its ticket no longer resolves
// Every member function runs with the caller's mutex held (wait() releases it
// while blocked, through the condition variable).  A ticket retires the first
// time a poll or a wait sees its request done: later polls and waits of that
// ticket answer "unknown".  Every thread already waiting when it retires still
// receives the result.  The record is freed by whichever of the retiring call
// and the waiters leaves last, so no thread reads it after it is freed and it
// is freed exactly once.
#pragma once

#include <chrono>
#include <condition_variable>
#include <mutex>
#include <unordered_map>
#include <vector>

namespace mg {
namespace tickets {

enum class Got { UNKNOWN, PENDING, DONE };

template <class R>
class Book {
 public:
  Book() = default;
  Book(const Book&) = delete;
  Book& operator=(const Book&) = delete;
  ~Book() { clear(); }

  void add(long long ticket, R* r) { live_[ticket] = r; }

  // Copy the request's state out through fill(const R&); retire it if done.
  template <class Fill>
  Got poll(long long ticket, Fill&& fill) {
    auto it = live_.find(ticket);
    if (it == live_.end()) return Got::UNKNOWN;
    R* r = it->second;
    fill(*r);
    if (!r->done) return Got::PENDING;
    retire(it);
    return Got::DONE;
  }

  // Block on cv (whose mutex lk holds) until the request is done or
  // timeout_s passes, then copy its state out through fill.
  template <class Fill>
  Got wait(long long ticket, std::unique_lock<std::mutex>& lk, std::condition_variable& cv,
           double timeout_s, Fill&& fill) {
    auto it = live_.find(ticket);
    if (it == live_.end()) return Got::UNKNOWN;
    R* r = it->second;
    ++r->waiters;
    const bool done = cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                  [r] { return r->done; });
    --r->waiters;
    fill(*r);
    if (!done) return Got::PENDING;  // not done, so not retired: still live
    if (!r->retired) {
      retire(live_.find(ticket));
    } else if (r->waiters == 0) {
      delete r;  // retired by another call while this thread waited; last one out
    }
    return Got::DONE;
  }

  // Free every live record (no thread may be waiting).
  void clear() {
    for (auto& kv : live_) delete kv.second;
    live_.clear();
  }

  size_t live() const { return live_.size(); }

 private:
  using Iter = typename std::unordered_map<long long, R*>::iterator;
  void retire(Iter it) {
    R* r = it->second;
    live_.erase(it);
    r->retired = true;
    if (r->waiters == 0) delete r;  // else the last waiter to leave frees it
  }

  std::unordered_map<long long, R*> live_;
};

}  // namespace tickets
}  // namespace mg
