// mg_admission.h -- the serving loop's admission policy, host code only.
//
// The server keeps grid hierarchies (solver contexts) resident on the device
// between requests.  Each resident hierarchy is keyed by what fixes its layout
// and constants (cells per side, cell width, boundary rule, the fixed boundary
// value, the multipole order).  A request is admitted when a hierarchy for
// its key is idle, or when a new one fits in the HBM budget, after evicting
// idle hierarchies in least-recently-used order if needed.  A request that
// cannot be admitted now waits; a later request in the queue may pass it, but
// only a bounded number of times, after which the queue head holds the next
// free slot (no starvation of large requests behind a stream of small ones).
//
// Nothing here touches CUDA: the caller creates and destroys the contexts the
// decisions name, so the policy is tested on the host alone.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace mg {
namespace admission {

struct Key {
  int n = 0, bc = 0, lmax = 0;
  double dx = 0.0, fixed_value = 0.0;
  bool host = false;  // requests with host buffers: the hierarchy holds device copies too
  int slots = 0;      // > 0: a batched hierarchy of that many grids of this shape
  int fk = 0;         // a rule per face (bc = 4): the kind of face q in bits 2q..2q+1
  double fv[6] = {};  // ... and the values of its fixed faces
  bool operator==(const Key& o) const {
    if (!(n == o.n && bc == o.bc && lmax == o.lmax && dx == o.dx &&
          fixed_value == o.fixed_value && host == o.host && slots == o.slots && fk == o.fk))
      return false;
    for (int q = 0; q < 6; ++q)
      if (fv[q] != o.fv[q]) return false;
    return true;
  }
};

struct Resident {
  uint64_t id = 0;      // stable name of the slot (indices move on eviction)
  Key key;
  void* ctx = nullptr;  // owned by the caller; null while being created
  size_t bytes = 0;
  bool busy = false;
  uint64_t last_used = 0;
};

enum class Act { USE, CREATE, WAIT, NEVER };

struct Decision {
  Act act = Act::WAIT;
  uint64_t id = 0;               // USE / CREATE: the slot taken
  void* ctx = nullptr;           // USE: its context
  std::vector<void*> evict;      // contexts to destroy before CREATE
};

class Pool {
 public:
  explicit Pool(size_t budget) : budget_(budget) {}

  size_t budget() const { return budget_; }
  size_t resident_bytes() const { return bytes_; }
  size_t peak_bytes() const { return peak_; }
  long long evictions() const { return evictions_; }
  long long created() const { return created_; }
  const std::vector<Resident>& residents() const { return res_; }

  // Admission of one request with key k whose hierarchy needs `need` bytes.
  // USE marks an idle matching hierarchy busy.  CREATE reserves `need` bytes
  // in a new busy slot (ctx null until set_ctx) after dropping the evicted
  // idle hierarchies from the pool.  WAIT changes nothing.  NEVER: the
  // hierarchy alone exceeds the budget.
  Decision admit(const Key& k, size_t need) {
    Decision d;
    for (size_t i = 0; i < res_.size(); ++i) {
      Resident& r = res_[i];
      if (!r.busy && r.ctx && r.key == k) {
        r.busy = true;
        r.last_used = ++clock_;
        d.act = Act::USE;
        d.id = r.id;
        d.ctx = r.ctx;
        return d;
      }
    }
    if (need > budget_) {  // never fits (the server refuses it at submission)
      d.act = Act::NEVER;
      return d;
    }
    size_t idle = 0;
    for (const Resident& r : res_)
      if (!r.busy && r.ctx) idle += r.bytes;
    if (bytes_ + need > budget_ + idle) return d;  // WAIT: busy hierarchies hold the room
    while (bytes_ + need > budget_) {
      int lru = -1;
      for (size_t i = 0; i < res_.size(); ++i)
        if (!res_[i].busy && res_[i].ctx &&
            (lru < 0 || res_[i].last_used < res_[(size_t)lru].last_used))
          lru = (int)i;
      d.evict.push_back(res_[(size_t)lru].ctx);
      bytes_ -= res_[(size_t)lru].bytes;
      res_.erase(res_.begin() + lru);
      ++evictions_;
    }
    Resident r;
    r.id = ++ids_;
    r.key = k;
    r.bytes = need;
    r.busy = true;
    r.last_used = ++clock_;
    res_.push_back(r);
    bytes_ += need;
    if (bytes_ > peak_) peak_ = bytes_;
    ++created_;
    d.act = Act::CREATE;
    d.id = r.id;
    return d;
  }

  // The caller created the context of CREATE slot `id`.
  void set_ctx(uint64_t id, void* ctx) {
    for (Resident& r : res_)
      if (r.id == id) r.ctx = ctx;
  }

  // Creating the context of CREATE slot `id` failed: give its bytes back.
  void drop(uint64_t id) {
    for (size_t i = 0; i < res_.size(); ++i)
      if (res_[i].id == id) {
        bytes_ -= res_[i].bytes;
        res_.erase(res_.begin() + (long)i);
        --created_;
        return;
      }
  }

  // The request on this context finished: the hierarchy stays resident, idle.
  void release(void* ctx) {
    for (Resident& r : res_)
      if (r.ctx == ctx) {
        r.busy = false;
        r.last_used = ++clock_;
        return;
      }
  }

  // Every idle context, removed from the pool (for shutdown).
  std::vector<void*> drain_idle() {
    std::vector<void*> out;
    for (size_t i = 0; i < res_.size();) {
      if (!res_[i].busy && res_[i].ctx) {
        out.push_back(res_[i].ctx);
        bytes_ -= res_[i].bytes;
        res_.erase(res_.begin() + (long)i);
      } else {
        ++i;
      }
    }
    return out;
  }

 private:
  size_t budget_;
  size_t bytes_ = 0, peak_ = 0;
  long long evictions_ = 0, created_ = 0;
  uint64_t clock_ = 0, ids_ = 0;
  std::vector<Resident> res_;
};

// Which queued request a free worker takes: the first one in arrival order
// that `admit` lets in, except that once the queue head has been passed
// `max_bypass` times only the head may go.  `try_admit(i)` runs the
// admission for queue entry i and returns true when it was admitted (it must
// leave the pool unchanged otherwise).  Returns the index taken or -1.
template <typename TryAdmit>
int pick(size_t queue_len, int& head_bypassed, int max_bypass, TryAdmit try_admit) {
  if (queue_len == 0) return -1;
  if (try_admit((size_t)0)) {
    head_bypassed = 0;
    return 0;
  }
  if (head_bypassed >= max_bypass) return -1;
  for (size_t i = 1; i < queue_len; ++i)
    if (try_admit(i)) {
      ++head_bypassed;
      return (int)i;
    }
  return -1;
}

}  // namespace admission
}  // namespace mg
