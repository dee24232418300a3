// noalloc_cache.h -- the per-context address cache of the allocation-free
// cost entry point (host code only, no CUDA types).
//
// A fixed table of (key, value) entries that are written once and never
// changed.  Inserts are serialised by the caller (a mutex); lookups take no
// lock: an entry is filled before the count that publishes it is stored
// (release), and a lookup reads the count first (acquire), so it only reads
// entries that are complete.  Keys are CUDA context ids, which the driver
// never reuses within a process; a key of 0 means "no context" and is never
// stored.  When the table is full, inserts are refused and callers simply do
// the lookup they would have cached.
#pragma once
#include <atomic>

namespace dfm {

template <class V, int Cap>
struct ScratchCache {
  unsigned long long keys[Cap] = {};
  V vals[Cap] = {};
  std::atomic<int> count{0};

  bool find(unsigned long long key, V* out) const {
    const int n = count.load(std::memory_order_acquire);
    for (int i = 0; i < n; ++i)
      if (keys[i] == key) {
        *out = vals[i];
        return true;
      }
    return false;
  }
  // Caller holds the insert lock.  False if the key is 0 or the table is full.
  bool insert(unsigned long long key, V val) {
    if (key == 0) return false;
    const int n = count.load(std::memory_order_relaxed);
    if (n >= Cap) return false;
    keys[n] = key;
    vals[n] = val;
    count.store(n + 1, std::memory_order_release);
    return true;
  }
};

}  // namespace dfm
