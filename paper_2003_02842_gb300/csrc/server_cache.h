// server_cache.h -- host-side index of the serving engine's resident
// coefficient rows (plain C++, no CUDA): rows keyed by (asset, t0, t1, N),
// pinned while requests in flight read or write them, published when the
// request that wrote them finishes, and evicted least recently used first.
// The device rows themselves live in the server; this class only hands out
// row numbers.
#pragma once

#include <stdint.h>
#include <string.h>

#include <list>
#include <unordered_map>
#include <vector>

namespace mmgpu {

struct CacheKey {
  int asset = 0;
  int N = 0;
  double t0 = 0, t1 = 0;
  bool operator==(const CacheKey& o) const {
    return asset == o.asset && N == o.N && memcmp(&t0, &o.t0, sizeof(double)) == 0 &&
           memcmp(&t1, &o.t1, sizeof(double)) == 0;
  }
};

struct CacheKeyHash {
  size_t operator()(const CacheKey& k) const {
    uint64_t a, b;
    memcpy(&a, &k.t0, 8);
    memcpy(&b, &k.t1, 8);
    uint64_t h = (uint64_t)(uint32_t)k.asset * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)(uint32_t)k.N + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
    h ^= a + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    h ^= b + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

class CoefCache {
 public:
  // n rows, all free
  void reset(int n) {
    rows_.assign(n, Row{});
    clear();
  }

  // every row free (the store the rows were computed from changed)
  void clear() {
    index_.clear();
    lru_.clear();
    free_.clear();
    for (int r = (int)rows_.size() - 1; r >= 0; --r) {
      rows_[r] = Row{};
      free_.push_back(r);
    }
  }

  int size() const { return (int)rows_.size(); }

  // the published row of k, pinned for the caller; -1 when absent
  int acquire(const CacheKey& k) {
    const auto it = index_.find(k);
    if (it == index_.end()) return -1;
    pin(it->second);
    return it->second;
  }

  // a row the caller will write for k, pinned and not yet visible to
  // acquire(): a free row, else the least recently used unpinned one
  // (dropped from the index); -1 when every row is in use
  int reserve(const CacheKey& k) {
    int r = -1;
    if (!free_.empty()) {
      r = free_.back();
      free_.pop_back();
    } else if (!lru_.empty()) {
      r = lru_.back();
      lru_.pop_back();
      index_.erase(rows_[r].key);
      rows_[r] = Row{};
    } else {
      return -1;
    }
    rows_[r].key = k;
    rows_[r].pins = 1;
    return r;
  }

  // a request is done with rows it acquired
  void unpin(int r) {
    Row& c = rows_[r];
    c.pins -= 1;
    if (c.pins == 0 && c.indexed) {
      lru_.push_front(r);
      c.lru = lru_.begin();
      c.in_lru = true;
    }
  }

  // a request is done with a row it reserved: with ok, the row is published
  // (unless its key was published meanwhile), else it is returned
  void finish_reserved(int r, bool ok) {
    Row& c = rows_[r];
    if (ok && index_.find(c.key) == index_.end()) {
      index_.emplace(c.key, r);
      c.indexed = true;
      unpin(r);
    } else {
      rows_[r] = Row{};
      free_.push_back(r);
    }
  }

  // counts for tests and statistics
  int published() const { return (int)index_.size(); }
  int evictable() const { return (int)lru_.size(); }
  int free_rows() const { return (int)free_.size(); }
  int pins(int r) const { return rows_[r].pins; }

 private:
  struct Row {
    CacheKey key;
    int pins = 0;          // requests in flight that read or write this row
    bool indexed = false;  // visible to acquire()
    bool in_lru = false;   // unpinned and indexed: evictable
    std::list<int>::iterator lru;
  };

  void pin(int r) {
    Row& c = rows_[r];
    if (c.in_lru) {
      lru_.erase(c.lru);
      c.in_lru = false;
    }
    c.pins += 1;
  }

  std::vector<Row> rows_;
  std::unordered_map<CacheKey, int, CacheKeyHash> index_;
  std::list<int> lru_;  // evictable rows, most recently used first
  std::vector<int> free_;
};

}  // namespace mmgpu
