// Host-side checks of the serving engine's coefficient-row index (no GPU):
// publish on success only, pins protect rows from eviction, eviction takes
// the least recently used unpinned row, a key published twice keeps one row,
// and clear() frees everything. Exits non-zero on the first failed check.
#include <stdio.h>

#include "server_cache.h"

using mmgpu::CacheKey;
using mmgpu::CoefCache;

static int fails = 0;
#define CHECK(c)                                              \
  do {                                                        \
    if (!(c)) {                                               \
      fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c); \
      ++fails;                                                \
    }                                                         \
  } while (0)

static CacheKey key(int asset, int N = 10, double t0 = 0.0, double t1 = 1.0) {
  CacheKey k;
  k.asset = asset;
  k.N = N;
  k.t0 = t0;
  k.t1 = t1;
  return k;
}

int main() {
  CoefCache c;
  c.reset(3);
  CHECK(c.size() == 3 && c.free_rows() == 3 && c.published() == 0);

  // a reserved row is invisible until published; a failed request returns it
  int r0 = c.reserve(key(0));
  CHECK(r0 >= 0 && c.acquire(key(0)) == -1);
  c.finish_reserved(r0, false);
  CHECK(c.free_rows() == 3 && c.published() == 0 && c.acquire(key(0)) == -1);

  // publish three rows: asset 0, 1, 2 (0 oldest)
  int r[3];
  for (int a = 0; a < 3; ++a) {
    r[a] = c.reserve(key(a));
    CHECK(r[a] >= 0);
  }
  CHECK(c.reserve(key(9)) == -1);  // every row pinned by its writer
  for (int a = 0; a < 3; ++a) c.finish_reserved(r[a], true);
  CHECK(c.published() == 3 && c.evictable() == 3 && c.free_rows() == 0);

  // keys differ by asset, cutoff and window
  CHECK(c.acquire(key(0, 11)) == -1 && c.acquire(key(0, 10, 0.0, 2.0)) == -1 && c.acquire(key(5)) == -1);

  // reading asset 0 makes it the most recently used; a pinned row is never evicted
  int h0 = c.acquire(key(0));
  CHECK(h0 == r[0] && c.pins(h0) == 1 && c.evictable() == 2);
  int n1 = c.reserve(key(3));  // evicts the least recently used unpinned row: asset 1
  CHECK(n1 == r[1] && c.acquire(key(1)) == -1 && c.published() == 2);
  c.finish_reserved(n1, true);
  c.unpin(h0);
  // order now (most recent first): 0, 3, 2 -> next eviction takes asset 2
  int n2 = c.reserve(key(4));
  CHECK(n2 == r[2] && c.acquire(key(2)) == -1);
  c.finish_reserved(n2, true);
  int a0 = c.acquire(key(0)), a3 = c.acquire(key(3)), a4 = c.acquire(key(4));
  CHECK(a0 == r[0] && a3 == n1 && a4 == n2);
  CHECK(c.reserve(key(7)) == -1);  // all three pinned by readers
  c.unpin(a0);
  c.unpin(a3);
  c.unpin(a4);

  // two writers of one key: the first to finish publishes, the other's row is returned
  c.clear();
  CHECK(c.free_rows() == 3 && c.published() == 0);
  int w1 = c.reserve(key(8)), w2 = c.reserve(key(8));
  CHECK(w1 >= 0 && w2 >= 0 && w1 != w2);
  c.finish_reserved(w2, true);
  c.finish_reserved(w1, true);
  CHECK(c.published() == 1 && c.free_rows() == 2 && c.acquire(key(8)) == w2);
  c.unpin(w2);
  CHECK(c.evictable() == 1);

  if (fails == 0) printf("cache ok\n");
  return fails == 0 ? 0 : 1;
}
