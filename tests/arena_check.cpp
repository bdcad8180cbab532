// Randomised check of the serving loop's arena allocator against a plain model:
// a bitmap of 256-byte units.  Every block alloc hands out must lie inside the
// arena, overlap no live block, and start at the first run of free units long
// enough for it (first fit over the merged free blocks); the free blocks must
// always be exactly the maximal free runs of the bitmap; used and peak must
// match the live bytes; and releasing everything must leave one block.
// Built and run by tests/test_arena.py; prints "ok" and exits 0 on success.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "arena.h"

namespace {

unsigned long long g_state = 0x9e3779b97f4a7c15ull;
unsigned long long next_u64() {  // splitmix64
  unsigned long long z = (g_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

int fail(const char* what, long long a, long long b) {
  std::printf("FAIL: %s (%lld, %lld)\n", what, a, b);
  return 1;
}

struct Live {
  long long off, bytes;
};

int run(long long arena_bytes, int ops, int max_units) {
  hp::Arena A;
  A.init(nullptr, arena_bytes);
  const long long units = arena_bytes / 256;
  std::vector<char> busy(units, 0);
  std::vector<Live> live;
  long long used = 0, peak = 0;
  for (int op = 0; op < ops; ++op) {
    const bool do_alloc = live.empty() || next_u64() % 100 < 55;
    if (do_alloc) {
      const long long bytes = 1 + (long long)(next_u64() % (unsigned long long)(max_units * 256));
      const long long need = (bytes + 255) / 256;
      long long want = -1;  // the model's first fit
      for (long long u = 0, run_len = 0; u < units; ++u) {
        run_len = busy[u] ? 0 : run_len + 1;
        if (run_len == need) {
          want = u - need + 1;
          break;
        }
      }
      long long off = -7;
      const bool ok = A.alloc(bytes, &off);
      if (ok != (want >= 0)) return fail("alloc succeeded iff a free run fits", ok, want);
      if (!ok) continue;
      if (off != want * 256) return fail("first fit offset", off, want * 256);
      if (off < 0 || off + need * 256 > units * 256) return fail("block inside the arena", off, need);
      for (long long u = 0; u < need; ++u) {
        if (busy[off / 256 + u]) return fail("overlap with a live block", off, u);
        busy[off / 256 + u] = 1;
      }
      live.push_back({off, bytes});
      used += need * 256;
      if (used > peak) peak = used;
    } else {
      const size_t k = (size_t)(next_u64() % live.size());
      const Live b = live[k];
      live[k] = live.back();
      live.pop_back();
      A.release(b.off, b.bytes);
      const long long need = (b.bytes + 255) / 256;
      for (long long u = 0; u < need; ++u) busy[b.off / 256 + u] = 0;
      used -= need * 256;
    }
    if (A.used != used) return fail("used bytes", A.used, used);
    if (A.peak != peak) return fail("peak bytes", A.peak, peak);
    // the free blocks are exactly the maximal free runs of the model
    auto it = A.free_blocks.begin();
    for (long long u = 0; u < units;) {
      if (busy[u]) {
        ++u;
        continue;
      }
      long long v = u;
      while (v < units && !busy[v]) ++v;
      if (it == A.free_blocks.end()) return fail("missing free block at", u * 256, (v - u) * 256);
      if (it->first != u * 256 || it->second != (v - u) * 256) return fail("free block", it->first, it->second);
      ++it;
      u = v;
    }
    if (it != A.free_blocks.end()) return fail("extra free block", it->first, it->second);
  }
  for (const Live& b : live) A.release(b.off, b.bytes);
  if (A.used != 0) return fail("used after releasing everything", A.used, 0);
  if (A.free_blocks.size() != 1 || A.free_blocks.begin()->first != 0 || A.free_blocks.begin()->second != units * 256)
    return fail("one free block after releasing everything", (long long)A.free_blocks.size(), units * 256);
  return 0;
}

}  // namespace

int main() {
  // a small arena with large requests (often full: refusals and merges), and a
  // larger one with small requests (many live blocks); an odd size rounds down
  if (run(64 * 256, 20000, 12)) return 1;
  if (run(4096 * 256 + 100, 20000, 40)) return 1;
  if (run(256, 1000, 1)) return 1;
  std::printf("ok\n");
  return 0;
}
