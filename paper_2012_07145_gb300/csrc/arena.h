// First-fit allocator over one device arena (the serving loop's request
// memory): offsets into a region reserved once, in 256-byte units, with the
// free blocks kept sorted by offset and merged with both neighbours on
// release.  Host-only bookkeeping: it never touches the device.
#pragma once

#include <algorithm>
#include <iterator>
#include <map>

namespace hp {

inline long long round256(long long v) { return (v + 255) / 256 * 256; }

struct Arena {
  char* base = nullptr;
  long long size = 0;
  std::map<long long, long long> free_blocks;  // offset -> size
  long long used = 0, peak = 0;

  // Reset to one free block of `bytes` (rounded down to 256) at offset 0.
  void init(char* b, long long bytes) {
    base = b;
    size = bytes;
    free_blocks.clear();
    free_blocks[0] = bytes / 256 * 256;
    used = peak = 0;
  }

  // The lowest-offset free block that holds `bytes` (rounded up to 256);
  // false when none does (the caller waits for a release).
  bool alloc(long long bytes, long long* off) {
    bytes = round256(bytes);
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const long long rest = it->second - bytes;
      const long long at = it->first + bytes;
      free_blocks.erase(it);
      if (rest > 0) free_blocks[at] = rest;
      used += bytes;
      peak = std::max(peak, used);
      return true;
    }
    return false;
  }

  // Returns a block that alloc gave out (same offset and size).
  void release(long long off, long long bytes) {
    bytes = round256(bytes);
    used -= bytes;
    auto it = free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
};

}  // namespace hp
