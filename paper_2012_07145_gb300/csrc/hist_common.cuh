// Device helpers shared by the histogram-equalization kernels (the three
// stage kernels and the fused one): warp-aggregated counting into a
// per-warp sub-histogram, the CDF and equalization table, and the table
// lookup of four packed bytes.  All counts are exact integers.
#pragma once

#include <cuda_runtime.h>

namespace hp {

// Division of a 32-bit chunk index by the chunks per row, a divisor fixed for
// the launch: one multiply-high, a subtract, an add and two shifts instead of
// an integer division (a long instruction sequence on the GPU, and the
// kernels' largest per-chunk cost when it was done in 64 bits).  The method is
// that of Granlund and Montgomery, "Division by invariant integers using
// multiplication" (1994), for every n < 2^32 and 1 <= d < 2^32: with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1 (which fits in 32
// bits), t = mulhi(m, n) and n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
  unsigned int d, m;
  int s1, s2;
};

inline FastDiv make_fastdiv(unsigned int d) {
  int l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (unsigned int)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ unsigned int fastdiv(unsigned int n, const FastDiv& f) {
  const unsigned int t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Adds byte value v to the warp's sub-histogram wh.  When every active lane
// holds the same value (flat regions, constant images: the worst case for
// contention) one lane adds the whole count.
__device__ __forceinline__ void count_byte(unsigned int* wh, unsigned int v, unsigned int active) {
  const int first = __ffs(active) - 1;
  const bool uniform = __all_sync(active, v == __shfl_sync(active, v, first));
  if (uniform) {
    if ((int)(threadIdx.x & 31) == first) atomicAdd(&wh[v], (unsigned int)__popc(active));
  } else {
    atomicAdd(&wh[v], 1u);
  }
}

// The CDF of the 256 counts and the equalization table, by one CTA: thread v
// (v < 256) passes the count of bin v in h and writes table entry v; the other
// threads of a larger CTA pass anything and only take part in the barriers.
//   N == cmin: LUT[v] = v;  cdf[v] < cmin: 0;
//   else ((cdf[v]-cmin)*510 + (N-cmin)) / (2*(N-cmin)) in 64-bit integers,
// N the pixel count and cmin the CDF at the first non-empty bin.
__device__ __forceinline__ void cdf_lut_cta(unsigned int h, unsigned char* __restrict__ lut) {
  __shared__ unsigned int warp_tot[8];
  __shared__ unsigned int s_cmin, s_first;
  const int v = threadIdx.x;
  const bool mine = v < 256;
  const int lane = v & 31, w = v >> 5;
  if (!mine) h = 0;
  unsigned int c = h;
  if (mine) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int t = __shfl_up_sync(0xffffffffu, c, o);
      if (lane >= o) c += t;
    }
    if (lane == 31) warp_tot[w] = c;
  }
  if (v == 0) s_first = 256;
  __syncthreads();
  if (mine) {
    unsigned int off = 0;
    for (int i = 0; i < w; ++i) off += warp_tot[i];
    c += off;
    if (h > 0) atomicMin(&s_first, (unsigned int)v);
  }
  __syncthreads();
  if (mine) {
    if (v == (int)s_first) s_cmin = c;
    if (s_first == 256 && v == 0) s_cmin = 0;
  }
  __syncthreads();
  if (!mine) return;
  unsigned long long n = 0;
  for (int i = 0; i < 8; ++i) n += warp_tot[i];
  unsigned long long cmin = s_cmin;
  unsigned int out;
  if (n == cmin) {
    out = (unsigned int)v;
  } else if (c < cmin) {
    out = 0;
  } else {
    unsigned long long den = n - cmin;
    out = (unsigned int)((((unsigned long long)c - cmin) * 510ull + den) / (2ull * den));
  }
  lut[v] = (unsigned char)out;
}

__device__ __forceinline__ unsigned int lut4(const unsigned char* t, unsigned int a) {
  return (unsigned int)t[a & 0xff] | ((unsigned int)t[(a >> 8) & 0xff] << 8) |
         ((unsigned int)t[(a >> 16) & 0xff] << 16) | ((unsigned int)t[a >> 24] << 24);
}

}  // namespace hp
