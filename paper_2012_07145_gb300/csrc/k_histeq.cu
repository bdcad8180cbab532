// Histogram equalization of a u8 image in one cooperative kernel: the image is
// read from memory once and written once.
//
// Each CTA takes a contiguous range of 16-pixel chunks (row-major over the
// image, a row's last chunk possibly partial) and holds them in registers
// (kEqK chunks per thread) while it counts them into per-warp sub-histograms
// (four interleaved copies per warp, one per lane mod 4, against same-address
// serialisation of the shared-memory atomics).  The CTA adds its counts to a device-wide histogram with
// one atomic per bin, then all CTAs meet at a grid-wide barrier -- they are
// co-resident because the launch is cooperative, and the wait is bounded --
// after which every CTA forms the CDF and the table itself (256 bins: cheaper
// than another launch) and writes its equalized chunks.  When an image has
// more chunks than the grid holds in registers, the CTA counts in rounds and
// reads its chunks again for the lookup.
//
// The device-wide state (two histograms, an arrival counter and a generation
// number) lives in a zero-initialised scratch that resets itself: launch g
// counts into histogram g & 1, and the last CTA to arrive clears the other
// histogram and the counter before it releases the others by bumping the
// generation, so the next launch (a CUDA-graph replay included) starts clean.
#include <cuda_runtime.h>

#include "hist_common.cuh"
#include "hp_internal.h"
#include "tma.cuh"

namespace hp {

namespace {

constexpr int kEqThreads = 1024;
constexpr int kEqWarps = kEqThreads / 32;
constexpr int kEqK = 8;  // chunks of 16 pixels per thread per round
constexpr int kEqSmem = kEqWarps * 256 * 4 * 4;

struct EqState {
  unsigned int gen, count, pad[2];
  unsigned int hist[2][256];
};

struct EqParams {
  ImgView in, out;
  EqState* st;
  int* err;
  long long n_chunks, per_cta;  // chunks in the image; chunks per CTA
  int cpr;                      // chunks per row
};

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int* a) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ int chunk_bytes(const EqParams& p, long long ch, const unsigned char** src,
                                           unsigned char** dst) {
  const int y = (int)(ch / p.cpr);
  const int x0 = (int)(ch - (long long)y * p.cpr) << 4;
  *src = (const unsigned char*)p.in.data + (long long)y * p.in.rs + x0;
  *dst = (unsigned char*)p.out.data + (long long)y * p.out.rs + x0;
  return min(16, p.in.w - x0);
}

__device__ __forceinline__ uint4 load_chunk(const unsigned char* src, int nb) {
  if (nb == 16) return __ldcs(reinterpret_cast<const uint4*>(src));
  unsigned int w[4] = {0u, 0u, 0u, 0u};
  for (int b = 0; b < nb; ++b) w[b >> 2] |= (unsigned int)src[b] << (8 * (b & 3));
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Counts a chunk into the lane's copy of the warp's sub-histogram: copy c of
// bin v is word 4 v + c, so lanes that hold the same value but use different
// copies hit different banks instead of serialising on one address.
__device__ __forceinline__ void count_chunk(unsigned int* wh, const uint4& q, int nb) {
  const unsigned int w[4] = {q.x, q.y, q.z, q.w};
  if (nb == 16) {
#pragma unroll
    for (int b = 0; b < 16; ++b) atomicAdd(&wh[((w[b >> 2] >> (8 * (b & 3))) & 0xffu) << 2], 1u);
  } else {
    for (int b = 0; b < nb; ++b) atomicAdd(&wh[((w[b >> 2] >> (8 * (b & 3))) & 0xffu) << 2], 1u);
  }
}

__device__ __forceinline__ void store_chunk(const unsigned char* t, const uint4& q, int nb, unsigned char* dst) {
  if (nb == 16) {
    __stcs(reinterpret_cast<uint4*>(dst), make_uint4(lut4(t, q.x), lut4(t, q.y), lut4(t, q.z), lut4(t, q.w)));
    return;
  }
  const unsigned int w[4] = {q.x, q.y, q.z, q.w};
  for (int b = 0; b < nb; ++b) dst[b] = t[(w[b >> 2] >> (8 * (b & 3))) & 0xffu];
}

__global__ void __launch_bounds__(kEqThreads, 1) k_histeq(const __grid_constant__ EqParams p) {
  extern __shared__ unsigned int sh_dyn[];  // per warp: 4 copies of 256 bins, interleaved
  unsigned int (*sh)[256 * 4] = reinterpret_cast<unsigned int (*)[256 * 4]>(sh_dyn);
  __shared__ unsigned char table[256];
  __shared__ unsigned int s_gen;
  __shared__ int s_last, s_ok;
  for (int i = threadIdx.x; i < kEqWarps * 256 * 4; i += blockDim.x) (&sh[0][0])[i] = 0;
  if (threadIdx.x == 0) s_gen = ld_relaxed(&p.st->gen);
  __syncthreads();
  const unsigned int gen = s_gen, buf = gen & 1u;
  unsigned int* wh = sh[threadIdx.x >> 5] + (threadIdx.x & 3);
  const long long c0 = (long long)blockIdx.x * p.per_cta;
  const long long c1 = min(p.n_chunks, c0 + p.per_cta);
  const long long round_span = (long long)kEqK * blockDim.x;
  const bool resident = c1 - c0 <= round_span;  // one round: the chunks stay in registers

  // ---- count ----
  uint4 q[kEqK];
  int nb[kEqK];
#pragma unroll
  for (int k = 0; k < kEqK; ++k) nb[k] = 0;
  for (long long base = c0; base < c1; base += round_span) {
#pragma unroll
    for (int k = 0; k < kEqK; ++k) {
      const long long ch = base + (long long)k * blockDim.x + threadIdx.x;
      nb[k] = 0;
      q[k] = make_uint4(0u, 0u, 0u, 0u);
      if (ch < c1) {
        const unsigned char* src;
        unsigned char* dst;
        nb[k] = chunk_bytes(p, ch, &src, &dst);
        q[k] = load_chunk(src, nb[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kEqK; ++k) count_chunk(wh, q[k], nb[k]);
  }
  __syncthreads();
  for (int v = threadIdx.x; v < 256; v += blockDim.x) {
    unsigned int s = 0;
    for (int w = 0; w < kEqWarps; ++w) s += sh[w][4 * v] + sh[w][4 * v + 1] + sh[w][4 * v + 2] + sh[w][4 * v + 3];
    if (s) atomicAdd(&p.st->hist[buf][v], s);
  }

  // ---- grid-wide barrier (bounded) ----
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&p.st->count, 1u) == gridDim.x - 1;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    // every CTA's counts are in: clear the other histogram and the counter for
    // the next launch, then release the others
    for (int v = threadIdx.x; v < 256; v += blockDim.x) p.st->hist[buf ^ 1u][v] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      p.st->count = 0;
      __threadfence();
      atomicExch(&p.st->gen, gen + 1u);
    }
  } else if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    while (ld_relaxed(&p.st->gen) == gen) {
      if (global_ns() - t0 > 1000000000ull) {
        s_ok = 0;
        atomicExch(p.err, 3);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  if (!s_ok) return;

  // ---- table, then the lookup ----
  cdf_lut_cta(threadIdx.x < 256 ? __ldcg(&p.st->hist[buf][threadIdx.x]) : 0u, table);
  __syncthreads();
  if (resident) {
#pragma unroll
    for (int k = 0; k < kEqK; ++k) {
      if (nb[k] == 0) continue;
      const long long ch = c0 + (long long)k * blockDim.x + threadIdx.x;
      const unsigned char* src;
      unsigned char* dst;
      chunk_bytes(p, ch, &src, &dst);
      store_chunk(table, q[k], nb[k], dst);
    }
    return;
  }
  for (long long ch = c0 + threadIdx.x; ch < c1; ch += blockDim.x) {
    const unsigned char* src;
    unsigned char* dst;
    const int n = chunk_bytes(p, ch, &src, &dst);
    store_chunk(table, load_chunk(src, n), n, dst);
  }
}

int max_coop_ctas() {
  static int n = 0;
  if (!n) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        allow_max_dynamic_smem((const void*)k_histeq) != 0 ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_histeq, kEqThreads, kEqSmem) != cudaSuccess || per < 1) {
      cudaGetLastError();
      return 152;
    }
    n = sms * per;
  }
  return n;
}

}  // namespace

size_t histeq_state_bytes() { return sizeof(EqState); }

// CTAs of the launch: one per 2048 chunks (32 KB of image), at most all
// co-resident ones.
int histeq_grid(int w, int h) {
  const long long chunks = (long long)((w + 15) / 16) * h;
  long long g = (chunks + 2047) / 2048;
  const int cap = max_coop_ctas();
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

int launch_histeq(const ImgView& in, const ImgView& out, void* state, int* err, int grid, void* stream) {
  static bool configured = false;
  if (!configured) {
    int e = allow_max_dynamic_smem((const void*)k_histeq);
    if (e) return e;
    configured = true;
  }
  EqParams p;
  p.in = in;
  p.out = out;
  p.st = reinterpret_cast<EqState*>(state);
  p.err = err;
  p.cpr = (in.w + 15) / 16;
  p.n_chunks = (long long)p.cpr * in.h;
  p.per_cta = (p.n_chunks + grid - 1) / grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kEqThreads, 1, 1);
  cfg.dynamicSmemBytes = kEqSmem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_histeq, p);
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)e;
}

}  // namespace hp
