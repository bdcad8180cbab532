// Histogram equalization of a u8 image in one cooperative kernel: the image is
// read from memory once and written once.
//
// Each CTA takes a contiguous range of 16-pixel chunks (row-major over the
// image, a row's last chunk possibly partial), keeps them in shared memory
// while it counts them into a lane-private histogram: counter (v, l) is word
// 32 v + l, so the 32 lanes of a shared-memory atomic always hit 32 different
// banks and never the same address, whatever the values (a low-contrast image
// puts most lanes of a warp on a few values).  The loops stay compact: each
// runs once or twice per thread, so its code must not be long (the instruction
// cache is cold).  The CTA adds its counts to a device-wide histogram with
// one atomic per bin, then all CTAs meet at a grid-wide barrier -- they are
// co-resident because the launch is cooperative, and the wait is bounded --
// after which every CTA forms the CDF and the table itself (256 bins: cheaper
// than another launch) and writes its equalized chunks.  When a CTA's slice
// does not fit in shared memory it reads its chunks again for the lookup.
//
// The device-wide state (two histograms of kEqCopies copies each -- CTA b adds
// into copy b % kEqCopies, so no counter takes more than a few atomics -- an
// arrival counter per launch parity and the launch number g) lives in a
// zero-initialised scratch that resets itself: launch g counts into histogram
// g & 1 and arrives at counter g & 1, and every CTA waits for that counter to
// reach the CTA count.  The last CTA to arrive advances g and clears the other
// parity's counter and histogram, which nothing reads in this launch, so the
// next launch (a CUDA-graph replay included) starts clean.
#include <cuda_runtime.h>

#include "hist_common.cuh"
#include "hp_internal.h"
#include "tma.cuh"

namespace hp {

namespace {

constexpr int kEqThreads = 1024;
constexpr int kEqU = 6;  // chunk loads in flight per thread
constexpr int kEqHistBytes = 256 * 32 * 4;               // 256 bins x 32 lanes
constexpr int kEqSmemMax = 227 * 1024 - 8 * 1024;        // dynamic shared memory limit used here
constexpr int kEqStageMax = kEqSmemMax - kEqHistBytes;    // bytes of image a CTA can keep

constexpr int kEqCopies = 8;  // device histogram copies (CTA b adds into copy b % 8)

struct EqState {
  unsigned int gen, count[2], pad;  // launch number; arrivals of the launches of each parity
  unsigned int hist[2][kEqCopies][256];
};

struct EqParams {
  ImgView in, out;
  EqState* st;                  // one state per image of the batch
  int* err;
  unsigned int n_chunks, per_cta;  // chunks in an image (< 2^32: at most its pixels); chunks per CTA
  FastDiv cpr;                     // chunks per row (the divisor of a chunk index)
  int staged;                   // per_cta chunks fit in shared memory: no second read
  int ctas;                     // CTAs per image (a batch's images take consecutive groups of CTAs)
};

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int* a) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ int chunk_bytes(const EqParams& p, int img, unsigned int ch, const unsigned char** src,
                                           unsigned char** dst) {
  const unsigned int y = fastdiv(ch, p.cpr);
  const int x0 = (int)(ch - y * p.cpr.d) << 4;
  *src = (const unsigned char*)p.in.data + (long long)img * p.in.ps + (long long)y * p.in.rs + x0;
  *dst = (unsigned char*)p.out.data + (long long)img * p.out.ps + (long long)y * p.out.rs + x0;
  return min(16, p.in.w - x0);
}

__device__ __forceinline__ uint4 load_chunk(const unsigned char* src, int nb) {
  if (nb == 16) return __ldcs(reinterpret_cast<const uint4*>(src));
  uint4 q = make_uint4(0u, 0u, 0u, 0u);
  for (int b = 0; b < nb; ++b) {
    const unsigned int v = (unsigned int)src[b] << (8 * (b & 3));
    if (b < 4) q.x |= v;
    else if (b < 8) q.y |= v;
    else if (b < 12) q.z |= v;
    else q.w |= v;
  }
  return q;
}

// Word b / 4 of a chunk without indexing a local array (a partial chunk's
// loop index is not a compile-time constant).
__device__ __forceinline__ unsigned int word_of(const uint4& q, int b) {
  return b < 8 ? (b < 4 ? q.x : q.y) : (b < 12 ? q.z : q.w);
}

// Counts a chunk into the lane's column (hl = hist + lane) of the CTA's
// lane-private histogram: bin v of this lane is word 32 v.
__device__ __forceinline__ void count_chunk(unsigned int* hl, const uint4& q, int nb) {
  const unsigned int w[4] = {q.x, q.y, q.z, q.w};
  if (nb == 16) {
#pragma unroll
    for (int b = 0; b < 16; ++b) atomicAdd(&hl[((w[b >> 2] >> (8 * (b & 3))) & 0xffu) << 5], 1u);
  } else {
    for (int b = 0; b < nb; ++b) atomicAdd(&hl[((word_of(q, b) >> (8 * (b & 3))) & 0xffu) << 5], 1u);
  }
}

__device__ __forceinline__ void store_chunk(const unsigned char* t, const uint4& q, int nb, unsigned char* dst) {
  if (nb == 16) {
    __stcs(reinterpret_cast<uint4*>(dst), make_uint4(lut4(t, q.x), lut4(t, q.y), lut4(t, q.z), lut4(t, q.w)));
    return;
  }
  for (int b = 0; b < nb; ++b) dst[b] = t[(word_of(q, b) >> (8 * (b & 3))) & 0xffu];
}

__global__ void __launch_bounds__(kEqThreads, 1) k_histeq(const __grid_constant__ EqParams p) {
  // dynamic shared memory: the lane-private histogram, then (when the slice
  // fits) the CTA's slice of the image
  extern __shared__ uint4 smem_dyn[];
  unsigned int* sh = reinterpret_cast<unsigned int*>(smem_dyn);
  uint4* stage = smem_dyn + kEqHistBytes / 16;
  __shared__ unsigned char table[256];
  __shared__ unsigned int s_gen;
  __shared__ int s_last, s_ok;
  // image of the batch and this CTA's place among the image's CTAs
  const int img = blockIdx.x / p.ctas, cta = blockIdx.x - img * p.ctas;
  EqState* const st = p.st + img;
  for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) sh[i] = 0;
  if (threadIdx.x == 0) s_gen = ld_relaxed(&st->gen);
  __syncthreads();
  const unsigned int gen = s_gen, buf = gen & 1u;
  unsigned int* hl = sh + (threadIdx.x & 31);
  const unsigned int c0 = (unsigned int)cta * p.per_cta;
  const unsigned int c1 = (unsigned int)min((unsigned long long)p.n_chunks, (unsigned long long)c0 + p.per_cta);
  const bool staged = p.staged != 0;  // the slice is kept in shared memory for the lookup

  // ---- count (kEqU loads in flight per thread) ----
  const unsigned int step = kEqU * blockDim.x;
#pragma unroll 1
  for (unsigned int base = c0 + threadIdx.x; base < c1; base += step) {
    uint4 q[kEqU];
    int nb[kEqU];
#pragma unroll
    for (int u = 0; u < kEqU; ++u) {
      const unsigned int ch = base + u * blockDim.x;
      nb[u] = 0;
      if (ch < c1) {
        const unsigned char* src;
        unsigned char* dst;
        nb[u] = chunk_bytes(p, img, ch, &src, &dst);
        q[u] = load_chunk(src, nb[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kEqU; ++u) {
      if (nb[u] == 0) continue;
      if (staged) stage[base + u * blockDim.x - c0] = q[u];
      count_chunk(hl, q[u], nb[u]);
    }
  }
  __syncthreads();
  {
    // all threads reduce: thread t sums bin t / 4 over 8 of the 32 lane
    // columns (8 (t % 4) .. 8 (t % 4) + 7, visited from a bin-dependent start
    // so that a warp's reads hit 32 different banks); the four partial sums of
    // a bin are adjacent lanes and are added by shuffles
    const int v = threadIdx.x >> 2, part = threadIdx.x & 3;
    const unsigned int* row = sh + v * 32 + 8 * part;
    unsigned int s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += row[(j + v) & 7];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0 && s) atomicAdd(&st->hist[buf][cta % kEqCopies][v], s);
  }

  // ---- grid-wide barrier (bounded) ----
  __syncthreads();
  if (threadIdx.x == 0) {
    // arrive, then wait until every CTA of this launch has: the barrier is
    // the arrival counter itself (no CTA has to release the others)
    __threadfence();
    const unsigned int need = (unsigned)p.ctas;
    const bool last = atomicAdd(&st->count[buf], 1u) == need - 1;
    s_last = last;
    s_ok = 1;
    if (!last) {
      const unsigned long long t0 = global_ns();
      while (ld_relaxed(&st->count[buf]) < need) {
        if (global_ns() - t0 > 1000000000ull) {
          s_ok = 0;
          atomicExch(p.err, 3);
          break;
        }
      }
    } else {
      // the next launch (parity buf ^ 1) finds its counter and histogram
      // zero and the launch number advanced; nothing in this launch reads them
      st->count[buf ^ 1u] = 0;
      st->gen = gen + 1u;
    }
    __threadfence();
  }
  __syncthreads();
  if (!s_ok) return;
  if (s_last)  // the other histogram, for the next launch
    for (int v = threadIdx.x; v < kEqCopies * 256; v += blockDim.x) (&st->hist[buf ^ 1u][0][0])[v] = 0;

  // ---- table, then the lookup ----
  unsigned int h = 0;
  if (threadIdx.x < 256)
#pragma unroll
    for (int c = 0; c < kEqCopies; ++c) h += __ldcg(&st->hist[buf][c][threadIdx.x]);
  cdf_lut_cta(h, table);
  __syncthreads();
  // two chunks per iteration, so that each thread has two independent
  // lookups in flight
#pragma unroll 1
  for (unsigned int base = c0 + threadIdx.x; base < c1; base += 2 * blockDim.x) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const unsigned int ch = base + u * blockDim.x;
      if (ch < c1) {
        const unsigned char* src;
        unsigned char* dst;
        const int n = chunk_bytes(p, img, ch, &src, &dst);
        store_chunk(table, staged ? stage[ch - c0] : load_chunk(src, n), n, dst);
      }
    }
  }
}

int max_coop_ctas() {
  static int n = 0;
  if (!n) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        allow_max_dynamic_smem((const void*)k_histeq) != 0 ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_histeq, kEqThreads, kEqSmemMax) != cudaSuccess ||
        per < 1) {
      cudaGetLastError();
      return 152;
    }
    n = sms * per;
  }
  return n;
}

}  // namespace

size_t histeq_state_bytes() { return sizeof(EqState); }  // per image of a batch

// CTAs per image: one per 2048 chunks (32 KB of image), at most the
// co-resident ones shared by the batch's images.
int histeq_grid(int w, int h, int batch) {
  const long long chunks = (long long)((w + 15) / 16) * h;
  long long g = (chunks + 2047) / 2048;
  const int cap = max_coop_ctas() / (batch > 1 ? batch : 1);
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

// grid: CTAs per image (histeq_grid); the launch has grid x batch CTAs, all
// co-resident (cooperative).
int launch_histeq(const ImgView& in, const ImgView& out, void* state, int* err, int grid, int batch, void* stream) {
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
  const unsigned long long n_chunks = (unsigned long long)((in.w + 15) / 16) * in.h;
  // 32-bit chunk indices, with room for a thread's last stride past the end
  // (the counters hold at most 2^32 - 1 pixels anyway)
  if (n_chunks > 0xffffffffull - 65536 || in.w < 1) return (int)cudaErrorInvalidValue;
  p.cpr = make_fastdiv((unsigned int)((in.w + 15) / 16));
  p.n_chunks = (unsigned int)n_chunks;
  p.per_cta = (unsigned int)((n_chunks + grid - 1) / grid);
  p.staged = (unsigned long long)p.per_cta * 16 <= (unsigned long long)kEqStageMax;
  p.ctas = grid;
  if (batch < 1) batch = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid * batch, 1, 1);
  cfg.blockDim = dim3(kEqThreads, 1, 1);
  cfg.dynamicSmemBytes = kEqHistBytes + (p.staged ? (int)p.per_cta * 16 : 0);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (t_probe) probe_kernel((const void*)k_histeq);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_histeq, p);
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)e;
}

}  // namespace hp
