// Histogram equalization kernels: a 256-bin histogram of a u8 image, the CDF
// scan and equalization lookup table, and the table lookup.
//
// Histogram: the parallel reduction the paper's histogram-equalize discussion
// calls for (atomics expose the data parallelism, Sec. 6.5 and Sec. 8).  Each
// warp keeps a private sub-histogram in shared memory and adds each byte with
// a shared-memory atomic; when every active lane of the warp holds the same
// value (flat regions, constant images: the worst case for contention) the
// warp aggregates and one lane adds the whole count.  The CTA's sub-histograms
// are summed and added to the global counters with one atomic per bin.  Each
// thread loads 4 x 16 bytes before counting so enough reads are in flight to
// keep HBM busy.  All counts are exact integers.
#include <cuda_runtime.h>

#include <mutex>

#include "hist_common.cuh"
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kHistThreads = 512;
constexpr int kHistWarps = kHistThreads / 32;

constexpr int kChunksPerIter = 4;

// cpr: the chunks per row (16-byte chunks); chunk indices are 32-bit (the
// host checks that the image's chunks fit).
__global__ void __launch_bounds__(kHistThreads) k_hist(const ImgView in, const FastDiv cpr, unsigned int* __restrict__ hist) {
  grid_dep_sync();
  __shared__ unsigned int sh[kHistWarps][256];
  for (int i = threadIdx.x; i < kHistWarps * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  unsigned int* wh = sh[threadIdx.x >> 5];
  const unsigned int n_chunks = cpr.d * (unsigned int)in.h;
  // a warp takes 32 x kChunksPerIter consecutive chunks per iteration; the
  // loop bound is warp-uniform, so the warp-wide votes below are legal
  const unsigned int per_iter = gridDim.x * blockDim.x * kChunksPerIter;
  const unsigned int warp_base = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * kChunksPerIter;
  const int lane = threadIdx.x & 31;
  for (unsigned int base = warp_base; base < n_chunks; base += per_iter) {
    unsigned int words[kChunksPerIter][4];
    int nbytes[kChunksPerIter];
#pragma unroll
    for (int u = 0; u < kChunksPerIter; ++u) {
      const unsigned int ch = base + u * 32 + lane;
      words[u][0] = words[u][1] = words[u][2] = words[u][3] = 0;
      nbytes[u] = 0;
      if (ch < n_chunks) {
        const unsigned int y = fastdiv(ch, cpr);
        const int x0 = (int)(ch - y * cpr.d) << 4;
        const unsigned char* row = (const unsigned char*)in.data + (long long)y * in.rs;
        nbytes[u] = min(16, in.w - x0);
        if (nbytes[u] == 16) {
          const uint4 q = __ldcs(reinterpret_cast<const uint4*>(row + x0));
          words[u][0] = q.x; words[u][1] = q.y; words[u][2] = q.z; words[u][3] = q.w;
        } else {
#pragma unroll
          for (int b = 0; b < 16; ++b)
            if (b < nbytes[u]) words[u][b >> 2] |= (unsigned int)row[x0 + b] << (8 * (b & 3));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kChunksPerIter; ++u) {
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        const unsigned int active = __ballot_sync(0xffffffffu, b < nbytes[u]);
        if (b < nbytes[u]) count_byte(wh, (words[u][b >> 2] >> (8 * (b & 3))) & 0xffu, active);
      }
    }
  }
  __syncthreads();
  for (int v = threadIdx.x; v < 256; v += blockDim.x) {
    unsigned int s = 0;
    for (int w = 0; w < kHistWarps; ++w) s += sh[w][v];
    if (s) atomicAdd(&hist[v], s);
  }
}

// One CTA of 256 threads: the CDF and the equalization table.
__global__ void __launch_bounds__(256) k_cdf_lut(const unsigned int* __restrict__ hist, unsigned char* __restrict__ lut) {
  grid_dep_sync();
  cdf_lut_cta(hist[threadIdx.x], lut);
}

__global__ void __launch_bounds__(256) k_lut_apply(const ImgView in, const ImgView out, const FastDiv cpr,
                                                   const unsigned char* __restrict__ lut) {
  grid_dep_sync();
  __shared__ unsigned char t[256];
  if (threadIdx.x < 256) t[threadIdx.x] = lut[threadIdx.x];
  __syncthreads();
  const unsigned int n_chunks = cpr.d * (unsigned int)in.h;
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int c0 = blockIdx.x * blockDim.x + threadIdx.x; c0 < n_chunks; c0 += stride * kChunksPerIter) {
    uint4 q[kChunksPerIter];
    int nb[kChunksPerIter];
    unsigned int chs[kChunksPerIter];
#pragma unroll
    for (int u = 0; u < kChunksPerIter; ++u) {
      const unsigned int ch = c0 + u * stride;
      chs[u] = ch;
      nb[u] = 0;
      if (ch < n_chunks) {
        const unsigned int y = fastdiv(ch, cpr);
        const int x0 = (int)(ch - y * cpr.d) << 4;
        nb[u] = min(16, in.w - x0);
        if (nb[u] == 16) q[u] = __ldcs(reinterpret_cast<const uint4*>((const unsigned char*)in.data + (long long)y * in.rs + x0));
      }
    }
#pragma unroll
    for (int u = 0; u < kChunksPerIter; ++u) {
      if (nb[u] == 0) continue;
      const unsigned int ch = chs[u];
      const unsigned int y = fastdiv(ch, cpr);
      const int x0 = (int)(ch - y * cpr.d) << 4;
      unsigned char* dst = (unsigned char*)out.data + (long long)y * out.rs + x0;
      if (nb[u] == 16) {
        __stcs(reinterpret_cast<uint4*>(dst), make_uint4(lut4(t, q[u].x), lut4(t, q[u].y), lut4(t, q[u].z), lut4(t, q[u].w)));
      } else {
        const unsigned char* src = (const unsigned char*)in.data + (long long)y * in.rs + x0;
        for (int b = 0; b < nb[u]; ++b) dst[b] = t[src[b]];
      }
    }
  }
}

// Chunk indices are 32-bit, with room for a thread's last stride past the end
// (at most 8 x 152 x 256 x 4 chunks); a histogram counts at most 2^32 - 1
// pixels anyway.
bool chunks_fit(long long chunks) { return chunks >= 0 && chunks <= 0xffffffffLL - (1LL << 24); }

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

int launch_hist(const HistArgs& a, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int e = (int)cudaMemsetAsync(a.hist, 0, 256 * sizeof(unsigned int), s);
  if (e) return e;
  long long chunks = (long long)((a.in.w + 15) / 16) * a.in.h;
  if (!chunks_fit(chunks)) return (int)cudaErrorInvalidValue;
  long long want = (chunks + kHistThreads * kChunksPerIter - 1) / (kHistThreads * kChunksPerIter);
  int blocks = (int)(want < 4LL * sm_count() ? want : 4LL * sm_count());
  if (blocks < 1) blocks = 1;
  const FastDiv cpr = make_fastdiv((unsigned int)((a.in.w + 15) / 16));
  { const int le_ = launch_kernel(k_hist, dim3(blocks), dim3(kHistThreads), 0, (void*)s, a.in, cpr, a.hist); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

int launch_cdf_lut(const LutArgs& a, void* stream) {
  { const int le_ = launch_kernel(k_cdf_lut, dim3(1), dim3(256), 0, stream, a.hist, a.lut); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

int launch_lut_apply(const LutApplyArgs& a, void* stream) {
  long long chunks = (long long)((a.in.w + 15) / 16) * a.in.h;
  if (!chunks_fit(chunks)) return (int)cudaErrorInvalidValue;
  long long want = (chunks + 256 * kChunksPerIter - 1) / (256 * kChunksPerIter);
  int blocks = (int)(want < 8LL * sm_count() ? want : 8LL * sm_count());
  if (blocks < 1) blocks = 1;
  const FastDiv cpr = make_fastdiv((unsigned int)((a.in.w + 15) / 16));
  { const int le_ = launch_kernel(k_lut_apply, dim3(blocks), dim3(256), 0, stream, a.in, a.out, cpr, a.lut); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp

// ---------------------------------------------------------------------------
// Allocation-free histogram equalization.
//
// Some callers cannot allocate device memory at the time they run a pipeline:
// a host framework that owns every byte of device memory through its own pool
// and forbids cudaMalloc from plugins, a real-time or serving loop that must
// not block (cudaMalloc can synchronise the device) or fail under memory
// pressure, or a deployment that reserves all memory once at start-up.  For
// them this entry point equalizes one u8 image with the three kernels above,
// taking its scratch -- the 256 histogram counters and the 256-entry table --
// from a fixed array in the library's device image instead of from an
// allocation.  The paper has no counterpart: it is a property of this library.
// ---------------------------------------------------------------------------
namespace hp {
namespace {

constexpr int kNoallocCounterBytes = 256 * 4;
constexpr int kNoallocBytes = kNoallocCounterBytes + 256;  // counters, then the LUT
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds these 1280 bytes until the process
// exits.  All calls share them: calls that overlap on the GPU race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

void* g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

}  // namespace

}  // namespace hp

extern "C" hp_status hp_histeq_u8_noalloc(const hp_buffer* input, const hp_buffer* output, void* stream) {
  using namespace hp;
  if (!input || !output || !input->data || !output->data)
    return report_error(HP_ERR_INVALID_ARG, "hp_histeq_u8_noalloc: null buffer");
  const hp_buffer* bufs[2] = {input, output};
  for (const hp_buffer* b : bufs) {
    if (b->dtype != HP_U8 || b->channels != 1)
      return report_error(HP_ERR_INVALID_ARG, "hp_histeq_u8_noalloc: buffers must be 1-channel u8");
    if (b->width < 1 || b->height < 1)
      return report_error(HP_ERR_INVALID_ARG, "hp_histeq_u8_noalloc: empty image");
    if (((uintptr_t)b->data & 15) || b->row_stride_bytes % 16 || b->row_stride_bytes < b->width)
      return report_error(HP_ERR_INVALID_ARG,
                          "hp_histeq_u8_noalloc: data must be 16-byte aligned and rows a multiple of 16 bytes");
  }
  if (input->width != output->width || input->height != output->height)
    return report_error(HP_ERR_INVALID_ARG, "hp_histeq_u8_noalloc: input and output sizes differ");
  if ((unsigned long long)input->width * (unsigned long long)input->height > HP_NOALLOC_MAX_PIXELS)
    return report_error(HP_ERR_INVALID_ARG,
                        "hp_histeq_u8_noalloc: image larger than HP_NOALLOC_MAX_PIXELS (the 32-bit counters)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return report_error(HP_ERR_CUDA, "hp_histeq_u8_noalloc: no usable current device");
  }
  void* base = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name of
    // the array is not a device address, so ask the runtime for the address
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return report_error(HP_ERR_CUDA, "hp_histeq_u8_noalloc: cudaGetSymbolAddress of the scratch array failed");
      }
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  ImgView in{}, out{};
  in.data = input->data; in.dtype = HP_U8; in.c = 1; in.w = input->width; in.h = input->height;
  in.rs = input->row_stride_bytes; in.ps = input->plane_stride_bytes;
  out.data = output->data; out.dtype = HP_U8; out.c = 1; out.w = output->width; out.h = output->height;
  out.rs = output->row_stride_bytes; out.ps = output->plane_stride_bytes;
  unsigned int* hist = reinterpret_cast<unsigned int*>(base);
  unsigned char* lut = reinterpret_cast<unsigned char*>(base) + kNoallocCounterBytes;
  HistArgs ha{};
  ha.in = in;
  ha.hist = hist;  // launch_hist clears the counters on the stream before counting
  int e = launch_hist(ha, stream);
  if (!e) {
    LutArgs la{};
    la.hist = hist;
    la.lut = lut;
    e = launch_cdf_lut(la, stream);
  }
  if (!e) {
    LutApplyArgs aa{};
    aa.in = in;
    aa.out = out;
    aa.lut = lut;
    e = launch_lut_apply(aa, stream);
  }
  if (e) return report_error(HP_ERR_CUDA, cudaGetErrorString((cudaError_t)e));
  return HP_OK;
}
