// Fused stencil-chain kernel: d consecutive 5x5 separable stencil stages per
// output tile, the long-range fusion of the stencil chain (Sec. 2, Fig. 1).
//
// One CTA computes one T_w x T_h output tile of one channel.
//  1. Stage 0, the input tile plus a halo of 2d pixels per side, is loaded into
//     shared memory by TMA (cp.async.bulk.tensor, mbarrier completion); where
//     the alignment rules of TMA do not hold it is loaded with clamped
//     per-thread loads instead.
//  2. Stage s = 1..d is computed over its own rectangle, which shrinks by 2 per
//     side each stage (the overlapped-tile recompute of Fig. 1), from the
//     previous stage's buffer into the other buffer of a ping-pong pair.  Each
//     thread owns a 4-column block and sweeps down a segment of rows ("serial"
//     thread tiling, Sec. 2 and Sec. 4.1): every producer row is read once with
//     two 128-bit shared loads, its x pass is evaluated for the 4 columns and
//     kept in a 5-row register window, and the y pass of the window gives one
//     output row (producers staged in registers, Sec. 4.7).
//  3. Tiles that touch the image border replicate the edge of every stage into
//     the out-of-image part of its rectangle, so each stage reads its producer
//     with the clamp-to-edge boundary on the producer's own domain.
//  4. The last stage is written to global memory with 128-bit (f32) or 64-bit
//     (f16/bf16) coalesced stores; an optional unsharp epilogue combines it
//     with the chain's input.
// Every value uses the separable x-then-y fma chain of stage_math.cuh and is
// rounded to the stage's storage type, so the result is bit-identical to the
// stage-per-kernel schedule (which is this kernel with d = 1).
#include <cuda.h>
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

struct ChainGeom {
  int W0, H0;   // stage-0 rectangle
  int P;        // row pitch of both buffers (floats)
  int BH, nby;  // TMA box rows and boxes stacked along y
  int R;        // rows allocated per buffer
};

__host__ __device__ inline ChainGeom chain_geom(int depth, int tw, int th) {
  ChainGeom g;
  g.W0 = tw + 4 * depth;
  g.H0 = th + 4 * depth;
  g.P = ((g.W0 + 3) & ~3) + 4;
  g.BH = g.H0 < 256 ? g.H0 : 256;
  g.nby = (g.H0 + g.BH - 1) / g.BH;
  g.R = g.nby * g.BH;
  return g;
}

constexpr int kSmemHeader = 128;  // mbarrier + alignment slack

struct ChainKParams {
  CUtensorMap tmap;
  ChainArgs a;
  int use_tma;
};

template <int RND>
__device__ __forceinline__ float rnd(float v, int dtype) {
  if (RND == 0) return v;
  if (RND == 1) return __half2float(__float2half_rn(v));
  if (RND == 2) return __bfloat162float(__float2bfloat16_rn(v));
  return round_storage(dtype, v);
}

__device__ __forceinline__ float4 xpass(const float* p, const float* wx) {
  const float4 lo = *reinterpret_cast<const float4*>(p);
  const float4 hi = *reinterpret_cast<const float4*>(p + 4);
  float4 h;
  h.x = tap5(wx, lo.x, lo.y, lo.z, lo.w, hi.x);
  h.y = tap5(wx, lo.y, lo.z, lo.w, hi.x, hi.y);
  h.z = tap5(wx, lo.z, lo.w, hi.x, hi.y, hi.z);
  h.w = tap5(wx, lo.w, hi.x, hi.y, hi.z, hi.w);
  return h;
}

template <int RND>
__device__ __forceinline__ float4 ypass(const float* wy, const float4& a, const float4& b, const float4& c,
                                        const float4& d, const float4& e, int dtype) {
  float4 v;
  v.x = rnd<RND>(tap5(wy, a.x, b.x, c.x, d.x, e.x), dtype);
  v.y = rnd<RND>(tap5(wy, a.y, b.y, c.y, d.y, e.y), dtype);
  v.z = rnd<RND>(tap5(wy, a.z, b.z, c.z, d.z, e.z), dtype);
  v.w = rnd<RND>(tap5(wy, a.w, b.w, c.w, d.w, e.w), dtype);
  return v;
}

// Output sink of a sweep: a shared buffer, or the global output (last stage).
struct SmemSink {
  float* dst;
  int P;
  __device__ __forceinline__ void put(int b, int y, const float4& v) const {
    *reinterpret_cast<float4*>(dst + y * P + 4 * b) = v;
  }
};

struct GlobalSink {
  const ChainArgs* a;
  int ox, oy, ch;
  __device__ __forceinline__ void put(int b, int y, float4 v) const {
    const int gy = oy + y;
    const int gx = ox + 4 * b;
    if (gy >= a->out.h || gx >= a->out.w) return;
    const int odt = a->out.dtype;
    if (a->epilogue == 1) {
      float vin[4];
      for (int i = 0; i < 4; ++i) vin[i] = gx + i < a->in.w ? load_px(a->in, ch, gx + i, gy) : 0.0f;
      v.x = round_storage(odt, op_unsharp(vin[0], v.x, a->amount));
      v.y = round_storage(odt, op_unsharp(vin[1], v.y, a->amount));
      v.z = round_storage(odt, op_unsharp(vin[2], v.z, a->amount));
      v.w = round_storage(odt, op_unsharp(vin[3], v.w, a->amount));
    }
    char* row = (char*)a->out.data + (long long)ch * a->out.ps + (long long)gy * a->out.rs;
    if (gx + 3 < a->out.w) {
      if (odt == HP_F32) {
        *reinterpret_cast<float4*>(row + 4LL * gx) = v;
        return;
      }
      if (odt == HP_F16) {
        __half2 p0 = __floats2half2_rn(v.x, v.y), p1 = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&p0);
        u.y = *reinterpret_cast<unsigned*>(&p1);
        *reinterpret_cast<uint2*>(row + 2LL * gx) = u;
        return;
      }
      if (odt == HP_BF16) {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v.x, v.y), p1 = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&p0);
        u.y = *reinterpret_cast<unsigned*>(&p1);
        *reinterpret_cast<uint2*>(row + 2LL * gx) = u;
        return;
      }
    }
    const float vv[4] = {v.x, v.y, v.z, v.w};
    for (int i = 0; i < 4 && gx + i < a->out.w; ++i) store_px(a->out, ch, gx + i, gy, vv[i]);
  }
};

// One stage over a Ws x Hs rectangle: work items are (4-column block, row
// segment); the producer rectangle starts 2 columns and 2 rows further out, so
// output (x, y) reads producer rows y..y+4 and columns x..x+4 (rect-relative).
template <int RND, class Sink>
__device__ __forceinline__ void sweep(const float* __restrict__ src, int P, int Ws, int Hs, int seg,
                                      const float* wx, const float* wy, int dtype, const Sink& sink) {
  const int nb = Ws >> 2;
  const int nseg = (Hs + seg - 1) / seg;
  const int items = nb * nseg;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int sg = it / nb;
    const int b = it - sg * nb;
    const int r0 = sg * seg;
    const int r1 = min(Hs, r0 + seg);
    const float* p = src + r0 * P + 4 * b;
    float4 h0 = xpass(p, wx);
    float4 h1 = xpass(p + P, wx);
    float4 h2 = xpass(p + 2 * P, wx);
    float4 h3 = xpass(p + 3 * P, wx);
    float4 h4;
    p += 4 * P;
    int y = r0;
    // Five steps per iteration so the 5-row window rotates without moves.
    while (true) {
      h4 = xpass(p, wx); p += P;
      sink.put(b, y, ypass<RND>(wy, h0, h1, h2, h3, h4, dtype));
      if (++y >= r1) break;
      h0 = xpass(p, wx); p += P;
      sink.put(b, y, ypass<RND>(wy, h1, h2, h3, h4, h0, dtype));
      if (++y >= r1) break;
      h1 = xpass(p, wx); p += P;
      sink.put(b, y, ypass<RND>(wy, h2, h3, h4, h0, h1, dtype));
      if (++y >= r1) break;
      h2 = xpass(p, wx); p += P;
      sink.put(b, y, ypass<RND>(wy, h3, h4, h0, h1, h2, dtype));
      if (++y >= r1) break;
      h3 = xpass(p, wx); p += P;
      sink.put(b, y, ypass<RND>(wy, h4, h0, h1, h2, h3, dtype));
      if (++y >= r1) break;
    }
  }
}

template <class Sink>
__device__ __forceinline__ void sweep_any(int rkind, const float* src, int P, int Ws, int Hs, int seg,
                                          const float* wx, const float* wy, int dtype, const Sink& sink) {
  switch (rkind) {
    case 0: sweep<0>(src, P, Ws, Hs, seg, wx, wy, dtype, sink); break;
    case 1: sweep<1>(src, P, Ws, Hs, seg, wx, wy, dtype, sink); break;
    case 2: sweep<2>(src, P, Ws, Hs, seg, wx, wy, dtype, sink); break;
    default: sweep<3>(src, P, Ws, Hs, seg, wx, wy, dtype, sink); break;
  }
}

// Replicates the in-image edge of a stage rectangle (origin (x0, y0) in image
// coordinates, Ws x Hs) into its out-of-image part.
__device__ void fixup(float* buf, int P, int x0, int y0, int Ws, int Hs, int W, int H) {
  const int cx0 = max(0, -x0), cx1 = min(Ws, W - x0);
  const int cy0 = max(0, -y0), cy1 = min(Hs, H - y0);
  const int band_rows = cy0 + (Hs - cy1);
  const int n1 = band_rows * Ws;
  const int side = cx0 + (Ws - cx1);
  const int n2 = (cy1 - cy0) * side;
  for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
    int x, y;
    if (i < n1) {
      int r = i / Ws;
      x = i - r * Ws;
      y = r < cy0 ? r : cy1 + (r - cy0);
    } else {
      int j = i - n1;
      int r = j / side;
      int k = j - r * side;
      y = cy0 + r;
      x = k < cx0 ? k : cx1 + (k - cx0);
    }
    buf[y * P + x] = buf[min(max(y, cy0), cy1 - 1) * P + min(max(x, cx0), cx1 - 1)];
  }
}

__device__ __forceinline__ int rkind_of(int dtype) {
  return dtype == HP_F32 ? 0 : dtype == HP_F16 ? 1 : dtype == HP_BF16 ? 2 : 3;
}

__global__ void __launch_bounds__(512) k_chain(const __grid_constant__ ChainKParams kp) {
  const ChainArgs& a = kp.a;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base);
  const int d = a.depth;
  const ChainGeom g = chain_geom(d, a.tile_w, a.tile_h);
  float* bufA = reinterpret_cast<float*>(base + kSmemHeader);
  float* bufB = bufA + g.P * g.R;
  const int ch = blockIdx.z;
  const int ox = blockIdx.x * a.tile_w, oy = blockIdx.y * a.tile_h;
  const int W = a.in.w, H = a.in.h;
  const int xin = ox - 2 * d, yin = oy - 2 * d;
  const bool border = xin < 0 || yin < 0 || xin + g.W0 > W || yin + g.H0 > H;

  // ---- stage 0: input tile + halo ----
  if (kp.use_tma) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(bar, (unsigned)(g.nby * g.BH * g.P * 4));
      for (int k = 0; k < g.nby; ++k) tma_load_3d(bufA + k * g.BH * g.P, &kp.tmap, xin, yin + k * g.BH, ch, bar);
    }
    if (!mbar_wait_bounded(bar, 0, 1u << 26)) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      return;
    }
    if (border) {
      fixup(bufA, g.P, xin, yin, g.W0, g.H0, W, H);
    }
  } else {
    const int n = g.W0 * g.H0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int y = i / g.W0;
      int x = i - y * g.W0;
      bufA[y * g.P + x] = load_px(a.in, ch, iclamp(xin + x, 0, W - 1), iclamp(yin + y, 0, H - 1));
    }
  }
  __syncthreads();

  // ---- stages 1..d ----
  for (int s = 1; s <= d; ++s) {
    const float* src = (s & 1) ? bufA : bufB;
    float* dst = (s & 1) ? bufB : bufA;
    const int Ws = a.tile_w + 4 * (d - s);
    const int Hs = a.tile_h + 4 * (d - s);
    float wx[5], wy[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      wx[k] = a.w[s - 1][k];
      wy[k] = a.w[s - 1][5 + k];
    }
    const int dt = a.storage[s - 1];
    const int rk = rkind_of(dt);
    if (s < d) {
      sweep_any(rk, src, g.P, Ws, Hs, a.seg, wx, wy, dt, SmemSink{dst, g.P});
      if (border) {
        __syncthreads();
        fixup(dst, g.P, ox - 2 * (d - s), oy - 2 * (d - s), Ws, Hs, W, H);
      }
      __syncthreads();
    } else {
      sweep_any(rk, src, g.P, Ws, Hs, a.seg, wx, wy, dt, GlobalSink{&a, ox, oy, ch});
    }
  }
}

}  // namespace

int chain_smem_bytes(int depth, int tile_w, int tile_h, int in_dtype) {
  (void)in_dtype;
  ChainGeom g = chain_geom(depth, tile_w, tile_h);
  return kSmemHeader + 128 + 2 * g.P * g.R * 4;
}

int launch_chain(const ChainArgs& a, int smem_bytes, void* stream) {
  static bool configured = false;
  if (smem_bytes > 48 * 1024 && !configured) {
    int e = allow_max_dynamic_smem((const void*)k_chain);
    if (e) return e;
    configured = true;
  }
  ChainKParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  ChainGeom g = chain_geom(a.depth, a.tile_w, a.tile_h);
  kp.use_tma = a.in.dtype == HP_F32 && (2 * a.depth * 4) % 16 == 0 && g.P <= 256 && g.BH <= 256;
  if (kp.use_tma) {
    int e = encode_tmap_3d(&kp.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs,
                           a.in.ps, g.P, g.BH);
    if (e) kp.use_tma = 0;  // fall back to clamped loads
  }
  dim3 grid(a.tiles_x, a.tiles_y, a.in.c);
  k_chain<<<grid, a.threads, smem_bytes, (cudaStream_t)stream>>>(kp);
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
