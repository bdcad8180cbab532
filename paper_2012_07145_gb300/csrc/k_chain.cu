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
//  4. The last stage goes straight from the y pass to global memory, one
//     128-bit (f32) or 64-bit (f16/bf16) store per 4-column row; with the
//     optional unsharp epilogue it is staged in shared memory and combined
//     with the chain's input on the way out.
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
  int buf;      // floats per buffer (a multiple of 32, so buffer B stays 128-byte aligned)
};

__host__ __device__ inline ChainGeom chain_geom(int depth, int tw, int th) {
  ChainGeom g;
  g.W0 = tw + 4 * depth;
  g.H0 = th + 4 * depth;
  g.P = (g.W0 + 3) & ~3;
  g.BH = g.H0 < 256 ? g.H0 : 256;
  g.nby = (g.H0 + g.BH - 1) / g.BH;
  // rows: the stacked TMA boxes, and the overshoot of a last row segment
  // (segments of up to 16 rows read 4 rows further)
  const int r_seg = ((g.H0 + 15) & ~15) + 4;
  g.R = g.nby * g.BH > r_seg ? g.nby * g.BH : r_seg;
  g.buf = (g.P * g.R + 31) & ~31;
  return g;
}

constexpr int kSmemHeader = 128;  // mbarrier, status word, alignment slack

// How stage 0 reaches shared memory.
enum { kLoadClamped = 0, kLoadTmaDirect = 1, kLoadTmaStaged = 2 };

struct ChainKParams {
  CUtensorMap tmap;
  ChainArgs a;
  int load_mode;
  int off;   // staged: column of the image's x = xin inside the staged box
  int sbw;   // staged: box width in elements
};

template <int RND>
__device__ __forceinline__ float rnd(float v, int dtype) {
  if (RND == 0) return v;
  if (RND == 1) return __half2float(__float2half_rn(v));
  if (RND == 2) return __bfloat162float(__float2bfloat16_rn(v));
  return round_storage(dtype, v);
}

// x pass of one producer row for 4 output columns.  (The paired FP32
// instructions of sm_100 were measured slower here: they issue on one FMA pipe
// only, and the x pass would need register moves to form its pairs.)
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

// Output sink of a sweep: the stage's shared buffer.
struct SmemSink {
  float* dst;
  int P;
  __device__ __forceinline__ void put(int b, int y, const float4& v) const {
    *reinterpret_cast<float4*>(dst + y * P + 4 * b) = v;
  }
};

// Output sink of the last stage (no epilogue): the output image, rows and
// columns past the tile or the image dropped.
template <int ODT>
struct GlobalSink {
  char* plane;
  long long rs;
  int ox, oy, th, tw, W, H;
  const ImgView* out;
  int ch;
  __device__ __forceinline__ void put(int b, int y, const float4& v) const {
    if (y >= th || oy + y >= H) return;
    const int x = 4 * b, gx = ox + x;
    char* row = plane + (long long)(oy + y) * rs;
    if (ODT != 3 && x + 3 < tw && gx + 3 < W) {
      if (ODT == 0) {
        *reinterpret_cast<float4*>(row + 4LL * gx) = v;
      } else {
        uint2 u;
        if (ODT == 1) {
          __half2 p0 = __floats2half2_rn(v.x, v.y), p1 = __floats2half2_rn(v.z, v.w);
          u.x = *reinterpret_cast<unsigned*>(&p0);
          u.y = *reinterpret_cast<unsigned*>(&p1);
        } else {
          __nv_bfloat162 p0 = __floats2bfloat162_rn(v.x, v.y), p1 = __floats2bfloat162_rn(v.z, v.w);
          u.x = *reinterpret_cast<unsigned*>(&p0);
          u.y = *reinterpret_cast<unsigned*>(&p1);
        }
        *reinterpret_cast<uint2*>(row + 2LL * gx) = u;
      }
    } else {
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (x + k < tw && gx + k < W) store_px(*out, ch, gx + k, oy + y, vv[k]);
    }
  }
};

// One stage over a Ws x Hs rectangle: work items are (4-column block, row
// segment of SEG rows); the producer rectangle starts 2 columns and 2 rows
// further out, so output (x, y) reads producer rows y..y+4 and columns x..x+4
// (rect-relative).  The segment is unrolled completely: SEG + 4 producer rows
// each get one x pass, kept in a 5-row register window for the y passes.  The
// last segment may run past Hs; those rows are computed from rows that exist
// in the buffer (it is allocated for that) and are never read by valid outputs.
template <int SEG, int RND, class Sink>
__device__ __forceinline__ void sweep(const float* __restrict__ src, int P, int Ws, int Hs,
                                      const float* wx, const float* wy, int dtype, const Sink& sink) {
  const int nb = Ws >> 2;
  const int nseg = (Hs + SEG - 1) / SEG;
  const int items = nb * nseg;
  // it / nb as a float product: (it + 0.5) / nb lies at least 0.5 / nb from an
  // integer, and the product (a correctly rounded reciprocal, one rounding)
  // is off by less than (it / nb) 2^-22, which is smaller for every it below
  // 2^21 (a tile has fewer than 2^12 items); the truncation is the exact quotient
  const float rnb = __frcp_rn((float)nb);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int sg = (int)(((float)it + 0.5f) * rnb);
    const int b = it - sg * nb;
    const int r0 = sg * SEG;
    const float* p = src + r0 * P + 4 * b;
    float4 h[SEG + 4];
#pragma unroll
    for (int k = 0; k < SEG + 4; ++k) {
      h[k] = xpass(p + k * P, wx);
      if (k >= 4) sink.put(b, r0 + k - 4, ypass<RND>(wy, h[k - 4], h[k - 3], h[k - 2], h[k - 1], h[k], dtype));
    }
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

__device__ __forceinline__ float staged_value(const unsigned char* st, int idx, int dtype) {
  if (dtype == HP_F16) return __half2float(reinterpret_cast<const __half*>(st)[idx]);
  if (dtype == HP_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(st)[idx]);
  return reinterpret_cast<const float*>(st)[idx];
}

// PC: the buffers' row pitch as a compile-time constant (0: the tile's own, at
// run time); with it every shared-memory row of a sweep is an immediate offset.
template <int RND, int ODT, int SEG, int PC>
__global__ void __launch_bounds__(512) k_chain(const __grid_constant__ ChainKParams kp) {
  grid_dep_sync();
  const ChainArgs& a = kp.a;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // align to 128 bytes by offsetting the shared array itself (not through an
  // integer cast), so every derived pointer stays a 32-bit shared address
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base);
  volatile int* status = reinterpret_cast<volatile int*>(base + 64);
  const int d = a.depth;
  const ChainGeom g = chain_geom(d, a.tile_w, a.tile_h);
  const int P = PC ? PC : g.P;
  float* bufA = reinterpret_cast<float*>(base + kSmemHeader);
  float* bufB = bufA + g.buf;
  const int ch = blockIdx.z;
  const int ox = blockIdx.x * a.tile_w, oy = blockIdx.y * a.tile_h;
  const int W = a.in.w, H = a.in.h;
  const int xin = ox - 2 * d, yin = oy - 2 * d;
  const bool border = xin < 0 || yin < 0 || xin + g.W0 > W || yin + g.H0 > H;

  // ---- stage 0: input tile + halo ----
  if (kp.load_mode != kLoadClamped) {
    const bool direct = kp.load_mode == kLoadTmaDirect;
    const int esize = a.in.dtype == HP_F32 ? 4 : 2;
    const int bw = direct ? g.P : kp.sbw;
    unsigned char* dst = direct ? reinterpret_cast<unsigned char*>(bufA) : reinterpret_cast<unsigned char*>(bufB);
    if (threadIdx.x == 0) {
      *status = 0;
      mbar_init(bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(bar, (unsigned)(g.nby * g.BH * bw * esize));
      for (int k = 0; k < g.nby; ++k)
        tma_load_3d(dst + (size_t)k * g.BH * bw * esize, &kp.tmap, xin - kp.off, yin + k * g.BH, ch, bar);
      // one thread waits (bounded); the others sleep in the barrier below
      if (!mbar_wait_bounded(bar, 0, 2000000000ull)) *status = 1;  // gives up after 2 s
    }
    __syncthreads();
    if (*status) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      return;
    }
    if (!direct) {
      // convert to f32 and shift to column 0 of buffer A (row-wise, coalesced)
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int y = warp; y < g.H0; y += nw)
        for (int x = lane; x < g.W0; x += 32)
          bufA[y * g.P + x] = staged_value(dst, y * bw + x + kp.off, a.in.dtype);
      __syncthreads();
    }
    if (border) {
      fixup(bufA, g.P, xin, yin, g.W0, g.H0, W, H);
    }
  } else {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int y = warp; y < g.H0; y += nw) {
      const int gy = iclamp(yin + y, 0, H - 1);
      for (int x = lane; x < g.W0; x += 32) bufA[y * g.P + x] = load_px(a.in, ch, iclamp(xin + x, 0, W - 1), gy);
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
    if (s == d && a.epilogue == 0) {
      // the last stage straight to the output; nothing reads shared memory after it
      GlobalSink<ODT> gs{(char*)a.out.data + (long long)ch * a.out.ps, a.out.rs, ox, oy, a.tile_h, a.tile_w,
                         a.out.w, a.out.h, &a.out, ch};
      sweep<SEG, RND>(src, P, Ws, Hs, wx, wy, dt, gs);
      return;
    }
    sweep<SEG, RND>(src, P, Ws, Hs, wx, wy, dt, SmemSink{dst, P});
    if (s < d && border) {
      __syncthreads();
      fixup(dst, g.P, ox - 2 * (d - s), oy - 2 * (d - s), Ws, Hs, W, H);
    }
    __syncthreads();
  }

  // ---- with the unsharp epilogue: combine and copy the last stage out with
  // coalesced 128-bit (f32) / 64-bit stores ----
  const float* last = (d & 1) ? bufB : bufA;
  const int hlim = min(a.tile_h, a.out.h - oy), wlim = min(a.tile_w, a.out.w - ox);
  const int nb4 = a.tile_w >> 2;
  char* plane = (char*)a.out.data + (long long)ch * a.out.ps;
  const int odt = a.out.dtype;
  for (int i = threadIdx.x; i < hlim * nb4; i += blockDim.x) {
    const int y = i / nb4;
    const int x = 4 * (i - y * nb4);
    if (x >= wlim) continue;
    float4 v = *reinterpret_cast<const float4*>(last + y * g.P + x);
    if (a.epilogue == 1) {
      // unsharp: combine with the chain's input at the same pixel (stage 0 is
      // still in buffer A when the chain has one stage)
      float vin[4];
      if (d == 1) {
        const float* s0 = bufA + (y + 2) * g.P + x + 2;
        vin[0] = s0[0]; vin[1] = s0[1]; vin[2] = s0[2]; vin[3] = s0[3];
      } else {
        for (int k = 0; k < 4; ++k) vin[k] = x + k < wlim ? load_px(a.in, ch, ox + x + k, oy + y) : 0.0f;
      }
      v.x = round_storage(odt, op_unsharp(vin[0], v.x, a.amount));
      v.y = round_storage(odt, op_unsharp(vin[1], v.y, a.amount));
      v.z = round_storage(odt, op_unsharp(vin[2], v.z, a.amount));
      v.w = round_storage(odt, op_unsharp(vin[3], v.w, a.amount));
    }
    char* row = plane + (long long)(oy + y) * a.out.rs;
    const int gx = ox + x;
    if (ODT != 3 && x + 3 < wlim) {
      if (ODT == 0) {
        *reinterpret_cast<float4*>(row + 4LL * gx) = v;
      } else {
        uint2 u;
        if (ODT == 1) {
          __half2 p0 = __floats2half2_rn(v.x, v.y), p1 = __floats2half2_rn(v.z, v.w);
          u.x = *reinterpret_cast<unsigned*>(&p0);
          u.y = *reinterpret_cast<unsigned*>(&p1);
        } else {
          __nv_bfloat162 p0 = __floats2bfloat162_rn(v.x, v.y), p1 = __floats2bfloat162_rn(v.z, v.w);
          u.x = *reinterpret_cast<unsigned*>(&p0);
          u.y = *reinterpret_cast<unsigned*>(&p1);
        }
        *reinterpret_cast<uint2*>(row + 2LL * gx) = u;
      }
    } else {
      const float vv[4] = {v.x, v.y, v.z, v.w};
      for (int k = 0; k < 4 && x + k < wlim; ++k) store_px(a.out, ch, gx + k, oy + y, vv[k]);
    }
  }
}

typedef void (*ChainKernel)(ChainKParams);

// The pitch of a 64-column tile of depth 4 (64 + 16 columns) is compiled in
// for the uniform-type kernels.
constexpr int kPitch64d4 = 80;

template <int RND, int ODT>
ChainKernel by_seg(int seg, int pitch) {
  if (RND != 3 && pitch == kPitch64d4)
    return seg == 4 ? k_chain<RND, ODT, 4, kPitch64d4> : seg == 16 ? k_chain<RND, ODT, 16, kPitch64d4>
                                                                  : k_chain<RND, ODT, 8, kPitch64d4>;
  return seg == 4 ? k_chain<RND, ODT, 4, 0> : seg == 16 ? k_chain<RND, ODT, 16, 0> : k_chain<RND, ODT, 8, 0>;
}

// Picks the instantiation: one rounding kind for every stage and a vector
// store for the output type when they agree, else the general one; and the
// unrolled segment length.
ChainKernel pick_kernel(const ChainArgs& a, int* variant) {
  int s0 = a.storage[0];
  bool uniform = true;
  for (int i = 1; i < a.depth; ++i) uniform &= a.storage[i] == s0;
  const int si = a.seg == 4 ? 0 : a.seg == 16 ? 2 : 1;
  const bool same = uniform && a.out.dtype == s0;
  const int pitch = chain_geom(a.depth, a.tile_w, a.tile_h).P;
  const int pc = pitch == kPitch64d4 ? 12 : 0;  // the compiled-pitch kernels' variant numbers follow
  if (same && s0 == HP_F32) { *variant = pc + 0 * 3 + si; return by_seg<0, 0>(a.seg, pitch); }
  if (same && s0 == HP_F16) { *variant = pc + 1 * 3 + si; return by_seg<1, 1>(a.seg, pitch); }
  if (same && s0 == HP_BF16) { *variant = pc + 2 * 3 + si; return by_seg<2, 2>(a.seg, pitch); }
  *variant = 3 * 3 + si;
  return by_seg<3, 3>(a.seg, pitch);
}

}  // namespace

int chain_smem_bytes(int depth, int tile_w, int tile_h, int in_dtype) {
  (void)in_dtype;
  ChainGeom g = chain_geom(depth, tile_w, tile_h);
  return kSmemHeader + 128 + 2 * g.buf * 4;
}

int launch_chain(const ChainArgs& a, int smem_bytes, void* stream) {
  static bool configured[24] = {};
  int variant = 0;
  ChainKernel kern = pick_kernel(a, &variant);
  if (!configured[variant]) {  // opt in once: static shared memory also counts against the default 48 KB
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[variant] = true;
  }
  ChainKParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  ChainGeom g = chain_geom(a.depth, a.tile_w, a.tile_h);
  const int dt = a.in.dtype;
  // every tile's x origin is a multiple of tile_w, itself a multiple of 8, so
  // the halo origin's alignment is that of -2d for every tile
  const int xin = -2 * a.depth;
  kp.load_mode = kLoadClamped;
  if (dt == HP_F32 || dt == HP_F16 || dt == HP_BF16) {
    const int esize = dt == HP_F32 ? 4 : 2;
    const int align = 16 / esize;
    const int off = ((xin % align) + align) % align;
    CUtensorMapDataType tdt = dt == HP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                              : dt == HP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (dt == HP_F32 && off == 0 && g.P <= 256) {
      if (!encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps, g.P, g.BH))
        kp.load_mode = kLoadTmaDirect;
    } else {
      const int sbw = (g.W0 + off + align - 1) / align * align;
      if (sbw <= 256 && (long long)g.nby * g.BH * sbw * esize <= (long long)g.buf * 4 &&
          !encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps, sbw, g.BH)) {
        kp.load_mode = kLoadTmaStaged;
        kp.off = off;
        kp.sbw = sbw;
      }
    }
  }
  dim3 grid(a.tiles_x, a.tiles_y, a.in.c);
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(a.threads), smem_bytes, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
