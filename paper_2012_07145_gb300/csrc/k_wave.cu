// Streaming ("wavefront") stencil-chain kernel: d fused 5x5 stages, one warp
// per stage, rows flowing through shared-memory ring buffers.
//
// One CTA owns a vertical strip of the output, tile_w columns by tile_h rows
// (one channel).  Stage s (warp s-1) works on its own column range,
// tile_w + 4(d-s) wide, 4 columns per lane, and on its rows top to bottom, one
// row per tick; all warps advance together, one __syncthreads per tick.  Stage
// s starts 5 ticks after stage s-1, so the producer rows y-2..y+2 a row y needs
// are always complete.  Each warp keeps the x passes of its last five producer
// rows in registers (the 5-row window), so every producer row is read from
// shared memory once and no row is computed twice: the only recompute left is
// the 2(d-s)-column halo per side of each stage (the overlapped tiles of
// Fig. 1 along x only) and the 2(d-s)-row halo at the strip's top and bottom.
// Stage 0 arrives by TMA, 8-row boxes into a 32-row ring, issued up to 24 rows
// ahead of stage 1 with one mbarrier per box slot.  Rows outside the image are
// never computed: a stage reads its producer's row min(max(y, 0), H-1), and
// border strips replicate the edge columns of every row they write.  The last
// stage writes global memory with 128-bit stores.
//
// Values use the same x-then-y fma chains and per-stage rounding as every other
// kernel (stage_math.cuh), so results are bit-identical to them.
#include <cuda.h>
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

constexpr int kWP = 132;                 // ring pitch in floats: 128 columns + 4
constexpr int kWRing = 8;                // rows of each inter-stage ring
constexpr int kWBox = 8;                 // rows per TMA box
constexpr int kWBoxes = 4;               // box slots in the input ring
constexpr int kWIn = kWBox * kWBoxes;    // rows of the input ring
constexpr int kWHeader = 128;

struct WaveKParams {
  CUtensorMap tmap;
  ChainArgs a;
};

template <int RND>
__device__ __forceinline__ float wrnd(float v, int dtype) {
  if (RND == 0) return v;
  if (RND == 1) return __half2float(__float2half_rn(v));
  if (RND == 2) return __bfloat162float(__float2bfloat16_rn(v));
  return round_storage(dtype, v);
}

__device__ __forceinline__ float4 wxpass(const float* p, const float* wx) {
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
__device__ __forceinline__ float4 wypass(const float* wy, const float4& a, const float4& b, const float4& c,
                                         const float4& d, const float4& e, int dtype) {
  float4 v;
  v.x = wrnd<RND>(tap5(wy, a.x, b.x, c.x, d.x, e.x), dtype);
  v.y = wrnd<RND>(tap5(wy, a.y, b.y, c.y, d.y, e.y), dtype);
  v.z = wrnd<RND>(tap5(wy, a.z, b.z, c.z, d.z, e.z), dtype);
  v.w = wrnd<RND>(tap5(wy, a.w, b.w, c.w, d.w, e.w), dtype);
  return v;
}

// A box holds image rows [y0_0 + 8b, y0_0 + 8b + 8); it is loaded only if some
// of them lie inside the image.
__device__ __forceinline__ bool box_useful(int b, int y0_0, int H) {
  const int yb = y0_0 + kWBox * b;
  return yb + kWBox > 0 && yb < H;
}

// Phase parity of box b on its barrier: how many useful boxes used the slot before.
__device__ __forceinline__ unsigned box_parity(int b, int y0_0, int H) {
  unsigned n = 0;
  for (int q = b % kWBoxes; q < b; q += kWBoxes) n += box_useful(q, y0_0, H) ? 1u : 0u;
  return n & 1u;
}

template <int RND, int ODT>
__global__ void __launch_bounds__(512) k_wave(const __grid_constant__ WaveKParams kp) {
  const ChainArgs& a = kp.a;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base);
  volatile int* status = reinterpret_cast<volatile int*>(base + 64);
  float* inring = reinterpret_cast<float*>(base + kWHeader);
  float* rings = inring + kWIn * kWP;
  const int d = a.depth;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = warp + 1;  // this warp's stage
  const int ch = blockIdx.z;
  const int ox = blockIdx.x * a.tile_w, oy = blockIdx.y * a.tile_h;
  const int W = a.in.w, H = a.in.h;
  const int x0_0 = ox - 2 * d, y0_0 = oy - 2 * d;
  const int W0 = a.tile_w + 4 * d;
  const int nboxes = (a.tile_h + 4 * d + kWBox - 1) / kWBox;
  const bool border_x = x0_0 < 0 || x0_0 + W0 > W;

  const int x0s = ox - 2 * (d - s), y0s = oy - 2 * (d - s);
  const int Hs = a.tile_h + 4 * (d - s);
  const int nb = (a.tile_w + 4 * (d - s)) >> 2;
  float wx[5], wy[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    wx[k] = a.w[s - 1][k];
    wy[k] = a.w[s - 1][5 + k];
  }
  const int dt = a.storage[s - 1];
  const float* src = s == 1 ? inring : rings + (s - 2) * kWRing * kWP;
  float* dst = rings + (s - 1) * kWRing * kWP;  // unused by the last stage

  int next_box = 0;     // thread 0: next box to issue
  int waited_box = -1;  // warp 0: boxes up to this one have landed and been fixed up
  auto issue_upto = [&](int last) {
    if (last >= nboxes) last = nboxes - 1;
    if (next_box > last) return;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the slots before TMA writes
    for (; next_box <= last; ++next_box) {
      const int b = next_box;
      if (!box_useful(b, y0_0, H)) continue;
      uint64_t* bar = &bars[b % kWBoxes];
      mbar_arrive_expect_tx(bar, (unsigned)(kWBox * kWP * 4));
      tma_load_3d(inring + (b % kWBoxes) * kWBox * kWP, &kp.tmap, x0_0, y0_0 + kWBox * b, ch, bar);
    }
  };
  if (threadIdx.x == 0) {
    *status = 0;
    for (int i = 0; i < kWBoxes; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
    // the first box holding an image row, and the three after it
    const int first_box = y0_0 < 0 ? (-y0_0) / kWBox : 0;
    next_box = first_box;
    issue_upto(first_box + kWBoxes - 1);
  }
  __syncthreads();

  // stage 1: make sure input virtual row v (and every row before it) has landed
  auto ensure_input = [&](int v) {
    const int want = v / kWBox;
    while (waited_box < want) {
      const int b = ++waited_box;
      if (!box_useful(b, y0_0, H)) continue;
      if (lane == 0 && !mbar_wait_bounded(&bars[b % kWBoxes], box_parity(b, y0_0, H), 2000000000ull)) *status = 1;
      __syncwarp();
      if (border_x) {
        // TMA filled columns outside the image with zeros: replicate the edges
        for (int r = 0; r < kWBox; ++r) {
          const int Y = y0_0 + kWBox * b + r;
          if (Y < 0 || Y >= H) continue;
          float* row = inring + ((b % kWBoxes) * kWBox + r) * kWP;
          for (int c = lane; c < W0; c += 32) {
            const int X = x0_0 + c;
            if (X < 0 || X >= W) row[c] = row[iclamp(X, 0, W - 1) - x0_0];
          }
        }
        __syncwarp();
      }
    }
  };
  // x pass of producer row Y (an image row inside [0, H))
  auto xp = [&](int Y) -> float4 {
    const int slot = s == 1 ? ((Y - y0_0) & (kWIn - 1)) : (Y & (kWRing - 1));
    return wxpass(src + slot * kWP + 4 * lane, wx);
  };
  const int odt = a.out.dtype;
  char* out_plane = (char*)a.out.data + (long long)ch * a.out.ps;
  const int wlim = min(a.tile_w, a.out.w - ox);
  auto emit = [&](int y, float4 v) {
    if (s < d) {
      if (lane < nb) *reinterpret_cast<float4*>(dst + (y & (kWRing - 1)) * kWP + 4 * lane) = v;
      if (border_x) {
        __syncwarp();
        float* row = dst + (y & (kWRing - 1)) * kWP;
        for (int c = lane; c < 4 * nb; c += 32) {
          const int X = x0s + c;
          if (X < 0 || X >= W) row[c] = row[iclamp(X, 0, W - 1) - x0s];
        }
      }
      return;
    }
    const int x = 4 * lane;
    if (x >= wlim) return;
    char* row = out_plane + (long long)y * a.out.rs;
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
      return;
    }
    const float vv[4] = {v.x, v.y, v.z, v.w};
    for (int k = 0; k < 4 && x + k < wlim; ++k) store_px(a.out, ch, gx + k, y, round_storage(odt, vv[k]));
  };

  const int first_row = max(0, y0s);
  const int ticks = 5 * (d - 1) + a.tile_h;
  float4 h0, h1, h2, h3, h4;
  int t = 0;
  // one tick: stage s computes its row y = y0s + (t - 5(s-1)) if that row is in the image
#define HP_WAVE_TICK(A, B, C, D, E)                                         \
  {                                                                         \
    const int k = t - 5 * (s - 1);                                          \
    const int y = y0s + k;                                                  \
    if (k >= 0 && k < Hs && y >= 0 && y < H) {                              \
      const int Y2 = min(y + 2, H - 1);                                     \
      if (s == 1) ensure_input(Y2 - y0_0);                                  \
      if (y == first_row) {                                                 \
        A = xp(max(y - 2, 0));                                              \
        B = xp(max(y - 1, 0));                                              \
        C = xp(y);                                                          \
        D = xp(min(y + 1, H - 1));                                          \
      }                                                                     \
      E = xp(Y2);                                                           \
      emit(y, wypass<RND>(wy, A, B, C, D, E, dt));                          \
      if (s == 1) {                                                         \
        __syncwarp(); /* every lane's reads of older slots are done */      \
        if (threadIdx.x == 0) issue_upto((Y2 - y0_0) / kWBox + kWBoxes - 1); \
      }                                                                     \
    }                                                                       \
    __syncthreads();                                                        \
    if (*status) break;                                                     \
    if (++t >= ticks) break;                                                \
  }
  while (true) {
    HP_WAVE_TICK(h0, h1, h2, h3, h4)
    HP_WAVE_TICK(h1, h2, h3, h4, h0)
    HP_WAVE_TICK(h2, h3, h4, h0, h1)
    HP_WAVE_TICK(h3, h4, h0, h1, h2)
    HP_WAVE_TICK(h4, h0, h1, h2, h3)
  }
#undef HP_WAVE_TICK
  if (*status && threadIdx.x == 0) atomicExch(a.err, 1);
}

typedef void (*WaveKernel)(WaveKParams);

}  // namespace

int wave_max_tile_w(int depth) { return ((128 - 4 * (depth - 1)) / 8) * 8; }

int wave_smem_bytes(int depth) { return kWHeader + 128 + 4 * (kWIn * kWP + (depth - 1) * kWRing * kWP); }

int launch_wave(const ChainArgs& a, int smem_bytes, void* stream) {
  int s0 = a.storage[0];
  bool uniform = true;
  for (int i = 1; i < a.depth; ++i) uniform &= a.storage[i] == s0;
  const bool same = uniform && a.out.dtype == s0;
  int variant;
  WaveKernel kern;
  if (same && s0 == HP_F32) { variant = 0; kern = k_wave<0, 0>; }
  else if (same && s0 == HP_F16) { variant = 1; kern = k_wave<1, 1>; }
  else if (same && s0 == HP_BF16) { variant = 2; kern = k_wave<2, 2>; }
  else { variant = 3; kern = k_wave<3, 3>; }
  static bool configured[4] = {};
  if (!configured[variant]) {  // opt in once: static shared memory also counts against the default 48 KB
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[variant] = true;
  }
  WaveKParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  if (a.in.dtype != HP_F32 ||
      encode_tmap_3d(&kp.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs,
                     a.in.ps, kWP, kWBox))
    return (int)cudaErrorInvalidValue;
  dim3 grid(a.tiles_x, a.tiles_y, a.in.c);
  kern<<<grid, 32 * a.depth, smem_bytes, (cudaStream_t)stream>>>(kp);
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
