// Fused Harris corner response: the whole Harris DAG (gray, 3x3 Sobel
// gradients, products, 3x3 box sums, det - k tr^2) in one kernel per output
// tile, with every intermediate in shared memory or registers (block- and
// thread-level fusion, Sec. 2 "Fusion Options").
//
// Per CTA (output tile T_w x T_h):
//  0. one 3-D TMA box brings the three input planes, tile + 2-pixel halo, into
//     a staging area (mbarrier completion, one waiting thread);
//  1. gray = 0.299 R + 0.587 G + 0.114 B over (T_w+4) x (T_h+4), edge-replicated
//     outside the image;
//  2. each thread sweeps a 4-column block down a row segment: the x passes of
//     both gradients share one read of each gray row, 3-row register windows
//     give Ix and Iy, and the three products are stored over (T_w+2) x (T_h+2)
//     (aliasing the dead staging area);
//  3. the same sweep over the three product buffers gives the box sums and the
//     response, written with 128-bit coalesced stores.
// All values come from the stage expressions of stage_math.cuh with each
// stage rounded to its storage type, so the result is bit-identical to any
// other schedule of the same pipeline.
#include <cuda.h>
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

struct HarrisGeom {
  int GW, GH, Pg;   // gray rectangle and pitch
  int PW, PH, Pp;   // product rectangles and pitch
  int A, off;       // staging: box x origin ox - A (16-byte aligned); gray column x is box column x + off
  int bw;           // staging box width (elements)
  int gray_floats, region_bytes;
};

__host__ __device__ inline HarrisGeom harris_geom(int tw, int th, int esize) {
  HarrisGeom g;
  g.GW = tw + 4;
  g.GH = th + 4;
  g.Pg = tw + 12;
  g.PW = tw + 2;
  g.PH = th + 2;
  g.Pp = tw + 8;
  g.A = 16 / esize;
  g.off = g.A - 2;
  g.bw = (g.GW + g.off + g.A - 1) / g.A * g.A;
  g.gray_floats = (g.Pg * g.GH + 31) & ~31;
  const int staging = g.bw * g.GH * 3 * esize;
  const int prods = 3 * g.Pp * g.PH * 4;
  g.region_bytes = ((staging > prods ? staging : prods) + 127) & ~127;
  return g;
}

constexpr int kHeader = 128;

struct HarrisKParams {
  CUtensorMap tmap;
  HarrisArgs a;
};

template <int RND>
__device__ __forceinline__ float rs(float v, int dtype) {
  return RND == 0 ? v : round_storage(dtype, v);
}

__device__ __forceinline__ void load6(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float2 b = *reinterpret_cast<const float2*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}

__device__ __forceinline__ float4 x3(const float* w, const float* v) {
  float4 h;
  h.x = tap3(w, v[0], v[1], v[2]);
  h.y = tap3(w, v[1], v[2], v[3]);
  h.z = tap3(w, v[2], v[3], v[4]);
  h.w = tap3(w, v[3], v[4], v[5]);
  return h;
}

__device__ __forceinline__ float4 y3(const float* w, const float4& a, const float4& b, const float4& c) {
  return make_float4(tap3(w, a.x, b.x, c.x), tap3(w, a.y, b.y, c.y), tap3(w, a.z, b.z, c.z), tap3(w, a.w, b.w, c.w));
}

__device__ void fixup_rect(float* buf, int P, int x0, int y0, int Ws, int Hs, int W, int H) {
  const int cx0 = max(0, -x0), cx1 = min(Ws, W - x0);
  const int cy0 = max(0, -y0), cy1 = min(Hs, H - y0);
  const int n = Ws * Hs;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int y = i / Ws, x = i - y * Ws;
    if (x >= cx0 && x < cx1 && y >= cy0 && y < cy1) continue;
    buf[y * P + x] = buf[min(max(y, cy0), cy1 - 1) * P + min(max(x, cx0), cx1 - 1)];
  }
}

template <int RND, int ODT>
__global__ void __launch_bounds__(512) k_harris(const __grid_constant__ HarrisKParams kp) {
  grid_dep_sync();
  const HarrisArgs& a = kp.a;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base);
  volatile int* status = reinterpret_cast<volatile int*>(base + 64);
  const int esize = a.in.dtype == HP_F32 ? 4 : 2;
  const HarrisGeom g = harris_geom(a.tile_w, a.tile_h, esize);
  float* G = reinterpret_cast<float*>(base + kHeader);
  unsigned char* region = base + kHeader + g.gray_floats * 4;
  const int ox = blockIdx.x * a.tile_w, oy = blockIdx.y * a.tile_h;
  const int W = a.in.w, H = a.in.h;
  const bool border = ox - 2 < 0 || oy - 2 < 0 || ox + a.tile_w + 2 > W || oy + a.tile_h + 2 > H;

  // ---- 0. TMA: three planes, tile + halo ----
  if (threadIdx.x == 0) {
    *status = 0;
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, (unsigned)(g.bw * g.GH * 3 * esize));
    tma_load_3d(region, &kp.tmap, ox - g.A, oy - 2, 3 * blockIdx.z, bar);  // image blockIdx.z of a batch
    if (!mbar_wait_bounded(bar, 0, 2000000000ull)) *status = 1;
  }
  __syncthreads();
  if (*status) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    return;
  }

  // ---- 1. gray over the (T_w+4) x (T_h+4) rectangle at (ox-2, oy-2) ----
  {
    const int plane = g.bw * g.GH;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int y = warp; y < g.GH; y += nw) {
      for (int x = lane; x < g.GW; x += 32) {
        const int i = y * g.bw + x + g.off;
        float r, gg, b;
        if (esize == 4) {
          const float* st = reinterpret_cast<const float*>(region);
          r = st[i]; gg = st[plane + i]; b = st[2 * plane + i];
        } else if (a.in.dtype == HP_BF16) {
          const __nv_bfloat16* st = reinterpret_cast<const __nv_bfloat16*>(region);
          r = __bfloat162float(st[i]); gg = __bfloat162float(st[plane + i]); b = __bfloat162float(st[2 * plane + i]);
        } else {
          const __half* st = reinterpret_cast<const __half*>(region);
          r = __half2float(st[i]); gg = __half2float(st[plane + i]); b = __half2float(st[2 * plane + i]);
        }
        G[y * g.Pg + x] = rs<RND>(op_gray(r, gg, b, a.gray_scale), a.st[0]);
      }
    }
    if (border) {
      __syncthreads();
      fixup_rect(G, g.Pg, ox - 2, oy - 2, g.GW, g.GH, W, H);
    }
    __syncthreads();
  }

  // ---- 2. gradients and products over (T_w+2) x (T_h+2) at (ox-1, oy-1) ----
  float* Pxx = reinterpret_cast<float*>(region);
  float* Pyy = Pxx + g.Pp * g.PH;
  float* Pxy = Pyy + g.Pp * g.PH;
  {
    const float* wxi = a.w[0];
    const float* wyi = a.w[0] + 3;
    const float* wxj = a.w[1];
    const float* wyj = a.w[1] + 3;
    float wa[3], wb[3], wc[3], wd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { wa[k] = wxi[k]; wb[k] = wyi[k]; wc[k] = wxj[k]; wd[k] = wyj[k]; }
    const int nb = (g.PW + 3) >> 2;
    const int nseg = (g.PH + a.seg - 1) / a.seg;
    for (int it = threadIdx.x; it < nb * nseg; it += blockDim.x) {
      const int sg = it / nb, b = it - sg * nb;
      const int r0 = sg * a.seg, r1 = min(g.PH, r0 + a.seg);
      const float* p = G + r0 * g.Pg + 4 * b;
      float v[6];
      float4 hx0, hx1, hx2, hy0, hy1, hy2;
      load6(p, v); hx0 = x3(wa, v); hy0 = x3(wc, v); p += g.Pg;
      load6(p, v); hx1 = x3(wa, v); hy1 = x3(wc, v); p += g.Pg;
      int y = r0;
      auto emit = [&](const float4& a0, const float4& a1, const float4& a2, const float4& b0, const float4& b1,
                      const float4& b2) {
        float4 ix = y3(wb, a0, a1, a2), iy = y3(wd, b0, b1, b2);
        ix.x = rs<RND>(ix.x, a.st[1]); ix.y = rs<RND>(ix.y, a.st[1]); ix.z = rs<RND>(ix.z, a.st[1]); ix.w = rs<RND>(ix.w, a.st[1]);
        iy.x = rs<RND>(iy.x, a.st[2]); iy.y = rs<RND>(iy.y, a.st[2]); iy.z = rs<RND>(iy.z, a.st[2]); iy.w = rs<RND>(iy.w, a.st[2]);
        float4 pxx, pyy, pxy;
        pxx.x = rs<RND>(__fmul_rn(ix.x, ix.x), a.st[3]); pxx.y = rs<RND>(__fmul_rn(ix.y, ix.y), a.st[3]);
        pxx.z = rs<RND>(__fmul_rn(ix.z, ix.z), a.st[3]); pxx.w = rs<RND>(__fmul_rn(ix.w, ix.w), a.st[3]);
        pyy.x = rs<RND>(__fmul_rn(iy.x, iy.x), a.st[4]); pyy.y = rs<RND>(__fmul_rn(iy.y, iy.y), a.st[4]);
        pyy.z = rs<RND>(__fmul_rn(iy.z, iy.z), a.st[4]); pyy.w = rs<RND>(__fmul_rn(iy.w, iy.w), a.st[4]);
        pxy.x = rs<RND>(__fmul_rn(ix.x, iy.x), a.st[5]); pxy.y = rs<RND>(__fmul_rn(ix.y, iy.y), a.st[5]);
        pxy.z = rs<RND>(__fmul_rn(ix.z, iy.z), a.st[5]); pxy.w = rs<RND>(__fmul_rn(ix.w, iy.w), a.st[5]);
        const int o = y * g.Pp + 4 * b;
        *reinterpret_cast<float4*>(Pxx + o) = pxx;
        *reinterpret_cast<float4*>(Pyy + o) = pyy;
        *reinterpret_cast<float4*>(Pxy + o) = pxy;
      };
      while (true) {
        load6(p, v); hx2 = x3(wa, v); hy2 = x3(wc, v); p += g.Pg;
        emit(hx0, hx1, hx2, hy0, hy1, hy2);
        if (++y >= r1) break;
        load6(p, v); hx0 = x3(wa, v); hy0 = x3(wc, v); p += g.Pg;
        emit(hx1, hx2, hx0, hy1, hy2, hy0);
        if (++y >= r1) break;
        load6(p, v); hx1 = x3(wa, v); hy1 = x3(wc, v); p += g.Pg;
        emit(hx2, hx0, hx1, hy2, hy0, hy1);
        if (++y >= r1) break;
      }
    }
    if (border) {
      __syncthreads();
      fixup_rect(Pxx, g.Pp, ox - 1, oy - 1, g.PW, g.PH, W, H);
      fixup_rect(Pyy, g.Pp, ox - 1, oy - 1, g.PW, g.PH, W, H);
      fixup_rect(Pxy, g.Pp, ox - 1, oy - 1, g.PW, g.PH, W, H);
    }
    __syncthreads();
  }

  // ---- 3. box sums and response over the T_w x T_h tile ----
  {
    float w[3][6];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int k = 0; k < 6; ++k) w[q][k] = a.w[2 + q][k];
    const int nb = a.tile_w >> 2;
    const int nseg = (a.tile_h + a.seg - 1) / a.seg;
    const int hlim = min(a.tile_h, a.out.h - oy), wlim = min(a.tile_w, a.out.w - ox);
    char* out_row0 = (char*)a.out.data + (long long)blockIdx.z * a.out.ps + (long long)oy * a.out.rs;
    for (int it = threadIdx.x; it < nb * nseg; it += blockDim.x) {
      const int sg = it / nb, b = it - sg * nb;
      const int r0 = sg * a.seg, r1 = min(a.tile_h, r0 + a.seg);
      const int o0 = r0 * g.Pp + 4 * b;
      float v[6];
      float4 s[3][3];  // [buffer][window row]
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        load6(Pxx + o0 + k * g.Pp, v); s[0][k] = x3(w[0], v);
        load6(Pyy + o0 + k * g.Pp, v); s[1][k] = x3(w[1], v);
        load6(Pxy + o0 + k * g.Pp, v); s[2][k] = x3(w[2], v);
      }
      int o = o0 + 2 * g.Pp;
      auto emit = [&](int y, int i0, int i1, int i2) {
        float4 sxx = y3(w[0] + 3, s[0][i0], s[0][i1], s[0][i2]);
        float4 syy = y3(w[1] + 3, s[1][i0], s[1][i1], s[1][i2]);
        float4 sxy = y3(w[2] + 3, s[2][i0], s[2][i1], s[2][i2]);
        const int odt = a.out.dtype;
        // ODT 0 and 2 round on the store itself (f32 is exact, bf16 packs with round-to-nearest)
        auto ro = [&](float q) { return ODT == 3 ? round_storage(odt, q) : q; };
        float4 r;
        r.x = ro(op_harris(rs<RND>(sxx.x, a.st[6]), rs<RND>(syy.x, a.st[7]), rs<RND>(sxy.x, a.st[8]), a.k));
        r.y = ro(op_harris(rs<RND>(sxx.y, a.st[6]), rs<RND>(syy.y, a.st[7]), rs<RND>(sxy.y, a.st[8]), a.k));
        r.z = ro(op_harris(rs<RND>(sxx.z, a.st[6]), rs<RND>(syy.z, a.st[7]), rs<RND>(sxy.z, a.st[8]), a.k));
        r.w = ro(op_harris(rs<RND>(sxx.w, a.st[6]), rs<RND>(syy.w, a.st[7]), rs<RND>(sxy.w, a.st[8]), a.k));
        const int x = 4 * b;
        if (y >= hlim || x >= wlim) return;
        char* row = out_row0 + (long long)y * a.out.rs;
        const int gx = ox + x;
        if (ODT != 3 && x + 3 < wlim) {
          if (ODT == 0) {
            *reinterpret_cast<float4*>(row + 4LL * gx) = r;
          } else {
            __nv_bfloat162 p0 = __floats2bfloat162_rn(r.x, r.y), p1 = __floats2bfloat162_rn(r.z, r.w);
            uint2 u;
            u.x = *reinterpret_cast<unsigned*>(&p0);
            u.y = *reinterpret_cast<unsigned*>(&p1);
            *reinterpret_cast<uint2*>(row + 2LL * gx) = u;
          }
          return;
        }
        const float vv[4] = {r.x, r.y, r.z, r.w};
        for (int i = 0; i < 4 && x + i < wlim; ++i) store_px(a.out, blockIdx.z, gx + i, oy + y, vv[i]);
      };
      int y = r0;
      while (true) {
        load6(Pxx + o, v); s[0][2] = x3(w[0], v);
        load6(Pyy + o, v); s[1][2] = x3(w[1], v);
        load6(Pxy + o, v); s[2][2] = x3(w[2], v);
        o += g.Pp;
        emit(y, 0, 1, 2);
        if (++y >= r1) break;
        load6(Pxx + o, v); s[0][0] = x3(w[0], v);
        load6(Pyy + o, v); s[1][0] = x3(w[1], v);
        load6(Pxy + o, v); s[2][0] = x3(w[2], v);
        o += g.Pp;
        emit(y, 1, 2, 0);
        if (++y >= r1) break;
        load6(Pxx + o, v); s[0][1] = x3(w[0], v);
        load6(Pyy + o, v); s[1][1] = x3(w[1], v);
        load6(Pxy + o, v); s[2][1] = x3(w[2], v);
        o += g.Pp;
        emit(y, 2, 0, 1);
        if (++y >= r1) break;
      }
    }
  }
}

typedef void (*HarrisKernel)(HarrisKParams);

}  // namespace

int harris_smem_bytes(int tile_w, int tile_h, int in_dtype) {
  const HarrisGeom g = harris_geom(tile_w, tile_h, in_dtype == HP_F32 ? 4 : 2);
  return kHeader + 128 + g.gray_floats * 4 + g.region_bytes;
}

int launch_harris(const HarrisArgs& a, int smem_bytes, void* stream) {
  bool inner_f32 = true;
  for (int i = 0; i < 9; ++i) inner_f32 &= a.st[i] == HP_F32;
  int variant;
  HarrisKernel kern;
  if (inner_f32 && a.out.dtype == HP_F32) { variant = 0; kern = k_harris<0, 0>; }
  else if (inner_f32 && a.out.dtype == HP_BF16) { variant = 1; kern = k_harris<0, 2>; }
  else { variant = 2; kern = k_harris<3, 3>; }
  static bool configured[3] = {false, false, false};
  if (!configured[variant]) {  // opt in once: static shared memory also counts against the default 48 KB
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[variant] = true;
  }
  HarrisKParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  const int dt = a.in.dtype;
  const int esize = dt == HP_F32 ? 4 : 2;
  const HarrisGeom g = harris_geom(a.tile_w, a.tile_h, esize);
  CUtensorMapDataType tdt = dt == HP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                            : dt == HP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (g.bw > 256 || g.GH > 256 ||
      encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps, g.bw, g.GH, 3))
    return (int)cudaErrorInvalidValue;
  dim3 grid(a.tiles_x, a.tiles_y, a.batch > 1 ? a.batch : 1);
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(a.threads), smem_bytes, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
