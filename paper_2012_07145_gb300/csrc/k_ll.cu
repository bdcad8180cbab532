// Local Laplacian kernels (the local Laplacian app of Sec. 6, after Paris et
// al. with K discrete intensity levels).
//
// k_ll_down: one pyramid level down for every channel of a level stack.  The
//   source is either a materialised level (f32 planes), or, for the first
//   level, the remap stack computed on the fly from the input: gray of the RGB
//   input, then the K remaps and gray itself (the inlined producers of Sec. 4).
//   Per CTA and channel: fill the clamped fine tile in shared memory, x pass at
//   even columns, y pass at even rows (binomial [1,4,6,4,1]/16 per axis).
//
// k_ll_level: one pyramid level of the output Laplacian and the collapse step,
//   per pixel: t = G_l[gray]*(K-1) picks the two levels k0, k0+1; for each of
//   them L = G_l[k] - U(G_{l+1}[k]) is formed only where it is used (the other
//   K-2 Laplacian channels are never computed); the blend is added to the
//   upsampled coarser result.  At level 0 the level stack itself is the remap
//   of gray, computed on the fly, and the colour reconstruction and u16
//   quantisation follow.
//
// Every value is the stage expression of stage_math.cuh rounded to its stage's
// storage type, so results are bit-identical to the generic kernels.
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

// Source value at clamped fine coordinates: a plane of the level (f32 fast
// path or any dtype) or, for the remap source, computed from the gray tile.
template <bool F32>
__device__ __forceinline__ float level_px(const ImgView& v, int c, int x, int y) {
  if (F32) return __ldg(reinterpret_cast<const float*>((const char*)v.data + (long long)c * v.ps + (long long)y * v.rs) + x);
  return load_px(v, c, x, y);
}

// Tile widths are powers of two (checked on the host): lg_tw = log2(tile_w).
template <bool REMAP, bool F32>
__global__ void __launch_bounds__(256) k_ll_down(const LLDownArgs a) {
  grid_dep_wait();
  extern __shared__ __align__(16) float sm[];
  __shared__ float gk_level[HP_MAX_PARAMS * 2 + 1];
  const int tw = a.tile_w, lg_tw = 31 - __clz(tw);
  const int FW = 2 * tw + 3, FH = 2 * a.tile_h + 3;
  const int plane = FW * FH;
  float* GR = sm;                           // gray tile (remap source only)
  float* S = GR + (REMAP ? plane : 0);      // C source planes
  float* HX = S + a.C * plane;              // C x-pass planes, FH x tile_w
  const int x0 = blockIdx.x * tw, y0 = blockIdx.y * a.tile_h;
  const int fx0 = 2 * x0 - 2, fy0 = 2 * y0 - 2;
  const int Wf = a.src.w, Hf = a.src.h;
  const int nt = blockDim.x;
  if (REMAP) {
    if (threadIdx.x < a.K) gk_level[threadIdx.x] = ll_level(threadIdx.x, a.K);
    // gray of the clamped fine tile, four pixels (12 loads) in flight per thread
    for (int i0 = threadIdx.x; i0 < plane; i0 += 4 * nt) {
      float rgb[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * nt;
        const int r = i / FW, q = i - r * FW;
        const int fy = iclamp(fy0 + r, 0, Hf - 1), fx = iclamp(fx0 + q, 0, Wf - 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) rgb[u][c] = i < plane ? load_px(a.src, c, fx, fy) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u * nt < plane)
          GR[i0 + u * nt] = round_storage(a.st_gray, op_gray(rgb[u][0], rgb[u][1], rgb[u][2], a.gray_scale));
    }
    __syncthreads();
    // every channel of the remap stack of one fine pixel per thread.  Outside
    // the band |g - g_k| <= sigma the remap is a multiply-add; a pixel lies in
    // the band of at most two levels when 2 sigma (K-1) < 2, so the power is
    // evaluated for those two only (the general case evaluates every level).
    for (int i = threadIdx.x; i < plane; i += nt) {
      const float g = GR[i];
      int ka = -1, kb = -1;
      bool many = false;
      for (int k = 0; k < a.K; ++k) {
        if (fabsf(__fsub_rn(g, gk_level[k])) <= a.sigma) {
          if (ka < 0) ka = k;
          else if (kb < 0) kb = k;
          else many = true;
        }
      }
      const float pa = ka >= 0 ? op_ll_remap(g, gk_level[ka], a.sigma, a.alpha, a.beta) : 0.0f;
      const float pb = kb >= 0 ? op_ll_remap(g, gk_level[kb], a.sigma, a.alpha, a.beta) : 0.0f;
      for (int c = 0; c < a.C; ++c) {
        float v;
        if (c >= a.K) {
          v = g;
        } else if (many) {
          v = op_ll_remap(g, gk_level[c], a.sigma, a.alpha, a.beta);
        } else if (c == ka) {
          v = pa;
        } else if (c == kb) {
          v = pb;
        } else {
          const float d = __fsub_rn(g, gk_level[c]);
          v = op_ll_remap_outside(d, fabsf(d), gk_level[c], a.sigma, a.beta);
        }
        S[c * plane + i] = round_storage(a.st_remap, v);
      }
    }
  } else {
    // every channel at once, four loads in flight per thread before any store
    const int total = a.C * plane;
    for (int i0 = threadIdx.x; i0 < total; i0 += 4 * nt) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * nt;
        const int c = i / plane, j = i - c * plane;
        const int r = j / FW, q = j - r * FW;
        v[u] = i < total ? level_px<F32>(a.src, c, iclamp(fx0 + q, 0, Wf - 1), iclamp(fy0 + r, 0, Hf - 1)) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u * nt < total) S[i0 + u * nt] = v[u];
    }
  }
  __syncthreads();
  const int hxp = FH << lg_tw;
  for (int c = 0; c < a.C; ++c)
    for (int j = threadIdx.x; j < hxp; j += nt) {
      const int r = j >> lg_tw, x = j & (tw - 1);
      const float* s = S + c * plane + r * FW + 2 * x;
      HX[c * hxp + j] = tap5_binomial16(s[0], s[1], s[2], s[3], s[4]);
    }
  __syncthreads();
  const int op = a.tile_h << lg_tw;
  for (int c = 0; c < a.C; ++c)
    for (int j = threadIdx.x; j < op; j += nt) {
      const int y = j >> lg_tw, x = j & (tw - 1);
      const int ox = x0 + x, oy = y0 + y;
      if (ox >= a.out.w || oy >= a.out.h) continue;
      const float* h = HX + c * hxp + 2 * y * tw + x;
      const float v = round_storage(a.st_out, tap5_binomial16(h[0], h[tw], h[2 * tw], h[3 * tw], h[4 * tw]));
      if (F32) {
        reinterpret_cast<float*>((char*)a.out.data + (long long)c * a.out.ps + (long long)oy * a.out.rs)[ox] = v;
      } else {
        store_px(a.out, c, ox, oy, v);
      }
    }
}

// Upsample of channel c of a coarse image at fine (X, Y): taps per axis by
// parity, coarse indices clamped; x pass over each needed coarse row, then y.
// Each coarse value is first rounded to `st` (the storage of the stage it
// stands for; a no-op when the buffer already holds that stage).
template <bool F32>
__device__ __forceinline__ float upsample_at(const ImgView& v, int c, int X, int Y, int st) {
  float wx[3], wy[3], xs[3], hs[3];
  int mx0, my0;
  const int nx = up_taps(X, &mx0, wx);
  const int ny = up_taps(Y, &my0, wy);
  for (int t = 0; t < ny; ++t) {
    const int yy = iclamp(my0 + t, 0, v.h - 1);
    for (int i = 0; i < nx; ++i) {
      const float raw = level_px<F32>(v, c, iclamp(mx0 + i, 0, v.w - 1), yy);
      xs[i] = F32 ? raw : round_storage(st, raw);
    }
    hs[t] = tapn(wx, xs, nx);
  }
  return tapn(wy, hs, ny);
}

// F32: every level buffer and every stage stored as f32 (no rounding steps).
template <bool LEVEL0, bool F32>
__global__ void __launch_bounds__(256) k_ll_level(const LLLevelArgs a) {
  grid_dep_wait();
  const int X = blockIdx.x * 32 + (threadIdx.x & 31);
  const int Y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (X >= a.W || Y >= a.H) return;
  auto rs = [](int st, float v) { return F32 ? v : round_storage(st, v); };
  const int K = a.K;
  float gray = 0.0f, rgb[3];
  float gK;
  if (LEVEL0) {
    for (int c = 0; c < 3; ++c) rgb[c] = load_px(a.in, c, X, Y);
    gray = rs(a.st_gray, op_gray(rgb[0], rgb[1], rgb[2], a.gray_scale));
    gK = rs(a.st_G, gray);
  } else {
    gK = level_px<F32>(a.G, K, X, Y);
  }
  int k0;
  float f;
  ll_interp_index(gK, K, &k0, &f);
  float Lk[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int k = k0 + j;
    const float g = LEVEL0 ? rs(a.st_G, op_ll_remap(gray, ll_level(k, K), a.sigma, a.alpha, a.beta))
                           : level_px<F32>(a.G, k, X, Y);
    const float u = rs(a.st_U, upsample_at<F32>(a.Gn, k, X, Y, HP_F32));
    Lk[j] = rs(a.st_L, op_binary(HP_OP_SUB, g, u));
  }
  const float lout = rs(a.st_Lout, op_ll_blend(Lk[0], Lk[1], f));
  const float ur = rs(a.st_UR, upsample_at<F32>(a.Rn, a.rn_ch, X, Y, a.rn_st));
  const float r = rs(a.st_R, op_binary(HP_OP_ADD, lout, ur));
  if (LEVEL0) {
    for (int c = 0; c < 3; ++c)
      store_px(a.out, c, X, Y, round_storage(a.out.dtype, op_ll_colour(rgb[c], gray, r, a.s_in, a.s_out)));
  } else {
    store_px(a.out, 0, X, Y, r);
  }
}

}  // namespace

int ll_down_smem_bytes(int tile_w, int tile_h, int channels, int remap) {
  const int FW = 2 * tile_w + 3, FH = 2 * tile_h + 3;
  return ((remap ? FW * FH : 0) + channels * FW * FH + channels * FH * tile_w) * 4;
}

int launch_ll_down(const LLDownArgs& a, int smem_bytes, void* stream) {
  typedef void (*K)(LLDownArgs);
  const bool f32 = a.src.dtype == HP_F32 && a.out.dtype == HP_F32 && a.st_out == HP_F32;
  const int variant = (a.remap ? 2 : 0) + (f32 ? 1 : 0);
  const K kernels[4] = {k_ll_down<false, false>, k_ll_down<false, true>, k_ll_down<true, false>,
                        k_ll_down<true, true>};
  static bool configured[4] = {};
  if (!configured[variant]) {  // opt in once: static shared memory also counts against the default 48 KB
    int e = allow_max_dynamic_smem((const void*)kernels[variant]);
    if (e) return e;
    configured[variant] = true;
  }
  dim3 grid(a.tiles_x, a.tiles_y, 1);
  { const int le_ = launch_kernel(kernels[variant], dim3(grid), dim3(256), smem_bytes, stream, a); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

int launch_ll_level(const LLLevelArgs& a, void* stream) {
  dim3 grid((a.W + 31) / 32, (a.H + 7) / 8, 1);
  bool f32 = a.Gn.dtype == HP_F32 && a.Rn.dtype == HP_F32 && a.rn_st == HP_F32 && a.st_G == HP_F32 &&
             a.st_U == HP_F32 && a.st_L == HP_F32 && a.st_Lout == HP_F32 && a.st_UR == HP_F32 && a.st_R == HP_F32;
  if (a.level0) {
    f32 = f32 && a.st_gray == HP_F32;
    if (f32) { const int le_ = launch_kernel(k_ll_level<true, true>, dim3(grid), dim3(256), 0, stream, a); if (le_) return le_; }
    else { const int le_ = launch_kernel(k_ll_level<true, false>, dim3(grid), dim3(256), 0, stream, a); if (le_) return le_; }
  } else {
    f32 = f32 && a.G.dtype == HP_F32;
    if (f32) { const int le_ = launch_kernel(k_ll_level<false, true>, dim3(grid), dim3(256), 0, stream, a); if (le_) return le_; }
    else { const int le_ = launch_kernel(k_ll_level<false, false>, dim3(grid), dim3(256), 0, stream, a); if (le_) return le_; }
  }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
