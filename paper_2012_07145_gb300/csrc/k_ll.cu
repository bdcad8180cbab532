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

__global__ void __launch_bounds__(256) k_ll_down(const LLDownArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int FW = 2 * a.tile_w + 3, FH = 2 * a.tile_h + 3;
  float* GR = sm;                 // gray tile (remap source only)
  float* S = GR + FW * FH;        // source channel tile
  float* HX = S + FW * FH;        // x-pass results, FH x tile_w
  const int x0 = blockIdx.x * a.tile_w, y0 = blockIdx.y * a.tile_h;
  const int fx0 = 2 * x0 - 2, fy0 = 2 * y0 - 2;
  const int Wf = a.src.w, Hf = a.src.h;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (a.remap) {
    for (int r = warp; r < FH; r += nw) {
      const int fy = iclamp(fy0 + r, 0, Hf - 1);
      for (int q = lane; q < FW; q += 32) {
        const int fx = iclamp(fx0 + q, 0, Wf - 1);
        GR[r * FW + q] = round_storage(a.st_gray, op_gray(load_px(a.src, 0, fx, fy), load_px(a.src, 1, fx, fy),
                                                          load_px(a.src, 2, fx, fy), a.gray_scale));
      }
    }
    __syncthreads();
  }
  for (int c = 0; c < a.C; ++c) {
    if (a.remap) {
      const float gk = c < a.K ? ll_level(c, a.K) : 0.0f;
      for (int r = warp; r < FH; r += nw)
        for (int q = lane; q < FW; q += 32) {
          const float g = GR[r * FW + q];
          S[r * FW + q] = round_storage(a.st_remap, c < a.K ? op_ll_remap(g, gk, a.sigma, a.alpha, a.beta) : g);
        }
    } else {
      for (int r = warp; r < FH; r += nw) {
        const int fy = iclamp(fy0 + r, 0, Hf - 1);
        for (int q = lane; q < FW; q += 32) S[r * FW + q] = load_px(a.src, c, iclamp(fx0 + q, 0, Wf - 1), fy);
      }
    }
    __syncthreads();
    for (int r = warp; r < FH; r += nw)
      for (int x = lane; x < a.tile_w; x += 32) {
        const float* s = S + r * FW + 2 * x;
        HX[r * a.tile_w + x] = tap5_binomial16(s[0], s[1], s[2], s[3], s[4]);
      }
    __syncthreads();
    for (int y = warp; y < a.tile_h; y += nw) {
      const int oy = y0 + y;
      for (int x = lane; x < a.tile_w; x += 32) {
        const int ox = x0 + x;
        if (ox >= a.out.w || oy >= a.out.h) continue;
        const float* h = HX + 2 * y * a.tile_w + x;
        const int tw = a.tile_w;
        store_px(a.out, c, ox, oy,
                 round_storage(a.st_out, tap5_binomial16(h[0], h[tw], h[2 * tw], h[3 * tw], h[4 * tw])));
      }
    }
    __syncthreads();
  }
}

// Upsample of channel c of a coarse image at fine (X, Y): taps per axis by
// parity, coarse indices clamped; x pass over each needed coarse row, then y.
// Each coarse value is first rounded to `st` (the storage of the stage it
// stands for; a no-op when the buffer already holds that stage).
__device__ __forceinline__ float upsample_at(const ImgView& v, int c, int X, int Y, int st = HP_F32) {
  float wx[3], wy[3], xs[3], hs[3];
  int mx0, my0;
  const int nx = up_taps(X, &mx0, wx);
  const int ny = up_taps(Y, &my0, wy);
  for (int t = 0; t < ny; ++t) {
    const int yy = iclamp(my0 + t, 0, v.h - 1);
    for (int i = 0; i < nx; ++i) xs[i] = round_storage(st, load_px(v, c, iclamp(mx0 + i, 0, v.w - 1), yy));
    hs[t] = tapn(wx, xs, nx);
  }
  return tapn(wy, hs, ny);
}

__global__ void __launch_bounds__(256) k_ll_level(const LLLevelArgs a) {
  const int X = blockIdx.x * 32 + (threadIdx.x & 31);
  const int Y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (X >= a.W || Y >= a.H) return;
  const int K = a.K;
  float gray = 0.0f, rgb[3];
  float gK;
  if (a.level0) {
    for (int c = 0; c < 3; ++c) rgb[c] = load_px(a.in, c, X, Y);
    gray = round_storage(a.st_gray, op_gray(rgb[0], rgb[1], rgb[2], a.gray_scale));
    gK = round_storage(a.st_G, gray);
  } else {
    gK = load_px(a.G, K, X, Y);
  }
  int k0;
  float f;
  ll_interp_index(gK, K, &k0, &f);
  float Lk[2];
  for (int j = 0; j < 2; ++j) {
    const int k = k0 + j;
    const float g = a.level0 ? round_storage(a.st_G, op_ll_remap(gray, ll_level(k, K), a.sigma, a.alpha, a.beta))
                             : load_px(a.G, k, X, Y);
    const float u = round_storage(a.st_U, upsample_at(a.Gn, k, X, Y));
    Lk[j] = round_storage(a.st_L, op_binary(HP_OP_SUB, g, u));
  }
  const float lout = round_storage(a.st_Lout, op_ll_blend(Lk[0], Lk[1], f));
  const float ur = round_storage(a.st_UR, upsample_at(a.Rn, a.rn_ch, X, Y, a.rn_st));
  const float r = round_storage(a.st_R, op_binary(HP_OP_ADD, lout, ur));
  if (a.level0) {
    for (int c = 0; c < 3; ++c)
      store_px(a.out, c, X, Y, round_storage(a.out.dtype, op_ll_colour(rgb[c], gray, r, a.s_in, a.s_out)));
  } else {
    store_px(a.out, 0, X, Y, r);
  }
}

}  // namespace

int ll_down_smem_bytes(int tile_w, int tile_h) {
  const int FW = 2 * tile_w + 3, FH = 2 * tile_h + 3;
  return (2 * FW * FH + FH * tile_w) * 4;
}

int launch_ll_down(const LLDownArgs& a, int smem_bytes, void* stream) {
  static bool configured = false;
  if (!configured) {  // opt in once: static shared memory also counts against the default 48 KB
    int e = allow_max_dynamic_smem((const void*)k_ll_down);
    if (e) return e;
    configured = true;
  }
  dim3 grid(a.tiles_x, a.tiles_y, 1);
  k_ll_down<<<grid, 256, smem_bytes, (cudaStream_t)stream>>>(a);
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

int launch_ll_level(const LLLevelArgs& a, void* stream) {
  dim3 grid((a.W + 31) / 32, (a.H + 7) / 8, 1);
  k_ll_level<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
