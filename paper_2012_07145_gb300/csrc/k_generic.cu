// Generic fused-group kernel: an interpreter over any group of stencil,
// point-wise, downsample and upsample stages.
//
// One CTA computes one output tile of the group.  Every member except the
// output is computed over the rectangle its consumers need (halo bounds
// inference, recomputing the overlap between neighbouring tiles: Sec. 2
// "Fusion Options", Fig. 1) into shared memory, in topological order; the
// output member is written straight to global memory.  A group of one stage is
// the stage-per-kernel ("compute root") form of that stage.  Reads of the
// group's inputs go to global memory (L1/L2) at clamped coordinates.
//
// Every value is produced by the expressions of stage_math.cuh, so this kernel
// and the specialised ones give bit-identical results.
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

struct Ctx {
  const GPlan* g;
  const Rect* rects;
  const float* sm;
};

// Value of input ref (node index or -1-external) at clamped (x, y).
__device__ __forceinline__ float fetch(const Ctx& k, int ref, int c, int x, int y) {
  if (ref < 0) {
    const ImgView& e = k.g->ext[-1 - ref];
    return load_px(e, c, iclamp(x, 0, e.w - 1), iclamp(y, 0, e.h - 1));
  }
  const GNode& p = k.g->nodes[ref];
  x = iclamp(x, 0, p.dom_w - 1);
  y = iclamp(y, 0, p.dom_h - 1);
  const Rect r = k.rects[ref];
  const int ly = y - r.y0, lx = x - r.x0;
  // bounds inference guarantees the read lies in the rectangle this tile
  // computed for the producer (not only in its allocation, which is the
  // largest rectangle over all tiles); record a miss instead of reading
  if ((unsigned)ly >= (unsigned)(r.y1 - r.y0) || (unsigned)lx >= (unsigned)(r.x1 - r.x0) ||
      (unsigned)c >= (unsigned)p.channels) {
    atomicExch(k.g->err, 2);
    return 0.0f;
  }
  return k.sm[p.smem_off + (c * p.rows + ly) * p.pitch + lx];
}

__device__ float eval_node(const Ctx& k, const GNode& nd, int c, int x, int y) {
  const float* P = k.g->params + nd.p_off;
  switch (nd.kind) {
    case HP_STENCIL: {
      const float* wx = k.g->weights + nd.w_off;
      const float* wy = wx + 2 * nd.rx + 1;
      float hs[2 * HP_MAX_RADIUS + 1];
      float xs[2 * HP_MAX_RADIUS + 1];
      for (int j = 0; j <= 2 * nd.ry; ++j) {
        int yy = y + j - nd.ry;
        for (int i = 0; i <= 2 * nd.rx; ++i) xs[i] = fetch(k, nd.in[0], c, x + i - nd.rx, yy);
        hs[j] = tapn(wx, xs, 2 * nd.rx + 1);
      }
      return tapn(wy, hs, 2 * nd.ry + 1);
    }
    case HP_MAX_STENCIL: {  // exact: the maximum is the same in any order
      float mv = fetch(k, nd.in[0], c, x - nd.rx, y - nd.ry);
      for (int j = -nd.ry; j <= nd.ry; ++j)
        for (int i = -nd.rx; i <= nd.rx; ++i) mv = fmaxf(mv, fetch(k, nd.in[0], c, x + i, y + j));
      return mv;
    }
    case HP_DOWNSAMPLE2: {
      float hs[5];
      for (int j = 0; j < 5; ++j) {
        int yy = 2 * y + j - 2;
        hs[j] = tap5_binomial16(fetch(k, nd.in[0], c, 2 * x - 2, yy), fetch(k, nd.in[0], c, 2 * x - 1, yy),
                                fetch(k, nd.in[0], c, 2 * x, yy), fetch(k, nd.in[0], c, 2 * x + 1, yy),
                                fetch(k, nd.in[0], c, 2 * x + 2, yy));
      }
      return tap5_binomial16(hs[0], hs[1], hs[2], hs[3], hs[4]);
    }
    case HP_UPSAMPLE2: {
      float wxs[3], wys[3], xs[3], hs[3];
      int mx0, my0;
      int nx = up_taps(x, &mx0, wxs);
      int ny = up_taps(y, &my0, wys);
      for (int t = 0; t < ny; ++t) {
        for (int i = 0; i < nx; ++i) xs[i] = fetch(k, nd.in[0], c, mx0 + i, my0 + t);
        hs[t] = tapn(wxs, xs, nx);
      }
      return tapn(wys, hs, ny);
    }
    default:
      break;
  }
  switch (nd.op) {
    case HP_OP_GRAY:
      return op_gray(fetch(k, nd.in[0], 0, x, y), fetch(k, nd.in[0], 1, x, y), fetch(k, nd.in[0], 2, x, y), P[0]);
    case HP_OP_MUL: case HP_OP_ADD: case HP_OP_SUB:
      return op_binary(nd.op, fetch(k, nd.in[0], c, x, y), fetch(k, nd.in[1], c, x, y));
    case HP_OP_HARRIS:
      return op_harris(fetch(k, nd.in[0], 0, x, y), fetch(k, nd.in[1], 0, x, y), fetch(k, nd.in[2], 0, x, y), P[0]);
    case HP_OP_UNSHARP:
      return op_unsharp(fetch(k, nd.in[0], c, x, y), fetch(k, nd.in[1], c, x, y), P[0]);
    case HP_OP_LL_REMAP: {
      int K = (int)P[3];
      float g = fetch(k, nd.in[0], 0, x, y);
      return c < K ? op_ll_remap(g, ll_level(c, K), P[0], P[1], P[2]) : g;
    }
    case HP_OP_LL_INTERP: {
      int K = (int)P[0];
      int k0;
      float f;
      ll_interp_index(fetch(k, nd.in[0], K, x, y), K, &k0, &f);
      return op_ll_blend(fetch(k, nd.in[1], k0, x, y), fetch(k, nd.in[1], k0 + 1, x, y), f);
    }
    case HP_OP_LL_COLOUR:
      return op_ll_colour(fetch(k, nd.in[0], c, x, y), fetch(k, nd.in[1], 0, x, y), fetch(k, nd.in[2], 0, x, y), P[0],
                          P[1]);
    case HP_OP_SELECT:
      return fetch(k, nd.in[0], (int)P[0], x, y);
    case HP_OP_PREMUL:
      return op_premul(fetch(k, nd.in[0], c, x, y), fetch(k, nd.in[0], 3, x, y), c);
    case HP_OP_OVER:
      return op_over(fetch(k, nd.in[0], c, x, y), fetch(k, nd.in[0], 3, x, y), fetch(k, nd.in[1], c, x, y));
    case HP_OP_UNPREMUL:
      return op_unpremul(fetch(k, nd.in[0], c, x, y), fetch(k, nd.in[0], 3, x, y));
    case HP_OP_ZBLUR: {  // along the range levels: channel 2z + q from 2 clamp(z + j) + q
      const int gz = (int)P[0], z = c >> 1, q = c & 1;
      float t[5];
      for (int j = 0; j < 5; ++j) t[j] = fetch(k, nd.in[0], 2 * iclamp(z + j - 2, 0, gz - 1) + q, x, y);
      return tap5_binomial16(t[0], t[1], t[2], t[3], t[4]);
    }
    default:  // HP_OP_SCALE
      return op_scale(fetch(k, nd.in[0], c, x, y), P[0], P[1]);
  }
}

__global__ void __launch_bounds__(1024) k_generic(const __grid_constant__ GPlan g) {
  grid_dep_sync();
  extern __shared__ float4 smem4[];
  __shared__ Rect rects[kMaxGNodes];
  float* sm = reinterpret_cast<float*>(smem4);
  if (threadIdx.x == 0) infer_rects(g, blockIdx.x * g.tile_w, blockIdx.y * g.tile_h, rects);
  __syncthreads();
  Ctx k{&g, rects, sm};
  for (int n = 0; n < g.n_nodes; ++n) {
    const Rect r = rects[n];
    if (!rect_empty(r)) {
      const GNode& nd = g.nodes[n];
      const int rw = r.x1 - r.x0, rh = r.y1 - r.y0;
      const int plane = rw * rh;
      const int total = plane * nd.channels;
      const bool last = n == g.n_nodes - 1;
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int c = idx / plane;
        int rem = idx - c * plane;
        int yy = rem / rw;
        int xx = rem - yy * rw;
        float v = round_storage(nd.storage, eval_node(k, nd, c, r.x0 + xx, r.y0 + yy));
        if (last) {
          store_px(g.out, c, r.x0 + xx, r.y0 + yy, v);
        } else {
          sm[nd.smem_off + (c * nd.rows + yy) * nd.pitch + xx] = v;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

int launch_generic(const GPlan& g, int threads, int smem_bytes, void* stream) {
  static bool configured = false;
  if (!configured) {  // opt in once: static shared memory also counts against the default 48 KB
    int e = allow_max_dynamic_smem((const void*)k_generic);
    if (e) return e;
    configured = true;
  }
  dim3 grid(g.tiles_x, g.tiles_y, 1);
  { const int le_ = launch_kernel(k_generic, dim3(grid), dim3(threads), smem_bytes, stream, g); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

const char* cuda_error_string(int e) { return cudaGetErrorString((cudaError_t)e); }

int allow_max_dynamic_smem(const void* func) {
  cudaFuncAttributes fa;
  int e = (int)cudaFuncGetAttributes(&fa, func);
  if (e) return e;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  e = (int)cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e) return e;
  return (int)cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   optin - (int)fa.sharedSizeBytes);
}

}  // namespace hp
