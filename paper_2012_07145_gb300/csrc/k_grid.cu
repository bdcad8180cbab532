// Bilateral grid (the bilateral grid app of Sec. 6, after Chen, Paris and
// Durand): the splat of a gray image into a grid of s x s pixel cells and
// range levels of size r, and the trilinear slice of the blurred grid back to
// the image.  The grid is a (ceil(W/s)+1) x (ceil(H/s)+1) image of 2 GZ
// channels: channel 2z holds the sum of the values of range level z, channel
// 2z+1 their count.  The blur between them (a point-wise op along the range
// levels and two 5-tap stencils) is one streaming kernel, k_grid_blur, below;
// any other grouping of those stages runs on the generic kernel.
//
// k_grid_splat: one thread per cell (any s) or four (s = 8, k_grid_splat8: two
//   pixel rows each, their copies added in a fixed order); each walks its
//   pixels in row order and adds them to its range level's pair of
//   accumulators, which sit in lane-private shared memory (every access of a
//   warp hits 32 banks), so the sums are formed in the same order every time.
// k_grid_slice: per pixel, trilinear interpolation (x, then y, then the range
//   level) of the value and the weight, then their ratio; four pixels of a row
//   per thread.
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

constexpr int kSplatThreads = 128;
constexpr int kMaxGZ = 31;

__device__ __forceinline__ float gray_at(const ImgView& v, int x, int y) {
  return fminf(fmaxf(load_px(v, 0, x, y), 0.0f), 1.0f);
}

__device__ __forceinline__ int range_level(float v, float inv_r, int gz) {
  return iclamp((int)floorf(__fmaf_rn(v, inv_r, 0.5f)), 0, gz - 1);
}

// Any cell size s: one thread per cell walks its s x s pixels in row order.
__global__ void __launch_bounds__(kSplatThreads) k_grid_splat(const GridArgs a) {
  grid_dep_sync();
  __shared__ float acc[2 * kMaxGZ * kSplatThreads];
  const int t = threadIdx.x;
  const int gx = blockIdx.x * kSplatThreads + t, gy = blockIdx.y;
  if (gx >= a.grid.w) return;  // no barrier below: each thread owns its column of acc
  for (int j = 0; j < 2 * a.gz; ++j) acc[j * kSplatThreads + t] = 0.0f;
  const int W = a.in.w, H = a.in.h;
  const int s = a.s;
  for (int j = 0; j < s; ++j) {
    const int y = iclamp(gy * s + j - s / 2, 0, H - 1);
    for (int i = 0; i < s; ++i) {
      const float v = gray_at(a.in, iclamp(gx * s + i - s / 2, 0, W - 1), y);
      const int z = range_level(v, a.inv_r, a.gz);
      float* p = acc + 2 * z * kSplatThreads + t;
      p[0] = __fadd_rn(p[0], v);
      p[kSplatThreads] = __fadd_rn(p[kSplatThreads], 1.0f);
    }
  }
  for (int j = 0; j < 2 * a.gz; ++j)
    reinterpret_cast<float*>((char*)a.grid.data + (long long)j * a.grid.ps + (long long)gy * a.grid.rs)[gx] =
        acc[j * kSplatThreads + t];
}

// The splat of 8 x 8-pixel cells: a block of 4 warps takes 32 consecutive
// cells of a grid row, lane = cell, warp w = the cell's pixel rows 2w and 2w+1
// (two 128-bit loads per row for interior cells); each warp accumulates into
// its own lane-private copy, then the four copies are added in warp order.
__global__ void __launch_bounds__(128) k_grid_splat8(const GridArgs a) {
  grid_dep_sync();
  __shared__ float acc[4][2 * kMaxGZ][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gx = blockIdx.x * 32 + lane, gy = blockIdx.y;
  const bool valid = gx < a.grid.w;
  for (int j = 0; j < 2 * a.gz; ++j) acc[w][j][lane] = 0.0f;
  if (valid) {
    const int W = a.in.w, H = a.in.h;
    const int x0 = gx * 8 - 4;
    const bool inner = x0 >= 0 && x0 + 7 <= W - 1 && a.in.dtype == HP_F32;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int y = iclamp(gy * 8 + 2 * w + jj - 4, 0, H - 1);
      float v[8];
      if (inner) {
        const float4* row = reinterpret_cast<const float4*>((const char*)a.in.data + (long long)y * a.in.rs) + (x0 >> 2);
        const float4 f0 = __ldg(row), f1 = __ldg(row + 1);
        v[0] = f0.x; v[1] = f0.y; v[2] = f0.z; v[3] = f0.w; v[4] = f1.x; v[5] = f1.y; v[6] = f1.z; v[7] = f1.w;
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fminf(fmaxf(v[i], 0.0f), 1.0f);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = gray_at(a.in, iclamp(x0 + i, 0, W - 1), y);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int z = range_level(v[i], a.inv_r, a.gz);
        acc[w][2 * z][lane] = __fadd_rn(acc[w][2 * z][lane], v[i]);
        acc[w][2 * z + 1][lane] = __fadd_rn(acc[w][2 * z + 1][lane], 1.0f);
      }
    }
  }
  __syncthreads();
  if (!valid) return;
  for (int j = w; j < 2 * a.gz; j += 4) {
    const float t = __fadd_rn(__fadd_rn(__fadd_rn(acc[0][j][lane], acc[1][j][lane]), acc[2][j][lane]), acc[3][j][lane]);
    reinterpret_cast<float*>((char*)a.grid.data + (long long)j * a.grid.ps + (long long)gy * a.grid.rs)[gx] = t;
  }
}

__device__ __forceinline__ float lerp(float a, float b, float f) { return __fmaf_rn(f, __fsub_rn(b, a), a); }

// Four consecutive pixels of one row per thread (a warp: 128 pixels; a block:
// 8 rows): one 128-bit load of the image and one 128-bit store of the output
// where the row allows, and the grid-row addresses shared by the four pixels.
// Each pixel's arithmetic is the per-pixel expression above, unchanged.
__global__ void __launch_bounds__(256) k_grid_slice(const GridArgs a) {
  grid_dep_sync();
  const int xb = (blockIdx.x * 32 + (threadIdx.x & 31)) * 4;
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (xb >= a.in.w || y >= a.in.h) return;
  const ImgView& g = a.grid;
  const float gyf = __fmul_rn((float)y, a.inv_s);
  const float fly = floorf(gyf), fy = __fsub_rn(gyf, fly);
  const int y0 = iclamp((int)fly, 0, g.h - 1), y1 = iclamp((int)fly + 1, 0, g.h - 1);
  const char* g0 = (const char*)g.data + (long long)y0 * g.rs;
  const char* g1 = (const char*)g.data + (long long)y1 * g.rs;
  const int n = imin(4, a.in.w - xb);
  const bool vec = n == 4 && a.in.dtype == HP_F32 && (((size_t)a.in.data | (size_t)a.in.rs | (size_t)a.out.data | (size_t)a.out.rs) & 15) == 0;
  float v[4];
  if (vec) {
    const float4 q = __ldg(reinterpret_cast<const float4*>((const char*)a.in.data + (long long)y * a.in.rs) + (xb >> 2));
    v[0] = fminf(fmaxf(q.x, 0.0f), 1.0f); v[1] = fminf(fmaxf(q.y, 0.0f), 1.0f);
    v[2] = fminf(fmaxf(q.z, 0.0f), 1.0f); v[3] = fminf(fmaxf(q.w, 0.0f), 1.0f);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = gray_at(a.in, imin(xb + k, a.in.w - 1), y);
  }
  float o[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float gxf = __fmul_rn((float)(xb + k), a.inv_s), gzf = __fmul_rn(v[k], a.inv_r);
    const float flx = floorf(gxf), flz = floorf(gzf);
    const float fx = __fsub_rn(gxf, flx), fz = __fsub_rn(gzf, flz);
    const int x0 = iclamp((int)flx, 0, g.w - 1), x1 = iclamp((int)flx + 1, 0, g.w - 1);
    const int z0 = iclamp((int)flz, 0, a.gz - 1), z1 = iclamp((int)flz + 1, 0, a.gz - 1);
    float r[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {  // value, weight
      float zs[2];
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const long long off = (long long)(2 * (d ? z1 : z0) + q) * g.ps;
        const float* p0 = reinterpret_cast<const float*>(g0 + off);
        const float* p1 = reinterpret_cast<const float*>(g1 + off);
        const float a0 = lerp(__ldg(p0 + x0), __ldg(p0 + x1), fx);
        const float a1 = lerp(__ldg(p1 + x0), __ldg(p1 + x1), fx);
        zs[d] = lerp(a0, a1, fy);
      }
      r[q] = lerp(zs[0], zs[1], fz);
    }
    o[k] = r[1] > 0.0f ? __fdiv_rn(r[0], r[1]) : v[k];
  }
  float* orow = reinterpret_cast<float*>((char*)a.out.data + (long long)y * a.out.rs);
  if (vec) {
    reinterpret_cast<float4*>(orow)[xb >> 2] = make_float4(o[0], o[1], o[2], o[3]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < n) orow[xb + k] = o[k];
  }
}

}  // namespace

int grid_max_levels() { return kMaxGZ; }

int launch_grid_splat(const GridArgs& a, void* stream) {
  if (a.gz < 1 || a.gz > kMaxGZ || a.s < 1 || a.grid.dtype != HP_F32 || a.grid.c < 2 * a.gz) return (int)cudaErrorInvalidValue;
  if (a.s == 8) {
    dim3 grid8((a.grid.w + 31) / 32, a.grid.h, 1);
    { const int le_ = launch_kernel(k_grid_splat8, grid8, dim3(128), 0, stream, a); if (le_) return le_; }
  } else {
    dim3 grid((a.grid.w + kSplatThreads - 1) / kSplatThreads, a.grid.h, 1);
    { const int le_ = launch_kernel(k_grid_splat, grid, dim3(kSplatThreads), 0, stream, a); if (le_) return le_; }
  }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

int launch_grid_slice(const GridArgs& a, void* stream) {
  if (a.gz < 1 || a.grid.dtype != HP_F32 || a.out.dtype != HP_F32 || a.grid.c < 2 * a.gz) return (int)cudaErrorInvalidValue;
  dim3 grid((a.in.w + 127) / 128, (a.in.h + 7) / 8, 1);
  { const int le_ = launch_kernel(k_grid_slice, grid, dim3(256), 0, stream, a); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}


// ---- the blur of the grid (the group: range-level blur, x blur, y blur) ----
//
// k_grid_blur: one warp per strip of 28 grid columns (lanes 0, 1, 30, 31 only
// feed their neighbours), one of the two halves of a cell (values or weights)
// and a chunk of 4 range levels, walking down a run of grid rows.  Per row it
// loads the chunk's levels and two more on each side (clamped), blurs along
// the levels, then along x (neighbours by warp shuffles); the y blur is five
// accumulators per level, each fed its taps in order as the rows arrive, so
// the float operations are those of the three stages one after the other.
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kZC = 4;          // range levels per unit
constexpr int kBlurStrip = 28;  // grid columns per warp

struct GridBlurParams {
  GridBlurArgs a;
  int strips, zchunks, runs, units;
};

struct BlurRun {
  const GridBlurParams& P;
  int x, k, z0, y0, nout, T;
  bool prod;
  float acc[kZC][5];
  float ld[kZC + 4];  // the row's levels z0-2 .. z0+kZC+1 (clamped), in flight

  __device__ __forceinline__ explicit BlurRun(const GridBlurParams& p) : P(p) {}

  __device__ __forceinline__ void fetch(int t) {
    const ImgView& g = P.a.in;
    const int y = iclamp(y0 - 2 + t, 0, g.h - 1);
    const int xc = iclamp(x, 0, g.w - 1);
    const char* row = (const char*)g.data + (long long)y * g.rs;
#pragma unroll
    for (int i = 0; i < kZC + 4; ++i) {
      const int c = 2 * iclamp(z0 - 2 + i, 0, P.a.gz - 1) + k;
      ld[i] = __ldg(reinterpret_cast<const float*>(row + c * g.ps) + xc);
    }
  }

  // Input row t (grid row y0 - 2 + t) into the accumulators; PH = t mod 5.
  // Row t is tap j of output row t - j (run-relative, outputs 0 .. nout-1):
  // tap 0 starts output t, tap 4 completes output t - 4.
  template <int PH>
  __device__ __forceinline__ void row(int t) {
    float v[kZC + 4];
#pragma unroll
    for (int i = 0; i < kZC + 4; ++i) v[i] = ld[i];
    if (t + 1 < T) fetch(t + 1);
    const float w[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
    const int ofin = t - 4;
    const bool st = prod && ofin >= 0 && ofin < nout;
#pragma unroll
    for (int q = 0; q < kZC; ++q) {
      const float zb = tap5_binomial16(v[q], v[q + 1], v[q + 2], v[q + 3], v[q + 4]);
      const float l2 = __shfl_up_sync(kFull, zb, 2), l1 = __shfl_up_sync(kFull, zb, 1);
      const float r1 = __shfl_down_sync(kFull, zb, 1), r2 = __shfl_down_sync(kFull, zb, 2);
      const float h = tap5(w, l2, l1, zb, r1, r2);
      // slot of output t - j is (t - j) mod 5 = (PH - j) mod 5
      float& fin = acc[q][(PH + 1) % 5];                 // output t - 4: tap 4, complete
      fin = __fmaf_rn(w[4], h, fin);
      if (st && z0 + q < P.a.gz) {
        const ImgView& o = P.a.out;
        reinterpret_cast<float*>((char*)o.data + (long long)(2 * (z0 + q) + k) * o.ps +
                                 (long long)(y0 + ofin) * o.rs)[x] = fin;
      }
      acc[q][(PH + 2) % 5] = __fmaf_rn(w[3], h, acc[q][(PH + 2) % 5]);  // output t - 3
      acc[q][(PH + 3) % 5] = __fmaf_rn(w[2], h, acc[q][(PH + 3) % 5]);  // output t - 2
      acc[q][(PH + 4) % 5] = __fmaf_rn(w[1], h, acc[q][(PH + 4) % 5]);  // output t - 1
      acc[q][PH] = __fmul_rn(w[0], h);                                  // output t: tap 0
    }
  }

  __device__ __forceinline__ void run(int u) {
    const int lane = threadIdx.x & 31;
    const int strip = u % P.strips;
    int rest = u / P.strips;
    const int zc = rest % P.zchunks;
    rest /= P.zchunks;
    k = rest & 1;
    const int run_idx = rest >> 1;
    x = strip * kBlurStrip + lane - 2;
    prod = lane >= 2 && lane < 2 + kBlurStrip && x < P.a.in.w;
    z0 = zc * kZC;
    y0 = run_idx * P.a.rows;
    nout = imin(P.a.rows, P.a.in.h - y0);
    T = nout + 4;  // grid rows y0 - 2 .. y0 + nout + 1
#pragma unroll
    for (int q = 0; q < kZC; ++q)
#pragma unroll
      for (int s = 0; s < 5; ++s) acc[q][s] = 0.0f;
    fetch(0);
    for (int t = 0; t < T; t += 5) {
      row<0>(t);
      if (t + 1 >= T) break;
      row<1>(t + 1);
      if (t + 2 >= T) break;
      row<2>(t + 2);
      if (t + 3 >= T) break;
      row<3>(t + 3);
      if (t + 4 >= T) break;
      row<4>(t + 4);
    }
  }
};

__global__ void __launch_bounds__(256, 2) k_grid_blur(const GridBlurParams P) {
  grid_dep_wait();
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < P.units; u += nw) {
    BlurRun r(P);
    r.run(u);
  }
}

}  // namespace

int grid_blur_units(const GridBlurArgs& a) {
  const int strips = (a.in.w + kBlurStrip - 1) / kBlurStrip;
  const int zchunks = (a.gz + kZC - 1) / kZC;
  return strips * zchunks * 2 * ((a.in.h + a.rows - 1) / a.rows);
}

int launch_grid_blur(const GridBlurArgs& a, int grid, void* stream) {
  if (a.gz < 1 || a.rows < 1 || grid < 1 || a.in.dtype != HP_F32 || a.out.dtype != HP_F32 || a.in.c < 2 * a.gz ||
      a.out.c < 2 * a.gz)
    return (int)cudaErrorInvalidValue;
  GridBlurParams kp;
  kp.a = a;
  kp.strips = (a.in.w + kBlurStrip - 1) / kBlurStrip;
  kp.zchunks = (a.gz + kZC - 1) / kZC;
  kp.runs = (a.in.h + a.rows - 1) / a.rows;
  kp.units = kp.strips * kp.zchunks * 2 * kp.runs;
  { const int le_ = launch_kernel(k_grid_blur, dim3(grid), dim3(256), 0, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
