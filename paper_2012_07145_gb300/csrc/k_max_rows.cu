// Max filter, streaming (the max filter app of Sec. 6): per channel, the
// maximum over the (2RX+1) x (2RY+1) window at clamped coordinates, for a
// group of one window-maximum stage (square, horizontal or vertical) or of a
// horizontal and a vertical one of the same radius (the same values as the
// square window: the clamp acts on each coordinate separately).
//
// One warp per strip of 120 columns of one plane walks down a run of rows.
// Lane l holds the 4 columns x0 + 4 (l - 1) .. + 3 of every input row (lanes 0
// and 31 only feed their neighbours, R <= 4 columns each side); the next row's
// loads are in flight while a row is processed.  (Keeping 2RY+1 rows of loads
// in flight cost registers, hence occupancy, and measured slower.)  Per row: the
// horizontal maxima of the lane's 4 columns from its own values and its
// neighbours' (warp shuffles), kept in a ring of 2RY+1 rows; from row 2RY on,
// the maximum over the ring is an output row.  Maxima are exact, so the order
// of the comparisons does not matter; the group's storage roundings are
// applied to the final maximum (rounding is monotone, so rounding the maximum
// equals the maximum of rounded values).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStripW = 120;  // output columns per warp

struct MaxParams {
  MaxArgs a;
  int strips, runs, units;
};

template <int IDT>
__device__ __forceinline__ void load_row(const MaxArgs& a, int plane, int y, int x0, bool vec, float (&v)[4]) {
  const char* row = (const char*)a.in.data + (long long)plane * a.in.ps + (long long)y * a.in.rs;
  if (IDT == HP_F32 && vec) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(row) + (x0 >> 2));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if (IDT == HP_BF16 && vec) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(row) + (x0 >> 2));
    v[0] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(q.x & 0xffffu)));
    v[1] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(q.x >> 16)));
    v[2] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(q.y & 0xffffu)));
    v[3] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(q.y >> 16)));
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = load_px(a.in, plane, iclamp(x0 + k, 0, a.in.w - 1), y);
  }
}

template <int IDT, int RX, int RY, bool RND>
struct MaxRun {
  static constexpr int N = 2 * RY + 1;  // rows of the ring of horizontal maxima = rows per unrolled step
  const MaxParams& P;
  int plane, x0, y0, nout, lane, n_in;
  bool vec, prod;
  float ring[N][4];
  float nxt[4];    // the next input row, in flight

  __device__ __forceinline__ explicit MaxRun(const MaxParams& p) : P(p) {}

  __device__ __forceinline__ void fetch(int t, float (&dst)[4]) {
    load_row<IDT>(P.a, plane, iclamp(y0 - RY + t, 0, P.a.in.h - 1), x0, vec, dst);
  }

  // Input row t of the run into ring slot S (the load of row t + 1 is issued
  // first); from t = 2RY on, output row t - 2RY.
  template <int S>
  __device__ __forceinline__ void row(int t) {
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = nxt[k];
    if (t + 1 < n_in) fetch(t + 1, nxt);
    // a[0..11]: the left lane's 4 columns, this lane's, the right lane's
    float a[12];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = __shfl_up_sync(kFull, v[k], 1);
      a[4 + k] = v[k];
      a[8 + k] = __shfl_down_sync(kFull, v[k], 1);
    }
    // column k's window is a[4 + k - RX .. 4 + k + RX]
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float m = a[4 + k - RX];
#pragma unroll
      for (int i = 5 + k - RX; i <= 4 + k + RX; ++i) m = fmaxf(m, a[i]);
      ring[S][k] = m;
    }
    if (t >= 2 * RY) {
      float o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float m = ring[0][k];
#pragma unroll
        for (int s = 1; s < N; ++s) m = fmaxf(m, ring[s][k]);
        o[k] = RND ? round_storage(P.a.st_out, round_storage(P.a.st_mid, m)) : m;
      }
      if (prod) {
        const int y = y0 + t - 2 * RY;
        const ImgView& ov = P.a.out;
        if (!RND && x0 + 3 < ov.w) {
          reinterpret_cast<float4*>((char*)ov.data + (long long)plane * ov.ps + (long long)y * ov.rs)[x0 >> 2] =
              make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (x0 + k < ov.w) store_px(ov, plane, x0 + k, y, o[k]);
        }
      }
    }
  }

  template <int SS>
  __device__ __forceinline__ bool step(int t) {
    if (t + SS >= n_in) return false;
    row<SS>(t + SS);
    return true;
  }

  __device__ __forceinline__ void run(int u) {
    lane = threadIdx.x & 31;
    const int per_plane = P.strips * P.runs;
    plane = u / per_plane;
    const int v = u - plane * per_plane;
    const int run_idx = v / P.strips, strip = v - run_idx * P.strips;
    x0 = strip * kStripW + 4 * (lane - 1);
    const int W = P.a.in.w;
    vec = x0 >= 0 && x0 + 3 <= W - 1;
    prod = lane >= 1 && lane <= 30 && x0 < W;
    y0 = run_idx * P.a.rows;
    nout = imin(P.a.rows, P.a.in.h - y0);
    n_in = nout + 2 * RY;
    fetch(0, nxt);
    for (int t = 0; t < n_in; t += N) {
      if (!step<0>(t)) return;
      if (N > 1 && !step<(N > 1 ? 1 : 0)>(t)) return;
      if (N > 2 && !step<(N > 2 ? 2 : 0)>(t)) return;
      if (N > 3 && !step<(N > 3 ? 3 : 0)>(t)) return;
      if (N > 4 && !step<(N > 4 ? 4 : 0)>(t)) return;
      if (N > 5 && !step<(N > 5 ? 5 : 0)>(t)) return;
      if (N > 6 && !step<(N > 6 ? 6 : 0)>(t)) return;
      if (N > 7 && !step<(N > 7 ? 7 : 0)>(t)) return;
      if (N > 8 && !step<(N > 8 ? 8 : 0)>(t)) return;
    }
  }
};

// RND: a storage rounding or a non-f32 output (else plain maxima, float4 stores).
// Three CTAs per SM, except the vertical-only windows of radius 3 and 4, whose
// ring of 2r+1 row maxima needs more registers than that leaves (they run at
// two CTAs per SM rather than spill).
template <int RX, int RY>
constexpr int max_rows_min_blocks() { return RX == 0 && RY >= 3 ? 2 : 3; }

template <int IDT, int RX, int RY, bool RND>
__global__ void __launch_bounds__(256, max_rows_min_blocks<RX, RY>()) k_max_rows(const MaxParams P) {
  grid_dep_wait();
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < P.units; u += nw) {
    MaxRun<IDT, RX, RY, RND> r(P);
    r.run(u);
  }
}

typedef void (*MaxKernel)(MaxParams);

// shape 0: square window, 1: horizontal only, 2: vertical only
template <int IDT, int R, bool RND>
MaxKernel by_shape(int shape) {
  return shape == 1 ? k_max_rows<IDT, R, 0, RND> : shape == 2 ? k_max_rows<IDT, 0, R, RND> : k_max_rows<IDT, R, R, RND>;
}

template <int IDT, bool RND>
MaxKernel by_radius(int r, int shape) {
  return r == 1 ? by_shape<IDT, 1, RND>(shape) : r == 2 ? by_shape<IDT, 2, RND>(shape)
                : r == 3 ? by_shape<IDT, 3, RND>(shape) : by_shape<IDT, 4, RND>(shape);
}

MaxKernel pick_kernel(const MaxArgs& a) {
  const bool plain = a.st_mid == HP_F32 && a.st_out == HP_F32 && a.out.dtype == HP_F32;
  if (a.in.dtype == HP_F32) return plain ? by_radius<HP_F32, false>(a.radius, a.shape) : by_radius<HP_F32, true>(a.radius, a.shape);
  if (a.in.dtype == HP_BF16) return by_radius<HP_BF16, true>(a.radius, a.shape);
  return by_radius<-1, true>(a.radius, a.shape);
}

}  // namespace

int max_rows_strip_w() { return kStripW; }

int max_rows_grid(const MaxArgs& a, int units, int threads) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick_kernel(a), threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return need < 2 * 152 ? need : 2 * 152;  // no device to ask: two CTAs on each of 152 SMs
  }
  return need < sms * per_sm ? need : sms * per_sm;
}

int launch_max_rows(const MaxArgs& a, int grid, void* stream) {
  if (a.radius < 1 || a.radius > 4 || a.shape < 0 || a.shape > 2 || a.rows < 1 || a.threads < 32 || a.threads > 256 || a.threads % 32 || grid < 1)
    return (int)cudaErrorInvalidValue;
  MaxParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  kp.strips = (a.in.w + kStripW - 1) / kStripW;
  kp.runs = (a.in.h + a.rows - 1) / a.rows;
  kp.units = kp.strips * kp.runs * a.in.c;
  { const int le_ = launch_kernel(pick_kernel(a), dim3(grid), dim3(a.threads), 0, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
