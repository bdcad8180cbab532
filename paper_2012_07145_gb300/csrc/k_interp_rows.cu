// One level of the interpolate app's composite (Sec. 6 app list), streaming:
// I_l = D_l over U(I_{l+1}) for the 4 premultiplied channels, and at the
// finest level the division by coverage, out = I_0.rgb / I_0.a.
//
// One warp per strip of 30 coarse columns walks down a run of coarse rows.
// Lane l owns coarse column m = 30 s + l - 1 and the fine columns 2m and 2m+1.
// Per coarse row it loads the 4 channels of I_{l+1} at its column and takes
// the x pass of the upsample for its two fine columns (coarse neighbours m-1,
// m+1 by warp shuffles): even fine columns 1/8, 6/8, 1/8 over m-1, m, m+1; odd
// ones 1/2, 1/2 over m, m+1.  A window of three x-passed coarse rows (in
// registers) gives the y pass of fine rows 2n (1/8, 6/8, 1/8 over n-1, n, n+1)
// and 2n+1 (1/2, 1/2 over n, n+1); the composite with D_l follows per pixel.
// Lanes 0 and 31 only feed their neighbours.  The operations are those of the
// per-pixel expressions (x pass over each coarse row, then the y pass, in tap
// order; op_over, op_unpremul), so results are bit-identical to the generic
// kernel.  All stages are stored as f32 (the host checks).
#include <cuda_runtime.h>

#include <cstring>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStripW = 30;  // coarse columns per warp

struct InterpParams {
  InterpArgs a;
  int strips, units;
};

template <bool FINAL>
struct InterpRun {
  const InterpParams& P;
  int m, cm, X0, X1, n0, nrun;
  bool pair, prod, ok1;
  float hx[3][4][2];  // x-passed coarse rows (window slot, channel, fine column)
  float raw[4];       // the next coarse row, in flight

  __device__ __forceinline__ explicit InterpRun(const InterpParams& p) : P(p) {}

  __device__ __forceinline__ void load_raw(int q) {
    const ImgView& c = P.a.coarse;
    const char* row = (const char*)c.data + (long long)iclamp(n0 - 1 + q, 0, c.h - 1) * c.rs;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) raw[ch] = __ldg(reinterpret_cast<const float*>(row + ch * c.ps) + cm);
  }

  template <int S>
  __device__ __forceinline__ void xpass() {
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const float l = __shfl_up_sync(kFull, raw[ch], 1);
      const float r = __shfl_down_sync(kFull, raw[ch], 1);
      hx[S][ch][0] = __fmaf_rn(0.125f, r, __fmaf_rn(0.75f, raw[ch], __fmul_rn(0.125f, l)));
      hx[S][ch][1] = __fmaf_rn(0.5f, r, __fmul_rn(0.5f, raw[ch]));
    }
  }

  // Fine row Y from window slots of coarse rows n-1 (A), n (B), n+1 (C).
  template <bool ODD, int A, int B, int C>
  __device__ __forceinline__ void emit(int Y) const {
    const ImgView& f = P.a.fine;
    const char* frow = (const char*)f.data + (long long)Y * f.rs;
    float d[4][2];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const float* q = reinterpret_cast<const float*>(frow + ch * f.ps);
      if (pair && P.a.vec) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(q) + (X0 >> 1));
        d[ch][0] = v.x;
        d[ch][1] = v.y;
      } else {
        d[ch][0] = __ldg(q + X0);
        d[ch][1] = __ldg(q + X1);
      }
    }
    float o[4][2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        const float u = ODD ? __fmaf_rn(0.5f, hx[C][ch][j], __fmul_rn(0.5f, hx[B][ch][j]))
                            : __fmaf_rn(0.125f, hx[C][ch][j], __fmaf_rn(0.75f, hx[B][ch][j], __fmul_rn(0.125f, hx[A][ch][j])));
        o[ch][j] = op_over(d[ch][j], d[3][j], u);
      }
      if (FINAL) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) o[ch][j] = op_unpremul(o[ch][j], o[3][j]);
      }
    }
    if (!prod) return;
    const ImgView& ov = P.a.out;
    char* orow = (char*)ov.data + (long long)Y * ov.rs;
#pragma unroll
    for (int ch = 0; ch < (FINAL ? 3 : 4); ++ch) {
      float* q = reinterpret_cast<float*>(orow + ch * ov.ps);
      if (ok1 && P.a.vec) {
        reinterpret_cast<float2*>(q)[X0 >> 1] = make_float2(o[ch][0], o[ch][1]);
      } else {
        q[X0] = o[ch][0];
        if (ok1) q[X1] = o[ch][1];
      }
    }
  }

  template <int PH>
  __device__ __forceinline__ void step(int i) {
    constexpr int A = PH, B = (PH + 1) % 3, C = (PH + 2) % 3;
    xpass<C>();
    if (i + 3 <= nrun + 1) load_raw(i + 3);
    const int Y = 2 * (n0 + i);
    emit<false, A, B, C>(Y);
    if (Y + 1 < P.a.fine.h) emit<true, A, B, C>(Y + 1);
  }

  __device__ __forceinline__ void run(int strip, int run_idx) {
    const int lane = threadIdx.x & 31;
    const int W = P.a.fine.w;
    m = strip * kStripW + lane - 1;
    cm = iclamp(m, 0, P.a.coarse.w - 1);
    X0 = iclamp(2 * m, 0, W - 1);
    X1 = iclamp(2 * m + 1, 0, W - 1);
    pair = 2 * m >= 0 && 2 * m + 1 <= W - 1;
    prod = lane >= 1 && lane <= kStripW && 2 * m <= W - 1;
    ok1 = prod && 2 * m + 1 <= W - 1;
    n0 = run_idx * P.a.rows;
    nrun = imin(P.a.rows, P.a.coarse.h - n0);
    load_raw(0);
    xpass<0>();
    load_raw(1);
    xpass<1>();
    load_raw(2);
    for (int i = 0; i < nrun; i += 3) {
      step<0>(i);
      if (i + 1 >= nrun) break;
      step<1>(i + 1);
      if (i + 2 >= nrun) break;
      step<2>(i + 2);
    }
  }
};

template <bool FINAL>
__global__ void __launch_bounds__(256, 3) k_interp_rows(const InterpParams P) {
  grid_dep_wait();
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < P.units; u += nw) {
    InterpRun<FINAL> r(P);
    r.run(u % P.strips, u / P.strips);
  }
}

typedef void (*InterpKernel)(InterpParams);

InterpKernel pick_kernel(const InterpArgs& a) { return a.final_div ? k_interp_rows<true> : k_interp_rows<false>; }

}  // namespace

int interp_rows_strip_w() { return kStripW; }

int interp_rows_grid(const InterpArgs& a, int units, int threads) {
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

int launch_interp_rows(const InterpArgs& a_in, int grid, void* stream) {
  InterpArgs a = a_in;
  if (a.rows < 1 || a.threads < 32 || a.threads > 256 || a.threads % 32 || grid < 1) return (int)cudaErrorInvalidValue;
  if (a.fine.dtype != HP_F32 || a.coarse.dtype != HP_F32 || a.out.dtype != HP_F32 || a.fine.c < 4 || a.coarse.c < 4 ||
      a.out.c < (a.final_div ? 3 : 4))
    return (int)cudaErrorInvalidValue;
  auto al = [](const ImgView& v) { return (long long)(size_t)v.data % 8 == 0 && v.rs % 8 == 0 && v.ps % 8 == 0; };
  a.vec = al(a.fine) && al(a.out);
  InterpParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  kp.strips = (a.coarse.w + kStripW - 1) / kStripW;
  kp.units = kp.strips * ((a.coarse.h + a.rows - 1) / a.rows);
  { const int le_ = launch_kernel(pick_kernel(a), dim3(grid), dim3(a.threads), 0, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
