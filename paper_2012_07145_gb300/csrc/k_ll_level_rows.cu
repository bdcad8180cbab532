// One level of the local-Laplacian output pyramid and its collapse step,
// streaming (the local Laplacian app of Sec. 6, after Paris et al. with K = 8
// discrete intensity levels).  Per fine pixel of level l:
//   t = G_l[gray] (K-1) picks the levels k0 and k0+1 (weight f);
//   L_k = G_l[k] - U(G_{l+1}[k]) for those two;  L' = (1-f) L_k0 + f L_k0+1;
//   R_l = L' + U(R_{l+1}).
// At level 0 the level stack is the remap of gray, computed on the fly from
// the RGB input, and the colour reconstruction and output quantisation follow.
//
// One warp per strip of 30 coarse columns walks down a run of coarse rows.
// Lane l owns coarse column m = 30 s + l - 1 and the fine columns 2m and 2m+1.
// Per coarse row it loads channels 0..K-1 of G_{l+1} and R_{l+1} at its column
// and takes the x pass of the upsample for its two fine columns (coarse
// neighbours m-1, m+1 by warp shuffles): even fine columns 1/8, 6/8, 1/8 over
// m-1, m, m+1; odd ones 1/2, 1/2 over m, m+1.  A window of three x-passed
// coarse rows gives the y pass of fine rows 2n (1/8, 6/8, 1/8 over n-1, n, n+1)
// and 2n+1 (1/2, 1/2 over n, n+1).  The window of the K levels sits in shared
// memory, lane-private (word (slot, level, column) x 32 + lane: every access
// of a warp hits 32 banks), so a pixel reads just the two levels it blends; no
// global load depends on the pixel's level.  R_{l+1}'s window stays in
// registers.  Lanes 0 and 31 only feed their neighbours.  The operations
// are those of the per-pixel expression (x pass over each coarse row, then the
// y pass, in tap order), so results are bit-identical to the other kernels.
// All stages are stored as f32 in the pipelines this kernel takes (the host
// checks), so there are no rounding steps between them.
#include <cuda_runtime.h>

#include <cstring>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

constexpr int kK = 8;        // intensity levels
constexpr int kNC = kK + 1;  // x-passed channels per coarse row: the K levels of G_{l+1}, then R_{l+1}
constexpr int kStripW = 30;  // coarse columns per warp
constexpr int kSlotF = kK * 2 * 32;      // floats per window slot of a warp: K levels x 2 columns x 32 lanes
constexpr int kWarpF = 3 * kSlotF;       // floats per warp: three slots
constexpr int kMaxWarps = 8;             // 256 threads

struct LevelRowsParams {
  LLLevelArgs a;
  float gk[kK];   // level values k / (K-1), correctly rounded
  int strips, rows, units;
  int vec_in;     // level 0: u16 pair loads and stores aligned
  int vec_out;    // pair stores of the output aligned
  int vec_g;      // float2 loads of G_l aligned
};

// One fine row of the level-0 input (RGB u16) at the lane's two fine columns.
struct RGBPair {
  unsigned w[3];
  __device__ __forceinline__ float get(int c, int j) const { return (float)(j ? (w[c] >> 16) : (w[c] & 0xffffu)); }
};

template <bool LEVEL0, int ODT>
struct LevelRun {
  const LevelRowsParams& P;
  const float* gks;  // the level table in shared memory (dynamic index)
  float* win;        // this lane's column of the warp's window: word (slot, level, column) x 32
  int m, cm, X0, X1, n0, nrun;
  bool pair, prod, ok1;  // pair: both fine columns inside the image; ok1: fine column 2m+1 exists
  float hr[3][2];        // x-passed coarse rows of R_{l+1} (window slot, fine column)
  float raw[kNC];        // the next coarse row, in flight
  RGBPair pin[2], pin_nxt[2];   // level 0: input rows 2n, 2n+1 of this step and the next
  float2 gkp[2], gkp_nxt[2];    // above level 0: G_l[K] at rows 2n, 2n+1

  __device__ __forceinline__ LevelRun(const LevelRowsParams& p, const float* g, float* w) : P(p), gks(g), win(w) {}

  __device__ __forceinline__ void load_raw(int q) {
    const LLLevelArgs& a = P.a;
    const int cy = iclamp(n0 - 1 + q, 0, a.Gn.h - 1);
    const char* g = (const char*)a.Gn.data + (long long)cy * a.Gn.rs;
#pragma unroll
    for (int c = 0; c < kK; ++c) raw[c] = __ldg(reinterpret_cast<const float*>(g + c * a.Gn.ps) + cm);
    const int ry = iclamp(n0 - 1 + q, 0, a.Rn.h - 1);
    raw[kK] = __ldg(reinterpret_cast<const float*>((const char*)a.Rn.data + (long long)a.rn_ch * a.Rn.ps +
                                                   (long long)ry * a.Rn.rs) + iclamp(m, 0, a.Rn.w - 1));
  }

  // x pass of the loaded coarse row into window slot S
  template <int S>
  __device__ __forceinline__ void xpass() {
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const float l = __shfl_up_sync(0xffffffffu, raw[c], 1);
      const float r = __shfl_down_sync(0xffffffffu, raw[c], 1);
      const float h0 = __fmaf_rn(0.125f, r, __fmaf_rn(0.75f, raw[c], __fmul_rn(0.125f, l)));
      const float h1 = __fmaf_rn(0.5f, r, __fmul_rn(0.5f, raw[c]));
      if (c < kK) {
        win[S * kSlotF + (2 * c) * 32] = h0;
        win[S * kSlotF + (2 * c + 1) * 32] = h1;
      } else {
        hr[S][0] = h0;
        hr[S][1] = h1;
      }
    }
  }

  // own-pixel inputs of fine row Y (level 0: RGB; above: G_l[K])
  __device__ __forceinline__ void load_px_row(int Y, RGBPair& rgb, float2& gk) const {
    const LLLevelArgs& a = P.a;
    if (LEVEL0) {
      const char* row = (const char*)a.in.data + (long long)Y * a.in.rs;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const char* q = row + c * a.in.ps;
        if (pair && P.vec_in) {
          rgb.w[c] = __ldg(reinterpret_cast<const unsigned*>(q) + (X0 >> 1));
        } else {
          const unsigned short* s = reinterpret_cast<const unsigned short*>(q);
          rgb.w[c] = (unsigned)__ldg(s + X0) | ((unsigned)__ldg(s + X1) << 16);
        }
      }
    } else {
      const float* q = reinterpret_cast<const float*>((const char*)a.G.data + (long long)kK * a.G.ps +
                                                      (long long)Y * a.G.rs);
      gk = pair && P.vec_g ? __ldg(reinterpret_cast<const float2*>(q) + (X0 >> 1)) : make_float2(__ldg(q + X0), __ldg(q + X1));
    }
  }

  __device__ __forceinline__ void load_step(int i, RGBPair (&rgb)[2], float2 (&gk)[2]) const {
    const int Y = 2 * (n0 + i);
    load_px_row(Y, rgb[0], gk[0]);
    load_px_row(imin(Y + 1, P.a.H - 1), rgb[1], gk[1]);
  }

  // Fine row Y from the window slots of coarse rows n-1 (A), n (B), n+1 (C);
  // odd rows use B and C only.
  template <bool ODD, int A, int B, int C>
  __device__ __forceinline__ void emit(int Y, const RGBPair& rgb, float2 gkv) const {
    const LLLevelArgs& a = P.a;
    float res[2], gray[2], rgbf[2][3];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float gK, g0, g1;
      int k0;
      float f;
      if (LEVEL0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) rgbf[j][c] = rgb.get(c, j);
        gray[j] = op_gray(rgbf[j][0], rgbf[j][1], rgbf[j][2], a.gray_scale);
        gK = gray[j];
      } else {
        gK = j ? gkv.y : gkv.x;
      }
      ll_interp_index(gK, kK, &k0, &f);
      if (LEVEL0) {
        g0 = op_ll_remap(gray[j], gks[k0], a.sigma, a.alpha, a.beta);
        g1 = op_ll_remap(gray[j], gks[k0 + 1], a.sigma, a.alpha, a.beta);
      } else {
        const float* q = reinterpret_cast<const float*>((const char*)a.G.data + (long long)Y * a.G.rs) + (j ? X1 : X0);
        g0 = __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(q) + (long long)k0 * a.G.ps));
        g1 = __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(q) + (long long)(k0 + 1) * a.G.ps));
      }
      // y pass of the two levels this pixel blends (k0 and k0 + 1), and of R
      const float* wl = win + (2 * k0 + j) * 32;  // level k0, this column; level k0 + 1 is 64 further
      float ulo, uhi, ur;
      if (ODD) {
        ulo = __fmaf_rn(0.5f, wl[C * kSlotF], __fmul_rn(0.5f, wl[B * kSlotF]));
        uhi = __fmaf_rn(0.5f, wl[C * kSlotF + 64], __fmul_rn(0.5f, wl[B * kSlotF + 64]));
        ur = __fmaf_rn(0.5f, hr[C][j], __fmul_rn(0.5f, hr[B][j]));
      } else {
        ulo = __fmaf_rn(0.125f, wl[C * kSlotF], __fmaf_rn(0.75f, wl[B * kSlotF], __fmul_rn(0.125f, wl[A * kSlotF])));
        uhi = __fmaf_rn(0.125f, wl[C * kSlotF + 64],
                        __fmaf_rn(0.75f, wl[B * kSlotF + 64], __fmul_rn(0.125f, wl[A * kSlotF + 64])));
        ur = __fmaf_rn(0.125f, hr[C][j], __fmaf_rn(0.75f, hr[B][j], __fmul_rn(0.125f, hr[A][j])));
      }
      const float L0 = __fsub_rn(g0, ulo);
      const float L1 = __fsub_rn(g1, uhi);
      res[j] = __fadd_rn(op_ll_blend(L0, L1, f), ur);
    }
    if (!prod) return;
    const ImgView& o = a.out;
    char* row = (char*)o.data + (long long)Y * o.rs;
    if (LEVEL0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float v[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) v[j] = round_storage(ODT, op_ll_colour(rgbf[j][c], gray[j], res[j], a.s_in, a.s_out));
        char* q = row + c * o.ps;
        if (ODT == HP_U16) {
          unsigned short* s = reinterpret_cast<unsigned short*>(q);
          if (ok1 && P.vec_out) {
            reinterpret_cast<unsigned*>(s)[X0 >> 1] = (unsigned)(unsigned short)v[0] | ((unsigned)(unsigned short)v[1] << 16);
          } else {
            s[X0] = (unsigned short)v[0];
            if (ok1) s[X1] = (unsigned short)v[1];
          }
        } else {
          float* s = reinterpret_cast<float*>(q);
          if (ok1 && P.vec_out) {
            reinterpret_cast<float2*>(s)[X0 >> 1] = make_float2(v[0], v[1]);
          } else {
            s[X0] = v[0];
            if (ok1) s[X1] = v[1];
          }
        }
      }
    } else {
      float* s = reinterpret_cast<float*>(row);
      if (ok1 && P.vec_out) {
        reinterpret_cast<float2*>(s)[X0 >> 1] = make_float2(res[0], res[1]);
      } else {
        s[X0] = res[0];
        if (ok1) s[X1] = res[1];
      }
    }
  }

  // Coarse step i: x pass of coarse row n+1 = n0+i+1 (window slot (PH+2)%3),
  // the next coarse row's loads, then fine rows 2n and 2n+1.
  template <int PH>
  __device__ __forceinline__ void step(int i) {
    constexpr int A = PH, B = (PH + 1) % 3, C = (PH + 2) % 3;
    xpass<C>();
    if (i + 3 <= nrun + 1) load_raw(i + 3);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      pin[r] = pin_nxt[r];
      gkp[r] = gkp_nxt[r];
    }
    if (i + 1 < nrun) load_step(i + 1, pin_nxt, gkp_nxt);
    const int Y = 2 * (n0 + i);
    emit<false, A, B, C>(Y, pin[0], gkp[0]);
    if (Y + 1 < P.a.H) emit<true, A, B, C>(Y + 1, pin[1], gkp[1]);
  }

  __device__ __forceinline__ void run(int strip, int run_idx) {
    const LLLevelArgs& a = P.a;
    const int lane = threadIdx.x & 31;
    m = strip * kStripW + lane - 1;
    cm = iclamp(m, 0, a.Gn.w - 1);
    X0 = iclamp(2 * m, 0, a.W - 1);
    X1 = iclamp(2 * m + 1, 0, a.W - 1);
    pair = 2 * m >= 0 && 2 * m + 1 <= a.W - 1;
    prod = lane >= 1 && lane <= kStripW && 2 * m <= a.W - 1;
    ok1 = prod && 2 * m + 1 <= a.W - 1;
    n0 = run_idx * P.rows;
    nrun = imin(P.rows, a.Gn.h - n0);  // coarse rows n0 .. n0+nrun-1 give fine rows 2n, 2n+1
    load_raw(0);
    xpass<0>();
    load_raw(1);
    xpass<1>();
    load_raw(2);
    load_step(0, pin_nxt, gkp_nxt);
    for (int i = 0; i < nrun; i += 3) {
      step<0>(i);
      if (i + 1 >= nrun) break;
      step<1>(i + 1);
      if (i + 2 >= nrun) break;
      step<2>(i + 2);
    }
  }
};

template <bool LEVEL0, int ODT>
__global__ void __launch_bounds__(256, 3) k_ll_level_rows(const LevelRowsParams P) {
  grid_dep_wait();
  __shared__ float gks[kK];
  extern __shared__ float wins[];  // kWarpF floats per warp (dynamic: 48 KB for 8 warps)
  if (threadIdx.x < kK) gks[threadIdx.x] = P.gk[threadIdx.x];
  __syncthreads();
  float* win = wins + (threadIdx.x >> 5) * kWarpF + (threadIdx.x & 31);
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < P.units; u += nw) {
    LevelRun<LEVEL0, ODT> r(P, gks, win);
    r.run(u % P.strips, u / P.strips);
  }
}

typedef void (*LevelKernel)(LevelRowsParams);

LevelKernel pick_kernel(const LLLevelArgs& a) {
  if (!a.level0) return k_ll_level_rows<false, HP_F32>;
  return a.out.dtype == HP_U16 ? k_ll_level_rows<true, HP_U16> : k_ll_level_rows<true, HP_F32>;
}

}  // namespace

int ll_level_rows_strip_w() { return kStripW; }

// K = 8 levels, every stage and level buffer stored as f32; level 0 reads a
// u16 RGB input and writes u16 or f32 (views' dtypes as set by the caller).
int ll_level_rows_ok(const LLLevelArgs& a) {
  const bool st = a.st_G == HP_F32 && a.st_U == HP_F32 && a.st_L == HP_F32 && a.st_Lout == HP_F32 &&
                  a.st_UR == HP_F32 && a.st_R == HP_F32 && a.rn_st == HP_F32 && a.Gn.dtype == HP_F32 &&
                  a.Rn.dtype == HP_F32 && a.Gn.c >= kK;
  if (a.K != kK || !st) return 0;
  if (a.level0) return a.st_gray == HP_F32 && a.in.dtype == HP_U16 && (a.out.dtype == HP_U16 || a.out.dtype == HP_F32);
  return a.G.dtype == HP_F32 && a.G.c >= kK + 1 && a.out.dtype == HP_F32;
}

static int level_smem_bytes(int threads) { return (threads / 32) * kWarpF * 4; }

int ll_level_rows_grid(const LLLevelArgs& a, int units, int threads) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      allow_max_dynamic_smem((const void*)pick_kernel(a)) != 0 ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick_kernel(a), threads, level_smem_bytes(threads)) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return need < 2 * 152 ? need : 2 * 152;  // no device to ask: two CTAs on each of 152 SMs
  }
  return need < sms * per_sm ? need : sms * per_sm;
}

int launch_ll_level_rows(const LLLevelArgs& a, int rows, int threads, int grid, void* stream) {
  if (!ll_level_rows_ok(a)) return (int)cudaErrorInvalidValue;
  if (rows < 1 || threads < 32 || threads > 256 || threads % 32 || grid < 1) return (int)cudaErrorInvalidValue;
  LevelRowsParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  // k / (K-1) in IEEE single precision: the correctly rounded quotient, equal
  // to the device's __fdiv_rn of the same operands.
  for (int k = 0; k < kK; ++k) kp.gk[k] = (float)k / (float)(kK - 1);
  kp.strips = (a.Gn.w + kStripW - 1) / kStripW;
  kp.rows = rows;
  kp.units = kp.strips * ((a.Gn.h + rows - 1) / rows);
  auto al = [](const ImgView& v, long long n) {
    return (long long)(size_t)v.data % n == 0 && v.rs % n == 0 && v.ps % n == 0;
  };
  kp.vec_in = a.level0 ? al(a.in, 4) : 0;
  kp.vec_out = al(a.out, a.out.dtype == HP_U16 ? 4 : 8);
  kp.vec_g = a.level0 ? 0 : al(a.G, 8);
  static bool configured[3] = {};
  const int variant = !a.level0 ? 0 : a.out.dtype == HP_U16 ? 1 : 2;
  if (!configured[variant]) {  // the window (48 KB for 8 warps) and the level table pass the default 48 KB
    const int e = allow_max_dynamic_smem((const void*)pick_kernel(a));
    if (e) return e;
    configured[variant] = true;
  }
  { const int le_ = launch_kernel(pick_kernel(a), dim3(grid), dim3(threads), level_smem_bytes(threads), stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
