// Streaming pyramid downsample kernels of the local Laplacian app (Sec. 6,
// after Paris et al. with K discrete intensity levels): the first level of the
// remap pyramid straight from the input (gray and the K remaps inlined into the
// downsample, as the producers of Sec. 4), and one level down of a stack of f32
// planes (the coarser levels).
//
// One warp per strip of 30 coarse columns walks down a run of coarse rows.
// Lane l owns coarse column x = 30 s + l - 1 and with it the fine columns 2x
// and 2x+1 (clamped).  For every fine row it forms the source values at its two
// fine columns (remap: loads their RGB, forms gray, the K remapped values and
// gray itself as channel K; planes: loads them) and per channel takes the x
// pass of the binomial [1,4,6,4,1]/16 at fine column 2x from its own pair and
// its neighbours' (warp shuffles).  Lanes 0 and 31 only feed their neighbours.
// The y pass is three accumulators per channel: each fine row adds its tap to
// the (up to three) outputs whose 5-row window holds it, in tap order, so the
// float operations are exactly those of the two-pass expression (x pass, then
// y pass over the x-pass values).  An output completes at every second fine
// row and is stored then.  Nothing goes through shared memory.
//
// Remap cost: outside the band |g - g_k| <= sigma the remap is one
// multiply-add (op_ll_remap_outside, bit-identical to op_ll_remap there).  The
// host selects the remap kernel only when no gray value can lie in the band of
// three levels (sigma below the level spacing 1/(K-1), with a margin for the
// rounding of g - g_k and of g_k), so the full remap (divide and power) runs
// for the first two levels of the band at most, whatever the image.
#include <cuda_runtime.h>

#include <cstring>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

constexpr int kK = 8;            // intensity levels
constexpr int kC = kK + 1;       // channels: the K remaps, then gray
constexpr int kStripW = 30;      // coarse columns per warp

struct LLRowsParams {
  LLDownArgs a;
  float gk[kK];                  // level values k / (K-1), correctly rounded
  int strips, rows, units, vec;  // vec: pair loads are aligned (data, row and plane strides)
};

// x pass at fine column 2x from this lane's pair (2x, 2x+1) and its
// neighbours' (2x-2, 2x-1 from lane - 1; 2x+2 from lane + 1).
__device__ __forceinline__ float xpass(float v0, float v1) {
  const float l0 = __shfl_up_sync(0xffffffffu, v0, 1);
  const float l1 = __shfl_up_sync(0xffffffffu, v1, 1);
  const float r0 = __shfl_down_sync(0xffffffffu, v0, 1);
  return tap5_binomial16(l0, l1, v0, v1, r0);
}

// The y taps of fine row t (PH = t mod 6) for one channel: output o collects
// rows 2o .. 2o+4 into acc[o mod 3].  On even rows returns output t/2 - 2,
// which this row completes.
template <int PH>
__device__ __forceinline__ float ytaps(float (&acc)[3], float h) {
  constexpr int m = PH >> 1;  // t/2 mod 3 (even t), (t-1)/2 mod 3 (odd t)
  float fin = 0.0f;
  if ((PH & 1) == 0) {
    fin = __fmaf_rn(0.0625f, h, acc[(m + 1) % 3]);          // tap 4 of output t/2 - 2
    acc[(m + 2) % 3] = __fmaf_rn(0.375f, h, acc[(m + 2) % 3]);  // tap 2 of output t/2 - 1
    acc[m] = __fmul_rn(0.0625f, h);                             // tap 0 of output t/2
  } else {
    acc[m] = __fmaf_rn(0.25f, h, acc[m]);                       // tap 1 of output (t-1)/2
    acc[(m + 2) % 3] = __fmaf_rn(0.25f, h, acc[(m + 2) % 3]);  // tap 3 of output (t-1)/2 - 1
  }
  return fin;
}

// Geometry of one warp's run: coarse rows [y0, y0 + nout) at coarse column x.
struct RunGeom {
  int x, cx0, cx1, fy0, nout, T, y0;
  bool pair, prod;
  __device__ __forceinline__ void init(int strip, int run_idx, int rows, int Wf, int Wc, int Hc, bool vec) {
    const int lane = threadIdx.x & 31;
    x = strip * kStripW + lane - 1;
    cx0 = iclamp(2 * x, 0, Wf - 1);
    cx1 = iclamp(2 * x + 1, 0, Wf - 1);
    pair = vec && 2 * x >= 0 && 2 * x + 1 <= Wf - 1;
    prod = lane >= 1 && lane <= kStripW && x < Wc;
    y0 = run_idx * rows;
    nout = imin(rows, Hc - y0);
    fy0 = 2 * y0 - 2;
    T = 2 * nout + 3;  // fine rows 2 y0 - 2 .. 2 (y0 + nout - 1) + 2
  }
};

// Runs row<PH>(t) for t = 0 .. T-1 with PH = t mod 6 known at compile time.
template <class R>
__device__ __forceinline__ void walk_rows(R& r, int T) {
  for (int t = 0; t < T; t += 6) {
    r.template row<0>(t);
    if (t + 1 >= T) break;
    r.template row<1>(t + 1);
    if (t + 2 >= T) break;
    r.template row<2>(t + 2);
    if (t + 3 >= T) break;
    r.template row<3>(t + 3);
    if (t + 4 >= T) break;
    r.template row<4>(t + 4);
    if (t + 5 >= T) break;
    r.template row<5>(t + 5);
  }
}

// One fine row of the input at the lane's two fine columns.
template <int IDT>
struct Px;

template <>
struct Px<HP_U16> {
  unsigned w[3];
  __device__ __forceinline__ float get(int c, int j) const { return (float)(j ? (w[c] >> 16) : (w[c] & 0xffffu)); }
  __device__ __forceinline__ void load(const char* row, long long ps, int cx0, int cx1, bool pair) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const char* q = row + c * ps;
      if (pair) {
        w[c] = __ldg(reinterpret_cast<const unsigned*>(q) + (cx0 >> 1));
      } else {
        const unsigned short* s = reinterpret_cast<const unsigned short*>(q);
        w[c] = (unsigned)__ldg(s + cx0) | ((unsigned)__ldg(s + cx1) << 16);
      }
    }
  }
};

template <>
struct Px<HP_F32> {
  float2 w[3];
  __device__ __forceinline__ float get(int c, int j) const { return j ? w[c].y : w[c].x; }
  __device__ __forceinline__ void load(const char* row, long long ps, int cx0, int cx1, bool pair) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const char* q = row + c * ps;
      if (pair) {
        w[c] = __ldg(reinterpret_cast<const float2*>(q) + (cx0 >> 1));
      } else {
        const float* s = reinterpret_cast<const float*>(q);
        w[c] = make_float2(__ldg(s + cx0), __ldg(s + cx1));
      }
    }
  }
};

// The remap source: gray of the input, its K remaps and gray itself.
// F32S: gray, remap and output stored as f32 (no rounding steps).
template <int IDT, bool F32S>
struct RemapRun {
  const LLRowsParams& P;
  const float* gks;    // the level table in shared memory (dynamic index)
  RunGeom G;
  float acc[kC][3];
  Px<IDT> cur, nxt;

  __device__ __forceinline__ RemapRun(const LLRowsParams& p, const float* g) : P(p), gks(g) {}

  __device__ __forceinline__ float rs(int st, float v) const { return F32S ? v : round_storage(st, v); }

  __device__ __forceinline__ void fetch(Px<IDT>& px, int t) const {
    const int f = iclamp(G.fy0 + t, 0, P.a.src.h - 1);
    px.load((const char*)P.a.src.data + (long long)f * P.a.src.rs, P.a.src.ps, G.cx0, G.cx1, G.pair);
  }

  __device__ __forceinline__ void store(int c, int y, float v) const {
    if (F32S) {
      reinterpret_cast<float*>((char*)P.a.out.data + (long long)c * P.a.out.ps + (long long)y * P.a.out.rs)[G.x] = v;
    } else {
      store_px(P.a.out, c, G.x, y, round_storage(P.a.st_out, v));
    }
  }

  template <int PH>
  __device__ __forceinline__ void row(int t) {
    const LLDownArgs& a = P.a;
    if (t + 1 < G.T) fetch(nxt, t + 1);
    float g[2], pa[2], pb[2];
    int ka[2], kb[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      g[j] = rs(a.st_gray, op_gray(cur.get(0, j), cur.get(1, j), cur.get(2, j), a.gray_scale));
      unsigned m = 0;
#pragma unroll
      for (int k = 0; k < kK; ++k) m |= fabsf(__fsub_rn(g[j], P.gk[k])) <= a.sigma ? 1u << k : 0u;
      ka[j] = __ffs(m) - 1;            // first level in the band, -1 if none
      kb[j] = __ffs(m & (m - 1)) - 1;  // second level, -1 if none
      pa[j] = op_ll_remap(g[j], gks[ka[j] & (kK - 1)], a.sigma, a.alpha, a.beta);
      pb[j] = op_ll_remap(g[j], gks[kb[j] & (kK - 1)], a.sigma, a.alpha, a.beta);
    }
    const int ofin = (t >> 1) - 2;
    const bool st = (PH & 1) == 0 && G.prod && ofin >= 0 && ofin < G.nout;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      float v[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float r;
        if (c < kK) {
          const float d = __fsub_rn(g[j], P.gk[c]);
          r = op_ll_remap_outside(d, fabsf(d), P.gk[c], a.sigma, a.beta);
          r = c == ka[j] ? pa[j] : r;
          r = c == kb[j] ? pb[j] : r;
        } else {
          r = g[j];
        }
        v[j] = rs(a.st_remap, r);
      }
      const float fin = ytaps<PH>(acc[c], xpass(v[0], v[1]));
      if (st) store(c, G.y0 + ofin, fin);
    }
    cur = nxt;
  }

  __device__ __forceinline__ void run(int strip, int run_idx) {
    G.init(strip, run_idx, P.rows, P.a.src.w, P.a.out.w, P.a.out.h, P.vec);
#pragma unroll
    for (int c = 0; c < kC; ++c)
#pragma unroll
      for (int s = 0; s < 3; ++s) acc[c][s] = 0.0f;
    fetch(cur, 0);
    walk_rows(*this, G.T);
  }
};

// The plane source: CG channels (from channel c0) of a stack of f32 planes.
// F32S: the output stored as f32.
template <int CG, bool F32S>
struct PlaneRun {
  const LLRowsParams& P;
  RunGeom G;
  int c0;
  float acc[CG][3];
  float2 cur[CG], nxt[CG], nxt2[CG];  // rows t, t+1, t+2: two rows of loads in flight

  __device__ __forceinline__ explicit PlaneRun(const LLRowsParams& p) : P(p) {}

  __device__ __forceinline__ void fetch(float2 (&px)[CG], int t) const {
    const int f = iclamp(G.fy0 + t, 0, P.a.src.h - 1);
    const char* row = (const char*)P.a.src.data + (long long)c0 * P.a.src.ps + (long long)f * P.a.src.rs;
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      const float* q = reinterpret_cast<const float*>(row + c * P.a.src.ps);
      px[c] = G.pair ? __ldg(reinterpret_cast<const float2*>(q) + (G.cx0 >> 1))
                     : make_float2(__ldg(q + G.cx0), __ldg(q + G.cx1));
    }
  }

  __device__ __forceinline__ void store(int c, int y, float v) const {
    if (F32S) {
      reinterpret_cast<float*>((char*)P.a.out.data + (long long)c * P.a.out.ps + (long long)y * P.a.out.rs)[G.x] = v;
    } else {
      store_px(P.a.out, c, G.x, y, round_storage(P.a.st_out, v));
    }
  }

  template <int PH>
  __device__ __forceinline__ void row(int t) {
    if (t + 2 < G.T) fetch(nxt2, t + 2);
    const int ofin = (t >> 1) - 2;
    const bool st = (PH & 1) == 0 && G.prod && ofin >= 0 && ofin < G.nout;
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      const float fin = ytaps<PH>(acc[c], xpass(cur[c].x, cur[c].y));
      if (st) store(c0 + c, G.y0 + ofin, fin);
    }
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      cur[c] = nxt[c];
      nxt[c] = nxt2[c];
    }
  }

  __device__ __forceinline__ void run(int strip, int run_idx, int group) {
    G.init(strip, run_idx, P.rows, P.a.src.w, P.a.out.w, P.a.out.h, P.vec);
    c0 = group * CG;
#pragma unroll
    for (int c = 0; c < CG; ++c)
#pragma unroll
      for (int s = 0; s < 3; ++s) acc[c][s] = 0.0f;
    fetch(cur, 0);
    fetch(nxt, 1);  // T >= 5
    walk_rows(*this, G.T);
  }
};

template <int IDT, bool F32S>
__global__ void __launch_bounds__(256, 2) k_ll_remap_rows(const LLRowsParams P) {
  grid_dep_wait();
  __shared__ float gks[kK];
  if (threadIdx.x < kK) gks[threadIdx.x] = P.gk[threadIdx.x];
  __syncthreads();
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < P.units; u += nw) {
    RemapRun<IDT, F32S> r(P, gks);
    r.run(u % P.strips, u / P.strips);
  }
}

// One level down of C f32 planes, CG channels per warp unit.
template <int CG, bool F32S>
__global__ void __launch_bounds__(256, 2) k_ll_down_rows(const LLRowsParams P) {
  grid_dep_wait();
  const int groups = P.a.C / CG;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < P.units; u += nw) {
    const int rest = u / P.strips;
    PlaneRun<CG, F32S> r(P);
    r.run(u % P.strips, rest / groups, rest % groups);
  }
}

typedef void (*RemapKernel)(LLRowsParams);

// Three channels per unit where the count allows (nine would hold 27
// accumulators and 54 prefetched values per lane, past the register budget).
RemapKernel pick_down_kernel(int C, bool f32s) {
  static const RemapKernel ks[4] = {k_ll_down_rows<1, false>, k_ll_down_rows<1, true>, k_ll_down_rows<3, false>,
                                    k_ll_down_rows<3, true>};
  return ks[(C % 3 == 0 ? 2 : 0) + (f32s ? 1 : 0)];
}

int down_group(int C) { return C % 3 == 0 ? 3 : 1; }

int resident_ctas(RemapKernel kern, int threads, int need) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return need < 2 * 152 ? need : 2 * 152;  // no device to ask: two CTAs on each of 152 SMs
  }
  return need < sms * per_sm ? need : sms * per_sm;
}

RemapKernel pick_kernel(int in_dtype, bool f32s, int* variant) {
  const int v = (in_dtype == HP_F32 ? 2 : 0) + (f32s ? 1 : 0);
  static const RemapKernel ks[4] = {k_ll_remap_rows<HP_U16, false>, k_ll_remap_rows<HP_U16, true>,
                                    k_ll_remap_rows<HP_F32, false>, k_ll_remap_rows<HP_F32, true>};
  *variant = v;
  return ks[v];
}

bool all_f32(const LLDownArgs& a) {
  return a.st_gray == HP_F32 && a.st_remap == HP_F32 && a.st_out == HP_F32 && a.out.dtype == HP_F32;
}

}  // namespace

int ll_remap_rows_strip_w() { return kStripW; }

// The streaming kernel covers K = 8 levels with gray as channel K, u16 or f32
// input, and sigma below the level spacing: |g - g_k| <= sigma can then hold
// for two levels at most.  (Computed |g - g_k| is within 2^-24 sigma
// of the exact value when it is <= sigma, and g_k within 2^-24 of k/(K-1); the
// 1e-6 margin covers both.)  sigma must be positive: at sigma <= 0 the full
// remap's d = 0 case is not inside the band.
int ll_remap_rows_ok(const LLDownArgs& a, int in_dtype) {
  return a.remap && a.K == kK && a.C == kC && (in_dtype == HP_U16 || in_dtype == HP_F32) && a.sigma > 0.0f &&
         2.0 * (double)a.sigma + 1e-6 < 2.0 / (kK - 1);
}

int ll_remap_rows_grid(int in_dtype, int units, int threads) {
  const int nw = threads / 32;
  int variant = 0;
  return resident_ctas(pick_kernel(in_dtype, true, &variant), threads, (units + nw - 1) / nw);
}

// The plane kernel covers any channel count of f32 planes (3 or 1 channels
// per warp unit).
int ll_down_rows_ok(const LLDownArgs& a, int src_dtype) { return !a.remap && src_dtype == HP_F32 && a.C >= 1; }

int ll_down_rows_groups(int C) { return C / down_group(C); }

int ll_down_rows_grid(int C, int units, int threads) {
  const int nw = threads / 32;
  return resident_ctas(pick_down_kernel(C, true), threads, (units + nw - 1) / nw);
}

int launch_ll_down_rows(const LLDownArgs& a, int rows, int threads, int grid, void* stream) {
  if (a.src.dtype != HP_F32 || a.remap) return (int)cudaErrorInvalidValue;
  if (rows < 1 || threads < 32 || threads > 256 || threads % 32 || grid < 1) return (int)cudaErrorInvalidValue;
  LLRowsParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  kp.strips = (a.out.w + kStripW - 1) / kStripW;
  kp.rows = rows;
  kp.units = kp.strips * ll_down_rows_groups(a.C) * ((a.out.h + rows - 1) / rows);
  kp.vec = ((long long)(size_t)a.src.data % 8 == 0) && a.src.rs % 8 == 0 && a.src.ps % 8 == 0;
  const bool f32s = a.st_out == HP_F32 && a.out.dtype == HP_F32;
  { const int le_ = launch_kernel(pick_down_kernel(a.C, f32s), dim3(grid), dim3(threads), 0, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

int launch_ll_remap_rows(const LLDownArgs& a, int rows, int threads, int grid, void* stream) {
  if (a.src.dtype != HP_U16 && a.src.dtype != HP_F32) return (int)cudaErrorInvalidValue;
  if (rows < 1 || threads < 32 || threads > 256 || threads % 32 || grid < 1) return (int)cudaErrorInvalidValue;
  LLRowsParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  // k / (K-1) in IEEE single precision: the correctly rounded quotient, equal
  // to the device's __fdiv_rn of the same operands.
  for (int k = 0; k < kK; ++k) kp.gk[k] = (float)k / (float)(kK - 1);
  kp.strips = (a.out.w + kStripW - 1) / kStripW;
  kp.rows = rows;
  kp.units = kp.strips * ((a.out.h + rows - 1) / rows);
  const long long al = a.src.dtype == HP_F32 ? 8 : 4;
  kp.vec = ((long long)(size_t)a.src.data % al == 0) && a.src.rs % al == 0 && a.src.ps % al == 0;
  int variant;
  RemapKernel kern = pick_kernel(a.src.dtype, all_f32(a), &variant);
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(threads), 0, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
