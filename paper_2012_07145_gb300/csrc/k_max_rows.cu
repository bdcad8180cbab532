// Max filter, streaming (the max filter app of Sec. 6): per channel, the
// maximum over the (2RX+1) x (2RY+1) window at clamped coordinates, for a
// group of one window-maximum stage (square, horizontal or vertical) or of a
// horizontal and a vertical one of the same radius (the same values as the
// square window: the clamp acts on each coordinate separately).
//
// One warp per strip of 120 columns of one plane walks down a run of rows.
// Lane l holds the 4 columns x0 + 4 (l - 1) .. + 3 of every input row (lanes 0
// and 31 only feed their neighbours, R <= 4 columns each side).  f32, f16 and
// bf16 inputs arrive as TMA boxes of 4 rows x 128 columns through a ring of 3
// shared-memory slots private to the warp, issued in the order the warp will
// read them (across its runs), so up to 12 rows per warp are in flight without
// holding registers; other input types are loaded row by row from global
// memory, the next row's loads in flight while a row is processed.  Per row:
// the horizontal maxima of the lane's 4 columns from its own values and its
// neighbours' (warp shuffles), kept in a ring of 2RY+1 rows; from row 2RY on,
// the maximum over the ring is an output row.  Clamp to edge: from TMA boxes,
// a column outside the image takes the edge column's value (a shuffle from the
// lane that holds it), row 0's maxima also stand for the rows above it and
// row H - 1's for the rows below.  Maxima are exact, so the order
// of the comparisons does not matter; the group's storage roundings are
// applied to the final maximum (rounding is monotone, so rounding the maximum
// equals the maximum of rounded values).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStripW = 120;  // output columns per warp
constexpr int kBoxRows = 4;     // rows per TMA box
constexpr int kRing = 3;        // boxes per warp ring
constexpr int kBarBytes = 512;  // mbarriers of up to 16 warps x kRing

struct MaxParams {
  CUtensorMap tmap;
  MaxArgs a;
  int strips, runs, units;
};

// TMA boxes start at the strip's first column less 4 (lane 0's), less `pad`
// columns where that start is not 16-byte aligned (2-byte inputs); a box row
// is a multiple of 16 bytes, and every slot starts on a 128-byte boundary (the
// shared-memory destination of a tensor copy).
struct BoxGeom {
  int pad, box_w, box_bytes, slot_bytes;
};

__host__ __device__ inline BoxGeom box_geom(int esize) {
  BoxGeom g;
  g.pad = esize == 2 ? 4 : 0;
  g.box_w = esize == 2 ? 136 : 128;
  g.box_bytes = g.box_w * kBoxRows * esize;
  g.slot_bytes = (g.box_bytes + 127) / 128 * 128;
  return g;
}

__device__ __forceinline__ int dt_size(int dt) { return dt == HP_F32 ? 4 : 2; }

// A run of rows of one strip of one plane: input rows y0 - RY .. y0 + nout + RY - 1.
struct Unit {
  int plane, xs, y0, nout, n_in, nbox;
};

__device__ __forceinline__ Unit unit_geom(const MaxParams& P, int u, int ry) {
  Unit U;
  const int per_plane = P.strips * P.runs;
  U.plane = u / per_plane;
  const int v = u - U.plane * per_plane;
  const int run = v / P.strips, strip = v - run * P.strips;
  U.xs = strip * kStripW;
  U.y0 = run * P.a.rows;
  U.nout = imin(P.a.rows, P.a.in.h - U.y0);
  U.n_in = U.nout + 2 * ry;
  U.nbox = (U.n_in + kBoxRows - 1) / kBoxRows;
  return U;
}

// The warp's ring: box q (in issue order, which is the order of use) lives in
// slot q % kRing and completes phase (q / kRing) & 1 of that slot's mbarrier.
struct Ring {
  unsigned char* slots;
  uint64_t* bars;
  unsigned issued, released;
  int iu, ij;  // next box to issue: unit and box within it
  Unit IU;     // geometry of unit iu
};

__device__ __forceinline__ void issue_one(const MaxParams& P, const BoxGeom& g, Ring& R, int stride, int lane, int ry) {
  if (R.iu >= P.units) return;
  if (lane == 0) {
    const int s = R.issued % kRing;
    // the warp's reads of this slot (its previous box) come before the copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(R.bars + s, (unsigned)g.box_bytes);
    tma_load_3d(R.slots + s * g.slot_bytes, &P.tmap, R.IU.xs - 4 - g.pad, R.IU.y0 - ry + R.ij * kBoxRows, R.IU.plane,
                R.bars + s);
  }
  ++R.issued;
  if (++R.ij == R.IU.nbox) {
    R.ij = 0;
    R.iu += stride;
    if (R.iu < P.units) R.IU = unit_geom(P, R.iu, ry);
  }
}

// Every lane's value at a column outside [0, W) becomes the value at the
// nearest column inside, fetched from the lane that holds it.
__device__ __forceinline__ void clamp_cols(float (&v)[4], int c0, int x0, int W) {
  float o[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + k;
    const int s = min(max(c, 0), W - 1);
    const int off = s - x0;
    const int sl = off >> 2, sk = off & 3;
    const float t0 = __shfl_sync(kFull, v[0], sl), t1 = __shfl_sync(kFull, v[1], sl);
    const float t2 = __shfl_sync(kFull, v[2], sl), t3 = __shfl_sync(kFull, v[3], sl);
    const float t = sk == 0 ? t0 : sk == 1 ? t1 : sk == 2 ? t2 : t3;
    o[k] = c == s ? v[k] : t;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = o[k];
}

template <int IDT>
__device__ __forceinline__ void load4_smem(const unsigned char* p, float (&v)[4]) {
  if (IDT == HP_F32) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    const unsigned u[2] = {q.x, q.y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const unsigned short lo = (unsigned short)(u[i] & 0xffffu), hi = (unsigned short)(u[i] >> 16);
      if (IDT == HP_BF16) {
        v[2 * i] = __bfloat162float(__ushort_as_bfloat16(lo));
        v[2 * i + 1] = __bfloat162float(__ushort_as_bfloat16(hi));
      } else {
        v[2 * i] = __half2float(__ushort_as_half(lo));
        v[2 * i + 1] = __half2float(__ushort_as_half(hi));
      }
    }
  }
}

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

// The same run with f32 or bf16 input rows taken from the warp's TMA ring.
template <int IDT, int RX, int RY, bool RND>
struct MaxRunTma {
  static constexpr int N = 2 * RY + 1;
  static constexpr int kEsize = IDT == HP_F32 ? 4 : 2;
  const MaxParams& P;
  const BoxGeom& g;
  Ring& R;
  const Unit U;
  const int lane, stride, c0, W, H;
  const bool hb, vedge, prod;
  const unsigned char* slot;
  unsigned q;  // box being read
  int rr;      // row within it
  float ring[N][4];

  __device__ __forceinline__ MaxRunTma(const MaxParams& P_, const BoxGeom& g_, Ring& R_, const Unit& U_, int lane_,
                                       int stride_)
      : P(P_), g(g_), R(R_), U(U_), lane(lane_), stride(stride_), c0(U_.xs - 4 + 4 * lane_), W(P_.a.in.w),
        H(P_.a.in.h), hb(U_.xs - 4 < 0 || U_.xs + 124 > P_.a.in.w), vedge(U_.y0 < RY || U_.y0 + U_.nout + RY > P_.a.in.h),
        prod(lane_ >= 1 && lane_ <= 30 && U_.xs - 4 + 4 * lane_ < P_.a.out.w), slot(nullptr), q(R_.released), rr(0) {}

  __device__ __forceinline__ bool wait_box() {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_poll(R.bars + q % kRing, (q / kRing) & 1u, 2000000000ull);
    __syncwarp();
    ok = __shfl_sync(kFull, ok, 0);
    slot = R.slots + (q % kRing) * g.slot_bytes + (4 * lane + g.pad) * kEsize;
    return ok != 0;
  }

  __device__ __forceinline__ void release_box() {
    ++q;
    __syncwarp();
    R.released = q;
    issue_one(P, g, R, stride, lane, RY);
  }

  // Input row t of the run (image row y0 - RY + t) into ring slot S; from
  // t = 2RY on, output row t - 2RY.  False: a box never arrived.
  template <int S>
  __device__ __forceinline__ bool row(int t) {
    if (rr == 0 && !wait_box()) return false;
    float v[4];
    load4_smem<IDT>(slot + rr * g.box_w * kEsize, v);
    if (++rr == kBoxRows) {
      rr = 0;
      release_box();
    }
    if (hb) clamp_cols(v, c0, U.xs - 4, W);
    float a[12];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = __shfl_up_sync(kFull, v[k], 1);
      a[4 + k] = v[k];
      a[8 + k] = __shfl_down_sync(kFull, v[k], 1);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float m = a[4 + k - RX];
#pragma unroll
      for (int i = 5 + k - RX; i <= 4 + k + RX; ++i) m = fmaxf(m, a[i]);
      ring[S][k] = m;
    }
    if (vedge) {
      const int r = U.y0 - RY + t;
      if (r == 0) {  // rows -RY .. -1 are row 0
#pragma unroll
        for (int j = 1; j <= RY; ++j)
#pragma unroll
          for (int k = 0; k < 4; ++k) ring[(S + N - j) % N][k] = ring[S][k];
      }
      if (r >= H) {  // rows below the image are row H - 1
#pragma unroll
        for (int k = 0; k < 4; ++k) ring[S][k] = ring[(S + N - 1) % N][k];
      }
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
        const int y = U.y0 + t - 2 * RY;
        const ImgView& ov = P.a.out;
        if (!RND && c0 + 3 < ov.w) {
          reinterpret_cast<float4*>((char*)ov.data + (long long)U.plane * ov.ps + (long long)y * ov.rs)[c0 >> 2] =
              make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (c0 + k < ov.w) store_px(ov, U.plane, c0 + k, y, o[k]);
        }
      }
    }
    return true;
  }

  // 1: the row ran, 0: past the run's end, -1: a box never arrived
  template <int SS>
  __device__ __forceinline__ int step(int t) {
    if (t + SS >= U.n_in) return 0;
    return row<SS>(t + SS) ? 1 : -1;
  }

  __device__ __forceinline__ bool run() {
    for (int t = 0; t < U.n_in; t += N) {
      int e;
      if ((e = step<0>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 1 && (e = step<(N > 1 ? 1 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 2 && (e = step<(N > 2 ? 2 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 3 && (e = step<(N > 3 ? 3 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 4 && (e = step<(N > 4 ? 4 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 5 && (e = step<(N > 5 ? 5 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 6 && (e = step<(N > 6 ? 6 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 7 && (e = step<(N > 7 ? 7 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
      if (N > 8 && (e = step<(N > 8 ? 8 : 0)>(t)) <= 0) { if (e < 0) return false; break; }
    }
    if (rr != 0) release_box();  // the run's last box, partly read
    return true;
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

template <int IDT, int RX, int RY, bool RND>
__global__ void __launch_bounds__(256, max_rows_min_blocks<RX, RY>()) k_max_rows_tma(const __grid_constant__ MaxParams P) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gw = blockIdx.x * nw + warp, stride = gridDim.x * nw;
  if (gw >= P.units) return;
  const BoxGeom g = box_geom(IDT == HP_F32 ? 4 : 2);
  Ring R;
  R.bars = reinterpret_cast<uint64_t*>(base) + warp * kRing;
  R.slots = base + kBarBytes + warp * kRing * g.slot_bytes;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < kRing; ++i) mbar_init(R.bars + i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  R.issued = R.released = 0;
  R.iu = gw;
  R.ij = 0;
  R.IU = unit_geom(P, gw, RY);
  for (int i = 0; i < kRing; ++i) issue_one(P, g, R, stride, lane, RY);
  for (int u = gw; u < P.units; u += stride) {
    MaxRunTma<IDT, RX, RY, RND> r(P, g, R, unit_geom(P, u, RY), lane, stride);
    if (!r.run()) {
      // a box never arrived: report, wait (bounded) for the copies still in
      // flight into this warp's slots, and stop
      if (lane == 0) {
        atomicExch(P.a.err, 1);
        for (unsigned b = R.released; b < R.issued; ++b) mbar_wait_poll(R.bars + b % kRing, (b / kRing) & 1u, 100000000ull);
      }
      __syncwarp();
      return;
    }
  }
}

typedef void (*MaxKernel)(MaxParams);

// shape 0: square window, 1: horizontal only, 2: vertical only; f32 and bf16
// inputs take the TMA ring
template <int IDT, int R, bool RND>
MaxKernel by_shape(int shape) {
  if (IDT == HP_F32 || IDT == HP_BF16) {
    constexpr int T = IDT == HP_F32 || IDT == HP_BF16 ? IDT : HP_F32;
    return shape == 1 ? k_max_rows_tma<T, R, 0, RND> : shape == 2 ? k_max_rows_tma<T, 0, R, RND>
                                                                  : k_max_rows_tma<T, R, R, RND>;
  }
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

bool uses_tma(const MaxArgs& a) { return a.in.dtype == HP_F32 || a.in.dtype == HP_BF16; }

}  // namespace

int max_rows_strip_w() { return kStripW; }

int max_rows_smem_bytes(const MaxArgs& a, int threads) {
  if (!uses_tma(a)) return 0;
  return 128 + kBarBytes + (threads / 32) * kRing * box_geom(a.in.dtype == HP_F32 ? 4 : 2).slot_bytes;
}

int max_rows_grid(const MaxArgs& a, int units, int threads) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0;
  const MaxKernel kern = pick_kernel(a);
  const int smem = max_rows_smem_bytes(a, threads);
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      (smem && allow_max_dynamic_smem((const void*)kern) != 0) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) {
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
  const MaxKernel kern = pick_kernel(a);
  const int smem = max_rows_smem_bytes(a, a.threads);
  if (smem) {
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    const int esize = a.in.dtype == HP_F32 ? 4 : 2;
    const CUtensorMapDataType tdt = a.in.dtype == HP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps,
                       box_geom(esize).box_w, kBoxRows, 1))
      return (int)cudaErrorInvalidValue;
  }
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(a.threads), smem, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
