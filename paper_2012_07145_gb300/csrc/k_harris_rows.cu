// Streaming Harris corner response: the whole Harris DAG (gray, 3x3 Sobel
// gradients, products, 3x3 box sums, det - k tr^2) in one kernel with every
// intermediate in registers (thread-level fusion, Sec. 2 "Fusion Options").
//
// Each warp owns a strip of output columns, four per lane, and walks down a run
// of rows.  Input rows arrive as TMA boxes (three planes, kBoxRows rows, 128
// columns) through a ring of shared-memory slots private to the warp: while the
// warp computes on one box the next kRing - 1 are in flight, and no barrier
// wider than the warp is ever taken.  Horizontal neighbours come from warp
// shuffles (the outer lanes only feed their neighbours), vertical neighbours
// from 3-row register windows, so a value is computed once per strip.  Stage
// expressions and per-stage rounding are those of stage_math.cuh, so the result
// is bit-identical to every other schedule of the pipeline.
//
// Boundary conditions (each stencil clamps on its own producer, Sec. 3): an x
// pass at the image's first or last column takes the edge column itself as the
// missing neighbour (a select on the shuffled value); rows outside take the
// nearest edge row of the same stage (a copy inside the register window).
#include <cuda.h>
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

// Box heights stay a power of two: boxes of 3 or 5 rows measured several
// times slower to arrive than boxes of 2 or 4.
constexpr int kBoxRows = 2;       // rows per TMA box
constexpr int kRing = 4;          // boxes per warp ring
constexpr int kBarBytes = 512;    // mbarriers of up to 16 warps x kRing
constexpr unsigned kFull = 0xffffffffu;

struct StripGeom {
  int halo_lanes;  // lanes on each side that only feed neighbours
  int strip_w;     // output columns per strip: 4 (32 - 2 halo_lanes)
  int slot_bytes;  // one ring slot: 128 columns x kBoxRows rows x 3 planes
};

// A TMA box must start on a 16-byte boundary: 4 columns of a 4-byte input,
// 8 of a 2-byte one, which sets the halo on the left (and, by symmetry, right).
__host__ __device__ inline StripGeom strip_geom(int esize) {
  StripGeom g;
  g.halo_lanes = esize == 4 ? 1 : 2;
  g.strip_w = 4 * (32 - 2 * g.halo_lanes);
  g.slot_bytes = 128 * kBoxRows * 3 * esize;
  return g;
}

struct RowsParams {
  CUtensorMap tmap;
  HarrisArgs a;
  int strips, units, rows;  // strips across the image; units = strips x row runs; rows per run
};

struct Unit {
  int x0, oy, n_in, nbox;  // x0: image column of lane 0's first column; n_in input rows from oy - 2
  int img;                 // image of a batch (input planes 3 img .. 3 img + 2, output plane img)
};

__device__ __forceinline__ Unit unit_geom(const RowsParams& kp, const StripGeom& g, int u) {
  Unit U;
  const int per_img = kp.units / (kp.a.batch > 1 ? kp.a.batch : 1);
  U.img = u / per_img;
  u -= U.img * per_img;
  const int s = u % kp.strips, r = u / kp.strips;
  U.x0 = s * g.strip_w - 4 * g.halo_lanes;
  U.oy = r * kp.rows;
  U.n_in = min(kp.rows, kp.a.out.h - U.oy) + 4;
  U.nbox = (U.n_in + kBoxRows - 1) / kBoxRows;
  return U;
}

// The warp's ring: boxes are numbered in issue order (which is also the order
// of use); box q lives in slot q % kRing and completes phase (q / kRing) & 1
// of that slot's mbarrier.
struct Ring {
  unsigned char* slots;
  uint64_t* bars;
  unsigned issued, released;
  int iu, ij;   // next box to issue: unit and box within the unit
  Unit IU;      // geometry of unit iu
};

__device__ __forceinline__ void issue_one(const RowsParams& kp, const StripGeom& g, Ring& R, int stride, int lane) {
  if (R.iu >= kp.units) return;
  if (lane == 0) {
    const int s = R.issued % kRing;
    mbar_arrive_expect_tx(R.bars + s, (unsigned)g.slot_bytes);
    tma_load_3d(R.slots + s * g.slot_bytes, &kp.tmap, R.IU.x0, R.IU.oy - 2 + R.ij * kBoxRows, 3 * R.IU.img,
                R.bars + s);
  }
  ++R.issued;
  if (++R.ij == R.IU.nbox) {
    R.ij = 0;
    R.iu += stride;
    if (R.iu < kp.units) R.IU = unit_geom(kp, g, R.iu);
  }
}

// Left and right neighbours of the lane's four columns for a 3-tap x pass,
// with the boundary condition of the stage they belong to: the neighbour
// outside the image is the edge column itself.  Column 0 always sits first in
// a lane (strips start on multiples of 4); column W - 1 may sit anywhere.
struct Edges {
  bool left;      // the lane's first column is column 0
  bool right[4];  // column k of the lane is column W - 1
};

__device__ __forceinline__ void neighbours(const float (&v)[4], const Edges& e, float (&l)[4], float (&r)[4]) {
  const float up = __shfl_up_sync(kFull, v[3], 1), dn = __shfl_down_sync(kFull, v[0], 1);
  l[0] = e.left ? v[0] : up;
  l[1] = v[0];
  l[2] = v[1];
  l[3] = v[2];
  r[0] = e.right[0] ? v[0] : v[1];
  r[1] = e.right[1] ? v[1] : v[2];
  r[2] = e.right[2] ? v[2] : v[3];
  r[3] = e.right[3] ? v[3] : dn;
}


// The stencil weights of the five 3x3 stages (x taps then y taps, in the
// order Ix, Iy, Sxx, Syy, Sxy).  With SPEC the weights are the Sobel and box
// constants the pipeline was checked to hold, as compile-time values: the
// compiler then drops the exact products by 1 and -1 and turns fma(1, c, s)
// into the same-rounded c + s, so the arithmetic, and every result bit, is
// that of the runtime-weight expression.
template <bool SPEC>
struct Weights {
  const float (&w)[5][6];
  __device__ __forceinline__ Weights(const float (&w_)[5][6]) : w(w_) {}
  __device__ __forceinline__ float operator()(int q, int k) const { return w[q][k]; }
};
template <>
struct Weights<true> {
  __device__ __forceinline__ Weights(const float (&)[5][6]) {}
  __device__ __forceinline__ float operator()(int q, int k) const {
    // Ix: x [-1 0 1], y [1 2 1]; Iy: x [1 2 1], y [-1 0 1]; box sums: [1 1 1] both ways
    return q == 0 ? (k < 3 ? (float)(k - 1) : (k == 4 ? 2.0f : 1.0f))
         : q == 1 ? (k < 3 ? (k == 1 ? 2.0f : 1.0f) : (float)(k - 4))
                  : 1.0f;
  }
};

template <bool SPEC>
__device__ __forceinline__ float tapw(const Weights<SPEC>& w, int q, int k0, float a, float b, float c) {
  if (SPEC) {
    // w0 * a is exact for w0 = +-1: start from +-a (what tap3v's first product
    // rounds to) and keep its two fused steps; fma(1, c, s) is c + s either way
    const float w0 = w(q, k0), w1 = w(q, k0 + 1), w2 = w(q, k0 + 2);
    if (w0 == 1.0f || w0 == -1.0f) {
      const float s = __fmaf_rn(w1, b, w0 == 1.0f ? a : -a);
      return __fmaf_rn(w2, c, s);
    }
  }
  return tap3v(w(q, k0), w(q, k0 + 1), w(q, k0 + 2), a, b, c);
}

template <bool SPEC>
__device__ __forceinline__ void xpass3(const Weights<SPEC>& w, int q, const float (&l)[4], const float (&v)[4],
                                       const float (&r)[4], float (&h)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = tapw(w, q, 0, l[k], v[k], r[k]);
}

// A stage value rounded to its storage: RND 0 = every stage f32 (nothing to
// do), 2 = every stage bf16 (known at compile time), 3 = per stage.
template <int RND>
__device__ __forceinline__ float rs(float v, int dtype) {
  if (RND == 0) return v;
  if (RND == 2) return __bfloat162float(__float2bfloat16_rn(v));
  return round_storage(dtype, v);
}

// Four values rounded to the storage type; bf16 two at a time (one paired
// conversion, round-to-nearest-even per value: the same values as rs).
template <int RND>
__device__ __forceinline__ void rs4(float (&v)[4], int dtype) {
  if (RND == 2) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2 f = __bfloat1622float2(__floats2bfloat162_rn(v[2 * q], v[2 * q + 1]));
      v[2 * q] = f.x;
      v[2 * q + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = rs<RND>(v[k], dtype);
  }
}

__device__ __forceinline__ void load4(const unsigned char* p, int dtype, float (&v)[4]) {
  if (dtype == HP_F32) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    const unsigned u[2] = {q.x, q.y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const unsigned short lo = (unsigned short)(u[i] & 0xffffu), hi = (unsigned short)(u[i] >> 16);
      if (dtype == HP_BF16) {
        v[2 * i] = __bfloat162float(__ushort_as_bfloat16(lo));
        v[2 * i + 1] = __bfloat162float(__ushort_as_bfloat16(hi));
      } else {
        v[2 * i] = __half2float(__ushort_as_half(lo));
        v[2 * i + 1] = __half2float(__ushort_as_half(hi));
      }
    }
  }
}

// One run of rows of one strip.  Rows are numbered from the first input row
// (image row oy - 2): step t reads input row t, forms gradient/product row t - 1
// (from t >= 2) and emits output row t - 2 (from t >= 4).  Windows are indexed
// by row mod 3, so a loop unrolled three times keeps them in fixed registers.
template <int RND, int ODT, bool SPEC>
struct StripRun {
  const RowsParams& kp;
  const StripGeom& g;
  Ring& R;
  const Unit U;
  const int lane, stride, c0, esize;
  const Weights<SPEC> w;
  Edges e;
  const bool vedge;          // the run reads rows outside the image
  bool st_full, st_part;     // the lane stores four columns / some of its columns
  char* out_row;             // the next output row
  float hA[3][4], hB[3][4];  // x passes of gray with the Ix and Iy x-weights
  float sm[3][3][4];         // x passes of the three products
  unsigned q;                // box being read
  int rr;                    // row within it
  const unsigned char* slot;

  __device__ __forceinline__ StripRun(const RowsParams& kp_, const StripGeom& g_, Ring& R_, const Unit& U_, int lane_,
                                      int stride_)
      : kp(kp_), g(g_), R(R_), U(U_), lane(lane_), stride(stride_), c0(U_.x0 + 4 * lane_),
        esize(kp_.a.in.dtype == HP_F32 ? 4 : 2), w(kp_.a.w), vedge(U_.oy < 2 || U_.oy + U_.n_in - 2 > kp_.a.in.h),
        q(R_.released), rr(0), slot(nullptr) {
    const int W = kp.a.in.w;
    e.left = c0 == 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) e.right[k] = c0 + k == W - 1;
    const bool mine = lane >= g.halo_lanes && lane < 32 - g.halo_lanes;
    st_full = mine && c0 + 3 < W && ODT != 3;
    st_part = mine && c0 < W && !st_full;
    out_row = (char*)kp.a.out.data + (long long)U.img * kp.a.out.ps + (long long)U.oy * kp.a.out.rs;
  }

  // Waits for box q (one lane polls, bounded), then the warp reads it.
  __device__ __forceinline__ bool wait_box() {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_poll(R.bars + q % kRing, (q / kRing) & 1u, 2000000000ull);
    __syncwarp();
    ok = __shfl_sync(kFull, ok, 0);
    slot = R.slots + (q % kRing) * g.slot_bytes + lane * 4 * esize;
    return ok != 0;
  }

  // Frees box q's slot for the box kRing later in issue order.
  __device__ __forceinline__ void release_box() {
    ++q;
    __syncwarp();
    R.released = q;
    issue_one(kp, g, R, stride, lane);
  }

  // gray of input row r into window slot M, then both x passes.
  template <int M>
  __device__ __forceinline__ bool row_in(int r, bool edge) {
    const HarrisArgs& a = kp.a;
    if (rr == 0 && !wait_box()) return false;
    const unsigned char* p = slot + rr * 128 * esize;
    const int plane = 128 * kBoxRows * esize;
    float cr[4], cg[4], cb[4], gv[4];
    load4(p, a.in.dtype, cr);
    load4(p + plane, a.in.dtype, cg);
    load4(p + 2 * plane, a.in.dtype, cb);
    if (++rr == kBoxRows) {
      rr = 0;
      release_box();
    }
    if (SPEC || a.gray_scale == 1.0f) {  // x * 1 is exact: the same value as op_gray with scale 1
#pragma unroll
      for (int k = 0; k < 4; ++k) gv[k] = __fmaf_rn(0.114f, cb[k], __fmaf_rn(0.587f, cg[k], __fmul_rn(0.299f, cr[k])));
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) gv[k] = op_gray(cr[k], cg[k], cb[k], a.gray_scale);
    }
    rs4<RND>(gv, a.st[0]);
    float l[4], rt[4];
    neighbours(gv, e, l, rt);
    xpass3(w, 0, l, gv, rt, hA[M]);
    xpass3(w, 1, l, gv, rt, hB[M]);
    constexpr int P = (M + 2) % 3;  // the previous row's slot
    if (!edge) return true;
    if (r == 0) {                   // row -1 of gray is row 0
#pragma unroll
      for (int k = 0; k < 4; ++k) { hA[P][k] = hA[M][k]; hB[P][k] = hB[M][k]; }
    }
    if (r == a.in.h) {              // row H of gray is row H - 1
#pragma unroll
      for (int k = 0; k < 4; ++k) { hA[M][k] = hA[P][k]; hB[M][k] = hB[P][k]; }
    }
    return true;
  }

  // Gradients and products of row r - 1 (window rows r-2, r-1, r), then the x
  // passes of the box sums, into product slot (M + 2) % 3.
  template <int M>
  __device__ __forceinline__ void row_grad(int r, bool edge) {
    const HarrisArgs& a = kp.a;
    constexpr int I0 = (M + 1) % 3, I1 = (M + 2) % 3, I2 = M;
    constexpr int S = (M + 2) % 3, SP = (M + 1) % 3;  // this product row's slot; the previous one's
    float pr[3][4], ix[4], iy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ix[k] = tapw(w, 0, 3, hA[I0][k], hA[I1][k], hA[I2][k]);
      iy[k] = tapw(w, 1, 3, hB[I0][k], hB[I1][k], hB[I2][k]);
    }
    rs4<RND>(ix, a.st[1]);
    rs4<RND>(iy, a.st[2]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pr[0][k] = __fmul_rn(ix[k], ix[k]);
      pr[1][k] = __fmul_rn(iy[k], iy[k]);
      pr[2][k] = __fmul_rn(ix[k], iy[k]);
    }
    rs4<RND>(pr[0], a.st[3]);
    rs4<RND>(pr[1], a.st[4]);
    rs4<RND>(pr[2], a.st[5]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float l[4], rt[4];
      neighbours(pr[b], e, l, rt);
      xpass3(w, 2 + b, l, pr[b], rt, sm[S][b]);
    }
    if (!edge) return;
    if (r == 1) {           // product row 0 was just formed: row -1 is row 0
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 4; ++k) sm[SP][b][k] = sm[S][b][k];
    }
    if (r == a.in.h + 1) {  // product row H is row H - 1
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 4; ++k) sm[S][b][k] = sm[SP][b][k];
    }
  }

  // Box sums (y pass over product rows r-3, r-2, r-1) and the response of
  // output row r - 2 = image row y.
  template <int M>
  __device__ __forceinline__ void row_out() {
    const HarrisArgs& a = kp.a;
    constexpr int J0 = M, J1 = (M + 1) % 3, J2 = (M + 2) % 3;
    float o[4], sxx[4], syy[4], sxy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sxx[k] = tapw(w, 2, 3, sm[J0][0][k], sm[J1][0][k], sm[J2][0][k]);
      syy[k] = tapw(w, 3, 3, sm[J0][1][k], sm[J1][1][k], sm[J2][1][k]);
      sxy[k] = tapw(w, 4, 3, sm[J0][2][k], sm[J1][2][k], sm[J2][2][k]);
    }
    rs4<RND>(sxx, a.st[6]);
    rs4<RND>(syy, a.st[7]);
    rs4<RND>(sxy, a.st[8]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float v = op_harris(sxx[k], syy[k], sxy[k], a.k);
      o[k] = ODT == 3 ? round_storage(a.out.dtype, v) : v;
    }
    char* row = out_row;
    out_row += a.out.rs;
    if (st_full) {
      if (ODT == 0) {
        *reinterpret_cast<float4*>(row + 4LL * c0) = make_float4(o[0], o[1], o[2], o[3]);
      } else {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(o[0], o[1]), p1 = __floats2bfloat162_rn(o[2], o[3]);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&p0);
        u.y = *reinterpret_cast<unsigned*>(&p1);
        *reinterpret_cast<uint2*>(row + 2LL * c0) = u;
      }
    } else if (st_part) {
      const int y = (int)((row - (char*)a.out.data - (long long)U.img * a.out.ps) / a.out.rs);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (c0 + k < a.out.w) store_px(a.out, U.img, c0 + k, y, o[k]);
    }
  }

  template <int M>
  __device__ __forceinline__ bool step(int t) {
    const int r = U.oy - 2 + t;
    const bool edge = vedge && (r < 2 || r >= kp.a.in.h);  // a window row outside the image may need a copy
    if (!row_in<M>(r, edge)) return false;
    if (t >= 2) row_grad<M>(r, edge);
    if (t >= 4) row_out<M>();
    return true;
  }

  __device__ __forceinline__ bool run() {
    const int n = U.n_in;
    int t = 0;
    while (true) {
      if (!step<0>(t)) return false;
      if (++t >= n) break;
      if (!step<1>(t)) return false;
      if (++t >= n) break;
      if (!step<2>(t)) return false;
      if (++t >= n) break;
    }
    if (rr != 0) {  // the unit's last box had rows to spare
      rr = 0;
      release_box();
    }
    return true;
  }
};

template <int RND, int ODT, bool SPEC>
__global__ void __launch_bounds__(256, 2) k_harris_rows(const __grid_constant__ RowsParams kp) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const StripGeom g = strip_geom(kp.a.in.dtype == HP_F32 ? 4 : 2);
  const int gw = blockIdx.x * nw + warp, stride = gridDim.x * nw;
  if (gw >= kp.units) return;
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
  R.IU = unit_geom(kp, g, gw);
  for (int i = 0; i < kRing; ++i) issue_one(kp, g, R, stride, lane);
  for (int u = gw; u < kp.units; u += stride) {
    StripRun<RND, ODT, SPEC> run(kp, g, R, unit_geom(kp, g, u), lane, stride);
    if (!run.run()) {
      // a box never arrived: report, wait (bounded) for the copies still in
      // flight into this warp's slots, and stop
      if (lane == 0) {
        atomicExch(kp.a.err, 1);
        for (unsigned b = R.released; b < R.issued; ++b)
          mbar_wait_poll(R.bars + b % kRing, (b / kRing) & 1u, 100000000ull);
      }
      __syncwarp();
      return;
    }
  }
}

typedef void (*RowsKernel)(RowsParams);

// True when the stencil weights are the Sobel and box constants and the gray
// scale is 1 (the pipeline built by the Harris app), so the specialised
// instantiation applies.
bool sobel_box_weights(const HarrisArgs& a) {
  const float d[3] = {-1.0f, 0.0f, 1.0f}, m[3] = {1.0f, 2.0f, 1.0f}, b[3] = {1.0f, 1.0f, 1.0f};
  bool ok = a.gray_scale == 1.0f;
  for (int k = 0; k < 3; ++k) {
    ok &= a.w[0][k] == d[k] && a.w[0][3 + k] == m[k] && a.w[1][k] == m[k] && a.w[1][3 + k] == d[k];
    for (int q = 2; q < 5; ++q) ok &= a.w[q][k] == b[k] && a.w[q][3 + k] == b[k];
  }
  return ok;
}

RowsKernel pick_kernel(const HarrisArgs& a, int* variant) {
  bool inner_f32 = true;
  for (int i = 0; i < 9; ++i) inner_f32 &= a.st[i] == HP_F32;
  const bool spec = sobel_box_weights(a);
  if (inner_f32 && a.out.dtype == HP_F32) {
    *variant = spec ? 0 : 1;
    return spec ? k_harris_rows<0, 0, true> : k_harris_rows<0, 0, false>;
  }
  if (inner_f32 && a.out.dtype == HP_BF16) {
    *variant = spec ? 2 : 3;
    return spec ? k_harris_rows<0, 2, true> : k_harris_rows<0, 2, false>;
  }
  bool inner_bf16 = true;
  for (int i = 0; i < 9; ++i) inner_bf16 &= a.st[i] == HP_BF16;
  if (inner_bf16 && a.out.dtype == HP_BF16) {  // the bf16-storage pipeline
    *variant = spec ? 5 : 6;
    return spec ? k_harris_rows<2, 2, true> : k_harris_rows<2, 2, false>;
  }
  *variant = 4;
  return k_harris_rows<3, 3, false>;
}

}  // namespace

int harris_rows_strip_w(int in_dtype) { return strip_geom(in_dtype == HP_F32 ? 4 : 2).strip_w; }

int harris_rows_smem_bytes(int threads, int in_dtype) {
  const StripGeom g = strip_geom(in_dtype == HP_F32 ? 4 : 2);
  return 128 + kBarBytes + (threads / 32) * kRing * g.slot_bytes;
}

// Persistent grid: enough CTAs to fill every SM at the kernel's occupancy, or
// fewer when there are fewer units.
int harris_rows_grid(const HarrisArgs& a, int units, int threads, int smem_bytes) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0, variant = 0;
  RowsKernel kern = pick_kernel(a, &variant);
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      allow_max_dynamic_smem((const void*)kern) != 0 ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem_bytes) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return need < 2 * 152 ? need : 2 * 152;  // no device to ask: two CTAs on each of 152 SMs
  }
  return need < sms * per_sm ? need : sms * per_sm;
}

int launch_harris_rows(const HarrisArgs& a, int rows, int grid, int smem_bytes, void* stream) {
  int variant;
  RowsKernel kern = pick_kernel(a, &variant);
  static bool configured[7] = {};
  if (!configured[variant]) {
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[variant] = true;
  }
  RowsParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  const int dt = a.in.dtype;
  const int esize = dt == HP_F32 ? 4 : 2;
  const StripGeom g = strip_geom(esize);
  kp.strips = (a.out.w + g.strip_w - 1) / g.strip_w;
  kp.rows = rows;
  kp.units = kp.strips * ((a.out.h + rows - 1) / rows) * (a.batch > 1 ? a.batch : 1);
  CUtensorMapDataType tdt = dt == HP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                            : dt == HP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps, 128, kBoxRows, 3))
    return (int)cudaErrorInvalidValue;
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(a.threads), smem_bytes, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
