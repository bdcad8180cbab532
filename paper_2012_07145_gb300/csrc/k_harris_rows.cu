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
  int strips, units, rows;  // strips across the image; units = strips x row runs x images; rows per run
};

// A run of output rows oy .. ye-1 of one strip of one image.  Input rows are
// read from y0 = max(oy - 2, 0): n_steps steps in all, of which the first n_in
// read a row inside the image.
struct Unit {
  int x0, oy, ye, y0, n_steps, n_in, nbox;  // x0: image column of lane 0's first column
  int img;                                  // image of a batch (input planes 3 img .. 3 img + 2, output plane img)
};

__device__ __forceinline__ Unit unit_geom(const RowsParams& kp, const StripGeom& g, int u) {
  Unit U;
  const int per_img = kp.units / (kp.a.batch > 1 ? kp.a.batch : 1);
  U.img = u / per_img;
  u -= U.img * per_img;
  const int s = u % kp.strips, r = u / kp.strips;
  const int H = kp.a.in.h;
  U.x0 = s * g.strip_w - 4 * g.halo_lanes;
  U.oy = r * kp.rows;
  U.ye = min(U.oy + kp.rows, kp.a.out.h);
  U.y0 = max(U.oy - 2, 0);
  U.n_steps = U.ye - U.y0 + 2;
  U.n_in = min(U.y0 + U.n_steps, H) - U.y0;
  U.nbox = (U.n_in + kBoxRows - 1) / kBoxRows;
  return U;
}

// Issues box j of unit U (input rows y0 + 2j, y0 + 2j + 1 of its image's three
// planes) into ring slot q % kRing.  Called by one lane; the fence orders the
// warp's earlier reads of the slot before the copy that overwrites it.
__device__ __forceinline__ void issue_box(const CUtensorMap* tmap, unsigned char* slots, uint64_t* bars,
                                          int slot_bytes, unsigned q, const Unit& U, int j) {
  const int s = q % kRing;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bars + s, (unsigned)slot_bytes);
  tma_load_3d(slots + s * slot_bytes, tmap, U.x0, U.y0 + j * kBoxRows, 3 * U.img, bars + s);
}

// Left and right neighbours of the lane's four columns for a 3-tap x pass.  In
// a strip past an image edge (HE), the neighbour outside the image is the edge
// column itself (column 0 always sits first in a lane: strips start on
// multiples of 4; column W - 1 may sit anywhere).
struct Edges {
  bool left;      // the lane's first column is column 0
  bool right[4];  // column k of the lane is column W - 1
};

template <bool HE>
__device__ __forceinline__ void neighbours(const float (&v)[4], const Edges& e, float (&l)[4], float (&r)[4]) {
  const float up = __shfl_up_sync(kFull, v[3], 1), dn = __shfl_down_sync(kFull, v[0], 1);
  l[0] = HE && e.left ? v[0] : up;
  l[1] = v[0];
  l[2] = v[1];
  l[3] = v[2];
  r[0] = HE && e.right[0] ? v[0] : v[1];
  r[1] = HE && e.right[1] ? v[1] : v[2];
  r[2] = HE && e.right[2] ? v[2] : v[3];
  r[3] = HE && e.right[3] ? v[3] : dn;
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

// One run of rows of one strip.  Step t reads input row r = y0 + t: gray row
// r and its two x passes; the Sobel y passes complete gradient row r - 1, whose
// products and box-sum x passes follow; the box y passes complete output row
// r - 2.  Every 3-tap y pass keeps two partial sums per column instead of a
// window of rows: when row i's x pass x arrives, output row i - 1 takes its
// last tap, row i its middle one, and row i + 1 starts -- the taps of each row
// still applied oldest first, as tap3v applies them, so every value is the
// same.  The two partial sums swap slots every step (see ystep), so a box of
// two steps keeps fixed registers.  The stage values that a clamp may repeat below
// the image (the newest x passes) are kept.
template <int RND, int ODT, bool SPEC>
struct HarrisRun {
  static constexpr int kODT = ODT;
  const HarrisArgs& a;
  const Weights<SPEC> w;
  float pA[2][4], pB[2][4];     // Sobel y partial sums (Ix, Iy)
  float pS[3][2][4];            // box-sum y partial sums (xx, yy, xy)
  float hA[4], hB[4];           // newest x passes of gray (Ix and Iy x-weights)
  float hS[3][4];               // newest x passes of the products
  Edges e;
  int y0, H;
  bool top;
  float o[4];                   // the response row of the latest step

  __device__ __forceinline__ HarrisRun(const HarrisArgs& a_) : a(a_), w(a_.w) {}

  // A 3-tap y pass step of weight set q over slot pair P (two partial sums):
  // returns the completed row, advances the sums.
  // Slot PH & 1 holds the partial sum of the row that completes now (two
  // taps in), slot (PH + 1) & 1 that of the next row (one tap in); after the
  // update the roles of the slots swap, which the next step's phase follows.
  template <int PH>
  __device__ __forceinline__ float ystep(int q, float x, float (&p)[2][4], int k) {
    constexpr int s0 = PH & 1, s1 = (PH + 1) & 1;
    const float out = __fmaf_rn(w(q, 5), x, p[s0][k]);
    const float w3 = w(q, 3);
    p[s1][k] = __fmaf_rn(w(q, 4), x, p[s1][k]);
    if (SPEC && (w3 == 1.0f || w3 == -1.0f))
      p[s0][k] = w3 == 1.0f ? x : -x;   // w3 * x is exact for w3 = +-1: the product tap3v's first step rounds to
    else
      p[s0][k] = __fmul_rn(w3, x);
    return out;
  }

  // Gray row r (input row v of the three planes) and its two x passes.
  template <bool HE>
  __device__ __forceinline__ void gray_x(const float (&cr)[4], const float (&cg)[4], const float (&cb)[4]) {
    float gv[4];
    if (SPEC || a.gray_scale == 1.0f) {  // x * 1 is exact: the same value as op_gray with scale 1
#pragma unroll
      for (int k = 0; k < 4; ++k) gv[k] = __fmaf_rn(0.114f, cb[k], __fmaf_rn(0.587f, cg[k], __fmul_rn(0.299f, cr[k])));
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) gv[k] = op_gray(cr[k], cg[k], cb[k], a.gray_scale);
    }
    rs4<RND>(gv, a.st[0]);
    float l[4], rt[4];
    neighbours<HE>(gv, e, l, rt);
    xpass3(w, 0, l, gv, rt, hA);
    xpass3(w, 1, l, gv, rt, hB);
  }

  // The Sobel y passes with the newest gray x passes (gradient row i - 1),
  // then that row's products and their box-sum x passes into hS.  DUP: the
  // gray row also stands for the row above it (image row 0).
  template <int PH, bool HE>
  __device__ __forceinline__ void grad_prod(bool valid) {
    float ix[4], iy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ix[k] = ystep<PH>(0, hA[k], pA, k);
      iy[k] = ystep<PH>(1, hB[k], pB, k);
    }
    if (!valid) return;   // the gradient row is above the run's first: its products are not needed
    rs4<RND>(ix, a.st[1]);
    rs4<RND>(iy, a.st[2]);
    float pr[3][4];
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
      neighbours<HE>(pr[b], e, l, rt);
      xpass3(w, 2 + b, l, pr[b], rt, hS[b]);
    }
  }

  // The box-sum y passes with the newest product x passes, then the response
  // of the completed row into o.
  template <int PH>
  __device__ __forceinline__ void box_resp() {
    float sxx[4], syy[4], sxy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sxx[k] = ystep<PH>(2, hS[0][k], pS[0], k);
      syy[k] = ystep<PH>(3, hS[1][k], pS[1], k);
      sxy[k] = ystep<PH>(4, hS[2][k], pS[2], k);
    }
    rs4<RND>(sxx, a.st[6]);
    rs4<RND>(syy, a.st[7]);
    rs4<RND>(sxy, a.st[8]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float v = op_harris(sxx[k], syy[k], sxy[k], a.k);
      o[k] = ODT == 3 ? round_storage(a.out.dtype, v) : v;
    }
  }

  // Step t (t & 1 = PH) on input row (cr, cg, cb); EDGE: the image's top
  // or bottom rows are near (clamped rows), HE: the strip reaches past an
  // image edge.
  template <int PH, bool EDGE, bool HE>
  __device__ __forceinline__ void step(int t, const float (&cr)[4], const float (&cg)[4], const float (&cb)[4]) {
    if (!EDGE) {
      gray_x<HE>(cr, cg, cb);
      grad_prod<PH, HE>(true);
      box_resp<PH>();
      return;
    }
    const int r = y0 + t;                     // gray row
    if (r < H) gray_x<HE>(cr, cg, cb);        // else row H - 1's x passes stand for row r (clamped)
    if (top && r == 0) grad_prod<(PH + 1) & 1, HE>(false);   // gray row -1 is row 0
    // gradient row r - 1: its products when it lies in the image; below it
    // the product row is row H - 1's, whose x passes hS still hold
    grad_prod<PH, HE>(r - 1 >= 0 && r - 1 < H);
    if (top && r == 1) box_resp<(PH + 1) & 1>();             // product row -1 is row 0
    box_resp<PH>();
  }
};

template <int ODT>
__device__ __forceinline__ void store_out(char* row, int c0, bool full, bool part, const ImgView& out, int img, int y,
                                          const float (&o)[4]) {
  if (full) {
    if (ODT == 0) {
      *reinterpret_cast<float4*>(row + 4LL * c0) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
      __nv_bfloat162 p0 = __floats2bfloat162_rn(o[0], o[1]), p1 = __floats2bfloat162_rn(o[2], o[3]);
      uint2 u;
      u.x = *reinterpret_cast<unsigned*>(&p0);
      u.y = *reinterpret_cast<unsigned*>(&p1);
      *reinterpret_cast<uint2*>(row + 2LL * c0) = u;
    }
  } else if (part) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (c0 + k < out.w) store_px(out, img, c0 + k, y, o[k]);
  }
}

// The two steps of one box; EDGE: check each step against the run's end.
template <bool EDGE, bool HE, class Run>
__device__ __forceinline__ void box_steps(Run& R, int t0, int n, const unsigned char* slot, int dtype, int esize,
                                          int t_store, char*& out_row, int c0, bool full, bool part, const Unit& U,
                                          const ImgView& out) {
  constexpr int ODT = Run::kODT;
  const int plane = 128 * kBoxRows * esize;
#pragma unroll
  for (int u = 0; u < kBoxRows; ++u) {
    const int t = t0 + u;
    if (EDGE && t >= n) return;
    float cr[4], cg[4], cb[4];
    if (!EDGE || U.y0 + t < R.H) {
      const unsigned char* p = slot + u * 128 * esize;
      load4(p, dtype, cr);
      load4(p + plane, dtype, cg);
      load4(p + 2 * plane, dtype, cb);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) cr[k] = cg[k] = cb[k] = 0.0f;
    }
    if (u == 0) R.template step<0, EDGE, HE>(t, cr, cg, cb);
    else R.template step<1, EDGE, HE>(t, cr, cg, cb);
    if (t >= t_store) {
      // lanes with only some columns inside the image exist past the right
      // edge alone; the general output type stores column by column everywhere
      store_out<ODT>(out_row, c0, full, (HE || ODT == 3) && part, out, U.img, U.y0 + t - 2, R.o);
      out_row += out.rs;
    }
  }
}

template <int RND, int ODT, bool SPEC>
__global__ void __launch_bounds__(256) k_harris_rows(const __grid_constant__ RowsParams kp) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int esize = kp.a.in.dtype == HP_F32 ? 4 : 2;
  const StripGeom g = strip_geom(esize);
  const int gw = blockIdx.x * nw + warp, stride = gridDim.x * nw;
  if (gw >= kp.units) return;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base) + warp * kRing;
  unsigned char* slots = base + kBarBytes + warp * kRing * g.slot_bytes;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < kRing; ++i) mbar_init(bars + i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  HarrisRun<RND, ODT, SPEC> R(kp.a);
  const int W = kp.a.in.w, H = kp.a.in.h;
  R.H = H;
  unsigned qbase = 0;  // boxes this warp has issued before the current unit
  for (int u = gw; u < kp.units; u += stride) {
    const Unit U = unit_geom(kp, g, u);
    if (lane == 0)
      for (int j = 0; j < kRing && j < U.nbox; ++j) issue_box(&kp.tmap, slots, bars, g.slot_bytes, qbase + j, U, j);
    const int c0 = U.x0 + 4 * lane;
    R.y0 = U.y0;
    R.top = U.y0 == 0;
    R.e.left = c0 == 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) R.e.right[k] = c0 + k == W - 1;
    const bool he = U.x0 < 0 || U.x0 + 128 > W;
    const bool mine = lane >= g.halo_lanes && lane < 32 - g.halo_lanes;
    const bool st_full = mine && c0 + 3 < kp.a.out.w && ODT != 3;
    const bool st_part = mine && c0 < kp.a.out.w && !st_full;
    char* out_row = (char*)kp.a.out.data + (long long)U.img * kp.a.out.ps + (long long)U.oy * kp.a.out.rs;
    const int n = U.n_steps;
    const int t_store = U.oy - U.y0 + 2;          // first step whose output row is the run's
    const int t_edge = H - U.y0;                   // from this step on the gray row lies below the image
    const int t_top = R.top ? 1 : -1;              // steps 0 .. t_top: gray row 0 or 1 of a top run
    int failed = 0;
#pragma unroll 1
    for (int j = 0; kBoxRows * j < n; ++j) {
      const int t0 = kBoxRows * j;
      const unsigned char* slot = nullptr;
      if (t0 < U.n_in) {
        const unsigned q = qbase + j;
        int ok = 1;
        if (lane == 0) ok = mbar_wait_poll(bars + q % kRing, (q / kRing) & 1u, 2000000000ull);
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok) {
          failed = 1;
          break;
        }
        slot = slots + (q % kRing) * g.slot_bytes + lane * 4 * esize;
      }
      const bool edge = t0 <= t_top || t0 + kBoxRows - 1 >= t_edge || t0 + kBoxRows > n;
      if (edge) {
        if (he) box_steps<true, true>(R, t0, n, slot, kp.a.in.dtype, esize, t_store, out_row, c0, st_full, st_part, U, kp.a.out);
        else box_steps<true, false>(R, t0, n, slot, kp.a.in.dtype, esize, t_store, out_row, c0, st_full, st_part, U, kp.a.out);
      } else {
        if (he) box_steps<false, true>(R, t0, n, slot, kp.a.in.dtype, esize, t_store, out_row, c0, st_full, st_part, U, kp.a.out);
        else box_steps<false, false>(R, t0, n, slot, kp.a.in.dtype, esize, t_store, out_row, c0, st_full, st_part, U, kp.a.out);
      }
      if (j + kRing < U.nbox) {  // this box's slot is read: refill it
        __syncwarp();
        if (lane == 0) issue_box(&kp.tmap, slots, bars, g.slot_bytes, qbase + j + kRing, U, j + kRing);
      }
    }
    if (failed) {
      // a box never arrived: report, wait (bounded) for the copies still in
      // flight into this warp's slots, and stop
      if (lane == 0) {
        atomicExch(kp.a.err, 1);
        for (int j = 0; j < U.nbox; ++j) {
          const unsigned q = qbase + j;
          mbar_wait_poll(bars + q % kRing, (q / kRing) & 1u, 100000000ull);
        }
      }
      __syncwarp();
      return;
    }
    qbase += U.nbox;
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
