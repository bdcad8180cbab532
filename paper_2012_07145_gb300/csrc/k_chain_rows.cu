// Streaming stencil chain: D successive 5x5 stencils (D = 2 or 4) fused in
// registers, per channel plane -- the long-range fusion of the stencil chain
// (Sec. 2, Fig. 1) with every intermediate kept in registers (Sec. 4.7).
//
// Each warp owns a strip of columns, C consecutive ones per lane (C = 4 or 8),
// and walks down a run of rows.  Input rows arrive as TMA boxes (32 C columns
// x 4 rows) through a ring of shared-memory slots private to the warp.  Every
// step reads one input row and pushes it through all D stages: a stage's x
// pass takes its two neighbours on each side from the adjacent lanes (warp
// shuffles), its y pass runs over a 5-row register window of its x-pass
// results, and its output row feeds the next stage's x pass at once.  Stage s
// lags the input by 2(s+1) rows.  Each stage loses two columns of validity on
// each side, so whole lanes of halo (2D columns at least) surround the strip.
// No barrier wider than the warp is taken and no intermediate touches shared
// or global memory; a run's only shared-memory traffic is one load per input
// row and lane.
//
// A run of R output rows starting at row oy reads input rows from
// y0 = max(oy - 2D, 0) and takes R + 4D steps (R + 2D + oy at the image top).
// In a run that starts inside the image, the first steps of the later stages
// run on rows that are not valid yet; their results fall out of the windows
// before any valid output reads them, so every stage runs at every step and
// the steady loop has no per-stage test.  Boundary conditions, per stage on
// its own producer (clamp to edge): at the image top, a stage's first input
// row (row 0) also fills the two window rows above it; below the image, a
// stage's window repeats its row H - 1 instead of an x pass; in strips that
// touch the left or right image edge, each stage's input row takes the edge
// column's value outside the image (shuffled from the lane that holds it).
//
// Stage expressions and per-stage rounding are those of stage_math.cuh, so the
// result is bit-identical to every other schedule.
#include <cuda.h>
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

// Box heights stay a power of two: boxes of 3 or 5 rows measured several
// times slower to arrive than boxes of 2 or 4.
constexpr int kBoxRows = 4;      // rows per TMA box
constexpr int kRing = 3;         // boxes per warp ring
constexpr int kMaxWarps = 8;     // warps per block (256 threads)
constexpr int kBarBytes = 256;   // mbarriers of up to kMaxWarps x kRing
constexpr unsigned kFull = 0xffffffffu;

struct StripGeom {
  int cols;        // columns per lane (4 or 8)
  int halo_lanes;  // lanes on each side that only feed neighbours
  int strip_w;     // output columns per strip: cols (32 - 2 halo_lanes)
  int box_w;       // columns per TMA box row: 32 cols
  int slot_bytes;  // one ring slot: box_w columns x kBoxRows rows
};

// 2D columns of halo on each side, in whole lanes; a TMA box must also start
// on a 16-byte boundary (8 columns of a 2-byte input).
__host__ __device__ inline StripGeom strip_geom(int depth, int cols, int esize) {
  StripGeom g;
  g.cols = cols;
  int hl = (2 * depth + cols - 1) / cols;
  if (esize == 2 && (cols * hl) % 8) hl += 1;
  g.halo_lanes = hl;
  g.strip_w = cols * (32 - 2 * hl);
  g.box_w = 32 * cols;
  g.slot_bytes = g.box_w * kBoxRows * esize;
  return g;
}

struct CRowsParams {
  CUtensorMap tmap;
  ChainArgs a;
  int strips, runs, units, rows;  // per plane: strips x runs units of `rows` output rows
};

struct Unit {
  int x0, oy, ye, y0, plane, n_steps, n_in, nbox;  // x0: image column of lane 0's first column
};

__device__ __forceinline__ Unit unit_geom(const CRowsParams& kp, const StripGeom& g, int u, int depth) {
  Unit U;
  const int per_plane = kp.strips * kp.runs;
  U.plane = u / per_plane;
  const int v = u - U.plane * per_plane;
  const int run = v / kp.strips, s = v - run * kp.strips;
  const int H = kp.a.in.h;
  U.x0 = s * g.strip_w - g.cols * g.halo_lanes;
  U.oy = run * kp.rows;
  U.ye = min(U.oy + kp.rows, kp.a.out.h);
  U.y0 = max(U.oy - 2 * depth, 0);
  U.n_steps = U.ye - U.y0 + 2 * depth;
  U.n_in = min(U.y0 + U.n_steps, H) - U.y0;  // input rows inside the image
  U.nbox = (U.n_in + kBoxRows - 1) / kBoxRows;
  return U;
}

// Per-unit description of the image's left and right edges inside a strip:
// a stage's input row takes, at columns outside [0, W), the value of the
// nearest column inside (clamp to edge), fetched from the lane that holds it
// with one shuffle per edge.
struct EdgeFix {
  int lmask, rmask;  // per lane: bit k set if column c0 + k lies left of 0 / right of W - 1
  int l_lane;        // lane holding column 0 (at its element 0)
  int r_lane, r_k;   // lane and element holding column W - 1
};

__device__ __forceinline__ EdgeFix edge_fix_of(int c0, int x0, int W, int C) {
  EdgeFix f;
  f.lmask = f.rmask = 0;
  for (int k = 0; k < C; ++k) {
    if (c0 + k < 0) f.lmask |= 1 << k;
    if (c0 + k > W - 1) f.rmask |= 1 << k;
  }
  f.l_lane = (0 - x0) / C;
  f.r_lane = (W - 1 - x0) / C;
  f.r_k = (W - 1 - x0) - f.r_lane * C;
  return f;
}

// A select the compiler keeps as a select (a chain of compare-and-select over
// an array's elements would otherwise become an indexed load from local memory).
__device__ __forceinline__ float sel(bool p, float a, float b) {
  float r;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %3, 0;\n\tselp.f32 %0, %1, %2, q;\n\t}" : "=f"(r) : "f"(a), "f"(b), "r"((int)p));
  return r;
}

template <int C>
__device__ __forceinline__ void clamp_cols(float (&v)[C], const EdgeFix& f, bool left, bool right) {
  if (left) {
    const float e = __shfl_sync(kFull, v[0], f.l_lane);
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = (f.lmask >> k) & 1 ? e : v[k];
  }
  if (right) {
    float mine = v[0];
#pragma unroll
    for (int k = 1; k < C; ++k) mine = sel(f.r_k == k, v[k], mine);
    const float e = __shfl_sync(kFull, mine, f.r_lane);
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = (f.rmask >> k) & 1 ? e : v[k];
  }
}

template <int C>
__device__ __forceinline__ void load_row(const unsigned char* p, int dtype, float (&v)[C]) {
  if (dtype == HP_F32) {
#pragma unroll
    for (int q = 0; q < C / 4; ++q) {
      const float4 f = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < C / 4; ++q) {
      const uint2 u2 = reinterpret_cast<const uint2*>(p)[q];
      const unsigned u[2] = {u2.x, u2.y};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const unsigned short lo = (unsigned short)(u[i] & 0xffffu), hi = (unsigned short)(u[i] >> 16);
        if (dtype == HP_BF16) {
          v[4 * q + 2 * i] = __bfloat162float(__ushort_as_bfloat16(lo));
          v[4 * q + 2 * i + 1] = __bfloat162float(__ushort_as_bfloat16(hi));
        } else {
          v[4 * q + 2 * i] = __half2float(__ushort_as_half(lo));
          v[4 * q + 2 * i + 1] = __half2float(__ushort_as_half(hi));
        }
      }
    }
  }
}

// Issues box j of unit U (input rows y0 + 4j ..) into ring slot q % kRing.
// Called by one lane; the fence orders the warp's earlier reads of the slot
// (generic proxy) before the copy that overwrites it (async proxy).
__device__ __forceinline__ void issue_box(const CUtensorMap* tmap, unsigned char* slots, uint64_t* bars,
                                          int slot_bytes, unsigned q, const Unit& U, int j) {
  const int s = q % kRing;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bars + s, (unsigned)slot_bytes);
  tma_load_3d(slots + s * slot_bytes, tmap, U.x0, U.y0 + j * kBoxRows, U.plane, bars + s);
}

// Weight classes a stage's taps can be specialised for: the kernel is then
// compiled with the taps as constants (the same float values the pipeline
// stores, so the arithmetic is unchanged), which frees the registers and the
// loads the runtime taps would take.  Class 1: binomial [1,4,6,4,1]/16 on both
// axes; class 2: box 1/5 on both axes; 0: the taps passed at run time.
// A pattern WP holds the class of stage s in bits 2s..2s+1 (WP = 0: all
// runtime).
constexpr int kClassBinomial = 1, kClassBox = 2;

__host__ __device__ constexpr float class_tap(int cls, int k) {
  return cls == kClassBox ? 0.2f : (k == 0 || k == 4) ? 0.0625f : k == 2 ? 0.375f : 0.25f;
}

// One run of rows of one strip of one plane.  Step t reads input row y0 + t;
// stage s's input row at that step is i = y0 + t - 2s, and its y pass
// completes its output row i - 2; the last stage's output row is y0 + t - 2D.
//
// The y pass keeps, per stage and column, four partial sums instead of a
// window of x-pass rows: when the x-pass row h of input row i arrives, the
// partial sum of output row i - 2 takes its last tap and leaves, those of rows
// i - 1, i and i + 1 take one tap each, and row i + 2's starts.  The taps of
// every output row are still applied oldest row first, as tap5 applies them,
// so the sums are bit-identical to the window form, and each update writes the
// next slot's register: the loop body is a single step, with no rotation of
// registers and no unrolling (the kernel's code stays small enough for the
// instruction cache).  All state is in registers: the partial sums, the
// newest x-pass row of every stage and the runtime taps (loaded once).
// RND: 0 every storage type f32 (no rounding), 1 all f16, 2 all bf16, 3 per
// stage at run time.  ODT: output stores 0 f32, 1 f16, 2 bf16, 3 any type.
template <int D, int C, int RND, int ODT, int WP>
struct RunState {
  static constexpr int kD = D, kC = C, kODT = ODT;
  float w[D][10];            // per stage: x taps, then y taps (runtime class)
  int st[D];                 // per stage: storage type (RND = 3)
  float acc[D][4][C];        // per stage: partial sums of its output rows i - 1 .. i + 2
  float h[D][C];             // per stage: its newest x-pass row (below the image it stays row H - 1)
  int y0, H;
  bool top;                  // the run starts at image row 0
  EdgeFix ef;
  bool hl, hr, he;           // the strip reaches past the left / right / either image edge

  template <int S>
  __device__ __forceinline__ float tap(int k) const {
    constexpr int cls = (WP >> (2 * S)) & 3;
    if constexpr (cls != 0) return class_tap(cls, k % 5);
    else return w[S][k];
  }

  template <int S>
  __device__ __forceinline__ float rnd(float b) const {
    if (RND == 1) return __half2float(__float2half_rn(b));
    if (RND == 2) return __bfloat162float(__float2bfloat16_rn(b));
    if (RND == 3) return round_storage(st[S], b);
    return b;
  }

  // x pass of stage S over its input row v (columns c0-2 .. c0+C+1: two
  // neighbours on each side from the adjacent lanes) into h[S].  In a strip
  // that reaches past an image edge the row first takes the edge values.
  template <int S, bool HE>
  __device__ __forceinline__ void xpass(float (&v)[C]) {
    if (HE) clamp_cols<C>(v, ef, hl, hr);
    const float l2 = __shfl_up_sync(kFull, v[C - 2], 1), l1 = __shfl_up_sync(kFull, v[C - 1], 1);
    const float r1 = __shfl_down_sync(kFull, v[0], 1), r2 = __shfl_down_sync(kFull, v[1], 1);
    float e[C + 4];
    e[0] = l2; e[1] = l1;
#pragma unroll
    for (int k = 0; k < C; ++k) e[k + 2] = v[k];
    e[C + 2] = r1; e[C + 3] = r2;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      float sum = __fmul_rn(tap<S>(0), e[k]);
      sum = __fmaf_rn(tap<S>(1), e[k + 1], sum);
      sum = __fmaf_rn(tap<S>(2), e[k + 2], sum);
      sum = __fmaf_rn(tap<S>(3), e[k + 3], sum);
      h[S][k] = __fmaf_rn(tap<S>(4), e[k + 4], sum);
    }
  }

  // y pass of stage S with h[S] as its newest row, at phase P (the step
  // number minus 2S, mod 4): the partial sums advance one row and o receives
  // the completed output row (rounded to the stage's storage type).  Partial
  // sum j (output row i - 1 + j after the update) lives in slot (j + P) & 3, so
  // every update reads and writes one slot: no register moves.
  template <int S, int P>
  __device__ __forceinline__ void ypass(float (&o)[C]) {
    constexpr int q0 = (P + 3) & 3, q1 = P & 3, q2 = (P + 1) & 3, q3 = (P + 2) & 3;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const float x = h[S][k];
      const float b = __fmaf_rn(tap<S>(9), x, acc[S][q0][k]);
      acc[S][q1][k] = __fmaf_rn(tap<S>(8), x, acc[S][q1][k]);
      acc[S][q2][k] = __fmaf_rn(tap<S>(7), x, acc[S][q2][k]);
      acc[S][q3][k] = __fmaf_rn(tap<S>(6), x, acc[S][q3][k]);
      acc[S][q0][k] = __fmul_rn(tap<S>(5), x);
      o[k] = rnd<S>(b);
    }
  }

  float o[C];                // the last stage's row of the latest step

  // Step t (t mod 4 = U): the input row (from the box's slot while it lies
  // inside the image) through all D stages into o.
  template <int U, bool EDGE, bool HE>
  __device__ __forceinline__ void step(int t, const unsigned char* slot, int dtype, int esize, int box_w) {
    float v[C];
    if (!EDGE || y0 + t < H) {
      load_row<C>(slot + U * box_w * esize, dtype, v);
    } else {
#pragma unroll
      for (int k = 0; k < C; ++k) v[k] = 0.0f;
    }
    stages<0, U, EDGE, HE>(t, v, o);
  }

  // Stages S.. at step t, whose number mod 4 is U; v is stage S's input row.
  // EDGE: the step may need the top or bottom boundary handling.  Returns the
  // last stage's row in o.
  template <int S, int U, bool EDGE, bool HE>
  __device__ __forceinline__ void stages(int t, float (&v)[C], float (&o)[C]) {
    constexpr int P = ((U - 2 * S) % 4 + 4) % 4;
    if (EDGE) {
      const int i = y0 + t - 2 * S;
      if (i < H) {  // else below the image: h[S] still holds row H - 1, the clamped row
        xpass<S, HE>(v);
        if (top && i == 0) {  // rows -2 and -1 of this stage's producer are its row 0
          ypass<S, (P + 2) & 3>(o);
          ypass<S, (P + 3) & 3>(o);
        }
      }
    } else {
      xpass<S, HE>(v);
    }
    if constexpr (S + 1 < D) {
      float m[C];
      ypass<S, P>(m);
      stages<S + 1, U, EDGE, HE>(t, m, o);
    } else {
      ypass<S, P>(o);
    }
  }
};

// Stores a lane's output columns.  full: all C columns lie inside the image
// (one vector store); part: some do (one store per column inside).
template <int C, int ODT>
__device__ __forceinline__ void store_row(char* row, int c0, bool full, bool part, const ImgView& out, int plane,
                                          int y, const float (&o)[C]) {
  if (ODT == 3) {
    if (full || part) {
#pragma unroll
      for (int k = 0; k < C; ++k)
        if (c0 + k < out.w) store_px(out, plane, c0 + k, y, o[k]);
    }
    return;
  }
  if (ODT == 0) {
    float* p = reinterpret_cast<float*>(row) + c0;
    if (full) {
#pragma unroll
      for (int q4 = 0; q4 < C / 4; ++q4)
        reinterpret_cast<float4*>(p)[q4] = make_float4(o[4 * q4], o[4 * q4 + 1], o[4 * q4 + 2], o[4 * q4 + 3]);
    } else if (part) {
#pragma unroll
      for (int k = 0; k < C; ++k)
        if (c0 + k < out.w) p[k] = o[k];
    }
    return;
  }
  unsigned short hv[C];
#pragma unroll
  for (int k = 0; k < C; ++k)
    hv[k] = ODT == 1 ? __half_as_ushort(__float2half_rn(o[k])) : __bfloat16_as_ushort(__float2bfloat16_rn(o[k]));
  unsigned short* p = reinterpret_cast<unsigned short*>(row) + c0;
  if (full) {
#pragma unroll
    for (int q4 = 0; q4 < C / 4; ++q4)
      reinterpret_cast<uint2*>(p)[q4] = make_uint2(hv[4 * q4] | (unsigned)hv[4 * q4 + 1] << 16,
                                                  hv[4 * q4 + 2] | (unsigned)hv[4 * q4 + 3] << 16);
  } else if (part) {
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (c0 + k < out.w) p[k] = hv[k];
  }
}

// The store of step t's output row, once the chain's output is the run's.
// Lanes with only some columns inside the image exist in strips past the
// right image edge (HE) alone.
template <int C, int ODT, bool HE>
__device__ __forceinline__ void store_if(int t, int t_store, char*& out_row, int c0, bool full, bool part,
                                         const ImgView& out, const Unit& U, int D, const float (&o)[C]) {
  if (t >= t_store) {
    store_row<C, ODT>(out_row, c0, full, HE && part, out, U.plane, U.y0 + t - 2 * D, o);
    out_row += out.rs;
  }
}

// The four steps of one box (steps t0 .. t0 + 3, those below n).  EDGE: some
// step needs the top or bottom boundary handling; HE: the strip reaches past
// an image edge.
template <bool EDGE, bool HE, class RS>
__device__ __forceinline__ void box_steps(RS& S, int t0, int n, const unsigned char* slot, const CRowsParams& kp,
                                          int esize, int box_w, int t_store, char*& out_row, int c0, bool full,
                                          bool part, const Unit& U) {
  constexpr int C = RS::kC, ODT = RS::kODT, D = RS::kD;
  S.template step<0, EDGE, HE>(t0, slot, kp.a.in.dtype, esize, box_w);
  store_if<C, ODT, HE>(t0, t_store, out_row, c0, full, part, kp.a.out, U, D, S.o);
  if (EDGE && t0 + 1 >= n) return;
  S.template step<1, EDGE, HE>(t0 + 1, slot, kp.a.in.dtype, esize, box_w);
  store_if<C, ODT, HE>(t0 + 1, t_store, out_row, c0, full, part, kp.a.out, U, D, S.o);
  if (EDGE && t0 + 2 >= n) return;
  S.template step<2, EDGE, HE>(t0 + 2, slot, kp.a.in.dtype, esize, box_w);
  store_if<C, ODT, HE>(t0 + 2, t_store, out_row, c0, full, part, kp.a.out, U, D, S.o);
  if (EDGE && t0 + 3 >= n) return;
  S.template step<3, EDGE, HE>(t0 + 3, slot, kp.a.in.dtype, esize, box_w);
  store_if<C, ODT, HE>(t0 + 3, t_store, out_row, c0, full, part, kp.a.out, U, D, S.o);
}

template <int D, int C, int RND, int ODT, int WP>
__global__ void __maxnreg__(200) k_chain_rows(const __grid_constant__ CRowsParams kp) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int esize = kp.a.in.dtype == HP_F32 ? 4 : 2;
  const StripGeom g = strip_geom(D, C, esize);
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
  RunState<D, C, RND, ODT, WP> S;
#pragma unroll
  for (int s = 0; s < D; ++s) {
#pragma unroll
    for (int k = 0; k < 10; ++k) S.w[s][k] = kp.a.w[s][k];
    S.st[s] = kp.a.storage[s];
  }
  const int W = kp.a.in.w, H = kp.a.in.h, OW = kp.a.out.w;
  S.H = H;
  unsigned qbase = 0;  // boxes this warp has issued before the current unit
  for (int u = gw; u < kp.units; u += stride) {
    const Unit U = unit_geom(kp, g, u, D);
    if (lane == 0)
      for (int j = 0; j < kRing && j < U.nbox; ++j) issue_box(&kp.tmap, slots, bars, g.slot_bytes, qbase + j, U, j);
    const int c0 = U.x0 + C * lane;
    S.y0 = U.y0;
    S.top = U.y0 == 0;
    S.hl = U.x0 < 0;
    S.hr = U.x0 + 32 * C > W;
    S.ef = edge_fix_of(c0, U.x0, W, C);
    S.he = S.hl || S.hr;
#pragma unroll
    for (int s = 0; s < D; ++s)
#pragma unroll
      for (int k = 0; k < C; ++k) {
        S.h[s][k] = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) S.acc[s][j][k] = 0.0f;
      }
    const bool mine = lane >= g.halo_lanes && lane < 32 - g.halo_lanes;
    const bool st_full = mine && c0 + C - 1 < OW;
    const bool st_part = mine && c0 < OW && !st_full;
    char* out_row = (char*)kp.a.out.data + (long long)U.plane * kp.a.out.ps + (long long)U.oy * kp.a.out.rs;
    const int n = U.n_steps;
    const int t_store = U.oy - U.y0 + 2 * D;       // first step whose output row is the run's
    const int t_edge = H - 1 - U.y0;               // from this step on some stage's input row is H - 1 or below
    const int edge_lo = S.top ? 2 * (D - 1) : -1;  // steps 0 .. edge_lo: some stage's input row is row 0
    int failed = 0;
    // One box (4 input rows) per iteration, its four steps unrolled so that
    // each stage's partial sums keep fixed registers.  Boxes whose steps are
    // all away from the image's top and bottom rows take the plain steps.
#pragma unroll 1
    for (int j = 0; 4 * j < n; ++j) {
      const int t0 = 4 * j;
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
        slot = slots + (q % kRing) * g.slot_bytes + lane * C * esize;
      }
      if (t0 > edge_lo && t0 + 3 < t_edge && t0 + 3 < n) {
        if (S.he) box_steps<false, true>(S, t0, n, slot, kp, esize, g.box_w, t_store, out_row, c0, st_full, st_part, U);
        else box_steps<false, false>(S, t0, n, slot, kp, esize, g.box_w, t_store, out_row, c0, st_full, st_part, U);
      } else {
        if (S.he) box_steps<true, true>(S, t0, n, slot, kp, esize, g.box_w, t_store, out_row, c0, st_full, st_part, U);
        else box_steps<true, false>(S, t0, n, slot, kp, esize, g.box_w, t_store, out_row, c0, st_full, st_part, U);
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

typedef void (*CRowsKernel)(CRowsParams);

// The class of a stage's taps (kClassBinomial / kClassBox when all ten taps
// equal that class's values bit for bit, else 0).
int stage_class(const float (&w)[10]) {
  for (int cls : {kClassBinomial, kClassBox}) {
    bool eq = true;
    for (int k = 0; k < 10; ++k) {
      const float t = class_tap(cls, k % 5);
      eq &= memcmp(&w[k], &t, sizeof t) == 0;
    }
    if (eq) return cls;
  }
  return 0;
}

// Specialised tap patterns: alternating binomial/box from either class, and
// all binomial; any other pattern takes the runtime taps.
template <int D>
constexpr int pattern_of(int c0, int c1) {
  int p = 0;
  for (int s = 0; s < D; ++s) p |= ((s & 1) ? c1 : c0) << (2 * s);
  return p;
}

template <int D, int C, int RND, int ODT>
CRowsKernel pick_wp(const ChainArgs& a, int* variant) {
  int p = 0;
  for (int s = 0; s < D; ++s) p |= stage_class(a.w[s]) << (2 * s);
  constexpr int BX = pattern_of<D>(kClassBinomial, kClassBox), XB = pattern_of<D>(kClassBox, kClassBinomial);
  constexpr int BB = pattern_of<D>(kClassBinomial, kClassBinomial);
  if (RND != 3) {
    if (p == BX) { *variant = 1; return k_chain_rows<D, C, RND, ODT, BX>; }
    if (p == XB) { *variant = 2; return k_chain_rows<D, C, RND, ODT, XB>; }
    if (p == BB) { *variant = 3; return k_chain_rows<D, C, RND, ODT, BB>; }
  }
  *variant = 0;
  return k_chain_rows<D, C, RND, ODT, 0>;
}

// Rounding and store type: one type for every stage and the output, or the
// general (runtime) form.
template <int D, int C>
CRowsKernel pick_dc(const ChainArgs& a, int* variant) {
  const int s0 = a.storage[0];
  bool uniform = true;
  for (int s = 1; s < D; ++s) uniform &= a.storage[s] == s0;
  uniform &= a.out.dtype == s0;
  int v = 0;
  CRowsKernel k;
  if (uniform && s0 == HP_F32) k = pick_wp<D, C, 0, 0>(a, &v), v += 0;
  else if (uniform && s0 == HP_F16) k = pick_wp<D, C, 1, 1>(a, &v), v += 4;
  else if (uniform && s0 == HP_BF16) k = pick_wp<D, C, 2, 2>(a, &v), v += 8;
  else k = pick_wp<D, C, 3, 3>(a, &v), v += 12;
  *variant = v;
  return k;
}

// Instantiations: 4 columns per lane at depth 2 and 4, 8 columns at depth 2
// (at depth 4 the partial sums of 8 columns would not fit in registers).
CRowsKernel pick_kernel(const ChainArgs& a, int cols, int* variant) {
  int base = 0;
  CRowsKernel k;
  if (a.depth == 2 && cols == 8) k = pick_dc<2, 8>(a, variant), base = 32;
  else if (a.depth == 2) k = pick_dc<2, 4>(a, variant), base = 0;
  else k = pick_dc<4, 4>(a, variant), base = 16;
  *variant += base;
  return k;
}

int esize_of(int dtype) { return dtype == HP_F32 ? 4 : 2; }

}  // namespace

bool chain_rows_depth_ok(int depth) { return depth == 2 || depth == 4; }

// Strip width with `cols` columns per lane (4, the default, or 8) for this
// depth and input type.
int chain_rows_strip_w(int depth, int in_dtype, int cols) { return strip_geom(depth, cols, esize_of(in_dtype)).strip_w; }

// Columns per lane a schedule's tile width selects (4 or 8), or 0 if the width
// is not a strip width of this depth and input type.
int chain_rows_cols(int depth, int in_dtype, int tile_w) {
  for (int c : {4, 8})
    if ((c == 4 || depth == 2) && strip_geom(depth, c, esize_of(in_dtype)).strip_w == tile_w) return c;
  return 0;
}

int chain_rows_smem_bytes(int depth, int cols, int threads, int in_dtype) {
  const StripGeom g = strip_geom(depth, cols, esize_of(in_dtype));
  return 128 + kBarBytes + (threads / 32) * kRing * g.slot_bytes;
}

// Persistent grid: enough CTAs to fill every SM at the kernel's occupancy, or
// fewer when there are fewer units.
int chain_rows_grid(const ChainArgs& a, int cols, int units, int threads, int smem_bytes) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0, variant = 0;
  CRowsKernel kern = pick_kernel(a, cols, &variant);
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      allow_max_dynamic_smem((const void*)kern) != 0 ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem_bytes) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return need < 2 * 152 ? need : 2 * 152;  // no device to ask: two CTAs on each of 152 SMs
  }
  return need < sms * per_sm ? need : sms * per_sm;
}

int launch_chain_rows(const ChainArgs& a, int cols, int rows, int grid, int smem_bytes, void* stream) {
  int variant;
  CRowsKernel kern = pick_kernel(a, cols, &variant);
  static bool configured[48] = {};
  if (!configured[variant]) {
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[variant] = true;
  }
  if (a.threads / 32 > kMaxWarps) return (int)cudaErrorInvalidValue;
  CRowsParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  const int dt = a.in.dtype;
  const int esize = esize_of(dt);
  const StripGeom g = strip_geom(a.depth, cols, esize);
  kp.strips = (a.out.w + g.strip_w - 1) / g.strip_w;
  kp.runs = (a.out.h + rows - 1) / rows;
  kp.rows = rows;
  kp.units = kp.strips * kp.runs * a.out.c;
  CUtensorMapDataType tdt = dt == HP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                            : dt == HP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps, g.box_w, kBoxRows, 1))
    return (int)cudaErrorInvalidValue;
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(a.threads), smem_bytes, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
