// Streaming stencil chain: D successive 5x5 stencils (D = 2 or 4) fused in
// registers, per channel plane.
//
// Each warp owns a strip of output columns, four per lane, and walks down a
// run of rows.  Input rows arrive as TMA boxes through a ring of shared-memory
// slots private to the warp.  Every step reads one input row and pushes it
// through all D stages: a stage's x pass takes its two neighbours on each side
// from the adjacent lanes, its y pass runs over a 5-row register window of its
// x-pass results, and its output row feeds the next stage's x pass at once.
// Stage s therefore lags the input by 2(s+1) rows; the run starts 2D rows
// above its first output row and ends 2D rows below its last.  Each stage
// loses two columns of validity on each side, so 2D columns of halo (the outer
// lanes) surround the strip.  No barrier wider than the warp is taken and no
// intermediate touches shared or global memory.
//
// Stage expressions and per-stage rounding are those of stage_math.cuh, so the
// result is bit-identical to every other schedule.  Boundary conditions, per
// stage on its own producer (clamp to edge, Sec. 3): in strips that touch the
// left or right image edge, each stage's input row takes the edge column's
// value outside the image (shuffled from the lane that holds it); rows outside
// the image take the nearest edge row's x-pass result (a copy in the window).
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
constexpr int kBarBytes = 512;   // mbarriers of up to 16 warps x kRing
constexpr unsigned kFull = 0xffffffffu;

struct StripGeom {
  int halo_lanes;  // lanes on each side that only feed neighbours
  int strip_w;     // output columns per strip: 4 (32 - 2 halo_lanes)
  int slot_bytes;  // one ring slot: 128 columns x kBoxRows rows
};

// 2D columns of halo on each side, in whole lanes; a TMA box must also start
// on a 16-byte boundary (8 columns of a 2-byte input).
__host__ __device__ inline StripGeom strip_geom(int depth, int esize) {
  StripGeom g;
  int hl = (2 * depth + 3) / 4;
  if (esize == 2 && hl < 2) hl = 2;
  g.halo_lanes = hl;
  g.strip_w = 4 * (32 - 2 * hl);
  g.slot_bytes = 128 * kBoxRows * esize;
  return g;
}

struct CRowsParams {
  CUtensorMap tmap;
  ChainArgs a;
  int strips, runs, units, rows;  // per plane: strips x runs units of `rows` output rows
};

struct Unit {
  int x0, oy, plane, n_in, nbox;  // x0: image column of lane 0's first column; n_in input rows
};

__device__ __forceinline__ Unit unit_geom(const CRowsParams& kp, const StripGeom& g, int u, int depth) {
  Unit U;
  const int per_plane = kp.strips * kp.runs;
  U.plane = u / per_plane;
  const int v = u - U.plane * per_plane;
  const int run = v / kp.strips, s = v - run * kp.strips;
  U.x0 = s * g.strip_w - 4 * g.halo_lanes;
  U.oy = run * kp.rows;
  U.n_in = min(kp.rows, kp.a.out.h - U.oy) + 4 * depth;
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

template <int D>
__device__ __forceinline__ void issue_one(const CRowsParams& kp, const StripGeom& g, Ring& R, int stride, int lane) {
  if (R.iu >= kp.units) return;
  if (lane == 0) {
    const int s = R.issued % kRing;
    mbar_arrive_expect_tx(R.bars + s, (unsigned)g.slot_bytes);
    tma_load_3d(R.slots + s * g.slot_bytes, &kp.tmap, R.IU.x0, R.IU.oy - 2 * D + R.ij * kBoxRows, R.IU.plane,
                R.bars + s);
  }
  ++R.issued;
  if (++R.ij == R.IU.nbox) {
    R.ij = 0;
    R.iu += stride;
    if (R.iu < kp.units) R.IU = unit_geom(kp, g, R.iu, D);
  }
}

// Every lane's value at a column outside [0, W) becomes the value at the
// nearest column inside, fetched from the lane that holds it.  (Out of line,
// by value: only strips at the image's left and right edges call it.)
__device__ __noinline__ float4 clamp_cols4(float4 q, int c0, int x0, int W) {
  const float v[4] = {q.x, q.y, q.z, q.w};
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
  return make_float4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ void clamp_cols(float (&v)[4], int c0, int x0, int W) {
  const float4 r = clamp_cols4(make_float4(v[0], v[1], v[2], v[3]), c0, x0, W);
  v[0] = r.x; v[1] = r.y; v[2] = r.z; v[3] = r.w;
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

__host__ __device__ constexpr int mod5(int x) { return ((x % 5) + 5) % 5; }

// One run of rows of one strip of one plane.  Step t reads input row t of the
// run (image row oy - 2D + t); stage s's input row at that step is t - 2s, its
// output row t - 2(s+1), valid from t = 4(s+1) on; the last stage's output row
// t - 2D is image row oy + t - 4D.  Windows are indexed by row mod 5, so a
// loop unrolled five times keeps them in fixed registers.  F32: every storage
// type is f32 (no rounding).  ODT: 0 f32, 1 f16, 2 bf16 packed stores, 3 any.
template <int D, int ODT, bool F32>
struct ChainRun {
  const CRowsParams& kp;
  const StripGeom& g;
  Ring& R;
  const Unit U;
  const int lane, stride, c0, esize;
  const bool hb;             // the strip touches the left or right image edge
  const bool vedge;          // the run reads rows outside the image
  float hx[D][5][4];         // per stage: x-pass results of its last 5 input rows
  bool st_full, st_part;     // the lane stores four columns / some of its columns
  char* out_row;             // the next output row
  unsigned q;                // box being read
  int rr;                    // row within it
  const unsigned char* slot;

  __device__ __forceinline__ ChainRun(const CRowsParams& kp_, const StripGeom& g_, Ring& R_, const Unit& U_,
                                      int lane_, int stride_)
      : kp(kp_), g(g_), R(R_), U(U_), lane(lane_), stride(stride_), c0(U_.x0 + 4 * lane_),
        esize(kp_.a.in.dtype == HP_F32 ? 4 : 2), hb(U_.x0 < 0 || U_.x0 + 128 > kp_.a.in.w),
        vedge(U_.oy < 2 * D || U_.oy + U_.n_in - 2 * D > kp_.a.in.h), q(R_.released), rr(0), slot(nullptr) {
    const int W = kp.a.out.w;
    const bool mine = lane >= g.halo_lanes && lane < 32 - g.halo_lanes;
    st_full = mine && c0 + 3 < W && ODT != 3;
    st_part = mine && c0 < W && !st_full;
    out_row = (char*)kp.a.out.data + (long long)U.plane * kp.a.out.ps + (long long)U.oy * kp.a.out.rs;
  }

  __device__ __forceinline__ bool wait_box() {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_poll(R.bars + q % kRing, (q / kRing) & 1u, 2000000000ull);
    __syncwarp();
    ok = __shfl_sync(kFull, ok, 0);
    slot = R.slots + (q % kRing) * g.slot_bytes + lane * 4 * esize;
    return ok != 0;
  }

  __device__ __forceinline__ void release_box() {
    ++q;
    __syncwarp();
    R.released = q;
    issue_one<D>(kp, g, R, stride, lane);
  }

  // x pass of stage S over a row (columns c0-2 .. c0+5) into window slot J,
  // then the window copies of the image's top and bottom boundary rows (y is
  // the row's image row).
  template <int S, int J>
  __device__ __forceinline__ void xpass(const float (&v)[4], int y) {
    const float* w = kp.a.w[S];
    const float l2 = __shfl_up_sync(kFull, v[2], 1), l1 = __shfl_up_sync(kFull, v[3], 1);
    const float r1 = __shfl_down_sync(kFull, v[0], 1), r2 = __shfl_down_sync(kFull, v[1], 1);
    hx[S][J][0] = tap5(w, l2, l1, v[0], v[1], v[2]);
    hx[S][J][1] = tap5(w, l1, v[0], v[1], v[2], v[3]);
    hx[S][J][2] = tap5(w, v[0], v[1], v[2], v[3], r1);
    hx[S][J][3] = tap5(w, v[1], v[2], v[3], r1, r2);
    if (vedge) {
      if (y == 0) {  // rows -2 and -1 of this stage's input are row 0
#pragma unroll
        for (int k = 0; k < 4; ++k) { hx[S][mod5(J - 1)][k] = hx[S][J][k]; hx[S][mod5(J - 2)][k] = hx[S][J][k]; }
      }
      if (y >= kp.a.in.h) {  // rows H and H + 1 are row H - 1
#pragma unroll
        for (int k = 0; k < 4; ++k) hx[S][J][k] = hx[S][mod5(J - 1)][k];
      }
    }
  }

  // y pass of stage S whose newest window row sits in slot J; then either the
  // next stage's x pass or the store.
  template <int S, int M>
  __device__ __forceinline__ void stage(int t) {
    constexpr int J = mod5(M - 2 * S);
    const float* w = kp.a.w[S] + 5;
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float b = tap5(w, hx[S][mod5(J + 1)][k], hx[S][mod5(J + 2)][k], hx[S][mod5(J + 3)][k], hx[S][mod5(J + 4)][k],
                     hx[S][J][k]);
      if (!F32) b = round_storage(kp.a.storage[S], b);
      o[k] = b;
    }
    if constexpr (S + 1 < D) {
      if (hb) clamp_cols(o, c0, U.x0, kp.a.in.w);
      xpass<S + 1, mod5(M - 2 * (S + 1))>(o, U.oy - 2 * D + t - 2 * (S + 1));
      stage<S + 1, M>(t);
      return;
    }
    if (t < 4 * D) return;  // the chain's output is not valid yet
    char* row = out_row;
    out_row += kp.a.out.rs;
    if (st_full) {
      if (ODT == 0) {
        *reinterpret_cast<float4*>(row + 4LL * c0) = make_float4(o[0], o[1], o[2], o[3]);
      } else {
        uint2 u;
        if (ODT == 1) {
          __half2 p0 = __floats2half2_rn(o[0], o[1]), p1 = __floats2half2_rn(o[2], o[3]);
          u.x = *reinterpret_cast<unsigned*>(&p0);
          u.y = *reinterpret_cast<unsigned*>(&p1);
        } else {
          __nv_bfloat162 p0 = __floats2bfloat162_rn(o[0], o[1]), p1 = __floats2bfloat162_rn(o[2], o[3]);
          u.x = *reinterpret_cast<unsigned*>(&p0);
          u.y = *reinterpret_cast<unsigned*>(&p1);
        }
        *reinterpret_cast<uint2*>(row + 2LL * c0) = u;
      }
    } else if (st_part) {
      const int y = U.oy + t - 4 * D;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (c0 + k < kp.a.out.w) store_px(kp.a.out, U.plane, c0 + k, y, o[k]);
    }
  }

  template <int M>
  __device__ __forceinline__ bool step(int t) {
    if (rr == 0 && !wait_box()) return false;
    float v[4];
    load4(slot + rr * 128 * esize, kp.a.in.dtype, v);
    if (++rr == kBoxRows) {
      rr = 0;
      release_box();
    }
    if (hb) clamp_cols(v, c0, U.x0, kp.a.in.w);
    xpass<0, M>(v, U.oy - 2 * D + t);
    stage<0, M>(t);
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
      if (!step<3>(t)) return false;
      if (++t >= n) break;
      if (!step<4>(t)) return false;
      if (++t >= n) break;
    }
    if (rr != 0) {  // the unit's last box had rows to spare
      rr = 0;
      release_box();
    }
    return true;
  }
};

template <int D, int ODT, bool F32>
__global__ void __launch_bounds__(256, 2) k_chain_rows(const __grid_constant__ CRowsParams kp) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const StripGeom g = strip_geom(D, kp.a.in.dtype == HP_F32 ? 4 : 2);
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
  R.IU = unit_geom(kp, g, gw, D);
  for (int i = 0; i < kRing; ++i) issue_one<D>(kp, g, R, stride, lane);
  for (int u = gw; u < kp.units; u += stride) {
    ChainRun<D, ODT, F32> run(kp, g, R, unit_geom(kp, g, u, D), lane, stride);
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

typedef void (*CRowsKernel)(CRowsParams);

template <int D>
CRowsKernel pick_d(const ChainArgs& a, int* variant) {
  bool f32 = a.in.dtype == HP_F32 && a.out.dtype == HP_F32;
  for (int s = 0; s < D; ++s) f32 &= a.storage[s] == HP_F32;
  const int odt = a.out.dtype == HP_F32 ? 0 : a.out.dtype == HP_F16 ? 1 : a.out.dtype == HP_BF16 ? 2 : 3;
  if (f32) { *variant = 0; return k_chain_rows<D, 0, true>; }
  *variant = 1 + odt;
  switch (odt) {
    case 0: return k_chain_rows<D, 0, false>;
    case 1: return k_chain_rows<D, 1, false>;
    case 2: return k_chain_rows<D, 2, false>;
    default: return k_chain_rows<D, 3, false>;
  }
}

CRowsKernel pick_kernel(const ChainArgs& a, int* variant) {
  if (a.depth == 2) return pick_d<2>(a, variant);
  CRowsKernel k = pick_d<4>(a, variant);
  *variant += 5;
  return k;
}

}  // namespace

bool chain_rows_depth_ok(int depth) { return depth == 2 || depth == 4; }

int chain_rows_strip_w(int depth, int in_dtype) { return strip_geom(depth, in_dtype == HP_F32 ? 4 : 2).strip_w; }

int chain_rows_smem_bytes(int depth, int threads, int in_dtype) {
  const StripGeom g = strip_geom(depth, in_dtype == HP_F32 ? 4 : 2);
  return 128 + kBarBytes + (threads / 32) * kRing * g.slot_bytes;
}

// Persistent grid: enough CTAs to fill every SM at the kernel's occupancy, or
// fewer when there are fewer units.
int chain_rows_grid(const ChainArgs& a, int units, int threads, int smem_bytes) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0, variant = 0;
  CRowsKernel kern = pick_kernel(a, &variant);
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

int launch_chain_rows(const ChainArgs& a, int rows, int grid, int smem_bytes, void* stream) {
  int variant;
  CRowsKernel kern = pick_kernel(a, &variant);
  static bool configured[10] = {};
  if (!configured[variant]) {
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[variant] = true;
  }
  CRowsParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  const int dt = a.in.dtype;
  const int esize = dt == HP_F32 ? 4 : 2;
  const StripGeom g = strip_geom(a.depth, esize);
  kp.strips = (a.out.w + g.strip_w - 1) / g.strip_w;
  kp.runs = (a.out.h + rows - 1) / rows;
  kp.rows = rows;
  kp.units = kp.strips * kp.runs * a.out.c;
  CUtensorMapDataType tdt = dt == HP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                            : dt == HP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps, 128, kBoxRows, 1))
    return (int)cudaErrorInvalidValue;
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(a.threads), smem_bytes, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
