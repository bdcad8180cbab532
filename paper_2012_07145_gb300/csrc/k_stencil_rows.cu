// Streaming single 5x5 stencil, optionally followed by the unsharp-mask
// combine (out = in + amount (in - blur)), per channel plane.
//
// Each warp owns a strip of output columns, four per lane, of one plane and
// walks down a run of rows.  Input rows arrive as TMA boxes (kBoxRows rows, 128
// columns) through a ring of shared-memory slots private to the warp, so the
// loads of later rows overlap the arithmetic on the current one and no barrier
// wider than the warp is taken.  The x pass takes its two neighbours on each
// side from the adjacent lanes (the outer lanes only feed them), the y pass
// runs over a 5-row register window of x-pass results, and the unsharp
// combine reads the input row from a matching 5-row window.  The stencil and
// combine expressions are those of stage_math.cuh, so the result is
// bit-identical to every other schedule of the pipeline.
//
// Boundary condition (clamp to edge on the stencil's input): in strips that
// touch the left or right image edge the input row's columns outside the image
// take the edge column's value (shuffled from the lane that holds it); rows
// outside take the nearest edge row's x-pass result (a copy inside the window).
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

// A TMA box must start on a 16-byte boundary: 4 columns of a 4-byte input, 8
// of a 2-byte one; that sets the halo lanes (two columns of halo are needed).
__host__ __device__ inline StripGeom strip_geom(int esize) {
  StripGeom g;
  g.halo_lanes = esize == 4 ? 1 : 2;
  g.strip_w = 4 * (32 - 2 * g.halo_lanes);
  g.slot_bytes = 128 * kBoxRows * esize;
  return g;
}

struct SRowsParams {
  CUtensorMap tmap;
  ChainArgs a;  // depth 1: storage[0], w[0] (wx then wy), epilogue, amount
  int strips, runs, units, rows;  // per plane: strips x runs units of `rows` output rows
};

struct Unit {
  int x0, oy, plane, n_in, nbox;  // x0: image column of lane 0's first column
};

__device__ __forceinline__ Unit unit_geom(const SRowsParams& kp, const StripGeom& g, int u) {
  Unit U;
  const int per_plane = kp.strips * kp.runs;
  U.plane = u / per_plane;
  const int v = u - U.plane * per_plane;
  const int run = v / kp.strips, s = v - run * kp.strips;
  U.x0 = s * g.strip_w - 4 * g.halo_lanes;
  U.oy = run * kp.rows;
  U.n_in = min(kp.rows, kp.a.out.h - U.oy) + 4;
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

__device__ __forceinline__ void issue_one(const SRowsParams& kp, const StripGeom& g, Ring& R, int stride, int lane) {
  if (R.iu >= kp.units) return;
  if (lane == 0) {
    const int s = R.issued % kRing;
    mbar_arrive_expect_tx(R.bars + s, (unsigned)g.slot_bytes);
    tma_load_3d(R.slots + s * g.slot_bytes, &kp.tmap, R.IU.x0, R.IU.oy - 2 + R.ij * kBoxRows, R.IU.plane,
                R.bars + s);
  }
  ++R.issued;
  if (++R.ij == R.IU.nbox) {
    R.ij = 0;
    R.iu += stride;
    if (R.iu < kp.units) R.IU = unit_geom(kp, g, R.iu);
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

// One run of rows of one strip of one plane.  Step t reads input row t
// (image row oy - 2 + t) and, from t = 4 on, emits output row t - 4 of the
// run.  Windows are indexed by row mod 5, so a loop unrolled five times keeps
// them in fixed registers.  F32 = every storage type is f32 (no rounding, one
// 128-bit store per lane and row).
// The binomial [1,4,6,4,1]/16 taps (the unsharp blur, the same float values
// the pipeline stores) as compile-time constants.
__device__ __forceinline__ float tap5_binomial_const(float a, float b, float c, float d, float e) {
  float s = __fmul_rn(0.0625f, a);
  s = __fmaf_rn(0.25f, b, s);
  s = __fmaf_rn(0.375f, c, s);
  s = __fmaf_rn(0.25f, d, s);
  return __fmaf_rn(0.0625f, e, s);
}

// BIN: both passes take the binomial taps (checked bit for bit on the host),
// compiled as constants: no registers for the taps, which lets the unsharp
// kernel keep five CTAs of 128 threads per SM without spilling.
template <bool F32, bool EPI, bool BIN>
struct StripRun {
  const SRowsParams& kp;
  const StripGeom& g;
  Ring& R;
  const Unit U;
  const int lane, stride, c0, esize;
  const bool hb;             // the strip touches the left or right image edge
  const bool vedge;          // the run reads rows outside the image
  float wx[5], wy[5];
  float hx[5][4];            // x-pass results
  float raw[5][4];           // input values (for the unsharp combine)
  bool st_full, st_part;     // the lane stores four columns / some of its columns
  char* out_row;             // the next output row
  unsigned q;                // box being read
  int rr;                    // row within it
  const unsigned char* slot;

  __device__ __forceinline__ StripRun(const SRowsParams& kp_, const StripGeom& g_, Ring& R_, const Unit& U_,
                                      int lane_, int stride_)
      : kp(kp_), g(g_), R(R_), U(U_), lane(lane_), stride(stride_), c0(U_.x0 + 4 * lane_),
        esize(kp_.a.in.dtype == HP_F32 ? 4 : 2), hb(U_.x0 < 0 || U_.x0 + 128 > kp_.a.in.w),
        vedge(U_.oy < 2 || U_.oy + U_.n_in - 2 > kp_.a.in.h), q(R_.released),
        rr(0), slot(nullptr) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      wx[k] = kp.a.w[0][k];
      wy[k] = kp.a.w[0][5 + k];
    }
    const int W = kp.a.out.w;
    const bool mine = lane >= g.halo_lanes && lane < 32 - g.halo_lanes;
    st_full = mine && c0 + 3 < W && F32;
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
    issue_one(kp, g, R, stride, lane);
  }

  template <int M>
  __device__ __forceinline__ bool step(int t) {
    const ChainArgs& a = kp.a;
    const int r = U.oy - 2 + t;
    if (rr == 0 && !wait_box()) return false;
    float v[4];
    load4(slot + rr * 128 * esize, F32 ? HP_F32 : a.in.dtype, v);
    if (++rr == kBoxRows) {
      rr = 0;
      release_box();
    }
    if (hb) clamp_cols(v, c0, U.x0, a.in.w);
#pragma unroll
    for (int k = 0; k < 4; ++k) raw[M][k] = v[k];
    // x pass: columns c0-2 .. c0+5
    const float l2 = __shfl_up_sync(kFull, v[2], 1), l1 = __shfl_up_sync(kFull, v[3], 1);
    const float r1 = __shfl_down_sync(kFull, v[0], 1), r2 = __shfl_down_sync(kFull, v[1], 1);
    hx[M][0] = BIN ? tap5_binomial_const(l2, l1, v[0], v[1], v[2]) : tap5(wx, l2, l1, v[0], v[1], v[2]);
    hx[M][1] = BIN ? tap5_binomial_const(l1, v[0], v[1], v[2], v[3]) : tap5(wx, l1, v[0], v[1], v[2], v[3]);
    hx[M][2] = BIN ? tap5_binomial_const(v[0], v[1], v[2], v[3], r1) : tap5(wx, v[0], v[1], v[2], v[3], r1);
    hx[M][3] = BIN ? tap5_binomial_const(v[1], v[2], v[3], r1, r2) : tap5(wx, v[1], v[2], v[3], r1, r2);
    if (vedge && (r < 1 || r >= a.in.h)) {
      if (r == 0) {  // rows -2 and -1 are row 0
#pragma unroll
        for (int k = 0; k < 4; ++k) { hx[(M + 3) % 5][k] = hx[M][k]; hx[(M + 4) % 5][k] = hx[M][k]; }
      }
      if (r >= a.in.h) {  // rows H and H + 1 are row H - 1
#pragma unroll
        for (int k = 0; k < 4; ++k) hx[M][k] = hx[(M + 4) % 5][k];
      }
    }
    if (t >= 4) {
      // y pass over rows t-4 .. t -> output row t - 4 of the run (input row t - 2)
      constexpr int J0 = (M + 1) % 5, J1 = (M + 2) % 5, J2 = (M + 3) % 5, J3 = (M + 4) % 5;
      float o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float b = BIN ? tap5_binomial_const(hx[J0][k], hx[J1][k], hx[J2][k], hx[J3][k], hx[M][k])
                      : tap5(wy, hx[J0][k], hx[J1][k], hx[J2][k], hx[J3][k], hx[M][k]);
        if (!F32) b = round_storage(a.storage[0], b);
        if (EPI) {
          b = op_unsharp(raw[J2][k], b, a.amount);
          if (!F32) b = round_storage(a.out.dtype, b);
        }
        o[k] = b;
      }
      char* row = out_row;
      out_row += a.out.rs;
      if (st_full) {
        *reinterpret_cast<float4*>(row + 4LL * c0) = make_float4(o[0], o[1], o[2], o[3]);
      } else if (st_part) {
        const int y = U.oy + t - 4;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (c0 + k < a.out.w) store_px(a.out, U.plane, c0 + k, y, o[k]);
      }
    }
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

template <bool F32, bool EPI, bool BIN>
__global__ void __maxnreg__(BIN ? 96 : 128) k_stencil_rows(const __grid_constant__ SRowsParams kp) {
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
    StripRun<F32, EPI, BIN> run(kp, g, R, unit_geom(kp, g, u), lane, stride);
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

typedef void (*SRowsKernel)(SRowsParams);

// Whether both passes' taps are the binomial ones, bit for bit.
bool binomial_taps(const ChainArgs& a) {
  static const float b[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
  return memcmp(a.w[0], b, sizeof b) == 0 && memcmp(a.w[0] + 5, b, sizeof b) == 0;
}

template <bool BIN>
SRowsKernel pick_fe(bool f32, bool epi) {
  if (epi) return f32 ? k_stencil_rows<true, true, BIN> : k_stencil_rows<false, true, BIN>;
  return f32 ? k_stencil_rows<true, false, BIN> : k_stencil_rows<false, false, BIN>;
}

SRowsKernel pick_kernel(const ChainArgs& a, int* variant) {
  const bool f32 = a.in.dtype == HP_F32 && a.storage[0] == HP_F32 && a.out.dtype == HP_F32;
  const bool epi = a.epilogue == 1;
  const bool bin = binomial_taps(a);
  *variant = (f32 ? 0 : 1) + (epi ? 2 : 0) + (bin ? 4 : 0);
  return bin ? pick_fe<true>(f32, epi) : pick_fe<false>(f32, epi);
}

}  // namespace

int stencil_rows_strip_w(int in_dtype) { return strip_geom(in_dtype == HP_F32 ? 4 : 2).strip_w; }

int stencil_rows_smem_bytes(int threads, int in_dtype) {
  const StripGeom g = strip_geom(in_dtype == HP_F32 ? 4 : 2);
  return 128 + kBarBytes + (threads / 32) * kRing * g.slot_bytes;
}

// Persistent grid: enough CTAs to fill every SM at the kernel's occupancy, or
// fewer when there are fewer units.
int stencil_rows_grid(const ChainArgs& a, int units, int threads, int smem_bytes) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0, variant = 0;
  SRowsKernel kern = pick_kernel(a, &variant);
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

int launch_stencil_rows(const ChainArgs& a, int rows, int grid, int smem_bytes, void* stream) {
  int variant;
  SRowsKernel kern = pick_kernel(a, &variant);
  static bool configured[8] = {};
  if (!configured[variant]) {
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[variant] = true;
  }
  SRowsParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  const int dt = a.in.dtype;
  const int esize = dt == HP_F32 ? 4 : 2;
  const StripGeom g = strip_geom(esize);
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
