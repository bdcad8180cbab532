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
// Lanes 0 and 31 only feed their neighbours.  The two fine rows of D_l a
// coarse step composites arrive as one TMA box (68 fine columns from a 16-byte
// aligned start, 2 rows, the 4 planes) through a ring of 3 shared-memory slots
// private to the warp, issued in the order the warp will read them (across its
// runs), so the fine loads are in flight well ahead of their use without
// holding registers.  The operations are those of the
// per-pixel expressions (x pass over each coarse row, then the y pass, in tap
// order; op_over, op_unpremul), so results are bit-identical to the generic
// kernel.  All stages are stored as f32 (the host checks).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStripW = 30;   // coarse columns per warp
constexpr int kBoxW = 68;     // fine columns per box: lanes 0..31's 64, from 4 left of lane 1's first (16-byte aligned)
constexpr int kBoxBytes = kBoxW * 2 * 4 * 4;          // 2 fine rows x 4 planes x f32
constexpr int kSlotBytes = (kBoxBytes + 127) / 128 * 128;  // slots start on 128-byte boundaries
constexpr int kRing = 3;      // boxes per warp ring
constexpr int kBarBytes = 512;  // mbarriers of up to 16 warps x kRing

struct InterpParams {
  CUtensorMap tmap;  // the fine level D_l: (W, H, planes), box (kBoxW, 2, 4)
  InterpArgs a;
  int strips, units;
};

// The warp's ring: box q (in issue order, which is the order of use) lives in
// slot q % kRing and completes phase (q / kRing) & 1 of that slot's mbarrier.
// Box j of a run holds fine rows 2 (n0 + j) and 2 (n0 + j) + 1.
struct Ring {
  unsigned char* slots;
  uint64_t* bars;
  unsigned issued, released;
  int iu, ij, inrun, ix, iy;  // next box: unit, box within it, the unit's boxes, its fine origin
};

__device__ __forceinline__ void set_unit(const InterpParams& P, Ring& R) {
  const int strip = R.iu % P.strips, run = R.iu / P.strips;
  const int n0 = run * P.a.rows;
  R.inrun = imin(P.a.rows, P.a.coarse.h - n0);
  R.ix = 2 * (strip * kStripW) - 4;
  R.iy = 2 * n0;
}

__device__ __forceinline__ void issue_one(const InterpParams& P, Ring& R, int stride, int lane) {
  if (R.iu >= P.units) return;
  if (lane == 0) {
    const int s = R.issued % kRing;
    // the warp's reads of this slot (its previous box) come before the copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(R.bars + s, (unsigned)kBoxBytes);
    tma_load_3d(R.slots + s * kSlotBytes, &P.tmap, R.ix, R.iy + 2 * R.ij, 0, R.bars + s);
  }
  ++R.issued;
  if (++R.ij == R.inrun) {
    R.ij = 0;
    R.iu += stride;
    if (R.iu < P.units) set_unit(P, R);
  }
}

template <bool FINAL>
struct InterpRun {
  const InterpParams& P;
  Ring& R;
  const int stride;
  int m, cm, X0, X1, n0, nrun, c0, c1;  // c0, c1: X0, X1 as columns of the box
  bool pair, prod, ok1;
  unsigned q;                 // box being read
  const float* box;           // its slot
  float hx[3][4][2];  // x-passed coarse rows (window slot, channel, fine column)
  float raw[4];       // the next coarse row, in flight

  __device__ __forceinline__ InterpRun(const InterpParams& p, Ring& r, int stride_)
      : P(p), R(r), stride(stride_), q(r.released), box(nullptr) {}

  __device__ __forceinline__ bool wait_box(int lane) {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_poll(R.bars + q % kRing, (q / kRing) & 1u, 2000000000ull);
    __syncwarp();
    ok = __shfl_sync(kFull, ok, 0);
    box = reinterpret_cast<const float*>(R.slots + (q % kRing) * kSlotBytes);
    return ok != 0;
  }

  __device__ __forceinline__ void release_box(int lane) {
    ++q;
    __syncwarp();
    R.released = q;
    issue_one(P, R, stride, lane);
  }

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

  // Fine row Y (row ODD of the current box) from window slots of coarse rows
  // n-1 (A), n (B), n+1 (C).
  template <bool ODD, int A, int B, int C>
  __device__ __forceinline__ void emit(int Y) const {
    float d[4][2];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const float* q = box + (2 * ch + (ODD ? 1 : 0)) * kBoxW;
      if (pair) {
        const float2 v = *reinterpret_cast<const float2*>(q + c0);
        d[ch][0] = v.x;
        d[ch][1] = v.y;
      } else {
        d[ch][0] = q[c0];
        d[ch][1] = q[c1];
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

  // False: a box never arrived.
  template <int PH>
  __device__ __forceinline__ bool step(int i, int lane) {
    constexpr int A = PH, B = (PH + 1) % 3, C = (PH + 2) % 3;
    xpass<C>();
    if (i + 3 <= nrun + 1) load_raw(i + 3);
    if (!wait_box(lane)) return false;
    const int Y = 2 * (n0 + i);
    emit<false, A, B, C>(Y);
    if (Y + 1 < P.a.fine.h) emit<true, A, B, C>(Y + 1);
    release_box(lane);
    return true;
  }

  __device__ __forceinline__ bool run(int strip, int run_idx) {
    const int lane = threadIdx.x & 31;
    const int W = P.a.fine.w;
    m = strip * kStripW + lane - 1;
    cm = iclamp(m, 0, P.a.coarse.w - 1);
    X0 = iclamp(2 * m, 0, W - 1);
    X1 = iclamp(2 * m + 1, 0, W - 1);
    c0 = X0 - (2 * (strip * kStripW) - 4);
    c1 = X1 - (2 * (strip * kStripW) - 4);
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
      if (!step<0>(i, lane)) return false;
      if (i + 1 >= nrun) break;
      if (!step<1>(i + 1, lane)) return false;
      if (i + 2 >= nrun) break;
      if (!step<2>(i + 2, lane)) return false;
    }
    return true;
  }
};

template <bool FINAL>
__global__ void __launch_bounds__(256, 3) k_interp_rows(const __grid_constant__ InterpParams P) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gw = blockIdx.x * nw + warp, stride = gridDim.x * nw;
  if (gw >= P.units) return;
  Ring R;
  R.bars = reinterpret_cast<uint64_t*>(base) + warp * kRing;
  R.slots = base + kBarBytes + warp * kRing * kSlotBytes;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < kRing; ++i) mbar_init(R.bars + i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  R.issued = R.released = 0;
  R.iu = gw;
  R.ij = 0;
  set_unit(P, R);
  for (int i = 0; i < kRing; ++i) issue_one(P, R, stride, lane);
  for (int u = gw; u < P.units; u += stride) {
    InterpRun<FINAL> r(P, R, stride);
    if (!r.run(u % P.strips, u / P.strips)) {
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

typedef void (*InterpKernel)(InterpParams);

InterpKernel pick_kernel(const InterpArgs& a) { return a.final_div ? k_interp_rows<true> : k_interp_rows<false>; }

}  // namespace

int interp_rows_strip_w() { return kStripW; }

int interp_rows_smem_bytes(int threads) { return 128 + kBarBytes + (threads / 32) * kRing * kSlotBytes; }

int interp_rows_grid(const InterpArgs& a, int units, int threads) {
  const int nw = threads / 32;
  const int need = (units + nw - 1) / nw;
  int dev = 0, sms = 0, per_sm = 0;
  const InterpKernel kern = pick_kernel(a);
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      allow_max_dynamic_smem((const void*)kern) != 0 ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, interp_rows_smem_bytes(threads)) != cudaSuccess ||
      per_sm < 1) {
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
  const InterpKernel kern = pick_kernel(a);
  int e = allow_max_dynamic_smem((const void*)kern);
  if (e) return e;
  if (encode_tmap_3d(&kp.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.fine.data, a.fine.w, a.fine.h, a.fine.c, a.fine.rs,
                     a.fine.ps, kBoxW, 2, 4))
    return (int)cudaErrorInvalidValue;
  { const int le_ = launch_kernel(kern, dim3(grid), dim3(a.threads), interp_rows_smem_bytes(a.threads), stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
