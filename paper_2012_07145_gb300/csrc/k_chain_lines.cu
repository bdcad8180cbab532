// Line-buffer stencil chain: D consecutive 5x5 separable stencil stages
// (D even, 2..8) fused in one CTA per T_w x T_h output tile -- the long-range
// fusion of the stencil chain (Sec. 2, Fig. 1) with the producer/consumer
// rows staged on chip (Sec. 4.7), in a line-buffered order instead of whole
// overlapped tiles.
//
// Every stage owns its own threads, each computing one block of 8 columns of
// that stage for every row of the tile, so the x pass of a row is never
// recomputed and no 2-D halo is carried: stage s covers columns
// [ox - 2(D - s), ox + T_w + 2(D - s)) and rows [oy - 2(D - s), oy + T_h + 2(D - s))
// clamped to the image.  Rows flow through shared-memory rings: stage 0 (the
// input) arrives as TMA boxes of 4 rows into a 16-row ring; stage s = 1..D-1
// writes its rows into a 12-row ring of its own; stage D stores to global
// memory.  The CTA advances in steps of 4 rows with one barrier per step;
// stage s runs 2 steps behind stage s - 1, so every row it reads was written
// in an earlier step and no row is overwritten before its last reader is done.
//
// A thread keeps its stage's y pass as four running partial sums per column
// (tap k of output row o is added when row o + k - 2 arrives, in tap order),
// so the y pass is the same fma chain as the stage-per-kernel schedule's and
// the result is bit-identical to it.  The x pass of a row reads 12 values
// with three 128-bit shared loads.  The threads of stages 2p+1 and 2p+2 are
// interleaved lane by lane and their rings start 16 bytes apart modulo 128,
// so each quarter warp's 128-bit accesses cover all 32 banks once.
//
// Boundaries, per stage on its own producer (clamp to edge): at the image top,
// the first row supplies the two rows above it (its x pass enters three taps
// at once); at the bottom, the last row is fed again for the two rows below;
// in tiles that reach past the left or right edge, the threads whose 12
// columns leave the image read them at clamped columns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"
#include "tma.cuh"

namespace hp {

namespace {

constexpr int kStep = 4;       // rows per step, and rows per TMA box
constexpr int kRing = 12;      // rows per ring of stages 1..D-1
constexpr int kGroups = 4;     // TMA boxes held in the input ring (16 rows)
constexpr int kMaxPairs = kLinesMaxDepth / 2;
constexpr int kHeader = 128;   // mbarriers and the abort flag

struct LinesGeom {
  int D, tw, th;
  int P0;                      // input ring pitch in elements (= TMA box width)
  int P;                       // pitch of rings 1..D-1 in floats
  int npairs;
  int tbase[kMaxPairs + 1];    // first thread of each stage pair; tbase[npairs] = threads in use
  int ring_off[kLinesMaxDepth];  // byte offset of ring r from the aligned base
  int threads, smem;
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

LinesGeom lines_geom(int D, int tw, int th, int esize) {
  LinesGeom g;
  memset(&g, 0, sizeof g);
  g.D = D;
  g.tw = tw;
  g.th = th;
  g.npairs = D / 2;
  g.tbase[0] = 0;
  int widest = 0;
  for (int p = 0; p < g.npairs; ++p) {
    const int w_odd = tw + 4 * (D - (2 * p + 1));  // the wider stage of the pair
    const int nb = (w_odd + 7) / 8;
    widest = nb > widest ? nb : widest;
    g.tbase[p + 1] = g.tbase[p] + 2 * nb;
  }
  g.threads = round_up(g.tbase[g.npairs], 32);
  // the input ring: a 128-byte multiple per row, at least the stage-0 width
  g.P0 = round_up(tw + 4 * D, 128 / esize);
  // rings 1..D-1: 8 columns per block of the widest pair (reads past it fall
  // into the next row and only feed columns that are never used)
  g.P = round_up(8 * widest, 32);
  int off = kHeader;
  g.ring_off[0] = off;
  off += kGroups * kStep * g.P0 * esize;
  for (int r = 1; r < D; ++r) {
    off = round_up(off, 128) + 16 * (r & 1);
    g.ring_off[r] = off;
    off += kRing * g.P * 4;
  }
  // slack for the last ring's reads past its end, and for aligning the base
  g.smem = round_up(off, 128) + 128 + 128;
  return g;
}

struct LinesParams {
  CUtensorMap tmap;
  ChainArgs a;
  LinesGeom g;
};

template <int T>
__device__ __forceinline__ float rnd_t(float v) {
  if (T == 1) return __half2float(__float2half_rn(v));
  if (T == 2) return __bfloat162float(__float2bfloat16_rn(v));
  return v;
}

template <int T>
__device__ __forceinline__ float elem(const unsigned char* row, int c) {
  if (T == 1) return __half2float(reinterpret_cast<const __half*>(row)[c]);
  if (T == 2) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[c]);
  return reinterpret_cast<const float*>(row)[c];
}

__device__ __forceinline__ void unpack2(unsigned u, float* x, int T) {
  if (T == 1) {
    const __half2 h = *reinterpret_cast<const __half2*>(&u);
    x[0] = __low2float(h);
    x[1] = __high2float(h);
  } else {
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&u);
    x[0] = __low2float(h);
    x[1] = __high2float(h);
  }
}

// 12 consecutive values from column c of a ring row (16-byte aligned).
template <int T>
__device__ __forceinline__ void load12(const unsigned char* row, int c, float* x) {
  if (T == 0) {
    const float* p = reinterpret_cast<const float*>(row) + c;
    const float4 q0 = *reinterpret_cast<const float4*>(p);
    const float4 q1 = *reinterpret_cast<const float4*>(p + 4);
    const float4 q2 = *reinterpret_cast<const float4*>(p + 8);
    x[0] = q0.x; x[1] = q0.y; x[2] = q0.z; x[3] = q0.w;
    x[4] = q1.x; x[5] = q1.y; x[6] = q1.z; x[7] = q1.w;
    x[8] = q2.x; x[9] = q2.y; x[10] = q2.z; x[11] = q2.w;
  } else {
    const unsigned char* p = row + 2 * c;
    const uint4 q0 = *reinterpret_cast<const uint4*>(p);
    const uint2 q1 = *reinterpret_cast<const uint2*>(p + 16);
    unpack2(q0.x, x + 0, T);
    unpack2(q0.y, x + 2, T);
    unpack2(q0.z, x + 4, T);
    unpack2(q0.w, x + 6, T);
    unpack2(q1.x, x + 8, T);
    unpack2(q1.y, x + 10, T);
  }
}

template <int T>
__device__ __forceinline__ void store8_global(char* row, const float* v) {
  if (T == 0) {
    *reinterpret_cast<float4*>(row) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(row + 16) = make_float4(v[4], v[5], v[6], v[7]);
  } else {
    uint4 u;
    unsigned* w = reinterpret_cast<unsigned*>(&u);
    for (int k = 0; k < 4; ++k) {
      if (T == 1) {
        __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<unsigned*>(&h);
      } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<unsigned*>(&h);
      }
    }
    *reinterpret_cast<uint4*>(row) = u;
  }
}

// Input type, every stage's storage and the output type are T (0: f32, 1: f16, 2: bf16).
template <int T>
__global__ void __launch_bounds__(kLinesMaxThreads) k_chain_lines(const __grid_constant__ LinesParams kp) {
  grid_dep_sync();
  const ChainArgs& a = kp.a;
  const LinesGeom& g = kp.g;
  constexpr int esize = T == 0 ? 4 : 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(base + 64);
  unsigned char* ring0 = base + g.ring_off[0];

  const int D = g.D;
  const int W = a.in.w, H = a.in.h;
  const int ch = blockIdx.z;
  const int ox = blockIdx.x * g.tw, oy = blockIdx.y * g.th;
  const int a0 = max(oy - 2 * D, 0), b0 = min(oy + g.th + 2 * D, H);
  const int ngroups = (b0 - a0 + kStep - 1) / kStep;
  // steps: stage D starts at step 2D - 1 and is the last to finish
  const int K = 2 * D - 1 + (min(oy + g.th, H) + 2 - max(oy - 2, 0) + kStep - 1) / kStep;

  // ---- this thread's stage s (1..D; 0: idle) and column block b ----
  const int t = threadIdx.x;
  int s = 0, b = 0;
#pragma unroll
  for (int q = 0; q < kMaxPairs; ++q)
    if (q < g.npairs && t >= g.tbase[q] && t < g.tbase[q + 1]) {
      const int j = t - g.tbase[q];
      s = 2 * q + 1 + (j & 1);
      b = j >> 1;
    }
  const int sp = s > 0 ? s : 1;
  const int Xp = ox - 2 * (D - sp + 1);  // producer rectangle's first image column
  const int ap = max(oy - 2 * (D - sp + 1), 0), bp = min(oy + g.th + 2 * (D - sp + 1), H);
  const int top = ap == 0;
  // feeds: producer rows ap.. (the last one repeated below the image) until
  // the stage's own last row, min(oy + th + 2(D - s), H) - 1, has its five taps
  const int nfeed = min(oy + g.th + 2 * (D - sp), H) + 2 - ap;
  const int Ls = 2 * sp - 1;
  const int nsteps = (nfeed + kStep - 1) / kStep;
  const int c0 = Xp + 8 * b;
  const bool xedge = c0 < 0 || c0 + 11 > W - 1;
  const bool last = s == D;
  float wx[5], wy[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    wx[k] = a.w[sp - 1][k];
    wy[k] = a.w[sp - 1][5 + k];
  }
  const unsigned char* src = base + g.ring_off[sp - 1];
  float* dst = reinterpret_cast<float*>(base + g.ring_off[sp < D ? sp : 0]);
  const int row_elems = sp == 1 ? g.P0 : g.P;
  const int src_pitch = sp == 1 ? g.P0 * esize : g.P * 4;
  char* out_plane = (char*)a.out.data + (long long)ch * a.out.ps;
  const int gx = ox + 8 * b;  // last stage: first output column of the block
  const bool out_block = last && 8 * b < g.tw && gx < a.out.w;
  const bool out_full = out_block && 8 * b + 8 <= g.tw && gx + 8 <= a.out.w;

  if (t == 0) {
    *abort_flag = 0;
    for (int k = 0; k < kGroups; ++k) mbar_init(bar + k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int gi) {
    uint64_t* bb = bar + (gi & (kGroups - 1));
    mbar_arrive_expect_tx(bb, (unsigned)(kStep * g.P0 * esize));
    tma_load_3d(ring0 + (size_t)(gi & (kGroups - 1)) * kStep * g.P0 * esize, &kp.tmap, ox - 2 * D, a0 + kStep * gi,
                ch, bb);
  };
  if (t == 0 && ngroups > 0) issue(0);

  float acc[4][8];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[u][c] = 0.0f;

  int k = 0;
  for (; k < K; ++k) {
    if (t == 0 && k + 1 < ngroups) issue(k + 1);
    if (s != 0 && k >= Ls && k < Ls + nsteps) {
      if (s == 1 && k - 1 < ngroups) {
        const int gi = k - 1;
        if (!mbar_wait_bounded(bar + (gi & (kGroups - 1)), (unsigned)((gi >> 2) & 1), 2000000000ull))
          *abort_flag = 1;  // gives up after 2 s; the whole block stops after this step
      }
      const int f0 = (k - Ls) * kStep;
#pragma unroll
      for (int u = 0; u < kStep; ++u) {
        const int i = f0 + u;
        if (i < nfeed) {
          const int r = min(ap + i, bp - 1);  // producer row of this feed
          const unsigned char* row =
              src + (size_t)(s == 1 ? ((r - a0) & (kGroups * kStep - 1)) : (r % kRing)) * src_pitch;
          float x[12];
          if (!xedge) {
            if (s == 1)
              load12<T>(row, 8 * b, x);
            else
              load12<0>(row, 8 * b, x);
          } else {
            // clamp to the image, and keep the columns of blocks that only
            // feed unused outputs inside the ring row
#pragma unroll
            for (int q = 0; q < 12; ++q) {
              const int cc = min(min(max(c0 + q, 0), W - 1) - Xp, row_elems - 1);
              x[q] = s == 1 ? elem<T>(row, cc) : elem<0>(row, cc);
            }
          }
          float h[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) h[c] = tap5(wx, x[c], x[c + 1], x[c + 2], x[c + 3], x[c + 4]);
          if (u == 0 && top && i == 0) {
            // rows -2 and -1 are row 0: its x pass enters three taps of output
            // row 0, two of row 1 and one of row 2
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              float o0 = __fmul_rn(wy[0], h[c]);
              o0 = __fmaf_rn(wy[1], h[c], o0);
              acc[2][c] = __fmaf_rn(wy[2], h[c], o0);
              const float o1 = __fmul_rn(wy[0], h[c]);
              acc[3][c] = __fmaf_rn(wy[1], h[c], o1);
              acc[0][c] = o1;
            }
          } else {
            if (i >= 4 - 2 * top) {
              // output row o completes with its fifth tap
              const int o = ap + i - 2;
              float v[8];
#pragma unroll
              for (int c = 0; c < 8; ++c) v[c] = rnd_t<T>(__fmaf_rn(wy[4], h[c], acc[u][c]));
              if (!last) {
                float* d = dst + (size_t)(o % kRing) * g.P + 8 * b;
                *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
                *reinterpret_cast<float4*>(d + 4) = make_float4(v[4], v[5], v[6], v[7]);
              } else if (out_full) {
                store8_global<T>(out_plane + (long long)o * a.out.rs + (long long)gx * esize, v);
              } else if (out_block) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                  if (8 * b + c < g.tw && gx + c < a.out.w) store_px(a.out, ch, gx + c, o, v[c]);
              }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              acc[(u + 1) & 3][c] = __fmaf_rn(wy[3], h[c], acc[(u + 1) & 3][c]);
              acc[(u + 2) & 3][c] = __fmaf_rn(wy[2], h[c], acc[(u + 2) & 3][c]);
              acc[(u + 3) & 3][c] = __fmaf_rn(wy[1], h[c], acc[(u + 3) & 3][c]);
              acc[u][c] = __fmul_rn(wy[0], h[c]);
            }
          }
        }
      }
    }
    __syncthreads();
    if (*abort_flag) break;
  }
  if (k < K) {
    // a box did not arrive: wait (bounded) for the boxes still in flight, then report
    if (t == 0) {
      for (int gi = max(k - 1, 0); gi < ngroups && gi <= k + 1; ++gi)
        mbar_wait_bounded(bar + (gi & (kGroups - 1)), (unsigned)((gi >> 2) & 1), 100000000ull);
      atomicExch(a.err, 1);
    }
  }
}

typedef void (*LinesKernel)(LinesParams);

}  // namespace

bool chain_lines_ok(int depth, int tile_w, int tile_h, int dtype) {
  if (depth < 2 || depth > kLinesMaxDepth || depth % 2) return false;
  if (dtype != HP_F32 && dtype != HP_F16 && dtype != HP_BF16) return false;
  const int esize = dtype == HP_F32 ? 4 : 2;
  // the TMA box starts at column ox - 2 depth: 16-byte aligned for every tile
  if ((2 * depth * esize) % 16) return false;
  if (tile_w < 8 || tile_w % 8 || tile_h < 2 * depth + 2) return false;
  const LinesGeom g = lines_geom(depth, tile_w, tile_h, esize);
  return g.P0 <= 256 && g.threads <= kLinesMaxThreads && g.smem <= kSmemLimit;
}

int chain_lines_threads(int depth, int tile_w, int tile_h, int dtype) {
  return lines_geom(depth, tile_w, tile_h, dtype == HP_F32 ? 4 : 2).threads;
}

int chain_lines_smem_bytes(int depth, int tile_w, int tile_h, int dtype) {
  return lines_geom(depth, tile_w, tile_h, dtype == HP_F32 ? 4 : 2).smem;
}

int launch_chain_lines(const ChainArgs& a, void* stream) {
  static bool configured[3] = {};
  const int dt = a.in.dtype;
  const int vi = dt == HP_F16 ? 1 : dt == HP_BF16 ? 2 : 0;
  LinesKernel kern = vi == 0 ? k_chain_lines<0> : vi == 1 ? k_chain_lines<1> : k_chain_lines<2>;
  if (!configured[vi]) {
    int e = allow_max_dynamic_smem((const void*)kern);
    if (e) return e;
    configured[vi] = true;
  }
  const int esize = vi == 0 ? 4 : 2;
  LinesParams kp;
  memset(&kp, 0, sizeof kp);
  kp.a = a;
  kp.g = lines_geom(a.depth, a.tile_w, a.tile_h, esize);
  const CUtensorMapDataType tdt = vi == 0   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : vi == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (encode_tmap_3d(&kp.tmap, tdt, esize, a.in.data, a.in.w, a.in.h, a.in.c, a.in.rs, a.in.ps, kp.g.P0, kStep))
    return (int)cudaErrorInvalidValue;
  dim3 grid(a.tiles_x, a.tiles_y, a.in.c);
  { const int le_ = launch_kernel(kern, grid, dim3(kp.g.threads), kp.g.smem, stream, kp); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
