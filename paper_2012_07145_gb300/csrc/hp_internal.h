// Internal structures shared by the host runtime (pipeline.cpp) and the CUDA
// kernels.  Plain C++ structs only: they are passed by value as kernel
// parameters.
#pragma once

#include <stdint.h>

#include <cuda_runtime.h>

#include "../../include/hp.h"

#if defined(__CUDACC__)
#define HPHD __host__ __device__ __forceinline__
#else
#define HPHD inline
#endif

#if defined(__CUDACC__)
// First statement of every kernel launched by launch_kernel: wait until the
// grid it depends on has completed (a no-op for a plain launch).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The same, then let the next kernel's launch begin at once: its blocks take
// the SMs this grid's last wave leaves free (and wait there).  For kernels
// that run in several waves; a persistent grid (one wave) gains nothing, and
// the local-Laplacian sequence measured slower with it.
__device__ __forceinline__ void grid_dep_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

namespace hp {

// A planar [C][H][W] image in device memory.  Strides in bytes.
struct ImgView {
  void* data;
  int dtype;
  int c, w, h;
  int pad_;
  long long rs, ps;
};

struct Rect {
  int x0, y0, x1, y1;  // half-open; empty when x1 <= x0 or y1 <= y0
};

HPHD int imin(int a, int b) { return a < b ? a : b; }
HPHD int imax(int a, int b) { return a > b ? a : b; }
HPHD int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
HPHD int floordiv2(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }
HPHD int ceildiv2(int v) { return -floordiv2(-v); }

// ---------------------------------------------------------------------------
// Group plan for the generic fused-group kernel (and the host bounds
// inference, which runs the same rect propagation).
// ---------------------------------------------------------------------------
constexpr int kMaxGNodes = 48;
constexpr int kMaxGExt = 8;
constexpr int kMaxGWeights = 512;
constexpr int kMaxGParams = 192;

struct GNode {
  int kind, op, channels, storage;
  int n_in;
  int in[HP_MAX_INPUTS];  // >= 0: node index inside the group; < 0: -1-e, external e
  int rx, ry;
  int w_off;              // wx (2rx+1) then wy (2ry+1) in GPlan::weights
  int p_off, n_params;    // in GPlan::params
  int dom_w, dom_h;
  int smem_off;           // float offset of this node's tile (channels * pitch * rows)
  int pitch, rows;        // allocation bounds of the tile
};

struct GPlan {
  int n_nodes;            // the output node is n_nodes - 1
  int n_ext;
  int tile_w, tile_h, tiles_x, tiles_y;
  int smem_floats;
  int pad_;
  int* err;               // device error word: set when a read falls outside its tile
  GNode nodes[kMaxGNodes];
  ImgView ext[kMaxGExt];
  ImgView out;
  float weights[kMaxGWeights];
  float params[kMaxGParams];
};

// Footprint of consumer `kind` (reading input slot `slot`) over its rect,
// expressed in the producer's coordinates, before clamping.
HPHD Rect footprint(int kind, int slot, int rx, int ry, Rect r) {
  Rect f = r;
  if (kind == HP_STENCIL || kind == HP_MAX_STENCIL) {
    f.x0 = r.x0 - rx; f.x1 = r.x1 + rx; f.y0 = r.y0 - ry; f.y1 = r.y1 + ry;
  } else if (kind == HP_DOWNSAMPLE2) {
    f.x0 = 2 * r.x0 - 2; f.x1 = 2 * r.x1 + 1; f.y0 = 2 * r.y0 - 2; f.y1 = 2 * r.y1 + 1;
  } else if (kind == HP_UPSAMPLE2) {
    if (slot == 1) { f.x0 = f.x1 = 0; f.y0 = f.y1 = 0; return f; }  // size reference: not read
    f.x0 = ceildiv2(r.x0 - 2); f.x1 = floordiv2(r.x1 + 1) + 1;
    f.y0 = ceildiv2(r.y0 - 2); f.y1 = floordiv2(r.y1 + 1) + 1;
  }
  return f;
}

HPHD bool rect_empty(Rect r) { return r.x1 <= r.x0 || r.y1 <= r.y0; }

// Rect of every node for the output tile at (tx0, ty0): the output node gets
// the tile clipped to its domain; each producer gets the union of its
// consumers' footprints clipped to its own domain (reverse topological order).
HPHD void infer_rects(const GPlan& g, int tx0, int ty0, Rect* rects) {
  for (int n = 0; n < g.n_nodes; ++n) rects[n] = Rect{0, 0, 0, 0};
  const GNode& o = g.nodes[g.n_nodes - 1];
  rects[g.n_nodes - 1] = Rect{tx0, ty0, imin(tx0 + g.tile_w, o.dom_w), imin(ty0 + g.tile_h, o.dom_h)};
  for (int n = g.n_nodes - 1; n >= 0; --n) {
    Rect r = rects[n];
    if (rect_empty(r)) continue;
    const GNode& nd = g.nodes[n];
    for (int s = 0; s < nd.n_in; ++s) {
      int m = nd.in[s];
      if (m < 0) continue;
      Rect f = footprint(nd.kind, s, nd.rx, nd.ry, r);
      if (rect_empty(f)) continue;
      const GNode& p = g.nodes[m];
      f.x0 = imax(f.x0, 0); f.y0 = imax(f.y0, 0);
      f.x1 = imin(f.x1, p.dom_w); f.y1 = imin(f.y1, p.dom_h);
      if (rect_empty(f)) continue;
      Rect& q = rects[m];
      if (rect_empty(q)) {
        q = f;
      } else {
        q.x0 = imin(q.x0, f.x0); q.y0 = imin(q.y0, f.y0);
        q.x1 = imax(q.x1, f.x1); q.y1 = imax(q.y1, f.y1);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Parameters of the specialised kernels.
// ---------------------------------------------------------------------------
constexpr int kSmemLimit = 227 * 1024 - 1024;  // opt-in maximum less static shared memory
constexpr int kChainMax = 32;

struct ChainArgs {
  ImgView in, out;
  int depth;
  int tile_w, tile_h, tiles_x, tiles_y;
  int threads, seg;
  int cols;                // streaming chain kernel: columns per lane (4 or 8)
  int storage[kChainMax];
  float w[kChainMax][10];  // per stage: wx[5] then wy[5]
  int epilogue;            // 0: none; 1: unsharp out = in + amount*(in - chain(in))
  float amount;
  int* err;                // device error word (bounded waits)
};

// Max filter group (k_max_rows.cu): window of radius 1..4, square (shape 0),
// horizontal (1) or vertical (2).
struct MaxArgs {
  ImgView in, out;
  int radius, shape, rows, threads;
  int st_mid, st_out;  // storages of the two stages (the same for a one-stage group)
  int* err;            // device error word (bounded waits)
};

// Interpolate level group (k_interp_rows.cu): I = D over U(coarse), optionally
// followed by the division by coverage.
struct InterpArgs {
  ImgView fine, coarse, out;  // D_l (4 ch), I_{l+1} (4 ch), the group's output
  int rows, threads, final_div, vec;
  int* err;  // device error word (bounded waits)
};

// Bilateral grid splat / slice (k_grid.cu).
struct GridArgs {
  ImgView in;    // the 1-channel image
  ImgView grid;  // (ceil(W/s)+1) x (ceil(H/s)+1), 2 gz channels
  ImgView out;   // slice: the 1-channel output
  int s, gz;
  float inv_s, inv_r;
};

// Blur of a bilateral grid (k_grid.cu): [1,4,6,4,1]/16 along the range levels,
// then x, then y; rows per run of the streaming kernel.
struct GridBlurArgs {
  ImgView in, out;
  int gz, rows;
};

// One point-wise stage over f32 images (k_pointwise.cu).
struct PwArgs {
  ImgView in[HP_MAX_INPUTS];
  ImgView out;
  int n_in, op;
  float p0, p1;
};

struct PointwiseArgs {
  int op, n_in, channels, storage;
  ImgView in[HP_MAX_INPUTS];
  ImgView out;
  float params[HP_MAX_PARAMS];
};

struct ResampleArgs {  // downsample / upsample, per channel
  ImgView in, out;
  int storage;
};

// Harris group: gray -> (Ix, Iy) 3x3 separable stencils -> products
// (Ixx, Iyy, Ixy) -> 3x3 separable sums (Sxx, Syy, Sxy) -> response.
struct HarrisArgs {
  ImgView in, out;          // in: 3 ch; out: 1 ch
  float gray_scale, k;
  // storage of: gray, Ix, Iy, Ixx, Iyy, Ixy, Sxx, Syy, Sxy (the response uses out.dtype)
  int st[9];
  // 3 x-taps then 3 y-taps of: Ix, Iy, Sxx, Syy, Sxy
  float w[5][6];
  int tile_w, tile_h, tiles_x, tiles_y, threads, seg;
  int batch;                // images stacked in the buffers (in: 3 planes each, out: 1)
  int* err;
};

// Downsample of every channel of a source level (binomial per axis at 2x, 2y);
// with remap = 1 the source is the local-Laplacian remap stack of the gray of
// an RGB input, computed on the fly.
struct LLDownArgs {
  ImgView src, out;
  int C;                       // channels produced
  int remap;
  float gray_scale, sigma, alpha, beta;
  int K;
  int st_gray, st_remap, st_out;
  int tile_w, tile_h, tiles_x, tiles_y;
};

// One level of the local-Laplacian output pyramid and its collapse step
// (see k_ll.cu).
struct LLLevelArgs {
  ImgView G, Gn, Rn, out, in;
  int rn_ch, rn_st;            // channel of Rn read by the upsample; storage it is rounded to
  int level0;
  float gray_scale, sigma, alpha, beta, s_in, s_out;
  int K;
  int st_gray, st_G, st_U, st_L, st_Lout, st_UR, st_R;
  int W, H;
};

struct HistArgs {
  ImgView in;               // 1 ch u8
  unsigned int* hist;       // 256 counters
  int blocks;
};

struct LutArgs {
  const unsigned int* hist;
  unsigned char* lut;       // 256 entries
  ImgView lut_view;         // where the LUT stage is materialised (256x1 u8)
};

struct LutApplyArgs {
  ImgView in, out;          // u8, 1 ch
  const unsigned char* lut;
};

// Launchers (defined in the .cu files).  Return a cudaError_t as int.
int launch_chain(const ChainArgs& a, int smem_bytes, void* stream);
// streaming stencil chain (2 or 4 stages in registers): one warp per strip of one plane
bool chain_rows_depth_ok(int depth);
int chain_rows_strip_w(int depth, int in_dtype, int cols = 4);
int chain_rows_cols(int depth, int in_dtype, int tile_w);
int chain_rows_smem_bytes(int depth, int cols, int threads, int in_dtype);
int chain_rows_grid(const ChainArgs& a, int cols, int units, int threads, int smem_bytes);
int launch_chain_rows(const ChainArgs& a, int cols, int rows, int grid, int smem_bytes, void* stream);
int chain_smem_bytes(int depth, int tile_w, int tile_h, int in_dtype);
// line-buffer stencil chain (an even number of stages <= kLinesMaxDepth, one
// thread block per tile, every stage on its own threads, rows through rings)
constexpr int kLinesMaxDepth = 8;
constexpr int kLinesMaxThreads = 256;
bool chain_lines_ok(int depth, int tile_w, int tile_h, int dtype);
int chain_lines_threads(int depth, int tile_w, int tile_h, int dtype);
int chain_lines_smem_bytes(int depth, int tile_w, int tile_h, int dtype);
int launch_chain_lines(const ChainArgs& a, void* stream);
int launch_generic(const GPlan& g, int threads, int smem_bytes, void* stream);
int launch_pointwise(const PointwiseArgs& a, void* stream);
int launch_downsample(const ResampleArgs& a, void* stream);
int launch_upsample(const ResampleArgs& a, void* stream);
int launch_harris(const HarrisArgs& a, int smem_bytes, void* stream);
int harris_smem_bytes(int tile_w, int tile_h, int in_dtype);
// streaming Harris: one warp per strip of harris_rows_strip_w columns, a.tile_h rows per run
int harris_rows_strip_w(int in_dtype);
int harris_rows_smem_bytes(int threads, int in_dtype);
int harris_rows_grid(const HarrisArgs& a, int units, int threads, int smem_bytes);
int launch_harris_rows(const HarrisArgs& a, int rows, int grid, int smem_bytes, void* stream);
// streaming single 5x5 stencil (+ unsharp combine): one warp per strip of one plane
int stencil_rows_strip_w(int in_dtype);
int stencil_rows_smem_bytes(int threads, int in_dtype);
int stencil_rows_grid(const ChainArgs& a, int units, int threads, int smem_bytes);
int launch_stencil_rows(const ChainArgs& a, int rows, int grid, int smem_bytes, void* stream);
// histogram equalization in one cooperative kernel; `state` is histeq_state_bytes() of zeroed device memory
size_t histeq_state_bytes();
int histeq_grid(int w, int h, int batch);
int launch_histeq(const ImgView& in, const ImgView& out, void* state, int* err, int grid, int batch, void* stream);
int launch_ll_down(const LLDownArgs& a, int smem_bytes, void* stream);
int ll_down_smem_bytes(int tile_w, int tile_h, int channels, int remap);
int launch_ll_level(const LLLevelArgs& a, void* stream);
int ll_remap_rows_strip_w();
int ll_remap_rows_ok(const LLDownArgs& a, int in_dtype);
int ll_remap_rows_grid(int in_dtype, int units, int threads);
int launch_ll_remap_rows(const LLDownArgs& a, int rows, int threads, int grid, void* stream);
int ll_down_rows_ok(const LLDownArgs& a, int src_dtype);
int ll_down_rows_groups(int C);
int ll_down_rows_grid(int C, int units, int threads);
int launch_ll_down_rows(const LLDownArgs& a, int rows, int threads, int grid, void* stream);
int ll_level_rows_strip_w();
int ll_level_rows_ok(const LLLevelArgs& a);
int ll_level_rows_grid(const LLLevelArgs& a, int units, int threads);
int launch_ll_level_rows(const LLLevelArgs& a, int rows, int threads, int grid, void* stream);
int max_rows_strip_w();
int max_rows_grid(const MaxArgs& a, int units, int threads);
// dynamic shared memory of the max filter kernel (the per-warp TMA rings; 0 when it loads from global memory)
int max_rows_smem_bytes(const MaxArgs& a, int threads);
int launch_max_rows(const MaxArgs& a, int grid, void* stream);
int interp_rows_strip_w();
int interp_rows_grid(const InterpArgs& a, int units, int threads);
// dynamic shared memory of the interpolate level kernel (the per-warp TMA rings of the fine level)
int interp_rows_smem_bytes(int threads);
int launch_interp_rows(const InterpArgs& a, int grid, void* stream);
int pw_rows_op_ok(int op);
int launch_pw_rows(const PwArgs& p, void* stream);
int grid_max_levels();
int launch_grid_splat(const GridArgs& a, void* stream);
int launch_grid_slice(const GridArgs& a, void* stream);
int grid_blur_units(const GridBlurArgs& a);
int launch_grid_blur(const GridBlurArgs& a, int grid, void* stream);
int launch_hist(const HistArgs& a, void* stream);
int launch_cdf_lut(const LutArgs& a, void* stream);
int launch_lut_apply(const LutApplyArgs& a, void* stream);
const char* cuda_error_string(int e);
// Raises a kernel's dynamic shared-memory limit to the device's opt-in maximum
// minus the kernel's static shared memory.  Returns a cudaError_t as int.
int allow_max_dynamic_smem(const void* func);

extern unsigned long long g_launches;

// Programmatic dependent launch: when t_overlap is set (by the realize of a
// pipeline with HP_OPT_OVERLAP on, for its own thread), kernels are launched
// so that the next one's blocks may be scheduled while the previous kernel's
// last blocks finish.  Every such kernel first waits for its predecessor grid
// to complete and its memory to be visible (grid_dep_sync), before any global
// memory access, so the order of reads and writes is that of plain launches.
extern thread_local int t_overlap;

// Register and local-memory (spill) figures of the kernels a realize
// launches, gathered when the pipeline's HP_OPT_PROBE_ATTRS is on (for the
// tuner's pruning): t_probe points at the realizing pipeline's record.
struct KernelProbe {
  int kernels;
  int max_regs;
  long long max_local;
};
extern thread_local KernelProbe* t_probe;
void probe_kernel(const void* func);

template <typename... KArgs, typename... Args>
inline int launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, void* stream, Args... args) {
  if (t_probe) probe_kernel((const void*)kern);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = t_overlap ? 1 : 0;
  return (int)cudaLaunchKernelEx(&cfg, kern, args...);
}

// Sets the thread's hp_last_error() message and returns s.
hp_status report_error(hp_status s, const char* msg);

}  // namespace hp
