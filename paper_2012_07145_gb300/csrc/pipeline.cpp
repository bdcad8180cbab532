// Pipeline IR, schedule validation, halo bounds inference, lowering of fusion
// groups onto kernels, scratch management and the C ABI of include/hp.h.
//
// The algorithm (stages and their footprints) is fixed independently of the
// schedule (Sec. 1).  A schedule assigns every stage a compute location: its
// own kernel ("root"), a fusion group computed per output tile in shared memory
// and registers, or inline (Sec. 2 "Fusion Options", Sec. 4 decision 1), plus
// the tile and thread shape of each group (Sec. 2 "Tiling", Sec. 4.1-4.3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "hp_internal.h"

namespace hp {

unsigned long long g_launches = 0;
thread_local int t_overlap = 0;
thread_local KernelProbe* t_probe = nullptr;

void probe_kernel(const void* func) {
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, func) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  ++t_probe->kernels;
  if (at.numRegs > t_probe->max_regs) t_probe->max_regs = at.numRegs;
  if ((long long)at.localSizeBytes > t_probe->max_local) t_probe->max_local = (long long)at.localSizeBytes;
}

namespace {

thread_local std::string t_err;

hp_status fail(hp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

hp_status cuda_fail(int e, const char* what) {
  return fail(HP_ERR_CUDA, "%s: %s", what, cuda_error_string(e));
}

int dtype_bytes(int d) {
  switch (d) {
    case HP_U8: return 1;
    case HP_U16: case HP_F16: case HP_BF16: return 2;
    default: return 4;
  }
}

bool valid_dtype(int d) { return d >= HP_U8 && d <= HP_U32; }

long long round16(long long v) { return (v + 15) / 16 * 16; }


struct Stage {
  int kind = 0, op = 0, channels = 1, storage = HP_F32;
  std::vector<int> inputs;
  int rx = 0, ry = 0;
  std::vector<float> wx, wy, params;
};

struct Dom {
  int w = 0, h = 0;
};

// Roles of a local-Laplacian level group (see k_ll.cu).
struct LLRoles {
  int U, L, Lout, UR, R, colour;   // stage ids (colour -1 above level 0)
  int Gl, Gn, Rn;                  // refs: the level stack, the next coarser stack, the coarser result
  int gray, remap, select;         // inlined producers (-1 if absent)
};

// One fusion group after lowering for a given set of input sizes.
struct GroupPlan {
  int kernel = HP_KERNEL_GENERIC;
  int output = -1;
  std::vector<int> members;  // stage ids (inlined copies included), ascending
  int tile_w = 0, tile_h = 0, threads = 0, seg = 0;
  int grid_x = 1, grid_y = 1, grid_z = 1;
  int smem = 0;
  // kernel-specific
  ChainArgs chain{};
  HarrisArgs harris{};
  LLDownArgs lldown{};
  LLLevelArgs lllevel{};
  MaxArgs maxa{};
  InterpArgs interp{};
  PwArgs pw{};
  GridArgs grid{};
  GridBlurArgs gblur{};
  LLRoles llroles{};
  std::unique_ptr<GPlan> gplan;
  std::vector<int> ext_refs;  // generic: external refs (stage id or -1-k)
  size_t aux_bytes = 0;       // kernel state kept across launches (zeroed once at allocation)
  void* aux = nullptr;
};

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// A captured launch sequence for one set of buffer addresses.
struct GraphEntry {
  std::vector<long long> key;    // data pointers and strides of the inputs and the output
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;
  unsigned long long last_use = 0;
};

struct Plan {
  std::vector<Dom> dom;          // per stage
  std::vector<Dom> in_dom;       // per input
  std::vector<GroupPlan> groups; // in execution order
  std::map<int, Scratch> bufs;   // exported stage -> device buffer
  std::vector<Scratch> staging;  // hp_realize_host device copies (inputs..., output)
  std::vector<Scratch> staging_async[2];  // hp_realize_host_async's two alternating sets
  std::vector<GraphEntry> graphs;
  std::vector<std::vector<long long>> seen;  // keys realized once without a graph
  bool allocated = false;
};

constexpr size_t kMaxGraphs = 16;

}  // namespace

// Records a failure message for hp_last_error() from other translation units.
hp_status report_error(hp_status s, const char* msg) { return fail(s, "%s", msg); }

}  // namespace hp

struct hp_pipeline {
  std::vector<int> in_dtypes, in_channels;
  std::vector<hp::Stage> stages;
  int output = -1;
  bool has_schedule = false;
  std::vector<int> group_of;              // per stage
  int n_groups = 0;
  std::vector<int> tile_w, tile_h, threads, serial_y, impl;
  std::map<std::vector<int>, std::unique_ptr<hp::Plan>> plans;
  int* d_err = nullptr;
  bool use_graph = false;
  bool overlap = true;   // programmatic dependent launch between the realize's kernels
  int batch = 1;         // images per realize (a server's batched copy; see clone_pipeline)
  unsigned long long graph_replays = 0;  // realizes served by an instantiated graph
  bool probe = false;    // gather the launched kernels' register / local-memory figures
  hp::KernelProbe probed{0, 0, 0};
  cudaStream_t capture_stream = nullptr;
  unsigned long long uses = 0;
  // hp_realize_host_async: its copy-in and copy-out streams, and per staging
  // set the events "inputs copied", "realized" and "output copied back"
  cudaStream_t host_in = nullptr, host_out = nullptr;
  cudaEvent_t ev_in[2] = {}, ev_done[2] = {}, ev_free[2] = {};
  unsigned long long async_calls = 0;
};

namespace hp {
namespace {

int stage_channels_of_ref(const hp_pipeline* p, int ref) {
  return ref < 0 ? p->in_channels[-1 - ref] : p->stages[ref].channels;
}

int stage_dtype_of_ref(const hp_pipeline* p, int ref) {
  return ref < 0 ? p->in_dtypes[-1 - ref] : p->stages[ref].storage;
}

// Range levels of a bilateral grid with range cell r: floor(1/r + 1/2) + 1.
int grid_levels(float r) { return (int)floor(1.0 / (double)r + 0.5) + 1; }

hp_status validate_stage(const hp_pipeline* p, const hp_stage_desc* d) {
  int nst = (int)p->stages.size();
  if (d->n_inputs < 1 || d->n_inputs > HP_MAX_INPUTS || !d->inputs)
    return fail(HP_ERR_INVALID_ARG, "stage needs 1..%d inputs", HP_MAX_INPUTS);
  for (int i = 0; i < d->n_inputs; ++i) {
    int r = d->inputs[i];
    if (r >= nst || (r < 0 && -1 - r >= (int)p->in_dtypes.size()))
      return fail(HP_ERR_INVALID_ARG, "input %d refers to unknown stage/input %d", i, r);
  }
  if (!valid_dtype(d->storage)) return fail(HP_ERR_INVALID_ARG, "bad storage dtype %d", d->storage);
  if (d->boundary != 0) return fail(HP_ERR_UNSUPPORTED, "only clamp-to-edge boundaries are supported");
  if (d->n_params < 0 || d->n_params > HP_MAX_PARAMS || (d->n_params > 0 && !d->params))
    return fail(HP_ERR_INVALID_ARG, "bad params");
  int c0 = stage_channels_of_ref(p, d->inputs[0]);
  auto need = [&](int n, int ch) -> hp_status {
    if (d->n_inputs != n) return fail(HP_ERR_INVALID_ARG, "kind %d op %d takes %d inputs", d->kind, d->op, n);
    if (d->channels != ch)
      return fail(HP_ERR_INVALID_ARG, "kind %d op %d produces %d channels, desc says %d", d->kind, d->op, ch,
                  d->channels);
    return HP_OK;
  };
  hp_status s;
  switch (d->kind) {
    case HP_STENCIL:
      if ((s = need(1, c0))) return s;
      if (d->rx < 0 || d->ry < 0 || d->rx > HP_MAX_RADIUS || d->ry > HP_MAX_RADIUS || !d->wx || !d->wy)
        return fail(HP_ERR_INVALID_ARG, "stencil radii must be in [0,%d] with taps", HP_MAX_RADIUS);
      if (d->storage == HP_U32) return fail(HP_ERR_UNSUPPORTED, "u32 storage is for histograms only");
      return HP_OK;
    case HP_MAX_STENCIL:
      if ((s = need(1, c0))) return s;
      if (d->rx < 0 || d->ry < 0 || d->rx > HP_MAX_RADIUS || d->ry > HP_MAX_RADIUS)
        return fail(HP_ERR_INVALID_ARG, "max-stencil radii must be in [0,%d]", HP_MAX_RADIUS);
      if (d->storage == HP_U32) return fail(HP_ERR_UNSUPPORTED, "u32 storage is for histograms only");
      return HP_OK;
    case HP_GRID_SPLAT: {
      if (d->n_params < 2 || !(d->params[0] >= 1.0f && d->params[0] <= 64.0f) || (float)(int)d->params[0] != d->params[0] ||
          !(d->params[1] >= 1.0f / 30.0f && d->params[1] <= 1.0f))
        return fail(HP_ERR_INVALID_ARG, "grid splat params: s an integer in [1, 64], r in [1/30, 1]");
      const int gz = grid_levels(d->params[1]);
      if ((s = need(1, 2 * gz))) return s;
      if (c0 != 1) return fail(HP_ERR_INVALID_ARG, "grid splat input is 1-channel");
      if (d->storage != HP_F32) return fail(HP_ERR_UNSUPPORTED, "the grid is stored as f32");
      return HP_OK;
    }
    case HP_GRID_SLICE: {
      if ((s = need(2, 1))) return s;
      if (d->n_params < 2 || !(d->params[0] >= 1.0f) || !(d->params[1] > 0.0f))
        return fail(HP_ERR_INVALID_ARG, "grid slice params: s >= 1, r > 0");
      const int gz = grid_levels(d->params[1]);
      if (c0 != 2 * gz || stage_channels_of_ref(p, d->inputs[1]) != 1)
        return fail(HP_ERR_INVALID_ARG, "grid slice inputs: a 2 GZ-channel grid and a 1-channel image");
      if (d->storage != HP_F32) return fail(HP_ERR_UNSUPPORTED, "the slice is stored as f32");
      return HP_OK;
    }
    case HP_DOWNSAMPLE2:
      if (d->storage == HP_U32) return fail(HP_ERR_UNSUPPORTED, "u32 storage is for histograms only");
      return need(1, c0);
    case HP_UPSAMPLE2:
      if (d->storage == HP_U32) return fail(HP_ERR_UNSUPPORTED, "u32 storage is for histograms only");
      return need(2, c0);
    case HP_HISTOGRAM:
      if ((s = need(1, 1))) return s;
      if (c0 != 1 || stage_dtype_of_ref(p, d->inputs[0]) != HP_U8)
        return fail(HP_ERR_INVALID_ARG, "histogram input must be a 1-channel u8 image");
      if (d->storage != HP_U32) return fail(HP_ERR_INVALID_ARG, "histogram storage must be u32");
      return HP_OK;
    case HP_CDF_LUT:
      if ((s = need(1, 1))) return s;
      if (d->inputs[0] < 0 || p->stages[d->inputs[0]].kind != HP_HISTOGRAM)
        return fail(HP_ERR_INVALID_ARG, "cdf_lut input must be a histogram stage");
      if (d->storage != HP_U8) return fail(HP_ERR_INVALID_ARG, "lut storage must be u8");
      return HP_OK;
    case HP_LUT_APPLY:
      if ((s = need(2, 1))) return s;
      if (c0 != 1 || stage_dtype_of_ref(p, d->inputs[0]) != HP_U8)
        return fail(HP_ERR_INVALID_ARG, "lut_apply image must be a 1-channel u8 image");
      if (d->inputs[1] < 0 || p->stages[d->inputs[1]].kind != HP_CDF_LUT)
        return fail(HP_ERR_INVALID_ARG, "lut_apply second input must be a cdf_lut stage");
      if (d->storage != HP_U8) return fail(HP_ERR_INVALID_ARG, "lut_apply storage must be u8");
      return HP_OK;
    case HP_POINTWISE:
      break;
    default:
      return fail(HP_ERR_UNSUPPORTED, "unknown stage kind %d", d->kind);
  }
  if (d->storage == HP_U32) return fail(HP_ERR_UNSUPPORTED, "u32 storage is for histograms only");
  auto chan = [&](int i) { return stage_channels_of_ref(p, d->inputs[i]); };
  auto nparams = [&](int n) -> hp_status {
    if (d->n_params < n) return fail(HP_ERR_INVALID_ARG, "op %d needs %d params", d->op, n);
    return HP_OK;
  };
  switch (d->op) {
    case HP_OP_GRAY:
      if ((s = need(1, 1)) || (s = nparams(1))) return s;
      if (c0 != 3) return fail(HP_ERR_INVALID_ARG, "gray needs a 3-channel input");
      return HP_OK;
    case HP_OP_MUL: case HP_OP_ADD: case HP_OP_SUB:
      if ((s = need(2, c0))) return s;
      if (chan(1) != c0) return fail(HP_ERR_INVALID_ARG, "binary op inputs differ in channels");
      return HP_OK;
    case HP_OP_HARRIS:
      if ((s = need(3, 1)) || (s = nparams(1))) return s;
      if (chan(0) != 1 || chan(1) != 1 || chan(2) != 1) return fail(HP_ERR_INVALID_ARG, "harris inputs are 1-channel");
      return HP_OK;
    case HP_OP_UNSHARP:
      if ((s = need(2, c0)) || (s = nparams(1))) return s;
      if (chan(1) != c0) return fail(HP_ERR_INVALID_ARG, "unsharp inputs differ in channels");
      return HP_OK;
    case HP_OP_LL_REMAP: {
      if ((s = nparams(4))) return s;
      int K = (int)d->params[3];
      if (K < 2 || K > 16 || (float)K != d->params[3]) return fail(HP_ERR_INVALID_ARG, "remap K must be 2..16");
      if ((s = need(1, K + 1))) return s;
      if (c0 != 1) return fail(HP_ERR_INVALID_ARG, "remap input is 1-channel");
      if (!(d->params[0] > 0.0f)) return fail(HP_ERR_INVALID_ARG, "sigma_r must be > 0");
      return HP_OK;
    }
    case HP_OP_LL_INTERP: {
      if ((s = need(2, 1)) || (s = nparams(1))) return s;
      int K = (int)d->params[0];
      if (K < 2 || chan(0) < K + 1 || chan(1) < K)
        return fail(HP_ERR_INVALID_ARG, "interp needs a K+1-channel G stack and a K-channel L stack");
      return HP_OK;
    }
    case HP_OP_PREMUL:
      if ((s = need(1, 4))) return s;
      if (c0 != 4) return fail(HP_ERR_INVALID_ARG, "premultiply needs a 4-channel (RGBA) input");
      return HP_OK;
    case HP_OP_OVER:
      if ((s = need(2, 4))) return s;
      if (chan(0) != 4 || chan(1) != 4) return fail(HP_ERR_INVALID_ARG, "over needs two 4-channel inputs");
      return HP_OK;
    case HP_OP_UNPREMUL:
      if ((s = need(1, 3))) return s;
      if (c0 != 4) return fail(HP_ERR_INVALID_ARG, "unpremultiply needs a 4-channel input");
      return HP_OK;
    case HP_OP_ZBLUR: {
      if ((s = nparams(1))) return s;
      const int gz = (int)d->params[0];
      if (gz < 1 || (float)gz != d->params[0] || c0 != 2 * gz) return fail(HP_ERR_INVALID_ARG, "zblur: params {GZ}, 2 GZ channels");
      return need(1, c0);
    }
    case HP_OP_LL_COLOUR:
      if ((s = need(3, 3)) || (s = nparams(2))) return s;
      if (chan(0) != 3 || chan(1) != 1 || chan(2) != 1) return fail(HP_ERR_INVALID_ARG, "colour inputs: 3, 1, 1 ch");
      return HP_OK;
    case HP_OP_SELECT: {
      if ((s = need(1, 1)) || (s = nparams(1))) return s;
      int c = (int)d->params[0];
      if (c < 0 || c >= c0) return fail(HP_ERR_INVALID_ARG, "select channel out of range");
      return HP_OK;
    }
    case HP_OP_SCALE:
      if ((s = need(1, c0)) || (s = nparams(2))) return s;
      return HP_OK;
    default:
      return fail(HP_ERR_UNSUPPORTED, "unknown point-wise op %d", d->op);
  }
}

// Domains of every stage for the given input sizes.
hp_status infer_domains(const hp_pipeline* p, const std::vector<Dom>& in_dom, std::vector<Dom>& dom) {
  dom.assign(p->stages.size(), Dom{});
  auto of = [&](int ref) { return ref < 0 ? in_dom[-1 - ref] : dom[ref]; };
  for (size_t s = 0; s < p->stages.size(); ++s) {
    const Stage& st = p->stages[s];
    Dom d0 = of(st.inputs[0]);
    switch (st.kind) {
      case HP_DOWNSAMPLE2: dom[s] = Dom{(d0.w + 1) / 2, (d0.h + 1) / 2}; break;
      case HP_UPSAMPLE2: {
        Dom r = of(st.inputs[1]);
        if ((r.w + 1) / 2 != d0.w || (r.h + 1) / 2 != d0.h)
          return fail(HP_ERR_INVALID_ARG, "stage %zu: upsample of %dx%d cannot produce %dx%d", s, d0.w, d0.h, r.w, r.h);
        dom[s] = r;
        break;
      }
      case HP_HISTOGRAM:
        // the bin counters (and the table's running sums) are 32-bit
        if ((unsigned long long)d0.w * (unsigned long long)d0.h > 4294967295ULL)
          return fail(HP_ERR_UNSUPPORTED, "stage %zu: a histogram counts at most 2^32 - 1 pixels (%dx%d given)", s, d0.w,
                      d0.h);
        dom[s] = Dom{256, 1};
        break;
      case HP_CDF_LUT: dom[s] = Dom{256, 1}; break;
      case HP_GRID_SPLAT: {
        const int gs = (int)st.params[0];
        dom[s] = Dom{(d0.w + gs - 1) / gs + 1, (d0.h + gs - 1) / gs + 1};
        break;
      }
      case HP_GRID_SLICE: {
        const int gs = (int)st.params[0];
        const Dom im = of(st.inputs[1]);
        if (d0.w != (im.w + gs - 1) / gs + 1 || d0.h != (im.h + gs - 1) / gs + 1)
          return fail(HP_ERR_INVALID_ARG, "stage %zu: a %dx%d grid does not fit a %dx%d image", s, d0.w, d0.h, im.w, im.h);
        dom[s] = im;
        break;
      }
      default: {
        dom[s] = d0;
        int first = st.kind == HP_LUT_APPLY ? 1 : (int)st.inputs.size();
        for (int i = 1; i < first; ++i) {
          Dom di = of(st.inputs[i]);
          if (di.w != d0.w || di.h != d0.h)
            return fail(HP_ERR_INVALID_ARG, "stage %zu: inputs differ in size (%dx%d vs %dx%d)", s, d0.w, d0.h, di.w, di.h);
        }
      }
    }
    if (dom[s].w < 1 || dom[s].h < 1) return fail(HP_ERR_INVALID_ARG, "stage %zu has an empty domain", s);
  }
  return HP_OK;
}

// Members of each group: assigned stages plus the inline closure.
struct GroupShape {
  std::vector<int> members;
  int output = -1;
};

hp_status group_shapes(const hp_pipeline* p, std::vector<GroupShape>& shapes) {
  int ns = (int)p->stages.size();
  int ng = p->n_groups;
  std::vector<std::vector<char>> in_group(ng, std::vector<char>(ns, 0));
  for (int s = 0; s < ns; ++s)
    if (p->group_of[s] >= 0) in_group[p->group_of[s]][s] = 1;
  // inline closure: walk producers of members through inlined stages
  for (int g = 0; g < ng; ++g) {
    for (int s = ns - 1; s >= 0; --s) {
      if (!in_group[g][s]) continue;
      for (int r : p->stages[s].inputs)
        if (r >= 0 && p->group_of[r] == HP_INLINE) in_group[g][r] = 1;
    }
  }
  // exported: stages read by a stage outside the group (or the output)
  shapes.assign(ng, GroupShape{});
  for (int g = 0; g < ng; ++g) {
    std::vector<int> exported;
    for (int s = 0; s < ns; ++s) {
      if (!in_group[g][s]) continue;
      shapes[g].members.push_back(s);
      if (p->group_of[s] != g) continue;  // inlined copies are never exported
      bool exp = s == p->output;
      for (int c = 0; c < ns && !exp; ++c) {
        bool reads = false;
        for (int r : p->stages[c].inputs) reads |= r == s;
        if (!reads) continue;
        if (p->group_of[c] >= 0 && p->group_of[c] != g) exp = true;
        if (p->group_of[c] == HP_INLINE) {
          for (int h = 0; h < ng; ++h)
            if (h != g && in_group[h][c]) exp = true;
        }
      }
      if (exp) exported.push_back(s);
    }
    if (shapes[g].members.empty()) return fail(HP_ERR_SCHEDULE, "group %d is empty", g);
    if (exported.size() != 1)
      return fail(HP_ERR_SCHEDULE, "group %d must have exactly one stage read outside it (has %zu)", g,
                  exported.size());
    int last_assigned = -1;
    for (int s : shapes[g].members)
      if (p->group_of[s] == g) last_assigned = s;
    if (exported[0] != last_assigned)
      return fail(HP_ERR_SCHEDULE, "group %d: its output stage %d must be its last member", g, exported[0]);
    shapes[g].output = exported[0];
    // inlined stages read after the output would be dead; nothing else to check
  }
  return HP_OK;
}

bool is_r2_stencil(const Stage& s) { return s.kind == HP_STENCIL && s.rx == 2 && s.ry == 2; }
bool is_r1_stencil(const Stage& s) { return s.kind == HP_STENCIL && s.rx == 1 && s.ry == 1; }

// Roles of a Harris-shaped group: gray, Ix, Iy, Pxx, Pyy, Pxy, Sxx, Syy, Sxy,
// response (stage ids), if the 10 members have exactly that structure.
bool match_harris(const hp_pipeline* p, const std::vector<int>& m, int roles[10]) {
  if (m.size() != 10) return false;
  auto st = [&](int i) -> const Stage& { return p->stages[m[i]]; };
  auto in_group = [&](int id) { return std::find(m.begin(), m.end(), id) != m.end(); };
  const Stage& g = st(0);
  if (!(g.kind == HP_POINTWISE && g.op == HP_OP_GRAY && !in_group(g.inputs[0]))) return false;
  roles[0] = m[0];
  int grads[2], ng = 0, prods[3], np = 0, sums[3], ns = 0, resp = -1;
  for (int i = 1; i < 10; ++i) {
    const Stage& s = st(i);
    if (is_r1_stencil(s) && s.inputs[0] == m[0] && ng < 2) grads[ng++] = m[i];
    else if (s.kind == HP_POINTWISE && s.op == HP_OP_MUL && np < 3) prods[np++] = m[i];
    else if (is_r1_stencil(s) && ns < 3) sums[ns++] = m[i];
    else if (s.kind == HP_POINTWISE && s.op == HP_OP_HARRIS) resp = m[i];
    else return false;
  }
  if (ng != 2 || np != 3 || ns != 3 || resp != m[9]) return false;
  roles[1] = grads[0];
  roles[2] = grads[1];
  auto is_prod = [&](int id, int a, int b) {
    const Stage& s = p->stages[id];
    return (s.inputs[0] == a && s.inputs[1] == b) || (s.inputs[0] == b && s.inputs[1] == a);
  };
  roles[3] = roles[4] = roles[5] = -1;
  for (int q : prods) {
    if (is_prod(q, grads[0], grads[0])) roles[3] = q;
    else if (is_prod(q, grads[1], grads[1])) roles[4] = q;
    else if (is_prod(q, grads[0], grads[1])) roles[5] = q;
  }
  if (roles[3] < 0 || roles[4] < 0 || roles[5] < 0) return false;
  for (int k = 0; k < 3; ++k) {
    roles[6 + k] = -1;
    for (int q : sums)
      if (p->stages[q].inputs[0] == roles[3 + k]) roles[6 + k] = q;
    if (roles[6 + k] < 0) return false;
  }
  const Stage& r = p->stages[resp];
  if (r.inputs[0] != roles[6] || r.inputs[1] != roles[7] || r.inputs[2] != roles[8]) return false;
  roles[9] = resp;
  return true;
}

// Downsample group: a single HP_DOWNSAMPLE (source read from memory), or the
// first local-Laplacian level, gray -> LL remap -> downsample, with gray and
// the remap in the group (inlined) and the RGB input outside it.
bool match_down(const hp_pipeline* p, const std::vector<int>& m, int* remap, int* gray, int* rm) {
  const Stage& last = p->stages[m.back()];
  if (last.kind != HP_DOWNSAMPLE2) return false;
  if (m.size() == 1) {
    *remap = 0;
    return true;
  }
  if (m.size() != 3) return false;
  const Stage& g = p->stages[m[0]];
  const Stage& r = p->stages[m[1]];
  if (!(g.kind == HP_POINTWISE && g.op == HP_OP_GRAY && g.inputs[0] < 0)) return false;
  if (!(r.kind == HP_POINTWISE && r.op == HP_OP_LL_REMAP && r.inputs[0] == m[0])) return false;
  if (last.inputs[0] != m[1]) return false;
  *remap = 1;
  *gray = m[0];
  *rm = m[1];
  return true;
}

bool match_ll_level(const hp_pipeline* p, const std::vector<int>& m, LLRoles& r) {
  auto in_m = [&](int id) { return id >= 0 && std::find(m.begin(), m.end(), id) != m.end(); };
  r = LLRoles{-1, -1, -1, -1, -1, -1, 0, 0, 0, -1, -1, -1};
  for (int id : m) {
    const Stage& s = p->stages[id];
    if (s.kind == HP_POINTWISE && s.op == HP_OP_LL_INTERP) {
      if (r.Lout >= 0) return false;
      r.Lout = id;
    }
  }
  if (r.Lout < 0) return false;
  const Stage& lo = p->stages[r.Lout];
  r.Gl = lo.inputs[0];
  r.L = lo.inputs[1];
  if (!in_m(r.L)) return false;
  const Stage& L = p->stages[r.L];
  if (!(L.kind == HP_POINTWISE && L.op == HP_OP_SUB && L.inputs[0] == r.Gl && in_m(L.inputs[1]))) return false;
  r.U = L.inputs[1];
  const Stage& U = p->stages[r.U];
  if (!(U.kind == HP_UPSAMPLE2 && U.inputs[1] == r.Gl && !in_m(U.inputs[0]))) return false;
  r.Gn = U.inputs[0];
  for (int id : m) {
    const Stage& s = p->stages[id];
    if (s.kind == HP_POINTWISE && s.op == HP_OP_ADD && s.inputs[0] == r.Lout) r.R = id;
  }
  if (r.R < 0) return false;
  r.UR = p->stages[r.R].inputs[1];
  if (!in_m(r.UR)) return false;
  const Stage& UR = p->stages[r.UR];
  if (!(UR.kind == HP_UPSAMPLE2 && UR.inputs[1] == r.Lout)) return false;
  r.Rn = UR.inputs[0];
  size_t expect = 5;
  if (in_m(r.Rn)) {
    const Stage& se = p->stages[r.Rn];
    if (!(se.kind == HP_POINTWISE && se.op == HP_OP_SELECT && !in_m(se.inputs[0]))) return false;
    r.select = r.Rn;
    ++expect;
  }
  if (in_m(r.Gl)) {  // level 0: the stack is the inlined remap of an inlined gray
    const Stage& rm = p->stages[r.Gl];
    if (!(rm.kind == HP_POINTWISE && rm.op == HP_OP_LL_REMAP && in_m(rm.inputs[0]))) return false;
    const Stage& g = p->stages[rm.inputs[0]];
    if (!(g.kind == HP_POINTWISE && g.op == HP_OP_GRAY && g.inputs[0] < 0)) return false;
    r.remap = r.Gl;
    r.gray = rm.inputs[0];
    for (int id : m) {
      const Stage& s = p->stages[id];
      if (s.kind == HP_POINTWISE && s.op == HP_OP_LL_COLOUR && s.inputs[1] == r.gray && s.inputs[2] == r.R &&
          s.inputs[0] == g.inputs[0])
        r.colour = id;
    }
    if (r.colour < 0) return false;
    expect += 3;
  } else if (in_m(r.Gn)) {
    return false;
  }
  if (m.size() != expect) return false;
  const int K = (int)lo.params[0];
  if (r.remap >= 0 && (int)p->stages[r.remap].params[3] != K) return false;
  if (r.select >= 0 && (int)p->stages[r.select].params[0] >= stage_channels_of_ref(p, p->stages[r.select].inputs[0]))
    return false;
  return m.back() == (r.colour >= 0 ? r.colour : r.R);
}

// Picks the kernel of a group from its shape.
int choose_kernel(const hp_pipeline* p, const GroupShape& gs, int impl) {
  const auto& m = gs.members;
  if (m.size() == 1) {
    const Stage& s = p->stages[m[0]];
    switch (s.kind) {
      case HP_STENCIL: return is_r2_stencil(s) && impl != HP_IMPL_GENERIC ? HP_KERNEL_STENCIL_CHAIN : HP_KERNEL_GENERIC;
      case HP_MAX_STENCIL: {  // square, horizontal or vertical window of radius 1..4
        const int r = s.rx > s.ry ? s.rx : s.ry;
        const bool shape_ok = s.rx == s.ry || s.rx == 0 || s.ry == 0;
        return shape_ok && r >= 1 && r <= 4 && impl != HP_IMPL_GENERIC ? HP_KERNEL_MAX_ROWS : HP_KERNEL_GENERIC;
      }
      case HP_POINTWISE: {  // f32 per-channel and RGBA ops: the vectorised point-wise kernel
        bool f32 = s.storage == HP_F32 && impl != HP_IMPL_GENERIC && pw_rows_op_ok(s.op);
        for (int r : s.inputs) f32 = f32 && stage_dtype_of_ref(p, r) == HP_F32;
        return f32 ? HP_KERNEL_PW_ROWS : HP_KERNEL_POINTWISE;
      }
      case HP_DOWNSAMPLE2: return impl == HP_IMPL_GENERIC ? HP_KERNEL_GENERIC : HP_KERNEL_DOWNSAMPLE;
      case HP_UPSAMPLE2: return HP_KERNEL_UPSAMPLE;
      case HP_HISTOGRAM: return HP_KERNEL_HISTOGRAM;
      case HP_GRID_SPLAT: return HP_KERNEL_GRID_SPLAT;
      case HP_GRID_SLICE: return HP_KERNEL_GRID_SLICE;
      case HP_CDF_LUT: return HP_KERNEL_CDF_LUT;
      case HP_LUT_APPLY: return HP_KERNEL_LUT_APPLY;
    }
  }
  if (m.size() == 3) {  // histogram -> table -> lookup of the same u8 image
    const Stage& h = p->stages[m[0]];
    const Stage& t = p->stages[m[1]];
    const Stage& l = p->stages[m[2]];
    if (h.kind == HP_HISTOGRAM && t.kind == HP_CDF_LUT && l.kind == HP_LUT_APPLY && t.inputs[0] == m[0] &&
        l.inputs[1] == m[1] && l.inputs[0] == h.inputs[0] && impl != HP_IMPL_GENERIC)
      return HP_KERNEL_HISTEQ;
  }
  for (int s : m) {
    int k = p->stages[s].kind;
    if (k == HP_HISTOGRAM || k == HP_CDF_LUT || k == HP_LUT_APPLY || k == HP_GRID_SPLAT || k == HP_GRID_SLICE) return -1;
  }
  if (impl == HP_IMPL_GENERIC) return HP_KERNEL_GENERIC;
  // bilateral grid blur: along the range levels, then x, then y (binomial/16)
  if (m.size() == 3) {
    const Stage& a = p->stages[m[0]];
    const Stage& b = p->stages[m[1]];
    const Stage& c = p->stages[m[2]];
    auto is_b16 = [](const std::vector<float>& w) {
      return w.size() == 5 && w[0] == 0.0625f && w[1] == 0.25f && w[2] == 0.375f && w[3] == 0.25f && w[4] == 0.0625f;
    };
    auto is_one = [](const std::vector<float>& w) { return w.size() == 1 && w[0] == 1.0f; };
    if (a.kind == HP_POINTWISE && a.op == HP_OP_ZBLUR && b.kind == HP_STENCIL && c.kind == HP_STENCIL &&
        b.inputs[0] == m[0] && c.inputs[0] == m[1] && b.rx == 2 && b.ry == 0 && c.rx == 0 && c.ry == 2 &&
        is_b16(b.wx) && is_one(b.wy) && is_one(c.wx) && is_b16(c.wy) && a.storage == HP_F32 && b.storage == HP_F32 &&
        c.storage == HP_F32 && stage_dtype_of_ref(p, a.inputs[0]) == HP_F32)
      return HP_KERNEL_GRID_BLUR;
  }
  // interpolate level: upsample of a coarse image, composite with the fine
  // level (and the division by coverage), every stage f32
  if (m.size() == 2 || m.size() == 3) {
    const Stage& u = p->stages[m[0]];
    const Stage& o = p->stages[m[1]];
    bool ok = u.kind == HP_UPSAMPLE2 && o.kind == HP_POINTWISE && o.op == HP_OP_OVER && o.inputs[1] == m[0] &&
              o.inputs[0] == u.inputs[1] && o.inputs[0] != m[0] && u.inputs[0] != m[1] && u.channels == 4 &&
              u.storage == HP_F32 && o.storage == HP_F32 && stage_dtype_of_ref(p, u.inputs[0]) == HP_F32 &&
              stage_dtype_of_ref(p, o.inputs[0]) == HP_F32 && stage_channels_of_ref(p, u.inputs[0]) == 4;
    if (ok && m.size() == 3) {
      const Stage& d = p->stages[m[2]];
      ok = d.kind == HP_POINTWISE && d.op == HP_OP_UNPREMUL && d.inputs[0] == m[1] && d.storage == HP_F32;
    }
    if (ok) return HP_KERNEL_INTERP_ROWS;
  }
  // a horizontal and a vertical window maximum of one radius (either order)
  if (m.size() == 2) {
    const Stage& a = p->stages[m[0]];
    const Stage& b = p->stages[m[1]];
    if (a.kind == HP_MAX_STENCIL && b.kind == HP_MAX_STENCIL && b.inputs[0] == m[0] && a.inputs[0] != m[1]) {
      const int r = a.rx + a.ry;
      if (r >= 1 && r <= 4 && a.rx * a.ry == 0 && b.rx * b.ry == 0 && b.rx + b.ry == r && a.rx != b.rx)
        return HP_KERNEL_MAX_ROWS;
    }
  }
  // linear chain of 5x5 stencils
  bool chain = (int)m.size() <= kChainMax;
  for (size_t i = 0; i < m.size() && chain; ++i) {
    const Stage& s = p->stages[m[i]];
    chain = is_r2_stencil(s) && (i == 0 ? (s.inputs[0] < 0 || std::find(m.begin(), m.end(), s.inputs[0]) == m.end())
                                       : s.inputs[0] == m[i - 1]);
  }
  if (chain) return HP_KERNEL_STENCIL_CHAIN;  // the builder picks the tiled or the streaming kernel
  {
    int remap, gray, rm;
    if (match_down(p, m, &remap, &gray, &rm)) return HP_KERNEL_DOWNSAMPLE;
    LLRoles llr;
    if (match_ll_level(p, m, llr)) return HP_KERNEL_LL_LEVEL;
  }
  int roles[10];
  if (match_harris(p, m, roles)) {
    int dt = stage_dtype_of_ref(p, p->stages[roles[0]].inputs[0]);
    if (dt == HP_F32 || dt == HP_F16 || dt == HP_BF16) return HP_KERNEL_HARRIS;
  }
  // 5x5 stencil + unsharp combine with the stencil's own input
  if (m.size() == 2) {
    const Stage& a = p->stages[m[0]];
    const Stage& b = p->stages[m[1]];
    if (is_r2_stencil(a) && b.kind == HP_POINTWISE && b.op == HP_OP_UNSHARP && b.inputs[1] == m[0] &&
        b.inputs[0] == a.inputs[0] && a.inputs[0] != m[0])
      return HP_KERNEL_UNSHARP;
  }
  return HP_KERNEL_GENERIC;
}

ImgView view_of(const hp_buffer& b) {
  ImgView v{};
  v.data = b.data;
  v.dtype = b.dtype;
  v.c = b.channels;
  v.w = b.width;
  v.h = b.height;
  v.rs = b.row_stride_bytes;
  v.ps = b.plane_stride_bytes;
  return v;
}

ImgView scratch_view(const Stage& s, Dom d, void* ptr) {
  ImgView v{};
  v.data = ptr;
  v.dtype = s.storage;
  v.c = s.channels;
  v.w = d.w;
  v.h = d.h;
  v.rs = round16((long long)d.w * dtype_bytes(s.storage));
  v.ps = round16(v.rs * d.h);
  return v;
}

size_t scratch_bytes(const Stage& s, Dom d) {
  ImgView v = scratch_view(s, d, nullptr);
  return (size_t)(v.ps * v.c);
}

// Domain of a reference: a stage's, or a pipeline input's (ref < 0).
Dom dom_of_ref(const Plan& plan, int ref) { return ref < 0 ? plan.in_dom[-1 - ref] : plan.dom[ref]; }

int pick(const std::vector<int>& v, int g, int dflt) {
  return g < (int)v.size() && v[g] > 0 ? v[g] : dflt;
}

// Default run length of the streaming kernels: about one run per resident warp
// over the image (strip_units = strips x planes), at least 8 rows so that the
// 4 warm-up rows of a run stay a modest overhead.
int default_run_rows(int h, int strip_units, long long resident_warps) {
  if (resident_warps < 1) resident_warps = 1;
  long long r = ((long long)h * strip_units + resident_warps - 1) / resident_warps;
  if (r < 8) r = 8;
  if (r > h) r = h < 8 ? 8 : h;
  return (int)r;
}

// Builds the generic plan (GPlan) of a group: nodes in member order, the
// output node last, external inputs listed once.
hp_status build_gplan(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  auto g = std::make_unique<GPlan>();
  memset(g.get(), 0, sizeof(GPlan));
  if ((int)gp.members.size() > kMaxGNodes) return fail(HP_ERR_SCHEDULE, "group has more than %d stages", kMaxGNodes);
  std::map<int, int> node_of;
  for (size_t i = 0; i < gp.members.size(); ++i) node_of[gp.members[i]] = (int)i;
  g->n_nodes = (int)gp.members.size();
  int wpos = 0, ppos = 0;
  for (size_t i = 0; i < gp.members.size(); ++i) {
    const Stage& s = p->stages[gp.members[i]];
    GNode& n = g->nodes[i];
    n.kind = s.kind; n.op = s.op; n.channels = s.channels; n.storage = s.storage;
    n.n_in = (int)s.inputs.size();
    for (int k = 0; k < n.n_in; ++k) {
      int r = s.inputs[k];
      auto it = node_of.find(r);
      if (r >= 0 && it != node_of.end()) {
        n.in[k] = it->second;
      } else {
        auto e = std::find(gp.ext_refs.begin(), gp.ext_refs.end(), r);
        int ei = (int)(e - gp.ext_refs.begin());
        if (e == gp.ext_refs.end()) {
          if ((int)gp.ext_refs.size() >= kMaxGExt) return fail(HP_ERR_SCHEDULE, "group reads more than %d buffers", kMaxGExt);
          gp.ext_refs.push_back(r);
        }
        n.in[k] = -1 - ei;
      }
    }
    n.rx = s.rx; n.ry = s.ry;
    n.w_off = wpos;
    if (s.kind == HP_STENCIL) {
      if (wpos + (int)s.wx.size() + (int)s.wy.size() > kMaxGWeights) return fail(HP_ERR_SCHEDULE, "too many taps");
      for (float w : s.wx) g->weights[wpos++] = w;
      for (float w : s.wy) g->weights[wpos++] = w;
    }
    n.p_off = ppos;
    n.n_params = (int)s.params.size();
    if (ppos + n.n_params > kMaxGParams) return fail(HP_ERR_SCHEDULE, "too many params");
    for (float v : s.params) g->params[ppos++] = v;
    n.dom_w = plan.dom[gp.members[i]].w;
    n.dom_h = plan.dom[gp.members[i]].h;
  }
  g->n_ext = (int)gp.ext_refs.size();
  g->tile_w = gp.tile_w;
  g->tile_h = gp.tile_h;
  Dom od = plan.dom[gp.output];
  g->tiles_x = (od.w + gp.tile_w - 1) / gp.tile_w;
  g->tiles_y = (od.h + gp.tile_h - 1) / gp.tile_h;
  // shared-memory bounds: the largest rect of each node over all tiles
  std::vector<int> maxw(g->n_nodes, 0), maxh(g->n_nodes, 0);
  std::vector<Rect> rects(g->n_nodes);
  for (int ty = 0; ty < g->tiles_y; ++ty)
    for (int tx = 0; tx < g->tiles_x; ++tx) {
      infer_rects(*g, tx * g->tile_w, ty * g->tile_h, rects.data());
      for (int n = 0; n < g->n_nodes; ++n) {
        if (rect_empty(rects[n])) continue;
        maxw[n] = std::max(maxw[n], rects[n].x1 - rects[n].x0);
        maxh[n] = std::max(maxh[n], rects[n].y1 - rects[n].y0);
      }
    }
  int off = 0;
  for (int n = 0; n + 1 < g->n_nodes; ++n) {
    GNode& nd = g->nodes[n];
    nd.pitch = maxw[n];
    nd.rows = maxh[n];
    nd.smem_off = off;
    off += nd.channels * nd.pitch * nd.rows;
  }
  g->smem_floats = off;
  gp.smem = off * 4;
  if (gp.smem > kSmemLimit)
    return fail(HP_ERR_SCHEDULE, "group needs %d bytes of shared memory (limit %d); use smaller tiles", gp.smem,
                kSmemLimit);
  gp.grid_x = g->tiles_x;
  gp.grid_y = g->tiles_y;
  gp.gplan = std::move(g);
  return HP_OK;
}

void chain_common_args(const hp_pipeline* p, GroupPlan& gp, bool unsharp) {
  ChainArgs& a = gp.chain;
  memset(&a, 0, sizeof a);
  std::vector<int> st = gp.members;
  if (unsharp) st.resize(1);
  a.depth = (int)st.size();
  for (int i = 0; i < a.depth; ++i) {
    const Stage& s = p->stages[st[i]];
    a.storage[i] = s.storage;
    for (int k = 0; k < 5; ++k) {
      a.w[i][k] = s.wx[k];
      a.w[i][5 + k] = s.wy[k];
    }
  }
  a.epilogue = unsharp ? 1 : 0;
  a.amount = unsharp ? p->stages[gp.members[1]].params[0] : 0.0f;
  a.tile_w = gp.tile_w;
  a.tile_h = gp.tile_h;
  a.threads = gp.threads;
  a.seg = gp.seg;
}

// A single 5x5 stencil (optionally with the unsharp combine) on the streaming
// kernel: strips of stencil_rows_strip_w columns, tile_h rows per run.
hp_status build_stencil_rows(const hp_pipeline* p, const Plan& plan, GroupPlan& gp, bool unsharp) {
  chain_common_args(p, gp, unsharp);
  ChainArgs& a = gp.chain;
  const int in_dt = stage_dtype_of_ref(p, p->stages[gp.members[0]].inputs[0]);
  const int sw = stencil_rows_strip_w(in_dt);
  if (a.tile_w != sw)
    return fail(HP_ERR_SCHEDULE, "streaming stencil strips are %d columns wide for this input type (tile_w %d)", sw,
                a.tile_w);
  if (a.threads % 32 != 0 || a.threads < 32 || a.threads > 256)
    return fail(HP_ERR_SCHEDULE, "streaming stencil threads per block must be a multiple of 32 in [32, 256]");
  Dom od = plan.dom[gp.output];
  const int planes = p->stages[gp.output].channels;
  a.tiles_x = (od.w + sw - 1) / sw;
  gp.smem = stencil_rows_smem_bytes(a.threads, in_dt);
  if (gp.smem > kSmemLimit) return fail(HP_ERR_SCHEDULE, "streaming stencil needs %d bytes of shared memory", gp.smem);
  a.in.dtype = in_dt;
  a.out.dtype = p->stages[gp.output].storage;
  if (a.tile_h == 0)
    gp.tile_h = a.tile_h = default_run_rows(od.h, a.tiles_x * planes,
                                            (long long)stencil_rows_grid(a, 1 << 30, a.threads, gp.smem) * (a.threads / 32));
  if (a.tile_h < 1 || a.tile_h > 65536) return fail(HP_ERR_SCHEDULE, "streaming stencil needs tile_h >= 1 rows per run");
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  gp.grid_x = stencil_rows_grid(a, a.tiles_x * a.tiles_y * planes, a.threads, gp.smem);
  gp.grid_y = 1;
  gp.grid_z = 1;
  return HP_OK;
}

hp_status build_chain(const hp_pipeline* p, const Plan& plan, GroupPlan& gp, bool unsharp) {
  chain_common_args(p, gp, unsharp);
  ChainArgs& a = gp.chain;
  std::vector<int> st = gp.members;
  if (unsharp) st.resize(1);
  if (a.tile_w % 8 != 0 || a.tile_w < 8 || a.tile_h < 1)
    return fail(HP_ERR_SCHEDULE, "stencil-chain tile width must be a positive multiple of 8");
  Dom od = plan.dom[gp.output];
  a.tiles_x = (od.w + a.tile_w - 1) / a.tile_w;
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  a.threads = gp.threads;
  a.seg = gp.seg;
  if (a.threads % 32 != 0 || a.threads < 32 || a.threads > 512)
    return fail(HP_ERR_SCHEDULE, "stencil-chain threads per block must be a multiple of 32 in [32, 512]");
  if (a.seg != 4 && a.seg != 8 && a.seg != 16)
    return fail(HP_ERR_SCHEDULE, "stencil-chain serial_y (rows per thread) must be 4, 8 or 16");
  int in_ref = p->stages[st[0]].inputs[0];
  int in_dtype = in_ref < 0 ? p->in_dtypes[-1 - in_ref] : p->stages[in_ref].storage;
  gp.smem = chain_smem_bytes(a.depth, a.tile_w, a.tile_h, in_dtype);
  if (gp.smem > kSmemLimit)
    return fail(HP_ERR_SCHEDULE, "stencil chain of depth %d with tile %dx%d needs %d bytes of shared memory", a.depth,
                a.tile_w, a.tile_h, gp.smem);
  gp.grid_x = a.tiles_x;
  gp.grid_y = a.tiles_y;
  gp.grid_z = p->stages[st[0]].channels;
  return HP_OK;
}

// Whether a chain group can take the line-buffer kernel: an even number of
// stages up to kLinesMaxDepth, the input, every stage and the output stored in
// one type (f32, f16 or bf16), and the group's tile within the kernel's limits.
bool chain_lines_group_ok(const hp_pipeline* p, const GroupPlan& gp) {
  const int in_dt = stage_dtype_of_ref(p, p->stages[gp.members[0]].inputs[0]);
  for (int m : gp.members)
    if (p->stages[m].storage != in_dt) return false;
  return chain_lines_ok((int)gp.members.size(), gp.tile_w, gp.tile_h, in_dt);
}

// A chain on the line-buffer kernel: one thread block per tile_w x tile_h
// output tile, every stage on its own threads (their count follows from the
// tile width and the depth; the schedule's threads and serial_y do not apply).
hp_status build_chain_lines(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  chain_common_args(p, gp, false);
  ChainArgs& a = gp.chain;
  const int in_dt = stage_dtype_of_ref(p, p->stages[gp.members[0]].inputs[0]);
  Dom od = plan.dom[gp.output];
  a.tiles_x = (od.w + a.tile_w - 1) / a.tile_w;
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  a.threads = chain_lines_threads(a.depth, a.tile_w, a.tile_h, in_dt);
  a.in.dtype = in_dt;
  a.out.dtype = p->stages[gp.output].storage;
  gp.threads = a.threads;
  gp.smem = chain_lines_smem_bytes(a.depth, a.tile_w, a.tile_h, in_dt);
  gp.grid_x = a.tiles_x;
  gp.grid_y = a.tiles_y;
  gp.grid_z = p->stages[gp.members[0]].channels;
  return HP_OK;
}

// A chain of 2 or 4 stencils on the streaming kernel: strips of
// chain_rows_strip_w columns, tile_h rows per run, every stage in registers.
hp_status build_chain_rows(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  chain_common_args(p, gp, false);
  ChainArgs& a = gp.chain;
  if (!chain_rows_depth_ok(a.depth))
    return fail(HP_ERR_SCHEDULE, "the streaming chain kernel fuses 2 or 4 stencils (group of %d)", a.depth);
  const int in_dt = stage_dtype_of_ref(p, p->stages[gp.members[0]].inputs[0]);
  const int cols = chain_rows_cols(a.depth, in_dt, a.tile_w);
  if (!cols)
    return fail(HP_ERR_SCHEDULE,
                "streaming chain strips of %d stages are %d (4 columns per lane) or %d (8) columns wide for this "
                "input type (tile_w %d)",
                a.depth, chain_rows_strip_w(a.depth, in_dt, 4), chain_rows_strip_w(a.depth, in_dt, 8), a.tile_w);
  const int sw = a.tile_w;
  a.cols = cols;
  if (a.threads % 32 != 0 || a.threads < 32 || a.threads > 256)
    return fail(HP_ERR_SCHEDULE, "streaming chain threads per block must be a multiple of 32 in [32, 256]");
  Dom od = plan.dom[gp.output];
  const int planes = p->stages[gp.output].channels;
  a.tiles_x = (od.w + sw - 1) / sw;
  gp.smem = chain_rows_smem_bytes(a.depth, cols, a.threads, in_dt);
  if (gp.smem > kSmemLimit) return fail(HP_ERR_SCHEDULE, "streaming chain needs %d bytes of shared memory", gp.smem);
  a.in.dtype = in_dt;
  a.out.dtype = p->stages[gp.output].storage;
  if (a.tile_h == 0)
    gp.tile_h = a.tile_h = default_run_rows(od.h, a.tiles_x * planes,
                                            (long long)chain_rows_grid(a, cols, 1 << 30, a.threads, gp.smem) * (a.threads / 32));
  if (a.tile_h < 1 || a.tile_h > 65536) return fail(HP_ERR_SCHEDULE, "streaming chain needs tile_h >= 1 rows per run");
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  gp.grid_x = chain_rows_grid(a, cols, a.tiles_x * a.tiles_y * planes, a.threads, gp.smem);
  gp.grid_y = 1;
  gp.grid_z = 1;
  return HP_OK;
}

void harris_common_args(const hp_pipeline* p, GroupPlan& gp, int roles[10]) {
  match_harris(p, gp.members, roles);
  HarrisArgs& a = gp.harris;
  memset(&a, 0, sizeof a);
  a.gray_scale = p->stages[roles[0]].params[0];
  a.k = p->stages[roles[9]].params[0];
  for (int i = 0; i < 9; ++i) a.st[i] = p->stages[roles[i]].storage;
  const int wst[5] = {roles[1], roles[2], roles[6], roles[7], roles[8]};
  for (int q = 0; q < 5; ++q)
    for (int k = 0; k < 3; ++k) {
      a.w[q][k] = p->stages[wst[q]].wx[k];
      a.w[q][3 + k] = p->stages[wst[q]].wy[k];
    }
  a.tile_w = gp.tile_w;
  a.tile_h = gp.tile_h;
  a.threads = gp.threads;
  a.seg = gp.seg;
  a.batch = p->batch;
}

hp_status build_harris(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  int roles[10];
  harris_common_args(p, gp, roles);
  HarrisArgs& a = gp.harris;
  if (a.tile_w % 8 != 0 || a.tile_w < 8 || a.tile_w > 232 || a.tile_h < 1 || a.tile_h > 252)
    return fail(HP_ERR_SCHEDULE, "Harris tile width must be a multiple of 8 in [8, 232], height in [1, 252]");
  if (a.threads % 32 != 0 || a.threads < 32 || a.threads > 512)
    return fail(HP_ERR_SCHEDULE, "Harris threads per block must be a multiple of 32 in [32, 512]");
  if (a.seg < 1) return fail(HP_ERR_SCHEDULE, "serial_y must be >= 1");
  Dom od = plan.dom[gp.output];
  a.tiles_x = (od.w + a.tile_w - 1) / a.tile_w;
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  gp.smem = harris_smem_bytes(a.tile_w, a.tile_h, stage_dtype_of_ref(p, p->stages[roles[0]].inputs[0]));
  if (gp.smem > kSmemLimit) return fail(HP_ERR_SCHEDULE, "Harris tile needs %d bytes of shared memory", gp.smem);
  gp.grid_x = a.tiles_x;
  gp.grid_y = a.tiles_y;
  gp.ext_refs.assign(1, p->stages[roles[0]].inputs[0]);
  return HP_OK;
}

hp_status build_harris_rows(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  int roles[10];
  harris_common_args(p, gp, roles);
  HarrisArgs& a = gp.harris;
  const int in_dt = stage_dtype_of_ref(p, p->stages[roles[0]].inputs[0]);
  const int sw = harris_rows_strip_w(in_dt);
  if (a.tile_w != sw)
    return fail(HP_ERR_SCHEDULE, "streaming Harris strips are %d columns wide for this input type (tile_w %d)", sw,
                a.tile_w);
  if (a.threads % 32 != 0 || a.threads < 32 || a.threads > 256)
    return fail(HP_ERR_SCHEDULE, "streaming Harris threads per block must be a multiple of 32 in [32, 256]");
  Dom od = plan.dom[gp.output];
  a.tiles_x = (od.w + sw - 1) / sw;
  gp.smem = harris_rows_smem_bytes(a.threads, in_dt);
  if (gp.smem > kSmemLimit) return fail(HP_ERR_SCHEDULE, "streaming Harris needs %d bytes of shared memory", gp.smem);
  a.in.dtype = in_dt;
  a.out.dtype = p->stages[gp.output].storage;
  if (a.tile_h == 0)
    gp.tile_h = a.tile_h = default_run_rows(od.h, a.tiles_x * p->batch,
                                            (long long)harris_rows_grid(a, 1 << 30, a.threads, gp.smem) * (a.threads / 32));
  if (a.tile_h < 4 || a.tile_h > 65536) return fail(HP_ERR_SCHEDULE, "streaming Harris needs tile_h >= 4 rows per run");
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  gp.grid_x = harris_rows_grid(a, a.tiles_x * a.tiles_y * p->batch, a.threads, gp.smem);
  gp.grid_y = 1;
  gp.ext_refs.assign(1, p->stages[roles[0]].inputs[0]);
  return HP_OK;
}

// Arguments shared by the tiled and the streaming downsample kernels.
void down_common_args(const hp_pipeline* p, GroupPlan& gp) {
  int remap = 0, gray = -1, rm = -1;
  match_down(p, gp.members, &remap, &gray, &rm);
  LLDownArgs& a = gp.lldown;
  memset(&a, 0, sizeof a);
  const Stage& d = p->stages[gp.output];
  a.remap = remap;
  a.C = d.channels;
  a.st_out = d.storage;
  if (remap) {
    const Stage& g = p->stages[gray];
    const Stage& r = p->stages[rm];
    a.gray_scale = g.params[0];
    a.st_gray = g.storage;
    a.sigma = r.params[0];
    a.alpha = r.params[1];
    a.beta = r.params[2];
    a.K = (int)r.params[3];
    a.st_remap = r.storage;
    gp.ext_refs.assign(1, g.inputs[0]);
  } else {
    gp.ext_refs.assign(1, d.inputs[0]);
  }
}

hp_status build_down(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  down_common_args(p, gp);
  LLDownArgs& a = gp.lldown;
  a.tile_w = gp.tile_w;
  a.tile_h = gp.tile_h;
  if (a.tile_w < 1 || a.tile_h < 1 || a.tile_w > 64 || a.tile_h > 64 || (a.tile_w & (a.tile_w - 1)))
    return fail(HP_ERR_SCHEDULE, "downsample tile width must be a power of two and tiles at most 64x64");
  if (a.remap && a.K > 2 * HP_MAX_PARAMS) return fail(HP_ERR_UNSUPPORTED, "too many intensity levels");
  Dom od = plan.dom[gp.output];
  a.tiles_x = (od.w + a.tile_w - 1) / a.tile_w;
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  gp.threads = 256;
  gp.smem = ll_down_smem_bytes(a.tile_w, a.tile_h, a.C, a.remap);
  if (gp.smem > kSmemLimit)
    return fail(HP_ERR_SCHEDULE, "downsample of %d channels with tile %dx%d needs %d bytes of shared memory", a.C,
                a.tile_w, a.tile_h, gp.smem);
  gp.grid_x = a.tiles_x;
  gp.grid_y = a.tiles_y;
  return HP_OK;
}

// Streaming downsample (the first level of the remap pyramid, or a stack of
// f32 planes): strips of 30 coarse columns, tile_h coarse rows per run (0:
// about one run per resident warp; the plane kernel, light per row, down to
// one row so that small levels still spread over the SMs).
hp_status build_ll_rows(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  down_common_args(p, gp);
  LLDownArgs& a = gp.lldown;
  const bool remap = gp.kernel == HP_KERNEL_LL_REMAP_ROWS;
  const int src_dt = stage_dtype_of_ref(p, gp.ext_refs[0]);
  if (remap ? !ll_remap_rows_ok(a, src_dt) : !ll_down_rows_ok(a, src_dt))
    return fail(HP_ERR_SCHEDULE, remap ? "the streaming remap downsample needs K = 8, u16 or f32 input and 0 < sigma < 1/7"
                                       : "the streaming downsample needs f32 planes");
  if (gp.tile_w != ll_remap_rows_strip_w())
    return fail(HP_ERR_SCHEDULE, "streaming downsample strips are %d coarse columns wide (tile_w %d)",
                ll_remap_rows_strip_w(), gp.tile_w);
  if (gp.threads % 32 != 0 || gp.threads < 32 || gp.threads > 256)
    return fail(HP_ERR_SCHEDULE, "streaming downsample threads per block must be a multiple of 32 in [32, 256]");
  Dom od = plan.dom[gp.output];
  a.tile_w = gp.tile_w;
  a.tiles_x = (od.w + a.tile_w - 1) / a.tile_w;
  const int units_per_row = a.tiles_x * (remap ? 1 : ll_down_rows_groups(a.C));
  auto grid_for = [&](int units) {
    return remap ? ll_remap_rows_grid(src_dt, units, gp.threads) : ll_down_rows_grid(a.C, units, gp.threads);
  };
  if (gp.tile_h == 0) {
    const long long warps = (long long)grid_for(1 << 30) * (gp.threads / 32);
    gp.tile_h = remap ? default_run_rows(od.h, units_per_row, warps)
                      : (int)std::max(1LL, ((long long)od.h * units_per_row + warps - 1) / warps);
  }
  if (gp.tile_h < 1 || gp.tile_h > 65536) return fail(HP_ERR_SCHEDULE, "streaming downsample needs tile_h >= 1");
  a.tile_h = gp.tile_h;
  a.tiles_y = (od.h + a.tile_h - 1) / a.tile_h;
  gp.smem = 0;
  gp.grid_x = grid_for(units_per_row * a.tiles_y);
  gp.grid_y = 1;
  return HP_OK;
}

hp_status build_ll_level(const hp_pipeline* p, const Plan& plan, GroupPlan& gp) {
  LLRoles& r = gp.llroles;
  match_ll_level(p, gp.members, r);
  LLLevelArgs& a = gp.lllevel;
  memset(&a, 0, sizeof a);
  a.K = (int)p->stages[r.Lout].params[0];
  a.level0 = r.remap >= 0;
  a.st_U = p->stages[r.U].storage;
  a.st_L = p->stages[r.L].storage;
  a.st_Lout = p->stages[r.Lout].storage;
  a.st_UR = p->stages[r.UR].storage;
  a.st_R = p->stages[r.R].storage;
  a.rn_ch = 0;
  a.rn_st = HP_F32;
  if (r.select >= 0) {
    a.rn_ch = (int)p->stages[r.select].params[0];
    a.rn_st = p->stages[r.select].storage;
  }
  if (a.level0) {
    const Stage& g = p->stages[r.gray];
    const Stage& rm = p->stages[r.remap];
    const Stage& c = p->stages[r.colour];
    a.gray_scale = g.params[0];
    a.st_gray = g.storage;
    a.sigma = rm.params[0];
    a.alpha = rm.params[1];
    a.beta = rm.params[2];
    a.st_G = rm.storage;
    a.s_in = c.params[0];
    a.s_out = c.params[1];
  } else {
    a.st_G = stage_dtype_of_ref(p, r.Gl);
  }
  Dom d = plan.dom[r.Lout];
  a.W = d.w;
  a.H = d.h;
  gp.threads = 256;
  gp.grid_x = (d.w + 31) / 32;
  gp.grid_y = (d.h + 7) / 8;
  gp.smem = 0;
  return HP_OK;
}

// The level kernel's arguments with the element types and channel counts of
// its views filled in from the stages they come from (at realize the views
// carry the same).
LLLevelArgs ll_level_view_types(const hp_pipeline* p, const GroupPlan& gp) {
  LLLevelArgs a = gp.lllevel;
  const LLRoles& r = gp.llroles;
  auto set = [&](ImgView& v, int ref) {
    v.dtype = stage_dtype_of_ref(p, ref);
    v.c = stage_channels_of_ref(p, ref);
  };
  if (a.level0) {
    set(a.in, p->stages[r.gray].inputs[0]);
  } else {
    set(a.G, r.Gl);
  }
  set(a.Gn, r.Gn);
  set(a.Rn, r.select >= 0 ? p->stages[r.select].inputs[0] : r.Rn);
  a.out.dtype = p->stages[gp.output].storage;
  a.out.c = p->stages[gp.output].channels;
  return a;
}

// Streaming level kernel: strips of 30 coarse columns (60 fine), tile_h coarse
// rows per run (0: about one run per resident warp, at least 2).
hp_status build_ll_level_rows(const hp_pipeline* p, const Plan& plan, GroupPlan& gp, const LLLevelArgs& probe) {
  if (gp.tile_w != ll_level_rows_strip_w())
    return fail(HP_ERR_SCHEDULE, "streaming level strips are %d coarse columns wide (tile_w %d)", ll_level_rows_strip_w(),
                gp.tile_w);
  if (gp.threads % 32 != 0 || gp.threads < 32 || gp.threads > 256)
    return fail(HP_ERR_SCHEDULE, "streaming level threads per block must be a multiple of 32 in [32, 256]");
  const Dom cd = dom_of_ref(plan, gp.llroles.Gn);
  const int strips = (cd.w + gp.tile_w - 1) / gp.tile_w;
  if (gp.tile_h == 0) {
    const long long warps = (long long)ll_level_rows_grid(probe, 1 << 30, gp.threads) * (gp.threads / 32);
    gp.tile_h = (int)std::max(2LL, ((long long)cd.h * strips + warps - 1) / warps);
  }
  if (gp.tile_h < 1 || gp.tile_h > 65536) return fail(HP_ERR_SCHEDULE, "streaming level needs tile_h >= 1");
  gp.grid_x = ll_level_rows_grid(probe, strips * ((cd.h + gp.tile_h - 1) / gp.tile_h), gp.threads);
  gp.grid_y = 1;
  gp.smem = 0;
  return HP_OK;
}

hp_status lower(hp_pipeline* p, const std::vector<Dom>& in_dom, Plan& plan) {
  plan.in_dom = in_dom;
  hp_status s = infer_domains(p, in_dom, plan.dom);
  if (s) return s;
  std::vector<GroupShape> shapes;
  if ((s = group_shapes(p, shapes))) return s;
  std::vector<int> order(p->n_groups);
  for (int g = 0; g < p->n_groups; ++g) order[g] = g;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return shapes[a].output < shapes[b].output; });
  plan.groups.clear();
  plan.groups.resize(p->n_groups);
  for (int oi = 0; oi < p->n_groups; ++oi) {
    int g = order[oi];
    GroupPlan& gp = plan.groups[oi];
    gp.members = shapes[g].members;
    gp.output = shapes[g].output;
    int impl = g < (int)p->impl.size() ? p->impl[g] : HP_IMPL_AUTO;
    gp.kernel = choose_kernel(p, shapes[g], impl);
    if (gp.kernel < 0) return fail(HP_ERR_UNSUPPORTED, "group %d mixes reductions with other stages", g);
    switch (gp.kernel) {
      case HP_KERNEL_STENCIL_CHAIN:
      case HP_KERNEL_UNSHARP: {
        // one stencil (+ unsharp combine): the streaming kernel at its strip
        // width (the default) or under HP_IMPL_WAVE; else the tiled chain kernel
        // a chain of 2 or 4: the streaming chain kernel likewise at its strip width
        const bool unsharp = gp.kernel == HP_KERNEL_UNSHARP;
        const bool single = unsharp || gp.members.size() == 1;
        const int in_dt = stage_dtype_of_ref(p, p->stages[gp.members[0]].inputs[0]);
        const int depth = (int)gp.members.size();
        const int sw = single ? stencil_rows_strip_w(in_dt) : chain_rows_depth_ok(depth) ? chain_rows_strip_w(depth, in_dt) : -1;
        gp.tile_w = pick(p->tile_w, g, single ? sw : 64);
        const bool strip_w = single ? gp.tile_w == sw : chain_rows_depth_ok(depth) && chain_rows_cols(depth, in_dt, gp.tile_w);
        const bool streaming = impl == HP_IMPL_WAVE || (impl == HP_IMPL_AUTO && strip_w);
        gp.tile_h = pick(p->tile_h, g, streaming ? 0 : 32);  // 0: the streaming kernels' adaptive run length
        gp.threads = pick(p->threads, g, 256);
        gp.seg = pick(p->serial_y, g, 8);
        if (!single && impl == HP_IMPL_LINES && chain_lines_group_ok(p, gp)) {
          gp.kernel = HP_KERNEL_STENCIL_LINES;
          s = build_chain_lines(p, plan, gp);
        } else if (single && streaming) {
          gp.kernel = HP_KERNEL_STENCIL_ROWS;
          s = build_stencil_rows(p, plan, gp, unsharp);
        } else if (streaming) {
          gp.kernel = HP_KERNEL_STENCIL_WAVE;
          s = build_chain_rows(p, plan, gp);
        } else {
          s = build_chain(p, plan, gp, unsharp);
        }
        break;
      }
      case HP_KERNEL_DOWNSAMPLE: {
        // the first remap level: the streaming kernel at its strip width (the
        // default) or under HP_IMPL_WAVE, where it covers the group
        // the first remap level and f32 plane stacks: the streaming kernels at
        // their strip width (the default) or under HP_IMPL_WAVE
        {
          GroupPlan probe;
          probe.members = gp.members;
          probe.output = gp.output;
          down_common_args(p, probe);
          const int sw = ll_remap_rows_strip_w();
          const int src_dt = stage_dtype_of_ref(p, probe.ext_refs[0]);
          const bool remap_ok = ll_remap_rows_ok(probe.lldown, src_dt);
          if (remap_ok || ll_down_rows_ok(probe.lldown, src_dt)) {
            gp.tile_w = pick(p->tile_w, g, sw);
            if (impl == HP_IMPL_WAVE || (impl == HP_IMPL_AUTO && gp.tile_w == sw)) {
              gp.kernel = remap_ok ? HP_KERNEL_LL_REMAP_ROWS : HP_KERNEL_LL_DOWN_ROWS;
              gp.tile_w = sw;
              gp.tile_h = pick(p->tile_h, g, 0);
              gp.threads = pick(p->threads, g, 256);
              s = build_ll_rows(p, plan, gp);
              break;
            }
          }
        }
        // default: 16x16 coarse tiles, halved (down to 4x4) for small levels so
        // that the grid still covers the SMs
        Dom od = plan.dom[gp.output];
        int t = 16;
        while (t > 4 && ((od.w + t - 1) / t) * ((od.h + t / 2 - 1) / (t / 2)) < 512) t /= 2;
        gp.tile_w = std::min(pick(p->tile_w, g, t), 64);
        gp.tile_h = std::min(pick(p->tile_h, g, std::max(2, t / 2)), 64);
        const int c = p->stages[gp.output].channels;
        while (ll_down_smem_bytes(gp.tile_w, gp.tile_h, c, 1) > kSmemLimit && gp.tile_w > 4) {
          gp.tile_w /= 2;
          gp.tile_h = std::max(4, gp.tile_h / 2);
        }
      }
        s = build_down(p, plan, gp);
        break;
      case HP_KERNEL_LL_LEVEL: {
        s = build_ll_level(p, plan, gp);
        if (s) break;
        // the streaming kernel at its strip width (the default) or under
        // HP_IMPL_WAVE, where it covers the group
        const int sw = ll_level_rows_strip_w();
        LLLevelArgs probe = ll_level_view_types(p, gp);
        if (ll_level_rows_ok(probe)) {
          gp.tile_w = pick(p->tile_w, g, sw);
          if (impl == HP_IMPL_WAVE || (impl == HP_IMPL_AUTO && gp.tile_w == sw)) {
            gp.kernel = HP_KERNEL_LL_LEVEL_ROWS;
            gp.tile_w = sw;
            gp.tile_h = pick(p->tile_h, g, 0);
            gp.threads = pick(p->threads, g, 256);
            s = build_ll_level_rows(p, plan, gp, probe);
          }
        }
        break;
      }
      case HP_KERNEL_HARRIS: {
        int roles[10];
        match_harris(p, gp.members, roles);
        const int sw = harris_rows_strip_w(stage_dtype_of_ref(p, p->stages[roles[0]].inputs[0]));
        gp.tile_w = pick(p->tile_w, g, sw);
        gp.tile_h = pick(p->tile_h, g, 0);
        gp.threads = pick(p->threads, g, 256);
        gp.seg = pick(p->serial_y, g, 8);
        if (impl == HP_IMPL_WAVE || (impl == HP_IMPL_AUTO && gp.tile_w == sw)) {
          gp.kernel = HP_KERNEL_HARRIS_ROWS;
          s = build_harris_rows(p, plan, gp);
        } else {
          if (gp.tile_h == 0) gp.tile_h = 32;
          s = build_harris(p, plan, gp);
        }
        break;
      }
      case HP_KERNEL_MAX_ROWS: {
        const Stage& first = p->stages[gp.members[0]];
        const Stage& last = p->stages[gp.output];
        MaxArgs& a = gp.maxa;
        memset(&a, 0, sizeof a);
        if (gp.members.size() == 1) {
          a.radius = first.rx > first.ry ? first.rx : first.ry;
          a.shape = first.rx == first.ry ? 0 : first.ry == 0 ? 1 : 2;
        } else {
          a.radius = first.rx + first.ry;
          a.shape = 0;
        }
        a.st_mid = first.storage;
        a.st_out = last.storage;
        gp.ext_refs.assign(1, first.inputs[0]);
        gp.tile_w = max_rows_strip_w();
        gp.threads = pick(p->threads, g, 256);
        if (gp.threads % 32 != 0 || gp.threads < 32 || gp.threads > 256) {
          s = fail(HP_ERR_SCHEDULE, "streaming max filter threads per block must be a multiple of 32 in [32, 256]");
          break;
        }
        a.threads = gp.threads;
        Dom od = plan.dom[gp.output];
        const int planes = last.channels;
        const int strips = (od.w + gp.tile_w - 1) / gp.tile_w;
        gp.tile_h = pick(p->tile_h, g, 0);
        if (gp.tile_h == 0) {
          a.in.dtype = stage_dtype_of_ref(p, first.inputs[0]);
          gp.tile_h = default_run_rows(od.h, strips * planes,
                                       (long long)max_rows_grid(a, 1 << 30, gp.threads) * (gp.threads / 32));
        }
        a.rows = gp.tile_h;
        a.in.dtype = stage_dtype_of_ref(p, first.inputs[0]);
        gp.grid_x = max_rows_grid(a, strips * planes * ((od.h + a.rows - 1) / a.rows), gp.threads);
        gp.grid_y = 1;
        gp.smem = max_rows_smem_bytes(a, gp.threads);
        break;
      }
      case HP_KERNEL_GRID_BLUR: {
        const Stage& zb = p->stages[gp.members[0]];
        GridBlurArgs& a = gp.gblur;
        memset(&a, 0, sizeof a);
        a.gz = (int)zb.params[0];
        gp.ext_refs.assign(1, zb.inputs[0]);
        gp.threads = 256;
        const Dom gd = plan.dom[gp.output];
        a.in.w = gd.w;
        a.in.h = gd.h;
        a.rows = 1;
        const long long per_row = grid_blur_units(a) / gd.h;  // column units per grid row
        gp.tile_h = pick(p->tile_h, g, 0);
        if (gp.tile_h == 0) gp.tile_h = (int)std::max(1LL, ((long long)gd.h * per_row + 2431) / 2432);
        a.rows = gp.tile_h;
        const int units = grid_blur_units(a);
        gp.grid_x = std::max(1, std::min((units + 7) / 8, 2 * 152));
        gp.grid_y = 1;
        break;
      }
      case HP_KERNEL_GRID_SPLAT:
      case HP_KERNEL_GRID_SLICE: {
        const Stage& st = p->stages[gp.output];
        GridArgs& a = gp.grid;
        memset(&a, 0, sizeof a);
        a.s = (int)st.params[0];
        a.gz = grid_levels(st.params[1]);
        a.inv_s = (float)(1.0 / (double)a.s);
        a.inv_r = (float)(1.0 / (double)st.params[1]);
        if (a.gz > grid_max_levels()) {
          s = fail(HP_ERR_UNSUPPORTED, "at most %d range levels", grid_max_levels());
          break;
        }
        gp.ext_refs = st.inputs;
        gp.threads = 256;
        break;
      }
      case HP_KERNEL_PW_ROWS: {
        const Stage& st = p->stages[gp.output];
        PwArgs& a = gp.pw;
        memset(&a, 0, sizeof a);
        a.op = st.op;
        a.n_in = (int)st.inputs.size();
        a.p0 = st.params.size() > 0 ? st.params[0] : 0.0f;
        a.p1 = st.params.size() > 1 ? st.params[1] : 0.0f;
        gp.ext_refs = st.inputs;
        gp.threads = 256;
        break;
      }
      case HP_KERNEL_INTERP_ROWS: {
        const Stage& u = p->stages[gp.members[0]];
        const Stage& o = p->stages[gp.members[1]];
        InterpArgs& a = gp.interp;
        memset(&a, 0, sizeof a);
        a.final_div = gp.members.size() == 3;
        gp.ext_refs.assign({o.inputs[0], u.inputs[0]});  // the fine level, the coarse image
        gp.tile_w = interp_rows_strip_w();
        gp.threads = pick(p->threads, g, 256);
        if (gp.threads % 32 != 0 || gp.threads < 32 || gp.threads > 256) {
          s = fail(HP_ERR_SCHEDULE, "streaming interpolate threads per block must be a multiple of 32 in [32, 256]");
          break;
        }
        a.threads = gp.threads;
        const Dom cd = dom_of_ref(plan, u.inputs[0]);
        const int strips = (cd.w + gp.tile_w - 1) / gp.tile_w;
        gp.tile_h = pick(p->tile_h, g, 0);
        if (gp.tile_h == 0) {
          const long long warps = (long long)interp_rows_grid(a, 1 << 30, gp.threads) * (gp.threads / 32);
          gp.tile_h = (int)std::max(2LL, ((long long)cd.h * strips + warps - 1) / warps);
        }
        a.rows = gp.tile_h;
        gp.grid_x = interp_rows_grid(a, strips * ((cd.h + a.rows - 1) / a.rows), gp.threads);
        gp.grid_y = 1;
        gp.smem = interp_rows_smem_bytes(gp.threads);
        break;
      }
      case HP_KERNEL_HISTEQ: {
        Dom od = plan.dom[gp.output];
        gp.threads = 1024;
        gp.grid_x = histeq_grid(od.w, od.h, p->batch);
        gp.aux_bytes = histeq_state_bytes() * p->batch;
        gp.ext_refs.assign(1, p->stages[gp.members[0]].inputs[0]);
        break;
      }
      case HP_KERNEL_HISTOGRAM: case HP_KERNEL_CDF_LUT: case HP_KERNEL_LUT_APPLY:
        gp.threads = 256;
        break;
      default: {
        bool single = gp.members.size() == 1;
        gp.tile_w = pick(p->tile_w, g, single ? 64 : 32);
        gp.tile_h = pick(p->tile_h, g, single ? 16 : 32);
        gp.threads = pick(p->threads, g, 256);
        if (gp.threads % 32 != 0 || gp.threads > 1024)
          return fail(HP_ERR_SCHEDULE, "threads per block must be a multiple of 32 in [32, 1024]");
        s = build_gplan(p, plan, gp);
      }
    }
    if (s) return s;
    if (p->batch > 1 && gp.kernel != HP_KERNEL_HARRIS && gp.kernel != HP_KERNEL_HARRIS_ROWS &&
        gp.kernel != HP_KERNEL_HISTEQ)
      return fail(HP_ERR_UNSUPPORTED, "a batch of %d images needs every group on a batch-aware kernel "
                                      "(fused Harris or histogram equalization)", p->batch);
  }
  return HP_OK;
}

// First realize of a plan: its buffers.  Kernel state is cleared on the
// realize's own stream (a synchronous memset would wait for every stream).
hp_status ensure_scratch(hp_pipeline* p, Plan& plan, cudaStream_t stream) {
  if (plan.allocated) return HP_OK;
  for (GroupPlan& gp : plan.groups) {
    if (gp.aux_bytes && !gp.aux) {
      if (cudaMalloc(&gp.aux, gp.aux_bytes) != cudaSuccess ||
          cudaMemsetAsync(gp.aux, 0, gp.aux_bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        gp.aux = nullptr;
        return fail(HP_ERR_OOM, "cudaMalloc of %zu bytes of kernel state failed", gp.aux_bytes);
      }
    }
  }
  for (const GroupPlan& gp : plan.groups) {
    if (gp.output == p->output) continue;
    const Stage& st = p->stages[gp.output];
    Scratch sc;
    sc.bytes = scratch_bytes(st, plan.dom[gp.output]);
    int e = cudaMalloc(&sc.ptr, sc.bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(HP_ERR_OOM, "cudaMalloc of %zu bytes for stage %d failed", sc.bytes, gp.output);
    }
    plan.bufs[gp.output] = sc;
  }
  plan.allocated = true;
  return HP_OK;
}

ImgView ref_view(const hp_pipeline* p, const Plan& plan, int ref, const hp_buffer* inputs,
                 const hp_buffer* output) {
  if (ref < 0) return view_of(inputs[-1 - ref]);
  if (ref == p->output) return view_of(*output);
  auto it = plan.bufs.find(ref);
  return scratch_view(p->stages[ref], plan.dom[ref], it->second.ptr);
}

hp_status check_buffer(const hp_buffer& b, int dtype, int channels, Dom d, const char* what, int idx) {
  if (!b.data) return fail(HP_ERR_INVALID_ARG, "%s %d: null data", what, idx);
  if (b.dtype != dtype) return fail(HP_ERR_INVALID_ARG, "%s %d: dtype %d, expected %d", what, idx, b.dtype, dtype);
  if (b.channels != channels)
    return fail(HP_ERR_INVALID_ARG, "%s %d: %d channels, expected %d", what, idx, b.channels, channels);
  if (d.w > 0 && (b.width != d.w || b.height != d.h))
    return fail(HP_ERR_INVALID_ARG, "%s %d: size %dx%d, expected %dx%d", what, idx, b.width, b.height, d.w, d.h);
  if (b.width < 1 || b.height < 1) return fail(HP_ERR_INVALID_ARG, "%s %d: empty image", what, idx);
  if (((uintptr_t)b.data & 15) != 0) return fail(HP_ERR_INVALID_ARG, "%s %d: data not 16-byte aligned", what, idx);
  if (b.row_stride_bytes % 16 != 0 || b.plane_stride_bytes % 16 != 0)
    return fail(HP_ERR_INVALID_ARG, "%s %d: strides must be multiples of 16 bytes", what, idx);
  if (b.row_stride_bytes < (long long)b.width * dtype_bytes(dtype) ||
      (b.channels > 1 && b.plane_stride_bytes < b.row_stride_bytes * b.height))
    return fail(HP_ERR_INVALID_ARG, "%s %d: strides too small for the image", what, idx);
  return HP_OK;
}

hp_status get_plan(hp_pipeline* p, const std::vector<Dom>& in_dom, Plan** out) {
  if (p->output < 0) return fail(HP_ERR_STATE, "no output stage set");
  std::vector<int> key;
  for (Dom d : in_dom) { key.push_back(d.w); key.push_back(d.h); }
  auto it = p->plans.find(key);
  if (it != p->plans.end()) { *out = it->second.get(); return HP_OK; }
  auto plan = std::make_unique<Plan>();
  hp_status s = lower(p, in_dom, *plan);
  if (s) return s;
  *out = plan.get();
  p->plans[key] = std::move(plan);
  return HP_OK;
}

void free_plan(Plan& plan) {
  for (auto& g : plan.graphs) cudaGraphExecDestroy(g.exec);
  plan.graphs.clear();
  plan.seen.clear();
  for (auto& kv : plan.bufs) cudaFree(kv.second.ptr);
  for (auto& gp : plan.groups)
    if (gp.aux) {
      cudaFree(gp.aux);
      gp.aux = nullptr;
    }
  for (auto& sc : plan.staging) cudaFree(sc.ptr);
  for (auto& set : plan.staging_async)
    for (auto& sc : set) cudaFree(sc.ptr);
  plan.bufs.clear();
  plan.staging.clear();
  for (auto& set : plan.staging_async) set.clear();
}

void drop_plans(hp_pipeline* p) {
  if (p->host_out) cudaStreamSynchronize(p->host_out);  // no hp_realize_host_async work in flight
  for (auto& kv : p->plans) free_plan(*kv.second);
  p->plans.clear();
}

void default_schedule(hp_pipeline* p) {
  int ns = (int)p->stages.size();
  p->group_of.resize(ns);
  for (int s = 0; s < ns; ++s) p->group_of[s] = s;
  p->n_groups = ns;
  p->tile_w.clear(); p->tile_h.clear(); p->threads.clear(); p->serial_y.clear(); p->impl.clear();
}

hp_status run_groups_impl(hp_pipeline* p, Plan& plan, const hp_buffer* inputs, const hp_buffer* output, void* stream);

// Launches every group's kernel in order on `stream`; with the overlap option
// each launch may begin while the previous kernel drains (every kernel waits
// for its predecessor before touching memory).
hp_status run_groups(hp_pipeline* p, Plan& plan, const hp_buffer* inputs, const hp_buffer* output, void* stream) {
  struct Overlap {
    int saved;
    KernelProbe* saved_probe;
    Overlap(int on, KernelProbe* probe) : saved(t_overlap), saved_probe(t_probe) {
      t_overlap = on;
      t_probe = probe;
    }
    ~Overlap() {
      t_overlap = saved;
      t_probe = saved_probe;
    }
  } guard(p->overlap ? 1 : 0, p->probe ? &p->probed : nullptr);
  if (p->probe) p->probed = KernelProbe{0, 0, 0};
  return run_groups_impl(p, plan, inputs, output, stream);
}

hp_status run_groups_impl(hp_pipeline* p, Plan& plan, const hp_buffer* inputs, const hp_buffer* output, void* stream) {
  for (GroupPlan& gp : plan.groups) {
    ImgView out = ref_view(p, plan, gp.output, inputs, output);
    int e = 0;
    switch (gp.kernel) {
      case HP_KERNEL_STENCIL_CHAIN:
      case HP_KERNEL_UNSHARP:
      case HP_KERNEL_STENCIL_WAVE:
      case HP_KERNEL_STENCIL_LINES: {
        ChainArgs a = gp.chain;
        int first = gp.members[0];
        a.in = ref_view(p, plan, p->stages[first].inputs[0], inputs, output);
        a.out = out;
        a.err = p->d_err;
        e = gp.kernel == HP_KERNEL_STENCIL_WAVE    ? launch_chain_rows(a, a.cols, a.tile_h, gp.grid_x, gp.smem, stream)
            : gp.kernel == HP_KERNEL_STENCIL_LINES ? launch_chain_lines(a, stream)
                                                   : launch_chain(a, gp.smem, stream);
        break;
      }
      case HP_KERNEL_STENCIL_ROWS: {
        ChainArgs a = gp.chain;
        a.in = ref_view(p, plan, p->stages[gp.members[0]].inputs[0], inputs, output);
        a.out = out;
        a.err = p->d_err;
        e = launch_stencil_rows(a, a.tile_h, gp.grid_x, gp.smem, stream);
        break;
      }
      case HP_KERNEL_DOWNSAMPLE: {
        LLDownArgs a = gp.lldown;
        a.src = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.out = out;
        e = launch_ll_down(a, gp.smem, stream);
        break;
      }
      case HP_KERNEL_GRID_BLUR: {
        GridBlurArgs a = gp.gblur;
        a.in = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.out = out;
        e = launch_grid_blur(a, gp.grid_x, stream);
        break;
      }
      case HP_KERNEL_GRID_SPLAT: {
        GridArgs a = gp.grid;
        a.in = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.grid = out;
        e = launch_grid_splat(a, stream);
        break;
      }
      case HP_KERNEL_GRID_SLICE: {
        GridArgs a = gp.grid;
        a.grid = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.in = ref_view(p, plan, gp.ext_refs[1], inputs, output);
        a.out = out;
        e = launch_grid_slice(a, stream);
        break;
      }
      case HP_KERNEL_PW_ROWS: {
        PwArgs a = gp.pw;
        for (int i = 0; i < a.n_in; ++i) a.in[i] = ref_view(p, plan, gp.ext_refs[i], inputs, output);
        a.out = out;
        e = launch_pw_rows(a, stream);
        break;
      }
      case HP_KERNEL_INTERP_ROWS: {
        InterpArgs a = gp.interp;
        a.fine = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.coarse = ref_view(p, plan, gp.ext_refs[1], inputs, output);
        a.out = out;
        a.err = p->d_err;
        e = launch_interp_rows(a, gp.grid_x, stream);
        break;
      }
      case HP_KERNEL_MAX_ROWS: {
        MaxArgs a = gp.maxa;
        a.in = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.out = out;
        a.err = p->d_err;
        e = launch_max_rows(a, gp.grid_x, stream);
        break;
      }
      case HP_KERNEL_LL_REMAP_ROWS:
      case HP_KERNEL_LL_DOWN_ROWS: {
        LLDownArgs a = gp.lldown;
        a.src = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.out = out;
        e = gp.kernel == HP_KERNEL_LL_REMAP_ROWS ? launch_ll_remap_rows(a, a.tile_h, gp.threads, gp.grid_x, stream)
                                                 : launch_ll_down_rows(a, a.tile_h, gp.threads, gp.grid_x, stream);
        break;
      }
      case HP_KERNEL_LL_LEVEL:
      case HP_KERNEL_LL_LEVEL_ROWS: {
        LLLevelArgs a = gp.lllevel;
        const LLRoles& r = gp.llroles;
        if (a.level0) {
          a.in = ref_view(p, plan, p->stages[r.gray].inputs[0], inputs, output);
        } else {
          a.G = ref_view(p, plan, r.Gl, inputs, output);
        }
        a.Gn = ref_view(p, plan, r.Gn, inputs, output);
        a.Rn = ref_view(p, plan, r.select >= 0 ? p->stages[r.select].inputs[0] : r.Rn, inputs, output);
        a.out = out;
        e = gp.kernel == HP_KERNEL_LL_LEVEL_ROWS ? launch_ll_level_rows(a, gp.tile_h, gp.threads, gp.grid_x, stream)
                                                 : launch_ll_level(a, stream);
        break;
      }
      case HP_KERNEL_HARRIS: {
        HarrisArgs a = gp.harris;
        a.in = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.out = out;
        a.err = p->d_err;
        e = launch_harris(a, gp.smem, stream);
        break;
      }
      case HP_KERNEL_HARRIS_ROWS: {
        HarrisArgs a = gp.harris;
        a.in = ref_view(p, plan, gp.ext_refs[0], inputs, output);
        a.out = out;
        a.err = p->d_err;
        e = launch_harris_rows(a, a.tile_h, gp.grid_x, gp.smem, stream);
        break;
      }
      case HP_KERNEL_HISTEQ:
        e = launch_histeq(ref_view(p, plan, gp.ext_refs[0], inputs, output), out, gp.aux, p->d_err, gp.grid_x,
                          p->batch, stream);
        break;
      case HP_KERNEL_HISTOGRAM: {
        HistArgs a{};
        a.in = ref_view(p, plan, p->stages[gp.output].inputs[0], inputs, output);
        a.hist = (unsigned int*)out.data;
        e = launch_hist(a, stream);
        break;
      }
      case HP_KERNEL_CDF_LUT: {
        LutArgs a{};
        a.hist = (const unsigned int*)ref_view(p, plan, p->stages[gp.output].inputs[0], inputs, output).data;
        a.lut = (unsigned char*)out.data;
        a.lut_view = out;
        e = launch_cdf_lut(a, stream);
        break;
      }
      case HP_KERNEL_LUT_APPLY: {
        LutApplyArgs a{};
        a.in = ref_view(p, plan, p->stages[gp.output].inputs[0], inputs, output);
        a.lut = (const unsigned char*)ref_view(p, plan, p->stages[gp.output].inputs[1], inputs, output).data;
        a.out = out;
        e = launch_lut_apply(a, stream);
        break;
      }
      default: {
        GPlan& g = *gp.gplan;
        for (size_t i = 0; i < gp.ext_refs.size(); ++i) g.ext[i] = ref_view(p, plan, gp.ext_refs[i], inputs, output);
        g.out = out;
        g.err = p->d_err;
        e = launch_generic(g, gp.threads, gp.smem, stream);
      }
    }
    if (e) return cuda_fail(e, "kernel launch");
  }
  return HP_OK;
}

// Replays the launch sequence as a CUDA graph.  The first realize for a set of
// buffer addresses runs uncaptured (it also sets kernel attributes); the second
// captures the sequence on a private stream and every later one launches the
// instantiated graph on the caller's stream.
hp_status run_graph(hp_pipeline* p, Plan& plan, const hp_buffer* inputs, int n_inputs, const hp_buffer* output,
                    void* stream) {
  std::vector<long long> key;
  for (int i = 0; i <= n_inputs; ++i) {
    const hp_buffer& b = i < n_inputs ? inputs[i] : *output;
    key.push_back((long long)(uintptr_t)b.data);
    key.push_back(b.row_stride_bytes);
    key.push_back(b.plane_stride_bytes);
  }
  ++p->uses;
  for (GraphEntry& g : plan.graphs) {
    if (g.key != key) continue;
    g.last_use = p->uses;
    int e = cudaGraphLaunch(g.exec, (cudaStream_t)stream);
    if (e) return cuda_fail(e, "cudaGraphLaunch");
    __atomic_add_fetch(&g_launches, g.kernels, __ATOMIC_RELAXED);
    ++p->graph_replays;
    return HP_OK;
  }
  if (std::find(plan.seen.begin(), plan.seen.end(), key) == plan.seen.end()) {
    if (plan.seen.size() > 4 * kMaxGraphs) plan.seen.clear();
    plan.seen.push_back(key);
    return run_groups(p, plan, inputs, output, stream);
  }
  if (!p->capture_stream) {
    int e = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking);
    if (e) return cuda_fail(e, "cudaStreamCreate");
  }
  // capture only records; the graph launch below orders after the caller's work
  unsigned long long before = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
  int e = cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e) return cuda_fail(e, "cudaStreamBeginCapture");
  hp_status st = run_groups(p, plan, inputs, output, p->capture_stream);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(p->capture_stream, &graph);
  unsigned long long kernels = __atomic_load_n(&g_launches, __ATOMIC_RELAXED) - before;
  __atomic_sub_fetch(&g_launches, kernels, __ATOMIC_RELAXED);  // captured, not executed
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e) return cuda_fail(e, "cudaGraphInstantiate");
  if (plan.graphs.size() >= kMaxGraphs) {
    auto lru = std::min_element(plan.graphs.begin(), plan.graphs.end(),
                                [](const GraphEntry& a, const GraphEntry& b) { return a.last_use < b.last_use; });
    cudaGraphExecDestroy(lru->exec);
    plan.graphs.erase(lru);
  }
  GraphEntry g;
  g.key = key;
  g.exec = exec;
  g.kernels = kernels;
  g.last_use = p->uses;
  plan.graphs.push_back(g);
  e = cudaGraphLaunch(exec, (cudaStream_t)stream);
  if (e) return cuda_fail(e, "cudaGraphLaunch");
  __atomic_add_fetch(&g_launches, kernels, __ATOMIC_RELAXED);
  return HP_OK;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" {

hp_status hp_pipeline_create(hp_pipeline** out, int n_inputs, const int* in_dtypes, const int* in_channels) {
  if (!out || n_inputs < 1 || n_inputs > 16 || !in_dtypes || !in_channels)
    return fail(HP_ERR_INVALID_ARG, "hp_pipeline_create: bad arguments");
  for (int i = 0; i < n_inputs; ++i) {
    if (!valid_dtype(in_dtypes[i]) || in_dtypes[i] == HP_U32)
      return fail(HP_ERR_INVALID_ARG, "input %d: bad dtype %d", i, in_dtypes[i]);
    if (in_channels[i] < 1 || in_channels[i] > 64) return fail(HP_ERR_INVALID_ARG, "input %d: bad channel count", i);
  }
  auto* p = new hp_pipeline();
  p->in_dtypes.assign(in_dtypes, in_dtypes + n_inputs);
  p->in_channels.assign(in_channels, in_channels + n_inputs);
  *out = p;
  t_err.clear();
  return HP_OK;
}

hp_status hp_add_stage(hp_pipeline* p, const hp_stage_desc* d, int* out_id) {
  if (!p || !d) return fail(HP_ERR_INVALID_ARG, "hp_add_stage: null argument");
  hp_status s = validate_stage(p, d);
  if (s) return s;
  Stage st;
  st.kind = d->kind;
  st.op = d->op;
  st.channels = d->channels;
  st.storage = d->storage;
  st.inputs.assign(d->inputs, d->inputs + d->n_inputs);
  st.rx = d->rx;
  st.ry = d->ry;
  if (d->kind == HP_STENCIL) {
    st.wx.assign(d->wx, d->wx + 2 * d->rx + 1);
    st.wy.assign(d->wy, d->wy + 2 * d->ry + 1);
  }
  if (d->n_params > 0) st.params.assign(d->params, d->params + d->n_params);
  p->stages.push_back(st);
  if (out_id) *out_id = (int)p->stages.size() - 1;
  p->has_schedule = false;
  drop_plans(p);
  return HP_OK;
}

hp_status hp_set_output(hp_pipeline* p, int stage_id) {
  if (!p || stage_id < 0 || stage_id >= (int)p->stages.size())
    return fail(HP_ERR_INVALID_ARG, "hp_set_output: bad stage id %d", stage_id);
  p->output = stage_id;
  if (!p->has_schedule) default_schedule(p);
  drop_plans(p);
  return HP_OK;
}

hp_status hp_schedule_set(hp_pipeline* p, const hp_schedule* s) {
  if (!p || !s) return fail(HP_ERR_INVALID_ARG, "hp_schedule_set: null argument");
  if (p->output < 0) return fail(HP_ERR_STATE, "set the output stage before the schedule");
  int ns = (int)p->stages.size();
  if (s->n_stages != ns || !s->group_of_stage || s->n_groups < 1 || s->n_groups > ns)
    return fail(HP_ERR_SCHEDULE, "schedule must cover all %d stages with 1..%d groups", ns, ns);
  for (int i = 0; i < ns; ++i) {
    int g = s->group_of_stage[i];
    if (g == HP_INLINE) {
      if (p->stages[i].kind != HP_POINTWISE) return fail(HP_ERR_SCHEDULE, "only point-wise stages can be inlined");
      if (i == p->output) return fail(HP_ERR_SCHEDULE, "the output stage cannot be inlined");
    } else if (g < 0 || g >= s->n_groups) {
      return fail(HP_ERR_SCHEDULE, "stage %d: group %d out of range", i, g);
    }
  }
  auto per_group = [&](const int* v, std::vector<int>& dst, int lo, int hi, const char* what) -> hp_status {
    dst.clear();
    if (!v) return HP_OK;
    dst.assign(v, v + s->n_groups);
    for (int x : dst)
      if (x != 0 && (x < lo || x > hi)) return fail(HP_ERR_SCHEDULE, "%s %d out of range [%d, %d]", what, x, lo, hi);
    return HP_OK;
  };
  // keep the old schedule until the new one validates
  hp_pipeline tmp;
  tmp.stages = p->stages;
  tmp.output = p->output;
  tmp.in_dtypes = p->in_dtypes;
  tmp.in_channels = p->in_channels;
  tmp.group_of.assign(s->group_of_stage, s->group_of_stage + ns);
  tmp.n_groups = s->n_groups;
  hp_status st;
  if ((st = per_group(s->tile_w, tmp.tile_w, 1, 4096, "tile_w")) || (st = per_group(s->tile_h, tmp.tile_h, 1, 4096, "tile_h")) ||
      (st = per_group(s->threads, tmp.threads, 32, 1024, "threads")) ||
      (st = per_group(s->serial_y, tmp.serial_y, 1, 256, "serial_y")) ||
      (st = per_group(s->impl, tmp.impl, 0, 3, "impl")))
    return st;
  std::vector<GroupShape> shapes;
  if ((st = group_shapes(&tmp, shapes))) return st;
  drop_plans(p);
  p->group_of = tmp.group_of;
  p->n_groups = tmp.n_groups;
  p->tile_w = tmp.tile_w; p->tile_h = tmp.tile_h; p->threads = tmp.threads;
  p->serial_y = tmp.serial_y; p->impl = tmp.impl;
  p->has_schedule = true;
  return HP_OK;
}

static hp_status collect_in_dom(hp_pipeline* p, const hp_buffer* inputs, int n_inputs, std::vector<Dom>& in_dom) {
  if (!p || !inputs || n_inputs != (int)p->in_dtypes.size())
    return fail(HP_ERR_INVALID_ARG, "expected %d input buffers", p ? (int)p->in_dtypes.size() : 0);
  in_dom.clear();
  for (int i = 0; i < n_inputs; ++i) {
    hp_status s = check_buffer(inputs[i], p->in_dtypes[i], p->in_channels[i] * p->batch, Dom{0, 0}, "input", i);
    if (s) return s;
    in_dom.push_back(Dom{inputs[i].width, inputs[i].height});
  }
  return HP_OK;
}

// The pipeline's device error word: allocated once, cleared on the caller's
// stream (no device-wide wait).
static hp_status alloc_error_word(hp_pipeline* p, void* stream) {
  if (cudaMalloc(&p->d_err, 16) != cudaSuccess) {
    cudaGetLastError();
    p->d_err = nullptr;
    return fail(HP_ERR_OOM, "cudaMalloc of the error word failed");
  }
  const cudaError_t e = cudaMemsetAsync(p->d_err, 0, 16, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->d_err);
    p->d_err = nullptr;
    return fail(HP_ERR_CUDA, "clearing the error word failed: %s", cudaGetErrorString(e));
  }
  return HP_OK;
}

hp_status hp_prepare(hp_pipeline* p, const int* widths, const int* heights, int n_inputs, void* stream) {
  if (!p || !widths || !heights || n_inputs != (int)p->in_dtypes.size())
    return fail(HP_ERR_INVALID_ARG, "hp_prepare: expected %d input sizes", p ? (int)p->in_dtypes.size() : 0);
  std::vector<Dom> in_dom;
  for (int i = 0; i < n_inputs; ++i) {
    if (widths[i] < 1 || heights[i] < 1) return fail(HP_ERR_INVALID_ARG, "hp_prepare: empty input %d", i);
    in_dom.push_back(Dom{widths[i], heights[i]});
  }
  Plan* plan = nullptr;
  hp_status s = get_plan(p, in_dom, &plan);
  if (s) return s;
  if (!p->d_err) {
    if ((s = alloc_error_word(p, stream))) return s;
  }
  return ensure_scratch(p, *plan, (cudaStream_t)stream);
}

hp_status hp_realize(hp_pipeline* p, const hp_buffer* inputs, int n_inputs, const hp_buffer* output, void* stream) {
  std::vector<Dom> in_dom;
  hp_status s = collect_in_dom(p, inputs, n_inputs, in_dom);
  if (s) return s;
  if (!output) return fail(HP_ERR_INVALID_ARG, "null output buffer");
  Plan* plan = nullptr;
  if ((s = get_plan(p, in_dom, &plan))) return s;
  const Stage& os = p->stages[p->output];
  if ((s = check_buffer(*output, os.storage, os.channels * p->batch, plan->dom[p->output], "output", 0))) return s;
  if (!p->d_err && (s = alloc_error_word(p, stream))) return s;
  if ((s = ensure_scratch(p, *plan, (cudaStream_t)stream))) return s;
  if (!p->use_graph) return run_groups(p, *plan, inputs, output, stream);
  return run_graph(p, *plan, inputs, n_inputs, output, stream);
}

hp_status hp_realize_host(hp_pipeline* p, const hp_buffer* inputs, int n_inputs, const hp_buffer* output,
                          void* stream) {
  std::vector<Dom> in_dom;
  if (!p || !inputs || n_inputs != (int)p->in_dtypes.size() || !output)
    return fail(HP_ERR_INVALID_ARG, "hp_realize_host: bad arguments");
  for (int i = 0; i < n_inputs; ++i) in_dom.push_back(Dom{inputs[i].width, inputs[i].height});
  Plan* plan = nullptr;
  hp_status s = get_plan(p, in_dom, &plan);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<hp_buffer> dev_in(n_inputs);
  if (plan->staging.empty()) {
    plan->staging.resize(n_inputs + 1);
    for (int i = 0; i <= n_inputs; ++i) {
      const hp_buffer& b = i < n_inputs ? inputs[i] : *output;
      size_t bytes = (size_t)round16((long long)b.width * dtype_bytes(b.dtype)) * b.height * b.channels;
      if (cudaMalloc(&plan->staging[i].ptr, bytes)) {
        cudaGetLastError();
        plan->staging.clear();
        return fail(HP_ERR_OOM, "cudaMalloc of %zu staging bytes failed", bytes);
      }
      plan->staging[i].bytes = bytes;
    }
  }
  for (int i = 0; i <= n_inputs; ++i) {
    const hp_buffer& b = i < n_inputs ? inputs[i] : *output;
    if (!b.data) return fail(HP_ERR_INVALID_ARG, "null host buffer");
    hp_buffer d = b;
    d.data = plan->staging[i].ptr;
    d.row_stride_bytes = round16((long long)b.width * dtype_bytes(b.dtype));
    d.plane_stride_bytes = d.row_stride_bytes * b.height;
    if (i < n_inputs) {
      dev_in[i] = d;
      for (int c = 0; c < b.channels; ++c) {
        int e = cudaMemcpy2DAsync((char*)d.data + c * d.plane_stride_bytes, d.row_stride_bytes,
                                  (const char*)b.data + c * b.plane_stride_bytes, b.row_stride_bytes,
                                  (size_t)b.width * dtype_bytes(b.dtype), b.height, cudaMemcpyHostToDevice, st);
        if (e) return cuda_fail(e, "host-to-device copy");
      }
    }
  }
  hp_buffer dev_out = *output;
  dev_out.data = plan->staging[n_inputs].ptr;
  dev_out.row_stride_bytes = round16((long long)output->width * dtype_bytes(output->dtype));
  dev_out.plane_stride_bytes = dev_out.row_stride_bytes * output->height;
  if ((s = hp_realize(p, dev_in.data(), n_inputs, &dev_out, stream))) return s;
  for (int c = 0; c < output->channels; ++c) {
    int e = cudaMemcpy2DAsync((char*)output->data + c * output->plane_stride_bytes, output->row_stride_bytes,
                              (const char*)dev_out.data + c * dev_out.plane_stride_bytes, dev_out.row_stride_bytes,
                              (size_t)output->width * dtype_bytes(output->dtype), output->height,
                              cudaMemcpyDeviceToHost, st);
    if (e) return cuda_fail(e, "device-to-host copy");
  }
  int e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(e, "stream synchronize");
  return HP_OK;
}

hp_status hp_realize_host_async(hp_pipeline* p, const hp_buffer* inputs, int n_inputs, const hp_buffer* output,
                                void* stream) {
  std::vector<Dom> in_dom;
  if (!p || !inputs || n_inputs != (int)p->in_dtypes.size() || !output)
    return fail(HP_ERR_INVALID_ARG, "hp_realize_host_async: bad arguments");
  for (int i = 0; i <= n_inputs; ++i)
    if (!(i < n_inputs ? inputs[i] : *output).data) return fail(HP_ERR_INVALID_ARG, "null host buffer");
  for (int i = 0; i < n_inputs; ++i) in_dom.push_back(Dom{inputs[i].width, inputs[i].height});
  Plan* plan = nullptr;
  hp_status s = get_plan(p, in_dom, &plan);
  if (s) return s;
  if (!p->host_in) {
    cudaStream_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) || cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking)) {
      cudaGetLastError();
      if (a) cudaStreamDestroy(a);
      return fail(HP_ERR_CUDA, "hp_realize_host_async: stream creation failed");
    }
    for (int j = 0; j < 2; ++j)
      if (cudaEventCreateWithFlags(&p->ev_in[j], cudaEventDisableTiming) ||
          cudaEventCreateWithFlags(&p->ev_done[j], cudaEventDisableTiming) ||
          cudaEventCreateWithFlags(&p->ev_free[j], cudaEventDisableTiming)) {
        cudaGetLastError();
        cudaStreamDestroy(a);
        cudaStreamDestroy(b);
        return fail(HP_ERR_CUDA, "hp_realize_host_async: event creation failed");
      }
    p->host_in = a;
    p->host_out = b;
  }
  const int j = (int)(p->async_calls & 1);
  std::vector<Scratch>& set = plan->staging_async[j];
  if (set.empty()) {
    set.resize(n_inputs + 1);
    for (int i = 0; i <= n_inputs; ++i) {
      const hp_buffer& b = i < n_inputs ? inputs[i] : *output;
      const size_t bytes = (size_t)round16((long long)b.width * dtype_bytes(b.dtype)) * b.height * b.channels;
      if (cudaMalloc(&set[i].ptr, bytes)) {
        cudaGetLastError();
        for (int k = 0; k < i; ++k) cudaFree(set[k].ptr);
        set.clear();
        return fail(HP_ERR_OOM, "cudaMalloc of %zu staging bytes failed", bytes);
      }
      set[i].bytes = bytes;
    }
  }
  std::vector<hp_buffer> dev_in(n_inputs);
  hp_buffer dev_out = *output;
  for (int i = 0; i <= n_inputs; ++i) {
    const hp_buffer& b = i < n_inputs ? inputs[i] : *output;
    hp_buffer d = b;
    d.data = set[i].ptr;
    d.row_stride_bytes = round16((long long)b.width * dtype_bytes(b.dtype));
    d.plane_stride_bytes = d.row_stride_bytes * b.height;
    if (i < n_inputs) dev_in[i] = d;
    else dev_out = d;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the set's previous copy out (two calls back) is done before its staging is reused
  if (cudaStreamWaitEvent(p->host_in, p->ev_free[j], 0)) return cuda_fail(cudaGetLastError(), "stream wait");
  for (int i = 0; i < n_inputs; ++i)
    for (int c = 0; c < inputs[i].channels; ++c) {
      int e = cudaMemcpy2DAsync((char*)dev_in[i].data + c * dev_in[i].plane_stride_bytes, dev_in[i].row_stride_bytes,
                                (const char*)inputs[i].data + c * inputs[i].plane_stride_bytes, inputs[i].row_stride_bytes,
                                (size_t)inputs[i].width * dtype_bytes(inputs[i].dtype), inputs[i].height,
                                cudaMemcpyHostToDevice, p->host_in);
      if (e) return cuda_fail(e, "host-to-device copy");
    }
  if (cudaEventRecord(p->ev_in[j], p->host_in) || cudaStreamWaitEvent(st, p->ev_in[j], 0))
    return cuda_fail(cudaGetLastError(), "event record / wait");
  if ((s = hp_realize(p, dev_in.data(), n_inputs, &dev_out, stream))) return s;
  if (cudaEventRecord(p->ev_done[j], st) || cudaStreamWaitEvent(p->host_out, p->ev_done[j], 0))
    return cuda_fail(cudaGetLastError(), "event record / wait");
  for (int c = 0; c < output->channels; ++c) {
    int e = cudaMemcpy2DAsync((char*)output->data + c * output->plane_stride_bytes, output->row_stride_bytes,
                              (const char*)dev_out.data + c * dev_out.plane_stride_bytes, dev_out.row_stride_bytes,
                              (size_t)output->width * dtype_bytes(output->dtype), output->height,
                              cudaMemcpyDeviceToHost, p->host_out);
    if (e) return cuda_fail(e, "device-to-host copy");
  }
  if (cudaEventRecord(p->ev_free[j], p->host_out)) return cuda_fail(cudaGetLastError(), "event record");
  ++p->async_calls;
  return HP_OK;
}

hp_status hp_realize_host_wait(hp_pipeline* p) {
  if (!p) return fail(HP_ERR_INVALID_ARG, "null pipeline");
  if (!p->host_out) return HP_OK;
  int e = cudaStreamSynchronize(p->host_out);
  if (e) return cuda_fail(e, "stream synchronize");
  return HP_OK;
}

hp_status hp_group_count(hp_pipeline* p, int* n) {
  if (!p || !n) return fail(HP_ERR_INVALID_ARG, "null argument");
  if (p->output < 0) return fail(HP_ERR_STATE, "no output stage set");
  *n = p->n_groups;
  return HP_OK;
}

static hp_status plan_for_sizes(hp_pipeline* p, const int* ws, const int* hs, Plan** plan) {
  if (!p || !ws || !hs) return fail(HP_ERR_INVALID_ARG, "null argument");
  std::vector<Dom> in_dom;
  for (size_t i = 0; i < p->in_dtypes.size(); ++i) {
    if (ws[i] < 1 || hs[i] < 1) return fail(HP_ERR_INVALID_ARG, "input %zu: empty size", i);
    in_dom.push_back(Dom{ws[i], hs[i]});
  }
  return get_plan(p, in_dom, plan);
}

hp_status hp_group_info_get(hp_pipeline* p, const int* ws, const int* hs, int group, hp_group_info* info) {
  Plan* plan = nullptr;
  hp_status s = plan_for_sizes(p, ws, hs, &plan);
  if (s) return s;
  if (!info || group < 0 || group >= (int)plan->groups.size()) return fail(HP_ERR_INVALID_ARG, "bad group");
  const GroupPlan& gp = plan->groups[group];
  info->kernel = gp.kernel;
  info->output_stage = gp.output;
  info->n_members = (int)gp.members.size();
  info->tile_w = gp.tile_w;
  info->tile_h = gp.tile_h;
  info->threads = gp.threads;
  info->grid_x = gp.grid_x;
  info->grid_y = gp.grid_y;
  info->grid_z = gp.grid_z;
  info->smem_bytes = gp.smem;
  return HP_OK;
}

hp_status hp_infer_bounds(hp_pipeline* p, const int* ws, const int* hs, int group, int x0, int y0, int w, int h,
                          int* rects, int n_rects) {
  Plan* plan = nullptr;
  hp_status s = plan_for_sizes(p, ws, hs, &plan);
  if (s) return s;
  if (group < 0 || group >= (int)plan->groups.size() || !rects || n_rects < (int)p->stages.size() || w < 1 || h < 1)
    return fail(HP_ERR_INVALID_ARG, "bad group, tile or rects array");
  const GroupPlan& gp = plan->groups[group];
  // same propagation as the kernels, for this tile size
  GPlan g;
  memset(&g, 0, sizeof g);
  std::map<int, int> node_of;
  for (size_t i = 0; i < gp.members.size(); ++i) node_of[gp.members[i]] = (int)i;
  g.n_nodes = (int)gp.members.size();
  g.tile_w = w;
  g.tile_h = h;
  for (size_t i = 0; i < gp.members.size(); ++i) {
    const Stage& st = p->stages[gp.members[i]];
    GNode& n = g.nodes[i];
    n.kind = st.kind;
    n.n_in = (int)st.inputs.size();
    for (int k = 0; k < n.n_in; ++k) {
      auto it = node_of.find(st.inputs[k]);
      n.in[k] = st.inputs[k] >= 0 && it != node_of.end() ? it->second : -1;
    }
    n.rx = st.rx;
    n.ry = st.ry;
    n.dom_w = plan->dom[gp.members[i]].w;
    n.dom_h = plan->dom[gp.members[i]].h;
  }
  std::vector<Rect> r(g.n_nodes);
  infer_rects(g, x0, y0, r.data());
  for (size_t i = 0; i < p->stages.size(); ++i) {
    rects[4 * i] = rects[4 * i + 1] = rects[4 * i + 2] = rects[4 * i + 3] = 0;
  }
  for (int n = 0; n < g.n_nodes; ++n) {
    int sid = gp.members[n];
    rects[4 * sid] = r[n].x0;
    rects[4 * sid + 1] = r[n].y0;
    rects[4 * sid + 2] = r[n].x1;
    rects[4 * sid + 3] = r[n].y1;
  }
  return HP_OK;
}

}  // extern "C"

namespace hp {

// True when every stage acts on each channel separately, so B images can be
// stacked plane-wise into one image of B times the channels.
bool pipeline_stackable(const hp_pipeline* p) {
  for (const Stage& s : p->stages) {
    if (s.kind == HP_STENCIL || s.kind == HP_MAX_STENCIL || s.kind == HP_DOWNSAMPLE2 || s.kind == HP_UPSAMPLE2) continue;
    if (s.kind == HP_POINTWISE && (s.op == HP_OP_MUL || s.op == HP_OP_ADD || s.op == HP_OP_SUB ||
                                   s.op == HP_OP_UNSHARP || s.op == HP_OP_SCALE))
      continue;
    return false;
  }
  return true;
}

unsigned long long pipeline_graph_replays(const hp_pipeline* p) { return p->graph_replays; }

hp_pipeline* clone_pipeline(const hp_pipeline* p, int batch);

// Whether `batch` images of these input sizes can be realized by one call of a
// batched copy of p: a stackable pipeline always; otherwise its lowering for
// the sizes must put every group on a batch-aware kernel.
// Size, channels and storage type of p's output for these input sizes (one image).
hp_status pipeline_output_shape(hp_pipeline* p, const int* widths, const int* heights, int n_inputs, int* w, int* h,
                                int* channels, int* dtype) {
  std::vector<Dom> in_dom;
  for (int i = 0; i < n_inputs; ++i) in_dom.push_back(Dom{widths[i], heights[i]});
  Plan* plan = nullptr;
  hp_status st = get_plan(p, in_dom, &plan);
  if (st) return st;
  const Stage& os = p->stages[p->output];
  *w = plan->dom[p->output].w;
  *h = plan->dom[p->output].h;
  *channels = os.channels;
  *dtype = os.storage;
  return HP_OK;
}

bool pipeline_batch_ok(const hp_pipeline* p, const int* widths, const int* heights, int n_inputs, int batch) {
  if (batch <= 1 || pipeline_stackable(p)) return true;
  hp_pipeline* c = clone_pipeline(p, batch);
  std::vector<Dom> in_dom;
  for (int i = 0; i < n_inputs; ++i) in_dom.push_back(Dom{widths[i], heights[i]});
  Plan* plan = nullptr;
  const bool ok = get_plan(c, in_dom, &plan) == HP_OK;
  hp_pipeline_destroy(c);
  return ok;
}

// A copy of the pipeline's algorithm and schedule (no plans, no scratch) for
// `batch` images stacked as planes: a stackable pipeline (every stage acts on
// each channel separately) gets every channel count multiplied by batch; any
// other pipeline keeps its channels and realizes `batch` images per call,
// which its kernels must support (lowering refuses the batch otherwise).
hp_pipeline* clone_pipeline(const hp_pipeline* p, int batch) {
  auto* c = new hp_pipeline();
  c->in_dtypes = p->in_dtypes;
  c->in_channels = p->in_channels;
  c->stages = p->stages;
  if (batch > 1 && pipeline_stackable(p)) {
    for (int& ch : c->in_channels) ch *= batch;
    for (Stage& s : c->stages) s.channels *= batch;
  } else {
    c->batch = batch;
  }
  c->output = p->output;
  c->has_schedule = p->has_schedule;
  c->group_of = p->group_of;
  c->n_groups = p->n_groups;
  c->tile_w = p->tile_w;
  c->tile_h = p->tile_h;
  c->threads = p->threads;
  c->serial_y = p->serial_y;
  c->impl = p->impl;
  return c;
}

}  // namespace hp

extern "C" {

hp_status hp_check_device_error(hp_pipeline* p, int* code) {
  if (!p || !code) return fail(HP_ERR_INVALID_ARG, "null argument");
  *code = 0;
  if (!p->d_err) return HP_OK;
  int e = cudaMemcpy(code, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) return cuda_fail(e, "reading the device error word");
  e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e) return cuda_fail(e, "clearing the device error word");
  return HP_OK;
}

hp_status hp_set_option(hp_pipeline* p, int option, long long value) {
  if (!p) return fail(HP_ERR_INVALID_ARG, "null pipeline");
  switch (option) {
    case HP_OPT_CUDA_GRAPH:
      if (p->use_graph != (value != 0)) {
        for (auto& kv : p->plans) {
          for (auto& g : kv.second->graphs) cudaGraphExecDestroy(g.exec);
          kv.second->graphs.clear();
          kv.second->seen.clear();
        }
      }
      p->use_graph = value != 0;
      return HP_OK;
    case HP_OPT_OVERLAP:
      if (p->overlap != (value != 0)) {  // captured graphs hold the old launch attributes
        for (auto& kv : p->plans) {
          for (auto& g : kv.second->graphs) cudaGraphExecDestroy(g.exec);
          kv.second->graphs.clear();
          kv.second->seen.clear();
        }
      }
      p->overlap = value != 0;
      return HP_OK;
    case HP_OPT_PROBE_ATTRS:
      p->probe = value != 0;
      p->probed = hp::KernelProbe{0, 0, 0};
      return HP_OK;
    default:
      return fail(HP_ERR_INVALID_ARG, "unknown option %d", option);
  }
}

hp_status hp_pipeline_destroy(hp_pipeline* p) {
  if (!p) return fail(HP_ERR_INVALID_ARG, "null pipeline");
  drop_plans(p);
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  if (p->host_in) cudaStreamDestroy(p->host_in);
  if (p->host_out) cudaStreamDestroy(p->host_out);
  for (int j = 0; j < 2; ++j) {
    if (p->ev_in[j]) cudaEventDestroy(p->ev_in[j]);
    if (p->ev_done[j]) cudaEventDestroy(p->ev_done[j]);
    if (p->ev_free[j]) cudaEventDestroy(p->ev_free[j]);
  }
  if (p->d_err) cudaFree(p->d_err);
  delete p;
  return HP_OK;
}

const char* hp_last_error(void) { return t_err.c_str(); }

unsigned long long hp_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

}  // extern "C"

hp_status hp_kernel_attrs_get(hp_pipeline* p, int* n_kernels, int* max_registers, long long* max_local_bytes) {
  using namespace hp;
  if (!p || !n_kernels || !max_registers || !max_local_bytes) return fail(HP_ERR_INVALID_ARG, "null argument");
  *n_kernels = p->probed.kernels;
  *max_registers = p->probed.max_regs;
  *max_local_bytes = p->probed.max_local;
  return HP_OK;
}
