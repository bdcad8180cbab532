// One point-wise stage over f32 images (the inlined producers of Sec. 4 when
// they run as their own kernel): 4 pixels of one row per thread, 128-bit loads
// and stores, every output channel.  Covers the per-channel ops (add, sub,
// mul, scale, unsharp combine) and the RGBA ops of the interpolate app
// (premultiply, over, unpremultiply); the values are the stage_math.cuh
// expressions, so they equal the generic kernel's bit for bit.
#include <cuda_runtime.h>

#include "hp_internal.h"
#include "stage_math.cuh"

namespace hp {

namespace {

__device__ __forceinline__ float4 ld4(const ImgView& v, int c, int y, int x4, bool full) {
  const float* row = reinterpret_cast<const float*>((const char*)v.data + (long long)c * v.ps + (long long)y * v.rs);
  if (full) return __ldg(reinterpret_cast<const float4*>(row) + (x4 >> 2));
  float t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) t[k] = x4 + k < v.w ? __ldg(row + x4 + k) : 0.0f;
  return make_float4(t[0], t[1], t[2], t[3]);
}

template <int OP>
__device__ __forceinline__ float pw(float a, float b, float alpha, int c, const PwArgs& p) {
  switch (OP) {
    case HP_OP_MUL: case HP_OP_ADD: case HP_OP_SUB: return op_binary(OP, a, b);
    case HP_OP_UNSHARP: return op_unsharp(a, b, p.p0);
    case HP_OP_SCALE: return op_scale(a, p.p0, p.p1);
    case HP_OP_PREMUL: return op_premul(a, alpha, c);
    case HP_OP_OVER: return op_over(a, alpha, b);
    default: return op_unpremul(a, alpha);  // HP_OP_UNPREMUL
  }
}

template <int OP>
__global__ void __launch_bounds__(256) k_pw(const PwArgs p) {
  grid_dep_sync();
  const int x4 = (blockIdx.x * 64 + (threadIdx.x & 63)) * 4;
  const int y = blockIdx.y * 4 + (threadIdx.x >> 6);
  if (y >= p.out.h || x4 >= p.out.w) return;
  const bool full = x4 + 3 < p.out.w;
  constexpr bool kAlpha = OP == HP_OP_PREMUL || OP == HP_OP_OVER || OP == HP_OP_UNPREMUL;
  constexpr bool kTwo = OP == HP_OP_MUL || OP == HP_OP_ADD || OP == HP_OP_SUB || OP == HP_OP_UNSHARP || OP == HP_OP_OVER;
  float4 al = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (kAlpha) al = ld4(p.in[0], 3, y, x4, full);
  char* orow = (char*)p.out.data + (long long)y * p.out.rs;
  for (int c = 0; c < p.out.c; ++c) {
    const float4 a = ld4(p.in[0], c, y, x4, full);
    const float4 b = kTwo ? ld4(p.in[1], c, y, x4, full) : a;
    const float4 o = make_float4(pw<OP>(a.x, b.x, al.x, c, p), pw<OP>(a.y, b.y, al.y, c, p),
                                 pw<OP>(a.z, b.z, al.z, c, p), pw<OP>(a.w, b.w, al.w, c, p));
    float* q = reinterpret_cast<float*>(orow + (long long)c * p.out.ps);
    if (full) {
      reinterpret_cast<float4*>(q)[x4 >> 2] = o;
    } else {
      const float t[4] = {o.x, o.y, o.z, o.w};
      for (int k = 0; k < 4 && x4 + k < p.out.w; ++k) q[x4 + k] = t[k];
    }
  }
}

typedef void (*PwKernel)(PwArgs);

PwKernel pick_kernel(int op) {
  switch (op) {
    case HP_OP_MUL: return k_pw<HP_OP_MUL>;
    case HP_OP_ADD: return k_pw<HP_OP_ADD>;
    case HP_OP_SUB: return k_pw<HP_OP_SUB>;
    case HP_OP_UNSHARP: return k_pw<HP_OP_UNSHARP>;
    case HP_OP_SCALE: return k_pw<HP_OP_SCALE>;
    case HP_OP_PREMUL: return k_pw<HP_OP_PREMUL>;
    case HP_OP_OVER: return k_pw<HP_OP_OVER>;
    case HP_OP_UNPREMUL: return k_pw<HP_OP_UNPREMUL>;
    default: return nullptr;
  }
}

}  // namespace

int pw_rows_op_ok(int op) { return pick_kernel(op) != nullptr; }

int launch_pw_rows(const PwArgs& p, void* stream) {
  PwKernel k = pick_kernel(p.op);
  if (!k) return (int)cudaErrorInvalidValue;
  for (int i = 0; i < p.n_in; ++i)
    if (p.in[i].dtype != HP_F32 || p.in[i].w != p.out.w || p.in[i].h != p.out.h) return (int)cudaErrorInvalidValue;
  if (p.out.dtype != HP_F32) return (int)cudaErrorInvalidValue;
  dim3 grid((p.out.w + 255) / 256, (p.out.h + 3) / 4, 1);
  { const int le_ = launch_kernel(k, grid, dim3(256), 0, stream, p); if (le_) return le_; }
  __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
  return (int)cudaGetLastError();
}

}  // namespace hp
