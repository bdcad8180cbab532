// Per-stage float expressions.  They are part of the algorithm: every kernel
// (stage-per-kernel, fused chain, Harris, generic interpreter) evaluates a stage
// through these functions, with explicitly rounded operations so that FMA
// contraction cannot differ between inlining contexts.  That is what makes any
// two schedules of a pipeline give bit-identical results.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "hp_internal.h"

namespace hp {

// ---- storage -------------------------------------------------------------
// A stage's value is rounded to its storage dtype wherever it is kept.
__device__ __forceinline__ float round_storage(int dtype, float v) {
  switch (dtype) {
    case HP_F16: return __half2float(__float2half_rn(v));
    case HP_BF16: return __bfloat162float(__float2bfloat16_rn(v));
    case HP_U8: return fminf(fmaxf(rintf(v), 0.0f), 255.0f);
    case HP_U16: return fminf(fmaxf(rintf(v), 0.0f), 65535.0f);
    default: return v;
  }
}

__device__ __forceinline__ const char* px_ptr(const ImgView& v, int c, int x, int y, int esize) {
  return (const char*)v.data + (long long)c * v.ps + (long long)y * v.rs + (long long)x * esize;
}

__device__ __forceinline__ int dtype_size(int dtype) {
  return dtype == HP_U8 ? 1 : (dtype == HP_U16 || dtype == HP_F16 || dtype == HP_BF16) ? 2 : 4;
}

__device__ __forceinline__ float load_px(const ImgView& v, int c, int x, int y) {
  const char* p = (const char*)v.data + (long long)c * v.ps + (long long)y * v.rs;
  switch (v.dtype) {
    case HP_U8: return (float)((const unsigned char*)p)[x];
    case HP_U16: return (float)((const unsigned short*)p)[x];
    case HP_F16: return __half2float(((const __half*)p)[x]);
    case HP_BF16: return __bfloat162float(((const __nv_bfloat16*)p)[x]);
    case HP_U32: return (float)((const unsigned int*)p)[x];
    default: return ((const float*)p)[x];
  }
}

// Stores a value already rounded to the view's dtype.
__device__ __forceinline__ void store_px(const ImgView& v, int c, int x, int y, float val) {
  char* p = (char*)v.data + (long long)c * v.ps + (long long)y * v.rs;
  switch (v.dtype) {
    case HP_U8: ((unsigned char*)p)[x] = (unsigned char)val; break;
    case HP_U16: ((unsigned short*)p)[x] = (unsigned short)val; break;
    case HP_F16: ((__half*)p)[x] = __float2half_rn(val); break;
    case HP_BF16: ((__nv_bfloat16*)p)[x] = __float2bfloat16_rn(val); break;
    case HP_U32: ((unsigned int*)p)[x] = (unsigned int)val; break;
    default: ((float*)p)[x] = val;
  }
}

// ---- stencils --------------------------------------------------------------
// One pass of a separable stencil: w[0]*x[0], then fma of each later tap, in tap
// order (the x pass runs first, then the y pass over the x-pass results).
__device__ __forceinline__ float tap5(const float* w, float a, float b, float c, float d, float e) {
  float s = __fmul_rn(w[0], a);
  s = __fmaf_rn(w[1], b, s);
  s = __fmaf_rn(w[2], c, s);
  s = __fmaf_rn(w[3], d, s);
  return __fmaf_rn(w[4], e, s);
}

__device__ __forceinline__ float tap3v(float w0, float w1, float w2, float a, float b, float c) {
  float s = __fmul_rn(w0, a);
  s = __fmaf_rn(w1, b, s);
  return __fmaf_rn(w2, c, s);
}
__device__ __forceinline__ float tap3(const float* w, float a, float b, float c) {
  return tap3v(w[0], w[1], w[2], a, b, c);
}

// Binomial [1,4,6,4,1]/16 (exact in float), the per-axis taps of the pyramid
// downsample.
__device__ __forceinline__ float tap5_binomial16(float a, float b, float c, float d, float e) {
  const float w[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
  return tap5(w, a, b, c, d, e);
}

// Upsample taps per axis for fine index X: returns the number of coarse taps
// (3 for even X at m-1, m, m+1 with 1/8, 6/8, 1/8; 2 for odd X at m, m+1 with
// 1/2, 1/2), the first coarse index and the weights.
__device__ __forceinline__ int up_taps(int X, int* m0, float* w) {
  int m = X >> 1;
  if ((X & 1) == 0) {
    *m0 = m - 1; w[0] = 0.125f; w[1] = 0.75f; w[2] = 0.125f;
    return 3;
  }
  *m0 = m; w[0] = 0.5f; w[1] = 0.5f;
  return 2;
}

__device__ __forceinline__ float tapn(const float* w, const float* x, int n) {
  float s = __fmul_rn(w[0], x[0]);
  for (int i = 1; i < n; ++i) s = __fmaf_rn(w[i], x[i], s);
  return s;
}

// ---- point-wise ops --------------------------------------------------------

__device__ __forceinline__ float op_gray(float r, float g, float b, float scale) {
  float rs = __fmul_rn(r, scale), gs = __fmul_rn(g, scale), bs = __fmul_rn(b, scale);
  return __fmaf_rn(0.114f, bs, __fmaf_rn(0.587f, gs, __fmul_rn(0.299f, rs)));
}

__device__ __forceinline__ float op_harris(float sxx, float syy, float sxy, float k) {
  float det = __fmaf_rn(sxx, syy, -__fmul_rn(sxy, sxy));
  float tr = __fadd_rn(sxx, syy);
  return __fmaf_rn(-k, __fmul_rn(tr, tr), det);
}

__device__ __forceinline__ float op_unsharp(float in, float blur, float amount) {
  return __fmaf_rn(amount, __fsub_rn(in, blur), in);
}

// Paris et al. remap of intensity i around level g (sigma_r, alpha, beta):
//   |d| <= sigma: g + sign(d) sigma (|d|/sigma)^alpha;  else g + sign(d) (beta (|d| - sigma) + sigma)
// with d = i - g.  The power is CUDA's fast __powf (x = |d|/sigma lies in
// (0, 1]); both branches are evaluated and one is selected, so a warp never
// splits on the band test.
__device__ __forceinline__ float op_ll_remap(float i, float g, float sigma, float alpha, float beta) {
  const float d = __fsub_rn(i, g);
  const float ad = fabsf(d);
  const float x = __fdiv_rn(ad, sigma);
  const float inside = __fmul_rn(sigma, __powf(x, alpha));
  const float outside = __fmaf_rn(beta, __fsub_rn(ad, sigma), sigma);
  const float mag = ad <= sigma ? inside : outside;
  return ad == 0.0f ? g : __fadd_rn(g, copysignf(mag, d));
}

// The remap outside the band (|d| > sigma), bit-identical to op_ll_remap there.
__device__ __forceinline__ float op_ll_remap_outside(float d, float ad, float g, float sigma, float beta) {
  return __fadd_rn(g, copysignf(__fmaf_rn(beta, __fsub_rn(ad, sigma), sigma), d));
}

__device__ __forceinline__ float ll_level(int k, int K) { return __fdiv_rn((float)k, (float)(K - 1)); }

__device__ __forceinline__ void ll_interp_index(float gk, int K, int* k0, float* f) {
  float t = __fmul_rn(gk, (float)(K - 1));
  int k = (int)floorf(t);
  k = k > K - 2 ? K - 2 : k;
  k = k < 0 ? 0 : k;
  *k0 = k;
  *f = __fsub_rn(t, (float)k);
}

__device__ __forceinline__ float op_ll_blend(float lo, float hi, float f) {
  return __fmaf_rn(f, hi, __fmul_rn(__fsub_rn(1.0f, f), lo));
}

__device__ __forceinline__ float op_ll_colour(float in, float gray, float out_gray, float s_in, float s_out) {
  float v = __fmul_rn(in, s_in);
  float r = gray > 0.0f ? __fmul_rn(v, __fdiv_rn(out_gray, gray)) : out_gray;
  return __fmul_rn(r, s_out);
}

__device__ __forceinline__ float op_binary(int op, float a, float b) {
  switch (op) {
    case HP_OP_MUL: return __fmul_rn(a, b);
    case HP_OP_ADD: return __fadd_rn(a, b);
    default: return __fsub_rn(a, b);
  }
}

__device__ __forceinline__ float op_scale(float a, float s, float o) { return __fmaf_rn(a, s, o); }

// Interpolate app: premultiplied colour, compositing of a level over the
// upsampled coarser result, and the final division by coverage.
__device__ __forceinline__ float op_premul(float v, float a, int c) { return c < 3 ? __fmul_rn(v, a) : a; }

__device__ __forceinline__ float op_over(float front, float front_a, float back) {
  return __fmaf_rn(__fsub_rn(1.0f, front_a), back, front);
}

__device__ __forceinline__ float op_unpremul(float v, float a) { return a > 0.0f ? __fdiv_rn(v, a) : 0.0f; }

}  // namespace hp
