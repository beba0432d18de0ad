// cnn.cuh -- internal interface between the conv-stack driver (cnn.cu) and the
// tensor-core hidden-layer kernel (cnn_tc.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace acpr {

__device__ __forceinline__ float bf16r(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

// Standard normal CDF Phi(x) in float32 from the rational approximation of
// Abramowitz & Stegun, Handbook of Mathematical Functions, eq. 7.1.26 (after
// Hastings): for z >= 0, erfc(z) = t (a1 + t (a2 + t (a3 + t (a4 + t a5))))
// exp(-z^2) + e(z), t = 1 / (1 + p z), |e(z)| <= 1.5e-7.  With z = |x| / sqrt 2,
// Phi(-|x|) = erfc(z) / 2 and Phi(|x|) = 1 - Phi(-|x|): the negative tail is
// formed without the cancellation of 1 + erf.  Absolute error about 1e-7,
// far under the bf16 rounding the activations then take, in about a third of
// the instructions of 0.5 (1 + erff(x / sqrt 2)).
__device__ __forceinline__ float phi_as(float x) {
    const float z = fabsf(x) * 0.70710678118654752440f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
    float p = fmaf(t, 1.061405429f, -1.453152027f);
    p = fmaf(t, p, 1.421413741f);
    p = fmaf(t, p, -0.284496736f);
    p = fmaf(t, p, 0.254829592f);
    const float q = 0.5f * (p * t) * __expf(-z * z);  // Phi(-|x|)
    return x >= 0.0f ? 1.0f - q : q;
}

// Paired float32 arithmetic: two lanes in one 64-bit register, operated on by
// the sm_100-family .f32x2 instructions (one issue for two results), each
// lane rounded exactly as the scalar add / mul / fma.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2split(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// Hardware approximations: 1/x and 2^x (PTX rcp.approx, ex2.approx).
__device__ __forceinline__ float rcp_hw(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_hw(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// GELU x Phi(x) of two lanes with the paired instructions: the same
// Abramowitz & Stegun 7.1.26 form as phi_as, q = Phi(-|x|) = erfc(z)/2 with
// the 1/2 folded into the coefficients (exact: a power of two) and
// exp(-z^2) = 2^(-x^2 log2(e) / 2); then x Phi(x) = max(x, 0) - |x| q for
// either sign of x.
__device__ __forceinline__ f32x2 gelu2(f32x2 x) {
    float x0, x1;
    f2split(x, x0, x1);
    const f32x2 nx = f2(-fabsf(x0), -fabsf(x1));
    const f32x2 rx = f2(fmaxf(x0, 0.0f), fmaxf(x1, 0.0f));
    const f32x2 z = f2_mul(nx, f2(-0.70710678118654752440f, -0.70710678118654752440f));
    float d0, d1;
    f2split(f2_fma(z, f2(0.3275911f, 0.3275911f), f2(1.0f, 1.0f)), d0, d1);
    const f32x2 t = f2(rcp_hw(d0), rcp_hw(d1));
    f32x2 p = f2_fma(t, f2(0.5307027145f, 0.5307027145f), f2(-0.7265760135f, -0.7265760135f));
    p = f2_fma(t, p, f2(0.7107068705f, 0.7107068705f));
    p = f2_fma(t, p, f2(-0.142248368f, -0.142248368f));
    p = f2_fma(t, p, f2(0.127414796f, 0.127414796f));
    float w0, w1;  // -x^2 log2(e) / 2
    f2split(f2_mul(f2_mul(x, x), f2(-0.72134752044448170368f, -0.72134752044448170368f)), w0, w1);
    const f32x2 q = f2_mul(f2_mul(p, t), f2(ex2_hw(w0), ex2_hw(w1)));  // Phi(-|x|)
    return f2_fma(nx, q, rx);
}

// One lane of gelu2 with the same roundings (scalar kernels and the paired
// ones give the same bits for the same input).
__device__ __forceinline__ float gelu1(float x) {
    const float nx = -fabsf(x);
    const float z = __fmul_rn(nx, -0.70710678118654752440f);
    const float t = rcp_hw(__fmaf_rn(z, 0.3275911f, 1.0f));
    float p = __fmaf_rn(t, 0.5307027145f, -0.7265760135f);
    p = __fmaf_rn(t, p, 0.7107068705f);
    p = __fmaf_rn(t, p, -0.142248368f);
    p = __fmaf_rn(t, p, 0.127414796f);
    const float q = __fmul_rn(__fmul_rn(p, t), ex2_hw(__fmul_rn(__fmul_rn(x, x), -0.72134752044448170368f)));
    return __fmaf_rn(nx, q, fmaxf(x, 0.0f));
}

// Activation after every conv but the last: tanh, or GELU x * Phi(x)
// (float32: gelu1 / gelu2; float64: 0.5 (1 + erf(x / sqrt 2))).
__device__ __forceinline__ float act_apply_gelu(float x) { return gelu1(x); }
__device__ __forceinline__ double act_apply_gelu(double x) {
    return 0.5 * x * (1.0 + erf(x * 0.70710678118654752440));
}

template <typename T>
__device__ __forceinline__ T act_apply(int act, T x) {
    if (act == AC_ACT_TANH) return tanh(x);
    return act_apply_gelu(x);
}

// The activation fixed at compile time (kernels instantiated per activation,
// so that no code of the other one sits in their loops).
template <int ACT>
__device__ __forceinline__ float act_c(float x) {
    if constexpr (ACT == AC_ACT_TANH) return tanhf(x);
    else return act_apply_gelu(x);
}

// act_c of two lanes (GELU with the paired instructions).
template <int ACT>
__device__ __forceinline__ f32x2 act2(f32x2 x) {
    if constexpr (ACT == AC_ACT_TANH) {
        float a, b;
        f2split(x, a, b);
        return f2(tanhf(a), tanhf(b));
    } else {
        return gelu2(x);
    }
}

int check_cnn(const cnn_desc* d);
int coarse_step(const cnn_desc* d, int n, int batch, const void* u_in, void* u_out, cudaStream_t st);
// Batch entry b reads the field at u_in + in_map[b] * in_bs and writes the
// field at u_out + out_map[b] * out_bs (a NULL map means b; strides in
// elements).
int coarse_step_mapped(const cnn_desc* d, int n, int batch, const void* u_in, long long in_bs,
                       const int* in_map, void* u_out, long long out_bs, const int* out_map,
                       cudaStream_t st);
size_t work_bytes_for(const cnn_desc* d, int n, int batch);
// Last conv layer (C -> 1, residual) of the AC_F32 path and, with
// d->mass_fix, the mACNN mass shift; zpart: batch * max(1, n^2/256) doubles of
// scratch (one per block of the last layer).
int last_layer_bf16(const cnn_desc* d, int n, int batch, const __nv_bfloat16* a, float* out, const float* W,
                    const float* Bv, const float* u, double* zpart, cudaStream_t st);

// Packed bf16 weights of the hidden C -> C layers, per layer
// [tap 9][k-chunk C/8][cout C][8 input channels] (the K-major core-matrix
// layout of the tcgen05 B operand).
size_t packed_hidden_bytes(const cnn_desc* d);
int pack_hidden_weights(const cnn_desc* d, cudaStream_t st);

// Hidden layer l (1 <= l <= layers - 2) on the tensor cores:
// in/out are [batch][C/8][n][n][8] bf16.  Returns AC_ERR_UNSUPPORTED when the
// shape has no tensor-core kernel.
// Derivative of act_apply: 1 - tanh^2, or Phi(x) + x phi(x).
__device__ __forceinline__ float act_grad_gelu(float x) {
    return phi_as(x) + x * __expf(-0.5f * x * x) * 0.39894228040143267794f;
}
__device__ __forceinline__ double act_grad_gelu(double x) {
    return 0.5 * (1.0 + erf(x * 0.70710678118654752440)) + x * exp(-0.5 * x * x) * 0.39894228040143267794;
}

template <typename T>
__device__ __forceinline__ T act_grad(int act, T x) {
    if (act == AC_ACT_TANH) {
        const T t = tanh(x);
        return T(1) - t * t;
    }
    return act_grad_gelu(x);
}

template <int ACT>
__device__ __forceinline__ float act_grad_c(float x) {
    if constexpr (ACT == AC_ACT_TANH) {
        const float t = tanhf(x);
        return 1.0f - t * t;
    } else {
        return act_grad_gelu(x);
    }
}

// Every conv workspace (cnn_desc.work and the training workspace) starts
// with a header of kConvHeader bytes whose first int is the status word of
// the tensor-core kernels: a bounded wait that gives up stores a nonzero code
// there.  The header must be zero when the workspace is first used.
constexpr size_t kConvHeader = 256;
inline int* conv_status(void* ws) { return static_cast<int*>(ws); }

// AC_ERR_TIMEOUT (and the word cleared) if a bounded wait gave up since the
// last check of this status word.  Synchronises the stream.
int conv_check_status(int* status, cudaStream_t st);
// The same, unless `st` is being captured into a graph (then AC_OK: the
// graph's owner checks after a replay).
int conv_check_status_uncaptured(int* status, cudaStream_t st);
// Test hook: with polls > 0 the persistent tensor-core kernels' MMA issuer
// waits on an mbarrier that nothing arrives on, for `polls` polls.
void set_test_stall(int polls);

int hidden_layer_bf16(const cnn_desc* d, int l, int n, int batch, const __nv_bfloat16* in,
                      __nv_bfloat16* out, const float* w_master, const float* bias, int* status, cudaStream_t st,
                      float* zsave = nullptr);

// The last hidden layer (l = layers - 2) fused with the last layer's
// per-pixel projection (persistent tensor-core kernel, C = 32 or 64, n a
// multiple of 128): maps [batch][9][n][n] float32 receives, per pixel, the
// nine tap sums of W_last (bf16-rounded) with the layer's bf16 activations;
// act_out gets the activations and zsave the pre-activations only when zsave
// is not NULL (training).  AC_ERR_UNSUPPORTED for other shapes.
// Shapes of the persistent row-streaming kernel for (n, C) that a tuner may
// choose (input-ring depth, TMEM slots).
int conv_variant_count(int n, int C);
int conv_variant_describe(int n, int C, int index, int* ring, int* slots);
int conv_set_variant(int n, int C, int index);  // -1: automatic
int conv_get_variant(int n, int C);

// Weight gradient of a hidden C -> C layer on the tensor cores (C = 64, n a
// multiple of 128): writes the weight partials part[chunk][tap][co][ci] and
// the bias partials part[chunk][0][C*C + co] of `chunks` pixel chunks, for
// the fixed-order reduction of the CUDA-core path.  set_wgrad_tc(false)
// selects the CUDA-core path everywhere (tests).
void set_wgrad_tc(bool on);
bool wgrad_tc_supported(int C, int n);
int wgrad_tc_partials(int n, int batch, const __nv_bfloat16* a, const __nv_bfloat16* dz, float* part, int chunks,
                      int* status, cudaStream_t st);

bool hidden_last_fused_supported(int n, int C);
int hidden_last_fused(const cnn_desc* d, int l, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* act_out,
                      const float* bias, const float* w_last, float* maps, int* status, cudaStream_t st,
                      float* zsave = nullptr);
// The last layer from those maps: out = bias + sum_tap maps[tap](shifted) (+ u
// with the residual), the mass-shift block partials into zpart as
// last_layer_bf16, then (d->mass_fix) the shift itself.
int last_stencil_f32(const cnn_desc* d, int n, int batch, const float* maps, float* out, const float* Bv,
                     const float* u, double* zpart, cudaStream_t st);

// Backward through hidden layer l+1 into layer l's pre-activation gradient:
// dz_out = bf16(conv(dz_next, w_t) * act'(z_prev)), w_t from pack_hidden_t.
int hidden_dgrad_bf16(int C, int act, int n, int batch, const __nv_bfloat16* dz_next, __nv_bfloat16* dz_out,
                      const __nv_bfloat16* w_t, const float* z_prev, int* status, cudaStream_t st);
int pack_hidden_t(int C, const float* w_layer, __nv_bfloat16* out, cudaStream_t st);

}  // namespace acpr
