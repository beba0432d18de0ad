// cnn.cuh -- internal interface between the conv-stack driver (cnn.cu) and the
// tensor-core hidden-layer kernel (cnn_tc.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace acpr {

__device__ __forceinline__ float bf16r(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

// Activation after every conv but the last: tanh, or the exact (erf) GELU
// x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2)).
template <typename T>
__device__ __forceinline__ T act_apply(int act, T x) {
    if (act == AC_ACT_TANH) return tanh(x);
    return T(0.5) * x * (T(1) + erf(x * T(0.70710678118654752440)));
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
// d->mass_fix, the mACNN mass shift; zpart: batch * n^2/128 doubles of scratch.
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
// Derivative of act_apply.
template <typename T>
__device__ __forceinline__ T act_grad(int act, T x) {
    if (act == AC_ACT_TANH) {
        const T t = tanh(x);
        return T(1) - t * t;
    }
    // Phi(x) + x phi(x)
    return T(0.5) * (T(1) + erf(x * T(0.70710678118654752440))) +
           x * exp(T(-0.5) * x * x) * T(0.39894228040143267794);
}

// Device-side timeout flag of the tensor-core kernels: returns AC_ERR_TIMEOUT
// (and clears the flag) if a bounded wait gave up since the last call.
// Synchronises the stream.
int tc_check_status(cudaStream_t st);

int hidden_layer_bf16(const cnn_desc* d, int l, int n, int batch, const __nv_bfloat16* in,
                      __nv_bfloat16* out, const float* w_master, const float* bias, cudaStream_t st,
                      float* zsave = nullptr);

// Backward through hidden layer l+1 into layer l's pre-activation gradient:
// dz_out = bf16(conv(dz_next, w_t) * act'(z_prev)), w_t from pack_hidden_t.
int hidden_dgrad_bf16(int C, int act, int n, int batch, const __nv_bfloat16* dz_next, __nv_bfloat16* dz_out,
                      const __nv_bfloat16* w_t, const float* z_prev, cudaStream_t st);
int pack_hidden_t(int C, const float* w_layer, __nv_bfloat16* out, cudaStream_t st);

}  // namespace acpr
