// acnn.cuh -- internal declarations shared by acnn.cu (inference, loss, Adam,
// Algorithm 1) and acnn_train.cu (the per-layer forward/backward kernels) for
// the paper's ResBlock ACNN / mACNN coarse network (Sec. 3.2).
//
// Activation layout in HBM: channel-interleaved [field][n][n][C] (the C values
// of a pixel are contiguous, one 16-byte load for C = 4 float32); one-channel
// fields are [field][n][n].
#pragma once

#include "common.cuh"

namespace acpr {

struct AcnnIO {              // where field b of a batch lives
    const int* in_map;       // nullptr: field b at b * in_bs
    const int* out_map;
    long long in_bs, out_bs; // elements between consecutive fields
};

__device__ __forceinline__ long long acnn_sel(const int* map, int b) { return map ? map[b] : b; }

// tanh of the network.  float: the identity tanh x = 1 - 2 / (1 + e^{2x}) on
// the fast exponential and divide intrinsics (absolute error below 1e-6, exact
// limits +-1 for large |x|); double: the library tanh.
__device__ __forceinline__ float acnn_tanh(float x) { return 1.0f - __fdividef(2.0f, 1.0f + __expf(2.0f * x)); }
__device__ __forceinline__ double acnn_tanh(double x) { return tanh(x); }

inline int acnn_convs(int blocks) { return 2 + 2 * blocks; }

inline void acnn_dims(int C, int blocks, int l, int* cin, int* cout) {
    *cin = l == 0 ? 1 : C;
    *cout = l == acnn_convs(blocks) - 1 ? 1 : C;
}

// Offsets of conv l's weights and biases in the concatenated parameter arrays.
inline void acnn_offsets(int C, int blocks, int l, long long* wo, long long* bo) {
    long long w = 0, b = 0;
    for (int i = 0; i < l; ++i) {
        int ci, co;
        acnn_dims(C, blocks, i, &ci, &co);
        w += 9LL * ci * co;
        b += co;
    }
    *wo = w;
    *bo = b;
}

int acnn_check(const acnn_desc* d);

// Per-layer training path (acnn_train.cu).
size_t acnn_train_bytes_for(const acnn_desc* d, int n, int batch);
int acnn_forward_train_impl(const acnn_desc* d, int n, int batch, const void* u, void* out, void* ws,
                            cudaStream_t st);
int acnn_backward_impl(const acnn_desc* d, int n, int batch, const void* u, const void* gout, void* gw, void* gb,
                       void* ws, cudaStream_t st);

// Forward through the per-layer kernels for shapes the fused kernel does not
// cover (weights read from device memory); ws as for training.
int acnn_forward_layers(const acnn_desc* d, int n, int batch, const void* u, void* out, AcnnIO io, void* ws,
                        cudaStream_t st);

// Mass shift and limiter of a finished output conv: per-field sums of
// (out - in) reduced from `part` ([batch][parts] float64, written by the
// producing kernel), then out = clamp(out + shift).  Launched by both paths.
// With s_save (contiguous [batch][n][n]) the value before the clamp is kept
// there for the backward pass.
template <typename T>
int acnn_post(int n, int batch, const T* u, T* out, AcnnIO io, const double* part, int parts, int mass_fix,
              int limiter, double lo, double hi, cudaStream_t st, T* s_save = nullptr);

int acnn_precision(const acnn_net* net);

// acnn_forward with mapped fields (the Parareal driver's coarse sweeps).
int acnn_forward_mapped(const acnn_net* net, int n, int batch, const void* u, long long in_bs, const int* in_map,
                        void* out, long long out_bs, const int* out_map, void* work, size_t work_bytes,
                        cudaStream_t st);

}  // namespace acpr
