// cnn_tc.cu -- hidden C -> C conv layers of the coarse propagator on tcgen05.
#include "cnn.cuh"

namespace acpr {

// float32 master W[cout][cin][3][3] -> bf16 [tap][cin/8][cout][8]
__global__ void pack_hidden_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ out, int C) {
    const int total = 9 * C * C;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int i = idx % 8;
        const int o = (idx / 8) % C;
        const int kc = (idx / (8 * C)) % (C / 8);
        const int tap = idx / (8 * C * (C / 8));
        const int c = kc * 8 + i;
        out[idx] = __float2bfloat16_rn(w[(o * C + c) * 9 + tap]);
    }
}

size_t packed_hidden_bytes(const cnn_desc* d) {
    const int hidden = d->layers - 2;
    return size_t(hidden > 0 ? hidden : 0) * 9 * d->channels * d->channels * sizeof(__nv_bfloat16);
}

int pack_hidden_weights(const cnn_desc* d, cudaStream_t st) {
    const int C = d->channels;
    const float* w = static_cast<const float*>(d->w);
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(d->packed);
    size_t woff = size_t(C) * 9;
    for (int l = 1; l < d->layers - 1; ++l) {
        pack_hidden_kernel<<<64, 256, 0, st>>>(w + woff, p + size_t(l - 1) * 9 * C * C, C);
        ACPR_LAUNCH_CHECK();
        woff += size_t(C) * C * 9;
    }
    return AC_OK;
}

int hidden_layer_bf16(const cnn_desc*, int, int, int, const __nv_bfloat16*, __nv_bfloat16*,
                      const float*, const float*, cudaStream_t) {
    return AC_ERR_UNSUPPORTED;
}

}  // namespace acpr
