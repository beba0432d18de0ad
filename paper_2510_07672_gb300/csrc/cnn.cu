// cnn.cu -- the coarse propagator G (Sec. 3.2): a stack of 3x3 circular-padded
// convolutions 1 -> C -> ... -> C -> 1 with an activation after every layer but
// the last and a global residual connection, plus the optional mACNN mass
// shift and bound limiter.
//
// Two numeric paths:
//   AC_F64: float64 fields, weights and activations; planar [B][C][N][N]
//           hidden activations; CUDA-core direct convolution.
//   AC_F32: float32 fields; bf16 conv operands with float32 accumulation;
//           hidden activations stored as bf16 in the channel-chunked layout
//           [B][C/8][N][N][8] (16 bytes per pixel and chunk), the layout the
//           tensor-core layer kernel (cnn_tc.cu) consumes.  The first layer
//           (1 -> C, K = 9) and the last (C -> 1) run on CUDA cores; the
//           hidden C -> C layers run on tcgen05 (cnn_tc.cu) when available.
#include <cuda_bf16.h>

#include "cnn.cuh"
#include "common.cuh"

namespace acpr {

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------- float64 --
// One thread per output pixel, all output channels.
// Batch entry b of the input field starts at in + fi(b) * in_bs with
// fi(b) = in_map ? in_map[b] : b; the output field at out + fo(b) * out_bs with
// fo(b) = out_map ? out_map[b] : b.  Hidden activations are compact
// ([b][C]...).  in_mapped / out_mapped tell a layer whether its own input /
// output is a field (first / last layer) or an activation tensor.
struct BatchIO {
    const int* in_map;
    const int* out_map;
    long long in_bs, out_bs;
    int in_mapped, out_mapped;
};

__device__ __forceinline__ long long bsel(const int* map, int b) { return map ? map[b] : b; }

template <int COUT_MAX>
__global__ void conv_f64_kernel(const double* __restrict__ in, double* __restrict__ out,
                                const double* __restrict__ W, const double* __restrict__ bias,
                                int batch, int n, int cin, int cout, int act, int apply_act,
                                const double* __restrict__ resid, BatchIO io) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (pix >= nn * batch) return;
    const int b = int(pix / nn);
    const int y = int((pix % nn) / n), x = int(pix % n);
    const long long fi = bsel(io.in_map, b), fo = bsel(io.out_map, b);
    const double* inb = io.in_mapped ? in + fi * io.in_bs : in + (long long)b * cin * nn;
    double* outb = io.out_mapped ? out + fo * io.out_bs : out + (long long)b * cout * nn;
    double acc[COUT_MAX];
    for (int o = 0; o < cout; ++o) acc[o] = bias[o];
    for (int c = 0; c < cin; ++c) {
        const double* plane = inb + (long long)c * nn;
        double v[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int e = 0; e < 3; ++e) v[a * 3 + e] = plane[(long long)wrap(y + a - 1, n) * n + wrap(x + e - 1, n)];
        for (int o = 0; o < cout; ++o) {
            const double* w = W + ((long long)o * cin + c) * 9;
            double s = acc[o];
#pragma unroll
            for (int t = 0; t < 9; ++t) s += w[t] * v[t];
            acc[o] = s;
        }
    }
    for (int o = 0; o < cout; ++o) {
        double z = acc[o];
        if (apply_act) z = act_apply<double>(act, z);
        if (resid) z += resid[fi * io.in_bs + (long long)y * n + x];
        outb[(long long)o * nn + (long long)y * n + x] = z;
    }
}

// ------------------------------------------------------------ bf16 / f32 --
// First layer: float32 field -> bf16 chunked activations (K = 9 on CUDA cores).
// The bf16-rounded weights and the biases are staged in shared memory once per
// block (every thread reads the same entry: broadcast).  A thread computes two
// horizontally adjacent pixels (one weight load serves both), each output as
// the sum over taps in order, then the bias.
constexpr int kFirstPx = 2;
template <int C, int ACT>
__global__ void conv_first_bf16_kernel(const float* __restrict__ u, __nv_bfloat16* __restrict__ act,
                                       const float* __restrict__ W, const float* __restrict__ bias,
                                       int batch, int n, BatchIO io) {
    __shared__ float ws[C * 9], bs[C];
    for (int i = threadIdx.x; i < C * 9; i += blockDim.x) ws[i] = bf16r(W[i]);
    for (int i = threadIdx.x; i < C; i += blockDim.x) bs[i] = bias[i];
    __syncthreads();
    const long long pix = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * kFirstPx;
    const long long nn = (long long)n * n;
    if (pix >= nn * batch) return;
    const int lg = __ffs(n) - 1;  // n is a power of two
    const int b = int(pix >> (2 * lg));
    const int y = int(pix >> lg) & (n - 1), x = int(pix) & (n - 1);
    const float* f = u + bsel(io.in_map, b) * io.in_bs;
    float v[3][kFirstPx + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int e = 0; e < kFirstPx + 2; ++e)
            v[a][e] = bf16r(f[(long long)wrap(y + a - 1, n) * n + wrap(x + e - 1, n)]);
    static_assert(kFirstPx == 2, "the two pixels of a thread are the lanes of the paired instructions");
    f32x2 vp[3][3];  // the window of the pair: vp[dy][dx] = (v[dy][dx], v[dy][dx + 1])
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int e = 0; e < 3; ++e) vp[a][e] = f2(v[a][e], v[a][e + 1]);
#pragma unroll
    for (int kc = 0; kc < C / 8; ++kc) {
        __align__(16) __nv_bfloat16 o8[kFirstPx][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int o = kc * 8 + i;
            f32x2 s2 = f2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < 9; ++t) s2 = f2_fma(f2(ws[o * 9 + t], ws[o * 9 + t]), vp[t / 3][t % 3], s2);
            float a0, a1;
            f2split(act2<ACT>(f2_add(s2, f2(bs[o], bs[o]))), a0, a1);
            o8[0][i] = __float2bfloat16_rn(a0);
            o8[1][i] = __float2bfloat16_rn(a1);
        }
#pragma unroll
        for (int px = 0; px < kFirstPx; ++px)
            *reinterpret_cast<uint4*>(act + ((((long long)b * (C / 8) + kc) * nn) + ((pix + px) & (nn - 1))) * 8) =
                *reinterpret_cast<const uint4*>(o8[px]);
    }
}

// Hidden layer C -> C (CUDA-core path).  w: float32 masters [C][C][3][3].
template <int C>
__global__ void conv_hidden_bf16_cc_kernel(const __nv_bfloat16* __restrict__ in,
                                           __nv_bfloat16* __restrict__ out,
                                           const float* __restrict__ W,
                                           const float* __restrict__ bias, int batch, int n,
                                           int act_kind) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (pix >= nn * batch) return;
    const int b = int(pix / nn);
    const int y = int((pix % nn) / n), x = int(pix % n);
    float acc[C];
#pragma unroll
    for (int o = 0; o < C; ++o) acc[o] = 0.f;
    for (int kc = 0; kc < C / 8; ++kc) {
        const __nv_bfloat16* plane = in + ((long long)b * (C / 8) + kc) * nn * 8;
        for (int t = 0; t < 9; ++t) {
            const int yy = wrap(y + t / 3 - 1, n), xx = wrap(x + t % 3 - 1, n);
            const uint4 raw = *reinterpret_cast<const uint4*>(plane + ((long long)yy * n + xx) * 8);
            const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&raw);
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __bfloat162float(v8[i]);
#pragma unroll
            for (int o = 0; o < C; ++o) {
                float s = acc[o];
#pragma unroll
                for (int i = 0; i < 8; ++i) s = fmaf(bf16r(__ldg(W + ((o * C + kc * 8 + i) * 9 + t))), v[i], s);
                acc[o] = s;
            }
        }
    }
#pragma unroll
    for (int kc = 0; kc < C / 8; ++kc) {
        __align__(16) __nv_bfloat16 o8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            o8[i] = __float2bfloat16_rn(act_apply<float>(act_kind, acc[kc * 8 + i] + bias[kc * 8 + i]));
        *reinterpret_cast<uint4*>(out + ((((long long)b * (C / 8) + kc) * nn) + pix % nn) * 8) =
            *reinterpret_cast<const uint4*>(o8);
    }
}

// Last layer C -> 1 with the residual add in float32.  A block covers
// ppb = last_pixels(n) consecutive pixels of one field: nr = ppb / w rows of
// w = min(n, 256) columns starting at (y0, x0).  It first stages the input
// rows y0 - 1 .. y0 + nr (wrapped) over columns x0 - 1 .. x0 + w (wrapped), all
// C/8 chunk planes, and the bf16-rounded weights in shared memory, then one
// thread per pixel sums over (chunk, tap, channel) in that order.
// With zpart != NULL every block also writes the float64 sum of its stack
// outputs z (before the residual) to zpart[blockIdx.x], one warp adding the
// block's values in a fixed order (float64 arithmetic is scarce on this GPU:
// about one add per pixel, not one per thread and shuffle step).
constexpr int kLastThreads = 256;
template <int C>
__global__ void __launch_bounds__(kLastThreads)
conv_last_bf16_kernel(const __nv_bfloat16* __restrict__ in, float* __restrict__ out, const float* __restrict__ W,
                      const float* __restrict__ bias, const float* __restrict__ u, int batch, int n, int residual,
                      BatchIO io, double* __restrict__ zpart) {
    constexpr int KC = C / 8;
    extern __shared__ __align__(16) unsigned char lsm[];
    float* ws = reinterpret_cast<float*>(lsm);                       // [kc][tap][8]
    float* zsh = ws + C * 9;                                          // [ppb]
    uint4* tile = reinterpret_cast<uint4*>(zsh + kLastThreads);       // [nr + 2][KC][w + 2]
    const long long nn = (long long)n * n;
    const int ppb = int(nn < kLastThreads ? nn : kLastThreads);
    const int w = n < kLastThreads ? n : kLastThreads;
    const int nr = ppb / w;
    const long long p0 = (long long)blockIdx.x * ppb;
    const int b = int(p0 / nn);
    const int q0 = int(p0 % nn);
    const int y0 = q0 / n, x0 = q0 % n;
    for (int i = threadIdx.x; i < C * 9; i += blockDim.x) {
        const int e = i % 8, t = (i / 8) % 9, kc = i / 72;
        ws[i] = bf16r(W[(kc * 8 + e) * 9 + t]);
    }
    const __nv_bfloat16* ib = in + (long long)b * KC * nn * 8;
    const int tw = w + 2;
    for (int r = 0; r < nr + 2; ++r) {
        const int yy = wrap(y0 - 1 + r, n);
        for (int kc = 0; kc < KC; ++kc) {
            const uint4* src = reinterpret_cast<const uint4*>(ib + ((long long)kc * nn + (long long)yy * n) * 8);
            uint4* dst = tile + (r * KC + kc) * tw;
            for (int xx = threadIdx.x; xx < tw; xx += blockDim.x) dst[xx] = src[wrap(x0 - 1 + xx, n)];
        }
    }
    __syncthreads();
    const int tp = threadIdx.x;
    const bool valid = tp < ppb;
    float zs = 0.f;
    if (valid) {
        const int ry = tp / w, cx = tp % w;
        float acc = 0.f;
        for (int kc = 0; kc < KC; ++kc) {
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const uint4 raw = tile[((ry + t / 3) * KC + kc) * tw + cx + t % 3];
                const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&raw);
                const float4 w0 = reinterpret_cast<const float4*>(ws)[(kc * 9 + t) * 2];
                const float4 w1 = reinterpret_cast<const float4*>(ws)[(kc * 9 + t) * 2 + 1];
                const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int e = 0; e < 8; ++e) acc = fmaf(wv[e], __bfloat162float(v8[e]), acc);
            }
        }
        zs = acc + bias[0];
        const long long q = (long long)(y0 + ry) * n + x0 + cx;
        float z = zs;
        if (residual) z += u[bsel(io.in_map, b) * io.in_bs + q];
        out[bsel(io.out_map, b) * io.out_bs + q] = z;
    }
    if (zpart) {
        zsh[tp] = valid ? zs : 0.f;
        __syncthreads();
        if (tp < 32) {
            double v = 0.0;
            for (int i = tp; i < ppb; i += 32) v += double(zsh[i]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tp == 0) zpart[blockIdx.x] = v;
        }
    }
}

template <int C>
static size_t last_smem(int n) {
    const long long nn = (long long)n * n;
    const int ppb = int(nn < kLastThreads ? nn : kLastThreads);
    const int w = n < kLastThreads ? n : kLastThreads;
    const int nr = ppb / w;
    return sizeof(float) * (C * 9 + kLastThreads) + sizeof(uint4) * size_t(nr + 2) * (C / 8) * (w + 2);
}

// Last layer C -> 1 from the nine tap maps of the fused last hidden layer:
// z = (sum over taps (dy, dx) of maps[tap] at (y + dy - 1, x + dx - 1), wrapped)
// + bias, out = z (+ u), and the block's float64 sum of z when zpart != NULL
// (one block = last_pixels(n) pixels of one field, as conv_last_bf16_kernel).
__global__ void __launch_bounds__(kLastThreads)
last_stencil_kernel(const float* __restrict__ maps, float* __restrict__ out, const float* __restrict__ bias,
                    const float* __restrict__ u, int batch, int n, int residual, BatchIO io,
                    double* __restrict__ zpart) {
    __shared__ float zsh[kLastThreads];
    const long long nn = (long long)n * n;
    const int ppb = int(nn < kLastThreads ? nn : kLastThreads);
    const long long p0 = (long long)blockIdx.x * ppb;
    const int b = int(p0 / nn);
    const int tp = threadIdx.x;
    const bool valid = tp < ppb;
    float zs = 0.f;
    if (valid) {
        const long long q = p0 % nn + tp;
        const int y = int(q / n), x = int(q % n);
        const float* mb = maps + (long long)b * 9 * nn;
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < 9; ++t)
            acc += mb[t * nn + (long long)wrap(y + t / 3 - 1, n) * n + wrap(x + t % 3 - 1, n)];
        zs = acc + bias[0];
        float z = zs;
        if (residual) z += u[bsel(io.in_map, b) * io.in_bs + q];
        out[bsel(io.out_map, b) * io.out_bs + q] = z;
    }
    if (zpart) {
        zsh[tp] = valid ? zs : 0.f;
        __syncthreads();
        if (tp < 32) {
            double v = 0.0;
            for (int i = tp; i < ppb; i += 32) v += double(zsh[i]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tp == 0) zpart[blockIdx.x] = v;
        }
    }
}

// mACNN mass shift from the stack-output sums: out += -(sum z) / n^2 per
// field.  Grid (chunks, batch); each block forms the field's sum from its
// `bpf` block partials in a fixed order (deterministic), then shifts a chunk.
constexpr int kMassThreads = 256;
__global__ void mass_apply_kernel(float* __restrict__ out, const double* __restrict__ zpart, int bpf, int n,
                                  BatchIO io) {
    const long long nn = (long long)n * n;
    const int b = blockIdx.y;
    __shared__ double red[kMassThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < bpf; i += kMassThreads) s += zpart[(long long)b * bpf + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kMassThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const float shift = float(-red[0] / double(nn));
    float* ob = out + bsel(io.out_map, b) * io.out_bs;
    for (long long i = (long long)blockIdx.x * kMassThreads + threadIdx.x; i < nn;
         i += (long long)gridDim.x * kMassThreads)
        ob[i] += shift;
}

// mACNN mass shift then bound limiter, one block per field (deterministic
// float64 reduction of mean(u) - mean(out) in a fixed order).
template <typename T>
__global__ void post_kernel(const T* __restrict__ u, T* __restrict__ out, int n, int mass_fix,
                            int limiter, double lo, double hi, BatchIO io) {
    const long long nn = (long long)n * n;
    const T* ub = u + bsel(io.in_map, blockIdx.x) * io.in_bs;
    T* ob = out + bsel(io.out_map, blockIdx.x) * io.out_bs;
    __shared__ double red[32];
    double shift = 0.0;
    if (mass_fix) {
        double s = 0.0;
        for (long long i = threadIdx.x; i < nn; i += blockDim.x) s += double(ub[i]) - double(ob[i]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
            red[0] = t / double(nn);
        }
        __syncthreads();
        shift = red[0];
    }
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
        double v = double(ob[i]) + shift;
        if (limiter) v = v < lo ? lo : (v > hi ? hi : v);
        ob[i] = T(v);
    }
}

// ------------------------------------------------------------------ host --
static void layer_dims(const cnn_desc* d, int l, int* cin, int* cout) {
    *cin = l == 0 ? 1 : d->channels;
    *cout = l == d->layers - 1 ? 1 : d->channels;
}

int check_cnn(const cnn_desc* d) {
    ACPR_CHECK_ARG(d != nullptr, "cnn_desc is NULL");
    ACPR_CHECK_ARG(d->layers >= 2, "need at least 2 layers (1 -> C -> 1), got %d", d->layers);
    ACPR_CHECK_ARG(d->precision == AC_F64 || d->precision == AC_F32, "bad cnn precision");
    ACPR_CHECK_ARG(d->act == AC_ACT_TANH || d->act == AC_ACT_GELU, "bad activation %d", d->act);
    ACPR_CHECK_ARG(d->w && d->b, "null weight pointer");
    if (d->precision == AC_F64) {
        ACPR_CHECK_ARG(d->channels >= 1 && d->channels <= 64, "AC_F64 channels must be 1..64");
    } else if (!(d->channels == 16 || d->channels == 32 || d->channels == 64)) {
        set_error("AC_F32 conv: channels must be 16, 32 or 64 (got %d)", d->channels);
        return AC_ERR_UNSUPPORTED;
    }
    return AC_OK;
}

// Pixels per block of the last layer (a power of two dividing n^2, so a block
// never spans two fields).
static int last_pixels(int n) { return n * n >= kLastThreads ? kLastThreads : n * n; }

size_t work_bytes_for(const cnn_desc* d, int n, int batch) {
    const size_t act = size_t(batch) * d->channels * n * n * (d->precision == AC_F64 ? 8 : 2);
    const size_t zpart = size_t(batch) * (size_t(n) * n / last_pixels(n)) * sizeof(double);
    return kConvHeader + 2 * act + zpart;
}

// Last layer and (if d->mass_fix) the mass shift, for the AC_F32 path.
template <int C>
static int last_layer_f32(const cnn_desc* d, int n, int batch, const __nv_bfloat16* a, float* out,
                          const float* W, const float* Bv, const float* u, const BatchIO& io, double* zpart,
                          cudaStream_t st) {
    const int ppb = last_pixels(n);
    const long long pixels = (long long)n * n * batch;
    const unsigned blocks = unsigned(pixels / ppb);
    const size_t smem = last_smem<C>(n);
    static bool configured = false;
    if (!configured) {
        ACPR_CUDA(cudaFuncSetAttribute(conv_last_bf16_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(last_smem<C>(256))));
        configured = true;
    }
    conv_last_bf16_kernel<C><<<blocks, kLastThreads, smem, st>>>(a, out, W, Bv, u, batch, n, d->residual, io,
                                                                 d->mass_fix ? zpart : nullptr);
    ACPR_LAUNCH_CHECK();
    if (d->mass_fix) {
        const int bpf = int((long long)n * n / ppb);
        const long long chunks = ((long long)n * n + kMassThreads * 8 - 1) / (kMassThreads * 8);
        mass_apply_kernel<<<dim3(unsigned(chunks), unsigned(batch)), kMassThreads, 0, st>>>(out, zpart, bpf, n, io);
        ACPR_LAUNCH_CHECK();
    }
    return AC_OK;
}

int last_layer_bf16(const cnn_desc* d, int n, int batch, const __nv_bfloat16* a, float* out, const float* W,
                    const float* Bv, const float* u, double* zpart, cudaStream_t st) {
    BatchIO io{nullptr, nullptr, (long long)n * n, (long long)n * n, 1, 1};
    switch (d->channels) {
        case 16: return last_layer_f32<16>(d, n, batch, a, out, W, Bv, u, io, zpart, st);
        case 32: return last_layer_f32<32>(d, n, batch, a, out, W, Bv, u, io, zpart, st);
        default: return last_layer_f32<64>(d, n, batch, a, out, W, Bv, u, io, zpart, st);
    }
}

static int last_stencil_io(const cnn_desc* d, int n, int batch, const float* maps, float* out, const float* Bv,
                           const float* u, const BatchIO& io, double* zpart, cudaStream_t st) {
    const int ppb = last_pixels(n);
    const unsigned blocks = unsigned((long long)n * n * batch / ppb);
    last_stencil_kernel<<<blocks, kLastThreads, 0, st>>>(maps, out, Bv, u, batch, n, d->residual, io,
                                                         d->mass_fix ? zpart : nullptr);
    ACPR_LAUNCH_CHECK();
    if (d->mass_fix) {
        const int bpf = int((long long)n * n / ppb);
        const long long chunks = ((long long)n * n + kMassThreads * 8 - 1) / (kMassThreads * 8);
        mass_apply_kernel<<<dim3(unsigned(chunks), unsigned(batch)), kMassThreads, 0, st>>>(out, zpart, bpf, n, io);
        ACPR_LAUNCH_CHECK();
    }
    return AC_OK;
}

int last_stencil_f32(const cnn_desc* d, int n, int batch, const float* maps, float* out, const float* Bv,
                     const float* u, double* zpart, cudaStream_t st) {
    BatchIO io{nullptr, nullptr, (long long)n * n, (long long)n * n, 1, 1};
    return last_stencil_io(d, n, batch, maps, out, Bv, u, io, zpart, st);
}

template <int C>
static int run_f32(const cnn_desc* d, int n, int batch, const float* u, float* out, const BatchIO& io,
                   cudaStream_t st) {
    const long long pixels = (long long)n * n * batch;
    const int threads = 128;
    const unsigned blocks = unsigned((pixels + threads - 1) / threads);
    const float* W = static_cast<const float*>(d->w);
    const float* Bv = static_cast<const float*>(d->b);
    const size_t act_elems = size_t(batch) * C * n * n;
    unsigned char* wb = static_cast<unsigned char*>(d->work) + kConvHeader;
    int* status = conv_status(d->work);
    __nv_bfloat16* a0 = reinterpret_cast<__nv_bfloat16*>(wb);
    __nv_bfloat16* a1 = a0 + act_elems;
    const unsigned fblocks = unsigned((pixels / kFirstPx + threads - 1) / threads);
    if (d->act == AC_ACT_TANH)
        conv_first_bf16_kernel<C, AC_ACT_TANH><<<fblocks, threads, 0, st>>>(u, a0, W, Bv, batch, n, io);
    else
        conv_first_bf16_kernel<C, AC_ACT_GELU><<<fblocks, threads, 0, st>>>(u, a0, W, Bv, batch, n, io);
    ACPR_LAUNCH_CHECK();
    size_t woff = size_t(C) * 9, boff = C;
    double* zpart = reinterpret_cast<double*>(wb + 2 * act_elems * sizeof(__nv_bfloat16));
    for (int l = 1; l < d->layers - 1; ++l) {
        if (l == d->layers - 2 && hidden_last_fused_supported(n, C)) {
            // the last hidden layer also forms the last layer's nine tap maps
            // (in the other activation buffer: 36 B per pixel <= 2 C B)
            float* maps = reinterpret_cast<float*>(a1);
            const float* w_last = W + woff + size_t(C) * C * 9;
            int rc = hidden_last_fused(d, l, n, batch, a0, nullptr, Bv + boff, w_last, maps, status, st);
            if (rc) return rc;
            return last_stencil_io(d, n, batch, maps, out, Bv + boff + C, u, io, zpart, st);
        }
        int rc = hidden_layer_bf16(d, l, n, batch, a0, a1, W + woff, Bv + boff, status, st);
        if (rc == AC_ERR_UNSUPPORTED) {
            conv_hidden_bf16_cc_kernel<C><<<blocks, threads, 0, st>>>(a0, a1, W + woff, Bv + boff, batch, n, d->act);
            ACPR_LAUNCH_CHECK();
        } else if (rc) {
            return rc;
        }
        woff += size_t(C) * C * 9;
        boff += C;
        __nv_bfloat16* t = a0; a0 = a1; a1 = t;
    }
    return last_layer_f32<C>(d, n, batch, a0, out, W + woff, Bv + boff, u, io, zpart, st);
}

static int run_f64(const cnn_desc* d, int n, int batch, const double* u, double* out, const BatchIO& io,
                   cudaStream_t st) {
    const long long pixels = (long long)n * n * batch;
    const int threads = 128;
    const unsigned blocks = unsigned((pixels + threads - 1) / threads);
    const double* W = static_cast<const double*>(d->w);
    const double* Bv = static_cast<const double*>(d->b);
    const size_t act_elems = size_t(batch) * d->channels * n * n;
    double* a0 = reinterpret_cast<double*>(static_cast<unsigned char*>(d->work) + kConvHeader);
    double* a1 = a0 + act_elems;
    size_t woff = 0, boff = 0;
    const double* cur = u;
    for (int l = 0; l < d->layers; ++l) {
        int cin, cout;
        layer_dims(d, l, &cin, &cout);
        const bool last = l == d->layers - 1;
        double* dst = last ? out : (l % 2 == 0 ? a0 : a1);
        BatchIO lio = io;
        lio.in_mapped = l == 0;
        lio.out_mapped = last;
        conv_f64_kernel<64><<<blocks, threads, 0, st>>>(cur, dst, W + woff, Bv + boff, batch, n, cin, cout,
                                                        d->act, last ? 0 : 1, (last && d->residual) ? u : nullptr, lio);
        ACPR_LAUNCH_CHECK();
        cur = dst;
        woff += size_t(cin) * cout * 9;
        boff += cout;
    }
    return AC_OK;
}

int coarse_step_mapped(const cnn_desc* d, int n, int batch, const void* u_in, long long in_bs,
                       const int* in_map, void* u_out, long long out_bs, const int* out_map,
                       cudaStream_t st) {
    int rc = check_cnn(d);
    if (rc) return rc;
    ACPR_CHECK_ARG(batch >= 0, "batch must be >= 0");
    if (batch == 0) return AC_OK;
    if (!is_pow2(n) || n < 8 || n > 1024) {
        set_error("cnn_coarse_step: n=%d unsupported (power of two in [8, 1024])", n);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(u_in && u_out && u_in != u_out, "bad field pointers");
    ACPR_CHECK_ARG(d->work && d->work_bytes >= work_bytes_for(d, n, batch),
                   "cnn work buffer too small: need %zu bytes", work_bytes_for(d, n, batch));
    BatchIO io;
    io.in_map = in_map;
    io.out_map = out_map;
    io.in_bs = in_bs;
    io.out_bs = out_bs;
    io.in_mapped = 1;
    io.out_mapped = 1;
    if (d->precision == AC_F64) {
        rc = run_f64(d, n, batch, static_cast<const double*>(u_in), static_cast<double*>(u_out), io, st);
    } else {
        ACPR_CHECK_ARG(d->packed != nullptr || d->layers == 2, "AC_F32 conv needs the packed weight buffer");
        const float* ui = static_cast<const float*>(u_in);
        float* uo = static_cast<float*>(u_out);
        switch (d->channels) {
            case 16: rc = run_f32<16>(d, n, batch, ui, uo, io, st); break;
            case 32: rc = run_f32<32>(d, n, batch, ui, uo, io, st); break;
            default: rc = run_f32<64>(d, n, batch, ui, uo, io, st); break;
        }
    }
    if (rc) return rc;
    if ((d->precision == AC_F64 && d->mass_fix) || d->limiter) {
        if (d->precision == AC_F64)
            post_kernel<double><<<batch, 256, 0, st>>>(static_cast<const double*>(u_in), static_cast<double*>(u_out), n,
                                                       d->mass_fix, d->limiter, d->lo, d->hi, io);
        else
            post_kernel<float><<<batch, 256, 0, st>>>(static_cast<const float*>(u_in), static_cast<float*>(u_out), n,
                                                      0, d->limiter, d->lo, d->hi, io);
        ACPR_LAUNCH_CHECK();
    }
    return AC_OK;
}

int coarse_step(const cnn_desc* d, int n, int batch, const void* u_in, void* u_out, cudaStream_t st) {
    const long long nn = (long long)n * n;
    return coarse_step_mapped(d, n, batch, u_in, nn, nullptr, u_out, nn, nullptr, st);
}

size_t packed_bytes_for(const cnn_desc* d) {
    if (d->precision == AC_F64) return 0;
    return packed_hidden_bytes(d);
}

}  // namespace acpr

extern "C" size_t cnn_packed_bytes(const cnn_desc* desc) {
    if (acpr::check_cnn(desc)) return 0;
    return acpr::packed_bytes_for(desc);
}

extern "C" size_t cnn_work_bytes(const cnn_desc* desc, int n, int batch) {
    if (acpr::check_cnn(desc) || n <= 0 || batch < 0) return 0;
    return acpr::work_bytes_for(desc, n, batch);
}

extern "C" int cnn_pack_weights(const cnn_desc* desc, acpr_stream stream) {
    int rc = acpr::check_cnn(desc);
    if (rc) return rc;
    if (desc->precision == AC_F64) return AC_OK;
    if (!desc->packed) {
        acpr::set_error("cnn_pack_weights: packed buffer is NULL");
        return AC_ERR_ARG;
    }
    return acpr::pack_hidden_weights(desc, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cnn_coarse_step(const cnn_desc* desc, int n, int batch, const void* u_in, void* u_out,
                               acpr_stream stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = acpr::coarse_step(desc, n, batch, u_in, u_out, st);
    if (rc || batch <= 0 || desc->precision != AC_F32) return rc;
    // a bounded wait of the tensor-core kernels that gave up left its code in
    // the workspace header: report it here (this synchronises the stream)
    return acpr::conv_check_status_uncaptured(acpr::conv_status(desc->work), st);
}

extern "C" int cnn_conv_variant_count(int n, int channels) { return acpr::conv_variant_count(n, channels); }

extern "C" int cnn_conv_variant_shape(int n, int channels, int index, int* ring, int* slots) {
    using namespace acpr;
    ACPR_CHECK_ARG(ring && slots, "null output");
    const int rc = conv_variant_describe(n, channels, index, ring, slots);
    if (rc) set_error("cnn_conv_variant_shape: index %d out of range", index);
    return rc;
}

extern "C" int cnn_conv_set_variant(int n, int channels, int index) {
    return acpr::conv_set_variant(n, channels, index);
}

extern "C" int cnn_conv_get_variant(int n, int channels) { return acpr::conv_get_variant(n, channels); }

extern "C" int cnn_autotune(const cnn_desc* desc, int n, int batch, const void* u_in, void* u_out, float* ms_out,
                            acpr_stream stream) {
    using namespace acpr;
    int rc = check_cnn(desc);
    if (rc) return rc;
    ACPR_CHECK_ARG(desc->precision == AC_F32, "cnn_autotune: the tensor-core path is AC_F32 only");
    ACPR_CHECK_ARG(batch >= 1 && u_in && u_out, "bad autotune arguments");
    const int count = conv_variant_count(n, desc->channels);
    ACPR_CHECK_ARG(count > 0, "cnn_autotune: no persistent tile shape for n=%d, C=%d", n, desc->channels);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    ACPR_CUDA(cudaEventCreate(&e0));
    ACPR_CUDA(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < count && !rc; ++v) {
        conv_set_variant(n, desc->channels, v);
        rc = coarse_step(desc, n, batch, u_in, u_out, st);  // warm-up
        if (rc) break;
        ACPR_CUDA(cudaEventRecord(e0, st));
        for (int rep = 0; rep < 3 && !rc; ++rep) rc = coarse_step(desc, n, batch, u_in, u_out, st);
        ACPR_CUDA(cudaEventRecord(e1, st));
        ACPR_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        ACPR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 3.f;
        if (ms_out) ms_out[v] = ms;
        if (ms < best_ms) { best_ms = ms; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    conv_set_variant(n, desc->channels, rc ? -1 : best);
    if (!rc) rc = conv_check_status(conv_status(desc->work), st);
    return rc;
}

extern "C" int ac_conv_status(void* workspace, acpr_stream stream) {
    ACPR_CHECK_ARG(workspace != nullptr, "workspace is NULL");
    return acpr::conv_check_status(acpr::conv_status(workspace), reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ac_test_conv_stall(int polls) {
    acpr::set_test_stall(polls);
    return AC_OK;
}
