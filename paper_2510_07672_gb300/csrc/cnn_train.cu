// cnn_train.cu -- training of the coarse propagator (AC_F32 path): the
// forward pass that saves what the backward pass needs, the backward pass of
// the conv stack, Adam, and the mean-squared-error loss.
//
// The model is out = u + stack(u), stack = conv_L o act o ... o act o conv_1
// (Sec. 3.2), optionally with the mACNN mass shift out -= mean(stack(u)), in
// which case the stack receives the output gradient minus its mean.  With a_0 = bf16(u), z_l = conv_l(a_l) + b_l, a_{l+1} = bf16(act(z_l)):
//   dz_L     = g = dL/dout
//   dW_l     = sum over pixels of dz_l (x) shifted a_l,  db_l = sum dz_l
//   dz_{l-1} = act'(z_{l-1}) * conv^T(dz_l, W_l)      (bf16, the next operand)
//   du       = g + conv^T(dz_1, W_1)
// Operands use the forward's bf16 values (weights and activations), gradients
// of the pre-activations are rounded to bf16 before they enter a product, and
// every accumulation is float32; weight gradients are reduced over pixel
// chunks in a fixed order (deterministic).  Hidden-layer dgrads run on the
// tensor cores through the forward kernel with channel-transposed, tap-flipped
// weights; the first and last layers and the weight gradients on CUDA cores.
//
// Workspace (cnn_train_bytes), in this order:
//   A_l, l = 1..L-1   bf16 [B][C/8][n][n][8]     inputs of layers 1..L-1
//   Z_l, l = 0..L-2   f32  [B][C/8][n][n][8]     pre-activations of layers 0..L-2
//   dZ ping-pong      2 x bf16 [B][C/8][n][n][8]
//   Wt                bf16 (L-2) x 9*C*C          transposed, flipped hidden weights
//   partials          f32  kChunks x 9 x (C*C + C)  weight / bias gradient partials
//   g centred         f32  [B][n][n]               (mass shift only)
//   z partials        f64  block sums of the last layer (mass shift only)
#include <cuda_bf16.h>

#include "cnn.cuh"

namespace acpr {

constexpr int kChunks = 64;      // pixel chunks of the weight-gradient reduction
constexpr int kWgThreads = 256;

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

struct TrainLayout {
    size_t a_bytes, z_bytes;    // one layer
    size_t off_a, off_z, off_dz, off_wt, off_part, off_gc, off_zpart, off_maps, total;
};

static TrainLayout train_layout(const cnn_desc* d, int n, int batch) {
    TrainLayout t{};
    const size_t act = size_t(batch) * d->channels * n * n;
    const int L = d->layers;
    t.a_bytes = act * 2;
    t.z_bytes = act * 4;
    t.off_a = kConvHeader;  // the header holds the tensor-core kernels' status word
    t.off_z = t.off_a + t.a_bytes * (L - 1);
    t.off_dz = t.off_z + t.z_bytes * (L - 1);
    t.off_wt = t.off_dz + 2 * t.a_bytes;
    const size_t wt = size_t(L > 2 ? L - 2 : 0) * 9 * d->channels * d->channels * 2;
    t.off_part = (t.off_wt + wt + 255) / 256 * 256;
    t.off_gc = t.off_part + size_t(kChunks) * 9 * (size_t(d->channels) * d->channels + d->channels) * 4;
    t.off_zpart = t.off_gc + size_t(batch) * n * n * 4;
    t.off_maps = t.off_zpart + size_t(batch) * n * n * sizeof(double);  // >= the last layer's block partials
    t.total = t.off_maps + size_t(batch) * 9 * n * n * sizeof(float);
    return t;
}

// ------------------------------------------------------------- forward ----
// First layer with the float32 pre-activations saved (1 -> C, K = 9).
template <int C>
__global__ void first_fwd_save_kernel(const float* __restrict__ u, __nv_bfloat16* __restrict__ a1,
                                      float* __restrict__ z0, const float* __restrict__ W,
                                      const float* __restrict__ bias, int batch, int n, int act) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (pix >= nn * batch) return;
    const int b = int(pix / nn);
    const int y = int((pix % nn) / n), x = int(pix % n);
    const float* f = u + (long long)b * nn;
    float v[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) v[t] = bf16r(f[(long long)wrapi(y + t / 3 - 1, n) * n + wrapi(x + t % 3 - 1, n)]);
#pragma unroll
    for (int kc = 0; kc < C / 8; ++kc) {
        __align__(16) __nv_bfloat16 o8[8];
        __align__(16) float z8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int o = kc * 8 + i;
            float s = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) s = fmaf(bf16r(W[o * 9 + t]), v[t], s);
            z8[i] = s + bias[o];
            o8[i] = __float2bfloat16_rn(act_apply<float>(act, z8[i]));
        }
        const long long off = (((long long)b * (C / 8) + kc) * nn + pix % nn) * 8;
        *reinterpret_cast<uint4*>(a1 + off) = *reinterpret_cast<const uint4*>(o8);
        reinterpret_cast<float4*>(z0 + off)[0] = *reinterpret_cast<const float4*>(z8);
        reinterpret_cast<float4*>(z0 + off)[1] = *reinterpret_cast<const float4*>(z8 + 4);
    }
}

// ------------------------------------------------------------ backward ----
// gc = g - mean(g) per field (float64 sum in a fixed order), one block each.
__global__ void center_kernel(const float* __restrict__ g, float* __restrict__ gc, int n) {
    const long long nn = (long long)n * n;
    const float* gb = g + blockIdx.x * nn;
    float* ob = gc + blockIdx.x * nn;
    __shared__ double red[32];
    double s = 0.0;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) s += double(gb[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        red[0] = t / double(nn);
    }
    __syncthreads();
    const float mean = float(red[0]);
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) ob[i] = gb[i] - mean;
}

// Last layer: dz_{L-2} = bf16(act'(z_{L-2}) * sum_tap W_L[c][tap] g[p - off(tap)]).
template <int C>
__global__ void last_dgrad_kernel(const float* __restrict__ g, const float* __restrict__ W,
                                  const float* __restrict__ zprev, __nv_bfloat16* __restrict__ dz, int batch,
                                  int n, int act) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (pix >= nn * batch) return;
    const int b = int(pix / nn);
    const int y = int((pix % nn) / n), x = int(pix % n);
    float gv[9];
#pragma unroll
    for (int t = 0; t < 9; ++t)  // input p feeds output p - off(tap)
        gv[t] = bf16r(g[(long long)b * nn + (long long)wrapi(y - (t / 3 - 1), n) * n + wrapi(x - (t % 3 - 1), n)]);
#pragma unroll
    for (int kc = 0; kc < C / 8; ++kc) {
        const long long off = (((long long)b * (C / 8) + kc) * nn + pix % nn) * 8;
        __align__(16) __nv_bfloat16 o8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = kc * 8 + i;
            float s = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) s = fmaf(bf16r(W[c * 9 + t]), gv[t], s);
            o8[i] = __float2bfloat16_rn(s * act_grad<float>(act, zprev[off + i]));
        }
        *reinterpret_cast<uint4*>(dz + off) = *reinterpret_cast<const uint4*>(o8);
    }
}

// First layer: du = g + sum_{o,tap} W_1[o][tap] dz_0[o][p - off(tap)].
template <int C>
__global__ void first_dgrad_kernel(const float* __restrict__ g, const __nv_bfloat16* __restrict__ dz,
                                   const float* __restrict__ W, float* __restrict__ du, int batch, int n) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (pix >= nn * batch) return;
    const int b = int(pix / nn);
    const int y = int((pix % nn) / n), x = int(pix % n);
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const long long q = (long long)wrapi(y - (t / 3 - 1), n) * n + wrapi(x - (t % 3 - 1), n);
        for (int kc = 0; kc < C / 8; ++kc) {
            const uint4 raw = *reinterpret_cast<const uint4*>(dz + (((long long)b * (C / 8) + kc) * nn + q) * 8);
            const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                acc = fmaf(bf16r(__ldg(W + (kc * 8 + i) * 9 + t)), __bfloat162float(v8[i]), acc);
        }
    }
    du[pix] = g[pix] + acc;
}

// Weight and bias gradient partials of one layer, one (tap, chunk) per block:
//   part[chunk][tap][o][c] = sum_{pixels q of the chunk} dz[o][q] * a[c][q + off(tap)]
//   part[chunk][tap][C*C + o] = sum dz[o][q]  (tap 0 blocks only)
// a: bf16 chunked activations, or (CIN == 1) the float32 field rounded to bf16.
// dz: bf16 chunked, or (COUT == 1) the float32 output gradient rounded to bf16.
// Block rows of 64 pixels are staged in shared memory; thread (o, c-group)
// accumulates a strip of input channels.
// Each thread owns a TO x TC block of (output, input) channel pairs and, per
// staged pixel, reads TO dz values and TC activations (vector loads) for its
// TO * TC fused multiply-adds; every pair still sums its pixels in order.
template <int PER> struct WgTile;
template <> struct WgTile<1> { static constexpr int TO = 1, TC = 1; };
template <> struct WgTile<4> { static constexpr int TO = 2, TC = 2; };
template <> struct WgTile<16> { static constexpr int TO = 4, TC = 4; };

template <int K>
__device__ __forceinline__ void lds_vec(const float* p, float (&v)[K]) {
    if constexpr (K == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (K == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = *p;
    }
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgThreads)
wgrad_kernel(const void* __restrict__ a_src, const void* __restrict__ dz_src, float* __restrict__ part,
             int batch, int n, int C) {
    constexpr int TP = 64;                       // pixels per staged strip
    constexpr int PAIRS = CIN * COUT;
    constexpr int PER = (PAIRS + kWgThreads - 1) / kWgThreads;
    constexpr int TO = WgTile<PER>::TO, TC = WgTile<PER>::TC;
    constexpr int NCB = CIN / TC;                // input-channel blocks
    constexpr int NTH = (COUT / TO) * NCB;       // threads that own pairs
    constexpr int PA = CIN >= 4 ? CIN + 4 : CIN + 1;    // row pitches (16-byte rows for vector loads)
    constexpr int PD = COUT >= 4 ? COUT + 4 : COUT + 1;
    __shared__ __align__(16) float s_a[TP][PA];
    __shared__ __align__(16) float s_dz[TP][PD];
    const int tap = blockIdx.x % 9;
    const int chunk = blockIdx.x / 9;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int lg = __ffs(n) - 1;                 // n is a power of two
    const long long nn = (long long)n * n;
    const long long total = nn * batch;
    const long long per_chunk = (total + kChunks - 1) / kChunks;
    const long long p0 = chunk * per_chunk;
    const long long p1 = p0 + per_chunk < total ? p0 + per_chunk : total;
    const int ob = threadIdx.x / NCB, cb = threadIdx.x % NCB;
    const bool owner = threadIdx.x < NTH;
    float acc[TO][TC];
    float bacc = 0.f;
#pragma unroll
    for (int i = 0; i < TO; ++i)
#pragma unroll
        for (int k = 0; k < TC; ++k) acc[i][k] = 0.f;
    for (long long base = p0; base < p1; base += TP) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < TP * CIN; idx += kWgThreads) {
            const int pi = idx / CIN, c = idx % CIN;
            const long long p = base + pi;
            float v = 0.f;
            if (p < p1) {
                const int b = int(p >> (2 * lg));
                const int y = wrapi((int(p >> lg) & (n - 1)) + dy, n), x = wrapi((int(p) & (n - 1)) + dx, n);
                const long long q = (long long)y * n + x;
                if constexpr (CIN == 1) {
                    v = bf16r(static_cast<const float*>(a_src)[(long long)b * nn + q]);
                } else {
                    v = __bfloat162float(static_cast<const __nv_bfloat16*>(a_src)[
                        (((long long)b * (CIN / 8) + c / 8) * nn + q) * 8 + c % 8]);
                }
            }
            s_a[pi][c] = v;
        }
        for (int idx = threadIdx.x; idx < TP * COUT; idx += kWgThreads) {
            const int pi = idx / COUT, o = idx % COUT;
            const long long p = base + pi;
            float v = 0.f;
            if (p < p1) {
                const int b = int(p >> (2 * lg));
                const long long q = p & (nn - 1);
                if constexpr (COUT == 1) {
                    v = bf16r(static_cast<const float*>(dz_src)[(long long)b * nn + q]);
                } else {
                    v = __bfloat162float(static_cast<const __nv_bfloat16*>(dz_src)[
                        (((long long)b * (COUT / 8) + o / 8) * nn + q) * 8 + o % 8]);
                }
            }
            s_dz[pi][o] = v;
        }
        __syncthreads();
        if (owner) {
#pragma unroll 4
            for (int pi = 0; pi < TP; ++pi) {
                float dv[TO], av[TC];
                lds_vec<TO>(&s_dz[pi][ob * TO], dv);
                lds_vec<TC>(&s_a[pi][cb * TC], av);
#pragma unroll
                for (int i = 0; i < TO; ++i)
#pragma unroll
                    for (int k = 0; k < TC; ++k) acc[i][k] = fmaf(dv[i], av[k], acc[i][k]);
            }
        }
        if (tap == 0 && threadIdx.x < COUT)
            for (int pi = 0; pi < TP; ++pi) bacc += s_dz[pi][threadIdx.x];
    }
    float* out = part + ((long long)chunk * 9 + tap) * (C * C + C);
    if (owner) {
#pragma unroll
        for (int i = 0; i < TO; ++i)
#pragma unroll
            for (int k = 0; k < TC; ++k) out[(ob * TO + i) * CIN + cb * TC + k] = acc[i][k];
    }
    if (tap == 0 && threadIdx.x < COUT) out[C * C + threadIdx.x] = bacc;
}
// The same partials for the first (CIN = 1) and last (COUT = 1) layers, where
// one side has K = C channels and the other one: a thread walks its own pixels
// of the (tap, chunk) block with all K channel sums in registers (the K-side
// operand comes as 16-byte chunk vectors), then the block sums its threads in
// a fixed order (a shuffle tree per warp, then the warps in order).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgThreads)
wgrad_thin_kernel(const void* __restrict__ a_src, const void* __restrict__ dz_src, float* __restrict__ part,
                  int batch, int n, int C) {
    static_assert(CIN == 1 || COUT == 1, "one side of the layer has one channel");
    constexpr int K = CIN > COUT ? CIN : COUT;
    constexpr int KC = K / 8;
    constexpr int NW = kWgThreads / 32;
    __shared__ float red[NW][K + 1];
    const int tap = blockIdx.x % 9;
    const int chunk = blockIdx.x / 9;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int lg = __ffs(n) - 1;  // n is a power of two
    const long long nn = (long long)n * n;
    const long long total = nn * batch;
    const long long per_chunk = (total + kChunks - 1) / kChunks;
    const long long p0 = chunk * per_chunk;
    const long long p1 = p0 + per_chunk < total ? p0 + per_chunk : total;
    const bool bias = tap == 0;
    float acc[K], bacc[CIN == 1 ? K : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.f;
#pragma unroll
    for (int k = 0; k < (CIN == 1 ? K : 1); ++k) bacc[k] = 0.f;
    for (long long p = p0 + threadIdx.x; p < p1; p += kWgThreads) {
        const int b = int(p >> (2 * lg));
        const long long pl = p & (nn - 1);
        const int y = wrapi((int(p >> lg) & (n - 1)) + dy, n), x = wrapi((int(p) & (n - 1)) + dx, n);
        const long long q = (long long)y * n + x;
        if constexpr (CIN == 1) {
            // first layer: a = the float32 field (bf16-rounded), dz = C bf16 channels at p
            const float av = bf16r(static_cast<const float*>(a_src)[(long long)b * nn + q]);
            const __nv_bfloat16* dz = static_cast<const __nv_bfloat16*>(dz_src);
#pragma unroll
            for (int kc = 0; kc < KC; ++kc) {
                const uint4 raw = *reinterpret_cast<const uint4*>(dz + (((long long)b * KC + kc) * nn + pl) * 8);
                const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float dv = __bfloat162float(v8[i]);
                    acc[kc * 8 + i] = fmaf(dv, av, acc[kc * 8 + i]);
                    if (bias) bacc[kc * 8 + i] += dv;
                }
            }
        } else {
            // last layer: dz = the float32 output gradient (bf16-rounded), a = C bf16 channels at q
            const float dv = bf16r(static_cast<const float*>(dz_src)[(long long)b * nn + pl]);
            const __nv_bfloat16* a = static_cast<const __nv_bfloat16*>(a_src);
#pragma unroll
            for (int kc = 0; kc < KC; ++kc) {
                const uint4 raw = *reinterpret_cast<const uint4*>(a + (((long long)b * KC + kc) * nn + q) * 8);
                const __nv_bfloat16* v8 = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[kc * 8 + i] = fmaf(dv, __bfloat162float(v8[i]), acc[kc * 8 + i]);
            }
            if (bias) bacc[0] += dv;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* out = part + ((long long)chunk * 9 + tap) * (C * C + C);
    // weight partials: index o * CIN + c is k on both sides (the other index is 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t += red[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    if (bias) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < COUT; ++k) {
            float v = bacc[CIN == 1 ? k : 0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < COUT) {
            float t = 0.f;
            for (int w = 0; w < NW; ++w) t += red[w][threadIdx.x];
            out[C * C + threadIdx.x] = t;
        }
    }
}

// Fixed-order sum of the chunk partials into the float32 gradients
// (W[o][c][tap] layout of the masters; overwrite or accumulate).
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, float* __restrict__ gw, float* __restrict__ gb,
                                    int cin, int cout, int C, int accumulate) {
    const int nw = cout * cin * 9;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < nw) {
        const int o = idx / (cin * 9), c = (idx / 9) % cin, tap = idx % 9;
        float s = 0.f;
        for (int ch = 0; ch < kChunks; ++ch) s += part[((long long)ch * 9 + tap) * (C * C + C) + o * cin + c];
        gw[idx] = accumulate ? gw[idx] + s : s;
    } else if (idx < nw + cout) {
        const int o = idx - nw;
        float s = 0.f;
        for (int ch = 0; ch < kChunks; ++ch) s += part[((long long)ch * 9) * (C * C + C) + C * C + o];
        gb[o] = accumulate ? gb[o] + s : s;
    }
}

// ------------------------------------------------------------- host side --
static int check_train(const cnn_desc* d) {
    int rc = check_cnn(d);
    if (rc) return rc;
    if (d->precision != AC_F32 || d->limiter || !d->residual) {
        set_error("conv training: only the AC_F32 residual stack without limiter");
        return AC_ERR_UNSUPPORTED;
    }
    return AC_OK;
}

template <int CIN, int COUT>
static int wgrad(const void* a, const void* dz, float* part, float* gw, float* gb, int batch, int n, int C,
                 int accumulate, cudaStream_t st) {
    if constexpr (CIN == 1 || COUT == 1)
        wgrad_thin_kernel<CIN, COUT><<<kChunks * 9, kWgThreads, 0, st>>>(a, dz, part, batch, n, C);
    else
        wgrad_kernel<CIN, COUT><<<kChunks * 9, kWgThreads, 0, st>>>(a, dz, part, batch, n, C);
    ACPR_LAUNCH_CHECK();
    const int total = COUT * CIN * 9 + COUT;
    wgrad_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(part, gw, gb, CIN, COUT, C, accumulate);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

template <int C>
static int forward_train(const cnn_desc* d, int n, int batch, const float* u, float* out, unsigned char* ws,
                         cudaStream_t st) {
    const TrainLayout t = train_layout(d, n, batch);
    const long long pixels = (long long)n * n * batch;
    const unsigned blocks = unsigned((pixels + 127) / 128);
    const float* W = static_cast<const float*>(d->w);
    const float* Bv = static_cast<const float*>(d->b);
    auto A = [&](int l) { return reinterpret_cast<__nv_bfloat16*>(ws + t.off_a + t.a_bytes * (l - 1)); };
    auto Z = [&](int l) { return reinterpret_cast<float*>(ws + t.off_z + t.z_bytes * l); };
    first_fwd_save_kernel<C><<<blocks, 128, 0, st>>>(u, A(1), Z(0), W, Bv, batch, n, d->act);
    ACPR_LAUNCH_CHECK();
    size_t woff = size_t(C) * 9, boff = C;
    for (int l = 1; l < d->layers - 1; ++l) {
        int rc = hidden_layer_bf16(d, l, n, batch, A(l), A(l + 1), W + woff, Bv + boff, conv_status(ws), st, Z(l));
        if (rc) return rc;
        woff += size_t(C) * C * 9;
        boff += C;
    }
    // the inference path's last layer and mass shift, so that the training
    // forward equals cnn_coarse_step bit for bit
    double* zpart = reinterpret_cast<double*>(ws + t.off_zpart);
    return last_layer_bf16(d, n, batch, A(d->layers - 1), out, W + woff, Bv + boff, u, zpart, st);
}

// The same forward pass where the inference path fuses the last hidden layer
// with the last layer's projection (see hidden_last_fused).
template <int C>
static int forward_train_fused(const cnn_desc* d, int n, int batch, const float* u, float* out, unsigned char* ws,
                               cudaStream_t st) {
    const TrainLayout t = train_layout(d, n, batch);
    const long long pixels = (long long)n * n * batch;
    const unsigned blocks = unsigned((pixels + 127) / 128);
    const float* W = static_cast<const float*>(d->w);
    const float* Bv = static_cast<const float*>(d->b);
    auto A = [&](int l) { return reinterpret_cast<__nv_bfloat16*>(ws + t.off_a + t.a_bytes * (l - 1)); };
    auto Z = [&](int l) { return reinterpret_cast<float*>(ws + t.off_z + t.z_bytes * l); };
    first_fwd_save_kernel<C><<<blocks, 128, 0, st>>>(u, A(1), Z(0), W, Bv, batch, n, d->act);
    ACPR_LAUNCH_CHECK();
    size_t woff = size_t(C) * 9, boff = C;
    const int L = d->layers;
    for (int l = 1; l < L - 2; ++l) {
        int rc = hidden_layer_bf16(d, l, n, batch, A(l), A(l + 1), W + woff, Bv + boff, conv_status(ws), st, Z(l));
        if (rc) return rc;
        woff += size_t(C) * C * 9;
        boff += C;
    }
    float* maps = reinterpret_cast<float*>(ws + t.off_maps);
    int rc = hidden_last_fused(d, L - 2, n, batch, A(L - 2), A(L - 1), Bv + boff, W + woff + size_t(C) * C * 9, maps,
                               conv_status(ws), st, Z(L - 2));
    if (rc) return rc;
    double* zpart = reinterpret_cast<double*>(ws + t.off_zpart);
    return last_stencil_f32(d, n, batch, maps, out, Bv + boff + C, u, zpart, st);
}

template <int C>
static int backward(const cnn_desc* d, int n, int batch, const float* u, const float* g, float* du, float* gw,
                    float* gb, int accumulate, unsigned char* ws, cudaStream_t st) {
    const TrainLayout t = train_layout(d, n, batch);
    const int L = d->layers;
    const long long pixels = (long long)n * n * batch;
    const unsigned blocks = unsigned((pixels + 127) / 128);
    const float* W = static_cast<const float*>(d->w);
    auto A = [&](int l) { return reinterpret_cast<__nv_bfloat16*>(ws + t.off_a + t.a_bytes * (l - 1)); };
    auto Z = [&](int l) { return reinterpret_cast<float*>(ws + t.off_z + t.z_bytes * l); };
    __nv_bfloat16* dz[2] = {reinterpret_cast<__nv_bfloat16*>(ws + t.off_dz),
                            reinterpret_cast<__nv_bfloat16*>(ws + t.off_dz + t.a_bytes)};
    __nv_bfloat16* wt = reinterpret_cast<__nv_bfloat16*>(ws + t.off_wt);
    float* part = reinterpret_cast<float*>(ws + t.off_part);
    // parameter offsets per layer
    size_t woffs[64], boffs[64];
    size_t wo = 0, bo = 0;
    for (int l = 0; l < L; ++l) {
        const int ci = l == 0 ? 1 : C, co = l == L - 1 ? 1 : C;
        woffs[l] = wo; boffs[l] = bo;
        wo += size_t(ci) * co * 9; bo += co;
    }
    int rc;
    // the stack's output gradient: g, or g minus its mean under the mass shift
    const float* gs = g;
    if (d->mass_fix) {
        float* gc = reinterpret_cast<float*>(ws + t.off_gc);
        center_kernel<<<batch, 256, 0, st>>>(g, gc, n);
        ACPR_LAUNCH_CHECK();
        gs = gc;
    }
    // last layer
    rc = wgrad<C, 1>(A(L - 1), gs, part, gw + woffs[L - 1], gb + boffs[L - 1], batch, n, C, accumulate, st);
    if (rc) return rc;
    last_dgrad_kernel<C><<<blocks, 128, 0, st>>>(gs, W + woffs[L - 1], Z(L - 2), dz[0], batch, n, d->act);
    ACPR_LAUNCH_CHECK();
    int cur = 0;
    // hidden layers L-2 .. 1: dz[cur] holds dz_l
    for (int l = L - 2; l >= 1; --l) {
        if (wgrad_tc_supported(C, n)) {
            rc = wgrad_tc_partials(n, batch, A(l), dz[cur], part, kChunks, conv_status(ws), st);
            if (rc) return rc;
            const int tot = C * C * 9 + C;
            wgrad_reduce_kernel<<<(tot + 255) / 256, 256, 0, st>>>(part, gw + woffs[l], gb + boffs[l], C, C, C,
                                                                   accumulate);
            ACPR_LAUNCH_CHECK();
        } else {
            rc = wgrad<C, C>(A(l), dz[cur], part, gw + woffs[l], gb + boffs[l], batch, n, C, accumulate, st);
        }
        if (rc) return rc;
        __nv_bfloat16* wl = wt + size_t(l - 1) * 9 * C * C;
        rc = pack_hidden_t(C, W + woffs[l], wl, st);
        if (rc) return rc;
        rc = hidden_dgrad_bf16(C, d->act, n, batch, dz[cur], dz[cur ^ 1], wl, Z(l - 1), conv_status(ws), st);
        if (rc) return rc;
        cur ^= 1;
    }
    // first layer: dz[cur] holds dz_0
    rc = wgrad<1, C>(u, dz[cur], part, gw + woffs[0], gb + boffs[0], batch, n, C, accumulate, st);
    if (rc) return rc;
    if (du) {
        first_dgrad_kernel<C><<<blocks, 128, 0, st>>>(g, dz[cur], W + woffs[0], du, batch, n);
        ACPR_LAUNCH_CHECK();
    }
    return AC_OK;
}

// ------------------------------------------------------------- Adam / MSE --
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long count, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// grad = 2 * scale * (pred - target); per-block float64 partial sums of
// scale * (pred - target)^2 into part, finished by mse_finish_kernel.
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ target, long long count,
                           float scale, float* __restrict__ grad, int grad_accumulate, double* __restrict__ part) {
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        if (grad) grad[i] = grad_accumulate ? grad[i] + 2.f * scale * d : 2.f * scale * d;
        s += double(d) * double(d);
    }
    __shared__ double sh[8];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[blockIdx.x] = t * double(scale);
    }
}

__global__ void mse_finish_kernel(const double* __restrict__ part, int blocks, double* __restrict__ loss,
                                  int accumulate) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < blocks; ++i) t += part[i];
        loss[0] = accumulate ? loss[0] + t : t;
    }
}

}  // namespace acpr

extern "C" size_t cnn_train_bytes(const cnn_desc* desc, int n, int batch) {
    using namespace acpr;
    if (check_train(desc) || n <= 0 || batch <= 0) return 0;
    return train_layout(desc, n, batch).total + 64 * sizeof(double);
}

extern "C" int cnn_forward_train(const cnn_desc* desc, int n, int batch, const float* u_in, float* u_out,
                                 void* train_ws, acpr_stream stream) {
    using namespace acpr;
    int rc = check_train(desc);
    if (rc) return rc;
    ACPR_CHECK_ARG(n >= 8 && is_pow2(n) && batch >= 1, "need n a power of two >= 8 and batch >= 1");
    ACPR_CHECK_ARG(u_in && u_out && train_ws && desc->packed, "null pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(train_ws);
    const bool fused = desc->layers >= 3 && hidden_last_fused_supported(n, desc->channels);
    switch (desc->channels) {
        case 16: rc = forward_train<16>(desc, n, batch, u_in, u_out, ws, st); break;
        case 32:
            rc = fused ? forward_train_fused<32>(desc, n, batch, u_in, u_out, ws, st)
                       : forward_train<32>(desc, n, batch, u_in, u_out, ws, st);
            break;
        default:
            rc = fused ? forward_train_fused<64>(desc, n, batch, u_in, u_out, ws, st)
                       : forward_train<64>(desc, n, batch, u_in, u_out, ws, st);
            break;
    }
    // a bounded tensor-core wait that gave up is reported here (synchronises)
    return rc ? rc : conv_check_status_uncaptured(conv_status(train_ws), st);
}

extern "C" int cnn_backward(const cnn_desc* desc, int n, int batch, const float* u_in, const float* grad_out,
                            float* grad_in, float* grad_w, float* grad_b, int accumulate, void* train_ws,
                            acpr_stream stream) {
    using namespace acpr;
    int rc = check_train(desc);
    if (rc) return rc;
    ACPR_CHECK_ARG(n >= 8 && is_pow2(n) && batch >= 1, "need n a power of two >= 8 and batch >= 1");
    ACPR_CHECK_ARG(u_in && grad_out && grad_w && grad_b && train_ws, "null pointer");
    ACPR_CHECK_ARG(desc->layers >= 3 && desc->layers <= 64, "training needs 3..64 layers");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(train_ws);
    switch (desc->channels) {
        case 16: rc = backward<16>(desc, n, batch, u_in, grad_out, grad_in, grad_w, grad_b, accumulate, ws, st); break;
        case 32: rc = backward<32>(desc, n, batch, u_in, grad_out, grad_in, grad_w, grad_b, accumulate, ws, st); break;
        default: rc = backward<64>(desc, n, batch, u_in, grad_out, grad_in, grad_w, grad_b, accumulate, ws, st); break;
    }
    return rc ? rc : conv_check_status_uncaptured(conv_status(train_ws), st);
}

extern "C" int cnn_adam_step(float* w, const float* grad, float* m, float* v, long long count, double lr,
                             double beta1, double beta2, double eps, int t, acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(w && grad && m && v && count >= 0 && t >= 1, "bad Adam arguments");
    if (count == 0) return AC_OK;
    const float c1 = float(1.0 - pow(beta1, t)), c2 = float(1.0 - pow(beta2, t));
    const long long want = (count + 255) / 256;
    adam_kernel<<<unsigned(want < 1024 ? want : 1024), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        w, grad, m, v, count, float(lr), float(beta1), float(beta2), float(eps), c1, c2);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

extern "C" int mse_loss_grad(const float* pred, const float* target, long long count, double scale, float* grad,
                             int grad_accumulate, double* loss_dev, double* scratch_dev, int accumulate,
                             acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(pred && target && loss_dev && scratch_dev && count > 0, "bad MSE arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = 64;
    mse_kernel<<<blocks, 256, 0, st>>>(pred, target, count, float(scale), grad, grad_accumulate, scratch_dev);
    ACPR_LAUNCH_CHECK();
    mse_finish_kernel<<<1, 32, 0, st>>>(scratch_dev, blocks, loss_dev, accumulate);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}
