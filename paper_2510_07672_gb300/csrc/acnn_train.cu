// acnn_train.cu -- per-layer kernels of the ResBlock ACNN / mACNN (Sec. 3.2):
// the forward pass that saves every activation, and the backward pass to the
// parameter gradients.  Used for training (Algorithm 1) and for inference of
// shapes the fused kernel in acnn.cu does not cover.
//
// Every layer is one launch over all pixels of the batch; a thread owns
// kPix pixels of a 256 x kPix chunk (one field: n^2 >= 1024).  Activations
// are channel-interleaved [field][n][n][C], so one pixel's channels are one
// vector load; neighbours come through L1/L2 (a 16-field 256^2 C = 4 batch is
// 4 MB per activation, resident in L2).  Weight gradients reduce per block in
// a fixed order and then over blocks in a fixed order: deterministic.
#include "acnn.cuh"

namespace acpr {

namespace {

constexpr int kThreads = 256;
constexpr int kPix = 4;                        // pixels per thread in the conv kernels
constexpr int kChunk = kThreads * kPix;        // pixels per block (1024)
constexpr int kWgPix = 16;                     // pixels per thread in the weight-gradient kernel

template <typename T, int N>
__device__ __forceinline__ void load_px(const T* p, T (&r)[N]) {
    if constexpr (N % 4 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < N; k += 4) {
            const float4 q = *reinterpret_cast<const float4*>(p + k);
            r[k] = q.x; r[k + 1] = q.y; r[k + 2] = q.z; r[k + 3] = q.w;
        }
    } else if constexpr (N % 2 == 0 && sizeof(T) == 8) {
#pragma unroll
        for (int k = 0; k < N; k += 2) {
            const double2 q = *reinterpret_cast<const double2*>(p + k);
            r[k] = q.x; r[k + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) r[k] = p[k];
    }
}

template <typename T, int N>
__device__ __forceinline__ void store_px(T* p, const T (&r)[N]) {
    if constexpr (N % 4 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < N; k += 4) *reinterpret_cast<float4*>(p + k) = make_float4(r[k], r[k + 1], r[k + 2], r[k + 3]);
    } else if constexpr (N % 2 == 0 && sizeof(T) == 8) {
#pragma unroll
        for (int k = 0; k < N; k += 2) *reinterpret_cast<double2*>(p + k) = make_double2(r[k], r[k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) p[k] = r[k];
    }
}

enum { kModeTanh = 0, kModeBlockOut = 1 };

// The 9 taps are unrolled only while their weights fit in registers; beyond
// that the compiler would hoist every weight out of the pixel loop and spill.
template <typename T, int CIN, int COUT>
constexpr int taps_unroll() { return 9 * CIN * COUT * int(sizeof(T)) > 640 ? 1 : 9; }

// One 3x3 circular correlation CIN -> COUT over the batch (not the output conv).
//   kModeTanh:     out = tanh(conv(in) + b)
//   kModeBlockOut: out = t = tanh(conv(in) + b), out2 = skip + t
// in/out fields: base + sel(map, b) * bs (internal buffers: contiguous).
template <typename T, int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kThreads) conv_kernel(const T* __restrict__ in, long long in_bs,
                                                        const int* __restrict__ in_map, T* __restrict__ out,
                                                        long long out_bs, const int* __restrict__ out_map,
                                                        const T* __restrict__ W, const T* __restrict__ bias,
                                                        const T* __restrict__ skip, T* __restrict__ out2, int n,
                                                        int lg) {
    __shared__ T sw[9 * CIN * COUT];  // [tap][cin][cout]
    __shared__ T sb[COUT];
    for (int k = threadIdx.x; k < 9 * CIN * COUT; k += kThreads) {
        const int co = k / (9 * CIN), ci = (k / 9) % CIN, tap = k % 9;
        sw[(tap * CIN + ci) * COUT + co] = W[k];
    }
    if (threadIdx.x < COUT) sb[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const long long nn = 1LL << (2 * lg);
    const long long first = (long long)blockIdx.x * kChunk;
    const int b = int(first >> (2 * lg));
    const T* src = in + acnn_sel(in_map, b) * in_bs;
    T* dst = out + acnn_sel(out_map, b) * out_bs;
    const int mask = n - 1;
#pragma unroll 1
    for (int k = 0; k < kPix; ++k) {
        const int q = int((first & (nn - 1)) + threadIdx.x + k * kThreads);
        const int i = q >> lg, j = q & mask;
        T acc[COUT];
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = sb[co];
#pragma unroll(taps_unroll<T, CIN, COUT>())
        for (int tap = 0; tap < 9; ++tap) {
                const int a = tap / 3, e = tap % 3;
                const int s = (((i + a - 1) & mask) << lg) | ((j + e - 1) & mask);
                T v[CIN];
                load_px<T, CIN>(src + (long long)s * CIN, v);
                const T* w = sw + tap * CIN * COUT;
#pragma unroll
                for (int ci = 0; ci < CIN; ++ci)
#pragma unroll
                    for (int co = 0; co < COUT; ++co) acc[co] = fma(w[ci * COUT + co], v[ci], acc[co]);
            }
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = acnn_tanh(acc[co]);
        store_px<T, COUT>(dst + (long long)q * COUT, acc);
        if constexpr (MODE == kModeBlockOut) {
            T x[COUT];
            load_px<T, COUT>(skip + ((long long)b * nn + q) * COUT, x);
#pragma unroll
            for (int co = 0; co < COUT; ++co) x[co] += acc[co];
            store_px<T, COUT>(out2 + ((long long)b * nn + q) * COUT, x);
        }
    }
}

// The output conv C -> 1 (no activation); with `part` it also writes the
// block's sum of (out - u), u the one-channel network input, for the mass
// shift.
template <typename T, int CIN>
__global__ void __launch_bounds__(kThreads) out_conv_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                            long long out_bs, const int* __restrict__ out_map,
                                                            const T* __restrict__ W, const T* __restrict__ bias,
                                                            const T* __restrict__ u, long long u_bs,
                                                            const int* __restrict__ u_map, double* __restrict__ part,
                                                            int n, int lg) {
    __shared__ T sw[9 * CIN];  // [tap][cin]
    __shared__ double red[kThreads / 32];
    for (int k = threadIdx.x; k < 9 * CIN; k += kThreads) {
        const int ci = k / 9, tap = k % 9;
        sw[tap * CIN + ci] = W[k];
    }
    __syncthreads();
    const T b0 = bias[0];
    const long long nn = 1LL << (2 * lg);
    const long long first = (long long)blockIdx.x * kChunk;
    const int b = int(first >> (2 * lg));
    const T* src = in + (long long)b * nn * CIN;
    T* dst = out + acnn_sel(out_map, b) * out_bs;
    const T* ub = u + acnn_sel(u_map, b) * u_bs;
    const int mask = n - 1;
    T msum = T(0);
#pragma unroll 1
    for (int k = 0; k < kPix; ++k) {
        const int q = int((first & (nn - 1)) + threadIdx.x + k * kThreads);
        const int i = q >> lg, j = q & mask;
        T acc = b0;
#pragma unroll(taps_unroll<T, CIN, 1>())
        for (int tap = 0; tap < 9; ++tap) {
                const int a = tap / 3, e = tap % 3;
                const int s = (((i + a - 1) & mask) << lg) | ((j + e - 1) & mask);
                T v[CIN];
                load_px<T, CIN>(src + (long long)s * CIN, v);
#pragma unroll
                for (int ci = 0; ci < CIN; ++ci) acc = fma(sw[tap * CIN + ci], v[ci], acc);
            }
        dst[q] = acc;
        if (part) msum += acc - ub[q];
    }
    if (part) {
        double s = double(msum);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            part[blockIdx.x] = t;
        }
    }
}

// Input gradient of a 3x3 circular correlation COUT <- CIN (the adjoint:
// g_in[q] = sum_tap W[tap]^T g_out[q - d_tap]), then
//   raw = g_in + add   (stored when `raw` is set; `add` may be null)
//   gz  = raw * (1 - A^2)   (A: the tanh output feeding this gradient)
template <typename T, int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) dgrad_kernel(const T* __restrict__ g_out, const T* __restrict__ W,
                                                         const T* __restrict__ add, const T* __restrict__ A,
                                                         T* __restrict__ raw, T* __restrict__ gz, int n, int lg) {
    __shared__ T sw[9 * CIN * COUT];  // [tap][cout][cin]
    for (int k = threadIdx.x; k < 9 * CIN * COUT; k += kThreads) {
        const int co = k / (9 * CIN), ci = (k / 9) % CIN, tap = k % 9;
        sw[(tap * COUT + co) * CIN + ci] = W[k];
    }
    __syncthreads();
    const long long nn = 1LL << (2 * lg);
    const long long first = (long long)blockIdx.x * kChunk;
    const int b = int(first >> (2 * lg));
    const T* g = g_out + (long long)b * nn * COUT;
    const long long base = (long long)b * nn * CIN;
    const int mask = n - 1;
#pragma unroll 1
    for (int k = 0; k < kPix; ++k) {
        const int q = int((first & (nn - 1)) + threadIdx.x + k * kThreads);
        const int i = q >> lg, j = q & mask;
        T acc[CIN];
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) acc[ci] = T(0);
#pragma unroll(taps_unroll<T, CIN, COUT>())
        for (int tap = 0; tap < 9; ++tap) {
                const int a = tap / 3, e = tap % 3;
                const int s = (((i + 1 - a) & mask) << lg) | ((j + 1 - e) & mask);
                T v[COUT];
                load_px<T, COUT>(g + (long long)s * COUT, v);
                const T* w = sw + tap * COUT * CIN;
#pragma unroll
                for (int co = 0; co < COUT; ++co)
#pragma unroll
                    for (int ci = 0; ci < CIN; ++ci) acc[ci] = fma(w[co * CIN + ci], v[co], acc[ci]);
            }
        const long long o = base + (long long)q * CIN;
        if (add) {
            T ad[CIN];
            load_px<T, CIN>(add + o, ad);
#pragma unroll
            for (int ci = 0; ci < CIN; ++ci) acc[ci] += ad[ci];
        }
        if (raw) store_px<T, CIN>(raw + o, acc);
        T av[CIN];
        load_px<T, CIN>(A + o, av);
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) acc[ci] *= T(1) - av[ci] * av[ci];
        store_px<T, CIN>(gz + o, acc);
    }
}

// Weight-gradient partials of one conv: block (x, y) sums, over its
// kThreads * kWgPix pixels, g[p][co] in[p + d_tap][ci] for the co/ci chunk y
// (and g[p][co] for the biases, in chunk ci = 0), in a fixed order; the
// layer's parameters are [COUT][CIN][9] then [COUT].
template <typename T, int CIN, int COUT, int CI_CH, int CO_CH>
__global__ void __launch_bounds__(kThreads) wgrad_kernel(const T* __restrict__ in, const T* __restrict__ g,
                                                         double* __restrict__ part, long long total, int n, int lg) {
    constexpr int NW = CO_CH * CI_CH * 9;
    constexpr int NACC = NW + CO_CH;
    constexpr int NP = COUT * CIN * 9 + COUT;
    constexpr int CI_CHUNKS = CIN / CI_CH;
    __shared__ T red[kThreads / 32][NACC];
    const int co0 = (blockIdx.y / CI_CHUNKS) * CO_CH, ci0 = (blockIdx.y % CI_CHUNKS) * CI_CH;
    T acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = T(0);
    const long long nn = 1LL << (2 * lg);
    const int mask = n - 1;
    const long long first = (long long)blockIdx.x * kThreads * kWgPix;
#pragma unroll 1
    for (int k = 0; k < kWgPix; ++k) {
        const long long p = first + threadIdx.x + (long long)k * kThreads;
        if (p >= total) break;
        const long long b = p >> (2 * lg);
        const int q = int(p & (nn - 1));
        const int i = q >> lg, j = q & mask;
        T gv[CO_CH];
#pragma unroll
        for (int c = 0; c < CO_CH; ++c) gv[c] = g[p * COUT + co0 + c];
#pragma unroll
        for (int c = 0; c < CO_CH; ++c) acc[NW + c] += gv[c];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const int s = (((i + a - 1) & mask) << lg) | ((j + e - 1) & mask);
                T v[CI_CH];
                load_px<T, CI_CH>(in + (b * nn + s) * CIN + ci0, v);
#pragma unroll
                for (int c = 0; c < CO_CH; ++c)
#pragma unroll
                    for (int d = 0; d < CI_CH; ++d) acc[(c * CI_CH + d) * 9 + a * 3 + e] = fma(gv[c], v[d], acc[(c * CI_CH + d) * 9 + a * 3 + e]);
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
        T s = acc[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NACC; k += kThreads) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += double(red[w][k]);
        int idx;
        if (k < NW) {
            const int c = k / (CI_CH * 9), d = (k / 9) % CI_CH, tap = k % 9;
            idx = ((co0 + c) * CIN + ci0 + d) * 9 + tap;
        } else {
            if (ci0 != 0) continue;
            idx = COUT * CIN * 9 + co0 + (k - NW);
        }
        part[(long long)blockIdx.x * NP + idx] = s;
    }
}

// Sum the weight-gradient partials of `blocks` blocks in block order.
template <typename T>
__global__ void wgrad_finish_kernel(const double* __restrict__ part, int blocks, int nw, int nb, T* __restrict__ gw,
                                    T* __restrict__ gb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int np = nw + nb;
    if (k >= np) return;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += part[(long long)b * np + k];
    if (k < nw) gw[k] = T(s);
    else gb[k - nw] = T(s);
}

// dL/d(output conv) from dL/d(network output): the limiter's mask (pass where
// lo < s < hi, s the value before the clamp) and, with the mass shift, per-block
// sums for its field mean.
template <typename T>
__global__ void __launch_bounds__(kThreads) gmask_kernel(const T* __restrict__ gout, const T* __restrict__ s,
                                                         T* __restrict__ go, double* __restrict__ part, int limiter,
                                                         double lo, double hi) {
    __shared__ double red[kThreads / 32];
    const long long first = (long long)blockIdx.x * kChunk;
    T sum = T(0);
    for (int k = 0; k < kPix; ++k) {
        const long long p = first + threadIdx.x + k * kThreads;
        T g = gout[p];
        if (limiter) {
            const double v = double(s[p]);
            if (!(v > lo && v < hi)) g = T(0);
        }
        go[p] = g;
        sum += g;
    }
    if (part) {
        double d = double(sum);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            part[blockIdx.x] = t;
        }
    }
}

// go -= field mean of go (the transpose of the mass shift).
template <typename T>
__global__ void __launch_bounds__(kThreads) gcenter_kernel(T* __restrict__ go, const double* __restrict__ part,
                                                           int parts, int lg) {
    const long long first = (long long)blockIdx.x * kChunk;
    const int b = int(first >> (2 * lg));
    __shared__ double mean;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < parts; ++k) t += part[(long long)b * parts + k];
        mean = t / double(1LL << (2 * lg));
    }
    __syncthreads();
    for (int k = 0; k < kPix; ++k) {
        const long long p = first + threadIdx.x + k * kThreads;
        go[p] = T(double(go[p]) - mean);
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Ws {
    void *x, *h, *t, *s, *go, *gx, *gz, *gh;
    double *part, *fpart;
};

int wgrad_blocks(long long total) { return int((total + kThreads * kWgPix - 1) / (kThreads * kWgPix)); }

size_t ws_layout(const acnn_desc* d, int n, int batch, Ws* wout, void* base) {
    Ws tmp;
    Ws* w = wout ? wout : &tmp;
    const size_t es = elem_size(d->precision);
    const long long nn = (long long)n * n, px = nn * batch;
    const int C = d->channels, R = d->blocks;
    const size_t sizes[8] = {es * px * C * (R + 1), es * px * C * (R > 0 ? R : 1), es * px * C * (R > 0 ? R : 1),
                             es * px, es * px, es * px * C, es * px * C, es * px * C};
    const size_t npmax = size_t(9 * C * C + C);
    const size_t part_bytes = sizeof(double) * npmax * size_t(wgrad_blocks(px));
    const size_t fpart_bytes = sizeof(double) * size_t(px / kChunk + 1);
    size_t off = 0;
    char* p = static_cast<char*>(base);
    void** slots[8] = {&w->x, &w->h, &w->t, &w->s, &w->go, &w->gx, &w->gz, &w->gh};
    for (int k = 0; k < 8; ++k) {
        *slots[k] = p ? p + off : nullptr;
        off += align256(sizes[k]);
    }
    w->part = p ? reinterpret_cast<double*>(p + off) : nullptr;
    off += align256(part_bytes);
    w->fpart = p ? reinterpret_cast<double*>(p + off) : nullptr;
    off += align256(fpart_bytes);
    return off;
}

template <typename T, int C>
int forward_layers_t(const acnn_desc* d, int n, int batch, const T* u, T* out, AcnnIO io, const Ws& w,
                     cudaStream_t st) {
    const int lg = __builtin_ctz(n);
    const long long nn = (long long)n * n, px = nn * batch;
    const int R = d->blocks;
    const unsigned grid = unsigned(px / kChunk);
    const T* W = static_cast<const T*>(d->w);
    const T* B = static_cast<const T*>(d->b);
    T* x = static_cast<T*>(w.x);
    T* h = static_cast<T*>(w.h);
    T* t = static_cast<T*>(w.t);
    long long wo, bo;
    acnn_offsets(C, R, 0, &wo, &bo);
    conv_kernel<T, 1, C, kModeTanh><<<grid, kThreads, 0, st>>>(u, io.in_bs, io.in_map, x, nn * C, nullptr, W + wo,
                                                                B + bo, nullptr, nullptr, n, lg);
    ACPR_LAUNCH_CHECK();
    for (int r = 0; r < R; ++r) {
        T* xr = x + (long long)r * px * C;
        T* hr = h + (long long)r * px * C;
        T* tr = t + (long long)r * px * C;
        acnn_offsets(C, R, 1 + 2 * r, &wo, &bo);
        conv_kernel<T, C, C, kModeTanh><<<grid, kThreads, 0, st>>>(xr, nn * C, nullptr, hr, nn * C, nullptr, W + wo,
                                                                    B + bo, nullptr, nullptr, n, lg);
        ACPR_LAUNCH_CHECK();
        acnn_offsets(C, R, 2 + 2 * r, &wo, &bo);
        conv_kernel<T, C, C, kModeBlockOut><<<grid, kThreads, 0, st>>>(hr, nn * C, nullptr, tr, nn * C, nullptr,
                                                                        W + wo, B + bo, xr, xr + px * C, n, lg);
        ACPR_LAUNCH_CHECK();
    }
    acnn_offsets(C, R, 1 + 2 * R, &wo, &bo);
    out_conv_kernel<T, C><<<grid, kThreads, 0, st>>>(x + (long long)R * px * C, out, io.out_bs, io.out_map, W + wo,
                                                     B + bo, u, io.in_bs, io.in_map, d->mass_fix ? w.fpart : nullptr,
                                                     n, lg);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

template <typename T>
int forward_layers(const acnn_desc* d, int n, int batch, const void* u, void* out, AcnnIO io, const Ws& w,
                   cudaStream_t st) {
    int rc = d->channels == 4 ? forward_layers_t<T, 4>(d, n, batch, static_cast<const T*>(u), static_cast<T*>(out), io, w, st)
                              : forward_layers_t<T, 16>(d, n, batch, static_cast<const T*>(u), static_cast<T*>(out), io, w, st);
    if (rc) return rc;
    if (d->mass_fix || d->limiter)
        return acnn_post<T>(n, batch, static_cast<const T*>(u), static_cast<T*>(out), io, w.fpart,
                            int((long long)n * n / kChunk), d->mass_fix, d->limiter, d->lo, d->hi, st);
    return AC_OK;
}

template <typename T, int CIN, int COUT>
int wgrad(const T* in, const T* g, T* gw, T* gb, double* part, long long px, int n, int lg, cudaStream_t st) {
    constexpr int CI_CH = CIN < 4 ? CIN : 4;
    constexpr int CO_CH = sizeof(T) == 8 ? (COUT < 2 ? COUT : 2) : (COUT < 4 ? COUT : 4);
    const int blocks = wgrad_blocks(px);
    dim3 grid(blocks, (COUT / CO_CH) * (CIN / CI_CH));
    wgrad_kernel<T, CIN, COUT, CI_CH, CO_CH><<<grid, kThreads, 0, st>>>(in, g, part, px, n, lg);
    ACPR_LAUNCH_CHECK();
    const int np = COUT * CIN * 9 + COUT;
    wgrad_finish_kernel<T><<<(np + 127) / 128, 128, 0, st>>>(part, blocks, COUT * CIN * 9, COUT, gw, gb);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

template <typename T, int C>
int backward_t(const acnn_desc* d, int n, int batch, const T* u, const T* gout, T* gw, T* gb, const Ws& w,
               cudaStream_t st) {
    const int lg = __builtin_ctz(n);
    const long long nn = (long long)n * n, px = nn * batch;
    const int R = d->blocks;
    const unsigned grid = unsigned(px / kChunk);
    const T* W = static_cast<const T*>(d->w);
    T* x = static_cast<T*>(w.x);
    T* h = static_cast<T*>(w.h);
    T* t = static_cast<T*>(w.t);
    T* go = static_cast<T*>(w.go);
    T* gx = static_cast<T*>(w.gx);
    T* gz = static_cast<T*>(w.gz);
    T* gh = static_cast<T*>(w.gh);
    gmask_kernel<T><<<grid, kThreads, 0, st>>>(gout, static_cast<const T*>(w.s), go, d->mass_fix ? w.fpart : nullptr,
                                               d->limiter, d->lo, d->hi);
    ACPR_LAUNCH_CHECK();
    if (d->mass_fix) {
        gcenter_kernel<T><<<grid, kThreads, 0, st>>>(go, w.fpart, int(nn / kChunk), lg);
        ACPR_LAUNCH_CHECK();
    }
    long long wo, bo;
    int rc;
    // output conv: parameters, then dL/dx_R (raw into gx) and, for the last
    // block, dL/dz2 = gx (1 - t^2); with no blocks dL/dz_in = gx (1 - x_0^2)
    acnn_offsets(C, R, 1 + 2 * R, &wo, &bo);
    if ((rc = wgrad<T, C, 1>(x + (long long)R * px * C, go, gw + wo, gb + bo, w.part, px, n, lg, st))) return rc;
    const T* A = R > 0 ? t + (long long)(R - 1) * px * C : x;
    dgrad_kernel<T, C, 1><<<grid, kThreads, 0, st>>>(go, W + wo, nullptr, A, gx, gz, n, lg);
    ACPR_LAUNCH_CHECK();
    for (int r = R - 1; r >= 0; --r) {
        T* xr = x + (long long)r * px * C;
        T* hr = h + (long long)r * px * C;
        // conv2: dW2 from (h_r, gz); dL/dz1 = conv2^T(gz) (1 - h_r^2) into gh
        acnn_offsets(C, R, 2 + 2 * r, &wo, &bo);
        if ((rc = wgrad<T, C, C>(hr, gz, gw + wo, gb + bo, w.part, px, n, lg, st))) return rc;
        dgrad_kernel<T, C, C><<<grid, kThreads, 0, st>>>(gz, W + wo, nullptr, hr, nullptr, gh, n, lg);
        ACPR_LAUNCH_CHECK();
        // conv1: dW1 from (x_r, gh); dL/dx_r = gx + conv1^T(gh), and the next
        // gradient to propagate: times (1 - t_{r-1}^2), or (1 - x_0^2) at r = 0
        acnn_offsets(C, R, 1 + 2 * r, &wo, &bo);
        if ((rc = wgrad<T, C, C>(xr, gh, gw + wo, gb + bo, w.part, px, n, lg, st))) return rc;
        const T* An = r > 0 ? t + (long long)(r - 1) * px * C : x;
        dgrad_kernel<T, C, C><<<grid, kThreads, 0, st>>>(gh, W + wo, gx, An, gx, gz, n, lg);
        ACPR_LAUNCH_CHECK();
    }
    acnn_offsets(C, R, 0, &wo, &bo);
    return wgrad<T, 1, C>(u, gz, gw + wo, gb + bo, w.part, px, n, lg, st);
}

}  // namespace

size_t acnn_train_bytes_for(const acnn_desc* d, int n, int batch) { return ws_layout(d, n, batch, nullptr, nullptr); }

int acnn_forward_layers(const acnn_desc* d, int n, int batch, const void* u, void* out, AcnnIO io, void* ws,
                        cudaStream_t st) {
    Ws w;
    ws_layout(d, n, batch, &w, ws);
    return d->precision == AC_F64 ? forward_layers<double>(d, n, batch, u, out, io, w, st)
                                  : forward_layers<float>(d, n, batch, u, out, io, w, st);
}

template <typename T>
__global__ void save_s_kernel(const T* __restrict__ out, T* __restrict__ s, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) s[i] = out[i];
}

int acnn_forward_train_impl(const acnn_desc* d, int n, int batch, const void* u, void* out, void* ws,
                            cudaStream_t st) {
    Ws w;
    ws_layout(d, n, batch, &w, ws);
    const long long nn = (long long)n * n;
    AcnnIO io{nullptr, nullptr, nn, nn};
    int rc;
    if (d->precision == AC_F64) {
        rc = d->channels == 4 ? forward_layers_t<double, 4>(d, n, batch, static_cast<const double*>(u), static_cast<double*>(out), io, w, st)
                              : forward_layers_t<double, 16>(d, n, batch, static_cast<const double*>(u), static_cast<double*>(out), io, w, st);
    } else {
        rc = d->channels == 4 ? forward_layers_t<float, 4>(d, n, batch, static_cast<const float*>(u), static_cast<float*>(out), io, w, st)
                              : forward_layers_t<float, 16>(d, n, batch, static_cast<const float*>(u), static_cast<float*>(out), io, w, st);
    }
    if (rc) return rc;
    // the value before the limiter (after the mass shift) is what the
    // backward pass masks with; acnn_post saves it when asked
    const int parts = int(nn / kChunk);
    if (d->mass_fix || d->limiter) {
        if (d->precision == AC_F64)
            return acnn_post<double>(n, batch, static_cast<const double*>(u), static_cast<double*>(out), io,
                                     w.fpart, parts, d->mass_fix, d->limiter, d->lo, d->hi, st,
                                     static_cast<double*>(w.s));
        return acnn_post<float>(n, batch, static_cast<const float*>(u), static_cast<float*>(out), io, w.fpart, parts,
                                d->mass_fix, d->limiter, d->lo, d->hi, st, static_cast<float*>(w.s));
    }
    const long long count = nn * batch;
    if (d->precision == AC_F64)
        save_s_kernel<double><<<unsigned((count + 255) / 256), 256, 0, st>>>(static_cast<const double*>(out),
                                                                            static_cast<double*>(w.s), count);
    else
        save_s_kernel<float><<<unsigned((count + 255) / 256), 256, 0, st>>>(static_cast<const float*>(out),
                                                                          static_cast<float*>(w.s), count);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

int acnn_backward_impl(const acnn_desc* d, int n, int batch, const void* u, const void* gout, void* gw, void* gb,
                       void* ws, cudaStream_t st) {
    Ws w;
    ws_layout(d, n, batch, &w, ws);
    if (d->precision == AC_F64) {
        auto* W = static_cast<double*>(gw);
        auto* B = static_cast<double*>(gb);
        return d->channels == 4 ? backward_t<double, 4>(d, n, batch, static_cast<const double*>(u), static_cast<const double*>(gout), W, B, w, st)
                                : backward_t<double, 16>(d, n, batch, static_cast<const double*>(u), static_cast<const double*>(gout), W, B, w, st);
    }
    auto* W = static_cast<float*>(gw);
    auto* B = static_cast<float*>(gb);
    return d->channels == 4 ? backward_t<float, 4>(d, n, batch, static_cast<const float*>(u), static_cast<const float*>(gout), W, B, w, st)
                            : backward_t<float, 16>(d, n, batch, static_cast<const float*>(u), static_cast<const float*>(gout), W, B, w, st);
}

}  // namespace acpr
