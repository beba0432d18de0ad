// acnn.cu -- the paper's ResBlock ACNN / mACNN coarse propagator (Sec. 3.2):
// fused inference kernel, mass shift and limiter, the scheme-residual loss
// (Eq. loss_ACN) with its gradient, Adam, and the training loop of
// Algorithm 1.  The per-layer forward/backward kernels are in acnn_train.cu.
//
// Fused inference (C = 4, up to 3 blocks): one CTA per 32 x 32 output tile and
// field.  The CTA loads the input tile with a halo of 2 blocks + 2 pixels
// (periodic wrap), then runs every convolution in shared memory, each on a
// region one pixel smaller per side than the last, and writes only the 32 x 32
// result: HBM sees one read and one write per pixel.  The parameters (669
// floats for two blocks) travel as a __grid_constant__ kernel argument, so the
// fully unrolled FMAs take them straight from the constant bank.
#include "acnn.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

struct acnn_net {
    acnn_desc d;                 // w, b point at the handle's own device copy
    void* dev_params = nullptr;  // device copy (per-layer path)
    std::vector<char> host;      // packed kernel argument (fused path)
    bool fused = false;
};

namespace acpr {

namespace {

constexpr int kTile = 32;
constexpr int kThreads = 256;

template <typename T, int R>
struct FusedParams {
    T win[4][9];
    T bin[4];
    T wb[2 * R > 0 ? 2 * R : 1][4][4][9];  // [conv][cout][cin][tap]
    T bb[2 * R > 0 ? 2 * R : 1][4];
    T wout[4][9];
    T bout;
    T lo, hi;
    int mass_fix, limiter;
};

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T (&r)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
    }
}

template <typename T>
__device__ __forceinline__ void sts4(T* p, const T (&r)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(r[2], r[3]);
    }
}

template <typename T, int R>
struct FusedShape {
    static constexpr int H = 2 * R + 2;         // halo: one pixel per conv
    static constexpr int S0 = kTile + 2 * H;    // input tile side
    static constexpr int S1 = S0 - 2;           // side of the C-channel frames
    static constexpr size_t smem = sizeof(T) * (size_t(S0) * S0 + 2 * size_t(S1) * S1 * 4);
};

// Every convolution of the fused kernel covers a square frame region whose
// side M is a compile-time constant (and even), so the index arithmetic is
// multiply-shift.  A thread computes two vertically adjacent pixels: it loads
// their 4 x 3 window of 16-byte pixel vectors once (consecutive lanes read
// consecutive pixels, no bank conflicts), then walks the weights in the outer
// loop, each weight feeding both accumulators.

// Hidden C -> C conv L over frame rows/cols [LO, LO + M) of `src`; emit(i, j, acc)
// receives each tanh output.
template <typename T, int R, int L, int LO, int M, typename Emit>
__device__ __forceinline__ void hidden_conv(const FusedParams<T, R>& P, const T* __restrict__ src, Emit emit) {
    constexpr int S1 = FusedShape<T, R>::S1;
    static_assert(M % 2 == 0, "regions have even sides");
    for (int idx = threadIdx.x; idx < M * M / 2; idx += kThreads) {
        const int i = LO + 2 * (idx / M), j = LO + idx % M;
        T v[4][3][4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int e = 0; e < 3; ++e) lds4(src + ((i + rr - 1) * S1 + (j + e - 1)) * 4, v[rr][e]);
        T acc[2][4];
#pragma unroll
        for (int co = 0; co < 4; ++co) acc[0][co] = acc[1][co] = P.bb[L][co];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int ci = 0; ci < 4; ++ci)
#pragma unroll
                    for (int co = 0; co < 4; ++co) {
                        const T w = P.wb[L][co][ci][a * 3 + e];
                        acc[0][co] = fma(w, v[a][e][ci], acc[0][co]);
                        acc[1][co] = fma(w, v[a + 1][e][ci], acc[1][co]);
                    }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
#pragma unroll
            for (int co = 0; co < 4; ++co) acc[p][co] = acnn_tanh(acc[p][co]);
            emit(i + p, j, acc[p]);
        }
    }
}

template <typename T, int R, int r>
__device__ __forceinline__ void run_blocks(const FusedParams<T, R>& P, T* X, T* Hb) {
    if constexpr (r < R) {
        constexpr int S1 = FusedShape<T, R>::S1;
        // conv1: X valid on [2r, S1-2r) -> Hb on [2r+1, S1-2r-1)
        hidden_conv<T, R, 2 * r, 2 * r + 1, S1 - 4 * r - 2>(
            P, X, [&](int i, int j, const T (&h)[4]) { sts4(Hb + (i * S1 + j) * 4, h); });
        __syncthreads();
        // conv2 + skip: X += tanh(conv2(Hb)) on [2r+2, S1-2r-2); conv2 reads Hb only
        hidden_conv<T, R, 2 * r + 1, 2 * r + 2, S1 - 4 * r - 4>(P, Hb, [&](int i, int j, const T (&t)[4]) {
            T x[4];
            lds4(X + (i * S1 + j) * 4, x);
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] += t[c];
            sts4(X + (i * S1 + j) * 4, x);
        });
        __syncthreads();
        run_blocks<T, R, r + 1>(P, X, Hb);
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreads) acnn_fused_kernel(const __grid_constant__ FusedParams<T, R> P,
                                                              const T* __restrict__ u, T* __restrict__ out,
                                                              AcnnIO io, double* __restrict__ part, int n, int lg) {
    using Sh = FusedShape<T, R>;
    constexpr int S0 = Sh::S0, S1 = Sh::S1, H = Sh::H;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* X = reinterpret_cast<T*>(smem_raw);            // [S1][S1][4]
    T* Hb = X + S1 * S1 * 4;                          // [S1][S1][4]
    T* su = Hb + S1 * S1 * 4;                         // [S0][S0]
    const int tiles_x = n >> 5;
    const int ty = blockIdx.x / tiles_x, tx = blockIdx.x % tiles_x;
    const int b = blockIdx.y;
    const T* ub = u + acnn_sel(io.in_map, b) * io.in_bs;
    T* ob = out + acnn_sel(io.out_map, b) * io.out_bs;
    const int mask = n - 1;
    const int y0 = ty * kTile - H, x0 = tx * kTile - H;
    for (int idx = threadIdx.x; idx < S0 * S0; idx += kThreads) {
        const int i = idx / S0, j = idx % S0;
        su[idx] = ub[(long long)((y0 + i) & mask) * n + ((x0 + j) & mask)];
    }
    __syncthreads();
    // input conv 1 -> 4 with tanh over the whole frame: frame (i, j) sits at
    // su (i + 1, j + 1); pairs of rows as in hidden_conv
    for (int idx = threadIdx.x; idx < S1 * S1 / 2; idx += kThreads) {
        const int i = 2 * (idx / S1), j = idx % S1;
        T v[4][3];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int e = 0; e < 3; ++e) v[rr][e] = su[(i + rr) * S0 + (j + e)];
        T acc[2][4];
#pragma unroll
        for (int co = 0; co < 4; ++co) acc[0][co] = acc[1][co] = P.bin[co];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int co = 0; co < 4; ++co) {
                    const T w = P.win[co][a * 3 + e];
                    acc[0][co] = fma(w, v[a][e], acc[0][co]);
                    acc[1][co] = fma(w, v[a + 1][e], acc[1][co]);
                }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
#pragma unroll
            for (int co = 0; co < 4; ++co) acc[p][co] = acnn_tanh(acc[p][co]);
            sts4(X + ((i + p) * S1 + j) * 4, acc[p]);
        }
    }
    __syncthreads();
    run_blocks<T, R, 0>(P, X, Hb);
    // output conv 4 -> 1 on [2R+1, S1-2R-1): exactly the 32 x 32 tile
    constexpr int lo = 2 * R + 1;
    T msum = T(0);
    for (int idx = threadIdx.x; idx < kTile * kTile / 4; idx += kThreads) {
        const int ii = 4 * (idx >> 5), jj = idx & 31;
        const int i = lo + ii, j = lo + jj;
        T v[6][3][4];
#pragma unroll
        for (int rr = 0; rr < 6; ++rr)
#pragma unroll
            for (int e = 0; e < 3; ++e) lds4(X + ((i + rr - 1) * S1 + (j + e - 1)) * 4, v[rr][e]);
        T acc[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[p] = P.bout;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int ci = 0; ci < 4; ++ci) {
                    const T w = P.wout[ci][a * 3 + e];
#pragma unroll
                    for (int p = 0; p < 4; ++p) acc[p] = fma(w, v[p + a][e][ci], acc[p]);
                }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const long long g = (long long)(ty * kTile + ii + p) * n + tx * kTile + jj;
            T o = acc[p];
            if (P.mass_fix) {
                msum += o - su[(i + p + 1) * S0 + (j + 1)];
            } else if (P.limiter) {
                o = o < P.lo ? P.lo : (o > P.hi ? P.hi : o);
            }
            ob[g] = o;
        }
    }
    if (P.mass_fix) {
        __shared__ double red[kThreads / 32];
        double s = double(msum);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            part[(long long)b * gridDim.x + blockIdx.x] = t;
        }
    }
    (void)lg;
}

// out = clamp(out + shift_b), shift_b = -(sum of the field's partials) / n^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) post_kernel(T* __restrict__ out, AcnnIO io,
                                                        const double* __restrict__ part, int parts, int mass_fix,
                                                        int limiter, double lo, double hi, T* __restrict__ s_save,
                                                        int lg, int per_block) {
    const int b = blockIdx.y;
    __shared__ double shift;
    if (threadIdx.x == 0) {
        double t = 0.0;
        if (mass_fix)
            for (int k = 0; k < parts; ++k) t += part[(long long)b * parts + k];
        shift = -t / double(1LL << (2 * lg));
    }
    __syncthreads();
    T* ob = out + acnn_sel(io.out_map, b) * io.out_bs;
    const long long nn = 1LL << (2 * lg);
    const long long first = (long long)blockIdx.x * per_block;
    for (int k = threadIdx.x; k < per_block; k += kThreads) {
        const long long q = first + k;
        double v = double(ob[q]) + shift;
        if (s_save) s_save[b * nn + q] = T(v);
        if (limiter) v = v < lo ? lo : (v > hi ? hi : v);
        ob[q] = T(v);
    }
}

// ------------------------------------------------------------------ loss --
constexpr int kLossPix = 4;  // pixels per thread: a block covers 1024 pixels of one field

__device__ __forceinline__ double dsum_block(double s, double* red) {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

template <typename T>
__device__ __forceinline__ T fdw(T u) { return u - u * u * u; }

// Per-block sums of f(U0) and f(U1) (mass-conserving variant only).
template <typename T>
__global__ void __launch_bounds__(kThreads) loss_fsum_kernel(const T* __restrict__ U0, const T* __restrict__ U1,
                                                             double* __restrict__ fpart) {
    __shared__ double red[kThreads / 32];
    const long long first = (long long)blockIdx.x * kThreads * kLossPix;
    T s0 = T(0), s1 = T(0);
    for (int k = 0; k < kLossPix; ++k) {
        const long long p = first + threadIdx.x + k * kThreads;
        s0 += fdw(U0[p]);
        s1 += fdw(U1[p]);
    }
    const double t0 = dsum_block(double(s0), red);
    const double t1 = dsum_block(double(s1), red);
    if (threadIdx.x == 0) {
        fpart[2 * blockIdx.x] = t0;
        fpart[2 * blockIdx.x + 1] = t1;
    }
}

// r = U1 - U0 - dt/2 (eps^2 Lap_h (U1 + U0) + f(U1) + f(U0) - g1 - g0) and the
// block's sums of r and r^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) loss_resid_kernel(const T* __restrict__ U0, const T* __restrict__ U1,
                                                              T* __restrict__ r, const double* __restrict__ fpart,
                                                              double* __restrict__ rpart, int parts, int lg,
                                                              double half_dt, double e2_h2, int mass) {
    __shared__ double red[kThreads / 32];
    __shared__ double gsum;
    const long long nn = 1LL << (2 * lg);
    const long long first = (long long)blockIdx.x * kThreads * kLossPix;
    const long long b = first >> (2 * lg);
    if (threadIdx.x == 0) {
        double t = 0.0;
        if (mass)
            for (int k = 0; k < parts; ++k) t += fpart[2 * (b * parts + k)] + fpart[2 * (b * parts + k) + 1];
        gsum = t / double(nn);
    }
    __syncthreads();
    const T g = T(gsum);
    const int n = 1 << lg, mask = n - 1;
    const T* a0 = U0 + b * nn;
    const T* a1 = U1 + b * nn;
    T s = T(0), s2 = T(0);
    for (int k = 0; k < kLossPix; ++k) {
        const int q = int((first & (nn - 1)) + threadIdx.x + k * kThreads);
        const int i = q >> lg, j = q & mask;
        const int up = (((i - 1) & mask) << lg) | j, dn = (((i + 1) & mask) << lg) | j;
        const int lf = (i << lg) | ((j - 1) & mask), rt = (i << lg) | ((j + 1) & mask);
        const T c0 = a0[q], c1 = a1[q];
        const T lap = (a0[up] + a1[up]) + (a0[dn] + a1[dn]) + (a0[lf] + a1[lf]) + (a0[rt] + a1[rt]) -
                      T(4) * (c0 + c1);
        const T rv = c1 - c0 - T(half_dt) * (T(e2_h2) * lap + fdw(c1) + fdw(c0) - g);
        r[b * nn + q] = rv;
        s += rv;
        s2 += rv * rv;
    }
    const double t = dsum_block(double(s), red);
    const double t2 = dsum_block(double(s2), red);
    if (threadIdx.x == 0) {
        rpart[2 * blockIdx.x] = t;
        rpart[2 * blockIdx.x + 1] = t2;
    }
}

// grad = 2/(B n^2) (r - dt/2 (eps^2 Lap_h r + f'(U1) r - [mass] f'(U1) mean r)); block 0
// also writes the loss (sum of all r^2 partials in order) / (B n^2).
template <typename T>
__global__ void __launch_bounds__(kThreads) loss_grad_kernel(const T* __restrict__ U1, const T* __restrict__ r,
                                                             const double* __restrict__ rpart, int parts,
                                                             int total_blocks, T* __restrict__ grad,
                                                             double* __restrict__ loss, int lg, double half_dt,
                                                             double e2_h2, int mass, double scale) {
    __shared__ double rmean;
    const long long nn = 1LL << (2 * lg);
    const long long first = (long long)blockIdx.x * kThreads * kLossPix;
    const long long b = first >> (2 * lg);
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < parts; ++k) t += rpart[2 * (b * parts + k)];
        rmean = t / double(nn);
        if (blockIdx.x == 0) {
            double l = 0.0;
            for (int k = 0; k < total_blocks; ++k) l += rpart[2 * k + 1];
            *loss = l * scale * 0.5;
        }
    }
    __syncthreads();
    if (!grad) return;
    const T rm = T(rmean);
    const int n = 1 << lg, mask = n - 1;
    const T* rb = r + b * nn;
    for (int k = 0; k < kLossPix; ++k) {
        const int q = int((first & (nn - 1)) + threadIdx.x + k * kThreads);
        const int i = q >> lg, j = q & mask;
        const int up = (((i - 1) & mask) << lg) | j, dn = (((i + 1) & mask) << lg) | j;
        const int lf = (i << lg) | ((j - 1) & mask), rt = (i << lg) | ((j + 1) & mask);
        const T rv = rb[q];
        const T lap = rb[up] + rb[dn] + rb[lf] + rb[rt] - T(4) * rv;
        const T u = U1[b * nn + q];
        const T fp = T(1) - T(3) * u * u;
        const T jr = T(e2_h2) * lap + fp * rv - (mass ? fp * rm : T(0));
        grad[b * nn + q] = T(scale) * (rv - T(half_dt) * jr);
    }
}

template <typename T>
__global__ void adam_kernel(T* __restrict__ w, const T* __restrict__ g, T* __restrict__ m, T* __restrict__ v,
                            long long count, T lr, T b1, T b2, T eps, T c1, T c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const T gi = g[i];
    const T mi = b1 * m[i] + (T(1) - b1) * gi;
    const T vi = b2 * v[i] + (T(1) - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
}

template <typename T, int R>
void pack_fused(const acnn_desc& d, const T* w, const T* b, std::vector<char>& out) {
    FusedParams<T, R> P;
    std::memset(&P, 0, sizeof(P));
    int wo = 0, bo = 0;
    for (int co = 0; co < 4; ++co) {
        for (int t = 0; t < 9; ++t) P.win[co][t] = w[wo + co * 9 + t];
        P.bin[co] = b[bo + co];
    }
    wo += 36;
    bo += 4;
    for (int l = 0; l < 2 * R; ++l) {
        for (int co = 0; co < 4; ++co) {
            for (int ci = 0; ci < 4; ++ci)
                for (int t = 0; t < 9; ++t) P.wb[l][co][ci][t] = w[wo + (co * 4 + ci) * 9 + t];
            P.bb[l][co] = b[bo + co];
        }
        wo += 144;
        bo += 4;
    }
    for (int ci = 0; ci < 4; ++ci)
        for (int t = 0; t < 9; ++t) P.wout[ci][t] = w[wo + ci * 9 + t];
    P.bout = b[bo];
    P.lo = T(d.lo);
    P.hi = T(d.hi);
    P.mass_fix = d.mass_fix;
    P.limiter = d.limiter;
    out.resize(sizeof(P));
    std::memcpy(out.data(), &P, sizeof(P));
}

template <typename T, int R>
int launch_fused_r(const acnn_net* net, int n, int batch, const T* u, T* out, AcnnIO io, double* part,
                   cudaStream_t st) {
    using Sh = FusedShape<T, R>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(acnn_fused_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(Sh::smem));
    });
    ACPR_CUDA(attr_err);
    FusedParams<T, R> P;
    std::memcpy(&P, net->host.data(), sizeof(P));
    const int tiles = (n / kTile) * (n / kTile);
    acnn_fused_kernel<T, R><<<dim3(tiles, batch), kThreads, Sh::smem, st>>>(P, u, out, io, part, n, __builtin_ctz(n));
    ACPR_LAUNCH_CHECK();
    if (net->d.mass_fix)
        return acnn_post<T>(n, batch, u, out, io, part, tiles, 1, net->d.limiter, net->d.lo, net->d.hi, st);
    return AC_OK;
}

template <typename T>
int launch_fused(const acnn_net* net, int n, int batch, const T* u, T* out, AcnnIO io, double* part,
                 cudaStream_t st) {
    switch (net->d.blocks) {
        case 0: return launch_fused_r<T, 0>(net, n, batch, u, out, io, part, st);
        case 1: return launch_fused_r<T, 1>(net, n, batch, u, out, io, part, st);
        case 2: return launch_fused_r<T, 2>(net, n, batch, u, out, io, part, st);
        default: return launch_fused_r<T, 3>(net, n, batch, u, out, io, part, st);
    }
}

size_t fused_work_bytes(int n, int batch) { return sizeof(double) * size_t(n / kTile) * (n / kTile) * batch; }

bool supported_n(int n) { return is_pow2(n) && n >= 32 && n <= 1024; }

}  // namespace

template <typename T>
int acnn_post(int n, int batch, const T* u, T* out, AcnnIO io, const double* part, int parts, int mass_fix,
              int limiter, double lo, double hi, cudaStream_t st, T* s_save) {
    (void)u;
    const long long nn = (long long)n * n;
    const int per_block = nn >= 4096 ? 4096 : int(nn);
    post_kernel<T><<<dim3(unsigned(nn / per_block), batch), kThreads, 0, st>>>(out, io, part, parts, mass_fix, limiter,
                                                                                lo, hi, s_save, __builtin_ctz(n),
                                                                                per_block);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

template int acnn_post<float>(int, int, const float*, float*, AcnnIO, const double*, int, int, int, double, double,
                              cudaStream_t, float*);
template int acnn_post<double>(int, int, const double*, double*, AcnnIO, const double*, int, int, int, double, double,
                               cudaStream_t, double*);

int acnn_check(const acnn_desc* d) {
    ACPR_CHECK_ARG(d != nullptr, "acnn_desc is NULL");
    if (d->channels != 4 && d->channels != 16) {
        set_error("ACNN: channels=%d not built (4 or 16)", d->channels);
        return AC_ERR_UNSUPPORTED;
    }
    if (d->blocks < 0 || d->blocks > 4) {
        set_error("ACNN: blocks=%d not built (0..4)", d->blocks);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(d->precision == AC_F64 || d->precision == AC_F32, "bad ACNN precision");
    ACPR_CHECK_ARG(d->w && d->b, "null ACNN parameter pointer");
    ACPR_CHECK_ARG(!d->limiter || d->lo < d->hi, "limiter needs lo < hi");
    return AC_OK;
}

int acnn_precision(const acnn_net* net) { return net->d.precision; }

// Coarse evaluation for the Parareal driver.
int acnn_forward_mapped(const acnn_net* net, int n, int batch, const void* u, long long in_bs, const int* in_map,
                        void* out, long long out_bs, const int* out_map, void* work, size_t work_bytes,
                        cudaStream_t st) {
    ACPR_CHECK_ARG(net, "null ACNN handle");
    if (batch == 0) return AC_OK;
    ACPR_CHECK_ARG(batch > 0, "batch must be >= 0");
    if (!supported_n(n)) {
        set_error("acnn_forward: n=%d unsupported (power of two in [32, 1024])", n);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(u && out && u != out, "bad field pointers");
    const size_t need = acnn_work_bytes(net, n, batch);
    ACPR_CHECK_ARG(work && work_bytes >= need, "ACNN work buffer too small: need %zu bytes", need);
    AcnnIO io{in_map, out_map, in_bs, out_bs};
    if (net->fused) {
        if (net->d.precision == AC_F64)
            return launch_fused<double>(net, n, batch, static_cast<const double*>(u), static_cast<double*>(out), io,
                                        static_cast<double*>(work), st);
        return launch_fused<float>(net, n, batch, static_cast<const float*>(u), static_cast<float*>(out), io,
                                   static_cast<double*>(work), st);
    }
    return acnn_forward_layers(&net->d, n, batch, u, out, io, work, st);
}

}  // namespace acpr

using namespace acpr;

extern "C" long long acnn_param_count(int channels, int blocks, long long* num_bias) {
    if ((channels != 4 && channels != 16) || blocks < 0 || blocks > 4) return -1;
    long long wo, bo;
    acnn_offsets(channels, blocks, acnn_convs(blocks), &wo, &bo);
    if (num_bias) *num_bias = bo;
    return wo;
}

extern "C" int acnn_create(const acnn_desc* desc, acnn_net** out) {
    ACPR_CHECK_ARG(out, "null output pointer");
    *out = nullptr;
    int rc = acnn_check(desc);
    if (rc) return rc;
    long long nb = 0;
    const long long nw = acnn_param_count(desc->channels, desc->blocks, &nb);
    const size_t es = elem_size(desc->precision);
    auto* net = new acnn_net();
    net->d = *desc;
    if (cudaMalloc(&net->dev_params, es * size_t(nw + nb)) != cudaSuccess) {
        delete net;
        set_error("acnn_create: cudaMalloc failed");
        return AC_ERR_NOMEM;
    }
    std::vector<char> hw(es * size_t(nw)), hb(es * size_t(nb));
    cudaError_t e = cudaMemcpy(hw.data(), desc->w, hw.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hb.data(), desc->b, hb.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(net->dev_params, hw.data(), hw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(static_cast<char*>(net->dev_params) + hw.size(), hb.data(), hb.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(net->dev_params);
        delete net;
        set_error("acnn_create: parameter copy failed: %s", cudaGetErrorString(e));
        return AC_ERR_CUDA;
    }
    net->d.w = net->dev_params;
    net->d.b = static_cast<char*>(net->dev_params) + hw.size();
    net->fused = desc->channels == 4 && desc->blocks <= 3;
    if (net->fused) {
        if (desc->precision == AC_F64) {
            const auto* w = reinterpret_cast<const double*>(hw.data());
            const auto* b = reinterpret_cast<const double*>(hb.data());
            switch (desc->blocks) {
                case 0: pack_fused<double, 0>(*desc, w, b, net->host); break;
                case 1: pack_fused<double, 1>(*desc, w, b, net->host); break;
                case 2: pack_fused<double, 2>(*desc, w, b, net->host); break;
                default: pack_fused<double, 3>(*desc, w, b, net->host); break;
            }
        } else {
            const auto* w = reinterpret_cast<const float*>(hw.data());
            const auto* b = reinterpret_cast<const float*>(hb.data());
            switch (desc->blocks) {
                case 0: pack_fused<float, 0>(*desc, w, b, net->host); break;
                case 1: pack_fused<float, 1>(*desc, w, b, net->host); break;
                case 2: pack_fused<float, 2>(*desc, w, b, net->host); break;
                default: pack_fused<float, 3>(*desc, w, b, net->host); break;
            }
        }
    }
    *out = net;
    return AC_OK;
}

extern "C" void acnn_destroy(acnn_net* net) {
    if (!net) return;
    cudaFree(net->dev_params);
    delete net;
}

extern "C" size_t acnn_work_bytes(const acnn_net* net, int n, int batch) {
    if (!net || !supported_n(n) || batch < 0) return 0;
    if (net->fused) return fused_work_bytes(n, batch);
    return acnn_train_bytes_for(&net->d, n, batch);
}

extern "C" int acnn_forward(const acnn_net* net, int n, int batch, const void* u_in, void* u_out, void* work,
                            size_t work_bytes, acpr_stream stream) {
    const long long nn = (long long)n * n;
    return acnn_forward_mapped(net, n, batch, u_in, nn, nullptr, u_out, nn, nullptr, work, work_bytes,
                               reinterpret_cast<cudaStream_t>(stream));
}

extern "C" size_t acnn_train_bytes(const acnn_desc* desc, int n, int batch) {
    if (acnn_check(desc) || !supported_n(n) || batch <= 0) return 0;
    return acnn_train_bytes_for(desc, n, batch);
}

extern "C" int acnn_forward_train(const acnn_desc* desc, int n, int batch, const void* u_in, void* u_out,
                                  void* train_ws, acpr_stream stream) {
    int rc = acnn_check(desc);
    if (rc) return rc;
    if (!supported_n(n)) {
        set_error("acnn_forward_train: n=%d unsupported (power of two in [32, 1024])", n);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(batch > 0 && u_in && u_out && train_ws && u_in != u_out, "bad acnn_forward_train arguments");
    return acnn_forward_train_impl(desc, n, batch, u_in, u_out, train_ws, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int acnn_backward(const acnn_desc* desc, int n, int batch, const void* u_in, const void* grad_out,
                             void* grad_w, void* grad_b, void* train_ws, acpr_stream stream) {
    int rc = acnn_check(desc);
    if (rc) return rc;
    if (!supported_n(n)) {
        set_error("acnn_backward: n=%d unsupported (power of two in [32, 1024])", n);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(batch > 0 && u_in && grad_out && grad_w && grad_b && train_ws, "bad acnn_backward arguments");
    return acnn_backward_impl(desc, n, batch, u_in, grad_out, grad_w, grad_b, train_ws,
                              reinterpret_cast<cudaStream_t>(stream));
}

extern "C" size_t loss_acn_work_bytes(int n, int batch) {
    if (!supported_n(n) || batch <= 0) return 0;
    const size_t blocks = size_t(n) * n * batch / (kThreads * kLossPix);
    return 8 * size_t(n) * n * batch + 2 * sizeof(double) * blocks * 2 + 256;
}

extern "C" int loss_acn(const ac_params* params, int batch, const void* U0, const void* U1, double* loss_dev,
                        void* grad, void* work, acpr_stream stream) {
    ACPR_CHECK_ARG(params, "null params");
    const int n = params->n;
    if (!supported_n(n)) {
        set_error("loss_acn: n=%d unsupported (power of two in [32, 1024])", n);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(batch > 0 && U0 && U1 && loss_dev && work, "bad loss_acn arguments");
    ACPR_CHECK_ARG(params->precision == AC_F64 || params->precision == AC_F32, "bad precision");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int lg = __builtin_ctz(n);
    const long long nn = (long long)n * n;
    const int parts = int(nn / (kThreads * kLossPix));
    const int blocks = parts * batch;
    const double h = params->length / n;
    const double half_dt = 0.5 * params->dt, e2_h2 = params->eps * params->eps / (h * h);
    const int mass = params->variant == AC_MASS_CONSERVING;
    const double scale = 2.0 / (double(batch) * double(nn));
    char* wp = static_cast<char*>(work);
    void* r = wp;
    double* fpart = reinterpret_cast<double*>(wp + 8 * nn * batch);
    double* rpart = fpart + 2 * blocks;
    if (params->precision == AC_F64) {
        const auto* a = static_cast<const double*>(U0);
        const auto* c = static_cast<const double*>(U1);
        if (mass) {
            loss_fsum_kernel<double><<<blocks, kThreads, 0, st>>>(a, c, fpart);
            ACPR_LAUNCH_CHECK();
        }
        loss_resid_kernel<double><<<blocks, kThreads, 0, st>>>(a, c, static_cast<double*>(r), fpart, rpart, parts, lg,
                                                               half_dt, e2_h2, mass);
        ACPR_LAUNCH_CHECK();
        loss_grad_kernel<double><<<grad ? blocks : 1, kThreads, 0, st>>>(c, static_cast<double*>(r), rpart, parts,
                                                                         blocks, static_cast<double*>(grad), loss_dev,
                                                                         lg, half_dt, e2_h2, mass, scale);
    } else {
        const auto* a = static_cast<const float*>(U0);
        const auto* c = static_cast<const float*>(U1);
        if (mass) {
            loss_fsum_kernel<float><<<blocks, kThreads, 0, st>>>(a, c, fpart);
            ACPR_LAUNCH_CHECK();
        }
        loss_resid_kernel<float><<<blocks, kThreads, 0, st>>>(a, c, static_cast<float*>(r), fpart, rpart, parts, lg,
                                                              half_dt, e2_h2, mass);
        ACPR_LAUNCH_CHECK();
        loss_grad_kernel<float><<<grad ? blocks : 1, kThreads, 0, st>>>(c, static_cast<float*>(r), rpart, parts,
                                                                        blocks, static_cast<float*>(grad), loss_dev,
                                                                        lg, half_dt, e2_h2, mass, scale);
    }
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

extern "C" int acnn_adam_step(int precision, void* w, const void* grad, void* m, void* v, long long count, double lr,
                              double beta1, double beta2, double eps, int t, acpr_stream stream) {
    ACPR_CHECK_ARG(w && grad && m && v && count >= 0 && t >= 1, "bad acnn_adam_step arguments");
    ACPR_CHECK_ARG(precision == AC_F64 || precision == AC_F32, "bad precision");
    if (count == 0) return AC_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double c1 = 1.0 - std::pow(beta1, t), c2 = 1.0 - std::pow(beta2, t);
    const unsigned grid = unsigned((count + 255) / 256);
    if (precision == AC_F64)
        adam_kernel<double><<<grid, 256, 0, st>>>(static_cast<double*>(w), static_cast<const double*>(grad),
                                                  static_cast<double*>(m), static_cast<double*>(v), count, lr, beta1,
                                                  beta2, eps, c1, c2);
    else
        adam_kernel<float><<<grid, 256, 0, st>>>(static_cast<float*>(w), static_cast<const float*>(grad),
                                                 static_cast<float*>(m), static_cast<float*>(v), count, float(lr),
                                                 float(beta1), float(beta2), float(eps), float(c1), float(c2));
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

// Workspace of acnn_train_alg1, 256-byte aligned pieces: U, U1, G ([q][n][n]
// each), the parameter gradients, the training and the loss workspaces.
struct Alg1Layout {
    size_t u, u1, g, gp, ws, lw, total;
};
static Alg1Layout alg1_layout(const acnn_desc* desc, int n, int q) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t es = elem_size(desc->precision);
    long long nb = 0;
    const long long nw = acnn_param_count(desc->channels, desc->blocks, &nb);
    const size_t field = up(es * size_t(n) * n * q);
    Alg1Layout L{};
    L.u = 0;
    L.u1 = L.u + field;
    L.g = L.u1 + field;
    L.gp = L.g + field;
    L.ws = L.gp + up(es * size_t(nw + nb));
    L.lw = L.ws + up(acnn_train_bytes_for(desc, n, q));
    L.total = L.lw + up(loss_acn_work_bytes(n, q));
    return L;
}

extern "C" size_t acnn_train_alg1_bytes(const acnn_desc* desc, int n, int q) {
    if (!desc || n <= 0 || q <= 0) return 0;
    return alg1_layout(desc, n, q).total;
}

extern "C" int acnn_train_alg1(const ac_params* params, const acnn_desc* desc, int R, const void* U0s,
                               const int* perm, int epochs, int q, int steps, int b_inner, double lr, double beta1,
                               double beta2, double eps, void* adam_m, void* adam_v, int* t, double* losses_dev,
                               void* workspace, size_t workspace_bytes, acpr_stream stream) {
    int rc = acnn_check(desc);
    if (rc) return rc;
    ACPR_CHECK_ARG(params && U0s && perm && adam_m && adam_v && t && losses_dev, "null acnn_train_alg1 argument");
    ACPR_CHECK_ARG(params->precision == desc->precision, "params and network precision differ");
    ACPR_CHECK_ARG(R > 0 && q > 0 && R % q == 0, "R must be a positive multiple of q");
    ACPR_CHECK_ARG(epochs >= 0 && steps >= 0 && b_inner >= 0, "negative loop count");
    const int n = params->n;
    if (!supported_n(n)) {
        set_error("acnn_train_alg1: n=%d unsupported (power of two in [32, 1024])", n);
        return AC_ERR_UNSUPPORTED;
    }
    for (int e = 0; e < epochs; ++e)
        for (int k = 0; k < R; ++k)
            ACPR_CHECK_ARG(perm[e * R + k] >= 0 && perm[e * R + k] < R, "perm[%d][%d] out of range", e, k);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = elem_size(desc->precision);
    const long long nn = (long long)n * n;
    long long nb = 0;
    const long long nw = acnn_param_count(desc->channels, desc->blocks, &nb);
    const Alg1Layout lay = alg1_layout(desc, n, q);
    ACPR_CHECK_ARG(workspace && workspace_bytes >= lay.total, "acnn_train_alg1: workspace needs %zu bytes",
                   lay.total);
    ACPR_CHECK_ARG(reinterpret_cast<uintptr_t>(workspace) % 256 == 0, "workspace must be 256-byte aligned");
    char* wsb = static_cast<char*>(workspace);
    void* U = wsb + lay.u;
    void* U1 = wsb + lay.u1;
    void* G = wsb + lay.g;
    void* gp = wsb + lay.gp;
    void* ws = wsb + lay.ws;
    void* lw = wsb + lay.lw;
    char* gw = static_cast<char*>(gp);
    char* gb = gw + es * nw;
    char* mw = static_cast<char*>(adam_m);
    char* vw = static_cast<char*>(adam_v);
    long long li = 0;
    for (int e = 0; e < epochs && !rc; ++e)
        for (int sub = 0; sub < R / q && !rc; ++sub) {
            for (int j = 0; j < q; ++j) {
                const int src = perm[e * R + sub * q + j];
                if (cudaMemcpyAsync(static_cast<char*>(U) + es * nn * j, static_cast<const char*>(U0s) + es * nn * src,
                                    es * nn, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                    set_error("acnn_train_alg1: copy of initial conditions failed");
                    rc = AC_ERR_CUDA;
                }
            }
            for (int s = 0; s < steps && !rc; ++s) {
                for (int k = 0; k < b_inner && !rc; ++k) {
                    if ((rc = acnn_forward_train_impl(desc, n, q, U, U1, ws, st))) break;
                    if ((rc = loss_acn(params, q, U, U1, losses_dev + li, G, lw, stream))) break;
                    ++li;
                    if ((rc = acnn_backward_impl(desc, n, q, U, G, gw, gb, ws, st))) break;
                    *t += 1;
                    if ((rc = acnn_adam_step(desc->precision, desc->w, gw, mw, vw, nw, lr, beta1, beta2, eps, *t,
                                             stream)))
                        break;
                    rc = acnn_adam_step(desc->precision, desc->b, gb, mw + es * nw, vw + es * nw, nb, lr, beta1, beta2,
                                        eps, *t, stream);
                }
                if (b_inner > 0) std::swap(U, U1);  // U <- the prediction of the last inner update
            }
        }
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc) return rc;
    ACPR_CUDA(e);
    return AC_OK;
}
