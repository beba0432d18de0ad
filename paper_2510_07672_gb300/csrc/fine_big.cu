// fine_big.cu -- the fine propagator for fields too large for one cluster's
// shared memory (1024 x 1024 float32: 4 MB), in two passes per step through
// L2/HBM.  Same step and same arithmetic layout as fine.cu (Sec. 3.1): rows
// 2p and 2p+1 of a field share a complex line, the row spectra Z_p[k] are
// split into the two rows' half spectra by the column owner (DC and Nyquist
// columns packed in column 0), and rebuilt before the inverse row FFT.
//   rows kernel:    [inverse row FFT of the previous step] -> pointwise
//                   right-hand side -> forward row FFT -> Z[p][k]
//   columns kernel: split -> column FFT -> symbol -> inverse column FFT ->
//                   V[r][c] (c < N/2)
// One warp owns one line (B = 32 threads, A = N/32 values each), so the
// exchange inside a 1D transform needs only __syncwarp().  Z and V live in a
// library-owned device workspace (allocated on first use, kept until exit).
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fft_reg.cuh"

namespace acpr {

constexpr int kBigWarps = 8;  // lines per CTA

// Two-pass transform of one line by one warp; buf holds A*(B+1) values (the
// +1 pitch keeps the pass-2 reads free of bank conflicts).
template <typename T, int N, int A, int B, int SIGN>
__device__ __forceinline__ void warp_line_fft(vec2_t<T> (&x)[A], const vec2_t<T>* __restrict__ tw,
                                              vec2_t<T>* buf, int j) {
    static_assert(B == 32 && A * B == N && A % B == 0, "one warp per line");
    T re[A], im[A];
#pragma unroll
    for (int t = 0; t < A; ++t) { re[t] = x[t].x; im[t] = x[t].y; }
    reg_dft<T, A, SIGN>(re, im);
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) {
        const vec2_t<T> w = tw[(j * k1) & (N - 1)];
        const T c = w.x;
        const T s = SIGN < 0 ? w.y : -w.y;
        const T r = re[k1] * c - im[k1] * s;
        im[k1] = re[k1] * s + im[k1] * c;
        re[k1] = r;
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
        vec2_t<T> v;
        v.x = re[k1];
        v.y = im[k1];
        buf[k1 * (B + 1) + j] = v;
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < A / B; ++m) {
        const int k1 = j + B * m;
        T br[B], bi[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) {
            const vec2_t<T> v = buf[k1 * (B + 1) + n2];
            br[n2] = v.x;
            bi[n2] = v.y;
        }
        reg_dft<T, B, SIGN>(br, bi);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            x[m + (A / B) * k2].x = br[k2];
            x[m + (A / B) * k2].y = bi[k2];
        }
    }
}

struct BigArgs {
    const void* in;   // physical fields read by the first pass
    void* out;        // physical fields written by the last pass
    // field f = g * per_group + i reads field map[g] * in_gs + in_off + i of
    // `in` and writes field map[g] * out_gs + out_off + i of `out`
    int per_group;
    long long in_gs, in_off, out_gs, out_off;
    const int* map;
    void* Z;          // [fields][N/2][N] complex
    void* V;          // [fields][N][N/2] complex
    const double* mean;  // [fields] entry means (mass-conserving)
    const void* tw;   // [N] exp(-2 pi i k / N), float64-rounded once per call
    const void* lam;  // [N] dt eps^2 (4/h^2) sin^2(pi k / N)
    int mass;
    double a, dt, lam_scale;
};

enum { kRowsFirst = 0, kRowsMid = 1, kRowsLast = 2 };

__device__ __forceinline__ long long big_field(const BigArgs& a, int f, bool out) {
    const int g = f / a.per_group, i = f % a.per_group;
    const long long pg = a.map ? a.map[g] : g;
    return out ? pg * a.out_gs + a.out_off + i : pg * a.in_gs + a.in_off + i;
}

template <typename T, int N, int A>
__global__ void __launch_bounds__(kBigWarps * 32)
big_rows_kernel(BigArgs args, int mode) {
    using V2 = vec2_t<T>;
    constexpr int B = 32, HALF = N / 2, PB = A * (B + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* tw = reinterpret_cast<V2*>(smem_raw);
    V2* bufs = tw + N;
    const int lanes = threadIdx.x & 31, w = threadIdx.x >> 5, j = lanes;
    const int blocks_per_field = HALF / kBigWarps;
    const int f = blockIdx.x / blocks_per_field;
    const int p = (blockIdx.x % blocks_per_field) * kBigWarps + w;  // row pair: rows 2p, 2p+1
    for (int k = threadIdx.x; k < N; k += blockDim.x) tw[k] = static_cast<const V2*>(args.tw)[k];
    __syncthreads();
    V2* buf = bufs + w * PB;
    const size_t NN = size_t(N) * N;
    V2 x[A];
    if (mode == kRowsFirst) {
        const T* u = static_cast<const T*>(args.in) + size_t(big_field(args, f, false)) * NN + size_t(2 * p) * N;
#pragma unroll
        for (int t = 0; t < A; ++t) {
            x[t].x = u[j + B * t];
            x[t].y = u[N + j + B * t];
        }
    } else {
        // rebuild Z'[k] = V_{2p}[k] + i V_{2p+1}[k] with V[N - k] = conj(V[k])
        const V2* v0 = static_cast<const V2*>(args.V) + size_t(f) * NN / 2 + size_t(2 * p) * HALF;
        const V2* v1 = v0 + HALF;
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int k = j + B * t;
            V2 z;
            if (k == 0 || k == HALF) {
                const V2 va = v0[0], vb = v1[0];
                if (k == 0) { z.x = va.x; z.y = vb.x; }
                else        { z.x = va.y; z.y = vb.y; }
            } else if (k < HALF) {
                const V2 va = v0[k], vb = v1[k];
                z.x = va.x - vb.y;
                z.y = va.y + vb.x;
            } else {
                const V2 va = v0[N - k], vb = v1[N - k];
                z.x = va.x + vb.y;
                z.y = vb.x - va.y;
            }
            x[t] = z;
        }
        warp_line_fft<T, N, A, B, +1>(x, tw, buf, j);
        if (mode == kRowsLast) {
            T* u = static_cast<T*>(args.out) + size_t(big_field(args, f, true)) * NN + size_t(2 * p) * N;
#pragma unroll
            for (int t = 0; t < A; ++t) {
                u[j + B * t] = x[t].x;
                u[N + j + B * t] = x[t].y;
            }
            return;
        }
    }
    const T a = T(args.a), dt = T(args.dt);
#pragma unroll
    for (int t = 0; t < A; ++t) {
        const T ur = x[t].x, ui = x[t].y;
        x[t].x = a * ur + dt * (ur - ur * ur * ur);
        x[t].y = a * ui + dt * (ui - ui * ui * ui);
    }
    warp_line_fft<T, N, A, B, -1>(x, tw, buf, j);
    V2* z = static_cast<V2*>(args.Z) + size_t(f) * NN / 2 + size_t(p) * N;
#pragma unroll
    for (int t = 0; t < A; ++t) z[j + B * t] = x[t];
}

template <typename T, int N, int A>
__global__ void __launch_bounds__(kBigWarps * 32)
big_cols_kernel(BigArgs args) {
    using V2 = vec2_t<T>;
    constexpr int B = 32, HALF = N / 2, PB = A * (B + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* tw = reinterpret_cast<V2*>(smem_raw);
    T* lam = reinterpret_cast<T*>(tw + N);
    V2* bufs = reinterpret_cast<V2*>(lam + N);  // max(transform buffers, staging)
    const int j = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int blocks_per_field = HALF / kBigWarps;
    const int f = blockIdx.x / blocks_per_field;
    const int c0 = (blockIdx.x % blocks_per_field) * kBigWarps;
    const int col = c0 + w;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        tw[k] = static_cast<const V2*>(args.tw)[k];
        lam[k] = static_cast<const T*>(args.lam)[k];
    }
    __syncthreads();
    V2* buf = bufs + w * PB;
    const size_t NN = size_t(N) * N;
    const V2* Z = static_cast<const V2*>(args.Z) + size_t(f) * NN / 2;
    const T half = T(0.5);
    V2 x[A];
    // stage, for every row pair, the block's kBigWarps columns and their
    // partner columns (N - c; N/2 for c = 0) with row-contiguous loads:
    // in[pp][s], s < kBigWarps: Z[pp][c0 + s]; s >= kBigWarps: the partner of
    // c0 + s - kBigWarps (pitch 2 kBigWarps + 1: the split's reads of 16 row
    // pairs at one column fall in distinct banks)
    constexpr int SP = 2 * kBigWarps + 1;
    V2* in = bufs;  // [HALF][SP], before the transform buffers are used
    for (int idx = threadIdx.x; idx < HALF * 2 * kBigWarps; idx += blockDim.x) {
        const int pp = idx / (2 * kBigWarps), sl = idx % (2 * kBigWarps);
        const int cc = c0 + (sl % kBigWarps);
        const int cz = sl < kBigWarps ? cc : (cc == 0 ? HALF : N - cc);
        in[pp * SP + sl] = Z[size_t(pp) * N + cz];
    }
    __syncthreads();
    // split each row pair into its two rows' half spectra (column col)
#pragma unroll
    for (int t = 0; t < A; ++t) {
        const int r = j + B * t;
        const int pp = r >> 1;
        const V2 za = in[pp * SP + w], zb = in[pp * SP + kBigWarps + w];
        V2 v;
        if (col == 0) {
            if ((r & 1) == 0) { v.x = za.x; v.y = zb.x; }
            else              { v.x = za.y; v.y = zb.y; }
        } else if ((r & 1) == 0) {
            v.x = half * (za.x + zb.x);
            v.y = half * (za.y - zb.y);
        } else {
            v.x = half * (za.y + zb.y);
            v.y = half * (zb.x - za.x);
        }
        x[t] = v;
    }
    __syncthreads();  // the staged rows are read before the transform buffers overwrite them
    warp_line_fft<T, N, A, B, -1>(x, tw, buf, j);
    const T a = T(args.a);
    const T inv_nn = T(1.0 / double(NN));
    if (col != 0) {
        const T lam_l = lam[col];
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const T s = inv_nn / (a + (lam[j + B * t] + lam_l));
            x[t].x *= s;
            x[t].y *= s;
        }
    } else {
        // C'[k] = C[k] (s0 + sN) / 2 + conj(C[N - k]) (s0 - sN) / 2 (columns 0 and N/2)
        __syncwarp();
#pragma unroll
        for (int t = 0; t < A; ++t) buf[j + B * t] = x[t];
        __syncwarp();
        const T lam_n = lam[HALF];
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int k = j + B * t;
            const V2 zc = x[t];
            const V2 zp = buf[(N - k) & (N - 1)];
            const T lk = lam[k];
            const T s0 = inv_nn / (a + lk);
            const T sn = inv_nn / (a + (lk + lam_n));
            const T sp = half * (s0 + sn), sm = half * (s0 - sn);
            x[t].x = zc.x * sp + zp.x * sm;
            x[t].y = zc.y * sp - zp.y * sm;
            if (k == 0 && args.mass) {
                x[t].x = T(args.mean[f]);
                x[t].y = zc.y * sn;
            }
        }
    }
    warp_line_fft<T, N, A, B, +1>(x, tw, buf, j);
    // V[r][col] for every row, staged so that each row's kBigWarps columns are
    // written as one contiguous run
    __syncthreads();  // every warp is done with its transform buffer
    V2* stage = bufs;  // [N][kBigWarps + 1]
#pragma unroll
    for (int t = 0; t < A; ++t) stage[(j + B * t) * (kBigWarps + 1) + w] = x[t];
    __syncthreads();
    V2* Vf = static_cast<V2*>(args.V) + size_t(f) * NN / 2;
    for (int idx = threadIdx.x; idx < N * kBigWarps; idx += blockDim.x) {
        const int r = idx / kBigWarps, cc = idx % kBigWarps;
        Vf[size_t(r) * HALF + c0 + cc] = stage[r * (kBigWarps + 1) + cc];
    }
}

// The twiddle and symbol tables of one call, in float64 then rounded (float64
// arithmetic is scarce on this GPU: once per call, not once per block).
template <typename T, int N>
__global__ void big_tables_kernel(vec2_t<T>* __restrict__ tw, T* __restrict__ lam, double lam_scale) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * double(k) / N, &sn, &cs);
        tw[k].x = T(cs);
        tw[k].y = T(sn);
        const double s = sinpi(double(k) / N);
        lam[k] = T(lam_scale * s * s);
    }
}

// float64 mean of each field (fixed order): one block per field.
template <typename T>
__global__ void big_mean_kernel(BigArgs args, long long nn, double* __restrict__ mean) {
    const T* u = static_cast<const T*>(args.in) + size_t(big_field(args, blockIdx.x, false)) * nn;
    double s = 0.0;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) s += double(u[i]);
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        mean[blockIdx.x] = t / double(nn);
    }
}

namespace {
struct BigWorkspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_big_mutex;
std::vector<BigWorkspace> g_big_ws;  // per device
}  // namespace

static int big_workspace(size_t bytes, void** out) {
    int dev = 0;
    ACPR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_big_mutex);
    if (int(g_big_ws.size()) <= dev) g_big_ws.resize(dev + 1);
    BigWorkspace& ws = g_big_ws[dev];
    if (ws.bytes < bytes) {
        if (ws.ptr) {
            ACPR_CUDA(cudaDeviceSynchronize());
            cudaFree(ws.ptr);
            ws.ptr = nullptr;
            ws.bytes = 0;
        }
        if (cudaMalloc(&ws.ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("fine (large fields): workspace allocation of %zu bytes failed", bytes);
            return AC_ERR_NOMEM;
        }
        ws.bytes = bytes;
    }
    *out = ws.ptr;
    return AC_OK;
}

bool fine_big_supported(int n, int precision) { return n == 1024 && precision == AC_F32; }

size_t fine_big_workspace_bytes(int n, int fields) {
    // Z and V spectra, the means, then the tables (16-byte aligned)
    return size_t(n) * n * sizeof(float2) * fields + fields * sizeof(double) + 256 + size_t(n) * 12;
}

// The two-pass fine propagation of `fields` fields (mapping as in BigArgs).
// ws: device workspace of fine_big_workspace_bytes (NULL: the library's own,
// allocated on first use; calls on different streams must then not overlap).
int fine_big_run(const ac_params* p, int groups, int per_group, int steps, const void* in, long long in_gs,
                 long long in_off, void* out, long long out_gs, long long out_off, const int* map, void* ws,
                 cudaStream_t st) {
    constexpr int N = 1024, A = 32;
    using T = float;
    if (!fine_big_supported(p->n, p->precision)) {
        set_error("fine (large fields): n=%d precision %d not built", p->n, p->precision);
        return AC_ERR_UNSUPPORTED;
    }
    const int fields = groups * per_group;
    if (fields == 0) return AC_OK;
    const size_t NN = size_t(N) * N;
    const size_t zbytes = NN / 2 * sizeof(vec2_t<T>) * fields;
    if (!ws) {
        int rc = big_workspace(fine_big_workspace_bytes(N, fields), &ws);
        if (rc) return rc;
    }
    unsigned char* base = static_cast<unsigned char*>(ws);
    BigArgs a{};
    a.in = in;
    a.out = out;
    a.per_group = per_group;
    a.in_gs = in_gs;
    a.in_off = in_off;
    a.out_gs = out_gs;
    a.out_off = out_off;
    a.map = map;
    a.Z = base;
    a.V = base + zbytes;
    double* mean = reinterpret_cast<double*>(base + 2 * zbytes);
    a.mean = mean;
    const size_t toff = (2 * zbytes + size_t(fields) * sizeof(double) + 255) / 256 * 256;
    vec2_t<T>* tw_tab = reinterpret_cast<vec2_t<T>*>(base + toff);
    T* lam_tab = reinterpret_cast<T*>(tw_tab + N);
    a.tw = tw_tab;
    a.lam = lam_tab;
    a.mass = p->variant == AC_MASS_CONSERVING;
    a.a = 1.0 + p->S * p->dt;
    a.dt = p->dt;
    const double h = p->length / p->n;
    a.lam_scale = p->dt * p->eps * p->eps * 4.0 / (h * h);
    big_tables_kernel<T, N><<<(N + 255) / 256, 256, 0, st>>>(tw_tab, lam_tab, a.lam_scale);
    ACPR_LAUNCH_CHECK();
    if (a.mass) {
        big_mean_kernel<T><<<fields, 1024, 0, st>>>(a, (long long)NN, mean);
        ACPR_LAUNCH_CHECK();
    }
    // the columns kernel's shared area serves, one after the other, the
    // staged input columns, the warps' transform buffers and the output staging
    constexpr size_t kIn = size_t(N / 2) * (2 * kBigWarps + 1);
    constexpr size_t kXf = size_t(kBigWarps) * A * 33;
    constexpr size_t kOut = size_t(N) * (kBigWarps + 1);
    constexpr size_t kBufs = kIn > kXf ? (kIn > kOut ? kIn : kOut) : (kXf > kOut ? kXf : kOut);
    const size_t smem_rows = sizeof(vec2_t<T>) * (N + size_t(kBigWarps) * A * 33);
    const size_t smem_cols = sizeof(vec2_t<T>) * (N + kBufs) + sizeof(T) * N;
    static bool configured = false;
    if (!configured) {
        ACPR_CUDA(cudaFuncSetAttribute(big_rows_kernel<T, N, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem_rows)));
        ACPR_CUDA(cudaFuncSetAttribute(big_cols_kernel<T, N, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem_cols)));
        configured = true;
    }
    const unsigned blocks = unsigned(fields * (N / 2 / kBigWarps));
    if (steps == 0) {
        // one forward and one inverse row pass would round; copy instead
        for (int f = 0; f < fields; ++f) {
            const int g = f / per_group, i = f % per_group;
            int pg = g;
            if (map) ACPR_CUDA(cudaMemcpy(&pg, map + g, sizeof(int), cudaMemcpyDeviceToHost));
            ACPR_CUDA(cudaMemcpyAsync(static_cast<T*>(out) + (pg * out_gs + out_off + i) * NN,
                                      static_cast<const T*>(in) + (pg * in_gs + in_off + i) * NN, NN * sizeof(T),
                                      cudaMemcpyDeviceToDevice, st));
        }
        return AC_OK;
    }
    for (int s = 0; s < steps; ++s) {
        big_rows_kernel<T, N, A><<<blocks, kBigWarps * 32, smem_rows, st>>>(a, s == 0 ? kRowsFirst : kRowsMid);
        ACPR_LAUNCH_CHECK();
        big_cols_kernel<T, N, A><<<blocks, kBigWarps * 32, smem_cols, st>>>(a);
        ACPR_LAUNCH_CHECK();
    }
    big_rows_kernel<T, N, A><<<blocks, kBigWarps * 32, smem_rows, st>>>(a, kRowsLast);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

}  // namespace acpr
