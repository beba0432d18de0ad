// fine3d.cu -- the stabilised semi-implicit fine step on the periodic cube
// (d = 3; the 3D experiments of Sec. 4): the 7-point Laplacian, solved by a
// 3D FFT.
//
// A 128^3 float32 field is 8 MB, beyond one thread-block cluster, so a step is
// five passes over L2/HBM, each a batch of 1D transforms of length N done in
// shared memory by one CTA for 16 lines at a time:
//   X  pointwise right-hand side, forward FFT along k (contiguous rows)
//   Y  forward FFT along j
//   Z  forward FFT along i, divide by the symbol, inverse FFT along i
//   Y' inverse FFT along j
//   X' inverse FFT along k, scale, write the new fields
// Two real fields travel as the real and imaginary parts of one complex
// field: the operator is real with an even symbol, so it acts on both parts
// separately and a complex transform serves two fields.  The mass-conserving
// variant holds the zero mode at N^3 times the field's mean, taken once per
// call (the scheme conserves it exactly; the same reading as the 2D kernel).
#include "common.cuh"

#include <cmath>

namespace acpr {

namespace {

constexpr int kLines = 16;    // lines per CTA
constexpr int kThreads = 256;
constexpr int kMeanChunks = 64;

enum { kPassX = 0, kPassY = 1, kPassZ = 2, kPassYi = 3, kPassXi = 4 };

template <typename T>
__device__ __forceinline__ vec2_t<T> cmul(vec2_t<T> a, vec2_t<T> b) {
    vec2_t<T> r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <int N>
__device__ __forceinline__ int bitrev(int x) {
    constexpr int LG = N == 32 ? 5 : (N == 64 ? 6 : 7);
    return int(__brev(unsigned(x)) >> (32 - LG));
}

// Radix-2 decimation in time over the kLines lines of s (bit-reversed input,
// natural output); tw[k] = exp(-2 pi i k / N), conjugated for the inverse.
template <typename T, int N, bool INV>
__device__ __forceinline__ void fft_dit(vec2_t<T>* s, const vec2_t<T>* tw) {
    for (int half = 1; half < N; half <<= 1) {
        for (int bt = threadIdx.x; bt < kLines * N / 2; bt += kThreads) {
            const int l = bt / (N / 2), t = bt % (N / 2);
            const int pos = t & (half - 1);
            const int i0 = (t - pos) * 2 + pos, i1 = i0 + half;
            vec2_t<T> w = tw[pos * (N / (2 * half))];
            if (INV) w.y = -w.y;
            vec2_t<T>* x = s + l * N;
            const vec2_t<T> a = x[i0];
            const vec2_t<T> b = cmul<T>(x[i1], w);
            x[i0].x = a.x + b.x;
            x[i0].y = a.y + b.y;
            x[i1].x = a.x - b.x;
            x[i1].y = a.y - b.y;
        }
        __syncthreads();
    }
}

// Radix-2 decimation in frequency (natural input, bit-reversed output).
template <typename T, int N, bool INV>
__device__ __forceinline__ void fft_dif(vec2_t<T>* s, const vec2_t<T>* tw) {
    for (int half = N / 2; half >= 1; half >>= 1) {
        for (int bt = threadIdx.x; bt < kLines * N / 2; bt += kThreads) {
            const int l = bt / (N / 2), t = bt % (N / 2);
            const int pos = t & (half - 1);
            const int i0 = (t - pos) * 2 + pos, i1 = i0 + half;
            vec2_t<T> w = tw[pos * (N / (2 * half))];
            if (INV) w.y = -w.y;
            vec2_t<T>* x = s + l * N;
            const vec2_t<T> a = x[i0];
            const vec2_t<T> b = x[i1];
            x[i0].x = a.x + b.x;
            x[i0].y = a.y + b.y;
            vec2_t<T> d;
            d.x = a.x - b.x;
            d.y = a.y - b.y;
            x[i1] = cmul<T>(d, w);
        }
        __syncthreads();
    }
}

struct Step3 {
    double c0;       // 1 + S dt
    double dt;
    int mass;
    int fields;      // real fields (the last pair may have no imaginary field)
};

// One pass of the step over all pairs.  u: real fields [F][N][N][N]; W:
// complex [P][N][N][N]; tables: tw[N/2] then s2[N] (dt eps^2 4/h^2 sin^2(pi m/N));
// means: [F] per-field means (mass variant).
template <typename T, int N, int PASS>
__global__ void __launch_bounds__(kThreads) fine3d_pass(const T* __restrict__ u, T* __restrict__ uo,
                                                        vec2_t<T>* __restrict__ W,
                                                        const vec2_t<T>* __restrict__ tw_g,
                                                        const T* __restrict__ s2_g, const double* __restrict__ part,
                                                        Step3 prm) {
    using C2 = vec2_t<T>;
    constexpr long long NN = (long long)N * N, NNN = NN * N;
    __shared__ C2 s[kLines * N];
    __shared__ C2 tw[N / 2];
    __shared__ T s2[N];
    for (int k = threadIdx.x; k < N / 2; k += kThreads) tw[k] = tw_g[k];
    if (PASS == kPassZ)
        for (int k = threadIdx.x; k < N; k += kThreads) s2[k] = s2_g[k];
    const int b = blockIdx.x;
    if constexpr (PASS == kPassX || PASS == kPassXi) {
        // lines along k: rows r0 .. r0 + 15 of the [P][N][N] row space
        const long long r0 = (long long)b * kLines;
        const int p = int(r0 / NN);
        const long long ij0 = r0 % NN;
        const int fa = 2 * p, fb = 2 * p + 1;
        const bool has_b = fb < prm.fields;
        if constexpr (PASS == kPassX) {
            const T c0 = T(prm.c0), dt = T(prm.dt);
            for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
                const int l = e / N, k = e % N;
                const long long off = (ij0 + l) * N + k;
                const T ua = u[fa * NNN + off];
                const T ub = has_b ? u[fb * NNN + off] : T(0);
                C2 v;
                v.x = c0 * ua + dt * (ua - ua * ua * ua);
                v.y = has_b ? c0 * ub + dt * (ub - ub * ub * ub) : T(0);
                s[l * N + bitrev<N>(k)] = v;
            }
            __syncthreads();
            fft_dit<T, N, false>(s, tw);
            for (int e = threadIdx.x; e < kLines * N; e += kThreads) W[(long long)p * NNN + (ij0 + e / N) * N + e % N] = s[e];
        } else {
            for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
                const int l = e / N, k = e % N;
                s[l * N + bitrev<N>(k)] = W[(long long)p * NNN + (ij0 + l) * N + k];
            }
            __syncthreads();
            fft_dit<T, N, true>(s, tw);
            const T scale = T(1.0 / double(NNN));
            for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
                const long long off = (ij0 + e / N) * N + e % N;
                uo[fa * NNN + off] = s[e].x * scale;
                if (has_b) uo[fb * NNN + off] = s[e].y * scale;
            }
        }
    } else {
        // lines along j (PASS Y, Y') at fixed (p, i) or along i (PASS Z) at fixed
        // (p, j); 16 consecutive k per CTA
        constexpr int KC = N / kLines;
        const int kc = b % KC, q = (b / KC) % N, p = b / (KC * N);
        const int k0 = kc * kLines;
        auto addr = [&](int idx, int l) -> long long {
            // idx runs along the transformed axis
            if constexpr (PASS == kPassZ) return (long long)p * NNN + (long long)idx * NN + (long long)q * N + k0 + l;
            else return (long long)p * NNN + (long long)q * NN + (long long)idx * N + k0 + l;
        };
        __syncthreads();
        for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
            const int idx = e / kLines, l = e % kLines;
            s[l * N + bitrev<N>(idx)] = W[addr(idx, l)];
        }
        __syncthreads();
        if constexpr (PASS == kPassZ) {
            fft_dit<T, N, false>(s, tw);
            // s[l][a]: mode (a, q, k0 + l); divide by the symbol
            const bool dc_block = prm.mass && q == 0 && k0 == 0;
            if (dc_block && threadIdx.x == 0) {
                double ta = 0.0, tb = 0.0;
                for (int c = 0; c < kMeanChunks; ++c) {
                    ta += part[(2 * p) * kMeanChunks + c];
                    if (2 * p + 1 < prm.fields) tb += part[(2 * p + 1) * kMeanChunks + c];
                }
                s[0].x = T(ta);  // sums over the field: N^3 times the mean
                s[0].y = T(tb);
            }
            for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
                const int l = e / N, a = e % N;
                if (dc_block && e == 0) continue;
                const T D = T(prm.c0) + s2[a] + s2[q] + s2[k0 + l];
                const T inv = T(1) / D;
                s[e].x *= inv;
                s[e].y *= inv;
            }
            __syncthreads();
            fft_dif<T, N, true>(s, tw);
            for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
                const int idx = e / kLines, l = e % kLines;
                W[addr(idx, l)] = s[l * N + bitrev<N>(idx)];
            }
        } else {
            fft_dit<T, N, PASS == kPassYi>(s, tw);
            for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
                const int idx = e / kLines, l = e % kLines;
                W[addr(idx, l)] = s[l * N + idx];
            }
        }
    }
}

// Twiddles exp(-2 pi i k / N) and the symbol table, once per call.
template <typename T, int N>
__global__ void fine3d_tables(vec2_t<T>* tw, T* s2, double coef) {
    const int k = threadIdx.x;
    if (k < N / 2) {
        double sn, cs;
        sincospi(2.0 * k / N, &sn, &cs);
        tw[k].x = T(cs);
        tw[k].y = T(-sn);
    }
    if (k < N) {
        const double sv = sinpi(double(k) / N);
        s2[k] = T(coef * sv * sv);
    }
}

// Per-field partial sums (float64 across threads) of the field, for the mean.
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) fine3d_sums(const T* __restrict__ u, double* __restrict__ part) {
    constexpr long long NNN = (long long)N * N * N;
    constexpr long long chunk = NNN / kMeanChunks;
    const int f = blockIdx.y, c = blockIdx.x;
    const T* base = u + f * NNN + c * chunk;
    T acc = T(0);
    for (long long i = threadIdx.x; i < chunk; i += kThreads) acc += base[i];
    double d = double(acc);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    __shared__ double red[kThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        part[f * kMeanChunks + c] = t;
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t work_layout(int n, int fields, int precision, size_t* w_off, size_t* tw_off, size_t* s2_off,
                   size_t* part_off) {
    const size_t es = elem_size(precision);
    const size_t nnn = size_t(n) * n * n;
    const size_t pairs = size_t(fields + 1) / 2;
    size_t off = 0;
    *w_off = off;
    off += align256(2 * es * nnn * pairs);
    *tw_off = off;
    off += align256(2 * es * size_t(n / 2));
    *s2_off = off;
    off += align256(es * size_t(n));
    *part_off = off;
    off += align256(sizeof(double) * kMeanChunks * size_t(fields));
    return off;
}

template <typename T, int N>
int propagate3d(const ac_params* p, int steps, int fields, const T* u_in, T* u_out, char* work, cudaStream_t st) {
    using C2 = vec2_t<T>;
    size_t w_off, tw_off, s2_off, part_off;
    work_layout(N, fields, p->precision, &w_off, &tw_off, &s2_off, &part_off);
    C2* W = reinterpret_cast<C2*>(work + w_off);
    C2* tw = reinterpret_cast<C2*>(work + tw_off);
    T* s2 = reinterpret_cast<T*>(work + s2_off);
    double* part = reinterpret_cast<double*>(work + part_off);
    const double h = p->length / N;
    fine3d_tables<T, N><<<1, N, 0, st>>>(tw, s2, 4.0 * p->dt * p->eps * p->eps / (h * h));
    ACPR_LAUNCH_CHECK();
    if (p->variant == AC_MASS_CONSERVING) {
        fine3d_sums<T, N><<<dim3(kMeanChunks, fields), kThreads, 0, st>>>(u_in, part);
        ACPR_LAUNCH_CHECK();
    }
    Step3 prm{1.0 + p->S * p->dt, p->dt, p->variant == AC_MASS_CONSERVING, fields};
    const int pairs = (fields + 1) / 2;
    const unsigned gx = unsigned((long long)pairs * N * N / kLines);
    const unsigned gyz = unsigned((long long)pairs * N * (N / kLines));
    const T* src = u_in;
    for (int s = 0; s < steps; ++s) {
        fine3d_pass<T, N, kPassX><<<gx, kThreads, 0, st>>>(src, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassY><<<gyz, kThreads, 0, st>>>(nullptr, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassZ><<<gyz, kThreads, 0, st>>>(nullptr, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassYi><<<gyz, kThreads, 0, st>>>(nullptr, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassXi><<<gx, kThreads, 0, st>>>(nullptr, u_out, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        src = u_out;
    }
    if (steps == 0 && u_out != u_in) {
        ACPR_CUDA(cudaMemcpyAsync(u_out, u_in, sizeof(T) * size_t(N) * N * N * fields, cudaMemcpyDeviceToDevice, st));
    }
    return AC_OK;
}

bool supported3d(int n, int precision) {
    return (n == 32 || n == 64 || n == 128) && (precision == AC_F32 || precision == AC_F64);
}

}  // namespace

}  // namespace acpr

using namespace acpr;

extern "C" int ac_fine3d_supported(int n, int precision) { return supported3d(n, precision) ? 1 : 0; }

extern "C" size_t ac_fine3d_work_bytes(int n, int num_fields, int precision) {
    if (!supported3d(n, precision) || num_fields <= 0) return 0;
    size_t a, b, c, d;
    return work_layout(n, num_fields, precision, &a, &b, &c, &d);
}

extern "C" int ac_fine3d_propagate(const ac_params* params, int steps, int num_fields, const void* u_in, void* u_out,
                                   void* work, size_t work_bytes, acpr_stream stream) {
    ACPR_CHECK_ARG(params, "null params");
    const int n = params->n;
    if (!supported3d(n, params->precision)) {
        set_error("ac_fine3d_propagate: n=%d precision=%d not built (n = 32, 64, 128)", n, params->precision);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(steps >= 0 && num_fields >= 0, "negative steps or field count");
    if (num_fields == 0) return AC_OK;
    ACPR_CHECK_ARG(u_in && u_out && work, "null pointer");
    const size_t need = ac_fine3d_work_bytes(n, num_fields, params->precision);
    ACPR_CHECK_ARG(work_bytes >= need, "ac_fine3d_propagate: work buffer too small (need %zu bytes)", need);
    ACPR_CHECK_ARG(params->variant == AC_CLASSIC || params->variant == AC_MASS_CONSERVING, "bad variant");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(work);
    if (params->precision == AC_F64) {
        const auto* a = static_cast<const double*>(u_in);
        auto* o = static_cast<double*>(u_out);
        if (n == 32) return propagate3d<double, 32>(params, steps, num_fields, a, o, w, st);
        if (n == 64) return propagate3d<double, 64>(params, steps, num_fields, a, o, w, st);
        return propagate3d<double, 128>(params, steps, num_fields, a, o, w, st);
    }
    const auto* a = static_cast<const float*>(u_in);
    auto* o = static_cast<float*>(u_out);
    if (n == 32) return propagate3d<float, 32>(params, steps, num_fields, a, o, w, st);
    if (n == 64) return propagate3d<float, 64>(params, steps, num_fields, a, o, w, st);
    return propagate3d<float, 128>(params, steps, num_fields, a, o, w, st);
}
