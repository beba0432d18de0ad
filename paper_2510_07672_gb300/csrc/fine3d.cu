// fine3d.cu -- the stabilised semi-implicit fine step on the periodic cube
// (d = 3; the 3D experiments of Sec. 4): the 7-point Laplacian, solved by a
// 3D FFT.
//
// A 128^3 float32 field is 8 MB, beyond one thread-block cluster, so a step is
// five passes over L2/HBM, each a batch of 1D transforms of length N, 16 lines
// per CTA:
//   X  pointwise right-hand side, forward FFT along k (contiguous rows)
//   Y  forward FFT along j
//   Z  forward FFT along i, divide by the symbol, inverse FFT along i
//   Y' inverse FFT along j
//   X' inverse FFT along k, scale, write the new fields
// Each line is transformed in registers by a group of lanes of one warp
// (line_fft: one shared-memory exchange, warp barriers only).
// Two real fields travel as the real and imaginary parts of one complex
// field: the operator is real with an even symbol, so it acts on both parts
// separately and a complex transform serves two fields.  The mass-conserving
// variant holds the zero mode at N^3 times the field's mean, taken once per
// call (the scheme conserves it exactly; the same reading as the 2D kernel).
#include "common.cuh"
#include "fft_reg.cuh"

#include <cmath>

namespace acpr {

namespace {

constexpr int kLines = 16;    // lines per CTA
constexpr int kMeanChunks = 64;
constexpr int kSumThreads = 256;

enum { kPassX = 0, kPassY = 1, kPassZ = 2, kPassYi = 3, kPassXi = 4 };

// A line of N points is transformed by B lanes of one warp holding A = N / B
// points each (line_fft: one shared-memory exchange, warp barriers only).
template <int N> struct Split;
template <> struct Split<32> { static constexpr int A = 8, B = 4; };
template <> struct Split<64> { static constexpr int A = 8, B = 8; };
template <> struct Split<128> { static constexpr int A = 16, B = 8; };

struct Step3 {
    double c0;       // 1 + S dt
    double dt;
    int mass;
    int fields;      // real fields (the last pair may have no imaginary field)
};

// One pass of the step over all pairs.  u: real fields [F][N][N][N]; W:
// complex [P][N][N][N]; tw_g: the line_fft table (N entries); s2_g[m] =
// dt eps^2 (4/h^2) sin^2(pi m/N); part: per-field partial sums (mass variant).
// CTA: 16 lines x B lanes; thread (l, j) holds points j + B t of line l.
template <typename T, int N, int PASS>
__global__ void __launch_bounds__(kLines * Split<N>::B) fine3d_pass(const T* __restrict__ u, T* __restrict__ uo,
                                                                    vec2_t<T>* __restrict__ W,
                                                                    const vec2_t<T>* __restrict__ tw_g,
                                                                    const T* __restrict__ s2_g,
                                                                    const double* __restrict__ part, Step3 prm) {
    using C2 = vec2_t<T>;
    constexpr int A = Split<N>::A, B = Split<N>::B;
    constexpr long long NN = (long long)N * N, NNN = NN * N;
    constexpr int XL = xlen<N, B>();
    __shared__ C2 ex[kLines * XL];
    __shared__ C2 tw[N];
    __shared__ T s2[N];
    for (int k = threadIdx.x; k < N; k += kLines * B) {
        tw[k] = tw_g[k];
        if (PASS == kPassZ) s2[k] = s2_g[k];
    }
    __syncthreads();
    const int l = threadIdx.x / B, j = threadIdx.x % B;
    C2* line = ex + l * XL;
    const unsigned wmask = 0xffffffffu;
    const int b = blockIdx.x;
    C2 x[A];
    if constexpr (PASS == kPassX || PASS == kPassXi) {
        // lines along k: row r0 + l of the [P][N][N] row space
        const long long r0 = (long long)b * kLines;
        const int p = int(r0 / NN);
        const long long row = r0 % NN + l;
        const int fa = 2 * p, fb = 2 * p + 1;
        const bool has_b = fb < prm.fields;
        if constexpr (PASS == kPassX) {
            const T c0 = T(prm.c0), dt = T(prm.dt);
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const long long off = row * N + j + B * t;
                const T ua = u[fa * NNN + off];
                const T ub = has_b ? u[fb * NNN + off] : T(0);
                x[t].x = c0 * ua + dt * (ua - ua * ua * ua);
                x[t].y = has_b ? c0 * ub + dt * (ub - ub * ub * ub) : T(0);
            }
            line_fft<T, N, A, B, -1>(x, tw, line, j, wmask);
#pragma unroll
            for (int t = 0; t < A; ++t) W[(long long)p * NNN + row * N + j + B * t] = x[t];
        } else {
#pragma unroll
            for (int t = 0; t < A; ++t) x[t] = W[(long long)p * NNN + row * N + j + B * t];
            line_fft<T, N, A, B, 1>(x, tw, line, j, wmask);
            const T scale = T(1.0 / double(NNN));
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const long long off = row * N + j + B * t;
                uo[fa * NNN + off] = x[t].x * scale;
                if (has_b) uo[fb * NNN + off] = x[t].y * scale;
            }
        }
    } else {
        // lines along j (Y, Y') at fixed (p, i = q) or along i (Z) at fixed
        // (p, j = q); line l is k = k0 + l
        constexpr int KC = N / kLines;
        const int kc = b % KC, q = (b / KC) % N, p = b / (KC * N);
        const int k = kc * kLines + l;
        auto addr = [&](int idx) -> long long {
            if constexpr (PASS == kPassZ) return (long long)p * NNN + (long long)idx * NN + (long long)q * N + k;
            else return (long long)p * NNN + (long long)q * NN + (long long)idx * N + k;
        };
#pragma unroll
        for (int t = 0; t < A; ++t) x[t] = W[addr(j + B * t)];
        if constexpr (PASS == kPassZ) {
            line_fft<T, N, A, B, -1>(x, tw, line, j, wmask);
            // x[t]: mode (a = j + B t, q, k); divide by the symbol
            const T base = T(prm.c0) + s2[q] + s2[k];
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const T inv = T(1) / (base + s2[j + B * t]);
                x[t].x *= inv;
                x[t].y *= inv;
            }
            if (prm.mass && q == 0 && k == 0 && j == 0) {
                double ta = 0.0, tb = 0.0;
                for (int c = 0; c < kMeanChunks; ++c) {
                    ta += part[(2 * p) * kMeanChunks + c];
                    if (2 * p + 1 < prm.fields) tb += part[(2 * p + 1) * kMeanChunks + c];
                }
                x[0].x = T(ta);  // sums over the field: N^3 times the mean
                x[0].y = T(tb);
            }
            line_fft<T, N, A, B, 1>(x, tw, line, j, wmask);
        } else {
            line_fft<T, N, A, B, PASS == kPassYi ? 1 : -1>(x, tw, line, j, wmask);
        }
#pragma unroll
        for (int t = 0; t < A; ++t) W[addr(j + B * t)] = x[t];
    }
}

// The line_fft table tw[k1 B + j] = exp(-2 pi i ((j k1) mod N) / N) and the
// symbol table, once per call.
template <typename T, int N>
__global__ void fine3d_tables(vec2_t<T>* tw, T* s2, double coef) {
    constexpr int B = Split<N>::B;
    const int e = threadIdx.x;
    if (e < N) {
        const int k1 = e / B, j = e % B;
        double sn, cs;
        sincospi(2.0 * double((j * k1) % N) / N, &sn, &cs);
        tw[e].x = T(cs);
        tw[e].y = T(-sn);
        const double sv = sinpi(double(e) / N);
        s2[e] = T(coef * sv * sv);
    }
}

// Per-field partial sums (float64 across threads) of the field, for the mean.
template <typename T, int N>
__global__ void __launch_bounds__(kSumThreads) fine3d_sums(const T* __restrict__ u, double* __restrict__ part) {
    constexpr long long NNN = (long long)N * N * N;
    constexpr long long chunk = NNN / kMeanChunks;
    const int f = blockIdx.y, c = blockIdx.x;
    const T* base = u + f * NNN + c * chunk;
    T acc = T(0);
    for (long long i = threadIdx.x; i < chunk; i += kSumThreads) acc += base[i];
    double d = double(acc);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    __shared__ double red[kSumThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kSumThreads / 32; ++w) t += red[w];
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
    off += align256(2 * es * size_t(n));
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
        fine3d_sums<T, N><<<dim3(kMeanChunks, fields), kSumThreads, 0, st>>>(u_in, part);
        ACPR_LAUNCH_CHECK();
    }
    Step3 prm{1.0 + p->S * p->dt, p->dt, p->variant == AC_MASS_CONSERVING, fields};
    const int pairs = (fields + 1) / 2;
    const unsigned gx = unsigned((long long)pairs * N * N / kLines);
    const unsigned gyz = unsigned((long long)pairs * N * (N / kLines));
    constexpr int threads = kLines * Split<N>::B;
    const T* src = u_in;
    for (int s = 0; s < steps; ++s) {
        fine3d_pass<T, N, kPassX><<<gx, threads, 0, st>>>(src, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassY><<<gyz, threads, 0, st>>>(nullptr, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassZ><<<gyz, threads, 0, st>>>(nullptr, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassYi><<<gyz, threads, 0, st>>>(nullptr, nullptr, W, tw, s2, part, prm);
        ACPR_LAUNCH_CHECK();
        fine3d_pass<T, N, kPassXi><<<gx, threads, 0, st>>>(nullptr, u_out, W, tw, s2, part, prm);
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
