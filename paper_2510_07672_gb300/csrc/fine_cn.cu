// fine_cn.cu -- the paper's own fine scheme (Sec. 3.1): a Crank-Nicolson step
//   (U' - U)/dt = eps^2 Lap_h (U' + U)/2 + (f(U') + f(U))/2 - g(U, U'),
// g = 0 (classic) or the mean of (f(U') + f(U))/2 (mass-conserving), solved by
// Picard iteration: U^0 = U and
//   (I + hmu) U^{m+1} = (I - hmu) U + dt/2 (f(U) + f(U^m)) - dt g,
// hmu = -dt/2 eps^2 Lap_h (diagonal in the DFT basis: dt/2 eps^2 (mu_k + mu_l)),
// until max |U^{m+1} - U^m| <= tol or max_iters iterations.
//
// GB300 mapping: the cluster layout of fine.cu (one cluster of P CTAs per
// field, two rows of the field per complex line, row FFTs, DSMEM transposes,
// half spectra with the DC and Nyquist columns packed in column 0, column
// FFTs).  A step holds, per field, the spectrum of U in shared memory (from
// the previous step's last solve, or one extra forward transform at launch);
// it forms A = (1 - hmu) U_hat + dt/2 FFT(f(U)) once and then iterates: a
// Picard iteration is a forward transform of f(U^m) (skipped for m = 0, whose
// transform is that of f(U)), the division by (1 + hmu), the inverse
// transform, and the max |U^{m+1} - U^m| over the field (warp shuffle, shared
// memory, then the cluster's CTAs through DSMEM), which every CTA evaluates
// identically.  In the mass-conserving variant the mean mode is held at the
// float64 entry mean: the scheme conserves it exactly in exact arithmetic.
#include "common.cuh"
#include "fft_reg.cuh"

namespace cg = cooperative_groups;

namespace acpr {
namespace {

struct CnArgs {
    const void* in;
    void* out;
    int num_fields;
    int steps;
    int mass;
    int max_iters;
    double tol;
    double lamh_scale;  // dt/2 eps^2 (4 / h^2)
    double dt;
    int* iters;         // optional: total Picard iterations per field
    // work list (overrides the plain field index and `steps`): field f reads
    // field work[f].x of `in`, writes field work[f].y of `out`, runs
    // work[f].z steps
    const int4* work;
};

template <int P>
__device__ __forceinline__ void cn_cluster_barrier() {
    if constexpr (P > 1) {
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

template <int P, typename V>
__device__ __forceinline__ V* cn_peer(V* local, int rank) {
    if constexpr (P > 1) {
        return cg::this_cluster().map_shared_rank(local, rank);
    } else {
        return local;
    }
}

__host__ __device__ constexpr int cn_exchange_pitch(int len, int B) {
    return B >= 16 ? len + 1 : len + (((B - len) % 16) + 16) % 16;
}
__host__ __device__ constexpr int cn_transpose_pitch(int L, int B) {
    return ((L / (16 / B)) | 1) * (16 / B) >= L ? ((L / (16 / B)) | 1) * (16 / B)
                                                 : ((L / (16 / B)) + 2 | 1) * (16 / B);
}

template <typename T, int N, int P, int A, int B>
struct CnShape {
    static constexpr int R = N / P, L = R / 2, HALF = N / 2, THREADS = L * B;
    static constexpr int XP = cn_exchange_pitch(xlen<N, B>(), B);
    static constexpr int TP = cn_transpose_pitch(L, B);
    // bufR, bufC (transpose targets, position-major), bufX (exchanges), the
    // A and last-solve spectra [L][N], tables, cluster max slots
    static constexpr size_t V2 = sizeof(vec2_t<T>);
    static constexpr size_t SMEM = V2 * (2 * size_t(N) * TP + size_t(L) * XP + 2 * size_t(L) * N + N) +
                                   sizeof(T) * N + 8 * sizeof(double);
    static_assert(R >= 2 && R % 2 == 0 && B <= 16 && TP >= L, "shape");
};

template <typename T, int N, int P, int A, int B>
__global__ void __launch_bounds__(CnShape<T, N, P, A, B>::THREADS, 1)
fine_cn_kernel(CnArgs args) {
    using Sh = CnShape<T, N, P, A, B>;
    using V = vec2_t<T>;
    constexpr int R = Sh::R, L = Sh::L, HALF = Sh::HALF, TP = Sh::TP, XP = Sh::XP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* bufR = reinterpret_cast<V*>(smem_raw);
    V* bufC = bufR + N * TP;
    V* bufX = bufC + N * TP;
    V* Ahat = bufX + L * XP;      // [line][k]: A = (1 - hmu) U_hat + dt/2 FFT(f(U))
    V* Shat = Ahat + L * N;       // [line][k]: spectrum of the current U
    V* tw = Shat + L * N;
    T* lamh = reinterpret_cast<T*>(tw + N);                 // dt/2 eps^2 mu_k
    double* part = reinterpret_cast<double*>(lamh + N);     // [0]: mass partial, [2..3]: cluster max slots

    const int tid = threadIdx.x;
    const int j = tid % B, line = tid / B;
    constexpr unsigned WMASK = Sh::THREADS >= 32 ? 0xffffffffu : ((1u << Sh::THREADS) - 1u);
    int rank = 0;
    if constexpr (P > 1) rank = int(cg::this_cluster().block_rank());
    const int field = blockIdx.x / P;
    const size_t NN = size_t(N) * N;
    long long fin = field, fout = field;
    int nsteps = args.steps;
    if (args.work) {
        const int4 w = args.work[field];
        fin = w.x;
        fout = w.y;
        nsteps = w.z;
    }
    const T* in = static_cast<const T*>(args.in) + size_t(fin) * NN + size_t(rank) * R * N;
    T* out = static_cast<T*>(args.out) + size_t(fout) * NN + size_t(rank) * R * N;

    for (int k = tid; k < N; k += Sh::THREADS) {
        double sn, cs;
        sincospi(-2.0 * double(((k % B) * (k / B)) & (N - 1)) / N, &sn, &cs);
        tw[k].x = T(cs);
        tw[k].y = T(sn);
        const double s = sinpi(double(k) / N);
        lamh[k] = T(args.lamh_scale * s * s);
    }
    double msum = 0.0;
    for (int idx = tid; idx < R * N; idx += Sh::THREADS) {
        const int row = idx / N, c = idx % N;
        const T v = in[idx];
        msum += double(v);
        reinterpret_cast<T*>(bufR)[2 * (c * TP + row % L) + row / L] = v;
    }
    double mean = 0.0;
    if (args.mass) {
        constexpr int WARP = Sh::THREADS < 32 ? Sh::THREADS : 32;
        constexpr unsigned MASK = WARP == 32 ? 0xffffffffu : ((1u << WARP) - 1u);
#pragma unroll
        for (int o = WARP / 2; o > 0; o >>= 1) msum += __shfl_xor_sync(MASK, msum, o, WARP);
        double* wsum = reinterpret_cast<double*>(bufC);
        if ((tid % WARP) == 0) wsum[tid / WARP] = msum;
        __syncthreads();
        if (tid == 0) {
            double sa = 0.0;
            for (int w = 0; w < Sh::THREADS / WARP; ++w) sa += wsum[w];
            part[0] = sa;
        }
        cn_cluster_barrier<P>();
        double sa = 0.0;
        for (int q = 0; q < P; ++q) sa += *cn_peer<P>(part, q);
        mean = sa / double(NN);
        cn_cluster_barrier<P>();
    }
    __syncthreads();

    V* myR = bufR + line;
    V* myC = bufC + line;
    V* myX = bufX + line * XP;
    V* myA = Ahat + line * N;
    V* myS = Shat + line * N;
    const int pair = rank * L + line;
    const int col = rank * L + line;
    const T half = T(0.5), hdt = T(0.5 * args.dt);
    const T inv_nn = T(1.0 / double(NN));
    const T dc_mass = T(mean * double(NN));  // held mean mode, forward-transform scale

    V u[A];  // current iterate, row layout (physical)
#pragma unroll
    for (int t = 0; t < A; ++t) u[t] = myR[(j + B * t) * TP];

    // forward 2D transform: x (row layout, two real rows per line) ->
    // x (column layout, half spectra, columns 0 and N/2 packed in column 0)
    auto forward2d = [&](V (&x)[A]) {
        line_fft<T, N, A, B, -1>(x, tw, myX, j, WMASK);
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int k = j + B * t;
            const int c = (k == HALF) ? 0 : (k < HALF ? k : N - k);
            const int slot = (k == 0 || k < HALF) ? 0 : 1;
            V* dst = cn_peer<P>(bufC, c / L);
            dst[(slot * HALF + pair) * TP + c % L] = x[t];
        }
        cn_cluster_barrier<P>();
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int r = j + B * t;
            const int lr = r % R;
            const int pp = (r / R) * L + (lr % L);
            const V za = myC[pp * TP], zb = myC[(HALF + pp) * TP];
            V v;
            if (col == 0) {
                if (lr < L) { v.x = za.x; v.y = zb.x; }
                else        { v.x = za.y; v.y = zb.y; }
            } else if (lr < L) {
                v.x = half * (za.x + zb.x);
                v.y = half * (za.y - zb.y);
            } else {
                v.x = half * (za.y + zb.y);
                v.y = half * (zb.x - za.x);
            }
            x[t] = v;
        }
        line_fft<T, N, A, B, -1>(x, tw, myX, j, WMASK);
    };
    // inverse 2D transform: column layout -> row layout (unnormalised)
    auto inverse2d = [&](V (&x)[A]) {
        line_fft<T, N, A, B, +1>(x, tw, myX, j, WMASK);
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int r = j + B * t;
            const int lr = r % R;
            V* dst = cn_peer<P>(bufR, r / R);
            dst[((lr / L) * HALF + col) * TP + lr % L] = x[t];
        }
        cn_cluster_barrier<P>();
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int k = j + B * t;
            V z;
            if (k == 0 || k == HALF) {
                const V va = myR[0], vb = myR[HALF * TP];
                if (k == 0) { z.x = va.x; z.y = vb.x; }
                else        { z.x = va.y; z.y = vb.y; }
            } else if (k < HALF) {
                const V va = myR[k * TP], vb = myR[(HALF + k) * TP];
                z.x = va.x - vb.y;
                z.y = va.y + vb.x;
            } else {
                const V va = myR[(N - k) * TP], vb = myR[(HALF + N - k) * TP];
                z.x = va.x + vb.y;
                z.y = vb.x - va.y;
            }
            x[t] = z;
        }
        line_fft<T, N, A, B, +1>(x, tw, myX, j, WMASK);
    };
    // multiply the column-layout spectrum by a per-mode factor phi(hmu):
    // columns c != 0 by phi(lamh[k] + lamh[c]); the packed column 0 (columns
    // 0 and N/2 as F0 + i FN) by separating the two with C[N - k]:
    // C'[k] = C[k] (p0 + pN)/2 + conj(C[N - k]) (p0 - pN)/2
    auto scale = [&](V (&x)[A], auto phi) {
        if (col != 0) {
            const T lc = lamh[col];
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const T s = phi(lamh[j + B * t] + lc);
                x[t].x *= s;
                x[t].y *= s;
            }
        }
        __syncwarp(WMASK);
        if (col == 0) {
#pragma unroll
            for (int t = 0; t < A; ++t) myX[j + B * t] = x[t];
        }
        __syncwarp(WMASK);
        if (col == 0) {
            const T ln = lamh[HALF];
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const int k = j + B * t;
                const V zc = x[t];
                const V zp = myX[(N - k) & (N - 1)];
                const T p0 = phi(lamh[k]), pn = phi(lamh[k] + ln);
                const T sp = half * (p0 + pn), sm = half * (p0 - pn);
                x[t].x = zc.x * sp + zp.x * sm;
                x[t].y = zc.y * sp - zp.y * sm;
            }
        }
    };
    auto one_minus = [](T hm) { return T(1) - hm; };
    auto inv_one_plus = [](T hm) { return T(1) / (T(1) + hm); };

    // spectrum of the entry field
    {
        V x[A];
#pragma unroll
        for (int t = 0; t < A; ++t) x[t] = u[t];
        forward2d(x);
#pragma unroll
        for (int t = 0; t < A; ++t) myS[j + B * t] = x[t];
    }
    // every CTA has read its column data before the next transform writes
    // bufC again
    cn_cluster_barrier<P>();
    int iters_total = 0;
    int slot = 0;  // cluster-max slot, alternating
    const T tol = T(args.tol);
    __shared__ T warp_max[32];
    for (int step = 0; step < nsteps; ++step) {
        // fm = F0 = FFT(f(U)); A = (1 - hmu) U_hat + dt/2 F0
        V fm[A];
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const T ur = u[t].x, ui = u[t].y;
            fm[t].x = ur - ur * ur * ur;
            fm[t].y = ui - ui * ui * ui;
        }
        forward2d(fm);
        {
            V s[A];
#pragma unroll
            for (int t = 0; t < A; ++t) s[t] = myS[j + B * t];
            scale(s, one_minus);
#pragma unroll
            for (int t = 0; t < A; ++t) {
                myA[j + B * t].x = s[t].x + hdt * fm[t].x;
                myA[j + B * t].y = s[t].y + hdt * fm[t].y;
            }
        }
        // Picard: rhs = A + dt/2 FFT(f(U^m)) (fm = F0 for m = 0)
        for (int m = 0; m < args.max_iters; ++m) {
            V x[A];
#pragma unroll
            for (int t = 0; t < A; ++t) {
                x[t].x = myA[j + B * t].x + hdt * fm[t].x;
                x[t].y = myA[j + B * t].y + hdt * fm[t].y;
            }
            scale(x, inv_one_plus);
            if (args.mass && col == 0 && j == 0) {
                // mode (0, 0) in slot 0 of the packed column: real part = column 0's DC
                x[0].x = dc_mass;
            }
#pragma unroll
            for (int t = 0; t < A; ++t) {
                myS[j + B * t] = x[t];
                x[t].x *= inv_nn;
                x[t].y *= inv_nn;
            }
            inverse2d(x);
            // max |U^{m+1} - U^m| over the field
            T d = T(0);
#pragma unroll
            for (int t = 0; t < A; ++t) {
                d = fmax(d, fabs(x[t].x - u[t].x));
                d = fmax(d, fabs(x[t].y - u[t].y));
                u[t] = x[t];
            }
            ++iters_total;
            constexpr int WARP = Sh::THREADS < 32 ? Sh::THREADS : 32;
            constexpr unsigned MASK = WARP == 32 ? 0xffffffffu : ((1u << WARP) - 1u);
#pragma unroll
            for (int o = WARP / 2; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(MASK, d, o, WARP));
            if ((tid % WARP) == 0) warp_max[tid / WARP] = d;
            __syncthreads();
            if (tid == 0) {
                T c = T(0);
                for (int w = 0; w < Sh::THREADS / WARP; ++w) c = fmax(c, warp_max[w]);
                part[2 + slot] = double(c);
            }
            cn_cluster_barrier<P>();
            double g = 0.0;
            for (int q = 0; q < P; ++q) g = fmax(g, cn_peer<P>(part, q)[2 + slot]);
            slot ^= 1;
            if (g <= double(tol) || m + 1 == args.max_iters) break;
            // next iterate's nonlinearity in spectral form
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const T ur = u[t].x, ui = u[t].y;
                fm[t].x = ur - ur * ur * ur;
                fm[t].y = ui - ui * ui * ui;
            }
            forward2d(fm);
        }
    }
    if (args.iters && tid == 0 && rank == 0) args.iters[field] = iters_total;

    // store rows through bufR
    __syncthreads();
#pragma unroll
    for (int t = 0; t < A; ++t) myR[(j + B * t) * TP] = u[t];
    __syncthreads();
    for (int idx = tid; idx < R * N; idx += Sh::THREADS) {
        const int row = idx / N, c = idx % N;
        out[idx] = reinterpret_cast<const T*>(bufR)[2 * (c * TP + row % L) + row / L];
    }
    cn_cluster_barrier<P>();  // peers may still read this CTA's cluster-max slot
}

template <typename T, int N, int P, int A, int B>
int launch_cn(const CnArgs& args, cudaStream_t st) {
    using Sh = CnShape<T, N, P, A, B>;
    auto kern = fine_cn_kernel<T, N, P, A, B>;
    static bool configured = false;
    if (!configured) {
        ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::SMEM)));
        if (P > 8) ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(args.num_fields * P), 1, 1);
    cfg.blockDim = dim3(Sh::THREADS, 1, 1);
    cfg.dynamicSmemBytes = Sh::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ACPR_CUDA(cudaLaunchKernelEx(&cfg, kern, args));
    count_launch();
    return AC_OK;
}

}  // namespace

static int cn_launch(const ac_params* p, const CnArgs& a, cudaStream_t st) {
    if (p->precision == AC_F32) {
        switch (p->n) {
            case 64: return launch_cn<float, 64, 2, 8, 8>(a, st);
            case 128: return launch_cn<float, 128, 4, 16, 8>(a, st);
            case 256: return launch_cn<float, 256, 8, 16, 16>(a, st);
            default: break;
        }
    } else {
        switch (p->n) {
            case 64: return launch_cn<double, 64, 2, 8, 8>(a, st);
            default: break;
        }
    }
    set_error("ac_cn_propagate_slices: n=%d not built for precision %d (64, 128, 256 f32; 64 f64)", p->n,
              p->precision);
    return AC_ERR_UNSUPPORTED;
}

bool cn_supported(int n, int precision) {
    return precision == AC_F32 ? (n == 64 || n == 128 || n == 256) : (precision == AC_F64 && n == 64);
}

static int cn_check(const ac_params* p, double tol, int max_iters) {
    ACPR_CHECK_ARG(p != nullptr, "ac_params is NULL");
    ACPR_CHECK_ARG(p->precision == AC_F32 || p->precision == AC_F64, "bad precision %d", p->precision);
    ACPR_CHECK_ARG(p->variant == AC_CLASSIC || p->variant == AC_MASS_CONSERVING, "bad variant %d", p->variant);
    ACPR_CHECK_ARG(p->length > 0 && p->dt > 0 && p->eps >= 0, "need length > 0, dt > 0, eps >= 0");
    ACPR_CHECK_ARG(max_iters >= 1 && tol >= 0, "need max_iters >= 1 and tol >= 0");
    return AC_OK;
}

static CnArgs cn_args(const ac_params* p, double tol, int max_iters) {
    CnArgs a{};
    a.mass = p->variant == AC_MASS_CONSERVING;
    a.max_iters = max_iters;
    a.tol = tol;
    const double h = p->length / p->n;
    a.lamh_scale = 0.5 * p->dt * p->eps * p->eps * 4.0 / (h * h);
    a.dt = p->dt;
    return a;
}

// Work-list form (the Parareal driver's fine sweep): item f advances field
// work[f].x of `in` by work[f].z steps into field work[f].y of `out`.
int cn_run_work(const ac_params* p, int count, const int4* work, const void* in, void* out, double tol,
                int max_iters, cudaStream_t st) {
    int rc = cn_check(p, tol, max_iters);
    if (rc) return rc;
    ACPR_CHECK_ARG(count >= 0 && work && in && out, "bad work-list arguments");
    if (count == 0) return AC_OK;
    CnArgs a = cn_args(p, tol, max_iters);
    a.in = in;
    a.out = out;
    a.num_fields = count;
    a.work = work;
    return cn_launch(p, a, st);
}

int cn_propagate(const ac_params* p, int num_fields, int steps, const void* in, void* out, double tol,
                 int max_iters, int* iters_dev, cudaStream_t st) {
    int rc = cn_check(p, tol, max_iters);
    if (rc) return rc;
    ACPR_CHECK_ARG(num_fields >= 0 && steps >= 0, "bad counts");
    if (num_fields == 0) return AC_OK;
    ACPR_CHECK_ARG(in && out && in != out, "bad field pointers");
    ACPR_CHECK_ARG((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16 == 0,
                   "fields must be 16-byte aligned");
    ACPR_CHECK_ARG(num_fields < (1 << 24), "too many fields");
    CnArgs a = cn_args(p, tol, max_iters);
    a.in = in;
    a.out = out;
    a.num_fields = num_fields;
    a.steps = steps;
    a.iters = iters_dev;
    return cn_launch(p, a, st);
}

}  // namespace acpr

extern "C" int ac_cn_propagate_slices(const ac_params* params, int num_fields, int steps, const void* u_in,
                                      void* u_out, double tol, int max_iters, int* picard_iters,
                                      acpr_stream stream) {
    return acpr::cn_propagate(params, num_fields, steps, u_in, u_out, tol, max_iters, picard_iters,
                              reinterpret_cast<cudaStream_t>(stream));
}
