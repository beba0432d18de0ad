// fine.cu -- the fine propagator F: stabilised semi-implicit Allen-Cahn steps
// on a periodic n x n grid, many independent fields at once.
//
// One step (Sec. 3.1 fine operator, the stabilised linear scheme):
//   r      = (1 + S dt) u + dt f(u),                f(u) = u - u^3
//   u_hat' = FFT2(r)_kl / (N^2 D_kl),   D_kl = 1 + S dt + dt eps^2 (mu_k + mu_l),
//   u'     = IFFT2(u_hat')               (unnormalised inverse),
// mu_k = (4/h^2) sin^2(pi k / N) (minus the eigenvalues of the periodic 5-point
// Laplacian).  For the mass-conserving model (Eq. mass_AC_eq) the Lagrange
// multiplier beta = mean f(u) only moves the (0,0) mode, where it cancels
// dt * mean f(u); the (0,0) mode of u_hat' is therefore the mean of u, which
// the kernel holds at the float64 mean taken when the field was loaded.
//
// GB300 mapping.  A thread-block cluster of P CTAs owns one field for all
// `steps` steps; CTA q holds rows [qR, qR + R), R = N / P.  The field is real,
// so two rows of the same field travel as the real and imaginary parts of one
// complex line (rows qR + l and qR + l + R/2): every rounding then depends on
// this field alone, which makes F a deterministic function of its input, the
// property that lets converged Parareal slices stop changing bitwise.
//   row phase:    R/2 complex lines per CTA, N-point row FFTs;
//   transpose:    the row spectra Z_p[k] go straight into the peer CTAs'
//                 shared memory (DSMEM), column c receiving Z_p[c] and
//                 Z_p[N - c] of every row pair p;
//   column phase: the column owner splits each pair into the two real rows'
//                 half spectra (Hermitian symmetry), N/2 complex columns per
//                 field with the real DC and Nyquist columns packed into
//                 column 0, N-point column FFTs, symbol divide, inverse;
//   and back the same way.  Each 1D transform is a two-pass radix-A x radix-B
// register FFT with one shared-memory exchange.  Two cluster barriers per step
// order the transposes; HBM is read once when the field is loaded and written
// once when it is stored.
#include "common.cuh"
#include "fft_reg.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace acpr {

namespace {
// Set by a fine kernel whose bounded wait on its exchange mbarrier gave up
// (fine_check_status() reports and clears it).
__device__ int g_fine_timeout = 0;
constexpr long long kFineSpin = 20000000LL;  // polls (each try_wait suspends briefly): seconds
}

// Shared::cluster address of `local_addr` (a shared::cta address) in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_map(uint32_t local_addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}

// Bulk copy of `bytes` (multiple of 16, 16-byte aligned ends) from this CTA's
// shared memory to a peer's, completing `bytes` transaction bytes on the
// peer's mbarrier.
__device__ __forceinline__ void bulk_s2peer(uint32_t dst_cluster, uint32_t src_cta, uint32_t bytes,
                                            uint32_t mbar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_cluster),
        "r"(src_cta), "r"(bytes), "r"(mbar_cluster)
        : "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the async
// proxy (the bulk copies issued after the next barrier).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct FineArgs {
    const void* in;
    void* out;
    int num_fields;
    int steps;
    // Field f = g * per_group + i reads field (map[g] * in_gs + in_off + i) of
    // `in` and writes field (map[g] * out_gs + out_off + i) of `out` (map NULL:
    // identity).  Plain batched calls use per_group = num_fields.
    int per_group;
    long long in_gs, in_off, out_gs, out_off;
    const int* map;
    // Work list (overrides the mapping above and `steps`): field f reads field
    // work[f].x of `in`, writes field work[f].y of `out`, runs work[f].z steps.
    const int4* work;
    int mass;        // 1: hold the (0,0) mode at the entry mean
    // adjoint = 1 runs the transposed steps: lambda_n = a mu + dt f'(u_n) * (mu -
    // [mass] mean mu), mu = A^{-1} lambda_{n+1}, with u_n read from
    // states[n][field] (n = steps-1 .. 0, plain field index).
    int adjoint;
    const void* states;
    // traj != NULL stores the state before the first step and after every
    // step: traj[s][field] for s = 0..steps (plain field index).
    void* traj;
    double a;        // 1 + S dt
    double dt;
    double lam_scale;  // dt eps^2 (4 / h^2)
};

// Smallest value >= len that is congruent to B modulo 16 (B < 16); B = 16
// (one line per half-warp) takes len + 1.
__host__ __device__ constexpr int exchange_pitch(int len, int B) {
    return B >= 16 ? len + 1 : len + (((B - len) % 16) + 16) % 16;
}

// Smallest odd multiple of 16/B that is >= L (B <= 16).
__host__ __device__ constexpr int transpose_pitch(int L, int B) {
    return ((L / (16 / B)) | 1) * (16 / B) >= L ? ((L / (16 / B)) | 1) * (16 / B)
                                                 : ((L / (16 / B)) + 2 | 1) * (16 / B);
}

// NOX: no separate exchange buffer; the line FFTs of the row phase exchange
// through bufR and those of the column phase through bufC, each free at that
// time (asynchronous exchange only), which saves a third of the shared memory.
template <typename T, int N, int P, int A, int B, bool NOX = false>
struct FineShape {
    static constexpr int R = N / P;           // rows per CTA
    static constexpr int L = R / 2;           // lines per CTA (row pairs, then columns)
    static constexpr int HALF = N / 2;
    static constexpr int THREADS = L * B;     // (line, lane) pairs
    // bufX: one padded exchange area per line.  A half-warp holds 16/B lines;
    // with XP = B (mod 16) their areas start 2B banks apart and the exchange
    // writes and reads of those lines fall in distinct banks.
    static constexpr int XP = exchange_pitch(xlen<N, B>(), B);
    // bufR, bufC (transpose targets): position-major, element (pos, line) at
    // pos * TP + line.  A sender's B lanes write B consecutive lines at one
    // position (one contiguous run in the peer's memory); a reader's half-warp
    // (16/B lines, B positions each, TP elements apart) hits distinct banks
    // when TP is an odd multiple of 16/B.
    static constexpr int TP = transpose_pitch(L, B);
    static constexpr int BUFT_ELEMS = NOX && L * XP > N * TP ? L * XP : N * TP;
    static constexpr size_t BUFT = sizeof(vec2_t<T>) * size_t(BUFT_ELEMS);
    static constexpr size_t BUFX = NOX ? 0 : sizeof(vec2_t<T>) * size_t(L) * XP;
    static constexpr size_t SMEM = 2 * BUFT + BUFX + sizeof(vec2_t<T>) * N + sizeof(T) * N + 4 * sizeof(double) +
                                   2 * sizeof(uint64_t);
    // asynchronous exchange: a peer's share of a transpose is L positions of
    // TP elements per half (2 bulk copies per peer), 16-byte aligned
    static constexpr uint32_t RUN_BYTES = uint32_t(sizeof(vec2_t<T>) * L * TP);
    static constexpr bool ASYNC_OK = (RUN_BYTES % 16 == 0) && ((sizeof(vec2_t<T>) * HALF * TP) % 16 == 0) &&
                                     (BUFT % 16 == 0);
    static_assert(R >= 2 && R % 2 == 0, "need at least two rows per CTA");
    static_assert(B <= 16 && TP >= L, "transpose layout");
};

// Division where float32 round-off of a couple of ulp is harmless (the
// symbol); float64 keeps the IEEE division.
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

template <int P>
__device__ __forceinline__ void cluster_barrier() {
    if constexpr (P > 1) {
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

template <int P, typename V>
__device__ __forceinline__ V* peer_ptr(V* local, int rank) {
    if constexpr (P > 1) {
        return cg::this_cluster().map_shared_rank(local, rank);
    } else {
        return local;
    }
}

// MINB: CTAs per SM the register allocation must allow (occupancy target).
// ASYNC (P > 1, no adjoint mode): the two transposes of a step travel as bulk
// shared-memory copies to the peers, completing on one mbarrier per receive
// buffer, instead of direct DSMEM stores ordered by two cluster barriers.  A
// CTA stages the data for peer d in its own receive buffer's region for data
// *from* d (that region is next written by d only after d has received this
// CTA's data, so it is free), and the element for itself directly in the
// other buffer.  No cluster-wide barrier and no release fence in the step
// loop: a CTA waits only for the bytes it receives.
template <typename T, int N, int P, int A, int B, int MINB, bool ASYNC = false, bool NOX = false>
__global__ void __launch_bounds__(FineShape<T, N, P, A, B, NOX>::THREADS, MINB)
fine_field_kernel(FineArgs args) {
    using Sh = FineShape<T, N, P, A, B, NOX>;
    using V = vec2_t<T>;
    constexpr int R = Sh::R, L = Sh::L, HALF = Sh::HALF, TP = Sh::TP, XP = Sh::XP;
    static_assert(!NOX || ASYNC, "the shared exchange areas need the asynchronous exchange");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* bufR = reinterpret_cast<V*>(smem_raw);         // row phase: [pos][line]
    V* bufC = bufR + Sh::BUFT_ELEMS;                   // column phase: [pos][line]
    V* bufX = bufC + Sh::BUFT_ELEMS;                   // line-FFT exchanges (not with NOX)
    V* tw = bufX + (NOX ? 0 : L * XP);                 // line_fft twiddle table
    T* lam = reinterpret_cast<T*>(tw + N);             // dt eps^2 mu_k
    double* part = reinterpret_cast<double*>(lam + N); // mass partial, adjoint mean
    uint64_t* xbar = reinterpret_cast<uint64_t*>(part + 4);  // [0]: bufC received, [1]: bufR received
    static_assert(!ASYNC || (P > 1 && Sh::ASYNC_OK), "asynchronous exchange layout");
    constexpr uint32_t XBYTES = uint32_t(P - 1) * 2u * Sh::RUN_BYTES;  // bytes received per transpose

    const int tid = threadIdx.x;
    // the B lanes of a line are consecutive lanes of one warp, so the line
    // FFTs' exchanges need warp barriers only
    const int j = tid % B;       // lane within a line
    const int line = tid / B;    // local line index
    constexpr unsigned WMASK = Sh::THREADS >= 32 ? 0xffffffffu : ((1u << Sh::THREADS) - 1u);
    int rank = 0;
    if constexpr (P > 1) rank = int(cg::this_cluster().block_rank());
    const int field = blockIdx.x / P;
    const size_t NN = size_t(N) * N;
    long long fin, fout;
    int nsteps = args.steps;
    if (args.work) {
        const int4 w = args.work[field];
        fin = w.x;
        fout = w.y;
        nsteps = w.z;
    } else {
        const int g = field / args.per_group, i = field % args.per_group;
        const long long pg = args.map ? args.map[g] : g;
        fin = pg * args.in_gs + args.in_off + i;
        fout = pg * args.out_gs + args.out_off + i;
    }
    const T* in = static_cast<const T*>(args.in) + size_t(fin) * NN + size_t(rank) * R * N;
    T* out = static_cast<T*>(args.out) + size_t(fout) * NN + size_t(rank) * R * N;

    for (int k = tid; k < N; k += Sh::THREADS) {
        double sn, cs;
        sincospi(-2.0 * double(((k % B) * (k / B)) & (N - 1)) / N, &sn, &cs);
        tw[k].x = T(cs);
        tw[k].y = T(sn);
        const double s = sinpi(double(k) / N);
        lam[k] = T(args.lam_scale * s * s);
    }
    if constexpr (ASYNC) {
        if (tid == 0) {
            tc::mbar_init(&xbar[0], 1);
            tc::mbar_init(&xbar[1], 1);
            tc::fence_mbar_init();
            if (nsteps > 0) {
                tc::mbar_arrive_expect_tx(&xbar[0], XBYTES);
                tc::mbar_arrive_expect_tx(&xbar[1], XBYTES);
            }
        }
        // every peer's barriers exist before anyone sends
        cluster_barrier<P>();
    }

    // load rows [rank R, rank R + R): line l holds rows l (real) and l + L (imag)
    double msum = 0.0;
    T* traj0 = args.traj ? static_cast<T*>(args.traj) + size_t(field) * NN + size_t(rank) * R * N : nullptr;
    const size_t traj_step = size_t(args.num_fields) * NN;
    for (int idx = tid; idx < R * N; idx += Sh::THREADS) {
        const int row = idx / N, c = idx % N;
        const T v = in[idx];
        msum += double(v);
        reinterpret_cast<T*>(bufR)[2 * (c * TP + row % L) + row / L] = v;
        if (traj0) traj0[idx] = v;
    }
    double mean = 0.0;
    if (args.mass && !args.adjoint) {
        // float64 sum: warp shuffle, one value per warp, then the cluster
        constexpr int WARP = Sh::THREADS < 32 ? Sh::THREADS : 32;
        constexpr unsigned MASK = WARP == 32 ? 0xffffffffu : ((1u << WARP) - 1u);
#pragma unroll
        for (int o = WARP / 2; o > 0; o >>= 1) msum += __shfl_xor_sync(MASK, msum, o, WARP);
        double* wsum = reinterpret_cast<double*>(bufC);  // scratch before first use
        if ((tid % WARP) == 0) wsum[tid / WARP] = msum;
        __syncthreads();
        if (tid == 0) {
            double sa = 0.0;
            for (int w = 0; w < Sh::THREADS / WARP; ++w) sa += wsum[w];
            part[0] = sa;
        }
        cluster_barrier<P>();
        double sa = 0.0;
        for (int q = 0; q < P; ++q) sa += *peer_ptr<P>(part, q);
        mean = sa / double(NN);
        cluster_barrier<P>();  // peers are done reading `part`
    }
    __syncthreads();

    V x[A];
    V* myR = bufR + line;  // element pos of this line at myR[pos * TP]
    V* myC = bufC + line;
    // this line's exchange areas of the row and the column phase
    V* myXR = (NOX ? bufR : bufX) + line * XP;
    V* myXC = (NOX ? bufC : bufX) + line * XP;
#pragma unroll
    for (int t = 0; t < A; ++t) x[t] = myR[(j + B * t) * TP];
    if constexpr (NOX) __syncthreads();  // bufR read before it serves as exchange area

    const T a = T(args.a);
    const T dt = T(args.dt);
    const T inv_nn = T(1.0 / double(NN));
    const T half = T(0.5);
    const int pair = rank * L + line;  // global row-pair index (row phase)
    const int col = rank * L + line;   // global column index (column phase)
    // Exchange buffers and barriers per step.  Every line FFT, and the
    // column-0 separation, exchanges through the line's own area of bufX,
    // which only the line's lanes (one warp) touch: warp barriers order it.
    // bufR and bufC are only transpose targets (and the load/store staging),
    // ordered by the two cluster barriers.
    // Asynchronous exchange (ASYNC): `src` holds, at the region of each peer d
    // (positions h HALF + d L .. + L, h = 0, 1), the data for d; it goes to
    // d's `dst` at the region of this CTA, completing on d's barrier `bar`.
    bool xabort = false;  // a bounded wait gave up: skip later waits
    auto exchange_send = [&](V* src, V* dst, uint64_t* bar) {
        fence_proxy_async_smem();
        __syncthreads();
        if (tid < 2 * (P - 1)) {
            const int dd = tid >> 1, h = tid & 1;
            const int d = dd < rank ? dd : dd + 1;
            const uint32_t s_addr = tc::smem_u32(src + (h * HALF + d * L) * TP);
            const uint32_t d_addr = cluster_map(tc::smem_u32(dst + (h * HALF + rank * L) * TP), uint32_t(d));
            bulk_s2peer(d_addr, s_addr, Sh::RUN_BYTES, cluster_map(tc::smem_u32(bar), uint32_t(d)));
        }
    };
    auto exchange_wait = [&](int b, int stp) {
        bool ok = xabort;
        for (long long i = 0; !ok && i < kFineSpin; ++i) ok = tc::mbar_try_wait(&xbar[b], uint32_t(stp & 1));
        if (!ok) {
            xabort = true;
            atomicExch(&g_fine_timeout, 1);
        }
        // arm the next phase (its bytes come only after this CTA's next send)
        if (tid == 0 && stp + 1 < nsteps) tc::mbar_arrive_expect_tx(&xbar[b], XBYTES);
    };
    (void)exchange_send;
    (void)exchange_wait;
    for (int step = 0; step < nsteps; ++step) {
        if (!args.adjoint) {
            // pointwise right-hand side on both rows of the line
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const T ur = x[t].x, ui = x[t].y;
                x[t].x = a * ur + dt * (ur - ur * ur * ur);
                x[t].y = a * ui + dt * (ui - ui * ui * ui);
            }
        }
        line_fft<T, N, A, B, -1>(x, tw, myXR, j, WMASK);
        // row spectra Z_p[k] -> column min(k, N - k) (k = 0, N/2 -> column 0)
        if constexpr (ASYNC) {
            __syncthreads();  // every rebuild read of bufR (now the staging area) is done
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const int k = j + B * t;
                const int c = (k == HALF) ? 0 : (k < HALF ? k : N - k);
                const int slot = (k == 0 || k < HALF) ? 0 : 1;
                const int d = c / L;
                if (d == rank) bufC[(slot * HALF + pair) * TP + c % L] = x[t];
                else bufR[(slot * HALF + d * L + line) * TP + c % L] = x[t];
            }
            exchange_send(bufR, bufC, &xbar[0]);
            exchange_wait(0, step);
        } else {
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const int k = j + B * t;
                const int c = (k == HALF) ? 0 : (k < HALF ? k : N - k);
                const int slot = (k == 0 || k < HALF) ? 0 : 1;
                V* dst = peer_ptr<P>(bufC, c / L);
                dst[(slot * HALF + pair) * TP + c % L] = x[t];
            }
            cluster_barrier<P>();
        }
        // split each row pair into its two rows' half spectra
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int r = j + B * t;
            const int lr = r % R;
            const int pp = (r / R) * L + (lr % L);
            const V za = myC[pp * TP], zb = myC[(HALF + pp) * TP];
            V v;
            if (col == 0) {  // packed DC and Nyquist columns
                if (lr < L) { v.x = za.x; v.y = zb.x; }
                else        { v.x = za.y; v.y = zb.y; }
            } else if (lr < L) {  // (za + conj zb) / 2
                v.x = half * (za.x + zb.x);
                v.y = half * (za.y - zb.y);
            } else {              // (za - conj zb) / (2i)
                v.x = half * (za.y + zb.y);
                v.y = half * (zb.x - za.x);
            }
            x[t] = v;
        }
        if constexpr (NOX) __syncthreads();  // every split read of bufC is done
        line_fft<T, N, A, B, -1>(x, tw, myXC, j, WMASK);
        // divide by the symbol, with 1/N^2 of the inverse folded in
        if (col != 0) {
            const T lam_l = lam[col];
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const T s = fast_div(inv_nn, a + (lam[j + B * t] + lam_l));
                x[t].x *= s;
                x[t].y *= s;
            }
        }
        {
            // column 0 carries columns 0 and N/2 as C = F0 + i FN: separate
            // them with C[N - k], scale each by its own symbol, recombine:
            // C'[k] = C[k] (s0 + sN) / 2 + conj(C[N - k]) (s0 - sN) / 2
            // (through this line's area of bufX, after the FFT's reads)
            __syncwarp(WMASK);
            if (col == 0) {
#pragma unroll
                for (int t = 0; t < A; ++t) myXC[j + B * t] = x[t];
            }
            __syncwarp(WMASK);
            if (col == 0) {
                const T lam_n = lam[HALF];
#pragma unroll
                for (int t = 0; t < A; ++t) {
                    const int k = j + B * t;
                    const V zc = x[t];
                    const V zp = myXC[(N - k) & (N - 1)];
                    const T lk = lam[k];
                    const T s0 = fast_div(inv_nn, a + lk);
                    const T sn = fast_div(inv_nn, a + (lk + lam_n));
                    const T sp = half * (s0 + sn), sm = half * (s0 - sn);
                    x[t].x = zc.x * sp + zp.x * sm;
                    x[t].y = zc.y * sp - zp.y * sm;
                    if (k == 0 && args.mass) {
                        if (!args.adjoint) {
                            // mean mode of u held at the entry mean (F0'(0) = mean)
                            x[t].x = T(mean);
                            x[t].y = zc.y * sn;
                        } else {
                            // F0'(0) is mean(mu): hand it to every CTA of the
                            // cluster before the barrier that ends the phase
                            for (int q = 0; q < P; ++q) peer_ptr<P>(part, q)[1] = double(x[t].x);
                        }
                    }
                }
            }
        }
        line_fft<T, N, A, B, +1>(x, tw, myXC, j, WMASK);
        // column values V_r[c] -> owner of row r, slot (row role) and column c
        if constexpr (ASYNC) {
            __syncthreads();  // every split read of bufC (now the staging area) is done
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const int r = j + B * t;
                const int lr = r % R;
                const int d = r / R;
                if (d == rank) bufR[((lr / L) * HALF + col) * TP + lr % L] = x[t];
                else bufC[((lr / L) * HALF + d * L + line) * TP + lr % L] = x[t];
            }
            exchange_send(bufC, bufR, &xbar[1]);
            exchange_wait(1, step);
        } else {
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const int r = j + B * t;
                const int lr = r % R;
                V* dst = peer_ptr<P>(bufR, r / R);
                dst[((lr / L) * HALF + col) * TP + lr % L] = x[t];
            }
            cluster_barrier<P>();
        }
        // rebuild each pair's full row spectrum from the half spectra
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int k = j + B * t;
            V z;
            if (k == 0 || k == HALF) {
                const V va = myR[0], vb = myR[HALF * TP];
                if (k == 0) { z.x = va.x; z.y = vb.x; }
                else        { z.x = va.y; z.y = vb.y; }
            } else if (k < HALF) {  // Va + i Vb
                const V va = myR[k * TP], vb = myR[(HALF + k) * TP];
                z.x = va.x - vb.y;
                z.y = va.y + vb.x;
            } else {                // conj(Va) + i conj(Vb) at N - k
                const V va = myR[(N - k) * TP], vb = myR[(HALF + N - k) * TP];
                z.x = va.x + vb.y;
                z.y = vb.x - va.y;
            }
            x[t] = z;
        }
        if constexpr (NOX) __syncthreads();  // every rebuild read of bufR is done
        line_fft<T, N, A, B, +1>(x, tw, myXR, j, WMASK);
        if (args.adjoint) {
            // lambda_n = a mu + dt f'(u_n) (mu - mean mu), rows r0 (real) and r1 (imag)
            const int n_state = nsteps - 1 - step;
            const T* un = static_cast<const T*>(args.states) + (size_t(n_state) * args.num_fields + field) * NN +
                          size_t(rank * R + line) * N;
            const T mbar = args.mass ? T(part[1]) : T(0);
#pragma unroll
            for (int t = 0; t < A; ++t) {
                const int c = j + B * t;
                const T u0 = un[c], u1 = un[size_t(L) * N + c];
                const T f0 = T(1) - T(3) * u0 * u0, f1 = T(1) - T(3) * u1 * u1;
                x[t].x = a * x[t].x + dt * f0 * (x[t].x - mbar);
                x[t].y = a * x[t].y + dt * f1 * (x[t].y - mbar);
            }
        }
        if (args.traj) {
            __syncthreads();
#pragma unroll
            for (int t = 0; t < A; ++t) myR[(j + B * t) * TP] = x[t];
            __syncthreads();
            T* ts = static_cast<T*>(args.traj) + (size_t(step + 1) * traj_step) + size_t(field) * NN +
                    size_t(rank) * R * N;
            for (int idx = tid; idx < R * N; idx += Sh::THREADS) {
                const int row = idx / N, c = idx % N;
                ts[idx] = reinterpret_cast<const T*>(bufR)[2 * (c * TP + row % L) + row / L];
            }
            if constexpr (NOX) __syncthreads();  // bufR read before the next row FFT's exchange
        }
    }

    // store rows, coalesced, through bufR
    if constexpr (ASYNC) {
        // every CTA has received all its bytes, so no copy of this cluster is
        // still reading or writing shared memory when its CTAs exit
        cluster_barrier<P>();
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < A; ++t) myR[(j + B * t) * TP] = x[t];
    __syncthreads();
    for (int idx = tid; idx < R * N; idx += Sh::THREADS) {
        const int row = idx / N, c = idx % N;
        out[idx] = reinterpret_cast<const T*>(bufR)[2 * (c * TP + row % L) + row / L];
    }
}

// ---------------------------------------------------------------- launch --
template <typename T, int N, int P, int A, int B, int MINB, bool ASYNC = false, bool NOX = false>
static int launch_fine(const FineArgs& args, cudaStream_t stream) {
    using Sh = FineShape<T, N, P, A, B, NOX>;
    auto kern = fine_field_kernel<T, N, P, A, B, MINB, ASYNC, NOX>;
    static bool configured = false;  // per instantiation, once per process
    if (!configured) {
        ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::SMEM)));
        if (P > 8)
            ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(args.num_fields * P), 1, 1);
    cfg.blockDim = dim3(Sh::THREADS, 1, 1);
    cfg.dynamicSmemBytes = Sh::SMEM;
    cfg.stream = stream;
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

// Launch shapes built for each (precision, n): cluster size P, threads per
// CTA, occupancy target.  Entry 0 is the default; ac_fine_autotune times them
// all on the caller's problem and keeps the fastest.
struct FineVariant {
    const char* name;
    int (*launch)(const FineArgs&, cudaStream_t);
    bool async;  // asynchronous exchange: no adjoint mode
    int P;       // CTAs per field (the split that fixes the rounding)
};

#define ACPR_FV(T, N, P, A, B, M) {"P" #P "_A" #A "_B" #B "_occ" #M, &launch_fine<T, N, P, A, B, M>, false, P}
#define ACPR_FVA(T, N, P, A, B, M) \
    {"P" #P "_A" #A "_B" #B "_occ" #M "_async", &launch_fine<T, N, P, A, B, M, true>, true, P}
#define ACPR_FVN(T, N, P, A, B, M) \
    {"P" #P "_A" #A "_B" #B "_occ" #M "_async_nox", &launch_fine<T, N, P, A, B, M, true, true>, true, P}

template <typename T>
static const FineVariant* fine_variants(int n, int* count) {
    static const FineVariant v8[] = {ACPR_FV(T, 8, 1, 4, 2, 1)};
    static const FineVariant v16[] = {ACPR_FV(T, 16, 1, 4, 4, 1)};
    static const FineVariant v32[] = {ACPR_FV(T, 32, 1, 8, 4, 1)};
    static const FineVariant v64[] = {ACPR_FV(T, 64, 1, 8, 8, 2), ACPR_FV(T, 64, 2, 8, 8, 3)};
    if constexpr (sizeof(T) == 4) {
        static const FineVariant v128[] = {ACPR_FV(T, 128, 2, 16, 8, 2), ACPR_FV(T, 128, 4, 16, 8, 3),
                                           ACPR_FV(T, 128, 1, 16, 8, 1), ACPR_FVA(T, 128, 4, 16, 8, 3),
                                           ACPR_FVA(T, 128, 2, 16, 8, 2)};
        // entry 0 (clusters of 8, asynchronous exchange, no separate exchange
        // buffer, 3 CTAs per SM) measured fastest on large batches (512 fields,
        // 20 steps: 2.46 ms; with the exchange buffer 2.56 ms; cluster
        // barriers 2.97 ms).  16-CTA clusters are 10% faster on 16 fields, but a
        // shape change alters the rounding, and F must stay one function within
        // a solve and between a Parareal solve and its sequential reference
        // (exactness at k = s): the default does not depend on the batch size.
        static const FineVariant v256[] = {ACPR_FVN(T, 256, 8, 16, 16, 3), ACPR_FVA(T, 256, 8, 16, 16, 2),
                                           ACPR_FVA(T, 256, 16, 16, 16, 3), ACPR_FVA(T, 256, 4, 16, 16, 1),
                                           ACPR_FV(T, 256, 8, 16, 16, 2), ACPR_FV(T, 256, 4, 16, 16, 1),
                                           ACPR_FV(T, 256, 16, 16, 16, 3), ACPR_FV(T, 256, 8, 16, 16, 1),
                                           ACPR_FVN(T, 256, 8, 16, 16, 2)};
        static const FineVariant v512[] = {ACPR_FV(T, 512, 16, 32, 16, 1), ACPR_FVA(T, 512, 16, 32, 16, 1)};
        switch (n) {
            case 128: *count = 5; return v128;
            case 256: *count = 9; return v256;
            case 512: *count = 2; return v512;
            default: break;
        }
    } else {
        static const FineVariant v128[] = {ACPR_FV(T, 128, 4, 16, 8, 1), ACPR_FV(T, 128, 2, 16, 8, 1),
                                           ACPR_FVA(T, 128, 4, 16, 8, 1)};
        static const FineVariant v256[] = {ACPR_FV(T, 256, 8, 16, 16, 1), ACPR_FV(T, 256, 16, 16, 16, 2),
                                           ACPR_FVA(T, 256, 8, 16, 16, 1)};
        switch (n) {
            case 128: *count = 3; return v128;
            case 256: *count = 3; return v256;
            default: break;
        }
    }
    switch (n) {
        case 8: *count = 1; return v8;
        case 16: *count = 1; return v16;
        case 32: *count = 1; return v32;
        case 64: *count = 2; return v64;
        default: *count = 0; return nullptr;
    }
}
#undef ACPR_FV
#undef ACPR_FVA
#undef ACPR_FVN

namespace {
int g_variant[2][11] = {};  // [precision][log2 n]: chosen launch shape
}

static const FineVariant* pick_variant(int n, int precision, int* count) {
    const FineVariant* v = precision == AC_F64 ? fine_variants<double>(n, count) : fine_variants<float>(n, count);
    return v;
}

template <typename T>
static int dispatch_fine(int n, const FineArgs& args, cudaStream_t stream) {
    int count = 0;
    const FineVariant* v = fine_variants<T>(n, &count);
    if (!v || !count) {
        set_error("ac_fine: n=%d not built for %s", n, sizeof(T) == 8 ? "AC_F64" : "AC_F32");
        return AC_ERR_UNSUPPORTED;
    }
    const int pr = sizeof(T) == 8 ? AC_F64 : AC_F32;
    int idx = g_variant[pr][ilog2(n)];
    if (idx < 0 || idx >= count) idx = 0;
    // the adjoint's mean broadcast is ordered by cluster barriers: take the
    // barrier-exchange shape of the same split (same rounding), else the first
    if (args.adjoint && v[idx].async) {
        const int want = v[idx].P;
        int alt = -1;
        for (int i = 0; i < count && alt < 0; ++i)
            if (!v[i].async && v[i].P == want) alt = i;
        for (int i = 0; i < count && alt < 0; ++i)
            if (!v[i].async) alt = i;
        idx = alt < 0 ? count : alt;
        if (idx == count) {
            set_error("ac_fine: no barrier-exchange shape for the adjoint at n=%d", n);
            return AC_ERR_UNSUPPORTED;
        }
    }
    return v[idx].launch(args, stream);
}

// Device-side timeout flag of the fine kernels' bounded exchange waits:
// AC_ERR_TIMEOUT (and the flag cleared) if one gave up since the last call.
// Synchronises the stream.
int fine_check_status(cudaStream_t st) {
    int flag = 0;
    ACPR_CUDA(cudaMemcpyFromSymbolAsync(&flag, g_fine_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    ACPR_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        const int zero = 0;
        ACPR_CUDA(cudaMemcpyToSymbolAsync(g_fine_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        ACPR_CUDA(cudaStreamSynchronize(st));
        set_error("fine step: a bounded exchange wait gave up");
        return AC_ERR_TIMEOUT;
    }
    return AC_OK;
}

bool fine_big_supported(int n, int precision);
int fine_big_run(const ac_params* p, int groups, int per_group, int steps, const void* in, long long in_gs,
                 long long in_off, void* out, long long out_gs, long long out_off, const int* map, void* ws,
                 cudaStream_t st);

static bool fine_built(int n, int precision) {
    int count = 0;
    if (fine_big_supported(n, precision)) return true;
    return is_pow2(n) && n <= 1024 && pick_variant(n, precision, &count) != nullptr && count > 0;
}

bool fine_supported_internal(int n, int precision) { return is_pow2(n) && fine_built(n, precision); }

static int check_params(const ac_params* p) {
    ACPR_CHECK_ARG(p != nullptr, "ac_params is NULL");
    ACPR_CHECK_ARG(p->precision == AC_F32 || p->precision == AC_F64, "bad precision %d", p->precision);
    ACPR_CHECK_ARG(p->variant == AC_CLASSIC || p->variant == AC_MASS_CONSERVING, "bad variant %d", p->variant);
    ACPR_CHECK_ARG(p->length > 0 && p->dt > 0 && p->eps >= 0 && p->S >= 0,
                   "need length > 0, dt > 0, eps >= 0, S >= 0");
    if (!is_pow2(p->n) || !fine_built(p->n, p->precision)) {
        set_error("ac_fine: n=%d (precision %d) not supported", p->n, p->precision);
        return AC_ERR_UNSUPPORTED;
    }
    return AC_OK;
}

size_t fine_big_workspace_bytes(int n, int fields);

int fine_run(const ac_params* p, int groups, int per_group, int steps, const void* in, long long in_gs,
             long long in_off, void* out, long long out_gs, long long out_off, const int* map, int adjoint,
             const void* states, void* traj, cudaStream_t stream, void* big_ws = nullptr,
             size_t big_ws_bytes = 0);

int fine_run(const ac_params* p, int groups, int per_group, int steps, const void* in, long long in_gs,
             long long in_off, void* out, long long out_gs, long long out_off, const int* map, int adjoint,
             const void* states, void* traj, cudaStream_t stream, void* big_ws, size_t big_ws_bytes) {
    int rc = check_params(p);
    if (rc) return rc;
    ACPR_CHECK_ARG(groups >= 0 && per_group >= 0 && steps >= 0, "counts must be >= 0");
    if (groups == 0 || per_group == 0) return AC_OK;
    ACPR_CHECK_ARG(in && out, "null field pointer");
    ACPR_CHECK_ARG(in != out, "u_in and u_out must not overlap");
    ACPR_CHECK_ARG((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16 == 0,
                   "field pointers must be 16-byte aligned");
    ACPR_CHECK_ARG((long long)groups * per_group < (1LL << 30), "too many fields");
    if (fine_big_supported(p->n, p->precision)) {
        if (adjoint || traj || states) {
            set_error("ac_fine: n=%d supports plain propagation only (no trajectory or adjoint mode)", p->n);
            return AC_ERR_UNSUPPORTED;
        }
        if (big_ws) {
            const size_t need = fine_big_workspace_bytes(p->n, groups * per_group);
            ACPR_CHECK_ARG(big_ws_bytes >= need, "ac_fine: workspace needs %zu bytes", need);
            ACPR_CHECK_ARG(reinterpret_cast<uintptr_t>(big_ws) % 256 == 0, "workspace must be 256-byte aligned");
        }
        return fine_big_run(p, groups, per_group, steps, in, in_gs, in_off, out, out_gs, out_off, map, big_ws,
                            stream);
    }
    FineArgs a{};
    a.in = in;
    a.out = out;
    a.num_fields = groups * per_group;
    a.steps = steps;
    a.per_group = per_group;
    a.in_gs = in_gs;
    a.in_off = in_off;
    a.out_gs = out_gs;
    a.out_off = out_off;
    a.map = map;
    a.work = nullptr;
    a.adjoint = adjoint;
    a.states = states;
    a.traj = traj;
    a.mass = p->variant == AC_MASS_CONSERVING;
    a.a = 1.0 + p->S * p->dt;
    a.dt = p->dt;
    const double h = p->length / p->n;
    a.lam_scale = p->dt * p->eps * p->eps * 4.0 / (h * h);
    if (p->precision == AC_F64) return dispatch_fine<double>(p->n, a, stream);
    return dispatch_fine<float>(p->n, a, stream);
}

int fine_propagate_mapped(const ac_params* p, int groups, int per_group, int steps, const void* in,
                          long long in_gs, long long in_off, void* out, long long out_gs,
                          long long out_off, const int* map, cudaStream_t stream, void* big_ws,
                          size_t big_ws_bytes) {
    return fine_run(p, groups, per_group, steps, in, in_gs, in_off, out, out_gs, out_off, map, 0, nullptr,
                    nullptr, stream, big_ws, big_ws_bytes);
}

// Work-list launch: `count` fields, field f = (in field, out field, steps)
// from the device array work[f] (int4 x, y, z).
int fine_run_work(const ac_params* p, int count, const int4* work, const void* in, void* out, cudaStream_t stream) {
    int rc = check_params(p);
    if (rc) return rc;
    ACPR_CHECK_ARG(count >= 0 && (count == 0 || (work && in && out)), "bad work list");
    ACPR_CHECK_ARG(reinterpret_cast<uintptr_t>(work) % 16 == 0, "work list must be 16-byte aligned");
    if (fine_big_supported(p->n, p->precision)) {
        set_error("ac_fine: n=%d has no work-list launch (uniform steps only)", p->n);
        return AC_ERR_UNSUPPORTED;
    }
    if (!count) return AC_OK;
    FineArgs a{};
    a.in = in;
    a.out = out;
    a.num_fields = count;
    a.steps = 0;
    a.per_group = count;
    a.work = work;
    a.mass = p->variant == AC_MASS_CONSERVING;
    a.a = 1.0 + p->S * p->dt;
    a.dt = p->dt;
    const double h = p->length / p->n;
    a.lam_scale = p->dt * p->eps * p->eps * 4.0 / (h * h);
    if (p->precision == AC_F64) return dispatch_fine<double>(p->n, a, stream);
    return dispatch_fine<float>(p->n, a, stream);
}

int fine_propagate(const ac_params* p, int num_fields, int steps, const void* in, void* out,
                   cudaStream_t stream) {
    return fine_propagate_mapped(p, 1, num_fields, steps, in, 0, 0, out, 0, 0, nullptr, stream, nullptr, 0);
}

}  // namespace acpr

extern "C" int ac_fine_supported(int n, int precision) {
    return acpr::is_pow2(n) && acpr::fine_built(n, precision) ? 1 : 0;
}

extern "C" int ac_fine_step(const ac_params* params, int batch, const void* u_in, void* u_out,
                            acpr_stream stream) {
    return acpr::fine_propagate(params, batch, 1, u_in, u_out, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ac_fine_propagate_slices(const ac_params* params, int num_fields, int steps_per_slice,
                                        const void* u_starts, void* u_ends, acpr_stream stream) {
    return acpr::fine_propagate(params, num_fields, steps_per_slice, u_starts, u_ends,
                                reinterpret_cast<cudaStream_t>(stream));
}

extern "C" size_t ac_fine_workspace_bytes(int n, int num_fields, int precision) {
    if (num_fields <= 0 || !acpr::fine_big_supported(n, precision)) return 0;
    return acpr::fine_big_workspace_bytes(n, num_fields);
}

extern "C" int ac_fine_propagate_slices_ws(const ac_params* params, int num_fields, int steps_per_slice,
                                           const void* u_starts, void* u_ends, void* workspace,
                                           size_t workspace_bytes, acpr_stream stream) {
    using namespace acpr;
    if (params && fine_big_supported(params->n, params->precision) && num_fields > 0)
        ACPR_CHECK_ARG(workspace != nullptr, "ac_fine_propagate_slices_ws: n=%d needs a workspace", params->n);
    return fine_propagate_mapped(params, 1, num_fields, steps_per_slice, u_starts, 0, 0, u_ends, 0, 0, nullptr,
                                 reinterpret_cast<cudaStream_t>(stream), workspace, workspace_bytes);
}

extern "C" int ac_fine_trajectory(const ac_params* params, int num_fields, int steps, const void* u0, void* traj,
                                  acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(traj != nullptr, "traj is NULL");
    // the final state also lands in traj[steps]; `out` receives it too
    const size_t esz = params ? elem_size(params->precision) : 8;
    void* last = params ? static_cast<char*>(traj) + size_t(steps) * num_fields * params->n * params->n * esz
                        : nullptr;
    return fine_run(params, 1, num_fields, steps, u0, 0, 0, last, 0, 0, nullptr, 0, nullptr, traj,
                    reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ac_fine_adjoint(const ac_params* params, int num_fields, int steps, const void* states,
                               const void* lam_end, void* lam_start, acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(states != nullptr, "states is NULL");
    return fine_run(params, 1, num_fields, steps, lam_end, 0, 0, lam_start, 0, 0, nullptr, 1, states, nullptr,
                    reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ac_fine_variant_count(int n, int precision) {
    int count = 0;
    if (!acpr::is_pow2(n) || n > 1024 || (precision != AC_F32 && precision != AC_F64)) return 0;
    acpr::pick_variant(n, precision, &count);
    return count;
}

extern "C" const char* ac_fine_variant_name(int n, int precision, int index) {
    int count = ac_fine_variant_count(n, precision);
    if (index < 0 || index >= count) return "";
    return acpr::pick_variant(n, precision, &count)[index].name;
}

extern "C" int ac_fine_get_variant(int n, int precision) {
    if (!ac_fine_variant_count(n, precision)) return -1;
    return acpr::g_variant[precision][acpr::ilog2(n)];
}

extern "C" int ac_fine_set_variant(int n, int precision, int index) {
    using namespace acpr;
    const int count = ac_fine_variant_count(n, precision);
    ACPR_CHECK_ARG(count > 0, "n=%d precision %d not built", n, precision);
    ACPR_CHECK_ARG(index >= 0 && index < count, "variant %d out of range (%d built)", index, count);
    g_variant[precision][ilog2(n)] = index;
    return AC_OK;
}

extern "C" int ac_fine_autotune(const ac_params* params, int num_fields, int steps, const void* u_in, void* u_out,
                                float* ms_out, acpr_stream stream) {
    using namespace acpr;
    int rc = check_params(params);
    if (rc) return rc;
    ACPR_CHECK_ARG(num_fields >= 1 && steps >= 1 && u_in && u_out, "bad autotune arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int count = ac_fine_variant_count(params->n, params->precision);
    cudaEvent_t e0, e1;
    ACPR_CUDA(cudaEventCreate(&e0));
    ACPR_CUDA(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < count; ++v) {
        g_variant[params->precision][ilog2(params->n)] = v;
        rc = fine_propagate(params, num_fields, steps, u_in, u_out, st);  // warm-up
        if (rc) break;
        ACPR_CUDA(cudaEventRecord(e0, st));
        for (int rep = 0; rep < 2 && !rc; ++rep) rc = fine_propagate(params, num_fields, steps, u_in, u_out, st);
        ACPR_CUDA(cudaEventRecord(e1, st));
        ACPR_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        ACPR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms *= 0.5f;
        if (ms_out) ms_out[v] = ms;
        if (ms < best_ms) { best_ms = ms; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_variant[params->precision][ilog2(params->n)] = best;
    return rc ? rc : AC_OK;
}

extern "C" int ac_fine_propagate_work(const ac_params* params, int count, const void* work, const void* u_in,
                                      void* u_out, acpr_stream stream) {
    return acpr::fine_run_work(params, count, static_cast<const int4*>(work), u_in, u_out,
                               reinterpret_cast<cudaStream_t>(stream));
}
