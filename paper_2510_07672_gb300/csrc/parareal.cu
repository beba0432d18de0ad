// parareal.cu -- Parareal correction, convergence increment and the iteration
// driver of Algorithm 2 (Sec. 3.3) for a batch of independent problems.
//
// Device state per problem p (precision T):
//   Ua, Ub [s+1][n][n]  trajectories U^{k-1} and U^k (swapped every iteration)
//   Gold   [s][n][n]    stored coarse values G(U^{k-1}_n), reused at iteration k
//   Fres   [s][n][n]    fine results F(U^{k-1}_n)
// Iteration k >= 1:
//   1. Fres[n] = F(Ua[n]), n = k-1..s-1              one batched fine launch
//   2. Ub[k-1] = Ua[k-1]                               newest frozen slice
//      Ub[k]   = Fres[k-1] + (Gold[k-1] - Gold[k-1])  (U^k_{k-1} = U^{k-1}_{k-1})
//   3. for n = k..s-1 in order: g = G(Ub[n]);
//      Ub[n+1] = Fres[n] + (g - Gold[n]);  Gold[n] = g
//   4. increment of Ub against Ua over slices 1..s, float64
// The frozen prefix Ub[0..k-2] already equals Ua[0..k-2] (both hold the exact
// fine values), so step 2 copies one slice only.  The summation order
// F + (G_new - G_old) keeps U^k_k bitwise equal to the fine result.
#include <mutex>
#include <vector>

#include "cnn.cuh"
#include "common.cuh"

namespace acpr {

int fine_propagate_mapped(const ac_params* p, int groups, int per_group, int steps, const void* in,
                          long long in_gs, long long in_off, void* out, long long out_gs,
                          long long out_off, const int* map, cudaStream_t stream);

// ------------------------------------------------------------- kernels ----
constexpr int kResThreads = 256;
constexpr int kResBlocksPerProblem = 64;

// Per (problem, block) partials of sum (a - b)^2, sum a^2, max |a - b| over
// `count` elements starting at a + map[p] * a_ps + off (same for b), float64.
template <typename T>
__global__ void increment_partials_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                          long long a_ps, long long b_ps, long long off,
                                          long long count, const int* __restrict__ map,
                                          double* __restrict__ part) {
    const int p = blockIdx.y;
    const long long pp = map ? map[p] : p;
    const T* ap = a + pp * a_ps + off;
    const T* bp = b + pp * b_ps + off;
    double num = 0.0, den = 0.0, mx = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = double(ap[i]), d = x - double(bp[i]);
        num += d * d;
        den += x * x;
        mx = fmax(mx, fabs(d));
        if (!(d == d)) mx = d;  // keep NaN visible (fmax drops it)
    }
    __shared__ double sh[3][kResThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
        const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = (m2 != m2) ? m2 : fmax(mx, m2);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sh[0][w] = num; sh[1][w] = den; sh[2][w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double n0 = 0.0, d0 = 0.0, m0 = 0.0;
        for (int i = 0; i < kResThreads / 32; ++i) {
            n0 += sh[0][i];
            d0 += sh[1][i];
            m0 = (sh[2][i] != sh[2][i]) ? sh[2][i] : fmax(m0, sh[2][i]);
        }
        double* o = part + ((long long)p * gridDim.x + blockIdx.x) * 3;
        o[0] = n0; o[1] = d0; o[2] = m0;
    }
}

// Fixed-order reduction of the block partials: res[p] = (rel_l2, max_abs, num, den).
__global__ void increment_finish_kernel(const double* __restrict__ part, int blocks, int problems,
                                        double* __restrict__ res) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= problems) return;
    double num = 0.0, den = 0.0, mx = 0.0;
    for (int i = 0; i < blocks; ++i) {
        const double* q = part + ((long long)p * blocks + i) * 3;
        num += q[0];
        den += q[1];
        mx = (q[2] != q[2]) ? q[2] : fmax(mx, q[2]);
    }
    res[4 * p + 0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
    res[4 * p + 1] = mx;
    res[4 * p + 2] = num;
    res[4 * p + 3] = den;
}

// Ub[n+1] = Fres[n] + (g - Gold[n]) and optionally Gold[n] = g, for the mapped
// problems.  g = G(Ub[n]) is compact [batch][nn]; if g is NULL, Gold[n] is used
// in its place (the exact slice) and Gold is left alone.
template <typename T>
__global__ void correct_kernel(T* __restrict__ Ub, T* __restrict__ Gold, const T* __restrict__ Fres,
                               const T* __restrict__ g, int slice, int s, long long nn, int batch,
                               const int* __restrict__ map) {
    const long long total = nn * batch;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = int(idx / nn);
        const long long i = idx % nn;
        const long long p = map ? map[b] : b;
        T* go = Gold + (p * s + slice) * nn + i;
        const T gold = *go;
        const T gn = g ? g[(long long)b * nn + i] : gold;
        Ub[(p * (s + 1) + slice + 1) * nn + i] = Fres[(p * s + slice) * nn + i] + (gn - gold);
        if (g) *go = gn;
    }
}

// ----------------------------------------------------- standalone residual --
namespace {
struct ResidualScratch {
    double* part = nullptr;
    double* res = nullptr;
    double* host = nullptr;  // pinned
};
std::mutex g_res_mutex;
std::vector<ResidualScratch> g_res_scratch;  // per device
}  // namespace

template <typename T>
static int launch_increment(const void* a, const void* b, long long a_ps, long long b_ps, long long off,
                            long long count, const int* map, int problems, double* part, double* res,
                            cudaStream_t st) {
    dim3 grid(kResBlocksPerProblem, problems);
    increment_partials_kernel<T><<<grid, kResThreads, 0, st>>>(static_cast<const T*>(a), static_cast<const T*>(b),
                                                                a_ps, b_ps, off, count, map, part);
    ACPR_LAUNCH_CHECK();
    increment_finish_kernel<<<(problems + 127) / 128, 128, 0, st>>>(part, kResBlocksPerProblem, problems, res);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

static int increment(int precision, const void* a, const void* b, long long a_ps, long long b_ps, long long off,
                     long long count, const int* map, int problems, double* part, double* res, cudaStream_t st) {
    if (precision == AC_F64) return launch_increment<double>(a, b, a_ps, b_ps, off, count, map, problems, part, res, st);
    return launch_increment<float>(a, b, a_ps, b_ps, off, count, map, problems, part, res, st);
}

int residual(int num_slices, int n, int precision, const void* U_new, const void* U_old, double* l2,
             double* mx, cudaStream_t st) {
    ACPR_CHECK_ARG(num_slices >= 1 && n >= 1, "need num_slices >= 1 and n >= 1");
    ACPR_CHECK_ARG(precision == AC_F64 || precision == AC_F32, "bad precision");
    ACPR_CHECK_ARG(U_new && U_old && l2 && mx, "null pointer");
    std::lock_guard<std::mutex> lock(g_res_mutex);
    int dev = 0;
    ACPR_CUDA(cudaGetDevice(&dev));
    if (int(g_res_scratch.size()) <= dev) g_res_scratch.resize(dev + 1);
    ResidualScratch& sc = g_res_scratch[dev];
    if (!sc.part) {
        ACPR_CUDA(cudaMalloc(&sc.part, sizeof(double) * 3 * kResBlocksPerProblem));
        ACPR_CUDA(cudaMalloc(&sc.res, sizeof(double) * 4));
        ACPR_CUDA(cudaMallocHost(&sc.host, sizeof(double) * 4));
    }
    const long long nn = (long long)n * n;
    int rc = increment(precision, U_new, U_old, 0, 0, nn, nn * num_slices, nullptr, 1, sc.part, sc.res, st);
    if (rc) return rc;
    ACPR_CUDA(cudaMemcpyAsync(sc.host, sc.res, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
    ACPR_CUDA(cudaStreamSynchronize(st));
    *l2 = sc.host[0];
    *mx = sc.host[1];
    if (!std::isfinite(sc.host[0]) || !std::isfinite(sc.host[1])) {
        set_error("parareal_residual: non-finite increment");
        return AC_ERR_NONFINITE;
    }
    return AC_OK;
}

// ------------------------------------------- allocation-free residual -----
// The same two kernels as parareal_residual, but the block partials live in
// a fixed file-scope device array instead of memory from cudaMalloc, and the
// results go to a device buffer the caller passes.  One block reduces at most
// kNoAllocElemsPerBlock elements, so the array bounds the problem size.
namespace {
constexpr int kNoAllocMaxBlocks = 2048;                  // 3 doubles each: 48 KiB
constexpr long long kNoAllocElemsPerBlock = 16384;       // 64 per thread
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_scratch[3 * kNoAllocMaxBlocks];
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};          // device address per device
std::mutex g_noalloc_mutex;
}  // namespace

int residual_noalloc(int num_slices, int n, int precision, const void* U_new, const void* U_old,
                     double* out_dev, cudaStream_t st) {
    ACPR_CHECK_ARG(num_slices >= 1 && n >= 1, "need num_slices >= 1 and n >= 1");
    ACPR_CHECK_ARG(precision == AC_F64 || precision == AC_F32, "bad precision");
    const long long count = (long long)n * n * num_slices;
    const long long blocks = (count + kNoAllocElemsPerBlock - 1) / kNoAllocElemsPerBlock;
    if (blocks > kNoAllocMaxBlocks) {
        set_error("parareal_residual_noalloc: %lld elements exceed the fixed scratch limit of %lld "
                  "(%d blocks x %lld elements); use parareal_residual",
                  count, (long long)kNoAllocMaxBlocks * kNoAllocElemsPerBlock, kNoAllocMaxBlocks,
                  kNoAllocElemsPerBlock);
        return AC_ERR_UNSUPPORTED;
    }
    ACPR_CHECK_ARG(U_new && U_old && out_dev, "null pointer");
    int dev = 0;
    ACPR_CUDA(cudaGetDevice(&dev));
    ACPR_CHECK_ARG(dev >= 0 && dev < kNoAllocMaxDevices, "device index %d out of range", dev);
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            // host code only sees a stand-in for the array: ask the runtime for
            // its address on this device (once per device)
            void* addr = nullptr;
            ACPR_CUDA(cudaGetSymbolAddress(&addr, g_noalloc_scratch));
            g_noalloc_ptr[dev] = static_cast<double*>(addr);
        }
        scratch = g_noalloc_ptr[dev];
    }
    const long long nn = (long long)n * n;
    dim3 grid(unsigned(blocks), 1);
    // every scratch slot the finish kernel reads is written by this call's
    // partials kernel first, so nothing needs clearing
    if (precision == AC_F64)
        increment_partials_kernel<double><<<grid, kResThreads, 0, st>>>(
            static_cast<const double*>(U_new), static_cast<const double*>(U_old), 0, 0, nn, count, nullptr, scratch);
    else
        increment_partials_kernel<float><<<grid, kResThreads, 0, st>>>(
            static_cast<const float*>(U_new), static_cast<const float*>(U_old), 0, 0, nn, count, nullptr, scratch);
    ACPR_LAUNCH_CHECK();
    increment_finish_kernel<<<1, 128, 0, st>>>(scratch, int(blocks), 1, out_dev);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

}  // namespace acpr

// ---------------------------------------------------------------- driver ---
struct ac_parareal {
    ac_params p;
    cnn_desc g;
    int problems = 0, s = 0, c = 0;
    size_t esz = 0;
    long long nn = 0;
    void* Ua = nullptr;
    void* Ub = nullptr;
    void* Gold = nullptr;
    void* Fres = nullptr;
    void* gtmp = nullptr;   // [problems][nn] coarse output of one sweep step
    void* work = nullptr;   // conv activations
    void* packed = nullptr; // bf16 weights
    int* d_map = nullptr;   // active problem indices
    int* h_map = nullptr;   // pinned
    double* d_part = nullptr;
    double* d_res = nullptr;
    double* h_res = nullptr;  // pinned [problems][4]
    std::vector<char> active;
    std::vector<char> synced;  // inactive problem whose trajectory is in both buffers
    int k_next = 0;
    bool timing = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ac_parareal_stats stats{};
};

namespace acpr {

static void free_state(ac_parareal* st) {
    if (!st) return;
    for (void* ptr : {st->Ua, st->Ub, st->Gold, st->Fres, st->gtmp, st->work, st->packed,
                      static_cast<void*>(st->d_map), static_cast<void*>(st->d_part), static_cast<void*>(st->d_res)})
        if (ptr) cudaFree(ptr);
    if (st->h_map) cudaFreeHost(st->h_map);
    if (st->h_res) cudaFreeHost(st->h_res);
    for (cudaEvent_t e : st->ev)
        if (e) cudaEventDestroy(e);
    delete st;
}

// Upload the active-problem list; returns the count.
static int upload_map(ac_parareal* st, cudaStream_t stream, int* count) {
    int m = 0;
    for (int p = 0; p < st->problems; ++p)
        if (st->active[p]) st->h_map[m++] = p;
    *count = m;
    if (m) ACPR_CUDA(cudaMemcpyAsync(st->d_map, st->h_map, sizeof(int) * m, cudaMemcpyHostToDevice, stream));
    return AC_OK;
}

template <typename T>
static int launch_correct(ac_parareal* st, void* Ub, int slice, const void* g, int m, cudaStream_t stream) {
    const long long total = st->nn * m;
    const int threads = 256;
    const long long want = (total + threads - 1) / threads;
    const unsigned blocks = unsigned(want < 152 * 16 ? want : 152 * 16);
    correct_kernel<T><<<blocks, threads, 0, stream>>>(static_cast<T*>(Ub), static_cast<T*>(st->Gold),
                                                      static_cast<const T*>(st->Fres), static_cast<const T*>(g),
                                                      slice, st->s, st->nn, m, st->d_map);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

static int correct(ac_parareal* st, void* Ub, int slice, const void* g, int m, cudaStream_t stream) {
    if (st->p.precision == AC_F64) return launch_correct<double>(st, Ub, slice, g, m, stream);
    return launch_correct<float>(st, Ub, slice, g, m, stream);
}

static int iterate(ac_parareal* st, int* k_inout, double* l2_out, double* mx_out, cudaStream_t stream) {
    const int k = *k_inout;
    ACPR_CHECK_ARG(k == st->k_next, "iteration %d requested, state is at %d", k, st->k_next);
    ACPR_CHECK_ARG(k <= st->s, "k = %d exceeds the slice count %d", k, st->s);
    const long long nn = st->nn;
    const int s = st->s;
    const size_t fb = st->esz * nn;  // bytes per field
    int m = 0;
    int rc = upload_map(st, stream, &m);
    if (rc) return rc;
    const bool tm = st->timing;
    auto mark = [&](int i) -> int {
        if (tm) ACPR_CUDA(cudaEventRecord(st->ev[i], stream));
        return AC_OK;
    };
    if (k == 0) {
        // U^0_0 = u0 (already in Ua[0]); sequential coarse sweep
        if ((rc = mark(1))) return rc;
        for (int n = 0; n < s; ++n) {
            rc = coarse_step_mapped(&st->g, st->p.n, m, static_cast<char*>(st->Ua) + n * fb, nn * (s + 1),
                                    st->d_map, static_cast<char*>(st->Gold) + n * fb, nn * s, st->d_map,
                                    stream);
            if (rc) return rc;
            for (int i = 0; i < m; ++i) {
                const int p = st->h_map[i];
                ACPR_CUDA(cudaMemcpyAsync(static_cast<char*>(st->Ua) + (size_t(p) * (s + 1) + n + 1) * fb,
                                          static_cast<char*>(st->Gold) + (size_t(p) * s + n) * fb, fb,
                                          cudaMemcpyDeviceToDevice, stream));
            }
            st->stats.coarse_calls += 1;
            st->stats.coarse_cells += (long long)m * nn;
        }
        if ((rc = mark(2))) return rc;
        if (tm) {
            float ms = 0.f;
            ACPR_CUDA(cudaEventSynchronize(st->ev[2]));
            ACPR_CUDA(cudaEventElapsedTime(&ms, st->ev[1], st->ev[2]));
            st->stats.coarse_ms += ms;
        }
        st->k_next = 1;
        *k_inout = 1;
        return AC_OK;
    }
    // an inactive problem keeps its last trajectory in both buffers, so that
    // the buffer swap below never exposes a stale one
    for (int p = 0; p < st->problems; ++p) {
        if (st->active[p] || st->synced[p]) continue;
        ACPR_CUDA(cudaMemcpyAsync(static_cast<char*>(st->Ub) + size_t(p) * (s + 1) * fb,
                                  static_cast<char*>(st->Ua) + size_t(p) * (s + 1) * fb, fb * (s + 1),
                                  cudaMemcpyDeviceToDevice, stream));
        st->synced[p] = 1;
    }
    if (m == 0) {
        std::swap(st->Ua, st->Ub);
        st->k_next = k + 1;
        *k_inout = k + 1;
        return AC_OK;
    }
    // 1. fine solves of slices k-1 .. s-1 of every active problem (one launch)
    if ((rc = mark(0))) return rc;
    rc = fine_propagate_mapped(&st->p, m, s - k + 1, st->c, st->Ua, s + 1, k - 1, st->Fres, s, k - 1,
                               st->d_map, stream);
    if (rc) return rc;
    st->stats.fine_launches += 1;
    st->stats.fine_cell_steps += (long long)m * (s - k + 1) * st->c * nn;
    if ((rc = mark(1))) return rc;
    // 2. newest frozen slice and the exact slice k
    for (int i = 0; i < m; ++i) {
        const int p = st->h_map[i];
        ACPR_CUDA(cudaMemcpyAsync(static_cast<char*>(st->Ub) + (size_t(p) * (s + 1) + k - 1) * fb,
                                  static_cast<char*>(st->Ua) + (size_t(p) * (s + 1) + k - 1) * fb, fb,
                                  cudaMemcpyDeviceToDevice, stream));
    }
    rc = correct(st, st->Ub, k - 1, nullptr, m, stream);
    if (rc) return rc;
    // 3. sequential correction sweep
    for (int n = k; n < s; ++n) {
        rc = coarse_step_mapped(&st->g, st->p.n, m, static_cast<char*>(st->Ub) + n * fb, nn * (s + 1),
                                st->d_map, st->gtmp, nn, nullptr, stream);
        if (rc) return rc;
        rc = correct(st, st->Ub, n, st->gtmp, m, stream);
        if (rc) return rc;
        st->stats.coarse_calls += 1;
        st->stats.coarse_cells += (long long)m * nn;
    }
    if ((rc = mark(2))) return rc;
    // 4. increments over slices 1..s
    rc = increment(st->p.precision, st->Ub, st->Ua, nn * (s + 1), nn * (s + 1), nn, nn * s, st->d_map, m,
                   st->d_part, st->d_res, stream);
    if (rc) return rc;
    if ((rc = mark(3))) return rc;
    ACPR_CUDA(cudaMemcpyAsync(st->h_res, st->d_res, sizeof(double) * 4 * m, cudaMemcpyDeviceToHost, stream));
    ACPR_CUDA(cudaStreamSynchronize(stream));
    st->stats.iterations += 1;
    if (tm) {
        float a = 0.f, b = 0.f, c = 0.f;
        ACPR_CUDA(cudaEventElapsedTime(&a, st->ev[0], st->ev[1]));
        ACPR_CUDA(cudaEventElapsedTime(&b, st->ev[1], st->ev[2]));
        ACPR_CUDA(cudaEventElapsedTime(&c, st->ev[2], st->ev[3]));
        st->stats.fine_ms += a;
        st->stats.coarse_ms += b;
        st->stats.increment_ms += c;
    }
    bool nonfinite = false;
    for (int i = 0; i < m; ++i) {
        const int p = st->h_map[i];
        if (l2_out) l2_out[p] = st->h_res[4 * i];
        if (mx_out) mx_out[p] = st->h_res[4 * i + 1];
        if (!std::isfinite(st->h_res[4 * i]) || !std::isfinite(st->h_res[4 * i + 1])) nonfinite = true;
    }
    std::swap(st->Ua, st->Ub);
    st->k_next = k + 1;
    *k_inout = k + 1;
    if (nonfinite) {
        set_error("parareal_iterate: non-finite increment at k = %d", k);
        return AC_ERR_NONFINITE;
    }
    return AC_OK;
}

}  // namespace acpr

extern "C" int parareal_residual(int num_slices, int n, int precision, const void* U_new, const void* U_old,
                                 double* rel_l2_out, double* max_abs_out, acpr_stream stream) {
    return acpr::residual(num_slices, n, precision, U_new, U_old, rel_l2_out, max_abs_out,
                          reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int parareal_residual_noalloc(int num_slices, int n, int precision, const void* U_new,
                                         const void* U_old, double* out_dev, acpr_stream stream) {
    return acpr::residual_noalloc(num_slices, n, precision, U_new, U_old, out_dev,
                                  reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ac_parareal_create(const ac_params* params, const cnn_desc* coarse, int problems,
                                  int num_slices, int steps_per_slice, const void* u0, ac_parareal** out) {
    using namespace acpr;
    ACPR_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    ACPR_CHECK_ARG(params && coarse && u0, "null argument");
    ACPR_CHECK_ARG(problems >= 1 && num_slices >= 1 && steps_per_slice >= 0, "bad counts");
    ACPR_CHECK_ARG(coarse->precision == params->precision, "coarse and fine precision differ");
    int rc = check_cnn(coarse);
    if (rc) return rc;
    if (!ac_fine_supported(params->n, params->precision)) {
        set_error("ac_parareal_create: n=%d not supported", params->n);
        return AC_ERR_UNSUPPORTED;
    }
    ac_parareal* st = new ac_parareal();
    st->p = *params;
    st->g = *coarse;
    st->problems = problems;
    st->s = num_slices;
    st->c = steps_per_slice;
    st->esz = elem_size(params->precision);
    st->nn = (long long)params->n * params->n;
    st->active.assign(problems, 1);
    st->synced.assign(problems, 0);
    const size_t fb = st->esz * st->nn;
    const size_t traj = fb * size_t(problems) * (num_slices + 1);
    const size_t slc = fb * size_t(problems) * num_slices;
    auto alloc = [&](void** p, size_t bytes) -> bool { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = alloc(&st->Ua, traj) && alloc(&st->Ub, traj) && alloc(&st->Gold, slc) && alloc(&st->Fres, slc) &&
              alloc(&st->gtmp, fb * problems);
    const size_t wb = work_bytes_for(coarse, params->n, problems);
    ok = ok && alloc(&st->work, wb);
    const size_t pb = cnn_packed_bytes(coarse);
    if (ok && pb) ok = alloc(&st->packed, pb);
    ok = ok && alloc(reinterpret_cast<void**>(&st->d_map), sizeof(int) * problems) &&
         alloc(reinterpret_cast<void**>(&st->d_part), sizeof(double) * 3 * kResBlocksPerProblem * problems) &&
         alloc(reinterpret_cast<void**>(&st->d_res), sizeof(double) * 4 * problems);
    ok = ok && cudaMallocHost(&st->h_map, sizeof(int) * problems) == cudaSuccess &&
         cudaMallocHost(&st->h_res, sizeof(double) * 4 * problems) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_state(st);
        set_error("ac_parareal_create: device allocation failed");
        return AC_ERR_NOMEM;
    }
    st->g.work = st->work;
    st->g.work_bytes = wb;
    st->g.packed = st->packed;
    if (pb) {
        rc = cnn_pack_weights(&st->g, nullptr);
        if (rc) { free_state(st); return rc; }
    }
    // U0[p][0] = u0[p]
    if (cudaMemcpy2D(st->Ua, fb * (num_slices + 1), u0, fb, fb, problems, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        set_error("ac_parareal_create: copy of u0 failed: %s", cudaGetErrorString(cudaGetLastError()));
        free_state(st);
        return AC_ERR_CUDA;
    }
    *out = st;
    return AC_OK;
}

extern "C" int parareal_iterate(ac_parareal* state, int* k_inout, double* rel_l2_out, double* max_abs_out,
                                acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(state && k_inout, "null argument");
    return iterate(state, k_inout, rel_l2_out, max_abs_out, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ac_parareal_set_active(ac_parareal* state, int problem, int active) {
    using namespace acpr;
    ACPR_CHECK_ARG(state && problem >= 0 && problem < state->problems, "bad problem index");
    state->active[problem] = active ? 1 : 0;
    if (active) state->synced[problem] = 0;
    return AC_OK;
}

extern "C" const void* ac_parareal_trajectory(const ac_parareal* state) {
    return state ? state->Ua : nullptr;
}

extern "C" int ac_parareal_copy_trajectory(const ac_parareal* state, void* dst, acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(state && dst, "null argument");
    const size_t bytes = state->esz * state->nn * size_t(state->problems) * (state->s + 1);
    ACPR_CUDA(cudaMemcpyAsync(dst, state->Ua, bytes, cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)));
    return AC_OK;
}

extern "C" int ac_parareal_solve(ac_parareal* state, double tol, int kmax, int* iters_out, double* rel_l2_out,
                                 acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(state && iters_out && rel_l2_out, "null argument");
    ACPR_CHECK_ARG(kmax >= 1, "kmax must be >= 1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int P = state->problems;
    std::vector<double> l2(P, 0.0), mx(P, 0.0);
    for (int p = 0; p < P; ++p) { iters_out[p] = 0; rel_l2_out[p] = 0.0; }
    int k = state->k_next;
    int rc = AC_OK;
    if (k == 0) {
        rc = iterate(state, &k, nullptr, nullptr, st);
        if (rc) return rc;
    }
    const int klim = kmax < state->s ? kmax : state->s;
    bool any = true;
    bool saw_nonfinite = false;
    while (k <= klim && any) {
        const int kk = k;
        rc = iterate(state, &k, l2.data(), mx.data(), st);
        // A non-finite increment means a diverging iterate beyond the exact
        // prefix; slices <= k stay fine-solver values, so keep iterating: the
        // loop still ends with the exact trajectory at k = s.
        if (rc == AC_ERR_NONFINITE) saw_nonfinite = true;
        else if (rc) return rc;
        any = false;
        for (int p = 0; p < P; ++p) {
            if (!state->active[p]) continue;
            iters_out[p] = kk;
            rel_l2_out[p] = l2[p];
            // converged on the tolerance, or exact because k reached s
            if (l2[p] < tol || kk == state->s) state->active[p] = 0;
            else any = true;
        }
    }
    if (any) {
        set_error("ac_parareal_solve: not converged within kmax = %d%s", kmax,
                  saw_nonfinite ? " (non-finite increments met)" : "");
        return AC_ERR_NOT_CONVERGED;
    }
    return AC_OK;
}

extern "C" int ac_parareal_reset(ac_parareal* state, const void* u0, acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(state && u0, "null argument");
    const size_t fb = state->esz * state->nn;
    ACPR_CUDA(cudaMemcpy2DAsync(state->Ua, fb * (state->s + 1), u0, fb, fb, state->problems,
                                cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)));
    state->active.assign(state->problems, 1);
    state->synced.assign(state->problems, 0);
    state->k_next = 0;
    return AC_OK;
}

extern "C" int ac_parareal_enable_timing(ac_parareal* state, int on) {
    using namespace acpr;
    ACPR_CHECK_ARG(state, "null state");
    if (on && !state->ev[0])
        for (cudaEvent_t& e : state->ev) ACPR_CUDA(cudaEventCreate(&e));
    state->timing = on != 0;
    return AC_OK;
}

extern "C" int ac_parareal_get_stats(const ac_parareal* state, ac_parareal_stats* out) {
    using namespace acpr;
    ACPR_CHECK_ARG(state && out, "null argument");
    *out = state->stats;
    return AC_OK;
}

extern "C" int ac_parareal_reset_stats(ac_parareal* state) {
    using namespace acpr;
    ACPR_CHECK_ARG(state, "null state");
    state->stats = ac_parareal_stats{};
    return AC_OK;
}

extern "C" void ac_parareal_destroy(ac_parareal* state) { acpr::free_state(state); }
