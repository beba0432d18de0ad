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
//   4. increment of Ub against Ua over slices 1..s, float64: the corrections
//      of steps 2 and 3 leave per-block partial sums of the slices they write,
//      one small kernel adds them up (no second pass over the trajectories)
// The frozen prefix Ub[0..k-2] already equals Ua[0..k-2] (both hold the exact
// fine values), so step 2 copies one slice only.  The summation order
// F + (G_new - G_old) keeps U^k_k bitwise equal to the fine result.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "acnn.cuh"
#include "cnn.cuh"
#include "common.cuh"

namespace acpr {

int fine_propagate_mapped(const ac_params* p, int groups, int per_group, int steps, const void* in,
                          long long in_gs, long long in_off, void* out, long long out_gs,
                          long long out_off, const int* map, cudaStream_t stream, void* big_ws,
                          size_t big_ws_bytes);
size_t fine_big_workspace_bytes(int n, int fields);
bool fine_big_supported(int n, int precision);
int fine_run_work(const ac_params* p, int count, const int4* work, const void* in, void* out, cudaStream_t stream);
int cn_run_work(const ac_params* p, int count, const int4* work, const void* in, void* out, double tol,
                int max_iters, cudaStream_t st);
bool cn_supported(int n, int precision);
bool fine_supported_internal(int n, int precision);
int fine_check_status(cudaStream_t st);

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

// ------------------------------------------- correction fused with the increment --
// The correction kernel also accumulates, for the slice it writes, the three
// sums of the convergence test against the previous iterate: sum (U - U_old)^2,
// sum U^2 and max |U - U_old|, per (problem, slice, block) in float64, so the
// increment needs no second pass over the trajectories.
//
// float32 fields: each thread accumulates without rounding error that
// matters, in float32 arithmetic (float64 arithmetic is scarce on this GPU):
// d = a - b is split exactly into s + e (Knuth's TwoSum), d^2 = s^2 + (2 s e
// + e^2) with s^2 split exactly by a fused multiply-add (Dekker's product),
// and the sums are carried as unevaluated float pairs (hi + lo); the exact
// max |d| is tracked as the pair (|s|, sign(s) e), compared
// lexicographically (rounding is monotone).  The pairs become float64 once
// per thread.  Relative error of the sums about 2^-44.
// (The _rn intrinsics are never contracted into fused multiply-adds, which
// the error-free transformations below rely on.)
__device__ __forceinline__ void acc_two_sum(float& hi, float& lo, float p, float t) {
    const float x = __fadd_rn(hi, p);
    const float bv = __fsub_rn(x, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(x, bv)), __fsub_rn(p, bv));
    hi = x;
    lo = __fadd_rn(lo, __fadd_rn(err, t));
}

struct IncAcc32 {
    float nh = 0.f, nl = 0.f, dh = 0.f, dl = 0.f, ms = 0.f, me = 0.f;
    bool bad = false;
    __device__ __forceinline__ void add(float a, float b) {
        const float s = __fsub_rn(a, b);
        const float bb = __fsub_rn(s, a);
        const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
        const float p = __fmul_rn(s, s);
        float t = fmaf(s, s, -p);
        t = fmaf(__fmul_rn(2.0f, s), e, t);
        t = fmaf(e, e, t);
        acc_two_sum(nh, nl, p, t);
        const float q = __fmul_rn(a, a);
        acc_two_sum(dh, dl, q, fmaf(a, a, -q));
        const float as = fabsf(s), ae = s < 0.f ? -e : e;
        if (as > ms || (as == ms && ae > me)) { ms = as; me = ae; }
        if (!(s - s == 0.f)) bad = true;  // NaN or Inf
    }
    __device__ __forceinline__ void result(double& num, double& den, double& mx) const {
        num = double(nh) + double(nl);
        den = double(dh) + double(dl);
        mx = bad ? __longlong_as_double(0x7ff8000000000000LL) : double(ms) + double(me);
    }
};

struct IncAcc64 {
    double num = 0.0, den = 0.0, mx = 0.0;
    __device__ __forceinline__ void add(double a, double b) {
        const double d = a - b;
        num += d * d;
        den += a * a;
        mx = fmax(mx, fabs(d));
        if (!(d == d)) mx = d;
    }
    __device__ __forceinline__ void result(double& n, double& d, double& m) const { n = num; d = den; m = mx; }
};

template <typename T> struct IncAccT;
template <> struct IncAccT<float> { using type = IncAcc32; };
template <> struct IncAccT<double> { using type = IncAcc64; };

// Block sum of (num, den) and max (NaN kept) in a fixed order; thread 0 writes.
__device__ __forceinline__ void block_partials(double num, double den, double mx, double* out) {
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
        out[0] = n0; out[1] = d0; out[2] = m0;
    }
}

// Ub[n+1] = Fres[n] + (g - Gold[n]) (and Gold[n] = g; if g is NULL, Gold[n] is
// used in its place: the exact slice) for batch entry blockIdx.y, plus the
// block's increment partials of slice n + 1 against Ua into
// part[((p s + n) NB + blockIdx.x) * 3].
template <typename T>
__global__ void __launch_bounds__(kResThreads)
correct_inc_kernel(T* __restrict__ Ub, const T* __restrict__ Ua, T* __restrict__ Gold, const T* __restrict__ Fres,
                   const T* __restrict__ g, int slice, int s, long long nn, const int* __restrict__ map,
                   double* __restrict__ part) {
    const int b = blockIdx.y;
    const long long p = map ? map[b] : b;
    T* go = Gold + (p * s + slice) * nn;
    const T* fr = Fres + (p * s + slice) * nn;
    const T* gb = g ? g + (long long)b * nn : nullptr;
    T* ub = Ub + (p * (s + 1) + slice + 1) * nn;
    const T* ua = Ua + (p * (s + 1) + slice + 1) * nn;
    typename IncAccT<T>::type acc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn;
         i += (long long)gridDim.x * blockDim.x) {
        const T gold = go[i];
        const T gn = gb ? gb[i] : gold;
        const T u = fr[i] + (gn - gold);
        ub[i] = u;
        if (gb) go[i] = gn;
        acc.add(u, ua[i]);
    }
    double num, den, mx;
    acc.result(num, den, mx);
    block_partials(num, den, mx, part + ((p * s + slice) * gridDim.x + blockIdx.x) * 3);
}

// Increment of iteration k for the mapped problems: slices k..s from this
// iteration's partials, slices 1..k-1 (frozen: U^k_j = U^{k-1}_j) contribute
// only sum U^2, kept from the iteration that last wrote them.  One warp per
// problem; lane t takes the slices j = t + 1, t + 33, ... in order, then a
// fixed shuffle tree: deterministic.  res[4 i + 0..3] = rel_l2, max, num, den.
__global__ void increment_fused_finish_kernel(const double* __restrict__ part, int nb, int s, int k,
                                              const int* __restrict__ map, int problems, double* __restrict__ res) {
    const int i = blockIdx.x;
    if (i >= problems) return;
    const long long p = map ? map[i] : i;
    const int lane = threadIdx.x;
    double num = 0.0, den = 0.0, mx = 0.0;
    for (int j = 1 + lane; j <= s; j += 32) {
        const double* q = part + (p * s + (j - 1)) * (long long)nb * 3;
        for (int bl = 0; bl < nb; ++bl) {
            den += q[bl * 3 + 1];
            if (j >= k) {
                num += q[bl * 3];
                mx = (q[bl * 3 + 2] != q[bl * 3 + 2]) ? q[bl * 3 + 2] : fmax(mx, q[bl * 3 + 2]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
        const double m2 = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = (m2 != m2) ? m2 : fmax(mx, m2);
    }
    if (lane == 0) {
        res[4 * i + 0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
        res[4 * i + 1] = mx;
        res[4 * i + 2] = num;
        res[4 * i + 3] = den;
    }
}

// dst field (map[b] * dst_ps + dst_slice) = src field (map[b] * src_ps + src_slice)
template <typename T>
__global__ void copy_slice_kernel(T* __restrict__ dst, const T* __restrict__ src, int dst_slice, int src_slice,
                                  long long dst_ps, long long src_ps, long long nn, int batch,
                                  const int* __restrict__ map) {
    const long long total = nn * batch;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = int(idx / nn);
        const long long i = idx % nn;
        const long long p = map ? map[b] : b;
        dst[(p * dst_ps + dst_slice) * nn + i] = src[(p * src_ps + src_slice) * nn + i];
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
// Problems of one handle share ac_params and the coarse net; each has its own
// slice count s_p and steps per slice c_p.  Arrays are laid out with the
// largest slice count s; slices past s_p are never written and stay zero in
// both trajectories, so the increments over slices 1..s are those over 1..s_p.
// Active problems are kept in order of decreasing s_p, so the problems still
// sweeping at slice n are a prefix of that list.
struct GraphKey {
    int k;
    std::vector<int> active;
    bool swapped;  // the trajectory buffers' roles (a graph holds their addresses)
    bool operator<(const GraphKey& o) const {
        if (k != o.k) return k < o.k;
        if (swapped != o.swapped) return swapped < o.swapped;
        return active < o.active;
    }
};

struct ac_parareal {
    ac_params p;
    cnn_desc g;
    int problems = 0, s = 0;
    std::vector<int> sp, cp;    // per-problem slices and steps per slice
    bool uniform = true;        // every problem has the same slices and steps
    size_t esz = 0;
    long long nn = 0;
    void* Ua = nullptr;
    void* Ub = nullptr;
    void* Ua0 = nullptr;    // Ua as allocated (Ua and Ub swap every iteration)
    void* big_ws = nullptr; // workspace of the two-pass fine path (n = 1024)
    size_t big_ws_bytes = 0;
    void* Gold = nullptr;
    void* Fres = nullptr;
    void* gtmp = nullptr;   // [problems][nn] coarse output of one sweep step
    void* work = nullptr;   // conv activations
    void* packed = nullptr; // bf16 weights
    int* d_map = nullptr;   // active problems, decreasing s_p
    int* h_map = nullptr;   // pinned
    int4* d_fw = nullptr;   // fine work list
    int4* h_fw = nullptr;   // pinned
    double* d_part = nullptr;
    double* d_res = nullptr;
    double* h_res = nullptr;  // pinned [problems][4]
    std::vector<char> active;
    std::vector<char> synced;  // inactive problem whose trajectory is in both buffers
    int k_next = 0;
    int m_launched = 0;        // active count of the iteration in flight
    cudaStream_t stream_launched = nullptr;
    bool timing = false;
    bool graphs = false;
    bool has_cnn = false;            // created with a conv-stack G
    const acnn_net* acnn = nullptr;  // the ResBlock ACNN as G instead of the conv stack
    void* acnn_work = nullptr;
    size_t acnn_work_bytes = 0;
    int g_sub = 1;             // coarse composition: G applied g_sub times per slice
    void* gsub[2] = {nullptr, nullptr};  // [problems][nn] each: intermediate G applications
    int fine_scheme = 0;       // 0: stabilised semi-implicit step, 1: Crank-Nicolson + Picard
    double cn_tol = 1e-6;
    int cn_max_iters = 50;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t done = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream the graphs are captured on
    std::map<GraphKey, std::pair<cudaGraphExec_t, int>> graph_cache;  // exec, kernel nodes
    ac_parareal_stats stats{};
};

namespace acpr {

static void free_state(ac_parareal* st) {
    if (!st) return;
    for (void* ptr : {st->Ua, st->Ub, st->Gold, st->Fres, st->gtmp, st->work, st->packed, st->gsub[0], st->gsub[1],
                      st->big_ws,
                      st->acnn_work,
                      static_cast<void*>(st->d_map), static_cast<void*>(st->d_fw), static_cast<void*>(st->d_part),
                      static_cast<void*>(st->d_res)})
        if (ptr) cudaFree(ptr);
    if (st->h_map) cudaFreeHost(st->h_map);
    if (st->h_fw) cudaFreeHost(st->h_fw);
    if (st->h_res) cudaFreeHost(st->h_res);
    for (cudaEvent_t e : st->ev)
        if (e) cudaEventDestroy(e);
    if (st->done) cudaEventDestroy(st->done);
    for (auto& kv : st->graph_cache) cudaGraphExecDestroy(kv.second.first);
    if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
    delete st;
}

// One coarse evaluation of the sweep: G, or G composed g_sub times (the
// recursive composition of the remark after Algorithm 2: a coarse step that
// covers the slice in g_sub sub-steps).  The intermediate applications go
// through compact [mn][nn] buffers; the last one writes the mapped output.
static int coarse_once(ac_parareal* st, int mn, const void* in, long long in_bs, const int* in_map, void* out,
                       long long out_bs, const int* out_map, cudaStream_t stream) {
    if (st->acnn)
        return acnn_forward_mapped(st->acnn, st->p.n, mn, in, in_bs, in_map, out, out_bs, out_map, st->acnn_work,
                                   st->acnn_work_bytes, stream);
    ACPR_CHECK_ARG(st->has_cnn, "no coarse propagator: the handle was created without one and no ACNN is set");
    return coarse_step_mapped(&st->g, st->p.n, mn, in, in_bs, in_map, out, out_bs, out_map, stream);
}

static int coarse_apply(ac_parareal* st, int mn, const void* in, long long in_bs, const int* in_map, void* out,
                        long long out_bs, const int* out_map, cudaStream_t stream) {
    const void* cur = in;
    long long cur_bs = in_bs;
    const int* cur_map = in_map;
    for (int i = 0; i + 1 < st->g_sub; ++i) {
        void* dst = st->gsub[i & 1];
        int rc = coarse_once(st, mn, cur, cur_bs, cur_map, dst, st->nn, nullptr, stream);
        if (rc) return rc;
        cur = dst;
        cur_bs = st->nn;
        cur_map = nullptr;
    }
    return coarse_once(st, mn, cur, cur_bs, cur_map, out, out_bs, out_map, stream);
}

static unsigned grid_for(long long total, int threads) {
    const long long want = (total + threads - 1) / threads;
    return unsigned(want < 152 * 16 ? want : 152 * 16);
}

// Blocks per problem of the fused correction (at most 1024 elements per
// block, at most kIncBlocks blocks).
constexpr int kIncBlocks = 64;
static int inc_blocks(long long nn) {
    const long long want = (nn + 1023) / 1024;
    return int(want < kIncBlocks ? want : kIncBlocks);
}

template <typename T>
static int launch_correct(ac_parareal* st, void* Ub, int slice, const void* g, int m, cudaStream_t stream) {
    // Ub is U^k; the other trajectory buffer holds U^{k-1}
    const void* Uold = Ub == st->Ub ? st->Ua : st->Ub;
    correct_inc_kernel<T><<<dim3(unsigned(inc_blocks(st->nn)), unsigned(m)), kResThreads, 0, stream>>>(
        static_cast<T*>(Ub), static_cast<const T*>(Uold), static_cast<T*>(st->Gold),
        static_cast<const T*>(st->Fres), static_cast<const T*>(g), slice, st->s, st->nn, st->d_map, st->d_part);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

static int correct(ac_parareal* st, void* Ub, int slice, const void* g, int m, cudaStream_t stream) {
    if (st->p.precision == AC_F64) return launch_correct<double>(st, Ub, slice, g, m, stream);
    return launch_correct<float>(st, Ub, slice, g, m, stream);
}

static int copy_slice(ac_parareal* st, void* dst, const void* src, int dst_slice, int src_slice, long long dst_ps,
                      long long src_ps, int m, cudaStream_t stream) {
    if (st->p.precision == AC_F64)
        copy_slice_kernel<double><<<grid_for(st->nn * m, 256), 256, 0, stream>>>(
            static_cast<double*>(dst), static_cast<const double*>(src), dst_slice, src_slice, dst_ps, src_ps, st->nn,
            m, st->d_map);
    else
        copy_slice_kernel<float><<<grid_for(st->nn * m, 256), 256, 0, stream>>>(
            static_cast<float*>(dst), static_cast<const float*>(src), dst_slice, src_slice, dst_ps, src_ps, st->nn, m,
            st->d_map);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

// Number of active problems (a prefix of h_map) whose slice count exceeds n.
static int sweeping(const ac_parareal* st, int m, int n) {
    int c = 0;
    while (c < m && st->sp[st->h_map[c]] > n) ++c;
    return c;
}

// Host-side lists of iteration k: the active problems (decreasing s_p) and
// the fine work items (decreasing steps, the longest first).  Returns m.
static int build_lists(ac_parareal* st, int k, int* nwork) {
    std::vector<int> act;
    for (int p = 0; p < st->problems; ++p)
        if (st->active[p]) act.push_back(p);
    std::stable_sort(act.begin(), act.end(), [&](int a, int b) { return st->sp[a] > st->sp[b]; });
    for (size_t i = 0; i < act.size(); ++i) st->h_map[i] = act[i];
    int w = 0;
    if (k >= 1) {
        std::vector<int> byc(act);
        std::stable_sort(byc.begin(), byc.end(), [&](int a, int b) { return st->cp[a] > st->cp[b]; });
        for (int p : byc)
            for (int n = k - 1; n < st->sp[p]; ++n)
                st->h_fw[w++] = make_int4(p * (st->s + 1) + n, p * st->s + n, st->cp[p], 0);
    }
    *nwork = w;
    return int(act.size());
}

// All device work of iteration k (what a graph captures).
static int enqueue(ac_parareal* st, int k, int m, int nwork, cudaStream_t stream) {
    const long long nn = st->nn;
    const int s = st->s;
    const size_t fb = st->esz * nn;
    const bool tm = st->timing;
    int rc;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (tm) ACPR_CUDA(cudaStreamIsCapturing(stream, &cap));
    auto mark = [&](int i) -> int {
        // inside a capture only an "external" record becomes an event node
        if (tm) ACPR_CUDA(cudaEventRecordWithFlags(st->ev[i], stream,
                                                   cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                                        : cudaEventRecordDefault));
        return AC_OK;
    };
    if (k == 0) {
        // U^0_0 = u0 (already in Ua[0]); sequential coarse sweep U^0_{n+1} = G(U^0_n)
        if ((rc = mark(1))) return rc;
        for (int n = 0; n < s; ++n) {
            const int mn = sweeping(st, m, n);
            if (!mn) break;
            rc = coarse_apply(st, mn, static_cast<char*>(st->Ua) + n * fb, nn * (s + 1),
                                    st->d_map, static_cast<char*>(st->Gold) + n * fb, nn * s, st->d_map, stream);
            if (rc) return rc;
            if ((rc = copy_slice(st, st->Ua, st->Gold, n + 1, n, s + 1, s, mn, stream))) return rc;
        }
        return mark(2);
    }
    // 1. fine solves of slices k-1 .. s_p-1 of every active problem (one launch)
    if ((rc = mark(0))) return rc;
    if (st->uniform && st->p.n >= 1024) {
        // large fields: the two-pass path runs uniform launches only
        rc = fine_propagate_mapped(&st->p, m, s - k + 1, st->cp[0], st->Ua, s + 1, k - 1, st->Fres, s, k - 1,
                                   st->d_map, stream, st->big_ws, st->big_ws_bytes);
    } else if (st->fine_scheme == 1) {
        rc = cn_run_work(&st->p, nwork, st->d_fw, st->Ua, st->Fres, st->cn_tol, st->cn_max_iters, stream);
    } else {
        rc = fine_run_work(&st->p, nwork, st->d_fw, st->Ua, st->Fres, stream);
    }
    if (rc) return rc;
    if ((rc = mark(1))) return rc;
    // 2. newest frozen slice and the exact slice k
    if ((rc = copy_slice(st, st->Ub, st->Ua, k - 1, k - 1, s + 1, s + 1, m, stream))) return rc;
    if ((rc = correct(st, st->Ub, k - 1, nullptr, m, stream))) return rc;
    // 3. sequential correction sweep
    for (int n = k; n < s; ++n) {
        const int mn = sweeping(st, m, n);
        if (!mn) break;
        rc = coarse_apply(st, mn, static_cast<char*>(st->Ub) + n * fb, nn * (s + 1), st->d_map, st->gtmp, nn,
                          nullptr, stream);
        if (rc) return rc;
        if ((rc = correct(st, st->Ub, n, st->gtmp, mn, stream))) return rc;
    }
    if ((rc = mark(2))) return rc;
    // 4. increments over slices 1..s from the partials of the corrections
    increment_fused_finish_kernel<<<m, 32, 0, stream>>>(st->d_part, inc_blocks(nn), s, k, st->d_map, m, st->d_res);
    ACPR_LAUNCH_CHECK();
    return mark(3);
}

static void account(ac_parareal* st, int k, int m, int nwork) {
    if (k >= 1) {
        st->stats.fine_launches += 1;
        for (int i = 0; i < nwork; ++i) st->stats.fine_cell_steps += (long long)st->h_fw[i].z * st->nn;
    }
    for (int n = k; n < st->s; ++n) {
        const int mn = sweeping(st, m, n);
        if (!mn) break;
        st->stats.coarse_calls += st->g_sub;
        st->stats.coarse_cells += (long long)mn * st->nn * st->g_sub;
    }
}

// Launch iteration k (asynchronous); finish() completes it.
static int launch(ac_parareal* st, int k, cudaStream_t stream) {
    ACPR_CHECK_ARG(k == st->k_next, "iteration %d requested, state is at %d", k, st->k_next);
    ACPR_CHECK_ARG(k <= st->s, "k = %d exceeds the slice count %d", k, st->s);
    const size_t fb = st->esz * st->nn;
    int nwork = 0;
    const int m = build_lists(st, k, &nwork);
    st->m_launched = m;
    st->stream_launched = stream;
    if (k >= 1) {
        // an inactive problem keeps its last trajectory in both buffers, so
        // that the buffer swap never exposes a stale one
        for (int p = 0; p < st->problems; ++p) {
            if (st->active[p] || st->synced[p]) continue;
            ACPR_CUDA(cudaMemcpyAsync(static_cast<char*>(st->Ub) + size_t(p) * (st->s + 1) * fb,
                                      static_cast<char*>(st->Ua) + size_t(p) * (st->s + 1) * fb, fb * (st->s + 1),
                                      cudaMemcpyDeviceToDevice, stream));
            st->synced[p] = 1;
        }
    }
    if (m == 0) return AC_OK;
    ACPR_CUDA(cudaMemcpyAsync(st->d_map, st->h_map, sizeof(int) * m, cudaMemcpyHostToDevice, stream));
    if (nwork) ACPR_CUDA(cudaMemcpyAsync(st->d_fw, st->h_fw, sizeof(int4) * nwork, cudaMemcpyHostToDevice, stream));
    int rc;
    if (st->graphs) {
        GraphKey key{k, std::vector<int>(st->h_map, st->h_map + m), st->Ua != st->Ua0};
        auto it = st->graph_cache.find(key);
        if (it == st->graph_cache.end()) {
            // capture on a private stream (the caller's may be the legacy
            // default stream, which cannot be captured); nothing runs here
            if (!st->cap_stream) ACPR_CUDA(cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            ACPR_CUDA(cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeRelaxed));
            rc = enqueue(st, k, m, nwork, st->cap_stream);
            cudaError_t ec = cudaStreamEndCapture(st->cap_stream, &graph);
            if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
            ACPR_CUDA(ec);
            // kernel nodes, so that replays count towards ac_launch_count()
            size_t nodes = 0;
            int kernels = 0;
            if (cudaGraphGetNodes(graph, nullptr, &nodes) == cudaSuccess && nodes) {
                std::vector<cudaGraphNode_t> list(nodes);
                if (cudaGraphGetNodes(graph, list.data(), &nodes) == cudaSuccess)
                    for (size_t i = 0; i < nodes; ++i) {
                        cudaGraphNodeType t;
                        if (cudaGraphNodeGetType(list[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
                    }
            }
            cudaGraphExec_t exec = nullptr;
            cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            ACPR_CUDA(ei);
            // capture counted the kernels as launches already; undo that
            count_launch_add(-kernels);
            it = st->graph_cache.emplace(key, std::make_pair(exec, kernels)).first;
        }
        ACPR_CUDA(cudaGraphLaunch(it->second.first, stream));
        count_launch_add(it->second.second);
    } else {
        if ((rc = enqueue(st, k, m, nwork, stream))) return rc;
    }
    account(st, k, m, nwork);
    if (k >= 1)
        ACPR_CUDA(cudaMemcpyAsync(st->h_res, st->d_res, sizeof(double) * 4 * m, cudaMemcpyDeviceToHost, stream));
    ACPR_CUDA(cudaEventRecord(st->done, stream));
    return AC_OK;
}

static int finish(ac_parareal* st, int k, double* l2_out, double* mx_out) {
    const int m = st->m_launched;
    if (m) ACPR_CUDA(cudaEventSynchronize(st->done));
    int rc = st->work ? conv_check_status(conv_status(st->work), st->stream_launched) : AC_OK;
    if (!rc) rc = fine_check_status(st->stream_launched);
    if (rc) return rc;
    if (st->timing && m) {
        float a = 0.f, b = 0.f, c = 0.f;
        if (k == 0) {
            ACPR_CUDA(cudaEventElapsedTime(&b, st->ev[1], st->ev[2]));
        } else {
            ACPR_CUDA(cudaEventElapsedTime(&a, st->ev[0], st->ev[1]));
            ACPR_CUDA(cudaEventElapsedTime(&b, st->ev[1], st->ev[2]));
            ACPR_CUDA(cudaEventElapsedTime(&c, st->ev[2], st->ev[3]));
        }
        st->stats.fine_ms += a;
        st->stats.coarse_ms += b;
        st->stats.increment_ms += c;
    }
    st->k_next = k + 1;
    if (k == 0) return AC_OK;
    st->stats.iterations += 1;
    bool nonfinite = false;
    for (int i = 0; i < m; ++i) {
        const int p = st->h_map[i];
        if (l2_out) l2_out[p] = st->h_res[4 * i];
        if (mx_out) mx_out[p] = st->h_res[4 * i + 1];
        if (!std::isfinite(st->h_res[4 * i]) || !std::isfinite(st->h_res[4 * i + 1])) nonfinite = true;
    }
    std::swap(st->Ua, st->Ub);
    if (nonfinite) {
        set_error("parareal_iterate: non-finite increment at k = %d", k);
        return AC_ERR_NONFINITE;
    }
    return AC_OK;
}

static int iterate(ac_parareal* st, int* k_inout, double* l2_out, double* mx_out, cudaStream_t stream) {
    const int k = *k_inout;
    int rc = launch(st, k, stream);
    if (rc) return rc;
    rc = finish(st, k, l2_out, mx_out);
    *k_inout = st->k_next;
    return rc;
}

static int create(const ac_params* params, const cnn_desc* coarse, int problems, const int* slices,
                  const int* steps, const void* u0, ac_parareal** out) {
    ACPR_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    ACPR_CHECK_ARG(params && u0 && slices && steps, "null argument");
    ACPR_CHECK_ARG(problems >= 1, "need at least one problem");
    int smax = 0;
    for (int p = 0; p < problems; ++p) {
        ACPR_CHECK_ARG(slices[p] >= 1 && steps[p] >= 0, "problem %d: bad slice count or steps", p);
        smax = std::max(smax, slices[p]);
    }
    int rc = AC_OK;
    if (coarse) {
        ACPR_CHECK_ARG(coarse->precision == params->precision, "coarse and fine precision differ");
        if ((rc = check_cnn(coarse))) return rc;
    }
    if (!fine_supported_internal(params->n, params->precision)) {
        set_error("ac_parareal_create: n=%d not supported", params->n);
        return AC_ERR_UNSUPPORTED;
    }
    ac_parareal* st = new ac_parareal();
    st->p = *params;
    if (coarse) st->g = *coarse;
    st->has_cnn = coarse != nullptr;
    st->problems = problems;
    st->s = smax;
    st->sp.assign(slices, slices + problems);
    st->cp.assign(steps, steps + problems);
    for (int p = 1; p < problems; ++p)
        if (slices[p] != slices[0] || steps[p] != steps[0]) st->uniform = false;
    if (params->n >= 1024 && !st->uniform) {
        delete st;
        set_error("ac_parareal: n=%d needs equal slice counts and steps for all problems", params->n);
        return AC_ERR_UNSUPPORTED;
    }
    st->esz = elem_size(params->precision);
    st->nn = (long long)params->n * params->n;
    st->active.assign(problems, 1);
    st->synced.assign(problems, 0);
    const size_t fb = st->esz * st->nn;
    const size_t traj = fb * size_t(problems) * (smax + 1);
    const size_t slc = fb * size_t(problems) * smax;
    auto alloc = [&](void** p, size_t bytes) -> bool { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = alloc(&st->Ua, traj) && alloc(&st->Ub, traj) && alloc(&st->Gold, slc) && alloc(&st->Fres, slc) &&
              alloc(&st->gtmp, fb * problems);
    const size_t wb = coarse ? work_bytes_for(coarse, params->n, problems) : 0;
    if (wb) ok = ok && alloc(&st->work, wb);
    const size_t pb = coarse ? cnn_packed_bytes(coarse) : 0;
    if (ok && pb) ok = alloc(&st->packed, pb);
    if (ok && fine_big_supported(params->n, params->precision)) {
        st->big_ws_bytes = fine_big_workspace_bytes(params->n, problems * smax);
        ok = alloc(&st->big_ws, st->big_ws_bytes);
    }
    ok = ok && alloc(reinterpret_cast<void**>(&st->d_map), sizeof(int) * problems) &&
         alloc(reinterpret_cast<void**>(&st->d_fw), sizeof(int4) * size_t(problems) * smax) &&
         alloc(reinterpret_cast<void**>(&st->d_part), sizeof(double) * 3 * inc_blocks(st->nn) * problems * size_t(smax)) &&
         alloc(reinterpret_cast<void**>(&st->d_res), sizeof(double) * 4 * problems);
    ok = ok && cudaMallocHost(&st->h_map, sizeof(int) * problems) == cudaSuccess &&
         cudaMallocHost(&st->h_fw, sizeof(int4) * size_t(problems) * smax) == cudaSuccess &&
         cudaMallocHost(&st->h_res, sizeof(double) * 4 * problems) == cudaSuccess &&
         cudaEventCreateWithFlags(&st->done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_state(st);
        set_error("ac_parareal_create: device allocation failed");
        return AC_ERR_NOMEM;
    }
    st->Ua0 = st->Ua;
    st->g.work = st->work;
    st->g.work_bytes = wb;
    st->g.packed = st->packed;
    if (pb) {
        rc = cnn_pack_weights(&st->g, nullptr);
        if (rc) { free_state(st); return rc; }
    }
    // zero trajectories (slices past s_p stay zero), then U[p][0] = u0[p];
    // the conv workspace's status header starts at zero
    if ((st->work && cudaMemset(st->work, 0, kConvHeader) != cudaSuccess) ||
        cudaMemset(st->d_part, 0, sizeof(double) * 3 * inc_blocks(st->nn) * problems * size_t(smax)) != cudaSuccess ||
        cudaMemset(st->Ua, 0, traj) != cudaSuccess || cudaMemset(st->Ub, 0, traj) != cudaSuccess ||
        cudaMemcpy2D(st->Ua, fb * (smax + 1), u0, fb, fb, problems, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        set_error("ac_parareal_create: initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
        free_state(st);
        return AC_ERR_CUDA;
    }
    *out = st;
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

extern "C" int ac_parareal_create(const ac_params* params, const cnn_desc* coarse, int problems, int num_slices,
                                  int steps_per_slice, const void* u0, ac_parareal** out) {
    using namespace acpr;
    ACPR_CHECK_ARG(problems >= 1 && problems < (1 << 24), "bad problem count");
    std::vector<int> sl(problems, num_slices), st(problems, steps_per_slice);
    return create(params, coarse, problems, sl.data(), st.data(), u0, out);
}

extern "C" int ac_parareal_create_uneven(const ac_params* params, const cnn_desc* coarse, int problems,
                                         const int* num_slices, const int* steps_per_slice, const void* u0,
                                         ac_parareal** out) {
    return acpr::create(params, coarse, problems, num_slices, steps_per_slice, u0, out);
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

// Iterations of several handles at once: each iteration is launched on every
// handle's stream before any is waited for, so different grid sizes overlap.
static int solve_many(ac_parareal* const* states, int count, const cudaStream_t* streams, double tol, int kmax,
                      int* iters_out, double* rel_l2_out) {
    using namespace acpr;
    std::vector<std::vector<double>> l2(count), mx(count);
    std::vector<int> base(count, 0);
    int total = 0;
    for (int h = 0; h < count; ++h) {
        ACPR_CHECK_ARG(states[h], "null state %d", h);
        base[h] = total;
        total += states[h]->problems;
        l2[h].assign(states[h]->problems, 0.0);
        mx[h].assign(states[h]->problems, 0.0);
    }
    for (int i = 0; i < total; ++i) { iters_out[i] = 0; rel_l2_out[i] = 0.0; }
    int rc;
    for (int h = 0; h < count; ++h)
        if (states[h]->k_next == 0 && (rc = launch(states[h], 0, streams[h]))) return rc;
    for (int h = 0; h < count; ++h)
        if (states[h]->k_next == 0 && (rc = finish(states[h], 0, nullptr, nullptr))) return rc;
    std::vector<char> busy(count, 1);
    bool any = true, saw_nonfinite = false;
    while (any) {
        any = false;
        std::vector<int> kk(count, -1);
        for (int h = 0; h < count; ++h) {
            ac_parareal* st = states[h];
            const int klim = std::min(kmax, st->s);
            bool act = false;
            for (int p = 0; p < st->problems; ++p) act = act || st->active[p];
            if (!busy[h] || !act || st->k_next > klim) { busy[h] = 0; continue; }
            kk[h] = st->k_next;
            if ((rc = launch(st, kk[h], streams[h]))) return rc;
        }
        for (int h = 0; h < count; ++h) {
            if (kk[h] < 0) continue;
            ac_parareal* st = states[h];
            rc = finish(st, kk[h], l2[h].data(), mx[h].data());
            if (rc == AC_ERR_NONFINITE) saw_nonfinite = true;
            else if (rc) return rc;
            for (int p = 0; p < st->problems; ++p) {
                if (!st->active[p]) continue;
                iters_out[base[h] + p] = kk[h];
                rel_l2_out[base[h] + p] = l2[h][p];
                // converged on the tolerance, or exact because k reached s_p
                if (l2[h][p] < tol || kk[h] >= st->sp[p]) st->active[p] = 0;
                else any = true;
            }
        }
        bool left = false;
        for (int h = 0; h < count; ++h) {
            if (kk[h] < 0) continue;
            const int klim = std::min(kmax, states[h]->s);
            for (int p = 0; p < states[h]->problems; ++p)
                if (states[h]->active[p] && states[h]->k_next <= klim) left = true;
        }
        any = left;
    }
    for (int h = 0; h < count; ++h)
        for (int p = 0; p < states[h]->problems; ++p)
            if (states[h]->active[p]) {
                set_error("ac_parareal_solve: not converged within kmax = %d%s", kmax,
                          saw_nonfinite ? " (non-finite increments met)" : "");
                return AC_ERR_NOT_CONVERGED;
            }
    return AC_OK;
}

extern "C" int ac_parareal_solve(ac_parareal* state, double tol, int kmax, int* iters_out, double* rel_l2_out,
                                 acpr_stream stream) {
    using namespace acpr;
    ACPR_CHECK_ARG(state && iters_out && rel_l2_out, "null argument");
    ACPR_CHECK_ARG(kmax >= 1, "kmax must be >= 1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return solve_many(&state, 1, &st, tol, kmax, iters_out, rel_l2_out);
}

extern "C" int ac_parareal_solve_many(ac_parareal* const* states, int count, const acpr_stream* streams, double tol,
                                      int kmax, int* iters_out, double* rel_l2_out) {
    using namespace acpr;
    ACPR_CHECK_ARG(states && streams && iters_out && rel_l2_out && count >= 1, "null argument");
    ACPR_CHECK_ARG(kmax >= 1, "kmax must be >= 1");
    std::vector<cudaStream_t> sv(count);
    for (int h = 0; h < count; ++h) sv[h] = reinterpret_cast<cudaStream_t>(streams[h]);
    return solve_many(states, count, sv.data(), tol, kmax, iters_out, rel_l2_out);
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
    if (bool(on) != state->timing) {
        for (auto& kv : state->graph_cache) cudaGraphExecDestroy(kv.second.first);
        state->graph_cache.clear();  // captured graphs hold (or lack) the timing events
    }
    state->timing = on != 0;
    return AC_OK;
}

extern "C" int ac_parareal_enable_graphs(ac_parareal* state, int on) {
    using namespace acpr;
    ACPR_CHECK_ARG(state, "null state");
    state->graphs = on != 0;
    return AC_OK;
}

extern "C" int ac_parareal_set_coarse_acnn(ac_parareal* state, const acnn_net* net) {
    using namespace acpr;
    ACPR_CHECK_ARG(state, "null state");
    if (net) {
        ACPR_CHECK_ARG(acnn_precision(net) == state->p.precision, "ACNN precision differs from the handle's");
        const size_t need = acnn_work_bytes(net, state->p.n, state->problems);
        if (!need) {
            set_error("ac_parareal_set_coarse_acnn: n=%d not supported by the ACNN", state->p.n);
            return AC_ERR_UNSUPPORTED;
        }
        if (need > state->acnn_work_bytes) {
            if (state->acnn_work) cudaFree(state->acnn_work);
            state->acnn_work = nullptr;
            state->acnn_work_bytes = 0;
            ACPR_CUDA(cudaMalloc(&state->acnn_work, need));
            state->acnn_work_bytes = need;
        }
    }
    state->acnn = net;
    for (auto& kv : state->graph_cache) cudaGraphExecDestroy(kv.second.first);
    state->graph_cache.clear();
    return AC_OK;
}

extern "C" int ac_parareal_set_coarse_substeps(ac_parareal* state, int substeps) {
    using namespace acpr;
    ACPR_CHECK_ARG(state, "null state");
    ACPR_CHECK_ARG(substeps >= 1 && substeps <= 64, "coarse substeps must be 1..64 (got %d)", substeps);
    if (substeps > 1 && !state->gsub[0]) {
        const size_t bytes = state->esz * size_t(state->nn) * state->problems;
        ACPR_CUDA(cudaMalloc(&state->gsub[0], bytes));
        ACPR_CUDA(cudaMalloc(&state->gsub[1], bytes));
    }
    state->g_sub = substeps;
    for (auto& kv : state->graph_cache) cudaGraphExecDestroy(kv.second.first);
    state->graph_cache.clear();
    return AC_OK;
}

extern "C" int ac_parareal_set_fine_scheme(ac_parareal* state, int scheme, double tol, int max_iters) {
    using namespace acpr;
    ACPR_CHECK_ARG(state, "null state");
    ACPR_CHECK_ARG(scheme == 0 || scheme == 1, "fine scheme must be 0 (stabilised) or 1 (Crank-Nicolson)");
    if (scheme == 1) {
        ACPR_CHECK_ARG(tol >= 0 && max_iters >= 1, "need tol >= 0 and max_iters >= 1");
        if (!cn_supported(state->p.n, state->p.precision)) {
            set_error("Crank-Nicolson fine scheme not built for n=%d, precision %d", state->p.n, state->p.precision);
            return AC_ERR_UNSUPPORTED;
        }
        state->cn_tol = tol;
        state->cn_max_iters = max_iters;
    }
    state->fine_scheme = scheme;
    // captured iterations hold the previous scheme's launches
    for (auto& kv : state->graph_cache) cudaGraphExecDestroy(kv.second.first);
    state->graph_cache.clear();
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
