// energy.cu -- discrete energy, its gradient, and the gradient of the energy
// after `steps` fine steps with respect to the initial field (adjoint method
// with checkpointing).
//
// E_h(u) = h^2 sum_{ij} [ eps^2/2 (|D+x u|^2 + |D+y u|^2) + (u^2 - 1)^2 / 4 ]
// (the energy of Sec. 2, Eq. energy, with forward differences, consistent with
// the 5-point Laplacian: dE_h/du = h^2 (-eps^2 Lap_h u - f(u))).
// d E_h(u^M) / d u^0: forward pass storing a checkpoint every K steps, then per
// segment (last first) a recomputation of its states followed by the adjoint
// steps through them (ac_fine_adjoint), starting from dE_h/du at u^M.
#include "common.cuh"

namespace acpr {

int fine_run(const ac_params* p, int groups, int per_group, int steps, const void* in, long long in_gs,
             long long in_off, void* out, long long out_gs, long long out_off, const int* map, int adjoint,
             const void* states, void* traj, cudaStream_t stream, void* big_ws = nullptr, size_t big_ws_bytes = 0);

constexpr int kEnergyThreads = 1024;

// One block per field, float64 accumulation in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
energy_kernel(const T* __restrict__ u, int n, double h, double eps, double* __restrict__ e) {
    const long long nn = (long long)n * n;
    const T* f = u + blockIdx.x * nn;
    double s = 0.0;
    for (long long idx = threadIdx.x; idx < nn; idx += kEnergyThreads) {
        const int i = int(idx / n), j = int(idx % n);
        const double c = double(f[idx]);
        const double dx = (double(f[(long long)((i + 1) % n) * n + j]) - c) / h;
        const double dy = (double(f[(long long)i * n + (j + 1) % n]) - c) / h;
        const double w = c * c - 1.0;
        s += 0.5 * eps * eps * (dx * dx + dy * dy) + 0.25 * w * w;
    }
    __shared__ double red[kEnergyThreads / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kEnergyThreads / 32; ++w) t += red[w];
        e[blockIdx.x] = h * h * t;
    }
}

template <typename T>
__global__ void energy_grad_kernel(const T* __restrict__ u, T* __restrict__ g, int n, double h, double eps,
                                   long long total) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const long long nn = (long long)n * n;
    const T* f = u + (idx / nn) * nn;
    const int i = int((idx % nn) / n), j = int(idx % n);
    const double c = double(f[(long long)i * n + j]);
    const double lap = (double(f[(long long)((i + 1) % n) * n + j]) + double(f[(long long)((i + n - 1) % n) * n + j]) +
                        double(f[(long long)i * n + (j + 1) % n]) + double(f[(long long)i * n + (j + n - 1) % n]) -
                        4.0 * c) / (h * h);
    g[idx] = T(h * h * (-eps * eps * lap - (c - c * c * c)));
}

static int check_p(const ac_params* p) {
    ACPR_CHECK_ARG(p && p->n >= 2 && p->length > 0, "bad ac_params");
    ACPR_CHECK_ARG(p->precision == AC_F32 || p->precision == AC_F64, "bad precision");
    return AC_OK;
}

int energy(const ac_params* p, int fields, const void* u, double* e_dev, cudaStream_t st) {
    int rc = check_p(p);
    if (rc) return rc;
    ACPR_CHECK_ARG(fields >= 0 && u && e_dev, "bad energy arguments");
    if (!fields) return AC_OK;
    const double h = p->length / p->n;
    if (p->precision == AC_F64)
        energy_kernel<double><<<fields, kEnergyThreads, 0, st>>>(static_cast<const double*>(u), p->n, h, p->eps, e_dev);
    else
        energy_kernel<float><<<fields, kEnergyThreads, 0, st>>>(static_cast<const float*>(u), p->n, h, p->eps, e_dev);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

int energy_grad(const ac_params* p, int fields, const void* u, void* g, cudaStream_t st) {
    int rc = check_p(p);
    if (rc) return rc;
    ACPR_CHECK_ARG(fields >= 0 && u && g && u != g, "bad energy_grad arguments");
    const long long total = (long long)fields * p->n * p->n;
    if (!total) return AC_OK;
    const double h = p->length / p->n;
    const unsigned blocks = unsigned((total + 255) / 256);
    if (p->precision == AC_F64)
        energy_grad_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(u), static_cast<double*>(g),
                                                           p->n, h, p->eps, total);
    else
        energy_grad_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(u), static_cast<float*>(g), p->n,
                                                          h, p->eps, total);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

static size_t grad_ws_bytes(const ac_params* p, int steps, int K) {
    const size_t fb = elem_size(p->precision) * size_t(p->n) * p->n;
    const int nseg = (steps + K - 1) / K;
    return fb * (size_t(nseg + 1) + size_t(K + 1) + 2);
}

int energy_gradient_ic(const ac_params* p, int steps, int K, const void* u0, void* grad, void* ws, size_t ws_bytes,
                       cudaStream_t st) {
    int rc = check_p(p);
    if (rc) return rc;
    ACPR_CHECK_ARG(steps >= 0 && K >= 1 && u0 && grad && ws, "bad gradient arguments");
    ACPR_CHECK_ARG(ws_bytes >= grad_ws_bytes(p, steps, K), "workspace too small: need %zu bytes",
                   grad_ws_bytes(p, steps, K));
    const size_t fb = elem_size(p->precision) * size_t(p->n) * p->n;
    const int nseg = (steps + K - 1) / K;
    char* cp = static_cast<char*>(ws);                 // checkpoints c_0 .. c_nseg
    char* traj = cp + fb * (nseg + 1);                 // one segment's states
    char* lam[2] = {traj + fb * (K + 1), traj + fb * (K + 2)};
    ACPR_CUDA(cudaMemcpyAsync(cp, u0, fb, cudaMemcpyDeviceToDevice, st));
    for (int i = 0; i < nseg; ++i) {
        const int len = (i + 1) * K <= steps ? K : steps - i * K;
        rc = fine_run(p, 1, 1, len, cp + fb * i, 0, 0, cp + fb * (i + 1), 0, 0, nullptr, 0, nullptr, nullptr, st);
        if (rc) return rc;
    }
    rc = energy_grad(p, 1, cp + fb * nseg, lam[0], st);
    if (rc) return rc;
    int cur = 0;
    for (int i = nseg - 1; i >= 0; --i) {
        const int len = (i + 1) * K <= steps ? K : steps - i * K;
        // recompute the segment's states u_{iK} .. u_{iK+len} (traj[len] is not needed)
        rc = fine_run(p, 1, 1, len, cp + fb * i, 0, 0, traj + fb * len, 0, 0, nullptr, 0, nullptr, traj, st);
        if (rc) return rc;
        rc = fine_run(p, 1, 1, len, lam[cur], 0, 0, lam[cur ^ 1], 0, 0, nullptr, 1, traj, nullptr, st);
        if (rc) return rc;
        cur ^= 1;
    }
    ACPR_CUDA(cudaMemcpyAsync(grad, lam[cur], fb, cudaMemcpyDeviceToDevice, st));
    return AC_OK;
}

}  // namespace acpr

extern "C" int ac_energy(const ac_params* params, int num_fields, const void* u, double* energy_dev,
                         acpr_stream stream) {
    return acpr::energy(params, num_fields, u, energy_dev, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int ac_energy_grad(const ac_params* params, int num_fields, const void* u, void* grad,
                              acpr_stream stream) {
    return acpr::energy_grad(params, num_fields, u, grad, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" size_t ac_energy_gradient_workspace(const ac_params* params, int steps, int checkpoint_every) {
    if (!params || steps < 0 || checkpoint_every < 1 || params->n < 2) return 0;
    return acpr::grad_ws_bytes(params, steps, checkpoint_every);
}

extern "C" int ac_energy_gradient_ic(const ac_params* params, int steps, int checkpoint_every, const void* u0,
                                     void* grad, void* workspace, size_t workspace_bytes, acpr_stream stream) {
    return acpr::energy_gradient_ic(params, steps, checkpoint_every, u0, grad, workspace, workspace_bytes,
                                    reinterpret_cast<cudaStream_t>(stream));
}
