// common.cuh -- shared device/host helpers of the acpr library (not the oracle).
#pragma once

#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/acpr.h"

namespace acpr {

// Per-thread last error text (ac_last_error()).
void set_error(const char* fmt, ...);

#define ACPR_CUDA(call)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ::acpr::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call,            \
                              cudaGetErrorString(e_));                               \
            return AC_ERR_CUDA;                                                      \
        }                                                                            \
    } while (0)

#define ACPR_CHECK_ARG(cond, ...)                                                    \
    do {                                                                             \
        if (!(cond)) {                                                               \
            ::acpr::set_error(__VA_ARGS__);                                          \
            return AC_ERR_ARG;                                                       \
        }                                                                            \
    } while (0)

// Kernels launched by the library (ac_launch_count()).
void count_launch();
void count_launch_add(long long n);

// Check a kernel launch (configuration errors are reported synchronously) and
// count it.
#define ACPR_LAUNCH_CHECK()                                                          \
    do {                                                                             \
        ::acpr::count_launch();                                                      \
        cudaError_t e_ = cudaGetLastError();                                         \
        if (e_ != cudaSuccess) {                                                     \
            ::acpr::set_error("%s:%d: kernel launch: %s", __FILE__, __LINE__,        \
                              cudaGetErrorString(e_));                               \
            return AC_ERR_CUDA;                                                      \
        }                                                                            \
    } while (0)

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using vec2_t = typename Vec2<T>::type;

inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
inline size_t elem_size(int precision) { return precision == AC_F64 ? 8 : 4; }

// Bounded-wait budget for device spin loops (iterations of a polling loop with
// a ~100 ns sleep each: about 2 s).
constexpr long long kSpinLimit = 20000000LL;

}  // namespace acpr
