// errors.cu -- per-thread error text for ac_last_error().
#include <atomic>
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace acpr {
namespace {
thread_local char g_err[512] = {0};
std::atomic<long long> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launch_add(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

}  // namespace acpr

extern "C" const char* ac_last_error(void) { return acpr::g_err; }

extern "C" long long ac_launch_count(void) { return acpr::g_launches.load(std::memory_order_relaxed); }
