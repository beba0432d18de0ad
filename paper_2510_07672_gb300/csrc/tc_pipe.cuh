// tc_pipe.cuh -- pieces shared by the warp-specialised tensor-core kernels
// (the row-streaming conv and the weight gradient): bounded role waits, ring
// positions, the row cursor of a contiguous range of work units, and 16-byte
// cp.async copies that arrive on an mbarrier.
#pragma once

#include <cstdint>

#include "tc_ptx.cuh"

namespace acpr {

constexpr long long kTcSpin = 4000000;  // ~0.2 s of polls with 32 ns sleeps

// Bounded wait on phase `parity` of `bar` by one role of a warp-specialised
// kernel: gives up once another role has given up (abort flag in shared
// memory) or after `limit` polls, then raises the abort flag and stores 3 in
// the caller's status word.
__device__ __forceinline__ bool p_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                       long long limit = kTcSpin) {
    for (long long i = 0; i < limit; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        __nanosleep(32);
    }
    *abort_flag = 1;
    atomicExch(status, 3);
    return false;
}

// 16-byte global -> shared copy on the load/store path (cp.async), and an
// arrival on `bar` once all of this thread's earlier cp.async copies landed.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Position in a ring of `size` entries: index and the parity of the pass
// over the ring (the mbarrier phase it waits for), advanced without division.
struct RingPos {
    int idx = 0;
    uint32_t phase = 0;
    int size;
    __device__ explicit RingPos(int sz) : size(sz) {}
    __device__ void next() {
        if (++idx == size) {
            idx = 0;
            phase ^= 1u;
        }
    }
};

// Output row (field f, column block cb, row y) of work unit u, advanced by
// one unit at a time (one division per CTA, none in the loops).
struct RowCursor {
    int y, cb, NB, n;
    long long f;
    __device__ RowCursor(long long u, int n_, int nb) : NB(nb), n(n_) {
        y = int(u % n_);
        const long long t = u / n_;
        cb = int(t % nb);
        f = t / nb;
    }
    __device__ void next() {
        if (++y == n) {
            y = 0;
            if (++cb == NB) {
                cb = 0;
                ++f;
            }
        }
    }
};

}  // namespace acpr
