// cnn_wgrad_tc.cu -- weight gradient of a hidden C -> C conv layer (C = 64)
// on the tensor cores:
//   dW[tap][co][ci] = sum over pixels p of dz(p, co) * a(p + off(tap), ci),
// off(tap) = (tap / 3 - 1, tap % 3 - 1) with periodic wrap, dz the gradient of
// the layer's pre-activation and a its input activation, both bf16 in the
// chunked layout [f][C/8][n][n][8].  Per tap this is a GEMM with M = co, N = ci
// and K = pixels.  In the chunked layout the 8 channels of a pixel are 16
// contiguous bytes and consecutive pixels follow each other, which is the
// "MN-major" no-swizzle core-matrix layout of the tcgen05 operands (a core
// matrix = 8 pixels x 8 channels, 128 contiguous bytes); A and B are read
// transposed (instruction descriptor bits 15 and 16), LBO = 128 bytes between
// pixel groups, SBO = the chunk-plane stride.  One MMA = 64 x 64 x 16 (16
// pixels); the M = 64 accumulator puts rows 16 q .. 16 q + 15 in TMEM lanes
// 32 q .. 32 q + 15.
//
// Work: units (field, 128-column block, row) in order, split into kChunks
// contiguous ranges; each range is run by two CTAs, one for taps 0..4 and one
// for taps 5..8 (5 or 4 accumulators of 64 columns), so every CTA keeps its
// accumulators in TMEM over its whole range and writes one partial per tap at
// the end.  The CTA of taps 0..4 also forms the bias gradient sum_p dz(p, co)
// as one more 64 x 16 x 16 MMA per pixel group against a B of ones.  The
// partials are summed in a fixed order by the same reduction as the CUDA-core
// weight gradient, so the result is deterministic.
//   warp 0, producer: the input rows y - 1, y, y + 1 of a run start and then
//     row y + 1 per unit (128 columns plus one pixel each side, wrapped at the
//     field's edge: bulk copy per chunk plane, wrapped pixel by cp.async) into
//     a ring of activation rows, and row y of dz into a ring of dz rows;
//   warp 1 (lane 0), MMA issuer: per unit 8 pixel groups x its taps, then
//     releases the dz row and the activation row no later unit reads;
//   warps 2..5, epilogue: after the last MMA, read the accumulators and store
//     the partials.
// Every wait is bounded and sets the caller's status word when it gives up.
#include "cnn.cuh"
#include "tc_pipe.cuh"
#include "tc_ptx.cuh"

namespace acpr {

namespace {
constexpr int kWC = 64;                          // channels
constexpr int kWKC = kWC / 8;                    // chunk planes
constexpr int kWThreads = 32 * 6;                // producer, MMA, 4 epilogue warps
constexpr uint32_t kWAPlane = 130u * 16u;        // activation row: 128 pixels + 2 guard pixels
constexpr uint32_t kWASlot = kWKC * kWAPlane;
constexpr uint32_t kWDPlane = 128u * 16u;        // dz row: 128 pixels
constexpr uint32_t kWDSlot = kWKC * kWDPlane;
constexpr int kWRA = 7;                          // activation-row ring
constexpr int kWRD = 4;                          // dz-row ring
constexpr size_t kWOnesOff = size_t(kWRA) * kWASlot + size_t(kWRD) * kWDSlot;
constexpr uint32_t kWOnesPlane = 16u * 16u;      // B = ones for the bias: N = 16, K = 16, MN-major
constexpr size_t kWCtlOff = kWOnesOff + 2 * kWOnesPlane;
constexpr size_t kWSmem = kWCtlOff + 256;

struct WCtl {
    uint64_t afull[kWRA], aempty[kWRA], dfull[kWRD], dempty[kWRD];
    uint64_t fin;
    uint32_t tmem;
    int abort;
};
static_assert(sizeof(WCtl) <= 256, "control block");

bool g_wgrad_tc = true;
}  // namespace

void set_wgrad_tc(bool on) { g_wgrad_tc = on; }

__global__ void __launch_bounds__(kWThreads, 1)
wgrad_tc_kernel(const __nv_bfloat16* __restrict__ a, const __nv_bfloat16* __restrict__ dz, float* __restrict__ part,
                int n, int batch, int chunks, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* aring = smem;
    unsigned char* dring = smem + size_t(kWRA) * kWASlot;
    WCtl* ctl = reinterpret_cast<WCtl*>(smem + kWCtlOff);
    volatile int* abort_flag = &ctl->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int group = blockIdx.x & 1;                 // taps 0..4 or 5..8
    const int tap0 = group ? 5 : 0, ntap = group ? 4 : 5;
    const int ch = blockIdx.x >> 1;                   // pixel chunk of the reduction
    const int NB = n / 128;
    const size_t nn = size_t(n) * n;
    const long long total = (long long)batch * NB * n;
    const long long u0 = total * ch / chunks;
    const long long u1 = total * (ch + 1) / chunks;

    if (tid == 0) {
        for (int i = 0; i < kWRA; ++i) {
            tc::mbar_init(&ctl->afull[i], 1 + 32);  // byte count + the producer lanes' cp.async
            tc::mbar_init(&ctl->aempty[i], 1);
        }
        for (int i = 0; i < kWRD; ++i) {
            tc::mbar_init(&ctl->dfull[i], 1);
            tc::mbar_init(&ctl->dempty[i], 1);
        }
        tc::mbar_init(&ctl->fin, 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
    }
    if (group == 0) {
        uint32_t* ones = reinterpret_cast<uint32_t*>(smem + kWOnesOff);
        for (int i = tid; i < int(2 * kWOnesPlane / 4); i += blockDim.x) ones[i] = 0x3F803F80u;  // bf16 1.0 pairs
        tc::fence_proxy_async_smem();
    }
    if (warp == 1) tc::tmem_alloc(&ctl->tmem, 512u);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0) {
        // ---- producer warp
        long long ja = 0, jd = 0;
        RingPos ra(kWRA), rd(kWRD);
        RowCursor cur(u0, n, NB);
        bool ok = true;
        for (long long u = u0; u < u1 && ok; ++u, cur.next()) {
            const int y = cur.y;
            const long long f = cur.f;
            const bool start = (u == u0) || (y == 0);
            const int x0 = cur.cb * 128;
            const bool wl = x0 == 0, wr = x0 + 128 == n;
            const int bx = wl ? x0 : x0 - 1;
            const uint32_t bbytes = uint32_t(130 - int(wl) - int(wr)) * 16u;
            const uint32_t boff = wl ? 16u : 0u;
            for (int k = start ? 0 : 2; k < 3; ++k) {
                int yin = y - 1 + k;
                yin = yin < 0 ? yin + n : (yin >= n ? yin - n : yin);
                const int slot = ra.idx;
                bool free_slot = true;
                if (lane == 0 && ja >= kWRA) free_slot = p_wait(&ctl->aempty[slot], ra.phase ^ 1u, abort_flag, status);
                if (!__shfl_sync(0xffffffffu, free_slot, 0)) {
                    ok = false;
                    break;
                }
                unsigned char* dst = aring + size_t(slot) * kWASlot;
                const __nv_bfloat16* src = a + (size_t(f) * kWKC * nn + size_t(yin) * n) * 8;
                if (lane == 0) {
                    tc::mbar_arrive_expect_tx(&ctl->afull[slot], uint32_t(kWKC) * bbytes);
                    for (int kc = 0; kc < kWKC; ++kc)
                        tc::bulk_g2s(dst + size_t(kc) * kWAPlane + boff, src + (size_t(kc) * nn + size_t(bx)) * 8,
                                     bbytes, &ctl->afull[slot]);
                }
                if (lane < kWKC) {
                    unsigned char* d = dst + size_t(lane) * kWAPlane;
                    const __nv_bfloat16* r = src + size_t(lane) * nn * 8;
                    if (wl) cp_async16(d, r + size_t(n - 1) * 8);
                    if (wr) cp_async16(d + 129 * 16, r);
                }
                cp_async_arrive(&ctl->afull[slot]);
                ++ja;
                ra.next();
            }
            if (!ok) break;
            // dz row y of this unit
            const int slot = rd.idx;
            bool free_slot = true;
            if (lane == 0 && jd >= kWRD) free_slot = p_wait(&ctl->dempty[slot], rd.phase ^ 1u, abort_flag, status);
            if (!__shfl_sync(0xffffffffu, free_slot, 0)) break;
            if (lane == 0) {
                unsigned char* dst = dring + size_t(slot) * kWDSlot;
                const __nv_bfloat16* src = dz + (size_t(f) * kWKC * nn + size_t(y) * n + size_t(x0)) * 8;
                tc::mbar_arrive_expect_tx(&ctl->dfull[slot], kWDSlot);
                for (int kc = 0; kc < kWKC; ++kc)
                    tc::bulk_g2s(dst + size_t(kc) * kWDPlane, src + size_t(kc) * nn * 8, kWDPlane, &ctl->dfull[slot]);
            }
            ++jd;
            rd.next();
        }
        // drain: every issued copy lands before the CTA may exit
        if (lane == 0) {
            for (long long x = ja > kWRA ? ja - kWRA : 0; x < ja; ++x)
                tc::mbar_wait_bounded(&ctl->afull[x % kWRA], uint32_t((x / kWRA) & 1), kTcSpin);
            for (long long x = jd > kWRD ? jd - kWRD : 0; x < jd; ++x)
                tc::mbar_wait_bounded(&ctl->dfull[x % kWRD], uint32_t((x / kWRD) & 1), kTcSpin);
        }
        cp_async_wait_all();
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            // bf16 A and B, f32 D, both operands MN-major (transposed), M = 64, N = 64
            constexpr uint32_t idesc = tc::idesc_bf16_f32(64, 64) | (1u << 15) | (1u << 16);
            constexpr uint32_t idesc_b = tc::idesc_bf16_f32(64, 16) | (1u << 15) | (1u << 16);
            const uint64_t ones_d = tc::smem_desc(tc::smem_u32(smem + kWOnesOff), 128, kWOnesPlane);
            const uint64_t a_hi = tc::smem_desc(0, 128, kWDPlane);  // A = dz rows
            const uint64_t b_hi = tc::smem_desc(0, 128, kWAPlane);  // B = activation rows
            const uint32_t aring_u = tc::smem_u32(aring) >> 4, dring_u = tc::smem_u32(dring) >> 4;
            RingPos ra(kWRA), rd(kWRD);
            // ring positions of the unit's rows y - 1, y, y + 1
            int pos[3] = {0, 0, 0};
            uint32_t par[3] = {0, 0, 0};
            bool ok = true, first = true;
            int y = int(u0 % n);
            for (long long u = u0; u < u1 && ok; ++u, y = (y + 1 == n ? 0 : y + 1)) {
                const bool start = (u == u0) || (y == 0);
                if (start) {
                    for (int k = 0; k < 3; ++k, ra.next()) {
                        pos[k] = ra.idx;
                        par[k] = ra.phase;
                    }
                } else {
                    pos[0] = pos[1];
                    par[0] = par[1];
                    pos[1] = pos[2];
                    par[1] = par[2];
                    pos[2] = ra.idx;
                    par[2] = ra.phase;
                    ra.next();
                }
                for (int k = start ? 0 : 2; k < 3 && ok; ++k) ok = p_wait(&ctl->afull[pos[k]], par[k], abort_flag, status);
                if (ok) ok = p_wait(&ctl->dfull[rd.idx], rd.phase, abort_flag, status);
                if (!ok) break;
                // the wrapped pixels came by cp.async (generic proxy); the MMAs read through the async proxy
                tc::fence_proxy_async_smem();
                tc::fence_after_sync();
                const uint32_t d_u = dring_u + uint32_t(rd.idx) * (kWDSlot >> 4);
#pragma unroll 1
                for (int kg = 0; kg < 8; ++kg) {
                    const uint64_t ad = a_hi | uint64_t(d_u + uint32_t(kg * 16));
                    for (int t = 0; t < ntap; ++t) {
                        const int tap = tap0 + t, dy = tap / 3, dx = tap % 3;
                        const uint32_t r_u = aring_u + uint32_t(pos[dy]) * (kWASlot >> 4);
                        const uint64_t bd = b_hi | uint64_t(r_u + uint32_t(kg * 16 + dx));
                        tc::mma_bf16(tmem + uint32_t(t * kWC), ad, bd, idesc, (first && kg == 0) ? 0u : 1u);
                    }
                    if (group == 0)  // bias: every column of this accumulator is sum_p dz(p, co)
                        tc::mma_bf16(tmem + uint32_t(5 * kWC), ad, ones_d, idesc_b, (first && kg == 0) ? 0u : 1u);
                }
                first = false;
                tc::mma_commit(&ctl->dempty[rd.idx]);
                rd.next();
                // row y - 1 is read by no later unit; at the end of a run neither are y, y + 1
                const bool cont = (u + 1 < u1) && (y + 1 != n);
                tc::mma_commit(&ctl->aempty[pos[0]]);
                if (!cont) {
                    tc::mma_commit(&ctl->aempty[pos[1]]);
                    tc::mma_commit(&ctl->aempty[pos[2]]);
                }
            }
            // every MMA issued completes before the accumulators are read and TMEM is freed
            tc::mma_commit(&ctl->fin);
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---- epilogue: the accumulators of this CTA's taps -> partials
        const int q = warp & 3;
        const bool ok = tc::mbar_wait_bounded(&ctl->fin, 0, kTcSpin);
        if (!ok) atomicExch(status, 3);
        tc::fence_after_sync();
        if (ok && !*abort_flag) {
            const int co = 16 * q + lane;  // valid for lanes 0..15
            for (int t = 0; t < ntap; ++t) {
                float* dst = part + (size_t(ch) * 9 + size_t(tap0 + t)) * (kWC * kWC + kWC) + size_t(co) * kWC;
#pragma unroll 1
                for (int c0 = 0; c0 < kWC; c0 += 8) {
                    uint32_t v[8];
                    tc::tmem_ld8(tmem + (uint32_t(q * 32) << 16) + uint32_t(t * kWC + c0), v);
                    tc::tmem_wait_ld();
                    if (lane < 16) {
                        reinterpret_cast<float4*>(dst + c0)[0] =
                            make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]),
                                        __uint_as_float(v[3]));
                        reinterpret_cast<float4*>(dst + c0)[1] =
                            make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]), __uint_as_float(v[6]),
                                        __uint_as_float(v[7]));
                    }
                }
            }
            if (group == 0) {
                uint32_t v[8];
                tc::tmem_ld8(tmem + (uint32_t(q * 32) << 16) + uint32_t(5 * kWC), v);
                tc::tmem_wait_ld();
                if (lane < 16) part[(size_t(ch) * 9) * (kWC * kWC + kWC) + kWC * kWC + co] = __uint_as_float(v[0]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        // the MMA issuer's own completion wait (also when the epilogue gave up)
        if (lane == 0) tc::mbar_wait_bounded(&ctl->fin, 0, kTcSpin);
        __syncwarp();
        tc::tmem_dealloc(tmem, 512u);
    }
}

bool wgrad_tc_supported(int C, int n) { return g_wgrad_tc && C == kWC && n >= 128 && n % 128 == 0 && n <= 1024; }

int wgrad_tc_partials(int n, int batch, const __nv_bfloat16* a, const __nv_bfloat16* dz, float* part, int chunks,
                      int* status, cudaStream_t st) {
    if (!status) {
        set_error("tensor-core weight gradient: no status word");
        return AC_ERR_ARG;
    }
    static bool configured = false;
    if (!configured) {
        ACPR_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kWSmem)));
        configured = true;
    }
    wgrad_tc_kernel<<<2 * chunks, kWThreads, kWSmem, st>>>(a, dz, part, n, batch, chunks, status);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

}  // namespace acpr

extern "C" int cnn_train_set_wgrad_tc(int on) {
    acpr::set_wgrad_tc(on != 0);
    return AC_OK;
}
