// cnn_tc.cu -- hidden C -> C layers of the coarse propagator as implicit GEMMs
// on the 5th-generation tensor cores (tcgen05, accumulators in TMEM).
//
// One CTA computes TY full rows (all n columns) of one field for all C output
// channels.  Its input tile, rows y0-1 .. y0+TY with one wrapped column on each
// side, sits in shared memory in the K-major "no swizzle" core-matrix layout:
// for each chunk of 8 input channels a plane of pixels, 16 bytes (8 bf16) per
// pixel, pixels of a row consecutive, W = n + 2 pixels per row.  For a tap
// (dy, dx) the A operand of 128 consecutive output positions is then the same
// plane read from a start address shifted by dy*W + dx - 1 pixels: the 9-tap
// implicit GEMM needs no im2col copy, only 9 descriptors.  Output positions
// that fall on a wrap column are computed and discarded (2 of every n + 2).
//   GEMM per 128-position M tile: M = 128, N = C (cout), K = 9 * C (tap, cin),
//   issued as 9 * C/16 tcgen05.mma (K = 16 each) into TMEM columns [mt*C, +C).
// Weights: bf16 [tap][cin/8][cout][8] (cnn_pack_weights), the B operand.
// Loads: cp.async.bulk (one weight copy, three copies per input row: the row
// and its two wrap pixels), completing on an mbarrier.  The epilogue reads
// TMEM with tcgen05.ld, adds the float32 bias, applies the activation, rounds
// to bf16 and stores 16-byte channel chunks.  All waits are bounded; a timeout
// sets the caller's status word (the first int of the conv workspace), which
// conv_check_status() reports as AC_ERR_TIMEOUT.
// Fields with n >= 128 take the persistent, warp-specialised kernel below.
#include <algorithm>

#include "cnn.cuh"
#include "tc_pipe.cuh"
#include "tc_ptx.cuh"

namespace acpr {

namespace {
constexpr int kTcThreads = 256;
// Test hook (ac_test_conv_stall): > 0 makes the next persistent conv launches'
// MMA issuer wait, with this poll limit, on an mbarrier nothing arrives on.
int g_test_stall = 0;
}

void set_test_stall(int polls) { g_test_stall = polls > 0 ? polls : 0; }

int conv_check_status_uncaptured(int* status, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    ACPR_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return AC_OK;
    return conv_check_status(status, st);
}

int conv_check_status(int* status, cudaStream_t st) {
    if (!status) return AC_OK;
    int flag = 0;
    ACPR_CUDA(cudaMemcpyAsync(&flag, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    ACPR_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        ACPR_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
        ACPR_CUDA(cudaStreamSynchronize(st));
        set_error("tensor-core conv: bounded wait gave up (%s)",
                  flag == 1 ? "operand loads" : flag == 2 ? "MMA completion" : "pipeline wait");
        return AC_ERR_TIMEOUT;
    }
    return AC_OK;
}

// float32 master W[cout][cin][3][3] -> bf16 [tap][cin/8][cout][8]
__global__ void pack_hidden_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ out, int C) {
    const int total = 9 * C * C;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int i = idx % 8;
        const int o = (idx / 8) % C;
        const int kc = (idx / (8 * C)) % (C / 8);
        const int tap = idx / (8 * C * (C / 8));
        const int c = kc * 8 + i;
        out[idx] = __float2bfloat16_rn(w[(o * C + c) * 9 + tap]);
    }
}

size_t packed_hidden_bytes(const cnn_desc* d) {
    const int hidden = d->layers - 2;
    return size_t(hidden > 0 ? hidden : 0) * 9 * d->channels * d->channels * sizeof(__nv_bfloat16);
}

int pack_hidden_weights(const cnn_desc* d, cudaStream_t st) {
    const int C = d->channels;
    const float* w = static_cast<const float*>(d->w);
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(d->packed);
    size_t woff = size_t(C) * 9;
    for (int l = 1; l < d->layers - 1; ++l) {
        pack_hidden_kernel<<<64, 256, 0, st>>>(w + woff, p + size_t(l - 1) * 9 * C * C, C);
        ACPR_LAUNCH_CHECK();
        woff += size_t(C) * C * 9;
    }
    return AC_OK;
}

struct TcShape {
    int TY = 0, W = 0, n_mt = 0, plane_px = 0, ncols = 0;
    size_t smem = 0;
};

static TcShape tc_shape(int n, int C, int TY) {
    TcShape s;
    s.TY = TY;
    s.W = n + 2;
    const int pos = TY * s.W;
    s.n_mt = (pos + 127) / 128;
    // guard of 8 pixels, then reads up to the last M tile shifted by 2 rows + 1
    const int need = 8 + s.n_mt * 128 + 2 * s.W + 1;
    s.plane_px = (need + 7) / 8 * 8;
    int cols = 32;
    while (cols < s.n_mt * C) cols *= 2;
    s.ncols = cols;
    s.smem = size_t(C / 8) * s.plane_px * 16 + size_t(9) * C * C * 2 + 64;
    return s;
}

// Largest row count per CTA that fits: prefer shapes that let two CTAs share
// an SM (<= 113 KB shared memory and <= 256 TMEM columns each).
static TcShape pick_shape(int n, int C) {
    TcShape best;
    for (int pass = 0; pass < 2 && best.TY == 0; ++pass) {
        for (int TY = 8; TY >= 1; TY /= 2) {
            if (n % TY) continue;
            TcShape s = tc_shape(n, C, TY);
            const bool fits = pass == 0 ? (s.smem <= 113 * 1024 && s.ncols <= 256)
                                        : (s.smem <= 227 * 1024 && s.ncols <= 512);
            if (fits) { best = s; break; }
        }
    }
    return best;
}

// Epilogue modes: kFwd writes bf16(act(acc + bias)) and, if zio != NULL, the
// float32 pre-activation acc + bias to zio (training forward); kDgrad writes
// bf16(acc * act'(zio)) (backward through a hidden layer: acc is the
// transposed-and-flipped conv of the next layer's gradient, zio the saved
// pre-activation of this layer's input).  zio is float32 [f][C/8][n][n][8].
// kFwdLast (persistent kernel, the last hidden layer): as kFwd, and the
// epilogue also projects each pixel's bf16 activations onto the last
// layer's nine taps, maps[f][tap][pixel] = sum_c W_last[tap][c] a(pixel, c)
// (float32, bf16-rounded weights, channels in order); the C -> 1 conv is then
// a nine-point stencil of these maps (last_stencil).  The activations
// themselves are stored only when zio != NULL (training needs them).
enum { kFwd = 0, kDgrad = 1, kFwdLast = 2 };

template <int C, int ACT>
__global__ void __launch_bounds__(kTcThreads)
conv_hidden_tc_kernel(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out,
                      const __nv_bfloat16* __restrict__ wpk, const float* __restrict__ bias, int n, int TY,
                      int n_mt, int plane_px, int ncols, int mode, float* __restrict__ zio,
                      int* __restrict__ status) {
    constexpr int KC = C / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = n + 2;
    const int tiles = n / TY;
    const int f = blockIdx.x / tiles;
    const int y0 = (blockIdx.x % tiles) * TY;
    const uint32_t plane_bytes = uint32_t(plane_px) * 16;
    unsigned char* a_tile = smem;
    unsigned char* w_tile = a_tile + KC * plane_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(w_tile + 9 * C * C * 2);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t nn = size_t(n) * n;

    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0) tc::tmem_alloc(slot, uint32_t(ncols));
    if (tid == 0) {
        const uint32_t wbytes = 9 * C * C * 2;
        const uint32_t rowbytes = uint32_t(n) * 16;
        tc::mbar_arrive_expect_tx(&bars[0], wbytes + KC * (TY + 2) * (rowbytes + 32));
        tc::bulk_g2s(w_tile, wpk, wbytes, &bars[0]);
        for (int kc = 0; kc < KC; ++kc) {
            for (int r = 0; r < TY + 2; ++r) {
                int y = y0 - 1 + r;
                y = y < 0 ? y + n : (y >= n ? y - n : y);
                const __nv_bfloat16* src = in + ((size_t(f) * KC + kc) * nn + size_t(y) * n) * 8;
                unsigned char* dst = a_tile + kc * plane_bytes + size_t(8 + r * W) * 16;
                tc::bulk_g2s(dst + 16, src, rowbytes, &bars[0]);           // x = 0..n-1
                tc::bulk_g2s(dst, src + size_t(n - 1) * 8, 16, &bars[0]);  // x = n-1 on the left
                tc::bulk_g2s(dst + size_t(n + 1) * 16, src, 16, &bars[0]); // x = 0 on the right
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;

    bool ok = tc::mbar_wait_bounded(&bars[0], 0, kTcSpin);
    ok = __syncthreads_and(ok);
    if (ok) {
        if (tid == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(128, C);
            const uint32_t a0 = tc::smem_u32(a_tile), w0 = tc::smem_u32(w_tile);
            for (int mt = 0; mt < n_mt; ++mt) {
                for (int tap = 0; tap < 9; ++tap) {
                    const uint32_t apx = uint32_t(8 + mt * 128 + (tap / 3) * W + (tap % 3) - 1);
#pragma unroll
                    for (int ks = 0; ks < C / 16; ++ks) {
                        const uint64_t ad = tc::smem_desc(a0 + 2 * ks * plane_bytes + apx * 16, plane_bytes, 128);
                        const uint64_t bd = tc::smem_desc(w0 + uint32_t((tap * KC + 2 * ks) * C * 16), C * 16, 128);
                        tc::mma_bf16(tmem + uint32_t(mt * C), ad, bd, idesc, (tap | ks) != 0);
                    }
                }
            }
            tc::mma_commit(&bars[1]);
        }
        ok = tc::mbar_wait_bounded(&bars[1], 0, kTcSpin);
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (tid == 0) atomicExch(status, 2);
            tc::mbar_wait_bounded(&bars[1], 0, kTcSpin);  // let the MMAs drain
        }
    } else {
        if (tid == 0) atomicExch(status, 1);
        tc::mbar_wait_bounded(&bars[0], 0, kTcSpin);  // let in-flight copies land
    }
    if (ok) {
        tc::fence_after_sync();
        const int qw = warp & 3, half = warp >> 2;
        for (int mt = 0; mt < n_mt; ++mt) {
            const int q = mt * 128 + qw * 32 + lane;
            const int yl = q / W, xs = q % W;
            const bool valid = yl < TY && xs >= 1 && xs <= n;
            const size_t pix = size_t(y0 + yl) * n + (xs - 1);
#pragma unroll
            for (int h = 0; h < KC / 2; ++h) {
                const int kc = half * (KC / 2) + h;
                uint32_t v[8];
                tc::tmem_ld8(tmem + (uint32_t(qw * 32) << 16) + uint32_t(mt * C + kc * 8), v);
                tc::tmem_wait_ld();
                if (valid) {
                    const size_t off = ((size_t(f) * KC + kc) * nn + pix) * 8;
                    __align__(16) __nv_bfloat16 o8[8];
                    if (mode == kFwd) {
                        __align__(16) float z8[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            z8[i] = __uint_as_float(v[i]) + __ldg(bias + kc * 8 + i);
                            o8[i] = __float2bfloat16_rn(act_c<ACT>(z8[i]));
                        }
                        if (zio) {
                            reinterpret_cast<float4*>(zio + off)[0] = *reinterpret_cast<const float4*>(z8);
                            reinterpret_cast<float4*>(zio + off)[1] = *reinterpret_cast<const float4*>(z8 + 4);
                        }
                    } else {
                        const float4 za = reinterpret_cast<const float4*>(zio + off)[0];
                        const float4 zb = reinterpret_cast<const float4*>(zio + off)[1];
                        const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            o8[i] = __float2bfloat16_rn(__uint_as_float(v[i]) * act_grad_c<ACT>(zz[i]));
                    }
                    *reinterpret_cast<uint4*>(out + off) = *reinterpret_cast<const uint4*>(o8);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, uint32_t(ncols));
}

// ------------------------------------------------------- row streaming --
// Persistent kernel that reads each input row once and folds the vertical
// taps in TMEM.  Output row y of a 3x3 conv is
//   out(y) = D(y-1)[dy=0] + D(y)[dy=1] + D(y+1)[dy=2],
//   D(y')[dy](x, co) = sum_dx sum_ci in(y', x + dx - 1, ci) W(dy, dx, ci, co),
// so one GEMM per input row y' (M = 128 positions, N = 3C = (dy, co),
// K = 3 (dx) x C (ci)) gives the row's contribution to three output rows.
// N = 3C keeps the tensor core busier per byte of A read from shared memory
// than the tap-major form (N = C, each input row read nine times).
// Work unit = one output row of one 128-column block (field f, block cb, row
// y), ordered (f, cb, y); CTA c takes a contiguous range and streams the input
// rows y-1, y, y+1 at the start of a block run and one new row (y+1) per unit
// after that.
//   warp 0, producer: each streamed input row (128 columns plus one pixel
//     each side, wrapped at the field's edge, all C/8 chunk planes) into a
//     ring slot: one bulk copy per plane, wrapped pixels by cp.async, all
//     completing on full[slot];
//   warps 1 and 2 (lane 0), MMA issuers of the even and odd rows: 3 x C/16
//     MMAs of 128 x 3C x 16 per streamed row into TMEM slot j % DS (DS slots
//     of 3C columns, padded); tcgen05.commit releases the ring slot (empty)
//     and marks the TMEM slot full (dfull);
//   warps 3 .. 2 + 4 EPW, epilogue: a warp reads its TMEM lane quarter and
//     its C/32 (at least one) 8-channel chunks of the three dy blocks, frees
//     the TMEM slot (dempty) and keeps two partial output rows in registers:
//       finish out(y'-1) = P + D(y')[2];  P = P' + D(y')[1];  P' = D(y')[0] + b.
//     Every output is ((D(y-1)[0] + b) + D(y)[1]) + D(y+1)[2] with each
//     D accumulated over (dx, K-step) in order, whatever the ring depth, TMEM
//     slot count or CTA count: G is bitwise the same under every shape.
// kFwdLast: the nine-tap projection of each pixel's activations is summed
// per warp over its channels and then over the warps of a lane quarter in a
// fixed order through shared memory.
constexpr int kRMaxRing = 24;
constexpr int kRMaxD = 5;

struct RCtl {
    uint64_t never;  // test hook: nothing ever arrives here
    uint64_t full[kRMaxRing];
    uint64_t empty[kRMaxRing];
    uint64_t dfull[kRMaxD];
    uint64_t dempty[kRMaxD];
    uint64_t qbar[2][4];  // kFwdLast: the partial projections of a lane quarter are in shared memory
    uint64_t fin;  // completion of every MMA the CTA issued
    uint32_t tmem;
    int abort;
    alignas(16) float bias[64];
    alignas(16) float wl[64 * 10];  // kFwdLast: bf16-rounded last-layer weights [channel][tap], tap 9 = 0
};
constexpr size_t kRCtlBytes = 4096;
constexpr size_t kRScratchBytes = size_t(2) * 4 * 4 * 9 * 32 * sizeof(float);  // [2][quarter][warp][tap][lane]

// TMEM columns of one slot: 3C rounded up to a power of two, so that every
// slot starts on a multiple of its own width.
__host__ __device__ constexpr int r_dcols(int C) { return C <= 16 ? 64 : (C <= 32 ? 128 : 256); }
__host__ __device__ constexpr uint32_t r_slot_bytes(int C) { return uint32_t(C / 8) * 130u * 16u; }

// Epilogue geometry: CPW 8-channel chunks per warp, EPW warps per TMEM lane
// quarter, THREADS = producer warp + two MMA warps + 4 EPW epilogue warps.
template <int C>
struct RGeom {
    static constexpr int KC = C / 8;
    static constexpr int CPW = KC >= 4 ? KC / 4 : 1;
    static constexpr int EPW = KC / CPW;
    static constexpr int THREADS = 32 * (3 + 4 * EPW);
};

template <int C, int ACT, int mode>
__global__ void __launch_bounds__(RGeom<C>::THREADS, 1)
conv_rows_tc(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out,
             const __nv_bfloat16* __restrict__ wpk, const float* __restrict__ bias, int n, int batch, int RING,
             int DS, float* __restrict__ zio, int* __restrict__ status, int stall,
             const float* __restrict__ wlast, float* __restrict__ maps) {
    constexpr int KC = C / 8;
    constexpr int N3 = 3 * C;
    constexpr int DCOLS = r_dcols(C);
    constexpr int CPW = RGeom<C>::CPW;  // chunks per epilogue warp
    constexpr int EPW = RGeom<C>::EPW;  // epilogue warps per lane quarter
    constexpr uint32_t WBYTES = 9u * C * C * 2u;
    constexpr uint32_t PLANE = 130u * 16u;
    constexpr uint32_t SLOT = r_slot_bytes(C);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* w_tile = smem;  // [dx][kc][dy][cout][8]: B of the (dx, K-step) MMA is one block
    unsigned char* ring = smem + WBYTES;
    RCtl* ctl = reinterpret_cast<RCtl*>(ring + size_t(RING) * SLOT);
    float* scratch = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(ctl) + kRCtlBytes);
    volatile int* abort_flag = &ctl->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NB = n / 128;
    const size_t nn = size_t(n) * n;
    const long long total = (long long)batch * NB * n;
    const long long u0 = total * blockIdx.x / gridDim.x;
    const long long u1 = total * (blockIdx.x + 1) / gridDim.x;

    if (tid == 0) {
        for (int i = 0; i < RING; ++i) {
            tc::mbar_init(&ctl->full[i], 1 + 32);  // producer's byte count + 32 lanes' cp.async
            tc::mbar_init(&ctl->empty[i], 1);
        }
        for (int i = 0; i < DS; ++i) {
            tc::mbar_init(&ctl->dfull[i], 1);
            tc::mbar_init(&ctl->dempty[i], 4 * EPW);
        }
        for (int i = 0; i < 8; ++i) tc::mbar_init(&ctl->qbar[i / 4][i % 4], EPW);
        tc::mbar_init(&ctl->fin, 2);
        tc::mbar_init(&ctl->never, 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
    }
    static_assert(sizeof(RCtl) <= kRCtlBytes, "control block");
    __syncthreads();

    if (warp == 0) {
        // ---- producer warp: starts at once; the other warps stage the weights
        // meanwhile.  Per streamed row and chunk plane lane 0 issues one bulk
        // copy from the first to the last pixel that lies in the row (guard
        // pixels included where they are interior); a wrapped guard pixel is a
        // 16-byte cp.async by lane kc (a 16-byte bulk copy costs the copy
        // engine about as much as a 2 KB one).  Every lane then arrives on
        // full[slot] once its cp.async copies have landed.
        long long j = 0;
        RingPos rp(RING);
        RowCursor cur(u0, n, NB);
        bool ok = true;
        for (long long u = u0; u < u1 && ok; ++u, cur.next()) {
            const int y = cur.y;
            const long long f = cur.f;
            const bool start = (u == u0) || (y == 0);
            const int x0 = cur.cb * 128;
            const bool wl = x0 == 0, wr = x0 + 128 == n;
            const int bx = wl ? x0 : x0 - 1;                                  // first pixel of the bulk copy
            const uint32_t bbytes = uint32_t(130 - int(wl) - int(wr)) * 16u;  // its bytes
            const uint32_t boff = wl ? 16u : 0u;                              // its offset in the plane
            for (int k = start ? 0 : 2; k < 3; ++k) {
                int yin = y - 1 + k;
                yin = yin < 0 ? yin + n : (yin >= n ? yin - n : yin);
                const int slot = rp.idx;
                bool free_slot = true;
                if (lane == 0 && j >= RING) free_slot = p_wait(&ctl->empty[slot], rp.phase ^ 1u, abort_flag, status);
                if (!__shfl_sync(0xffffffffu, free_slot, 0)) {
                    ok = false;
                    break;
                }
                unsigned char* dst = ring + size_t(slot) * SLOT;
                const __nv_bfloat16* src = in + (size_t(f) * KC * nn + size_t(yin) * n) * 8;
                if (lane == 0) {
                    tc::mbar_arrive_expect_tx(&ctl->full[slot], uint32_t(KC) * bbytes);
                    for (int kc = 0; kc < KC; ++kc)
                        tc::bulk_g2s(dst + size_t(kc) * PLANE + boff, src + (size_t(kc) * nn + size_t(bx)) * 8, bbytes,
                                     &ctl->full[slot]);
                }
                if (lane < KC) {
                    unsigned char* d = dst + size_t(lane) * PLANE;
                    const __nv_bfloat16* r = src + size_t(lane) * nn * 8;
                    if (wl) cp_async16(d, r + size_t(n - 1) * 8);
                    if (wr) cp_async16(d + 129 * 16, r);
                }
                cp_async_arrive(&ctl->full[slot]);
                ++j;
                rp.next();
            }
        }
        // drain: every issued copy lands before the CTA may exit
        if (lane == 0)
            for (long long x = j > RING ? j - RING : 0; x < j; ++x)
                tc::mbar_wait_bounded(&ctl->full[x % RING], uint32_t((x / RING) & 1), kTcSpin);
        cp_async_wait_all();
        __syncwarp();
    } else {
        // ---- weights (permuted to [dx][kc][dy][cout][8]), bias, last-layer taps
        const uint4* wsrc = reinterpret_cast<const uint4*>(wpk);
        uint4* wdst = reinterpret_cast<uint4*>(w_tile);
        for (int e = tid - 32; e < 9 * KC * C; e += blockDim.x - 32) {
            const int co = e % C, kc = (e / C) % KC, tap = e / (C * KC);
            wdst[((tap % 3) * KC + kc) * N3 + (tap / 3) * C + co] = wsrc[e];
        }
        tc::fence_proxy_async_smem();
        if (tid - 32 < C) ctl->bias[tid - 32] = (mode != kDgrad) ? bias[tid - 32] : 0.f;
        if constexpr (mode == kFwdLast)
            for (int e = tid - 32; e < 10 * C; e += blockDim.x - 32) {
                const int tap = e % 10, c = e / 10;
                ctl->wl[e] = tap < 9 ? bf16r(wlast[c * 9 + tap]) : 0.f;
            }
        if (warp == 1) tc::tmem_alloc(&ctl->tmem, 512u);
        tc::fence_before_sync();
        tc::bar_sync(1, blockDim.x - 32);
        tc::fence_after_sync();
        const uint32_t tmem = ctl->tmem;

        if (warp == 1 || warp == 2) {
            if (lane == 0) {
                // ---- MMA issuers: warp 1 takes the even stream positions, warp 2
                // the odd ones, so that one issuer's waits and address
                // arithmetic overlap the other's MMAs
                const long long mine = warp - 1;
                bool ok = true;
                // test hook: a wait that cannot succeed, so the bounded-wait path runs
                if (stall > 0) ok = p_wait(&ctl->never, 0, abort_flag, status, stall);
                const uint32_t idesc = tc::idesc_bf16_f32(128, N3);
                const uint64_t a_hi = tc::smem_desc(0, PLANE, 128);
                const uint64_t b_hi = tc::smem_desc(0, N3 * 16, 128);
                // start-address fields count 16-byte units; one pixel (8 channels) is one unit
                const uint32_t ring_u = tc::smem_u32(ring) >> 4, w_u = tc::smem_u32(w_tile) >> 4;
                long long j = 0;
                RingPos rp(RING), dp(DS);
                int y = int(u0 % n);
                for (long long u = u0; u < u1 && ok; ++u, y = (y + 1 == n ? 0 : y + 1)) {
                    const bool start = (u == u0) || (y == 0);
                    for (int k = start ? 0 : 2; k < 3; ++k, ++j, rp.next(), dp.next()) {
                        if ((j & 1) != mine) continue;
                        const int slot = rp.idx;
                        const int ds = dp.idx;
                        if (j >= DS && !(ok = p_wait(&ctl->dempty[ds], dp.phase ^ 1u, abort_flag, status))) break;
                        if (!(ok = p_wait(&ctl->full[slot], rp.phase, abort_flag, status))) break;
                        // the guard pixels came by cp.async (generic proxy); the MMAs read
                        // the slot through the async proxy
                        tc::fence_proxy_async_smem();
                        tc::fence_after_sync();
                        const uint32_t in_u = ring_u + uint32_t(slot) * (SLOT >> 4);
                        const uint32_t d_addr = tmem + uint32_t(ds * DCOLS);
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                            for (int ks = 0; ks < C / 16; ++ks) {
                                const uint64_t ad = a_hi | uint64_t(in_u + uint32_t(dx) + uint32_t(2 * ks) * (PLANE >> 4));
                                const uint64_t bd = b_hi | uint64_t(w_u + uint32_t((dx * KC + 2 * ks) * N3));
                                tc::mma_bf16(d_addr, ad, bd, idesc, (dx | ks) != 0);
                            }
                        }
                        tc::mma_commit(&ctl->empty[slot]);
                        tc::mma_commit(&ctl->dfull[ds]);
                    }
                }
                // every MMA issued so far (by both issuers) completes before TMEM is freed
                tc::mma_commit(&ctl->fin);
                tc::mbar_wait_bounded(&ctl->fin, 0, kTcSpin);
            }
        } else if (warp >= 3) {
            // ---- epilogue
            const int q = warp & 3;         // TMEM lane quarter: pixels 32 q .. 32 q + 31
            const int g = (warp - 3) >> 2;  // chunk group: chunks g CPW .. g CPW + CPW - 1
            const f32x2* bias2 = reinterpret_cast<const f32x2*>(ctl->bias);
            f32x2 P[CPW][4], Pn[CPW][4];  // partial sums of output rows y and y + 1, channel pairs
#pragma unroll
            for (int c = 0; c < CPW; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) P[c][e] = Pn[c][e] = f2(0.f, 0.f);
            RingPos dp(DS);
            RowCursor cur(u0, n, NB);
            int rows_done = 0;
            bool ok = true;
            for (long long u = u0; u < u1 && ok; ++u, cur.next()) {
                const int y = cur.y;
                const long long f = cur.f;
                const bool start = (u == u0) || (y == 0);
                const size_t pix = size_t(y) * n + size_t(cur.cb * 128 + q * 32 + lane);
                for (int k = start ? 0 : 2; k < 3; ++k, dp.next()) {
                    const int ds = dp.idx;
                    if (!(ok = p_wait(&ctl->dfull[ds], dp.phase, abort_flag, status))) break;
                    tc::fence_after_sync();
                    const uint32_t trow = tmem + (uint32_t(q * 32) << 16) + uint32_t(ds * DCOLS);
                    f32x2 pt2[5];  // kFwdLast: the nine-tap projection, tap pairs
#pragma unroll
                    for (int m = 0; m < 5; ++m) pt2[m] = f2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < CPW; ++c) {
                        const int kc = g * CPW + c;
                        uint32_t v[3][8];
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy) tc::tmem_ld8(trow + uint32_t(dy * C + kc * 8), v[dy]);
                        tc::tmem_wait_ld();
                        if (c == CPW - 1) {
                            // the slot is in registers: the MMA issuer may refill it
                            tc::fence_before_sync();
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(&ctl->dempty[ds]);
                        }
                        f32x2 d[3][4];
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                d[dy][e] = f2(__uint_as_float(v[dy][2 * e]), __uint_as_float(v[dy][2 * e + 1]));
                        if (k == 2) {
                            // output row y is complete: ((D(y-1)[0] + b) + D(y)[1]) + D(y+1)[2]
                            const size_t off = ((size_t(f) * KC + kc) * nn + pix) * 8;
                            f32x2 z[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) z[e] = f2_add(P[c][e], d[2][e]);
                            uint32_t packed[4];
                            if constexpr (mode != kDgrad) {
                                float a8[8];
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    float a0, a1;
                                    f2split(act2<ACT>(z[e]), a0, a1);
                                    const __nv_bfloat162 hh = __floats2bfloat162_rn(a0, a1);
                                    packed[e] = *reinterpret_cast<const uint32_t*>(&hh);
                                    if constexpr (mode == kFwdLast) {
                                        a8[2 * e] = __low2float(hh);
                                        a8[2 * e + 1] = __high2float(hh);
                                    }
                                }
                                if (zio) {
                                    f32x2* z2 = reinterpret_cast<f32x2*>(zio + off);
#pragma unroll
                                    for (int e = 0; e < 4; ++e) z2[e] = z[e];
                                }
                                if constexpr (mode == kFwdLast) {
                                    // channels in order, taps in pairs: each tap's sum is the
                                    // same fma chain as one tap at a time
#pragma unroll
                                    for (int i = 0; i < 8; ++i) {
                                        const f32x2* w2 = reinterpret_cast<const f32x2*>(ctl->wl + (kc * 8 + i) * 10);
                                        const f32x2 ai = f2(a8[i], a8[i]);
#pragma unroll
                                        for (int m = 0; m < 5; ++m) pt2[m] = f2_fma(w2[m], ai, pt2[m]);
                                    }
                                }
                            } else {
                                const float4 za = reinterpret_cast<const float4*>(zio + off)[0];
                                const float4 zb = reinterpret_cast<const float4*>(zio + off)[1];
                                const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    float a0, a1;
                                    f2split(z[e], a0, a1);
                                    const __nv_bfloat162 hh = __floats2bfloat162_rn(a0 * act_grad_c<ACT>(zz[2 * e]),
                                                                                    a1 * act_grad_c<ACT>(zz[2 * e + 1]));
                                    packed[e] = *reinterpret_cast<const uint32_t*>(&hh);
                                }
                            }
                            // kFwdLast stores the activations only for training (zio)
                            if (mode != kFwdLast || zio)
                                *reinterpret_cast<uint4*>(out + off) =
                                    make_uint4(packed[0], packed[1], packed[2], packed[3]);
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            P[c][e] = f2_add(Pn[c][e], d[1][e]);
                            if constexpr (mode == kDgrad) Pn[c][e] = d[0][e];
                            else Pn[c][e] = f2_add(d[0][e], bias2[kc * 4 + e]);  // the bias enters first
                        }
                    }
                    if (mode == kFwdLast && k == 2) {
                        // the quarter's EPW partial projections, summed in warp order
                        const int par = rows_done & 1;
                        float* sc = scratch + size_t(par * 4 + q) * (4 * 9 * 32);
#pragma unroll
                        for (int m = 0; m < 5; ++m) {
                            float t0, t1;
                            f2split(pt2[m], t0, t1);
                            sc[(g * 9 + 2 * m) * 32 + lane] = t0;
                            if (m < 4) sc[(g * 9 + 2 * m + 1) * 32 + lane] = t1;
                        }
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&ctl->qbar[par][q]);
                        if (!(ok = p_wait(&ctl->qbar[par][q], uint32_t((rows_done >> 1) & 1), abort_flag,
                                          status)))
                            break;
                        for (int tp = g; tp < 9; tp += EPW) {
                            float s_ = sc[tp * 32 + lane];
#pragma unroll
                            for (int w = 1; w < EPW; ++w) s_ = __fadd_rn(s_, sc[(w * 9 + tp) * 32 + lane]);
                            maps[(size_t(f) * 9 + tp) * nn + pix] = s_;
                        }
                    }
                    if (k == 2) ++rows_done;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(ctl->tmem, 512u);
}

struct RShape {
    int RING = 0, DS = 0;
    size_t smem = 0;
};

// ring_mode: 0 as deep as shared memory allows (up to kRMaxRing slots),
// 1 at most 12, 2 at most 6; ds: TMEM slots (0: as many as fit, up to kRMaxD).
static RShape r_shape_with(int n, int C, int ring_mode, int ds, bool last) {
    RShape s;
    if (n < 128 || n % 128 || !(C == 16 || C == 32 || C == 64)) return s;
    const int dmax = std::min(kRMaxD, 512 / r_dcols(C));
    s.DS = ds ? ds : dmax;
    if (s.DS < 2 || s.DS > dmax) return RShape{};
    const size_t fixed = size_t(9) * C * C * 2 + kRCtlBytes + (last ? kRScratchBytes : 0);
    int ring = int((size_t(227) * 1024 - fixed) / r_slot_bytes(C));
    ring = std::min(ring, kRMaxRing);
    if (ring_mode == 1) ring = std::min(ring, 12);
    if (ring_mode == 2) ring = std::min(ring, 6);
    if (ring < 2) return RShape{};
    s.RING = ring;
    s.smem = fixed + size_t(ring) * r_slot_bytes(C);
    // one CTA per SM: it owns all 512 TMEM columns
    if (s.smem < size_t(116) * 1024) s.smem = size_t(116) * 1024;
    return s;
}

// Shape of the row-streaming kernel per (channels, log2 n): index into
// conv_variants() (-1: automatic, the first).  A shape is a ring depth mode
// and a TMEM slot count; every shape gives the same bits.
namespace {
int g_conv_pick[3][11] = {{-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                          {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                          {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1}};
int cidx(int C) { return C == 16 ? 0 : (C == 32 ? 1 : 2); }
int lg2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
struct ConvVariant { int ring_mode, ds; };
constexpr ConvVariant kConvVariants[] = {{0, 0}, {1, 0}, {2, 0}, {0, 2}, {0, 3}, {1, 2}};
constexpr int kConvVariantCount = int(sizeof(kConvVariants) / sizeof(kConvVariants[0]));
}  // namespace

// The valid, distinct shapes for (n, C), in kConvVariants order.
static int conv_variants(int n, int C, int* out) {
    int cnt = 0;
    RShape seen[kConvVariantCount];
    for (int i = 0; i < kConvVariantCount; ++i) {
        const RShape r = r_shape_with(n, C, kConvVariants[i].ring_mode, kConvVariants[i].ds, false);
        if (!r.RING) continue;
        bool dup = false;
        for (int k = 0; k < cnt; ++k) dup = dup || (seen[k].RING == r.RING && seen[k].DS == r.DS);
        if (dup) continue;
        seen[cnt] = r;
        out[cnt++] = i;
    }
    return cnt;
}

// The shape a hidden layer of (n, C) runs with (RING 0: the one-shot kernel);
// `last` leaves room for the fused last layer's reduction scratch.
static RShape conv_plan(int n, int C, bool last) {
    const int pick = (C == 16 || C == 32 || C == 64) && n >= 1 && n <= 1024 ? g_conv_pick[cidx(C)][lg2(n)] : -1;
    int idx[kConvVariantCount];
    const int cnt = conv_variants(n, C, idx);
    if (cnt == 0) return RShape{};
    const ConvVariant v = kConvVariants[idx[pick >= 0 && pick < cnt ? pick : 0]];
    return r_shape_with(n, C, v.ring_mode, v.ds, last);
}

int conv_variant_count(int n, int C) {
    if (!(C == 16 || C == 32 || C == 64) || n < 1 || n > 1024) return 0;
    int idx[kConvVariantCount];
    return conv_variants(n, C, idx);
}

int conv_variant_describe(int n, int C, int index, int* ring, int* slots) {
    int idx[kConvVariantCount];
    const int cnt = conv_variant_count(n, C) ? conv_variants(n, C, idx) : 0;
    if (index < 0 || index >= cnt) return AC_ERR_ARG;
    const RShape r = r_shape_with(n, C, kConvVariants[idx[index]].ring_mode, kConvVariants[idx[index]].ds, false);
    *ring = r.RING;
    *slots = r.DS;
    return AC_OK;
}

int conv_set_variant(int n, int C, int index) {
    ACPR_CHECK_ARG(C == 16 || C == 32 || C == 64, "channels must be 16, 32 or 64");
    ACPR_CHECK_ARG(n >= 1 && n <= 1024 && (n & (n - 1)) == 0, "n must be a power of two <= 1024");
    ACPR_CHECK_ARG(index >= -1 && index < conv_variant_count(n, C), "variant %d out of range", index);
    g_conv_pick[cidx(C)][lg2(n)] = index;
    return AC_OK;
}

int conv_get_variant(int n, int C) {
    if (!(C == 16 || C == 32 || C == 64) || n < 1 || n > 1024) return -1;
    return g_conv_pick[cidx(C)][lg2(n)];
}

static int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 1;
    }
    return sms;
}

template <int C, int ACT, int MODE>
static int launch_rows_mode(const RShape& s, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                            const __nv_bfloat16* w, const float* bias, float* zio, int* status, cudaStream_t st,
                            const float* wlast, float* maps) {
    auto kern = conv_rows_tc<C, ACT, MODE>;
    static bool configured = false;
    if (!configured) {
        ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(227 * 1024)));
        configured = true;
    }
    const long long units = (long long)batch * (n / 128) * n;
    const int grid = int(units < num_sms() ? units : num_sms());
    kern<<<grid, RGeom<C>::THREADS, s.smem, st>>>(in, out, w, bias, n, batch, s.RING, s.DS, zio, status,
                                                  g_test_stall, wlast, maps);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

template <int C, int ACT>
static int launch_rows_act(const RShape& s, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                           const __nv_bfloat16* w, const float* bias, int mode, float* zio, int* status,
                           cudaStream_t st, const float* wlast, float* maps) {
    if (mode == kDgrad)
        return launch_rows_mode<C, ACT, kDgrad>(s, n, batch, in, out, w, bias, zio, status, st, wlast, maps);
    if constexpr (C >= 32)
        if (mode == kFwdLast)
            return launch_rows_mode<C, ACT, kFwdLast>(s, n, batch, in, out, w, bias, zio, status, st, wlast, maps);
    return launch_rows_mode<C, ACT, kFwd>(s, n, batch, in, out, w, bias, zio, status, st, wlast, maps);
}

template <int C>
static int launch_rows(const RShape& r, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                       const __nv_bfloat16* w, const float* bias, int act, int mode, float* zio, int* status,
                       cudaStream_t st, const float* wlast = nullptr, float* maps = nullptr) {
    if (act == AC_ACT_TANH)
        return launch_rows_act<C, AC_ACT_TANH>(r, n, batch, in, out, w, bias, mode, zio, status, st, wlast, maps);
    return launch_rows_act<C, AC_ACT_GELU>(r, n, batch, in, out, w, bias, mode, zio, status, st, wlast, maps);
}

template <int C>
static int launch_hidden(int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out, const __nv_bfloat16* w,
                         const float* bias, int act, int mode, float* zio, int* status, cudaStream_t st) {
    if (batch <= 0) return AC_OK;
    if (!status) {
        set_error("tensor-core conv: no status word");
        return AC_ERR_ARG;
    }
    const RShape plan = conv_plan(n, C, false);
    if (plan.RING) return launch_rows<C>(plan, n, batch, in, out, w, bias, act, mode, zio, status, st);
    const TcShape s = pick_shape(n, C);
    if (s.TY == 0) return AC_ERR_UNSUPPORTED;
    auto kern = act == AC_ACT_TANH ? conv_hidden_tc_kernel<C, AC_ACT_TANH> : conv_hidden_tc_kernel<C, AC_ACT_GELU>;
    static bool configured[2] = {false, false};
    if (!configured[act == AC_ACT_TANH]) {
        ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(227 * 1024)));
        configured[act == AC_ACT_TANH] = true;
    }
    const long long blocks = (long long)batch * (n / s.TY);
    kern<<<unsigned(blocks), kTcThreads, s.smem, st>>>(in, out, w, bias, n, s.TY, s.n_mt, s.plane_px, s.ncols, mode,
                                                       zio, status);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

int hidden_layer_bf16(const cnn_desc* d, int l, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                      const float* /*w_master*/, const float* bias, int* status, cudaStream_t st, float* zsave) {
    if (n < 8) return AC_ERR_UNSUPPORTED;
    const int C = d->channels;
    const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(d->packed) + size_t(l - 1) * 9 * C * C;
    switch (C) {
        case 16: return launch_hidden<16>(n, batch, in, out, w, bias, d->act, kFwd, zsave, status, st);
        case 32: return launch_hidden<32>(n, batch, in, out, w, bias, d->act, kFwd, zsave, status, st);
        case 64: return launch_hidden<64>(n, batch, in, out, w, bias, d->act, kFwd, zsave, status, st);
        default: return AC_ERR_UNSUPPORTED;
    }
}

bool hidden_last_fused_supported(int n, int C) { return C >= 32 && C <= 64 && conv_plan(n, C, true).RING > 0; }

int hidden_last_fused(const cnn_desc* d, int l, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* act_out,
                      const float* bias, const float* w_last, float* maps, int* status, cudaStream_t st,
                      float* zsave) {
    const int C = d->channels;
    if (batch <= 0) return AC_OK;
    if (!hidden_last_fused_supported(n, C)) return AC_ERR_UNSUPPORTED;
    if (!status) {
        set_error("tensor-core conv: no status word");
        return AC_ERR_ARG;
    }
    const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(d->packed) + size_t(l - 1) * 9 * C * C;
    const RShape plan = conv_plan(n, C, true);
    if (C == 32)
        return launch_rows<32>(plan, n, batch, in, act_out, w, bias, d->act, kFwdLast, zsave, status, st, w_last, maps);
    return launch_rows<64>(plan, n, batch, in, act_out, w, bias, d->act, kFwdLast, zsave, status, st, w_last, maps);
}

int hidden_dgrad_bf16(int C, int act, int n, int batch, const __nv_bfloat16* dz_next, __nv_bfloat16* dz_out,
                      const __nv_bfloat16* w_t, const float* z_prev, int* status, cudaStream_t st) {
    if (n < 8) return AC_ERR_UNSUPPORTED;
    float* zp = const_cast<float*>(z_prev);
    switch (C) {
        case 16: return launch_hidden<16>(n, batch, dz_next, dz_out, w_t, nullptr, act, kDgrad, zp, status, st);
        case 32: return launch_hidden<32>(n, batch, dz_next, dz_out, w_t, nullptr, act, kDgrad, zp, status, st);
        case 64: return launch_hidden<64>(n, batch, dz_next, dz_out, w_t, nullptr, act, kDgrad, zp, status, st);
        default: return AC_ERR_UNSUPPORTED;
    }
}

// float32 master W[cout][cin][3][3] -> bf16 [tap][cout/8][cin][8] of the
// channel-transposed, tap-flipped kernel: the B operand of the dgrad GEMM.
__global__ void pack_hidden_t_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ out, int C) {
    const int total = 9 * C * C;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int i = idx % 8;                     // old output channel within its chunk
        const int c = (idx / 8) % C;               // new output channel = old input channel
        const int oc = (idx / (8 * C)) % (C / 8);  // chunk of old output channels
        const int tap = idx / (8 * C * (C / 8));
        const int o = oc * 8 + i;
        out[idx] = __float2bfloat16_rn(w[(o * C + c) * 9 + (8 - tap)]);
    }
}

int pack_hidden_t(int C, const float* w_layer, __nv_bfloat16* out, cudaStream_t st) {
    pack_hidden_t_kernel<<<64, 256, 0, st>>>(w_layer, out, C);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

}  // namespace acpr
