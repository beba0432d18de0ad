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
#include "cnn.cuh"
#include "tc_ptx.cuh"

namespace acpr {

namespace {
constexpr int kTcThreads = 256;
constexpr long long kTcSpin = 4000000;  // ~0.2 s of polls with 32 ns sleeps
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

// ------------------------------------------------------------ persistent --
// Persistent, warp-specialised form of the same GEMM for n >= 128 (n a
// multiple of 128), one CTA per SM.  Work unit = (field f, column block cb,
// row block yb): TY output rows y0 = yb TY .. y0 + TY - 1, each cut into MG
// M-tiles of 128 consecutive positions, columns [cb CW, cb CW + CW),
// CW = 128 MG.  Units are ordered (f, cb, yb) and CTA c takes a contiguous
// range of them, so consecutive units of a CTA mostly slide down TY rows and
// need TY new input rows.
//   warp 0 (lane 0), producer: input row segments (the CW columns of a row
//     plus one wrapped pixel on each side, all C/8 chunk planes) into a ring
//     of RING slots by cp.async.bulk, each completing on full[slot];
//   warp 1 (lane 0), MMA issuer: for tap (dy, dx) the A operand of output row
//     y0 + r, M-tile m, is slot(row y0 + r - 1 + dy) read from pixel
//     m*128 + dx, so an M-tile never leaves its slot.  The TY * MG
//     accumulators of a unit fill one of two TMEM stages of 256 columns.
//     Descriptors are formed by integer adds on their start-address field, so
//     issuing an MMA costs a few instructions.  tcgen05.commit marks the stage
//     full and releases (empty[slot]) the input rows no later unit reads;
//   warps 2..17, epilogue: tcgen05.ld of the stage, bias + activation (or the
//     act' product), bf16 16-byte stores; then the stage is marked empty.
// Loads of later rows, MMAs of the next unit and the epilogue of the current
// one overlap.  Every output is the same sum in the same order (tap, then
// K-step) as in the one-shot kernel, so both produce the same bits.  Every
// wait is bounded and also stops once another role has given up (abort flag
// in shared memory); before exit the CTA drains its in-flight copies and MMAs
// and frees TMEM.
constexpr int kPEpiWarps = 16;
constexpr int kPThreads = 32 * (2 + kPEpiWarps);
constexpr int kPStages = 2;
constexpr int kPStageCols = 256;
constexpr int kPMaxRing = 16;

struct PShape {
    int MG = 0, CW = 0, TY = 0, RING = 0;
    int areuse = 0;  // MMAs that share an input row read its A operand once (collector buffer)
    uint32_t slot_bytes = 0;
    size_t smem = 0;
};

// Tile shape: mg = M-tiles per row segment (0: automatic), ring_mode = depth
// of the input-row ring (0: one unit of prefetch, 2 TY + 2 rows; 1: no
// prefetch, TY + 2; 2: as deep as shared memory allows, up to kPMaxRing).
static PShape p_shape_with(int n, int C, int mg, int ring_mode, int areuse = 0) {
    PShape s;
    s.areuse = areuse;
    if (n < 128 || n % 128) return s;
    // C = 64 keeps one M-tile per row so that a ring slot stays small
    s.MG = mg ? mg : ((C >= 64 || n < 256) ? 1 : 2);
    if (s.MG < 1 || s.MG > 2 || (s.MG == 2 && (C >= 64 || n < 256))) return PShape{};
    s.CW = 128 * s.MG;
    s.TY = kPStageCols / (s.MG * C);
    if (s.TY < 1 || n % s.TY) return PShape{};
    s.slot_bytes = uint32_t(C / 8) * uint32_t(s.CW + 2) * 16u;
    const size_t wbytes = size_t(9) * C * C * 2;
    const size_t ctrl = 4096;  // PCtl
    const size_t avail = size_t(227) * 1024 - wbytes - ctrl;
    int ring = int(avail / s.slot_bytes);
    if (ring > kPMaxRing) ring = kPMaxRing;
    if (ring_mode == 0 && ring > 2 * s.TY + 2) ring = 2 * s.TY + 2;  // one unit of prefetch
    if (ring_mode == 1 && ring > s.TY + 2) ring = s.TY + 2;
    if (ring < s.TY + 2) return PShape{};
    s.RING = ring;
    s.smem = wbytes + size_t(ring) * s.slot_bytes + ctrl;
    // more than half an SM's shared memory: at most one such CTA per SM, so
    // the CTAs' TMEM stages (all 512 columns) never contend
    if (s.smem < size_t(116) * 1024) s.smem = size_t(116) * 1024;
    return s;
}

// Tile shapes a tuner may pick, per (channels, log2 n): index into
// conv_variants() (-1: automatic).
namespace {
int g_conv_pick[3][11] = {{-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                          {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                          {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1}};
int cidx(int C) { return C == 16 ? 0 : (C == 32 ? 1 : 2); }
int lg2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
struct ConvVariant { int mg, ring_mode, areuse; };
constexpr ConvVariant kConvVariants[] = {{0, 0, 0}, {1, 0, 0}, {2, 0, 0}, {1, 1, 0}, {2, 1, 0}, {1, 2, 0}, {2, 2, 0},
                                         {0, 0, 1}, {1, 0, 1}, {2, 0, 1}, {1, 2, 1}, {2, 2, 1}};
constexpr int kConvVariantCount = int(sizeof(kConvVariants) / sizeof(kConvVariants[0]));
}  // namespace

// The valid, distinct shapes for (n, C), in kConvVariants order.
static int conv_variants(int n, int C, int* out) {
    int cnt = 0;
    PShape seen[kConvVariantCount];
    for (int i = 0; i < kConvVariantCount; ++i) {
        const PShape s = p_shape_with(n, C, kConvVariants[i].mg, kConvVariants[i].ring_mode, kConvVariants[i].areuse);
        if (!s.RING) continue;
        bool dup = false;
        for (int k = 0; k < cnt; ++k)
            dup = dup || (seen[k].MG == s.MG && seen[k].RING == s.RING && seen[k].areuse == s.areuse);
        if (dup) continue;
        seen[cnt] = s;
        out[cnt++] = i;
    }
    return cnt;
}

static PShape p_shape(int n, int C) {
    const int pick = (C == 16 || C == 32 || C == 64) && n >= 1 && n <= 1024 ? g_conv_pick[cidx(C)][lg2(n)] : -1;
    if (pick >= 0) {
        int idx[kConvVariantCount];
        const int cnt = conv_variants(n, C, idx);
        if (pick < cnt) {
            const ConvVariant v = kConvVariants[idx[pick]];
            return p_shape_with(n, C, v.mg, v.ring_mode, v.areuse);
        }
    }
    return p_shape_with(n, C, 0, 0);
}

int conv_variant_count(int n, int C) {
    if (!(C == 16 || C == 32 || C == 64) || n < 1 || n > 1024) return 0;
    int idx[kConvVariantCount];
    return conv_variants(n, C, idx);
}

int conv_variant_describe(int n, int C, int index, int* mg, int* ty, int* ring, int* areuse) {
    int idx[kConvVariantCount];
    const int cnt = conv_variant_count(n, C) ? conv_variants(n, C, idx) : 0;
    if (index < 0 || index >= cnt) return AC_ERR_ARG;
    const ConvVariant v = kConvVariants[idx[index]];
    const PShape s = p_shape_with(n, C, v.mg, v.ring_mode, v.areuse);
    *mg = s.MG;
    *ty = s.TY;
    *ring = s.RING;
    *areuse = s.areuse;
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

struct PCtl {
    uint64_t never;  // test hook: nothing ever arrives here
    uint64_t full[kPMaxRing];
    uint64_t empty[kPMaxRing];
    uint64_t accf[kPStages];
    uint64_t acce[kPStages];
    uint64_t wbar;  // the weight copy
    uint64_t fin;   // completion of every MMA the CTA issued
    uint32_t tmem;
    int abort;
    alignas(16) float bias[64];
    alignas(16) float wl[64 * 9];  // kFwdLast: bf16-rounded last-layer weights [kc][tap][8]
};

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

template <int C, int MG, int ACT>
__global__ void __launch_bounds__(kPThreads, 1)
conv_hidden_tc_persistent(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          const __nv_bfloat16* __restrict__ wpk, const float* __restrict__ bias, int n,
                          int batch, int RING, uint32_t slot_bytes, int mode, float* __restrict__ zio,
                          int* __restrict__ status, int stall, const float* __restrict__ wlast,
                          float* __restrict__ maps, int areuse) {
    constexpr int KC = C / 8;
    constexpr int TY = kPStageCols / (MG * C);
    constexpr int NACC = TY * MG;
    constexpr int CW = 128 * MG;
    constexpr uint32_t WBYTES = 9u * C * C * 2u;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* w_tile = smem;
    unsigned char* ring = smem + WBYTES;
    PCtl* ctl = reinterpret_cast<PCtl*>(ring + size_t(RING) * slot_bytes);
    volatile int* abort_flag = &ctl->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NB = n / CW;
    const int NYB = n / TY;
    const uint32_t plane_b = uint32_t(CW + 2) * 16u;
    const size_t nn = size_t(n) * n;
    const long long total = (long long)batch * NB * NYB;
    const long long u0 = total * blockIdx.x / gridDim.x;
    const long long u1 = total * (blockIdx.x + 1) / gridDim.x;

    if (tid == 0) {
        for (int i = 0; i < RING; ++i) {
            tc::mbar_init(&ctl->full[i], 1);
            tc::mbar_init(&ctl->empty[i], 1);
        }
        for (int i = 0; i < kPStages; ++i) {
            tc::mbar_init(&ctl->accf[i], 1);
            tc::mbar_init(&ctl->acce[i], kPEpiWarps);
        }
        tc::mbar_init(&ctl->wbar, 1);
        tc::mbar_init(&ctl->fin, 1);
        tc::mbar_init(&ctl->never, 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
    }
    static_assert(sizeof(PCtl) <= 4096, "control block");
    if (tid < C) ctl->bias[tid] = (mode != kDgrad) ? bias[tid] : 0.f;
    if (mode == kFwdLast)
        for (int e = tid; e < 9 * C; e += blockDim.x) {
            // wl[kc][tap][i] = bf16(W_last[0][kc 8 + i][tap])
            const int i = e % 8, tap = (e / 8) % 9, kc = e / 72;
            ctl->wl[e] = bf16r(wlast[(kc * 8 + i) * 9 + tap]);
        }
    __syncthreads();
    if (warp == 1) tc::tmem_alloc(&ctl->tmem, uint32_t(kPStages * kPStageCols));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0 && lane == 0) {
        // ---- producer
        tc::mbar_arrive_expect_tx(&ctl->wbar, WBYTES);
        tc::bulk_g2s(w_tile, wpk, WBYTES, &ctl->wbar);
        long long s = 0;
        bool ok = true;
        for (long long u = u0; u < u1 && ok; ++u) {
            const int yb = int(u % NYB);
            const long long t = u / NYB;
            const int cb = int(t % NB);
            const long long f = t / NB;
            const int y0 = yb * TY;
            const bool start = (u == u0) || (yb == 0);
            // input rows y0 - 1 .. y0 + TY (segment start) or y0 + 1 .. y0 + TY
            for (int r = start ? -1 : 1; r <= TY && ok; ++r) {
                int yin = y0 + r;
                yin = yin < 0 ? yin + n : (yin >= n ? yin - n : yin);
                const int slot = int(s % RING);
                const long long k = s / RING;
                if (k >= 1 && !p_wait(&ctl->empty[slot], uint32_t((k - 1) & 1), abort_flag, status)) {
                    ok = false;
                    break;
                }
                tc::mbar_arrive_expect_tx(&ctl->full[slot], uint32_t(KC) * plane_b);
                const int x0 = cb * CW;
                const int xl = x0 == 0 ? n - 1 : x0 - 1;
                const int xr = x0 + CW == n ? 0 : x0 + CW;
                for (int kc = 0; kc < KC; ++kc) {
                    const __nv_bfloat16* src = in + ((size_t(f) * KC + kc) * nn + size_t(yin) * n) * 8;
                    unsigned char* dst = ring + size_t(slot) * slot_bytes + size_t(kc) * plane_b;
                    tc::bulk_g2s(dst + 16, src + size_t(x0) * 8, uint32_t(CW) * 16u, &ctl->full[slot]);
                    tc::bulk_g2s(dst, src + size_t(xl) * 8, 16u, &ctl->full[slot]);
                    tc::bulk_g2s(dst + size_t(CW + 1) * 16, src + size_t(xr) * 8, 16u, &ctl->full[slot]);
                }
                ++s;
            }
        }
        // drain: every issued copy lands before the CTA may exit
        const long long first = s > RING ? s - RING : 0;
        for (long long x = first; x < s; ++x)
            tc::mbar_wait_bounded(&ctl->full[x % RING], uint32_t((x / RING) & 1), kTcSpin);
        tc::mbar_wait_bounded(&ctl->wbar, 0, kTcSpin);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        bool ok = p_wait(&ctl->wbar, 0, abort_flag, status);
        // test hook: a wait that cannot succeed, so the bounded-wait path runs
        if (ok && stall > 0) ok = p_wait(&ctl->never, 0, abort_flag, status, stall);
        const uint32_t idesc = tc::idesc_bf16_f32(128, C);
        const uint64_t a_hi = tc::smem_desc(0, plane_b, 128);
        const uint64_t b_hi = tc::smem_desc(0, C * 16, 128);
        // start-address fields count 16-byte units; one pixel (8 channels) is one unit
        const uint32_t ring_u = tc::smem_u32(ring) >> 4, w_u = tc::smem_u32(w_tile) >> 4;
        const uint32_t slot_u = slot_bytes >> 4, plane_u = plane_b >> 4;
        int a = 0, snext = 0;  // load index of the unit's first input row (a CTA's loads are few)
        int i = 0;
        for (long long u = u0; u < u1 && ok; ++u, ++i) {
            const int yb = int(u % NYB);
            const bool start = (u == u0) || (yb == 0);
            if (start) {
                a = snext;
                snext += TY + 2;
            } else {
                a += TY;
                snext += TY;
            }
            const int stage = i & 1;
            const int kk = i >> 1;
            if (kk >= 1 && !p_wait(&ctl->acce[stage], uint32_t((kk - 1) & 1), abort_flag, status)) break;
            const int aslot = a % RING;
            for (int d = 0; d < TY + 2 && ok; ++d)
                ok = p_wait(&ctl->full[(a + d) % RING], uint32_t(((a + d) / RING) & 1), abort_flag, status);
            if (!ok) break;
            tc::fence_after_sync();
            const uint32_t dbase = tmem + uint32_t(stage * kPStageCols);
            if (areuse) {
                // input row rho of the unit serves output rows rho - dy (dy =
                // 0, 1, 2): its A operand (shift dx, K-step ks, M-tile m) is
                // read into the collector once and used for up to three MMAs.
                // Each accumulator still receives its MMAs in (tap, K-step)
                // order, so the sums are those of the loop below, bit for bit.
#pragma unroll 1
                for (int rho = 0; rho < TY + 2; ++rho) {
                    int sl = aslot + rho;
                    sl = sl >= RING ? sl - RING : sl;
                    const uint32_t in_u = ring_u + uint32_t(sl) * slot_u;
                    const int dy_lo = rho - (TY - 1) > 0 ? rho - (TY - 1) : 0;
                    const int dy_hi = rho < 2 ? rho : 2;
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                        for (int ks = 0; ks < C / 16; ++ks) {
#pragma unroll
                            for (int m = 0; m < MG; ++m) {
                                const uint64_t ad = a_hi | uint64_t(in_u + uint32_t(dx) + uint32_t(2 * ks) * plane_u +
                                                                    uint32_t(m * 128));
#pragma unroll
                                for (int dy = 0; dy < 3; ++dy) {
                                    if (dy < dy_lo || dy > dy_hi) continue;
                                    const int tap = dy * 3 + dx;
                                    const int acc = (rho - dy) * MG + m;
                                    const uint64_t bd = b_hi | uint64_t(w_u + uint32_t((tap * KC + 2 * ks) * C));
                                    const uint32_t d_addr = dbase + uint32_t(acc * C);
                                    const uint32_t accum = (tap | ks) != 0;
                                    if (dy_lo == dy_hi) tc::mma_bf16(d_addr, ad, bd, idesc, accum);
                                    else if (dy == dy_lo) tc::mma_bf16_coll<1>(d_addr, ad, bd, idesc, accum);
                                    else if (dy == dy_hi) tc::mma_bf16_coll<3>(d_addr, ad, bd, idesc, accum);
                                    else tc::mma_bf16_coll<2>(d_addr, ad, bd, idesc, accum);
                                }
                            }
                        }
                    }
                }
            } else
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap % 3;
                // start of each output row's input row for this tap
                uint32_t row_u[TY];
#pragma unroll
                for (int r = 0; r < TY; ++r) {
                    int sl = aslot + r + dy;
                    sl = sl >= RING ? sl - RING : sl;
                    row_u[r] = ring_u + uint32_t(sl) * slot_u + uint32_t(dx);
                }
#pragma unroll
                for (int ks = 0; ks < C / 16; ++ks) {
                    const uint64_t bd = b_hi | uint64_t(w_u + uint32_t((tap * KC + 2 * ks) * C));
#pragma unroll
                    for (int acc = 0; acc < NACC; ++acc) {
                        const int r = acc / MG, m = acc % MG;
                        const uint64_t ad =
                            a_hi | uint64_t(row_u[r] + uint32_t(2 * ks) * plane_u + uint32_t(m * 128));
                        tc::mma_bf16(dbase + uint32_t(acc * C), ad, bd, idesc, (tap | ks) != 0);
                    }
                }
            }
            tc::mma_commit(&ctl->accf[stage]);
            const bool cont = (u + 1 < u1) && (yb != NYB - 1);
            const int nrel = cont ? TY : TY + 2;
            for (int d = 0; d < nrel; ++d) tc::mma_commit(&ctl->empty[(a + d) % RING]);
        }
        // every MMA issued so far completes before TMEM is freed
        tc::mma_commit(&ctl->fin);
        tc::mbar_wait_bounded(&ctl->fin, 0, kTcSpin);
    } else if (warp >= 2) {
        // ---- epilogue: kPEpiWarps warps in kPEpiWarps / 4 groups; a warp
        // reads TMEM lanes 32 (warp % 4) .. + 31 (one pixel per lane of an
        // M-tile) and owns its group's accumulators acc = grp, grp + NG, ...:
        // all C channels of its pixel come in W-column TMEM loads (one wait
        // per W channels), then bias + activation (or the act' product),
        // bf16, 16-byte stores per 8-channel chunk.  kFwdLast also projects
        // the pixel's activations onto the last layer's nine taps.
        constexpr int NG = kPEpiWarps / 4;
        constexpr int W = 16;
        const int grp = (warp - 2) >> 2;
        const int q = warp & 3;
        const float4* bias4 = reinterpret_cast<const float4*>(ctl->bias);
        int i = 0;
        for (long long u = u0; u < u1; ++u, ++i) {
            const int yb = int(u % NYB);
            const long long t = u / NYB;
            const int cb = int(t % NB);
            const long long f = t / NB;
            const int stage = i & 1;
            if (!p_wait(&ctl->accf[stage], uint32_t((i >> 1) & 1), abort_flag, status)) break;
            tc::fence_after_sync();
            const size_t pix0 = size_t(yb * TY) * n + size_t(cb * CW + q * 32 + lane);
            const uint32_t trow = tmem + (uint32_t(q * 32) << 16) + uint32_t(stage * kPStageCols);
            for (int acc = grp; acc < NACC; acc += NG) {
                const int r = acc / MG, m = acc % MG;
                const size_t pix = pix0 + size_t(r) * n + size_t(m) * 128;
                float pt[9];
#pragma unroll
                for (int tp = 0; tp < 9; ++tp) pt[tp] = 0.f;
#pragma unroll 1
                for (int kc0 = 0; kc0 < KC; kc0 += W / 8) {
                    uint32_t v[W];
                    tc::tmem_ldw<W>(trow + uint32_t(acc * C + kc0 * 8), v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int h = 0; h < W / 8; ++h) {
                        const int kc = kc0 + h;
                        const size_t off = ((size_t(f) * KC + kc) * nn + pix) * 8;
                        uint32_t packed[4];
                        if (mode != kDgrad) {
                            const float4 b0 = bias4[kc * 2], b1 = bias4[kc * 2 + 1];
                            __align__(16) float z8[8] = {
                                __uint_as_float(v[h * 8 + 0]) + b0.x, __uint_as_float(v[h * 8 + 1]) + b0.y,
                                __uint_as_float(v[h * 8 + 2]) + b0.z, __uint_as_float(v[h * 8 + 3]) + b0.w,
                                __uint_as_float(v[h * 8 + 4]) + b1.x, __uint_as_float(v[h * 8 + 5]) + b1.y,
                                __uint_as_float(v[h * 8 + 6]) + b1.z, __uint_as_float(v[h * 8 + 7]) + b1.w};
                            float a8[8];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const __nv_bfloat162 hh = __floats2bfloat162_rn(act_c<ACT>(z8[2 * e]),
                                                                                act_c<ACT>(z8[2 * e + 1]));
                                packed[e] = *reinterpret_cast<const uint32_t*>(&hh);
                                a8[2 * e] = __low2float(hh);
                                a8[2 * e + 1] = __high2float(hh);
                            }
                            if (zio) {
                                reinterpret_cast<float4*>(zio + off)[0] = *reinterpret_cast<const float4*>(z8);
                                reinterpret_cast<float4*>(zio + off)[1] = *reinterpret_cast<const float4*>(z8 + 4);
                            }
                            if (mode == kFwdLast) {
                                const float4* wl4 = reinterpret_cast<const float4*>(ctl->wl + kc * 72);
#pragma unroll
                                for (int tp = 0; tp < 9; ++tp) {
                                    const float4 w0 = wl4[tp * 2], w1 = wl4[tp * 2 + 1];
                                    float s_ = pt[tp];
                                    s_ = fmaf(w0.x, a8[0], s_);
                                    s_ = fmaf(w0.y, a8[1], s_);
                                    s_ = fmaf(w0.z, a8[2], s_);
                                    s_ = fmaf(w0.w, a8[3], s_);
                                    s_ = fmaf(w1.x, a8[4], s_);
                                    s_ = fmaf(w1.y, a8[5], s_);
                                    s_ = fmaf(w1.z, a8[6], s_);
                                    s_ = fmaf(w1.w, a8[7], s_);
                                    pt[tp] = s_;
                                }
                            }
                        } else {
                            const float4 za = reinterpret_cast<const float4*>(zio + off)[0];
                            const float4 zb = reinterpret_cast<const float4*>(zio + off)[1];
                            const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const __nv_bfloat162 hh = __floats2bfloat162_rn(
                                    __uint_as_float(v[h * 8 + 2 * e]) * act_grad_c<ACT>(zz[2 * e]),
                                    __uint_as_float(v[h * 8 + 2 * e + 1]) * act_grad_c<ACT>(zz[2 * e + 1]));
                                packed[e] = *reinterpret_cast<const uint32_t*>(&hh);
                            }
                        }
                        // kFwdLast stores the activations only for training (zio)
                        if (mode != kFwdLast || zio)
                            *reinterpret_cast<uint4*>(out + off) =
                                make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    }
                }
                if (mode == kFwdLast) {
#pragma unroll
                    for (int tp = 0; tp < 9; ++tp) maps[(size_t(f) * 9 + tp) * nn + pix] = pt[tp];
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&ctl->acce[stage]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, uint32_t(kPStages * kPStageCols));
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

template <int C, int MG, int ACT>
static int launch_persistent_act(const PShape& s, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                                 const __nv_bfloat16* w, const float* bias, int mode, float* zio, int* status,
                                 cudaStream_t st, const float* wlast, float* maps) {
    auto kern = conv_hidden_tc_persistent<C, MG, ACT>;
    static bool configured = false;
    if (!configured) {
        ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(227 * 1024)));
        configured = true;
    }
    const long long units = (long long)batch * (n / s.CW) * (n / s.TY);
    const int grid = int(units < num_sms() ? units : num_sms());
    kern<<<grid, kPThreads, s.smem, st>>>(in, out, w, bias, n, batch, s.RING, s.slot_bytes, mode, zio, status,
                                          g_test_stall, wlast, maps, s.areuse);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

template <int C, int MG>
static int launch_persistent_mg(const PShape& s, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                                const __nv_bfloat16* w, const float* bias, int act, int mode, float* zio,
                                int* status, cudaStream_t st, const float* wlast = nullptr, float* maps = nullptr) {
    if (act == AC_ACT_TANH)
        return launch_persistent_act<C, MG, AC_ACT_TANH>(s, n, batch, in, out, w, bias, mode, zio, status, st, wlast,
                                                         maps);
    return launch_persistent_act<C, MG, AC_ACT_GELU>(s, n, batch, in, out, w, bias, mode, zio, status, st, wlast,
                                                     maps);
}

template <int C>
static int launch_persistent(const PShape& s, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                             const __nv_bfloat16* w, const float* bias, int act, int mode, float* zio,
                             int* status, cudaStream_t st, const float* wlast = nullptr, float* maps = nullptr) {
    if (s.MG == 1)
        return launch_persistent_mg<C, 1>(s, n, batch, in, out, w, bias, act, mode, zio, status, st, wlast, maps);
    if constexpr (C < 64)
        return launch_persistent_mg<C, 2>(s, n, batch, in, out, w, bias, act, mode, zio, status, st, wlast, maps);
    set_error("conv: no persistent kernel for C=%d, MG=%d", C, s.MG);
    return AC_ERR_UNSUPPORTED;
}

template <int C>
static int launch_hidden(int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out, const __nv_bfloat16* w,
                         const float* bias, int act, int mode, float* zio, int* status, cudaStream_t st) {
    if (batch <= 0) return AC_OK;
    if (!status) {
        set_error("tensor-core conv: no status word");
        return AC_ERR_ARG;
    }
    const PShape ps = p_shape(n, C);
    if (ps.RING) return launch_persistent<C>(ps, n, batch, in, out, w, bias, act, mode, zio, status, st);
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

bool hidden_last_fused_supported(int n, int C) { return C >= 32 && C <= 64 && p_shape(n, C).RING > 0; }

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
    const PShape ps = p_shape(n, C);
    if (C == 32)
        return launch_persistent<32>(ps, n, batch, in, act_out, w, bias, d->act, kFwdLast, zsave, status, st, w_last,
                                     maps);
    return launch_persistent<64>(ps, n, batch, in, act_out, w, bias, d->act, kFwdLast, zsave, status, st, w_last,
                                 maps);
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
