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
// sets a device flag that tc_check_status() reports as AC_ERR_TIMEOUT.
#include "cnn.cuh"
#include "tc_ptx.cuh"

namespace acpr {

namespace {
__device__ int g_tc_timeout = 0;
constexpr int kTcThreads = 256;
constexpr long long kTcSpin = 4000000;  // ~0.2 s of polls with 32 ns sleeps
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
enum { kFwd = 0, kDgrad = 1 };

template <int C>
__global__ void __launch_bounds__(kTcThreads)
conv_hidden_tc_kernel(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out,
                      const __nv_bfloat16* __restrict__ wpk, const float* __restrict__ bias, int n, int TY,
                      int n_mt, int plane_px, int ncols, int act, int mode, float* __restrict__ zio) {
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
            if (tid == 0) atomicExch(&g_tc_timeout, 2);
            tc::mbar_wait_bounded(&bars[1], 0, kTcSpin);  // let the MMAs drain
        }
    } else {
        if (tid == 0) atomicExch(&g_tc_timeout, 1);
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
                            o8[i] = __float2bfloat16_rn(act_apply<float>(act, z8[i]));
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
                            o8[i] = __float2bfloat16_rn(__uint_as_float(v[i]) * act_grad<float>(act, zz[i]));
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

template <int C>
static int launch_hidden(int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out, const __nv_bfloat16* w,
                         const float* bias, int act, int mode, float* zio, cudaStream_t st) {
    const TcShape s = pick_shape(n, C);
    if (s.TY == 0) return AC_ERR_UNSUPPORTED;
    auto kern = conv_hidden_tc_kernel<C>;
    static size_t configured = 0;
    if (configured < s.smem) {
        ACPR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(227 * 1024)));
        configured = 227 * 1024;
    }
    const long long blocks = (long long)batch * (n / s.TY);
    kern<<<unsigned(blocks), kTcThreads, s.smem, st>>>(in, out, w, bias, n, s.TY, s.n_mt, s.plane_px, s.ncols, act,
                                                       mode, zio);
    ACPR_LAUNCH_CHECK();
    return AC_OK;
}

int hidden_layer_bf16(const cnn_desc* d, int l, int n, int batch, const __nv_bfloat16* in, __nv_bfloat16* out,
                      const float* /*w_master*/, const float* bias, cudaStream_t st, float* zsave) {
    if (n < 8) return AC_ERR_UNSUPPORTED;
    const int C = d->channels;
    const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(d->packed) + size_t(l - 1) * 9 * C * C;
    switch (C) {
        case 16: return launch_hidden<16>(n, batch, in, out, w, bias, d->act, kFwd, zsave, st);
        case 32: return launch_hidden<32>(n, batch, in, out, w, bias, d->act, kFwd, zsave, st);
        case 64: return launch_hidden<64>(n, batch, in, out, w, bias, d->act, kFwd, zsave, st);
        default: return AC_ERR_UNSUPPORTED;
    }
}

int hidden_dgrad_bf16(int C, int act, int n, int batch, const __nv_bfloat16* dz_next, __nv_bfloat16* dz_out,
                      const __nv_bfloat16* w_t, const float* z_prev, cudaStream_t st) {
    if (n < 8) return AC_ERR_UNSUPPORTED;
    float* zp = const_cast<float*>(z_prev);
    switch (C) {
        case 16: return launch_hidden<16>(n, batch, dz_next, dz_out, w_t, nullptr, act, kDgrad, zp, st);
        case 32: return launch_hidden<32>(n, batch, dz_next, dz_out, w_t, nullptr, act, kDgrad, zp, st);
        case 64: return launch_hidden<64>(n, batch, dz_next, dz_out, w_t, nullptr, act, kDgrad, zp, st);
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

int tc_check_status(cudaStream_t st) {
    int flag = 0;
    ACPR_CUDA(cudaMemcpyFromSymbolAsync(&flag, g_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    ACPR_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        const int zero = 0;
        ACPR_CUDA(cudaMemcpyToSymbolAsync(g_tc_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        ACPR_CUDA(cudaStreamSynchronize(st));
        set_error("tensor-core conv: bounded wait gave up (%s)", flag == 1 ? "operand loads" : "MMA completion");
        return AC_ERR_TIMEOUT;
    }
    return AC_OK;
}

}  // namespace acpr
