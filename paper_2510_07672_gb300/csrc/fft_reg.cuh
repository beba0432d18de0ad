// fft_reg.cuh -- small complex DFTs held entirely in one thread's registers,
// and the two-pass (four-step) 1D transform of length N = A * B that a group of
// B lanes of one warp performs on one line of a field with one shared-memory
// exchange.
//
// Layout invariant ("stride layout"): thread j of a line holds element
// j + B * t in slot t, t = 0..A-1, both before and after a 1D transform (the
// output is in natural frequency order).  This lets a forward and an inverse
// transform follow each other without any reordering.
#pragma once

#include "common.cuh"

namespace acpr {

// cos(2 pi m / 32) for m = 0..8; other angles follow by symmetry.
__host__ __device__ constexpr double cos32_quarter(int m) {
    return m == 0 ? 1.0
         : m == 1 ? 0.98078528040323044912618223613424
         : m == 2 ? 0.92387953251128675612818318939679
         : m == 3 ? 0.83146961230254523707878837761791
         : m == 4 ? 0.70710678118654752440084436210485
         : m == 5 ? 0.55557023301960222474283081394853
         : m == 6 ? 0.38268343236508977172845998403040
         : m == 7 ? 0.19509032201612826784828486847702
                  : 0.0;
}

__host__ __device__ constexpr double cos32(int m) {
    // cos(2 pi m / 32), m in [0, 32)
    return m <= 8 ? cos32_quarter(m)
         : m <= 16 ? -cos32_quarter(16 - m)
         : m <= 24 ? -cos32_quarter(m - 16)
                   : cos32_quarter(32 - m);
}
__host__ __device__ constexpr double sin32(int m) {
    // sin(2 pi m / 32) = cos(2 pi (m - 8) / 32)
    return cos32((m + 24) & 31);
}

__host__ __device__ constexpr int bit_reverse(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int ilog2(int m) { return m <= 1 ? 0 : 1 + ilog2(m / 2); }

// (vr + i vi) *= exp(SIGN * 2 pi i m / 32), m a compile-time constant after
// unrolling; quarter turns are done as swaps.
template <typename T, int SIGN>
__device__ __forceinline__ void twiddle32(int m, T& vr, T& vi) {
    if (m == 0) return;
    if (m == 8) {  // multiply by SIGN * i
        T t = vr;
        vr = -T(SIGN) * vi;
        vi = T(SIGN) * t;
        return;
    }
    const T c = T(cos32(m));
    const T s = T(SIGN) * T(sin32(m));
    T r = vr * c - vi * s;
    vi = vr * s + vi * c;
    vr = r;
}

// Radix-2 butterfly (u, v) -> (u + w v, u - w v) with w = exp(SIGN 2 pi i m / 32),
// m a compile-time constant.  Quarter turns are swaps.  A general twiddle is
// folded into the butterfly with the larger of |cos|, |sin| factored out
// (the fused multiply-add form of Linzer and Feig, IBM J. Res. Dev. 37
// (1993)): with q = sin/cos, w v = cos (v_r - q v_i, v_i + q v_r), and the two
// outputs are u +- cos (...) -- six fused multiply-adds instead of two
// multiplies, two multiply-adds and four adds.
template <typename T, int SIGN>
__device__ __forceinline__ void butterfly32(int m, T& ur, T& ui, T& vr, T& vi) {
    if (m == 0 || m == 8) {
        twiddle32<T, SIGN>(m, vr, vi);
        const T ar = ur, ai = ui;
        ur = ar + vr;
        ui = ai + vi;
        vr = ar - vr;
        vi = ai - vi;
        return;
    }
    const double cd = cos32(m), sd = double(SIGN) * sin32(m);
    T a, b, f;
    if ((cd < 0 ? -cd : cd) >= (sd < 0 ? -sd : sd)) {
        const T q = T(sd / cd);
        f = T(cd);
        a = fma(-q, vi, vr);  // (c v_r - s v_i) / c
        b = fma(q, vr, vi);   // (s v_r + c v_i) / c
    } else {
        const T q = T(cd / sd);
        f = T(sd);
        a = fma(q, vr, -vi);  // (c v_r - s v_i) / s
        b = fma(q, vi, vr);   // (s v_r + c v_i) / s
    }
    const T ar = ur, ai = ui;
    ur = fma(f, a, ar);
    ui = fma(f, b, ai);
    vr = fma(-f, a, ar);
    vi = fma(-f, b, ai);
}

// One butterfly stage of span LEN, then the next (template recursion keeps
// every index a compile-time constant so the arrays stay in registers).
template <typename T, int M, int SIGN, int LEN>
__device__ __forceinline__ void dit_stages(T (&re)[M], T (&im)[M]) {
    if constexpr (LEN <= M) {
#pragma unroll
        for (int i = 0; i < M; i += LEN) {
#pragma unroll
            for (int k = 0; k < LEN / 2; ++k)
                butterfly32<T, SIGN>(k * (32 / LEN), re[i + k], im[i + k], re[i + k + LEN / 2],
                                     im[i + k + LEN / 2]);
        }
        dit_stages<T, M, SIGN, 2 * LEN>(re, im);
    }
}

// In-register radix-2 DIT DFT of size M (M <= 32, power of two),
// X_k = sum_j x_j exp(SIGN 2 pi i j k / M), natural order in and out.
template <typename T, int M, int SIGN>
__device__ __forceinline__ void reg_dft(T (&re)[M], T (&im)[M]) {
    static_assert(M >= 1 && M <= 32 && (M & (M - 1)) == 0, "M must be a power of two <= 32");
    constexpr int bits = ilog2(M);
    T r2[M], i2[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        r2[bit_reverse(i, bits)] = re[i];
        i2[bit_reverse(i, bits)] = im[i];
    }
#pragma unroll
    for (int i = 0; i < M; ++i) { re[i] = r2[i]; im[i] = i2[i]; }
    dit_stages<T, M, SIGN, 2>(re, im);
}

// Shared-memory position of element e = k1 * B + n2 of a line's exchange area:
// one pad slot after every B elements, so that the pass-2 reads (B lanes
// reading elements B apart) fall in distinct banks.
template <int B>
__host__ __device__ constexpr int xpos(int k1, int n2) { return k1 * (B + 1) + n2; }

// Exchange-area length (complex elements) a line needs.
template <int N, int B>
__host__ __device__ constexpr int xlen() { return N + N / B; }

// One line transform of length N = A * B by the B lanes of that line, which
// are B consecutive lanes of one warp (B divides 32).
//   x:    this thread's A elements (stride layout), transformed in place.
//   tw:   shared table, entry k1 * B + j = exp(-2 pi i ((j k1) mod N) / N)
//         (the inverse uses the conjugates): the B lanes of a line read B
//         consecutive entries.
//   line: base of this line's exchange area in shared memory (>= xlen<N, B>()
//         elements), read and written by this line's lanes only;
//   j:    this thread's lane within the line;
//   wmask: the warp's lanes that run this code (all lanes of every line in
//         the warp).
// Unnormalised, X_k = sum_n x_n exp(SIGN 2 pi i n k / N).  Only warp-level
// barriers: the lanes that exchange data share a warp.
template <typename T, int N, int A, int B, int SIGN>
__device__ __forceinline__ void line_fft(vec2_t<T> (&x)[A], const vec2_t<T>* __restrict__ tw,
                                         vec2_t<T>* line, int j, unsigned wmask) {
    static_assert(A * B == N && A % B == 0, "N = A * B with B | A");
    static_assert(B <= 32 && 32 % B == 0, "a line's lanes must fit in one warp");
    T re[A], im[A];
#pragma unroll
    for (int t = 0; t < A; ++t) { re[t] = x[t].x; im[t] = x[t].y; }
    // pass 1: A-point DFT over n1 of x[B n1 + j]
    reg_dft<T, A, SIGN>(re, im);
    // twiddle exp(SIGN 2 pi i j k1 / N)
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) {
        const vec2_t<T> w = tw[k1 * B + j];
        const T c = w.x;
        const T s = SIGN < 0 ? w.y : -w.y;
        const T r = re[k1] * c - im[k1] * s;
        im[k1] = re[k1] * s + im[k1] * c;
        re[k1] = r;
    }
    __syncwarp(wmask);  // this line's earlier readers of `line` are done
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
        vec2_t<T> v;
        v.x = re[k1];
        v.y = im[k1];
        line[xpos<B>(k1, j)] = v;
    }
    __syncwarp(wmask);
    // pass 2: for k1 = j + B m, a B-point DFT over n2
#pragma unroll
    for (int m = 0; m < A / B; ++m) {
        const int k1 = j + B * m;
        T br[B], bi[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) {
            const vec2_t<T> v = line[xpos<B>(k1, n2)];
            br[n2] = v.x;
            bi[n2] = v.y;
        }
        reg_dft<T, B, SIGN>(br, bi);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            // output index k1 + A k2 = j + B (m + (A/B) k2)
            x[m + (A / B) * k2].x = br[k2];
            x[m + (A / B) * k2].y = bi[k2];
        }
    }
}

}  // namespace acpr
