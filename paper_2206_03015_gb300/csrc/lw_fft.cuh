// Shared FFT building blocks of liblw.so (not part of the ABI): complex
// helpers, the twiddle table exp(+2 pi i t/N) and an in-place radix-2
// transform of interleaved sequences in shared memory.
#pragma once

#include "lw_internal.cuh"

namespace lw {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) {
    C r;
    r.x = a.x + b.x;
    r.y = a.y + b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C csub(C a, C b) {
    C r;
    r.x = a.x - b.x;
    r.y = a.y - b.y;
    return r;
}

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) {
    return __brev(x) >> (32 - bits);
}

// twiddle table tw[t] = exp(+2 pi i t / N), t = 0..N-1, evaluated in FP64
template <typename T>
__global__ void twiddle_kernel(typename V2<T>::type* tw, int64_t N) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)t / (double)N, &s, &c);
        typename V2<T>::type w;
        w.x = (T)c;
        w.y = (T)s;
        tw[t] = w;
    }
}

// In-place radix-2 transform of C interleaved sequences of length L stored
// as buf[j * C + c] in bit-reversed order, evaluated R <= 4 radix-2 stages at
// a time: a pass over stages s .. s+R-1 gives each thread a group of 2^R
// elements i0 + m h (h = 2^(s-1), m = 0 .. 2^R - 1) held in registers.  In stage
// s+t the element m pairs with m + 2^t under the twiddle exp(2 pi i q / 2^(s+t)),
// q = q0 + (m mod 2^t) h, q0 = the group's offset in its block; this factors
// into the table value tw[q0 * N / 2^(s+t)] (tw[x] = exp(2 pi i x / N)) times
// the constant root exp(2 pi i (m mod 2^t) / 2^(t+1)).  Per pass a group makes
// 2^R reads and writes of shared memory and R table reads.  fft_smem picks R per
// transform so that the passes keep every thread busy.
template <typename C> struct Root;
template <> struct Root<double2> {
    // exp(2 pi i k / 16), k = 0..15 (cos and sin of multiples of pi/8)
    __device__ static double2 get(int k) {
        constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173;
        constexpr double c2 = 0.70710678118654752440;
        const double cs[5] = {1.0, c1, c2, s1, 0.0};   // cos(k pi/8), k = 0..4
        const int kk = k & 15;
        const int q = kk & 3, o = kk >> 2;             // k = 4 o + q
        // (cos, sin) of (q pi / 8), rotated by o quarter turns
        const double c = cs[q], s = cs[4 - q];
        double2 r;
        if (o == 0) { r.x = c; r.y = s; }
        else if (o == 1) { r.x = -s; r.y = c; }
        else if (o == 2) { r.x = -c; r.y = -s; }
        else { r.x = s; r.y = -c; }
        return r;
    }
};
template <> struct Root<float2> {
    __device__ static float2 get(int k) {
        const double2 d = Root<double2>::get(k);
        return make_float2((float)d.x, (float)d.y);
    }
};

template <typename C, int R>
__device__ __forceinline__ void fft_pass(C* buf, int L, int Cn, int s, const C* __restrict__ tw,
                                         int64_t N) {
    constexpr int G = 1 << R;
    const int h = 1 << (s - 1);
    const int ng = (L >> R) * Cn;
    for (int t = threadIdx.x; t < ng; t += blockDim.x) {
        const int c = t % Cn;
        const int g = t / Cn;
        const int q0 = g & (h - 1);
        const int i0 = ((g >> (s - 1)) << (s - 1 + R)) + q0;
        C x[G];
#pragma unroll
        for (int m = 0; m < G; ++m) x[m] = buf[(i0 + m * h) * Cn + c];
#pragma unroll
        for (int st = 0; st < R; ++st) {
            const C wb = tw[(int64_t)q0 * (N >> (s + st))];
            const int half = 1 << st;
#pragma unroll
            for (int m = 0; m < G; ++m) {
                if (m & half) continue;
                const int r = m & (half - 1);
                // constant root exp(2 pi i r / 2^(st+1)) = 16th root number r * 8 / half
                const C w = r == 0 ? wb : cmul(wb, Root<C>::get(r * (8 >> st)));
                const C v = cmul(x[m + half], w);
                const C u = x[m];
                x[m] = cadd(u, v);
                x[m + half] = csub(u, v);
            }
        }
#pragma unroll
        for (int m = 0; m < G; ++m) buf[(i0 + m * h) * Cn + c] = x[m];
    }
    __syncthreads();
}

// Passes of R stages, R the largest of 2..4 that still gives every thread of the
// CTA a group ((L >> R) * Cn >= blockDim.x), the remaining stages first.
template <typename C>
__device__ void fft_smem(C* buf, int L, int logL, int Cn, const C* __restrict__ tw, int64_t N) {
    int R = 4;
    while (R > 2 && (int64_t)(L >> R) * Cn < (int64_t)blockDim.x) --R;
    if (R > logL) R = logL;
    int s = 1;
    const int lead = R > 0 ? logL % R : 0;
    if (lead == 1) fft_pass<C, 1>(buf, L, Cn, s, tw, N);
    if (lead == 2) fft_pass<C, 2>(buf, L, Cn, s, tw, N);
    if (lead == 3) fft_pass<C, 3>(buf, L, Cn, s, tw, N);
    s += lead;
    for (; s <= logL; s += R) {
        if (R == 4)
            fft_pass<C, 4>(buf, L, Cn, s, tw, N);
        else if (R == 3)
            fft_pass<C, 3>(buf, L, Cn, s, tw, N);
        else if (R == 2)
            fft_pass<C, 2>(buf, L, Cn, s, tw, N);
        else
            fft_pass<C, 1>(buf, L, Cn, s, tw, N);
    }
}


}  // namespace lw
