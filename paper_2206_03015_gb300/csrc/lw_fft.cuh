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
// as buf[j * C + c] in bit-reversed order; twiddle exp(2 pi i q/len) is
// tw[q * (N / len)] (tw covers the full length N).
template <typename C>
__device__ void fft_smem(C* buf, int L, int logL, int Cn, const C* __restrict__ tw, int64_t N) {
    const int nbf = (L >> 1) * Cn;
    for (int s = 1; s <= logL; ++s) {
        const int len = 1 << s, half = len >> 1;
        const int64_t stride = N >> s;
        for (int t = threadIdx.x; t < nbf; t += blockDim.x) {
            const int c = t % Cn;
            const int b = t / Cn;
            const int q = b & (half - 1);
            const int i0 = ((b >> (s - 1)) << s) + q;
            const int i1 = i0 + half;
            const C w = tw[q * stride];
            const C u = buf[i0 * Cn + c];
            const C v = cmul(buf[i1 * Cn + c], w);
            buf[i0 * Cn + c] = cadd(u, v);
            buf[i1 * Cn + c] = csub(u, v);
        }
        __syncthreads();
    }
}


}  // namespace lw
