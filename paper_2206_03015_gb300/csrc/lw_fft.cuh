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
// tw[q * (N / len)] (tw covers the full length N).  Two consecutive radix-2
// stages s, s+1 run in one pass over groups of four elements (i0, i0+h,
// i0+2h, i0+3h), h = 2^(s-1): the same butterflies and twiddles as stage by
// stage, with half the shared-memory traffic and barriers; an odd first stage
// runs alone.
template <typename C>
__device__ void fft_smem(C* buf, int L, int logL, int Cn, const C* __restrict__ tw, int64_t N) {
    int s = 1;
    if (logL & 1) {   // stage 1 (len 2, twiddle 1)
        const int nbf = (L >> 1) * Cn;
        for (int t = threadIdx.x; t < nbf; t += blockDim.x) {
            const int c = t % Cn;
            const int i0 = 2 * (t / Cn);
            const C u = buf[i0 * Cn + c];
            const C v = cmul(buf[(i0 + 1) * Cn + c], tw[0]);
            buf[i0 * Cn + c] = cadd(u, v);
            buf[(i0 + 1) * Cn + c] = csub(u, v);
        }
        __syncthreads();
        s = 2;
    }
    for (; s < logL; s += 2) {
        const int h = 1 << (s - 1);
        const int64_t st0 = N >> s, st1 = N >> (s + 1);
        const int ng = (L >> 2) * Cn;
        for (int t = threadIdx.x; t < ng; t += blockDim.x) {
            const int c = t % Cn;
            const int g = t / Cn;
            const int q = g & (h - 1);
            const int i0 = ((g >> (s - 1)) << (s + 1)) + q;
            const C w0 = tw[q * st0];
            const C x0 = buf[i0 * Cn + c];
            const C x1 = cmul(buf[(i0 + h) * Cn + c], w0);
            const C x2 = buf[(i0 + 2 * h) * Cn + c];
            const C x3 = cmul(buf[(i0 + 3 * h) * Cn + c], w0);
            const C b0 = cadd(x0, x1), b1 = csub(x0, x1), b2 = cadd(x2, x3), b3 = csub(x2, x3);
            const C c2 = cmul(b2, tw[q * st1]);
            const C c3 = cmul(b3, tw[(q + h) * st1]);
            buf[i0 * Cn + c] = cadd(b0, c2);
            buf[(i0 + 2 * h) * Cn + c] = csub(b0, c2);
            buf[(i0 + h) * Cn + c] = cadd(b1, c3);
            buf[(i0 + 3 * h) * Cn + c] = csub(b1, c3);
        }
        __syncthreads();
    }
}


}  // namespace lw
