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
// (s.x^2 + d.x^2, s.y^2 + d.y^2)
template <typename C> __device__ __forceinline__ C sumsq2(C s, C d) {
    C r;
    r.x = s.x * s.x + d.x * d.x;
    r.y = s.y * s.y + d.y * d.y;
    return r;
}
__device__ __forceinline__ float2 sumsq2(float2 s, float2 d) {
    return __ffma2_rn(d, d, __fmul2_rn(s, s));
}
// FP32 pairs: one packed instruction each (a - b as the exact b * (-1) + a)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) {
    return __brev(x) >> (32 - bits);
}

// Shared-memory slot of element j of sequence c in a buffer of CN interleaved sequences:
// j * CN + c, plus (PAD) one padding slot per 2^sh elements.  With sh = logL - 5 the 32
// rows that a warp's bit-reversed stores of 32 consecutive inputs hit (they differ in the
// top five bits of j) start on 32 different banks modulo the odd factor s * CN + 1, so
// those stores are conflict-free; consecutive rows stay contiguous for the passes.
__host__ __device__ __forceinline__ int fft_pad_shift(int logL) { return logL > 5 ? logL - 5 : 0; }
template <int CN, bool PAD>
__device__ __forceinline__ int fft_slot(int j, int c, int sh) {
    return j * CN + (PAD ? (j >> sh) : 0) + c;
}
// slots a padded buffer of L rows of Cn sequences needs
__host__ __device__ __forceinline__ int fft_slots(int L, int logL, int Cn) {
    return L * Cn + (L >> fft_pad_shift(logL));
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

// In-place transform (sign +) of CN interleaved sequences of length L held in
// bit-reversed order at buf[fft_slot<CN, PAD>(j, c, sh)], as passes over R <= 4 radix-2
// stages at a time.  A pass over stages s .. s+R-1 gives each thread a group of G = 2^R
// elements x_m at i0 + m h (h = 2^(s-1), m = 0 .. G-1), the length-h transforms at offset
// q0 of G consecutive blocks, block m holding the sub-sequence of offset rev_R(m) (R-bit
// reversal).  The combined length-G h transform at q0 + k h is
//   sum_m exp(2 pi i (q0 + k h) rev_R(m) / (G h)) x_m
//     = sum_m exp(2 pi i k rev_R(m) / G) [exp(2 pi i q0 rev_R(m) / (G h)) x_m],
// so each x_m is first multiplied by the table value tw[q0 rev_R(m) N / (G h)]
// (tw[t] = exp(2 pi i t / N)) and the G-point transform of the bit-reversed group is then
// evaluated by radix-2 stages whose roots exp(2 pi i r / 2^(t+1)) are constants:
// 1, i and the odd eighth roots cost no or two multiplications.  fft_smem picks R per
// transform so that the passes keep every thread busy.
__host__ __device__ constexpr int rev_bits(int m, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((m >> b) & 1) << (bits - 1 - b);
    return r;
}

// x * exp(2 pi i k / 16), k = 0..7 (k is a constant once the stage loops are unrolled)
template <typename C>
__device__ __forceinline__ C mul_root16(C x, int k) {
    using T = decltype(x.x);
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;   // cos, sin pi/8
    const T r2 = (T)0.70710678118654752440;                                     // sqrt(1/2)
    C y;
    switch (k) {
        case 0: return x;
        case 4: y.x = -x.y; y.y = x.x; return y;                          // i
        case 2: y.x = (x.x - x.y) * r2; y.y = (x.x + x.y) * r2; return y;   // (1 + i)/sqrt 2
        case 6: y.x = -(x.x + x.y) * r2; y.y = (x.x - x.y) * r2; return y;  // (-1 + i)/sqrt 2
        case 1: return cmul(x, C{c1, s1});
        case 3: return cmul(x, C{s1, c1});
        case 5: return cmul(x, C{-s1, c1});
        default: return cmul(x, C{-c1, s1});                               // k = 7
    }
}

template <typename C, int CN, bool PAD, int R>
__device__ __forceinline__ void fft_pass(C* buf, int L, int sh, int s, const C* __restrict__ tw,
                                         int N) {
    constexpr int G = 1 << R;
    const int h = 1 << (s - 1);
    const int ng = (L >> R) * CN;
    const int tstep = N >> (R + s - 1);   // table step of exp(2 pi i / (G h))
    for (int t = threadIdx.x; t < ng; t += blockDim.x) {
        const int c = t % CN;
        const int g = t / CN;
        const int q0 = g & (h - 1);
        const int i0 = ((g >> (s - 1)) << (s - 1 + R)) + q0;
        C x[G];
#pragma unroll
        for (int m = 0; m < G; ++m) x[m] = buf[fft_slot<CN, PAD>(i0 + m * h, c, sh)];
        if (h > 1) {   // uniform; the pre-twiddles are all 1 in the first pass
            const int b = q0 * tstep;
#pragma unroll
            for (int m = 1; m < G; ++m) x[m] = cmul(x[m], tw[b * rev_bits(m, R)]);
        }
#pragma unroll
        for (int st = 0; st < R; ++st) {
            const int half = 1 << st;
#pragma unroll
            for (int m = 0; m < G; ++m) {
                if (m & half) continue;
                // root exp(2 pi i r / 2^(st+1)) = 16th root number r * 8 / half
                const C v = mul_root16(x[m + half], (m & (half - 1)) * (8 >> st));
                const C u = x[m];
                x[m] = cadd(u, v);
                x[m + half] = csub(u, v);
            }
        }
#pragma unroll
        for (int m = 0; m < G; ++m) buf[fft_slot<CN, PAD>(i0 + m * h, c, sh)] = x[m];
    }
    __syncthreads();
}

// Passes of R stages, R the largest of 2..4 that still gives every thread of the
// CTA a group ((L >> R) * CN >= blockDim.x), the remaining stages first.  sh is the
// padding shift of a PAD layout (fft_slot).
template <typename C, int CN, bool PAD>
__device__ void fft_smem(C* buf, int L, int logL, const C* __restrict__ tw, int N, int sh = 0) {
    int R = 4;
    while (R > 2 && (L >> R) * CN < (int)blockDim.x) --R;
    if (R > logL) R = logL;
    int s = 1;
    const int lead = R > 0 ? logL % R : 0;
    if (lead == 1) fft_pass<C, CN, PAD, 1>(buf, L, sh, s, tw, N);
    if (lead == 2) fft_pass<C, CN, PAD, 2>(buf, L, sh, s, tw, N);
    if (lead == 3) fft_pass<C, CN, PAD, 3>(buf, L, sh, s, tw, N);
    s += lead;
    for (; s <= logL; s += R) {
        if (R == 4)
            fft_pass<C, CN, PAD, 4>(buf, L, sh, s, tw, N);
        else if (R == 3)
            fft_pass<C, CN, PAD, 3>(buf, L, sh, s, tw, N);
        else if (R == 2)
            fft_pass<C, CN, PAD, 2>(buf, L, sh, s, tw, N);
        else
            fft_pass<C, CN, PAD, 1>(buf, L, sh, s, tw, N);
    }
}

// The same transform with the length 2^LOGL, the pass plan and the layout fixed at
// compile time, for CTAs of kFftThreads threads.  Element i0 + m h of a group is at
// slot base + off(m) with base = i0 CN + c + (i0 >> SH) and off(m) = m h CN +
// ((m h) >> SH): the bits of the block start, of q0 < h and of m h are disjoint, so the
// padding shift splits over them, and every group reads and writes at immediate
// offsets from one base.
constexpr int kFftThreads = 256;

template <int CN, int LOGL>
__host__ __device__ constexpr int fft_fixed_radix() {
    int R = 4;
    while (R > 2 && ((1 << LOGL) >> R) * CN < kFftThreads) --R;
    return R < LOGL ? R : LOGL;
}

template <typename C, int CN, bool PAD, int LOGL, int R, int S>
__device__ __forceinline__ void fft_pass_fixed(C* buf, const C* __restrict__ tw, int N) {
    constexpr int G = 1 << R;
    constexpr int h = 1 << (S - 1);
    constexpr int SH = PAD ? (LOGL > 5 ? LOGL - 5 : 0) : 31;
    constexpr int ng = ((1 << LOGL) >> R) * CN;
    const int tstep = N >> (R + S - 1);   // table step of exp(2 pi i / (G h))
#pragma unroll 1
    for (int t = threadIdx.x; t < ng; t += kFftThreads) {
        const int c = t % CN;
        const int g = t / CN;
        const int q0 = g & (h - 1);
        const int i0 = ((g >> (S - 1)) << (S - 1 + R)) + q0;
        C* bp = buf + (i0 * CN + c + (PAD ? (i0 >> SH) : 0));
        C x[G];
#pragma unroll
        for (int m = 0; m < G; ++m) x[m] = bp[m * h * CN + (PAD ? ((m * h) >> SH) : 0)];
        if (h > 1) {
            const int b = q0 * tstep;
#pragma unroll
            for (int m = 1; m < G; ++m) x[m] = cmul(x[m], tw[b * rev_bits(m, R)]);
        }
#pragma unroll
        for (int st = 0; st < R; ++st) {
            const int half = 1 << st;
#pragma unroll
            for (int m = 0; m < G; ++m) {
                if (m & half) continue;
                const C v = mul_root16(x[m + half], (m & (half - 1)) * (8 >> st));
                const C u = x[m];
                x[m] = cadd(u, v);
                x[m + half] = csub(u, v);
            }
        }
#pragma unroll
        for (int m = 0; m < G; ++m) bp[m * h * CN + (PAD ? ((m * h) >> SH) : 0)] = x[m];
    }
    __syncthreads();
}

template <typename C, int CN, bool PAD, int LOGL, int S = 1>
__device__ __forceinline__ void fft_smem_fixed(C* buf, const C* __restrict__ tw, int N) {
    if constexpr (S <= LOGL) {
        constexpr int R = fft_fixed_radix<CN, LOGL>();
        constexpr int lead = LOGL % R;
        constexpr int RR = (S == 1 && lead) ? lead : R;
        fft_pass_fixed<C, CN, PAD, LOGL, RR, S>(buf, tw, N);
        fft_smem_fixed<C, CN, PAD, LOGL, S + RR>(buf, tw, N);
    }
}

}  // namespace lw
