// Internal helpers of liblw.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lw.h"

namespace lw {

// Speed of light and vacuum permittivity (SI, exact / CODATA 2018).
constexpr double kC0 = 299792458.0;
constexpr double kInvC0 = 1.0 / 299792458.0;   // correctly rounded at compile time
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

constexpr int kSms = 152;   // GB300 streaming multiprocessors (2 dies x 76)

// Anchor record of the mixed section (32 bytes): the block's light-front time
// tau_b = t_b - z_b/c0 in FP64 and its position as unevaluated FP32 pairs (hi, lo),
// hi = fl32(x), lo = fl32(x - hi), per component.
struct alignas(32) Anchor {
    double tau;
    float x_hi, x_lo, y_hi, y_lo, z_hi, z_lo;
};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LW_OK : LW_ECUDA;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__device__ __forceinline__ void status_or(int32_t* st, int bits) {
    if (st && bits) atomicOr(st, bits);
}

// Block-wide OR of status bits, one atomic per block.
__device__ __forceinline__ void block_status_or(int32_t* st, int bits) {
    int any = __syncthreads_or(bits);
    if (any) {
        // gather the union of bits through shared memory
        __shared__ int s_bits;
        if (threadIdx.x == 0) s_bits = 0;
        __syncthreads();
        if (bits) atomicOr(&s_bits, bits);
        __syncthreads();
        if (threadIdx.x == 0 && st) atomicOr(st, s_bits);
    }
}

// Asynchronous global -> shared copies (cp.async, sm_80 and later): issued without
// holding registers, completed by cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// all but the most recently committed group complete
__device__ __forceinline__ void cp_async_wait_one() {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
// 8- and 16-byte copies that write zeros instead when !valid (src-size 0 reads nothing)
__device__ __forceinline__ void cp_async8_zfill(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                 : "memory");
}

// double -> float, round to nearest even, on the integer pipe (IEEE 754 binary64 and
// binary32 layouts); magnitudes below the smallest normal float become signed zero,
// above the largest float infinity, NaN stays NaN.
__device__ __forceinline__ float to_float_bits(unsigned hi, unsigned lo) {
    const unsigned a = hi & 0x7fffffffu;   // biased exponent and the top 20 mantissa bits
    // round to nearest even at bit 29 of the magnitude's 64-bit pattern: adding half an
    // ulp less one, plus the kept lsb, carries into bit 29 exactly when rounding up
    unsigned long long v = ((unsigned long long)a << 32) | lo;
    v += 0x0fffffffull + ((lo >> 29) & 1u);
    unsigned f = (unsigned)(v >> 29) - (896u << 23);   // rebias 1023 -> 127
    // selects, not branches, so that loads ahead of a conversion stay in flight
    f = a < (897u << 20) ? 0u : f;   // below the smallest normal float
    const unsigned big = a > 0x7ff00000u || (a == 0x7ff00000u && lo) ? 0x7fc00000u : 0x7f800000u;
    f = a >= (1151u << 20) ? big : f;   // beyond the largest float, infinity or NaN
    return __uint_as_float((hi & 0x80000000u) | f);
}
__device__ __forceinline__ float to_float(double v) {
    return to_float_bits((unsigned)__double2hiint(v), (unsigned)__double2loint(v));
}

// Far-field advanced time t_a = t - (n . r) / c0 in FP64 with the documented
// operation order ((n_x x + n_y y) + n_z z), one rounding per operation.
__device__ __forceinline__ double advanced_time_fp64(double nx, double ny, double nz, double x,
                                                     double y, double z, double t) {
    double nr = __dmul_rn(nx, x);
    nr = __dadd_rn(nr, __dmul_rn(ny, y));
    nr = __dadd_rn(nr, __dmul_rn(nz, z));
    return __dsub_rn(t, __dmul_rn(nr, kInvC0));
}

// Order-preserving map double -> uint64 (for atomic min/max).
__device__ __forceinline__ unsigned long long ordered_key(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_to_double(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

}  // namespace lw
