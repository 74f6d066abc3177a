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

// 32-byte aligned quadruple of doubles (anchor records of the mixed section)
struct alignas(32) D4 {
    double x, y, z, w;
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

// double -> float, round to nearest even, on the integer pipe (IEEE 754 binary64 and
// binary32 layouts); magnitudes below the smallest normal float become signed zero,
// above the largest float infinity, NaN stays NaN.
__device__ __forceinline__ float to_float(double v) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0x7ff)
        return __uint_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
    const int ef = e - 1023 + 127;
    if (ef <= 0) return __uint_as_float(sign);
    if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);   // top 23 of the 52 bits
    const unsigned rest = lo & 0x1fffffffu;                    // the 29 dropped bits
    unsigned f = sign | ((unsigned)ef << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ++f;   // carries into e
    return __uint_as_float(f);
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
