// Pipe peaks of the GPU this library runs on, for the deposit's roofline: the
// rates of the operations the time-domain deposit is made of, each measured by a
// kernel that does nothing else.
//
//   red_f32 / red_f64 / red_v4   L2 reductions (red.global.add) to addresses that
//                                are 128 bytes apart across a warp (every lane its
//                                own cache line, as when the lanes of a warp update
//                                different pixels' records) or consecutive
//                                (one line per warp), on a buffer that fits in L2
//   fma_f32 / fma_f64            dependent-chain-free FMA throughput
//   lds_v4                       conflict-free 16-byte shared-memory loads (one
//                                128-byte wavefront per 8 lanes)
//
// Every kernel indexes its buffer with a mask of a power-of-two length, so all
// accesses stay in bounds; none waits on anything.  The host times them with
// CUDA events on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ void red_add_f32(float* p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_f64(double* p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add_v4f32(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

// lane stride in elements: 32 (distinct 128-byte lines for 4-byte values) or 1
template <typename T, int V>
__global__ void red_kernel(T* buf, uint64_t mask, int iters, int stride_elems) {
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    // each warp walks its own region; consecutive iterations jump by a large odd
    // multiple of the warp's span so that lines are revisited rarely
    const uint64_t span = 32ull * stride_elems * V;
    uint64_t base = warp * span * 7;
    for (int r = 0; r < iters; ++r) {
        const uint64_t idx = (base + (uint64_t)lane * stride_elems * V) & mask;
        if (V == 4)
            red_add_v4f32(reinterpret_cast<float*>(buf) + idx, 1.0f, 1.0f, 1.0f, 1.0f);
        else if (sizeof(T) == 8)
            red_add_f64(reinterpret_cast<double*>(buf) + idx, 1.0);
        else
            red_add_f32(reinterpret_cast<float*>(buf) + idx, 1.0f);
        base += span * 4099;
    }
}

template <typename T>
__global__ void fma_kernel(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j);
    for (int r = 0; r < iters; ++r) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = x[j] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains
}

__global__ void lds_kernel(float* out, int iters) {
    __shared__ float4 s[1024];
    for (int q = threadIdx.x; q < 1024; q += blockDim.x)
        s[q] = make_float4((float)q, 1.0f, 2.0f, 3.0f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < iters; ++r) {
        const float4 v = s[(warp * 32 + lane + r * 32) & 1023];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = acc.x;
}

int status() { return cudaGetLastError() == cudaSuccess ? 0 : -3; }

}  // namespace

extern "C" {

// kind: 0 red.f32, 1 red.f64, 2 red.v4.f32 (buf: floats / doubles, n_elems a power of two).
// stride_elems: 32 (one line per lane) or 1 (consecutive).  Returns 0 or -3.
int lwp_red(int kind, void* buf, int64_t n_elems, int stride_elems, int blocks, int threads,
            int iters, void* stream) {
    if (!buf || n_elems < 1024 || (n_elems & (n_elems - 1)) || blocks < 1 || threads < 32 ||
        (threads & 31) || iters < 1 || (stride_elems != 1 && stride_elems != 32))
        return -1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t mask = (uint64_t)n_elems - 1;
    if (kind == 0)
        red_kernel<float, 1><<<blocks, threads, 0, st>>>(static_cast<float*>(buf), mask, iters,
                                                        stride_elems);
    else if (kind == 1)
        red_kernel<double, 1><<<blocks, threads, 0, st>>>(static_cast<double*>(buf), mask, iters,
                                                         stride_elems);
    else if (kind == 2)
        // v4: mask in floats, rounded down to a multiple of 4 so every vector stays inside
        red_kernel<float, 4><<<blocks, threads, 0, st>>>(static_cast<float*>(buf), mask & ~3ull,
                                                        iters, stride_elems);
    else
        return -1;
    return status();
}

// kind: 0 FP32, 1 FP64.  out: blocks * threads elements of the kind's type.
int lwp_fma(int kind, void* out, int blocks, int threads, int iters, void* stream) {
    if (!out || blocks < 1 || threads < 32 || iters < 1) return -1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (kind == 0)
        fma_kernel<float><<<blocks, threads, 0, st>>>(static_cast<float*>(out), iters, 0.999f,
                                                      0.001f);
    else if (kind == 1)
        fma_kernel<double><<<blocks, threads, 0, st>>>(static_cast<double*>(out), iters, 0.999,
                                                       0.001);
    else
        return -1;
    return status();
}

// out: blocks * threads floats.
int lwp_lds(float* out, int blocks, int threads, int iters, void* stream) {
    if (!out || blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1)
        return -1;
    lds_kernel<<<blocks, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters);
    return status();
}

}  // extern "C"
