// Trajectory upload (device layout) and observer-grid bounds.
//
// lw_trajectories_upload builds up to two device sections from the caller's
// FP64 trajectories:
//   FP64   plain copies of t, r, beta, beta_dot (inputs of the FP64 deposit);
//   MIXED  per sample a float4 (tau - tau_b, x - x_b, y - y_b, z - z_b) with the
//          light-front time tau = t - z/c0 taken relative to the first sample of
//          the sample's anchoring block, six floats of field data
//          (beta_x, beta_y, beta_dot_x, beta_dot_y, 1 - beta_z, beta_dot_z), and per block the anchor
//          (tau_b in FP64, x_b, y_b, z_b as FP32 pairs).  Subtracting the anchor in FP64 keeps the FP32
//          numbers small, so the FP32 part of the bin coordinate stays accurate.
// lw_grid_bounds evaluates Eqs. (tu_min) and (tu_max).
#include <math.h>

#include <algorithm>

#include "lw_internal.cuh"

namespace lw {
namespace {

// Buckets of the electron ordering (light-front time of the first sample).
constexpr int kOrderBuckets = 4096;

struct TrajLayout {
    size_t status = 0, ends = 0, t = 0, r = 0, beta = 0, beta_dot = 0, scan = 0, field = 0,
           anchor = 0, order = 0, order_tmp = 0;
    size_t total = 0;
    int64_t n_t = 0;
    int n_blocks = 0;
};

TrajLayout make_layout(int64_t n_e, int64_t n_s, int t_per_e, int sections, int block) {
    TrajLayout L;
    const int64_t ns1 = n_s + 1;
    L.n_t = (t_per_e ? n_e : 1) * ns1;
    L.n_blocks = (int)((ns1 + block - 1) / block);
    size_t off = 0;
    L.status = off;
    off = align256(off + sizeof(int32_t));
    L.ends = off;
    off = align256(off + sizeof(double) * 8 * (size_t)n_e);
    if (sections & LW_SECTION_FP64) {
        L.t = off;
        off = align256(off + sizeof(double) * (size_t)L.n_t);
        L.r = off;
        off = align256(off + sizeof(double) * 3 * (size_t)(n_e * ns1));
        L.beta = off;
        off = align256(off + sizeof(double) * 3 * (size_t)(n_e * ns1));
        L.beta_dot = off;
        off = align256(off + sizeof(double) * 3 * (size_t)(n_e * ns1));
    }
    if (sections & LW_SECTION_MIXED) {
        L.scan = off;
        off = align256(off + sizeof(float4) * (size_t)(n_e * ns1));
        L.field = off;
        off = align256(off + sizeof(float) * 6 * (size_t)(n_e * ns1));
        L.anchor = off;
        off = align256(off + sizeof(Anchor) * (size_t)(n_e * L.n_blocks));
    }
    L.order = off;
    off = align256(off + sizeof(int32_t) * (size_t)n_e);
    L.order_tmp = off;   // two ordered keys (range) + kOrderBuckets counters
    off = align256(off + 2 * sizeof(unsigned long long) + sizeof(int32_t) * kOrderBuckets);
    L.total = off;
    return L;
}

// One pass over the samples (CTA = 256 consecutive samples of one electron;
// grid x = sample chunks, y = electrons): input checks of every sample --
// finite values, |beta| < 1 (evaluated as ((bx*bx + by*by) + bz*bz) < 1),
// strictly increasing lab time, and with `check_steps` consecutive samples
// closer than c0 dt (LW_ST_STEP otherwise) -- and, when `scan` is non-null, the mixed
// section (block-relative float4, the field records as a float4 and a float2, per-block
// anchor).
// The [sample][3] inputs are copied into shared memory (cp.async, the next electron's chunk
// while this one is converted) so that every global load is a contiguous run; the outputs
// are one float4 and one float2 store per sample.
constexpr int kPrepThreads = 256;

// isfinite on the exponent bits (integer pipe; the FP64 pipe is the upload's bound)
__device__ __forceinline__ bool finite_bits(double v) {
    return ((__double2hiint(v) >> 20) & 0x7ff) != 0x7ff;
}


// Blocks (of at least 16 samples) that one chunk of kPrepThreads samples can meet.
constexpr int kChunkBlocks = kPrepThreads / 16 + 1;

__global__ void __launch_bounds__(kPrepThreads)
    prepare_kernel(const double* __restrict__ t, int t_per_e, const double* __restrict__ r,
                   const double* __restrict__ beta, const double* __restrict__ bdot, int64_t n_e,
                   int ns1, int block_shift, int n_blocks, float4* __restrict__ scan,
                   float4* __restrict__ field4, float2* __restrict__ field2,
                   Anchor* __restrict__ anchor, int check_steps, int32_t* __restrict__ status) {
    // two buffers: the next electron's chunk is copied in (cp.async) while this one is
    // converted, so the loads of one chunk overlap the arithmetic and stores of the other
    __shared__ double s_in[2][3][3 * kPrepThreads];   // r, beta, beta_dot of the chunk
    __shared__ double s_t[2][kPrepThreads];           // its times (per-electron time axes)
    __shared__ double s_blk[2][4][kChunkBlocks];      // (t, x, y, z) of its block starts
    __shared__ double s_taub[2][kChunkBlocks];        // their light-front times
    int bits = 0;
    const int i_first = blockIdx.x * kPrepThreads;
    const int cnt = min(kPrepThreads, ns1 - i_first);
    const int b_first = i_first >> block_shift;
    const int n_b = ((i_first + cnt - 1) >> block_shift) - b_first + 1;   // blocks met
    const int l = threadIdx.x;
    const int i = i_first + l;
    // a shared time axis is the same for every electron
    const double t_shared = (!t_per_e && l < cnt) ? t[i] : 0.0;
    auto prefetch = [&](int64_t k, int buf) {
        const int64_t s0 = k * ns1 + i_first;
        for (int q = l; q < 3 * cnt; q += kPrepThreads) {
            cp_async8(&s_in[buf][0][q], r + 3 * s0 + q);
            cp_async8(&s_in[buf][1][q], beta + 3 * s0 + q);
            cp_async8(&s_in[buf][2][q], bdot + 3 * s0 + q);
        }
        if (t_per_e && l < cnt) cp_async8(&s_t[buf][l], t + s0 + l);
        if (scan && l < n_b) {
            const int64_t sb = k * ns1 + ((int64_t)(b_first + l) << block_shift);
            cp_async8(&s_blk[buf][0][l], t + (t_per_e ? sb : sb - k * ns1));
            for (int c = 0; c < 3; ++c) cp_async8(&s_blk[buf][1 + c][l], r + 3 * sb + c);
        }
        cp_async_commit();
    };
    int buf = 0;
    if (blockIdx.y < n_e) prefetch(blockIdx.y, 0);
    for (int64_t k = blockIdx.y; k < n_e; k += gridDim.y, buf ^= 1) {
        const int64_t s0 = k * ns1 + i_first;
        const int64_t kn = k + gridDim.y;
        // the other buffer was released by the previous iteration's last barrier
        if (kn < n_e) {
            prefetch(kn, buf ^ 1);
            cp_async_wait_one();   // this chunk's group is complete, the next may be in flight
        } else {
            cp_async_wait_all();
        }
        // a block start's light-front time, by the thread that copied it (its own copies
        // are complete), once per block
        if (scan && l < n_b) s_taub[buf][l] = s_blk[buf][0][l] - s_blk[buf][3][l] * kInvC0;
        __syncthreads();
        const bool check_t = t_per_e || k == 0;
        if (l < cnt) {
            const int64_t s = s0 + l;
            // the staged values are read as (lo, hi) integer words: those that are only
            // checked and rounded to FP32 never become FP64 registers (which costs FP64-pipe
            // instructions, the pass's bound); FP64 values are formed where FP64 arithmetic
            // needs them
            const double* in0 = s_in[buf][0];
            const uint2* u1 = reinterpret_cast<const uint2*>(s_in[buf][1]);
            const uint2* u2 = reinterpret_cast<const uint2*>(s_in[buf][2]);
            const uint2* u0 = reinterpret_cast<const uint2*>(in0);
            const uint2 xu = u0[3 * l], yu = u0[3 * l + 1], zu = u0[3 * l + 2];
            const double x = __hiloint2double((int)xu.y, (int)xu.x);
            const double y = __hiloint2double((int)yu.y, (int)yu.x);
            const double z = __hiloint2double((int)zu.y, (int)zu.x);
            const uint2 b0u = u1[3 * l], b1u = u1[3 * l + 1], b2u = u1[3 * l + 2];
            const uint2 a0u = u2[3 * l], a1u = u2[3 * l + 1], a2u = u2[3 * l + 2];
            const double b2 = __hiloint2double((int)b2u.y, (int)b2u.x);
            const double ti = t_per_e ? s_t[buf][l] : t_shared;
            auto fu = [](uint2 v) { return ((v.y >> 20) & 0x7ffu) != 0x7ffu; };   // isfinite
            const bool fin = finite_bits(x) & finite_bits(y) & finite_bits(z) &
                             fu(b0u) & fu(b1u) & fu(b2u) & fu(a0u) & fu(a1u) & fu(a2u) &
                             finite_bits(ti);
            if (!fin) bits |= LW_ST_NONFINITE;
            // |beta| < 1: decided in FP32 when 1 - beta^2 is far above its FP32 rounding,
            // else by the FP64 expression ((bx*bx + by*by) + bz*bz) < 1
            const float b0f = to_float_bits(b0u.y, b0u.x), b1f = to_float_bits(b1u.y, b1u.x);
            const float epsf = to_float(1.0 - b2);   // exact in FP64 for b2 in [0.5, 2]
            const float perp = fmaf(b0f, b0f, b1f * b1f);
            const float one_minus = fmaf(-epsf, epsf, 2.0f * epsf) - perp;   // 1 - beta^2
            // b2 >= 0.5 on the bits: non-negative and exponent >= -1 (NaN goes on to the
            // FP64 test and fails it)
            const bool b2_half = __double2hiint(b2) >= 0x3fe00000;
            if (!(b2_half && one_minus > 1.0e-5f * (2.0f * epsf + perp))) {
                const double b0 = __hiloint2double((int)b0u.y, (int)b0u.x);
                const double b1 = __hiloint2double((int)b1u.y, (int)b1u.x);
                const double bb = __dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)),
                                            __dmul_rn(b2, b2));
                if (!(bb < 1.0)) bits |= LW_ST_BETA;
            }
            const double* tk = t + (t_per_e ? k * ns1 : 0);
            if (check_t && i > 0 && !(ti > tk[i - 1])) bits |= LW_ST_TIME;
            if (check_steps && i > 0) {   // |r_i - r_(i-1)| < c0 (t_i - t_(i-1)), in FP64
                const double* pr = l > 0 ? &in0[3 * (l - 1)] : r + 3 * (s - 1);
                const double dx = x - pr[0], dy = y - pr[1], dz = z - pr[2];
                const double ct = kC0 * (ti - tk[i - 1]);
                if (!(dx * dx + dy * dy + dz * dz < ct * ct)) bits |= LW_ST_STEP;
            }
            if (scan) {
                const int ib = (i >> block_shift) << block_shift;
                const int jb = (i >> block_shift) - b_first;
                const double xb = s_blk[buf][1][jb], yb = s_blk[buf][2][jb],
                             zb = s_blk[buf][3][jb];
                const double tau = ti - z * kInvC0;
                const double taub = s_taub[buf][jb];
                scan[s] = make_float4(to_float(tau - taub), to_float(x - xb), to_float(y - yb),
                                      to_float(z - zb));
                // (beta_x, beta_y, beta_dot_x, beta_dot_y) and (1 - beta_z, beta_dot_z): one
                // 16-byte and one 8-byte record, each a single shared-memory load in the
                // deposit; the x and y pairs are operands of its packed FP32x2 arithmetic
                field4[s] = make_float4(b0f, b1f, to_float_bits(a0u.y, a0u.x),
                                        to_float_bits(a1u.y, a1u.x));
                field2[s] = make_float2(epsf, to_float_bits(a2u.y, a2u.x));
                if (i == ib) {   // position as FP32 pairs: hi = fl32(x), lo = fl32(x - hi)
                    Anchor an;
                    an.tau = taub;
                    an.x_hi = __double2float_rn(xb);
                    an.x_lo = __double2float_rn(xb - (double)an.x_hi);
                    an.y_hi = __double2float_rn(yb);
                    an.y_lo = __double2float_rn(yb - (double)an.y_hi);
                    an.z_hi = __double2float_rn(zb);
                    an.z_lo = __double2float_rn(zb - (double)an.z_hi);
                    anchor[k * n_blocks + (i >> block_shift)] = an;
                }
            }
        }
        __syncthreads();   // both buffers are free for the next prefetch
    }
    block_status_or(status, bits);
}

__global__ void ends_kernel(const double* __restrict__ t, int t_per_e,
                            const double* __restrict__ r, int64_t n_e, int64_t ns1,
                            double* __restrict__ ends) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_e;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double* tk = t + (t_per_e ? k * ns1 : 0);
        const double* x0 = r + 3 * (k * ns1);
        const double* x1 = r + 3 * (k * ns1 + ns1 - 1);
        double* e = ends + 8 * k;
        e[0] = tk[0];
        e[1] = x0[0];
        e[2] = x0[1];
        e[3] = x0[2];
        e[4] = tk[ns1 - 1];
        e[5] = x1[0];
        e[6] = x1[1];
        e[7] = x1[2];
    }
}

// Electron ordering for the mixed deposit: electrons sorted (by buckets of
// 1/kOrderBuckets of the range) on the light-front time tau = t - z/c0 of their
// first sample, which orders their arrival at detectors near the z axis.  The
// deposit visits electrons in this order, so the electrons in flight at any
// time update a narrow band of observer bins.
__device__ __forceinline__ double first_tau(const double* e) { return e[0] - e[3] * kInvC0; }

__global__ void order_range_kernel(const double* __restrict__ ends, int64_t n_e,
                                   unsigned long long* keys) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_e;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double v = first_tau(ends + 8 * k);
        if (isfinite(v)) {
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&keys[0], ordered_key(lo));
        atomicMax(&keys[1], ordered_key(hi));
    }
}

__device__ __forceinline__ int order_bucket(const double* e, const unsigned long long* keys) {
    const double lo = key_to_double(keys[0]), hi = key_to_double(keys[1]);
    const double v = first_tau(e);
    if (!(hi > lo) || !isfinite(v)) return 0;
    const double x = (v - lo) / (hi - lo) * kOrderBuckets;
    return (int)fmin(fmax(x, 0.0), (double)(kOrderBuckets - 1));
}

__global__ void order_count_kernel(const double* __restrict__ ends, int64_t n_e,
                                   const unsigned long long* __restrict__ keys,
                                   int32_t* __restrict__ counts) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_e;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&counts[order_bucket(ends + 8 * k, keys)], 1);
}

// Exclusive prefix sum of the bucket counts, in place (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) order_scan_kernel(int32_t* counts) {
    constexpr int kPer = kOrderBuckets / 1024;
    __shared__ int32_t s_sum[1024];
    int32_t v[kPer];
    int32_t sum = 0;
    for (int i = 0; i < kPer; ++i) {
        v[i] = counts[threadIdx.x * kPer + i];
        sum += v[i];
    }
    s_sum[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {   // Hillis-Steele inclusive scan of the sums
        const int32_t add = threadIdx.x >= d ? s_sum[threadIdx.x - d] : 0;
        __syncthreads();
        s_sum[threadIdx.x] += add;
        __syncthreads();
    }
    int32_t run = s_sum[threadIdx.x] - sum;
    for (int i = 0; i < kPer; ++i) {
        counts[threadIdx.x * kPer + i] = run;
        run += v[i];
    }
}

__global__ void order_scatter_kernel(const double* __restrict__ ends, int64_t n_e,
                                     const unsigned long long* __restrict__ keys,
                                     int32_t* __restrict__ offsets, int32_t* __restrict__ order) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_e;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&offsets[order_bucket(ends + 8 * k, keys)], 1);
        order[pos] = (int32_t)k;
    }
}

__global__ void bounds_init_kernel(unsigned long long* keys) {
    keys[0] = ordered_key(INFINITY);
    keys[1] = ordered_key(-INFINITY);
}

// One thread per (pixel, electron); Eqs. (tu_min), (tu_max).
__global__ void bounds_kernel(const double* __restrict__ ends, int64_t n_e,
                              const double* __restrict__ n_hat, int64_t n_pix,
                              unsigned long long* keys) {
    double lo = INFINITY, hi = -INFINITY;
    const int64_t total = n_e * n_pix;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = s / n_e;
        const int64_t k = s - m * n_e;
        const double nx = n_hat[3 * m], ny = n_hat[3 * m + 1], nz = n_hat[3 * m + 2];
        const double* e = ends + 8 * k;
        double a0 = advanced_time_fp64(nx, ny, nz, e[1], e[2], e[3], e[0]);
        double a1 = advanced_time_fp64(nx, ny, nz, e[5], e[6], e[7], e[4]);
        lo = fmin(lo, a0);
        hi = fmax(hi, a1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&keys[0], ordered_key(lo));
        atomicMax(&keys[1], ordered_key(hi));
    }
}

__global__ void bounds_finish_kernel(unsigned long long* keys) {
    double* out = reinterpret_cast<double*>(keys);
    double lo = key_to_double(keys[0]);
    double hi = key_to_double(keys[1]);
    out[0] = lo;
    out[1] = hi;
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)kSms * 32;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace
}  // namespace lw

using namespace lw;

extern "C" int lw_trajectories_upload(const lw_traj_in* in, int32_t sections, int32_t block,
                                      void* ws, size_t* ws_bytes, lw_traj* out, void* stream) {
    if (!in || !ws_bytes || !out) return LW_EINVAL;
    if (in->n_e < 1 || in->n_s < 1) return LW_EINVAL;
    if (in->n_s >= (int64_t(1) << 30) || in->n_e >= (int64_t(1) << 31)) return LW_EUNSUPPORTED;
    if (!in->t || !in->r || !in->beta || !in->beta_dot) return LW_EINVAL;
    if (sections <= 0 || (sections & ~(LW_SECTION_FP64 | LW_SECTION_MIXED))) return LW_EINVAL;
    if (block == 0) block = 512;
    if (block < 16 || block > 1024 || (block & (block - 1))) return LW_EINVAL;
    const int t_per_e = in->t_per_electron ? 1 : 0;
    const TrajLayout L = make_layout(in->n_e, in->n_s, t_per_e, sections, block);
    if (!ws) {
        *ws_bytes = L.total;
        return LW_OK;
    }
    if (*ws_bytes < L.total) {
        *ws_bytes = L.total;
        return LW_ESIZE;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) return LW_EINVAL;
    cudaStream_t st = as_stream(stream);
    char* base = static_cast<char*>(ws);
    const int64_t ns1 = in->n_s + 1;
    const size_t vec_bytes = sizeof(double) * 3 * (size_t)(in->n_e * ns1);

    lw_traj v{};
    v.n_e = in->n_e;
    v.n_s = in->n_s;
    v.t_per_electron = t_per_e;
    v.sections = sections;
    v.block = block;
    v.n_blocks = L.n_blocks;
    int32_t* status = reinterpret_cast<int32_t*>(base + L.status);
    v.input_status = status;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return LW_ECUDA;

    const double *t = in->t, *r = in->r, *beta = in->beta, *bdot = in->beta_dot;
    if (sections & LW_SECTION_FP64) {
        double* dt = reinterpret_cast<double*>(base + L.t);
        double* dr = reinterpret_cast<double*>(base + L.r);
        double* db = reinterpret_cast<double*>(base + L.beta);
        double* dd = reinterpret_cast<double*>(base + L.beta_dot);
        if (cudaMemcpyAsync(dt, in->t, sizeof(double) * (size_t)L.n_t, cudaMemcpyDefault, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(dr, in->r, vec_bytes, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaMemcpyAsync(db, in->beta, vec_bytes, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaMemcpyAsync(dd, in->beta_dot, vec_bytes, cudaMemcpyDefault, st) != cudaSuccess)
            return LW_ECUDA;
        v.t = dt;
        v.r = dr;
        v.beta = db;
        v.beta_dot = dd;
        t = dt;
        r = dr;
        beta = db;
        bdot = dd;
    }
    const int threads = 256;
    double* ends = reinterpret_cast<double*>(base + L.ends);
    ends_kernel<<<grid_for(in->n_e, threads), threads, 0, st>>>(t, t_per_e, r, in->n_e, ns1,
                                                                 ends);
    if (launch_status() != LW_OK) return LW_ECUDA;
    v.ends = ends;
    float4* scan = nullptr;
    float* field = nullptr;
    Anchor* anchor = nullptr;
    if (sections & LW_SECTION_MIXED) {
        scan = reinterpret_cast<float4*>(base + L.scan);
        field = reinterpret_cast<float*>(base + L.field);
        anchor = reinterpret_cast<Anchor*>(base + L.anchor);
        v.scan = scan;
        v.field = field;
        v.anchor = reinterpret_cast<const double*>(anchor);
    }
    int shift = 0;
    while ((1 << shift) < block) ++shift;
    const dim3 g((unsigned)((ns1 + kPrepThreads - 1) / kPrepThreads),
                 (unsigned)std::min<int64_t>(in->n_e, 65535));
    prepare_kernel<<<g, kPrepThreads, 0, st>>>(t, t_per_e, r, beta, bdot, in->n_e, (int)ns1, shift,
                                          L.n_blocks, scan, reinterpret_cast<float4*>(field),
                                          field ? reinterpret_cast<float2*>(
                                                      field + 4 * (size_t)(in->n_e * ns1))
                                                : nullptr,
                                          anchor,
                                          (sections & LW_SECTION_FP64) ? 1 : 0, status);
    if (launch_status() != LW_OK) return LW_ECUDA;
    {
        int32_t* order = reinterpret_cast<int32_t*>(base + L.order);
        unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + L.order_tmp);
        int32_t* counts = reinterpret_cast<int32_t*>(keys + 2);
        if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * kOrderBuckets, st) != cudaSuccess)
            return LW_ECUDA;
        bounds_init_kernel<<<1, 1, 0, st>>>(keys);
        const int ge = grid_for(in->n_e, threads);
        order_range_kernel<<<ge, threads, 0, st>>>(ends, in->n_e, keys);
        order_count_kernel<<<ge, threads, 0, st>>>(ends, in->n_e, keys, counts);
        order_scan_kernel<<<1, 1024, 0, st>>>(counts);
        order_scatter_kernel<<<ge, threads, 0, st>>>(ends, in->n_e, keys, counts, order);
        if (launch_status() != LW_OK) return LW_ECUDA;
        v.order = order;
    }
    *out = v;
    *ws_bytes = L.total;
    return LW_OK;
}

extern "C" int lw_grid_bounds(const lw_traj* traj, const lw_detector* det, double* bounds,
                              void* stream) {
    if (!traj || !det || !bounds || !det->n_hat || det->n_pix < 1) return LW_EINVAL;
    if (!traj->ends || traj->n_e < 1) return LW_EINVAL;
    cudaStream_t st = as_stream(stream);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(bounds);
    bounds_init_kernel<<<1, 1, 0, st>>>(keys);
    if (launch_status() != LW_OK) return LW_ECUDA;
    const int threads = 256;
    bounds_kernel<<<grid_for(traj->n_e * det->n_pix, threads), threads, 0, st>>>(
        traj->ends, traj->n_e, det->n_hat, det->n_pix, keys);
    if (launch_status() != LW_OK) return LW_ECUDA;
    bounds_finish_kernel<<<1, 1, 0, st>>>(keys);
    return launch_status();
}
