// Time-domain deposit (Algorithm 2 of the paper) for every pixel.
//
// Thread mapping (both precisions): one thread owns one (mixed: PIX) detector
// pixel(s) -- the paper's "detector parallelization" on one GPU -- and a CTA
// walks a chunk of electrons; the samples of the current electron are staged
// in shared memory once per CTA and read by all of its pixels as broadcasts.
// The field (Eq. far_efield) and the interpolation weights are evaluated only
// for steps whose interval (t_b, t_a] contains grid points, and those
// contributions are added to the record with global atomics (pixels of
// different CTAs share bins through electrons of other chunks).
//
// FP64 path: every step costs the time map and one compare.  Every operation
// of the time map, the bin index, the field and the weights is written with
// explicit round-to-nearest intrinsics in the order documented in lw.h, so
// advanced times, bin indices and per-sample contributions are bit-identical
// to a plain C loop without FMA contraction; only the order of the atomic
// additions differs.
//
// Mixed path: the bin coordinate u = (t_a - t_min)/dt_u is anchored once per
// block of samples in double-FP32 arithmetic (integer part + FP32 fraction)
// and evaluated per sample with three FP32 FMAs of small, block-relative
// quantities.  Because t_a increases along a subluminal trajectory, a block
// needs one coordinate per pixel (its last sample) to know which grid points
// it reaches; each grid point's step is then found by a bracketed search
// (regula falsi, then bisection) over the staged block.  The field is FP32 in
// the stable form
//   D = (1 - n_z) + n_z (1 - beta_z) - n_perp . beta_perp,
// and contributions are added with FP64 atomics, a compensated pair of FP32
// atomics, or FP32 atomics (the three mixed records).
#include <math.h>

#include <algorithm>
#include <vector>

#include "lw_internal.cuh"

namespace lw {
namespace {

struct DepositArgs {
    int64_t n_e, ns1;
    int t_per_e;
    const double* t;
    const double* r;
    const double* beta;
    const double* bdot;
    const float4* scan;
    const float4* field4;    // (beta_x, beta_y, beta_dot_x, beta_dot_y) per sample
    const float2* field2;    // (1 - beta_z, beta_dot_z) per sample
    const Anchor* anchor;
    int block, n_blocks;
    const int32_t* input_status;
    const double* ends;
    const int32_t* order;   // mixed: electron visiting order (may be null)
    const double* n_hat;
    int64_t n_pix;
    double R;
    double t_min, dt_u, inv_dtu;
    // FP32 constants of the mixed path, rounded once on the host: 1/dt_u, c0 dt_u (a pixel
    // direction from its slope) and c0/R (velocity field).  Kernel parameters can be FMA
    // operands directly; a value converted from the FP64 fields inside the kernel would
    // be recomputed on the FP64 pipe wherever the compiler chooses not to keep it.
    float s32, inv_sc, c0_over_R;
    int64_t n_bins;
    uint32_t flags;
    void* record;
    int32_t* status;
    int e_chunk;
};

// ------------------------------------------------------------------ FP64

constexpr int kFp64Threads = 128;
constexpr int kFp64Tile = 64;

// Field of one sample with the oracle's operation order (see lw.h).
__device__ int field_fp64(double nx, double ny, double nz, double R, uint32_t flags,
                          const double* __restrict__ b, const double* __restrict__ a,
                          double F[3]) {
    F[0] = F[1] = F[2] = 0.0;
    const double b0 = b[0], b1 = b[1], b2v = b[2];
    const double bb = __dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)),
                                __dmul_rn(b2v, b2v));
    const double nb = __dadd_rn(__dadd_rn(__dmul_rn(nx, b0), __dmul_rn(ny, b1)),
                                __dmul_rn(nz, b2v));
    const double D = __dsub_rn(1.0, nb);
    if (!(bb < 1.0) || !(D > 0.0)) return LW_ST_BETA;
    const double D3 = __dmul_rn(__dmul_rn(D, D), D);
    const double m0 = __dsub_rn(nx, b0), m1 = __dsub_rn(ny, b1), m2 = __dsub_rn(nz, b2v);
    if (flags & LW_FIELD_ACCEL) {
        const double a0 = a[0], a1 = a[1], a2 = a[2];
        // inner = (n - beta) x beta_dot
        const double i0 = __dsub_rn(__dmul_rn(m1, a2), __dmul_rn(m2, a1));
        const double i1 = __dsub_rn(__dmul_rn(m2, a0), __dmul_rn(m0, a2));
        const double i2 = __dsub_rn(__dmul_rn(m0, a1), __dmul_rn(m1, a0));
        // outer = n x inner
        const double o0 = __dsub_rn(__dmul_rn(ny, i2), __dmul_rn(nz, i1));
        const double o1 = __dsub_rn(__dmul_rn(nz, i0), __dmul_rn(nx, i2));
        const double o2 = __dsub_rn(__dmul_rn(nx, i1), __dmul_rn(ny, i0));
        F[0] = __ddiv_rn(o0, D3);
        F[1] = __ddiv_rn(o1, D3);
        F[2] = __ddiv_rn(o2, D3);
    }
    if (flags & LW_FIELD_VELOCITY) {
        const double g = __ddiv_rn(__dmul_rn(kC0, __dsub_rn(1.0, bb)), __dmul_rn(D3, R));
        F[0] = __dadd_rn(F[0], __dmul_rn(m0, g));
        F[1] = __dadd_rn(F[1], __dmul_rn(m1, g));
        F[2] = __dadd_rn(F[2], __dmul_rn(m2, g));
    }
    return 0;
}

// State of Algorithm 2's walk over one (pixel, electron): the previous sample's
// advanced time, coordinate and field.
struct ScanState {
    double tb, ub;
    bool ok_b;
    double Fb[3];
    int64_t fb_step;
    __device__ void reset() {
        tb = ub = 0.0;
        ok_b = false;
        Fb[0] = Fb[1] = Fb[2] = 0.0;
        fb_step = -1;
    }
};

// One sample i = (t, x, y, z) of Algorithm 2's walk for the pixel (nx, ny, nz): the
// step (t_a,i-1, t_a,i] deposits every grid point it holds, in the oracle's order.
__device__ __forceinline__ void scan_sample(const DepositArgs& p, double nx, double ny,
                                            double nz, double* rec, const double* bk,
                                            const double* ak, int64_t i, double t, double x,
                                            double y, double z, ScanState& S, int& bits) {
    const double ta = advanced_time_fp64(nx, ny, nz, x, y, z, t);
    const double ua = __dmul_rn(__dsub_rn(ta, p.t_min), p.inv_dtu);
    const bool ok_a = fabs(ua) < 4.0e18;
    if (i > 0) {
        if (!ok_a || !S.ok_b) {
            bits |= LW_ST_NONFINITE;
        } else {
            const int64_t j_hi = (int64_t)floor(ua);
            const int64_t j_lo = (int64_t)floor(S.ub) + 1;
            if (!(ta > S.tb)) bits |= LW_ST_TA_ORDER;
            if (j_lo <= j_hi) {
                int64_t ja = j_lo, jz = j_hi;
                if (ja < 0) {
                    ja = 0;
                    bits |= LW_ST_CLIP;
                }
                if (jz > p.n_bins - 1) {
                    jz = p.n_bins - 1;
                    bits |= LW_ST_CLIP;
                }
                if (ja <= jz) {
                    if (S.fb_step != i - 1)
                        field_fp64(nx, ny, nz, p.R, p.flags, bk + 3 * (i - 1), ak + 3 * (i - 1),
                                   S.Fb);
                    double Fa[3];
                    field_fp64(nx, ny, nz, p.R, p.flags, bk + 3 * i, ak + 3 * i, Fa);
                    const double den = __dsub_rn(ta, S.tb);
                    for (int64_t j = ja; j <= jz; ++j) {
                        const double tu = __dadd_rn(p.t_min, __dmul_rn((double)j, p.dt_u));
                        const double wa = __ddiv_rn(__dsub_rn(ta, tu), den);
                        const double wb = __ddiv_rn(__dsub_rn(tu, S.tb), den);
                        for (int c = 0; c < 3; ++c)
                            atomicAdd(rec + c * p.n_bins + j,
                                      __dadd_rn(__dmul_rn(S.Fb[c], wa), __dmul_rn(Fa[c], wb)));
                    }
                    S.Fb[0] = Fa[0];
                    S.Fb[1] = Fa[1];
                    S.Fb[2] = Fa[2];
                    S.fb_step = i;
                }
            }
        }
    }
    S.tb = ta;
    S.ub = ua;
    S.ok_b = ok_a;
}

// Algorithm 2 literally: every step of every (pixel, electron), in the oracle's
// operation order (CTA = kFp64Threads pixels x p.e_chunk electrons).
__device__ void fp64_scan_cta(const DepositArgs& p) {
    __shared__ double s_t[kFp64Tile];
    __shared__ double s_r[kFp64Tile * 3];
    const int64_t m = (int64_t)blockIdx.x * kFp64Threads + threadIdx.x;
    const bool active = m < p.n_pix;
    double nx = 0.0, ny = 0.0, nz = 1.0;
    if (active) {
        nx = p.n_hat[3 * m];
        ny = p.n_hat[3 * m + 1];
        nz = p.n_hat[3 * m + 2];
    }
    double* rec = static_cast<double*>(p.record) + (active ? m * 3 * p.n_bins : 0);
    int bits = 0;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && p.input_status)
        bits |= *p.input_status;
    const int64_t k0 = (int64_t)blockIdx.y * p.e_chunk;
    const int64_t k1 = min(k0 + p.e_chunk, p.n_e);
    for (int64_t k = k0; k < k1; ++k) {
        const double* tk = p.t + (p.t_per_e ? k * p.ns1 : 0);
        const double* rk = p.r + 3 * k * p.ns1;
        const double* bk = p.beta + 3 * k * p.ns1;
        const double* ak = p.bdot + 3 * k * p.ns1;
        ScanState S;
        S.reset();
        for (int64_t i0 = 0; i0 < p.ns1; i0 += kFp64Tile) {
            const int n = (int)min((int64_t)kFp64Tile, p.ns1 - i0);
            __syncthreads();
            for (int q = threadIdx.x; q < n; q += kFp64Threads) {
                s_t[q] = tk[i0 + q];
                s_r[3 * q] = rk[3 * (i0 + q)];
                s_r[3 * q + 1] = rk[3 * (i0 + q) + 1];
                s_r[3 * q + 2] = rk[3 * (i0 + q) + 2];
            }
            __syncthreads();
            if (!active) continue;
            for (int q = 0; q < n; ++q)
                scan_sample(p, nx, ny, nz, rec, bk, ak, i0 + q, s_t[q], s_r[3 * q],
                            s_r[3 * q + 1], s_r[3 * q + 2], S, bits);
        }
    }
    block_status_or(p.status, bits);
}

// ------------------------------------------------------------------ mixed

constexpr int kMixThreads = 256;
constexpr int kMixPix = 2;            // pixels per thread: tiles of 512 pixels
#ifndef LW_MIX_MIN_BLOCKS
#define LW_MIX_MIN_BLOCKS 3
#endif
constexpr int kMixMinBlocks = LW_MIX_MIN_BLOCKS;   // resident CTAs per SM
#ifndef LW_MIX_MAX_CHUNK
#define LW_MIX_MAX_CHUNK 1
#endif
constexpr int kMixMaxChunk = LW_MIX_MAX_CHUNK;   // electrons per CTA at most
// With the interleaved record one L2 sector takes a grid point's update, so a wider band of
// electrons in flight costs little and several electrons per CTA share its pixel set-up.
#ifndef LW_MIX_MAX_CHUNK_X4
#define LW_MIX_MAX_CHUNK_X4 4
#endif
constexpr int kMixMaxChunkX4 = LW_MIX_MAX_CHUNK_X4;

struct DF {   // unevaluated sum hi + lo of two floats
    float hi, lo;
};

__device__ __forceinline__ DF split_double(double x) {
    DF r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - (double)r.hi);
    return r;
}

// Compensated atomic accumulation into a (sum, compensation) pair: the
// rounding error of the atomic add is recovered exactly from the returned old
// value (two-sum) and added to the compensation word.
__device__ __forceinline__ void kahan_atomic_add(float2* p, float v) {
    const float old = atomicAdd(&p->x, v);
    const float s = __fadd_rn(old, v);
    const float bb = __fsub_rn(s, old);
    const float err = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    if (err != 0.0f) atomicAdd(&p->y, err);
}

struct PixelConst {
    float nx, ny, nz, omnz;   // direction and 1 - n_z (stable)
};

// rcp.approx.ftz.f32: the reciprocal to about 1 ulp, far below the FP32 field's own error
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per-sample FP32 field in the stable form, for the field terms FL (LW_FIELD_* mask, a
// compile-time constant); zero if D <= 0.
// f4 = (beta_x, beta_y, beta_dot_x, beta_dot_y), f2 = (1 - beta_z, beta_dot_z).
template <int FL>
__device__ __forceinline__ void field_fp32(const PixelConst& pc, float4 f4, float2 f2,
                                           float c0_over_R, float F[3]) {
    const float bx = f4.x, by = f4.y, eps = f2.x;
    const float ax = f4.z, ay = f4.w, az = f2.y;
    const float D = fmaf(-pc.ny, by, fmaf(-pc.nx, bx, fmaf(pc.nz, eps, pc.omnz)));
    const float mx = pc.nx - bx, my = pc.ny - by, mz = eps - pc.omnz;
    const float invD = rcp_approx(D);
    const float invD3 = invD * invD * invD;
    float F0 = 0.0f, F1 = 0.0f, F2 = 0.0f;
    if (FL & LW_FIELD_ACCEL) {
        const float na = fmaf(pc.nz, az, fmaf(pc.ny, ay, pc.nx * ax));
        F0 = fmaf(mx, na, -D * ax) * invD3;
        F1 = fmaf(my, na, -D * ay) * invD3;
        F2 = fmaf(mz, na, -D * az) * invD3;
    }
    if (FL & LW_FIELD_VELOCITY) {
        const float g2 = fmaf(-by, by, fmaf(-bx, bx, eps * (2.0f - eps)));   // 1 - beta^2
        const float g = c0_over_R * g2 * invD3;
        F0 = fmaf(mx, g, F0);
        F1 = fmaf(my, g, F1);
        F2 = fmaf(mz, g, F2);
    }
    const bool ok = D > 0.0f;   // selects: no branch around the loads
    F[0] = ok ? F0 : 0.0f;
    F[1] = ok ? F1 : 0.0f;
    F[2] = ok ? F2 : 0.0f;
}

// One end of a step for the deposit, with Eq. far_efield expanded: since n . (n - beta) =
// D, n x ((n - beta) x beta_dot) / D^3 = (k m - beta_dot) / D^2 with m = n - beta and
// k = n . beta_dot / D; the velocity field adds c0/R (1 - beta^2) / D to k.  Returns
// k m - beta_dot (x and y packed for the FP32x2 instructions, z) and the scale
// weight / D^2 (zero if D <= 0), so that the interpolated value is t_a s_a + t_b s_b.
template <int FL>
__device__ __forceinline__ void end_terms(const PixelConst& pc, float2 nxy, float4 f4, float2 ez,
                                          float c0_over_R, float weight, float2& txy,
                                          float& tz, float& sc) {
    const float2 b = make_float2(f4.x, f4.y), a = make_float2(f4.z, f4.w);   // beta, beta_dot
    const float D = fmaf(-pc.ny, b.y, fmaf(-pc.nx, b.x, fmaf(pc.nz, ez.x, pc.omnz)));
    const float2 m = __ffma2_rn(b, make_float2(-1.0f, -1.0f), nxy);
    const float mz = ez.x - pc.omnz;
    const float invD = rcp_approx(D);
    float k = 0.0f;
    if (FL & LW_FIELD_ACCEL) k = fmaf(pc.nz, ez.y, fmaf(pc.ny, a.y, pc.nx * a.x)) * invD;
    if (FL & LW_FIELD_VELOCITY) {
        const float g2 = fmaf(-b.y, b.y, fmaf(-b.x, b.x, ez.x * (2.0f - ez.x)));   // 1 - beta^2
        k = fmaf(c0_over_R * g2, invD, k);
    }
    if (FL & LW_FIELD_ACCEL) {
        txy = __ffma2_rn(m, make_float2(k, k), make_float2(-a.x, -a.y));
        tz = fmaf(mz, k, -ez.y);
    } else {
        txy = __fmul2_rn(m, make_float2(k, k));
        tz = mz * k;
    }
    sc = D > 0.0f ? weight * (invD * invD) : 0.0f;
}

// Grid points of one pixel and block above which the owning lane deposits them
// itself instead of handing them to the warp (keeps the warp's job count in int).
constexpr int kMaxWarpJobs = 1 << 20;
// Jobs of a warp and block listed explicitly (slot, grid point); later ones are
// located by bisection over the slots' job offsets.
constexpr int kJobTable = 128;
// Step searches: regula falsi (linear interpolation inside the bracket) for this many
// probes, then bisection.  On Boris trajectories of a 10,000-electron bunch in a
// 0.8 um laser (10,000 steps, 64 x 64 pixels, 65,536 bins) it needs 2.1 probes per grid point
// on average (at most 5); alternating interpolation and bisection needed 3.2.
constexpr int kFalsiProbes = 8;

// Record accumulation of the mixed modes: FP64 (red.global.add.f64), compensated FP32
// pair, FP32 (red.global.add.f32), or FP32 interleaved per grid point as (x, y, z, 0) and
// added by one vector reduction (red.global.add.v4.f32: one L2 sector operation instead of
// three).
enum { kAccF64 = 0, kAccKahan = 1, kAccF32 = 2, kAccF32X4 = 3 };

template <int ACC>
__device__ __forceinline__ void accumulate(void* rec, int64_t idx, float v) {
    if (ACC == kAccKahan) {
        kahan_atomic_add(static_cast<float2*>(rec) + idx, v);
    } else if (ACC == kAccF32) {
        atomicAdd(static_cast<float*>(rec) + idx, v);
    } else {
        atomicAdd(static_cast<double*>(rec) + idx, (double)v);
    }
}

// Adds the three components (v0, v1, v2) of grid point j to the pixel row starting at
// `row` (the pixel's [3][N] values, or its [N][4] floats for the interleaved record).
template <int ACC>
__device__ __forceinline__ void deposit3_row(unsigned char* row, int j, int64_t n_bins,
                                             float v0, float v1, float v2) {
    if (ACC == kAccF32X4) {
        float* p = reinterpret_cast<float*>(row + 16ull * (unsigned)j);
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v0),
                     "f"(v1), "f"(v2), "f"(0.0f)
                     : "memory");
    } else {
        accumulate<ACC>(row, j, v0);
        accumulate<ACC>(row, j + n_bins, v1);
        accumulate<ACC>(row, j + 2 * n_bins, v2);
    }
}

// Accumulation form and record size of a precision.
__host__ __device__ constexpr int acc_of(int precision) {
    return precision == LW_MIXED_KAHAN ? kAccKahan
           : precision == LW_MIXED_F32 ? kAccF32
           : precision == LW_MIXED_F32X4 ? kAccF32X4 : kAccF64;
}
// 4-byte words per (pixel, grid point): three doubles or float pairs, three floats, or
// one float4
__host__ __device__ constexpr int record_words(int precision) {
    return precision == LW_MIXED_F32 ? 3 : precision == LW_MIXED_F32X4 ? 4 : 6;
}

// FP64 bin index of a trajectory end sample, with the FP64 path's operation order.
__device__ __forceinline__ int exact_bin(const double* e, double nx, double ny, double nz,
                                         double t_min, double inv_dtu) {
    const double ta = advanced_time_fp64(nx, ny, nz, e[1], e[2], e[3], e[0]);
    double u = __dmul_rn(__dsub_rn(ta, t_min), inv_dtu);
    u = fmin(fmax(u, -1.0e9), 1.0e9);
    return (int)floor(u);
}

// The same, kept out of line: the mixed deposit needs it only for trajectory end samples
// whose mixed bin coordinate lies within rounding of an integer, and a call keeps its
// FP64 instructions out of the common path.
__device__ __noinline__ int exact_bin_rare(const double* e, const double* n, double t_min,
                                           double inv_dtu) {
    return exact_bin(e, n[0], n[1], n[2], t_min, inv_dtu);
}

// Bin coordinate of a staged sample relative to its block's anchor, without the
// anchor fraction f: u - I - f = s dtau + w . dr, with sc = (dtau, dr) and
// w = (w_x, w_y, w_z) the pixel's slope (FP32 hi parts), s = 1/dt_u.
__device__ __forceinline__ float coord(float4 w, float s, float4 sc) {
    return fmaf(w.z, sc.w, fmaf(w.y, sc.z, fmaf(w.x, sc.y, s * sc.x)));
}

// Staging of the mixed deposit: a ring of kMixStages shared buffers filled by the
// tensor memory accelerator's bulk copies (cp.async.bulk, issued by one thread,
// completion counted in bytes on one mbarrier per buffer), kMixStages - 1 blocks ahead
// of the block being processed.  One buffer holds block b's samples i0 .. i0+B-1 as
// float4 (block-relative light-front time and position), the field records of samples
// i0 .. i0+B (the next block's first sample included) as a float4 array and a float2
// array and, with block 0 and with every block b of b % 32 == 31, the FP64 anchors of the
// next 32 blocks.
#ifndef LW_MIX_STAGES
#define LW_MIX_STAGES 2
#endif
constexpr int kMixStages = LW_MIX_STAGES;
constexpr int kAnchorBatch = 32;
__host__ __device__ constexpr size_t stage_f4_off(int B) { return 16 * (size_t)B; }
__host__ __device__ constexpr size_t stage_f2_off(int B) {
    return stage_f4_off(B) + 16 * ((size_t)B + 1);
}
__host__ __device__ constexpr size_t stage_anchor_off(int B) {
    // float2 records: 8 (B + 1) bytes copied from a 16-byte aligned start up to 8 bytes early
    return (stage_f2_off(B) + 8 * ((size_t)B + 1) + 8 + 15 + 31) / 32 * 32;
}
__host__ __device__ constexpr size_t stage_bytes(int B) {
    return stage_anchor_off(B) + sizeof(Anchor) * kAnchorBatch;
}

// mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk).
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of `bar` with the given parity to complete; gives up after a
// bounded number of polls (each poll may suspend the thread for a hardware-chosen time)
// and returns false.
constexpr int kMaxPolls = 1 << 24;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (int i = 0; i < kMaxPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Half-width of the band around an integer inside which a trajectory end sample's bin
// is recomputed in FP64: the double-FP32 anchor of an end sample is exact to far below
// 2^-30 bins, the FP32 coordinate of a last sample that is not an anchor to a few ulps
// of its block-relative value.
constexpr float kFirstGuard = 1.0f / (1 << 20);
__device__ __forceinline__ float last_guard(float v) {
    return (fabsf(v) + 1.0f) * (1.0f / (1 << 18));
}

// Precision check of the mixed deposit.  An FP32 block-relative coordinate carries an
// absolute error of about an ulp of the terms it sums; the interpolation weight
// (t_J - x_a)/(x_b - x_a) of a step of du bins then errs by about
// kCoordEps (|x_a| + |x_b| + |t_J|) / du, and the deposited value by that fraction of the
// field's change across the step; the fields themselves carry the rounding of their
// Doppler factor.  A separate launch of the same CTA routine (CHECK, which deposits
// nothing) evaluates a sample of the units -- every kCheckStride-th electron chunk -- and
// adds up the squares of these estimates and of the values; a unit whose root-mean-square
// ratio exceeds kPrecisionTol sets LW_ST_PRECISION.  The deposit itself carries none of
// this arithmetic.
constexpr float kCoordEps = 1.0f / (1 << 23);
constexpr int kCheckStride = 64;
constexpr float kPrecisionTol = 1.0f / (1 << 11);

// Sum of the sizes of the terms of coord(): its rounding is about an ulp of this.
__device__ __forceinline__ float coord_mag(float4 w, float s, float4 sc) {
    return fabsf(s * sc.x) + fabsf(w.x * sc.y) + fabsf(w.y * sc.z) + fabsf(w.z * sc.w);
}

// Relative error of an FP32 field through its Doppler factor: D sums terms of size
// (1 - n_z) + n_z (1 - beta_z) + |n_x beta_x| + |n_y beta_y|, each rounded to about an ulp,
// and enters the field as D^-3.
__device__ __forceinline__ float fd_rel(const PixelConst& pc, float4 f4, float2 f2) {
    const float2 f01 = make_float2(f4.x, f4.y);
    const float eps = f2.x;
    const float D = fmaf(-pc.ny, f01.y, fmaf(-pc.nx, f01.x, fmaf(pc.nz, eps, pc.omnz)));
    const float mag = fabsf(pc.nx * f01.x) + fabsf(pc.ny * f01.y) + pc.omnz + pc.nz * eps;
    return D > 0.0f ? 3.0f * kCoordEps * mag / D : 0.0f;
}

// floor(I + f) - I for a double-FP32 fraction f that lies within rounding of [0, 1)
__device__ __forceinline__ int frac_floor(float f) { return f >= 1.0f ? 1 : (f < 0.0f ? -1 : 0); }

// The work of one CTA: pixel tile `tile` (kMixThreads * PIX pixels) and electron
// chunk `chunk` (p.e_chunk electrons) of one variant.  Returns the status bits.
//
// The advanced time of a subluminal particle increases strictly along its
// trajectory (dt_a/dt = 1 - n.beta > 0).  Block b owns the steps (t_{i-1}, t_i] of
// Algorithm 2 that end at samples i0+1 .. i0+B, i.e. from its own anchor (sample i0)
// to the next block's anchor, so per pixel the grid points it reaches form one run
// (j_done, floor(u(i0+B))] whose end is the next anchor's coordinate, evaluated once per
// pixel and block in double-FP32 arithmetic (it is the next block's start as well).
// Each grid point of the run lies in exactly one of the block's steps: the first
// sample whose coordinate reaches it.  The grid points of the warp's 32 * PIX pixels
// are spread over its 32 lanes (prefix sum of the runs, one grid point per lane and
// round); a lane predicts the step from the linear interpolation between the block's
// two anchors, confirms it with the two samples around it (or narrows the bracket
// with regula falsi and bisection when the prediction misses), evaluates the FP32
// fields at both ends of the step and adds the interpolated value.
// The bins of the trajectory's first and last samples, where a one-bin rounding flip
// would add or drop a whole sample (Algorithm 2's half-open interval), are recomputed
// with the FP64 path's operation order when the mixed value lies within a guard band
// of an integer.
template <int PIX, int ACC, int FL, bool CHECK>
__device__ __forceinline__ int mixed_cta(const DepositArgs& p, int64_t tile, int64_t chunk) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int kSlots = kMixThreads * PIX;
    const int B = p.block;
    const size_t sbytes = stage_bytes(B);
    constexpr int kWarpsMix = kMixThreads / 32;
    // Slot numbering: lane-major, wslot + lane * PIX + q for pixel q of a lane -- the
    // order in which the warp's jobs are listed, so that the 32 jobs of a round, which
    // mostly belong to consecutive slots, read consecutive per-slot records.
    __shared__ float4 s_wh[kSlots];                   // slope hi parts (w_x, w_y, w_z), row
    __shared__ int4 s_job[kSlots];                    // block: I, f, x_end
    __shared__ int s_ja[kSlots];                      // block: first grid point
    __shared__ int s_kp[kSlots];                      // block: job offset (lane-major)
    __shared__ int2 s_tab[kWarpsMix][kJobTable];      // block: (slot, grid point) of job t
    __shared__ __align__(8) uint64_t s_full[kMixStages];   // stage filled (bytes arrived)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wslot = warp * 32 * PIX;
    const float s32 = p.s32;
    const float c0_over_R = (FL & LW_FIELD_VELOCITY) ? p.c0_over_R : 0.0f;
    const float inv_sc = p.inv_sc;   // direction from slope: n_x = -w_x c0 dt_u
    const int nb = (int)p.n_bins;
    const int64_t pix0 = tile * kSlots;
    unsigned act = 0;
    float wlo[PIX][3];   // slope lo parts of this thread's pixels (its anchors only)
    float whi[PIX][3];   // and their hi parts (the copies in s_wh serve other lanes' jobs)
    __syncthreads();   // shared arrays may still be read by the previous unit
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMixStages; ++s) mbar_init(&s_full[s], 1);
        mbar_init_fence();
    }
    for (int q = 0; q < PIX; ++q) {
        const int64_t m = pix0 + q * kMixThreads + threadIdx.x;
        double nx = 0.0, ny = 0.0, nz = 1.0;
        if (m < p.n_pix) {
            act |= 1u << q;
            nx = p.n_hat[3 * m];
            ny = p.n_hat[3 * m + 1];
            nz = p.n_hat[3 * m + 2];
        }
        // 1 - n_z: its FP64 cancellation error (<= 2^-53 absolute) moves the anchor by
        // 2^-53 |z_b| / (c0 dt_u) bins, below 1e-8 while |z_b| < 1e8 c0 dt_u -- far
        // below the FP32 coordinate's own rounding
        const double omnz = 1.0 - nz;
        const double sc = kInvC0 * p.inv_dtu;
        const DF wx = split_double(-nx * sc), wy = split_double(-ny * sc);
        const DF wz = split_double(omnz * sc);
        // .w: the pixel's row in the tile (bits of an unsigned), for the record address
        s_wh[wslot + lane * PIX + q] =
            make_float4(wx.hi, wy.hi, wz.hi, __uint_as_float(q * kMixThreads + threadIdx.x));
        wlo[q][0] = wx.lo;
        wlo[q][1] = wy.lo;
        wlo[q][2] = wz.lo;
        whi[q][0] = wx.hi;
        whi[q][1] = wy.hi;
        whi[q][2] = wz.hi;
    }
    __syncthreads();   // barriers initialised
    int bits = 0;
    if (tile == 0 && chunk == 0 && threadIdx.x == 0 && p.input_status) bits |= *p.input_status;
    float err2 = 0.0f, val2 = 0.0f;   // CHECK: squared error estimates and squared values

    // the tile's first record row; a pixel row is 4 * record_words bytes per grid point
    const uint64_t row_bytes =
        4ull * (ACC == kAccF32X4 ? 4 : ACC == kAccF32 ? 3 : 6) * (uint64_t)p.n_bins;
    unsigned char* const tile_rec =
        CHECK ? nullptr : static_cast<unsigned char*>(p.record) + (uint64_t)pix0 * row_bytes;
    auto electron = [&](int64_t kk) -> int64_t { return p.order ? (int64_t)p.order[kk] : kk; };
    // blocks with at least one step: ceil((ns1 - 1) / B)
    const int nbs = (int)((p.ns1 - 2) / B + 1);
    // float2 field records of a block start 0 or 8 bytes into their area: the bulk copy
    // starts at the 16-byte boundary at or before the block's first record
    auto field_shift = [&](int64_t k, int b) -> int {
        return (int)((k * p.ns1 + (int64_t)b * B) & 1) * 8;
    };
    // one thread stages block b of electron k into buffer `buf`
    auto issue = [&](int64_t k, int b, int buf) {
        unsigned char* base = smem_raw + buf * sbytes;
        const int64_t i0 = (int64_t)b * B;
        const int ns = (int)min((int64_t)B, p.ns1 - 1 - i0);   // steps of the block
        const unsigned scan_bytes = 16u * (unsigned)min((int64_t)B, p.ns1 - i0);
        const int sh = field_shift(k, b);
        const unsigned f4_bytes = 16u * (unsigned)(ns + 1);
        const unsigned f2_bytes = (8u * (unsigned)(ns + 1) + (unsigned)sh + 15u) & ~15u;
        const int a0 = b == 0 ? 0 : ((b & (kAnchorBatch - 1)) == kAnchorBatch - 1 ? b + 1 : -1);
        const unsigned anc_bytes =
            a0 >= 0 ? (unsigned)(sizeof(Anchor) * min(kAnchorBatch, p.n_blocks - a0)) : 0u;
        fence_proxy_async_smem();   // the buffer's previous contents were read by the CTA
        mbar_expect_tx(&s_full[buf], scan_bytes + f4_bytes + f2_bytes + anc_bytes);
        bulk_g2s(base, p.scan + k * p.ns1 + i0, scan_bytes, &s_full[buf]);
        bulk_g2s(base + stage_f4_off(B), p.field4 + k * p.ns1 + i0, f4_bytes, &s_full[buf]);
        bulk_g2s(base + stage_f2_off(B),
                 reinterpret_cast<const unsigned char*>(p.field2 + k * p.ns1 + i0) - sh,
                 f2_bytes, &s_full[buf]);
        if (anc_bytes)
            bulk_g2s(base + stage_anchor_off(B), p.anchor + k * p.n_blocks + a0, anc_bytes,
                     &s_full[buf]);
    };

    const int64_t k0 = chunk * p.e_chunk;
    const int64_t k1 = min(k0 + p.e_chunk, p.n_e);
    // ring: the unit's (electron, block) stages in order, kMixStages - 1 in flight ahead;
    // every thread keeps the bookkeeping, thread 0 issues the copies
    int64_t iss_kk = k0;   // next stage to issue
    int iss_b = 0;
    unsigned pending = 0;   // bit s: buffer s has a copy in flight
    auto issue_next = [&](int buf) {
        if (iss_kk < k1) {
            if (threadIdx.x == 0) issue(electron(iss_kk), iss_b, buf);
            pending |= 1u << buf;
            if (++iss_b == nbs) {
                iss_b = 0;
                ++iss_kk;
            }
        }
    };
    for (int st = 0; st + 1 < kMixStages; ++st) issue_next(st);
    int cur = 0;               // buffer of the block being processed
    unsigned phase = 0;        // bit s: parity of buffer s's next completion
    bool timed_out = false;
    // FP64 bin of an end sample (0 first, 1 last) of electron k for this lane's pixel q,
    // in the FP64 path's operation order
    auto end_bin = [&](int64_t k, int q, int which) -> int {
        const int64_t m = (act >> q & 1u) ? pix0 + q * kMixThreads + threadIdx.x : 0;
        return exact_bin_rare(p.ends + 8 * k + 4 * which, p.n_hat + 3 * m, p.t_min, p.inv_dtu);
    };
    // anchor U = T + W . R_b of pixel q in double-FP32 arithmetic -> I + f
    auto anchor_of = [&](const float (&an)[8], const float4& wh, int q, int& Iout, float& fout) {
        const float whc[3] = {wh.x, wh.y, wh.z};
        float s = an[0], e = an[1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float Rh = an[2 + 2 * c], Rl = an[3 + 2 * c];
            const float pr = __fmul_rn(whc[c], Rh);
            float pe = fmaf(whc[c], Rh, -pr);
            pe = fmaf(whc[c], Rl, fmaf(wlo[q][c], Rh, pe));
            const float s2 = __fadd_rn(s, pr);
            const float bb = __fsub_rn(s2, s);
            const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(pr, bb));
            s = s2;
            e = __fadd_rn(e, __fadd_rn(err, pe));
        }
        s = fminf(fmaxf(s, -1.0e9f), 1.0e9f);
        const float Is = floorf(s);
        Iout = (int)Is;
        fout = __fadd_rn(__fsub_rn(s, Is), e);
    };
    // FP32 pairs of an anchor (T = (tau_b - t_min)/dt_u, x_b, y_b, z_b); the position's
    // pairs are stored, T depends on the grid
    auto split_anchor = [&](const Anchor& a, float (&an)[8]) {
        const DF T = split_double((a.tau - p.t_min) * p.inv_dtu);
        an[0] = T.hi;
        an[1] = T.lo;
        an[2] = a.x_hi;
        an[3] = a.x_lo;
        an[4] = a.y_hi;
        an[5] = a.y_lo;
        an[6] = a.z_hi;
        an[7] = a.z_lo;
    };

    for (int64_t kk = k0; kk < k1 && !timed_out; ++kk) {
        const int64_t k = electron(kk);
        // per pixel: (Is, fs) = the block's start anchor, jdone = last grid point reached
        // so far (absolute; from the first sample's bin in block 0)
        int Is[PIX], jdone[PIX];
        float fs[PIX];
        float anc32[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (int b = 0; b < nbs; ++b) {
            const int64_t i0 = (int64_t)b * B;
            const int ns = (int)min((int64_t)B, p.ns1 - 1 - i0);   // steps: (i0+r-1, i0+r], r=1..ns
            const bool ok = mbar_wait(&s_full[cur], (phase >> cur) & 1u);
            // every warp is done with the previous block's buffer; a wait that ran out
            // anywhere stops the whole CTA
            if (__syncthreads_or(!ok)) {
                timed_out = true;
                break;
            }
            phase ^= 1u << cur;
            pending &= ~(1u << cur);
            issue_next(cur == 0 ? kMixStages - 1 : cur - 1);
            const unsigned char* base = smem_raw + cur * sbytes;
            const float4* s_scan = reinterpret_cast<const float4*>(base);
            const float4* s_f4 = reinterpret_cast<const float4*>(base + stage_f4_off(B));
            const float2* s_f2 =
                reinterpret_cast<const float2*>(base + stage_f2_off(B) + field_shift(k, b));
            const Anchor* s_anc = reinterpret_cast<const Anchor*>(base + stage_anchor_off(B));
            cur = cur + 1 == kMixStages ? 0 : cur + 1;
            // anchors: lane l holds the FP32 pairs of anchor 32c + l (c = batch); block b's
            // end anchor is b + 1
            const int ab = b & (kAnchorBatch - 1);
            if (b == 0) {
                if (lane < p.n_blocks) split_anchor(s_anc[lane], anc32);
                float an0[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) an0[c] = __shfl_sync(0xffffffffu, anc32[c], 0);
#pragma unroll
                for (int q = 0; q < PIX; ++q) {   // block 0's anchor is sample 0
                    anchor_of(an0, make_float4(whi[q][0], whi[q][1], whi[q][2], 0.0f), q,
                              Is[q], fs[q]);
                    const int fl = frac_floor(fs[q]);
                    const float fr = fs[q] - (float)fl;
                    jdone[q] = Is[q] + fl;
                    if (fr < kFirstGuard || fr > 1.0f - kFirstGuard) jdone[q] = end_bin(k, q, 0);
                }
            }
            const bool end_anchor = i0 + B <= p.ns1 - 1;   // the block ends at anchor b + 1
            const bool traj_end = i0 + ns == p.ns1 - 1;    // ... at the trajectory's last sample
            float ane[8];
            if (end_anchor) {
                if (ab == kAnchorBatch - 1) {   // the next batch was staged with this block
                    if (lane < p.n_blocks - (b + 1)) split_anchor(s_anc[lane], anc32);
                }
                const int src = ab == kAnchorBatch - 1 ? 0 : ab + 1;
#pragma unroll
                for (int c = 0; c < 8; ++c) ane[c] = __shfl_sync(0xffffffffu, anc32[c], src);
            }
            int K[PIX], big[PIX], JA[PIX];
            int tot = 0;
#pragma unroll
            for (int q = 0; q < PIX; ++q) {
                const int sl = wslot + lane * PIX + q;
                const float4 wh = make_float4(whi[q][0], whi[q][1], whi[q][2], 0.0f);
                int Ie = 0, jend;
                float fe = 0.0f, xe;
                if (end_anchor) {
                    anchor_of(ane, wh, q, Ie, fe);
                    const int fl = frac_floor(fe);
                    jend = Ie + fl;
                    if (traj_end) {
                        const float fr = fe - (float)fl;
                        if (fr < kFirstGuard || fr > 1.0f - kFirstGuard) jend = end_bin(k, q, 1);
                    }
                    // end coordinate relative to the start anchor, without its fraction
                    xe = __fadd_rn((float)(Ie - Is[q]), __fsub_rn(fe, fs[q]));
                } else {   // the trajectory's last sample, inside this block
                    xe = coord(wh, s32, s_scan[ns]);
                    const float v = __fadd_rn(xe, fs[q]);
                    const float fv = floorf(v), d = v - fv, gd = last_guard(v);
                    jend = Is[q] + (int)fv;
                    if (d < gd || d > 1.0f - gd || !(fabsf(v) < 1.0e9f)) jend = end_bin(k, q, 1);
                }
                int ja = jdone[q] + 1, jz = jend, kq = 0;
                if ((act >> q & 1u) && jz >= ja) {
                    if (ja < 0) {
                        ja = 0;
                        bits |= LW_ST_CLIP;
                    }
                    if (jz > nb - 1) {
                        jz = nb - 1;
                        bits |= LW_ST_CLIP;
                    }
                    kq = max(0, jz - ja + 1);
                }
                if (jend > jdone[q]) jdone[q] = jend;
                s_job[sl] = make_int4(Is[q], __float_as_int(fs[q]), __float_as_int(xe), 0);
                s_ja[sl] = ja;
                JA[q] = ja;
                big[q] = kq > kMaxWarpJobs ? kq : 0;
                K[q] = kq > kMaxWarpJobs ? 0 : kq;
                tot += K[q];
                Is[q] = Ie;
                fs[q] = fe;
            }
            // Grid point j (absolute) of slot sl with block data I, f, xe (coordinate of the
            // block's last sample relative to the anchor) and slope w: its step ends at the
            // first sample r in 1..ns whose coordinate reaches fl(J - f), J = j - I (the
            // last one if none does).  x(0) = 0 (the anchor) and x(ns) = xe bracket it.
            auto job = [&](int sl, int j) {
                const int4 jb = s_job[sl];
                const float4 w = s_wh[sl];
                const float f = __int_as_float(jb.y), xe = __int_as_float(jb.z);
                const float tJ = __fsub_rn((float)(j - jb.x), f);
                int a = 0, hb = ns;
                float xa = 0.0f, xb = xe;
                if (xe < tJ) {   // beyond the FP32 coordinate of the last sample: last step
                    a = ns - 1;
                    xa = a > 0 ? coord(w, s32, s_scan[a]) : 0.0f;
                } else if (ns > 1) {
                    // predicted step end g: the interpolated crossing between the anchors
                    const float fr = __fdividef(tJ, xe);
                    int g = (int)ceilf(fr * (float)ns);
                    g = min(max(g, 1), ns);
                    const float xl = g > 1 ? coord(w, s32, s_scan[g - 1]) : 0.0f;
                    const float xg = g < ns ? coord(w, s32, s_scan[g]) : xe;
                    if (xg < tJ) {
                        a = g;
                        xa = xg;
                    } else if (xl >= tJ) {
                        if (g > 1) {
                            hb = g - 1;
                            xb = xl;
                        } else {   // at or before the anchor (FP32 rounding): first step
                            hb = 1;
                            xb = xg;
                        }
                    } else {
                        a = g - 1;
                        xa = xl;
                        hb = g;
                        xb = xg;
                    }
                    int probes = 0;
                    while (hb - a > 1) {   // the prediction missed: narrow the bracket
                        int g2 = (a + hb) >> 1;
                        if (probes < kFalsiProbes) {
                            const float r = __fdividef(tJ - xa, xb - xa);
                            const float gf = ceilf(r * (float)(hb - a));
                            g2 = a + (int)fminf(fmaxf(gf, 1.0f), (float)(hb - a - 1));
                        }
                        ++probes;
                        const float xg2 = coord(w, s32, s_scan[g2]);
                        if (xg2 >= tJ) {
                            hb = g2;
                            xb = xg2;
                        } else {
                            a = g2;
                            xa = xg2;
                        }
                    }
                }
                // step (a, hb]: field records a and hb (record r = sample i0 + r)
                PixelConst pc;
                pc.nx = -w.x * inv_sc;
                pc.ny = -w.y * inv_sc;
                pc.omnz = w.z * inv_sc;
                pc.nz = 1.0f - pc.omnz;
                const float du = __fsub_rn(xb, xa);
                const float wb = du > 0.0f ? __fdividef(__fsub_rn(tJ, xa), du) : 0.0f;
                const float wa = 1.0f - wb;
                if (CHECK) {   // error estimate instead of the deposit
                    if (!(du > 0.0f)) return;
                    float Fb[3], Fa[3];
                    field_fp32<FL>(pc, s_f4[a], s_f2[a], c0_over_R, Fb);
                    field_fp32<FL>(pc, s_f4[hb], s_f2[hb], c0_over_R, Fa);
                    const float v0 = fmaf(Fb[0], wa, Fa[0] * wb);
                    const float v1 = fmaf(Fb[1], wa, Fa[1] * wb);
                    const float v2 = fmaf(Fb[2], wa, Fa[2] * wb);
                    // the weight's: the field's change times the weight's rounding, from the
                    // sizes of the terms the two coordinates sum (the anchor's is exact, the
                    // next anchor's a double-FP32 difference)
                    const float ma = a > 0 ? coord_mag(w, s32, s_scan[a]) : 0.0f;
                    const float mb = (hb < ns || !end_anchor) ? coord_mag(w, s32, s_scan[hb])
                                                              : fabsf(xb);
                    const float dw = kCoordEps * (ma + mb + fabsf(tJ)) / du;
                    float e = dw * (fabsf(Fa[0] - Fb[0]) + fabsf(Fa[1] - Fb[1]) +
                                    fabsf(Fa[2] - Fb[2]));
                    // the fields': D in FP32 loses the terms' size over D, three times in D^3
                    e = fmaf(fd_rel(pc, s_f4[a], s_f2[a]) * wa,
                             fabsf(Fb[0]) + fabsf(Fb[1]) + fabsf(Fb[2]), e);
                    e = fmaf(fd_rel(pc, s_f4[hb], s_f2[hb]) * wb,
                             fabsf(Fa[0]) + fabsf(Fa[1]) + fabsf(Fa[2]), e);
                    // squares of the values scaled by 2^-100 (fields of up to ~1e35 /s stay in
                    // range)
                    e *= 0x1p-50f;
                    err2 = fmaf(e, e, err2);
                    const float u0 = v0 * 0x1p-50f, u1 = v1 * 0x1p-50f, u2 = v2 * 0x1p-50f;
                    val2 = fmaf(u0, u0, fmaf(u1, u1, fmaf(u2, u2, val2)));
                } else {
                    // wa F(a) + wb F(hb), both ends in the expanded form
                    const float2 nxy = make_float2(pc.nx, pc.ny);
                    float2 tb, ta;
                    float tbz, taz, sb, sa;
                    end_terms<FL>(pc, nxy, s_f4[a], s_f2[a], c0_over_R, wa, tb, tbz, sb);
                    end_terms<FL>(pc, nxy, s_f4[hb], s_f2[hb], c0_over_R, wb, ta, taz, sa);
                    const float2 vxy =
                        __ffma2_rn(tb, make_float2(sb, sb), __fmul2_rn(ta, make_float2(sa, sa)));
                    const float vz = fmaf(tbz, sb, taz * sa);
                    deposit3_row<ACC>(tile_rec + (uint64_t)__float_as_uint(w.w) * row_bytes, j,
                                      p.n_bins, vxy.x, vxy.y, vz);
                }
            };
            // the warp's grid points: prefix sum of the runs over the warp's slots, and the
            // first kJobTable of them listed as (slot, grid point) by their owners
            int incl = tot;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            const int T = __shfl_sync(0xffffffffu, incl, 31);
            int run = incl - tot;
#pragma unroll
            for (int q = 0; q < PIX; ++q) {
                const int sl = wslot + lane * PIX + q;
                s_kp[sl] = run;
                for (int t = 0; t < K[q] && run + t < kJobTable; ++t)
                    s_tab[warp][run + t] = make_int2(sl, JA[q] + t);
                run += K[q];
            }
            __syncwarp();
            // slot of the warp's job t beyond the table: the last slot whose offset is <= t
            auto slot_of = [&](int t) -> int {
                int pos = 0;
#pragma unroll
                for (int step = 16 * PIX; step > 0; step >>= 1)
                    if (s_kp[wslot + pos + step] <= t) pos += step;
                return wslot + pos;
            };
            for (int t = lane; t < T; t += 32) {
                if (t < kJobTable) {
                    const int2 e = s_tab[warp][t];
                    job(e.x, e.y);
                } else {
                    const int sl = slot_of(t);
                    job(sl, s_ja[sl] + (t - s_kp[sl]));
                }
            }
#pragma unroll
            for (int q = 0; q < PIX; ++q) {   // runs too long for the warp's job count
                const int sl = wslot + lane * PIX + q;
                for (int t = 0; t < big[q]; ++t) job(sl, JA[q] + t);
            }
            __syncwarp();   // s_job / s_kp are rewritten for the next block
        }
    }
    if (CHECK) {   // the unit's estimated error against the values it would deposit
        __shared__ float s_err[2];
        if (threadIdx.x == 0) s_err[0] = s_err[1] = 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            err2 += __shfl_xor_sync(0xffffffffu, err2, o);
            val2 += __shfl_xor_sync(0xffffffffu, val2, o);
        }
        __syncthreads();
        if (lane == 0) {
            atomicAdd(&s_err[0], err2);
            atomicAdd(&s_err[1], val2);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_err[0] > kPrecisionTol * kPrecisionTol * s_err[1])
            bits |= LW_ST_PRECISION;
    }
    if (timed_out) {
        bits |= LW_ST_TIMEOUT;
        // copies may still be in flight into the ring: wait for each one, again with a
        // bounded wait, before the CTA leaves
        for (int s = 0; s < kMixStages; ++s)
            if (pending >> s & 1u) mbar_wait(&s_full[s], (phase >> s) & 1u);
    }
    __syncthreads();   // every stage consumed; the barriers can be retired
    if (threadIdx.x == 0)
        for (int s = 0; s < kMixStages; ++s) mbar_inval(&s_full[s]);
    return bits;
}

// FP64 deposit for trajectories whose advanced time increases (no LW_ST_STEP
// from the upload): per pixel and block of samples, the grid points reached
// are the run (floor(u_b), floor(u_end)]; each is located, by a bracketed
// search over the staged block, at the first sample whose coordinate reaches
// it -- the step of Algorithm 2 that holds it -- and deposited with the scan's
// FP64 expressions in the oracle's operation order, so every contribution is
// bit-identical to the literal scan (only the order of the atomic additions
// differs).  With LW_ST_STEP set the literal scan runs instead, and electrons that
// reach more than half a grid point per step (on average over the CTA's pixels) are
// walked step by step, like the scan, from the same staged blocks.
constexpr int kF64Block = 256;   // samples staged per block

__global__ void __launch_bounds__(kFp64Threads) deposit_fp64_jobs_kernel(DepositArgs p) {
    if (p.input_status && (*p.input_status & LW_ST_STEP)) {
        fp64_scan_cta(p);
        return;
    }
    constexpr int kWarpsF = kFp64Threads / 32;
    __shared__ double s_t[2][kF64Block + 1];        // sample i0-1 first
    __shared__ double s_r[2][3 * (kF64Block + 1)];
    __shared__ double s_n[kFp64Threads][3];         // pixel directions
    __shared__ double s_ua[kFp64Threads];           // block: coordinate before the block
    __shared__ double s_ue[kFp64Threads];           // block: coordinate of its last sample
    __shared__ int s_ja[kFp64Threads];              // block: first grid point of the run
    __shared__ int s_kp[kFp64Threads];              // block: job offset in the warp
    __shared__ int2 s_tab[kWarpsF][kJobTable];      // block: (slot, grid point) of job t
    __shared__ unsigned long long s_pts[2];         // grid points of the electron (alternating)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wslot = warp * 32;
    const int64_t pix0 = (int64_t)blockIdx.x * kFp64Threads;
    const int n_act = (int)min((int64_t)kFp64Threads, p.n_pix - pix0);
    const int64_t m = pix0 + threadIdx.x;
    const bool active = m < p.n_pix;
    const int nb = (int)p.n_bins;
    double nx = 0.0, ny = 0.0, nz = 1.0;
    if (active) {
        nx = p.n_hat[3 * m];
        ny = p.n_hat[3 * m + 1];
        nz = p.n_hat[3 * m + 2];
    }
    s_n[threadIdx.x][0] = nx;
    s_n[threadIdx.x][1] = ny;
    s_n[threadIdx.x][2] = nz;
    int bits = 0;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && p.input_status)
        bits |= *p.input_status;
    const int nblk = (int)((p.ns1 + kF64Block - 1) / kF64Block);
    auto electron = [&](int64_t kk) -> int64_t { return p.order ? (int64_t)p.order[kk] : kk; };
    auto issue = [&](int64_t k, int b, int buf) {
        const int64_t i0 = (int64_t)b * kF64Block;
        const int n = (int)min((int64_t)kF64Block, p.ns1 - i0);
        const double* tk = p.t + (p.t_per_e ? k * p.ns1 : 0) + i0;
        const double* rk = p.r + 3 * (k * p.ns1 + i0);
        for (int q = (b == 0 ? 1 : 0) + threadIdx.x; q <= n; q += kFp64Threads)
            cp_async8(&s_t[buf][q], tk + (q - 1));
        for (int q = (b == 0 ? 3 : 0) + threadIdx.x; q < 3 * (n + 1); q += kFp64Threads)
            cp_async8(&s_r[buf][q], rk + (q - 3));
        cp_async_commit();
    };
    // coordinate u = (t_a - t_min) / dt_u of staged sample q, the scan's expression
    auto coord64 = [&](const double* n3, int buf, int q) -> double {
        const double ta = advanced_time_fp64(n3[0], n3[1], n3[2], s_r[buf][3 * q],
                                             s_r[buf][3 * q + 1], s_r[buf][3 * q + 2],
                                             s_t[buf][q]);
        return __dmul_rn(__dsub_rn(ta, p.t_min), p.inv_dtu);
    };
    const int64_t k0 = (int64_t)blockIdx.y * p.e_chunk;
    const int64_t k1 = min(k0 + p.e_chunk, p.n_e);
    int buf = 0;
    if (k0 < k1) issue(electron(k0), 0, 0);
    for (int64_t kk = k0; kk < k1; ++kk) {
        const int64_t k = electron(kk);
        const double* bk = p.beta + 3 * k * p.ns1;
        const double* ak = p.bdot + 3 * k * p.ns1;
        const double* e0 = p.ends + 8 * k;
        const double u0 = __dmul_rn(__dsub_rn(advanced_time_fp64(nx, ny, nz, e0[1], e0[2], e0[3],
                                                                 e0[0]),
                                              p.t_min),
                                    p.inv_dtu);
        bool ok = fabs(u0) < 4.0e18;
        if (active && !ok) bits |= LW_ST_NONFINITE;
        int64_t jdone = ok ? (int64_t)floor(u0) : 0;
        double uprev = u0;
        // More than half a grid point per step on average over the CTA's pixels: walk
        // every step (fields once per step, shared by the grid points it holds) instead
        // of locating each grid point -- the choice is the CTA's, per electron.
        const double ul = __dmul_rn(__dsub_rn(advanced_time_fp64(nx, ny, nz, e0[5], e0[6], e0[7],
                                                                 e0[4]),
                                              p.t_min),
                                    p.inv_dtu);
        unsigned long long pts = 0;
        if (active && ok && fabs(ul) < 4.0e18) {
            const double lo = fmax(floor(u0), -1.0), hi = fmin(floor(ul), (double)nb - 1.0);
            if (hi > lo) pts = (unsigned long long)(hi - lo);
        }
        for (int o = 16; o > 0; o >>= 1) pts += __shfl_down_sync(0xffffffffu, pts, o);
        const int ci = (int)(kk & 1);
        if (threadIdx.x == 0) s_pts[ci] = 0;
        __syncthreads();
        if (lane == 0) atomicAdd(&s_pts[ci], pts);
        __syncthreads();
        const bool per_step = 2 * s_pts[ci] > (unsigned long long)n_act * (unsigned long long)(p.ns1 - 1);
        ScanState S;
        S.reset();
        double* rec_m = static_cast<double*>(p.record) + (active ? m * 3 * p.n_bins : 0);
        for (int b = 0; b < nblk; ++b) {
            const int64_t i0 = (int64_t)b * kF64Block;
            const int n = (int)min((int64_t)kF64Block, p.ns1 - i0);
            cp_async_wait_all();
            __syncthreads();   // block b staged; every warp is done with block b-1
            if (b + 1 < nblk)
                issue(k, b + 1, buf ^ 1);
            else if (kk + 1 < k1)
                issue(electron(kk + 1), 0, buf ^ 1);
            const int cb = buf;
            buf ^= 1;
            if (per_step) {
                if (active)
                    for (int q = 1; q <= n; ++q)
                        scan_sample(p, nx, ny, nz, rec_m, bk, ak, i0 + q - 1, s_t[cb][q],
                                    s_r[cb][3 * q], s_r[cb][3 * q + 1], s_r[cb][3 * q + 2], S,
                                    bits);
                continue;
            }
            const int lo0 = (b == 0) ? 1 : 0;   // sample 0 ends no step
            const double ue = coord64(s_n[threadIdx.x], cb, n);
            int K = 0, ja = 0, big = 0;
            if (active && ok && n > lo0) {
                if (!(fabs(ue) < 4.0e18)) {
                    bits |= LW_ST_NONFINITE;
                    ok = false;
                } else {
                    const int64_t jend = (int64_t)floor(ue);
                    int64_t a = jdone + 1, z = jend;
                    if (a <= z) {
                        if (a < 0) {
                            a = 0;
                            bits |= LW_ST_CLIP;
                        }
                        if (z > nb - 1) {
                            z = nb - 1;
                            bits |= LW_ST_CLIP;
                        }
                        if (a <= z) {
                            K = (int)(z - a + 1);
                            ja = (int)a;
                            if (K > kMaxWarpJobs) {
                                big = K;
                                K = 0;
                            }
                        }
                    }
                    if (jend > jdone) jdone = jend;
                }
            }
            s_ja[threadIdx.x] = ja;
            s_ua[threadIdx.x] = b == 0 ? u0 : uprev;
            s_ue[threadIdx.x] = ue;
            uprev = ue;
            // the warp's grid points: prefix sum, the first kJobTable listed by owners
            int incl = K;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            const int T = __shfl_sync(0xffffffffu, incl, 31);
            const int run = incl - K;
            s_kp[threadIdx.x] = run;
            for (int t = 0; t < K && run + t < kJobTable; ++t)
                s_tab[warp][run + t] = make_int2(threadIdx.x, ja + t);
            __syncwarp();
            // grid point j of slot sl: locate its step in the staged block and deposit
            auto job = [&](int sl, int j) {
                const double* n3 = s_n[sl];
                const double J = (double)j;
                // first staged sample in [lo0, n-1] (local index) with u >= j
                int a = lo0 - 1, hb = n - 1;
                double xa = s_ua[sl], xb = s_ue[sl];
                int probes = 0;
                while (hb - a > 1) {
                    int g = (a + hb) >> 1;
                    if (probes < kFalsiProbes) {
                        const float fr = __fdividef((float)(J - xa), (float)(xb - xa));
                        const float gf = ceilf(fr * (float)(hb - a));
                        g = a + (int)fminf(fmaxf(gf, 1.0f), (float)(hb - a - 1));
                    }
                    ++probes;
                    const double xg = coord64(n3, cb, g + 1);
                    if (xg >= J) {
                        hb = g;
                        xb = xg;
                    } else {
                        a = g;
                        xa = xg;
                    }
                }
                const int i = hb;   // local index of the step's end sample
                const int q = i + 1;
                const double ta = advanced_time_fp64(n3[0], n3[1], n3[2], s_r[cb][3 * q],
                                                     s_r[cb][3 * q + 1], s_r[cb][3 * q + 2],
                                                     s_t[cb][q]);
                const double tb = advanced_time_fp64(n3[0], n3[1], n3[2], s_r[cb][3 * q - 3],
                                                     s_r[cb][3 * q - 2], s_r[cb][3 * q - 1],
                                                     s_t[cb][q - 1]);
                const int64_t gi = i0 + i;   // global sample index of the step's end
                double Fb[3], Fa[3];
                field_fp64(n3[0], n3[1], n3[2], p.R, p.flags, bk + 3 * (gi - 1), ak + 3 * (gi - 1),
                           Fb);
                field_fp64(n3[0], n3[1], n3[2], p.R, p.flags, bk + 3 * gi, ak + 3 * gi, Fa);
                const double den = __dsub_rn(ta, tb);
                const double tu = __dadd_rn(p.t_min, __dmul_rn(J, p.dt_u));
                const double wa = __ddiv_rn(__dsub_rn(ta, tu), den);
                const double wb = __ddiv_rn(__dsub_rn(tu, tb), den);
                double* rec = static_cast<double*>(p.record) + (pix0 + sl) * 3 * p.n_bins + j;
                for (int c = 0; c < 3; ++c)
                    atomicAdd(rec + c * p.n_bins,
                              __dadd_rn(__dmul_rn(Fb[c], wa), __dmul_rn(Fa[c], wb)));
            };
            for (int t = lane; t < T; t += 32) {
                if (t < kJobTable) {
                    const int2 e = s_tab[warp][t];
                    job(e.x, e.y);
                } else {
                    int pos = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (s_kp[wslot + pos + step] <= t) pos += step;
                    const int sl = wslot + pos;
                    job(sl, s_ja[sl] + (t - s_kp[sl]));
                }
            }
            for (int t = 0; t < big; ++t) job(threadIdx.x, ja + t);   // runs beyond the warp count
            __syncwarp();
        }
    }
    cp_async_wait_all();
    block_status_or(p.status, bits);
}

template <int PIX, int ACC, int FL>
__global__ void __launch_bounds__(kMixThreads, kMixMinBlocks) deposit_mixed_kernel(DepositArgs p) {
    // the precision check launched after this grid (programmatic dependent launch) may
    // start once every CTA of this grid has started: it fills the SMs of the last wave
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int bits = mixed_cta<PIX, ACC, FL, false>(p, blockIdx.x, blockIdx.y);
    block_status_or(p.status, bits);
}

// Precision check of a mixed deposit: the units of every `stride`-th electron chunk
// (grid y = sampled chunks), evaluated without depositing.  Launched as a programmatic
// dependent of the deposit, it runs beside the deposit's last CTAs and, before it ends,
// waits for the deposit grid to complete (griddepcontrol.wait: its completion and memory
// flush), so that work after it in the stream sees the finished record; without that
// launch attribute the wait returns at once.
template <int PIX, int FL>
__global__ void __launch_bounds__(kMixThreads, kMixMinBlocks)
    deposit_check_kernel(DepositArgs p, int stride) {
    const int bits =
        mixed_cta<PIX, kAccF32X4, FL, true>(p, blockIdx.x, (int64_t)blockIdx.y * stride);
    block_status_or(p.status, bits & LW_ST_PRECISION);
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Persistent form: CTAs pull (variant, pixel tile, electron chunk) units from a
// list in decreasing order of work until the list is exhausted.
struct BatchUnit {
    int variant;
    int tile;
    int chunk;
    int pad;
};

// The variants' arguments of the batch being deposited, copied from the plan's
// workspace before each launch: read through the constant cache with a
// CTA-uniform index, they cost the shared-memory pipe nothing.
constexpr int kBatchMaxItems = 256;
__constant__ DepositArgs c_batch_vars[kBatchMaxItems];

template <int PIX, int ACC, int FL>
__global__ void __launch_bounds__(kMixThreads, kMixMinBlocks)
    deposit_batched_kernel(const BatchUnit* __restrict__ units, int n_units, int* counter) {
    __shared__ int s_unit;
    while (true) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= n_units) break;
        const BatchUnit un = units[u];
        const DepositArgs& p = c_batch_vars[un.variant];
        const int bits = mixed_cta<PIX, ACC, FL, false>(p, un.tile, un.chunk);
        block_status_or(p.status, bits);
    }
}

// Precision check of a batched deposit: every `stride`-th unit of the list.
template <int PIX, int FL>
__global__ void __launch_bounds__(kMixThreads, kMixMinBlocks)
    deposit_batched_check_kernel(const BatchUnit* __restrict__ units, int n_units, int stride) {
    const int u = blockIdx.x * stride;
    if (u >= n_units) return;
    const BatchUnit un = units[u];
    const DepositArgs& p = c_batch_vars[un.variant];
    const int bits = mixed_cta<PIX, kAccF32X4, FL, true>(p, un.tile, un.chunk);
    block_status_or(p.status, bits & LW_ST_PRECISION);
}

// Zeroes every variant's record (n_pix * n_bins * words 4-byte words): grid y =
// variant, x = CTAs striding over it, with 16-byte stores where the record is
// 16-byte aligned (an odd last value is stored alone).
__global__ void zero_records_kernel(const DepositArgs* __restrict__ vars, int words) {
    const DepositArgs& a = vars[blockIdx.y];
    const int64_t n = a.n_pix * a.n_bins * words;   // 4-byte words
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float* rec = static_cast<float*>(a.record);
    if ((reinterpret_cast<uintptr_t>(a.record) & 15) == 0) {
        float4* rec4 = static_cast<float4*>(a.record);
        for (int64_t i = i0; i < n / 4; i += stride) rec4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t i = (n / 4) * 4 + i0; i < n; i += stride) rec[i] = 0.0f;
    } else {
        for (int64_t i = i0; i < n; i += stride) rec[i] = 0.0f;
    }
}

// Kernel instances by accumulation form and field terms (LW_FIELD_* mask 1, 2 or 3).
using MixedKernel = void (*)(DepositArgs);
using BatchedKernel = void (*)(const BatchUnit*, int, int*);
template <int ACC>
MixedKernel mixed_kernel_fl(uint32_t fl) {
    return fl == 1 ? deposit_mixed_kernel<kMixPix, ACC, 1>
           : fl == 2 ? deposit_mixed_kernel<kMixPix, ACC, 2> : deposit_mixed_kernel<kMixPix, ACC, 3>;
}
MixedKernel mixed_kernel(int acc, uint32_t fl) {
    return acc == kAccKahan ? mixed_kernel_fl<kAccKahan>(fl)
           : acc == kAccF32 ? mixed_kernel_fl<kAccF32>(fl)
           : acc == kAccF32X4 ? mixed_kernel_fl<kAccF32X4>(fl) : mixed_kernel_fl<kAccF64>(fl);
}
template <int ACC>
BatchedKernel batched_kernel_fl(uint32_t fl) {
    return fl == 1 ? deposit_batched_kernel<kMixPix, ACC, 1>
           : fl == 2 ? deposit_batched_kernel<kMixPix, ACC, 2>
                     : deposit_batched_kernel<kMixPix, ACC, 3>;
}
using CheckKernel = void (*)(DepositArgs, int);
CheckKernel check_kernel(uint32_t fl) {
    return fl == 1 ? deposit_check_kernel<kMixPix, 1>
           : fl == 2 ? deposit_check_kernel<kMixPix, 2> : deposit_check_kernel<kMixPix, 3>;
}
using BatchedCheckKernel = void (*)(const BatchUnit*, int, int);
BatchedCheckKernel batched_check_kernel(uint32_t fl) {
    return fl == 1 ? deposit_batched_check_kernel<kMixPix, 1>
           : fl == 2 ? deposit_batched_check_kernel<kMixPix, 2>
                     : deposit_batched_check_kernel<kMixPix, 3>;
}
BatchedKernel batched_kernel(int acc, uint32_t fl) {
    return acc == kAccKahan ? batched_kernel_fl<kAccKahan>(fl)
           : acc == kAccF32 ? batched_kernel_fl<kAccF32>(fl)
           : acc == kAccF32X4 ? batched_kernel_fl<kAccF32X4>(fl) : batched_kernel_fl<kAccF64>(fl);
}

// The mixed path's FP32 constants from the FP64 grid and detector fields (each the FP32
// rounding of its correctly rounded FP64 value).
void set_fp32_constants(DepositArgs& a) {
    a.s32 = (float)a.inv_dtu;
    a.inv_sc = (float)(kC0 * a.dt_u);
    a.c0_over_R = (float)(kC0 / a.R);
}

}  // namespace
}  // namespace lw

using namespace lw;

extern "C" int lw_deposit_time_domain(const lw_traj* traj, const lw_detector* det,
                                      const lw_grid* grid, int32_t precision,
                                      uint32_t field_flags, void* record, int32_t accumulate,
                                      int32_t* status, void* stream) {
    if (!traj || !det || !grid || !record || !det->n_hat) return LW_EINVAL;
    if (det->n_pix < 1 || grid->n_bins < 1 || grid->n_bins > (int64_t(1) << 30)) return LW_EINVAL;
    if (!(grid->dt_u > 0.0) || !isfinite(grid->dt_u) || !isfinite(grid->t_min)) return LW_EINVAL;
    if (field_flags == 0 || (field_flags & ~(LW_FIELD_ACCEL | LW_FIELD_VELOCITY))) return LW_EINVAL;
    if ((field_flags & LW_FIELD_VELOCITY) && !(det->R > 0.0)) return LW_EINVAL;
    if (precision != LW_FP64 && precision != LW_MIXED && precision != LW_MIXED_KAHAN &&
        precision != LW_MIXED_F32 && precision != LW_MIXED_F32X4)
        return LW_EINVAL;
    if (precision == LW_FP64 && !(traj->sections & LW_SECTION_FP64)) return LW_EINVAL;
    if (precision != LW_FP64 && !(traj->sections & LW_SECTION_MIXED)) return LW_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (!accumulate &&
        cudaMemsetAsync(record, 0, 4 * (size_t)record_words(precision) *
                                       (size_t)(det->n_pix * grid->n_bins), st) != cudaSuccess)
        return LW_ECUDA;

    DepositArgs a{};
    a.n_e = traj->n_e;
    a.ns1 = traj->n_s + 1;
    a.t_per_e = traj->t_per_electron;
    a.t = traj->t;
    a.r = traj->r;
    a.beta = traj->beta;
    a.bdot = traj->beta_dot;
    a.scan = static_cast<const float4*>(traj->scan);
    a.field4 = static_cast<const float4*>(traj->field);
    a.field2 = traj->field
                   ? reinterpret_cast<const float2*>(a.field4 + traj->n_e * (traj->n_s + 1))
                   : nullptr;
    a.anchor = reinterpret_cast<const Anchor*>(traj->anchor);
    a.block = traj->block;
    a.n_blocks = traj->n_blocks;
    a.input_status = traj->input_status;
    a.ends = traj->ends;
    a.order = traj->order;
    a.n_hat = det->n_hat;
    a.n_pix = det->n_pix;
    a.R = det->R > 0.0 ? det->R : 1.0;
    a.t_min = grid->t_min;
    a.dt_u = grid->dt_u;
    a.inv_dtu = 1.0 / grid->dt_u;
    set_fp32_constants(a);
    a.n_bins = grid->n_bins;
    a.flags = field_flags;
    a.record = record;
    a.status = status;

    if (precision == LW_FP64) {
        const int64_t tiles = (det->n_pix + kFp64Threads - 1) / kFp64Threads;
        a.e_chunk = (int)std::max<int64_t>(1, (traj->n_e + 65534) / 65535);
        dim3 g((unsigned)tiles, (unsigned)((traj->n_e + a.e_chunk - 1) / a.e_chunk));
        deposit_fp64_jobs_kernel<<<g, kFp64Threads, 0, st>>>(a);
        return launch_status();
    }
    constexpr int PIX = kMixPix;
    const int64_t tiles = (det->n_pix + kMixThreads * PIX - 1) / (kMixThreads * PIX);
    // a few consecutive electrons (in arrival order) per CTA row -- enough rows for
    // about eight waves of resident CTAs -- dispatched tile-fastest: the electrons in
    // flight stay consecutive in arrival order, so the record bins they update are few
    // enough to be served from L2, and each CTA's pixel set-up serves several electrons
    const int64_t rows_wanted = (int64_t)kSms * kMixMinBlocks * 8 / std::max<int64_t>(1, tiles);
    int64_t ec = traj->n_e / std::max<int64_t>(1, rows_wanted);
    ec = std::min<int64_t>(std::max<int64_t>(ec, 1),
                           precision == LW_MIXED_F32X4 ? kMixMaxChunkX4 : kMixMaxChunk);
    a.e_chunk = (int)std::max<int64_t>(ec, (traj->n_e + 65534) / 65535);
    dim3 g((unsigned)tiles, (unsigned)((traj->n_e + a.e_chunk - 1) / a.e_chunk));
    const size_t smem = kMixStages * stage_bytes(traj->block);   // staging ring
    // static tables + double-buffered staging exceed the 48 KB default: opt in
    const MixedKernel kern = mixed_kernel(acc_of(precision), field_flags);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return LW_ECUDA;
    kern<<<g, kMixThreads, smem, st>>>(a);
    if (launch_status() != LW_OK) return LW_ECUDA;
    if (status) {   // the precision check on a sample of the electron chunks (LW_ST_PRECISION)
        const int64_t chunks = g.y;
        const int stride = chunks > kCheckStride ? kCheckStride : 1;
        const CheckKernel ck = check_kernel(field_flags);
        if (cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return LW_ECUDA;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g.x, (unsigned)((chunks + stride - 1) / stride));
        cfg.blockDim = dim3(kMixThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, ck, a, stride) != cudaSuccess) return LW_ECUDA;
    }
    return launch_status();
}

// ---------------------------------------------------------------------------
// Batched form: several independent problems in one persistent launch.
namespace lw {
namespace {

struct BatchHeader {
    int n_items, n_units, precision, smem;
};

size_t batch_layout(int n_items, int64_t n_units, size_t* off_vars, size_t* off_units,
                    size_t* off_counter) {
    size_t off = 0;
    *off_counter = off;
    off = align256(off + sizeof(int));
    *off_vars = off;
    off = align256(off + sizeof(DepositArgs) * (size_t)n_items);
    *off_units = off;
    off = align256(off + sizeof(BatchUnit) * (size_t)n_units);
    return off;
}

}  // namespace
}  // namespace lw

extern "C" int lw_batch_plan(const lw_batch_item* items, int32_t n_items, int32_t precision,
                             uint32_t field_flags, void* ws, size_t* ws_bytes, lw_batch* plan,
                             void* stream) {
    constexpr int PIX = kMixPix;
    if (!items || n_items < 1 || !ws_bytes || !plan) return LW_EINVAL;
    if (n_items > kBatchMaxItems) return LW_EUNSUPPORTED;
    if (precision != LW_MIXED && precision != LW_MIXED_KAHAN && precision != LW_MIXED_F32 &&
        precision != LW_MIXED_F32X4)
        return LW_EUNSUPPORTED;
    if (field_flags == 0 || (field_flags & ~(LW_FIELD_ACCEL | LW_FIELD_VELOCITY))) return LW_EINVAL;
    std::vector<DepositArgs> vars((size_t)n_items);
    std::vector<BatchUnit> units;
    std::vector<int64_t> unit_work;
    int max_block = 16;
    int64_t total = 0;
    const int64_t px_per_cta = (int64_t)kMixThreads * PIX;
    for (int v = 0; v < n_items; ++v) {
        const lw_batch_item& it = items[v];
        if (!it.traj || !it.det || !it.record || !it.det->n_hat || it.det->n_pix < 1) return LW_EINVAL;
        if (!(it.traj->sections & LW_SECTION_MIXED)) return LW_EINVAL;
        if (it.grid.n_bins < 1 || it.grid.n_bins > (int64_t(1) << 30)) return LW_EINVAL;
        if (!(it.grid.dt_u > 0.0) || !isfinite(it.grid.dt_u) || !isfinite(it.grid.t_min))
            return LW_EINVAL;
        if ((field_flags & LW_FIELD_VELOCITY) && !(it.det->R > 0.0)) return LW_EINVAL;
        total += it.traj->n_e * it.traj->n_s * it.det->n_pix;
        if (it.traj->block > max_block) max_block = it.traj->block;
    }
    // unit size: aim at ~8 units per resident CTA over the whole batch
    const int64_t target = total / ((int64_t)kSms * 5 * 8) + 1;
    for (int v = 0; v < n_items; ++v) {
        const lw_batch_item& it = items[v];
        DepositArgs& a = vars[(size_t)v];
        a = DepositArgs{};
        a.n_e = it.traj->n_e;
        a.ns1 = it.traj->n_s + 1;
        a.t_per_e = it.traj->t_per_electron;
        a.scan = static_cast<const float4*>(it.traj->scan);
        a.field4 = static_cast<const float4*>(it.traj->field);
        a.field2 = it.traj->field ? reinterpret_cast<const float2*>(
                                        a.field4 + it.traj->n_e * (it.traj->n_s + 1))
                                  : nullptr;
        a.anchor = reinterpret_cast<const Anchor*>(it.traj->anchor);
        a.block = it.traj->block;
        a.n_blocks = it.traj->n_blocks;
        a.input_status = it.traj->input_status;
        a.ends = it.traj->ends;
        a.order = it.traj->order;
        a.n_hat = it.det->n_hat;
        a.n_pix = it.det->n_pix;
        a.R = it.det->R > 0.0 ? it.det->R : 1.0;
        a.t_min = it.grid.t_min;
        a.dt_u = it.grid.dt_u;
        a.inv_dtu = 1.0 / it.grid.dt_u;
        set_fp32_constants(a);
        a.n_bins = it.grid.n_bins;
        a.flags = field_flags;
        a.record = it.record;
        a.status = it.status;
        const int64_t tiles = (a.n_pix + px_per_cta - 1) / px_per_cta;
        int64_t chunk = it.e_chunk;
        if (chunk <= 0) {
            chunk = target / (px_per_cta * it.traj->n_s);
            if (chunk < 1) chunk = 1;
        }
        if (chunk > a.n_e) chunk = a.n_e;
        a.e_chunk = (int)chunk;
        const int64_t chunks = (a.n_e + chunk - 1) / chunk;
        for (int64_t c = 0; c < chunks; ++c)
            for (int64_t t = 0; t < tiles; ++t) {
                units.push_back(BatchUnit{v, (int)t, (int)c, 0});
                const int64_t ne = std::min(chunk, a.n_e - c * chunk);
                const int64_t np = std::min(px_per_cta, a.n_pix - t * px_per_cta);
                unit_work.push_back(ne * it.traj->n_s * np);
            }
    }
    // largest units first
    // variants largest first (their total work), each variant's units in their own
    // order (electron chunks in arrival order, tiles fastest), so that the units in
    // flight keep the record band of one variant narrow
    std::vector<int64_t> var_work((size_t)n_items, 0);
    for (size_t i = 0; i < units.size(); ++i) var_work[(size_t)units[i].variant] += unit_work[i];
    std::vector<size_t> order(units.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        const int vx = units[x].variant, vy = units[y].variant;
        if (vx == vy) return false;
        if (var_work[(size_t)vx] != var_work[(size_t)vy])
            return var_work[(size_t)vx] > var_work[(size_t)vy];
        return vx < vy;
    });
    std::vector<BatchUnit> sorted(units.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = units[order[i]];
    size_t o_vars, o_units, o_counter;
    const size_t need = batch_layout(n_items, (int64_t)sorted.size(), &o_vars, &o_units, &o_counter);
    if (!ws) {
        *ws_bytes = need;
        return LW_OK;
    }
    if (*ws_bytes < need) {
        *ws_bytes = need;
        return LW_ESIZE;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) return LW_EINVAL;
    cudaStream_t st = as_stream(stream);
    char* base = static_cast<char*>(ws);
    if (cudaMemcpyAsync(base + o_vars, vars.data(), sizeof(DepositArgs) * vars.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(base + o_units, sorted.data(), sizeof(BatchUnit) * sorted.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return LW_ECUDA;
    // pageable sources: make sure the copies have consumed them before returning
    if (cudaStreamSynchronize(st) != cudaSuccess) return LW_ECUDA;
    plan->ws = ws;
    plan->n_items = n_items;
    plan->n_units = (int32_t)sorted.size();
    plan->precision = precision;
    plan->smem_bytes = (int32_t)(kMixStages * stage_bytes(max_block));
    plan->field_flags = (int32_t)field_flags;
    plan->reserved = 0;
    plan->offsets[0] = (int64_t)o_counter;
    plan->offsets[1] = (int64_t)o_vars;
    plan->offsets[2] = (int64_t)o_units;
    *ws_bytes = need;
    return LW_OK;
}

extern "C" int lw_batch_deposit(const lw_batch* plan, void* stream) {
    constexpr int PIX = kMixPix;
    if (!plan || !plan->ws || plan->n_items < 1) return LW_EINVAL;
    cudaStream_t st = as_stream(stream);
    char* base = static_cast<char*>(plan->ws);
    int* counter = reinterpret_cast<int*>(base + plan->offsets[0]);
    const DepositArgs* vars = reinterpret_cast<const DepositArgs*>(base + plan->offsets[1]);
    const BatchUnit* units = reinterpret_cast<const BatchUnit*>(base + plan->offsets[2]);
    if (plan->n_items > kBatchMaxItems) return LW_EUNSUPPORTED;
    zero_records_kernel<<<dim3(kSms * 4, (unsigned)plan->n_items), 256, 0, st>>>(
        vars, record_words(plan->precision));
    if (launch_status() != LW_OK) return LW_ECUDA;
    if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return LW_ECUDA;
    if (cudaMemcpyToSymbolAsync(c_batch_vars, vars, sizeof(DepositArgs) * (size_t)plan->n_items,
                                0, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return LW_ECUDA;
    if (plan->field_flags < 1 || plan->field_flags > 3) return LW_EINVAL;
    const BatchedKernel kern = batched_kernel(acc_of(plan->precision), (uint32_t)plan->field_flags);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             plan->smem_bytes) != cudaSuccess)
        return LW_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMixThreads,
                                                      plan->smem_bytes) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int dev = 0, sms = kSms;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(plan->n_units, sms * per_sm);
    kern<<<grid, kMixThreads, plan->smem_bytes, st>>>(units, plan->n_units, counter);
    if (launch_status() != LW_OK) return LW_ECUDA;
    // the precision check on every kCheckStride-th unit (LW_ST_PRECISION into the variants'
    // status words)
    const int stride = plan->n_units > kCheckStride ? kCheckStride : 1;
    const BatchedCheckKernel ck = batched_check_kernel((uint32_t)plan->field_flags);
    if (cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             plan->smem_bytes) != cudaSuccess)
        return LW_ECUDA;
    ck<<<(plan->n_units + stride - 1) / stride, kMixThreads, plan->smem_bytes, st>>>(
        units, plan->n_units, stride);
    return launch_status();
}
