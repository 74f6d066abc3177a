// Adjoint of lw_deposit_time_domain followed by lw_spectrum (FP64, and mixed precision below).
//
// Given g = dL/dS and the saved X' = sqrt(K) dt_u X, the record gradient is
//   dL/drec_c[j] = 2 sqrt(K) dt_u Re( sum_{l=0}^{N/2} g_l conj(X'_c(l)) e^{+2 pi i j l/N} ),
// evaluated as one complex FFT of two Hermitian-extended rows (both outputs
// are real, so they travel as the real and imaginary part of one transform).
// The deposit's adjoint is its transpose: a gather over the same
// (electron, step, pixel) intervals.  For grid point j in (t_b, t_a] with
// w = (t_j - t_b)/(t_a - t_b) the record received F_b (1 - w) + F_a w, so
//   dL/dF_b += R (1 - w),  dL/dF_a += R w,
//   dL/dt_a += -(R.(F_a - F_b)) w / (t_a - t_b),
//   dL/dt_b += -(R.(F_a - F_b)) (1 - w) / (t_a - t_b),
// and, per sample, with t_a = t - n.r/c0 and F = [(n-beta)(n.bdot) - D bdot]/D^3:
//   dL/dr    = -(dL/dt_a) n / c0,
//   dL/dbdot = [n ((n-beta).G) - D G] / D^3,
//   dL/dbeta = [-(n.bdot) G + n (bdot.G)] / D^3 + 3 n (F.G) / D,     G = dL/dF.
// Contributions of the 32 pixels of a warp to the same sample are summed with
// shuffles before one atomic add per component.
#include <math.h>

#include "lw_fft.cuh"

namespace lw {
namespace {

// ------------------------------------------------------------ adjoint FFT

struct AdjLoader {
    const double2* X;     // [n_pix][3][nl] (FP64 forward)
    const float2* Xf;     // the same from a mixed-precision forward (X unused when set)
    const double* g;      // [n_pix][nl]
    int64_t rows;         // 3 * n_pix
    int64_t nl;
    double two_sigma;     // 2 sqrt(K) dt_u

    __device__ double2 H(int64_t row, int64_t l) const {   // 2 sigma g_l conj(X'_l)
        double2 h;
        if (row >= rows) {
            h.x = h.y = 0.0;
            return h;
        }
        const int64_t m = row / 3;
        double2 x;
        if (Xf) {
            const float2 xf = Xf[row * nl + l];
            x.x = xf.x;
            x.y = xf.y;
        } else {
            x = X[row * nl + l];
        }
        const double s = two_sigma * g[m * nl + l];
        h.x = s * x.x;
        h.y = -s * x.y;
        return h;
    }
    // Hermitian extension of H at index l of a length-N transform
    __device__ double2 Ht(int64_t row, int64_t l, int64_t N) const {
        const int64_t half = N / 2;
        double2 h;
        if (l == 0 || l == half) {
            h = H(row, l);
            h.y = 0.0;
        } else if (l < half) {
            h = H(row, l);
            h.x *= 0.5;
            h.y *= 0.5;
        } else {
            h = H(row, N - l);
            h.x *= 0.5;
            h.y = -0.5 * h.y;
        }
        return h;
    }
    __device__ double2 operator()(int64_t pair, int64_t l, int64_t N) const {
        const double2 a = Ht(2 * pair, l, N), b = Ht(2 * pair + 1, l, N);
        double2 z;
        z.x = a.x - b.y;
        z.y = a.y + b.x;
        return z;
    }
};

__device__ __forceinline__ void adj_store(double* out, int64_t rows, int64_t pair, int64_t N,
                                          int64_t j, double2 z) {
    const int64_t ra = 2 * pair, rb = 2 * pair + 1;
    out[ra * N + j] = z.x;
    if (rb < rows) out[rb * N + j] = z.y;
}

__global__ void adj_direct_kernel(AdjLoader ld, int N, int logN, const double2* __restrict__ tw,
                                  double* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int64_t pair = blockIdx.x;
    for (int l = threadIdx.x; l < N; l += blockDim.x) buf[bitrev(l, logN)] = ld(pair, l, N);
    __syncthreads();
    fft_smem<double2, 1, false>(buf, N, logN, tw, N);
    for (int j = threadIdx.x; j < N; j += blockDim.x) adj_store(out, ld.rows, pair, N, j, buf[j]);
}

template <int CT>
__global__ void adj_pass1_kernel(AdjLoader ld, int N, int N1, int logN1, int N2,
                                 const double2* __restrict__ tw, double2* __restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);   // [N1][CT]
    const int64_t pair = blockIdx.y;
    const int c0 = blockIdx.x * CT;
    for (int t = threadIdx.x; t < N1 * CT; t += blockDim.x) {
        const int c = t % CT, n1 = t / CT;
        buf[bitrev(n1, logN1) * CT + c] = ld(pair, (int64_t)n1 * N2 + c0 + c, N);
    }
    __syncthreads();
    fft_smem<double2, CT, false>(buf, N1, logN1, tw, N);
    double2* Yp = Y + pair * (int64_t)N;
    for (int t = threadIdx.x; t < N1 * CT; t += blockDim.x) {
        const int c = t % CT, k1 = t / CT;
        const int n2 = c0 + c;
        Yp[(int64_t)k1 * N2 + n2] = cmul(buf[k1 * CT + c], tw[((int64_t)n2 * k1) & (N - 1)]);
    }
}

// rows k1 .. k1+CT-1 of the pass-1 output: transform over n2, write X[k1 + N1 k2]
template <int CT>
__global__ void adj_pass2_kernel(int64_t rows, int N, int N1, int N2, int logN2,
                                 const double2* __restrict__ tw, const double2* __restrict__ Y,
                                 double* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);   // [N2][CT]
    const int64_t pair = blockIdx.y;
    const int k10 = blockIdx.x * CT;
    const double2* Yp = Y + pair * (int64_t)N;
    for (int t = threadIdx.x; t < N2 * CT; t += blockDim.x) {
        const int n2 = t % N2, c = t / N2;
        buf[bitrev(n2, logN2) * CT + c] = Yp[(int64_t)(k10 + c) * N2 + n2];
    }
    __syncthreads();
    fft_smem<double2, CT, false>(buf, N2, logN2, tw, N);
    for (int t = threadIdx.x; t < N2 * CT; t += blockDim.x) {
        const int c = t % CT, k2 = t / CT;
        adj_store(out, rows, pair, N, (int64_t)(k10 + c) + (int64_t)N1 * k2, buf[k2 * CT + c]);
    }
}

// ------------------------------------------------------------ adjoint deposit

struct AdjArgs {
    int64_t n_e, ns1;
    int t_per_e;
    const double* t;
    const double* r;
    const double* beta;
    const double* bdot;
    const double* n_hat;
    int64_t n_pix;
    double t_min, dt_u, inv_dtu;
    int64_t n_bins;
    const double* dLdrec;   // [n_pix][3][n_bins]
    const float* dLdrec_f;  // mixed: dLdrec * 2^-e in FP32 (|values| < 2)
    const double* rscale;   // mixed: 2^e (device scalar)
    float* f_grad;          // mixed: per sample 12 floats, (dL/du_a n, dL/dbeta, dL/dbdot, 0)
                            // on the record gradient's scale, FP32 sums
    double* g_r;
    double* g_beta;
    double* g_bdot;
    int e_chunk;
};

constexpr int kAdjThreads = 128;
constexpr int kAdjTile = 64;

// acceleration field (the FP64 forward kernel's formula; one reciprocal of D^3 instead
// of three divisions -- the adjoint needs the field, not its last bit)
__device__ void field_acc_fp64(double nx, double ny, double nz, const double* __restrict__ b,
                               const double* __restrict__ a, double F[3]) {
    const double b0 = b[0], b1 = b[1], b2v = b[2];
    const double bb = __dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)),
                                __dmul_rn(b2v, b2v));
    const double D = __dsub_rn(1.0, __dadd_rn(__dadd_rn(__dmul_rn(nx, b0), __dmul_rn(ny, b1)),
                                              __dmul_rn(nz, b2v)));
    F[0] = F[1] = F[2] = 0.0;
    if (!(bb < 1.0) || !(D > 0.0)) return;
    const double D3 = __dmul_rn(__dmul_rn(D, D), D);
    const double m0 = __dsub_rn(nx, b0), m1 = __dsub_rn(ny, b1), m2 = __dsub_rn(nz, b2v);
    const double i0 = __dsub_rn(__dmul_rn(m1, a[2]), __dmul_rn(m2, a[1]));
    const double i1 = __dsub_rn(__dmul_rn(m2, a[0]), __dmul_rn(m0, a[2]));
    const double i2 = __dsub_rn(__dmul_rn(m0, a[1]), __dmul_rn(m1, a[0]));
    const double iD3 = 1.0 / D3;
    F[0] = __dsub_rn(__dmul_rn(ny, i2), __dmul_rn(nz, i1)) * iD3;
    F[1] = __dsub_rn(__dmul_rn(nz, i0), __dmul_rn(nx, i2)) * iD3;
    F[2] = __dsub_rn(__dmul_rn(nx, i1), __dmul_rn(ny, i0)) * iD3;
}

// (dL/dF, dL/dt_a) of one sample -> (dL/dr, dL/dbeta, dL/dbdot)
__device__ void sample_chain(double nx, double ny, double nz, const double* __restrict__ b,
                             const double* __restrict__ a, const double G[3], double gta,
                             double out[9]) {
    out[0] = -gta * nx * kInvC0;
    out[1] = -gta * ny * kInvC0;
    out[2] = -gta * nz * kInvC0;
    const double D = 1.0 - (nx * b[0] + ny * b[1] + nz * b[2]);
    if (!(D > 0.0) || !(b[0] * b[0] + b[1] * b[1] + b[2] * b[2] < 1.0)) {
        for (int c = 3; c < 9; ++c) out[c] = 0.0;
        return;
    }
    const double iD = 1.0 / D, iD3 = iD * iD * iD;
    const double mx = nx - b[0], my = ny - b[1], mz = nz - b[2];
    const double nbd = nx * a[0] + ny * a[1] + nz * a[2];
    const double bG = a[0] * G[0] + a[1] * G[1] + a[2] * G[2];
    const double mG = mx * G[0] + my * G[1] + mz * G[2];
    const double Fx = (mx * nbd - D * a[0]) * iD3, Fy = (my * nbd - D * a[1]) * iD3,
                 Fz = (mz * nbd - D * a[2]) * iD3;
    const double FG = Fx * G[0] + Fy * G[1] + Fz * G[2];
    out[3] = (-nbd * G[0] + nx * bG) * iD3 + 3.0 * nx * FG * iD;
    out[4] = (-nbd * G[1] + ny * bG) * iD3 + 3.0 * ny * FG * iD;
    out[5] = (-nbd * G[2] + nz * bG) * iD3 + 3.0 * nz * FG * iD;
    out[6] = (nx * mG - D * G[0]) * iD3;
    out[7] = (ny * mG - D * G[1]) * iD3;
    out[8] = (nz * mG - D * G[2]) * iD3;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// finish sample i: chain rule, warp sum over pixels, atomics into the gradients
__device__ __forceinline__ void flush_sample(const AdjArgs& p, bool act, double nx, double ny,
                                             double nz, int64_t k, int64_t i, const double G[3],
                                             double gta, bool nonzero) {
    if (!__any_sync(0xffffffffu, nonzero)) return;
    double o[9];
    const int64_t s = k * p.ns1 + i;
    if (nonzero && act) {
        sample_chain(nx, ny, nz, p.beta + 3 * s, p.bdot + 3 * s, G, gta, o);
    } else {
        for (int c = 0; c < 9; ++c) o[c] = 0.0;
    }
    for (int c = 0; c < 9; ++c) o[c] = warp_sum(o[c]);
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 3; ++c) {
            atomicAdd(p.g_r + 3 * s + c, o[c]);
            atomicAdd(p.g_beta + 3 * s + c, o[3 + c]);
            atomicAdd(p.g_bdot + 3 * s + c, o[6 + c]);
        }
    }
}

__global__ void __launch_bounds__(kAdjThreads) adj_deposit_kernel(AdjArgs p) {
    __shared__ double s_t[kAdjTile];
    __shared__ double s_r[kAdjTile * 3];
    const int64_t m = (int64_t)blockIdx.x * kAdjThreads + threadIdx.x;
    const bool active = m < p.n_pix;
    double nx = 0.0, ny = 0.0, nz = 1.0;
    if (active) {
        nx = p.n_hat[3 * m];
        ny = p.n_hat[3 * m + 1];
        nz = p.n_hat[3 * m + 2];
    }
    const double* R = p.dLdrec + (active ? m * 3 * p.n_bins : 0);
    const int64_t k0 = (int64_t)blockIdx.y * p.e_chunk;
    const int64_t k1 = min(k0 + p.e_chunk, p.n_e);
    for (int64_t k = k0; k < k1; ++k) {
        const double* tk = p.t + (p.t_per_e ? k * p.ns1 : 0);
        const double* rk = p.r + 3 * k * p.ns1;
        const double* bk = p.beta + 3 * k * p.ns1;
        const double* ak = p.bdot + 3 * k * p.ns1;
        double tb = 0.0, ub = 0.0;
        double Fb[3] = {0.0, 0.0, 0.0};
        int64_t fb_step = -1;
        double Gc[3] = {0.0, 0.0, 0.0}, gtc = 0.0;   // carry: sample i-1 so far
        bool nzc = false;
        for (int64_t i0 = 0; i0 < p.ns1; i0 += kAdjTile) {
            const int n = (int)min((int64_t)kAdjTile, p.ns1 - i0);
            __syncthreads();
            for (int q = threadIdx.x; q < n; q += kAdjThreads) {
                s_t[q] = tk[i0 + q];
                s_r[3 * q] = rk[3 * (i0 + q)];
                s_r[3 * q + 1] = rk[3 * (i0 + q) + 1];
                s_r[3 * q + 2] = rk[3 * (i0 + q) + 2];
            }
            __syncthreads();
            for (int q = 0; q < n; ++q) {
                const int64_t i = i0 + q;
                const double ta = advanced_time_fp64(nx, ny, nz, s_r[3 * q], s_r[3 * q + 1],
                                                     s_r[3 * q + 2], s_t[q]);
                const double ua = __dmul_rn(__dsub_rn(ta, p.t_min), p.inv_dtu);
                double Gn[3] = {0.0, 0.0, 0.0}, gtn = 0.0;   // contributions to sample i
                bool nzn = false;
                if (i > 0 && active && fabs(ua) < 4.0e18 && fabs(ub) < 4.0e18) {
                    int64_t ja = (int64_t)floor(ub) + 1, jz = (int64_t)floor(ua);
                    if (ja < 0) ja = 0;
                    if (jz > p.n_bins - 1) jz = p.n_bins - 1;
                    if (ja <= jz) {
                        if (fb_step != i - 1)
                            field_acc_fp64(nx, ny, nz, bk + 3 * (i - 1), ak + 3 * (i - 1), Fb);
                        double Fa[3];
                        field_acc_fp64(nx, ny, nz, bk + 3 * i, ak + 3 * i, Fa);
                        const double den = __dsub_rn(ta, tb);
                        const double iden = 1.0 / den;   // one division per step
                        for (int64_t j = ja; j <= jz; ++j) {
                            const double tu = __dadd_rn(p.t_min, __dmul_rn((double)j, p.dt_u));
                            const double wa = __dsub_rn(ta, tu) * iden;
                            const double wb = __dsub_rn(tu, tb) * iden;
                            const double R0 = R[j], R1 = R[p.n_bins + j], R2 = R[2 * p.n_bins + j];
                            Gc[0] += R0 * wa;
                            Gc[1] += R1 * wa;
                            Gc[2] += R2 * wa;
                            Gn[0] += R0 * wb;
                            Gn[1] += R1 * wb;
                            Gn[2] += R2 * wb;
                            const double dw = R0 * (Fa[0] - Fb[0]) + R1 * (Fa[1] - Fb[1]) +
                                              R2 * (Fa[2] - Fb[2]);
                            gtn -= dw * wb * iden;
                            gtc -= dw * wa * iden;
                        }
                        nzc = true;
                        nzn = true;
                        Fb[0] = Fa[0];
                        Fb[1] = Fa[1];
                        Fb[2] = Fa[2];
                        fb_step = i;
                    }
                }
                if (i > 0) flush_sample(p, active, nx, ny, nz, k, i - 1, Gc, gtc, nzc);
                Gc[0] = Gn[0];
                Gc[1] = Gn[1];
                Gc[2] = Gn[2];
                gtc = gtn;
                nzc = nzn;
                tb = ta;
                ub = ua;
            }
        }
        flush_sample(p, active, nx, ny, nz, k, p.ns1 - 1, Gc, gtc, nzc);
    }
}

// ------------------------------------------------------------ mixed-precision adjoint
//
// The same transpose in mixed precision: the bin coordinate of each tile's first sample in
// FP64 and, within the tile of 64 samples, each sample's as an integer plus an FP32
// fraction advanced by the step's FP32 increment (from FP64-differenced samples), so the
// weights are computed from numbers of the size of a step; everything else in FP32:
// the fields in the stable form
// D = (1 - n_z) + n_z (1 - beta_z) - n_perp . beta_perp, the weights from bin coordinates
// relative to the step's first grid point, the sums over grid points and the per-sample
// chain rule.  The record gradient enters scaled by a power of two 2^-e (|values| < 2,
// e from its largest magnitude), so that its products with fields of up to ~1e30 /s stay
// in FP32 range; the warp sums are unscaled in FP64 before the FP64 atomics.

// largest |dL/drec| as ordered bits (non-negative doubles compare as integers)
__global__ void adj_absmax_kernel(const double* __restrict__ R, int64_t n,
                                  unsigned long long* __restrict__ mx) {
    unsigned long long v = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(R[i]));
        v = b > v ? b : v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(mx, v);
}

// 2^e >= the largest |dL/drec| / 2 (1 when it is zero or not finite)
__device__ __forceinline__ int adj_exponent(unsigned long long mx) {
    const int e = (int)(mx >> 52) - 1023;
    return (mx == 0 || e > 1000 || e < -1000) ? 0 : e;
}

__global__ void adj_to_f32_kernel(const double* __restrict__ R, int64_t n,
                                  const unsigned long long* __restrict__ mx,
                                  float* __restrict__ Rf, double* __restrict__ rscale) {
    const int e = adj_exponent(*mx);
    const double down = ldexp(1.0, -e);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        Rf[i] = (float)(R[i] * down);
    if (blockIdx.x == 0 && threadIdx.x == 0) *rscale = ldexp(1.0, e);
}

struct NF {   // a pixel direction in FP32 with 1 - n_z kept exactly
    float x, y, z, omz;
};

// acceleration field (n - beta) (n . bdot) - D bdot) / D^3 in FP32; zero when |beta| >= 1
// (b.w == 0) or D <= 0
__device__ __forceinline__ void field_acc_f32(const NF& n, float4 b, float4 a, float F[3]) {
    const float D = fmaf(-n.y, b.y, fmaf(-n.x, b.x, fmaf(n.z, b.z, n.omz)));
    const float mx = n.x - b.x, my = n.y - b.y, mz = b.z - n.omz;
    const float nbd = fmaf(n.z, a.z, fmaf(n.y, a.y, n.x * a.x));
    const float iD = __fdividef(1.0f, D);
    const float iD3 = (b.w != 0.0f && D > 0.0f) ? iD * iD * iD : 0.0f;
    F[0] = fmaf(mx, nbd, -D * a.x) * iD3;
    F[1] = fmaf(my, nbd, -D * a.y) * iD3;
    F[2] = fmaf(mz, nbd, -D * a.z) * iD3;
}

// (dL/dF, dL/du_a) of one sample -> (dL/du_a n, dL/dbeta, dL/dbdot) in FP32, on the scale
// of the record gradient; dL/dr = -(dL/du_a) n / (c0 dt_u) is completed by the caller
__device__ __forceinline__ void sample_chain_f32(const NF& n, float4 b, float4 a,
                                                 const float G[3], float gu, float o[9]) {
    o[0] = gu * n.x;
    o[1] = gu * n.y;
    o[2] = gu * n.z;
    const float D = fmaf(-n.y, b.y, fmaf(-n.x, b.x, fmaf(n.z, b.z, n.omz)));
    if (b.w == 0.0f || !(D > 0.0f)) {
        for (int c = 3; c < 9; ++c) o[c] = 0.0f;
        return;
    }
    const float iD = __fdividef(1.0f, D), iD3 = iD * iD * iD;
    const float mx = n.x - b.x, my = n.y - b.y, mz = b.z - n.omz;
    const float nbd = fmaf(n.z, a.z, fmaf(n.y, a.y, n.x * a.x));
    const float bG = fmaf(a.z, G[2], fmaf(a.y, G[1], a.x * G[0]));
    const float mG = fmaf(mz, G[2], fmaf(my, G[1], mx * G[0]));
    const float Fx = fmaf(mx, nbd, -D * a.x) * iD3, Fy = fmaf(my, nbd, -D * a.y) * iD3,
                Fz = fmaf(mz, nbd, -D * a.z) * iD3;
    const float FG3 = 3.0f * fmaf(Fz, G[2], fmaf(Fy, G[1], Fx * G[0])) * iD;
    o[3] = fmaf(fmaf(-nbd, G[0], n.x * bG), iD3, n.x * FG3);
    o[4] = fmaf(fmaf(-nbd, G[1], n.y * bG), iD3, n.y * FG3);
    o[5] = fmaf(fmaf(-nbd, G[2], n.z * bG), iD3, n.z * FG3);
    o[6] = fmaf(n.x, mG, -D * G[0]) * iD3;
    o[7] = fmaf(n.y, mG, -D * G[1]) * iD3;
    o[8] = fmaf(n.z, mG, -D * G[2]) * iD3;
}

__device__ __forceinline__ void flush_sample_f32(const AdjArgs& p, bool act, const NF& n,
                                                 int64_t k, int64_t i, float4 b, float4 a,
                                                 const float G[3], float gu, bool nonzero,
                                                 double r_scale, double u_scale) {
    if (!__any_sync(0xffffffffu, nonzero)) return;
    float o[9];
    if (nonzero && act) {
        sample_chain_f32(n, b, a, G, gu, o);
    } else {
        for (int c = 0; c < 9; ++c) o[c] = 0.0f;
    }
    for (int c = 0; c < 9; ++c)
        for (int s = 16; s > 0; s >>= 1) o[c] += __shfl_xor_sync(0xffffffffu, o[c], s);
    if ((threadIdx.x & 31) == 0) {   // three 16-byte FP32 reductions (no FP64 in the loop)
        float* f = p.f_grad + 12 * (k * p.ns1 + i);
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(f), "f"(o[0]),
                     "f"(o[1]), "f"(o[2]), "f"(o[3]) : "memory");
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(f + 4), "f"(o[4]),
                     "f"(o[5]), "f"(o[6]), "f"(o[7]) : "memory");
        asm volatile("red.global.add.f32 [%0], %1;" ::"l"(f + 8), "f"(o[8]) : "memory");
    }
}

// the FP32 sums in FP64, unscaled, added to the caller's gradients
__global__ void adj_finish_kernel(const float* __restrict__ f, int64_t n_samples,
                                  const double* __restrict__ rscale, double inv_dtu,
                                  double* __restrict__ g_r, double* __restrict__ g_b,
                                  double* __restrict__ g_a) {
    const double r_scale = *rscale;
    const double u_scale = -r_scale * inv_dtu * kInvC0;   // dL/dr = -(dL/du_a) n / (c0 dt_u)
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_samples;
         s += (int64_t)gridDim.x * blockDim.x) {
        const float* q = f + 12 * s;
        for (int c = 0; c < 3; ++c) {
            g_r[3 * s + c] += (double)q[c] * u_scale;
            g_b[3 * s + c] += (double)q[3 + c] * r_scale;
            g_a[3 * s + c] += (double)q[6 + c] * r_scale;
        }
    }
}

// Half-width of the band around an integer inside which a sample's bin coordinate is
// recomputed in FP64: far above the FP32 chain's rounding over a tile (64 steps of a few
// ulps of the step's terms).
constexpr float kAdjGuard = 1.0f / (1 << 12);

__global__ void __launch_bounds__(kAdjThreads) adj_deposit_mixed_kernel(AdjArgs p) {
    // one tile of samples i0 .. i0 + kAdjTile - 1, staged once per CTA: each sample's step
    // from the previous one (FP64 differences rounded to FP32) and its fields' inputs
    __shared__ float4 s_d[kAdjTile];   // (tau_i - tau_i-1, r_i - r_i-1), tau = t - z/c0
    __shared__ float4 s_b[kAdjTile];   // (beta_x, beta_y, 1 - beta_z, |beta| < 1)
    __shared__ float4 s_a[kAdjTile];   // (beta_dot, 0)
    __shared__ double s_anc[4];        // (t, r) of sample i0
    const int64_t m = (int64_t)blockIdx.x * kAdjThreads + threadIdx.x;
    const bool active = m < p.n_pix;
    double nx = 0.0, ny = 0.0, nz = 1.0;
    if (active) {
        nx = p.n_hat[3 * m];
        ny = p.n_hat[3 * m + 1];
        nz = p.n_hat[3 * m + 2];
    }
    NF nf;
    nf.x = (float)nx;
    nf.y = (float)ny;
    nf.z = (float)nz;
    nf.omz = (float)(1.0 - nz);
    // bin coordinate u = (t_a - t_min)/dt_u = (tau - t_min)/dt_u + w . r with the pixel's
    // slope w = (-n_x, -n_y, 1 - n_z) / (c0 dt_u): in FP64 at each tile's first sample; from
    // there on as J + f (integer, FP32 fraction) advanced by each step's FP32 increment
    // s dtau + w . dr, so that the weights see small numbers
    const double sw = kInvC0 * p.inv_dtu;
    const double wx = -nx * sw, wy = -ny * sw, wz = (1.0 - nz) * sw;
    const float s32 = (float)p.inv_dtu, wx32 = (float)wx, wy32 = (float)wy, wz32 = (float)wz;
    const double r_scale = *p.rscale;
    // dL/dr = -(dL/du_a) n / (c0 dt_u), on the record gradient's scale
    const double u_scale = -r_scale * p.inv_dtu * kInvC0;
    const float* R = p.dLdrec_f + (active ? m * 3 * p.n_bins : 0);
    const bool vec = (p.n_bins & 3) == 0;
    // the FP64 adjoint's bin coordinate of a sample, and its split into floor + fraction
    auto u_fp64 = [&](double t, double x, double y, double z) {
        return __dmul_rn(__dsub_rn(advanced_time_fp64(nx, ny, nz, x, y, z, t), p.t_min),
                         p.inv_dtu);
    };
    auto exact_coord = [&](double u, int64_t& Jo, float& fo) {
        u = fmin(fmax(u, -1.0e15), 1.0e15);
        const double fl = floor(u);
        Jo = (int64_t)fl;
        fo = (float)(u - fl);
    };
    const int64_t k0 = (int64_t)blockIdx.y * p.e_chunk;
    const int64_t k1 = min(k0 + p.e_chunk, p.n_e);
    for (int64_t k = k0; k < k1; ++k) {
        const double* tk = p.t + (p.t_per_e ? k * p.ns1 : 0);
        const double* rk = p.r + 3 * k * p.ns1;
        const double* bk = p.beta + 3 * k * p.ns1;
        const double* ak = p.bdot + 3 * k * p.ns1;
        float Fb[3] = {0.0f, 0.0f, 0.0f};
        int64_t fb_step = -1;
        float Gc[3] = {0.0f, 0.0f, 0.0f}, guc = 0.0f;   // carry: sample i-1 so far
        bool nzc = false;
        float4 pb = make_float4(0.f, 0.f, 0.f, 0.f), pa = pb;   // sample i-1
        int64_t J = 0;   // sample i-1 at J + f
        // the pixel's record-gradient rows are read in increasing j: with n_bins a multiple
        // of 4 (16-byte aligned rows) a lane keeps the 16-byte chunk of each row holding the
        // current j, one vector load per row and 4 bins instead of one scalar per bin (the
        // lanes of a warp read 32 different rows, so loads cost one L1 wavefront per lane)
        int64_t jc = -4;
        float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0, c2 = c0;
        float f = 0.0f;
        for (int64_t i0 = 0; i0 < p.ns1; i0 += kAdjTile) {
            const int n = (int)min((int64_t)kAdjTile, p.ns1 - i0);
            __syncthreads();
            for (int q = threadIdx.x; q < n; q += kAdjThreads) {
                const int64_t i = i0 + q;
                const double* rq = rk + 3 * i;
                const double* bq = bk + 3 * i;
                const double* aq = ak + 3 * i;
                if (i > 0) {
                    const double tau = tk[i] - rq[2] * kInvC0;
                    const double taup = tk[i - 1] - rq[-1] * kInvC0;
                    s_d[q] = make_float4((float)(tau - taup), (float)(rq[0] - rq[-3]),
                                         (float)(rq[1] - rq[-2]), (float)(rq[2] - rq[-1]));
                }
                const double bb = __dadd_rn(__dadd_rn(__dmul_rn(bq[0], bq[0]),
                                                      __dmul_rn(bq[1], bq[1])),
                                            __dmul_rn(bq[2], bq[2]));
                s_b[q] = make_float4((float)bq[0], (float)bq[1], (float)(1.0 - bq[2]),
                                     bb < 1.0 ? 1.0f : 0.0f);
                s_a[q] = make_float4((float)aq[0], (float)aq[1], (float)aq[2], 0.0f);
            }
            if (threadIdx.x == 0) {
                s_anc[0] = tk[i0];
                s_anc[1] = rk[3 * i0];
                s_anc[2] = rk[3 * i0 + 1];
                s_anc[3] = rk[3 * i0 + 2];
            }
            __syncthreads();
            // sample i0 with the FP64 adjoint's expression: J0 + f0
            int64_t J0;
            float f0;
            exact_coord(u_fp64(s_anc[0], s_anc[1], s_anc[2], s_anc[3]), J0, f0);
            for (int q = 0; q < n; ++q) {
                const int64_t i = i0 + q;
                const float4 cb = s_b[q], ca = s_a[q];
                // sample i at Ji + fi: the tile's first from the FP64 anchor, the others
                // advanced from sample i-1 by the step's FP32 increment, and recomputed in
                // FP64 when the fraction lies within kAdjGuard of an integer, so that the
                // floors -- which grid points a step holds -- are those of the FP64 adjoint
                int64_t Ji;
                float fi;
                if (q == 0) {
                    Ji = J0;
                    fi = f0;
                } else {
                    const float4 d = s_d[q];
                    float u = f + fmaf(wz32, d.w, fmaf(wy32, d.z, fmaf(wx32, d.y, s32 * d.x)));
                    u = fminf(fmaxf(u, -1.0e9f), 1.0e9f);
                    const float fl = floorf(u);
                    Ji = J + (int64_t)fl;
                    fi = u - fl;
                    if (fi < kAdjGuard || fi > 1.0f - kAdjGuard) {
                        const double* rq = rk + 3 * i;
                        exact_coord(u_fp64(tk[i], rq[0], rq[1], rq[2]), Ji, fi);
                    }
                }
                // the step (i-1, i] relative to Jf = J_(i-1): ub = f_(i-1), ua = u_i - Jf
                const int64_t Jf = J, dJ = Ji - J;
                const float ub = f;
                const float ua = (dJ > -(1 << 24) && dJ < (1 << 24)) ? (float)dJ + fi : 1.0e9f;
                float Gn[3] = {0.0f, 0.0f, 0.0f}, gun = 0.0f;   // contributions to sample i
                bool nzn = false;
                if (i > 0 && active) {
                    int64_t ja = J + 1, jz = Ji;
                    if (ja < 0) ja = 0;
                    if (jz > p.n_bins - 1) jz = p.n_bins - 1;
                    if (ja <= jz) {
                        if (fb_step != i - 1) field_acc_f32(nf, pb, pa, Fb);
                        float Fa[3];
                        field_acc_f32(nf, cb, ca, Fa);
                        const float iden = __fdividef(1.0f, ua - ub);
                        const float d0 = Fa[0] - Fb[0], d1 = Fa[1] - Fb[1], d2 = Fa[2] - Fb[2];
                        for (int64_t j = ja; j <= jz; ++j) {
                            const float tj = (float)(j - Jf);
                            const float wa = (ua - tj) * iden, wb = (tj - ub) * iden;
                            float R0, R1, R2;
                            if (vec) {   // 16-byte chunks of the three rows, reloaded per 4 bins
                                if ((j & ~int64_t(3)) != jc) {
                                    jc = j & ~int64_t(3);
                                    c0 = __ldg(reinterpret_cast<const float4*>(R + jc));
                                    c1 = __ldg(reinterpret_cast<const float4*>(R + p.n_bins + jc));
                                    c2 = __ldg(reinterpret_cast<const float4*>(R + 2 * p.n_bins + jc));
                                }
                                const int e = (int)(j & 3);
                                R0 = e == 0 ? c0.x : e == 1 ? c0.y : e == 2 ? c0.z : c0.w;
                                R1 = e == 0 ? c1.x : e == 1 ? c1.y : e == 2 ? c1.z : c1.w;
                                R2 = e == 0 ? c2.x : e == 1 ? c2.y : e == 2 ? c2.z : c2.w;
                            } else {
                                R0 = R[j];
                                R1 = R[p.n_bins + j];
                                R2 = R[2 * p.n_bins + j];
                            }
                            Gc[0] = fmaf(R0, wa, Gc[0]);
                            Gc[1] = fmaf(R1, wa, Gc[1]);
                            Gc[2] = fmaf(R2, wa, Gc[2]);
                            Gn[0] = fmaf(R0, wb, Gn[0]);
                            Gn[1] = fmaf(R1, wb, Gn[1]);
                            Gn[2] = fmaf(R2, wb, Gn[2]);
                            const float dw = fmaf(R2, d2, fmaf(R1, d1, R0 * d0)) * iden;
                            gun = fmaf(-dw, wb, gun);
                            guc = fmaf(-dw, wa, guc);
                        }
                        nzc = true;
                        nzn = true;
                        Fb[0] = Fa[0];
                        Fb[1] = Fa[1];
                        Fb[2] = Fa[2];
                        fb_step = i;
                    }
                }
                if (i > 0)
                    flush_sample_f32(p, active, nf, k, i - 1, pb, pa, Gc, guc, nzc, r_scale,
                                     u_scale);
                Gc[0] = Gn[0];
                Gc[1] = Gn[1];
                Gc[2] = Gn[2];
                guc = gun;
                nzc = nzn;
                J = Ji;
                f = fi;
                pb = cb;
                pa = ca;
            }
        }
        flush_sample_f32(p, active, nf, k, p.ns1 - 1, pb, pa, Gc, guc, nzc, r_scale, u_scale);
    }
}

int pick_chunk(int64_t n_e, int64_t tiles) {
    const int64_t target = (int64_t)kSms * 16;
    int64_t chunk = (n_e * tiles + target - 1) / target;
    if (chunk < 1) chunk = 1;
    if (chunk > n_e) chunk = n_e;
    return (int)chunk;
}

}  // namespace
}  // namespace lw

using namespace lw;

extern "C" int lw_spectrum_grad(const lw_traj* traj, const lw_detector* det, const lw_grid* grid,
                                int32_t precision, uint32_t field_flags, const void* X_save,
                                const double* dL_dS, double q, double* dL_dr, double* dL_dbeta,
                                double* dL_dbeta_dot, void* ws, size_t* ws_bytes, void* stream) {
    if (!traj || !det || !grid || !ws_bytes || !det->n_hat || det->n_pix < 1) return LW_EINVAL;
    const bool mixed = precision == LW_MIXED || precision == LW_MIXED_KAHAN ||
                       precision == LW_MIXED_F32 || precision == LW_MIXED_F32X4;
    if (precision != LW_FP64 && !mixed) return LW_EUNSUPPORTED;
    if (field_flags != LW_FIELD_ACCEL) return LW_EUNSUPPORTED;
    if (!(traj->sections & LW_SECTION_FP64)) return LW_EINVAL;
    const int64_t N = grid->n_bins;
    if (N < 2 || N > (int64_t(1) << 18) || (N & (N - 1))) return LW_EUNSUPPORTED;
    if (!(grid->dt_u > 0.0) || !isfinite(q)) return LW_EINVAL;
    int logN = 0;
    while ((int64_t(1) << logN) < N) ++logN;
    const bool direct = N <= 4096;
    const int64_t rows = 3 * det->n_pix;
    const int64_t pairs = (rows + 1) / 2;
    const size_t rec_bytes = align256(sizeof(double) * (size_t)(rows * N));
    const size_t tw_bytes = align256(sizeof(double2) * (size_t)N);
    const size_t y_bytes = direct ? 0 : align256(sizeof(double2) * (size_t)(pairs * N));
    // mixed: the scaled FP32 record gradient, its largest magnitude and the scale
    const size_t gsum_bytes = mixed ? align256(sizeof(float) * 12 * (size_t)(traj->n_e * (traj->n_s + 1))) : 0;
    const size_t f_bytes = mixed ? align256(sizeof(float) * (size_t)(rows * N)) + 256 + gsum_bytes : 0;
    const size_t need = rec_bytes + tw_bytes + y_bytes + f_bytes;
    if (!ws) {
        *ws_bytes = need;
        return LW_OK;
    }
    if (*ws_bytes < need) {
        *ws_bytes = need;
        return LW_ESIZE;
    }
    if (!X_save || !dL_dS || !dL_dr || !dL_dbeta || !dL_dbeta_dot) return LW_EINVAL;
    cudaStream_t st = as_stream(stream);
    char* base = static_cast<char*>(ws);
    double* dLdrec = reinterpret_cast<double*>(base);
    double2* tw = reinterpret_cast<double2*>(base + rec_bytes);
    double2* Y = reinterpret_cast<double2*>(base + rec_bytes + tw_bytes);
    const double K = q * q / (16.0 * kPi * kPi * kPi * kEps0 * kC0);
    AdjLoader ld;
    ld.X = mixed ? nullptr : static_cast<const double2*>(X_save);
    ld.Xf = mixed ? static_cast<const float2*>(X_save) : nullptr;
    ld.g = dL_dS;
    ld.rows = rows;
    ld.nl = N / 2 + 1;
    ld.two_sigma = 2.0 * sqrt(K) * grid->dt_u;

    const int tw_grid = (int)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024);
    twiddle_kernel<double><<<tw_grid, 256, 0, st>>>(tw, N);
    if (launch_status() != LW_OK) return LW_ECUDA;
    if (direct) {
        const size_t smem = sizeof(double2) * (size_t)N;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(adj_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return LW_ECUDA;
        adj_direct_kernel<<<(unsigned)pairs, 256, smem, st>>>(ld, (int)N, logN, tw, dLdrec);
    } else {
        const int logN2 = (logN + 1) / 2, logN1 = logN - logN2;
        const int N1 = 1 << logN1, N2 = 1 << logN2;
        constexpr int CT = 16;
        size_t smem = sizeof(double2) * (size_t)N1 * CT;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(adj_pass1_kernel<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return LW_ECUDA;
        adj_pass1_kernel<CT><<<dim3((unsigned)(N2 / CT), (unsigned)pairs), 256, smem, st>>>(
            ld, (int)N, N1, logN1, N2, tw, Y);
        if (launch_status() != LW_OK) return LW_ECUDA;
        smem = sizeof(double2) * (size_t)N2 * CT;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(adj_pass2_kernel<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return LW_ECUDA;
        adj_pass2_kernel<CT><<<dim3((unsigned)(N1 / CT), (unsigned)pairs), 256, smem, st>>>(
            rows, (int)N, N1, N2, logN2, tw, Y, dLdrec);
    }
    if (launch_status() != LW_OK) return LW_ECUDA;

    AdjArgs a{};
    a.n_e = traj->n_e;
    a.ns1 = traj->n_s + 1;
    a.t_per_e = traj->t_per_electron;
    a.t = traj->t;
    a.r = traj->r;
    a.beta = traj->beta;
    a.bdot = traj->beta_dot;
    a.n_hat = det->n_hat;
    a.n_pix = det->n_pix;
    a.t_min = grid->t_min;
    a.dt_u = grid->dt_u;
    a.inv_dtu = 1.0 / grid->dt_u;
    a.n_bins = N;
    a.dLdrec = dLdrec;
    a.g_r = dL_dr;
    a.g_beta = dL_dbeta;
    a.g_bdot = dL_dbeta_dot;
    const int64_t tiles = (det->n_pix + kAdjThreads - 1) / kAdjThreads;
    a.e_chunk = pick_chunk(traj->n_e, tiles);
    dim3 g((unsigned)tiles, (unsigned)((traj->n_e + a.e_chunk - 1) / a.e_chunk));
    if (!mixed) {
        adj_deposit_kernel<<<g, kAdjThreads, 0, st>>>(a);
        return launch_status();
    }
    char* fbase = base + rec_bytes + tw_bytes + y_bytes;
    float* Rf = reinterpret_cast<float*>(fbase);
    unsigned long long* mx =
        reinterpret_cast<unsigned long long*>(fbase + align256(sizeof(float) * (size_t)(rows * N)));
    double* rscale = reinterpret_cast<double*>(mx + 1);
    if (cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st) != cudaSuccess) return LW_ECUDA;
    const int64_t n_rec = rows * N;
    const int rg = (int)std::min<int64_t>((n_rec + 255) / 256, (int64_t)kSms * 8);
    adj_absmax_kernel<<<rg, 256, 0, st>>>(dLdrec, n_rec, mx);
    adj_to_f32_kernel<<<rg, 256, 0, st>>>(dLdrec, n_rec, mx, Rf, rscale);
    if (launch_status() != LW_OK) return LW_ECUDA;
    a.dLdrec_f = Rf;
    a.rscale = rscale;
    a.f_grad = reinterpret_cast<float*>(fbase + align256(sizeof(float) * (size_t)(rows * N)) + 256);
    const int64_t n_samples = traj->n_e * (traj->n_s + 1);
    if (cudaMemsetAsync(a.f_grad, 0, sizeof(float) * 12 * (size_t)n_samples, st) != cudaSuccess)
        return LW_ECUDA;
    adj_deposit_mixed_kernel<<<g, kAdjThreads, 0, st>>>(a);
    if (launch_status() != LW_OK) return LW_ECUDA;
    const int fg = (int)std::min<int64_t>((n_samples + 255) / 256, (int64_t)kSms * 8);
    adj_finish_kernel<<<fg, 256, 0, st>>>(a.f_grad, n_samples, rscale, a.inv_dtu, a.g_r, a.g_beta,
                                          a.g_bdot);
    return launch_status();
}
