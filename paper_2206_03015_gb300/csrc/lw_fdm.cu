// Frequency-domain method (Eq. inty_dft / Algorithm 1 of the paper), the
// comparison method of the time-domain path, on a uniform frequency grid
// omega_w = omega0 + w * d_omega:
//   S(n, omega) = q^2 dt^2 / (16 pi^3 eps0 c0)
//                 | sum_k sum_i A_k(n, t_i) exp(j omega (t_i - n.r_ki / c0)) |^2,
//   A = n x ((n - beta) x beta_dot) / (1 - n.beta)^2.
//
// One CTA owns one pixel and 1024 frequencies (4 per thread).  Per staged
// sample one thread computes in FP64 the phase time tau, the vector A (then
// rounded to FP32) and three phases reduced modulo 2 pi: omega_base tau,
// 32 d_omega tau and d_omega tau (kept as FP32 hi + lo pairs).  The twiddles
// exp(j (omega_base + 32 a d_omega) tau) and exp(j b d_omega tau), a, b = 0..31,
// follow in double-FP32 arithmetic (exact products, reduction by a two-float
// 2 pi) and one FP32 sincos each; a thread's twiddle for frequency w = 32 a + b
// is one complex product.  Per sample and frequency that leaves one complex
// product and six FMAs; partial sums over a staged chunk are FP32 and are
// added to compensated (two-float) totals.
#include <math.h>

#include "lw_internal.cuh"

namespace lw {
namespace {

constexpr int kFdmThreads = 256;
constexpr int kFdmFreq = 1024;          // frequencies per CTA
constexpr int kFdmPer = kFdmFreq / kFdmThreads;
constexpr int kFdmChunk = 16;           // samples staged per round

struct FdmArgs {
    int64_t n_e, ns1;
    int t_per_e;
    const double* t;
    const double* r;
    const double* beta;
    const double* bdot;
    const double* n_hat;
    int64_t n_pix;
    double omega0, d_omega;
    int64_t n_omega;
    double scale;   // q^2 dt^2 / (16 pi^3 eps0 c0)
    double* S;
};

__device__ __forceinline__ double mod2pi(double x) {
    constexpr double two_pi = 2.0 * kPi;
    constexpr double inv_two_pi = 1.0 / (2.0 * kPi);
    return x - two_pi * floor(x * inv_two_pi);
}

// exp(j (base + a * step)) with base, step in [0, 2 pi) given as FP32 hi + lo pairs
__device__ __forceinline__ float2 twiddle(float bh, float bl, float sh, float sl, float a) {
    constexpr float two_pi_hi = 6.28318548202514648f;              // fl(2 pi)
    constexpr float two_pi_lo = -1.7484555314695172e-7f;           // 2 pi - fl(2 pi)
    const float p = a * sh;
    const float e = fmaf(a, sh, -p);                                // exact product error
    const float hi = __fadd_rn(p, bh);
    const float bb = __fsub_rn(hi, p);
    const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(hi, bb)), __fsub_rn(bh, bb));
    const float lo = fmaf(a, sl, e) + bl + err;
    const float kq = rintf(hi * 0.159154943091895336f);
    const float ph = fmaf(-kq, two_pi_lo, fmaf(-kq, two_pi_hi, hi)) + lo;
    float s, c;
    sincosf(ph, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

__global__ void __launch_bounds__(kFdmThreads) fdm_kernel(FdmArgs p) {
    __shared__ float2 s_e1[kFdmChunk][32];   // exp(j (omega_base + 32 a d_omega) tau)
    __shared__ float2 s_e2[kFdmChunk][32];   // exp(j b d_omega tau)
    __shared__ float s_A[kFdmChunk][3];
    __shared__ float s_ph[kFdmChunk][6];     // (base, 32 d_omega, d_omega) phases, hi/lo
    const int64_t m = blockIdx.x;
    const int64_t w0 = (int64_t)blockIdx.y * kFdmFreq;
    const double nx = p.n_hat[3 * m], ny = p.n_hat[3 * m + 1], nz = p.n_hat[3 * m + 2];
    const double omega_base = p.omega0 + (double)w0 * p.d_omega;
    // compensated accumulators: [freq][component] real and imaginary, hi and lo
    float hr[kFdmPer][3], hi_[kFdmPer][3], lr[kFdmPer][3], li[kFdmPer][3];
    for (int f = 0; f < kFdmPer; ++f)
        for (int c = 0; c < 3; ++c) hr[f][c] = hi_[f][c] = lr[f][c] = li[f][c] = 0.0f;
    const int64_t total = p.n_e * p.ns1;
    for (int64_t s0 = 0; s0 < total; s0 += kFdmChunk) {
        const int ns = (int)min((int64_t)kFdmChunk, total - s0);
        __syncthreads();
        if (threadIdx.x < ns) {   // FP64 per sample: tau, A, reduced phases
            const int s = threadIdx.x;
            const int64_t g = s0 + s;
            const int64_t k = g / p.ns1, i = g - k * p.ns1;
            const double* x = p.r + 3 * g;
            const double tt = p.t_per_e ? p.t[g] : p.t[i];
            const double tau = tt - ((nx * x[0] + ny * x[1]) + nz * x[2]) * kInvC0;
            const double ph[3] = {mod2pi(omega_base * tau), mod2pi(32.0 * p.d_omega * tau),
                                  mod2pi(p.d_omega * tau)};
            for (int c = 0; c < 3; ++c) {
                const float h = (float)ph[c];
                s_ph[s][2 * c] = h;
                s_ph[s][2 * c + 1] = (float)(ph[c] - (double)h);
            }
            const double* b = p.beta + 3 * g;
            const double* a = p.bdot + 3 * g;
            const double D = 1.0 - ((nx * b[0] + ny * b[1]) + nz * b[2]);
            const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
            double A0 = 0.0, A1 = 0.0, A2 = 0.0;
            if (D > 0.0 && bb < 1.0) {
                const double m0 = nx - b[0], m1 = ny - b[1], m2 = nz - b[2];
                const double i0 = m1 * a[2] - m2 * a[1];
                const double i1 = m2 * a[0] - m0 * a[2];
                const double i2 = m0 * a[1] - m1 * a[0];
                const double iD2 = 1.0 / (D * D);
                A0 = (ny * i2 - nz * i1) * iD2;
                A1 = (nz * i0 - nx * i2) * iD2;
                A2 = (nx * i1 - ny * i0) * iD2;
            }
            s_A[s][0] = (float)A0;
            s_A[s][1] = (float)A1;
            s_A[s][2] = (float)A2;
        }
        __syncthreads();
        for (int job = threadIdx.x; job < ns * 64; job += kFdmThreads) {
            const int s = job / 64, which = job % 64;
            const float* ph = s_ph[s];
            if (which < 32)
                s_e1[s][which] = twiddle(ph[0], ph[1], ph[2], ph[3], (float)which);
            else
                s_e2[s][which - 32] = twiddle(0.0f, 0.0f, ph[4], ph[5], (float)(which - 32));
        }
        __syncthreads();
        float pr[kFdmPer][3], pi[kFdmPer][3];
        for (int f = 0; f < kFdmPer; ++f)
            for (int c = 0; c < 3; ++c) pr[f][c] = pi[f][c] = 0.0f;
        for (int s = 0; s < ns; ++s) {
            const float A0 = s_A[s][0], A1 = s_A[s][1], A2 = s_A[s][2];
#pragma unroll
            for (int f = 0; f < kFdmPer; ++f) {
                const int w = threadIdx.x + f * kFdmThreads;
                const float2 tw = cmulf(s_e1[s][w >> 5], s_e2[s][w & 31]);
                pr[f][0] = fmaf(A0, tw.x, pr[f][0]);
                pi[f][0] = fmaf(A0, tw.y, pi[f][0]);
                pr[f][1] = fmaf(A1, tw.x, pr[f][1]);
                pi[f][1] = fmaf(A1, tw.y, pi[f][1]);
                pr[f][2] = fmaf(A2, tw.x, pr[f][2]);
                pi[f][2] = fmaf(A2, tw.y, pi[f][2]);
            }
        }
        for (int f = 0; f < kFdmPer; ++f)
            for (int c = 0; c < 3; ++c) {
                two_sum_add(hr[f][c], lr[f][c], pr[f][c]);
                two_sum_add(hi_[f][c], li[f][c], pi[f][c]);
            }
    }
    for (int f = 0; f < kFdmPer; ++f) {
        const int64_t w = w0 + threadIdx.x + f * kFdmThreads;
        if (w >= p.n_omega) continue;
        double sum = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double re = (double)hr[f][c] + (double)lr[f][c];
            const double im = (double)hi_[f][c] + (double)li[f][c];
            sum += re * re + im * im;
        }
        p.S[m * p.n_omega + w] = p.scale * sum;
    }
}

}  // namespace
}  // namespace lw

using namespace lw;

extern "C" int lw_spectrum_fdm(const lw_traj* traj, const lw_detector* det, double omega0,
                               double d_omega, int64_t n_omega, double dt, double q,
                               double* spectrum, void* stream) {
    if (!traj || !det || !spectrum || !det->n_hat || det->n_pix < 1 || n_omega < 1)
        return LW_EINVAL;
    if (!(traj->sections & LW_SECTION_FP64) || !traj->t || !traj->r) return LW_EINVAL;
    if (!isfinite(omega0) || !isfinite(d_omega) || !(dt > 0.0) || !isfinite(q)) return LW_EINVAL;
    if (det->n_pix > 2147483647LL || (n_omega + kFdmFreq - 1) / kFdmFreq > 65535)
        return LW_EUNSUPPORTED;
    FdmArgs a{};
    a.n_e = traj->n_e;
    a.ns1 = traj->n_s + 1;
    a.t_per_e = traj->t_per_electron;
    a.t = traj->t;
    a.r = traj->r;
    a.beta = traj->beta;
    a.bdot = traj->beta_dot;
    a.n_hat = det->n_hat;
    a.n_pix = det->n_pix;
    a.omega0 = omega0;
    a.d_omega = d_omega;
    a.n_omega = n_omega;
    a.scale = q * q * dt * dt / (16.0 * kPi * kPi * kPi * kEps0 * kC0);
    a.S = spectrum;
    dim3 g((unsigned)det->n_pix, (unsigned)((n_omega + kFdmFreq - 1) / kFdmFreq));
    fdm_kernel<<<g, kFdmThreads, 0, as_stream(stream)>>>(a);
    return launch_status();
}
