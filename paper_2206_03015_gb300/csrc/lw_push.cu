// Boris pusher on the GPU (FP64), the trajectory update of Algorithm 2 ("update
// trajectory" in the step loop), for the in-situ form of the time-domain path:
// trajectories are produced one block of steps at a time and deposited at once,
// so only the current block is ever stored.  The same step, carried out on
// forward-mode derivative numbers, gives the gradient of a loss of the samples
// with respect to the initial momenta and the laser's a0 and waist.
//
// Laser: lowest-order paraxial Gaussian beam polarised along x, propagating
// along -z, focused at z = 0 and peaking there at t = 0:
//   E_x = E0 (w0/w) exp(-rho^2/w^2) exp(-(t + z/c)^2/(2 sigma^2))
//         cos(omega (t + z/c) + k rho^2 zeta/(2 (zeta^2 + zR^2)) - atan(zeta/zR)),
//   B_y = -E_x/c0,  zeta = -z,  w = w0 sqrt(1 + zeta^2/zR^2),  zR = pi w0^2/lam,
//   E0 = a0 m c0 omega / e,  sigma = FWHM_intensity / (2 sqrt(ln 2)).
// Step: drift half a step, Boris kick (half electric, magnetic rotation, half
// electric) with the fields at the midpoint, drift half a step; samples hold
// (t, r, beta, beta_dot) with beta_dot the Lorentz-force derivative
//   beta_dot = q/(m gamma c0) [E + c0 beta x B - beta (beta . E)].
#include <math.h>

#include "lw_internal.cuh"

namespace lw {
namespace {

constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;

using ::atan;
using ::cos;
using ::exp;
using ::sqrt;

// Forward-mode derivative numbers: a value and its derivatives along N directions.
template <int N>
struct Dual {
    double v;
    double d[N];
};
template <int N>
__device__ __forceinline__ Dual<N> mk(double v) {
    Dual<N> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = 0.0;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) {
    Dual<N> r = a;
    r.v = a.v + b;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(double a, const Dual<N>& b) { return b + a; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) { return a + (-b); }
template <int N>
__device__ __forceinline__ Dual<N> operator-(double a, const Dual<N>& b) { return (-b) + a; }
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
    Dual<N> r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N>
__device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) { return mk<N>(a) / b; }
template <int N>
__device__ __forceinline__ Dual<N> sqrt(const Dual<N>& a) {
    Dual<N> r;
    r.v = sqrt(a.v);
    const double h = 0.5 / r.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * h;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> exp(const Dual<N>& a) {
    Dual<N> r;
    r.v = exp(a.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * r.v;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> cos(const Dual<N>& a) {
    Dual<N> r;
    double sn, cs;
    sincos(a.v, &sn, &cs);
    r.v = cs;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i] * sn;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> atan(const Dual<N>& a) {
    Dual<N> r;
    r.v = atan(a.v);
    const double h = 1.0 / (1.0 + a.v * a.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * h;
    return r;
}

// Laser constants (T = double, or Dual when derivatives along a0 and w0 are carried).
template <typename T>
struct LaserT {
    double omega, k, sigma;
    T E0, zR, w0;
};
using Laser = LaserT<double>;

template <typename T>
__device__ __forceinline__ void fields(const LaserT<T>& L, const T& x, const T& y, const T& z,
                                       double t, T& Ex, T& By) {
    const T zeta = -z;
    const T w = L.w0 * sqrt(1.0 + (zeta / L.zR) * (zeta / L.zR));
    const T rho2 = x * x + y * y;
    const T xi = t + z * kInvC0;
    const T env = exp(-rho2 / (w * w)) * exp(-(xi * xi) / (2.0 * L.sigma * L.sigma));
    const T phase =
        L.omega * xi + L.k * rho2 * zeta / (2.0 * (zeta * zeta + L.zR * L.zR)) - atan(zeta / L.zR);
    Ex = L.E0 * (L.w0 / w) * env * cos(phase);
    By = -Ex * kInvC0;
}

// The sample at (r, u): beta = u / gamma and the Lorentz-force beta_dot.
template <typename T>
__device__ __forceinline__ void sample(const LaserT<T>& L, double qm, const T r[3], const T u[3],
                                       double t, T b[3], T a[3]) {
    const T gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    b[0] = u[0] / gam;
    b[1] = u[1] / gam;
    b[2] = u[2] / gam;
    T Ex, By;
    fields(L, r[0], r[1], r[2], t, Ex, By);
    // E = (Ex, 0, 0), B = (0, By, 0): beta x B = (-b_z By, 0, b_x By)
    const T bE = b[0] * Ex;
    const T f = qm / (gam * kC0);
    a[0] = f * (Ex + kC0 * (-b[2] * By) - b[0] * bE);
    a[1] = f * (-b[1] * bE);
    a[2] = f * (kC0 * (b[0] * By) - b[2] * bE);
}

// One Boris step from time ti: drift dt/2, kick with the fields at the midpoint, drift.
template <typename T>
__device__ __forceinline__ void boris_step(const LaserT<T>& L, double qm, double dt, double ti,
                                           T x[3], T v[3]) {
    const double eps = qm * dt / (2.0 * kC0);
    T gam = sqrt(1.0 + v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const T rh[3] = {x[0] + 0.5 * dt * kC0 * v[0] / gam, x[1] + 0.5 * dt * kC0 * v[1] / gam,
                     x[2] + 0.5 * dt * kC0 * v[2] / gam};
    T Ex, By;
    fields(L, rh[0], rh[1], rh[2], ti + 0.5 * dt, Ex, By);
    const T um[3] = {v[0] + eps * Ex, v[1], v[2]};
    const T gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    const T tv = qm * dt / (2.0 * gm) * By;   // t vector = (0, tv, 0)
    // u' = um + um x t ; s = 2 t / (1 + t^2) ; u+ = um + u' x s
    const T up[3] = {um[0] - um[2] * tv, um[1], um[2] + um[0] * tv};
    const T sv = 2.0 * tv / (1.0 + tv * tv);
    v[0] = um[0] - up[2] * sv + eps * Ex;
    v[1] = um[1];
    v[2] = um[2] + up[0] * sv;
    gam = sqrt(1.0 + v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    x[0] = rh[0] + 0.5 * dt * kC0 * v[0] / gam;
    x[1] = rh[1] + 0.5 * dt * kC0 * v[1] / gam;
    x[2] = rh[2] + 0.5 * dt * kC0 * v[2] / gam;
}

__device__ __forceinline__ void store_sample(const Laser& L, double qm, const double r[3],
                                             const double u[3], double t, double* ro,
                                             double* bo, double* ao) {
    double b[3], a[3];
    sample(L, qm, r, u, t, b, a);
    for (int c = 0; c < 3; ++c) {
        ro[c] = r[c];
        bo[c] = b[c];
        ao[c] = a[c];
    }
}

__global__ void push_kernel(double* __restrict__ r, double* __restrict__ u, int64_t n_e,
                            double t0, double dt, int64_t step0, int n_steps, Laser L, double qm,
                            double* __restrict__ ro, double* __restrict__ bo,
                            double* __restrict__ ao) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_e;
         k += (int64_t)gridDim.x * blockDim.x) {
        double x[3] = {r[3 * k], r[3 * k + 1], r[3 * k + 2]};
        double v[3] = {u[3 * k], u[3 * k + 1], u[3 * k + 2]};
        const int64_t base = k * (int64_t)(n_steps + 1);
        store_sample(L, qm, x, v, t0 + dt * (double)step0, ro + 3 * base, bo + 3 * base,
                     ao + 3 * base);
        for (int s = 0; s < n_steps; ++s) {
            boris_step(L, qm, dt, t0 + dt * (double)(step0 + s), x, v);
            const int64_t o = 3 * (base + s + 1);
            store_sample(L, qm, x, v, t0 + dt * (double)(step0 + s + 1), ro + o, bo + o, ao + o);
        }
        r[3 * k] = x[0];
        r[3 * k + 1] = x[1];
        r[3 * k + 2] = x[2];
        u[3 * k] = v[0];
        u[3 * k + 1] = v[1];
        u[3 * k + 2] = v[2];
    }
}

// Gradient of a loss L(samples) with respect to each electron's initial momentum u0 and
// the laser's a0 and w0, by forward-mode differentiation of the push: one thread per
// (electron, direction) pushes the electron again carrying the derivative of its state
// along one of u0_x, u0_y, u0_z, a0 and w0 (Dual<1>) and contracts each sample's
// derivative with dL/d(r, beta, beta_dot) of that sample.  Five threads per electron
// rather than one thread with all five directions: the push is a sequential FP64 chain
// per electron, and GB300's FP64 rate per SM sub-partition makes a single warp's
// instructions slow, so the work is spread over five times as many warps.  Per-electron
// a0 and w0 parts are added to dL_dlaser with FP64 atomics.
constexpr int kTan = 5;
__global__ void push_tangent_kernel(const double* __restrict__ r0, const double* __restrict__ u0,
                                    int64_t n_e, double t0, double dt, int n_steps, Laser L0,
                                    double e0_per_a0, double zr_per_w0, double qm,
                                    const double* __restrict__ g_r, const double* __restrict__ g_b,
                                    const double* __restrict__ g_a, double* __restrict__ dL_du0,
                                    double* __restrict__ dL_dlaser) {
    using D = Dual<1>;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_e * kTan;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / kTan;
        const int dir = (int)(t - k * kTan);   // 0..2: u0 components, 3: a0, 4: w0
        LaserT<D> L;
        L.omega = L0.omega;
        L.k = L0.k;
        L.sigma = L0.sigma;
        L.E0 = D{L0.E0, {dir == 3 ? e0_per_a0 : 0.0}};
        L.zR = D{L0.zR, {dir == 4 ? zr_per_w0 : 0.0}};
        L.w0 = D{L0.w0, {dir == 4 ? 1.0 : 0.0}};
        D x[3], v[3];
        for (int c = 0; c < 3; ++c) {
            x[c] = mk<1>(r0[3 * k + c]);
            v[c] = mk<1>(u0[3 * k + c]);
            v[c].d[0] = dir == c ? 1.0 : 0.0;
        }
        double acc = 0.0;
        const int64_t base = k * (int64_t)(n_steps + 1);
        auto contract = [&](int64_t o, double tt) {
            D b[3], a[3];
            sample(L, qm, x, v, tt, b, a);
            for (int c = 0; c < 3; ++c)
                acc = fma(g_r[3 * o + c], x[c].d[0],
                          fma(g_b[3 * o + c], b[c].d[0], fma(g_a[3 * o + c], a[c].d[0], acc)));
        };
        contract(base, t0);
        for (int s = 0; s < n_steps; ++s) {
            boris_step(L, qm, dt, t0 + dt * (double)s, x, v);
            contract(base + s + 1, t0 + dt * (double)(s + 1));
        }
        if (dir < 3)
            dL_du0[3 * k + dir] += acc;
        else
            atomicAdd(dL_dlaser + (dir - 3), acc);
    }
}

__global__ void times_kernel(double* t_out, double t0, double dt, int64_t step0, int n_steps) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= n_steps; s += gridDim.x * blockDim.x)
        t_out[s] = t0 + dt * (double)(step0 + s);
}

}  // namespace
}  // namespace lw

using namespace lw;

extern "C" int lw_boris_push(double* r, double* u, int64_t n_e, double t0, double dt,
                             int64_t step0, int32_t n_steps, const lw_laser* laser,
                             double charge, double mass,
                             double* t_out, double* r_out, double* beta_out, double* bdot_out,
                             void* stream) {
    if (!r || !u || !laser || !t_out || !r_out || !beta_out || !bdot_out) return LW_EINVAL;
    if (n_e < 1 || n_steps < 1 || step0 < 0 || step0 > (int64_t(1) << 52) || !(dt > 0.0) ||
        !isfinite(t0) || !(mass > 0.0))
        return LW_EINVAL;
    if (!(laser->lam > 0.0) || !(laser->w0 > 0.0) || !(laser->fwhm > 0.0)) return LW_EINVAL;
    Laser L;
    L.omega = 2.0 * kPi * kC0 / laser->lam;
    L.k = L.omega * kInvC0;
    L.sigma = laser->fwhm / (2.0 * sqrt(log(2.0)));
    L.E0 = laser->a0 * kMe * kC0 * L.omega / kQe;
    L.zR = kPi * laser->w0 * laser->w0 / laser->lam;
    L.w0 = laser->w0;
    cudaStream_t st = as_stream(stream);
    times_kernel<<<(n_steps + 256) / 256, 256, 0, st>>>(t_out, t0, dt, step0, n_steps);
    if (launch_status() != LW_OK) return LW_ECUDA;
    // one warp per block: a push is a sequential FP64 chain per electron, so the few
    // warps of a small bunch are spread over as many SMs as possible
    const int threads = 32;
    const int blocks = (int)((n_e + threads - 1) / threads);
    push_kernel<<<blocks, threads, 0, st>>>(r, u, n_e, t0, dt, step0, n_steps, L, charge / mass, r_out,
                                            beta_out, bdot_out);
    return launch_status();
}

extern "C" int lw_boris_push_grad(const double* r0, const double* u0, int64_t n_e, double t0,
                                  double dt, int32_t n_steps, const lw_laser* laser,
                                  double charge, double mass, const double* dL_dr,
                                  const double* dL_dbeta, const double* dL_dbeta_dot,
                                  double* dL_du0, double* dL_dlaser, void* stream) {
    if (!r0 || !u0 || !laser || !dL_dr || !dL_dbeta || !dL_dbeta_dot || !dL_du0 || !dL_dlaser)
        return LW_EINVAL;
    if (n_e < 1 || n_steps < 1 || !(dt > 0.0) || !isfinite(t0) || !(mass > 0.0))
        return LW_EINVAL;
    if (!(laser->lam > 0.0) || !(laser->w0 > 0.0) || !(laser->fwhm > 0.0)) return LW_EINVAL;
    Laser L;
    L.omega = 2.0 * kPi * kC0 / laser->lam;
    L.k = L.omega * kInvC0;
    L.sigma = laser->fwhm / (2.0 * sqrt(log(2.0)));
    const double e0_per_a0 = kMe * kC0 * L.omega / kQe;
    L.E0 = laser->a0 * e0_per_a0;
    L.zR = kPi * laser->w0 * laser->w0 / laser->lam;
    L.w0 = laser->w0;
    const double zr_per_w0 = 2.0 * kPi * laser->w0 / laser->lam;
    // one warp per block: the warps spread over the SMs' sub-partitions
    const int threads = 32;
    const int64_t work = n_e * kTan;
    const int blocks = (int)std::min<int64_t>((work + threads - 1) / threads, 1 << 20);
    push_tangent_kernel<<<blocks, threads, 0, as_stream(stream)>>>(
        r0, u0, n_e, t0, dt, n_steps, L, e0_per_a0, zr_per_w0, charge / mass, dL_dr, dL_dbeta,
        dL_dbeta_dot, dL_du0, dL_dlaser);
    return launch_status();
}
