// Boris pusher on the GPU (FP64), the trajectory update of Algorithm 2 ("update
// trajectory" in the step loop), for the in-situ form of the time-domain path:
// trajectories are produced one block of steps at a time and deposited at once,
// so only the current block is ever stored.
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

struct Laser {
    double omega, k, sigma, E0, zR, w0;
};

__device__ __forceinline__ void fields(const Laser& L, double x, double y, double z, double t,
                                       double& Ex, double& By) {
    const double zeta = -z;
    const double w = L.w0 * sqrt(1.0 + (zeta / L.zR) * (zeta / L.zR));
    const double rho2 = x * x + y * y;
    const double xi = t + z * kInvC0;
    const double env = exp(-rho2 / (w * w)) * exp(-(xi * xi) / (2.0 * L.sigma * L.sigma));
    const double phase =
        L.omega * xi + L.k * rho2 * zeta / (2.0 * (zeta * zeta + L.zR * L.zR)) - atan(zeta / L.zR);
    Ex = L.E0 * (L.w0 / w) * env * cos(phase);
    By = -Ex * kInvC0;
}

__device__ __forceinline__ void store_sample(const Laser& L, double qm, const double r[3],
                                             const double u[3], double t, double* ro,
                                             double* bo, double* ao) {
    const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double b[3] = {u[0] / gam, u[1] / gam, u[2] / gam};
    double Ex, By;
    fields(L, r[0], r[1], r[2], t, Ex, By);
    // E = (Ex, 0, 0), B = (0, By, 0): beta x B = (-b_z By, 0, b_x By)
    const double bE = b[0] * Ex;
    const double f = qm / (gam * kC0);
    ro[0] = r[0];
    ro[1] = r[1];
    ro[2] = r[2];
    bo[0] = b[0];
    bo[1] = b[1];
    bo[2] = b[2];
    ao[0] = f * (Ex + kC0 * (-b[2] * By) - b[0] * bE);
    ao[1] = f * (-b[1] * bE);
    ao[2] = f * (kC0 * (b[0] * By) - b[2] * bE);
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
        const double eps = qm * dt / (2.0 * kC0);
        for (int s = 0; s < n_steps; ++s) {
            const double ti = t0 + dt * (double)(step0 + s);
            double gam = sqrt(1.0 + v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            const double rh[3] = {x[0] + 0.5 * dt * kC0 * v[0] / gam,
                                  x[1] + 0.5 * dt * kC0 * v[1] / gam,
                                  x[2] + 0.5 * dt * kC0 * v[2] / gam};
            double Ex, By;
            fields(L, rh[0], rh[1], rh[2], ti + 0.5 * dt, Ex, By);
            const double um[3] = {v[0] + eps * Ex, v[1], v[2]};
            const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
            const double tv = qm * dt / (2.0 * gm) * By;   // t vector = (0, tv, 0)
            // u' = um + um x t ; s = 2 t / (1 + t^2) ; u+ = um + u' x s
            const double up[3] = {um[0] - um[2] * tv, um[1], um[2] + um[0] * tv};
            const double sv = 2.0 * tv / (1.0 + tv * tv);
            v[0] = um[0] - up[2] * sv + eps * Ex;
            v[1] = um[1];
            v[2] = um[2] + up[0] * sv;
            gam = sqrt(1.0 + v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            x[0] = rh[0] + 0.5 * dt * kC0 * v[0] / gam;
            x[1] = rh[1] + 0.5 * dt * kC0 * v[1] / gam;
            x[2] = rh[2] + 0.5 * dt * kC0 * v[2] / gam;
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
    const int threads = 128;
    const int blocks = (int)((n_e + threads - 1) / threads);
    push_kernel<<<blocks, threads, 0, st>>>(r, u, n_e, t0, dt, step0, n_steps, L, charge / mass, r_out,
                                            beta_out, bdot_out);
    return launch_status();
}
