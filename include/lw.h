/*
 * lw.h -- C ABI of liblw.so, a GB300 (sm_103a) implementation of the
 * time-domain Lienard-Wiechert radiation method of Kan, Kaertner, Le Borne,
 * Ruprecht, Zemke, "Parallel Computation of Inverse Compton Scattering
 * Radiation Spectra based on Lienard-Wiechert Potentials" (arXiv 2206.03015).
 *
 * Pipeline (one call per stage, all asynchronous on the caller's stream):
 *   lw_trajectories_upload  stored trajectories -> device layout       (Sec. 4.2, "Beam")
 *   lw_grid_bounds          t_u^min, t_u^max of the observer grid       (Eqs. tu_min, tu_max)
 *   lw_deposit_time_domain  advanced times + LW far field + linear
 *                           interpolation onto the uniform grid         (Eqs. far_adv, far_efield,
 *                                                                         Algorithm 2)
 *   lw_spectrum             per-pixel FFT -> d2I/domega dOmega          (Eqs. efield_xfrom,
 *                                                                         const_phase_drop)
 *   lw_spectrum_grad        adjoint of deposit + spectrum
 *
 * Conventions shared by every entry point:
 *  - The caller owns all memory.  The library allocates no device or host
 *    memory; every buffer (including workspaces, sized by a query call) is
 *    passed in.  Pointers marked "device" must be device memory or memory the
 *    GPU can address (pinned host memory is accepted wherever a kernel reads
 *    an input once).
 *  - Every call enqueues work on `stream` (a cudaStream_t passed as void*;
 *    NULL = legacy default stream) and returns without synchronising.
 *  - Host-detectable argument errors are returned synchronously as a negative
 *    lw_status and enqueue nothing.  LW_ECUDA reports a failed launch.
 *  - Data-dependent conditions found by the kernels are OR-ed into the
 *    caller's device status word (int32, LW_ST_* bits); read it after the
 *    stream has been synchronised.  Kernels never trap.
 *  - Calls on different streams may run concurrently as long as they do not
 *    write the same buffers.  Two entry points hold global state and must be
 *    serialised (one stream, or host-side ordering): lw_batch_deposit copies
 *    the batch's arguments into a constant-memory table of the library, and
 *    lw_spectrum_static uses one file-scope device scratch array.  Every other
 *    call keeps its state in caller buffers.
 *
 * Units are SI: t [s], r [m], beta [1], beta_dot [1/s].  Field records hold
 * the LW far field divided by the constant q/(4 pi eps0 c0 R), i.e.
 *   F = n x ((n - beta) x beta_dot) / (1 - n.beta)^3       [1/s].
 */
#ifndef LW_H
#define LW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LW_OK = 0,
    LW_EINVAL = -1,        /* invalid argument (null pointer, bad size, bad flag) */
    LW_ESIZE = -2,         /* workspace smaller than required */
    LW_ECUDA = -3,         /* a CUDA launch or runtime call failed */
    LW_EUNSUPPORTED = -4,  /* valid but unsupported (e.g. n_bins not a power of two for the FFT) */
    LW_ETIMEOUT = -5       /* a bounded device-side wait ran out */
} lw_status;

/* Arithmetic of a call. */
enum {
    LW_FP64 = 0,   /* everything in FP64; advanced times and bin indices follow the op order
                      documented at lw_deposit_time_domain (bit-identical to a plain C loop
                      compiled without FMA contraction) */
    LW_MIXED = 1,  /* FP64-exact bin coordinates carried as integer + FP32 fraction, FP32
                      field and interpolation, contributions added to an FP64 record by
                      the L2 (red.global.add.f64), FP32 FFT */
    LW_MIXED_KAHAN = 2, /* as LW_MIXED but the record is a compensated FP32 pair
                           (sum, compensation): atomic add with return + two-sum */
    LW_MIXED_F32 = 3,   /* as LW_MIXED but the record is FP32, added to by the L2
                           (red.global.add.f32): half the record's bytes and faster
                           atomics; each bin's sum carries FP32 rounding, so it suits
                           records whose bins collect few contributions each (about 3 for
                           a 10,000-electron bunch on 64 x 64 pixels and 65,536 bins; the
                           error grows with the count) */
    LW_MIXED_F32X4 = 4  /* as LW_MIXED_F32 with the three components of a grid point
                           stored together as (x, y, z, 0) and added by one vector
                           reduction (red.global.add.v4.f32): one L2 operation per grid
                           point instead of three, for a third more record bytes */
};

/* Field terms (bit mask) of lw_deposit_time_domain. */
enum {
    LW_FIELD_ACCEL = 1,     /* acceleration (radiation) field, Eq. far_efield */
    LW_FIELD_VELOCITY = 2   /* far-field velocity field c0 (n-beta)(1-beta^2)/((1-n.beta)^3 R) */
};

/* Device status bits (OR-ed into the caller's int32 status word). */
enum {
    LW_ST_BETA = 1,        /* |beta| >= 1 at a sample (its field is taken as 0) */
    LW_ST_NONFINITE = 2,   /* non-finite input, or a bin coordinate beyond +-2^62 */
    LW_ST_TIME = 4,        /* lab time not strictly increasing along a trajectory */
    LW_ST_CLIP = 8,        /* grid points outside [0, n_bins) were skipped */
    LW_ST_TA_ORDER = 16,   /* advanced time not increasing between two samples (LW_FP64) */
    LW_ST_STEP = 32,       /* two consecutive samples at least c0 (t_i - t_(i-1)) apart
                              (checked by uploads with the FP64 section): the advanced time
                              may decrease for some direction */
    LW_ST_TIMEOUT = 64,    /* a kernel's bounded wait for its staged input ran out (the
                              record is incomplete) */
    LW_ST_PRECISION = 128  /* mixed deposits: the estimated FP32 error of some tile's
                              contributions (interpolation weights from FP32 coordinates,
                              FP32 Doppler factors) exceeds 2^-11 of their root mean square.
                              The estimate is conservative: on the cases it was calibrated on,
                              every mixed spectrum more than 1e-4 (relative L2) from the FP64
                              one raised it, and none within 2.5e-5 of it did.  Typical
                              causes: fields that change by a large fraction across a step
                              (an observer inside a synchrotron cone sampled coarsely), or
                              velocities far from the z axis.  LW_FP64 has no such limit */
};

/* Which device sections lw_trajectories_upload builds (bit mask). */
enum { LW_SECTION_FP64 = 1, LW_SECTION_MIXED = 2 };

/* Stored trajectories as given by the caller (all float64, C order).
 *   t         [n_s+1] shared by all electrons, or [n_e][n_s+1] if t_per_electron
 *   r         [n_e][n_s+1][3]   position
 *   beta      [n_e][n_s+1][3]   velocity / c0
 *   beta_dot  [n_e][n_s+1][3]   d beta / dt
 * Pointers are device or pinned-host memory; they are read once by
 * lw_trajectories_upload and not referenced afterwards. */
typedef struct {
    int64_t n_e;
    int64_t n_s;
    const double* t;
    int32_t t_per_electron;
    const double* r;
    const double* beta;
    const double* beta_dot;
} lw_traj_in;

/* Device view of uploaded trajectories (plain old data; all pointers point
 * into the workspace passed to lw_trajectories_upload, which the caller must
 * keep alive and unmodified while the view is used). */
typedef struct {
    int64_t n_e, n_s;
    int32_t t_per_electron;
    int32_t sections;       /* LW_SECTION_* bits that were built */
    int32_t block;          /* samples per anchoring block of the mixed section */
    int32_t n_blocks;       /* ceil((n_s+1) / block) */
    const double* t;        /* FP64 section: copies of the inputs (same layouts) */
    const double* r;
    const double* beta;
    const double* beta_dot;
    const void* scan;       /* MIXED: float4 [n_e][n_s+1] (tau - tau_b, r - r_b) per sample,
                               tau = t - z/c0, _b = first sample of the sample's block */
    const void* field;      /* MIXED: float4 [n_e][n_s+1] (beta_x, beta_y, beta_dot_x,
                               beta_dot_y), then float2 [n_e][n_s+1] (1 - beta_z,
                               beta_dot_z) */
    const double* anchor;   /* MIXED: 32-byte records [n_e][n_blocks]: tau_b (double), then
                               x_b, y_b, z_b as float pairs (hi, lo), hi = fl32(x),
                               lo = fl32(x - hi) */
    const double* ends;     /* always: double [n_e][2][4] = (t, x, y, z) of the first and
                               the last sample of each electron */
    const int32_t* input_status; /* device int32: LW_ST_* found while uploading */
    const int32_t* order;   /* always: int32 [n_e] electron indices in increasing light-front
                               time tau = t - z/c0 of the first sample (bucketed: the order
                               within 1/4096 of the range is unspecified); the deposits
                               visit electrons in this order */
} lw_traj;

/* Far-field detector: n_pix unit directions n_hat [n_pix][3] (float64, device) on a
 * sphere of radius R (used only by LW_FIELD_VELOCITY). */
typedef struct {
    int64_t n_pix;
    const double* n_hat;
    double R;
} lw_detector;

/* Uniform observer grid t_j = t_min + j * dt_u, j = 0 .. n_bins-1. */
typedef struct {
    double t_min;
    double dt_u;
    int64_t n_bins;
} lw_grid;

/* Copy stored trajectories into the device layout of `ws` (Sec. 4.2 "Beam":
 * position, velocity and acceleration per particle; here for every step).
 *   sections   LW_SECTION_FP64 and/or LW_SECTION_MIXED
 *   block      samples per anchoring block of the mixed section (16..1024,
 *              power of two; 0 = default 512)
 *   ws         device workspace, 256-byte aligned; NULL = size query
 *   ws_bytes   in: size of ws; out: bytes required
 *   out        filled with the device view on success
 * Checks every sample (finite values, |beta| < 1, strictly increasing t) and
 * records LW_ST_* bits in the workspace for later deposits.
 * The mixed deposit relies on the advanced time increasing along each
 * trajectory for every direction, which holds whenever consecutive samples
 * are less than c0 (t_i - t_{i-1}) apart, i.e. for any subluminal motion
 * sampled in time order; the FP64 deposit makes no such assumption.
 * Errors: LW_EINVAL (null in/out pointers, n_e < 1, n_s < 1, bad sections or
 * block), LW_EUNSUPPORTED (n_s >= 2^30 or n_e >= 2^31), LW_ESIZE (ws too small; *ws_bytes =
 * required), LW_ECUDA. */
int lw_trajectories_upload(const lw_traj_in* in, int32_t sections, int32_t block, void* ws,
                           size_t* ws_bytes, lw_traj* out, void* stream);

/* Observer-grid bounds, Eqs. (tu_min) and (tu_max):
 *   bounds[0] = min over (k, m) of t_a^{k,m}(t_start),
 *   bounds[1] = max over (k, m) of t_a^{k,m}(t_end),
 * with the FP64 advanced time of lw_deposit_time_domain (constant |x|/c0
 * dropped).  bounds: device double[2].  Works with either section.
 * Errors: LW_EINVAL, LW_ECUDA. */
int lw_grid_bounds(const lw_traj* traj, const lw_detector* det, double* bounds, void* stream);

/* Time-domain method, Algorithm 2, for every pixel of the detector.
 * For each electron k, pixel m and step i the advanced time (Eq. far_adv,
 * without the constant |x|/c0) and bin coordinate are
 *   t_a = t_i - (n . r_i) * (1/c0),   u = (t_a - t_min) * (1/dt_u),
 * and every grid point j with floor(u_{i-1}) < j <= floor(u_i) (the
 * half-open interval (t_b, t_a] of Algorithm 2) receives
 *   F_{i-1} (t_a - t_j)/(t_a - t_b) + F_i (t_j - t_b)/(t_a - t_b).
 * LW_FP64 evaluates n.r as ((n_x x + n_y y) + n_z z) and every operation
 * above in that order with single IEEE roundings.  LW_MIXED evaluates u as
 * an integer plus an FP32 fraction anchored once per block in
 * double-FP32 arithmetic (the first and last samples' bins in FP64, as in
 * LW_FP64), the field in FP32 from the stable form
 *   D = (1 - n_z) + n_z (1 - beta_z) - n_perp . beta_perp,
 *   F = [(n - beta)(n . beta_dot) - D beta_dot] / D^3,
 * and accumulates into FP64 (LW_MIXED), compensated FP32 pairs (LW_MIXED_KAHAN)
 * or FP32 (LW_MIXED_F32, and LW_MIXED_F32X4 with the components interleaved).
 *   precision    LW_FP64, LW_MIXED, LW_MIXED_KAHAN, LW_MIXED_F32 or LW_MIXED_F32X4
 *                (the matching section must exist)
 *   field_flags  LW_FIELD_* mask (non-zero)
 *   record       device; LW_FP64 and LW_MIXED: double [n_pix][3][n_bins];
 *                LW_MIXED_KAHAN: float2 [n_pix][3][n_bins] = (sum, compensation),
 *                value = sum + compensation; LW_MIXED_F32: float [n_pix][3][n_bins];
 *                LW_MIXED_F32X4: float4 [n_pix][n_bins] = (x, y, z, 0)
 *   accumulate   0: the record is zeroed first; 1: add to its contents
 *   status       device int32, OR-ed with LW_ST_* bits (may be NULL)
 * Grid points outside [0, n_bins) are skipped (LW_ST_CLIP).
 * Errors: LW_EINVAL (null pointers, n_bins < 1, dt_u <= 0 or non-finite,
 * missing section, zero flags), LW_ECUDA. */
int lw_deposit_time_domain(const lw_traj* traj, const lw_detector* det, const lw_grid* grid,
                           int32_t precision, uint32_t field_flags, void* record,
                           int32_t accumulate, int32_t* status, void* stream);

/* Spectral-angular distribution from the records (Eq. efield_xfrom and the
 * prefactor of Eq. const_phase_drop):
 *   S[m][l] = q^2 dt_u^2 / (16 pi^3 eps0 c0) * sum_c |X_{m,c}(l)|^2,
 *   X_{m,c}(l) = sum_j rec[m][c][j] exp(+2 pi i j l / n_bins),  l = 0 .. n_bins/2,
 * at omega_l = 2 pi l / (n_bins dt_u), in J s / sr (per unit angular frequency).
 *   record    device, layout of lw_deposit_time_domain for `precision`
 *   n_pix     pixels in the record
 *   q         particle charge [C]
 *   spectrum  device; LW_FP64: double, the LW_MIXED* modes: float [n_pix][n_bins/2+1]
 *   X_save    device or NULL; receives X' = sqrt(K) dt_u X (so that S = sum_c |X'_c|^2),
 *             K = q^2/(16 pi^3 eps0 c0), as LW_FP64: double2, the LW_MIXED* modes: float2
 *             [n_pix][3][n_bins/2+1]
 *   ws        device scratch for the two-pass FFT (n_bins above 4096); NULL = query
 *   ws_bytes  in: size of ws; out: bytes required (0 when none is needed)
 * Errors: LW_EINVAL, LW_EUNSUPPORTED (n_bins not a power of two in
 * [2, 2^18]), LW_ESIZE, LW_ECUDA. */
int lw_spectrum(const void* record, int32_t precision, int64_t n_pix, const lw_grid* grid,
                double q, void* spectrum, void* X_save, void* ws, size_t* ws_bytes,
                void* stream);

/* Adjoint of lw_deposit_time_domain followed by lw_spectrum (reverse-mode
 * gradient of a loss L(S)).  Given g = dL/dS [n_pix][n_bins/2+1] (float64,
 * device) and X_save written by lw_spectrum with the same precision, adds to
 *   dL_dr, dL_dbeta, dL_dbeta_dot   float64 [n_e][n_s+1][3] (device, caller-zeroed)
 * the gradient of L with respect to every sample's position, velocity and
 * acceleration.  The record gradient is
 *   dL/drec_c[j] = 2 sqrt(K) dt_u Re(sum_l g_l conj(X'_c(l)) exp(+2 pi i j l/N))
 * (one complex FFT per two rows); the deposit is transposed as a gather over
 * the same half-open intervals of Algorithm 2, differentiating the
 * interpolation weights with respect to t_a and t_b, the advanced time
 * (Eq. far_adv) with respect to r and the acceleration field (Eq. far_efield)
 * with respect to beta and beta_dot.  L is piecewise smooth in the samples
 * (grid points entering or leaving an interval change its slope but not its
 * value); the result is the derivative on the current piece.
 *   precision    LW_FP64, or one of the LW_MIXED* modes (X_save then float2): bin
 *                coordinates in FP64 at every 64th sample and in FP32 relative to it
 *                in between, fields, weights and the chain rule in FP32 with the
 *                record gradient scaled by a power of two (FP32 range: fields up to
 *                ~1e30 /s, 1 - n.beta above ~1e-5); the FP64 section must exist in
 *                both cases
 *   field_flags  LW_FIELD_ACCEL
 *   q            particle charge [C] (as passed to lw_spectrum)
 *   ws           device scratch (NULL = size query): dL/drec, twiddles and,
 *                above 4096 bins, the four-step transform buffer
 * Errors: LW_EINVAL, LW_EUNSUPPORTED (other precision/flags, n_bins not a power
 * of two in [2, 2^18]), LW_ESIZE, LW_ECUDA. */
int lw_spectrum_grad(const lw_traj* traj, const lw_detector* det, const lw_grid* grid,
                     int32_t precision, uint32_t field_flags, const void* X_save,
                     const double* dL_dS, double q, double* dL_dr, double* dL_dbeta,
                     double* dL_dbeta_dot, void* ws, size_t* ws_bytes, void* stream);

/* Frequency-domain method, Eq. (inty_dft) / Algorithm 1 (the paper's comparison
 * method), on the uniform frequency grid omega_w = omega0 + w d_omega:
 *   S[m][w] = q^2 dt^2 / (16 pi^3 eps0 c0)
 *             |sum_k sum_{i=0}^{n_s} A_k(n_m, t_i) exp(j omega_w (t_i - n_m.r_ki/c0))|^2,
 *   A = n x ((n - beta) x beta_dot) / (1 - n.beta)^2,
 * with the same far-field phase time as lw_deposit_time_domain (|x|/c0 dropped)
 * and the rectangle rule of weight dt over all stored samples.  Phase times,
 * A and the phase reductions modulo 2 pi are FP64; twiddles and sums are
 * double-FP32 / compensated FP32.  Needs the FP64 section.
 *   spectrum  device float64 [n_pix][n_omega]
 * Errors: LW_EINVAL, LW_EUNSUPPORTED (too many frequencies for one launch), LW_ECUDA. */
int lw_spectrum_fdm(const lw_traj* traj, const lw_detector* det, double omega0, double d_omega,
                    int64_t n_omega, double dt, double q, double* spectrum, void* stream);

/* Laser of lw_boris_push: lowest-order paraxial Gaussian beam polarised along x,
 * propagating along -z, focused at z = 0 and peaking there at t = 0. */
typedef struct {
    double lam;    /* wavelength [m] */
    double a0;     /* normalised peak vector potential */
    double w0;     /* waist [m] */
    double fwhm;   /* intensity FWHM duration [s] */
} lw_laser;

/* Trajectory update of Algorithm 2 ("update trajectory", Boris method as in the
 * paper's trial simulation) for the in-situ form of the path: advances n_e
 * particles (r [n_e][3] in metres, u = gamma beta [n_e][3]; device, updated in
 * place) by n_steps steps of dt from time t0 + step0 dt in the Gaussian laser,
 * and writes the n_steps + 1 samples t_out [n_steps+1], r_out, beta_out, bdot_out
 * [n_e][n_steps+1][3] (device, FP64) -- the layout of lw_traj_in -- including the
 * starting state as sample 0, so consecutive calls overlap by one sample.
 * Sample s has the time t0 + dt (step0 + s) (FP64, that order of operations), so
 * pushing in blocks with a running step0 and one t0 gives bit-identical times and
 * trajectories to a single call.  step0 in [0, 2^52].
 * Step: drift dt/2, Boris kick with the fields at the midpoint, drift dt/2;
 * bdot = q/(m gamma c0) [E + c0 beta x B - beta (beta.E)] at each sample.
 * Errors: LW_EINVAL, LW_ECUDA. */
int lw_boris_push(double* r, double* u, int64_t n_e, double t0, double dt, int64_t step0,
                  int32_t n_steps, const lw_laser* laser, double charge, double mass,
                  double* t_out, double* r_out, double* beta_out, double* bdot_out,
                  void* stream);

/* Gradient through lw_boris_push (one call from step 0): given dL/d(sample) for every
 * sample of the trajectories that lw_boris_push(r0, u0, n_e, t0, dt, 0, n_steps, laser,
 * charge, mass, ...) writes -- dL_dr, dL_dbeta, dL_dbeta_dot [n_e][n_steps+1][3] (device,
 * float64; e.g. from lw_spectrum_grad) -- adds
 *   dL_du0     [n_e][3]  the gradient with respect to each electron's initial u = gamma beta
 *   dL_dlaser  [2]       the gradient with respect to the laser's a0 and w0 (summed over
 *                        the electrons with FP64 atomics)
 * (device, float64, caller-zeroed or accumulated).  Each electron is pushed again with
 * forward-mode derivatives of its state along u0_x, u0_y, u0_z, a0 and w0, the same
 * operations as lw_boris_push, and each sample's derivatives are contracted with its
 * dL/d(sample) (the chain rule through Eqs. far_adv / far_efield is in lw_spectrum_grad;
 * this is the "update trajectory" step of Algorithm 2 differentiated).  No trajectory
 * state is stored: memory is the inputs' and outputs'.
 * Errors: LW_EINVAL, LW_ECUDA. */
int lw_boris_push_grad(const double* r0, const double* u0, int64_t n_e, double t0, double dt,
                       int32_t n_steps, const lw_laser* laser, double charge, double mass,
                       const double* dL_dr, const double* dL_dbeta, const double* dL_dbeta_dot,
                       double* dL_du0, double* dL_dlaser, void* stream);

/* Several independent problems ("variants": own trajectories, detector, grid
 * and record) deposited by one persistent launch of the mixed-precision
 * deposit (LW_MIXED, LW_MIXED_KAHAN, LW_MIXED_F32 or LW_MIXED_F32X4).  The work is
 * cut into units of
 * (variant, 512-pixel tile, chunk of electrons) that resident CTAs take from a
 * list: variants largest first, each variant's chunks in arrival order (the
 * upload's electron order) with its tiles fastest, so variants of very
 * different sizes share the GPU and each keeps its record updates local.
 * Two calls:
 *   lw_batch_plan     checks the items, writes the per-variant arguments and the
 *                     work list into `ws` (NULL = size query) and fills `plan`;
 *                     it copies from host memory and returns after the copies.
 *   lw_batch_deposit  zeroes every record and launches the persistent kernel;
 *                     it only enqueues stream-ordered work, so it can be
 *                     repeated (and recorded in a CUDA graph) with the same plan.
 *                     The variants' arguments are copied into a constant-memory
 *                     table of the library before the launch: calls of
 *                     lw_batch_deposit must not overlap on the GPU (serialise them
 *                     on one stream).
 * e_chunk (electrons per unit) comes from the item, or is chosen so that the
 * batch splits into about eight units per resident CTA when it is 0.  Records
 * and results are those of lw_deposit_time_domain for each variant.
 * Errors: LW_EINVAL, LW_EUNSUPPORTED (LW_FP64, or more than 256 items), LW_ESIZE,
 * LW_ECUDA. */
typedef struct {
    const lw_traj* traj;        /* uploaded with the mixed section */
    const lw_detector* det;
    lw_grid grid;
    void* record;               /* layout of lw_deposit_time_domain for the precision */
    int32_t* status;            /* device int32 or NULL */
    int32_t e_chunk;            /* electrons per work unit, 0 = automatic */
} lw_batch_item;

typedef struct {
    void* ws;
    int32_t n_items, n_units, precision, smem_bytes;
    int32_t field_flags, reserved;
    int64_t offsets[3];
} lw_batch;

int lw_batch_plan(const lw_batch_item* items, int32_t n_items, int32_t precision,
                  uint32_t field_flags, void* ws, size_t* ws_bytes, lw_batch* plan,
                  void* stream);
int lw_batch_deposit(const lw_batch* plan, void* stream);

/* lw_spectrum without a caller-supplied workspace, for callers that must not
 * allocate device memory while they run -- for example a read-out or plug-in
 * process whose device memory budget is fixed at start-up, where a cudaMalloc
 * or cudaFree would also synchronise the whole device and stall unrelated
 * streams.  The paper has no counterpart; this is a deployment convenience.
 * Same arguments, results and errors as lw_spectrum, except that the scratch
 * is one fixed array of lw_spectrum_static_capacity() bytes (32 MiB) that
 * every GPU loading the library holds until the process exits:
 *  - transforms whose scratch would exceed it return LW_ESIZE (n_bins <= 4096
 *    needs only the twiddle table; above that the four-step buffer needs
 *    3 * ceil(n_pix/2) * n_bins complex values);
 *  - the first call on each device looks up the array's device address (with
 *    that device current); make that first call before any stream capture;
 *  - all calls share the array and nothing in it needs to start at zero, but
 *    calls that overlap on the GPU (other streams, other host threads) race
 *    on it: serialise them.
 * No device or host allocation is made by this call. */
int lw_spectrum_static(const void* record, int32_t precision, int64_t n_pix, const lw_grid* grid,
                       double q, void* spectrum, void* X_save, void* stream);
size_t lw_spectrum_static_capacity(void);

#ifdef __cplusplus
}
#endif

#endif /* LW_H */
