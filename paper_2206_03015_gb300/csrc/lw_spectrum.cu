// Per-pixel spectra from the time records (Eq. efield_xfrom with the
// prefactor of Eq. const_phase_drop):
//   S[m][l] = sum_c |X'_{m,c}(l)|^2,  X' = sqrt(K) dt_u X,  K = q^2/(16 pi^3 eps0 c0),
//   X_{m,c}(l) = sum_j rec[m][c][j] exp(+2 pi i j l / N),  l = 0..N/2.
//
// Two real rows are transformed together as one complex sequence
// z = a + i b; with Z = FFT(z):
//   A(l) = (Z_l + conj Z_{N-l}) / 2,   B(l) = (Z_l - conj Z_{N-l}) / (2i).
// A pixel pair (m0, m1) gives three sequences: (x0 + i y0), (x1 + i y1),
// (z0 + i z1).  Transforms run in shared memory as passes of up to four radix-2
// stages (lw_fft.cuh: each group pre-multiplied by twiddles from a table
// e^{+2 pi i t/N} built once per call, then constant-root stages):
//   N <= 4096   one CTA per pixel pair, all three sequences in turn;
//   N >  4096   four-step: N = N1 * N2, pass 1 transforms the N2 columns of
//               length N1 (coalesced column tiles) and applies the twiddles
//               e^{2 pi i j2 l1 / N}, pass 2 transforms rows l1 .. l1+3 together
//               with their mirror rows N1 - l1, which hold the Z_{N-l} needed by
//               the split above, for the three sequences of a pixel pair at
//               once, so each spectrum value is written exactly once.  Both
//               passes are instantiated per row length (2^6 .. 2^9) with the
//               pass plan fixed at compile time.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "lw_fft.cuh"

namespace lw {
namespace {

// Record formats of the mixed modes.
enum { kRecF64 = 0, kRecKahan = 1, kRecF32 = 2, kRecF32X4 = 3 };

// Record readers.  load() fetches an element's raw bits, cvt() turns them into T; pass 1
// issues a batch of loads before it converts any, so that they are all in flight.
template <typename T> struct RecReader;
template <> struct RecReader<double> {
    using Raw = double;
    const double* rec;
    __device__ double load(int64_t row, int64_t N, int64_t j) const { return __ldcs(rec + row * N + j); }
    __device__ double cvt(double v) const { return v; }
    __device__ double cvt_fp64(double v) const { return v; }
    __device__ double operator()(int64_t row, int64_t N, int64_t j) const {
        return cvt(load(row, N, j));
    }
};
template <> struct RecReader<float> {
    using Raw = uint2;   // a double, a (sum, compensation) float pair, or a float in .x
    const void* rec;
    int kind;   // kRecF64 double, kRecKahan (sum, compensation) pairs, kRecF32 float,
                // kRecF32X4 float4 (x, y, z, 0) per pixel and grid point
    __device__ uint2 load(int64_t row, int64_t N, int64_t j) const {
        if (kind == kRecF32)
            return make_uint2(__float_as_uint(__ldcs(static_cast<const float*>(rec) + row * N + j)),
                              0u);
        if (kind == kRecF32X4) {   // row = 3 m + c
            const int64_t m = row / 3;
            return make_uint2(__float_as_uint(__ldcs(static_cast<const float*>(rec) +
                                                     ((m * N + j) << 2) + (row - 3 * m))),
                              0u);
        }
        return __ldcs(static_cast<const uint2*>(rec) + row * N + j);
    }
    __device__ float cvt(uint2 v) const {   // double -> float on the integer pipe
        if (kind == kRecF32 || kind == kRecF32X4) return __uint_as_float(v.x);
        if (kind == kRecKahan) return __uint_as_float(v.x) + __uint_as_float(v.y);
        return to_float_bits(v.y, v.x);   // little-endian double: v.y holds the high word
    }
    // the same rounding by the FP64 pipe's conversion: pass 1 converts one row of each
    // pair this way and one on the integer pipe, which its index work already loads
    // (results differ only below the smallest normal float, which this one keeps)
    __device__ float cvt_fp64(uint2 v) const {
        if (kind == kRecF32 || kind == kRecF32X4) return __uint_as_float(v.x);
        if (kind == kRecKahan) return __uint_as_float(v.x) + __uint_as_float(v.y);
        return __double2float_rn(__hiloint2double((int)v.y, (int)v.x));
    }
    __device__ float operator()(int64_t row, int64_t N, int64_t j) const {
        return cvt(load(row, N, j));
    }
};

struct SeqRows {   // the two real rows of complex sequence (pair, kind)
    int64_t ra, rb;   // record rows (m * 3 + c), -1 = zero row
    int64_t ma, mb;   // pixels receiving |A|^2 and |B|^2 (-1 = none)
    int ca, cb;       // components of A and B
};

__device__ __forceinline__ SeqRows seq_rows(int64_t pair, int kind, int64_t n_pix) {
    const int64_t m0 = 2 * pair, m1 = 2 * pair + 1;
    const bool has1 = m1 < n_pix;
    SeqRows s;
    if (kind == 0) {
        s.ra = m0 * 3 + 0; s.rb = m0 * 3 + 1; s.ma = m0; s.mb = m0; s.ca = 0; s.cb = 1;
    } else if (kind == 1) {
        s.ra = has1 ? m1 * 3 + 0 : -1; s.rb = has1 ? m1 * 3 + 1 : -1;
        s.ma = has1 ? m1 : -1; s.mb = has1 ? m1 : -1; s.ca = 0; s.cb = 1;
    } else {
        s.ra = m0 * 3 + 2; s.rb = has1 ? m1 * 3 + 2 : -1;
        s.ma = m0; s.mb = has1 ? m1 : -1; s.ca = 2; s.cb = 2;
    }
    return s;
}

// Split Z_l / Z_{N-l} into the two real rows' spectra and accumulate the powers.
template <typename T, typename C>
__device__ __forceinline__ void emit(const SeqRows& sr, int64_t l, C zl, C zn, int64_t nl,
                                     T* __restrict__ S, C* __restrict__ X, bool atomic) {
    C A, B;
    A.x = (T)0.5 * (zl.x + zn.x);
    A.y = (T)0.5 * (zl.y - zn.y);
    B.x = (T)0.5 * (zl.y + zn.y);
    B.y = (T)0.5 * (zn.x - zl.x);
    const T pa = A.x * A.x + A.y * A.y;
    const T pb = B.x * B.x + B.y * B.y;
    if (sr.ma >= 0) {
        if (atomic) atomicAdd(S + sr.ma * nl + l, pa);
        else S[sr.ma * nl + l] += pa;
        if (X) X[(sr.ma * 3 + sr.ca) * nl + l] = A;
    }
    if (sr.mb >= 0) {
        if (atomic) atomicAdd(S + sr.mb * nl + l, pb);
        else S[sr.mb * nl + l] += pb;
        if (X) X[(sr.mb * 3 + sr.cb) * nl + l] = B;
    }
}

// ---------------------------------------------------------------- direct path

template <typename T>
__global__ void spectrum_direct_kernel(RecReader<T> rd, int64_t n_pix, int N, int logN, T scale,
                                       const typename V2<T>::type* __restrict__ tw,
                                       T* __restrict__ S, typename V2<T>::type* __restrict__ X) {
    using C = typename V2<T>::type;
    extern __shared__ unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);   // padded layout (fft_slot)
    const int sh = fft_pad_shift(logN);
    const int64_t pair = blockIdx.x;
    const int64_t nl = N / 2 + 1;
    for (int kind = 0; kind < 3; ++kind) {
        const SeqRows sr = seq_rows(pair, kind, n_pix);
        if (sr.ma < 0 && sr.mb < 0) continue;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            C z;
            z.x = sr.ra >= 0 ? (scale * rd(sr.ra, N, j)) * scale : (T)0;
            z.y = sr.rb >= 0 ? (scale * rd(sr.rb, N, j)) * scale : (T)0;
            buf[fft_slot<1, true>(bitrev(j, logN), 0, sh)] = z;
        }
        __syncthreads();
        fft_smem<C, 1, true>(buf, N, logN, tw, N, sh);
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
            const int ln = (N - l) & (N - 1);
            emit<T, C>(sr, l, buf[fft_slot<1, true>(l, 0, sh)], buf[fft_slot<1, true>(ln, 0, sh)], nl, S, X,
                       false);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- four-step

// Pass 1: tile of N1 = 2^LOGN1 rows x CT columns (columns j2 in [c0, c0+CT)) of sequence
// seq.
template <typename T, int CT, int LOGN1>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 4 : 2)
    spectrum_pass1_kernel(RecReader<T> rd, int64_t n_pix, int N, int N2, T scale,
                          const typename V2<T>::type* __restrict__ tw,
                          typename V2<T>::type* __restrict__ Y, int64_t seq0) {
    using C = typename V2<T>::type;
    constexpr int N1 = 1 << LOGN1, logN1 = LOGN1;
    extern __shared__ unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);   // [N1][CT]
    C* wrow = buf + N1 * CT;                    // [N1]
    const int64_t seq = seq0 + blockIdx.y;
    const int c0 = blockIdx.x * CT;
    const SeqRows sr = seq_rows(seq / 3, (int)(seq % 3), n_pix);
    // loads in batches of kBatch elements per thread, all in flight before any is converted
    constexpr int kBatch = 8;
    using Raw = typename RecReader<T>::Raw;
    for (int t0 = 0; t0 < N1 * CT; t0 += kBatch * kFftThreads) {
        Raw va[kBatch], vb[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int t = t0 + u * kFftThreads + threadIdx.x;
            const int64_t j = (int64_t)(t / CT) * N2 + c0 + t % CT;
            const bool in = t < N1 * CT;
            va[u] = in && sr.ra >= 0 ? rd.load(sr.ra, N, j) : Raw{};
            vb[u] = in && sr.rb >= 0 ? rd.load(sr.rb, N, j) : Raw{};
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int t = t0 + u * kFftThreads + threadIdx.x;
            if (t < N1 * CT) {
                C z;
                z.x = (scale * rd.cvt_fp64(va[u])) * scale;
                z.y = (scale * rd.cvt(vb[u])) * scale;
                buf[bitrev(t / CT, logN1) * CT + t % CT] = z;
            }
        }
    }
    // first twiddle factor tw[c0 l1] of each row, shared by the tile's CT columns
    for (int l1 = threadIdx.x; l1 < N1; l1 += kFftThreads)
        wrow[l1] = tw[((int64_t)c0 * l1) & (N - 1)];
    __syncthreads();
    fft_smem_fixed<C, CT, false, LOGN1>(buf, tw, N);
    C* Ys = Y + seq * (int64_t)N;
    // twiddle exp(2 pi i j2 l1 / N), j2 = c0 + c, as tw[c0 l1] tw[c l1]: the second factor
    // lies in the table's first CT * N1 entries, which stay in cache
    for (int t0 = 0; t0 < N1 * CT; t0 += kBatch * kFftThreads) {
        C w2[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int t = t0 + u * kFftThreads + threadIdx.x;
            w2[u] = t < N1 * CT ? tw[(t % CT) * (t / CT)] : C{};
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int t = t0 + u * kFftThreads + threadIdx.x;
            if (t < N1 * CT) {
                const int c = t % CT, l1 = t / CT;
                __stcs(Ys + (int64_t)l1 * N2 + c0 + c, cmul(buf[l1 * CT + c], cmul(wrow[l1], w2[u])));
            }
        }
    }
}

// Pass 2: rows l1 (ROWS consecutive values from blockIdx.x * ROWS, up to N1/2) and their
// mirrors N1 - l1 of the three sequences of one pixel pair, transformed together (6 *
// ROWS interleaved sequences); each spectrum value is written once (no atomics, no
// zeroing): every l <= N/2 has row l mod N1, which one CTA holds as l1 or as a mirror.
template <typename T, int ROWS, int LOGN2>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 4 : 2)
    spectrum_pass2_kernel(int64_t n_pix, int N, int N1,
                          const typename V2<T>::type* __restrict__ tw,
                          const typename V2<T>::type* __restrict__ Y, T* __restrict__ S,
                          typename V2<T>::type* __restrict__ X, int64_t pair0) {
    using C = typename V2<T>::type;
    constexpr int Cn = 6 * ROWS;   // column = (r*3 + kind)*2 + side
    constexpr int N2 = 1 << LOGN2, logN2 = LOGN2;
    constexpr int sh = LOGN2 > 5 ? LOGN2 - 5 : 0;
    extern __shared__ unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);   // [N2][Cn], padded (fft_slot)
    const int64_t pair = pair0 + blockIdx.y;
    const int r0 = blockIdx.x * ROWS;
    const int64_t m0 = 2 * pair, m1 = 2 * pair + 1;
    const bool has1 = m1 < n_pix;
    // every element of the tile is copied straight into its bit-reversed slot by
    // cp.async, all of them in flight at once; rows past N1/2 are zero-filled. A thread
    // keeps its j2 values (TPC threads per column, CPI columns per round) so that the
    // bit-reversed slot offsets are computed once. The rounds are unrolled: with one
    // column per round (N2 >= kFftThreads) every column's side, kind and source row
    // offset are constants of the code, and a copy is an address add and the copy.
    constexpr int TPC = N2 < kFftThreads ? N2 : kFftThreads;
    constexpr int CPI = kFftThreads / TPC;
    constexpr int JPT = N2 / TPC;
    const C* Yp = Y + pair * 3 * (int64_t)N;
    int jslot[JPT];
#pragma unroll
    for (int u = 0; u < JPT; ++u) {
        const int jr = bitrev(threadIdx.x % TPC + u * TPC, logN2);
        jslot[u] = jr * Cn + (jr >> sh);
    }
    const int col0 = CPI == 1 ? 0 : (int)threadIdx.x / TPC;
#pragma unroll
    for (int cc = 0; cc < (Cn + CPI - 1) / CPI; ++cc) {
        const int col = cc * CPI + col0;
        if (CPI > 1 && col >= Cn) break;
        const int side = col & 1, kind = (col >> 1) % 3, r = col / 6;
        const int l1 = r0 + r;
        const bool valid = l1 <= N1 / 2;
        const int row = valid ? (side ? (N1 - l1) & (N1 - 1) : l1) : 0;
        const C* src = Yp + (kind * N + row * N2 + threadIdx.x % TPC);
#pragma unroll
        for (int u = 0; u < JPT; ++u) {
            C* dst = buf + (jslot[u] + col);
            if (sizeof(C) == 8)
                cp_async8_zfill(dst, src + u * TPC, valid);
            else
                cp_async16_zfill(dst, src + u * TPC, valid);
        }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    fft_smem_fixed<C, Cn, true, LOGN2>(buf, tw, N);
    const int64_t nl = N / 2 + 1;
    const int half = N / 2;
    // split: thread t takes row r = t % ROWS of side (t / ROWS) % 2 for every
    // (2 ROWS)-th l2; both are fixed per thread since kFftThreads is a multiple of 2 ROWS
    constexpr int L2STEP = kFftThreads / (2 * ROWS);
    const int r = threadIdx.x % ROWS, side = (threadIdx.x / ROWS) & 1;
    const int l1 = r0 + r;
    if (l1 > N1 / 2) return;
    const int l1p = (N1 - l1) & (N1 - 1);
    if (side == 1 && l1p == l1) return;                 // self-mirrored row: once
    const int row = side ? l1p : l1;
    T* S0 = S + m0 * nl;
    T* S1 = S + m1 * nl;
    const C* bz = buf + (r * 6 + side);        // column (r*3 + kind)*2 + side, kind 0
    const C* bm = buf + (r * 6 + 1 - side);    // the other side's column
#pragma unroll 2
    for (int l2 = threadIdx.x / (2 * ROWS); l2 < N2; l2 += L2STEP) {
        const int l = row + N1 * l2;
        if (l > half) break;   // l grows with l2
        // mirror index N - l lives in the other side's column
        const int l2m = row == 0 ? (N2 - l2) & (N2 - 1) : N2 - 1 - l2;
        const int ol = l2 * Cn + (l2 >> sh), om = l2m * Cn + (l2m >> sh);
        T pw0 = (T)0, pw1 = (T)0;
#pragma unroll
        for (int kind = 0; kind < 3; ++kind) {
            const C zl = bz[ol + 2 * kind];
            const C zn = bm[om + 2 * kind];
            // s = zl + zn, d = zl - zn: the two real rows' spectra are A = (s.x, d.y) / 2
            // and B = (s.y, -d.x) / 2
            const C sv = cadd(zl, zn), dv = csub(zl, zn);
            C A, B;
            A.x = (T)0.5 * sv.x;
            A.y = (T)0.5 * dv.y;
            B.x = (T)0.5 * sv.y;
            B.y = (T)-0.5 * dv.x;
            T pa, pb;   // (x, y) of one pixel: pa = |A|^2 + |B|^2; (z0, z1): |A|^2, |B|^2
            if (kind < 2) {   // |A|^2 + |B|^2 = (|s|^2 + |d|^2) / 4
                const C q = sumsq2(sv, dv);
                pa = (T)0.25 * (q.x + q.y);
                pb = (T)0;
            } else {
                pa = (T)0.25 * (sv.x * sv.x + dv.y * dv.y);
                pb = (T)0.25 * (sv.y * sv.y + dv.x * dv.x);
            }
            if (kind == 0) {          // (x0, y0)
                pw0 += pa;
                if (X) {
                    X[(m0 * 3 + 0) * nl + l] = A;
                    X[(m0 * 3 + 1) * nl + l] = B;
                }
            } else if (kind == 1) {   // (x1, y1)
                pw1 += pa;
                if (X && has1) {
                    X[(m1 * 3 + 0) * nl + l] = A;
                    X[(m1 * 3 + 1) * nl + l] = B;
                }
            } else {                  // (z0, z1)
                pw0 += pa;
                pw1 += pb;
                if (X) {
                    X[(m0 * 3 + 2) * nl + l] = A;
                    if (has1) X[(m1 * 3 + 2) * nl + l] = B;
                }
            }
        }
        S0[l] = pw0;
        if (has1) S1[l] = pw1;
    }
}

template <typename T> void set_reader(RecReader<T>& rd, const void* rec, int kind);
template <> void set_reader<double>(RecReader<double>& rd, const void* rec, int) {
    rd.rec = static_cast<const double*>(rec);
}
template <> void set_reader<float>(RecReader<float>& rd, const void* rec, int kind) {
    rd.rec = rec;
    rd.kind = kind;
}

constexpr int64_t kPairsPerLaunch = 21845;   // 3 x pairs <= 65535 (grid y limit)

template <typename T>
int run_spectrum(const void* record, int kind, int64_t n_pix, const lw_grid* g, double q,
                 void* spectrum, void* X_save, void* ws, size_t* ws_bytes, cudaStream_t st) {
    using C = typename V2<T>::type;
    const int64_t N = g->n_bins;
    int logN = 0;
    while ((int64_t(1) << logN) < N) ++logN;
    const bool direct = N <= 4096;
    const int64_t n_pairs = (n_pix + 1) / 2;
    const int64_t n_seq = 3 * n_pairs;
    const size_t tw_bytes = align256(sizeof(C) * (size_t)N);
    const size_t y_bytes = direct ? 0 : align256(sizeof(C) * (size_t)N * (size_t)n_seq);
    const size_t need = tw_bytes + y_bytes;
    if (!ws) {
        *ws_bytes = need;
        return LW_OK;
    }
    if (*ws_bytes < need) {
        *ws_bytes = need;
        return LW_ESIZE;
    }
    C* tw = reinterpret_cast<C*>(ws);
    C* Y = reinterpret_cast<C*>(static_cast<char*>(ws) + tw_bytes);
    const double K = q * q / (16.0 * kPi * kPi * kPi * kEps0 * kC0);
    // inputs are multiplied twice by sqrt(sqrt(K) dt_u) so that no factor leaves the
    // normal FP32 range: X' = sqrt(K) dt_u X and S = |X'|^2
    const T scale = (T)sqrt(sqrt(K) * g->dt_u);
    RecReader<T> rd;
    set_reader<T>(rd, record, kind);
    T* S = static_cast<T*>(spectrum);
    C* X = static_cast<C*>(X_save);
    const int nl = (int)(N / 2 + 1);

    const int tw_grid = (int)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024);
    twiddle_kernel<T><<<tw_grid, 256, 0, st>>>(tw, N);
    if (launch_status() != LW_OK) return LW_ECUDA;
    if (direct) {
        if (cudaMemsetAsync(S, 0, sizeof(T) * (size_t)nl * (size_t)n_pix, st) != cudaSuccess)
            return LW_ECUDA;
        const size_t smem = sizeof(C) * (size_t)fft_slots((int)N, logN, 1);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(spectrum_direct_kernel<T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return LW_ECUDA;
        spectrum_direct_kernel<T><<<(unsigned)n_pairs, 256, smem, st>>>(
            rd, n_pix, (int)N, logN, scale, tw, S, X);
        return launch_status();
    }
    const int logN2 = (logN + 1) / 2, logN1 = logN - logN2;
    const int N1 = 1 << logN1, N2 = 1 << logN2;
    constexpr int CT = 16;
    // logN in 13..18: logN1 and logN2 in 6..9
    const int lsel1 = logN1 - 6, lsel2 = logN2 - 6;
    if (lsel1 < 0 || lsel1 > 3 || lsel2 < 0 || lsel2 > 3) return LW_EUNSUPPORTED;
    {
        using K1 = void (*)(RecReader<T>, int64_t, int, int, T, const C*, C*, int64_t);
        const K1 k1s[4] = {spectrum_pass1_kernel<T, CT, 6>, spectrum_pass1_kernel<T, CT, 7>,
                           spectrum_pass1_kernel<T, CT, 8>, spectrum_pass1_kernel<T, CT, 9>};
        const K1 kern = k1s[lsel1];
        const size_t smem = sizeof(C) * (size_t)N1 * (CT + 1);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return LW_ECUDA;
        // grid y is limited to 65535: sequences in chunks of 21845 pixel pairs
        for (int64_t p0 = 0; p0 < n_pairs; p0 += kPairsPerLaunch) {
            const int64_t np = std::min<int64_t>(kPairsPerLaunch, n_pairs - p0);
            dim3 grid((unsigned)(N2 / CT), (unsigned)(3 * np));
            kern<<<grid, kFftThreads, smem, st>>>(rd, n_pix, (int)N, N2, scale, tw, Y, 3 * p0);
            if (launch_status() != LW_OK) return LW_ECUDA;
        }
    }
    {
        // rows of pass 2 per CTA: up to 4, within 96 KB of shared memory
        int rows = 4;
        while (rows > 1 && sizeof(C) * (size_t)fft_slots(N2, logN2, 6 * rows) > 96 * 1024)
            rows >>= 1;
        const size_t smem = sizeof(C) * (size_t)fft_slots(N2, logN2, 6 * rows);
        using K2 = void (*)(int64_t, int, int, const C*, const C*, T*, C*, int64_t);
        const K2 k2s[3][4] = {
            {spectrum_pass2_kernel<T, 1, 6>, spectrum_pass2_kernel<T, 1, 7>,
             spectrum_pass2_kernel<T, 1, 8>, spectrum_pass2_kernel<T, 1, 9>},
            {spectrum_pass2_kernel<T, 2, 6>, spectrum_pass2_kernel<T, 2, 7>,
             spectrum_pass2_kernel<T, 2, 8>, spectrum_pass2_kernel<T, 2, 9>},
            {spectrum_pass2_kernel<T, 4, 6>, spectrum_pass2_kernel<T, 4, 7>,
             spectrum_pass2_kernel<T, 4, 8>, spectrum_pass2_kernel<T, 4, 9>}};
        const K2 kern = k2s[rows == 4 ? 2 : rows == 2 ? 1 : 0][lsel2];
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return LW_ECUDA;
        const int groups = (N1 / 2 + 1 + rows - 1) / rows;
        for (int64_t p0 = 0; p0 < n_pairs; p0 += kPairsPerLaunch) {
            const int64_t np = std::min<int64_t>(kPairsPerLaunch, n_pairs - p0);
            dim3 grid((unsigned)groups, (unsigned)np);
            kern<<<grid, kFftThreads, smem, st>>>(n_pix, (int)N, N1, tw, Y, S, X, p0);
            if (launch_status() != LW_OK) return LW_ECUDA;
        }
        return LW_OK;
    }
}

}  // namespace
}  // namespace lw

using namespace lw;

extern "C" int lw_spectrum(const void* record, int32_t precision, int64_t n_pix,
                           const lw_grid* grid, double q, void* spectrum, void* X_save, void* ws,
                           size_t* ws_bytes, void* stream) {
    if (!grid || !ws_bytes || n_pix < 1) return LW_EINVAL;
    if (precision != LW_FP64 && precision != LW_MIXED && precision != LW_MIXED_KAHAN &&
        precision != LW_MIXED_F32 && precision != LW_MIXED_F32X4)
        return LW_EINVAL;
    const int64_t N = grid->n_bins;
    if (N < 2 || N > (int64_t(1) << 18) || (N & (N - 1))) return LW_EUNSUPPORTED;
    if (!(grid->dt_u > 0.0) || !isfinite(q)) return LW_EINVAL;
    if (ws && (!record || !spectrum)) return LW_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (precision == LW_FP64)
        return run_spectrum<double>(record, 0, n_pix, grid, q, spectrum, X_save, ws, ws_bytes,
                                    st);
    const int kind = precision == LW_MIXED_KAHAN ? kRecKahan
                     : precision == LW_MIXED_F32 ? kRecF32
                     : precision == LW_MIXED_F32X4 ? kRecF32X4 : kRecF64;
    return run_spectrum<float>(record, kind, n_pix, grid, q, spectrum, X_save, ws, ws_bytes,
                               st);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of lw_spectrum.  Its scratch (twiddle table and, for
// n_bins above 4096, the four-step transform buffer) lives in one fixed
// device array owned by this library instead of a caller-supplied workspace.
namespace lw {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB per GPU
__device__ __align__(256) unsigned char g_spectrum_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_spectrum_scratch on the current device, looked up once
// per device (in host code the array's name is not a device address).
int static_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LW_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_spectrum_scratch) != cudaSuccess || !ptr)
            return LW_ECUDA;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return LW_OK;
}

}  // namespace
}  // namespace lw

extern "C" size_t lw_spectrum_static_capacity(void) { return lw::kStaticScratchBytes; }

extern "C" int lw_spectrum_static(const void* record, int32_t precision, int64_t n_pix,
                                  const lw_grid* grid, double q, void* spectrum, void* X_save,
                                  void* stream) {
    if (!grid || n_pix < 1 || !record || !spectrum) return LW_EINVAL;
    if (precision != LW_FP64 && precision != LW_MIXED && precision != LW_MIXED_KAHAN &&
        precision != LW_MIXED_F32 && precision != LW_MIXED_F32X4)
        return LW_EINVAL;
    const int64_t N = grid->n_bins;
    if (N < 2 || N > (int64_t(1) << 18) || (N & (N - 1))) return LW_EUNSUPPORTED;
    if (!(grid->dt_u > 0.0) || !isfinite(q)) return LW_EINVAL;
    size_t need = 0;
    int rc = lw_spectrum(record, precision, n_pix, grid, q, spectrum, X_save, nullptr, &need,
                         stream);
    if (rc != LW_OK) return rc;
    if (need > lw::kStaticScratchBytes) return LW_ESIZE;
    void* scratch = nullptr;
    rc = lw::static_scratch(&scratch);
    if (rc != LW_OK) return rc;
    size_t bytes = lw::kStaticScratchBytes;
    return lw_spectrum(record, precision, n_pix, grid, q, spectrum, X_save, scratch, &bytes,
                       stream);
}
