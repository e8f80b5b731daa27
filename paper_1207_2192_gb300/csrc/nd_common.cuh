// nd_common.cuh -- shared device helpers of the GB300 thin-nanodisk library:
// complex arithmetic, constant-bank twiddles, the Philox4x32-10 noise stream
// and the per-replica work descriptors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nd {

template <typename T> struct cplx { T x, y; };
template <typename T> struct vec3 { T x, y, z; };

template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b)  // a * conj(b)
{
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T> __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return {a.x, -a.y}; }
template <typename T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.x * s, a.y * s}; }

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T drsqrt(T x);
template <> __device__ __forceinline__ float drsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double drsqrt<double>(double x) { return 1.0 / sqrt(x); }

// ------------------------------------------------------------- Philox noise

// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds of the
// 32x32->64 multiply-xor round with the published multipliers and Weyl key
// increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Three standard normals of one cell and one time step: key = seed words,
// counter = (cell, step low, step high, 0); Box-Muller on the pairs (r0, r1)
// and (r2, r3) with u = (r + 1) 2^-32 and angle 2 pi r 2^-32.
template <typename T> __device__ __forceinline__ vec3<T> thermal_normals(uint64_t seed, uint32_t cell, uint64_t step);

template <> __device__ __forceinline__ vec3<float> thermal_normals<float>(uint64_t seed, uint32_t cell, uint64_t step)
{
    uint4 r = philox4x32_10(make_uint4(cell, (uint32_t)step, (uint32_t)(step >> 32), 0u), (uint32_t)seed,
                            (uint32_t)(seed >> 32));
    const float s32 = 2.3283064365386963e-10f;
    // u = (r + 1) 2^-32 in (0, 1]: the word rounded to float, scaled exactly, then offset
    float u0 = __fmaf_rn(__uint2float_rn(r.x), s32, s32), u2 = __fmaf_rn(__uint2float_rn(r.z), s32, s32);
    // the hardware approximations (absolute error ~2^-21 on these ranges, far
    // below the FP32 step's own rounding of sigma w); the clamp keeps
    // -2 log u >= 0 where u rounds to just below 1
    float ra = sqrtf(fmaxf(-2.0f * __logf(u0), 0.0f)), rb = sqrtf(fmaxf(-2.0f * __logf(u2), 0.0f));
    const float two_pi = 6.283185307179586f;
    float s1, c1;
    __sincosf(two_pi * (__uint2float_rn(r.y) * s32), &s1, &c1);
    const float c3 = __cosf(two_pi * (__uint2float_rn(r.w) * s32));
    return {ra * c1, ra * s1, rb * c3};
}

template <> __device__ __forceinline__ vec3<double> thermal_normals<double>(uint64_t seed, uint32_t cell, uint64_t step)
{
    uint4 r = philox4x32_10(make_uint4(cell, (uint32_t)step, (uint32_t)(step >> 32), 0u), (uint32_t)seed,
                            (uint32_t)(seed >> 32));
    const double s32 = 2.3283064365386963e-10;
    double u0 = ((double)r.x + 1.0) * s32, u2 = ((double)r.z + 1.0) * s32;
    double ra = sqrt(-2.0 * log(u0)), rb = sqrt(-2.0 * log(u2));
    double s1, c1, s3, c3;
    sincospi(2.0 * (double)r.y * s32, &s1, &c1);
    sincospi(2.0 * (double)r.w * s32, &s3, &c3);
    return {ra * c1, ra * s1, rb * c3};
}

// ------------------------------------------------------------ descriptors

// One replica (one disk state) as the kernels see it.
struct Replica {
    int D, Dpad;                 // grid side and padded row length of the state
    int disk;                    // disk index (geometry)
    int flags;                   // bit 0: thermal noise on
    long long state_off;         // element offset of this replica's [3][D][Dpad] block
    long long spec_off;          // complex-element offset of its [3][D][RS] spectrum (global path)
    const void *Ghat;            // [P/2+1 (kx)][P/2+1 (ky)][4] spectral kernel, incl. exchange and 1/P^2,
                                 // then the same values as [4][P/2+1][P/2+1]
    const unsigned char *mask;   // [D][D]
    const int *cells;            // the cells inside the disk, j*D+i in increasing order (ncells of them)
    int ncells, pad_cells;
    double chext[3];             // (a^2/lambda^2) h_ext
    double alpha, dtau, sigma;   // damping, dimensionless step, noise amplitude
    unsigned long long seed, step0;
    float fchext[3];             // single-precision copies for the FP32 kernels
    float falpha, fdtau, fsigma;
    // optional per-step external field (a pulse or any schedule): step s of
    // the stepping modes uses (a^2/lambda^2) H_ext(s)/Ms = sched[3 s ..] while
    // s < nsched, else chext; one array per kernel precision (null: none)
    const float *fsched;
    const double *dsched;
    long long nsched;
};

// Stepping parameters in the kernel's precision (no double arithmetic in the
// FP32 kernels: GB300's FP64 rate is a small fraction of its FP32 rate).
template <typename T> struct StepParams { T chext[3], alpha, dtau, sigma; };
template <typename T> __device__ __forceinline__ StepParams<T> step_params(const Replica &r);
template <> __device__ __forceinline__ StepParams<float> step_params<float>(const Replica &r)
{
    return {{r.fchext[0], r.fchext[1], r.fchext[2]}, r.falpha, r.fdtau, r.fsigma};
}
template <> __device__ __forceinline__ StepParams<double> step_params<double>(const Replica &r)
{
    return {{r.chext[0], r.chext[1], r.chext[2]}, r.alpha, r.dtau, r.sigma};
}

// The scaled external field (a^2/lambda^2) H_ext/Ms of step s of a stepping
// call: the disk's schedule while s < nsched, else the static field.
template <typename T> __device__ __forceinline__ vec3<T> step_chext(const Replica &r, const StepParams<T> &sp,
                                                                    unsigned long long s);
template <> __device__ __forceinline__ vec3<float> step_chext<float>(const Replica &r, const StepParams<float> &sp,
                                                                      unsigned long long s)
{
    if (r.fsched && s < (unsigned long long)r.nsched) return {r.fsched[3 * s], r.fsched[3 * s + 1], r.fsched[3 * s + 2]};
    return {sp.chext[0], sp.chext[1], sp.chext[2]};
}
template <> __device__ __forceinline__ vec3<double> step_chext<double>(const Replica &r, const StepParams<double> &sp,
                                                                        unsigned long long s)
{
    if (r.dsched && s < (unsigned long long)r.nsched) return {r.dsched[3 * s], r.dsched[3 * s + 1], r.dsched[3 * s + 2]};
    return {sp.chext[0], sp.chext[1], sp.chext[2]};
}

// Per-replica inputs and outputs of the constrained relaxation.
struct RelaxIO {
    double X[2];      // constraint centre in cell units relative to the grid centre
    double lam[2];    // Lagrange multipliers (start values in, final values out)
    double resid;     // residual max |m x e|/|e| of the last sweep
    int iters;        // sweeps applied
    int status;       // 0 converged, 1 max_iter reached
};

// Per-replica statistics accumulators (double precision sums).
struct StatsAcc {
    double n, sx, sy, sr2;   // samples with a vortex, sums of x, y, x^2 + y^2 (metres)
    double nv, sv2;          // speed samples and the sum of V^2 (m^2/s^2)
    double no_vortex;        // samples without a vortex
    double px, py;           // previous core position
    int have_prev, pad;
};

// Status word written by kernels (bit flags), read by the host after a sync.
enum : unsigned { ND_DEV_NAN = 1u, ND_DEV_TIMEOUT = 2u };

}  // namespace nd
