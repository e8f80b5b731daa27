// nd_fft.cuh -- register-resident FFTs for the padded grid sizes P = 16..1024.
//
// A length-P transform runs on a group of G threads (G consecutive lanes of one
// warp), each holding R1 = P/G points in registers.  Thread t owns the points
// with index = t (mod G) in natural order, both on input and on output:
//   register o of thread t  <->  element t + G*o.
// The transform is the two-pass ("four-step") split P = R1 x G:
//   1. an R1-point DFT in registers over the strided points of each thread,
//   2. a twiddle exp(-+2 pi i t k1 / P) read from a small shared table,
//   3. one transpose through a padded per-group shared scratch area,
//   4. R1/G G-point DFTs in registers,
// so every point crosses shared memory exactly once.  Register DFTs are
// radix-2 decimation in time, with one radix-3 or radix-5 stage on top for the
// sizes with those factors, and compile-time twiddles from the constant bank.
// G need not divide the warp: with G = 10 a warp holds three groups and its
// last two lanes idle.
#pragma once
#include "nd_common.cuh"

namespace nd {

// 32nd roots of unity exp(-2 pi i k / 32), k = 0..31, 24th roots
// exp(-2 pi i k / 24), k = 0..23 (for the stages of transforms with a factor
// 3) and 20th roots exp(-2 pi i k / 20), k = 0..19 (factor 5), in the constant
// bank.  Each translation unit that includes this header owns a copy, filled
// by its own upload hook (ND_DEFINE_TWIDDLE_UPLOAD).  Indices are compile-time
// constants in the register DFTs, so each use becomes a constant-bank operand.
static __constant__ float2 c_w32f[32];
static __constant__ double2 c_w32d[32];
static __constant__ float2 c_w24f[24];
static __constant__ double2 c_w24d[24];
static __constant__ float2 c_w20f[20];
static __constant__ double2 c_w20d[20];

template <typename T> __device__ __forceinline__ cplx<T> w32(int k);
template <> __device__ __forceinline__ cplx<float> w32<float>(int k) { float2 v = c_w32f[k]; return {v.x, v.y}; }
template <> __device__ __forceinline__ cplx<double> w32<double>(int k) { double2 v = c_w32d[k]; return {v.x, v.y}; }
template <typename T> __device__ __forceinline__ cplx<T> w24(int k);
template <> __device__ __forceinline__ cplx<float> w24<float>(int k) { float2 v = c_w24f[k]; return {v.x, v.y}; }
template <> __device__ __forceinline__ cplx<double> w24<double>(int k) { double2 v = c_w24d[k]; return {v.x, v.y}; }
template <typename T> __device__ __forceinline__ cplx<T> w20(int k);
template <> __device__ __forceinline__ cplx<float> w20<float>(int k) { float2 v = c_w20f[k]; return {v.x, v.y}; }
template <> __device__ __forceinline__ cplx<double> w20<double>(int k) { double2 v = c_w20d[k]; return {v.x, v.y}; }

// re/im: the 32 roots exp(-2 pi i k/32); the 24 and 20 roots are computed here.
#define ND_DEFINE_TWIDDLE_UPLOAD(name)                                                  \
    cudaError_t name(const double *re, const double *im)                                \
    {                                                                                   \
        float2 f[32];                                                                   \
        double2 d[32];                                                                  \
        for (int k = 0; k < 32; ++k) {                                                  \
            f[k] = make_float2((float)re[k], (float)im[k]);                             \
            d[k] = make_double2(re[k], im[k]);                                          \
        }                                                                               \
        float2 f24[24], f20[20];                                                        \
        double2 d24[24], d20[20];                                                       \
        for (int k = 0; k < 24; ++k) {                                                  \
            const double c = cos(2.0 * M_PI * k / 24.0), s = -sin(2.0 * M_PI * k / 24.0); \
            f24[k] = make_float2((float)c, (float)s);                                   \
            d24[k] = make_double2(c, s);                                                \
        }                                                                               \
        for (int k = 0; k < 20; ++k) {                                                  \
            const double c = cos(2.0 * M_PI * k / 20.0), s = -sin(2.0 * M_PI * k / 20.0); \
            f20[k] = make_float2((float)c, (float)s);                                   \
            d20[k] = make_double2(c, s);                                                \
        }                                                                               \
        cudaError_t e = cudaMemcpyToSymbol(c_w32f, f, sizeof(f));                        \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w32d, d, sizeof(d));             \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w24f, f24, sizeof(f24));         \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w24d, d24, sizeof(d24));         \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w20f, f20, sizeof(f20));         \
        if (e != cudaSuccess) return e;                                                 \
        return cudaMemcpyToSymbol(c_w20d, d20, sizeof(d20));                            \
    }

template <int P> struct FFTShape;
template <> struct FFTShape<16> { static constexpr int G = 4; };
template <> struct FFTShape<32> { static constexpr int G = 4; };
template <> struct FFTShape<64> { static constexpr int G = 8; };
template <> struct FFTShape<128> { static constexpr int G = 8; };
template <> struct FFTShape<256> { static constexpr int G = 16; };
template <> struct FFTShape<512> { static constexpr int G = 16; };
template <> struct FFTShape<1024> { static constexpr int G = 32; };
// 192 = 8 x 24 (a radix-3 stage in the 24-point register DFT): the smallest
// grid of the form 2^n or 3 * 2^n above 128 for disks of 65..96 cells
template <> struct FFTShape<192> { static constexpr int G = 8; };
// 200 = 10 x 20 (radix-5 stages in the 20- and 10-point register DFTs) for
// disks of 97..100 cells: ten-lane groups, three to a warp
template <> struct FFTShape<200> { static constexpr int G = 10; };

template <int P> struct FFTGeom {
    static constexpr int G = FFTShape<P>::G;
    static constexpr int R1 = P / G;
    static_assert(R1 % G == 0, "R1 must be a multiple of G");
    static constexpr int R2 = R1 / G;  // G-point DFTs per thread in pass 2
    // per-group scratch: R1 rows of G+1 (padding breaks the stride-G conflicts),
    // rounded so consecutive groups start 8 complex words apart modulo 16
    static constexpr int SROW = G + 1;
    static constexpr int SRAW = R1 * SROW;
    static constexpr int SCRATCH = SRAW + ((8 - SRAW % 16) + 16) % 16;
    static constexpr int GROUPS_PER_WARP = 32 / G;   // whole groups per warp
    static constexpr bool POW2 = (G & (G - 1)) == 0;   // groups tile the warp exactly
};

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }
__host__ __device__ constexpr int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// b * w^k for the N-th root w = exp(DIR 2 pi i / N) (DIR = -1 forward), N a
// power of two up to 32 or a divisor of 24 or of 20, with the trivial factors
// 1, -1 and -+i special-cased; k and N are constants after the register DFT
// loops are unrolled, so the branches fold away.
template <int DIR, typename T>
__device__ __forceinline__ cplx<T> twid(cplx<T> b, int k, int N)
{
    k %= N;
    if (k == 0) return b;
    if (2 * k == N) return cplx<T>{-b.x, -b.y};
    if (4 * k == N) {  // exp(DIR i pi / 2) = DIR * i
        return DIR < 0 ? cplx<T>{b.y, -b.x} : cplx<T>{-b.y, b.x};
    }
    if (4 * k == 3 * N) return DIR < 0 ? cplx<T>{-b.y, b.x} : cplx<T>{b.y, -b.x};
    cplx<T> w = (32 % N == 0) ? w32<T>(k * (32 / N)) : (24 % N == 0) ? w24<T>(k * (24 / N)) : w20<T>(k * (20 / N));
    return DIR < 0 ? cmul(b, w) : cmulc(b, w);
}

// In-register N-point DFT, natural order in and out:
// v[k] <- sum_n v[n] exp(DIR 2 pi i n k / N), for N a power of two up to 32
// (radix 2), or three or five times one (one radix-3 stage on top, N | 24, or
// one radix-5 stage, N | 20).
template <int N, int DIR, typename T>
__device__ __forceinline__ void dft_reg(cplx<T> *v)
{
    if constexpr ((N & (N - 1)) == 0) {
        constexpr int B = ilog2c(N);
        cplx<T> u[N];
#pragma unroll
        for (int i = 0; i < N; ++i) u[bitrev(i, B)] = v[i];
#pragma unroll
        for (int half = 1; half < N; half *= 2) {
#pragma unroll
            for (int g = 0; g < N; g += 2 * half) {
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    cplx<T> a = u[g + j];
                    cplx<T> b = twid<DIR>(u[g + j + half], j, 2 * half);
                    u[g + j] = cadd(a, b);
                    u[g + j + half] = csub(a, b);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = u[i];
    } else if constexpr (N % 5 == 0) {
        static_assert(20 % N == 0, "register DFT sizes: 2^n <= 32 or divisors of 24 or of 20");
        // decimation in time by 5: five N/5-point DFTs of the residues n = 5m + r,
        // then N/5 five-point butterflies over r of w_N^{rk} A_r[k]; with
        // c_j = cos(2 pi j/5), s_j = sin(2 pi j/5) and DIR i = exp(DIR i pi/2):
        //   X[k]      = b0 + (b1 + b4) + (b2 + b3)
        //   X[k +  M] = p1 + DIR i q1,  X[k + 4M] = p1 - DIR i q1
        //   X[k + 2M] = p2 + DIR i q2,  X[k + 3M] = p2 - DIR i q2
        // p1 = b0 + c1 (b1 + b4) + c2 (b2 + b3),  q1 = s1 (b1 - b4) + s2 (b2 - b3)
        // p2 = b0 + c2 (b1 + b4) + c1 (b2 + b3),  q2 = s2 (b1 - b4) - s1 (b2 - b3)
        constexpr int M = N / 5;
        cplx<T> a[5][M];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int r = 0; r < 5; ++r) a[r][m] = v[5 * m + r];
#pragma unroll
        for (int r = 0; r < 5; ++r) dft_reg<M, DIR>(a[r]);
        const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);   // cos(2 pi/5), cos(4 pi/5)
        const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);    // sin(2 pi/5), sin(4 pi/5)
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const cplx<T> b0 = a[0][k], b1 = twid<DIR>(a[1][k], k, N), b2 = twid<DIR>(a[2][k], 2 * k, N),
                          b3 = twid<DIR>(a[3][k], 3 * k, N), b4 = twid<DIR>(a[4][k], 4 * k, N);
            const cplx<T> t1 = cadd(b1, b4), t2 = cadd(b2, b3), t3 = csub(b1, b4), t4 = csub(b2, b3);
            const cplx<T> p1 = {b0.x + c1 * t1.x + c2 * t2.x, b0.y + c1 * t1.y + c2 * t2.y};
            const cplx<T> p2 = {b0.x + c2 * t1.x + c1 * t2.x, b0.y + c2 * t1.y + c1 * t2.y};
            const cplx<T> q1 = {s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
            const cplx<T> q2 = {s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
            // DIR i q = DIR (-q.y, q.x)
            const cplx<T> e1 = DIR < 0 ? cplx<T>{q1.y, -q1.x} : cplx<T>{-q1.y, q1.x};
            const cplx<T> e2 = DIR < 0 ? cplx<T>{q2.y, -q2.x} : cplx<T>{-q2.y, q2.x};
            v[k] = cadd(b0, cadd(t1, t2));
            v[k + M] = cadd(p1, e1);
            v[k + 4 * M] = csub(p1, e1);
            v[k + 2 * M] = cadd(p2, e2);
            v[k + 3 * M] = csub(p2, e2);
        }
    } else {
        static_assert(N % 3 == 0 && 24 % N == 0, "register DFT sizes: 2^n <= 32 or divisors of 24 or of 20");
        // decimation in time by 3: three N/3-point DFTs of the residues n = 3m + r,
        // then N/3 three-point butterflies with the twiddles w_N^{rk}
        constexpr int M = N / 3;
        cplx<T> a[M], b[M], c[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            a[m] = v[3 * m];
            b[m] = v[3 * m + 1];
            c[m] = v[3 * m + 2];
        }
        dft_reg<M, DIR>(a);
        dft_reg<M, DIR>(b);
        dft_reg<M, DIR>(c);
        const T h3 = T(0.86602540378443864676);   // sin(pi/3)
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const cplx<T> bk = twid<DIR>(b[k], k, N), ck = twid<DIR>(c[k], 2 * k, N);
            const cplx<T> s = cadd(bk, ck), d = csub(bk, ck);
            const cplx<T> t = {a[k].x - T(0.5) * s.x, a[k].y - T(0.5) * s.y};
            // exp(DIR 2 pi i/3) = -1/2 + DIR i sin(pi/3): X[k + M] = t + DIR i h3 d, X[k + 2M] = t - DIR i h3 d
            const cplx<T> e = DIR < 0 ? cplx<T>{h3 * d.y, -h3 * d.x} : cplx<T>{-h3 * d.y, h3 * d.x};
            v[k] = cadd(a[k], s);
            v[k + M] = cadd(t, e);
            v[k + 2 * M] = csub(t, e);
        }
    }
}

// N-point DFT of an input whose upper half is zero (v[j] = 0 for j >= N/2):
// even outputs are the N/2-point DFT of v, odd outputs that of v[j] w^j.
template <int N, int DIR, typename T>
__device__ __forceinline__ void dft_reg_halfin(cplx<T> *v)
{
    cplx<T> a[N / 2], b[N / 2];
#pragma unroll
    for (int j = 0; j < N / 2; ++j) {
        a[j] = v[j];
        b[j] = twid<DIR>(v[j], j, N);
    }
    dft_reg<N / 2, DIR>(a);
    dft_reg<N / 2, DIR>(b);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = b[k];
    }
}

// N-point DFT of which only the outputs k < N/2 are needed (the others are
// left undefined): X[k] = A[k] + w^k B[k] over the even/odd halves.
template <int N, int DIR, typename T>
__device__ __forceinline__ void dft_reg_halfout(cplx<T> *v)
{
    cplx<T> a[N / 2], b[N / 2];
#pragma unroll
    for (int j = 0; j < N / 2; ++j) {
        a[j] = v[2 * j];
        b[j] = v[2 * j + 1];
    }
    dft_reg<N / 2, DIR>(a);
    dft_reg<N / 2, DIR>(b);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) v[k] = cadd(a[k], twid<DIR>(b[k], k, N));
}

enum : int { FFT_FULL = 0, FFT_HALF_IN = 1, FFT_HALF_OUT = 2 };

// Full P-point transform on a group of G threads.
//   v      : the thread's R1 points, element t + G*o in v[o]; replaced by the
//            transform in the same layout
//   t      : index of the thread in its group (0..G-1)
//   scr    : this group's private shared scratch, FFTGeom<P>::SCRATCH words
//   tw     : shared twiddle table [R1][G], tw[k1*G + t] = exp(-2 pi i t k1 / P)
//   gmask  : lane mask of the group (for __syncwarp)
//   FL     : FFT_HALF_IN when elements >= P/2 are zero (registers o >= R1/2
//            are then not read), FFT_HALF_OUT when only elements < P/2 of the
//            result are needed (registers o >= R1/2 are then undefined)
//   TWS    : row stride of the twiddle table (G by default; 2G reads the
//            table of a 2P-point transform, whose even rows are this one's)
template <int P, int DIR, int FL = FFT_FULL, int TWS = FFTGeom<P>::G, typename T>
__device__ __forceinline__ void fft_group(cplx<T> *v, int t, cplx<T> *scr, const cplx<T> *tw, unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, R2 = Gm::R2, SROW = Gm::SROW;
    if (FL & FFT_HALF_IN) dft_reg_halfin<R1, DIR>(v);
    else dft_reg<R1, DIR>(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
        cplx<T> w = tw[k1 * TWS + t];
        v[k1] = DIR < 0 ? cmul(v[k1], w) : cmulc(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) scr[k1 * SROW + t] = v[k1];
    __syncwarp(gmask);
#pragma unroll
    for (int i = 0; i < R2; ++i)
#pragma unroll
        for (int s = 0; s < G; ++s) v[i * G + s] = scr[(t + G * i) * SROW + s];
    __syncwarp(gmask);
#pragma unroll
    for (int i = 0; i < R2; ++i) {
        if (FL & FFT_HALF_OUT) dft_reg_halfout<G, DIR>(v + i * G);
        else dft_reg<G, DIR>(v + i * G);
    }
    // v[i*G + k2] holds X[t + G*i + R1*k2] = X[t + G*(i + R2*k2)]: reorder to o = i + R2*k2
    // (with FFT_HALF_OUT only k2 < G/2, i.e. o < R1/2, is defined)
    constexpr int K2 = (FL & FFT_HALF_OUT) ? G / 2 : G;
    cplx<T> o_[R1];
#pragma unroll
    for (int i = 0; i < R2; ++i)
#pragma unroll
        for (int k2 = 0; k2 < K2; ++k2) o_[i + R2 * k2] = v[i * G + k2];
#pragma unroll
    for (int o = 0; o < R2 * K2; ++o) v[o] = o_[o];
}

}  // namespace nd
