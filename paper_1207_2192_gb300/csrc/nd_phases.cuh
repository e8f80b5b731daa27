// nd_phases.cuh -- the three passes of one demagnetisation + exchange field
// evaluation (Section II.B convolution done with FFTs), written once and used
// both by the fused single-CTA kernel (spectrum in shared memory) and by the
// global-memory path (spectrum in HBM/L2).
//
// Spectrum layout: spec[c][y][RS] complex, c = x, y, z; row y = 0..D-1 of the
// zero-padded P x P grid (rows D..P-1 are zero and never stored); column
// kx = 0..P/2 of the half spectrum; RS words per row (SpecGeom).  After the inverse row pass the same rows,
// viewed as real arrays, hold the field b' = exchange + (a^2/lambda^2) h^M.
//
// Row pass (forward): the two real rows m_x(y), m_y(y) are transformed as one
// complex row m_x + i m_y, and the m_z rows are taken in pairs (y, y+1); the
// two real spectra are separated with the mirror element P-k.
// Column pass: kx = 1..P/2-1 are complex columns; the two real columns kx = 0
// and kx = P/2 are packed as one complex column.  Each column is transformed,
// multiplied by the spectral kernel, and transformed back, keeping rows < D.
// Row pass (inverse): the Hermitian half rows are completed by conjugation and
// pairs of real outputs are recovered from one complex inverse transform.
#pragma once
#include "nd_fft.cuh"

namespace nd {

template <int P> struct SpecGeom {
    // on chip (P <= 128) the two padding words keep the column reads free of
    // bank conflicts; in global memory (P > 128) four start each row on a
    // 32-byte sector, so the row passes move whole sectors
    static constexpr int RS = (P > 128) ? (P / 2 + 4) : (P >= 32) ? (P / 2 + 2) : (P / 2 + 2 + 8);
    static constexpr int KH = P / 2 + 1;   // kernel table side
};

template <typename T> struct GhatVal { T xx, yy, xy, zz; };

template <typename T> __device__ __forceinline__ GhatVal<T> load_ghat(const T *G, int idx);
template <> __device__ __forceinline__ GhatVal<float> load_ghat<float>(const float *G, int idx)
{
    float4 v = __ldg(reinterpret_cast<const float4 *>(G) + idx);
    return {v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ GhatVal<double> load_ghat<double>(const double *G, int idx)
{
    double2 a = __ldg(reinterpret_cast<const double2 *>(G) + 2 * idx);
    double2 b = __ldg(reinterpret_cast<const double2 *>(G) + 2 * idx + 1);
    return {a.x, a.y, b.x, b.y};
}

// Mirror element through the group's scratch: mirror_put stores the group's
// transform in natural order (element k at scr[k]); after a __syncwarp,
// mirror_get(scr, k) returns element (P - k) mod P.  The caller syncs the
// group again before the scratch is reused.
template <int P, typename T>
__device__ __forceinline__ void mirror_put(const cplx<T> *v, cplx<T> *scr, int t)
{
    using Gm = FFTGeom<P>;
#pragma unroll
    for (int o = 0; o < Gm::R1; ++o) scr[t + Gm::G * o] = v[o];
}
template <int P, typename T>
__device__ __forceinline__ cplx<T> mirror_get(const cplx<T> *scr, int k)
{
    return scr[k == 0 ? 0 : P - k];
}

// Number of row tasks: D complex xy rows plus ceil(D/2) z row pairs.
__host__ __device__ __forceinline__ int row_tasks(int D) { return D + (D + 1) / 2; }

// ---------------------------------------------------------------- row fwd

// Forward transform of one complex row v (held as a group's registers, element
// t + G o in v[o]; only the first half may be nonzero) whose real and imaginary
// parts are two real rows A and B, followed by their separation with the
// mirror element: the half spectra k = 0..P/2 go to dA and (if hasB) dB.
template <int P, typename T>
__device__ __forceinline__ void row_fwd_core(cplx<T> *v, bool active, cplx<T> *dA, cplx<T> *dB, bool hasB, int t,
                                             cplx<T> *scr, const cplx<T> *tw, unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1;
    fft_group<P, -1, FFT_HALF_IN>(v, t, scr, tw, gmask);
    mirror_put<P>(v, scr, t);
    __syncwarp(gmask);
    if (active) {
#pragma unroll
        for (int o = 0; o < R1; ++o) {
            const int k = t + G * o;
            if (k <= P / 2) {
                const cplx<T> w = mirror_get<P>(scr, k);
                const T h = T(0.5);
                cplx<T> A = {h * (v[o].x + w.x), h * (v[o].y - w.y)};
                cplx<T> B = {h * (v[o].y + w.y), -h * (v[o].x - w.x)};
                dA[k] = A;
                if (hasB) dB[k] = B;
            }
        }
    }
    __syncwarp(gmask);
}

// ms: stage magnetisation [3][D][ldm] (zero outside the disk); spec as above
// with component stride cstride (complex words).
template <int P, typename T>
__device__ __forceinline__ void row_fwd_task(int q, bool active, int D, const T *ms, int ldm, long long mstride,
                                             cplx<T> *spec, long long cstride, int t, int lane, cplx<T> *scr,
                                             const cplx<T> *tw, unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS;
    const bool isxy = q < D;
    const int y0 = isxy ? q : 2 * (q - D);
    const int y1 = y0 + 1;
    cplx<T> v[R1];
#pragma unroll
    for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
#pragma unroll
    for (int o = 0; o < R1 / 2; ++o) {   // D <= P/2: the upper half is zero padding
        const int x = t + G * o;
        if (active && x < D) {
            if (isxy) {
                v[o].x = ms[(long long)y0 * ldm + x];
                v[o].y = ms[mstride + (long long)y0 * ldm + x];
            } else {
                v[o].x = ms[2 * mstride + (long long)y0 * ldm + x];
                if (y1 < D) v[o].y = ms[2 * mstride + (long long)y1 * ldm + x];
            }
        }
    }
    cplx<T> *dA = isxy ? spec + (long long)y0 * RS : spec + 2 * cstride + (long long)y0 * RS;
    cplx<T> *dB = isxy ? spec + cstride + (long long)y0 * RS : spec + 2 * cstride + (long long)y1 * RS;
    const bool hasB = isxy || (y1 < D);
    row_fwd_core<P, T>(v, active, dA, dB, hasB, t, scr, tw, gmask);
}

// --------------------------------------------------------------- columns

// One row of the in-plane 2x2 block applied to the pair (a, b) = (X, Y):
// g0 a + g1 b.  Every path computes the block through this helper, so all
// schedules round the product identically.
template <typename T>
__device__ __forceinline__ cplx<T> tensor_row(T g0, cplx<T> a, T g1, cplx<T> b)
{
    return {g0 * a.x + g1 * b.x, g0 * a.y + g1 * b.y};
}

template <int P, typename T>
__device__ __forceinline__ void col_multiply(cplx<T> *vx, cplx<T> *vy, const T *Ghat, int kx, int t)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, KH = SpecGeom<P>::KH;
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        const int ky = t + G * o;
        const bool up = ky <= P / 2;
        const int kyr = up ? ky : P - ky;
        GhatVal<T> g = load_ghat<T>(Ghat, kx * KH + kyr);
        const T gxy = up ? g.xy : -g.xy;     // G_xy is odd in ky
        cplx<T> a = vx[o], b = vy[o];
        vx[o] = tensor_row(g.xx, a, gxy, b);
        vy[o] = tensor_row(gxy, a, g.yy, b);
    }
}

template <int P, typename T>
__device__ __forceinline__ void col_multiply_z(cplx<T> *vz, const T *Ghat, int kx, int t)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, KH = SpecGeom<P>::KH;
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        const int ky = t + G * o;
        const int kyr = ky <= P / 2 ? ky : P - ky;
        GhatVal<T> g = load_ghat<T>(Ghat, kx * KH + kyr);
        vz[o] = cscale(vz[o], g.zz);
    }
}

template <int P, typename T, int RS = SpecGeom<P>::RS>
__device__ __forceinline__ void col_load(cplx<T> *v, const cplx<T> *col, int D, int t, bool active)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1;
#pragma unroll
    for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
#pragma unroll
    for (int o = 0; o < R1 / 2; ++o) {   // rows >= D (and so >= P/2) are zero padding
        const int y = t + G * o;
        if (active && y < D) v[o] = col[(long long)y * RS];
    }
}

template <int P, typename T, int RS = SpecGeom<P>::RS>
__device__ __forceinline__ void col_store(const cplx<T> *v, cplx<T> *col, int D, int t, bool active)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1;
    if (!active) return;
#pragma unroll
    for (int o = 0; o < R1 / 2; ++o) {
        const int y = t + G * o;
        if (y < D) col[(long long)y * RS] = v[o];
    }
}

// Packed pair of real columns kx = 0 and kx = P/2 of component c (spectrum
// column base col): load as c0 + i c_{P/2}, forward transform, separate the
// two spectra with the mirror element, scale each by its diagonal kernel entry
// and re-pack, ready for the inverse transform.
template <int P, typename T>
__device__ __forceinline__ void packed_col_fwd_loaded(cplx<T> *v, int c, const T *Ghat, int t, cplx<T> *scr,
                                                      const cplx<T> *tw, unsigned gmask);

template <int P, typename T>
__device__ __forceinline__ void packed_col_fwd(cplx<T> *v, int c, bool active, int D, const cplx<T> *col,
                                               const T *Ghat, int t, int lane, cplx<T> *scr, const cplx<T> *tw,
                                               unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS;
#pragma unroll
    for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
#pragma unroll
    for (int o = 0; o < R1 / 2; ++o) {
        const int y = t + G * o;
        if (active && y < D) v[o] = {col[(long long)y * RS].x, col[(long long)y * RS + P / 2].x};
    }
    packed_col_fwd_loaded<P, T>(v, c, Ghat, t, scr, tw, gmask);
}

// The spectral step of a packed pair after its forward transform (v holds
// the transform of c0 + i c_{P/2}): separate the two column spectra with the
// mirror element, scale each by its diagonal kernel entry (s0 at kx = 0, s1 at
// kx = P/2) and re-pack them for the inverse transform.
template <int P, typename T>
__device__ __forceinline__ void packed_col_scale(cplx<T> *v, int c, const T *Ghat, int t, cplx<T> *scr,
                                                 unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, KH = SpecGeom<P>::KH;
    mirror_put<P>(v, scr, t);
    __syncwarp(gmask);
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        const int ky = t + G * o;
        const int kyr = ky <= P / 2 ? ky : P - ky;
        const cplx<T> w = mirror_get<P>(scr, ky);
        const int comp = c == 2 ? 3 : c;    // the diagonal entry: xx, yy or zz
        const T s0 = __ldg(Ghat + 4 * kyr + comp);
        const T s1 = __ldg(Ghat + 4 * ((P / 2) * KH + kyr) + comp);
        const T h = T(0.5);
        cplx<T> F0 = {h * (v[o].x + w.x), h * (v[o].y - w.y)};
        cplx<T> F1 = {h * (v[o].y + w.y), -h * (v[o].x - w.x)};
        F0 = cscale(F0, s0);
        F1 = cscale(F1, s1);
        v[o] = {F0.x - F1.y, F0.y + F1.x};
    }
    __syncwarp(gmask);
}

// The packed pair after loading (v = c0 + i c_{P/2}, rows < D, zero above).
template <int P, typename T>
__device__ __forceinline__ void packed_col_fwd_loaded(cplx<T> *v, int c, const T *Ghat, int t, cplx<T> *scr,
                                                      const cplx<T> *tw, unsigned gmask)
{
    fft_group<P, -1, FFT_HALF_IN>(v, t, scr, tw, gmask);
    packed_col_scale<P, T>(v, c, Ghat, t, scr, gmask);
}

// Rows < D of the inverse-transformed packed pair back to the two real columns.
template <int P, typename T>
__device__ __forceinline__ void packed_col_store(const cplx<T> *v, bool active, int D, cplx<T> *col, int t)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS;
    if (!active) return;
#pragma unroll
    for (int o = 0; o < R1 / 2; ++o) {
        const int y = t + G * o;
        if (y < D) {
            col[(long long)y * RS] = {v[o].x, T(0)};
            col[(long long)y * RS + P / 2] = {v[o].y, T(0)};
        }
    }
}

// Loads and stores of a column task of either kind (pk: the packed pair).
template <int P, typename T>
__device__ __forceinline__ void col_load_kind(cplx<T> *v, const cplx<T> *col, bool pk, int kx, int D, int t,
                                              bool active)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS;
    if (pk) {
#pragma unroll
        for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
#pragma unroll
        for (int o = 0; o < R1 / 2; ++o) {
            const int y = t + G * o;
            if (active && y < D) v[o] = {col[(long long)y * RS].x, col[(long long)y * RS + P / 2].x};
        }
    } else {
        col_load<P>(v, col + kx, D, t, active);
    }
}
template <int P, typename T>
__device__ __forceinline__ void col_store_kind(const cplx<T> *v, cplx<T> *col, bool pk, int kx, int D, int t,
                                               bool active)
{
    if (pk) packed_col_store<P, T>(v, active, D, col, t);
    else col_store<P>(v, col + kx, D, t, active);
}

// Column task q = 0..P/2-1: q = 0 is the packed pair of real columns kx = 0
// and kx = P/2, q >= 1 is column kx = q.  Both kinds run the same transform
// calls (x and y, then z), and only the loads, the spectral step and the
// stores differ, so that the groups of one warp never run the transforms of
// the two kinds one after the other.
template <int P, typename T>
__device__ __forceinline__ void col_task(int q, bool active, int D, cplx<T> *spec, long long cstride,
                                         const T *Ghat, int t, int lane, cplx<T> *scr, const cplx<T> *tw,
                                         unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int R1 = Gm::R1;
    const bool pk = q == 0;
    const int kx = pk ? 0 : (active ? q : 1);   // idle groups still run the transforms; keep their table reads in range
    cplx<T> vx[R1], vy[R1];
    col_load_kind<P, T>(vx, spec, pk, kx, D, t, active);
    col_load_kind<P, T>(vy, spec + cstride, pk, kx, D, t, active);
    fft_group<P, -1, FFT_HALF_IN>(vx, t, scr, tw, gmask);
    fft_group<P, -1, FFT_HALF_IN>(vy, t, scr, tw, gmask);
    if (pk) {   // G_xy vanishes on both real columns
        packed_col_scale<P, T>(vx, 0, Ghat, t, scr, gmask);
        packed_col_scale<P, T>(vy, 1, Ghat, t, scr, gmask);
    } else {
        col_multiply<P>(vx, vy, Ghat, kx, t);
    }
    fft_group<P, +1, FFT_HALF_OUT>(vx, t, scr, tw, gmask);
    fft_group<P, +1, FFT_HALF_OUT>(vy, t, scr, tw, gmask);
    col_store_kind<P, T>(vx, spec, pk, kx, D, t, active);
    col_store_kind<P, T>(vy, spec + cstride, pk, kx, D, t, active);
    cplx<T> vz[R1];
    col_load_kind<P, T>(vz, spec + 2 * cstride, pk, kx, D, t, active);
    fft_group<P, -1, FFT_HALF_IN>(vz, t, scr, tw, gmask);
    if (pk) packed_col_scale<P, T>(vz, 2, Ghat, t, scr, gmask);
    else col_multiply_z<P>(vz, Ghat, kx, t);
    fft_group<P, +1, FFT_HALF_OUT>(vz, t, scr, tw, gmask);
    col_store_kind<P, T>(vz, spec + 2 * cstride, pk, kx, D, t, active);
}

// ---------------------------------------------------------------- row inv

// Rows of row task q (q < D: the xy row y0 = q; else the z pair y0 = 2(q-D),
// y0 + 1) in the spectrum buffer: rA holds the spectrum of the row that ends in
// the real part, rB (if hasB) the one that ends in the imaginary part.
template <int P, typename T>
__device__ __forceinline__ void row_task_rows(int q, int D, cplx<T> *spec, long long cstride, cplx<T> *&rA,
                                              cplx<T> *&rB, bool &hasB)
{
    constexpr int RS = SpecGeom<P>::RS;
    const bool isxy = q < D;
    const int y0 = isxy ? q : 2 * (q - D);
    const int y1 = y0 + 1;
    hasB = isxy || (y1 < D);
    rA = isxy ? spec + (long long)y0 * RS : spec + 2 * cstride + (long long)y0 * RS;
    rB = isxy ? spec + cstride + (long long)y0 * RS : spec + 2 * cstride + (long long)y1 * RS;
}

// Inverse transform of row task q into the group's registers: afterwards the
// real parts of v[o], o < R1/2, are row A at x = t + G o and the imaginary
// parts row B.
// HALF_LOAD: read only the stored half rows k <= P/2 and take the mirrored
// entries k > P/2 from the group's scratch (for spectra in global memory,
// where each load is a round trip to L2; on chip the direct reads are cheaper).
template <int P, typename T, bool HALF_LOAD = false>
__device__ __forceinline__ void row_inv_fft(cplx<T> *v, bool active, const cplx<T> *rA, const cplx<T> *rB, bool hasB,
                                            int t, cplx<T> *scr, const cplx<T> *tw, unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1;
    if constexpr (HALF_LOAD) {
        static_assert(Gm::SCRATCH >= P + 2, "scratch holds both half rows");
        constexpr int KB = P / 2 + 1;   // B's half row starts here in the scratch
        constexpr int OH = R1 / 2 + 1;  // registers holding k <= P/2
        // every load first, so that all of them are in flight at once
        cplx<T> a[OH], b[OH];
#pragma unroll
        for (int o = 0; o < OH; ++o) {
            const int k = t + G * o;
            a[o] = b[o] = {T(0), T(0)};
            if (active && k <= P / 2) {
                a[o] = rA[k];
                if (hasB) b[o] = rB[k];
            }
        }
#pragma unroll
        for (int o = 0; o < OH; ++o) {
            const int k = t + G * o;
            if (k <= P / 2) {
                scr[k] = a[o];
                scr[KB + k] = b[o];
                v[o] = {a[o].x - b[o].y, a[o].y + b[o].x};
            }
        }
        __syncwarp(gmask);
#pragma unroll
        for (int o = 0; o < R1; ++o) {
            const int k = t + G * o;
            if (k > P / 2) {
                const cplx<T> a = scr[P - k], b = scr[KB + P - k];
                v[o] = {a.x + b.y, -a.y + b.x};   // conj(a) + i conj(b)
            }
        }
        __syncwarp(gmask);
    } else {
#pragma unroll
        for (int o = 0; o < R1; ++o) {
            const int k = t + G * o;
            const bool up = k <= P / 2;
            const int kk = up ? k : P - k;
            cplx<T> a = {T(0), T(0)}, b = {T(0), T(0)};
            if (active) {
                a = rA[kk];
                if (hasB) b = rB[kk];
            }
            if (!up) { a.y = -a.y; b.y = -b.y; }
            v[o] = {a.x - b.y, a.y + b.x};
        }
    }
    fft_group<P, +1, FFT_HALF_OUT>(v, t, scr, tw, gmask);
}

template <int P, typename T, bool HALF_LOAD = false>
__device__ __forceinline__ void row_inv_task(int q, bool active, int D, cplx<T> *spec, long long cstride, int t,
                                             cplx<T> *scr, const cplx<T> *tw, unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1;
    cplx<T> *rA, *rB;
    bool hasB;
    row_task_rows<P, T>(q, D, spec, cstride, rA, rB, hasB);
    cplx<T> v[R1];
    row_inv_fft<P, T, HALF_LOAD>(v, active, rA, rB, hasB, t, scr, tw, gmask);
    if (!active) return;
    T *oA = reinterpret_cast<T *>(rA), *oB = reinterpret_cast<T *>(rB);
#pragma unroll
    for (int o = 0; o < R1 / 2; ++o) {
        const int x = t + G * o;
        if (x < D) {
            oA[x] = v[o].x;
            if (hasB) oB[x] = v[o].y;
        }
    }
}

// ------------------------------------------------- half-length real rows

// One real row per task, as a transform of half the length (for P = 128,
// where the P/2-point transform runs on groups of the same width): 3D tasks
// of half the work each instead of D + D/2 paired ones, so that the row
// passes divide over the CTA's groups in finer steps.  With M = P/2 and
// W = exp(-2 pi i / P):
//   forward: z[n] = x[2n] + i x[2n+1] (n < M), Z = FFT_M(z),
//            X[k] = (Z[k] + conj Z[M-k])/2 - i W^k (Z[k] - conj Z[M-k])/2,
//            k = 0..M (X[M] = Re Z[0] - Im Z[0]);
//   inverse: Z[k] = (X[k] + conj X[M-k]) + i W^-k (X[k] - conj X[M-k]),
//            z = IFFT_M(Z), x[2n] = Re z[n], x[2n+1] = Im z[n]
// (both unnormalised, as the paired transforms).  twP is the P-point table
// [R1][G] of the groups' own transforms: its even rows are the M-point one's,
// and its row 1 holds W^t.
template <int P> struct HalfRows { static constexpr bool on = false; };
template <> struct HalfRows<128> { static constexpr bool on = FFTGeom<64>::G == FFTGeom<128>::G; };

// Forward: the real row x (x[i], i < D; zero beyond) to its half spectrum:
// X[k] for k = t + G o (k < M) left in v[o], X[M] (real) in xm on lane t = 0.
template <int P, typename T>
__device__ __forceinline__ void row_fwd_half_spectrum(bool active, const T *x, int D, cplx<T> *v, T &xm, int t,
                                                      cplx<T> *scr, const cplx<T> *twP, unsigned gmask)
{
    constexpr int M = P / 2, G = FFTGeom<M>::G, R1 = FFTGeom<M>::R1;
#pragma unroll
    for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
#pragma unroll
    for (int o = 0; o < R1 / 2; ++o) {   // D <= M: the upper half of z is zero padding
        const int n = t + G * o;
        if (active) {
            const T a = 2 * n < D ? x[2 * n] : T(0), b = 2 * n + 1 < D ? x[2 * n + 1] : T(0);
            v[o] = {a, b};
        }
    }
    fft_group<M, -1, FFT_HALF_IN, 2 * G>(v, t, scr, twP, gmask);
    mirror_put<M>(v, scr, t);
    __syncwarp(gmask);
    const cplx<T> w1 = twP[G + t];   // W^t
    const T h = T(0.5);
    xm = v[0].x - v[0].y;            // X[M] = Re Z[0] - Im Z[0] (used on lane 0)
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        const int k = t + G * o;
        const cplx<T> z = v[o], zm = mirror_get<M>(scr, k);
        const cplx<T> e = {h * (z.x + zm.x), h * (z.y - zm.y)};   // (Z[k] + conj Z[M-k]) / 2
        const cplx<T> d = {h * (z.x - zm.x), h * (z.y + zm.y)};   // (Z[k] - conj Z[M-k]) / 2
        const cplx<T> wd = cmul(twid<-1>(w1, o, P / G), d);        // W^k d, W^k = W^t W^(G o)
        v[o] = {e.x + wd.y, e.y - wd.x};                            // e - i W^k d
    }
    __syncwarp(gmask);
}

// Forward, stored: X[0..M] of the real row to dst.
template <int P, typename T>
__device__ __forceinline__ void row_fwd_half(bool active, const T *x, int D, cplx<T> *dst, int t, cplx<T> *scr,
                                             const cplx<T> *twP, unsigned gmask)
{
    constexpr int M = P / 2, G = FFTGeom<M>::G, R1 = FFTGeom<M>::R1;
    cplx<T> v[R1];
    T xm;
    row_fwd_half_spectrum<P, T>(active, x, D, v, xm, t, scr, twP, gmask);
    if (active) {
#pragma unroll
        for (int o = 0; o < R1; ++o) dst[t + G * o] = v[o];
        if (t == 0) dst[M] = {xm, T(0)};
    }
}

// Inverse: the half spectrum X[0..M] in src to the real row, x[i] for i < D
// written to out (which may alias src: every read precedes the writes).
template <int P, typename T>
__device__ __forceinline__ void row_inv_half(bool active, const cplx<T> *src, int D, T *out, int t, cplx<T> *scr,
                                             const cplx<T> *twP, unsigned gmask)
{
    constexpr int M = P / 2, G = FFTGeom<M>::G, R1 = FFTGeom<M>::R1;
    cplx<T> v[R1];
    const cplx<T> w1 = twP[G + t];
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        const int k = t + G * o;
        cplx<T> a = {T(0), T(0)}, b = {T(0), T(0)};
        if (active) {
            a = src[k];
            b = src[M - k];
        }
        const cplx<T> s = {a.x + b.x, a.y - b.y};                     // X[k] + conj X[M-k]
        const cplx<T> d = {a.x - b.x, a.y + b.y};                     // X[k] - conj X[M-k]
        const cplx<T> wk = twid<-1>(w1, o, P / G);                    // W^k
        const cplx<T> wd = {wk.x * d.x + wk.y * d.y, wk.x * d.y - wk.y * d.x};   // W^-k d
        v[o] = {s.x - wd.y, s.y + wd.x};                                // s + i W^-k d
    }
    fft_group<M, +1, FFT_HALF_OUT, 2 * G>(v, t, scr, twP, gmask);
    if (active) {
#pragma unroll
        for (int o = 0; o < R1 / 2; ++o) {
            const int n = t + G * o;
            if (2 * n < D) out[2 * n] = v[o].x;
            if (2 * n + 1 < D) out[2 * n + 1] = v[o].y;
        }
    }
}

// --------------------------------------------------------- group plumbing

// A thread's FFT group: GROUPS_PER_WARP groups of G consecutive lanes per
// warp, numbered warp by warp.  When G does not divide 32 (G = 10) the last
// lanes of each warp belong to no group: valid is false there, and they take
// no task and touch no scratch.
template <int P> struct GroupId {
    int group, t, lane;
    unsigned gmask;
    bool valid;
    __device__ __forceinline__ GroupId(int tid)
    {
        constexpr int G = FFTGeom<P>::G, GPW = FFTGeom<P>::GROUPS_PER_WARP;
        lane = tid & 31;
        if constexpr (FFTGeom<P>::POW2) {
            valid = true;
            group = tid / G;
            t = tid & (G - 1);
            gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
        } else {
            const int gw = lane / G;
            valid = gw < GPW;
            group = (tid >> 5) * GPW + gw;
            t = lane - gw * G;
            gmask = ((1u << G) - 1u) << (gw * G);
        }
    }
};

// FFT groups of a block of NT threads (whole warps).
template <int P, int NT> constexpr int groups_per_block() { return NT / 32 * FFTGeom<P>::GROUPS_PER_WARP; }

// Fill the [R1][G] twiddle table exp(-2 pi i t k1 / P) from the length-P table.
template <int P, typename T>
__device__ __forceinline__ void load_twiddles(cplx<T> *tw, const cplx<T> *twP, int tid, int nthreads)
{
    constexpr int G = FFTGeom<P>::G, R1 = FFTGeom<P>::R1;
    for (int i = tid; i < R1 * G; i += nthreads) {
        const int k1 = i / G, t = i % G;
        tw[i] = twP[(k1 * t) % P];
    }
}

}  // namespace nd
