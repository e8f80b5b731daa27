// nd_aux.cu -- once-per-geometry spectral kernel build and the small
// per-replica kernels: analytic vortex profile, vortex-core estimator, <m>,
// precision conversion and finiteness check.
#include <math.h>

#include "nd_common.cuh"
#include "nd_kernels.h"

namespace nd {

// --------------------------------------------------- spectral kernel build

// a^2 G at cell displacement (dx, dy) >= 0, lengths in units of a (Section
// II.B): G_zz = -l/(2 pi r s (s+r)), G_xx = l/(2 pi r^4) (x^2/s - y^2/(s+r)),
// G_xy = l/(2 pi r^4) (2s+r)/(s+r) x y/s, s = sqrt(r^2 + l^2); the origin holds
// the cell self terms -Nx, -Nx, 0, -Nz.
__global__ void k_green_quarter(int D, double l, double Nx, double Nz, double *Gq)
{
    const int n = D * D;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int dy = i / D, dx = i - dy * D;
        double xx, yy, xy, zz;
        if (dx == 0 && dy == 0) {
            xx = -Nx; yy = -Nx; xy = 0.0; zz = -Nz;
        } else {
            const double x = dx, y = dy, r2 = x * x + y * y, r = sqrt(r2), s = sqrt(r2 + l * l);
            const double pre = l / (2.0 * M_PI * r2 * r2);
            xx = pre * (x * x / s - y * y / (s + r));
            yy = pre * (y * y / s - x * x / (s + r));
            xy = pre * ((2.0 * s + r) / (s + r)) * (x * y / s);
            zz = -l / (2.0 * M_PI * r * s * (s + r));
        }
        Gq[i] = xx; Gq[n + i] = yy; Gq[2 * n + i] = xy; Gq[3 * n + i] = zz;
    }
}

// Thickness derivative of the table above, d(a^2 G)/dl at fixed displacement
// (lengths in units of a), and of the self terms:
//   dN_z/dl = r_o (r_o - q)/(q l^2),  dN_x/dl = r_o (q - r_o)/(2 q l^2),  q = sqrt(l^2 + r_o^2).
__global__ void k_green_quarter_dl(int D, double l, double dNx, double dNz, double *Gq)
{
    const int n = D * D;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int dy = i / D, dx = i - dy * D;
        double xx, yy, xy, zz;
        if (dx == 0 && dy == 0) {
            xx = -dNx; yy = -dNx; xy = 0.0; zz = -dNz;
        } else {
            const double x = dx, y = dy, r2 = x * x + y * y, r = sqrt(r2), s = sqrt(r2 + l * l);
            const double ds = l / s, r4 = r2 * r2;
            // G_xx = l/(2 pi r^4) (x^2/s - y^2/(s+r))
            xx = (1.0 / (2.0 * M_PI * r4)) * ((x * x / s - y * y / (s + r)) + l * (-x * x * ds / (s * s) + y * y * ds / ((s + r) * (s + r))));
            yy = (1.0 / (2.0 * M_PI * r4)) * ((y * y / s - x * x / (s + r)) + l * (-y * y * ds / (s * s) + x * x * ds / ((s + r) * (s + r))));
            // G_xy = g(l) x y / (2 pi r^4), g = l (2s+r)/((s+r) s)
            const double den = (s + r) * s;
            const double g = (2.0 * s + r) / den + l * ds * (2.0 * (s + r) * s - (2.0 * s + r) * (2.0 * s + r)) / (den * den);
            xy = g * x * y / (2.0 * M_PI * r4);
            // G_zz = -f(l)/(2 pi r), f = l/(s (s+r))
            const double f = (s * (s + r) - l * ds * (2.0 * s + r)) / (den * den);
            zz = -f / (2.0 * M_PI * r);
        }
        Gq[i] = xx; Gq[n + i] = yy; Gq[2 * n + i] = xy; Gq[3 * n + i] = zz;
    }
}

__global__ void k_trig_table(int P, double *cs)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * k / P, &s, &c);
        cs[2 * k] = c; cs[2 * k + 1] = s;
    }
}

// Pass 1 over dx: T1[c][dy][kx] = sum_dx w(dx) Gq[c][dy][dx] f_c(2 pi kx dx / P),
// f = cos for the even components (xx, yy, zz), sin for the odd one (xy),
// w = 1 at dx = 0 and 2 otherwise (the two signs of dx folded together).
__global__ void k_ghat_pass1(int P, int D, const double *Gq, const double *cs, double *T1)
{
    const int KH = P / 2 + 1, n = 4 * D * KH;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int kx = i % KH, dy = (i / KH) % D, c = i / (KH * D);
        const double *g = Gq + (size_t)c * D * D + (size_t)dy * D;
        const double *fc = cs + (c == 2 ? 1 : 0);
        double acc = g[0] * fc[0];
        // phase index kx*dx mod P, advanced by kx per term
        for (int dx = 1, k = kx; dx < D; ++dx, k = (k + kx >= P) ? k + kx - P : k + kx) acc += 2.0 * g[dx] * fc[2 * k];
        T1[i] = acc;
    }
}

// Pass 2 over dy and final assembly into [kx][ky][4], followed by the same
// values component-major, [4][kx][ky]:
//   Ghat_c = s_c sum_dy w(dy) T1[c][dy][kx] f_c(2 pi ky dy / P), s_xy = -1,
//   diagonal: (c Ghat + 2 cos(2 pi kx/P) + 2 cos(2 pi ky/P)) / P^2 (exchange folded in),
//   xy:       c Ghat_xy / P^2.
__global__ void k_ghat_pass2(int P, int D, double cfac, const double *T1, const double *cs, double *G64, float *G32,
                             int with_exchange)
{
    const int KH = P / 2 + 1, n = KH * KH;
    const double inv = 1.0 / ((double)P * (double)P);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int kx = i / KH, ky = i % KH;
        double v[4];
        for (int c = 0; c < 4; ++c) {
            const double *t1 = T1 + (size_t)c * D * KH + kx;
            const double *fc = cs + (c == 2 ? 1 : 0);
            double acc = t1[0] * fc[0];
            for (int dy = 1, k = ky; dy < D; ++dy, k = (k + ky >= P) ? k + ky - P : k + ky)
                acc += 2.0 * t1[(size_t)dy * KH] * fc[2 * k];
            v[c] = (c == 2) ? -acc : acc;
        }
        const double kex = with_exchange ? 2.0 * cs[2 * kx] + 2.0 * cs[2 * ky] : 0.0;
        const double o[4] = {(cfac * v[0] + kex) * inv, (cfac * v[1] + kex) * inv, cfac * v[2] * inv,
                             (cfac * v[3] + kex) * inv};
        for (int c = 0; c < 4; ++c) {
            G64[(size_t)i * 4 + c] = o[c];
            if (G32) G32[(size_t)i * 4 + c] = (float)o[c];
            // the same values component-major after the interleaved block
            G64[(size_t)(4 + c) * n + i] = o[c];
            if (G32) G32[(size_t)(4 + c) * n + i] = (float)o[c];
        }
    }
}

size_t build_ghat_work_doubles(int P, int D) { return (size_t)4 * D * D + (size_t)4 * D * (P / 2 + 1) + 2 * (size_t)P; }

cudaError_t build_ghat(int P, int D, double l, double Nx, double Nz, double cfac, const double *Gq_dev, double *G64,
                       float *G32, double *work, cudaStream_t st)
{
    double *Gq = work, *T1 = Gq + (size_t)4 * D * D, *cs = T1 + (size_t)4 * D * (P / 2 + 1);
    if (Gq_dev) {
        cudaError_t e = cudaMemcpyAsync(Gq, Gq_dev, sizeof(double) * 4 * D * D, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    } else {
        k_green_quarter<<<(D * D + 255) / 256, 256, 0, st>>>(D, l, Nx, Nz, Gq);
    }
    k_trig_table<<<(P + 255) / 256, 256, 0, st>>>(P, cs);
    const int KH = P / 2 + 1;
    k_ghat_pass1<<<(4 * D * KH + 255) / 256, 256, 0, st>>>(P, D, Gq, cs, T1);
    k_ghat_pass2<<<(KH * KH + 127) / 128, 128, 0, st>>>(P, D, cfac, T1, cs, G64, G32, 1);
    return cudaGetLastError();
}

cudaError_t build_ghat_dl(int P, int D, double l, double dNx, double dNz, double cfac, double *GL64, double *work,
                          cudaStream_t st)
{
    double *Gq = work, *T1 = Gq + (size_t)4 * D * D, *cs = T1 + (size_t)4 * D * (P / 2 + 1);
    k_green_quarter_dl<<<(D * D + 255) / 256, 256, 0, st>>>(D, l, dNx, dNz, Gq);
    k_trig_table<<<(P + 255) / 256, 256, 0, st>>>(P, cs);
    const int KH = P / 2 + 1;
    k_ghat_pass1<<<(4 * D * KH + 255) / 256, 256, 0, st>>>(P, D, Gq, cs, T1);
    k_ghat_pass2<<<(KH * KH + 127) / 128, 128, 0, st>>>(P, D, cfac, T1, cs, GL64, nullptr, 0);
    return cudaGetLastError();
}

// -------------------------------------------------------- vortex profile

// Planar q = +1 vortex at X0 (Section IV) with a seeded core:
// phi = atan2(y - y0, x - x0) + chirality pi/2, m_z = polarity exp(-rho^2/lambda^2).
template <typename T>
__global__ void k_init_vortex(const Replica *reps, const int *work, T *ybase, const double *X0, const int *pc,
                              double lam)
{
    const int ridx = work[blockIdx.y];
    const Replica r = reps[ridx];
    const int D = r.D, DD = D * D;
    const long long cs = (long long)D * r.Dpad;
    const double x0 = X0[2 * ridx], y0 = X0[2 * ridx + 1];
    const int pol = pc[2 * ridx], chi = pc[2 * ridx + 1];
    T *y = ybase + r.state_off;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < DD; cell += gridDim.x * blockDim.x) {
        const int j = cell / D, i = cell - j * D;
        const long long si = (long long)j * r.Dpad + i;
        double mx = 0, my = 0, mz = 0;
        if (r.mask[cell]) {
            const double x = i - 0.5 * (D - 1), yy = j - 0.5 * (D - 1);
            const double rho2 = (x - x0) * (x - x0) + (yy - y0) * (yy - y0);
            mz = pol * exp(-rho2 / (lam * lam));
            const double phi = atan2(yy - y0, x - x0) + chi * 0.5 * M_PI;
            const double sp = sqrt(1.0 - mz * mz);
            double sn, cn;
            sincos(phi, &sn, &cn);
            mx = sp * cn; my = sp * sn;
        }
        y[si] = (T)mx; y[cs + si] = (T)my; y[2 * cs + si] = (T)mz;
    }
    // cells of the padded columns stay untouched
}

cudaError_t launch_init_vortex(int prec, const Replica *reps, const int *work, int nwork, int maxD, void *y,
                               const double *X0, const int *pc, double lam, cudaStream_t st)
{
    dim3 g((maxD * maxD + 255) / 256, nwork);
    if (prec == ND_PREC_FP64) k_init_vortex<double><<<g, 256, 0, st>>>(reps, work, (double *)y, X0, pc, lam);
    else k_init_vortex<float><<<g, 256, 0, st>>>(reps, work, (float *)y, X0, pc, lam);
    return cudaGetLastError();
}

// ------------------------------------------------------------ vortex core

// Core position estimator (Section IV) in two kernels.  The plaquette
// windings and the m_z^2 corner sums are evaluated in double precision with
// no fused multiply-adds, in the same order as the CPU reference, so both
// take the same integer decisions from the same inputs.
//   k_core_scan: grid (nblk, replicas), each CTA scans a strided share of the
//     plaquettes for the winding +1 one with the largest corner sum (lowest
//     index on ties) and writes its candidate;
//   k_core_finish: one CTA per replica picks the best candidate (same rule)
//     and forms the m_z^2-weighted centroid over the disk cells within
//     4 lambda_ex of it, visiting only the bounding box of that circle.
template <typename T> struct CoreAt {
    const T *y;
    long long cs;
    int D, Dpad;
    __device__ __forceinline__ double operator()(int cell, int c) const
    {
        const int j = cell / D, i = cell - j * D;
        return (double)y[c * cs + (long long)j * Dpad + i];
    }
};

template <typename T>
__global__ void __launch_bounds__(256) k_core_scan(const Replica *reps, const int *work, const T *ybase, double *part,
                                                   int nblk)
{
    __shared__ double sw[256];
    __shared__ int si_[256];
    const int ridx = work[blockIdx.y];
    const Replica r = reps[ridx];
    const int D = r.D, tid = threadIdx.x;
    const CoreAt<T> at{ybase + r.state_off, (long long)D * r.Dpad, D, r.Dpad};
    double bw = -1.0;
    int bi = 0x7fffffff;
    const int np = (D - 1) * (D - 1);
    for (int p = blockIdx.x * 256 + tid; p < np; p += nblk * 256) {
        const int j = p / (D - 1), i = p - j * (D - 1);
        const int t = j * D + i;
        if (!(r.mask[t] && r.mask[t + 1] && r.mask[t + D] && r.mask[t + D + 1])) continue;
        const int c[4] = {t, t + 1, t + D + 1, t + D};
        // The winding is decided in double precision.  A single-precision pass
        // settles every plaquette whose angle sum lies within a quarter turn
        // of a multiple of 2 pi (its error, ~1e-6 rad, is far below that
        // margin, so the double sum rounds to the same integer); only the
        // others, and plaquettes with an in-plane component too small for
        // single-precision products, are summed again in double.
        float sf = 0.0f, amin = 1.0f;
        for (int q = 0; q < 4; ++q) {
            const int p0 = c[q], p1 = c[(q + 1) & 3];
            const float ax = (float)at(p0, 0), ay = (float)at(p0, 1), bx = (float)at(p1, 0), by = (float)at(p1, 1);
            sf += atan2f(ax * by - ay * bx, ax * bx + ay * by);
            amin = fminf(amin, ax * ax + ay * ay);
        }
        const float kf = sf * (float)(0.5 / M_PI);
        long long wind;
        if (amin > 1e-12f && fabsf(kf - rintf(kf)) < 0.25f) {
            wind = (long long)rintf(kf);
        } else {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) {
                const int p0 = c[q], p1 = c[(q + 1) & 3];
                const double ax = at(p0, 0), ay = at(p0, 1), bx = at(p1, 0), by = at(p1, 1);
                const double cr = __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
                const double dt = __dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by));
                s = __dadd_rn(s, atan2(cr, dt));
            }
            wind = llround(s / (2.0 * M_PI));
        }
        if (wind != 1) continue;
        const double z0 = at(t, 2), z1 = at(t + 1, 2), z2 = at(t + D, 2), z3 = at(t + D + 1, 2);
        double w = __dmul_rn(z0, z0);
        w = __dadd_rn(w, __dmul_rn(z1, z1));
        w = __dadd_rn(w, __dmul_rn(z2, z2));
        w = __dadd_rn(w, __dmul_rn(z3, z3));
        if (w > bw || (w == bw && t < bi)) { bw = w; bi = t; }
    }
    sw[tid] = bw; si_[tid] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) {
            const double w2 = sw[tid + o];
            const int i2 = si_[tid + o];
            if (w2 > sw[tid] || (w2 == sw[tid] && i2 < si_[tid])) { sw[tid] = w2; si_[tid] = i2; }
        }
        __syncthreads();
    }
    if (tid == 0) {
        double *o = part + 2 * ((size_t)ridx * nblk + blockIdx.x);
        o[0] = sw[0];
        o[1] = (double)si_[0];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_core_finish(const Replica *reps, const int *work, const T *ybase,
                                                     const double *part, int nblk, double rc2, double *out)
{
    __shared__ double sx[3][8];
    __shared__ int best_s;
    __shared__ double bw_s;
    const int ridx = work[blockIdx.x];
    const Replica r = reps[ridx];
    const int D = r.D, tid = threadIdx.x;
    const CoreAt<T> at{ybase + r.state_off, (long long)D * r.Dpad, D, r.Dpad};
    if (tid == 0) {
        double bw = -1.0;
        int bi = 0x7fffffff;
        for (int b = 0; b < nblk; ++b) {
            const double w = part[2 * ((size_t)ridx * nblk + b)];
            const int i = (int)part[2 * ((size_t)ridx * nblk + b) + 1];
            if (w > bw || (w == bw && i < bi)) { bw = w; bi = i; }
        }
        best_s = bi;
        bw_s = bw;
    }
    __syncthreads();
    const int best = best_s;
    const bool found = bw_s >= 0.0 && best != 0x7fffffff;
    double a0 = 0, a1 = 0, a2 = 0;
    if (found) {
        const int bj = best / D, bii = best - bj * D;
        const double cx = bii + 0.5 - 0.5 * (D - 1), cy = bj + 0.5 - 0.5 * (D - 1);
        const int rc = (int)ceil(sqrt(rc2)) + 1;
        const int i0 = max(0, bii - rc), i1 = min(D - 1, bii + 1 + rc), j0 = max(0, bj - rc), j1 = min(D - 1, bj + 1 + rc);
        const int w = i1 - i0 + 1, nbox = w * (j1 - j0 + 1);
        for (int k = tid; k < nbox; k += 256) {
            const int j = j0 + k / w, i = i0 + k % w, cell = j * D + i;
            if (!r.mask[cell]) continue;
            const double x = i - 0.5 * (D - 1), yy = j - 0.5 * (D - 1);
            const double dx = x - cx, dy = yy - cy;
            if (dx * dx + dy * dy >= rc2) continue;
            const double z = at(cell, 2), wz = z * z;
            a0 += wz; a1 += wz * x; a2 += wz * yy;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if ((tid & 31) == 0) { sx[0][tid >> 5] = a0; sx[1][tid >> 5] = a1; sx[2][tid >> 5] = a2; }
    __syncthreads();
    if (tid == 0) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int wv = 0; wv < 8; ++wv) { s0 += sx[0][wv]; s1 += sx[1][wv]; s2 += sx[2][wv]; }
        double *o = out + 4 * ridx;
        if (found && s0 > 0.0) { o[0] = s1 / s0; o[1] = s2 / s0; o[2] = 0.0; }
        else { o[0] = 0.0; o[1] = 0.0; o[2] = 1.0; }
        o[3] = found ? (double)best : -1.0;
    }
}

int core_scan_blocks(int D)
{
    const int np = (D - 1) * (D - 1);
    int n = np / 4096;
    return n < 1 ? 1 : (n > kCoreMaxBlocks ? kCoreMaxBlocks : n);
}

cudaError_t launch_vortex_core(int prec, const Replica *reps, const int *work, int nwork, int maxD, const void *y,
                               double rc2, double *part, double *out, cudaStream_t st)
{
    const int nblk = core_scan_blocks(maxD);
    dim3 g(nblk, nwork);
    if (prec == ND_PREC_FP64) {
        k_core_scan<double><<<g, 256, 0, st>>>(reps, work, (const double *)y, part, nblk);
        k_core_finish<double><<<nwork, 256, 0, st>>>(reps, work, (const double *)y, part, nblk, rc2, out);
    } else {
        k_core_scan<float><<<g, 256, 0, st>>>(reps, work, (const float *)y, part, nblk);
        k_core_finish<float><<<nwork, 256, 0, st>>>(reps, work, (const float *)y, part, nblk, rc2, out);
    }
    return cudaGetLastError();
}

// Advance the noise-step counter of every replica (graph replays continue the
// Philox stream where the previous replay stopped).
__global__ void k_advance_steps(Replica *reps, int n, long long steps)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) reps[r].step0 += (unsigned long long)steps;
}

cudaError_t launch_advance_steps(Replica *reps, int n, long long steps, cudaStream_t s)
{
    k_advance_steps<<<(n + 127) / 128, 128, 0, s>>>(reps, n, steps);
    return cudaGetLastError();
}

// ------------------------------------------------------------ statistics

// Per-replica accumulation of the core statistics of Sec. V.C in double
// precision with 64-bit histogram counts: samples where a vortex was found
// add r = |r_c| to <x>, <y>, <r^2> and to the r histogram; consecutive found
// samples add the speed V = |r_c(t) - r_c(t - dt)|/dt to <V^2> and the V
// histogram.  One thread per replica; core holds the estimator output in
// cell units ([4] per replica: x, y, status, plaquette).
__global__ void k_stats_update(const int *work, int nwork, const double *core, const double *a_of_rep,
                               StatsAcc *st, unsigned long long *hr, unsigned long long *hv, int rb, int vb,
                               double r_max, double v_max, double dt)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwork) return;
    const int r = work[w];
    const double *c = core + 4 * r;
    StatsAcc &S = st[r];
    if (c[2] != 0.0) {
        S.no_vortex += 1.0;
        S.have_prev = 0;
        return;
    }
    const double a = a_of_rep[r];
    const double x = c[0] * a, y = c[1] * a, rr = sqrt(x * x + y * y);
    S.n += 1.0; S.sx += x; S.sy += y; S.sr2 += x * x + y * y;
    const long long br = (long long)floor(rr / r_max * rb);
    if (br >= 0 && br < rb) hr[(size_t)r * rb + br] += 1ull;
    if (S.have_prev) {
        const double vx = (x - S.px) / dt, vy = (y - S.py) / dt, v = sqrt(vx * vx + vy * vy);
        S.nv += 1.0; S.sv2 += v * v;
        const long long bv = (long long)floor(v / v_max * vb);
        if (bv >= 0 && bv < vb) hv[(size_t)r * vb + bv] += 1ull;
    }
    S.px = x; S.py = y; S.have_prev = 1;
}

cudaError_t launch_stats_update(const int *work, int nwork, const double *core, const double *a_of_rep, StatsAcc *st,
                                unsigned long long *hr, unsigned long long *hv, int rb, int vb, double r_max,
                                double v_max, double dt, cudaStream_t s)
{
    k_stats_update<<<(nwork + 127) / 128, 128, 0, s>>>(work, nwork, core, a_of_rep, st, hr, hv, rb, vb, r_max, v_max, dt);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- <m>

template <typename T>
__global__ void __launch_bounds__(256) k_mean_m(const Replica *reps, const int *work, const T *ybase, double *out)
{
    __shared__ double sx[4][8];
    const int ridx = work[blockIdx.x];
    const Replica r = reps[ridx];
    const int D = r.D, tid = threadIdx.x;
    const long long cs = (long long)D * r.Dpad;
    const T *y = ybase + r.state_off;
    double a0 = 0, a1 = 0, a2 = 0, n = 0;
    for (int cell = tid; cell < D * D; cell += 256) {
        if (!r.mask[cell]) continue;
        const int j = cell / D, i = cell - j * D;
        const long long si = (long long)j * r.Dpad + i;
        a0 += (double)y[si]; a1 += (double)y[cs + si]; a2 += (double)y[2 * cs + si]; n += 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if ((tid & 31) == 0) { sx[0][tid >> 5] = a0; sx[1][tid >> 5] = a1; sx[2][tid >> 5] = a2; sx[3][tid >> 5] = n; }
    __syncthreads();
    if (tid == 0) {
        double s[4] = {0, 0, 0, 0};
        for (int w = 0; w < 8; ++w) for (int c = 0; c < 4; ++c) s[c] += sx[c][w];
        for (int c = 0; c < 3; ++c) out[3 * ridx + c] = s[c] / s[3];
    }
}

cudaError_t launch_mean_m(int prec, const Replica *reps, const int *work, int nwork, const void *y, double *out,
                          cudaStream_t st)
{
    if (prec == ND_PREC_FP64) k_mean_m<double><<<nwork, 256, 0, st>>>(reps, work, (const double *)y, out);
    else k_mean_m<float><<<nwork, 256, 0, st>>>(reps, work, (const float *)y, out);
    return cudaGetLastError();
}

// ---------------------------------------------------- conversion, checks

template <typename S, typename D_>
__global__ void k_convert(const S *src, D_ *dst, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (D_)src[i];
}

cudaError_t launch_convert(int to_prec, const void *src, void *dst, size_t n, cudaStream_t st)
{
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (n == 0) return cudaSuccess;
    if (to_prec == ND_PREC_FP64) k_convert<float, double><<<blocks, 256, 0, st>>>((const float *)src, (double *)dst, n);
    else k_convert<double, float><<<blocks, 256, 0, st>>>((const double *)src, (float *)dst, n);
    return cudaGetLastError();
}

// Sets ND_DEV_NAN in *flag if any component of a cell inside a disk is not
// finite (cells outside the disks and padding columns are ignored).
// grid = (cell blocks, replicas).
template <typename T>
__global__ void k_check_finite(const Replica *reps, const int *work, const T *ybase, unsigned *flag)
{
    const Replica &r = reps[work[blockIdx.y]];
    const int D = r.D, DD = D * D;
    const long long cs = (long long)D * r.Dpad;
    bool bad = false;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < DD; cell += gridDim.x * blockDim.x) {
        if (!r.mask[cell]) continue;
        const int j = cell / D, i = cell - j * D;
        const T *y = ybase + r.state_off + (long long)j * r.Dpad + i;
        bad |= !(isfinite(y[0]) && isfinite(y[cs]) && isfinite(y[2 * cs]));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, ND_DEV_NAN);
}

cudaError_t launch_check_finite(int prec, const Replica *reps, const int *work, int nwork, int maxD, const void *y,
                                unsigned *flag, cudaStream_t st)
{
    if (nwork == 0) return cudaSuccess;
    const int cells = maxD * maxD, bx = (cells + 255) / 256 < 64 ? (cells + 255) / 256 : 64;
    dim3 g(bx, nwork);
    if (prec == ND_PREC_FP64) k_check_finite<double><<<g, 256, 0, st>>>(reps, work, (const double *)y, flag);
    else k_check_finite<float><<<g, 256, 0, st>>>(reps, work, (const float *)y, flag);
    return cudaGetLastError();
}

}  // namespace nd
