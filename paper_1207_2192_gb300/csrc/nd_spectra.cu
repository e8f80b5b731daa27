// nd_spectra.cu -- time series of the average magnetisation <m> of every
// replica, and their averaged power spectra (Sec. V: the thermal power spectra
// of <m_x>, from whose peaks the gyrotropic frequency and the higher modes
// are read).
#include "nd_phases.cuh"
#include "nd_kernels.h"

namespace nd {

ND_DEFINE_TWIDDLE_UPLOAD(upload_tw_spectra)

// <m> of every replica of a size class (double sums over the disk cells)
// written at sample index *count of its series [replica][cap][3]; samples
// beyond cap are dropped (the counter keeps counting).
template <typename T>
__global__ void __launch_bounds__(256) k_series_append(const Replica *reps, const int *work, const T *ybase,
                                                       double *series, const unsigned long long *count, int cap)
{
    __shared__ double sx[4][8];
    const int ridx = work[blockIdx.x];
    const Replica &r = reps[ridx];
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
        const unsigned long long idx = *count;
        if (idx < (unsigned long long)cap) {
            double s[4] = {0, 0, 0, 0};
            for (int w = 0; w < 8; ++w)
                for (int c = 0; c < 4; ++c) s[c] += sx[c][w];
            double *o = series + ((size_t)ridx * cap + idx) * 3;
            for (int c = 0; c < 3; ++c) o[c] = s[c] / s[3];
        }
    }
}

__global__ void k_series_advance(unsigned long long *count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *count += 1ull;
}

// Periodogram of one window: group g of the CTA takes window
// blockIdx.x * NG + g of replica blockIdx.y, component comp; the window mean
// is removed and |X_k|^2, k = 0..W/2, is written to pw[replica][window][k].
template <int W>
__global__ void __launch_bounds__(128) k_window_power(const double *__restrict__ series, int cap, int comp, int nwin,
                                                      const cplx<double> *__restrict__ twW, double *__restrict__ pw)
{
    using Gm = FFTGeom<W>;
    constexpr int G = Gm::G, R1 = Gm::R1, NG = 128 / G, NK = W / 2 + 1;
    extern __shared__ __align__(16) unsigned char ssm[];
    cplx<double> *tw = reinterpret_cast<cplx<double> *>(ssm);
    cplx<double> *scratch = tw + R1 * G;
    load_twiddles<W>(tw, twW, threadIdx.x, 128);
    __syncthreads();
    GroupId<W> gid(threadIdx.x);
    const int r = blockIdx.y, w = blockIdx.x * NG + gid.group;
    if (w >= nwin) return;   // no CTA barrier follows
    const double *x = series + ((size_t)r * cap + (size_t)w * W) * 3 + comp;
    cplx<double> v[R1];
    double s = 0.0;
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        v[o] = {x[(size_t)(gid.t + G * o) * 3], 0.0};
        s += v[o].x;
    }
    for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(gid.gmask, s, off);
    const double mean = s / W;
#pragma unroll
    for (int o = 0; o < R1; ++o) v[o].x -= mean;
    fft_group<W, -1, FFT_FULL>(v, gid.t, scratch + gid.group * Gm::SCRATCH, tw, gid.gmask);
    double *out = pw + ((size_t)r * nwin + w) * NK;
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        const int k = gid.t + G * o;
        if (k < NK) out[k] = v[o].x * v[o].x + v[o].y * v[o].y;
    }
}

// One-sided averaged periodogram: psd[r][k] = scale * (2 or 1) * mean over
// windows of pw[r][w][k] (windows summed in order).
__global__ void k_psd_reduce(const double *__restrict__ pw, int nwin, int nk, int nrep, double scale,
                             double *__restrict__ psd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrep * nk) return;
    const int r = i / nk, k = i - r * nk;
    double s = 0.0;
    for (int w = 0; w < nwin; ++w) s += pw[((size_t)r * nwin + w) * nk + k];
    const double f = (k == 0 || k == nk - 1) ? 1.0 : 2.0;
    psd[i] = scale * f * s / nwin;
}

cudaError_t launch_series_append(int prec, const Replica *reps, const int *work, int nwork, const void *y,
                                 double *series, const unsigned long long *count, int cap, cudaStream_t st)
{
    if (nwork == 0) return cudaSuccess;
    if (prec == ND_PREC_FP64)
        k_series_append<double><<<nwork, 256, 0, st>>>(reps, work, (const double *)y, series, count, cap);
    else
        k_series_append<float><<<nwork, 256, 0, st>>>(reps, work, (const float *)y, series, count, cap);
    return cudaGetLastError();
}

cudaError_t launch_series_advance(unsigned long long *count, cudaStream_t st)
{
    k_series_advance<<<1, 32, 0, st>>>(count);
    return cudaGetLastError();
}

template <int W>
static cudaError_t window_power_w(const double *series, int cap, int comp, int nwin, int nrep, const void *twW,
                                  double *pw, cudaStream_t st)
{
    using Gm = FFTGeom<W>;
    constexpr int NG = 128 / Gm::G;
    const size_t smem = sizeof(cplx<double>) * ((size_t)Gm::R1 * Gm::G + (size_t)NG * Gm::SCRATCH);
    cudaError_t e = cudaFuncSetAttribute(k_window_power<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 g((nwin + NG - 1) / NG, nrep);
    k_window_power<W><<<g, 128, smem, st>>>(series, cap, comp, nwin, (const cplx<double> *)twW, pw);
    return cudaGetLastError();
}

cudaError_t launch_window_power(int W, const double *series, int cap, int comp, int nwin, int nrep, const void *twW,
                                double *pw, cudaStream_t st)
{
    switch (W) {
    case 64: return window_power_w<64>(series, cap, comp, nwin, nrep, twW, pw, st);
    case 128: return window_power_w<128>(series, cap, comp, nwin, nrep, twW, pw, st);
    case 256: return window_power_w<256>(series, cap, comp, nwin, nrep, twW, pw, st);
    case 512: return window_power_w<512>(series, cap, comp, nwin, nrep, twW, pw, st);
    case 1024: return window_power_w<1024>(series, cap, comp, nwin, nrep, twW, pw, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_psd_reduce(const double *pw, int nwin, int nk, int nrep, double scale, double *psd, cudaStream_t st)
{
    const int n = nrep * nk;
    k_psd_reduce<<<(n + 255) / 256, 256, 0, st>>>(pw, nwin, nk, nrep, scale, psd);
    return cudaGetLastError();
}

}  // namespace nd
