// nd_dispatch.cu -- precision dispatch between the instantiation units.
#include "nd_kernels.h"

namespace nd {

cudaError_t upload_tw_fused_f32(const double *, const double *);
cudaError_t upload_tw_fused_f64(const double *, const double *);
cudaError_t upload_tw_glob_f32(const double *, const double *);
cudaError_t upload_tw_glob_f64(const double *, const double *);
cudaError_t upload_tw_spectra(const double *, const double *);
size_t fused_smem_f32(int P, int D, int Dpad, bool wbuf, int variant);
size_t fused_smem_f64(int P, int D, int Dpad, bool wbuf, int variant);
int fused_blocks_per_sm_f32(int P, int mode, size_t smem, int variant);
int fused_blocks_per_sm_f64(int P, int mode, size_t smem, int variant);
int fused_variant_threads_f32(int P, int variant);
cudaError_t launch_fused_f32(int P, const LaunchArgs &a);
cudaError_t launch_fused_f64(int P, const LaunchArgs &a);
cudaError_t launch_global_f32(int P, const LaunchArgs &a, int maxD);
cudaError_t launch_global_f64(int P, const LaunchArgs &a, int maxD);
cudaError_t launch_relax_grad_f32(const LaunchArgs &a, int maxD, const void *grad, const double *gscale);
size_t cluster_smem_f32(int P, int D, int Dpad, bool wbuf, int nc);
size_t cluster_smem_f64(int P, int D, int Dpad, bool wbuf, int nc);
int cluster_max_active_f32(int P, int D, int Dpad, bool wbuf, int nc);
int cluster_max_active_f64(int P, int D, int Dpad, bool wbuf, int nc);
cudaError_t launch_cluster_f32(int P, const LaunchArgs &a, int maxD, int maxDpad, int nc);
cudaError_t launch_cluster_f64(int P, const LaunchArgs &a, int maxD, int maxDpad, int nc);
cudaError_t launch_relax_grad_f64(const LaunchArgs &a, int maxD, const void *grad, const double *gscale);

cudaError_t upload_twiddle_constants(const double *re, const double *im)
{
    cudaError_t e;
    if ((e = upload_tw_fused_f32(re, im)) != cudaSuccess) return e;
    if ((e = upload_tw_fused_f64(re, im)) != cudaSuccess) return e;
    if ((e = upload_tw_glob_f32(re, im)) != cudaSuccess) return e;
    if ((e = upload_tw_spectra(re, im)) != cudaSuccess) return e;
    return upload_tw_glob_f64(re, im);
}

size_t fused_smem(int P, int prec, int D, int Dpad, bool wbuf, int variant)
{
    return prec == ND_PREC_FP64 ? fused_smem_f64(P, D, Dpad, wbuf, variant) : fused_smem_f32(P, D, Dpad, wbuf, variant);
}

int fused_blocks_per_sm(int P, int prec, int mode, size_t smem, int variant)
{
    return prec == ND_PREC_FP64 ? fused_blocks_per_sm_f64(P, mode, smem, variant)
                                : fused_blocks_per_sm_f32(P, mode, smem, variant);
}

int fused_variant_threads(int P, int variant) { return fused_variant_threads_f32(P, variant); }

cudaError_t launch_fused(int P, int prec, const LaunchArgs &a)
{
    return prec == ND_PREC_FP64 ? launch_fused_f64(P, a) : launch_fused_f32(P, a);
}

cudaError_t launch_global(int P, int prec, const LaunchArgs &a, int maxD)
{
    return prec == ND_PREC_FP64 ? launch_global_f64(P, a, maxD) : launch_global_f32(P, a, maxD);
}

cudaError_t launch_relax_grad(int prec, const LaunchArgs &a, int maxD, const void *grad, const double *gscale)
{
    return prec == ND_PREC_FP64 ? launch_relax_grad_f64(a, maxD, grad, gscale) : launch_relax_grad_f32(a, maxD, grad, gscale);
}

size_t cluster_smem(int P, int prec, int D, int Dpad, bool wbuf, int nc)
{
    return prec == ND_PREC_FP64 ? cluster_smem_f64(P, D, Dpad, wbuf, nc) : cluster_smem_f32(P, D, Dpad, wbuf, nc);
}

int cluster_max_active(int P, int prec, int D, int Dpad, bool wbuf, int nc)
{
    return prec == ND_PREC_FP64 ? cluster_max_active_f64(P, D, Dpad, wbuf, nc)
                                : cluster_max_active_f32(P, D, Dpad, wbuf, nc);
}

cudaError_t launch_cluster(int P, int prec, const LaunchArgs &a, int maxD, int maxDpad, int nc)
{
    return prec == ND_PREC_FP64 ? launch_cluster_f64(P, a, maxD, maxDpad, nc)
                                : launch_cluster_f32(P, a, maxD, maxDpad, nc);
}

size_t spec_words(int P, int D)
{
    const int RS = (P > 128) ? (P / 2 + 4) : (P >= 32) ? (P / 2 + 2) : (P / 2 + 2 + 8);   // matches SpecGeom<P>::RS
    // rounded to 16 complex words (128 B for FP32) so every replica's spectrum,
    // and for P > 128 every row of it, starts on a 32-byte sector
    return ((size_t)3 * D * RS + 15) / 16 * 16;
}

}  // namespace nd
