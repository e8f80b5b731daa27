// nd_glob_f64.cu -- instantiations of the global-memory field path in FP64.
#include <math.h>

#include "nd_field_impl.cuh"

namespace nd {

ND_DEFINE_TWIDDLE_UPLOAD(upload_tw_glob_f64)

cudaError_t launch_global_f64(int P, const LaunchArgs &a, int maxD)
{
    switch (P) {
    case 16: return launch_global_p<16, double>(a, maxD);
    case 32: return launch_global_p<32, double>(a, maxD);
    case 64: return launch_global_p<64, double>(a, maxD);
    case 128: return launch_global_p<128, double>(a, maxD);
    case 192: return launch_global_p<192, double>(a, maxD);
    case 200: return launch_global_p<200, double>(a, maxD);
    case 256: return launch_global_p<256, double>(a, maxD);
    case 512: return launch_global_p<512, double>(a, maxD);
    case 1024: return launch_global_p<1024, double>(a, maxD);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_relax_grad_f64(const LaunchArgs &a, int maxD, const void *grad, const double *gscale)
{
    return launch_relax_grad_t<double>(a, maxD, grad, gscale);
}

}  // namespace nd
