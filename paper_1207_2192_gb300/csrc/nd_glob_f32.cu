// nd_glob_f32.cu -- instantiations of the global-memory field path in FP32.
#include <math.h>

#include "nd_field_impl.cuh"

namespace nd {

ND_DEFINE_TWIDDLE_UPLOAD(upload_tw_glob_f32)

cudaError_t launch_global_f32(int P, const LaunchArgs &a, int maxD)
{
    switch (P) {
    case 16: return launch_global_p<16, float>(a, maxD);
    case 32: return launch_global_p<32, float>(a, maxD);
    case 64: return launch_global_p<64, float>(a, maxD);
    case 128: return launch_global_p<128, float>(a, maxD);
    case 192: return launch_global_p<192, float>(a, maxD);
    case 200: return launch_global_p<200, float>(a, maxD);
    case 256: return launch_global_p<256, float>(a, maxD);
    case 512: return launch_global_p<512, float>(a, maxD);
    case 1024: return launch_global_p<1024, float>(a, maxD);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_relax_grad_f32(const LaunchArgs &a, int maxD, const void *grad, const double *gscale)
{
    return launch_relax_grad_t<float>(a, maxD, grad, gscale);
}

}  // namespace nd
