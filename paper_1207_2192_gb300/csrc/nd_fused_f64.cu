// nd_fused_f64.cu -- instantiations of the fused on-chip kernel in FP64.
#include "nd_field_impl.cuh"

namespace nd {

ND_DEFINE_TWIDDLE_UPLOAD(upload_tw_fused_f64)

size_t fused_smem_f64(int P, int D, int Dpad)
{
    switch (P) {
    case 16: return fused_smem_bytes<16, double>(D, Dpad, FusedNT<16>::v);
    case 32: return fused_smem_bytes<32, double>(D, Dpad, FusedNT<32>::v);
    case 64: return fused_smem_bytes<64, double>(D, Dpad, FusedNT<64>::v);
    case 128: return fused_smem_bytes<128, double>(D, Dpad, FusedNT<128>::v);
    default: return (size_t)-1;
    }
}

cudaError_t launch_fused_f64(int P, const LaunchArgs &a)
{
    switch (P) {
    case 16: return launch_fused_p<16, double>(a);
    case 32: return launch_fused_p<32, double>(a);
    case 64: return launch_fused_p<64, double>(a);
    case 128: return launch_fused_p<128, double>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace nd
