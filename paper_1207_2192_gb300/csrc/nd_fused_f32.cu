// nd_fused_f32.cu -- instantiations of the fused on-chip kernel in FP32.
#include "nd_cluster.cuh"

namespace nd {

static_assert(sizeof(Segment) == sizeof(SegmentHost), "segment layout");

ND_DEFINE_TWIDDLE_UPLOAD(upload_tw_fused_f32)

size_t fused_smem_f32(int P, int D, int Dpad, bool wbuf, int variant)
{
    const int nt = fused_nt(P, variant);
    if (nt == 0) return (size_t)-1;
    switch (P) {
    case 16: return fused_smem_bytes<16, float>(D, Dpad, nt, wbuf);
    case 32: return fused_smem_bytes<32, float>(D, Dpad, nt, wbuf);
    case 64: return fused_smem_bytes<64, float>(D, Dpad, nt, wbuf);
    case 128: return fused_smem_bytes<128, float>(D, Dpad, nt, wbuf);
    default: return (size_t)-1;
    }
}

template <int P>
static int occ_p(int mode, size_t smem, int variant)
{
    switch (mode) {
    case M_RK4: return fused_occupancy<P, float, M_RK4>(variant, smem);
    case M_HEUN: return fused_occupancy<P, float, M_HEUN>(variant, smem);
    default: return 0;
    }
}

int fused_blocks_per_sm_f32(int P, int mode, size_t smem, int variant)
{
    switch (P) {
    case 16: return occ_p<16>(mode, smem, variant);
    case 32: return occ_p<32>(mode, smem, variant);
    case 64: return occ_p<64>(mode, smem, variant);
    case 128: return occ_p<128>(mode, smem, variant);
    default: return 0;
    }
}

int fused_variant_threads_f32(int P, int variant) { return fused_nt(P, variant); }

cudaError_t launch_fused_f32(int P, const LaunchArgs &a)
{
    switch (P) {
    case 16: return launch_fused_p<16, float>(a);
    case 32: return launch_fused_p<32, float>(a);
    case 64: return launch_fused_p<64, float>(a);
    case 128: return launch_fused_p<128, float>(a);
    default: return cudaErrorInvalidValue;
    }
}

// Cluster plans: NC = 8 CTAs for every on-chip size, NC = 16 for P >= 32
// (where the P/2 column slots split over 16 CTAs), and P = 192 and 256 on 16
// CTAs (spectra too large for one CTA's shared memory).
#define ND_CLUSTER_CASES(X)      \
    X(16, 8) X(32, 8) X(64, 8) X(128, 8) X(32, 16) X(64, 16) X(128, 16) X(192, 16) X(256, 16)

size_t cluster_smem_f32(int P, int D, int Dpad, bool wbuf, int nc)
{
#define X(p, n) if (P == p && nc == n) return cluster_smem_bytes<p, float, n>(D, Dpad, wbuf);
    ND_CLUSTER_CASES(X)
#undef X
    return (size_t)-1;
}

int cluster_max_active_f32(int P, int D, int Dpad, bool wbuf, int nc)
{
#define X(p, n) if (P == p && nc == n) return cluster_max_active_t<p, float, n>(D, Dpad, wbuf);
    ND_CLUSTER_CASES(X)
#undef X
    return 0;
}

cudaError_t launch_cluster_f32(int P, const LaunchArgs &a, int maxD, int maxDpad, int nc)
{
#define X(p, n) if (P == p && nc == n) return launch_cluster_p<p, float, n>(a, maxD, maxDpad);
    ND_CLUSTER_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace nd
