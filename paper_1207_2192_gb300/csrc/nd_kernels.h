// nd_kernels.h -- host-side interface between the C-ABI layer and the CUDA
// kernels (no CUDA device code here, no torch types).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace nd {

enum { ND_PREC_FP32 = 0, ND_PREC_FP64 = 1 };
enum { M_FIELD = 0, M_RK4 = 1, M_HEUN = 2, M_ENERGY = 3, M_RELAX = 4 };

struct Replica;
struct RelaxIO;
struct StatsAcc;

struct LaunchArgs {
    int mode = M_FIELD;
    const Replica *reps = nullptr;   // device array of all replicas of the handle
    const int *work = nullptr;       // device array: replica indices handled by this launch
    int nwork = 0;
    void *y = nullptr;               // state y_n (user buffer, updated in place by steppers)
    void *acc = nullptr;             // stage accumulator scratch (same layout as y)
    void *out = nullptr;             // field output (field mode)
    void *ms = nullptr;              // global-path stage state (same layout as y)
    void *spec = nullptr;            // global-path spectrum scratch
    double *red = nullptr;           // per-replica reduction output (energy), indexed by replica
    const void *tw = nullptr;        // length-P twiddle table exp(-2 pi i k/P) of the precision
    long long nsteps = 1;
    unsigned long long step_base = 0;
    size_t smem = 0;
    cudaStream_t stream = 0;
    // relaxation
    RelaxIO *rio = nullptr;          // per replica, indexed like reps
    RelaxIO *rio_host = nullptr;     // host copy of the same array (global-path convergence checks)
    int n_rio = 0;                   // entries of rio
    const int *work_host = nullptr;  // host copy of work (nwork entries)
    double *part = nullptr;          // global-path relaxation partial sums: [replicas][kRelaxBlocks][6]
    double eta = 0.5, tol = 1e-6, rc2 = 0.0;
    int max_iter = 0;
    // time-sliced schedule (fused steppers): ncta CTAs run the segments
    // segs[seg_off[b] .. seg_off[b+1]) and hand replicas over through flags
    const void *segs = nullptr;
    const int *seg_off = nullptr;
    int *flags = nullptr;
    int ncta = 0;
    unsigned *status = nullptr;      // device status word (ND_DEV_* bits)
    int use_wbuf = 0;                // keep the Heun predictor's normals in shared memory
    int smem_optin = 0;              // per-block shared-memory limit of the device
    int variant = 0;                 // fused-kernel thread-count variant (stepping modes)
    int n_sm = 1;                    // multiprocessors of the device (persistent grids)
};

constexpr int kRelaxBlocks = 64;    // global-path relaxation: partial-sum blocks per replica

struct SegmentHost {                 // mirrors Segment in nd_field_impl.cuh
    int rep, wait, signal, pad;
    long long step_begin, nsteps;
};

cudaError_t upload_twiddle_constants(const double *re, const double *im);
size_t fused_smem(int P, int prec, int D, int Dpad, bool wbuf = false, int variant = 0);
int fused_blocks_per_sm(int P, int prec, int mode, size_t smem, int variant = 0);
int fused_variant_threads(int P, int variant);   // 0 if the variant does not exist
cudaError_t launch_fused(int P, int prec, const LaunchArgs &a);
// One replica per thread-block cluster of nc = 8 or 16 CTAs (P <= 128; P = 256
// on 16 CTAs; stepping modes), of cluster_cta_threads(P) threads per CTA.
constexpr int cluster_cta_threads(int P) { return P >= 256 ? 512 : 256; }
size_t cluster_smem(int P, int prec, int D, int Dpad, bool wbuf, int nc);   // (size_t)-1: no such size
int cluster_max_active(int P, int prec, int D, int Dpad, bool wbuf, int nc);  // 0: does not fit
cudaError_t launch_cluster(int P, int prec, const LaunchArgs &a, int maxD, int maxDpad, int nc);
cudaError_t launch_global(int P, int prec, const LaunchArgs &a, int maxD);
size_t spec_words(int P, int D);   // complex words of one replica's [3][D][RS] spectrum
// One constrained-relaxation sweep over a size class with the field taken
// from an energy gradient: b = gscale[r] * grad (a.y: the state, a.rio/a.part:
// multipliers and partial sums, a.tol: convergence threshold).
cudaError_t launch_relax_grad(int prec, const LaunchArgs &a, int maxD, const void *grad, const double *gscale);

// Spectral kernel build (Section II.B tensor, cell self terms, exchange folded in).
// Gq: optional device table [4][D][D] of a^2 G at displacements (dx, dy) >= 0 (comps xx, yy, xy, zz,
// self terms at the origin); when null it is computed from the paper's closed forms.
// Output: Ghat64 [P/2+1][P/2+1][4] doubles followed by the same values
// component-major, [4][P/2+1][P/2+1] (ghat_table_entries(P) doubles in all),
// and, if Ghat32 != null, a float copy of the same layout.
inline size_t ghat_table_entries(int P) { return (size_t)(P / 2 + 1) * (P / 2 + 1) * 8; }
cudaError_t build_ghat(int P, int D, double L_over_a, double Nx, double Nz, double c, const double *Gq_dev,
                       double *Ghat64, float *Ghat32, double *work, cudaStream_t st);
size_t build_ghat_work_doubles(int P, int D);
// Spectral kernel of c d(a^2 G)/dl (l = L/a, no exchange), same layout and 1/P^2 scale.
cudaError_t build_ghat_dl(int P, int D, double l, double dNx, double dNz, double cfac, double *GL64, double *work,
                          cudaStream_t st);

// Auxiliary kernels (nd_aux.cu).
cudaError_t launch_init_vortex(int prec, const Replica *reps, const int *work, int nwork, int maxD, void *y,
                               const double *X0_cells /*[nrep][2], units of a, device*/, const int *pol_chi,
                               double lambda_over_a, cudaStream_t st);
constexpr int kCoreMaxBlocks = 128;   // plaquette-scan CTAs per replica (candidates buffer: [B][128][2] doubles)
int core_scan_blocks(int D);
cudaError_t launch_vortex_core(int prec, const Replica *reps, const int *work, int nwork, int maxD, const void *y,
                               double rc2, double *part, double *out /*[nrep][4]: xc, yc (units of a), status, cell*/,
                               cudaStream_t st);
cudaError_t launch_stats_update(const int *work, int nwork, const double *core, const double *a_of_rep, StatsAcc *st,
                                unsigned long long *hr, unsigned long long *hv, int rb, int vb, double r_max,
                                double v_max, double dt, cudaStream_t s);
cudaError_t launch_advance_steps(Replica *reps, int n, long long steps, cudaStream_t s);
cudaError_t launch_mean_m(int prec, const Replica *reps, const int *work, int nwork, const void *y,
                          double *out /*[nrep][3]*/, cudaStream_t st);
cudaError_t launch_convert(int to_prec, const void *src, void *dst, size_t n, cudaStream_t st);

// Time series of <m> and their power spectra (nd_spectra.cu).
cudaError_t launch_series_append(int prec, const Replica *reps, const int *work, int nwork, const void *y,
                                 double *series /*[nrep][cap][3]*/, const unsigned long long *count, int cap,
                                 cudaStream_t st);
cudaError_t launch_series_advance(unsigned long long *count, cudaStream_t st);
cudaError_t launch_window_power(int W, const double *series, int cap, int comp, int nwin, int nrep,
                                const void *twW /*length-W FP64 table*/, double *pw /*[nrep][nwin][W/2+1]*/,
                                cudaStream_t st);
cudaError_t launch_psd_reduce(const double *pw, int nwin, int nk, int nrep, double scale, double *psd, cudaStream_t st);
cudaError_t launch_check_finite(int prec, const Replica *reps, const int *work, int nwork, int maxD, const void *y,
                                unsigned *flag, cudaStream_t st);

}  // namespace nd
