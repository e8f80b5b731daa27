// nd_api.cu -- the C ABI (include/nanodisk.h): handle, geometry and units on
// the host, device memory, staging of host buffers, and dispatch of each call
// to the fused on-chip kernel or to the global-memory path per FFT size class.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/nanodisk.h"
#include "nd_common.cuh"
#include "nd_kernels.h"

using namespace nd;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define ND_CUDA(call)                                                                                      \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return fail(ND_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

const double kMu0 = 4.0e-7 * M_PI;   // vacuum permeability (SI)
const double kBoltzmann = 1.380649e-23;

struct DiskInfo {
    nd_disk_desc desc;
    int D = 0, Dpad = 0, P = 0, C = 0;
    double lambda = 0, cfac = 0, B0 = 0, t0 = 0, J = 0, Nx = 0, Nz = 0;
    double h[3] = {0, 0, 0};   // H_ext / Ms
    std::vector<unsigned char> mask;
    unsigned char *mask_d = nullptr;
    int *cells_d = nullptr;    // the cells inside the disk (increasing j*D+i), C of them
    double *ghat64 = nullptr;  // [P/2+1][P/2+1][4]
    float *ghat32 = nullptr;
    double *ghatL = nullptr;   // thickness derivative of the demagnetisation kernel (FP64)
    double dNx = 0, dNz = 0;   // dN/d(L/a) of the self terms
    // per-step external field schedule, (a^2/lambda^2) H_ext(s)/Ms, [nsched][3]
    float *sched32 = nullptr;
    double *sched64 = nullptr;
    long long nsched = 0;
};

// Upload a disk's mask and its compacted cell list (the mask may change).
static cudaError_t upload_mask(DiskInfo &d)
{
    std::vector<int> cells;
    for (size_t i = 0; i < d.mask.size(); ++i)
        if (d.mask[i]) cells.push_back((int)i);
    cudaError_t e = cudaMemcpy(d.mask_d, d.mask.data(), d.mask.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !cells.empty())
        e = cudaMemcpy(d.cells_d, cells.data(), sizeof(int) * cells.size(), cudaMemcpyHostToDevice);
    return e;
}

struct SizeClass {
    int P = 0, maxD = 0, maxDpad = 0;
    std::vector<int> reps;     // replica indices
    int *work_d = nullptr;     // device copy of reps
    bool fused_main = false;   // fused kernel in the handle precision
    bool fused_fp64 = false;   // fused kernel in FP64 (energy)
    size_t smem_main = 0, smem_fp64 = 0;
    size_t smem_wbuf = 0;      // fused Heun with the normals kept in shared memory (0: does not fit)
    int plan[2] = {-1, -1};    // stepping plan for RK4 / Heun: -1 default, 0..2 fused variant, kPlanGlobal, kPlanCluster
    // time-sliced schedule, cached per (mode, n_steps)
    SegmentHost *segs_d = nullptr;
    int *seg_off_d = nullptr;
    int seg_mode = -1, seg_ncta = 0;
    long long seg_nsteps = -1;
};

constexpr int kPlanGlobal = 100;
constexpr int kPlanCluster = 200;     // one replica per thread-block cluster of 8 CTAs (P <= 128)
constexpr int kPlanCluster16 = 201;   // one replica per cluster of 16 CTAs (32 <= P <= 128)
static int plan_cluster_nc(int pl) { return pl == kPlanCluster ? 8 : pl == kPlanCluster16 ? 16 : 0; }

int next_pow2_at_least(int n)
{
    int p = 16;
    while (p < n) p *= 2;
    return p;
}

// Padded FFT side for a linear convolution of span n = 2D - 1: the next power
// of two, or with ND_GRID_3X the smallest of the register FFT's other sizes
// where it is smaller: 192 = 3 * 2^6 (n <= 192) and 200 = 2^3 * 5^2 (n <= 200).
int padded_size(int n, bool allow3)
{
    const int p2 = next_pow2_at_least(n);
    if (allow3 && n <= 192 && p2 > 192) return 192;
    if (allow3 && n <= 200 && p2 > 200) return 200;
    return p2;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace nd {
void set_last_error(const std::string &msg) { g_err = msg; }
}

struct nd_handle {
    int prec = ND_FP32;
    int device = 0;
    size_t elt = 4;                       // bytes per state element
    std::vector<DiskInfo> disks;
    std::vector<int> rep_disk;
    std::vector<long long> rep_off;
    std::vector<long long> rep_spec_off;  // complex words
    long long state_elems = 0;
    long long spec_words = 0;
    std::vector<double> alpha;
    std::vector<SizeClass> classes;
    static constexpr int kSlots = 4;      // ring of pinned parameter blocks
    Replica *reps_h = nullptr;            // current slot (points into reps_ring)
    Replica *reps_ring = nullptr;         // pinned [kSlots][B]
    cudaEvent_t slot_ev[kSlots] = {};
    int slot = 0;
    Replica *reps_d = nullptr;
    std::map<int, void *> tw64, tw32;     // P -> length-P twiddle tables
    void *acc = nullptr;                  // handle-precision scratch (state layout)
    void *ms = nullptr;                   // handle-precision stage state (global path)
    void *spec = nullptr;                 // spectrum scratch (global path), sized for FP64
    void *stage_in = nullptr, *stage_out = nullptr;   // staging of host buffers
    double *y64 = nullptr, *ms64 = nullptr;           // FP64 copies (energy of FP32 handles)
    double *red_d = nullptr;              // [B] reductions
    double *red_h = nullptr;              // pinned [B * 4]
    double *aux_d = nullptr;              // [B * 4] small per-replica inputs/outputs
    int *aux_i = nullptr;                 // [B * 2]
    RelaxIO *rio_d = nullptr;             // [B] relaxation inputs/outputs
    RelaxIO *rio_h = nullptr;             // pinned [B]
    double *relax_part = nullptr;         // global-path relaxation partial sums [B][kRelaxBlocks][6]
    double *series = nullptr;             // <m> time series [B][series_cap][3]
    unsigned long long *series_count = nullptr;   // device sample counter
    int series_cap = 0;
    double *psd_work = nullptr;           // per-window periodograms
    size_t psd_work_doubles = 0;
    // statistics (device resident, filled by nd_stats_sample)
    StatsAcc *stats = nullptr;
    unsigned long long *hist_r = nullptr, *hist_v = nullptr;
    int rbins = 0, vbins = 0;
    double r_max = 0, v_max = 0;
    double *core_d = nullptr;             // [B * 4] estimator output of the last sample
    double *core_part = nullptr;          // [B][kCoreMaxBlocks][2] plaquette-scan candidates
    double *a_rep = nullptr;              // [B] cell edge per replica
    size_t max_smem = 0;
    int n_sm = 0;
    // side streams and fork/join events: the stepping kernels of different
    // size classes run side by side (class 0 on the caller's stream)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join_ev;
    cudaEvent_t fork_ev = nullptr;
    int *flags_d = nullptr;               // [B] replica hand-over flags of the time-sliced schedule
    unsigned *status_d = nullptr;         // device status word (ND_DEV_* bits)
    unsigned long long rk4_step = 0;      // step index of the next nd_step_rk4 step (field schedules)
};

static int setup_class_paths(nd_handle *h)
{
    for (auto &c : h->classes) {
        const size_t w = fused_smem(c.P, h->prec, c.maxD, c.maxDpad, true);
        c.smem_wbuf = (w != (size_t)-1 && w + 1024 <= h->max_smem) ? w : 0;
        // 1 KiB of the per-block limit is left for the kernels' static shared variables
        c.smem_main = fused_smem(c.P, h->prec, c.maxD, c.maxDpad);
        c.fused_main = c.smem_main != (size_t)-1 && c.smem_main + 1024 <= h->max_smem;
        c.smem_fp64 = fused_smem(c.P, ND_PREC_FP64, c.maxD, c.maxDpad);
        c.fused_fp64 = c.smem_fp64 != (size_t)-1 && c.smem_fp64 + 1024 <= h->max_smem;
    }
    return ND_OK;
}

// Parameter blocks go through a ring of pinned host slots: a slot is reused
// only after the copy that last read it has executed.
static void next_slot(nd_handle *h)
{
    h->slot = (h->slot + 1) % nd_handle::kSlots;
    cudaEventSynchronize(h->slot_ev[h->slot]);
    h->reps_h = h->reps_ring + (size_t)h->slot * h->rep_disk.size();
}

static void upload_reps(nd_handle *h, cudaStream_t st)
{
    cudaMemcpyAsync(h->reps_d, h->reps_h, sizeof(Replica) * h->rep_disk.size(), cudaMemcpyHostToDevice, st);
    cudaEventRecord(h->slot_ev[h->slot], st);
}

enum { TAB_MAIN = 0, TAB_DL = 1 };

static void fill_reps(nd_handle *h, bool fp64_kernel, double dt_seconds, const double *Tk,
                      const unsigned long long *seed, unsigned long long step0, int table = TAB_MAIN)
{
    const int B = (int)h->rep_disk.size();
    next_slot(h);
    for (int r = 0; r < B; ++r) {
        const DiskInfo &d = h->disks[h->rep_disk[r]];
        Replica &R = h->reps_h[r];
        R.D = d.D;
        R.Dpad = d.Dpad;
        R.disk = h->rep_disk[r];
        R.state_off = h->rep_off[r];
        R.spec_off = h->rep_spec_off[r];
        R.Ghat = table == TAB_DL ? (const void *)d.ghatL : (fp64_kernel ? (const void *)d.ghat64 : (const void *)d.ghat32);
        R.mask = d.mask_d;
        R.cells = d.cells_d;
        R.ncells = d.C;
        for (int k = 0; k < 3; ++k) R.chext[k] = table == TAB_DL ? 0.0 : d.cfac * d.h[k];
        R.alpha = h->alpha[r];
        R.dtau = d.desc.gamma * d.B0 * dt_seconds;
        double Ts = Tk ? kBoltzmann * Tk[r] / d.J : 0.0;
        R.sigma = sqrt(2.0 * R.alpha * Ts * R.dtau);
        R.flags = (R.sigma > 0.0) ? 1 : 0;
        R.seed = seed ? seed[r] : 0ull;
        R.step0 = step0;
        for (int k = 0; k < 3; ++k) R.fchext[k] = (float)R.chext[k];
        R.falpha = (float)R.alpha;
        R.fdtau = (float)R.dtau;
        R.fsigma = (float)R.sigma;
        R.fsched = table == TAB_DL ? nullptr : d.sched32;
        R.dsched = table == TAB_DL ? nullptr : d.sched64;
        R.nsched = table == TAB_DL ? 0 : d.nsched;
    }
}

// Time-sliced schedule for more replicas than resident CTAs: the class's
// replica-steps (B_c x n) are cut into ncta equal, contiguous ranges; CTA i
// runs the start of the replica it shares with CTA i+1 first (and flags it),
// then its whole replicas, then the end of the replica it shares with CTA i-1
// after waiting for that flag.  Every CTA does the same number of steps.
static void build_segments(int Bc, long long n, int ncta, std::vector<SegmentHost> &segs, std::vector<int> &off)
{
    const long long W = (long long)Bc * n, s = (W + ncta - 1) / ncta;
    segs.clear();
    off.assign(ncta + 1, 0);
    for (int i = 0; i < ncta; ++i) {
        off[i] = (int)segs.size();
        const long long start = (long long)i * s, end = std::min(W, start + s);
        if (start >= end) continue;
        const int r0 = (int)(start / n), r1 = (int)((end - 1) / n);
        const long long o0 = start % n, o1 = (end - 1) % n + 1;
        if (r0 == r1) {
            segs.push_back({r0, o0 > 0 ? 1 : 0, o1 < n ? 1 : 0, 0, o0, o1 - o0});
            continue;
        }
        if (o1 < n) segs.push_back({r1, 0, 1, 0, 0, o1});             // start of the replica continued by CTA i+1
        for (int r = (o0 > 0 ? r0 + 1 : r0); r < r1; ++r) segs.push_back({r, 0, 0, 0, 0, n});
        if (o1 == n) segs.push_back({r1, 0, 0, 0, 0, n});
        if (o0 > 0) segs.push_back({r0, 1, 0, 0, o0, n - o0});          // end of the replica started by CTA i-1
    }
    off[ncta] = (int)segs.size();
}

// Whether a cluster plan of nc CTAs per replica exists for the class: the
// size has one, its shared memory fits, and the GPU can hold such a cluster.
static bool cluster_plan_fits(const nd_handle *h, const SizeClass &c, int prec, bool heun, int nc)
{
    const size_t sm = cluster_smem(c.P, prec, c.maxD, c.maxDpad, heun, nc);
    if (sm == (size_t)-1 || sm + 1024 > h->max_smem) return false;
    return cluster_max_active(c.P, prec, c.maxD, c.maxDpad, heun, nc) > 0;
}

// Run one mode over all replicas.  fp64 selects the FP64 kernels (with y a
// double buffer of the state layout), otherwise the handle precision.
static int run_mode(nd_handle *h, int mode, bool fp64, void *y, void *out, long long nsteps, cudaStream_t st,
                    const Replica *reps = nullptr, int only_class = -1)
{
    const int prec = fp64 ? ND_PREC_FP64 : (h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32);
    // The stepping kernels of the size classes are independent (each touches
    // only its replicas' state and scratch), so they run side by side on
    // forked streams: a class fills only the SMs of its replicas.  Not when a
    // class needs the time-sliced schedule, whose cooperative launch takes the
    // whole GPU.
    bool concurrent = (mode == M_RK4 || mode == M_HEUN) && only_class < 0 && h->classes.size() > 1 &&
                      h->side.size() + 1 == h->classes.size();
    for (const auto &c : h->classes)
        if ((int)c.reps.size() > h->n_sm) concurrent = false;
    if (concurrent) ND_CUDA(cudaEventRecord(h->fork_ev, st));
    const cudaStream_t st0 = st;
    for (int ci = 0; ci < (int)h->classes.size(); ++ci) {
        if (only_class >= 0 && ci != only_class) continue;
        auto &c = h->classes[ci];
        cudaStream_t st = st0;
        if (concurrent && ci > 0) {
            st = h->side[ci - 1];
            ND_CUDA(cudaStreamWaitEvent(st, h->fork_ev, 0));
        }
        LaunchArgs a;
        a.mode = mode;
        a.reps = reps ? reps : h->reps_d;
        a.work = c.work_d;
        a.nwork = (int)c.reps.size();
        a.y = y;
        a.out = out;
        a.red = h->red_d;
        a.nsteps = nsteps;
        a.step_base = 0;
        a.stream = st;
        a.tw = (prec == ND_PREC_FP64) ? h->tw64[c.P] : h->tw32[c.P];
        a.smem_optin = (int)h->max_smem;
        a.n_sm = h->n_sm;
        bool fused = fp64 ? c.fused_fp64 : c.fused_main;
        const bool stepping = (mode == M_HEUN || mode == M_RK4) && !fp64;
        int variant = 0;
        int cluster_nc = 0;
        if (stepping) {
            const int pl = c.plan[mode == M_RK4 ? 0 : 1];
            if (pl == kPlanGlobal) fused = false;
            else if (plan_cluster_nc(pl)) cluster_nc = plan_cluster_nc(pl);
            else if (pl > 0) variant = pl;
        }
        if (mode == M_RK4 || mode == M_HEUN) a.acc = h->acc;
        if (cluster_nc) {
            a.use_wbuf = mode == M_HEUN ? 1 : 0;
            a.status = h->status_d;
            ND_CUDA(launch_cluster(c.P, prec, a, c.maxD, c.maxDpad, cluster_nc));
        } else if (fused) {
            a.smem = fp64 ? c.smem_fp64 : c.smem_main;
            a.status = h->status_d;
            a.variant = variant;
            if (variant != 0) a.smem = fused_smem(c.P, prec, c.maxD, c.maxDpad, false, variant);
            if (mode == M_HEUN && !fp64) {
                const size_t w = variant == 0 ? c.smem_wbuf : fused_smem(c.P, prec, c.maxD, c.maxDpad, true, variant);
                if (w && w != (size_t)-1 && w + 1024 <= h->max_smem) {
                    a.smem = w;
                    a.use_wbuf = 1;
                }
            }
            if ((mode == M_HEUN || mode == M_RK4) && !fp64 && nsteps >= 2) {
                // localise the replicas' indices to the class: segments refer to positions in c.reps
                const int per_sm = fused_blocks_per_sm(c.P, prec, mode, a.smem, variant);
                const int ncta = per_sm * h->n_sm;
                const int Bc = (int)c.reps.size();
                if (per_sm > 0 && Bc > ncta) {
                    if (c.seg_mode != mode || c.seg_nsteps != nsteps || c.seg_ncta != ncta) {
                        std::vector<SegmentHost> segs;
                        std::vector<int> off;
                        build_segments(Bc, nsteps, ncta, segs, off);
                        for (auto &g : segs) g.rep = c.reps[g.rep];
                        cudaFree(c.segs_d);
                        cudaFree(c.seg_off_d);
                        c.segs_d = nullptr;
                        c.seg_off_d = nullptr;
                        ND_CUDA(cudaMalloc(&c.segs_d, sizeof(SegmentHost) * segs.size()));
                        ND_CUDA(cudaMalloc(&c.seg_off_d, sizeof(int) * off.size()));
                        ND_CUDA(cudaMemcpy(c.segs_d, segs.data(), sizeof(SegmentHost) * segs.size(), cudaMemcpyHostToDevice));
                        ND_CUDA(cudaMemcpy(c.seg_off_d, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
                        c.seg_mode = mode;
                        c.seg_nsteps = nsteps;
                        c.seg_ncta = ncta;
                    }
                    ND_CUDA(cudaMemsetAsync(h->flags_d, 0, sizeof(int) * h->rep_disk.size(), st));
                    a.segs = c.segs_d;
                    a.seg_off = c.seg_off_d;
                    a.flags = h->flags_d;
                    a.ncta = ncta;
                }
            }
            ND_CUDA(launch_fused(c.P, prec, a));
        } else {
            a.ms = fp64 ? (void *)h->ms64 : h->ms;
            a.spec = h->spec;
            if (!a.ms || !a.spec) return fail(ND_ERR_ARG, "global-path buffers are not allocated");
            ND_CUDA(launch_global(c.P, prec, a, c.maxD));
        }
        // a stepped state with a non-finite cell sets the NaN bit of the status word
        if (mode == M_RK4 || mode == M_HEUN)
            ND_CUDA(launch_check_finite(prec, a.reps, c.work_d, (int)c.reps.size(), c.maxD, y, h->status_d, st));
        if (concurrent && ci > 0) ND_CUDA(cudaEventRecord(h->join_ev[ci - 1], st));
    }
    if (concurrent)
        for (size_t k = 0; k < h->side.size(); ++k) ND_CUDA(cudaStreamWaitEvent(st0, h->join_ev[k], 0));
    return ND_OK;
}

static int ensure_alloc(void **p, size_t bytes)
{
    if (*p) return ND_OK;
    ND_CUDA(cudaMalloc(p, bytes));
    return ND_OK;
}

static int check_handle(const nd_handle *h)
{
    if (!h) return fail(ND_ERR_ARG, "null handle");
    return ND_OK;
}

// Prepare a state argument: device pointers pass through; host pointers are
// copied into a staging buffer.
static int stage_in(nd_handle *h, const void *m, void **dev, bool copy, cudaStream_t st, void **slot)
{
    if (!m) return fail(ND_ERR_ARG, "null state pointer");
    if (is_device_ptr(m)) {
        *dev = const_cast<void *>(m);
        return ND_OK;
    }
    size_t bytes = (size_t)h->state_elems * h->elt;
    int rc = ensure_alloc(slot, bytes);
    if (rc) return rc;
    if (copy) ND_CUDA(cudaMemcpyAsync(*slot, m, bytes, cudaMemcpyHostToDevice, st));
    *dev = *slot;
    return ND_OK;
}

static int stage_out(nd_handle *h, void *m, const void *dev, cudaStream_t st)
{
    if (dev == m) return ND_OK;
    ND_CUDA(cudaMemcpyAsync(m, dev, (size_t)h->state_elems * h->elt, cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    return ND_OK;
}

extern "C" {

const char *nd_last_error(void) { return g_err.c_str(); }

int nd_create_disk(const nd_disk_desc *disks, int n_disks, const int *replicas_per_disk, int precision,
                   nd_handle **out)
{
    if (!out) return fail(ND_ERR_ARG, "out is null");
    *out = nullptr;
    if (!disks || n_disks < 1) return fail(ND_ERR_ARG, "need at least one disk");
    const bool allow3 = (precision & ND_GRID_3X) != 0;
    precision &= ~ND_GRID_3X;
    if (precision != ND_FP32 && precision != ND_FP64)
        return fail(ND_ERR_ARG, "precision must be ND_FP32 or ND_FP64 (optionally with ND_GRID_3X)");
    nd_handle *h = new nd_handle();
    h->prec = precision;
    h->elt = precision == ND_FP64 ? 8 : 4;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return fail(ND_ERR_CUDA, "no CUDA device"); }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    h->max_smem = (size_t)optin;
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    // twiddle constants exp(-2 pi i k / 32)
    {
        double re[32], im[32];
        for (int k = 0; k < 32; ++k) { re[k] = cos(2.0 * M_PI * k / 32.0); im[k] = -sin(2.0 * M_PI * k / 32.0); }
        if (upload_twiddle_constants(re, im) != cudaSuccess) { delete h; return fail(ND_ERR_CUDA, "twiddle upload failed"); }
    }
    long long off = 0, soff = 0;
    for (int d = 0; d < n_disks; ++d) {
        const nd_disk_desc &ds = disks[d];
        if (!(ds.R > 0 && ds.L > 0 && ds.a > 0 && ds.Ms > 0 && ds.A > 0 && ds.gamma > 0)) {
            nd_destroy(h);
            return fail(ND_ERR_ARG, "disk " + std::to_string(d) + ": R, L, a, Ms, A, gamma must be positive");
        }
        DiskInfo di;
        di.desc = ds;
        di.D = (int)floor(2.0 * ds.R / ds.a + 0.5);
        if (di.D < 1) { nd_destroy(h); return fail(ND_ERR_ARG, "disk smaller than one cell"); }
        di.Dpad = (di.D + 3) / 4 * 4;
        di.P = padded_size(2 * di.D - 1, allow3);
        if (di.P > 1024) { nd_destroy(h); return fail(ND_ERR_ARG, "disk too large: padded grid above 1024"); }
        di.lambda = sqrt(2.0 * ds.A / (kMu0 * ds.Ms * ds.Ms));
        di.cfac = ds.a * ds.a / (di.lambda * di.lambda);
        di.B0 = 2.0 * ds.A / (ds.a * ds.a * ds.Ms);
        di.t0 = 1.0 / (ds.gamma * di.B0);
        di.J = 2.0 * ds.A * ds.L;
        const double ro = ds.a / sqrt(M_PI), q = sqrt(ds.L * ds.L + ro * ro);
        di.Nz = (ds.L + ro - q) / ds.L;
        di.Nx = (q - ro) / (2.0 * ds.L);
        {   // derivatives with respect to l = L/a (lengths in units of a)
            const double l = ds.L / ds.a, rol = 1.0 / sqrt(M_PI), ql = sqrt(l * l + rol * rol);
            di.dNz = rol * (rol - ql) / (ql * l * l);
            di.dNx = rol * (ql - rol) / (2.0 * ql * l * l);
        }
        for (int k = 0; k < 3; ++k) di.h[k] = ds.hext[k] / ds.Ms;
        di.mask.assign((size_t)di.D * di.D, 0);
        const double rr = (ds.R / ds.a) * (ds.R / ds.a);
        for (int j = 0; j < di.D; ++j)
            for (int i = 0; i < di.D; ++i) {
                const double x = i - 0.5 * (di.D - 1), y = j - 0.5 * (di.D - 1);
                const bool in = (x * x + y * y) <= rr;
                di.mask[(size_t)j * di.D + i] = in;
                di.C += in;
            }
        const int nr = replicas_per_disk ? replicas_per_disk[d] : 1;
        if (nr < 0) { nd_destroy(h); return fail(ND_ERR_ARG, "negative replica count"); }
        for (int k = 0; k < nr; ++k) {
            h->rep_disk.push_back(d);
            h->rep_off.push_back(off);
            h->rep_spec_off.push_back(soff);
            h->alpha.push_back(ds.alpha);
            off += 3LL * di.D * di.Dpad;
            soff += (long long)spec_words(di.P, di.D);
        }
        h->disks.push_back(std::move(di));
    }
    const int B = (int)h->rep_disk.size();
    if (B < 1) { nd_destroy(h); return fail(ND_ERR_ARG, "no replicas"); }
    h->state_elems = off;
    h->spec_words = soff;
    // size classes by P
    std::map<int, int> cls;
    for (int r = 0; r < B; ++r) {
        const DiskInfo &d = h->disks[h->rep_disk[r]];
        auto it = cls.find(d.P);
        if (it == cls.end()) {
            cls[d.P] = (int)h->classes.size();
            SizeClass c;
            c.P = d.P;
            h->classes.push_back(c);
            it = cls.find(d.P);
        }
        SizeClass &c = h->classes[it->second];
        c.reps.push_back(r);
        c.maxD = std::max(c.maxD, d.D);
        c.maxDpad = std::max(c.maxDpad, d.Dpad);
    }
    int rc = setup_class_paths(h);
    if (rc) { nd_destroy(h); return rc; }
    if (h->classes.size() > 1) {
        bool ok = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) == cudaSuccess;
        for (size_t k = 1; ok && k < h->classes.size(); ++k) {
            cudaStream_t s2 = nullptr;
            cudaEvent_t e2 = nullptr;
            ok = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) == cudaSuccess;
            if (s2) h->side.push_back(s2);
            if (e2) h->join_ev.push_back(e2);
        }
        if (!ok) { nd_destroy(h); return fail(ND_ERR_CUDA, "side streams for the size classes"); }
    }
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(e);
        nd_destroy(h);
        return fail(ND_ERR_CUDA, m);
    };
    cudaError_t e;
    for (auto &c : h->classes) {
        if ((e = cudaMalloc(&c.work_d, sizeof(int) * c.reps.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        if ((e = cudaMemcpy(c.work_d, c.reps.data(), sizeof(int) * c.reps.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy");
        if (!h->tw64.count(c.P)) {
            std::vector<double> t64(2 * c.P);
            std::vector<float> t32(2 * c.P);
            for (int k = 0; k < c.P; ++k) {
                t64[2 * k] = cos(2.0 * M_PI * k / c.P);
                t64[2 * k + 1] = -sin(2.0 * M_PI * k / c.P);
                t32[2 * k] = (float)t64[2 * k];
                t32[2 * k + 1] = (float)t64[2 * k + 1];
            }
            void *p64 = nullptr, *p32 = nullptr;
            if ((e = cudaMalloc(&p64, sizeof(double) * 2 * c.P)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
            h->tw64[c.P] = p64;
            if ((e = cudaMalloc(&p32, sizeof(float) * 2 * c.P)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
            h->tw32[c.P] = p32;
            cudaMemcpy(p64, t64.data(), sizeof(double) * 2 * c.P, cudaMemcpyHostToDevice);
            cudaMemcpy(p32, t32.data(), sizeof(float) * 2 * c.P, cudaMemcpyHostToDevice);
        }
    }
    if ((e = cudaMallocHost(&h->reps_ring, sizeof(Replica) * B * nd_handle::kSlots)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocHost");
    h->reps_h = h->reps_ring;
    for (int k = 0; k < nd_handle::kSlots; ++k)
        if ((e = cudaEventCreateWithFlags(&h->slot_ev[k], cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaMalloc(&h->reps_d, sizeof(Replica) * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->red_d, sizeof(double) * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMallocHost(&h->red_h, sizeof(double) * 4 * B)) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaMalloc(&h->aux_d, sizeof(double) * 4 * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->aux_i, sizeof(int) * 2 * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->acc, h->elt * h->state_elems)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->rio_d, sizeof(RelaxIO) * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->flags_d, sizeof(int) * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->status_d, sizeof(unsigned))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMemset(h->status_d, 0, sizeof(unsigned))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
    if ((e = cudaMallocHost(&h->rio_h, sizeof(RelaxIO) * B)) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    if ((e = cudaMalloc(&h->core_d, sizeof(double) * 4 * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->core_part, sizeof(double) * 2 * kCoreMaxBlocks * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&h->a_rep, sizeof(double) * B)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    {
        std::vector<double> av(B);
        for (int r = 0; r < B; ++r) av[r] = h->disks[h->rep_disk[r]].desc.a;
        cudaMemcpy(h->a_rep, av.data(), sizeof(double) * B, cudaMemcpyHostToDevice);
    }
    bool any_global = false, any_global64 = false;
    for (auto &c : h->classes) { any_global |= !c.fused_main; any_global64 |= !c.fused_fp64; }
    if (any_global || any_global64) {
        if ((e = cudaMalloc(&h->spec, sizeof(double) * 2 * h->spec_words)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    }
    if (any_global && (e = cudaMalloc(&h->ms, h->elt * h->state_elems)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if (h->prec == ND_FP32 && (e = cudaMalloc((void **)&h->y64, sizeof(double) * h->state_elems)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc");
    if (any_global64 && (e = cudaMalloc((void **)&h->ms64, sizeof(double) * h->state_elems)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc");
    for (int d = 0; d < n_disks; ++d) {
        DiskInfo &di = h->disks[d];
        const size_t kh = ghat_table_entries(di.P);
        if ((e = cudaMalloc(&di.mask_d, di.mask.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        if ((e = cudaMalloc(&di.cells_d, sizeof(int) * di.mask.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        if ((e = upload_mask(di)) != cudaSuccess) return cuda_fail(e, "mask upload");
        if ((e = cudaMalloc(&di.ghat64, sizeof(double) * kh)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        if ((e = cudaMalloc(&di.ghat32, sizeof(float) * kh)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        if ((e = cudaMalloc(&di.ghatL, sizeof(double) * kh)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    }
    for (int d = 0; d < n_disks; ++d) {
        rc = nd_set_green_tensor(h, d, nullptr);
        if (rc) { std::string m = g_err; nd_destroy(h); return fail(rc, m); }
    }
    *out = h;
    g_err.clear();
    return ND_OK;
}

void nd_destroy(nd_handle *h)
{
    if (!h) return;
    for (auto &d : h->disks) {
        cudaFree(d.mask_d); cudaFree(d.cells_d); cudaFree(d.ghat64); cudaFree(d.ghat32); cudaFree(d.ghatL);
        cudaFree(d.sched32); cudaFree(d.sched64);
    }
    for (auto st2 : h->side) { cudaStreamSynchronize(st2); cudaStreamDestroy(st2); }
    for (auto e2 : h->join_ev) cudaEventDestroy(e2);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    for (auto &c : h->classes) { cudaFree(c.work_d); cudaFree(c.segs_d); cudaFree(c.seg_off_d); }
    cudaFree(h->flags_d);
    cudaFree(h->status_d);
    for (auto &kv : h->tw64) cudaFree(kv.second);
    for (auto &kv : h->tw32) cudaFree(kv.second);
    for (int k = 0; k < nd_handle::kSlots; ++k)
        if (h->slot_ev[k]) { cudaEventSynchronize(h->slot_ev[k]); cudaEventDestroy(h->slot_ev[k]); }
    cudaFreeHost(h->reps_ring);
    cudaFree(h->reps_d);
    cudaFree(h->red_d);
    cudaFreeHost(h->red_h);
    cudaFree(h->aux_d);
    cudaFree(h->aux_i);
    cudaFree(h->rio_d);
    cudaFree(h->relax_part);
    cudaFree(h->series);
    cudaFree(h->series_count);
    cudaFree(h->psd_work);
    cudaFreeHost(h->rio_h);
    cudaFree(h->stats);
    cudaFree(h->hist_r);
    cudaFree(h->hist_v);
    cudaFree(h->core_d);
    cudaFree(h->core_part);
    cudaFree(h->a_rep);
    cudaFree(h->acc);
    cudaFree(h->ms);
    cudaFree(h->spec);
    cudaFree(h->stage_in);
    cudaFree(h->stage_out);
    cudaFree(h->y64);
    cudaFree(h->ms64);
    delete h;
}

int nd_get_info(const nd_handle *h, int *n_replicas, long long *state_elems)
{
    if (int rc = check_handle(h)) return rc;
    if (n_replicas) *n_replicas = (int)h->rep_disk.size();
    if (state_elems) *state_elems = h->state_elems;
    return ND_OK;
}

int nd_replica_layout(const nd_handle *h, int r, int *D, int *Dpad, int *P, long long *offset, int *n_cells)
{
    if (int rc = check_handle(h)) return rc;
    if (r < 0 || r >= (int)h->rep_disk.size()) return fail(ND_ERR_ARG, "replica index out of range");
    const DiskInfo &d = h->disks[h->rep_disk[r]];
    if (D) *D = d.D;
    if (Dpad) *Dpad = d.Dpad;
    if (P) *P = d.P;
    if (offset) *offset = h->rep_off[r];
    if (n_cells) *n_cells = d.C;
    return ND_OK;
}

int nd_disk_mask(const nd_handle *h, int d, unsigned char *mask_out)
{
    if (int rc = check_handle(h)) return rc;
    if (d < 0 || d >= (int)h->disks.size() || !mask_out) return fail(ND_ERR_ARG, "bad disk index or output");
    memcpy(mask_out, h->disks[d].mask.data(), h->disks[d].mask.size());
    return ND_OK;
}

int nd_units(const nd_handle *h, int d, double out[8])
{
    if (int rc = check_handle(h)) return rc;
    if (d < 0 || d >= (int)h->disks.size() || !out) return fail(ND_ERR_ARG, "bad disk index or output");
    const DiskInfo &di = h->disks[d];
    out[0] = di.lambda; out[1] = di.cfac; out[2] = di.B0; out[3] = di.t0;
    out[4] = di.J; out[5] = di.Nx; out[6] = di.Nz; out[7] = di.C;
    return ND_OK;
}

int nd_set_green_tensor(nd_handle *h, int d, const double *Gq)
{
    if (int rc = check_handle(h)) return rc;
    if (d < 0 || d >= (int)h->disks.size()) return fail(ND_ERR_ARG, "bad disk index");
    DiskInfo &di = h->disks[d];
    double *work = nullptr, *gq = nullptr;
    ND_CUDA(cudaMalloc(&work, sizeof(double) * build_ghat_work_doubles(di.P, di.D)));
    if (Gq) {
        if (cudaMalloc(&gq, sizeof(double) * 4 * di.D * di.D) != cudaSuccess) {
            cudaFree(work);
            return fail(ND_ERR_CUDA, "cudaMalloc");
        }
        cudaMemcpy(gq, Gq, sizeof(double) * 4 * di.D * di.D, cudaMemcpyDefault);
    }
    cudaError_t e = build_ghat(di.P, di.D, di.desc.L / di.desc.a, di.Nx, di.Nz, di.cfac, gq, di.ghat64, di.ghat32, work, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    // the thickness derivative always follows the paper's closed forms
    if (e == cudaSuccess) e = build_ghat_dl(di.P, di.D, di.desc.L / di.desc.a, di.dNx, di.dNz, di.cfac, di.ghatL, work, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(work);
    cudaFree(gq);
    if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("spectral kernel build: ") + cudaGetErrorString(e));
    return ND_OK;
}

int nd_set_mask(nd_handle *h, int d, const unsigned char *mask)
{
    if (int rc = check_handle(h)) return rc;
    if (d < 0 || d >= (int)h->disks.size() || !mask) return fail(ND_ERR_ARG, "bad disk index or null mask");
    DiskInfo &di = h->disks[d];
    int C = 0;
    for (size_t i = 0; i < di.mask.size(); ++i) {
        di.mask[i] = mask[i] ? 1 : 0;
        C += di.mask[i];
    }
    di.C = C;
    ND_CUDA(cudaDeviceSynchronize());   // kernels in flight may still read the old cell list
    ND_CUDA(upload_mask(di));
    return ND_OK;
}

int nd_set_field_schedule(nd_handle *h, int d, long long n_steps, const double *H)
{
    if (int rc = check_handle(h)) return rc;
    if (d < 0 || d >= (int)h->disks.size()) return fail(ND_ERR_ARG, "bad disk index");
    if (n_steps < 0 || (n_steps > 0 && !H)) return fail(ND_ERR_ARG, "need n_steps >= 0 and a field array");
    DiskInfo &di = h->disks[d];
    ND_CUDA(cudaDeviceSynchronize());   // kernels in flight may still read the old schedule
    cudaFree(di.sched32);
    cudaFree(di.sched64);
    di.sched32 = nullptr;
    di.sched64 = nullptr;
    di.nsched = 0;
    h->rk4_step = 0;
    if (n_steps == 0) return ND_OK;
    std::vector<double> v64(3 * (size_t)n_steps);
    std::vector<float> v32(3 * (size_t)n_steps);
    for (size_t i = 0; i < v64.size(); ++i) {
        v64[i] = di.cfac * (H[i] / di.desc.Ms);   // rounded as the static field is
        v32[i] = (float)v64[i];
    }
    ND_CUDA(cudaMalloc(&di.sched64, sizeof(double) * v64.size()));
    ND_CUDA(cudaMalloc(&di.sched32, sizeof(float) * v32.size()));
    ND_CUDA(cudaMemcpy(di.sched64, v64.data(), sizeof(double) * v64.size(), cudaMemcpyHostToDevice));
    ND_CUDA(cudaMemcpy(di.sched32, v32.data(), sizeof(float) * v32.size(), cudaMemcpyHostToDevice));
    di.nsched = n_steps;
    return ND_OK;
}

int nd_set_damping(nd_handle *h, const double *alpha)
{
    if (int rc = check_handle(h)) return rc;
    if (!alpha) return fail(ND_ERR_ARG, "null alpha");
    for (size_t r = 0; r < h->alpha.size(); ++r) h->alpha[r] = alpha[r];
    return ND_OK;
}

int nd_effective_field(nd_handle *h, const void *m, void *b, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr, *bd = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    if (!b) return fail(ND_ERR_ARG, "null output");
    if (int rc = stage_in(h, b, &bd, false, st, &h->stage_out)) return rc;
    ND_CUDA(cudaMemsetAsync(bd, 0, (size_t)h->state_elems * h->elt, st));
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    if (int rc = run_mode(h, M_FIELD, false, md, bd, 1, st)) return rc;
    return stage_out(h, b, bd, st);
}

int nd_energy(nd_handle *h, const void *m, double *E_out, double *dEdL_out, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!E_out) return fail(ND_ERR_ARG, "null E_out");
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    const int B = (int)h->rep_disk.size();
    void *y64 = md;
    if (h->prec == ND_FP32) {
        ND_CUDA(launch_convert(ND_PREC_FP64, md, h->y64, (size_t)h->state_elems, st));
        y64 = h->y64;
    }
    fill_reps(h, true, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    ND_CUDA(cudaMemsetAsync(h->red_d, 0, sizeof(double) * B, st));
    if (int rc = run_mode(h, M_ENERGY, true, y64, nullptr, 1, st)) return rc;
    ND_CUDA(cudaMemcpyAsync(h->red_h, h->red_d, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < B; ++r) E_out[r] = h->red_h[r];
    if (dEdL_out) {
        // -1/2 sum_i m_i . (c dh^M/dl)_i with the derivative kernel = d(E/J)/dl at fixed m;
        // then dE/dL = 2A E/J + J d(E/J)/dl / a  (E = J E/J, J = 2AL)
        fill_reps(h, true, 0.0, nullptr, nullptr, 0, TAB_DL);
        upload_reps(h, st);
        ND_CUDA(cudaMemsetAsync(h->red_d, 0, sizeof(double) * B, st));
        if (int rc = run_mode(h, M_ENERGY, true, y64, nullptr, 1, st)) return rc;
        ND_CUDA(cudaMemcpyAsync(h->red_h, h->red_d, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
        ND_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < B; ++r) {
            const DiskInfo &d = h->disks[h->rep_disk[r]];
            dEdL_out[r] = 2.0 * d.desc.A * E_out[r] + d.J * h->red_h[r] / d.desc.a;
        }
    }
    return ND_OK;
}

int nd_step_rk4(nd_handle *h, void *m, long long n_steps, double dt_seconds, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (n_steps < 0) return fail(ND_ERR_ARG, "negative n_steps");
    if (!(dt_seconds > 0)) return fail(ND_ERR_ARG, "dt must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    if (n_steps > 0) {
        fill_reps(h, h->prec == ND_FP64, dt_seconds, nullptr, nullptr, h->rk4_step);
        upload_reps(h, st);
        if (int rc = run_mode(h, M_RK4, false, md, nullptr, n_steps, st)) return rc;
        h->rk4_step += (unsigned long long)n_steps;
    }
    return stage_out(h, m, md, st);
}

int nd_step_heun(nd_handle *h, void *m, long long n_steps, double dt_seconds, const double *T_kelvin,
                 const unsigned long long *seed, unsigned long long step0, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (n_steps < 0) return fail(ND_ERR_ARG, "negative n_steps");
    if (!(dt_seconds > 0)) return fail(ND_ERR_ARG, "dt must be positive");
    if (!T_kelvin || !seed) return fail(ND_ERR_ARG, "T_kelvin and seed are required");
    for (size_t r = 0; r < h->rep_disk.size(); ++r)
        if (!(T_kelvin[r] >= 0)) return fail(ND_ERR_ARG, "temperatures must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    if (n_steps > 0) {
        fill_reps(h, h->prec == ND_FP64, dt_seconds, T_kelvin, seed, step0);
        upload_reps(h, st);
        if (int rc = run_mode(h, M_HEUN, false, md, nullptr, n_steps, st)) return rc;
    }
    return stage_out(h, m, md, st);
}

int nd_relax_constrained(nd_handle *h, void *m, const double *X, double tol, int max_iter, double *U_out,
                         double *lambda_out, int *iters_out, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!X) return fail(ND_ERR_ARG, "null X");
    if (max_iter < 0 || !(tol > 0)) return fail(ND_ERR_ARG, "max_iter must be >= 0 and tol > 0");
    bool any_global = false;
    for (auto &c : h->classes) any_global |= !c.fused_main;
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    const int B = (int)h->rep_disk.size();
    if (any_global) {
        if (int rc = ensure_alloc(&h->ms, h->elt * h->state_elems)) return rc;
        if (int rc = ensure_alloc(&h->spec, sizeof(double) * 2 * h->spec_words)) return rc;
        if (int rc = ensure_alloc((void **)&h->relax_part, sizeof(double) * 6 * kRelaxBlocks * (size_t)B)) return rc;
    }
    ND_CUDA(cudaStreamSynchronize(st));   // the pinned relaxation block is rewritten below
    for (int r = 0; r < B; ++r) {
        const DiskInfo &d = h->disks[h->rep_disk[r]];
        RelaxIO &R = h->rio_h[r];
        R.X[0] = X[2 * r] / d.desc.a;
        R.X[1] = X[2 * r + 1] / d.desc.a;
        R.lam[0] = R.lam[1] = 0.0;
        R.resid = 0.0;
        R.iters = 0;
        R.status = 1;
    }
    ND_CUDA(cudaMemcpyAsync(h->rio_d, h->rio_h, sizeof(RelaxIO) * B, cudaMemcpyHostToDevice, st));
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    const int prec = h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32;
    for (auto &c : h->classes) {
        const DiskInfo &d = h->disks[h->rep_disk[c.reps[0]]];
        const double rcut = 4.0 * d.lambda / d.desc.a;
        LaunchArgs a;
        a.mode = M_RELAX;
        a.reps = h->reps_d;
        a.work = c.work_d;
        a.nwork = (int)c.reps.size();
        a.y = md;
        a.red = h->red_d;
        a.tw = (prec == ND_PREC_FP64) ? h->tw64[c.P] : h->tw32[c.P];
        a.smem = c.smem_main;
        a.stream = st;
        a.rio = h->rio_d;
        a.eta = 0.5;
        a.tol = tol;
        a.rc2 = rcut * rcut;
        a.max_iter = max_iter;
        if (c.fused_main) {
            ND_CUDA(launch_fused(c.P, prec, a));
        } else {
            a.ms = h->ms;
            a.spec = h->spec;
            a.part = h->relax_part;
            a.rio_host = h->rio_h;
            a.n_rio = B;
            a.work_host = c.reps.data();
            a.n_sm = h->n_sm;
            ND_CUDA(launch_global(c.P, prec, a, c.maxD));
        }
    }
    ND_CUDA(cudaMemcpyAsync(h->rio_h, h->rio_d, sizeof(RelaxIO) * B, cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    int rc = ND_OK;
    for (int r = 0; r < B; ++r) {
        if (lambda_out) { lambda_out[2 * r] = h->rio_h[r].lam[0]; lambda_out[2 * r + 1] = h->rio_h[r].lam[1]; }
        if (iters_out) iters_out[r] = h->rio_h[r].iters;
        if (h->rio_h[r].status != 0) rc = ND_ERR_NOT_CONVERGED;
    }
    if (U_out) {
        int e = nd_energy(h, md, U_out, nullptr, stream);
        if (e) return e;
    }
    if (int e = stage_out(h, m, md, st)) return e;
    if (rc) g_err = "relaxation did not converge within max_iter in at least one replica";
    return rc;
}

int nd_relax_sweep_grad(nd_handle *h, void *m, const void *grad, const double *X, double *lambda, double tol,
                        double *resid_out, int *moved_out, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!m || !grad || !X || !lambda) return fail(ND_ERR_ARG, "null argument");
    if (!is_device_ptr(m) || !is_device_ptr(grad)) return fail(ND_ERR_ARG, "m and grad must be device buffers");
    if (!(tol >= 0)) return fail(ND_ERR_ARG, "tol must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int B = (int)h->rep_disk.size();
    if (int rc = ensure_alloc((void **)&h->relax_part, sizeof(double) * 6 * kRelaxBlocks * (size_t)B)) return rc;
    ND_CUDA(cudaStreamSynchronize(st));   // the pinned relaxation block and aux_d are rewritten below
    std::vector<double> gs(B);
    for (int r = 0; r < B; ++r) {
        const DiskInfo &d = h->disks[h->rep_disk[r]];
        RelaxIO &R = h->rio_h[r];
        R.X[0] = X[2 * r] / d.desc.a;
        R.X[1] = X[2 * r + 1] / d.desc.a;
        R.lam[0] = lambda[2 * r];
        R.lam[1] = lambda[2 * r + 1];
        R.resid = 0.0;
        R.iters = 0;
        R.status = 1;
        gs[r] = -1.0 / d.J;
    }
    ND_CUDA(cudaMemcpyAsync(h->rio_d, h->rio_h, sizeof(RelaxIO) * B, cudaMemcpyHostToDevice, st));
    ND_CUDA(cudaMemcpyAsync(h->aux_d, gs.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st));
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    const int prec = h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32;
    for (auto &c : h->classes) {
        const DiskInfo &d = h->disks[h->rep_disk[c.reps[0]]];
        const double rcut = 4.0 * d.lambda / d.desc.a;
        LaunchArgs a;
        a.reps = h->reps_d;
        a.work = c.work_d;
        a.nwork = (int)c.reps.size();
        a.y = m;
        a.stream = st;
        a.rio = h->rio_d;
        a.part = h->relax_part;
        a.eta = 0.5;
        a.tol = tol;
        a.rc2 = rcut * rcut;
        ND_CUDA(launch_relax_grad(prec, a, c.maxD, grad, h->aux_d));
    }
    ND_CUDA(cudaMemcpyAsync(h->rio_h, h->rio_d, sizeof(RelaxIO) * B, cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < B; ++r) {
        lambda[2 * r] = h->rio_h[r].lam[0];
        lambda[2 * r + 1] = h->rio_h[r].lam[1];
        if (resid_out) resid_out[r] = h->rio_h[r].resid;
        if (moved_out) moved_out[r] = h->rio_h[r].status != 0;
    }
    return ND_OK;
}

int nd_init_vortex(nd_handle *h, void *m, const double *X0, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!X0) return fail(ND_ERR_ARG, "null X0");
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, false, st, &h->stage_in)) return rc;
    const int B = (int)h->rep_disk.size();
    std::vector<double> xc(2 * B);
    std::vector<int> pc(2 * B);
    for (int r = 0; r < B; ++r) {
        const DiskInfo &d = h->disks[h->rep_disk[r]];
        xc[2 * r] = X0[2 * r] / d.desc.a;
        xc[2 * r + 1] = X0[2 * r + 1] / d.desc.a;
        pc[2 * r] = d.desc.polarity >= 0 ? 1 : -1;
        pc[2 * r + 1] = d.desc.chirality >= 0 ? 1 : -1;
    }
    ND_CUDA(cudaMemcpyAsync(h->aux_d, xc.data(), sizeof(double) * 2 * B, cudaMemcpyHostToDevice, st));
    ND_CUDA(cudaMemcpyAsync(h->aux_i, pc.data(), sizeof(int) * 2 * B, cudaMemcpyHostToDevice, st));
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    ND_CUDA(cudaMemsetAsync(md, 0, (size_t)h->state_elems * h->elt, st));
    for (auto &c : h->classes) {
        const DiskInfo &d = h->disks[h->rep_disk[c.reps[0]]];
        ND_CUDA(launch_init_vortex(h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32, h->reps_d, c.work_d,
                                   (int)c.reps.size(), c.maxD, md, h->aux_d, h->aux_i, d.lambda / d.desc.a, st));
    }
    ND_CUDA(cudaStreamSynchronize(st));   // the host arrays above go out of scope
    return stage_out(h, m, md, st);
}

int nd_vortex_core(nd_handle *h, const void *m, double *Xc_out, int *status, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!Xc_out) return fail(ND_ERR_ARG, "null Xc_out");
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    const int B = (int)h->rep_disk.size();
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    for (auto &c : h->classes) {
        const DiskInfo &d = h->disks[h->rep_disk[c.reps[0]]];
        for (int r : c.reps)
            if (h->disks[h->rep_disk[r]].lambda / h->disks[h->rep_disk[r]].desc.a != d.lambda / d.desc.a)
                return fail(ND_ERR_ARG, "vortex_core: disks of one size class must share lambda_ex / a");
        const double rcut = 4.0 * d.lambda / d.desc.a;
        ND_CUDA(launch_vortex_core(h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32, h->reps_d, c.work_d,
                                   (int)c.reps.size(), c.maxD, md, rcut * rcut, h->core_part, h->aux_d, st));
    }
    ND_CUDA(cudaMemcpyAsync(h->red_h, h->aux_d, sizeof(double) * 4 * B, cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    int rc = ND_OK;
    for (int r = 0; r < B; ++r) {
        const double a = h->disks[h->rep_disk[r]].desc.a;
        const bool none = h->red_h[4 * r + 2] != 0.0;
        Xc_out[2 * r] = none ? 0.0 : h->red_h[4 * r] * a;
        Xc_out[2 * r + 1] = none ? 0.0 : h->red_h[4 * r + 1] * a;
        if (status) status[r] = none ? ND_ERR_NO_VORTEX : ND_OK;
        if (none) rc = ND_ERR_NO_VORTEX;
    }
    if (rc) g_err = "no vortex found in at least one replica";
    return rc;
}

int nd_check_status(nd_handle *h, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    ND_CUDA(cudaStreamSynchronize(st));
    unsigned v = 0;
    ND_CUDA(cudaMemcpy(&v, h->status_d, sizeof(v), cudaMemcpyDeviceToHost));
    ND_CUDA(cudaMemset(h->status_d, 0, sizeof(v)));
    if (v & ND_DEV_TIMEOUT) return fail(ND_ERR_TIMEOUT, "a bounded device-side wait expired (replica hand-over)");
    if (v & ND_DEV_NAN) return fail(ND_ERR_NAN, "non-finite values in the state");
    return ND_OK;
}

int nd_selftest_handover_timeout(nd_handle *h, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    auto &c = h->classes[0];
    if (!c.fused_main || h->prec == ND_FP64)
        return fail(ND_ERR_ARG, "the hand-over self-test needs an on-chip FP32 size class first in the handle");
    cudaStream_t st = (cudaStream_t)stream;
    // one CTA, one segment of one step that waits for replica c.reps[0]'s flag,
    // which no segment signals
    const SegmentHost seg = {c.reps[0], 1, 0, 0, 0, 1};
    const int off[2] = {0, 1};
    void *segs_d = nullptr, *off_d = nullptr;
    ND_CUDA(cudaMalloc(&segs_d, sizeof(seg)));
    cudaError_t e = cudaMalloc(&off_d, sizeof(off));
    if (e == cudaSuccess) e = cudaMemcpy(segs_d, &seg, sizeof(seg), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(off_d, off, sizeof(off), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flags_d, 0, sizeof(int) * h->rep_disk.size(), st);
    if (e == cudaSuccess) {
        LaunchArgs a;
        a.mode = M_HEUN;
        a.reps = h->reps_d;
        a.work = c.work_d;
        a.nwork = (int)c.reps.size();
        a.y = h->acc;     // never touched: the segment gives up before reading any state
        a.acc = h->acc;
        a.tw = h->tw32[c.P];
        a.nsteps = 1;
        a.smem = c.smem_main;
        a.stream = st;
        a.status = h->status_d;
        a.segs = segs_d;
        a.seg_off = (const int *)off_d;
        a.flags = h->flags_d;
        a.ncta = 1;
        a.n_sm = h->n_sm;
        e = launch_fused(c.P, ND_PREC_FP32, a);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(segs_d);
    cudaFree(off_d);
    if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("hand-over self-test: ") + cudaGetErrorString(e));
    return ND_OK;
}

int nd_stats_reset(nd_handle *h, double r_max, int r_bins, double v_max, int v_bins)
{
    if (int rc = check_handle(h)) return rc;
    if (!(r_max > 0) || !(v_max > 0) || r_bins < 1 || v_bins < 1) return fail(ND_ERR_ARG, "bad histogram range");
    const int B = (int)h->rep_disk.size();
    cudaFree(h->stats); cudaFree(h->hist_r); cudaFree(h->hist_v);
    h->stats = nullptr; h->hist_r = h->hist_v = nullptr;
    ND_CUDA(cudaMalloc(&h->stats, sizeof(StatsAcc) * B));
    ND_CUDA(cudaMalloc(&h->hist_r, sizeof(unsigned long long) * B * r_bins));
    ND_CUDA(cudaMalloc(&h->hist_v, sizeof(unsigned long long) * B * v_bins));
    ND_CUDA(cudaMemset(h->stats, 0, sizeof(StatsAcc) * B));
    ND_CUDA(cudaMemset(h->hist_r, 0, sizeof(unsigned long long) * B * r_bins));
    ND_CUDA(cudaMemset(h->hist_v, 0, sizeof(unsigned long long) * B * v_bins));
    h->rbins = r_bins; h->vbins = v_bins; h->r_max = r_max; h->v_max = v_max;
    return ND_OK;
}

static int stats_launches(nd_handle *h, const void *m, double dt_sample_seconds, cudaStream_t st, const Replica *reps)
{
    for (auto &c : h->classes) {
        const DiskInfo &d = h->disks[h->rep_disk[c.reps[0]]];
        const double rcut = 4.0 * d.lambda / d.desc.a;
        ND_CUDA(launch_vortex_core(h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32, reps, c.work_d,
                                   (int)c.reps.size(), c.maxD, m, rcut * rcut, h->core_part, h->core_d, st));
        ND_CUDA(launch_stats_update(c.work_d, (int)c.reps.size(), h->core_d, h->a_rep, h->stats, h->hist_r, h->hist_v,
                                    h->rbins, h->vbins, h->r_max, h->v_max, dt_sample_seconds, st));
    }
    return ND_OK;
}

int nd_stats_sample(nd_handle *h, const void *m, double dt_sample_seconds, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!h->stats) return fail(ND_ERR_ARG, "call nd_stats_reset first");
    if (!(dt_sample_seconds > 0)) return fail(ND_ERR_ARG, "dt_sample must be positive");
    if (!m || !is_device_ptr(m)) return fail(ND_ERR_ARG, "nd_stats_sample needs a device state");
    cudaStream_t st = (cudaStream_t)stream;
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    return stats_launches(h, m, dt_sample_seconds, st, h->reps_d);
}

int nd_stats_read(nd_handle *h, double *moments, unsigned long long *r_hist, unsigned long long *v_hist, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!h->stats) return fail(ND_ERR_ARG, "call nd_stats_reset first");
    cudaStream_t st = (cudaStream_t)stream;
    const int B = (int)h->rep_disk.size();
    ND_CUDA(cudaStreamSynchronize(st));
    std::vector<StatsAcc> s(B);
    ND_CUDA(cudaMemcpy(s.data(), h->stats, sizeof(StatsAcc) * B, cudaMemcpyDeviceToHost));
    if (moments)
        for (int r = 0; r < B; ++r) {
            double *o = moments + 7 * r;
            o[0] = s[r].n; o[1] = s[r].sx; o[2] = s[r].sy; o[3] = s[r].sr2;
            o[4] = s[r].nv; o[5] = s[r].sv2; o[6] = s[r].no_vortex;
        }
    if (r_hist) ND_CUDA(cudaMemcpy(r_hist, h->hist_r, sizeof(unsigned long long) * B * h->rbins, cudaMemcpyDeviceToHost));
    if (v_hist) ND_CUDA(cudaMemcpy(v_hist, h->hist_v, sizeof(unsigned long long) * B * h->vbins, cudaMemcpyDeviceToHost));
    return ND_OK;
}

// Statistics record: tag, replica count, bin counts, ranges, then per replica
// the StatsAcc fields as doubles (have_prev as 0/1), then both histograms.
namespace {
constexpr unsigned long long kStatsTag = 0x3154535344444e4eull;   // "NNDDSST1"
constexpr int kStatsWords = 10;                                   // doubles per replica
}

size_t nd_stats_save_bytes(const nd_handle *h)
{
    if (!h || !h->stats) return 0;
    const size_t B = h->rep_disk.size();
    return sizeof(unsigned long long) * 4 + sizeof(double) * 2 + sizeof(double) * kStatsWords * B +
           sizeof(unsigned long long) * B * (size_t)(h->rbins + h->vbins);
}

int nd_stats_save(nd_handle *h, void *buf, size_t bytes, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!h->stats) return fail(ND_ERR_ARG, "no statistics to save (nd_stats_reset first)");
    if (!buf || bytes < nd_stats_save_bytes(h)) return fail(ND_ERR_ARG, "statistics record buffer too small");
    const int B = (int)h->rep_disk.size();
    ND_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<StatsAcc> s(B);
    ND_CUDA(cudaMemcpy(s.data(), h->stats, sizeof(StatsAcc) * B, cudaMemcpyDeviceToHost));
    unsigned char *p = static_cast<unsigned char *>(buf);
    const unsigned long long head[4] = {kStatsTag, (unsigned long long)B, (unsigned long long)h->rbins,
                                        (unsigned long long)h->vbins};
    std::memcpy(p, head, sizeof(head)); p += sizeof(head);
    const double range[2] = {h->r_max, h->v_max};
    std::memcpy(p, range, sizeof(range)); p += sizeof(range);
    for (int r = 0; r < B; ++r) {
        const double w[kStatsWords] = {s[r].n, s[r].sx, s[r].sy, s[r].sr2, s[r].nv, s[r].sv2, s[r].no_vortex,
                                       s[r].px, s[r].py, s[r].have_prev ? 1.0 : 0.0};
        std::memcpy(p, w, sizeof(w)); p += sizeof(w);
    }
    ND_CUDA(cudaMemcpy(p, h->hist_r, sizeof(unsigned long long) * B * h->rbins, cudaMemcpyDeviceToHost));
    p += sizeof(unsigned long long) * B * h->rbins;
    ND_CUDA(cudaMemcpy(p, h->hist_v, sizeof(unsigned long long) * B * h->vbins, cudaMemcpyDeviceToHost));
    return ND_OK;
}

int nd_stats_load(nd_handle *h, const void *buf, size_t bytes, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    const size_t hb = sizeof(unsigned long long) * 4 + sizeof(double) * 2;
    if (!buf || bytes < hb) return fail(ND_ERR_ARG, "statistics record too short");
    const unsigned char *p = static_cast<const unsigned char *>(buf);
    unsigned long long head[4];
    double range[2];
    std::memcpy(head, p, sizeof(head));
    std::memcpy(range, p + sizeof(head), sizeof(range));
    const int B = (int)h->rep_disk.size();
    if (head[0] != kStatsTag) return fail(ND_ERR_ARG, "not a statistics record");
    if (head[1] != (unsigned long long)B) return fail(ND_ERR_ARG, "statistics record of another replica count");
    if (head[2] < 1 || head[3] < 1 || head[2] > (1u << 24) || head[3] > (1u << 24))
        return fail(ND_ERR_ARG, "bad histogram sizes in the statistics record");
    const int rb = (int)head[2], vb = (int)head[3];
    const size_t need = hb + sizeof(double) * kStatsWords * B + sizeof(unsigned long long) * B * (size_t)(rb + vb);
    if (bytes < need) return fail(ND_ERR_ARG, "statistics record too short");
    ND_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (int rc = nd_stats_reset(h, range[0], rb, range[1], vb)) return rc;
    p += hb;
    std::vector<StatsAcc> s(B);
    for (int r = 0; r < B; ++r) {
        double w[kStatsWords];
        std::memcpy(w, p, sizeof(w)); p += sizeof(w);
        s[r] = StatsAcc{};
        s[r].n = w[0]; s[r].sx = w[1]; s[r].sy = w[2]; s[r].sr2 = w[3]; s[r].nv = w[4]; s[r].sv2 = w[5];
        s[r].no_vortex = w[6]; s[r].px = w[7]; s[r].py = w[8]; s[r].have_prev = w[9] != 0.0;
    }
    ND_CUDA(cudaMemcpy(h->stats, s.data(), sizeof(StatsAcc) * B, cudaMemcpyHostToDevice));
    ND_CUDA(cudaMemcpy(h->hist_r, p, sizeof(unsigned long long) * B * rb, cudaMemcpyHostToDevice));
    p += sizeof(unsigned long long) * B * rb;
    ND_CUDA(cudaMemcpy(h->hist_v, p, sizeof(unsigned long long) * B * vb, cudaMemcpyHostToDevice));
    return ND_OK;
}

int nd_mean_m(nd_handle *h, const void *m, double *out, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(ND_ERR_ARG, "null out");
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    const int B = (int)h->rep_disk.size();
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    for (auto &c : h->classes)
        ND_CUDA(launch_mean_m(h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32, h->reps_d, c.work_d, (int)c.reps.size(),
                              md, h->aux_d, st));
    ND_CUDA(cudaMemcpyAsync(h->red_h, h->aux_d, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < 3 * B; ++i) out[i] = h->red_h[i];
    return ND_OK;
}

// ---------------------------------------------------------- time series

static int series_launches(nd_handle *h, const void *md, cudaStream_t st, const Replica *reps)
{
    const int prec = h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32;
    for (auto &c : h->classes)
        ND_CUDA(launch_series_append(prec, reps ? reps : h->reps_d, c.work_d, (int)c.reps.size(), md, h->series,
                                     h->series_count, h->series_cap, st));
    ND_CUDA(launch_series_advance(h->series_count, st));
    return ND_OK;
}

int nd_series_reset(nd_handle *h, int capacity)
{
    if (int rc = check_handle(h)) return rc;
    if (capacity < 1) return fail(ND_ERR_ARG, "capacity must be >= 1");
    const int B = (int)h->rep_disk.size();
    cudaFree(h->series);
    h->series = nullptr;
    h->series_cap = 0;
    ND_CUDA(cudaMalloc(&h->series, sizeof(double) * 3 * (size_t)capacity * B));
    if (!h->series_count) ND_CUDA(cudaMalloc(&h->series_count, sizeof(unsigned long long)));
    ND_CUDA(cudaMemset(h->series_count, 0, sizeof(unsigned long long)));
    h->series_cap = capacity;
    return ND_OK;
}

int nd_series_sample(nd_handle *h, const void *m, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!h->series) return fail(ND_ERR_ARG, "nd_series_reset first");
    cudaStream_t st = (cudaStream_t)stream;
    void *md = nullptr;
    if (int rc = stage_in(h, m, &md, true, st, &h->stage_in)) return rc;
    fill_reps(h, h->prec == ND_FP64, 0.0, nullptr, nullptr, 0);
    upload_reps(h, st);
    return series_launches(h, md, st, nullptr);
}

int nd_series_read(nd_handle *h, double *out, long long *n_samples)
{
    if (int rc = check_handle(h)) return rc;
    if (!h->series) return fail(ND_ERR_ARG, "nd_series_reset first");
    unsigned long long n = 0;
    ND_CUDA(cudaDeviceSynchronize());
    ND_CUDA(cudaMemcpy(&n, h->series_count, sizeof(n), cudaMemcpyDeviceToHost));
    if (n_samples) *n_samples = (long long)n;
    const size_t kept = n < (unsigned long long)h->series_cap ? (size_t)n : (size_t)h->series_cap;
    if (out && kept) {
        const int B = (int)h->rep_disk.size();
        for (int r = 0; r < B; ++r)
            ND_CUDA(cudaMemcpy(out + (size_t)r * kept * 3, h->series + (size_t)r * h->series_cap * 3,
                               sizeof(double) * 3 * kept, cudaMemcpyDeviceToHost));
    }
    return ND_OK;
}

int nd_power_spectrum(nd_handle *h, int component, int window, double dt_sample_seconds, double *psd_out,
                      double *freq_out, int *n_windows, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (!h->series) return fail(ND_ERR_ARG, "nd_series_reset first");
    if (component < 0 || component > 2) return fail(ND_ERR_ARG, "component must be 0, 1 or 2");
    if (window != 64 && window != 128 && window != 256 && window != 512 && window != 1024)
        return fail(ND_ERR_ARG, "window must be 64, 128, 256, 512 or 1024");
    if (!(dt_sample_seconds > 0)) return fail(ND_ERR_ARG, "dt_sample_seconds must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    ND_CUDA(cudaStreamSynchronize(st));
    unsigned long long n = 0;
    ND_CUDA(cudaMemcpy(&n, h->series_count, sizeof(n), cudaMemcpyDeviceToHost));
    const long long kept = n < (unsigned long long)h->series_cap ? (long long)n : (long long)h->series_cap;
    const int nwin = (int)(kept / window), nk = window / 2 + 1;
    if (n_windows) *n_windows = nwin;
    if (nwin < 1) return fail(ND_ERR_ARG, "fewer recorded samples than one window");
    const int B = (int)h->rep_disk.size();
    if (!h->tw64.count(window)) {
        std::vector<double> t64(2 * window);
        for (int k = 0; k < window; ++k) {
            t64[2 * k] = cos(2.0 * M_PI * k / window);
            t64[2 * k + 1] = -sin(2.0 * M_PI * k / window);
        }
        void *p = nullptr;
        ND_CUDA(cudaMalloc(&p, sizeof(double) * 2 * window));
        h->tw64[window] = p;
        ND_CUDA(cudaMemcpy(p, t64.data(), sizeof(double) * 2 * window, cudaMemcpyHostToDevice));
    }
    const size_t need = (size_t)B * nwin * nk + (size_t)B * nk;
    if (need > h->psd_work_doubles) {
        cudaFree(h->psd_work);
        h->psd_work = nullptr;
        h->psd_work_doubles = 0;
        ND_CUDA(cudaMalloc(&h->psd_work, sizeof(double) * need));
        h->psd_work_doubles = need;
    }
    double *pw = h->psd_work, *psd = pw + (size_t)B * nwin * nk;
    ND_CUDA(launch_window_power(window, h->series, h->series_cap, component, nwin, B, h->tw64[window], pw, st));
    ND_CUDA(launch_psd_reduce(pw, nwin, nk, B, dt_sample_seconds / window, psd, st));
    if (psd_out) ND_CUDA(cudaMemcpyAsync(psd_out, psd, sizeof(double) * B * nk, cudaMemcpyDeviceToHost, st));
    ND_CUDA(cudaStreamSynchronize(st));
    if (freq_out)
        for (int k = 0; k < nk; ++k) freq_out[k] = k / (window * dt_sample_seconds);
    return ND_OK;
}

}  // extern "C"

// ------------------------------------------------------------- autotuning

// The plans a size class can step with in a mode: the one-CTA kernel's thread
// counts that fit, the global path, and the cluster plans the GPU can hold.
static std::vector<int> plan_candidates(const nd_handle *h, const SizeClass &c, int mode)
{
    const int prec = h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32;
    std::vector<int> cands;
    for (int v = 0; v < 3; ++v) {
        if (fused_variant_threads(c.P, v) == 0) continue;
        const size_t sm = fused_smem(c.P, prec, c.maxD, c.maxDpad, false, v);
        if (sm != (size_t)-1 && sm + 1024 <= h->max_smem) cands.push_back(v);
    }
    cands.push_back(kPlanGlobal);
    for (int pl : {kPlanCluster, kPlanCluster16})
        if (cluster_plan_fits(h, c, prec, mode == M_HEUN, plan_cluster_nc(pl))) cands.push_back(pl);
    return cands;
}

namespace {
// One handle being tuned: its method, a scratch state and its own stream.
struct TuneItem {
    nd_handle *h = nullptr;
    int mode = M_HEUN, slot = 1;
    void *tmp = nullptr;
    std::vector<double> T;
    std::vector<unsigned long long> sd;
    cudaStream_t st = nullptr;
};
}  // namespace

// The steps of every item side by side (each handle on its stream, forked
// from and joined back to st0); only_class >= 0 restricts a single item to
// that class.
static int tune_run(std::vector<TuneItem> &items, double dt, long long n_steps, cudaStream_t st0, cudaEvent_t fork,
                    const std::vector<cudaEvent_t> &joins, int only_class)
{
    const bool many = items.size() > 1;
    if (many) ND_CUDA(cudaEventRecord(fork, st0));
    for (size_t k = 0; k < items.size(); ++k) {
        TuneItem &it = items[k];
        const cudaStream_t s = many ? it.st : st0;
        if (many) ND_CUDA(cudaStreamWaitEvent(s, fork, 0));
        const bool heun = it.mode == M_HEUN;
        fill_reps(it.h, it.h->prec == ND_FP64, dt, heun ? it.T.data() : nullptr, heun ? it.sd.data() : nullptr, 0);
        upload_reps(it.h, s);
        if (int rc = run_mode(it.h, it.mode, false, it.tmp, nullptr, n_steps, s, nullptr, only_class)) return rc;
        if (many) {
            ND_CUDA(cudaEventRecord(joins[k], s));
            ND_CUDA(cudaStreamWaitEvent(st0, joins[k], 0));
        }
    }
    return ND_OK;
}

// One pass of coordinate descent over every class of every item: each
// candidate plan is timed (one warm-up, the fastest of three runs) on
// everything that shares the GPU -- the whole group of handles, or the whole
// handle when it has several classes, which step side by side -- with the
// other classes at their current plans.  A plan that is fastest alone (a
// cluster plan spreading few replicas over many SMs) can take SMs that the
// other classes need, so a class is never timed alone unless it is alone.
static int tune_items(std::vector<TuneItem> &items, double dt, long long n_steps, cudaStream_t st0)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr, fork = nullptr;
    std::vector<cudaEvent_t> joins(items.size(), nullptr);
    int rc = ND_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(ND_ERR_CUDA, "autotune events");
    for (auto &j : joins)
        if (rc == ND_OK && cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess)
            rc = fail(ND_ERR_CUDA, "autotune events");
    const bool whole = items.size() > 1 || items[0].h->classes.size() > 1;
    for (auto &it : items) {
        for (int ci = 0; ci < (int)it.h->classes.size() && rc == ND_OK; ++ci) {
            SizeClass &c = it.h->classes[ci];
            // the class's current plan is timed first and kept unless another
            // is faster by more than 2%, so that timing noise does not walk the
            // descent between near-equal plans
            std::vector<int> cands = plan_candidates(it.h, c, it.mode);
            int cur = c.plan[it.slot];
            if (cur == -1) cur = c.fused_main ? 0 : kPlanGlobal;   // what the default runs
            const auto pos = std::find(cands.begin(), cands.end(), cur);
            if (pos != cands.end()) std::rotate(cands.begin(), pos, pos + 1);
            float best_ms = 1e30f;
            int best = cands.front();
            for (int cand : cands) {
                c.plan[it.slot] = cand;
                const int only = whole ? -1 : ci;
                rc = tune_run(items, dt, n_steps, st0, fork, joins, only);   // warm-up, builds schedules
                if (rc) break;
                float ms = 1e30f;
                for (int rep = 0; rep < 3 && rc == ND_OK; ++rep) {
                    cudaEventRecord(e0, st0);
                    rc = tune_run(items, dt, n_steps, st0, fork, joins, only);
                    cudaEventRecord(e1, st0);
                    if (rc) break;
                    cudaEventSynchronize(e1);
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = std::min(ms, t);
                }
                if (rc) break;
                if (ms < (cand == cands.front() ? 1.0f : 0.98f) * best_ms) { best_ms = ms; best = cand; }
            }
            c.plan[it.slot] = best;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (fork) cudaEventDestroy(fork);
    for (auto j : joins)
        if (j) cudaEventDestroy(j);
    return rc;
}

// A tuning item for handle h: global-path buffers (a candidate), a scratch
// state holding the analytic centred vortex, 300 K and seeds 0..B-1.
static int tune_item_make(nd_handle *h, int method, cudaStream_t st, TuneItem &it)
{
    if (int rc = ensure_alloc(&h->ms, h->elt * h->state_elems)) return rc;
    if (int rc = ensure_alloc(&h->spec, sizeof(double) * 2 * h->spec_words)) return rc;
    const int B = (int)h->rep_disk.size();
    it.h = h;
    it.mode = method == ND_METHOD_RK4 ? M_RK4 : M_HEUN;
    it.slot = method == ND_METHOD_RK4 ? 0 : 1;
    ND_CUDA(cudaMalloc(&it.tmp, h->elt * h->state_elems));
    std::vector<double> X0(2 * B, 0.0);
    if (int rc = nd_init_vortex(h, it.tmp, X0.data(), st)) return rc;
    it.T.assign(B, 300.0);
    it.sd.resize(B);
    for (int r = 0; r < B; ++r) it.sd[r] = (unsigned long long)r;
    return ND_OK;
}

extern "C" {

int nd_autotune(nd_handle *h, int method, double dt_seconds, long long n_steps, void *stream)
{
    if (int rc = check_handle(h)) return rc;
    if (method != ND_METHOD_RK4 && method != ND_METHOD_HEUN) return fail(ND_ERR_ARG, "method must be RK4 or HEUN");
    if (n_steps < 1 || !(dt_seconds > 0)) return fail(ND_ERR_ARG, "n_steps >= 1 and dt > 0 required");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<TuneItem> items(1);
    int rc = tune_item_make(h, method, st, items[0]);
    if (rc == ND_OK) rc = tune_items(items, dt_seconds, n_steps, st);
    cudaFree(items[0].tmp);
    return rc;
}

int nd_autotune_group(nd_handle *const *hs, const int *methods, int n, double dt_seconds, long long n_steps,
                      void *stream)
{
    if (!hs || !methods || n < 1) return fail(ND_ERR_ARG, "no handles to tune");
    if (n_steps < 1 || !(dt_seconds > 0)) return fail(ND_ERR_ARG, "n_steps >= 1 and dt > 0 required");
    for (int k = 0; k < n; ++k) {
        if (int rc = check_handle(hs[k])) return rc;
        if (methods[k] != ND_METHOD_RK4 && methods[k] != ND_METHOD_HEUN)
            return fail(ND_ERR_ARG, "method must be RK4 or HEUN");
        for (int j = 0; j < k; ++j)
            if (hs[j] == hs[k]) return fail(ND_ERR_ARG, "a handle appears twice in the group");
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<TuneItem> items(n);
    int rc = ND_OK;
    for (int k = 0; k < n && rc == ND_OK; ++k) {
        rc = tune_item_make(hs[k], methods[k], st, items[k]);
        if (rc == ND_OK && n > 1 && cudaStreamCreateWithFlags(&items[k].st, cudaStreamNonBlocking) != cudaSuccess)
            rc = fail(ND_ERR_CUDA, "autotune streams");
    }
    if (rc == ND_OK) rc = tune_items(items, dt_seconds, n_steps, st);
    cudaStreamSynchronize(st);
    for (auto &it : items) {
        if (it.st) cudaStreamDestroy(it.st);
        cudaFree(it.tmp);
    }
    return rc;
}

int nd_set_plan(nd_handle *h, int cls, int method, int plan)
{
    if (int rc = check_handle(h)) return rc;
    if (cls < 0 || cls >= (int)h->classes.size()) return fail(ND_ERR_ARG, "no such size class");
    if (method != ND_METHOD_RK4 && method != ND_METHOD_HEUN) return fail(ND_ERR_ARG, "method must be RK4 or HEUN");
    SizeClass &c = h->classes[cls];
    const int prec = h->prec == ND_FP64 ? ND_PREC_FP64 : ND_PREC_FP32;
    if (plan_cluster_nc(plan)) {
        if (!cluster_plan_fits(h, c, prec, method == ND_METHOD_HEUN, plan_cluster_nc(plan)))
            return fail(ND_ERR_ARG, "no such cluster plan for this size class");
    } else if (plan == kPlanGlobal) {
        if (int rc = ensure_alloc(&h->ms, h->elt * h->state_elems)) return rc;
        if (int rc = ensure_alloc(&h->spec, sizeof(double) * 2 * h->spec_words)) return rc;
    } else if (plan >= 0) {
        if (fused_variant_threads(c.P, plan) == 0) return fail(ND_ERR_ARG, "no such fused variant for this size");
        const size_t sm = fused_smem(c.P, prec, c.maxD, c.maxDpad, false, plan);
        if (sm == (size_t)-1 || sm + 1024 > h->max_smem) return fail(ND_ERR_ARG, "variant does not fit in shared memory");
    } else if (plan != -1) {
        return fail(ND_ERR_ARG, "plan must be -1, 0..2, 100, 200 or 201");
    }
    c.plan[method == ND_METHOD_RK4 ? 0 : 1] = plan;
    return ND_OK;
}

int nd_plan_info(const nd_handle *h, int cls, int *P, int *n_replicas, int *plan_rk4, int *plan_heun, int *threads_rk4,
                 int *threads_heun)
{
    if (int rc = check_handle(h)) return rc;
    if (cls < 0 || cls >= (int)h->classes.size()) return fail(ND_ERR_ARG, "no such size class");
    const SizeClass &c = h->classes[cls];
    auto threads = [&](int pl) {
        if (pl == kPlanGlobal) return 0;
        if (plan_cluster_nc(pl)) return cluster_cta_threads(c.P) * plan_cluster_nc(pl);   // threads of the cluster
        if (!c.fused_main) return 0;
        return fused_variant_threads(c.P, pl < 0 ? 0 : pl);
    };
    if (P) *P = c.P;
    if (n_replicas) *n_replicas = (int)c.reps.size();
    if (plan_rk4) *plan_rk4 = c.plan[0];
    if (plan_heun) *plan_heun = c.plan[1];
    if (threads_rk4) *threads_rk4 = threads(c.plan[0]);
    if (threads_heun) *threads_heun = threads(c.plan[1]);
    return ND_OK;
}

// Kernel nodes of a graph, counting those inside child graphs.
static cudaError_t count_kernel_nodes(cudaGraph_t graph, int *count)
{
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(graph, nullptr, &n);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(n);
    if ((e = cudaGraphGetNodes(graph, nodes.data(), &n)) != cudaSuccess) return e;
    for (auto node : nodes) {
        cudaGraphNodeType t;
        if ((e = cudaGraphNodeGetType(node, &t)) != cudaSuccess) return e;
        if (t == cudaGraphNodeTypeKernel) {
            ++*count;
        } else if (t == cudaGraphNodeTypeGraph) {
            cudaGraph_t child = nullptr;
            if ((e = cudaGraphChildGraphNodeGetGraph(node, &child)) != cudaSuccess) return e;
            if ((e = count_kernel_nodes(child, count)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

struct nd_graph {
    nd_handle *h = nullptr;
    Replica *reps = nullptr;          // private parameter blocks (step counter advanced on the device)
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void nd_graph_destroy(nd_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap) cudaStreamDestroy(g->cap);
    cudaFree(g->reps);
    delete g;
}

int nd_graph_create(nd_handle *h, void *m, int method, long long n_steps, double dt_seconds, const double *T_kelvin,
                    const unsigned long long *seed, unsigned long long step0, int stats_sample, nd_graph **out)
{
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(ND_ERR_ARG, "out is null");
    *out = nullptr;
    if (method != ND_METHOD_RK4 && method != ND_METHOD_HEUN) return fail(ND_ERR_ARG, "method must be RK4 or HEUN");
    if (n_steps < 1 || !(dt_seconds > 0)) return fail(ND_ERR_ARG, "n_steps >= 1 and dt > 0 required");
    if (!m || !is_device_ptr(m)) return fail(ND_ERR_ARG, "a graph needs a device state buffer");
    if (method == ND_METHOD_HEUN && (!T_kelvin || !seed)) return fail(ND_ERR_ARG, "T_kelvin and seed are required");
    if ((stats_sample & ND_GRAPH_STATS) && !h->stats) return fail(ND_ERR_ARG, "statistics sample needs nd_stats_reset first");
    if ((stats_sample & ND_GRAPH_SERIES) && !h->series) return fail(ND_ERR_ARG, "series sample needs nd_series_reset first");
    const int B = (int)h->rep_disk.size();
    const int mode = method == ND_METHOD_RK4 ? M_RK4 : M_HEUN;
    nd_graph *g = new nd_graph();
    g->h = h;
    auto bail = [&](int code, const std::string &msg) {
        nd_graph_destroy(g);
        return fail(code, msg);
    };
    cudaError_t e = cudaMalloc(&g->reps, sizeof(Replica) * B);
    if (e != cudaSuccess) return bail(ND_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    fill_reps(h, h->prec == ND_FP64, dt_seconds, method == ND_METHOD_HEUN ? T_kelvin : nullptr,
              method == ND_METHOD_HEUN ? seed : nullptr, step0);
    e = cudaMemcpy(g->reps, h->reps_h, sizeof(Replica) * B, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(ND_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    // one plain run of the launch sequence prepares the cached schedules
    // (allocations are not allowed inside a capture); it works on a scratch
    // copy so the caller's state is untouched
    {
        void *tmp = nullptr;
        if ((e = cudaMalloc(&tmp, h->elt * h->state_elems)) != cudaSuccess)
            return bail(ND_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        cudaMemcpy(tmp, m, h->elt * h->state_elems, cudaMemcpyDeviceToDevice);
        Replica *r2 = nullptr;
        cudaMalloc(&r2, sizeof(Replica) * B);
        cudaMemcpy(r2, g->reps, sizeof(Replica) * B, cudaMemcpyDeviceToDevice);
        int rc = run_mode(h, mode, false, tmp, nullptr, n_steps, 0, r2);
        cudaDeviceSynchronize();
        cudaFree(tmp);
        cudaFree(r2);
        if (rc) { std::string msg = g_err; return bail(rc, msg); }
    }
    if ((e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(ND_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    if ((e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail(ND_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    int rc = run_mode(h, mode, false, m, nullptr, n_steps, g->cap, g->reps);
    if (rc == ND_OK && (stats_sample & ND_GRAPH_STATS)) rc = stats_launches(h, m, n_steps * dt_seconds, g->cap, g->reps);
    if (rc == ND_OK && (stats_sample & ND_GRAPH_SERIES)) rc = series_launches(h, m, g->cap, g->reps);
    if (rc == ND_OK && launch_advance_steps(g->reps, B, n_steps, g->cap) != cudaSuccess) rc = ND_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->cap, &graph);
    g->graph = graph;
    if (rc) { std::string msg = g_err; return bail(rc, "capture: " + msg); }
    if (e != cudaSuccess) return bail(ND_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    if ((e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
        return bail(ND_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    *out = g;
    return ND_OK;
}

int nd_graph_join(nd_graph *const *parts, int n_parts, nd_graph **out)
{
    if (!out) return fail(ND_ERR_ARG, "out is null");
    *out = nullptr;
    if (!parts || n_parts < 1) return fail(ND_ERR_ARG, "no graphs to join");
    for (int k = 0; k < n_parts; ++k)
        if (!parts[k] || !parts[k]->graph) return fail(ND_ERR_ARG, "null graph among the parts");
    nd_graph *g = new nd_graph();
    cudaError_t e = cudaGraphCreate(&g->graph, 0);
    for (int k = 0; k < n_parts && e == cudaSuccess; ++k) {
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, g->graph, nullptr, 0, parts[k]->graph);   // no edges: side by side
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        nd_graph_destroy(g);
        return fail(ND_ERR_CUDA, std::string("graph join: ") + cudaGetErrorString(e));
    }
    *out = g;
    return ND_OK;
}

int nd_graph_launch(nd_graph *g, void *stream)
{
    if (!g || !g->exec) return fail(ND_ERR_ARG, "null graph");
    ND_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return ND_OK;
}

int nd_graph_nodes(const nd_graph *g, int *n_kernel_nodes)
{
    if (!g || !g->graph || !n_kernel_nodes) return fail(ND_ERR_ARG, "null argument");
    int k = 0;
    ND_CUDA(count_kernel_nodes(g->graph, &k));
    *n_kernel_nodes = k;
    return ND_OK;
}

}  // extern "C"
