// nd_noalloc.cu -- nd_step_heun_noalloc: the stochastic Heun stepper for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// framework that owns every device allocation through its own pool, in a
// real-time loop where an allocation's implicit synchronisation is not
// acceptable, or in a plugin that may only touch the buffers its host hands
// it.  Such a caller cannot create a handle (nd_create_disk allocates the
// spectral kernel, masks and scratch), so this entry point takes the disk
// description directly and keeps all of its own working memory in one
// file-scope device array that exists as soon as the library is loaded.
//
// The array holds, for one FP32 disk geometry with P <= 128: the stage
// accumulator of the Heun scheme, the spectral kernel (built in place, and
// rebuilt only when the geometry changes), the disk mask and its list of
// cells, the FFT twiddles, the per-replica parameter blocks and the work list.  Every call on a device
// shares that device's copy and leaves the last call's contents behind;
// nothing in it has to start at zero (the accumulator is written before it is
// read), but calls whose kernels overlap on the GPU -- on different streams, or
// a kernel still running when the next call rewrites the parameters or the
// kernel table -- race on it.
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/nanodisk.h"
#include "nd_common.cuh"
#include "nd_kernels.h"

using namespace nd;

namespace {

constexpr size_t kAccFloats = ND_NOALLOC_MAX_STATE_FLOATS;   // stage accumulator capacity
constexpr int kMaxReplicas = ND_NOALLOC_MAX_REPLICAS;
constexpr int kMaxP = 128, kMaxD = 64, kKH = kMaxP / 2 + 1;
constexpr size_t kGhatEntries = (size_t)kKH * kKH * 8;   // interleaved and component-major copies

constexpr size_t align256(size_t n) { return (n + 255) / 256 * 256; }
// layout of the static array (byte offsets)
constexpr size_t kOffAcc = 0;
constexpr size_t kOffG32 = align256(kOffAcc + sizeof(float) * kAccFloats);
constexpr size_t kOffG64 = align256(kOffG32 + sizeof(float) * kGhatEntries);
constexpr size_t kOffWork = align256(kOffG64 + sizeof(double) * kGhatEntries);
constexpr size_t kWorkDoubles = (size_t)4 * kMaxD * kMaxD + (size_t)4 * kMaxD * kKH + 2 * (size_t)kMaxP;
constexpr size_t kOffMask = align256(kOffWork + sizeof(double) * kWorkDoubles);
constexpr size_t kOffCells = align256(kOffMask + (size_t)kMaxD * kMaxD);
constexpr size_t kOffTw = align256(kOffCells + sizeof(int) * (size_t)kMaxD * kMaxD);
constexpr size_t kOffReps = align256(kOffTw + sizeof(float) * 2 * kMaxP);
constexpr size_t kOffList = align256(kOffReps + sizeof(Replica) * kMaxReplicas);
constexpr size_t kStaticBytes = align256(kOffList + sizeof(int) * kMaxReplicas);

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_nd_noalloc_scratch[kStaticBytes];

namespace {

struct DeviceSlot {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of g_nd_noalloc_scratch on this device
    // geometry whose kernel table, mask and twiddles are currently in the array
    bool have_geom = false;
    int D = 0, P = 0, C = 0;
    double key[6] = {0, 0, 0, 0, 0, 0};
};

constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mu;
Replica g_reps_host[kMaxReplicas];   // host staging of the parameter blocks (no heap use per call)
int g_list_host[kMaxReplicas];

}  // namespace

namespace nd {
void set_last_error(const std::string &msg);   // nd_api.cu: backs nd_last_error()
}

namespace {
int fail(int code, const std::string &m)
{
    nd::set_last_error(m);
    return code;
}
}  // namespace

extern "C" int nd_step_heun_noalloc(const nd_disk_desc *disk, int n_replicas, float *m, long long n_steps,
                                    double dt_seconds, const double *T_kelvin, const unsigned long long *seed,
                                    unsigned long long step0, void *stream)
{
    if (!disk || !m || !T_kelvin || !seed) return fail(ND_ERR_ARG, "nd_step_heun_noalloc: null argument");
    if (n_replicas < 1 || n_replicas > kMaxReplicas)
        return fail(ND_ERR_ARG, "nd_step_heun_noalloc: n_replicas must be 1.." + std::to_string(kMaxReplicas));
    if (n_steps < 0 || !(dt_seconds > 0)) return fail(ND_ERR_ARG, "nd_step_heun_noalloc: bad n_steps or dt");
    const nd_disk_desc &ds = *disk;
    if (!(ds.R > 0 && ds.L > 0 && ds.a > 0 && ds.Ms > 0 && ds.A > 0 && ds.gamma > 0))
        return fail(ND_ERR_ARG, "nd_step_heun_noalloc: R, L, a, Ms, A, gamma must be positive");
    // geometry and units (same conventions as nd_create_disk)
    const int D = (int)floor(2.0 * ds.R / ds.a + 0.5);
    if (D < 1) return fail(ND_ERR_ARG, "nd_step_heun_noalloc: disk smaller than one cell");
    const int Dpad = (D + 3) / 4 * 4;
    int P = 16;
    while (P < 2 * D - 1) P *= 2;
    if (P > kMaxP)
        return fail(ND_ERR_ARG, "nd_step_heun_noalloc: padded grid " + std::to_string(P) + " above the static limit " +
                                    std::to_string(kMaxP) + " (disk diameter above 64 cells)");
    const size_t need = (size_t)n_replicas * 3 * D * Dpad;
    if (need > kAccFloats)
        return fail(ND_ERR_ARG, "nd_step_heun_noalloc: " + std::to_string(need) + " state floats exceed the static limit " +
                                    std::to_string(kAccFloats));
    for (int r = 0; r < n_replicas; ++r)
        if (!(T_kelvin[r] >= 0)) return fail(ND_ERR_ARG, "nd_step_heun_noalloc: temperatures must be >= 0");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(ND_ERR_CUDA, "nd_step_heun_noalloc: no usable current device");
    {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, m) != cudaSuccess || !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(ND_ERR_ARG, "nd_step_heun_noalloc: m must be a device pointer (host buffers would need staging memory)");
        }
        // the kernel runs on the current device: a buffer of another GPU would
        // be reached through peer access, which need not be enabled
        if (at.type == cudaMemoryTypeDevice && at.device != dev)
            return fail(ND_ERR_ARG, "nd_step_heun_noalloc: m lives on device " + std::to_string(at.device) +
                                        ", not on the current device " + std::to_string(dev));
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = fused_smem(P, ND_PREC_FP32, D, Dpad);
    if (smem == (size_t)-1 || smem + 1024 > (size_t)optin)
        return fail(ND_ERR_ARG, "nd_step_heun_noalloc: disk too large for the on-chip kernel (diameter above ~60 cells)");

    std::lock_guard<std::mutex> lock(g_mu);
    cudaStream_t st = (cudaStream_t)stream;
    {
        // the parameter blocks go up from one static host array, so a captured
        // call would replay whatever the last call left there, not its own T,
        // seeds and step0
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            return fail(ND_ERR_CUDA, "nd_step_heun_noalloc: cannot query the stream's capture status");
        }
        if (cs != cudaStreamCaptureStatusNone)
            return fail(ND_ERR_ARG, "nd_step_heun_noalloc: the stream is being captured; this call cannot be captured");
    }
    DeviceSlot &S = g_slots[dev];
    if (!S.ready) {
        // once per device, with the device current: resolve the array's device address
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_nd_noalloc_scratch);
        if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        double re[32], im[32];
        for (int k = 0; k < 32; ++k) { re[k] = cos(2.0 * M_PI * k / 32.0); im[k] = -sin(2.0 * M_PI * k / 32.0); }
        e = upload_twiddle_constants(re, im);
        if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("twiddle constants: ") + cudaGetErrorString(e));
        S.base = static_cast<unsigned char *>(p);
        S.ready = true;
    }
    const double kMu0 = 4.0e-7 * M_PI, kB = 1.380649e-23;
    const double lam = sqrt(2.0 * ds.A / (kMu0 * ds.Ms * ds.Ms));
    const double cfac = ds.a * ds.a / (lam * lam), B0 = 2.0 * ds.A / (ds.a * ds.a * ds.Ms), J = 2.0 * ds.A * ds.L;
    const double ro = ds.a / sqrt(M_PI), q = sqrt(ds.L * ds.L + ro * ro);
    const double Nz = (ds.L + ro - q) / ds.L, Nx = (q - ro) / (2.0 * ds.L);
    float *acc = reinterpret_cast<float *>(S.base + kOffAcc);
    float *g32 = reinterpret_cast<float *>(S.base + kOffG32);
    double *g64 = reinterpret_cast<double *>(S.base + kOffG64);
    double *work = reinterpret_cast<double *>(S.base + kOffWork);
    unsigned char *mask = S.base + kOffMask;
    int *cells = reinterpret_cast<int *>(S.base + kOffCells);
    float *tw = reinterpret_cast<float *>(S.base + kOffTw);
    Replica *reps = reinterpret_cast<Replica *>(S.base + kOffReps);
    int *list = reinterpret_cast<int *>(S.base + kOffList);

    const double key[6] = {(double)D, ds.L / ds.a, Nx, Nz, cfac, ds.R / ds.a};
    bool same = S.have_geom && S.D == D && S.P == P;
    for (int k = 0; k < 6 && same; ++k) same = S.key[k] == key[k];
    if (!same) {
        unsigned char mh[kMaxD * kMaxD];
        int ch[kMaxD * kMaxD];
        int nc = 0;
        const double rr = (ds.R / ds.a) * (ds.R / ds.a);
        for (int j = 0; j < D; ++j)
            for (int i = 0; i < D; ++i) {
                const double x = i - 0.5 * (D - 1), y = j - 0.5 * (D - 1);
                mh[j * D + i] = (x * x + y * y) <= rr;
                if (mh[j * D + i]) ch[nc++] = j * D + i;
            }
        float th[2 * kMaxP];
        for (int k = 0; k < P; ++k) { th[2 * k] = (float)cos(2.0 * M_PI * k / P); th[2 * k + 1] = (float)-sin(2.0 * M_PI * k / P); }
        cudaError_t e = cudaMemcpyAsync(mask, mh, (size_t)D * D, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && nc > 0) e = cudaMemcpyAsync(cells, ch, sizeof(int) * nc, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tw, th, sizeof(float) * 2 * P, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = build_ghat(P, D, ds.L / ds.a, Nx, Nz, cfac, nullptr, g64, g32, work, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host arrays above are on the stack
        if (e != cudaSuccess) { S.have_geom = false; return fail(ND_ERR_CUDA, std::string("geometry set-up: ") + cudaGetErrorString(e)); }
        S.have_geom = true; S.D = D; S.P = P; S.C = nc;
        for (int k = 0; k < 6; ++k) S.key[k] = key[k];
    }
    if (n_steps == 0) return ND_OK;
    const double dtau = ds.gamma * B0 * dt_seconds;
    for (int r = 0; r < n_replicas; ++r) {
        Replica &R = g_reps_host[r];
        memset(&R, 0, sizeof(R));
        R.D = D; R.Dpad = Dpad; R.disk = 0;
        R.state_off = (long long)r * 3 * D * Dpad;
        R.spec_off = 0;
        R.Ghat = g32; R.mask = mask;
        R.cells = cells; R.ncells = S.C;
        for (int k = 0; k < 3; ++k) R.chext[k] = cfac * (ds.hext[k] / ds.Ms);   // rounded as nd_create_disk does
        R.alpha = ds.alpha; R.dtau = dtau;
        R.sigma = sqrt(2.0 * ds.alpha * (kB * T_kelvin[r] / J) * dtau);
        R.flags = R.sigma > 0.0 ? 1 : 0;
        R.seed = seed[r]; R.step0 = step0;
        for (int k = 0; k < 3; ++k) R.fchext[k] = (float)R.chext[k];
        R.falpha = (float)R.alpha; R.fdtau = (float)R.dtau; R.fsigma = (float)R.sigma;
        g_list_host[r] = r;
    }
    cudaError_t e = cudaMemcpyAsync(reps, g_reps_host, sizeof(Replica) * n_replicas, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(list, g_list_host, sizeof(int) * n_replicas, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("parameter upload: ") + cudaGetErrorString(e));
    LaunchArgs a;
    a.mode = M_HEUN;
    a.reps = reps;
    a.work = list;
    a.nwork = n_replicas;
    a.y = m;
    a.acc = acc;
    a.tw = tw;
    a.nsteps = n_steps;
    a.smem = smem;
    a.stream = st;
    // (the host parameter blocks come from pageable memory, so each copy has
    // consumed them by the time cudaMemcpyAsync returns and the next call may
    // overwrite them)
    e = launch_fused(P, ND_PREC_FP32, a);
    if (e != cudaSuccess) return fail(ND_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return ND_OK;
}
