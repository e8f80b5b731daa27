// nd_field_impl.cuh -- field evaluation and time stepping kernels (templates;
// instantiated by nd_fused_f32.cu, nd_fused_f64.cu, nd_glob_f32.cu, nd_glob_f64.cu).
//
// Two drivers share the passes of nd_phases.cuh:
//  * k_fused<P, T, MODE>: one CTA owns one replica for a whole launch.  The
//    half spectrum, the stage magnetisation and the FFT scratch live in shared
//    memory; a launch runs n_steps full time steps (RK4: four field
//    evaluations per step, Heun: two) without touching the spectrum in HBM.
//    Used when the CTA's shared-memory footprint fits (P <= 128 in FP32).
//  * k_g_*: the same passes as separate grid-wide kernels with the spectrum
//    in global memory, for the large padded grids (P = 256..1024) and FP64 at
//    P = 128.
// The LLG right-hand side, the RK4 combine, the stochastic Heun predictor and
// corrector with Philox noise and the |m| = 1 renormalisation are fused into
// the epilogue that consumes the inverse transform.
#pragma once
#include "nd_kernels.h"
#include "nd_phases.cuh"

namespace nd {

// ------------------------------------------------------------- epilogue

template <typename T> __device__ __forceinline__ vec3<T> v3(T x, T y, T z) { return {x, y, z}; }
template <typename T> __device__ __forceinline__ vec3<T> cross3(vec3<T> a, vec3<T> b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T> __device__ __forceinline__ vec3<T> axpy3(T s, vec3<T> a, vec3<T> b)
{
    return {b.x + s * a.x, b.y + s * a.y, b.z + s * a.z};
}
template <typename T> __device__ __forceinline__ vec3<T> normalize3(vec3<T> v)
{
    T r = drsqrt<T>(v.x * v.x + v.y * v.y + v.z * v.z);
    return {v.x * r, v.y * r, v.z * r};
}
// Landau-Lifshitz right-hand side m x b - alpha m x (m x b) (Section III.A).
template <typename T> __device__ __forceinline__ vec3<T> llg_rhs(vec3<T> m, vec3<T> b, T alpha)
{
    vec3<T> p = cross3(m, b), q = cross3(m, p);
    return {p.x - alpha * q.x, p.y - alpha * q.y, p.z - alpha * q.z};
}
// One Heun stage change m x [g - alpha m x g], g = b dtau + sigma w (Section III.C).
template <typename T> __device__ __forceinline__ vec3<T> heun_dm(vec3<T> m, vec3<T> g, T alpha)
{
    vec3<T> p = cross3(m, g);
    return cross3(m, vec3<T>{g.x - alpha * p.x, g.y - alpha * p.y, g.z - alpha * p.z});
}

// Programmatic dependent launch: the global path's kernels are launched so
// that each may start while its predecessor in the stream drains; before it
// reads anything the predecessor wrote (or the parameter blocks) it waits
// here until that grid has completed and its writes are visible.  Without
// the launch attribute this is a no-op.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename T> struct V3Ptr {
    T *p;
    long long s;  // component stride
    __device__ __forceinline__ vec3<T> ld(long long i) const { return {p[i], p[s + i], p[2 * s + i]}; }
    // bypassing L1: for data another CTA may have written during this launch
    __device__ __forceinline__ vec3<T> ldcg(long long i) const
    {
        return {__ldcg(p + i), __ldcg(p + s + i), __ldcg(p + 2 * s + i)};
    }
    __device__ __forceinline__ void st(long long i, vec3<T> v) const { p[i] = v.x; p[s + i] = v.y; p[2 * s + i] = v.z; }
};

// The per-cell update of one stepping stage (Section III.A RK4, Section III.C
// Heun), as a function of the cell's stage input m, its induction b, y_n and
// the stage accumulator a (read by stages > 0) and, for Heun, the normals w:
// returns the next stage's input; acc_new and the flags say what else the
// stage writes (the accumulator, and y_n after the last stage).  Every path
// (on chip, global, fused row pass) calls this one definition, so all of them
// round identically.
template <typename T> struct StageOut {
    vec3<T> nm, acc;
    bool w_acc, w_yn;
};

template <typename T, int MODE>
__device__ __forceinline__ StageOut<T> stage_update(const StepParams<T> &sp, bool noise, int stage, vec3<T> m,
                                                    vec3<T> b, vec3<T> y, vec3<T> a, vec3<T> w)
{
    const T alpha = sp.alpha, dt = sp.dtau;
    StageOut<T> o;
    if (MODE == M_RK4) {
        vec3<T> k = llg_rhs(m, b, alpha);
        if (stage == 0) {
            o.acc = k;
            o.nm = axpy3(T(0.5) * dt, k, m);
            o.w_acc = true; o.w_yn = false;
        } else if (stage < 3) {
            o.acc = axpy3(T(2), k, a);
            o.nm = axpy3(stage == 1 ? T(0.5) * dt : dt, k, y);
            o.w_acc = true; o.w_yn = false;
        } else {
            vec3<T> s = {a.x + k.x, a.y + k.y, a.z + k.z};
            o.nm = normalize3(axpy3(dt / T(6), s, y));
            o.w_acc = false; o.w_yn = true;
        }
    } else {   // M_HEUN
        vec3<T> g = {b.x * dt, b.y * dt, b.z * dt};
        if (noise) { g.x += sp.sigma * w.x; g.y += sp.sigma * w.y; g.z += sp.sigma * w.z; }
        vec3<T> d = heun_dm(m, g, alpha);
        if (stage == 0) {
            o.acc = d;
            o.nm = normalize3(vec3<T>{m.x + d.x, m.y + d.y, m.z + d.z});
            o.w_acc = true; o.w_yn = false;
        } else {
            o.nm = normalize3(vec3<T>{y.x + T(0.5) * (a.x + d.x), y.y + T(0.5) * (a.y + d.y),
                                      y.z + T(0.5) * (a.z + d.z)});
            o.w_acc = false; o.w_yn = true;
        }
    }
    return o;
}

// Per-cell epilogue of one field evaluation.
//   ms  : stage magnetisation (read; overwritten with the next stage's input)
//   yn  : state y_n (user buffer), acc : stage accumulator (scratch)
//   b   : the full dimensionless induction b_i at this cell
// Returns the cell's contribution to the reduced quantity (energy mode).
// For Heun, wbuf (when not null) keeps the predictor's normals for the
// corrector, which then reads them instead of regenerating them.
// ynl, accl: where y_n and the accumulator are read from (the same arrays, or
// copies of them staged in shared memory); writes always go to yn and acc.
template <typename T, int MODE>
__device__ __forceinline__ double epilogue_cell(const Replica &r, int cell, long long si, long long mi, vec3<T> b,
                                                V3Ptr<T> ms, V3Ptr<T> yn, V3Ptr<T> acc, V3Ptr<T> out, int stage,
                                                unsigned long long step, V3Ptr<T> wbuf, V3Ptr<T> ynl, V3Ptr<T> accl)
{
    vec3<T> m = ms.ld(mi);
    if (MODE == M_FIELD) {
        out.st(si, b);
        return 0.0;
    } else if (MODE == M_ENERGY) {
        // E/J = -sum_i m_i . (b'_i / 2 + c h_ext), b' = b - c h_ext  (Eq. Hmm)
        double bx = (double)b.x - r.chext[0], by = (double)b.y - r.chext[1], bz = (double)b.z - r.chext[2];
        return -((double)m.x * (0.5 * bx + r.chext[0]) + (double)m.y * (0.5 * by + r.chext[1]) +
                 (double)m.z * (0.5 * bz + r.chext[2]));
    } else if (MODE == M_RK4 || MODE == M_HEUN) {
        const StepParams<T> sp = step_params<T>(r);
        const vec3<T> zero = {T(0), T(0), T(0)};
        vec3<T> y = zero, a = zero, w = zero;
        if (stage > 0) { a = accl.ld(si); y = ynl.ld(si); }
        const bool noise = MODE == M_HEUN && (r.flags & 1);
        if (noise) {
            if (wbuf.p && stage == 1) {
                w = wbuf.ld(mi);
            } else {
                w = thermal_normals<T>(r.seed, (uint32_t)cell, step);
                if (wbuf.p) wbuf.st(mi, w);
            }
        }
        const StageOut<T> o = stage_update<T, MODE>(sp, noise, stage, m, b, y, a, w);
        if (o.w_acc) acc.st(si, o.acc);
        if (o.w_yn) yn.st(si, o.nm);
        ms.st(mi, o.nm);
        return 0.0;
    }
    return 0.0;
}

template <typename T, int MODE>
__device__ __forceinline__ double epilogue_cell(const Replica &r, int cell, long long si, long long mi, vec3<T> b,
                                                V3Ptr<T> ms, V3Ptr<T> yn, V3Ptr<T> acc, V3Ptr<T> out, int stage,
                                                unsigned long long step, V3Ptr<T> wbuf = V3Ptr<T>{nullptr, 0})
{
    return epilogue_cell<T, MODE>(r, cell, si, mi, b, ms, yn, acc, out, stage, step, wbuf, yn, acc);
}

template <int MODE> struct ModeStages { static constexpr int n = 1; };
template <> struct ModeStages<M_RK4> { static constexpr int n = 4; };
template <> struct ModeStages<M_HEUN> { static constexpr int n = 2; };

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ fused path

template <int P, typename T>
__host__ __device__ __forceinline__ size_t fused_smem_bytes(int D, int Dpad, int nthreads, bool wbuf = false)
{
    using Gm = FFTGeom<P>;
    size_t tw = sizeof(cplx<T>) * Gm::R1 * Gm::G;
    size_t spec = sizeof(cplx<T>) * 3 * (size_t)D * SpecGeom<P>::RS;
    size_t scr = sizeof(cplx<T>) * (size_t)(nthreads / Gm::G) * Gm::SCRATCH;
    size_t ms = sizeof(T) * 3 * (size_t)D * Dpad;
    size_t red = sizeof(double) * 32;
    size_t w = wbuf ? sizeof(T) * 3 * (size_t)D * Dpad : 0;
    return tw + spec + scr + ms + red + w;
}

// A piece of one replica's trajectory run by one CTA (time-sliced schedule).
struct Segment {
    int rep;                 // replica index
    int wait;                // wait until flags[rep] is set before starting
    int signal;              // set flags[rep] when done
    int pad;
    long long step_begin;    // first time step (relative to the call's step0)
    long long nsteps;
};

// Bounded wait of thread 0 on a flag set by another CTA of the same
// (cooperative) launch; returns false after about 2^22 polls.
__device__ __forceinline__ bool wait_flag(int *flag)
{
    for (long long it = 0; it < (1LL << 22); ++it) {
        if (atomicAdd(flag, 0) != 0) {
            __threadfence();
            return true;
        }
        __nanosleep(256);
    }
    return false;
}

template <typename T> __device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_max_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One alignment of the constrained relaxation for a cell (reading of the
// Lagrange-constrained local alignment of Sec. IV): e = b + fictitious field,
// m' = normalise((1-eta) m + eta e/|e|); accumulates the constraint values
// and the exact 2x2 Jacobian of C(m'(lambda)) for cells of the window.
template <typename T> struct RelaxAcc { T C0, C1, J00, J01, J11, res; };

template <typename T>
__device__ __forceinline__ vec3<T> relax_cell(vec3<T> m, vec3<T> b, bool inW, T dx, T dy, T l0, T l1, T eta,
                                              RelaxAcc<T> &acc)
{
    vec3<T> e = b;
    if (inW) e.z += l0 * T(2) * m.z * dx + l1 * T(2) * m.z * dy;
    const T en = dsqrt<T>(e.x * e.x + e.y * e.y + e.z * e.z);
    const vec3<T> u = {e.x / en, e.y / en, e.z / en};
    const vec3<T> tq = cross3(m, u);
    acc.res = max(acc.res, dsqrt<T>(tq.x * tq.x + tq.y * tq.y + tq.z * tq.z));
    const vec3<T> v = {(T(1) - eta) * m.x + eta * u.x, (T(1) - eta) * m.y + eta * u.y, (T(1) - eta) * m.z + eta * u.z};
    const T vn = dsqrt<T>(v.x * v.x + v.y * v.y + v.z * v.z);
    const vec3<T> mp = {v.x / vn, v.y / vn, v.z / vn};
    if (inW) {
        const vec3<T> q = {-u.x * u.z / en, -u.y * u.z / en, (T(1) - u.z * u.z) / en};
        const T mq = mp.x * q.x + mp.y * q.y + mp.z * q.z;
        const T kap = eta * (q.z - mp.z * mq) / vn;
        const T w = T(4) * mp.z * m.z * kap;
        acc.C0 += mp.z * mp.z * dx;
        acc.C1 += mp.z * mp.z * dy;
        acc.J00 += w * dx * dx;
        acc.J01 += w * dx * dy;
        acc.J11 += w * dy * dy;
    }
    return mp;
}

// Thread counts of the fused kernel per padded size: variant 0 is the default
// (and the only one of the field, energy and relaxation modes); the stepping
// modes also have the alternatives the autotuner (nd_autotune) times.
template <int P, int V> struct NTV { static constexpr int v = 0; };
template <> struct NTV<128, 0> { static constexpr int v = 512; };
template <> struct NTV<128, 1> { static constexpr int v = 384; };
template <> struct NTV<64, 0> { static constexpr int v = 384; };
template <> struct NTV<64, 1> { static constexpr int v = 256; };
template <> struct NTV<64, 2> { static constexpr int v = 512; };
template <> struct NTV<32, 0> { static constexpr int v = 256; };
template <> struct NTV<32, 1> { static constexpr int v = 128; };
template <> struct NTV<16, 0> { static constexpr int v = 128; };
template <> struct NTV<16, 1> { static constexpr int v = 64; };
template <int P> struct FusedNT { static constexpr int v = NTV<P, 0>::v; };

// Minimum resident CTAs the compiler must allow: the default thread count
// keeps the whole register file for one CTA; the smaller variants are compiled
// lean (up to 512 threads per SM resident) so that several CTAs can share an SM.
template <int P, int NT> struct FusedMinBlocks {
    static constexpr int v = (NT == NTV<P, 0>::v || NT >= 512) ? 1 : 512 / NT;
};

template <int P, typename T, int MODE, int NT>
__global__ void __launch_bounds__(NT, (FusedMinBlocks<P, NT>::v))
    k_fused(const Replica *__restrict__ reps, const int *__restrict__ work, T *__restrict__ ybase,
            T *__restrict__ accbase, T *__restrict__ outbase, double *__restrict__ red_out,
            const cplx<T> *__restrict__ twP, long long nsteps, unsigned long long step_base,
            RelaxIO *__restrict__ rio, double eta_d, double tol_d, double rc2_d, int max_iter,
            const Segment *__restrict__ segs, const int *__restrict__ seg_off, int *__restrict__ flags,
            unsigned *__restrict__ status, int use_wbuf)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS, GPW = Gm::GROUPS_PER_WARP;
    constexpr int NW = NT / 32, NGRP = NT / G;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Replica r_sh;   // the descriptor stays in shared memory, not in registers
    __shared__ T lam_s[2];
    __shared__ int conv_s, ok_s;
    __shared__ RelaxAcc<T> racc[NW];
    const int tid = threadIdx.x, warp = tid >> 5;
    GroupId<P> gid(tid);
    const int gw = gid.group % GPW;
    constexpr int ncol = P / 2;

    cplx<T> *tw = reinterpret_cast<cplx<T> *>(smem);
    load_twiddles<P>(tw, twP, tid, NT);

    const int s_begin = segs ? seg_off[blockIdx.x] : 0, s_end = segs ? seg_off[blockIdx.x + 1] : 1;
    for (int sg = s_begin; sg < s_end; ++sg) {
        int ridx, wait = 0, signal = 0;
        long long sbeg = 0, nseg = nsteps;
        if (segs) {
            const Segment g = segs[sg];
            ridx = g.rep; wait = g.wait; signal = g.signal; sbeg = g.step_begin; nseg = g.nsteps;
        } else {
            ridx = work[blockIdx.x];
        }
        if (tid == 0) {
            ok_s = wait ? (int)wait_flag(flags + ridx) : 1;
            if (!ok_s) atomicOr(status, ND_DEV_TIMEOUT);
            r_sh = reps[ridx];
        }
        __syncthreads();
        if (!ok_s) break;
        const Replica &r = r_sh;
        const int D = r.D, Dpad = r.Dpad, DD = D * D;
        const long long cs = (long long)D * RS;           // spectrum component stride
        const long long ms_s = (long long)D * Dpad;       // stage-state component stride
        cplx<T> *spec = tw + R1 * G;
        cplx<T> *scratch = spec + 3 * cs;
        T *msm = reinterpret_cast<T *>(scratch + NGRP * Gm::SCRATCH);
        double *red = reinterpret_cast<double *>(msm + 3 * ms_s);
        T *wsm = use_wbuf ? reinterpret_cast<T *>(red + 32) : nullptr;
        cplx<T> *scr = scratch + gid.group * Gm::SCRATCH;

        V3Ptr<T> yn{ybase + r.state_off, ms_s};
        V3Ptr<T> acc{accbase ? accbase + r.state_off : nullptr, ms_s};
        V3Ptr<T> out{outbase ? outbase + r.state_off : nullptr, ms_s};
        V3Ptr<T> ms{msm, ms_s};
        V3Ptr<T> wb{wsm, ms_s};
        for (int cell = tid; cell < DD; cell += NT) {
            const int y = cell / D, x = cell - y * D;
            const long long si = (long long)y * Dpad + x;
            vec3<T> v = r.mask[cell] ? yn.ldcg(si) : vec3<T>{T(0), T(0), T(0)};   // may come from another CTA
            ms.st(si, v);
        }
        __syncthreads();

        // row tasks: one real row each (half-length transforms) at P = 128,
        // else a complex row pair each
        constexpr bool HR = HalfRows<P>::on;
        const int nrow = HR ? 3 * D : row_tasks(D);
        double esum = 0.0;
        T relX = 0, relY = 0;
        if (MODE == M_RELAX) {
            relX = (T)rio[ridx].X[0];
            relY = (T)rio[ridx].X[1];
            if (tid == 0) { lam_s[0] = (T)rio[ridx].lam[0]; lam_s[1] = (T)rio[ridx].lam[1]; conv_s = 0; }
            __syncthreads();
        }
        const long long nst = (MODE == M_FIELD || MODE == M_ENERGY) ? 1 : (MODE == M_RELAX ? (long long)max_iter : nseg);
        long long n = 0;
        T res_last = T(0);
        for (n = 0; n < nst; ++n) {
            for (int stage = 0; stage < ModeStages<MODE>::n; ++stage) {
                for (int qb = warp * GPW; qb < nrow; qb += NW * GPW) {
                    const int q = qb + gw;
                    if constexpr (HR) {
                        const int c = q / D, y = q - c * D;
                        const bool act = q < nrow;
                        const int cc = act ? c : 0, yy = act ? y : 0;
                        row_fwd_half<P, T>(act, msm + cc * ms_s + (long long)yy * Dpad, D,
                                           spec + cc * cs + (long long)yy * RS, gid.t, scr, tw, gid.gmask);
                    } else {
                        row_fwd_task<P, T>(q, q < nrow, D, msm, Dpad, ms_s, spec, cs, gid.t, gid.lane, scr, tw,
                                           gid.gmask);
                    }
                }
                __syncthreads();
                for (int qb = warp * GPW; qb < ncol; qb += NW * GPW) {
                    const int q = qb + gw;
                    col_task<P, T>(q, q < ncol, D, spec, cs, reinterpret_cast<const T *>(r.Ghat), gid.t, gid.lane,
                                   scr, tw, gid.gmask);
                }
                __syncthreads();
                for (int qb = warp * GPW; qb < nrow; qb += NW * GPW) {
                    const int q = qb + gw;
                    if constexpr (HR) {
                        const int c = q / D, y = q - c * D;
                        const bool act = q < nrow;
                        const int cc = act ? c : 0, yy = act ? y : 0;
                        cplx<T> *row = spec + cc * cs + (long long)yy * RS;
                        row_inv_half<P, T>(act, row, D, reinterpret_cast<T *>(row), gid.t, scr, tw, gid.gmask);
                    } else {
                        row_inv_task<P, T>(q, q < nrow, D, spec, cs, gid.t, scr, tw, gid.gmask);
                    }
                }
                __syncthreads();
                const T *hr = reinterpret_cast<const T *>(spec);
                const StepParams<T> sp = step_params<T>(r);
                if (MODE == M_RELAX) {
                    // sweep: trial alignment with the current multipliers, reductions
                    const T eta = (T)eta_d, rc2 = (T)rc2_d, l0 = lam_s[0], l1 = lam_s[1];
                    RelaxAcc<T> a = {T(0), T(0), T(0), T(0), T(0), T(0)};
                    for (int cell = tid; cell < DD; cell += NT) {
                        if (!r.mask[cell]) continue;
                        const int y = cell / D, x = cell - y * D;
                        const long long si = (long long)y * Dpad + x, hi = (long long)y * (2 * RS) + x;
                        vec3<T> b = {hr[hi] + sp.chext[0], hr[2 * cs + hi] + sp.chext[1], hr[4 * cs + hi] + sp.chext[2]};
                        const T dx = (T)x - T(0.5) * (T)(D - 1) - relX, dy = (T)y - T(0.5) * (T)(D - 1) - relY;
                        relax_cell<T>(ms.ld(si), b, dx * dx + dy * dy < rc2, dx, dy, l0, l1, eta, a);
                    }
                    a.C0 = warp_sum_t(a.C0); a.C1 = warp_sum_t(a.C1); a.J00 = warp_sum_t(a.J00);
                    a.J01 = warp_sum_t(a.J01); a.J11 = warp_sum_t(a.J11); a.res = warp_max_t(a.res);
                    if ((tid & 31) == 0) racc[warp] = a;
                    __syncthreads();
                    if (tid == 0) {
                        RelaxAcc<T> s = racc[0];
                        for (int w = 1; w < NW; ++w) {
                            s.C0 += racc[w].C0; s.C1 += racc[w].C1; s.J00 += racc[w].J00; s.J01 += racc[w].J01;
                            s.J11 += racc[w].J11; s.res = max(s.res, racc[w].res);
                        }
                        res_last = s.res;
                        if (s.res < (T)tol_d) {
                            conv_s = 1;
                        } else {
                            const T det = s.J00 * s.J11 - s.J01 * s.J01;
                            if (det != T(0) && isfinite(det)) {
                                lam_s[0] += -(s.J11 * s.C0 - s.J01 * s.C1) / det;
                                lam_s[1] += -(-s.J01 * s.C0 + s.J00 * s.C1) / det;
                            }
                        }
                    }
                    __syncthreads();
                    if (conv_s) break;   // leaves the stage loop; the step loop stops below
                    const T m0 = lam_s[0], m1 = lam_s[1];
                    for (int cell = tid; cell < DD; cell += NT) {
                        if (!r.mask[cell]) continue;
                        const int y = cell / D, x = cell - y * D;
                        const long long si = (long long)y * Dpad + x, hi = (long long)y * (2 * RS) + x;
                        vec3<T> b = {hr[hi] + sp.chext[0], hr[2 * cs + hi] + sp.chext[1], hr[4 * cs + hi] + sp.chext[2]};
                        const T dx = (T)x - T(0.5) * (T)(D - 1) - relX, dy = (T)y - T(0.5) * (T)(D - 1) - relY;
                        RelaxAcc<T> dummy = {T(0), T(0), T(0), T(0), T(0), T(0)};
                        ms.st(si, relax_cell<T>(ms.ld(si), b, dx * dx + dy * dy < rc2, dx, dy, m0, m1, eta, dummy));
                    }
                    __syncthreads();
                    continue;
                }
                const unsigned long long step = step_base + r.step0 + (unsigned long long)(sbeg + n);
                // Stages that read y_n and the accumulator get both copied, with
                // 16-byte loads all in flight at once, into the FFT scratch (idle
                // during the epilogue) instead of two dependent round trips to L2
                // per cell.
                V3Ptr<T> ynl = yn, accl = acc;
                if ((MODE == M_HEUN && stage == 1) || (MODE == M_RK4 && stage > 0)) {
                    const long long words = 3 * ms_s * (long long)sizeof(T) / 16;   // Dpad is a multiple of 4
                    const bool fits = 2 * words * 16 <= (long long)(NGRP * Gm::SCRATCH * sizeof(cplx<T>));
                    const bool aligned = ((reinterpret_cast<uintptr_t>(yn.p) | reinterpret_cast<uintptr_t>(acc.p)) & 15) == 0;
                    if (fits && aligned) {
                        int4 *dst = reinterpret_cast<int4 *>(scratch);
                        const int4 *gy = reinterpret_cast<const int4 *>(yn.p), *ga = reinterpret_cast<const int4 *>(acc.p);
                        for (long long i = tid; i < words; i += NT) {
                            const int4 u = __ldcg(gy + i), v = __ldcg(ga + i);
                            dst[i] = u;
                            dst[words + i] = v;
                        }
                        __syncthreads();
                        ynl = V3Ptr<T>{reinterpret_cast<T *>(scratch), ms_s};
                        accl = V3Ptr<T>{reinterpret_cast<T *>(scratch) + 3 * ms_s, ms_s};
                    }
                }
                // the external field of this step (a scheduled one in the stepping modes)
                const vec3<T> cx = (MODE == M_RK4 || MODE == M_HEUN) ? step_chext<T>(r, sp, step)
                                                                     : vec3<T>{sp.chext[0], sp.chext[1], sp.chext[2]};
                // over the disk's cells only (a compacted list), so that no warp
                // spends an iteration on cells outside the disk
                for (int k = tid; k < r.ncells; k += NT) {
                    const int cell = __ldg(r.cells + k);
                    const int y = cell / D, x = cell - y * D;
                    const long long si = (long long)y * Dpad + x;
                    const long long hi = (long long)y * (2 * RS) + x;
                    vec3<T> b = {hr[hi] + cx.x, hr[2 * cs + hi] + cx.y, hr[4 * cs + hi] + cx.z};
                    if (MODE == M_ENERGY)
                        esum += epilogue_cell<T, MODE>(r, cell, si, si, b, ms, yn, acc, out, stage, step);
                    else
                        epilogue_cell<T, MODE>(r, cell, si, si, b, ms, yn, acc, out, stage, step, wb, ynl, accl);
                }
                __syncthreads();
            }
            if (MODE == M_RELAX && conv_s) break;
        }
        if (MODE == M_RELAX) {
            // the relaxed state back to the caller's buffer
            for (int cell = tid; cell < DD; cell += NT) {
                if (!r.mask[cell]) continue;
                const int y = cell / D, x = cell - y * D;
                const long long si = (long long)y * Dpad + x;
                yn.st(si, ms.ld(si));
            }
            if (tid == 0) {
                rio[ridx].lam[0] = (double)lam_s[0];
                rio[ridx].lam[1] = (double)lam_s[1];
                rio[ridx].resid = (double)res_last;
                rio[ridx].iters = (int)n;
                rio[ridx].status = conv_s ? 0 : 1;
            }
        }
        if (MODE == M_ENERGY) {
            esum = warp_sum(esum);
            if ((tid & 31) == 0) red[warp] = esum;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < NW; ++w) s += red[w];
                red_out[ridx] = s;
            }
        }
        __syncthreads();   // every write of this segment is done before the flag and the next segment
        if (signal && tid == 0) {
            __threadfence();
            atomicExch(flags + ridx, 1);
        }
    }
}

// ----------------------------------------------------------- global path

// Resident CTAs per SM the row passes are compiled for: at P = 1024 (FP32) a
// cap of 80 registers leaves room for three CTAs of 256 threads, which the
// latency-bound row loads need.
template <int P, typename T> struct RowsMinB { static constexpr int v = (P == 1024 && sizeof(T) == 4) ? 3 : 1; };
template <int P, typename T, int NT>
__global__ void __launch_bounds__(NT, RowsMinB<P, T>::v)
    k_g_rows(const Replica *__restrict__ reps, const int *__restrict__ work, const T *__restrict__ msbase,
             cplx<T> *__restrict__ specbase, const cplx<T> *__restrict__ twP, int inverse)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS, NGRP = groups_per_block<P, NT>();
    extern __shared__ __align__(16) unsigned char gsm[];
    cplx<T> *tw = reinterpret_cast<cplx<T> *>(gsm);
    cplx<T> *scratch = tw + R1 * G;
    const int tid = threadIdx.x;
    load_twiddles<P>(tw, twP, tid, NT);   // constant: before the wait
    wait_prior_grid();
    const Replica r = reps[work[blockIdx.y]];
    const int D = r.D;
    __syncthreads();
    GroupId<P> gid(tid);
    const int q = blockIdx.x * NGRP + gid.group;
    const int nrow = row_tasks(D);
    if (blockIdx.x * NGRP >= nrow) return;   // CTA-uniform
    if (!gid.valid) return;                  // lanes past the warp's last group
    const long long cs = (long long)D * RS;
    cplx<T> *spec = specbase + r.spec_off;
    cplx<T> *scr = scratch + gid.group * Gm::SCRATCH;
    if (!inverse) {
        const long long ms_s = (long long)D * r.Dpad;
        row_fwd_task<P, T>(q, q < nrow, D, msbase + r.state_off, r.Dpad, ms_s, spec, cs, gid.t, gid.lane, scr, tw,
                           gid.gmask);
    } else {
        row_inv_task<P, T, true>(q, q < nrow, D, spec, cs, gid.t, scr, tw, gid.gmask);
    }
}

template <int P, typename T, int NT>
__global__ void __launch_bounds__(NT)
    k_g_cols(const Replica *__restrict__ reps, const int *__restrict__ work, cplx<T> *__restrict__ specbase,
             const cplx<T> *__restrict__ twP)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS, NGRP = groups_per_block<P, NT>();
    extern __shared__ __align__(16) unsigned char gsm[];
    cplx<T> *tw = reinterpret_cast<cplx<T> *>(gsm);
    cplx<T> *scratch = tw + R1 * G;
    const int tid = threadIdx.x;
    load_twiddles<P>(tw, twP, tid, NT);   // constant: before the wait
    wait_prior_grid();
    const Replica r = reps[work[blockIdx.y]];
    const int D = r.D;
    __syncthreads();
    GroupId<P> gid(tid);
    if (!gid.valid) return;   // lanes past the warp's last group
    const int q = blockIdx.x * NGRP + gid.group;
    const long long cs = (long long)D * RS;
    col_task<P, T>(q, q < P / 2, D, specbase + r.spec_off, cs, reinterpret_cast<const T *>(r.Ghat), gid.t, gid.lane,
                   scratch + gid.group * Gm::SCRATCH, tw, gid.gmask);
}

// Tiled column pass for the large grids.  A CTA takes a block of four
// adjacent columns kx0..kx0+3 and one FFT group per (column, component): the
// XY kernel the x and y components (eight groups; group 4c + j holds component
// c of column kx0 + j, its partner for the in-plane tensor is group ^ 4), the
// Z kernel the z component (four groups).  The block's [D][4] tiles move
// between the spectrum and the groups' scratch areas as row-contiguous runs
// of four complex words (one 32-byte sector per row: rows start on sectors,
// SpecGeom::RS), so every sector the pass reads or writes is used whole.  The
// packed real columns kx = 0, P/2 are group j = 0 of block 0.  Persistent
// grid over (replica, column block) tasks.
template <int P, typename T, bool XY> struct ColTile {
    static constexpr int G = FFTGeom<P>::G;
    static constexpr int NCOMP = XY ? 2 : 1;
    static constexpr int NG = 4 * NCOMP;
    // whole warps: with ten-lane groups (P = 200, three to a warp) the XY
    // block is three warps with one group slot and each warp's last two
    // lanes idle, the Z block two warps with two idle slots
    static constexpr bool POW2 = FFTGeom<P>::POW2;
    static constexpr int GPW = FFTGeom<P>::GROUPS_PER_WARP;
    static constexpr int NT = POW2 ? NG * G : (NG + GPW - 1) / GPW * 32;
    static constexpr int NCB = P / 2 / 4;
    // resident CTAs per SM the kernel is compiled for: 16 warps at 128
    // registers (FP64 columns take twice the registers)
    static constexpr int MINB = sizeof(T) == 8 ? 1 : 512 / NT;
    // How the packed pair is transformed.  With 32 points per thread (P = 512,
    // 1024) a second inlined transform for it pushes the kernel past its 128
    // registers (96-124 bytes of spills per thread in FP32), so the pair moves
    // through the tile like the other columns and runs the same transform
    // calls; with 16 or 24 points per thread nothing spills, and the pair
    // loads, transforms and stores its two columns itself, which measured 3%
    // faster at P = 256.
    static constexpr bool SHARED_PACKED = FFTGeom<P>::R1 >= 32;
};

template <int P, typename T, bool XY>
__global__ void __launch_bounds__(ColTile<P, T, XY>::NT, ColTile<P, T, XY>::MINB)
    k_g_cols_tile(const Replica *__restrict__ reps, const int *__restrict__ work, int nwork,
                  cplx<T> *__restrict__ specbase, const cplx<T> *__restrict__ twP)
{
    using Gm = FFTGeom<P>;
    using CT = ColTile<P, T, XY>;
    constexpr int G = Gm::G, R1 = Gm::R1, KH = SpecGeom<P>::KH, RS = SpecGeom<P>::RS, NT = CT::NT, SCR = Gm::SCRATCH;
    constexpr bool SP = CT::SHARED_PACKED;
    static_assert(RS % 4 == 0, "rows start on 32-byte sectors");
    extern __shared__ __align__(16) unsigned char gsm[];
    cplx<T> *tw = reinterpret_cast<cplx<T> *>(gsm);
    cplx<T> *scratch = tw + R1 * G;
    const int tid = threadIdx.x;
    load_twiddles<P>(tw, twP, tid, NT);   // constant: before the wait
    wait_prior_grid();
    GroupId<P> gid(tid);
    const int g = gid.group, j = g & 3, c = XY ? (g >> 2) : 2, t = gid.t;
    // a group of the block (idle slots and lanes take part in the tile moves
    // and the barriers only)
    const bool gv = CT::POW2 || (gid.valid && g < CT::NG);
    cplx<T> *scr = scratch + g * SCR;
    const cplx<T> *other = scratch + (g ^ 4) * SCR;   // XY only
    for (int task = blockIdx.x; task < nwork * CT::NCB; task += gridDim.x) {
        const int wi = task / CT::NCB, cb = task - wi * CT::NCB, kx0 = 4 * cb;
        const Replica &r = reps[work[wi]];
        const int D = r.D;
        const long long cs = (long long)D * RS;
        cplx<T> *spec = specbase + r.spec_off;
        const T *Ghat = reinterpret_cast<const T *>(r.Ghat);
        const bool packed = (cb == 0 && j == 0);
        const int kx = packed ? 1 : kx0 + j;   // (the packed group reads no kx column of the table)
        __syncthreads();   // twiddles filled / the previous task's tiles stored
        // tile load: thread -> column jj = tid & 3 of the block, rows tid/4 + k NT/4
        // (column 0 of block 0: the packed pair c_0 + i c_{P/2}, when it moves
        // through the tile)
        const int cbase = XY ? 0 : 2, jj = tid & 3;
        const bool ppair = cb == 0 && jj == 0;
        if (SP || !ppair) {
#pragma unroll
            for (int ci = 0; ci < CT::NCOMP; ++ci) {
                const cplx<T> *src = spec + (cbase + ci) * cs + kx0 + jj;
                cplx<T> *dst = scratch + (4 * ci + jj) * SCR;
                if (SP && ppair) {
                    for (int y = tid >> 2; y < D; y += NT / 4)
                        dst[y] = {src[(long long)y * RS].x, src[(long long)y * RS + P / 2].x};
                } else {
                    for (int y = tid >> 2; y < D; y += NT / 4) dst[y] = src[(long long)y * RS];
                }
            }
        }
        __syncthreads();
        cplx<T> v[R1];
        if (!gv) {
        } else if (!SP && packed) {
            packed_col_fwd<P, T>(v, c, true, D, spec + c * cs, Ghat, t, gid.lane, scr, tw, gid.gmask);
        } else {
#pragma unroll
            for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
#pragma unroll
            for (int o = 0; o < R1 / 2; ++o) {   // rows >= D (and so >= P/2) are zero padding
                const int y = t + G * o;
                if (y < D) v[o] = scr[y];
            }
            __syncwarp(gid.gmask);
            fft_group<P, -1, FFT_HALF_IN>(v, t, scr, tw, gid.gmask);
            if (XY) {
#pragma unroll
                for (int o = 0; o < R1; ++o) scr[o * G + t] = v[o];
            }
        }
        if (XY) __syncthreads();
        if (!gv) {
        } else if (packed) {
            // (the packed pair's partner is packed too and reads no spectrum of it)
            if (SP) packed_col_scale<P, T>(v, c, Ghat, t, scr, gid.gmask);
        } else {
            // the component-major copy of the table: each group reads only the
            // entries it uses (4 or 8 bytes per point instead of 16)
            constexpr int KK = KH * KH;
            const T *Gs = Ghat + 4 * KK + kx * KH;
            if (XY) {
                const T *gd = Gs + c * KK, *go = Gs + 2 * KK;   // diagonal entry (xx or yy), xy
#pragma unroll
                for (int o = 0; o < R1; ++o) {
                    const int ky = t + G * o;
                    const bool up = ky <= P / 2;
                    const int kyr = up ? ky : P - ky;
                    const T gdiag = __ldg(gd + kyr), gxy0 = __ldg(go + kyr);
                    const T gxy = up ? gxy0 : -gxy0;   // G_xy is odd in ky
                    const cplx<T> w = other[o * G + t];
                    v[o] = c == 0 ? tensor_row(gdiag, v[o], gxy, w) : tensor_row(gxy, w, gdiag, v[o]);
                }
            } else {
                const T *gz = Gs + 3 * KK;
#pragma unroll
                for (int o = 0; o < R1; ++o) {
                    const int ky = t + G * o;
                    const int kyr = ky <= P / 2 ? ky : P - ky;
                    v[o] = cscale(v[o], __ldg(gz + kyr));
                }
            }
        }
        if (XY) __syncthreads();   // the partner's spectrum is read before the scratch is reused
        if (gv) {
            fft_group<P, +1, FFT_HALF_OUT>(v, t, scr, tw, gid.gmask);
            __syncwarp(gid.gmask);
            if (!SP && packed) {
                packed_col_store<P, T>(v, true, D, spec + c * cs, t);
            } else {
#pragma unroll
                for (int o = 0; o < R1 / 2; ++o) {
                    const int y = t + G * o;
                    if (y < D) scr[y] = v[o];
                }
            }
        }
        __syncthreads();
        if (SP || !ppair) {
#pragma unroll
            for (int ci = 0; ci < CT::NCOMP; ++ci) {
                cplx<T> *dst = spec + (cbase + ci) * cs + kx0 + jj;
                const cplx<T> *src = scratch + (4 * ci + jj) * SCR;
                if (SP && ppair) {
                    for (int y = tid >> 2; y < D; y += NT / 4) {
                        const cplx<T> u = src[y];
                        dst[(long long)y * RS] = {u.x, T(0)};
                        dst[(long long)y * RS + P / 2] = {u.y, T(0)};
                    }
                } else {
                    for (int y = tid >> 2; y < D; y += NT / 4) dst[(long long)y * RS] = src[y];
                }
            }
        }
    }
}

// Elementwise epilogue of the global path.  grid = (cell blocks, replicas).
template <int P, typename T, int MODE>
__global__ void __launch_bounds__(256)
    k_g_epi(const Replica *__restrict__ reps, const int *__restrict__ work, T *__restrict__ msbase,
            T *__restrict__ ybase, T *__restrict__ accbase, T *__restrict__ outbase,
            const cplx<T> *__restrict__ specbase, double *__restrict__ red_out, int stage,
            unsigned long long step)
{
    constexpr int RS = SpecGeom<P>::RS;
    const int ridx = work[blockIdx.y];
    const Replica r = reps[ridx];
    const int D = r.D, DD = D * D;
    const long long ms_s = (long long)D * r.Dpad, cs = (long long)D * RS;
    const int cell = blockIdx.x * 256 + threadIdx.x;
    double e = 0.0;
    if (cell < DD && r.mask[cell]) {
        const int y = cell / D, x = cell - y * D;
        const long long si = (long long)y * r.Dpad + x;
        const T *hr = reinterpret_cast<const T *>(specbase + r.spec_off);
        const long long hi = (long long)y * (2 * RS) + x;
        const StepParams<T> sp = step_params<T>(r);
        const vec3<T> cx = (MODE == M_RK4 || MODE == M_HEUN) ? step_chext<T>(r, sp, step + r.step0)
                                                             : vec3<T>{sp.chext[0], sp.chext[1], sp.chext[2]};
        vec3<T> b = {hr[hi] + cx.x, hr[2 * cs + hi] + cx.y, hr[4 * cs + hi] + cx.z};
        V3Ptr<T> ms{msbase + r.state_off, ms_s}, yn{ybase + r.state_off, ms_s};
        V3Ptr<T> acc{accbase ? accbase + r.state_off : nullptr, ms_s}, out{outbase ? outbase + r.state_off : nullptr, ms_s};
        e = epilogue_cell<T, MODE>(r, cell, si, si, b, ms, yn, acc, out, stage, step + r.step0);
    }
    if (MODE == M_ENERGY) {
        __shared__ double red[8];
        e = warp_sum(e);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += red[w];
            atomicAdd(red_out + ridx, s);
        }
    }
}

// Four consecutive elements of a row (16-byte aligned): one 16-byte access in
// FP32, two in FP64.
template <typename T> struct Quad { T v[4]; };
template <typename T> __device__ __forceinline__ Quad<T> ld_quad(const T *p);
template <> __device__ __forceinline__ Quad<float> ld_quad<float>(const float *p)
{
    const float4 a = __ldcg(reinterpret_cast<const float4 *>(p));
    return {{a.x, a.y, a.z, a.w}};
}
template <> __device__ __forceinline__ Quad<double> ld_quad<double>(const double *p)
{
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p)), b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return {{a.x, a.y, b.x, b.y}};
}
template <typename T> __device__ __forceinline__ void st_quad(T *p, const Quad<T> &q);
template <> __device__ __forceinline__ void st_quad<float>(float *p, const Quad<float> &q)
{
    *reinterpret_cast<float4 *>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
template <> __device__ __forceinline__ void st_quad<double>(double *p, const Quad<double> &q)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(q.v[0], q.v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(q.v[2], q.v[3]);
}

// Epilogue of the global path for the stepping modes with quad access: each
// thread takes four consecutive cells of a row, loads the field rows (the
// spectrum buffer viewed as real rows) and the state rows it needs with
// 16-byte accesses, applies stage_update to the cells inside the disk and
// stores whole quads back (cells outside the disk and padding columns are
// written back unchanged).  grid = (quad blocks, replicas).  Requires 16-byte
// aligned state buffers (rows and replica blocks are multiples of 4
// elements; the spectrum rows start on 32-byte sectors).
template <int P, typename T, int MODE>
__global__ void __launch_bounds__(256)
    k_g_epi_quad(const Replica *__restrict__ reps, const int *__restrict__ work, T *__restrict__ msbase,
                 T *__restrict__ ybase, T *__restrict__ accbase, const cplx<T> *__restrict__ specbase, int stage,
                 unsigned long long step)
{
    constexpr int RS = SpecGeom<P>::RS;
    static_assert(RS % 2 == 0, "field rows start on 16-byte boundaries");
    wait_prior_grid();
    const Replica &r = reps[work[blockIdx.y]];
    const int D = r.D, Dpad = r.Dpad, qpr = Dpad / 4;
    const int qd = blockIdx.x * 256 + threadIdx.x;
    if (qd >= D * qpr) return;
    const int y = qd / qpr, x0 = 4 * (qd - y * qpr);
    const long long ms_s = (long long)D * Dpad, cs2 = 2LL * D * RS;   // component strides (state, field rows)
    const long long si = (long long)y * Dpad + x0;
    const T *hr = reinterpret_cast<const T *>(specbase + r.spec_off) + (long long)y * (2 * RS) + x0;
    T *msr = msbase + r.state_off + si, *ynr = ybase + r.state_off + si, *acr = accbase + r.state_off + si;
    unsigned in = 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (x0 + u < D && r.mask[y * D + x0 + u]) in |= 1u << u;
    if (!in) return;
    Quad<T> m[3], b[3], yv[3], av[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        m[c] = ld_quad<T>(msr + c * ms_s);
        b[c] = ld_quad<T>(hr + c * cs2);
        if (stage > 0) {
            yv[c] = ld_quad<T>(ynr + c * ms_s);
            av[c] = ld_quad<T>(acr + c * ms_s);
        } else {
            yv[c] = av[c] = Quad<T>{{T(0), T(0), T(0), T(0)}};
        }
    }
    const StepParams<T> sp = step_params<T>(r);
    const bool noise = MODE == M_HEUN && (r.flags & 1);
    const unsigned long long nstep = step + r.step0;
    const vec3<T> cx = step_chext<T>(r, sp, nstep);
    Quad<T> nm[3] = {m[0], m[1], m[2]}, na[3] = {av[0], av[1], av[2]}, ny[3] = {yv[0], yv[1], yv[2]};
    bool w_acc = false, w_yn = false;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (!((in >> u) & 1u)) continue;
        const vec3<T> mu = {m[0].v[u], m[1].v[u], m[2].v[u]};
        const vec3<T> bu = {b[0].v[u] + cx.x, b[1].v[u] + cx.y, b[2].v[u] + cx.z};
        const vec3<T> yu = {yv[0].v[u], yv[1].v[u], yv[2].v[u]}, au = {av[0].v[u], av[1].v[u], av[2].v[u]};
        const vec3<T> w = noise ? thermal_normals<T>(r.seed, (uint32_t)(y * D + x0 + u), nstep)
                                : vec3<T>{T(0), T(0), T(0)};
        const StageOut<T> o = stage_update<T, MODE>(sp, noise, stage, mu, bu, yu, au, w);
        nm[0].v[u] = o.nm.x; nm[1].v[u] = o.nm.y; nm[2].v[u] = o.nm.z;
        if (o.w_acc) { na[0].v[u] = o.acc.x; na[1].v[u] = o.acc.y; na[2].v[u] = o.acc.z; w_acc = true; }
        if (o.w_yn) { ny[0].v[u] = o.nm.x; ny[1].v[u] = o.nm.y; ny[2].v[u] = o.nm.z; w_yn = true; }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        st_quad<T>(msr + c * ms_s, nm[c]);
        if (w_acc) {
            if (stage == 0) {   // the accumulator was not loaded: outside cells keep their (unused) values
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if ((in >> u) & 1u) acr[c * ms_s + u] = na[c].v[u];
            } else {
                st_quad<T>(acr + c * ms_s, na[c]);
            }
        }
        if (w_yn) st_quad<T>(ynr + c * ms_s, ny[c]);
    }
}

// Copy y_n into the stage buffer (masked), for the global path.
template <typename T>
__global__ void k_g_load_stage(const Replica *__restrict__ reps, const int *__restrict__ work, const T *__restrict__ ybase,
                               T *__restrict__ msbase)
{
    wait_prior_grid();
    const Replica r = reps[work[blockIdx.y]];
    const int D = r.D, DD = D * D;
    const long long ms_s = (long long)D * r.Dpad;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < DD; cell += gridDim.x * blockDim.x) {
        const int y = cell / D, x = cell - y * D;
        const long long si = r.state_off + (long long)y * r.Dpad + x;
        const bool in = r.mask[cell];
        for (int c = 0; c < 3; ++c) msbase[si + c * ms_s] = in ? ybase[si + c * ms_s] : T(0);
    }
}

// Constrained relaxation on the global path (Sec. IV; same sweep as the fused
// kernel's relaxation mode): per iteration the field passes, then
//   k_g_relax_reduce  per-block partial sums of the constraint values C_k, the
//                     Jacobian J and the residual max |m x e|/|e| of the trial
//                     alignment with the current multipliers,
//   k_g_relax_newton  per replica: fixed-order total, convergence test, one
//                     Newton step on the multipliers,
//   k_g_relax_update  the damped alignment with the new multipliers.
// Replicas that have converged (status 0) are left untouched.
template <int P, typename T>
__global__ void __launch_bounds__(256)
    k_g_relax_reduce(const Replica *__restrict__ reps, const int *__restrict__ work, const T *__restrict__ msbase,
                     const cplx<T> *__restrict__ specbase, const RelaxIO *__restrict__ rio, double rc2_d,
                     double eta_d, double *__restrict__ part)
{
    constexpr int RS = SpecGeom<P>::RS;
    __shared__ RelaxAcc<T> racc[8];
    const int ridx = work[blockIdx.y], tid = threadIdx.x;
    if (rio[ridx].status == 0) return;   // CTA-uniform
    const Replica &r = reps[ridx];
    const int D = r.D, DD = D * D;
    const long long ms_s = (long long)D * r.Dpad, cs = (long long)D * RS;
    const T *hr = reinterpret_cast<const T *>(specbase + r.spec_off);
    const V3Ptr<T> ms{const_cast<T *>(msbase) + r.state_off, ms_s};
    const T relX = (T)rio[ridx].X[0], relY = (T)rio[ridx].X[1], l0 = (T)rio[ridx].lam[0], l1 = (T)rio[ridx].lam[1];
    const T eta = (T)eta_d, rc2 = (T)rc2_d;
    const StepParams<T> sp = step_params<T>(r);
    RelaxAcc<T> a = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int cell = blockIdx.x * 256 + tid; cell < DD; cell += kRelaxBlocks * 256) {
        if (!r.mask[cell]) continue;
        const int y = cell / D, x = cell - y * D;
        const long long si = (long long)y * r.Dpad + x, hi = (long long)y * (2 * RS) + x;
        const vec3<T> b = {hr[hi] + sp.chext[0], hr[2 * cs + hi] + sp.chext[1], hr[4 * cs + hi] + sp.chext[2]};
        const T dx = (T)x - T(0.5) * (T)(D - 1) - relX, dy = (T)y - T(0.5) * (T)(D - 1) - relY;
        relax_cell<T>(ms.ld(si), b, dx * dx + dy * dy < rc2, dx, dy, l0, l1, eta, a);
    }
    a.C0 = warp_sum_t(a.C0); a.C1 = warp_sum_t(a.C1); a.J00 = warp_sum_t(a.J00);
    a.J01 = warp_sum_t(a.J01); a.J11 = warp_sum_t(a.J11); a.res = warp_max_t(a.res);
    if ((tid & 31) == 0) racc[tid >> 5] = a;
    __syncthreads();
    if (tid == 0) {
        RelaxAcc<T> t = racc[0];
        for (int w = 1; w < 8; ++w) {
            t.C0 += racc[w].C0; t.C1 += racc[w].C1; t.J00 += racc[w].J00; t.J01 += racc[w].J01;
            t.J11 += racc[w].J11; t.res = max(t.res, racc[w].res);
        }
        double *o = part + ((size_t)ridx * kRelaxBlocks + blockIdx.x) * 6;
        o[0] = t.C0; o[1] = t.C1; o[2] = t.J00; o[3] = t.J01; o[4] = t.J11; o[5] = t.res;
    }
}

static __global__ void k_g_relax_newton(const int *__restrict__ work, int nwork, RelaxIO *__restrict__ rio,
                                 const double *__restrict__ part, double tol, int iter)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwork) return;
    const int ridx = work[w];
    RelaxIO &R = rio[ridx];
    if (R.status == 0) return;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < kRelaxBlocks; ++b) {
        const double *o = part + ((size_t)ridx * kRelaxBlocks + b) * 6;
        for (int k = 0; k < 5; ++k) s[k] += o[k];
        s[5] = fmax(s[5], o[5]);
    }
    R.resid = s[5];
    if (s[5] < tol) {
        R.status = 0;   // converged: iters keeps the number of sweeps applied
        return;
    }
    const double det = s[2] * s[4] - s[3] * s[3];
    if (det != 0.0 && isfinite(det)) {
        R.lam[0] += -(s[4] * s[0] - s[3] * s[1]) / det;
        R.lam[1] += -(-s[3] * s[0] + s[2] * s[1]) / det;
    }
    R.iters = iter + 1;
}

template <int P, typename T>
__global__ void __launch_bounds__(256)
    k_g_relax_update(const Replica *__restrict__ reps, const int *__restrict__ work, T *__restrict__ msbase,
                     const cplx<T> *__restrict__ specbase, const RelaxIO *__restrict__ rio, double rc2_d, double eta_d)
{
    constexpr int RS = SpecGeom<P>::RS;
    const int ridx = work[blockIdx.y];
    if (rio[ridx].status == 0) return;
    const Replica &r = reps[ridx];
    const int D = r.D, DD = D * D;
    const int cell = blockIdx.x * 256 + threadIdx.x;
    if (cell >= DD || !r.mask[cell]) return;
    const long long ms_s = (long long)D * r.Dpad, cs = (long long)D * RS;
    const T *hr = reinterpret_cast<const T *>(specbase + r.spec_off);
    V3Ptr<T> ms{msbase + r.state_off, ms_s};
    const T relX = (T)rio[ridx].X[0], relY = (T)rio[ridx].X[1], m0 = (T)rio[ridx].lam[0], m1 = (T)rio[ridx].lam[1];
    const StepParams<T> sp = step_params<T>(r);
    const int y = cell / D, x = cell - y * D;
    const long long si = (long long)y * r.Dpad + x, hi = (long long)y * (2 * RS) + x;
    const vec3<T> b = {hr[hi] + sp.chext[0], hr[2 * cs + hi] + sp.chext[1], hr[4 * cs + hi] + sp.chext[2]};
    const T dx = (T)x - T(0.5) * (T)(D - 1) - relX, dy = (T)y - T(0.5) * (T)(D - 1) - relY;
    RelaxAcc<T> dummy = {T(0), T(0), T(0), T(0), T(0), T(0)};
    ms.st(si, relax_cell<T>(ms.ld(si), b, dx * dx + dy * dy < (T)rc2_d, dx, dy, m0, m1, (T)eta_d, dummy));
}

// The same sweep driven by an externally computed energy gradient: the field
// is b_i = gscale[r] * grad_i with gscale = -1/J (grad = dE/dm in joules, in
// the state layout), read in place of the spectrum rows.  Used by
// nd_relax_sweep_grad.
template <typename T>
__global__ void __launch_bounds__(256)
    k_relax_grad_reduce(const Replica *__restrict__ reps, const int *__restrict__ work, const T *__restrict__ mbase,
                        const T *__restrict__ gbase, const double *__restrict__ gscale,
                        const RelaxIO *__restrict__ rio, double rc2_d, double eta_d, double *__restrict__ part)
{
    __shared__ RelaxAcc<T> racc[8];
    const int ridx = work[blockIdx.y], tid = threadIdx.x;
    if (rio[ridx].status == 0) return;   // CTA-uniform
    const Replica &r = reps[ridx];
    const int D = r.D, DD = D * D;
    const long long ms_s = (long long)D * r.Dpad;
    const V3Ptr<T> ms{const_cast<T *>(mbase) + r.state_off, ms_s}, gr{const_cast<T *>(gbase) + r.state_off, ms_s};
    const T relX = (T)rio[ridx].X[0], relY = (T)rio[ridx].X[1], l0 = (T)rio[ridx].lam[0], l1 = (T)rio[ridx].lam[1];
    const T eta = (T)eta_d, rc2 = (T)rc2_d, sc = (T)gscale[ridx];
    RelaxAcc<T> a = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int cell = blockIdx.x * 256 + tid; cell < DD; cell += kRelaxBlocks * 256) {
        if (!r.mask[cell]) continue;
        const int y = cell / D, x = cell - y * D;
        const long long si = (long long)y * r.Dpad + x;
        const vec3<T> g = gr.ld(si), b = {sc * g.x, sc * g.y, sc * g.z};
        const T dx = (T)x - T(0.5) * (T)(D - 1) - relX, dy = (T)y - T(0.5) * (T)(D - 1) - relY;
        relax_cell<T>(ms.ld(si), b, dx * dx + dy * dy < rc2, dx, dy, l0, l1, eta, a);
    }
    a.C0 = warp_sum_t(a.C0); a.C1 = warp_sum_t(a.C1); a.J00 = warp_sum_t(a.J00);
    a.J01 = warp_sum_t(a.J01); a.J11 = warp_sum_t(a.J11); a.res = warp_max_t(a.res);
    if ((tid & 31) == 0) racc[tid >> 5] = a;
    __syncthreads();
    if (tid == 0) {
        RelaxAcc<T> t = racc[0];
        for (int w = 1; w < 8; ++w) {
            t.C0 += racc[w].C0; t.C1 += racc[w].C1; t.J00 += racc[w].J00; t.J01 += racc[w].J01;
            t.J11 += racc[w].J11; t.res = max(t.res, racc[w].res);
        }
        double *o = part + ((size_t)ridx * kRelaxBlocks + blockIdx.x) * 6;
        o[0] = t.C0; o[1] = t.C1; o[2] = t.J00; o[3] = t.J01; o[4] = t.J11; o[5] = t.res;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_relax_grad_update(const Replica *__restrict__ reps, const int *__restrict__ work, T *__restrict__ mbase,
                        const T *__restrict__ gbase, const double *__restrict__ gscale,
                        const RelaxIO *__restrict__ rio, double rc2_d, double eta_d)
{
    const int ridx = work[blockIdx.y];
    if (rio[ridx].status == 0) return;
    const Replica &r = reps[ridx];
    const int D = r.D, DD = D * D;
    const int cell = blockIdx.x * 256 + threadIdx.x;
    if (cell >= DD || !r.mask[cell]) return;
    const long long ms_s = (long long)D * r.Dpad;
    V3Ptr<T> ms{mbase + r.state_off, ms_s};
    const V3Ptr<T> gr{const_cast<T *>(gbase) + r.state_off, ms_s};
    const T relX = (T)rio[ridx].X[0], relY = (T)rio[ridx].X[1], m0 = (T)rio[ridx].lam[0], m1 = (T)rio[ridx].lam[1];
    const T sc = (T)gscale[ridx];
    const int y = cell / D, x = cell - y * D;
    const long long si = (long long)y * r.Dpad + x;
    const vec3<T> g = gr.ld(si), b = {sc * g.x, sc * g.y, sc * g.z};
    const T dx = (T)x - T(0.5) * (T)(D - 1) - relX, dy = (T)y - T(0.5) * (T)(D - 1) - relY;
    RelaxAcc<T> dummy = {T(0), T(0), T(0), T(0), T(0), T(0)};
    ms.st(si, relax_cell<T>(ms.ld(si), b, dx * dx + dy * dy < (T)rc2_d, dx, dy, m0, m1, (T)eta_d, dummy));
}

// One gradient-driven sweep over the replicas of one size class.
template <typename T>
static cudaError_t launch_relax_grad_t(const LaunchArgs &a, int maxD, const void *grad, const double *gscale)
{
    const dim3 gp(kRelaxBlocks, a.nwork), gu((maxD * maxD + 255) / 256, a.nwork);
    k_relax_grad_reduce<T><<<gp, 256, 0, a.stream>>>(a.reps, a.work, (const T *)a.y, (const T *)grad, gscale, a.rio,
                                                     a.rc2, a.eta, a.part);
    k_g_relax_newton<<<(a.nwork + 127) / 128, 128, 0, a.stream>>>(a.work, a.nwork, a.rio, a.part, a.tol, 0);
    k_relax_grad_update<T><<<gu, 256, 0, a.stream>>>(a.reps, a.work, (T *)a.y, (const T *)grad, gscale, a.rio, a.rc2,
                                                     a.eta);
    return cudaGetLastError();
}

// The stage buffer back to the caller's state (cells inside the disk).
template <typename T>
__global__ void k_g_store_stage(const Replica *__restrict__ reps, const int *__restrict__ work, const T *__restrict__ msbase,
                                T *__restrict__ ybase)
{
    const Replica &r = reps[work[blockIdx.y]];
    const int D = r.D, DD = D * D;
    const long long ms_s = (long long)D * r.Dpad;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < DD; cell += gridDim.x * blockDim.x) {
        if (!r.mask[cell]) continue;
        const int y = cell / D, x = cell - y * D;
        const long long si = r.state_off + (long long)y * r.Dpad + x;
        for (int c = 0; c < 3; ++c) ybase[si + c * ms_s] = msbase[si + c * ms_s];
    }
}

// --------------------------------------------------------- launch helpers


inline int fused_nt(int P, int variant)
{
    switch (P) {
    case 16: return variant == 0 ? NTV<16, 0>::v : variant == 1 ? NTV<16, 1>::v : 0;
    case 32: return variant == 0 ? NTV<32, 0>::v : variant == 1 ? NTV<32, 1>::v : 0;
    case 64: return variant == 0 ? NTV<64, 0>::v : variant == 1 ? NTV<64, 1>::v : variant == 2 ? NTV<64, 2>::v : 0;
    case 128: return variant == 0 ? NTV<128, 0>::v : variant == 1 ? NTV<128, 1>::v : 0;
    default: return 0;
    }
}
template <int P> struct GlobNT { static constexpr int v = 256; };
// The tiled column pass runs above P = 128 (rows of the global spectrum start
// on 32-byte sectors there).
template <int P> struct GlobTiled { static constexpr bool v = P > 128; };

template <int P, typename T, int NT>
constexpr size_t glob_smem_bytes()
{
    return sizeof(cplx<T>) *
           ((size_t)FFTGeom<P>::R1 * FFTGeom<P>::G + (size_t)groups_per_block<P, NT>() * FFTGeom<P>::SCRATCH);
}


template <int P, typename T, int MODE, int NT>
static cudaError_t launch_fused_t(const LaunchArgs &a)
{
    auto kern = k_fused<P, T, MODE, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem);
    if (e != cudaSuccess) return e;
    const Segment *segs = reinterpret_cast<const Segment *>(a.segs);
    if (!segs) {
        kern<<<a.nwork, NT, a.smem, a.stream>>>(a.reps, a.work, (T *)a.y, (T *)a.acc, (T *)a.out, a.red,
                                                (const cplx<T> *)a.tw, a.nsteps, a.step_base, a.rio, a.eta, a.tol,
                                                a.rc2, a.max_iter, nullptr, nullptr, nullptr, a.status, a.use_wbuf);
        return cudaGetLastError();
    }
    // time-sliced schedule: the CTAs wait on one another, so they must all be
    // resident at once -- a cooperative launch guarantees it or fails
    const Replica *reps = a.reps;
    const int *work = a.work;
    T *y = (T *)a.y, *acc = (T *)a.acc, *out = (T *)a.out;
    double *red = a.red;
    const cplx<T> *tw = (const cplx<T> *)a.tw;
    long long nsteps = a.nsteps;
    unsigned long long step_base = a.step_base;
    RelaxIO *rio = a.rio;
    double eta = a.eta, tol = a.tol, rc2 = a.rc2;
    int max_iter = a.max_iter, use_wbuf = a.use_wbuf;
    const int *seg_off = a.seg_off;
    int *flags = a.flags;
    unsigned *status = a.status;
    void *args[] = {(void *)&reps, (void *)&work, (void *)&y, (void *)&acc, (void *)&out, (void *)&red, (void *)&tw,
                    (void *)&nsteps, (void *)&step_base, (void *)&rio, (void *)&eta, (void *)&tol, (void *)&rc2,
                    (void *)&max_iter, (void *)&segs, (void *)&seg_off, (void *)&flags, (void *)&status,
                    (void *)&use_wbuf};
    // cudaLaunchKernelEx with the cooperative attribute is also legal inside a
    // stream capture (graph kernel node)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.ncta);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = a.smem;
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void *)kern, args);
}

template <int P, typename T, int MODE, int NT>
static int fused_occupancy_nt(size_t smem)
{
    int n = 0;
    cudaFuncSetAttribute(k_fused<P, T, MODE, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<P, T, MODE, NT>, NT, smem) != cudaSuccess) return 0;
    return n;
}

template <int P, typename T, int MODE>
static int fused_occupancy(int variant, size_t smem)
{
    if (variant == 1) {
        if constexpr (NTV<P, 1>::v > 0) return fused_occupancy_nt<P, T, MODE, NTV<P, 1>::v>(smem);
        return 0;
    }
    if (variant == 2) {
        if constexpr (NTV<P, 2>::v > 0) return fused_occupancy_nt<P, T, MODE, NTV<P, 2>::v>(smem);
        return 0;
    }
    return fused_occupancy_nt<P, T, MODE, NTV<P, 0>::v>(smem);
}

template <int P, typename T, int MODE>
static cudaError_t launch_stepper(const LaunchArgs &a)
{
    if (a.variant == 1) {
        if constexpr (NTV<P, 1>::v > 0) return launch_fused_t<P, T, MODE, NTV<P, 1>::v>(a);
        return cudaErrorInvalidValue;
    }
    if (a.variant == 2) {
        if constexpr (NTV<P, 2>::v > 0) return launch_fused_t<P, T, MODE, NTV<P, 2>::v>(a);
        return cudaErrorInvalidValue;
    }
    return launch_fused_t<P, T, MODE, NTV<P, 0>::v>(a);
}

template <int P, typename T>
static cudaError_t launch_fused_p(const LaunchArgs &a)
{
    constexpr int NT0 = FusedNT<P>::v;
    switch (a.mode) {
    case M_FIELD: return launch_fused_t<P, T, M_FIELD, NT0>(a);
    case M_ENERGY: return launch_fused_t<P, T, M_ENERGY, NT0>(a);
    case M_RK4: return launch_stepper<P, T, M_RK4>(a);
    case M_HEUN: return launch_stepper<P, T, M_HEUN>(a);
    case M_RELAX: return launch_fused_t<P, T, M_RELAX, NT0>(a);
    default: return cudaErrorInvalidValue;
    }
}

template <int P, typename T, int MODE>
static void launch_g_epi(const LaunchArgs &a, dim3 ge, int stage, unsigned long long step)
{
    k_g_epi<P, T, MODE><<<ge, 256, 0, a.stream>>>(a.reps, a.work, (T *)a.ms, (T *)a.y, (T *)a.acc, (T *)a.out,
                                                   (const cplx<T> *)a.spec, a.red, stage, step);
}

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while its predecessor finishes, and waits for it in wait_prior_grid().
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// The stepping epilogue with quad access when the state buffers allow it.
template <int P, typename T, int MODE>
static void launch_g_epi_step(const LaunchArgs &a, int maxD, int stage, unsigned long long step)
{
    const bool quad = ((reinterpret_cast<uintptr_t>(a.y) | reinterpret_cast<uintptr_t>(a.ms) |
                        reinterpret_cast<uintptr_t>(a.acc)) & 15) == 0;
    if (quad) {
        const int maxq = maxD * ((maxD + 3) / 4);
        launch_pdl(k_g_epi_quad<P, T, MODE>, dim3((maxq + 255) / 256, a.nwork), dim3(256), 0, a.stream, a.reps,
                   a.work, (T *)a.ms, (T *)a.y, (T *)a.acc, (const cplx<T> *)a.spec, stage, step);
    } else {
        launch_g_epi<P, T, MODE>(a, dim3((maxD * maxD + 255) / 256, a.nwork), stage, step);
    }
}

// The FFT passes of one field evaluation on the global path: stage buffer ->
// spectrum (forward rows), the column pass, spectrum -> field rows in the
// spectrum buffer (inverse rows).
template <int P, typename T>
static void glob_rows(const LaunchArgs &a, int maxD, int inverse)
{
    constexpr int NT = GlobNT<P>::v, NGRP = groups_per_block<P, NT>();
    const int nrow = row_tasks(maxD);
    dim3 gr((nrow + NGRP - 1) / NGRP, a.nwork);
    launch_pdl(k_g_rows<P, T, NT>, gr, dim3(NT), glob_smem_bytes<P, T, NT>(), a.stream, a.reps, a.work,
               (const T *)a.ms, (cplx<T> *)a.spec, (const cplx<T> *)a.tw, inverse);
}

template <int P, typename T>
static void glob_cols(const LaunchArgs &a, int maxD)
{
    constexpr int NT = GlobNT<P>::v, NGRP = groups_per_block<P, NT>();
    if constexpr (GlobTiled<P>::v) {
        using CX = ColTile<P, T, true>;
        using CZ = ColTile<P, T, false>;
        const int ntask = a.nwork * CX::NCB;
        const int gx = ntask < a.n_sm * CX::MINB ? ntask : a.n_sm * CX::MINB;
        const int gz = ntask < a.n_sm * CZ::MINB ? ntask : a.n_sm * CZ::MINB;
        launch_pdl(k_g_cols_tile<P, T, true>, dim3(gx), dim3(CX::NT), glob_smem_bytes<P, T, CX::NT>(), a.stream,
                   a.reps, a.work, a.nwork, (cplx<T> *)a.spec, (const cplx<T> *)a.tw);
        launch_pdl(k_g_cols_tile<P, T, false>, dim3(gz), dim3(CZ::NT), glob_smem_bytes<P, T, CZ::NT>(), a.stream,
                   a.reps, a.work, a.nwork, (cplx<T> *)a.spec, (const cplx<T> *)a.tw);
    } else {
        dim3 gc((P / 2 + NGRP - 1) / NGRP, a.nwork);
        launch_pdl(k_g_cols<P, T, NT>, gc, dim3(NT), glob_smem_bytes<P, T, NT>(), a.stream, a.reps, a.work,
                   (cplx<T> *)a.spec, (const cplx<T> *)a.tw);
    }
}

template <int P, typename T>
static void glob_field_passes(const LaunchArgs &a, int maxD)
{
    glob_rows<P, T>(a, maxD, 0);
    glob_cols<P, T>(a, maxD);
    glob_rows<P, T>(a, maxD, 1);
}

// One field evaluation on the global path with its epilogue.
template <int P, typename T>
static cudaError_t glob_eval(const LaunchArgs &a, int maxD, int stage, int mode, unsigned long long step)
{
    glob_field_passes<P, T>(a, maxD);
    dim3 ge((maxD * maxD + 255) / 256, a.nwork);
    switch (mode) {
    case M_FIELD: launch_g_epi<P, T, M_FIELD>(a, ge, stage, step); break;
    case M_ENERGY: launch_g_epi<P, T, M_ENERGY>(a, ge, stage, step); break;
    case M_RK4: launch_g_epi_step<P, T, M_RK4>(a, maxD, stage, step); break;
    case M_HEUN: launch_g_epi_step<P, T, M_HEUN>(a, maxD, stage, step); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int P, typename T>
static cudaError_t launch_global_p(const LaunchArgs &a, int maxD)
{
    constexpr int NT = GlobNT<P>::v;
    const int sm = (int)glob_smem_bytes<P, T, NT>();
    cudaError_t e0 = cudaFuncSetAttribute(k_g_rows<P, T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e0 == cudaSuccess) e0 = cudaFuncSetAttribute(k_g_cols<P, T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if constexpr (GlobTiled<P>::v) {
        if (e0 == cudaSuccess)
            e0 = cudaFuncSetAttribute(k_g_cols_tile<P, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)glob_smem_bytes<P, T, ColTile<P, T, true>::NT>());
        if (e0 == cudaSuccess)
            e0 = cudaFuncSetAttribute(k_g_cols_tile<P, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)glob_smem_bytes<P, T, ColTile<P, T, false>::NT>());
    }
    if (e0 != cudaSuccess) return e0;

    dim3 gl((maxD * maxD + 255) / 256, a.nwork);
    launch_pdl(k_g_load_stage<T>, gl, dim3(256), 0, a.stream, a.reps, a.work, (const T *)a.y, (T *)a.ms);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.mode == M_RELAX) {
        if (!a.rio || !a.part || !a.rio_host || !a.work_host) return cudaErrorInvalidValue;
        const dim3 gp(kRelaxBlocks, a.nwork), gu((maxD * maxD + 255) / 256, a.nwork);
        constexpr int kCheck = 32;   // iterations between host checks for convergence of every replica
        for (int it = 0; it < a.max_iter; ++it) {
            glob_field_passes<P, T>(a, maxD);
            k_g_relax_reduce<P, T><<<gp, 256, 0, a.stream>>>(a.reps, a.work, (const T *)a.ms, (const cplx<T> *)a.spec,
                                                             a.rio, a.rc2, a.eta, a.part);
            k_g_relax_newton<<<(a.nwork + 127) / 128, 128, 0, a.stream>>>(a.work, a.nwork, a.rio, a.part, a.tol, it);
            k_g_relax_update<P, T><<<gu, 256, 0, a.stream>>>(a.reps, a.work, (T *)a.ms, (const cplx<T> *)a.spec, a.rio,
                                                             a.rc2, a.eta);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((it + 1) % kCheck == 0 || it + 1 == a.max_iter) {
                // a synchronous read of the parameter array; stop once every
                // replica of this launch has converged
                if ((e = cudaMemcpyAsync(a.rio_host, a.rio, sizeof(RelaxIO) * a.n_rio, cudaMemcpyDeviceToHost,
                                         a.stream)) != cudaSuccess)
                    return e;
                if ((e = cudaStreamSynchronize(a.stream)) != cudaSuccess) return e;
                bool running = false;
                for (int k = 0; k < a.nwork && !running; ++k) running = a.rio_host[a.work_host[k]].status != 0;
                if (!running) break;
            }
        }
        k_g_store_stage<T><<<gl, 256, 0, a.stream>>>(a.reps, a.work, (const T *)a.ms, (T *)a.y);
        return cudaGetLastError();
    }
    const int nst = (a.mode == M_RK4) ? 4 : (a.mode == M_HEUN ? 2 : 1);
    const long long nsteps = (a.mode == M_FIELD || a.mode == M_ENERGY) ? 1 : a.nsteps;
    for (long long n = 0; n < nsteps; ++n)
        for (int s = 0; s < nst; ++s) {
            e = glob_eval<P, T>(a, maxD, s, a.mode, a.step_base + n);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

}  // namespace nd
