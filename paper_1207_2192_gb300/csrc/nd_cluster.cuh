// nd_cluster.cuh -- one replica's time steps on a thread-block cluster of NC
// CTAs (one per SM): for the sizes P <= 128 when a class has too few replicas
// to fill the GPU with one CTA each, and for P = 192 and 256, whose spectra
// fit in the shared memory of 16 CTAs but not of one.
//
// The replica's rows are split over the cluster: CTA k owns rows
// [k rpc, (k+1) rpc) of the disk (rpc even, so z row pairs stay whole) and
// the column slots [k spc, (k+1) spc) of the P/2 slots of the half spectrum
// (slot 0: the real columns kx = 0 and P/2 packed as one complex column).
// Per field evaluation (Section II.B convolution):
//   1. forward rows: each CTA transforms its own rows (at P = 128 one real
//      row per task at half length, else row pairs) and stores every
//      spectrum entry straight into the shared memory of the CTA that owns
//      its column (st.async into distributed shared memory, counted on the
//      owner's transaction barrier: no thread waits on a remote load or on
//      its own stores);
//   2. each CTA waits until its column slots hold every row;
//   3. columns: one FFT group per (slot, component) transforms its column
//      from local shared memory, applies the spectral kernel (the x and y
//      groups of a column exchange their spectra for the in-plane 2x2 block;
//      the kernel's entries of the CTA's columns are staged in shared memory
//      once per launch), transforms back and stores the rows into the shared
//      memory of their owners (st.async again);
//   4. each CTA waits until its rows hold every column;
//   5. inverse rows and the per-cell epilogue (stage_update) on the CTA's own
//      rows; the next stage's forward rows read only those rows, so a CTA
//      barrier suffices until the next exchange.
// The state y_n, the stage accumulator and the Heun predictor's normals of the
// CTA's rows stay in its shared memory for the whole launch: global memory is
// read once at the start and written once at the end.  The waits on the
// transaction barriers give up after about two seconds, set ND_DEV_TIMEOUT in
// the status word and skip the remaining waits, so a launch always ends.
#pragma once
#include <cooperative_groups.h>

#include "nd_field_impl.cuh"

namespace nd {

namespace cgc = cooperative_groups;

template <int P, typename T, int NC> struct ClusterGeom {
    static constexpr int G = FFTGeom<P>::G;
    // threads per CTA: enough FFT groups for one per (column slot, component)
    static constexpr int NT = cluster_cta_threads(P);
    static constexpr int NGRP = NT / G;
    static constexpr int SPC = (P / 2) / NC;   // column slots per CTA
    static_assert(SPC >= 1 && (P / 2) % NC == 0, "column slots split evenly over the cluster");
    static_assert(3 * SPC <= NGRP, "one FFT group per (slot, component)");
    static constexpr int KH = SpecGeom<P>::KH;
    // column buffer [3][P/2][SW]: row y of the CTA's SPC column slots, SW = SPC + 1
    // words apart so that a group's column reads fall in different banks, and
    // the lanes of a row group store neighbouring slots of one row
    static constexpr int SW = SPC + 1;
    static constexpr int NTAB = SPC + 1;       // table slots: the CTA's columns, then kx = P/2
};

// Rows per CTA for a grid of D rows: even, so that z row pairs stay in one CTA.
__host__ __device__ __forceinline__ int cluster_rows(int D, int NC) { return 2 * ((D + 2 * NC - 1) / (2 * NC)); }

template <int P, typename T, int NC>
__host__ __device__ __forceinline__ size_t cluster_smem_bytes(int D, int Dpad, bool wbuf)
{
    using CG = ClusterGeom<P, T, NC>;
    const int rpc = cluster_rows(D, NC);
    size_t b = sizeof(cplx<T>) * ((size_t)FFTGeom<P>::R1 * FFTGeom<P>::G               // twiddles
                                  + (size_t)3 * (P / 2) * CG::SW                        // column buffer
                                  + (size_t)3 * rpc * SpecGeom<P>::RS                   // spectrum rows
                                  + (size_t)CG::NGRP * FFTGeom<P>::SCRATCH);            // FFT scratch
    b += sizeof(T) * (size_t)4 * CG::NTAB * CG::KH;                                     // kernel table
    b += sizeof(T) * (size_t)3 * rpc * Dpad * (wbuf ? 4 : 3);   // stage state, y_n, accumulator (+ normals)
    b += 2 * sizeof(int);                                                               // own cell range
    b += 16;                                                                            // two mbarriers
    return b;
}

// The spectral step of the packed real columns kx = 0 and P/2 of one
// component after the forward transform of c0 + i c_{P/2}: separation with
// the mirror element, the diagonal kernel entries s0 (kx = 0) and s1
// (kx = P/2) from shared memory, and re-packing for the inverse transform.
template <int P, typename T>
__device__ __forceinline__ void cluster_packed_scale(cplx<T> *v, const T *s0t, const T *s1t, int t, cplx<T> *scr,
                                                     unsigned gmask)
{
    using Gm = FFTGeom<P>;
    constexpr int G = Gm::G, R1 = Gm::R1;
    mirror_put<P>(v, scr, t);
    __syncwarp(gmask);
#pragma unroll
    for (int o = 0; o < R1; ++o) {
        const int ky = t + G * o;
        const int kyr = ky <= P / 2 ? ky : P - ky;
        const cplx<T> w = mirror_get<P>(scr, ky);
        const T h = T(0.5);
        cplx<T> F0 = {h * (v[o].x + w.x), h * (v[o].y - w.y)};
        cplx<T> F1 = {h * (v[o].y + w.y), -h * (v[o].x - w.x)};
        F0 = cscale(F0, s0t[kyr]);
        F1 = cscale(F1, s1t[kyr]);
        v[o] = {F0.x - F1.y, F0.y + F1.x};
    }
    __syncwarp(gmask);
}

// Distributed-shared-memory exchange with transaction barriers: a producer
// stores into another CTA's shared memory with st.async, which also counts
// the bytes on that CTA's mbarrier; the consumer waits until its barrier has
// seen all the bytes it expects.  No producer waits on its own stores, and
// each CTA waits only for the data it reads.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_async(uint32_t a, cplx<float> v, uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
                 :: "r"(a), "f"(v.x), "f"(v.y), "r"(mbar) : "memory");
}
__device__ __forceinline__ void st_async(uint32_t a, cplx<double> v, uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
                 :: "r"(a), "d"(v.x), "d"(v.y), "r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase of the given parity to complete, acquiring at
// cluster scope what the producers stored.  Gives up after about two seconds
// of the global timer (a producer that never delivers) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    unsigned long long t0 = 0;
    for (unsigned it = 0; it < (1u << 30); ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
        if ((it & 63) == 63) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > 2000000000ull) return false;
        }
    }
    return false;
}

template <int P, typename T, int MODE, int NC>
__global__ void __launch_bounds__(ClusterGeom<P, T, NC>::NT, 1)
    k_cluster(const Replica *__restrict__ reps, const int *__restrict__ work, T *__restrict__ ybase,
              const cplx<T> *__restrict__ twP, long long nsteps, unsigned long long step_base, int use_wbuf,
              unsigned *__restrict__ status)
{
    using Gm = FFTGeom<P>;
    using CG = ClusterGeom<P, T, NC>;
    constexpr int G = Gm::G, R1 = Gm::R1, RS = SpecGeom<P>::RS, KH = CG::KH, NT = CG::NT, NGRP = CG::NGRP;
    constexpr int SPC = CG::SPC, SW = CG::SW, NTAB = CG::NTAB;
    static_assert(MODE == M_RK4 || MODE == M_HEUN, "stepping modes");
    cgc::cluster_group cluster = cgc::this_cluster();
    const int rank = (int)cluster.block_rank();
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    GroupId<P> gid(tid);
    const int ridx = work[blockIdx.x / NC];
    const Replica &r = reps[ridx];
    const int D = r.D, Dpad = r.Dpad, rpc = cluster_rows(D, NC);
    const int ylo = rank * rpc, nloc = max(0, min(D, ylo + rpc) - ylo);   // this CTA's rows [ylo, ylo + nloc)
    const long long lcs = (long long)rpc * RS;                            // local spectrum component stride
    const long long lms = (long long)rpc * Dpad;                          // local state component stride
    const long long ms_s = (long long)D * Dpad;                           // global state component stride
    unsigned long long *mbars = reinterpret_cast<unsigned long long *>(smem);   // [0] columns, [1] rows
    const uint32_t mb_col = smem_addr(mbars), mb_row = smem_addr(mbars + 1);
    cplx<T> *tw = reinterpret_cast<cplx<T> *>(smem + 16);
    cplx<T> *colbuf = tw + R1 * G;                                        // [3][P/2][SW]
    cplx<T> *spec = colbuf + 3 * (P / 2) * SW;                            // [3][rpc][RS]
    cplx<T> *scratch = spec + 3 * lcs;
    T *gtab = reinterpret_cast<T *>(scratch + NGRP * Gm::SCRATCH);        // [4][NTAB][KH]
    T *msl = gtab + 4 * NTAB * KH;                                        // [3][rpc][Dpad]
    T *ynl = msl + 3 * lms, *accl = ynl + 3 * lms;
    T *wl = use_wbuf ? accl + 3 * lms : nullptr;
    int *crange = reinterpret_cast<int *>((use_wbuf ? wl : accl) + 3 * lms);
    cplx<T> *scr = scratch + gid.group * Gm::SCRATCH;
    load_twiddles<P>(tw, twP, tid, NT);
    const V3Ptr<T> ms{msl, lms}, wb{wl, lms}, ynv{ynl, lms}, accv{accl, lms}, none{nullptr, 0};
    const V3Ptr<T> yg{ybase + r.state_off, ms_s};
    // the state of the CTA's rows (zero outside the disk)
    for (int i = tid; i < nloc * D; i += NT) {
        const int lr = i / D, x = i - lr * D, y = ylo + lr;
        const long long si = (long long)y * Dpad + x, mi = (long long)lr * Dpad + x;
        const vec3<T> m0 = r.mask[y * D + x] ? yg.ldcg(si) : vec3<T>{T(0), T(0), T(0)};
        ms.st(mi, m0);
        ynv.st(mi, m0);
    }
    // the kernel's entries of the CTA's columns (and of kx = P/2), from the
    // component-major copy of the table
    {
        constexpr int KK = KH * KH;
        const T *Gc = reinterpret_cast<const T *>(r.Ghat) + 4 * KK;
        for (int i = tid; i < 4 * NTAB * KH; i += NT) {
            const int c = i / (NTAB * KH), rem = i - c * (NTAB * KH), j = rem / KH, ky = rem - j * KH;
            const int kx = j < SPC ? rank * SPC + j : P / 2;
            gtab[i] = __ldg(Gc + (long long)c * KK + kx * KH + ky);
        }
    }
    // the CTA's cells: a contiguous range of the ascending cell list
    if (tid == 0) {
        int lo = 0, hi = r.ncells;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (__ldg(r.cells + mid) < ylo * D) lo = mid + 1; else hi = mid; }
        crange[0] = lo;
        hi = r.ncells;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (__ldg(r.cells + mid) < (ylo + nloc) * D) lo = mid + 1; else hi = mid; }
        crange[1] = lo;
    }
    // row tasks of this CTA: one real row per (component, row) at P = 128
    // (half-length transforms), else xy rows 0..nloc-1, then z pairs (0,1), ...
    constexpr bool HR = HalfRows<P>::on;
    const int nrt = HR ? 3 * nloc : nloc + (nloc + 1) / 2;
    const int nrounds = (nrt + NGRP - 1) / NGRP;
    // column task of this group: slot j (column kx = rank SPC + j, slot 0 of
    // rank 0 being the packed pair), component c
    const int cj = gid.group % SPC, cc = gid.group / SPC;
    const bool ctask = gid.group < 3 * SPC;   // groups beyond 3 SPC idle in the column pass
    const int kslot = rank * SPC + cj;
    const bool packed = ctask && kslot == 0;
    if (tid == 0) {
        mbar_init(mb_col, 1);
        mbar_init(mb_row, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    bool bailed = false;   // this thread's wait ran out once: it skips every later wait
    // bytes each CTA receives from the other CTAs per stage (what it sends to
    // itself goes by plain stores, made visible by a CTA barrier): its SPC
    // column slots of every other CTA's rows, and the P/2 + 1 spectrum entries
    // of each own row from the other CTAs' column slots (rank 0 holds the
    // packed pair: SPC + 1 entries of its own)
    const uint32_t bytes_col = (uint32_t)(3 * (D - nloc) * SPC * sizeof(cplx<T>));
    const uint32_t bytes_row = (uint32_t)(3 * nloc * (P / 2 + 1 - SPC - (rank == 0 ? 1 : 0)) * sizeof(cplx<T>));
    uint32_t phase = 0;
    cluster.sync();   // every CTA runs, with its barriers initialised, before the first remote store
    const int c0 = crange[0], c1 = crange[1];

    for (long long n = 0; n < nsteps; ++n) {
        const unsigned long long step = step_base + r.step0 + (unsigned long long)n;
        for (int stage = 0; stage < ModeStages<MODE>::n; ++stage) {
            if (tid == 0) {
                mbar_expect(mb_col, bytes_col);
                mbar_expect(mb_row, bytes_row);
            }
            // 1. forward rows of the CTA's own rows, sent to the column owners
            if constexpr (HR) {
                for (int q = gid.group; q < nrounds * NGRP; q += NGRP) {
                    const bool act = q < nrt;
                    const int c = act ? q / nloc : 0, l = act ? q - c * nloc : 0, y = ylo + l;
                    cplx<T> v[FFTGeom<P / 2>::R1];
                    T xm;
                    row_fwd_half_spectrum<P, T>(act, msl + c * lms + (long long)l * Dpad, D, v, xm, gid.t, scr, tw,
                                                gid.gmask);
                    if (act) {
#pragma unroll
                        for (int o = 0; o < FFTGeom<P / 2>::R1; ++o) {
                            const int k = gid.t + G * o;   // k = 0 goes with k = P/2 into the packed slot
                            const int ow = k / SPC, j = k - ow * SPC;
                            const cplx<T> a = k == 0 ? cplx<T>{v[o].x, xm} : v[o];
                            const int i = (c * (P / 2) + y) * SW + j;
                            if (ow == rank) {
                                colbuf[i] = a;
                            } else {
                                st_async(cluster_addr(smem_addr(colbuf), ow) + (uint32_t)(i * sizeof(cplx<T>)), a,
                                         cluster_addr(mb_col, ow));
                            }
                        }
                    }
                }
            } else
            for (int q = gid.group; q < nrounds * NGRP; q += NGRP) {
                const bool act = q < nrt;
                const bool isxy = q < nloc;
                const int l0 = isxy ? q : 2 * (q - nloc), l1 = l0 + 1;
                const bool hasB = isxy || (l1 < nloc);
                cplx<T> v[R1];
#pragma unroll
                for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
#pragma unroll
                for (int o = 0; o < R1 / 2; ++o) {
                    const int x = gid.t + G * o;
                    if (act && x < D) {
                        if (isxy) v[o] = {msl[(long long)l0 * Dpad + x], msl[lms + (long long)l0 * Dpad + x]};
                        else v[o] = {msl[2 * lms + (long long)l0 * Dpad + x],
                                     hasB ? msl[2 * lms + (long long)l1 * Dpad + x] : T(0)};
                    }
                }
                fft_group<P, -1, FFT_HALF_IN>(v, gid.t, scr, tw, gid.gmask);
                mirror_put<P>(v, scr, gid.t);
                __syncwarp(gid.gmask);
                if (act) {
                    // A: the row ending in the real part (x, or the first z row),
                    // B: the one ending in the imaginary part (y, or the second z row)
                    const int cA = isxy ? 0 : 2, cB = isxy ? 1 : 2;
                    const int yA = ylo + l0, yB = isxy ? ylo + l0 : ylo + l1;
                    T rA0 = T(0), rB0 = T(0);   // lane t = 0: the real entries at k = 0 (then k = P/2)
#pragma unroll
                    for (int o = 0; o < R1; ++o) {
                        const int k = gid.t + G * o;
                        if (k <= P / 2) {
                            const cplx<T> w = mirror_get<P>(scr, k);
                            const T h = T(0.5);
                            const cplx<T> A = {h * (v[o].x + w.x), h * (v[o].y - w.y)};
                            const cplx<T> B = {h * (v[o].y + w.y), -h * (v[o].x - w.x)};
                            if (k == 0) {
                                rA0 = A.x;
                                rB0 = B.x;
                            } else {
                                const int ow = k == P / 2 ? 0 : k / SPC, j = k == P / 2 ? 0 : k - ow * SPC;
                                const cplx<T> a = k == P / 2 ? cplx<T>{rA0, A.x} : A;
                                const cplx<T> b2 = k == P / 2 ? cplx<T>{rB0, B.x} : B;
                                const int iA = (cA * (P / 2) + yA) * SW + j, iB = (cB * (P / 2) + yB) * SW + j;
                                if (ow == rank) {
                                    colbuf[iA] = a;
                                    if (hasB) colbuf[iB] = b2;
                                } else {
                                    const uint32_t base = cluster_addr(smem_addr(colbuf), ow);
                                    const uint32_t mb = cluster_addr(mb_col, ow);
                                    st_async(base + (uint32_t)(iA * sizeof(cplx<T>)), a, mb);
                                    if (hasB) st_async(base + (uint32_t)(iB * sizeof(cplx<T>)), b2, mb);
                                }
                            }
                        }
                    }
                }
                __syncwarp(gid.gmask);
            }
            // every row spectrum of this CTA's columns has arrived (the
            // barrier makes the CTA's own plain stores visible)
            if (!bailed && !mbar_wait(mb_col, phase & 1)) {
                bailed = true;
                atomicOr(status, ND_DEV_TIMEOUT);
            }
            __syncthreads();
            // 3. columns from the local column buffer, back to the row owners
            {
                cplx<T> v[R1];
#pragma unroll
                for (int o = 0; o < R1; ++o) v[o] = {T(0), T(0)};
                const int kx = packed ? 0 : kslot;
                if (ctask) {
                    const cplx<T> *col = colbuf + cc * (P / 2) * SW + cj;
#pragma unroll
                    for (int o = 0; o < R1 / 2; ++o) {
                        const int y = gid.t + G * o;
                        if (y < D) v[o] = col[y * SW];
                    }
                }
                // one transform call for both kinds of column, so that a warp
                // holding the packed slot does not run two transforms in turn
                if (ctask) fft_group<P, -1, FFT_HALF_IN>(v, gid.t, scr, tw, gid.gmask);
                if (packed) {
                    const int comp = cc == 2 ? 3 : cc;   // the diagonal entry: xx, yy or zz
                    cluster_packed_scale<P, T>(v, gtab + (comp * NTAB) * KH, gtab + (comp * NTAB + SPC) * KH, gid.t,
                                               scr, gid.gmask);
                }
                // the x and y groups of a column exchange their spectra
                if (ctask && !packed && cc < 2) {
#pragma unroll
                    for (int o = 0; o < R1; ++o) scr[o * G + gid.t] = v[o];
                }
                __syncthreads();
                if (ctask && !packed) {
                    if (cc < 2) {
                        const cplx<T> *other = scratch + ((1 - cc) * SPC + cj) * Gm::SCRATCH;
                        const T *gd = gtab + (cc * NTAB + cj) * KH, *go = gtab + (2 * NTAB + cj) * KH;
#pragma unroll
                        for (int o = 0; o < R1; ++o) {
                            const int ky = gid.t + G * o;
                            const bool up = ky <= P / 2;
                            const int kyr = up ? ky : P - ky;
                            const T gdiag = gd[kyr], gxy0 = go[kyr];
                            const T gxy = up ? gxy0 : -gxy0;   // G_xy is odd in ky
                            const cplx<T> w = other[o * G + gid.t];
                            v[o] = cc == 0 ? tensor_row(gdiag, v[o], gxy, w) : tensor_row(gxy, w, gdiag, v[o]);
                        }
                    } else {
                        const T *gz = gtab + (3 * NTAB + cj) * KH;
#pragma unroll
                        for (int o = 0; o < R1; ++o) {
                            const int ky = gid.t + G * o;
                            const int kyr = ky <= P / 2 ? ky : P - ky;
                            v[o] = cscale(v[o], gz[kyr]);
                        }
                    }
                }
                __syncthreads();   // the partners' spectra are read before the scratch is reused
                if (ctask) fft_group<P, +1, FFT_HALF_OUT>(v, gid.t, scr, tw, gid.gmask);
#pragma unroll
                for (int o = 0; o < R1 / 2; ++o) {
                    const int y = gid.t + G * o;
                    if (ctask && y < D) {
                        const int ow = y / rpc, lr = y - ow * rpc;   // the row's owner
                        cplx<T> *dst = spec + cc * lcs + (long long)lr * RS;
                        if (ow == rank) {
                            if (packed) {
                                dst[0] = {v[o].x, T(0)};
                                dst[P / 2] = {v[o].y, T(0)};
                            } else {
                                dst[kx] = v[o];
                            }
                        } else {
                            const uint32_t row = cluster_addr(smem_addr(dst), ow);
                            const uint32_t mb = cluster_addr(mb_row, ow);
                            if (packed) {
                                st_async(row, cplx<T>{v[o].x, T(0)}, mb);
                                st_async(row + (uint32_t)((P / 2) * sizeof(cplx<T>)), cplx<T>{v[o].y, T(0)}, mb);
                            } else {
                                st_async(row + (uint32_t)(kx * sizeof(cplx<T>)), v[o], mb);
                            }
                        }
                    }
                }
            }
            // every column entry of this CTA's rows has arrived
            if (!bailed && !mbar_wait(mb_row, phase & 1)) {
                bailed = true;
                atomicOr(status, ND_DEV_TIMEOUT);
            }
            __syncthreads();
            ++phase;
            // 5. inverse rows of the CTA's own rows (the field rows, in place)
            if constexpr (HR) {
                for (int q = gid.group; q < nrounds * NGRP; q += NGRP) {
                    const bool act = q < nrt;
                    const int c = act ? q / nloc : 0, l = act ? q - c * nloc : 0;
                    cplx<T> *row = spec + c * lcs + (long long)l * RS;
                    row_inv_half<P, T>(act, row, D, reinterpret_cast<T *>(row), gid.t, scr, tw, gid.gmask);
                }
            } else
            for (int q = gid.group; q < nrounds * NGRP; q += NGRP) {
                const bool act = q < nrt;
                const bool isxy = q < nloc;
                const int l0 = isxy ? q : 2 * (q - nloc), l1 = l0 + 1;
                const bool hasB = isxy || (l1 < nloc);
                cplx<T> *rA = isxy ? spec + (long long)l0 * RS : spec + 2 * lcs + (long long)l0 * RS;
                cplx<T> *rB = isxy ? spec + lcs + (long long)l0 * RS : spec + 2 * lcs + (long long)l1 * RS;
                cplx<T> v[R1];
                row_inv_fft<P, T>(v, act, rA, rB, hasB, gid.t, scr, tw, gid.gmask);
                if (act) {
                    T *oA = reinterpret_cast<T *>(rA), *oB = reinterpret_cast<T *>(rB);
#pragma unroll
                    for (int o = 0; o < R1 / 2; ++o) {
                        const int x = gid.t + G * o;
                        if (x < D) {
                            oA[x] = v[o].x;
                            if (hasB) oB[x] = v[o].y;
                        }
                    }
                }
            }
            __syncthreads();
            // the per-cell epilogue of the CTA's cells
            const StepParams<T> sp = step_params<T>(r);
            const vec3<T> cx = step_chext<T>(r, sp, step);
            const T *hr = reinterpret_cast<const T *>(spec);
            for (int k = c0 + tid; k < c1; k += NT) {
                const int cell = __ldg(r.cells + k);
                const int y = cell / D, x = cell - y * D, lr = y - ylo;
                const long long mi = (long long)lr * Dpad + x;
                const long long hi = (long long)lr * (2 * RS) + x;
                const vec3<T> b = {hr[hi] + cx.x, hr[2 * lcs + hi] + cx.y, hr[4 * lcs + hi] + cx.z};
                epilogue_cell<T, MODE>(r, cell, mi, mi, b, ms, ynv, accv, none, stage, step, wb, ynv, accv);
            }
            __syncthreads();
        }
    }
    // the final state of the CTA's cells back to the caller's buffer
    for (int k = c0 + tid; k < c1; k += NT) {
        const int cell = __ldg(r.cells + k);
        const int y = cell / D, x = cell - y * D;
        yg.st((long long)y * Dpad + x, ynv.ld((long long)(y - ylo) * Dpad + x));
    }
    cluster.sync();   // no CTA leaves while another may still access its shared memory
}

// Launch configuration of one replica per cluster of NC CTAs (the cluster
// shape is a launch attribute; NC = 16 is a non-portable size the GPU allows).
template <int P, typename T, int MODE, int NC>
static cudaError_t cluster_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int nwork, size_t sm,
                                  cudaStream_t st)
{
    auto kern = k_cluster<P, T, MODE, NC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess && NC > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(nwork * NC, 1, 1);
    cfg.blockDim = dim3(ClusterGeom<P, T, NC>::NT, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaSuccess;
}

template <int P, typename T, int MODE, int NC>
static cudaError_t launch_cluster_t(const LaunchArgs &a, int maxD, int maxDpad)
{
    const size_t sm = cluster_smem_bytes<P, T, NC>(maxD, maxDpad, a.use_wbuf != 0);
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = cluster_config<P, T, MODE, NC>(cfg, attr, a.nwork, sm, a.stream);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_cluster<P, T, MODE, NC>, a.reps, a.work, (T *)a.y, (const cplx<T> *)a.tw,
                              a.nsteps, a.step_base, a.use_wbuf, a.status);
}

// Clusters of the size class that can be resident at once (0: the cluster
// shape or its shared memory does not fit this GPU).
template <int P, typename T, int NC>
static int cluster_max_active_t(int maxD, int maxDpad, bool wbuf)
{
    const size_t sm = cluster_smem_bytes<P, T, NC>(maxD, maxDpad, wbuf);
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (cluster_config<P, T, M_HEUN, NC>(cfg, attr, 1, sm, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_cluster<P, T, M_HEUN, NC>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int P, typename T, int NC>
static cudaError_t launch_cluster_p(const LaunchArgs &a, int maxD, int maxDpad)
{
    if (a.mode == M_RK4) return launch_cluster_t<P, T, M_RK4, NC>(a, maxD, maxDpad);
    if (a.mode == M_HEUN) return launch_cluster_t<P, T, M_HEUN, NC>(a, maxD, maxDpad);
    return cudaErrorInvalidValue;
}

}  // namespace nd
