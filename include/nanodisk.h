/*
 * nanodisk.h -- C ABI of the GB300 thin-nanodisk micromagnetics library
 * (libnanodisk.so).
 *
 * The library computes the per-time-step effective field of thin circular
 * ferromagnetic disks discretised into a x a x L cells, following Wysin &
 * Figueiredo, "Thermal vortex dynamics in thin circular ferromagnetic
 * nanodisks" (2012):
 *   - the demagnetisation field of the thin-film Green's tensor (Sec. II.B),
 *     applied as a zero-padded FFT convolution over the square grid masked to
 *     the disk, plus the nearest-neighbour exchange field (Eq. Bi);
 *   - the Landau-Lifshitz equation with damping, stepped with RK4 at T = 0
 *     (Sec. III.A) or with the stochastic Heun scheme of the Langevin
 *     equation at T > 0 (Eq. LV, Sec. III.C);
 *   - the energy of Eq. Hmm, the vortex-core estimator of Sec. IV, the
 *     analytic vortex profile of Sec. IV, and the average magnetisation.
 *
 * Conventions common to every call
 * --------------------------------
 * Units.  Physical inputs are SI (metres, A/m, J/m, seconds, kelvin).  Fields
 * returned by the library are the dimensionless induction b_i of Eq. Bi (unit
 * B0 = 2A/(a^2 Ms)); energies are in units of J = 2AL of the replica's disk.
 *
 * Grid.  A disk of radius R and cell edge a has D = round(2R/a) cells per
 * side.  Cell (i, j) (column i = x index, row j = y index) has its centre at
 * ((i - (D-1)/2) a, (j - (D-1)/2) a) and belongs to the disk iff that centre
 * lies within R.  The FFT grid side P is the smallest power of two >= 2D - 1
 * (at least 16; 192 or 200 instead of 256 with ND_GRID_3X), which makes the circular
 * convolution equal the linear one.
 *
 * State layout.  One handle holds B replicas (disk-major: the replicas of disk
 * 0 first).  A state buffer is one contiguous array of the handle's precision
 * (float for ND_FP32, double for ND_FP64); replica r occupies
 * [3][D_r][Dpad_r] elements starting at the offset nd_replica_layout reports,
 * where Dpad_r = D_r rounded up to a multiple of 4 and components are x, y, z.
 * Cells outside the disk read as zero (any value stored there is ignored) and
 * are written as zero or left unchanged; padding columns are never touched.
 *
 * Pointers.  Array arguments named m or b may be device pointers or host
 * pointers (pageable or pinned); the library inspects each.  With a host
 * pointer the call copies the data to a device staging buffer, runs, copies
 * results back, and returns after synchronising the stream.  With device
 * pointers the call is asynchronous on `stream` (a cudaStream_t, NULL for the
 * legacy default stream) unless it returns host scalars, in which case it
 * synchronises `stream` before returning.  Scalar outputs (E_out, Xc_out, ...)
 * are always host pointers.  The caller owns every buffer it passes; the
 * handle owns its spectral kernels, twiddle tables and scratch.
 *
 * Errors.  Every call returns ND_OK (0) or a positive ND_ERR_* code; no
 * exception crosses the ABI.  nd_last_error() returns a description of the
 * most recent failure on the calling thread.  A handle is not thread-safe and
 * calls on one handle must be ordered (one stream, or synchronised).
 */
#ifndef NANODISK_H
#define NANODISK_H

#ifdef __cplusplus
extern "C" {
#endif

#define ND_OK 0
#define ND_ERR_ARG 1            /* invalid argument or unsupported size */
#define ND_ERR_CUDA 2           /* a CUDA runtime call failed */
#define ND_ERR_NOT_CONVERGED 3  /* relaxation hit max_iter */
#define ND_ERR_NO_VORTEX 4      /* no plaquette with winding +1 */
#define ND_ERR_TIMEOUT 5        /* a bounded device-side wait expired */
#define ND_ERR_NAN 6            /* a non-finite value appeared in the state */

#define ND_FP32 0               /* float state and fields, FP64 energies and core sums */
#define ND_METHOD_RK4 0         /* stepping methods (nd_autotune, nd_graph_create) */
#define ND_METHOD_HEUN 1
#define ND_FP64 1               /* double everywhere */
#define ND_GRID_3X 0x100        /* nd_create_disk flag (or-ed into precision): allow the padded
                                   sizes 192 = 3 * 64 for disks of 65..96 cells and
                                   200 = 8 * 25 for 97..100 cells (see there) */

typedef struct nd_handle nd_handle;

/* One disk geometry and material (SI).  hext is the uniform external field
 * H_ext in A/m (Eq. Hmm); alpha the damping of Sec. III.A; polarity (+1/-1)
 * and chirality (+1 counter-clockwise, -1 clockwise) are used by
 * nd_init_vortex only. */
typedef struct {
    double R, L, a;
    double Ms, A, gamma;
    double alpha;
    double hext[3];
    int polarity, chirality;
} nd_disk_desc;

/* Create a handle for n_disks geometries with replicas_per_disk[d] replicas
 * each (replicas_per_disk may be NULL: one replica per disk).  Builds each
 * disk's mask and its spectral kernel from the thin-film Green's tensor of
 * Sec. II.B (in-plane and out-of-plane components averaged over the
 * thickness, cell self terms -N_x, -N_x, -N_z of a cylinder of radius
 * a/sqrt(pi)) with the exchange stencil folded in.  Requires D >= 1 and
 * P <= 1024.  precision is ND_FP32 or ND_FP64, optionally or-ed with
 * ND_GRID_3X: then disks of 65..96 cells get the padded grid P = 192 = 8 x 24
 * (an FFT with one radix-3 stage) and disks of 97..100 cells P = 200 = 10 x 20
 * (radix-5 stages, ten-lane FFT groups) instead of 256 -- any P >= 2D - 1 makes
 * the circular convolution equal the linear one; the paper's power-of-two rule
 * (Sec. II.B) is a convenience -- with 44% and 39% fewer spectral points.
 * P = 200 runs on the global path only (no cluster plan).  On success
 * *out receives the handle; the call synchronises the current device. */
int nd_create_disk(const nd_disk_desc *disks, int n_disks, const int *replicas_per_disk, int precision,
                   nd_handle **out);

/* Release the handle and everything it owns.  NULL is accepted. */
void nd_destroy(nd_handle *h);

/* Description of the last error on this thread ("" if none). */
const char *nd_last_error(void);

/* Number of replicas and the total number of elements of a state buffer. */
int nd_get_info(const nd_handle *h, int *n_replicas, long long *state_elems);

/* Layout of replica r: grid side D, padded row Dpad, FFT side P, element
 * offset of its [3][D][Dpad] block in a state buffer, and its active cells
 * (cells inside the disk).  Any output pointer may be NULL. */
int nd_replica_layout(const nd_handle *h, int r, int *D, int *Dpad, int *P, long long *offset, int *n_cells);

/* Copy disk d's mask ([D][D] bytes, 1 inside the disk) to host memory. */
int nd_disk_mask(const nd_handle *h, int d, unsigned char *mask_out);

/* Units of disk d (Sec. III.A): out[0] lambda_ex (m), out[1] a^2/lambda_ex^2,
 * out[2] B0 (T), out[3] t0 = 1/(gamma B0) (s), out[4] J = 2AL (J),
 * out[5] N_x, out[6] N_z, out[7] cells inside the disk. */
int nd_units(const nd_handle *h, int d, double out[8]);

/* Rebuild disk d's spectral kernel (Sec. II.B, "FFT of the Green's matrix,
 * done only once").  Gq == NULL rebuilds it from the paper's closed forms.
 * Otherwise Gq is a host array [4][D][D] of a^2 G at cell displacements
 * (dx, dy) >= 0, components xx, yy, xy, zz, self terms at [.][0][0], extended
 * to negative displacements by the tensor's symmetry (xx, yy, zz even in both
 * axes, xy odd in both).  Synchronises the device. */
int nd_set_green_tensor(nd_handle *h, int d, const double *Gq);

/* Per-replica damping alpha (host array [B]); replaces the disks' values. */
int nd_set_damping(nd_handle *h, const double *alpha);

/* Variant of the geometry (Sec. II.A's element, not necessarily circular):
 * replace disk d's mask by any set of cells of its D x D grid.  mask is a host
 * array [D][D] (row j = y index, column i = x index), nonzero inside.  The grid
 * D, the padded size P and the spectral kernel stay (the kernel does not depend
 * on the mask, and the exchange folded into it stays exact because cells
 * outside the mask hold zero); every later call -- field, energy, stepping,
 * relaxation, core estimator, statistics -- uses the new cell set, and
 * nd_replica_layout / nd_units report its cell count.  State values outside
 * the new mask are ignored and left unchanged.  Synchronises the device. */
int nd_set_mask(nd_handle *h, int d, const unsigned char *mask);

/* Time-dependent external field (Sec. II.A's H_ext switched per time step: a
 * pulse, or any schedule): step s of the stepping calls uses H_ext = H[s]
 * (host array [n_steps][3], A/m) for all stages of that step while
 * s < n_steps, and the disk's static hext afterwards.  The step index s is the
 * Heun noise counter (step0 + k in nd_step_heun and in graphs) and, for RK4,
 * a counter of the handle that starts at 0 when the schedule is set and
 * advances by n_steps with every nd_step_rk4 call (RK4 graphs use their
 * step0 argument and advance it per replay), so a run split over several
 * calls sees the same field as one call.  nd_effective_field, nd_energy and
 * nd_relax_constrained use the static field.  n_steps = 0 removes the
 * schedule.  Synchronises the device. */
int nd_set_field_schedule(nd_handle *h, int d, long long n_steps, const double *H);

/* b <- effective induction of Eq. Bi for every replica's state m:
 * b_i = sum_{j in z(i), j in disk} m_j + (a^2/lambda_ex^2)(h_ext + h^M_i).
 * b has the state layout; cells outside the disks are written as zero. */
int nd_effective_field(nd_handle *h, const void *m, void *b, void *stream);

/* Energy of Eq. Hmm for every replica, in units of J = 2AL, evaluated with a
 * double-precision field and double-precision sums whatever the handle's
 * precision: E_out[r] = -{ sum_pairs m_i . m_j + (a^2/lambda^2) sum_i
 * (h_ext + h^M_i / 2) . m_i }.  If dEdL_out is not NULL it receives, per
 * replica, the derivative of the energy in joules, E = J E_out, with respect
 * to the thickness L at fixed m (J/m): dE/dL = 2A E_out + J d(E/J)/dL, the
 * second term from the thickness derivative of the Sec. II.B tensor and of
 * the self factors (always the paper's closed forms).  At a constrained
 * minimum this is dU/dL by the envelope theorem, which gives dk_F/dL from
 * two relaxed states (Eq. Ux).  E_out and dEdL_out are host arrays [B]; the
 * call synchronises `stream`. */
int nd_energy(nd_handle *h, const void *m, double *E_out, double *dEdL_out, void *stream);

/* n_steps classical RK4 steps of dm/dtau = m x b - alpha m x (m x b)
 * (Sec. III.A) for every replica, with the full field at all four stages
 * and |m_i| = 1 restored after each step; dtau = gamma B0 dt_seconds.
 * m is updated in place.  With more replicas than resident CTAs the steps
 * are spread evenly over one CTA per SM, replicas changing CTA between steps
 * (a cooperative launch; see nd_check_status). */
int nd_step_rk4(nd_handle *h, void *m, long long n_steps, double dt_seconds, void *stream);

/* n_steps stochastic Heun steps of the Langevin equation (Eq. LV, Sec.
 * III.C): g = b dtau + sigma_s w, dm = m x [g - alpha m x g], Euler predictor
 * and trapezoid corrector with the same w, |m| = 1 restored after each
 * stage, sigma_s = sqrt(2 alpha T~ dtau), T~ = k_B T_kelvin[r] / J.
 * w_i are three standard normals per cell drawn from Philox4x32-10 with
 * key = seed[r] and counter = (cell index j*D+i, step, 0) where step runs from
 * step0 to step0 + n_steps - 1 (Box-Muller on the two word pairs), so a run
 * split into several calls is bit-identical to one call.  T_kelvin and seed
 * are host arrays [B]; T_kelvin[r] == 0 gives deterministic Heun. */
int nd_step_heun(nd_handle *h, void *m, long long n_steps, double dt_seconds, const double *T_kelvin,
                 const unsigned long long *seed, unsigned long long step0, void *stream);

/* Lagrange-constrained relaxation pinning each replica's vortex core at
 * X[r] (host array [B][2], metres) (Sec. IV local spin alignment with the
 * fictitious constraint fields of a Lagrange multiplier; the constraint form
 * is a reading, the paper defers its details to a cited reference):
 *   C_k(m) = sum_{i in W} (m_i^z)^2 (r_ik - X_k)/a = 0, k = x, y, with the
 *   window W = disk cells with |r_i - X| < 4 lambda_ex.
 * Each sweep evaluates b (Eq. Bi), adds 2 lambda_k m_i^z (r_ik - X_k)/a zhat in
 * W, stops if max_i |m_i x e_i|/|e_i| < tol, otherwise takes one Newton step
 * on the two multipliers for C(m') = 0 with the exact 2x2 Jacobian and sets
 * m_i <- normalise(m_i/2 + e_i/(2|e_i|)).  Multipliers start at zero.  m is
 * updated in place.  Outputs (host arrays, any may be NULL): U_out[B] the
 * double-precision energy of the relaxed state (units of J), lambda_out[B][2],
 * iters_out[B] sweeps applied.  Size classes held on chip (P <= 128 in
 * ND_FP32, P <= 64 in ND_FP64) relax in one launch; larger ones run the sweeps
 * as grid-wide passes and check every 32 sweeps (a host synchronisation)
 * whether all their replicas have converged.  Returns ND_ERR_NOT_CONVERGED if
 * a replica reached max_iter.  Synchronises `stream`. */
int nd_relax_constrained(nd_handle *h, void *m, const double *X, double tol, int max_iter, double *U_out,
                         double *lambda_out, int *iters_out, void *stream);

/* One sweep of the constrained relaxation of nd_relax_constrained (same
 * constraint, window, damping eta = 1/2 and Newton step) whose effective field
 * is taken from an energy gradient the caller supplies, instead of being
 * evaluated by the library: b_i = -(1/J) grad_i, grad = dE/dm in joules in the
 * state layout of the handle's precision (for instance the backward of an
 * autograd energy, which may add terms of its own to the energy of Eq. Hmm).
 * With grad = -J b this is exactly the library's own sweep.  Per replica:
 * the residual max |m x e|/|e| of the current state is written to resid_out
 * (host [B], may be NULL); if it is below tol the replica is left unchanged
 * (moved_out[r] = 0), otherwise one Newton step on the multipliers lambda
 * (host [B][2], in/out; start from zero) and the damped alignment update m in
 * place (moved_out[r] = 1; moved_out may be NULL).  X: host [B][2] core
 * positions in metres.  m and grad must be device buffers.  Synchronises
 * `stream`.  The paper has no counterpart (its relaxation is the alignment of
 * Sec. IV with the library's own field). */
int nd_relax_sweep_grad(nd_handle *h, void *m, const void *grad, const double *X, double *lambda, double tol,
                        double *resid_out, int *moved_out, void *stream);

/* Synchronise `stream` and read (then clear) the handle's device status
 * word.  Returns ND_ERR_TIMEOUT if a bounded device-side wait expired since
 * the last check (the time-sliced stepping schedule hands replicas between
 * CTAs through flags and gives up rather than hang), ND_ERR_NAN if a kernel
 * flagged non-finite values, else ND_OK.  The paper has no counterpart. */
int nd_check_status(nd_handle *h, void *stream);

/* Failure-path self-test of the time-sliced schedule: launches the stepping
 * kernel as one CTA with one segment that waits for a replica hand-over flag
 * that no segment ever sets.  The wait is bounded (about one second of
 * polling); when it expires the kernel sets ND_DEV_TIMEOUT in the handle's
 * status word and returns without reading or writing any state, so the
 * context stays usable and the next nd_check_status returns ND_ERR_TIMEOUT.
 * Synchronises `stream`.  Needs an ND_FP32 handle whose first size class is
 * held on chip (P <= 128), else ND_ERR_ARG.  The paper has no counterpart. */
int nd_selftest_handover_timeout(nd_handle *h, void *stream);

/* Analytic q = +1 vortex centred at X0[r] = (x0, y0) metres (host array
 * [B][2]) for every replica (Sec. IV profile): in-plane angle atan2(y - y0,
 * x - x0) + chirality pi/2, m_z = polarity exp(-rho^2/lambda_ex^2), |m| = 1. */
int nd_init_vortex(nd_handle *h, void *m, const double *X0, void *stream);

/* Vortex core position (Sec. IV) of every replica: the vorticity centre is
 * the plaquette with winding +1 (largest m_z^2 sum of its corners on ties);
 * Xc_out[r] = sum (m_z)^2 r_i / sum (m_z)^2 over disk cells within
 * 4 lambda_ex of it, in metres (host array [B][2]).  status[r] (host [B],
 * may be NULL) is 0 or ND_ERR_NO_VORTEX.  Returns ND_ERR_NO_VORTEX if any
 * replica has none.  Synchronises `stream`. */
int nd_vortex_core(nd_handle *h, const void *m, double *Xc_out, int *status, void *stream);

/* Device-resident statistics of the vortex core for the equilibrium checks
 * of Sec. V.C (radial Boltzmann law Eq. pr, <r^2> = 2kT/k_F, speed law f(V)).
 * nd_stats_reset allocates and zeroes, per replica, double-precision sums and
 * two uint64 histograms: r = |r_c| in r_bins bins over [0, r_max) metres and
 * V in v_bins bins over [0, v_max) m/s.  nd_stats_sample runs the core
 * estimator of nd_vortex_core on the device state m and accumulates, without
 * synchronising: samples with a vortex add to n, sum x, sum y, sum r^2 and the
 * r histogram; two consecutive such samples, dt_sample_seconds apart, add the
 * speed V = |r_c(t) - r_c(t - dt)|/dt to n_V, sum V^2 and the V histogram;
 * samples without one count as no_vortex and break the speed chain.
 * nd_stats_read synchronises `stream` and copies out moments ([B][7]: n,
 * sum x, sum y, sum r^2, n_V, sum V^2, no_vortex), r_hist ([B][r_bins]) and
 * v_hist ([B][v_bins]); any output may be NULL. */
int nd_stats_reset(nd_handle *h, double r_max, int r_bins, double v_max, int v_bins);
int nd_stats_sample(nd_handle *h, const void *m, double dt_sample_seconds, void *stream);
int nd_stats_read(nd_handle *h, double *moments, unsigned long long *r_hist, unsigned long long *v_hist,
                  void *stream);

/* Checkpoint of the statistics accumulators, so that a run split over
 * processes accumulates exactly as one uninterrupted run (the noise stream
 * resumes from the step counter, nd_step_heun's step0).  nd_stats_save_bytes
 * gives the size of the record; nd_stats_save synchronises `stream` and
 * writes, into the caller's host buffer of that size, the histogram ranges,
 * every replica's sums and the previous core position that continues its
 * speed chain, and both histograms.  nd_stats_load checks the record (a
 * leading tag, the replica count of the handle) and restores it, allocating
 * as nd_stats_reset does.  ND_ERR_ARG for a null buffer, a short buffer, a
 * record of another replica count, or (save) a handle without statistics. */
size_t nd_stats_save_bytes(const nd_handle *h);
int nd_stats_save(nd_handle *h, void *buf, size_t bytes, void *stream);
int nd_stats_load(nd_handle *h, const void *buf, size_t bytes, void *stream);

/* Average magnetisation <m> = (1/N) sum_i m_i over each disk (Sec. IV);
 * out is a host array [B][3].  Synchronises `stream`. */
int nd_mean_m(nd_handle *h, const void *m, double *out, void *stream);

/* ------------------------------------------------------------------------
 * Time series of the average magnetisation and their power spectra (Sec. V:
 * the thermal power spectra of <m_x> whose peaks give the gyrotropic
 * frequency and the higher modes).
 *
 * nd_series_reset allocates, for every replica, room for `capacity` samples
 * of <m> = (<m_x>, <m_y>, <m_z>) (double precision, averages over the disk
 * cells) and zeroes the device sample counter.  nd_series_sample appends one
 * sample of every replica at the counter's index and advances it (samples
 * past capacity are dropped; graph replays can append, see ND_GRAPH_SERIES).
 * nd_series_read synchronises the device and reports the number of samples
 * taken (n_samples, which may exceed capacity) and, if out is not NULL, copies
 * the kept ones, min(n_samples, capacity) per replica, to out
 * [B][kept][3].
 *
 * nd_power_spectrum splits each replica's kept series of one component
 * (0 = x, 1 = y, 2 = z) into n_windows = kept / window non-overlapping windows
 * (window 64, 128, 256, 512 or 1024 samples), removes each window's mean, and
 * returns the averaged one-sided periodogram
 *   psd_out[r][k] = (2 or 1) (dt_sample / window) < |sum_t x_t e^{-2 pi i k t/window}|^2 >_windows,
 * k = 0..window/2 (factor 2 except at k = 0 and window/2), in (units of
 * <m>)^2 per hertz, with freq_out[k] = k / (window dt_sample) hertz.  psd_out
 * is a host array [B][window/2+1], freq_out [window/2+1] (either may be NULL).
 * ND_ERR_ARG if fewer than `window` samples are kept.  Synchronises `stream`. */
int nd_series_reset(nd_handle *h, int capacity);
int nd_series_sample(nd_handle *h, const void *m, void *stream);
int nd_series_read(nd_handle *h, double *out, long long *n_samples);
int nd_power_spectrum(nd_handle *h, int component, int window, double dt_sample_seconds, double *psd_out,
                      double *freq_out, int *n_windows, void *stream);

/* ------------------------------------------------------------------------
 * Autotuning of the stepping schedule.  The replicas of a handle are grouped
 * by padded FFT size P ("size classes"); each class can step on the fused
 * on-chip kernel with one of up to three thread counts (which set how many
 * FFT groups share the row and column passes), on the global-memory path, or
 * (P <= 128) with each replica spread over a thread-block cluster of 8 CTAs
 * (or 16 for P >= 32; P = 192 and 256 on 16) whose shared memories hold the
 * replica's rows and exchange columns through distributed shared memory (for
 * classes with too few replicas to fill the GPU with one CTA each).
 * nd_autotune times every candidate that fits, on a scratch copy of an
 * analytic vortex state, for n_steps steps of the given method (and, for
 * Heun, 300 K; the fastest of three runs), and keeps the fastest per class
 * for later nd_step_* calls and graphs (the class's current plan unless
 * another is faster by more than 2%).  In a handle of several classes,
 * which step side by side, each candidate is timed on the whole handle with
 * the other classes at their current plans (one pass over the classes).  nd_plan_info reports, for class cls (0-based, in order of first
 * appearance), its P, replica count, the chosen plans (-1 default, 0..2 fused
 * variant, 100 global path, 200/201 cluster of 8/16 CTAs) and the threads per replica (fused:
 * threads per CTA; cluster: threads of the cluster; 0: global path).  Returns
 * ND_ERR_ARG for cls out of range.  The paper has no counterpart. */
int nd_autotune(nd_handle *h, int method, double dt_seconds, long long n_steps, void *stream);

/* Autotuning of handles that will step side by side (for instance the RK4
 * and Heun handles of one batch whose graphs nd_graph_join replays as one):
 * like nd_autotune, but every candidate of every class of every handle is
 * timed on all n handles stepping together, each on its own stream, with the
 * other classes at their current plans, so that the plans share the GPU well
 * rather than each being fastest alone.  methods[k] is handle k's method.
 * ND_ERR_ARG for no handles, a repeated handle or a bad method. */
int nd_autotune_group(nd_handle *const *handles, const int *methods, int n, double dt_seconds, long long n_steps,
                      void *stream);
/* Force the plan of class cls for a method (-1 default, 0..2 fused variant,
 * 100 global path, 200 cluster of 8 CTAs, 201 cluster of 16 CTAs); ND_ERR_ARG
 * if it does not exist or does not fit.  Plans 0..2 compute the same
 * arithmetic per element, so trajectories do not depend on which of them
 * runs; plan 100 does too except at P = 128, where the on-chip kernel
 * transforms each real row at half length and the global path transforms
 * pairs of rows; the cluster plans split the column products over the x and
 * y groups.  These agree to rounding (a few units in the last place of FP32
 * per step). */
int nd_set_plan(nd_handle *h, int cls, int method, int plan);
int nd_plan_info(const nd_handle *h, int cls, int *P, int *n_replicas, int *plan_rk4, int *plan_heun, int *threads_rk4,
                 int *threads_heun);

/* ------------------------------------------------------------------------
 * Graph-captured stepping.  nd_graph_create records, once, the whole launch
 * sequence of n_steps RK4 or Heun steps of every replica of the handle on
 * the device state m, followed by the samples that the flags in stats_sample
 * select (ND_GRAPH_STATS: one nd_stats_sample; ND_GRAPH_SERIES: one
 * nd_series_sample), as a CUDA graph; the noise-step counter lives on the
 * device and advances by n_steps
 * at the end of every replay, so consecutive nd_graph_launch calls continue
 * the Philox stream exactly as nd_step_heun with step0 advanced would (the
 * trajectories are bit-identical).  The graph keeps its own copy of the
 * per-replica parameters (dt, T, seeds, damping at creation time) and works
 * on the buffer m given at creation.  Uneven multi-disk handles become one
 * graph with a launch per FFT size class; the classes' launches are
 * independent branches of the graph (and, outside graphs, run on side streams
 * of the handle) so that they share the GPU, unless a class has more replicas
 * than the GPU has SMs.  The paper has no counterpart (it is the batching of
 * Sec. III's integrators).  nd_graph_nodes reports the number of kernel nodes
 * of one replay, counting those inside joined graphs.
 *
 * nd_graph_join makes one graph of n_parts graphs (for example the RK4 graph
 * of a handle of T = 0 replicas and the Heun graph of a handle of the others)
 * as independent branches: one nd_graph_launch replays all parts side by
 * side, each advancing its own step counter as its own launch would.  The
 * parts must outlive the joined graph (it uses their device buffers); destroy
 * it with nd_graph_destroy.  ND_ERR_ARG for no parts or a null part. */
typedef struct nd_graph nd_graph;
#define ND_GRAPH_STATS 1
#define ND_GRAPH_SERIES 2
int nd_graph_create(nd_handle *h, void *m, int method, long long n_steps, double dt_seconds, const double *T_kelvin,
                    const unsigned long long *seed, unsigned long long step0, int stats_sample, nd_graph **out);
int nd_graph_join(nd_graph *const *parts, int n_parts, nd_graph **out);
int nd_graph_launch(nd_graph *g, void *stream);
int nd_graph_nodes(const nd_graph *g, int *n_kernel_nodes);
void nd_graph_destroy(nd_graph *g);

/* ------------------------------------------------------------------------
 * Allocation-free Heun stepping.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code running
 * inside a framework that owns every device allocation through its own pool,
 * real-time loops that cannot afford an allocation's implicit synchronisation,
 * or plugins that may only touch the buffers their host gives them.  Such a
 * caller cannot create a handle, so the disk is described directly.
 *
 * The call performs the same n_steps stochastic Heun steps as nd_step_heun on
 * a handle holding n_replicas replicas of *disk in ND_FP32 (same state layout:
 * replica r at element offset r * 3 * D * Dpad), with the same noise stream.
 * Its working memory -- the stage accumulator, the spectral kernel, the mask
 * and its cell list, the twiddles and the parameter blocks -- lives in one
 * file-scope device
 * array of fixed size that every GPU loading the library holds until exit
 * (about 9 MiB); nothing is allocated.  Limits, rejected with ND_ERR_ARG and
 * a message: padded grid P <= 128 (disk diameter up to 64 cells, and the
 * on-chip kernel must fit, about 60 cells), n_replicas <= ND_NOALLOC_MAX_REPLICAS,
 * n_replicas * 3 * D * Dpad <= ND_NOALLOC_MAX_STATE_FLOATS, and m must be a
 * device pointer on the current device (a buffer of another GPU is rejected).
 *
 * The first call on a device resolves the array's address on that device and
 * loads the FFT constants.  The call cannot be stream-captured (its parameter
 * blocks go up from one static host array, which a replay would not refresh):
 * on a capturing stream it returns ND_ERR_ARG before issuing any work.
 * A call with a new geometry rebuilds the spectral kernel and synchronises
 * `stream`.  Every call shares the array and leaves its contents behind, so
 * calls whose work overlaps on the GPU (other streams, other threads) race.
 */
#define ND_NOALLOC_MAX_STATE_FLOATS (1 << 21)
#define ND_NOALLOC_MAX_REPLICAS 4096
int nd_step_heun_noalloc(const nd_disk_desc *disk, int n_replicas, float *m, long long n_steps, double dt_seconds,
                         const double *T_kelvin, const unsigned long long *seed, unsigned long long step0,
                         void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NANODISK_H */
