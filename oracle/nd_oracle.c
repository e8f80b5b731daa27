/*
 * nd_oracle.c -- plain FP64 CPU oracle for the thin-nanodisk micromagnetics
 * hot path of Wysin & Figueiredo, "Thermal vortex dynamics in thin circular
 * ferromagnetic nanodisks" (2012).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  It shares no code, header, table or
 * constant generator with the CUDA path.  Only the test-suite, the smoke
 * entry point and the CPU-baseline leg of the benchmark load it.
 *
 * Everything is double precision.  Where the method has a plain definition
 * (the demagnetisation field, the effective field, the energy) the oracle is
 * that definition written out, with an O(C^2) direct sum over cell pairs.
 * The time steppers, the noise generator, the vortex-core estimator and the
 * constrained relaxation follow the paper's steps in its order.
 *
 * Grid and layout: a D x D square grid of a x a x L cells; cell (i, j) has its
 * centre at ((i - (D-1)/2) a, (j - (D-1)/2) a); a cell belongs to the disk iff
 * its centre lies within radius R.  Arrays of vectors are stored as
 * [3][D][D] (component, row j = y index, column i = x index), x fastest.
 * Cells outside the disk hold zero.
 *
 * Every function that has no closed-form or brute-force pin in the tests says
 * "parity unpinned" in its comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NDO_MU0 (4.0e-7 * M_PI)          /* vacuum permeability, SI */
#define NDO_KB 1.380649e-23              /* Boltzmann constant, J/K */

typedef struct {
    double R, L, a;        /* disk radius, thickness, cell edge (m) */
    double Ms, A, gamma;   /* saturation magnetisation (A/m), exchange stiffness (J/m), gyromagnetic ratio (1/(T s)) */
    double alpha;          /* damping */
    double hext[3];        /* external field H_ext (A/m) */
    int polarity, chirality;
} ndo_disk;

typedef struct {
    int D;                 /* grid side */
    int C;                 /* number of cells in the disk */
    double a, L, R;
    double lambda_ex;      /* exchange length (m) */
    double c;              /* a^2 / lambda_ex^2 */
    double B0, t0, J;      /* induction unit (T), time unit (s), energy unit (J) */
    double Nx, Nz;         /* cell self-demagnetisation factors */
    double h[3];           /* scaled external field H_ext / Ms */
    double alpha;
    int polarity, chirality;
    unsigned char *mask;   /* [D][D] */
    double *Gt;            /* a^2 G at displacement (dx, dy) cells: [4][2D-1][2D-1], comps xx, yy, xy, zz */
    double *sched;         /* optional per-step external field H_ext(s)/Ms, [nsched][3] */
    long nsched;
} ndo_model;

/* ------------------------------------------------------------------ units */

/* Units of Section III.A: J = 2AL (energy unit), lambda_ex = sqrt(2A/(mu0 Ms^2)),
 * B0 = 2A/(a^2 Ms), t0 = 1/(gamma B0). */
void ndo_units(double A, double Ms, double a, double L, double gamma,
               double *lambda_ex, double *B0, double *t0, double *J, double *c)
{
    double lam = sqrt(2.0 * A / (NDO_MU0 * Ms * Ms));
    double b0 = 2.0 * A / (a * a * Ms);
    if (lambda_ex) *lambda_ex = lam;
    if (B0) *B0 = b0;
    if (t0) *t0 = 1.0 / (gamma * b0);
    if (J) *J = 2.0 * A * L;
    if (c) *c = (a * a) / (lam * lam);
}

/* Scaled temperature T~ = kT / J with J = 2AL (Section III.B). */
double ndo_scaled_temperature(double T, double A, double L) { return NDO_KB * T / (2.0 * A * L); }

/* Noise amplitude sigma_s = sqrt(2 alpha T~ dtau) (Section III.C, from the FD theorem). */
double ndo_sigma_s(double alpha, double Ts, double dtau) { return sqrt(2.0 * alpha * Ts * dtau); }

/* Gyrovector G = 2 pi Q L Ms / gamma (Section IV). */
double ndo_gyrovector(double L, double Ms, double gamma, int Q) { return 2.0 * M_PI * Q * L * Ms / gamma; }

/* Dimensionless gyrotropic angular frequency Omega_G = -kF a^2 / (4 pi L A Q) (Eq. OG). */
double ndo_omega_G(double kF, double a, double L, double A, int Q) { return -kF * a * a / (4.0 * M_PI * L * A * Q); }

/* Force constant from two static energies: U(x) = U(0) + kF x^2 / 2 (Eq. Ux). */
double ndo_kF_from_energies(double U0, double Ux, double x) { return 2.0 * (Ux - U0) / (x * x); }

/* Radial Boltzmann density p(r) = beta kF r exp(-beta kF r^2 / 2) (Eq. pr). */
double ndo_p_r(double r, double kF, double kT) { double b = 1.0 / kT; return b * kF * r * exp(-0.5 * b * kF * r * r); }

/* Gyrotropic effective mass m_G = G^2 / k_F (Sec. VI), G the gyrovector (kg/s)
 * and k_F the force constant (N/m); kilograms. */
double ndo_gyro_mass(double G, double kF) { return G * G / kF; }

/* Boltzmann density of the vortex rotational speed (Sec. VI):
 *   f(V) = beta m_G V exp(-beta m_G V^2 / 2),  beta = 1/kT,
 * the image of p(r) under V = |omega_G| r. */
double ndo_f_V(double V, double mG, double kT)
{
    double b = 1.0 / kT;
    return b * mG * V * exp(-0.5 * b * mG * V * V);
}

/* Angular frequency of gyrotropic motion from a sampled core track (the
 * dynamic side of Eq. OG): the polar angle theta_k = atan2(y_k, x_k) of each
 * sample, made continuous by adding the multiple of 2 pi that keeps every step
 * theta_k - theta_{k-1} within (-pi, pi], then the least-squares slope of
 * theta against tau_k = k dtau.  Returns the slope (radians per time unit;
 * negative for clockwise motion). */
double ndo_omega_from_track(const double *xc, const double *yc, int n, double dtau)
{
    if (n < 2) return 0.0;
    double *th = (double *)malloc(sizeof(double) * n);
    th[0] = atan2(yc[0], xc[0]);
    for (int k = 1; k < n; ++k) {
        double a = atan2(yc[k], xc[k]), d = a - th[k - 1];
        d -= 2.0 * M_PI * floor((d + M_PI) / (2.0 * M_PI));   /* into [-pi, pi) */
        th[k] = th[k - 1] + d;
    }
    double st = 0.0, sth = 0.0;
    for (int k = 0; k < n; ++k) { st += k * dtau; sth += th[k]; }
    double tm = st / n, thm = sth / n, num = 0.0, den = 0.0;
    for (int k = 0; k < n; ++k) {
        double dt_ = k * dtau - tm;
        num += dt_ * (th[k] - thm);
        den += dt_ * dt_;
    }
    free(th);
    return num / den;
}

/* Averaged one-sided power spectrum of a sampled series (Sec. V, the thermal
 * power spectra of <m_x>): the series x[0..n) is cut into n_w = n / W
 * consecutive windows of W samples; each window's mean is removed; its DFT
 * X_k = sum_t x_t exp(-2 pi i k t / W) is summed directly; and
 *   psd[k] = c_k (dt / W) < |X_k|^2 >_windows,  k = 0..W/2,
 * with c_k = 2 except c_0 = c_{W/2} = 1.  Returns n_w (0 if n < W, psd
 * untouched). */
int ndo_power_spectrum(const double *x, long n, int W, double dt, double *psd)
{
    int nw = (int)(n / W);
    if (nw < 1 || W < 2) return 0;
    for (int k = 0; k <= W / 2; ++k) psd[k] = 0.0;
    for (int w = 0; w < nw; ++w) {
        const double *xs = x + (size_t)w * W;
        double mean = 0.0;
        for (int t = 0; t < W; ++t) mean += xs[t];
        mean /= W;
        for (int k = 0; k <= W / 2; ++k) {
            double re = 0.0, im = 0.0;
            for (int t = 0; t < W; ++t) {
                double ang = -2.0 * M_PI * (double)(((long)k * t) % W) / W;
                re += (xs[t] - mean) * cos(ang);
                im += (xs[t] - mean) * sin(ang);
            }
            psd[k] += re * re + im * im;
        }
    }
    for (int k = 0; k <= W / 2; ++k) {
        double c = (k == 0 || 2 * k == W) ? 1.0 : 2.0;
        psd[k] *= c * dt / W / nw;
    }
    return nw;
}

/* ------------------------------------------------------------- geometry */

int ndo_grid_side(double R, double a) { return (int)floor(2.0 * R / a + 0.5); }

/* Disk mask: cell centre inside radius R (cell-centre reading of the disk). */
int ndo_mask(double R, double a, int D, unsigned char *mask)
{
    int C = 0;
    double rr = (R / a) * (R / a);
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) {
            double x = i - 0.5 * (D - 1), y = j - 0.5 * (D - 1);
            int in = (x * x + y * y) <= rr;
            mask[j * D + i] = (unsigned char)in;
            C += in;
        }
    return C;
}

/* ------------------------------------------------------ Green's tensor */

/* Thin-film Green's tensor at in-plane displacement (x, y) != 0, thickness L
 * (Section II.B): returns G_xx, G_yy, G_xy, G_zz in 1/m^2.
 *   G_zz = (1/(2 pi L)) (1/sqrt(r^2+L^2) - 1/r), written as -L/(2 pi r s (s+r))
 *   G_xx = L/(2 pi r^4) (x^2/s - y^2/(s+r))
 *   G_xy = L/(2 pi r^4) (2s+r)/(s+r) x y / s,      s = sqrt(r^2 + L^2)
 *   G_yy = G_xx with x and y swapped. */
void ndo_green(double x, double y, double L, double g[4])
{
    double r2 = x * x + y * y, r = sqrt(r2), s = sqrt(r2 + L * L);
    double pre = L / (2.0 * M_PI * r2 * r2);
    g[0] = pre * (x * x / s - y * y / (s + r));
    g[1] = pre * (y * y / s - x * x / (s + r));
    g[2] = pre * ((2.0 * s + r) / (s + r)) * (x * y / s);
    g[3] = -L / (2.0 * M_PI * r * s * (s + r));
}

/* Cell self-demagnetisation factors of a cylinder of radius r_o = a/sqrt(pi)
 * and length L (Section II.B): N_z = (L + r_o - sqrt(L^2+r_o^2))/L and
 * N_x = N_y = (sqrt(L^2+r_o^2) - r_o)/(2L); G_zz(0) = -N_z, G_xx(0) = G_yy(0) = -N_x,
 * G_xy(0) = 0.  The sign of N_x is the reading that makes N_x+N_y+N_z = 1. */
void ndo_self_factors(double L, double a, double *Nx, double *Nz)
{
    double ro = a / sqrt(M_PI), q = sqrt(L * L + ro * ro);
    *Nz = (L + ro - q) / L;
    *Nx = (q - ro) / (2.0 * L);
}

/* ----------------------------------------------------------------- model */

int ndo_model_init(const ndo_disk *d, ndo_model *m)
{
    memset(m, 0, sizeof(*m));
    m->D = ndo_grid_side(d->R, d->a);
    if (m->D < 1) return -1;
    m->a = d->a; m->L = d->L; m->R = d->R;
    m->alpha = d->alpha; m->polarity = d->polarity; m->chirality = d->chirality;
    ndo_units(d->A, d->Ms, d->a, d->L, d->gamma, &m->lambda_ex, &m->B0, &m->t0, &m->J, &m->c);
    ndo_self_factors(d->L, d->a, &m->Nx, &m->Nz);
    for (int k = 0; k < 3; ++k) m->h[k] = d->hext[k] / d->Ms;
    int D = m->D, W = 2 * D - 1;
    m->mask = (unsigned char *)malloc((size_t)D * D);
    m->Gt = (double *)malloc(sizeof(double) * 4 * (size_t)W * W);
    if (!m->mask || !m->Gt) return -2;
    m->C = ndo_mask(d->R, d->a, D, m->mask);
    /* a^2 G(r) sampled at cell-centre displacements; self terms at the origin. */
    for (int dy = -(D - 1); dy <= D - 1; ++dy)
        for (int dx = -(D - 1); dx <= D - 1; ++dx) {
            double g[4];
            if (dx == 0 && dy == 0) {
                g[0] = -m->Nx; g[1] = -m->Nx; g[2] = 0.0; g[3] = -m->Nz;
            } else {
                ndo_green(dx * d->a, dy * d->a, d->L, g);
                for (int k = 0; k < 4; ++k) g[k] *= d->a * d->a;
            }
            size_t o = (size_t)(dy + D - 1) * W + (dx + D - 1);
            for (int k = 0; k < 4; ++k) m->Gt[(size_t)k * W * W + o] = g[k];
        }
    return 0;
}

/* Replace the model's table by a user table Gq of a^2 G at displacements
 * (dx, dy) >= 0 cells, laid out [4][D][D] (index [k][dy][dx], components xx,
 * yy, xy, zz, the self terms at dx = dy = 0), extended to negative
 * displacements by the symmetry of the Sec. II.B tensor: xx, yy and zz even
 * in dx and in dy, xy odd in each. */
void ndo_model_set_green(ndo_model *m, const double *Gq)
{
    const int D = m->D, W = 2 * D - 1;
    for (int dy = -(D - 1); dy <= D - 1; ++dy)
        for (int dx = -(D - 1); dx <= D - 1; ++dx) {
            int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
            /* sign(dx) sign(dy): an odd function of dx vanishes at dx = 0 */
            double sgn = (dx > 0) - (dx < 0);
            sgn *= (dy > 0) - (dy < 0);
            size_t q = (size_t)ay * D + ax, o = (size_t)(dy + D - 1) * W + (dx + D - 1);
            for (int k = 0; k < 4; ++k) {
                double v = Gq[(size_t)k * D * D + q];
                m->Gt[(size_t)k * W * W + o] = (k == 2) ? sgn * v : v;
            }
        }
}

void ndo_model_free(ndo_model *m)
{
    free(m->mask); free(m->Gt); free(m->sched);
    m->mask = NULL; m->Gt = NULL; m->sched = NULL; m->nsched = 0;
}

/* Replace the disk mask by any set of cells of the D x D grid (a variant of
 * the geometry of Sec. II.A: a non-circular element); mask is [D][D], nonzero
 * inside.  The Green's table does not depend on the mask.  Returns the new
 * number of cells. */
int ndo_model_set_mask(ndo_model *m, const unsigned char *mask)
{
    const int N = m->D * m->D;
    int C = 0;
    for (int t = 0; t < N; ++t) { m->mask[t] = mask[t] ? 1 : 0; C += m->mask[t]; }
    m->C = C;
    return C;
}

/* A time-dependent external field (Sec. II.A's H_ext, switched per time step:
 * a pulse or any other schedule): step s of a trajectory (the steppers'
 * global step index) uses H_ext = hs[s] (A/m, [n][3]) for all of its stages
 * while s < n, and the static field of the disk afterwards.  n = 0 clears. */
int ndo_model_set_schedule(ndo_model *m, long n, const double *hs, double Ms)
{
    free(m->sched);
    m->sched = NULL;
    m->nsched = 0;
    if (n <= 0) return 0;
    m->sched = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!m->sched) return -1;
    for (long i = 0; i < 3 * n; ++i) m->sched[i] = hs[i] / Ms;
    m->nsched = n;
    return 0;
}

/* The scaled external field H_ext/Ms of step s. */
static const double *step_field(const ndo_model *m, uint64_t s)
{
    return (m->sched && s < (uint64_t)m->nsched) ? m->sched + 3 * s : m->h;
}

int ndo_model_D(const ndo_model *m) { return m->D; }
int ndo_model_C(const ndo_model *m) { return m->C; }
size_t ndo_model_size(void) { return sizeof(ndo_model); }
void ndo_model_params(const ndo_model *m, double out[8])
{
    out[0] = m->lambda_ex; out[1] = m->c; out[2] = m->B0; out[3] = m->t0;
    out[4] = m->J; out[5] = m->Nx; out[6] = m->Nz; out[7] = (double)m->C;
}
void ndo_model_mask(const ndo_model *m, unsigned char *out) { memcpy(out, m->mask, (size_t)m->D * m->D); }
void ndo_model_set_alpha(ndo_model *m, double alpha) { m->alpha = alpha; }

/* ------------------------------------------------------ fields, energy */

/* Demagnetisation field by direct summation over all source cells in the disk:
 *   h^M_i = sum_{j in disk} a^2 G(r_i - r_j) m_j,
 * with the self term diag(-N_x, -N_x, -N_z) at j = i (Section II.B).  Output is
 * zero outside the disk. */
void ndo_demag(const ndo_model *m, const double *mv, double *hM)
{
    const int D = m->D, W = 2 * D - 1, N = D * D;
    const double *Gxx = m->Gt, *Gyy = m->Gt + (size_t)W * W, *Gxy = m->Gt + 2 * (size_t)W * W,
                 *Gzz = m->Gt + 3 * (size_t)W * W;
    const double *mx = mv, *my = mv + N, *mz = mv + 2 * N;
#pragma omp parallel for schedule(dynamic, 4) if (N > 256)
    for (int t = 0; t < N; ++t) {
        int it = t % D, jt = t / D;
        double hx = 0, hy = 0, hz = 0;
        if (m->mask[t]) {
            for (int s = 0; s < N; ++s) {
                if (!m->mask[s]) continue;
                int is = s % D, js = s / D;
                size_t o = (size_t)(jt - js + D - 1) * W + (it - is + D - 1);
                hx += Gxx[o] * mx[s] + Gxy[o] * my[s];
                hy += Gxy[o] * mx[s] + Gyy[o] * my[s];
                hz += Gzz[o] * mz[s];
            }
        }
        hM[t] = hx; hM[N + t] = hy; hM[2 * N + t] = hz;
    }
}

/* Sum of nearest-neighbour unit vectors inside the disk (free boundary). */
static void exchange_sum(const ndo_model *m, const double *mv, int t, double out[3])
{
    const int D = m->D, N = D * D;
    int i = t % D, j = t / D;
    out[0] = out[1] = out[2] = 0.0;
    int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
    for (int q = 0; q < 4; ++q) {
        int ii = nb[q][0], jj = nb[q][1];
        if (ii < 0 || jj < 0 || ii >= D || jj >= D) continue;
        int s = jj * D + ii;
        if (!m->mask[s]) continue;
        for (int k = 0; k < 3; ++k) out[k] += mv[k * N + s];
    }
}

/* Dimensionless effective induction (Eq. Bi) with the scaled external field hx:
 *   b_i = sum_{j in z(i)} m_j + (a^2/lambda_ex^2) (h_ext + h^M_i). */
static void field_h(const ndo_model *m, const double *mv, double *b, const double hx[3])
{
    const int N = m->D * m->D;
    ndo_demag(m, mv, b);
    for (int t = 0; t < N; ++t) {
        if (!m->mask[t]) { b[t] = b[N + t] = b[2 * N + t] = 0.0; continue; }
        double ex[3];
        exchange_sum(m, mv, t, ex);
        for (int k = 0; k < 3; ++k) b[k * N + t] = ex[k] + m->c * (hx[k] + b[k * N + t]);
    }
}

/* Eq. Bi with the disk's static external field. */
void ndo_field(const ndo_model *m, const double *mv, double *b) { field_h(m, mv, b, m->h); }

/* Effective induction at selected cells only (flat indices j*D+i), by the
 * same direct sum: for sampled checks of large grids.  out is [n][3]. */
void ndo_field_at(const ndo_model *m, const double *mv, const int *cells, int n, double *out)
{
    const int D = m->D, W = 2 * D - 1, N = D * D;
    const double *Gxx = m->Gt, *Gyy = m->Gt + (size_t)W * W, *Gxy = m->Gt + 2 * (size_t)W * W,
                 *Gzz = m->Gt + 3 * (size_t)W * W;
#pragma omp parallel for schedule(dynamic, 1) if (n > 1)
    for (int q = 0; q < n; ++q) {
        int t = cells[q], it = t % D, jt = t / D;
        double h[3] = {0, 0, 0}, ex[3];
        if (!m->mask[t]) { out[3 * q] = out[3 * q + 1] = out[3 * q + 2] = 0.0; continue; }
        for (int s = 0; s < N; ++s) {
            if (!m->mask[s]) continue;
            int is = s % D, js = s / D;
            size_t o = (size_t)(jt - js + D - 1) * W + (it - is + D - 1);
            h[0] += Gxx[o] * mv[s] + Gxy[o] * mv[N + s];
            h[1] += Gxy[o] * mv[s] + Gyy[o] * mv[N + s];
            h[2] += Gzz[o] * mv[2 * N + s];
        }
        exchange_sum(m, mv, t, ex);
        for (int k = 0; k < 3; ++k) out[3 * q + k] = ex[k] + m->c * (m->h[k] + h[k]);
    }
}

/* Same as ndo_field but with the demagnetisation part only (no exchange, no
 * external field, no a^2/lambda^2 factor): the plain h^M of the direct sum. */
void ndo_field_parts(const ndo_model *m, const double *mv, double *ex, double *hM)
{
    const int N = m->D * m->D;
    ndo_demag(m, mv, hM);
    for (int t = 0; t < N; ++t) {
        double e[3] = {0, 0, 0};
        if (m->mask[t]) exchange_sum(m, mv, t, e);
        for (int k = 0; k < 3; ++k) ex[k * N + t] = e[k];
    }
}

/* Total energy in units of J (Eq. Hmm):
 *   H/J = -{ sum_{(i,j)} m_i . m_j + (a^2/lambda^2) sum_i (h_ext + h^M_i / 2) . m_i },
 * the pair sum running once over each nearest-neighbour pair in the disk. */
double ndo_energy(const ndo_model *m, const double *mv)
{
    const int D = m->D, N = D * D;
    double *hM = (double *)malloc(sizeof(double) * 3 * N);
    ndo_demag(m, mv, hM);
    double pairs = 0.0, zee = 0.0;
    for (int t = 0; t < N; ++t) {
        if (!m->mask[t]) continue;
        int i = t % D, j = t / D;
        if (i + 1 < D && m->mask[t + 1])
            for (int k = 0; k < 3; ++k) pairs += mv[k * N + t] * mv[k * N + t + 1];
        if (j + 1 < D && m->mask[t + D])
            for (int k = 0; k < 3; ++k) pairs += mv[k * N + t] * mv[k * N + t + D];
        for (int k = 0; k < 3; ++k) zee += (m->h[k] + 0.5 * hM[k * N + t]) * mv[k * N + t];
    }
    free(hM);
    return -(pairs + m->c * zee);
}

/* Number of nearest-neighbour pairs inside the disk. */
long ndo_pair_count(const ndo_model *m)
{
    const int D = m->D;
    long n = 0;
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) {
            int t = j * D + i;
            if (!m->mask[t]) continue;
            if (i + 1 < D && m->mask[t + 1]) ++n;
            if (j + 1 < D && m->mask[t + D]) ++n;
        }
    return n;
}

/* ------------------------------------------------------- LLG dynamics */

static inline void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Landau-Lifshitz right-hand side with damping (Section III.A):
 *   dm/dtau = m x b - alpha m x (m x b). */
void ndo_llg_rhs(const ndo_model *m, const double *mv, const double *b, double alpha, double *f)
{
    const int N = m->D * m->D;
    for (int t = 0; t < N; ++t) {
        double mm[3] = {mv[t], mv[N + t], mv[2 * N + t]}, bb[3] = {b[t], b[N + t], b[2 * N + t]};
        double p[3], q[3];
        cross(mm, bb, p);
        cross(mm, p, q);
        for (int k = 0; k < 3; ++k) f[k * N + t] = m->mask[t] ? p[k] - alpha * q[k] : 0.0;
    }
}

static void normalize_all(const ndo_model *m, double *mv)
{
    const int N = m->D * m->D;
    for (int t = 0; t < N; ++t) {
        if (!m->mask[t]) { mv[t] = mv[N + t] = mv[2 * N + t] = 0.0; continue; }
        double n = sqrt(mv[t] * mv[t] + mv[N + t] * mv[N + t] + mv[2 * N + t] * mv[2 * N + t]);
        for (int k = 0; k < 3; ++k) mv[k * N + t] /= n;
    }
}

/* Classical fourth-order Runge-Kutta for the LLG equation with the full field
 * evaluated at all four stages (Section III.A); |m_i| = 1 restored after each
 * full step (the paper is silent on renormalisation; this is the reading the
 * CUDA path follows too).  dtau is the dimensionless step gamma B0 dt; the
 * steps are numbered from step0 (the index selects a scheduled field). */
void ndo_rk4_at(const ndo_model *m, double *mv, long nsteps, double dtau, uint64_t step0)
{
    const int N3 = 3 * m->D * m->D;
    double *b = malloc(sizeof(double) * N3), *k = malloc(sizeof(double) * N3),
           *acc = malloc(sizeof(double) * N3), *ys = malloc(sizeof(double) * N3);
    static const double wstage[3] = {0.5, 0.5, 1.0};
    for (long n = 0; n < nsteps; ++n) {
        const double *hx = step_field(m, step0 + (uint64_t)n);   /* one external field per step */
        memcpy(ys, mv, sizeof(double) * N3);
        for (int s = 0; s < 4; ++s) {
            field_h(m, ys, b, hx);
            ndo_llg_rhs(m, ys, b, m->alpha, k);
            for (int t = 0; t < N3; ++t) {
                acc[t] = (s == 0) ? k[t] : acc[t] + ((s == 3) ? 1.0 : 2.0) * k[t];
                if (s < 3) ys[t] = mv[t] + wstage[s] * dtau * k[t];
            }
        }
        for (int t = 0; t < N3; ++t) mv[t] += dtau / 6.0 * acc[t];
        normalize_all(m, mv);
    }
    free(b); free(k); free(acc); free(ys);
}

/* RK4 steps numbered from 0 (the step index selects a scheduled field). */
void ndo_rk4(const ndo_model *m, double *mv, long nsteps, double dtau) { ndo_rk4_at(m, mv, nsteps, dtau, 0); }

/* ---------------------------------------------------- noise generator */

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
 * ten rounds of two 32x32->64 multiplies with multipliers 0xD2511F53 and
 * 0xCD9E8D57, the key bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85
 * between rounds.  Written from the published round definition. */
void ndo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0, p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Three standard normals for one cell and one time step.  The stream is
 * Philox4x32-10 with key = (seed low word, seed high word) and counter =
 * (cell index j*D+i, step low word, step high word, 0); the four 32-bit words
 * r0..r3 feed two Box-Muller pairs:
 *   u = (r + 1) 2^-32 in (0, 1],  v = r 2^-32 in [0, 1),
 *   w_x = sqrt(-2 ln u0) cos(2 pi v1),  w_y = sqrt(-2 ln u0) sin(2 pi v1),
 *   w_z = sqrt(-2 ln u2) cos(2 pi v3).
 * The paper uses a different (sequential) generator and does not name a
 * Gaussian transform; this is the reading both implementations follow. */
void ndo_thermal_normals(uint64_t seed, uint32_t cell, uint64_t step, double w[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {cell, (uint32_t)step, (uint32_t)(step >> 32), 0u}, r[4];
    ndo_philox4x32_10(ctr, key, r);
    const double s32 = 2.3283064365386963e-10; /* 2^-32 */
    double u0 = ((double)r[0] + 1.0) * s32, v1 = (double)r[1] * s32;
    double u2 = ((double)r[2] + 1.0) * s32, v3 = (double)r[3] * s32;
    double ra = sqrt(-2.0 * log(u0)), rb = sqrt(-2.0 * log(u2));
    w[0] = ra * cos(2.0 * M_PI * v1);
    w[1] = ra * sin(2.0 * M_PI * v1);
    w[2] = rb * cos(2.0 * M_PI * v3);
}

/* Fill an array with n normals of cell 0.., for moment tests. */
void ndo_normals_block(uint64_t seed, uint64_t step, uint32_t ncell, double *out)
{
    for (uint32_t c = 0; c < ncell; ++c) ndo_thermal_normals(seed, c, step, out + 3 * (size_t)c);
}

/* Change of one cell in one Heun stage (Section III.C):
 *   g = b dtau + sigma_s w,   dm = m x [g - alpha (m x g)]. */
static inline void heun_dm(const double mm[3], const double bb[3], const double w[3],
                           double dtau, double sig, double alpha, double dm[3])
{
    double g[3], p[3], q[3];
    for (int k = 0; k < 3; ++k) g[k] = bb[k] * dtau + sig * w[k];
    cross(mm, g, p);
    for (int k = 0; k < 3; ++k) q[k] = g[k] - alpha * p[k];
    cross(mm, q, dm);
}

/* Stochastic Heun (H2) integration of the Langevin equation (Eq. LV) with
 * thermal noise of variance sigma_s^2 per component and step (Section III.C):
 * Euler predictor y~ = y + dm(y), corrector y' = y + (dm(y) + dm(y~))/2 with
 * the same random vector w_n in both stages; |m| = 1 restored after the
 * predictor and after the corrector.  Ts is kT/J; step0 is the global index of
 * the first step (the noise counter, which also selects a scheduled external
 * field). */
void ndo_heun(const ndo_model *m, double *mv, long nsteps, double dtau, double Ts,
              uint64_t seed, uint64_t step0)
{
    const int D = m->D, N = D * D;
    const double sig = ndo_sigma_s(m->alpha, Ts, dtau);
    double *b = malloc(sizeof(double) * 3 * N), *dm1 = malloc(sizeof(double) * 3 * N),
           *yp = malloc(sizeof(double) * 3 * N), *W = malloc(sizeof(double) * 3 * N);
    for (long n = 0; n < nsteps; ++n) {
        uint64_t step = step0 + (uint64_t)n;
        const double *hx = step_field(m, step);   /* one external field per step */
        for (int t = 0; t < N; ++t) {
            double w[3] = {0, 0, 0};
            if (sig > 0.0) ndo_thermal_normals(seed, (uint32_t)t, step, w);
            for (int k = 0; k < 3; ++k) W[k * N + t] = w[k];
        }
        field_h(m, mv, b, hx);
        for (int t = 0; t < N; ++t) {
            double mm[3] = {mv[t], mv[N + t], mv[2 * N + t]}, bb[3] = {b[t], b[N + t], b[2 * N + t]};
            double w[3] = {W[t], W[N + t], W[2 * N + t]}, d[3];
            heun_dm(mm, bb, w, dtau, sig, m->alpha, d);
            for (int k = 0; k < 3; ++k) { dm1[k * N + t] = d[k]; yp[k * N + t] = mm[k] + d[k]; }
        }
        normalize_all(m, yp);
        field_h(m, yp, b, hx);
        for (int t = 0; t < N; ++t) {
            double mm[3] = {yp[t], yp[N + t], yp[2 * N + t]}, bb[3] = {b[t], b[N + t], b[2 * N + t]};
            double w[3] = {W[t], W[N + t], W[2 * N + t]}, d[3];
            heun_dm(mm, bb, w, dtau, sig, m->alpha, d);
            for (int k = 0; k < 3; ++k) mv[k * N + t] += 0.5 * (dm1[k * N + t] + d[k]);
        }
        normalize_all(m, mv);
    }
    free(b); free(dm1); free(yp); free(W);
}

/* ------------------------------------------------------ vortex profile */

/* Planar vortex of vorticity q = +1 centred at (x0, y0) (Section IV), with
 * in-plane angle phi = atan2(y - y0, x - x0) + chirality pi/2 and a seeded core
 * m_z = polarity exp(-rho^2/lambda_ex^2), in-plane part scaled so |m| = 1.
 * (The printed tan^-1((x-x0)/(y-y0)) winds the other way; this reading gives
 * the q = +1 vortex the text describes.) */
void ndo_init_vortex(const ndo_model *m, double x0, double y0, double *mv)
{
    const int D = m->D, N = D * D;
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) {
            int t = j * D + i;
            if (!m->mask[t]) { mv[t] = mv[N + t] = mv[2 * N + t] = 0.0; continue; }
            double x = (i - 0.5 * (D - 1)) * m->a, y = (j - 0.5 * (D - 1)) * m->a;
            double rho2 = (x - x0) * (x - x0) + (y - y0) * (y - y0);
            double mz = m->polarity * exp(-rho2 / (m->lambda_ex * m->lambda_ex));
            double phi = atan2(y - y0, x - x0) + m->chirality * 0.5 * M_PI;
            double sp = sqrt(1.0 - mz * mz);
            mv[t] = sp * cos(phi); mv[N + t] = sp * sin(phi); mv[2 * N + t] = mz;
        }
}

/* ------------------------------------------------------ vortex core */

/* Winding number of the in-plane angle around plaquette (i, j)-(i+1, j+1),
 * corners taken counter-clockwise; each angle step is the signed angle between
 * consecutive in-plane vectors, atan2(cross, dot), in (-pi, pi]. */
static int plaquette_winding(const ndo_model *m, const double *mv, int i, int j)
{
    const int D = m->D, N = D * D;
    int c[4] = {j * D + i, j * D + i + 1, (j + 1) * D + i + 1, (j + 1) * D + i};
    double s = 0.0;
    for (int q = 0; q < 4; ++q) {
        int p0 = c[q], p1 = c[(q + 1) & 3];
        double ax = mv[p0], ay = mv[N + p0], bx = mv[p1], by = mv[N + p1];
        s += atan2(ax * by - ay * bx, ax * bx + ay * by);
    }
    return (int)lround(s / (2.0 * M_PI));
}

/* Vortex core position (Section IV): the vorticity centre r_v is the centre of
 * the plaquette with winding +1 (if several, the one whose four corners carry
 * the largest sum of m_z^2; ties keep the first in row-major order); then
 *   r_c = sum (m_z^2 r_i) / sum m_z^2  over disk cells with |r_i - r_v| < 4 lambda_ex.
 * Returns 0 and r_c in metres, or 1 when no plaquette has winding +1. */
int ndo_vortex_core(const ndo_model *m, const double *mv, double Xc[2], double rv[2])
{
    const int D = m->D, N = D * D;
    int best = -1;
    double bestw = -1.0;
    for (int j = 0; j + 1 < D; ++j)
        for (int i = 0; i + 1 < D; ++i) {
            int t = j * D + i;
            if (!(m->mask[t] && m->mask[t + 1] && m->mask[t + D] && m->mask[t + D + 1])) continue;
            if (plaquette_winding(m, mv, i, j) != 1) continue;
            const double *mz = mv + 2 * N;
            double w = mz[t] * mz[t];
            w = w + mz[t + 1] * mz[t + 1];
            w = w + mz[t + D] * mz[t + D];
            w = w + mz[t + D + 1] * mz[t + D + 1];
            if (w > bestw) { bestw = w; best = t; }
        }
    if (best < 0) return 1;
    int bi = best % D, bj = best / D;
    /* plaquette centre in cell units relative to the grid centre */
    double cx = bi + 0.5 - 0.5 * (D - 1), cy = bj + 0.5 - 0.5 * (D - 1);
    double rcut = 4.0 * m->lambda_ex / m->a, rc2 = rcut * rcut;
    double sw = 0.0, sx = 0.0, sy = 0.0;
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) {
            int t = j * D + i;
            if (!m->mask[t]) continue;
            double x = i - 0.5 * (D - 1), y = j - 0.5 * (D - 1);
            double dx = x - cx, dy = y - cy;
            if (dx * dx + dy * dy >= rc2) continue;
            double w = mv[2 * N + t] * mv[2 * N + t];
            sw += w; sx += w * x; sy += w * y;
        }
    if (rv) { rv[0] = cx * m->a; rv[1] = cy * m->a; }
    if (sw <= 0.0) return 1;
    Xc[0] = sx / sw * m->a;
    Xc[1] = sy / sw * m->a;
    return 0;
}

/* Average magnetisation <m> = (1/N) sum_i m_i over the disk cells (Section IV). */
void ndo_mean_m(const ndo_model *m, const double *mv, double out[3])
{
    const int N = m->D * m->D;
    double s[3] = {0, 0, 0};
    for (int t = 0; t < N; ++t)
        if (m->mask[t]) for (int k = 0; k < 3; ++k) s[k] += mv[k * N + t];
    for (int k = 0; k < 3; ++k) out[k] = s[k] / m->C;
}

/* ---------------------------------------------- constrained relaxation */

/* Lagrange-constrained relaxation that pins the vortex core at X (Section IV;
 * the constraint itself is given in a reference the paper cites, so this is a
 * reading, parity unpinned beyond its own fixed-point properties).
 *
 * Constraint: C_k(m) = sum_{i in W} (m_i^z)^2 d_ik = 0 for k = x, y, with
 * d_ik = (r_ik - X_k)/a and window W = disk cells with |r_i - X| < 4 lambda_ex
 * -- the core estimator r_c = X written without its denominator.
 * Fictitious field: lambda_k dC_k/dm_i = 2 lambda_k m_i^z d_ik zhat.
 *
 * One sweep, given m:
 *   1. b = field(m); s_ik = 2 m_i^z d_ik;  e_i = b_i + (sum_k lambda_k s_ik) zhat.
 *   2. residual = max_i |m_i x e_i| / |e_i|; stop if residual < tol.
 *   3. trial alignment m'_i = normalise((1-eta) m_i + eta e_i/|e_i|) and one
 *      Newton step on lambda for C(m'(lambda)) = 0 using the exact 2x2
 *      Jacobian J_lk = sum_i 4 m'^z_i m^z_i kappa_i d_il d_ik with
 *      kappa_i = eta (q^z_i - m'^z_i (m'_i . q_i)) / |v_i|,
 *      q_i = (zhat - u_i u^z_i)/|e_i|, u_i = e_i/|e_i|, v_i = (1-eta) m_i + eta u_i.
 *   4. m <- m'(lambda_new).
 * U is the energy of the returned state in units of J.
 * Returns 0 when converged, 1 when max_iter sweeps did not converge. */
static void relax_align(const ndo_model *m, const double *mv, const double *b, const double lam[2],
                        double X, double Y, double eta, double rc2, double *mout,
                        double Cout[2], double Jout[3], double *resid)
{
    const int D = m->D, N = D * D;
    double C0 = 0, C1 = 0, J00 = 0, J01 = 0, J11 = 0, res = 0;
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) {
            int t = j * D + i;
            if (!m->mask[t]) { mout[t] = mout[N + t] = mout[2 * N + t] = 0.0; continue; }
            double mm[3] = {mv[t], mv[N + t], mv[2 * N + t]};
            double e[3] = {b[t], b[N + t], b[2 * N + t]};
            double dx = (i - 0.5 * (D - 1)) - X, dy = (j - 0.5 * (D - 1)) - Y;
            int inW = (dx * dx + dy * dy) < rc2;
            if (inW) e[2] += lam[0] * 2.0 * mm[2] * dx + lam[1] * 2.0 * mm[2] * dy;
            double en = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            double u[3] = {e[0] / en, e[1] / en, e[2] / en}, tq[3];
            cross(mm, u, tq);
            double r = sqrt(tq[0] * tq[0] + tq[1] * tq[1] + tq[2] * tq[2]);
            if (r > res) res = r;
            double v[3];
            for (int k = 0; k < 3; ++k) v[k] = (1.0 - eta) * mm[k] + eta * u[k];
            double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            double mp[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
            for (int k = 0; k < 3; ++k) mout[k * N + t] = mp[k];
            if (inW) {
                double q[3] = {-u[0] * u[2] / en, -u[1] * u[2] / en, (1.0 - u[2] * u[2]) / en};
                double mq = mp[0] * q[0] + mp[1] * q[1] + mp[2] * q[2];
                double kap = eta * (q[2] - mp[2] * mq) / vn;
                double wgt = 4.0 * mp[2] * mm[2] * kap;
                C0 += mp[2] * mp[2] * dx;
                C1 += mp[2] * mp[2] * dy;
                J00 += wgt * dx * dx; J01 += wgt * dx * dy; J11 += wgt * dy * dy;
            }
        }
    if (Cout) { Cout[0] = C0; Cout[1] = C1; }
    if (Jout) { Jout[0] = J00; Jout[1] = J01; Jout[2] = J11; }
    if (resid) *resid = res;
}

/* Constraint values C_k(m) for a state (used by tests and by the relaxation). */
void ndo_constraint(const ndo_model *m, const double *mv, const double Xm[2], double Cout[2])
{
    const int D = m->D, N = D * D;
    double X = Xm[0] / m->a, Y = Xm[1] / m->a, rcut = 4.0 * m->lambda_ex / m->a, rc2 = rcut * rcut;
    double C0 = 0, C1 = 0;
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) {
            int t = j * D + i;
            if (!m->mask[t]) continue;
            double dx = (i - 0.5 * (D - 1)) - X, dy = (j - 0.5 * (D - 1)) - Y;
            if (dx * dx + dy * dy >= rc2) continue;
            double z2 = mv[2 * N + t] * mv[2 * N + t];
            C0 += z2 * dx; C1 += z2 * dy;
        }
    Cout[0] = C0; Cout[1] = C1;
}

/* One relaxation sweep (exposed for sweep-level parity tests). lam is updated
 * in place, mv is replaced by the new state; returns the residual computed
 * before the update. */
double ndo_relax_sweep(const ndo_model *m, double *mv, const double Xm[2], double lam[2], double eta)
{
    const int N3 = 3 * m->D * m->D;
    double X = Xm[0] / m->a, Y = Xm[1] / m->a, rcut = 4.0 * m->lambda_ex / m->a, rc2 = rcut * rcut;
    double *b = malloc(sizeof(double) * N3), *mp = malloc(sizeof(double) * N3);
    double Cv[2], Jv[3], res;
    ndo_field(m, mv, b);
    relax_align(m, mv, b, lam, X, Y, eta, rc2, mp, Cv, Jv, &res);
    double det = Jv[0] * Jv[2] - Jv[1] * Jv[1];
    if (det != 0.0 && isfinite(det)) {
        double d0 = -(Jv[2] * Cv[0] - Jv[1] * Cv[1]) / det;
        double d1 = -(-Jv[1] * Cv[0] + Jv[0] * Cv[1]) / det;
        lam[0] += d0; lam[1] += d1;
    }
    relax_align(m, mv, b, lam, X, Y, eta, rc2, mp, NULL, NULL, NULL);
    memcpy(mv, mp, sizeof(double) * N3);
    free(b); free(mp);
    return res;
}

int ndo_relax(const ndo_model *m, double *mv, const double Xm[2], double tol, int max_iter,
              double eta, double *U, double lam[2], int *iters, double *resid_out)
{
    const int N3 = 3 * m->D * m->D;
    double X = Xm[0] / m->a, Y = Xm[1] / m->a, rcut = 4.0 * m->lambda_ex / m->a, rc2 = rcut * rcut;
    double *b = malloc(sizeof(double) * N3), *mp = malloc(sizeof(double) * N3);
    int status = 1, it;
    double res = INFINITY;
    for (it = 0; it < max_iter; ++it) {
        double Cv[2], Jv[3];
        ndo_field(m, mv, b);
        relax_align(m, mv, b, lam, X, Y, eta, rc2, mp, Cv, Jv, &res);
        if (res < tol) { status = 0; break; }
        double det = Jv[0] * Jv[2] - Jv[1] * Jv[1];
        if (det != 0.0 && isfinite(det)) {
            double d0 = -(Jv[2] * Cv[0] - Jv[1] * Cv[1]) / det;
            double d1 = -(-Jv[1] * Cv[0] + Jv[0] * Cv[1]) / det;
            lam[0] += d0; lam[1] += d1;
        }
        relax_align(m, mv, b, lam, X, Y, eta, rc2, mp, NULL, NULL, NULL);
        memcpy(mv, mp, sizeof(double) * N3);
    }
    if (iters) *iters = it;
    if (resid_out) *resid_out = res;
    if (U) *U = ndo_energy(m, mv);
    free(b); free(mp);
    return status;
}

int ndo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
