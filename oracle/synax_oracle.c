/*
 * synax_oracle.c -- plain FP64 CPU oracle of the synchrotron ray march of
 * "synax: A Differentiable and GPU-accelerated Synchrotron Simulation
 * Package" (Diao, Li, Grumitt, Mao), Sec. 2.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is compared against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header, constant or helper
 * with the CUDA library: every formula below is written out again from the
 * paper (and, for the field models the paper does not print, from the model
 * definitions of the project's design notes).
 *
 * What it computes, per HEALPix pixel i (Sec. 2.3):
 *   1. the pixel centre (RING scheme, Gorski et al. 2005) -> (l_i, b_i), n_i;
 *   2. the ray length L_i (fixed r_max, or exit from the box l_x,l_y,l_z
 *      centred on the Galactic centre, Sec. 2.3) and dr_i = L_i / N_int;
 *   3. midpoints r_{i,n} = r_obs + (n - 1/2) dr_i n_i, n = 1..N_int;
 *   4. B, N0, n_e at each midpoint (field models below: analytic, or B
 *      interpolated trilinearly on a grid over the box);
 *   5. j_I (Eq. 2) and j_P (Eq. 5) literally, in cgs, with B_trans the norm
 *      of the component of B transverse to n_i;
 *   6. chi_0 from Eq. 8 (denominator read as B.e_l, see the design notes);
 *   7. RM at the midpoint from Eq. 7 with B_LOS = -B.n (signed), integrated
 *      as the exact integral of the piecewise-constant cell values up to the
 *      midpoint: sum_{m<n} f_m dr + f_n dr / 2 (rm_rule 0, the default);
 *      rm_rule 1 drops the own cell (sum_{m<n}), rule 2 takes all of it
 *      (sum_{m<=n}, a plain cumulative sum);
 *   8. chi = chi_0 + RM lambda^2 (Eq. 6), lambda = c / nu;
 *   9. I, Q, U as the discrete sums of Eq. 9;
 *  10. brightness temperature T = I c^2 / (2 k nu^2) (Rayleigh-Jeans).
 * Loop order: pixel -> step -> frequency, all in double precision, plain
 * summation.  Pixels are split over POSIX threads in contiguous ranges;
 * every pixel is computed by exactly one thread, so results do not depend on
 * the thread count.
 *
 * Units: positions and lengths in kpc, B in microgauss, densities in cm^-3
 * at the model level; converted to cgs (G, cm) before Eq. 2, 5, 7 and 9.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- physical constants, cgs (CODATA 2018 exact / recommended values) ---- */
#define OR_C      2.99792458e10          /* speed of light, cm s^-1 */
#define OR_QE     4.803204712570263e-10  /* electron charge, statcoulomb */
#define OR_ME     9.1093837015e-28       /* electron mass, g */
#define OR_KB     1.380649e-16           /* Boltzmann constant, erg K^-1 */
#define OR_KPC    3.0856775814913673e21  /* kiloparsec, cm */
#define OR_UG     1.0e-6                 /* microgauss, G */
#define OR_PI     3.14159265358979323846

/* ---- model identifiers (same meaning as the library's, typed again) ---- */
#define OR_MODEL_TOY  0
#define OR_MODEL_WMAP 1
#define OR_MODEL_JF12 2
#define OR_MODEL_GRID 3
#define OR_MODEL_WMAP_STACK 4

#define OR_MAX_FREQ  16
#define OR_MAX_THETA 32

typedef struct {
    int32_t nside;
    int32_t n_steps;
    double  r_max_kpc;
    int32_t box_clip;               /* 1: ray ends at the box boundary */
    double  box_kpc[3];             /* full box lengths (l_x, l_y, l_z) */
    double  obs_kpc[3];             /* observer position, galactocentric */
    int32_t n_freq;
    double  freq_hz[OR_MAX_FREQ];
    int32_t model_id;
    int32_t n_theta;
    double  theta[OR_MAX_THETA];
    int32_t rm_rule;                /* 0 half-cell, 1 exclusive, 2 inclusive */
    const double* grid;             /* grid model: B at cell centres, [nz][ny][nx][3] uG */
    int32_t grid_n[3];              /* (nx, ny, nz), each >= 2 */
} oracle_problem;

/* ======================================================================
 * HEALPix RING pixel centres (Gorski et al. 2005, Sec. 4).
 * Ring i = 1..4N-1 from the north pole.  North cap i < N: 4i pixels,
 * z = 1 - i^2/(3N^2), phi = pi/(2i) (j - 1/2).  Equatorial belt
 * N <= i <= 3N: 4N pixels, z = 4/3 - 2i/(3N), phi = pi/(2N) (j - 1 + s/2)
 * with s = (i - N + 1) mod 2 (pixel 4 of Nside 1 sits at phi = 0, as in
 * healpy).  South cap: mirror of ring 4N - i.  Pixels are numbered ring by
 * ring from the north, with increasing phi inside a ring.
 * ====================================================================== */
int oracle_healpix_centre(int64_t nside, int64_t pix, double* z_out, double* phi_out)
{
    int64_t N = nside;
    if (N < 1) return -1;
    int64_t npix = 12 * N * N;
    if (pix < 0 || pix >= npix) return -1;
    int64_t first = 0, ring = 0, j = 0;
    for (int64_t i = 1; i <= 4 * N - 1; ++i) {
        int64_t n_in_ring = (i < N) ? 4 * i : (i <= 3 * N ? 4 * N : 4 * (4 * N - i));
        if (pix < first + n_in_ring) { ring = i; j = pix - first + 1; break; }
        first += n_in_ring;
    }
    double z, phi;
    double Nd = (double)N;
    if (ring < N) {
        double id = (double)ring;
        z = 1.0 - id * id / (3.0 * Nd * Nd);
        phi = OR_PI / (2.0 * id) * ((double)j - 0.5);
    } else if (ring <= 3 * N) {
        int64_t s = (ring - N + 1) % 2;
        z = 4.0 / 3.0 - 2.0 * (double)ring / (3.0 * Nd);
        phi = OR_PI / (2.0 * Nd) * ((double)j - 1.0 + 0.5 * (double)s);
    } else {
        double kd = (double)(4 * N - ring);
        z = -(1.0 - kd * kd / (3.0 * Nd * Nd));
        phi = OR_PI / (2.0 * kd) * ((double)j - 0.5);
    }
    *z_out = z;
    *phi_out = phi;
    return 0;
}

/* Line of sight for one pixel: l = phi, b = pi/2 - theta (Sec. 2.3, healpy
 * angles); n = (cos b cos l, cos b sin l, sin b); e_l = d n / d l normalised,
 * e_b = d n / d b.  (n, e_l, e_b) is a right-handed orthonormal triad. */
static void los_basis(int64_t nside, int64_t pix, double n[3], double el[3], double eb[3],
                      double* l_out, double* b_out)
{
    double z, phi;
    oracle_healpix_centre(nside, pix, &z, &phi);
    double theta = acos(z);
    double l = phi, b = OR_PI / 2.0 - theta;
    n[0] = cos(b) * cos(l);  n[1] = cos(b) * sin(l);  n[2] = sin(b);
    el[0] = -sin(l);         el[1] = cos(l);          el[2] = 0.0;
    eb[0] = -sin(b) * cos(l); eb[1] = -sin(b) * sin(l); eb[2] = cos(b);
    if (l_out) *l_out = l;
    if (b_out) *b_out = b;
}

/* Distance from the observer (inside the box) to the box boundary along n
 * (Sec. 2.3: the LOS runs from the observer to the box boundary). */
static double box_exit(const double o[3], const double n[3], const double box[3])
{
    double t = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double h = 0.5 * box[k];
        if (n[k] > 0.0)      t = fmin(t, (h - o[k]) / n[k]);
        else if (n[k] < 0.0) t = fmin(t, (-h - o[k]) / n[k]);
    }
    return t;
}

/* ======================================================================
 * Field models.  Each returns B (microgauss, galactocentric Cartesian),
 * N0 (cm^-3) and n_e (cm^-3) at r (kpc).  t is the distance from the
 * observer, used only by the toy model's sphere.
 * ====================================================================== */
static double sech2(double x) { double c = cosh(x); return 1.0 / (c * c); }
static double smoothstep(double t)
{
    if (t <= 0.0) return 0.0;
    if (t >= 1.0) return 1.0;
    return t * t * (3.0 - 2.0 * t);
}
static double logistic(double x, double h, double w)
{
    /* JF12-style transition L(x; h, w) = 1 / (1 + exp(-2 (|x| - h) / w)) */
    return 1.0 / (1.0 + exp(-2.0 * (fabs(x) - h) / w));
}

/* CR density, WMAP form (Sec. 3.1, Eq. 12) N0 = C0 exp(-rho/h_r) sech^2(z/h_z),
 * h_r = 5 kpc, h_z = 1 kpc; C0 is fixed by the density N0_obs at the observer
 * (the paper fixes N0 at Earth to 4.0e-5 cm^-3). */
static double cr_density(const double r[3], const double obs[3], double n0_obs)
{
    double rho = hypot(r[0], r[1]);
    double rho_o = hypot(obs[0], obs[1]);
    double g = exp(-rho / 5.0) * sech2(r[2] / 1.0);
    double g_o = exp(-rho_o / 5.0) * sech2(obs[2] / 1.0);
    return n0_obs * g / g_o;
}

/* Cylindrical unit vectors; at rho = 0 the azimuth is taken as 0. */
static void cyl_basis(const double r[3], double* rho, double rh[3], double ph[3])
{
    *rho = hypot(r[0], r[1]);
    double c = 1.0, s = 0.0;
    if (*rho > 0.0) { c = r[0] / *rho; s = r[1] / *rho; }
    rh[0] = c;  rh[1] = s;  rh[2] = 0.0;
    ph[0] = -s; ph[1] = c;  ph[2] = 0.0;
}

/* Toy model (Sec. 2.4): uniform B, n_e, N0 inside a sphere of radius R0
 * around the observer, zero outside.  theta = [Bx, By, Bz (uG), n_e, N0
 * (cm^-3), p, R0 (kpc)]. */
static void field_toy(const double* th, double t, double B[3], double* N0, double* ne)
{
    int inside = t < th[6];
    B[0] = inside ? th[0] : 0.0;
    B[1] = inside ? th[1] : 0.0;
    B[2] = inside ? th[2] : 0.0;
    *ne = inside ? th[3] : 0.0;
    *N0 = inside ? th[4] : 0.0;
}

/* WMAP-type model (Sec. 3.1, Eq. 13) with an exponential envelope and a
 * uniform x field.  theta = [b0 (uG), psi0, psi1, chi0B (rad), Bux (uG),
 * N0_obs (cm^-3), p, ne0 (cm^-3)].
 *   B = b0 e^{-rho/8} e^{-|z|/1} [cos psi cos chi rho^ + sin psi cos chi phi^
 *       + sin chi z^] + (Bux, 0, 0),
 *   psi = psi0 + psi1 ln(rho / 8 kpc), chi = chi0B tanh(z / 1 kpc) for
 *   3 <= rho <= 20 kpc, both zero otherwise;
 *   n_e = ne0 e^{-rho/20} sech^2(z/1). */
static void field_wmap(const double* th, const double r[3], const double obs[3],
                       double B[3], double* N0, double* ne)
{
    double rho, rh[3], ph[3];
    cyl_basis(r, &rho, rh, ph);
    double psi = 0.0, chi = 0.0;
    if (rho >= 3.0 && rho <= 20.0) {
        psi = th[1] + th[2] * log(rho / 8.0);
        chi = th[3] * tanh(r[2] / 1.0);
    }
    double amp = th[0] * exp(-rho / 8.0) * exp(-fabs(r[2]) / 1.0);
    for (int k = 0; k < 3; ++k) {
        double zk = (k == 2) ? 1.0 : 0.0;
        B[k] = amp * (cos(psi) * cos(chi) * rh[k] + sin(psi) * cos(chi) * ph[k] + sin(chi) * zk);
    }
    B[0] += th[4];
    *N0 = cr_density(r, obs, th[5]);
    *ne = th[7] * exp(-rho / 20.0) * sech2(r[2] / 1.0);
}

/* JF12-type model (defined by this project after Jansson & Farrar 2012; the
 * paper cites it but prints no formula).  theta = [b_1..b_8 (uG), B_h (uG),
 * z_h (kpc), B_X (uG), theta_X (rad), N0_obs (cm^-3), p, h1 (kpc), h2 (kpc)].
 * Fixed structure:
 *   disc: 8 log-spiral arms, pitch i = 11.5 deg, reference radius 5 kpc.
 *     Arm coordinate u = 8 (phi - ln(rho/5)/tan i) / (2 pi) mod 8; arm k
 *     covers u in [k, k+1); weights w_k(u) = S((d+delta)/(2delta))
 *     - S((d-1+delta)/(2delta)), d = u - k wrapped to [-4, 4), delta = 1/2,
 *     S the cubic smoothstep; beta(u) = sum_k b_k w_k(u): the strength is
 *     b_k at the arm centre u = k + 1/2 and is interpolated C^1 between
 *     neighbouring centres.
 *     B_disc = beta (5/rho) W(rho) (1 - L(z; 0.4, 0.27)) (sin i rho^ + cos i phi^),
 *     W(rho) = S((rho - 4.75)/0.5) S((20.25 - rho)/0.5).
 *   toroidal halo: B_h e^{-|z|/z_h} L(z; 0.4, 0.27) (1 - L(rho; 9.22, 0.2)) s(z) phi^,
 *     s(z) = z / sqrt(z^2 + 0.1^2) (a smooth sign).
 *   X field: r_p = rho - |z| / tan theta_X; for r_p > 0:
 *     B_X e^{-r_p/4.8} (r_p/rho) (s(z) cos theta_X rho^ + sin theta_X z^).
 *   CR: WMAP form normalised at the observer (cr_density).
 *   n_e = 0.025 e^{-rho/20} e^{-|z|/h1} + 0.10 e^{-rho/4} e^{-|z|/h2}. */
static void field_jf12(const double* th, const double r[3], const double obs[3],
                       double B[3], double* N0, double* ne)
{
    double rho, rh[3], ph[3];
    cyl_basis(r, &rho, rh, ph);
    double z = r[2];
    double pitch = 11.5 * OR_PI / 180.0;
    double Lz = logistic(z, 0.4, 0.27);
    double sz = z / sqrt(z * z + 0.1 * 0.1);
    for (int k = 0; k < 3; ++k) B[k] = 0.0;

    /* disc */
    double W = smoothstep((rho - 4.75) / 0.5) * smoothstep((20.25 - rho) / 0.5);
    if (W > 0.0) {
        double phi = atan2(r[1], r[0]);
        double phi0 = phi - log(rho / 5.0) / tan(pitch);
        double u = fmod(8.0 * phi0 / (2.0 * OR_PI), 8.0);
        if (u < 0.0) u += 8.0;
        double beta = 0.0, delta = 0.5;
        for (int k = 0; k < 8; ++k) {
            double d = u - (double)k;
            if (d >= 4.0) d -= 8.0;
            if (d < -4.0) d += 8.0;
            double wk = smoothstep((d + delta) / (2.0 * delta))
                      - smoothstep((d - 1.0 + delta) / (2.0 * delta));
            beta += th[k] * wk;
        }
        double amp = beta * (5.0 / rho) * W * (1.0 - Lz);
        for (int k = 0; k < 3; ++k) B[k] += amp * (sin(pitch) * rh[k] + cos(pitch) * ph[k]);
    }

    /* toroidal halo */
    double Lr = 1.0 / (1.0 + exp(-2.0 * (rho - 9.22) / 0.2));
    double halo = th[8] * exp(-fabs(z) / th[9]) * Lz * (1.0 - Lr) * sz;
    for (int k = 0; k < 3; ++k) B[k] += halo * ph[k];

    /* X field */
    double thx = th[11];
    double rp = rho - fabs(z) / tan(thx);
    if (rp > 0.0) {
        double mag = th[10] * exp(-rp / 4.8) * (rp / rho);
        B[0] += mag * sz * cos(thx) * rh[0];
        B[1] += mag * sz * cos(thx) * rh[1];
        B[2] += mag * sin(thx);
    }

    *N0 = cr_density(r, obs, th[12]);
    *ne = 0.025 * exp(-rho / 20.0) * exp(-fabs(z) / th[14])
        + 0.10 * exp(-rho / 4.0) * exp(-fabs(z) / th[15]);
}

/* Grid model (Sec. 2.3: a field given on a regular 3D grid over the box and
 * found at the midpoints by 3D linear interpolation; Sec. 3.3 optimises such
 * a B grid).  The nodes span the box wall to wall: node i of n_x along x sits
 * at x_i = -l_x/2 + i l_x / (n_x - 1), likewise y and z, so every point of the
 * box lies inside the node hull.  A point's fractional node coordinate
 * u = (x + l_x/2) (n_x - 1) / l_x is clamped to [0, n_x - 1] (which only
 * matters for points on or beyond a wall), and B is the trilinear blend of the
 * 8 nodes around it.  theta = [N0_obs (cm^-3), p, ne0 (cm^-3)]: CR density as
 * in the WMAP-type model (cr_density), n_e = ne0 e^{-rho/20} sech^2(z/1). */
static void grid_axis(double x, double l, int n, int* i0, double* f)
{
    double u = (x + 0.5 * l) * (n - 1) / l;
    if (u < 0.0) u = 0.0;
    if (u > n - 1) u = n - 1;
    int i = (int)floor(u);
    if (i > n - 2) i = n - 2;
    *i0 = i;
    *f = u - i;
}

void oracle_grid_interp(const double* grid, const int32_t n[3], const double box[3], const double r[3],
                        double B[3])
{
    int i0, j0, k0;
    double fx, fy, fz;
    grid_axis(r[0], box[0], n[0], &i0, &fx);
    grid_axis(r[1], box[1], n[1], &j0, &fy);
    grid_axis(r[2], box[2], n[2], &k0, &fz);
    for (int c = 0; c < 3; ++c) B[c] = 0.0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                double w = (di ? fx : 1.0 - fx) * (dj ? fy : 1.0 - fy) * (dk ? fz : 1.0 - fz);
                size_t node = ((size_t)(k0 + dk) * n[1] + (size_t)(j0 + dj)) * n[0] + (size_t)(i0 + di);
                for (int c = 0; c < 3; ++c) B[c] += w * grid[node * 3 + c];
            }
}

static void field_grid(const oracle_problem* P, const double r[3], double B[3], double* N0, double* ne)
{
    oracle_grid_interp(P->grid, P->grid_n, P->box_kpc, r, B);
    double rho = sqrt(r[0] * r[0] + r[1] * r[1]);
    *N0 = cr_density(r, P->obs_kpc, P->theta[0]);
    *ne = P->theta[2] * exp(-rho / 20.0) * sech2(r[2] / 1.0);
}

/* Stacked WMAP model (Sec. 4.3, Eq. 16): four fields of the WMAP form of
 * Eq. 13, each B_k = b0_k [cos psi_k cos chi_k rho^ + sin psi_k cos chi_k
 * phi^ + sin chi_k z^] with psi_k = psi0_k + psi1_k ln(rho / 8 kpc) and
 * chi_k = chi0B_k tanh(z / 1 kpc) for 3 <= rho <= 20 kpc (both zero
 * otherwise; no envelope: |B_k| = b0_k), stacked with the weights and the
 * component permutations of Eq. 16:
 *   B_x = 0.6 B1_x + 0.3 B2_x + 0.1 B3_z + 0.3 B4_y
 *   B_y = 0.6 B1_y + 0.3 B2_z + 0.1 B3_y + 0.3 B4_x
 *   B_z = 0.6 B1_z + 0.3 B2_y + 0.1 B3_x + 0.3 B4_z
 * theta = [b0, psi0, psi1, chi0B for k = 1..4 (uG, rad), N0_obs (cm^-3), p,
 * ne0 (cm^-3)]; N0 and n_e as in the WMAP-type model. */
static void wmap_component(const double* th4, double rho, const double rh[3], const double ph[3], double z,
                           double Bk[3])
{
    double psi = 0.0, chi = 0.0;
    if (rho >= 3.0 && rho <= 20.0) {
        psi = th4[1] + th4[2] * log(rho / 8.0);
        chi = th4[3] * tanh(z / 1.0);
    }
    for (int k = 0; k < 3; ++k) {
        double zk = (k == 2) ? 1.0 : 0.0;
        Bk[k] = th4[0] * (cos(psi) * cos(chi) * rh[k] + sin(psi) * cos(chi) * ph[k] + sin(chi) * zk);
    }
}

static void field_wmap_stack(const double* th, const double r[3], const double obs[3],
                             double B[3], double* N0, double* ne)
{
    double rho, rh[3], ph[3];
    cyl_basis(r, &rho, rh, ph);
    double B1[3], B2[3], B3[3], B4[3];
    wmap_component(th + 0, rho, rh, ph, r[2], B1);
    wmap_component(th + 4, rho, rh, ph, r[2], B2);
    wmap_component(th + 8, rho, rh, ph, r[2], B3);
    wmap_component(th + 12, rho, rh, ph, r[2], B4);
    B[0] = 0.6 * B1[0] + 0.3 * B2[0] + 0.1 * B3[2] + 0.3 * B4[1];
    B[1] = 0.6 * B1[1] + 0.3 * B2[2] + 0.1 * B3[1] + 0.3 * B4[0];
    B[2] = 0.6 * B1[2] + 0.3 * B2[1] + 0.1 * B3[0] + 0.3 * B4[2];
    *N0 = cr_density(r, obs, th[16]);
    *ne = th[18] * exp(-rho / 20.0) * sech2(r[2] / 1.0);
}

static double spectral_index(const oracle_problem* P)
{
    switch (P->model_id) {
    case OR_MODEL_TOY:  return P->theta[5];
    case OR_MODEL_WMAP: return P->theta[6];
    case OR_MODEL_GRID: return P->theta[1];
    case OR_MODEL_WMAP_STACK: return P->theta[17];
    default:            return P->theta[13];
    }
}

/* Field evaluation exposed for unit tests. */
int oracle_fields(const oracle_problem* P, const double r[3], double t,
                  double B[3], double* N0, double* ne)
{
    switch (P->model_id) {
    case OR_MODEL_TOY:  field_toy(P->theta, t, B, N0, ne); return 0;
    case OR_MODEL_WMAP: field_wmap(P->theta, r, P->obs_kpc, B, N0, ne); return 0;
    case OR_MODEL_JF12: field_jf12(P->theta, r, P->obs_kpc, B, N0, ne); return 0;
    case OR_MODEL_WMAP_STACK: field_wmap_stack(P->theta, r, P->obs_kpc, B, N0, ne); return 0;
    case OR_MODEL_GRID:
        if (!P->grid) return -1;
        field_grid(P, r, B, N0, ne);
        return 0;
    default: return -1;
    }
}

/* ======================================================================
 * Emissivities (Sec. 2.1 Eq. 2 and Sec. 2.2 Eq. 5), cgs.  B_trans in G,
 * N0 in cm^-3, nu in Hz -> erg s^-1 cm^-3 Hz^-1 sr^-1.  The limit
 * B_trans -> 0 is 0 (p > -1).
 * ====================================================================== */
void oracle_emissivity(double nu, double p, double b_trans_g, double n0,
                       double* jI, double* jP)
{
    if (!(b_trans_g > 0.0)) { *jI = 0.0; *jP = 0.0; return; }
    double pre = sqrt(3.0) * OR_QE * OR_QE * OR_QE * b_trans_g * n0
               / (8.0 * OR_PI * OR_ME * OR_C * OR_C);
    double x = 4.0 * OR_PI * nu * OR_ME * OR_C / (3.0 * OR_QE * b_trans_g);
    double xp = pow(x, (1.0 - p) / 2.0);
    double g1 = tgamma(p / 4.0 - 1.0 / 12.0);
    *jI = pre * xp * pow(2.0, (p + 1.0) / 2.0) / (p + 1.0) * g1 * tgamma(p / 4.0 + 19.0 / 12.0);
    *jP = pre * xp * pow(2.0, (p - 3.0) / 2.0) * g1 * tgamma(p / 4.0 + 7.0 / 12.0);
}

/* RM prefactor q_e^3 / (2 pi m_e^2 c^4) of Eq. 7 (cgs: rad cm^-2 per
 * cm^-3 G cm). */
double oracle_rm_constant(void)
{
    return OR_QE * OR_QE * OR_QE / (2.0 * OR_PI * OR_ME * OR_ME * OR_C * OR_C * OR_C * OR_C);
}

/* Rayleigh-Jeans brightness temperature of a specific intensity (cgs). */
double oracle_brightness_temperature(double I, double nu)
{
    return I * OR_C * OR_C / (2.0 * OR_KB * nu * nu);
}

/* ======================================================================
 * The march for one pixel.  out[f*3 + s], s = 0 (I), 1 (Q), 2 (U), in K.
 * ====================================================================== */
static void march_pixel(const oracle_problem* P, int64_t pix, double* out)
{
    double n[3], el[3], eb[3];
    los_basis(P->nside, pix, n, el, eb, NULL, NULL);
    double L = P->box_clip ? box_exit(P->obs_kpc, n, P->box_kpc) : P->r_max_kpc;
    int N = P->n_steps;
    double dr_kpc = L / (double)N;
    double dr_cm = dr_kpc * OR_KPC;
    double p = spectral_index(P);
    double K = oracle_rm_constant();
    int F = P->n_freq;

    double I[OR_MAX_FREQ], Q[OR_MAX_FREQ], U[OR_MAX_FREQ];
    for (int f = 0; f < F; ++f) { I[f] = 0.0; Q[f] = 0.0; U[f] = 0.0; }

    double rm_prefix = 0.0; /* sum_{m<n} n_e B_LOS dr over earlier cells, cgs */
    for (int k = 1; k <= N; ++k) {
        double t = ((double)k - 0.5) * dr_kpc;
        double r[3];
        for (int c = 0; c < 3; ++c) r[c] = P->obs_kpc[c] + t * n[c];
        double B[3], N0, ne;
        oracle_fields(P, r, t, B, &N0, &ne);

        double bn = B[0] * n[0] + B[1] * n[1] + B[2] * n[2];
        double bperp[3];
        for (int c = 0; c < 3; ++c) bperp[c] = B[c] - bn * n[c];
        double b_trans = sqrt(bperp[0] * bperp[0] + bperp[1] * bperp[1] + bperp[2] * bperp[2]);

        /* Eq. 8 with the denominator read as B.e_l */
        double num = B[0] * eb[0] + B[1] * eb[1] + B[2] * eb[2];
        double den = B[0] * el[0] + B[1] * el[1] + B[2] * el[2];
        double chi0 = atan2(num, den);

        /* Eq. 7: signed B_LOS = -B.n (positive towards the observer) */
        double f = ne * (-bn * OR_UG);
        double own = P->rm_rule == 1 ? 0.0 : (P->rm_rule == 2 ? 1.0 : 0.5);
        double rm = K * (rm_prefix + own * f * dr_cm);
        rm_prefix += f * dr_cm;

        for (int q = 0; q < F; ++q) {
            double nu = P->freq_hz[q];
            double jI, jP;
            oracle_emissivity(nu, p, b_trans * OR_UG, N0, &jI, &jP);
            double lam = OR_C / nu;
            double chi = chi0 + rm * lam * lam;           /* Eq. 6 */
            I[q] += jI * dr_cm;                           /* Eq. 9 */
            Q[q] += jP * cos(2.0 * chi) * dr_cm;
            U[q] += jP * sin(2.0 * chi) * dr_cm;
        }
    }
    for (int q = 0; q < F; ++q) {
        double nu = P->freq_hz[q];
        out[q * 3 + 0] = oracle_brightness_temperature(I[q], nu);
        out[q * 3 + 1] = oracle_brightness_temperature(Q[q], nu);
        out[q * 3 + 2] = oracle_brightness_temperature(U[q], nu);
    }
}

/* ---- threading over pixel ranges ---- */
typedef struct {
    const oracle_problem* P;
    const int64_t* pix;
    int64_t n_pix, begin, end;
    double* maps;
} or_job;

static void* or_worker(void* arg)
{
    or_job* J = (or_job*)arg;
    int F = J->P->n_freq;
    double out[OR_MAX_FREQ * 3];
    for (int64_t i = J->begin; i < J->end; ++i) {
        int64_t pix = J->pix ? J->pix[i] : i;
        march_pixel(J->P, pix, out);
        for (int q = 0; q < F; ++q)
            for (int s = 0; s < 3; ++s)
                J->maps[((int64_t)q * 3 + s) * J->n_pix + i] = out[q * 3 + s];
    }
    return NULL;
}

/* Validate the problem; returns 0 when it can be marched. */
static int or_validate(const oracle_problem* P)
{
    if (P->nside < 1 || P->nside > 8192) return -1;
    if (P->n_steps < 1) return -1;
    if (P->n_freq < 1 || P->n_freq > OR_MAX_FREQ) return -1;
    if (P->model_id < OR_MODEL_TOY || P->model_id > OR_MODEL_WMAP_STACK) return -1;
    static const int need[5] = {7, 8, 16, 3, 19};
    if (P->n_theta != need[P->model_id]) return -1;
    if (!P->box_clip && !(P->r_max_kpc > 0.0)) return -1;
    if (P->model_id == OR_MODEL_GRID) {
        /* the grid spans the box, so rays end at its walls */
        if (!P->grid || !P->box_clip) return -1;
        for (int a = 0; a < 3; ++a)
            if (P->grid_n[a] < 2) return -1;
    }
    if (P->rm_rule < 0 || P->rm_rule > 2) return -1;
    return 0;
}

/*
 * Maps for the pixels in pix[0..n_pix) (or all 12 nside^2 pixels in RING
 * order when pix is NULL, n_pix then being 12 nside^2), written as
 * maps[f][s][i] (f frequency, s = I, Q, U, i position in the pixel list),
 * brightness temperature in K.  n_threads <= 0 uses one thread.
 */
int oracle_forward(const oracle_problem* P, const int64_t* pix, int64_t n_pix,
                   double* maps, int n_threads)
{
    if (or_validate(P) != 0) return -1;
    int64_t npix_all = 12LL * P->nside * P->nside;
    if (!pix && n_pix != npix_all) return -1;
    if (pix)
        for (int64_t i = 0; i < n_pix; ++i)
            if (pix[i] < 0 || pix[i] >= npix_all) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if ((int64_t)n_threads > n_pix) n_threads = (int)(n_pix > 0 ? n_pix : 1);

    or_job jobs[256];
    pthread_t tids[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].P = P;
        jobs[t].pix = pix;
        jobs[t].n_pix = n_pix;
        jobs[t].begin = n_pix * t / n_threads;
        jobs[t].end = n_pix * (t + 1) / n_threads;
        jobs[t].maps = maps;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&tids[t], NULL, or_worker, &jobs[t]);
    or_worker(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(tids[t], NULL);
    return 0;
}

/* Field evaluation at n points (positions r[3n], observer distances t[n]) for
 * unit tests: out[5i..5i+4] = B (3), N0, n_e. */
int oracle_fields_batch(const oracle_problem* P, int64_t n, const double* r, const double* t,
                        double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        double B[3], N0, ne;
        if (oracle_fields(P, r + 3 * i, t[i], B, &N0, &ne) != 0) return -1;
        out[5 * i + 0] = B[0];
        out[5 * i + 1] = B[1];
        out[5 * i + 2] = B[2];
        out[5 * i + 3] = N0;
        out[5 * i + 4] = ne;
    }
    return 0;
}

/* LOS basis exposed for unit tests: out = [n(3), e_l(3), e_b(3), l, b]. */
int oracle_los(int64_t nside, int64_t pix, double* out)
{
    if (nside < 1 || pix < 0 || pix >= 12 * nside * nside) return -1;
    los_basis(nside, pix, out, out + 3, out + 6, out + 9, out + 10);
    return 0;
}

/* Ray length for one pixel (kpc), for unit tests. */
double oracle_ray_length(const oracle_problem* P, int64_t pix)
{
    double n[3], el[3], eb[3];
    los_basis(P->nside, pix, n, el, eb, NULL, NULL);
    return P->box_clip ? box_exit(P->obs_kpc, n, P->box_kpc) : P->r_max_kpc;
}
