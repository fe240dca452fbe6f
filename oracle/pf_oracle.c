/*
 * pf_oracle.c -- plain, slow, FP64 CPU oracle for one explicit time step of the
 * grand-potential phase-field model for ternary eutectic directional
 * solidification (Bauer et al., "Massively parallel phase-field simulations for
 * ternary eutectic directional solidification", arXiv:1506.01684).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA path; it is
 * never part of the product path.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Everything is written for readability: ghost layers are materialised as
 * padded copies, every face value is recomputed from its defining formula for
 * each of its two cells, and sums run in the order the formulas are written.
 * Compile with -O2 -ffp-contract=off (no fused multiply-add).
 *
 * Model (Section 2 of the paper):
 *   Eq. 1  d(phi_a)/dt = -(1/(tau*eps)) (rhs_a - (1/N) sum_b rhs_b)
 *          (the sign reading: phi descends the functional; see below)
 *   Eq. 2  rhs_a = eps*T*(da/dphi_a - div(da/dgrad phi_a))
 *                  + (T/eps) domega/dphi_a + dpsi/dphi_a
 *   Eq. 3  dmu/dt = [dc/dmu]^-1 ( -dc/dphi dphi/dt - dc/dT dT/dt
 *                                 + div(M grad mu) - div(J_at) )
 *   Eq. 4  J_at = (pi eps/4) sum_{a != l} g_a h_l / sqrt(phi_a phi_l) dphi_a/dt
 *                 (n_a . n_l) (c^l - c^a) (x) n_a,   n = grad phi/|grad phi|
 *   Frozen temperature T = T0 + G (z - v t) (Section 2, "frozen temperature").
 *   Algorithm 1: phi-sweep, then mu-sweep using phi at both time levels.
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * project's design notes):
 *   R1  parabolic grand potentials
 *         psi_a(mu,T) = -(1/2) mu . K_a mu - mu . chat_a(T) + s_a (T - TE),
 *         chat_a(T)   = cE_a + kT_a (T - TE),
 *         c^a(mu,T)   = -d psi_a / d mu = K_a mu + chat_a(T),
 *       with K_a = (1/2) A_a^{-1} for the curvature A_a of the fitted Gibbs energy
 *       f_a(c,T) = c . A_a c + B_a(T) . c + C_a(T) (B_a, C_a linear in T): A_a a
 *       symmetric positive-definite 2x2 matrix (the general form), or A_a times the
 *       identity (the symmetric set, K_a = I/(2 A_a)).
 *   R2  h_a = phi_a^2 / sum_b phi_b^2.
 *   R3  a = sum_{a<b} gamma_ab |q_ab|^2,  q_ab = phi_a grad phi_b - phi_b grad phi_a;
 *       omega = (16/pi^2) sum_{a<b} gamma_ab phi_a phi_b
 *               + sum_{a<b<d} gamma_abd phi_a phi_b phi_d.
 *   R4  minus sign in Eq. 1 (gradient flow).
 *   R5  N = 4 in the Lagrange term.
 *   R6  Euclidean projection onto the Gibbs simplex (sort-based).
 *   R7  face gradients and face averages of the mu-sweep use phi^{n+1};
 *       dphi/dt uses both levels.
 *   R8  g_a = phi_a.
 *   R9  a J_at term is skipped when the face average of phi_a or phi_l is
 *       <= 0 or when |grad phi_a|^2 or |grad phi_l|^2 <= 1e-20/dx^2.
 *   R10 dc/dphi dphi/dt -> sum_a c^a(mu^n,T^n) (h_a(phi^{n+1}) - h_a(phi^n)),
 *       dc/dT dT/dt     -> sum_a h_a(phi^{n+1}) kT_a (-G v dt),
 *       susceptibility chi = sum_a h_a(phi^{n+1}) K_a (a 2x2 matrix; mu^{n+1} =
 *       mu^n + chi^{-1} (source)), mobility M = sum_a D_a h_a K_a at the face.
 *   R11 moving window: h = sum(1 - phi_l)/(nx ny); when h >= z_trig, shift by
 *       s = min(floor(h - z_trig) + 1, nz - 1) planes; fresh planes get
 *       phi = e_l and the old top plane's mu.
 *   R12 dt <= 0 requests 0.5 * min(tau_min dx^2/(12 gamma_max T_max), dx^2/(6 D_max)).
 *   R17 relaxation time per phase pair: tau(phi) = sum_{a<b} tau_ab phi_a phi_b /
 *       sum_{a<b} phi_a phi_b at the cell's phi^n, and tau on a cell where that
 *       denominator is 0 (a single phase); all tau_ab <= 0: tau everywhere.
 *   R13 Voronoi nuclei from splitmix64.
 *
 * Grid: cell (i,j,k), x fastest; fields are SoA: phi[c][k][j][i] (c = 0..3,
 * phase 3 is the liquid), mu[c][k][j][i] (c = 0..1).  Periodic in x and y,
 * zero-gradient (mirror) in z.  Cell centres sit at z = (k + off) dx.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NPH 4
#define NMU 2
#define LIQ 3
#define ORC_PI 3.14159265358979323846

typedef struct {
    double dx, eps, tau, dt;
    double gamma2[6]; /* pairs (01,02,03,12,13,23) */
    double gamma3[4]; /* triples (012,013,023,123) */
    double A[4];
    double Am[4][3]; /* A_a as a symmetric matrix (a11, a12, a22); a11 <= 0: A[a] I */
    double tau_ab[6]; /* pairs (01,02,03,12,13,23); all <= 0: tau everywhere */
    double cE[4][2];
    double kT[4][2];
    double s[4];
    double D[4];
    double TE, T0, G, v;
    int seed_layers, n_grains;
    double window_trigger_z;
} orc_params;

/* ------------------------------------------------------------------------- */
/* parameter tables                                                           */
/* ------------------------------------------------------------------------- */

/* index of the pair (a, b), a != b, in the order 01 02 03 12 13 23 */
static int gam2_index(int a, int b)
{
    static const int I[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
    return I[a][b];
}

static double gam2(const orc_params *p, int a, int b) { return p->gamma2[gam2_index(a, b)]; }

static double gam3(const orc_params *p, int a, int b, int c)
{
    /* the triple is named by the phase it leaves out: 3 -> 012, 2 -> 013, 1 -> 023, 0 -> 123 */
    int missing = 6 - a - b - c;
    return p->gamma3[3 - missing];
}

/* R1: K_a = dc^a/dmu = (1/2) A_a^{-1} (symmetric 2x2) */
void orc_kmat(const orc_params *p, int a, double K[2][2])
{
    if (p->Am[a][0] > 0.0) {
        double a11 = p->Am[a][0], a12 = p->Am[a][1], a22 = p->Am[a][2];
        double det = a11 * a22 - a12 * a12;
        K[0][0] = 0.5 * a22 / det;
        K[0][1] = -0.5 * a12 / det;
        K[1][0] = -0.5 * a12 / det;
        K[1][1] = 0.5 * a11 / det;
    } else {
        K[0][0] = 1.0 / (2.0 * p->A[a]);
        K[0][1] = 0.0;
        K[1][0] = 0.0;
        K[1][1] = 1.0 / (2.0 * p->A[a]);
    }
}

static int tau_interpolated(const orc_params *p)
{
    for (int q = 0; q < 6; q++)
        if (p->tau_ab[q] > 0.0) return 1;
    return 0;
}

/* R17: relaxation time at a cell with phase fractions phi */
double orc_tau(const orc_params *p, const double phi[4])
{
    if (!tau_interpolated(p)) return p->tau;
    double num = 0.0, den = 0.0;
    for (int a = 0; a < NPH; a++)
        for (int b = a + 1; b < NPH; b++) {
            double w = phi[a] * phi[b];
            num += p->tau_ab[gam2_index(a, b)] * w;
            den += w;
        }
    return den > 0.0 ? num / den : p->tau;
}

/* R12: explicit stability limits of the linearised phi and mu equations. */
double orc_default_dt(const orc_params *p, int nz)
{
    double gmax = 0.0, dmax = 0.0, tmin = p->tau;
    if (tau_interpolated(p))
        for (int q = 0; q < 6; q++)
            if (p->tau_ab[q] < tmin) tmin = p->tau_ab[q];
    for (int i = 0; i < 6; i++)
        if (p->gamma2[i] > gmax) gmax = p->gamma2[i];
    for (int a = 0; a < NPH; a++)
        if (p->D[a] > dmax) dmax = p->D[a];
    double Ttop = p->T0 + p->G * (double)(nz - 1) * p->dx;
    double Tmax = p->T0 > Ttop ? p->T0 : Ttop;
    double lim_phi = tmin * p->dx * p->dx / (12.0 * gmax * Tmax);
    double lim_mu = dmax > 0.0 ? p->dx * p->dx / (6.0 * dmax) : lim_phi;
    double lim = lim_phi < lim_mu ? lim_phi : lim_mu;
    return 0.5 * lim;
}

/* ------------------------------------------------------------------------- */
/* pointwise model functions                                                  */
/* ------------------------------------------------------------------------- */

/* frozen temperature T = T0 + G (z - v t) */
double orc_temperature(const orc_params *p, double z, double t)
{
    return p->T0 + p->G * (z - p->v * t);
}

/* R1: chat_a(T) = cE_a + kT_a (T - TE) */
static void chat(const orc_params *p, int a, double T, double out[2])
{
    for (int i = 0; i < NMU; i++) out[i] = p->cE[a][i] + p->kT[a][i] * (T - p->TE);
}

/* R1: grand potential of phase a */
double orc_psi_alpha(const orc_params *p, int a, const double mu[2], double T)
{
    double ch[2], K[2][2];
    chat(p, a, T, ch);
    orc_kmat(p, a, K);
    double muKmu = mu[0] * (K[0][0] * mu[0] + K[0][1] * mu[1]) + mu[1] * (K[1][0] * mu[0] + K[1][1] * mu[1]);
    return -0.5 * muKmu - (mu[0] * ch[0] + mu[1] * ch[1]) + p->s[a] * (T - p->TE);
}

/* R1: c^a(mu,T) = -d psi_a/d mu */
void orc_c_alpha(const orc_params *p, int a, const double mu[2], double T, double out[2])
{
    double ch[2], K[2][2];
    chat(p, a, T, ch);
    orc_kmat(p, a, K);
    for (int i = 0; i < NMU; i++) out[i] = K[i][0] * mu[0] + K[i][1] * mu[1] + ch[i];
}

/* R2: h_a = phi_a^2 / sum phi_b^2 */
void orc_h(const double phi[4], double out[4])
{
    double S = 0.0;
    for (int b = 0; b < NPH; b++) S += phi[b] * phi[b];
    for (int a = 0; a < NPH; a++) out[a] = phi[a] * phi[a] / S;
}

/* psi(phi,mu,T) = sum_a h_a psi_a */
double orc_psi(const orc_params *p, const double phi[4], const double mu[2], double T)
{
    double h[4], r = 0.0;
    orc_h(phi, h);
    for (int a = 0; a < NPH; a++) r += h[a] * orc_psi_alpha(p, a, mu, T);
    return r;
}

/* d psi/d phi_a = sum_b psi_b dh_b/dphi_a = 2 phi_a (psi_a - sum_b h_b psi_b) / sum_b phi_b^2 */
void orc_dpsi(const orc_params *p, const double phi[4], const double mu[2], double T, double out[4])
{
    double h[4], ps[4], S = 0.0, hpsi = 0.0;
    orc_h(phi, h);
    for (int b = 0; b < NPH; b++) S += phi[b] * phi[b];
    for (int b = 0; b < NPH; b++) ps[b] = orc_psi_alpha(p, b, mu, T);
    for (int b = 0; b < NPH; b++) hpsi += h[b] * ps[b];
    for (int a = 0; a < NPH; a++) out[a] = 2.0 * phi[a] * (ps[a] - hpsi) / S;
}

/* R3: gradient energy density a(phi, grad phi); g[b][d] = d phi_b / d x_d */
double orc_a(const orc_params *p, const double phi[4], const double g[4][3])
{
    double r = 0.0;
    for (int a = 0; a < NPH; a++)
        for (int b = a + 1; b < NPH; b++) {
            double q2 = 0.0;
            for (int d = 0; d < 3; d++) {
                double q = phi[a] * g[b][d] - phi[b] * g[a][d];
                q2 += q * q;
            }
            r += gam2(p, a, b) * q2;
        }
    return r;
}

/* da/dphi_a = 2 sum_{b != a} gamma_ab q_ab . grad phi_b */
void orc_dadphi(const orc_params *p, const double phi[4], const double g[4][3], double out[4])
{
    for (int a = 0; a < NPH; a++) {
        double r = 0.0;
        for (int b = 0; b < NPH; b++) {
            if (b == a) continue;
            double qg = 0.0;
            for (int d = 0; d < 3; d++) {
                double q = phi[a] * g[b][d] - phi[b] * g[a][d];
                qg += q * g[b][d];
            }
            r += gam2(p, a, b) * qg;
        }
        out[a] = 2.0 * r;
    }
}

/* da/d(grad phi_a) = -2 sum_{b != a} gamma_ab phi_b q_ab   (a 3-vector per phase) */
void orc_dadgrad(const orc_params *p, const double phi[4], const double g[4][3], double out[4][3])
{
    for (int a = 0; a < NPH; a++)
        for (int d = 0; d < 3; d++) {
            double r = 0.0;
            for (int b = 0; b < NPH; b++) {
                if (b == a) continue;
                double q = phi[a] * g[b][d] - phi[b] * g[a][d];
                r += gam2(p, a, b) * phi[b] * q;
            }
            out[a][d] = -2.0 * r;
        }
}

/* R3: multi-obstacle potential on the simplex */
double orc_omega(const orc_params *p, const double phi[4])
{
    double two = 0.0, three = 0.0;
    for (int a = 0; a < NPH; a++)
        for (int b = a + 1; b < NPH; b++) two += gam2(p, a, b) * phi[a] * phi[b];
    for (int a = 0; a < NPH; a++)
        for (int b = a + 1; b < NPH; b++)
            for (int c = b + 1; c < NPH; c++) three += gam3(p, a, b, c) * phi[a] * phi[b] * phi[c];
    return 16.0 / (ORC_PI * ORC_PI) * two + three;
}

void orc_domega(const orc_params *p, const double phi[4], double out[4])
{
    for (int a = 0; a < NPH; a++) {
        double two = 0.0, three = 0.0;
        for (int b = 0; b < NPH; b++)
            if (b != a) two += gam2(p, a, b) * phi[b];
        for (int b = 0; b < NPH; b++)
            for (int c = b + 1; c < NPH; c++)
                if (b != a && c != a) three += gam3(p, a, b, c) * phi[b] * phi[c];
        out[a] = 16.0 / (ORC_PI * ORC_PI) * two + three;
    }
}

/* R6: Euclidean projection of u onto {sum = 1, phi >= 0} (sort-based). */
void orc_project(const double u[4], double out[4])
{
    double s[4];
    memcpy(s, u, sizeof s);
    /* insertion sort, descending */
    for (int i = 1; i < 4; i++) {
        double x = s[i];
        int j = i - 1;
        while (j >= 0 && s[j] < x) {
            s[j + 1] = s[j];
            j--;
        }
        s[j + 1] = x;
    }
    double csum = 0.0, theta = 0.0;
    for (int j = 0; j < 4; j++) {
        csum += s[j];
        double t = (csum - 1.0) / (double)(j + 1);
        if (s[j] - t > 0.0) theta = t; /* the largest j passing the test wins */
    }
    for (int a = 0; a < 4; a++) {
        double r = u[a] - theta;
        out[a] = r > 0.0 ? r : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* padded copies (one ghost layer: periodic x/y, mirror z)                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nx, ny, nz, nc;
    double *v;
} padded;

static double *pv(const padded *f, int c, int i, int j, int k)
{
    size_t px = (size_t)f->nx + 2, py = (size_t)f->ny + 2, pz = (size_t)f->nz + 2;
    return f->v + (((size_t)c * pz + (size_t)(k + 1)) * py + (size_t)(j + 1)) * px + (size_t)(i + 1);
}

static double pget(const padded *f, int c, int i, int j, int k) { return *pv(f, c, i, j, k); }

static padded make_padded(const double *src, int nc, int nx, int ny, int nz)
{
    padded f = {nx, ny, nz, nc, NULL};
    size_t n = (size_t)nc * (nx + 2) * (ny + 2) * (nz + 2);
    f.v = (double *)malloc(n * sizeof(double));
    for (int c = 0; c < nc; c++)
        for (int k = -1; k <= nz; k++)
            for (int j = -1; j <= ny; j++)
                for (int i = -1; i <= nx; i++) {
                    int si = (i + nx) % nx, sj = (j + ny) % ny;
                    int sk = k < 0 ? 0 : (k >= nz ? nz - 1 : k);
                    *pv(&f, c, i, j, k) = src[(((size_t)c * nz + sk) * ny + sj) * nx + si];
                }
    return f;
}

static void cell4(const padded *f, int i, int j, int k, double out[4])
{
    for (int c = 0; c < NPH; c++) out[c] = pget(f, c, i, j, k);
}

static const int E[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

/* ------------------------------------------------------------------------- */
/* phi-sweep (Eq. 1, Eq. 2, projection)                                       */
/* ------------------------------------------------------------------------- */

/* (da/d grad phi_a)_d at the face between L and R = L + e_d: face average of phi,
 * face difference for the normal derivative (the d-component depends on no other). */
static void face_dadgrad(const orc_params *p, const double phL[4], const double phR[4], int d, double F[4])
{
    double pbar[4], g[4][3], out[4][3];
    for (int b = 0; b < NPH; b++) {
        pbar[b] = 0.5 * (phL[b] + phR[b]);
        for (int e = 0; e < 3; e++) g[b][e] = 0.0;
        g[b][d] = (phR[b] - phL[b]) / p->dx;
    }
    orc_dadgrad(p, pbar, g, out);
    for (int a = 0; a < NPH; a++) F[a] = out[a][d];
}

/* rhs_a of Eq. 2 at cell (i,j,k) of the padded fields. */
static void cell_rhs(const orc_params *p, const padded *ph, const padded *mu, int i, int j, int k, double t,
                     double off, double rhs[4])
{
    double phP[4], div[4] = {0, 0, 0, 0}, g[4][3], dadphi[4], dom[4], dps[4], muP[2];
    cell4(ph, i, j, k, phP);
    for (int d = 0; d < 3; d++) {
        double phPl[4], phMi[4], Fp[4], Fm[4];
        cell4(ph, i + E[d][0], j + E[d][1], k + E[d][2], phPl);
        cell4(ph, i - E[d][0], j - E[d][1], k - E[d][2], phMi);
        face_dadgrad(p, phP, phPl, d, Fp);
        face_dadgrad(p, phMi, phP, d, Fm);
        for (int a = 0; a < NPH; a++) div[a] += (Fp[a] - Fm[a]) / p->dx;
        for (int b = 0; b < NPH; b++) g[b][d] = (phPl[b] - phMi[b]) / (2.0 * p->dx);
    }
    orc_dadphi(p, phP, g, dadphi);
    orc_domega(p, phP, dom);
    double T = orc_temperature(p, ((double)k + off) * p->dx, t);
    muP[0] = pget(mu, 0, i, j, k);
    muP[1] = pget(mu, 1, i, j, k);
    orc_dpsi(p, phP, muP, T, dps);
    for (int a = 0; a < NPH; a++) rhs[a] = p->eps * T * (dadphi[a] - div[a]) + T / p->eps * dom[a] + dps[a];
}

/* phi^{n+1} = Proj(phi^n - dt/(tau eps) (rhs - mean rhs)).  phi_star (optional) receives
 * the value before projection. */
void orc_phi_sweep(const orc_params *p, int nx, int ny, int nz, double t, double off, const double *phi,
                   const double *mu, double *phi_new, double *phi_star, double *rhs_out)
{
    padded ph = make_padded(phi, NPH, nx, ny, nz);
    padded m = make_padded(mu, NMU, nx, ny, nz);
    size_t ncell = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double rhs[4], phP[4], st[4], pr[4];
                cell_rhs(p, &ph, &m, i, j, k, t, off, rhs);
                cell4(&ph, i, j, k, phP);
                double mean = (rhs[0] + rhs[1] + rhs[2] + rhs[3]) / (double)NPH;
                double tau = orc_tau(p, phP);
                for (int a = 0; a < NPH; a++) st[a] = phP[a] - p->dt / (tau * p->eps) * (rhs[a] - mean);
                orc_project(st, pr);
                size_t c0 = ((size_t)k * ny + j) * nx + i;
                for (int a = 0; a < NPH; a++) {
                    phi_new[a * ncell + c0] = pr[a];
                    if (phi_star) phi_star[a * ncell + c0] = st[a];
                    if (rhs_out) rhs_out[a * ncell + c0] = rhs[a];
                }
            }
    free(ph.v);
    free(m.v);
}

/* ------------------------------------------------------------------------- */
/* mu-sweep (Eq. 3, Eq. 4)                                                    */
/* ------------------------------------------------------------------------- */

/* v = M(phi_bar) grad mu - J_at on the face between L=(i,j,k) and R = L + e_d. */
static void face_flux(const orc_params *p, const padded *pn, const padded *po, const padded *mu, int i, int j,
                      int k, int d, double t, double off, double v[2])
{
    int ri = i + E[d][0], rj = j + E[d][1], rk = k + E[d][2];
    double nL[4], nR[4], oL[4], oR[4], pbar[4], mL[2], mR[2], mbar[2], h[4], G[4][3], pdot[4];
    cell4(pn, i, j, k, nL);
    cell4(pn, ri, rj, rk, nR);
    cell4(po, i, j, k, oL);
    cell4(po, ri, rj, rk, oR);
    for (int c = 0; c < NMU; c++) {
        mL[c] = pget(mu, c, i, j, k);
        mR[c] = pget(mu, c, ri, rj, rk);
        mbar[c] = 0.5 * (mL[c] + mR[c]);
    }
    for (int b = 0; b < NPH; b++) pbar[b] = 0.5 * (nL[b] + nR[b]);
    double zf = (double)k + off + (d == 2 ? 0.5 : 0.0);
    double Tf = orc_temperature(p, zf * p->dx, t);

    /* mobility M = sum_a D_a h_a K_a (a 2x2 matrix) */
    orc_h(pbar, h);
    double M[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int a = 0; a < NPH; a++) {
        double K[2][2];
        orc_kmat(p, a, K);
        for (int r = 0; r < NMU; r++)
            for (int c = 0; c < NMU; c++) M[r][c] += p->D[a] * h[a] * K[r][c];
    }
    double flux[2];
    for (int c = 0; c < NMU; c++) flux[c] = (M[c][0] * (mR[0] - mL[0]) + M[c][1] * (mR[1] - mL[1])) / p->dx;

    /* face gradient of phi^{n+1}: normal by difference, tangential by the average of
     * the two cells' central differences (the D3C19 stencil) */
    for (int e = 0; e < 3; e++) {
        if (e == d) {
            for (int b = 0; b < NPH; b++) G[b][e] = (nR[b] - nL[b]) / p->dx;
        } else {
            double lp[4], lm[4], rp[4], rm[4];
            cell4(pn, i + E[e][0], j + E[e][1], k + E[e][2], lp);
            cell4(pn, i - E[e][0], j - E[e][1], k - E[e][2], lm);
            cell4(pn, ri + E[e][0], rj + E[e][1], rk + E[e][2], rp);
            cell4(pn, ri - E[e][0], rj - E[e][1], rk - E[e][2], rm);
            for (int b = 0; b < NPH; b++) G[b][e] = (lp[b] - lm[b] + rp[b] - rm[b]) / (4.0 * p->dx);
        }
    }
    for (int b = 0; b < NPH; b++) pdot[b] = 0.5 * ((nL[b] - oL[b]) + (nR[b] - oR[b])) / p->dt;

    /* anti-trapping current, Eq. 4, with g_a = phi_a */
    double J[2] = {0.0, 0.0};
    double thr = 1e-20 / (p->dx * p->dx);
    double gl2 = G[LIQ][0] * G[LIQ][0] + G[LIQ][1] * G[LIQ][1] + G[LIQ][2] * G[LIQ][2];
    for (int a = 0; a < NPH; a++) {
        if (a == LIQ) continue;
        if (!(pbar[a] > 0.0 && pbar[LIQ] > 0.0)) continue;
        double ga2 = G[a][0] * G[a][0] + G[a][1] * G[a][1] + G[a][2] * G[a][2];
        if (!(ga2 > thr && gl2 > thr)) continue;
        double na = sqrt(ga2), nl = sqrt(gl2);
        double ndot = (G[a][0] * G[LIQ][0] + G[a][1] * G[LIQ][1] + G[a][2] * G[LIQ][2]) / (na * nl);
        double pref = ORC_PI * p->eps / 4.0 * (pbar[a] * h[LIQ] / sqrt(pbar[a] * pbar[LIQ])) * pdot[a] * ndot;
        double cl[2], ca[2];
        orc_c_alpha(p, LIQ, mbar, Tf, cl);
        orc_c_alpha(p, a, mbar, Tf, ca);
        for (int c = 0; c < NMU; c++) J[c] += pref * (cl[c] - ca[c]) * (G[a][d] / na);
    }
    for (int c = 0; c < NMU; c++) v[c] = flux[c] - J[c];
}

/* Flux values on every face, for tests: vout[c][d][k][j][i] is the face between
 * cell (i,j,k) and cell (i,j,k) + e_d (with the boundary rules). */
void orc_face_flux_field(const orc_params *p, int nx, int ny, int nz, double t, double off, const double *phi_old,
                         const double *phi_new, const double *mu, double *vout)
{
    padded pn = make_padded(phi_new, NPH, nx, ny, nz);
    padded po = make_padded(phi_old, NPH, nx, ny, nz);
    padded m = make_padded(mu, NMU, nx, ny, nz);
    size_t ncell = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                for (int d = 0; d < 3; d++) {
                    double v[2];
                    face_flux(p, &pn, &po, &m, i, j, k, d, t, off, v);
                    size_t c0 = ((size_t)k * ny + j) * nx + i;
                    for (int c = 0; c < NMU; c++) vout[((size_t)c * 3 + d) * ncell + c0] = v[c];
                }
    free(pn.v);
    free(po.v);
    free(m.v);
}

void orc_mu_sweep(const orc_params *p, int nx, int ny, int nz, double t, double off, const double *phi_old,
                  const double *phi_new, const double *mu, double *mu_new)
{
    padded pn = make_padded(phi_new, NPH, nx, ny, nz);
    padded po = make_padded(phi_old, NPH, nx, ny, nz);
    padded m = make_padded(mu, NMU, nx, ny, nz);
    size_t ncell = (size_t)nx * ny * nz;
    double dT = -p->G * p->v * p->dt;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double div[2] = {0.0, 0.0};
                for (int d = 0; d < 3; d++) {
                    double vp[2], vm[2];
                    face_flux(p, &pn, &po, &m, i, j, k, d, t, off, vp);
                    face_flux(p, &pn, &po, &m, i - E[d][0], j - E[d][1], k - E[d][2], d, t, off, vm);
                    for (int c = 0; c < NMU; c++) div[c] += (vp[c] - vm[c]) / p->dx;
                }
                double nP[4], oP[4], hN[4], hO[4], muP[2];
                cell4(&pn, i, j, k, nP);
                cell4(&po, i, j, k, oP);
                orc_h(nP, hN);
                orc_h(oP, hO);
                muP[0] = pget(&m, 0, i, j, k);
                muP[1] = pget(&m, 1, i, j, k);
                double T = orc_temperature(p, ((double)k + off) * p->dx, t);
                double chi[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
                for (int a = 0; a < NPH; a++) {
                    double K[2][2];
                    orc_kmat(p, a, K);
                    for (int r = 0; r < NMU; r++)
                        for (int c = 0; c < NMU; c++) chi[r][c] += hN[a] * K[r][c];
                }
                double src[2];
                for (int c = 0; c < NMU; c++) {
                    double dcdphi = 0.0, dcdT = 0.0;
                    for (int a = 0; a < NPH; a++) {
                        double ca[2];
                        orc_c_alpha(p, a, muP, T, ca);
                        dcdphi += ca[c] * (hN[a] - hO[a]);
                        dcdT += hN[a] * p->kT[a][c];
                    }
                    src[c] = p->dt * div[c] - dcdphi - dcdT * dT;
                }
                size_t c0 = ((size_t)k * ny + j) * nx + i;
                /* mu^{n+1} = mu^n + chi^{-1} src, the 2x2 inverse by its adjugate */
                double det = chi[0][0] * chi[1][1] - chi[0][1] * chi[1][0];
                double inc[2];
                inc[0] = (chi[1][1] * src[0] - chi[0][1] * src[1]) / det;
                inc[1] = (chi[0][0] * src[1] - chi[1][0] * src[0]) / det;
                for (int c = 0; c < NMU; c++) mu_new[c * ncell + c0] = muP[c] + inc[c];
            }
    free(pn.v);
    free(po.v);
    free(m.v);
}

/* ------------------------------------------------------------------------- */
/* reductions, window, step, initial condition                                */
/* ------------------------------------------------------------------------- */

/* Phase fractions (mean of phi_a), solute totals sum_cells c (c = sum_a h_a c^a(mu,T)),
 * interface height h = sum (1 - phi_l) / (nx ny), and a non-finite flag. */
void orc_reduce(const orc_params *p, int nx, int ny, int nz, double t, double off, const double *phi,
                const double *mu, double fractions[4], double solute[2], double *h_int, int *nonfinite)
{
    size_t ncell = (size_t)nx * ny * nz, nxy = (size_t)nx * ny;
    double *plane = (double *)calloc((size_t)nz * 8, sizeof(double));
    int *bad = (int *)calloc((size_t)nz, sizeof(int));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++) {
        double *acc = plane + (size_t)k * 8;
        double T = orc_temperature(p, ((double)k + off) * p->dx, t);
        for (size_t q = 0; q < nxy; q++) {
            size_t c0 = (size_t)k * nxy + q;
            double ph[4], h[4], m[2];
            for (int a = 0; a < NPH; a++) ph[a] = phi[a * ncell + c0];
            m[0] = mu[c0];
            m[1] = mu[ncell + c0];
            for (int a = 0; a < NPH; a++)
                if (!isfinite(ph[a])) bad[k] = 1;
            if (!isfinite(m[0]) || !isfinite(m[1])) bad[k] = 1;
            for (int a = 0; a < NPH; a++) acc[a] += ph[a];
            orc_h(ph, h);
            for (int c = 0; c < NMU; c++) {
                double cc = 0.0;
                for (int a = 0; a < NPH; a++) {
                    double ca[2];
                    orc_c_alpha(p, a, m, T, ca);
                    cc += h[a] * ca[c];
                }
                acc[4 + c] += cc;
            }
            acc[6] += 1.0 - ph[LIQ];
        }
    }
    double tot[8] = {0};
    int anybad = 0;
    for (int k = 0; k < nz; k++) {
        for (int q = 0; q < 8; q++) tot[q] += plane[(size_t)k * 8 + q];
        anybad |= bad[k];
    }
    for (int a = 0; a < NPH; a++) fractions[a] = tot[a] / (double)ncell;
    solute[0] = tot[4];
    solute[1] = tot[5];
    *h_int = tot[6] / (double)nxy;
    *nonfinite = anybad;
    free(plane);
    free(bad);
}

/* R11: returns the number of planes shifted (0 if none). */
int orc_window_shift(const orc_params *p, int nx, int ny, int nz, double h_int, double *off, double *phi, double *mu)
{
    if (!(p->window_trigger_z > 0.0) || !(h_int >= p->window_trigger_z)) return 0;
    int s = (int)floor(h_int - p->window_trigger_z) + 1;
    if (s > nz - 1) s = nz - 1;
    if (s <= 0) return 0;
    size_t nxy = (size_t)nx * ny, ncell = nxy * nz;
    double *topmu = (double *)malloc(2 * nxy * sizeof(double));
    for (int c = 0; c < NMU; c++) memcpy(topmu + c * nxy, mu + c * ncell + (size_t)(nz - 1) * nxy, nxy * sizeof(double));
    for (int c = 0; c < NPH; c++) {
        double *f = phi + c * ncell;
        memmove(f, f + (size_t)s * nxy, (size_t)(nz - s) * nxy * sizeof(double));
        for (size_t q = (size_t)(nz - s) * nxy; q < ncell; q++) f[q] = (c == LIQ) ? 1.0 : 0.0;
    }
    for (int c = 0; c < NMU; c++) {
        double *f = mu + c * ncell;
        memmove(f, f + (size_t)s * nxy, (size_t)(nz - s) * nxy * sizeof(double));
        for (int k = nz - s; k < nz; k++) memcpy(f + (size_t)k * nxy, topmu + c * nxy, nxy * sizeof(double));
    }
    free(topmu);
    *off += (double)s;
    return s;
}

/* Algorithm 1 (one explicit step, repeated nsteps times), then t += dt and the
 * window check.  Returns the total number of planes shifted. */
int orc_step(const orc_params *p, int nx, int ny, int nz, double *t, double *off, double *phi, double *mu,
             int nsteps)
{
    size_t ncell = (size_t)nx * ny * nz;
    double *pn = (double *)malloc(NPH * ncell * sizeof(double));
    double *mn = (double *)malloc(NMU * ncell * sizeof(double));
    int shifted = 0;
    for (int n = 0; n < nsteps; n++) {
        orc_phi_sweep(p, nx, ny, nz, *t, *off, phi, mu, pn, NULL, NULL);
        orc_mu_sweep(p, nx, ny, nz, *t, *off, phi, pn, mu, mn);
        memcpy(phi, pn, NPH * ncell * sizeof(double));
        memcpy(mu, mn, NMU * ncell * sizeof(double));
        *t += p->dt;
        if (p->window_trigger_z > 0.0) {
            double fr[4], so[2], h;
            int bad;
            orc_reduce(p, nx, ny, nz, *t, *off, phi, mu, fr, so, &h, &bad);
            shifted += orc_window_shift(p, nx, ny, nz, h, off, phi, mu);
        }
    }
    free(pn);
    free(mn);
    return shifted;
}

/* splitmix64 (Steele, Lea and Flood, 2014): state advances by the golden-ratio
 * increment; the output is the state passed through the variant-13 mixer. */
static uint64_t orc_splitmix64(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_n(uint64_t seed, int n, uint64_t *out)
{
    uint64_t st = seed;
    for (int q = 0; q < n; q++) out[q] = orc_splitmix64(&st);
    return st;
}

static double orc_unit(uint64_t *state) { return (double)(orc_splitmix64(state) >> 11) * (1.0 / 9007199254740992.0); }

/* R13 grain seeds: for grain g, four draws in order give sx = u nx, sy = u ny, sz = u H and
 * phase floor(3u).  seeds[g*4 + 0..2] = position, seeds[g*4+3] = phase. */
void orc_voronoi_seeds(int nx, int ny, int H, int n_grains, uint64_t seed, double *seeds)
{
    uint64_t st = seed;
    for (int g = 0; g < n_grains; g++) {
        seeds[4 * g + 0] = orc_unit(&st) * (double)nx;
        seeds[4 * g + 1] = orc_unit(&st) * (double)ny;
        seeds[4 * g + 2] = orc_unit(&st) * (double)H;
        seeds[4 * g + 3] = floor(3.0 * orc_unit(&st));
    }
}

/* Initial state (Section 2, simulation setting): cells with k < H take the phase of the nearest
 * seed (periodic distance in x and y, plain in z, cell centre at (i+.5, j+.5, k+.5); ties go to the
 * lowest grain index); liquid above; mu = 0.  grain_out (optional) receives the grain index or -1. */
void orc_init(const orc_params *p, int nx, int ny, int nz, uint64_t seed, double *phi, double *mu, int *grain_out)
{
    size_t ncell = (size_t)nx * ny * nz;
    int H = p->seed_layers < nz ? p->seed_layers : nz;
    int ng = p->n_grains;
    double *seeds = (double *)malloc((size_t)(ng > 0 ? ng : 1) * 4 * sizeof(double));
    orc_voronoi_seeds(nx, ny, p->seed_layers, ng, seed, seeds);
    memset(mu, 0, NMU * ncell * sizeof(double));
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c0 = ((size_t)k * ny + j) * nx + i;
                int ph = LIQ, best = -1;
                if (k < H && ng > 0) {
                    double bestd = 0.0;
                    for (int g = 0; g < ng; g++) {
                        double dx = fabs(((double)i + 0.5) - seeds[4 * g + 0]);
                        double dy = fabs(((double)j + 0.5) - seeds[4 * g + 1]);
                        double dz = fabs(((double)k + 0.5) - seeds[4 * g + 2]);
                        if ((double)nx - dx < dx) dx = (double)nx - dx;
                        if ((double)ny - dy < dy) dy = (double)ny - dy;
                        double d2 = dx * dx + dy * dy + dz * dz;
                        if (best < 0 || d2 < bestd) {
                            best = g;
                            bestd = d2;
                        }
                    }
                    ph = (int)seeds[4 * best + 3];
                }
                for (int a = 0; a < NPH; a++) phi[a * ncell + c0] = (a == ph) ? 1.0 : 0.0;
                if (grain_out) grain_out[c0] = best;
            }
    free(seeds);
}

/* Number of OpenMP threads the sweeps use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
#endif
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
