/*
 * fpd_oracle.c -- plain FP64 CPU oracle of the extended fluid particle dynamics
 * (FPD) step of arXiv 2212.14153: bead-spring fibers as smoothed high-viscosity
 * regions in a D2Q9 multiple-relaxation-time lattice Boltzmann fluid.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file; only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library and is deliberately slow and literal:
 *   - populations f_k stored as plain values in two full A/B arrays (pull
 *     streaming), never in-place;
 *   - the MRT collision in explicit 9x9 matrix form m = M f, f* = M^-1 m*;
 *   - a separate velocity-space BGK collision for the equal-rates check;
 *   - bead forces from the case-by-case expressions of Eqs. 11-12;
 *   - per-cell phi/viscosity/force fields stored as arrays.
 * Build with -ffp-contract=off so every rounding is plain IEEE RN.
 *
 * What is followed where (section / equation of the paper):
 *   Eq. 1  viscosity  eta(r) = eta_f + sum_i (eta_s - eta_f) phi_i(r)
 *   Eq. 2  phi_i(r) = 1/2 {tanh[(a - |r - R_i|)/xi] + 1}
 *   Eq. 4  force density f(r) = sum_i phi_i F_i / int phi_i
 *   Eq. 5  bead velocity V_i = int phi_i v / int phi_i
 *   Eq. 9  bead-spring energy (bending term read without the square, the
 *          form whose gradient is Eq. 12)
 *   Eq. 11 spring forces, Eq. 12 bending forces
 *   Sec. 2.3 time-step items (1)-(3): fields from R^n, LBM to v^{n+1},
 *          V^{n+1} from v^{n+1}, R^{n+1} = R^n + dt V^{n+1} (forward Euler)
 *   Sec. 2.3 "MRT collision" + "centered forcing": the paper does not print
 *          the formulas; the Lallemand-Luo D2Q9 moment basis (PRE 61, 6546,
 *          2000) and Guo's forcing (PRE 65, 046308, 2002) are used.
 *   Sec. 4.1 Couette cell: walls at z = 0 and z = H moving at -V0 and +V0,
 *          periodic in x; here the wall-normal axis is called y.
 *   Sec. 3.1 sandwich Couette: static solid layers phi(y) of Eq. 14.
 *   Sec. 3.2 driven particle: a box periodic in x and y, a constant force F_0
 *          on the particle, and eps_v = int phi (v - V_0)^2 / int phi.  The
 *          uniform counter-force -F_0 / (nx ny) on the fluid that keeps the
 *          periodic box from accelerating is the caller's body force (gx, gy).
 * Readings where the paper is silent (the same list is kept with the design
 * notes): half-way moving-wall bounce-back with rho_w = 1; hard phi cutoff at
 * |r - R_i| >= a + phi_cut*xi; minimum-image distance in x; the half-force
 * velocity uses the force of the collision just done; the bead velocity of
 * step n uses phi and S of R^{n-1}; excluded volume (not in the paper) is a
 * harmonic repulsion k_ev (d - r) for non-bonded pairs closer than d.
 *
 * Lattice units throughout: dx = dt = 1, rho_0 = 1, c_s^2 = 1/3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* D2Q9 lattice: rest, four axis and four diagonal velocities.          */
/* ------------------------------------------------------------------ */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Parameters of one simulation (all lattice units). Mirrored by ctypes. */
typedef struct {
    int32_t nx, ny;        /* cells in x (periodic) and y (between the walls) */
    double u_bottom;       /* wall speed at y = 0  (paper: -V0)                */
    double u_top;          /* wall speed at y = H  (paper: +V0)                */
    double nu_f;           /* fluid kinematic viscosity; <= 0: from re        */
    double re;             /* Re = gamma_dot * l_c^2 / nu_f                    */
    double visc_ratio;     /* r_eta = eta_s / eta_f                            */
    double xi;             /* interface thickness                              */
    double a;              /* bead radius; d = l_0 = 2a                        */
    int32_t n_beads;       /* N beads per fiber                                */
    int32_t n_fibers;      /* fibers                                           */
    double k_s;            /* spring constant of Eq. 9; < 0: 0.25*pi*a^2*l0^2  */
    double k_b;            /* bending constant; used when stiffness_K <= 0     */
    double stiffness_K;    /* K = 2 k_b / (eta_f gamma_dot l_c^2), Eq. 18      */
    double k_ev;           /* excluded-volume stiffness; < 0: k_s / l0^2       */
    double phi_cut;        /* support radius a + phi_cut * xi                  */
    double gx, gy;         /* uniform body force density                       */
    int32_t collision;     /* 0 MRT magic rates, 1 MRT Lallemand-Luo, 2 BGK    */
    double s_e, s_eps, s_q;/* constant rates for collision == 1               */
    int32_t init_couette;  /* 1: equilibrium at the linear wall profile       */
    int32_t threads;       /* OpenMP threads for the lattice loops (<=0: 1)   */
    double sandwich_zl;    /* > 0: static solid layers of Eq. 14 below zl ... */
    double sandwich_zr;    /* ... and above zr (interface width xi)           */
    int32_t periodic_y;    /* 1: periodic in y too, no walls (Sec. 3.2)       */
    double bead_fx, bead_fy; /* constant external force on every bead (F_0) */
} orc_params;

typedef struct {
    orc_params p;
    double nu_f, k_s, k_b, k_ev, l0, rcut, gamma_dot;
    int nb;              /* total beads = n_fibers * n_beads */
    long nstep;
    double *f, *ftmp;    /* [9][ny][nx] */
    double *fx, *fy;     /* force density of the current bead table, [ny][nx] */
    double *nu;          /* kinematic viscosity field, [ny][nx] */
    double *R, *V, *F, *S; /* bead table: R,V,F [nb][2], S [nb] */
} orc_sim;

#define IDX(k, j, i, nx, ny) (((size_t)(k) * (size_t)(ny) + (size_t)(j)) * (size_t)(nx) + (size_t)(i))

/* ------------------------------------------------------------------ */
/* Moment basis of Lallemand & Luo (2000): rho, e, eps, jx, qx, jy, qy, */
/* pxx, pxy, each row a polynomial in the lattice velocity.             */
/* ------------------------------------------------------------------ */
void orc_moment_matrix(double *M) {
    for (int k = 0; k < 9; ++k) {
        double cx = CX[k], cy = CY[k], c2 = cx * cx + cy * cy;
        M[0 * 9 + k] = 1.0;
        M[1 * 9 + k] = -4.0 + 3.0 * c2;
        M[2 * 9 + k] = 4.0 - 10.5 * c2 + 4.5 * c2 * c2;
        M[3 * 9 + k] = cx;
        M[4 * 9 + k] = (-5.0 + 3.0 * c2) * cx;
        M[5 * 9 + k] = cy;
        M[6 * 9 + k] = (-5.0 + 3.0 * c2) * cy;
        M[7 * 9 + k] = cx * cx - cy * cy;
        M[8 * 9 + k] = cx * cy;
    }
}

/* The rows of M are mutually orthogonal, so M^-1 = M^T diag(1/|row|^2). */
void orc_inverse_moment_matrix(double *Minv) {
    double M[81], n2[9];
    orc_moment_matrix(M);
    for (int r = 0; r < 9; ++r) {
        n2[r] = 0.0;
        for (int k = 0; k < 9; ++k) n2[r] += M[r * 9 + k] * M[r * 9 + k];
    }
    for (int k = 0; k < 9; ++k)
        for (int r = 0; r < 9; ++r) Minv[k * 9 + r] = M[r * 9 + k] / n2[r];
}

/* Second-order discrete equilibrium in velocity space. */
void orc_feq(double rho, double ux, double uy, double *feq) {
    double u2 = ux * ux + uy * uy;
    for (int k = 0; k < 9; ++k) {
        double cu = CX[k] * ux + CY[k] * uy;
        feq[k] = W[k] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
    }
}

/* Equilibrium moments in the Lallemand-Luo basis (incl. rho u = j). */
void orc_meq(double rho, double ux, double uy, double *meq) {
    double u2 = ux * ux + uy * uy;
    meq[0] = rho;
    meq[1] = -2.0 * rho + 3.0 * rho * u2;
    meq[2] = rho - 3.0 * rho * u2;
    meq[3] = rho * ux;
    meq[4] = -rho * ux;
    meq[5] = rho * uy;
    meq[6] = -rho * uy;
    meq[7] = rho * (ux * ux - uy * uy);
    meq[8] = rho * ux * uy;
}

/* Guo source term in velocity space: w_k [3 (c_k - u) + 9 (c_k.u) c_k] . F */
void orc_guo_velocity(double ux, double uy, double Fx, double Fy, double *S) {
    for (int k = 0; k < 9; ++k) {
        double cu = CX[k] * ux + CY[k] * uy;
        double ex = 3.0 * (CX[k] - ux) + 9.0 * cu * CX[k];
        double ey = 3.0 * (CY[k] - uy) + 9.0 * cu * CY[k];
        S[k] = W[k] * (ex * Fx + ey * Fy);
    }
}

/* The same source written directly in moment space. */
void orc_guo_moment(double ux, double uy, double Fx, double Fy, double *Sm) {
    double uF = ux * Fx + uy * Fy;
    Sm[0] = 0.0;
    Sm[1] = 6.0 * uF;
    Sm[2] = -6.0 * uF;
    Sm[3] = Fx;
    Sm[4] = -Fx;
    Sm[5] = Fy;
    Sm[6] = -Fy;
    Sm[7] = 2.0 * (ux * Fx - uy * Fy);
    Sm[8] = ux * Fy + uy * Fx;
}

/* Relaxation rates per moment: s = (s_rho, s_e, s_eps, s_j, s_q, s_j, s_q,
 * s_nu, s_nu).  s_nu from the local viscosity, nu = (1/s_nu - 1/2)/3. */
void orc_rates(int collision, double nu, double s_e_ll, double s_eps_ll, double s_q_ll, double *s) {
    double s_nu = 1.0 / (3.0 * nu + 0.5);
    double s_e, s_eps, s_q;
    if (collision == 1) {
        s_e = s_e_ll; s_eps = s_eps_ll; s_q = s_q_ll;
    } else {
        /* "magic" two-relaxation-time pairing: even non-conserved moments at
         * s_nu, energy flux at s_q with (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16 */
        s_e = s_nu; s_eps = s_nu;
        s_q = 1.0 / (0.5 + (3.0 / 16.0) / (1.0 / s_nu - 0.5));
    }
    s[0] = 1.0; s[1] = s_e; s[2] = s_eps; s[3] = 1.0; s[4] = s_q;
    s[5] = 1.0; s[6] = s_q; s[7] = s_nu; s[8] = s_nu;
}

/* MRT collision with Guo forcing, explicit matrix form, given M and M^-1. */
static void collide_mrt_with(const double *M, const double *Minv, const double *f, double Fx, double Fy,
                             const double *s, double *out) {
    double m[9], meq[9], Sv[9], Sm[9], ms[9];
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int k = 0; k < 9; ++k) { rho += f[k]; jx += f[k] * CX[k]; jy += f[k] * CY[k]; }
    double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
    for (int r = 0; r < 9; ++r) {
        m[r] = 0.0;
        for (int k = 0; k < 9; ++k) m[r] += M[r * 9 + k] * f[k];
    }
    orc_meq(rho, ux, uy, meq);
    orc_guo_velocity(ux, uy, Fx, Fy, Sv);
    for (int r = 0; r < 9; ++r) {
        Sm[r] = 0.0;
        for (int k = 0; k < 9; ++k) Sm[r] += M[r * 9 + k] * Sv[k];
    }
    for (int r = 0; r < 9; ++r) ms[r] = m[r] - s[r] * (m[r] - meq[r]) + (1.0 - 0.5 * s[r]) * Sm[r];
    for (int k = 0; k < 9; ++k) {
        out[k] = 0.0;
        for (int r = 0; r < 9; ++r) out[k] += Minv[k * 9 + r] * ms[r];
    }
}

void orc_collide_mrt(const double *f, double Fx, double Fy, const double *s, double *out) {
    double M[81], Minv[81];
    orc_moment_matrix(M);
    orc_inverse_moment_matrix(Minv);
    collide_mrt_with(M, Minv, f, Fx, Fy, s, out);
}

/* Single-relaxation-time BGK with Guo forcing, in velocity space only. */
void orc_collide_bgk(const double *f, double Fx, double Fy, double tau, double *out) {
    double feq[9], Sv[9];
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int k = 0; k < 9; ++k) { rho += f[k]; jx += f[k] * CX[k]; jy += f[k] * CY[k]; }
    double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
    orc_feq(rho, ux, uy, feq);
    orc_guo_velocity(ux, uy, Fx, Fy, Sv);
    for (int k = 0; k < 9; ++k) out[k] = f[k] - (f[k] - feq[k]) / tau + (1.0 - 0.5 / tau) * Sv[k];
}

/* ------------------------------------------------------------------ */
/* Derived parameters (Sec. 2.3 and Eq. 18).                           */
/* ------------------------------------------------------------------ */
static void derive(orc_sim *s) {
    const orc_params *p = &s->p;
    s->l0 = 2.0 * p->a;
    s->gamma_dot = (p->u_top - p->u_bottom) / (double)p->ny;
    double lc = p->n_beads * s->l0;
    if (p->nu_f > 0.0) s->nu_f = p->nu_f;
    else s->nu_f = fabs(s->gamma_dot) * lc * lc / p->re;
    s->k_s = (p->k_s < 0.0) ? 0.25 * M_PI * p->a * p->a * s->l0 * s->l0 : p->k_s;
    if (p->stiffness_K > 0.0) s->k_b = p->stiffness_K * s->nu_f * fabs(s->gamma_dot) * lc * lc / 2.0;
    else s->k_b = p->k_b;
    s->k_ev = (p->k_ev < 0.0) ? s->k_s / (s->l0 * s->l0) : p->k_ev;
    s->rcut = p->a + p->phi_cut * p->xi;
}

/* ------------------------------------------------------------------ */
/* Bead-spring forces (Eqs. 9, 11, 12) + excluded volume (extension).   */
/* ------------------------------------------------------------------ */

/* Unit tangent t_k = (R_{k+1} - R_k) / |R_{k+1} - R_k| of segment k
 * (1-based, k = 1..N-1) and its length; zero vector outside that range. */
static void tangent(const double *Rf, int N, int k, double *t, double *len) {
    if (k < 1 || k > N - 1) { t[0] = t[1] = 0.0; *len = 1.0; return; }
    double dx = Rf[2 * k] - Rf[2 * (k - 1)];
    double dy = Rf[2 * k + 1] - Rf[2 * (k - 1) + 1];
    double l = sqrt(dx * dx + dy * dy);
    t[0] = dx / l; t[1] = dy / l; *len = l;
}

/* v . (I - t t) / L  for a vector v and unit tangent t */
static void proj(const double *v, const double *t, double L, double *out) {
    double vt = v[0] * t[0] + v[1] * t[1];
    out[0] = (v[0] - vt * t[0]) / L;
    out[1] = (v[1] - vt * t[1]) / L;
}

static double min_image(double d, double L) { return d - L * floor(d / L + 0.5); }

static void forces_impl(const orc_params *p, double k_s, double k_b, double k_ev, const double *R, double *F) {
    const int N = p->n_beads, NF = p->n_fibers, nb = N * NF;
    const double l0 = 2.0 * p->a;
    for (int b = 0; b < 2 * nb; ++b) F[b] = 0.0;
    for (int fib = 0; fib < NF; ++fib) {
        const double *Rf = R + 2 * fib * N;
        double *Ff = F + 2 * fib * N;
        for (int i = 1; i <= N; ++i) {
            double tm1[2], ti[2], tm2[2], tp1[2], Lm1, Li, Lm2, Lp1;
            tangent(Rf, N, i - 1, tm1, &Lm1);
            tangent(Rf, N, i, ti, &Li);
            tangent(Rf, N, i - 2, tm2, &Lm2);
            tangent(Rf, N, i + 1, tp1, &Lp1);
            double Fs[2] = {0.0, 0.0}, Fb[2] = {0.0, 0.0};
            /* Eq. 11: spring (compression) forces */
            if (N >= 2) {
                if (i == 1) {
                    Fs[0] = k_s / (l0 * l0) * (Li - l0) * ti[0];
                    Fs[1] = k_s / (l0 * l0) * (Li - l0) * ti[1];
                } else if (i == N) {
                    Fs[0] = -k_s / (l0 * l0) * (Lm1 - l0) * tm1[0];
                    Fs[1] = -k_s / (l0 * l0) * (Lm1 - l0) * tm1[1];
                } else {
                    Fs[0] = -k_s / (l0 * l0) * ((Lm1 - l0) * tm1[0] - (Li - l0) * ti[0]);
                    Fs[1] = -k_s / (l0 * l0) * ((Lm1 - l0) * tm1[1] - (Li - l0) * ti[1]);
                }
            }
            /* Eq. 12: bending forces, case by case as printed; tangents of
             * segments that do not exist are zero (so N = 2, 3 are covered). */
            if (N >= 3) {
                double a1[2], a2[2], v[2];
                if (i == 1) {                      /* Eq. 12b */
                    double t2[2], L2; tangent(Rf, N, 2, t2, &L2);
                    proj(t2, ti, Li, a1);
                    Fb[0] = -k_b * a1[0]; Fb[1] = -k_b * a1[1];
                } else if (i == 2) {               /* Eq. 12c */
                    double t1[2], t2[2], t3[2], L1, L2, L3;
                    tangent(Rf, N, 1, t1, &L1); tangent(Rf, N, 2, t2, &L2); tangent(Rf, N, 3, t3, &L3);
                    proj(t2, t1, L1, a1);
                    v[0] = t3[0] + t1[0]; v[1] = t3[1] + t1[1];
                    proj(v, t2, L2, a2);
                    Fb[0] = k_b * (a1[0] - a2[0]); Fb[1] = k_b * (a1[1] - a2[1]);
                } else if (i == N) {               /* Eq. 12e */
                    double tn2[2], tn1[2], Ln2, Ln1;
                    tangent(Rf, N, N - 2, tn2, &Ln2); tangent(Rf, N, N - 1, tn1, &Ln1);
                    proj(tn2, tn1, Ln1, a1);
                    Fb[0] = k_b * a1[0]; Fb[1] = k_b * a1[1];
                } else if (i == N - 1) {           /* Eq. 12d */
                    double tn1[2], tn2[2], tn3[2], Ln1, Ln2, Ln3;
                    tangent(Rf, N, N - 1, tn1, &Ln1); tangent(Rf, N, N - 2, tn2, &Ln2);
                    tangent(Rf, N, N - 3, tn3, &Ln3);
                    v[0] = tn1[0] + tn3[0]; v[1] = tn1[1] + tn3[1];
                    proj(v, tn2, Ln2, a1);
                    proj(tn2, tn1, Ln1, a2);
                    Fb[0] = k_b * (a1[0] - a2[0]); Fb[1] = k_b * (a1[1] - a2[1]);
                } else {                           /* Eq. 12a, interior */
                    v[0] = ti[0] + tm2[0]; v[1] = ti[1] + tm2[1];
                    proj(v, tm1, Lm1, a1);
                    v[0] = tp1[0] + tm1[0]; v[1] = tp1[1] + tm1[1];
                    proj(v, ti, Li, a2);
                    Fb[0] = k_b * (a1[0] - a2[0]); Fb[1] = k_b * (a1[1] - a2[1]);
                }
            }
            Ff[2 * (i - 1)] += Fs[0] + Fb[0];
            Ff[2 * (i - 1) + 1] += Fs[1] + Fb[1];
        }
    }
    /* excluded volume: harmonic repulsion k_ev (d - r) r_hat between beads
     * closer than d = l0 that are not spring-connected */
    if (k_ev != 0.0) {
        for (int b1 = 0; b1 < nb; ++b1) {
            for (int b2 = b1 + 1; b2 < nb; ++b2) {
                int same = (b1 / N) == (b2 / N);
                if (same && (b2 - b1) < 2) continue;
                double dx = min_image(R[2 * b1] - R[2 * b2], (double)p->nx);
                double dy = R[2 * b1 + 1] - R[2 * b2 + 1];
                if (p->periodic_y) dy = min_image(dy, (double)p->ny);
                double r = sqrt(dx * dx + dy * dy);
                if (r < l0 && r > 0.0) {
                    double mag = k_ev * (l0 - r) / r;
                    F[2 * b1] += mag * dx; F[2 * b1 + 1] += mag * dy;
                    F[2 * b2] -= mag * dx; F[2 * b2 + 1] -= mag * dy;
                }
            }
        }
    }
    /* constant external force F_0 on every bead (driven particle, Sec. 3.2) */
    for (int b = 0; b < nb; ++b) {
        F[2 * b] += p->bead_fx;
        F[2 * b + 1] += p->bead_fy;
    }
}

/* Total energy: springs (Eq. 9, first sum) + bending (Eq. 9 second sum
 * without the square, i = 1..N-2) + excluded volume (1/2 k_ev (d - r)^2). */
static double energy_impl(const orc_params *p, double k_s, double k_b, double k_ev, const double *R) {
    const int N = p->n_beads, NF = p->n_fibers, nb = N * NF;
    const double l0 = 2.0 * p->a;
    double U = 0.0;
    for (int fib = 0; fib < NF; ++fib) {
        const double *Rf = R + 2 * fib * N;
        for (int k = 1; k <= N - 1; ++k) {
            double t[2], L; tangent(Rf, N, k, t, &L);
            U += k_s / (2.0 * l0 * l0) * (L - l0) * (L - l0);
        }
        for (int k = 1; k <= N - 2; ++k) {
            double t1[2], t2[2], L1, L2;
            tangent(Rf, N, k, t1, &L1); tangent(Rf, N, k + 1, t2, &L2);
            U -= k_b * (t1[0] * t2[0] + t1[1] * t2[1]);
        }
    }
    for (int b1 = 0; b1 < nb; ++b1)
        for (int b2 = b1 + 1; b2 < nb; ++b2) {
            int same = (b1 / N) == (b2 / N);
            if (same && (b2 - b1) < 2) continue;
            double dx = min_image(R[2 * b1] - R[2 * b2], (double)p->nx);
            double dy = R[2 * b1 + 1] - R[2 * b2 + 1];
            if (p->periodic_y) dy = min_image(dy, (double)p->ny);
            double r = sqrt(dx * dx + dy * dy);
            if (r < l0) U += 0.5 * k_ev * (l0 - r) * (l0 - r);
        }
    /* potential of the constant external force: -F_0 . R */
    for (int b = 0; b < nb; ++b) U -= p->bead_fx * R[2 * b] + p->bead_fy * R[2 * b + 1];
    return U;
}

/* ------------------------------------------------------------------ */
/* Public pure helpers on explicit constants (used by the pins).        */
/* ------------------------------------------------------------------ */
void orc_bead_forces(const orc_params *p, double k_s, double k_b, double k_ev, const double *R, double *F) {
    forces_impl(p, k_s, k_b, k_ev, R, F);
}
double orc_bead_energy(const orc_params *p, double k_s, double k_b, double k_ev, const double *R) {
    return energy_impl(p, k_s, k_b, k_ev, R);
}

/* Eq. 2 with the hard support cutoff, at separation (dx, dy) from R_i. */
static double phi_of(double dx, double dy, double a, double xi, double rcut) {
    double r2 = dx * dx + dy * dy;
    if (r2 >= rcut * rcut) return 0.0;
    double r = sqrt(r2);
    return 0.5 * (tanh((a - r) / xi) + 1.0);
}

/* Eq. 2 for a cell centre (xc, yc), minimum image in x. */
double orc_phi(double a, double xi, double rcut, double nx, double xc, double yc, double Rx, double Ry) {
    return phi_of(min_image(xc - Rx, nx), yc - Ry, a, xi, rcut);
}

/* Eq. 2 for the simulation's geometry: minimum image in x, and in y too
 * when the lattice is periodic in y. */
static double phi_at(const orc_sim *s, double xc, double yc, double Rx, double Ry) {
    double dy = yc - Ry;
    if (s->p.periodic_y) dy = min_image(dy, (double)s->p.ny);
    return phi_of(min_image(xc - Rx, (double)s->p.nx), dy, s->p.a, s->p.xi, s->rcut);
}

/* ------------------------------------------------------------------ */
/* Simulation object.                                                   */
/* ------------------------------------------------------------------ */

/* List every cell whose centre lies within the cutoff of a bead at (Rx, Ry),
 * each cell once (minimum image in x, clipped at the walls in y), with its
 * phi.  Returns the count; the arrays hold at most support_capacity(s). */
static int support_capacity(const orc_sim *s) {  /* cells of the bead's box */
    int w = 2 * ((int)ceil(s->rcut) + 2) + 1;
    int wx = w < s->p.nx ? w : s->p.nx, wy = w < s->p.ny ? w : s->p.ny;
    return wx * wy;
}

static int support_cells(const orc_sim *s, double Rx, double Ry, int *ci, int *cj, double *phi) {
    const int nx = s->p.nx, ny = s->p.ny;
    int j0 = (int)floor(Ry - s->rcut - 0.5) - 1, j1 = (int)ceil(Ry + s->rcut - 0.5) + 1;
    if (s->p.periodic_y) {
        if (j1 - j0 + 1 >= ny) { j0 = 0; j1 = ny - 1; }
    } else {
        if (j0 < 0) j0 = 0;
        if (j1 > ny - 1) j1 = ny - 1;
    }
    int i0 = (int)floor(Rx - s->rcut - 0.5) - 1, i1 = (int)ceil(Rx + s->rcut - 0.5) + 1;
    if (i1 - i0 + 1 >= nx) { i0 = 0; i1 = nx - 1; }
    int n = 0;
    for (int jj = j0; jj <= j1; ++jj)
        for (int ii = i0; ii <= i1; ++ii) {
            int i = ((ii % nx) + nx) % nx;
            int j = ((jj % ny) + ny) % ny;
            double ph = phi_at(s, i + 0.5, j + 0.5, Rx, Ry);
            if (ph == 0.0) continue;
            ci[n] = i; cj[n] = j; phi[n] = ph; ++n;
        }
    return n;
}

/* Item (1) of the time step: phi_i, S_i = int phi_i, F_i, f(r), nu(r) from R. */
static void overlay(orc_sim *s) {
    const int nx = s->p.nx, ny = s->p.ny;
    const size_t ncell = (size_t)nx * ny;
    forces_impl(&s->p, s->k_s, s->k_b, s->k_ev, s->R, s->F);
    double *Phi = (double *)calloc(ncell, sizeof(double));
    for (size_t c = 0; c < ncell; ++c) { s->fx[c] = s->p.gx; s->fy[c] = s->p.gy; }
    int cap = support_capacity(s);
    int *ci = (int *)malloc(cap * sizeof(int)), *cj = (int *)malloc(cap * sizeof(int));
    double *ph = (double *)malloc(cap * sizeof(double));
    for (int b = 0; b < s->nb; ++b) {
        int n = support_cells(s, s->R[2 * b], s->R[2 * b + 1], ci, cj, ph);
        double S = 0.0;
        for (int q = 0; q < n; ++q) S += ph[q];
        s->S[b] = S;
        double gxb = s->F[2 * b] / S, gyb = s->F[2 * b + 1] / S;
        for (int q = 0; q < n; ++q) {
            size_t c = (size_t)cj[q] * nx + ci[q];
            Phi[c] += ph[q];
            s->fx[c] += ph[q] * gxb;
            s->fy[c] += ph[q] * gyb;
        }
    }
    free(ci); free(cj); free(ph);
    /* Sec. 3.1 sandwich benchmark: static solid layers, Eq. 14, in the
     * wall-normal coordinate y (the paper's z), added to the bead profiles */
    if (s->p.sandwich_zl > 0.0) {
        for (int j = 0; j < ny; ++j) {
            double y = j + 0.5, ph;
            if (y <= 0.5 * ny) ph = 0.5 * (tanh((s->p.sandwich_zl - y) / s->p.xi) + 1.0);
            else ph = 0.5 * (tanh((y - s->p.sandwich_zr) / s->p.xi) + 1.0);
            for (int i = 0; i < nx; ++i) Phi[(size_t)j * nx + i] += ph;
        }
    }
    /* Eq. 1 for the kinematic viscosity (rho_0 = 1) */
    for (size_t c = 0; c < ncell; ++c) s->nu[c] = s->nu_f * (1.0 + (s->p.visc_ratio - 1.0) * Phi[c]);
    free(Phi);
}

/* Macroscopic velocity with the half-force shift of the current force field. */
static void velocity_at(const orc_sim *s, int i, int j, double *ux, double *uy, double *rho_out) {
    const int nx = s->p.nx, ny = s->p.ny;
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int k = 0; k < 9; ++k) {
        double fk = s->f[IDX(k, j, i, nx, ny)];
        rho += fk; jx += fk * CX[k]; jy += fk * CY[k];
    }
    size_t c = (size_t)j * nx + i;
    *ux = (jx + 0.5 * s->fx[c]) / rho;
    *uy = (jy + 0.5 * s->fy[c]) / rho;
    if (rho_out) *rho_out = rho;
}

/* Item (3): V_i = int phi_i v / int phi_i with phi, S of the current R,
 * then R <- R + dt V (dt = 1). */
static void advance_beads(orc_sim *s) {
    int cap = support_capacity(s);
    int *ci = (int *)malloc(cap * sizeof(int)), *cj = (int *)malloc(cap * sizeof(int));
    double *ph = (double *)malloc(cap * sizeof(double));
    for (int b = 0; b < s->nb; ++b) {
        int n = support_cells(s, s->R[2 * b], s->R[2 * b + 1], ci, cj, ph);
        double sx = 0.0, sy = 0.0;
        for (int q = 0; q < n; ++q) {
            double ux, uy;
            velocity_at(s, ci[q], cj[q], &ux, &uy, NULL);
            sx += ph[q] * ux;
            sy += ph[q] * uy;
        }
        s->V[2 * b] = sx / s->S[b];
        s->V[2 * b + 1] = sy / s->S[b];
    }
    free(ci); free(cj); free(ph);
    for (int b = 0; b < s->nb; ++b) {
        s->R[2 * b] += s->V[2 * b];
        s->R[2 * b + 1] += s->V[2 * b + 1];
    }
}

static void collide_all(orc_sim *s) {
    const int nx = s->p.nx, ny = s->p.ny;
    const int coll = s->p.collision;
    double M[81], Minv[81];
    orc_moment_matrix(M);
    orc_inverse_moment_matrix(Minv);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double f[9], out[9], rates[9];
            size_t c = (size_t)j * nx + i;
            for (int k = 0; k < 9; ++k) f[k] = s->f[IDX(k, j, i, nx, ny)];
            if (coll == 2) {
                orc_collide_bgk(f, s->fx[c], s->fy[c], 3.0 * s->nu[c] + 0.5, out);
            } else {
                orc_rates(coll, s->nu[c], s->p.s_e, s->p.s_eps, s->p.s_q, rates);
                collide_mrt_with(M, Minv, f, s->fx[c], s->fy[c], rates, out);
            }
            for (int k = 0; k < 9; ++k) s->ftmp[IDX(k, j, i, nx, ny)] = out[k];
        }
    }
}

/* Pull streaming, periodic in x (and in y when periodic_y); a population
 * that would come from beyond a wall is the reflected one of the same cell
 * with the moving-wall term -6 w_k rho_w (c_k . u_w), rho_w = 1, k the
 * direction into the wall. */
static void stream_all(orc_sim *s) {
    const int nx = s->p.nx, ny = s->p.ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            for (int k = 0; k < 9; ++k) {
                int sj = j - CY[k];
                int si = ((i - CX[k]) % nx + nx) % nx;
                if (s->p.periodic_y) sj = (sj % ny + ny) % ny;
                double v;
                if (sj >= 0 && sj < ny) {
                    v = s->ftmp[IDX(k, sj, si, nx, ny)];
                } else {
                    int kw = OPP[k];
                    double uw = (sj < 0) ? s->p.u_bottom : s->p.u_top;
                    v = s->ftmp[IDX(kw, j, i, nx, ny)] - 6.0 * W[kw] * 1.0 * (CX[kw] * uw);
                }
                s->f[IDX(k, j, i, nx, ny)] = v;
            }
        }
    }
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->f); free(s->ftmp); free(s->fx); free(s->fy); free(s->nu);
    free(s->R); free(s->V); free(s->F); free(s->S);
    free(s);
}

/* Create a simulation.  Beads: R0 (nb x 2) if given, else fiber f centred at
 * centres[2f..2f+1] with angle theta0[f] (radians):
 *   R_i = c + (i - (N+1)/2) l0 (cos theta, sin theta),  i = 1..N. */
orc_sim *orc_create(const orc_params *p, const double *R0, const double *centres, const double *theta0) {
    if (p->nx < 1 || p->ny < 1 || p->n_beads < 0 || p->n_fibers < 0) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    derive(s);
    const int nx = p->nx, ny = p->ny;
    const size_t ncell = (size_t)nx * ny;
    s->nb = p->n_beads * p->n_fibers;
    s->f = (double *)calloc(9 * ncell, sizeof(double));
    s->ftmp = (double *)calloc(9 * ncell, sizeof(double));
    s->fx = (double *)calloc(ncell, sizeof(double));
    s->fy = (double *)calloc(ncell, sizeof(double));
    s->nu = (double *)calloc(ncell, sizeof(double));
    int nbm = s->nb > 0 ? s->nb : 1;
    s->R = (double *)calloc(2 * nbm, sizeof(double));
    s->V = (double *)calloc(2 * nbm, sizeof(double));
    s->F = (double *)calloc(2 * nbm, sizeof(double));
    s->S = (double *)calloc(nbm, sizeof(double));
    for (int j = 0; j < ny; ++j) {
        double ux = p->init_couette ? p->u_bottom + (p->u_top - p->u_bottom) * (j + 0.5) / ny : 0.0;
        double feq[9];
        orc_feq(1.0, ux, 0.0, feq);
        for (int i = 0; i < nx; ++i)
            for (int k = 0; k < 9; ++k) s->f[IDX(k, j, i, nx, ny)] = feq[k];
    }
    if (R0) {
        memcpy(s->R, R0, sizeof(double) * 2 * s->nb);
    } else {
        for (int fib = 0; fib < p->n_fibers; ++fib) {
            double cx = centres[2 * fib], cy = centres[2 * fib + 1], th = theta0[fib];
            for (int i = 1; i <= p->n_beads; ++i) {
                double off = (i - (p->n_beads + 1) / 2.0) * s->l0;
                s->R[2 * (fib * p->n_beads + i - 1)] = cx + off * cos(th);
                s->R[2 * (fib * p->n_beads + i - 1) + 1] = cy + off * sin(th);
            }
        }
    }
#ifdef _OPENMP
    omp_set_num_threads(p->threads > 0 ? p->threads : 1);
#endif
    overlay(s);
    return s;
}

/* Advance n steps; each step is items (3) of the previous step [skipped at
 * step 0], then (1), (2): collision + streaming. */
int orc_step(orc_sim *s, long n) {
#ifdef _OPENMP
    omp_set_num_threads(s->p.threads > 0 ? s->p.threads : 1);
#endif
    for (long t = 0; t < n; ++t) {
        if (s->nstep >= 1 && s->nb > 0) {
            advance_beads(s);
            overlay(s);
        }
        collide_all(s);
        stream_all(s);
        s->nstep++;
    }
    return 0;
}

long orc_nstep(const orc_sim *s) { return s->nstep; }

/* Velocity (with the half-force of the current table) and density, [ny][nx]. */
void orc_fields(const orc_sim *s, double *ux, double *uy, double *rho) {
    const int nx = s->p.nx, ny = s->p.ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double a, b, r;
            velocity_at(s, i, j, &a, &b, &r);
            size_t c = (size_t)j * nx + i;
            if (ux) ux[c] = a;
            if (uy) uy[c] = b;
            if (rho) rho[c] = r;
        }
}

void orc_get_populations(const orc_sim *s, double *f) {
    memcpy(f, s->f, sizeof(double) * 9 * (size_t)s->p.nx * s->p.ny);
}
void orc_set_populations(orc_sim *s, const double *f) {
    memcpy(s->f, f, sizeof(double) * 9 * (size_t)s->p.nx * s->p.ny);
}

/* Force-density and viscosity fields of the current bead table, [ny][nx]. */
void orc_overlay_fields(const orc_sim *s, double *fx, double *fy, double *nu) {
    size_t n = (size_t)s->p.nx * s->p.ny;
    if (fx) memcpy(fx, s->fx, n * sizeof(double));
    if (fy) memcpy(fy, s->fy, n * sizeof(double));
    if (nu) memcpy(nu, s->nu, n * sizeof(double));
}

void orc_beads(const orc_sim *s, double *R, double *V, double *F, double *S) {
    if (R) memcpy(R, s->R, sizeof(double) * 2 * s->nb);
    if (V) memcpy(V, s->V, sizeof(double) * 2 * s->nb);
    if (F) memcpy(F, s->F, sizeof(double) * 2 * s->nb);
    if (S) memcpy(S, s->S, sizeof(double) * s->nb);
}

/* mass = sum f; momentum = sum f c (no half-force) */
void orc_totals(const orc_sim *s, double *out3) {
    const int nx = s->p.nx, ny = s->p.ny;
    double m = 0.0, px = 0.0, py = 0.0;
    for (int k = 0; k < 9; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double v = s->f[IDX(k, j, i, nx, ny)];
                m += v; px += v * CX[k]; py += v * CY[k];
            }
    out3[0] = m; out3[1] = px; out3[2] = py;
}

/* Strength of the residual flow inside each bead (Sec. 3.2):
 *   eps_v = sum_x phi_i (v - V_i)^2 / sum_x phi_i
 * with v the fluid velocity of orc_fields, phi_i and the sums over the
 * bead's support at its current R_i, and V_i its latest velocity. */
void orc_internal_flow(const orc_sim *s, double *eps) {
    int cap = support_capacity(s);
    int *ci = (int *)malloc(cap * sizeof(int)), *cj = (int *)malloc(cap * sizeof(int));
    double *ph = (double *)malloc(cap * sizeof(double));
    for (int b = 0; b < s->nb; ++b) {
        int n = support_cells(s, s->R[2 * b], s->R[2 * b + 1], ci, cj, ph);
        double num = 0.0, den = 0.0;
        for (int q = 0; q < n; ++q) {
            double ux, uy;
            velocity_at(s, ci[q], cj[q], &ux, &uy, NULL);
            double dx = ux - s->V[2 * b], dy = uy - s->V[2 * b + 1];
            num += ph[q] * (dx * dx + dy * dy);
            den += ph[q];
        }
        eps[b] = num / den;
    }
    free(ci); free(cj); free(ph);
}

/* nu_f, k_s, k_b, k_ev, l0, rcut, gamma_dot */
void orc_derived(const orc_sim *s, double *out7) {
    out7[0] = s->nu_f; out7[1] = s->k_s; out7[2] = s->k_b; out7[3] = s->k_ev;
    out7[4] = s->l0; out7[5] = s->rcut; out7[6] = s->gamma_dot;
}
