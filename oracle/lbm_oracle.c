/*
 * Plain FP64 CPU oracle of the consistent double-distribution lattice Boltzmann
 * model with body force and heat source (arxiv 2609.28679).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, loads or calls it, and it shares no code,
 * header, table or constant with the CUDA sources.
 *
 * One time step follows the paper's flowchart (Sec. II.E, Fig. "Structure of
 * the algorithm") in order, with every intermediate field held in a full-size
 * array so that each phase can be read against its equation:
 *
 *   A  rho = sum_i f_i,  J = sum_i c_i f_i,  G = sum_i g_i        (Eq. def_h)
 *   B  F = rho*a + F_K,  F_K = kappa rho grad(lap rho);  Q(x)    (Eqs. force_decomposition, korteweg_force)
 *   C  u = (J + F/2)/rho;  rho E = G + (u.F + Q)/2;  T(rho,e);  P   (Eqs. def_u, def_E, TdependsongenericEOS)
 *      theta = P/rho (Eq. theta), c_s^2, gamma, alpha (Eqs. corr_bulk, corr_heat_source)
 *   D  u*, theta*, Phi, T*, q^c                                   (Eqs. sh_vel_1, sh_temp_1, correction, sh_T_1, qc_1)
 *   E  f^eq, f*, g^eq, g*  (Eqs. LBMeq, LBMstar, LBMeqG, LBMgstar); beta (Eq. beta);
 *      collide and stream (Eqs. LBM_f, LBM_g) with lambda = dt = 1.
 *
 * Lattice units: dt = dx = c = 1, varsigma^2 = 1/3 (Eq. cs).  D = 3 uses the
 * paper's D3Q27 set (Eq. D3Q27c); D = 2 uses its tensor-product restriction
 * D2Q9 (the paper names no 2-D set).
 *
 * Readings of points the paper leaves open:
 *  - beta = 1/(2 tau + 1) with a constant tau per distribution (Eq. beta); the
 *    shear viscosity mu = tau P then follows the local pressure.  eta and k
 *    enter only through the ratios eta/mu and k/mu.  With mu > 0 the paper's
 *    own parameterisation is used instead: tau = mu / P of the cell (Sec. II.C,
 *    the relation after Eq. theta), the same tau for f and g, and beta per
 *    cell in the collision (flowchart, last box).
 *  - isothermal = 1 follows the isothermal tests of Sec. III.A, where the g
 *    equation is not solved: each cell keeps its initial temperature, the
 *    specific energy is e(rho, T) of the EoS, and g is left as initialised.
 *  - alpha*theta is evaluated as ((D+2)/D - eta/mu) theta - c_s^2, which equals
 *    alpha*theta of Eq. corr_bulk with theta = P/rho but has no removable
 *    singularity where P = 0 (spinodal region of van der Waals / Peng-Robinson).
 *  - The upwind-biased first derivative in Eq. correction (Sec. II.E, chosen
 *    there to make higher Mach numbers stable) is the third-order
 *    upwind-biased difference, two points on the side the local u_alpha comes
 *    from and one on the other: (2 X_{+1} + 3 X_0 - 6 X_{-1} + X_{-2}) / 6 for
 *    u >= 0, mirrored for u < 0.  The linear stability of uniform flow under
 *    this step (oracle/stability.py) singles it out: it keeps uniform flow
 *    stable to Ma 1.2 at theta = 0.1 where the central difference fails above
 *    Ma 0.9, while the fully one-sided second-order difference is unstable at
 *    every Mach number.  With phi_central = 1 the 2-point central difference
 *    is used (the liquid-vapour cases).  Laplacian and gradients are the
 *    standard (2D+1)-point and 2-point central differences (Sec. II.E).
 *  - Half-way bounce-back walls at the z faces (Sec. III.A, Poiseuille) act on
 *    both f and g.  For the macroscopic stencils, cells beyond a wall mirror
 *    the interior: scalars (rho, lap rho, T, h) even, velocity odd, so X_z is
 *    odd.
 *  - zwalls = 2, the non-equilibrium-extrapolation walls of App. B (thermal
 *    Couette): the walls lie on the boundary cells z = 0 and z = nz - 1 (B),
 *    whose neighbours N are z = 1 and z = nz - 2.  After phases A-C of a step
 *    (all cells, from their current populations), every B cell is rebuilt:
 *    u_B = u_W, T_B = T_W, f_B = f^eq(rho_B, u_W, theta_W) +
 *    f_N - f^eq(rho_N, u_N, theta_N) and g_B alike, with theta_W = P(rho_B,
 *    T_W)/rho_B and e_W = e(rho_B, T_W).  The text extrapolates rho_B =
 *    rho_N (wall_rho = 1); where T_W differs from T_N that sets a pressure
 *    step P_B - P_N across the wall link, mass leaks through the wall and the
 *    thermal Couette profile misses the paper's analytic one by a margin that
 *    does not shrink with resolution.  The default (wall_rho = 0) extrapolates
 *    the pressure instead, rho_B solving P(rho_B, T_W) = P(rho_N, T_N) by
 *    eight Newton steps from rho_N (rho_N again if that ends non-finite or
 *    non-positive), which is the text's rho_B = rho_N wherever T_W = T_N and
 *    converges to the analytic profile at second order.  With a force normal
 *    to the wall (the cross-flow Poiseuille flow of Sec. III.A) the pressure
 *    is not uniform at rest, P_B = P_N sets a pressure step against it and the
 *    channel again leaks; wall_rho = 2 extrapolates the pressure linearly from
 *    the two cells inside, P_B = 2 P_N - P_NN, which is P_N where the pressure
 *    is uniform and keeps the wall tight under any smooth pressure gradient.
 *    Its phase-C fields become those of
 *    the wall state and its force keeps the per-mass value of phase B
 *    (F_B scaled by the new rho_B over the old).  Phases D-E then run on all
 *    cells, B included.  A stencil reaching past a wall takes the value
 *    extrapolated linearly through the boundary cell, v(z_B - m) =
 *    2 v(z_B) - v(z_B + m) (mirrored for the upper wall), for every field.
 *    Populations streaming out through a wall face return reversed (as with
 *    zwalls = 1); B is rebuilt before they are used.  The moments reported
 *    for a B cell are the rebuilt ones.  Not combined with isothermal = 1.
 *  - Duct ends (Sec. III.A, Rayleigh and Fanno flows) reuse the boundary-cell
 *    rebuild with other boundary states (face_kind): a subsonic inlet takes
 *    the total pressure P0 and temperature T0 with the velocity of its
 *    neighbour, T = T0 - |u|^2/(2 c_p), P = P0 (T/T0)^(c_p/R) (ideal gas with
 *    constant c_v only); a supersonic inlet takes static P, T and u; a
 *    subsonic outlet takes static P with u and T of the neighbour; a
 *    supersonic outlet takes rho, u and T of the neighbour.  Where P and T are
 *    given, rho_B solves P(rho_B, T) = P by the same eight Newton steps.
 *    "Zero-order extrapolation" at the subsonic outlet is read as carrying
 *    over the neighbour's mass flux, u_B = u_N rho_N / rho_B: carrying u_N
 *    itself leaves a pressure step of ~15 % in the last cells and an energy
 *    flux that misses the heat input (Rayleigh flow), while the mass flux
 *    gives a smooth outlet and the Rayleigh and Fanno relations to 1e-4.
 *    The boundary cell's force and heat keep their non-friction part per
 *    unit mass; the friction force and its heat are evaluated again at the
 *    rebuilt (rho_B, u_B).  The
 *    text's 1-D duct runs as a 1 x 1 x nz column of D3Q27: with no x or y
 *    variation its populations summed over c_x, c_y follow the 1-D product
 *    form of the same model exactly, except that the normal viscous stress
 *    is the 3-D one, (4/3 mu + eta) du/dz (both are regularisers of the
 *    inviscid Rayleigh and Fanno solutions).
 *  - Duct resistance: the friction of Fanno flow F_f = -k rho |u| u (k =
 *    f_D/(2 D_h)) and the Darcy throttle of the throttling process F_t =
 *    -K phi(z) rho u (phi a Gaussian of width sigma at the middle of the
 *    duct), with the compensating heat Q_r = -F_r.u, added to F and Q of
 *    phase B.  u = (J + F/2)/rho then depends on F_r; the relation is solved
 *    exactly: with w = (J + (F_B + F_K)/2)/rho and a = 1 + K phi/2,
 *    |u| (a + k |u|/2) = |w|, so u = 2 w / (a + sqrt(a^2 + 2 k |w|)).
 *    The throttling inlet (face kind 5) holds static P and T with the
 *    neighbour's velocity.
 *  - Peng-Robinson: the paper names the model only.  The textbook form with the
 *    Soave alpha(T) and a constant ideal-part c_v is used; e(rho,T) follows by
 *    integrating Eq. de_rho at constant T from rho = 0.  T(rho,e) is found by
 *    Newton's method in T from the previous step's T (from Tc when there is
 *    none), stopping at |dT| <= 1e-14 T, at most 50 iterations (hits of the
 *    cap are counted).
 *  - c_v in Eq. sh_T_1 is the local (de/dT)_rho.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_IDEAL 0
#define ORC_VDW 1
#define ORC_PR 2

typedef struct {
    int dim;            /* 2 or 3 */
    int nx, ny, nz;     /* nz = 1 when dim = 2 */
    int zwalls;         /* 0: periodic in z; 1: half-way bounce-back walls at both z faces;
                           2: non-equilibrium-extrapolation walls on the cells z = 0 and z = nz - 1 */
    int eos;            /* ORC_IDEAL, ORC_VDW, ORC_PR */
    double R, cv;       /* gas constant; constant (ideal-part) specific heat */
    double a, b;        /* vdW / PR attraction and co-volume */
    double Tc, omega;   /* PR critical temperature and acentric factor */
    double kappa;       /* Korteweg capillarity coefficient */
    double eta_over_mu; /* bulk / shear viscosity ratio */
    double k_over_mu;   /* conductivity / shear viscosity ratio */
    double tau_f, tau_g;
    double accel[3];    /* body acceleration: F_B = rho * accel */
    double q;           /* volumetric heat source Q */
    int zlo, zhi;       /* Q acts where zlo <= z < zhi; zhi <= 0 means everywhere */
    int phi_central;    /* 0: upwind-biased derivative in Phi; 1: central difference;
                           2-5: other stencils, for the stability analysis only */
    double mu;          /* > 0: the paper's tau = mu / P per cell (Sec. II.C), one tau for f and g;
                           0: constant tau_f, tau_g */
    int isothermal;     /* 1: the g equation is not solved (Sec. III.A, isothermal tests); every cell
                           keeps its initial temperature, e = e(rho, T) from the EoS */
    double uw_lo[3], uw_hi[3]; /* zwalls = 2: velocities of the walls at z = 0 and z = nz - 1 */
    double Tw_lo, Tw_hi;       /* zwalls = 2: their temperatures */
    int wall_rho;              /* zwalls = 2: 0: rho_B from P(rho_B, T_W) = P_N; 1: rho_B = rho_N;
                                  2: rho_B from P(rho_B, T_W) = 2 P_N - P_NN (NN: two cells in) */
    int face_kind[2];          /* zwalls = 2: ORC_FACE_* of the faces z = 0 and z = nz - 1; walls take
                                  (uw, Tw) above, the open kinds take (uw, Tw, face_P) as their data */
    double face_P[2];          /* static pressure (inlet static, outlet) or total pressure (inlet total) */
    double friction;           /* duct friction k = f_D / (2 D_h): F = -k rho |u| u, with Q = -F.u */
    double throttle_K;         /* throttle (Sec. III.B, throttling): F = -K phi(z) rho u, with Q = -F.u, */
    double throttle_sigma;     /* phi(z) = exp(-((z - (nz - 1)/2) / sigma)^2)  (dim 3) */
} orc_params;

/* Boundary kinds of a z face with zwalls = 2 (App. B walls; Sec. III.A duct ends) */
#define ORC_FACE_WALL 0          /* wall: u_W, T_W; rho_B by wall_rho */
#define ORC_FACE_INLET_TOTAL 1   /* subsonic inlet: total P0, T0 given, u from the neighbour (ideal gas) */
#define ORC_FACE_INLET_STATIC 2  /* supersonic inlet: static P, T and u given */
#define ORC_FACE_OUTLET_P 3      /* subsonic outlet: static P given, u and T from the neighbour */
#define ORC_FACE_OUTLET_EXTRAP 4 /* supersonic outlet: rho, u, T from the neighbour */
#define ORC_FACE_INLET_PT 5      /* inlet with static P and T given, u from the neighbour (throttling) */

typedef struct {
    orc_params p;
    int Q;
    long N;
    int c[27][3];
    int opp[27];
    double *f, *g, *fn, *gn;         /* populations [Q][N] and the streaming targets */
    double *rho, *J, *G;             /* phase A */
    double *lap, *F, *Qs;            /* phase B */
    double *u, *T, *P, *theta, *h, *cvl, *gam, *athe, *E, *e; /* phase C */
    double *X;                       /* phase D helper: X_alpha = rho u_alpha^3 + 3 rho u_alpha (theta - 1/3) */
    double *Ffield, *Qfield;         /* optional per-cell body force F_B [3][N] and heat source [N] (or NULL) */
    long newton_cap_hits;
    long theta_nonpos;
} orc_state;

/* ------------------------------------------------------------------------- */
/* Lattice (Eq. D3Q27c; D2Q9 is its restriction to two axes).                */
/* Direction i has base-3 digits (d_x, d_y, d_z); digit 0,1,2 -> c = 0,+1,-1. */
/* ------------------------------------------------------------------------- */
static int digit_to_c(int d) { return d == 0 ? 0 : (d == 1 ? 1 : -1); }

int orc_lattice(int dim, int *c_out /* [27*3] */, int *opp_out /* [27] */)
{
    int Q = (dim == 2) ? 9 : 27;
    for (int i = 0; i < Q; ++i) {
        int d0 = i % 3, d1 = (i / 3) % 3, d2 = (i / 9) % 3;
        c_out[3 * i + 0] = digit_to_c(d0);
        c_out[3 * i + 1] = digit_to_c(d1);
        c_out[3 * i + 2] = dim == 3 ? digit_to_c(d2) : 0;
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            if (c_out[3 * j] == -c_out[3 * i] && c_out[3 * j + 1] == -c_out[3 * i + 1] &&
                c_out[3 * j + 2] == -c_out[3 * i + 2])
                opp_out[i] = j;
    return Q;
}

/* ------------------------------------------------------------------------- */
/* Product-form factor, Eq. phi:                                              */
/*   Psi(c; xi, zeta) = 1 - c^2 + ( (3c^2 - 2) zeta + c xi ) / 2             */
/* ------------------------------------------------------------------------- */
double orc_psi(int c, double xi, double zeta)
{
    double c2 = (double)(c * c);
    return 1.0 - c2 + 0.5 * ((3.0 * c2 - 2.0) * zeta + (double)c * xi);
}

/* f_i = rho prod_alpha Psi(c_i alpha; xi_alpha, zeta_alpha).
 * Eq. LBMeq with xi = u, zeta = theta + u^2; Eq. LBMstar with xi = u*,
 * zeta = theta* + u*^2 + Phi.  The caller supplies xi and zeta per axis. */
void orc_fprod(int dim, double rho, const double *xi, const double *zeta, double *out)
{
    int c[81], opp[27];
    int Q = orc_lattice(dim, c, opp);
    for (int i = 0; i < Q; ++i) {
        double v = rho;
        for (int a = 0; a < dim; ++a) v *= orc_psi(c[3 * i + a], xi[a], zeta[a]);
        out[i] = v;
    }
}

/* g^eq_i (Eq. LBMeqG): the product of Psi(c_alpha; O_alpha, O_alpha^2) applied to
 * the generating function E = e + |u|^2/2 (Eq. Egen), with
 * O_alpha = theta d/du_alpha + u_alpha (Eq. Oa).  The operators of different
 * axes commute and e does not depend on u, so the product splits:
 *   O 1 = u,  O^2 1 = theta + u^2                      -> Psi(c; u, theta + u^2) =: P0
 *   O (u^2/2) = theta u + u^3/2,
 *   O^2 (u^2/2) = theta^2 + (5/2) theta u^2 + u^4/2    -> H := Psi applied to u^2/2
 *   g_i = rho [ e prod_a P0_a + sum_b H_b prod_{a != b} P0_a ].
 * The test suite checks this expansion against direct symbolic application of
 * the operators. */
void orc_geq(int dim, double rho, const double *u, double e, double theta, double *out)
{
    int c[81], opp[27];
    int Q = orc_lattice(dim, c, opp);
    for (int i = 0; i < Q; ++i) {
        double P0[3], H[3];
        for (int a = 0; a < dim; ++a) {
            int ca = c[3 * i + a];
            double ua = u[a];
            P0[a] = orc_psi(ca, ua, theta + ua * ua);
            double o1 = theta * ua + 0.5 * ua * ua * ua;
            double o2 = theta * theta + 2.5 * theta * ua * ua + 0.5 * ua * ua * ua * ua;
            double c2 = (double)(ca * ca);
            H[a] = (1.0 - c2) * 0.5 * ua * ua + 0.5 * ((3.0 * c2 - 2.0) * o2 + (double)ca * o1);
        }
        double prod = 1.0;
        for (int a = 0; a < dim; ++a) prod *= P0[a];
        double sum = e * prod;
        for (int b = 0; b < dim; ++b) {
            double t = H[b];
            for (int a = 0; a < dim; ++a)
                if (a != b) t *= P0[a];
            sum += t;
        }
        out[i] = rho * sum;
    }
}

/* ------------------------------------------------------------------------- */
/* Equations of state                                                         */
/*   ideal (Eq. idealEOS):  P = rho R T,                      e = cv T       */
/*   vdW   (Eq. vdw_eos):   P = rho R T/(1 - b rho) - a rho^2, e = cv T - a rho */
/*   PR    (textbook, Soave alpha):                                          */
/*     P = rho R T/(1 - b rho) - a al(T) rho^2 / (1 + 2 b rho - b^2 rho^2),   */
/*     al(T) = (1 + k (1 - s))^2,  s = sqrt(T/Tc),                           */
/*     k = 0.37464 + 1.54226 omega - 0.26992 omega^2,                        */
/*     e = cv T - a (1 + k)(1 + k - k s) Lam(rho), where Lam(rho) is the      */
/*     integral of 1/(1 + 2 b r - b^2 r^2) from 0 to rho, which makes         */
/*     de = cv dT - [T dP/dT - P] drho/rho^2 (Eq. de_rho) hold exactly.       */
/* ------------------------------------------------------------------------- */
static double pr_k(const orc_params *p)
{
    return 0.37464 + 1.54226 * p->omega - 0.26992 * p->omega * p->omega;
}

static double pr_lambda(const orc_params *p, double rho)
{
    double s2 = sqrt(2.0);
    double br = p->b * rho;
    return log((1.0 + (1.0 + s2) * br) / (1.0 + (1.0 - s2) * br)) / (2.0 * s2 * p->b);
}

double orc_eos_P(const orc_params *p, double rho, double T)
{
    switch (p->eos) {
    case ORC_IDEAL:
        return rho * p->R * T;
    case ORC_VDW:
        return rho * p->R * T / (1.0 - p->b * rho) - p->a * rho * rho;
    default: {
        double k = pr_k(p);
        double s = sqrt(T / p->Tc);
        double al = (1.0 + k * (1.0 - s)) * (1.0 + k * (1.0 - s));
        double br = p->b * rho;
        return rho * p->R * T / (1.0 - br) - p->a * al * rho * rho / (1.0 + 2.0 * br - br * br);
    }
    }
}

double orc_eos_e(const orc_params *p, double rho, double T)
{
    switch (p->eos) {
    case ORC_IDEAL:
        return p->cv * T;
    case ORC_VDW:
        return p->cv * T - p->a * rho;
    default: {
        double k = pr_k(p);
        double s = sqrt(T / p->Tc);
        return p->cv * T - p->a * (1.0 + k) * (1.0 + k - k * s) * pr_lambda(p, rho);
    }
    }
}

/* (dP/dT) at constant rho */
double orc_eos_dPdT(const orc_params *p, double rho, double T)
{
    switch (p->eos) {
    case ORC_IDEAL:
        return rho * p->R;
    case ORC_VDW:
        return rho * p->R / (1.0 - p->b * rho);
    default: {
        double k = pr_k(p);
        double s = sqrt(T / p->Tc);
        /* d al/dT = 2 (1 + k(1-s)) (-k) / (2 s Tc) */
        double dal = -(1.0 + k * (1.0 - s)) * k / (s * p->Tc);
        double br = p->b * rho;
        return rho * p->R / (1.0 - br) - p->a * dal * rho * rho / (1.0 + 2.0 * br - br * br);
    }
    }
}

/* (dP/drho) at constant T */
double orc_eos_dPdrho(const orc_params *p, double rho, double T)
{
    switch (p->eos) {
    case ORC_IDEAL:
        return p->R * T;
    case ORC_VDW: {
        double d = 1.0 - p->b * rho;
        return p->R * T / (d * d) - 2.0 * p->a * rho;
    }
    default: {
        double k = pr_k(p);
        double s = sqrt(T / p->Tc);
        double al = (1.0 + k * (1.0 - s)) * (1.0 + k * (1.0 - s));
        double b = p->b;
        double d1 = 1.0 - b * rho;
        double den = 1.0 + 2.0 * b * rho - b * b * rho * rho;
        /* d/drho [rho^2/den] = (2 rho den - rho^2 (2b - 2 b^2 rho)) / den^2 */
        double dq = (2.0 * rho * den - rho * rho * (2.0 * b - 2.0 * b * b * rho)) / (den * den);
        return p->R * T / (d1 * d1) - p->a * al * dq;
    }
    }
}

/* c_v = (de/dT) at constant rho */
double orc_eos_cv(const orc_params *p, double rho, double T)
{
    if (p->eos != ORC_PR) return p->cv;
    double k = pr_k(p);
    double s = sqrt(T / p->Tc);
    /* d/dT [ -a (1+k)(1+k-k s) Lam ] = a (1+k) k Lam ds/dT,  ds/dT = 1/(2 s Tc) */
    return p->cv + p->a * (1.0 + k) * k * pr_lambda(p, rho) / (2.0 * s * p->Tc);
}

/* T from (rho, e).  Ideal and vdW: the explicit inversions of Eqs. idealgasT
 * and lbm_temp.  PR: Newton's method on e(rho,T) - e = 0 in T, started from
 * T_guess.  *iters receives the iteration count (cap 50). */
double orc_eos_T(const orc_params *p, double rho, double e, double T_guess, int *iters)
{
    if (iters) *iters = 0;
    switch (p->eos) {
    case ORC_IDEAL:
        return e / p->cv;
    case ORC_VDW:
        return (e + p->a * rho) / p->cv;
    default: {
        /* without a previous T (T_guess <= 0) start from the critical temperature */
        double T = T_guess > 0.0 ? T_guess : p->Tc;
        int it;
        for (it = 1; it <= 50; ++it) {
            double r = orc_eos_e(p, rho, T) - e;
            double dT = -r / orc_eos_cv(p, rho, T);
            T += dT;
            if (fabs(dT) <= 1e-14 * fabs(T)) break;
        }
        if (iters) *iters = it;
        return T;
    }
    }
}

/* vdW constants from critical data (Sec. III.B): a = 27 R^2 Tc^2/(64 Pc), b = R Tc/(8 Pc) */
void orc_vdw_from_critical(double R, double Tc, double Pc, double *a, double *b)
{
    *a = 27.0 * R * R * Tc * Tc / (64.0 * Pc);
    *b = R * Tc / (8.0 * Pc);
}

/* PR constants from critical data (textbook): a = 0.45724 R^2 Tc^2/Pc, b = 0.07780 R Tc/Pc */
void orc_pr_from_critical(double R, double Tc, double Pc, double *a, double *b)
{
    *a = 0.45724 * R * R * Tc * Tc / Pc;
    *b = 0.07780 * R * Tc / Pc;
}

/* ------------------------------------------------------------------------- */
/* State                                                                      */
/* ------------------------------------------------------------------------- */
static double *zalloc(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

orc_state *orc_create(const orc_params *p)
{
    if (!p || (p->dim != 2 && p->dim != 3) || p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->dim == 2 && (p->nz != 1 || p->zwalls)) return NULL;
    if (p->zwalls < 0 || p->zwalls > 2) return NULL;
    if (p->zwalls == 2 && (p->nz < 4 || p->isothermal || !(p->Tw_lo > 0) || !(p->Tw_hi > 0))) return NULL;
    if (p->wall_rho < 0 || p->wall_rho > 2) return NULL;
    for (int f = 0; f < 2; ++f) {
        if (p->face_kind[f] < ORC_FACE_WALL || p->face_kind[f] > ORC_FACE_INLET_PT) return NULL;
        if (p->face_kind[f] != ORC_FACE_WALL && p->zwalls != 2) return NULL;
        if (p->face_kind[f] == ORC_FACE_INLET_TOTAL && p->eos != ORC_IDEAL) return NULL;
        if ((p->face_kind[f] == ORC_FACE_INLET_TOTAL || p->face_kind[f] == ORC_FACE_INLET_STATIC ||
             p->face_kind[f] == ORC_FACE_OUTLET_P || p->face_kind[f] == ORC_FACE_INLET_PT) && !(p->face_P[f] > 0))
            return NULL;
    }
    if (!(p->friction >= 0) || !(p->throttle_K >= 0)) return NULL;
    if (p->throttle_K > 0 && (p->dim != 3 || !(p->throttle_sigma > 0))) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    s->p = *p;
    int cflat[81];
    s->Q = orc_lattice(p->dim, cflat, s->opp);
    for (int i = 0; i < s->Q; ++i)
        for (int a = 0; a < 3; ++a) s->c[i][a] = cflat[3 * i + a];
    s->N = (long)p->nx * p->ny * p->nz;
    long N = s->N, Q = s->Q;
    s->f = zalloc(Q * N); s->g = zalloc(Q * N);
    s->fn = zalloc(Q * N); s->gn = zalloc(Q * N);
    s->rho = zalloc(N); s->J = zalloc(3 * N); s->G = zalloc(N);
    s->lap = zalloc(N); s->F = zalloc(3 * N); s->Qs = zalloc(N);
    s->u = zalloc(3 * N); s->T = zalloc(N); s->P = zalloc(N); s->theta = zalloc(N);
    s->h = zalloc(N); s->cvl = zalloc(N); s->gam = zalloc(N); s->athe = zalloc(N);
    s->E = zalloc(N); s->e = zalloc(N); s->X = zalloc(3 * N);
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    double *arr[] = {s->f, s->g, s->fn, s->gn, s->rho, s->J, s->G, s->lap, s->F, s->Qs, s->u, s->T,
                     s->P, s->theta, s->h, s->cvl, s->gam, s->athe, s->E, s->e, s->X};
    for (size_t k = 0; k < sizeof(arr) / sizeof(arr[0]); ++k) free(arr[k]);
    free(s->Ffield);
    free(s->Qfield);
    free(s);
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static inline long cidx(const orc_state *s, int x, int y, int z)
{
    return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * (long)z);
}

static inline int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* Index of the cell whose value stands at (x,y,z) for a macroscopic stencil:
 * periodic in x, y (and z without walls); mirrored about a wall at z = -1/2
 * or z = nz - 1/2.  *sign is -1 where the mirror flips a velocity. */
static long stencil_idx(const orc_state *s, int x, int y, int z, int *mirrored)
{
    x = wrap(x, s->p.nx);
    y = wrap(y, s->p.ny);
    *mirrored = 0;
    if (s->p.zwalls) {
        int nz = s->p.nz;
        while (z < 0 || z >= nz) {
            if (z < 0) z = -1 - z;
            else z = 2 * nz - 1 - z;
            *mirrored ^= 1;
        }
    } else {
        z = wrap(z, s->p.nz);
    }
    return cidx(s, x, y, z);
}

/* Value past a non-equilibrium-extrapolation wall (zwalls = 2): linear
 * extrapolation through the boundary cell, 2 v(z_B) - v(2 z_B - z). */
static double nee_ghost(const orc_state *s, const double *fld, int x, int y, int z)
{
    int zb = z < 0 ? 0 : s->p.nz - 1;
    x = wrap(x, s->p.nx);
    y = wrap(y, s->p.ny);
    return 2.0 * fld[cidx(s, x, y, zb)] - fld[cidx(s, x, y, 2 * zb - z)];
}

/* scalar field value at the neighbour (x+dx, y+dy, z+dz) (even mirror) */
static inline double nb_scalar(const orc_state *s, const double *fld, int x, int y, int z, int dx, int dy, int dz)
{
    int m;
    if (s->p.zwalls == 2 && (z + dz < 0 || z + dz >= s->p.nz)) return nee_ghost(s, fld, x + dx, y + dy, z + dz);
    return fld[stencil_idx(s, x + dx, y + dy, z + dz, &m)];
}

/* component a of a vector field [3][N] at the neighbour; odd mirror */
static inline double nb_vector(const orc_state *s, const double *fld, int a, int x, int y, int z, int dx, int dy, int dz)
{
    int m;
    if (s->p.zwalls == 2 && (z + dz < 0 || z + dz >= s->p.nz))
        return nee_ghost(s, fld + (long)a * s->N, x + dx, y + dy, z + dz);
    long k = stencil_idx(s, x + dx, y + dy, z + dz, &m);
    double v = fld[(long)a * s->N + k];
    return m ? -v : v;
}

/* ------------------------------------------------------------------------- */
/* Initial state: f = f^eq(rho0, u0, theta0), g = g^eq (flowchart, first box) */
/* ------------------------------------------------------------------------- */
int orc_init(orc_state *s, const double *rho, const double *u /* [dim][N] */, const double *T)
{
    int D = s->p.dim, Q = s->Q;
    long N = s->N;
    for (long k = 0; k < N; ++k) {
        double r = rho[k], uu[3] = {0, 0, 0}, xi[3], zeta[3], tmp[27];
        for (int a = 0; a < D; ++a) uu[a] = u[(long)a * N + k];
        double P = orc_eos_P(&s->p, r, T[k]);
        double th = P / r;
        for (int a = 0; a < D; ++a) { xi[a] = uu[a]; zeta[a] = th + uu[a] * uu[a]; }
        orc_fprod(D, r, xi, zeta, tmp);
        for (int i = 0; i < Q; ++i) s->f[(long)i * N + k] = tmp[i];
        orc_geq(D, r, uu, orc_eos_e(&s->p, r, T[k]), th, tmp);
        for (int i = 0; i < Q; ++i) s->g[(long)i * N + k] = tmp[i];
        s->T[k] = T[k];
    }
    return 0;
}

/* K phi(z) of the throttle at layer z (0 without one) */
static double throttle_phi(const orc_params *p, long z)
{
    if (!(p->throttle_K > 0.0) || p->dim != 3) return 0.0;
    double d = ((double)z - 0.5 * (double)(p->nz - 1)) / p->throttle_sigma;
    return p->throttle_K * exp(-d * d);
}

/* ------------------------------------------------------------------------- */
/* Phases A-C: macroscopic fields of the current populations                 */
/* ------------------------------------------------------------------------- */
static void macro_fields(orc_state *s)
{
    const orc_params *p = &s->p;
    int D = p->dim, Q = s->Q;
    long N = s->N;
    int nx = p->nx, ny = p->ny, nz = p->nz;

    /* A: Eq. def_h and the raw first moments */
#pragma omp parallel for schedule(static)
    for (long k = 0; k < N; ++k) {
        double r = 0, j[3] = {0, 0, 0}, G = 0;
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[(long)i * N + k];
            r += fi;
            for (int a = 0; a < D; ++a) j[a] += s->c[i][a] * fi;
            G += s->g[(long)i * N + k];
        }
        s->rho[k] = r;
        for (int a = 0; a < 3; ++a) s->J[(long)a * N + k] = j[a];
        s->G[k] = G;
    }

    /* B1: Laplacian of rho, (2D+1)-point stencil */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = cidx(s, x, y, z);
                double L = 0;
                for (int a = 0; a < D; ++a) {
                    int e[3] = {0, 0, 0};
                    e[a] = 1;
                    L += nb_scalar(s, s->rho, x, y, z, e[0], e[1], e[2]) - 2.0 * s->rho[k] +
                         nb_scalar(s, s->rho, x, y, z, -e[0], -e[1], -e[2]);
                }
                s->lap[k] = L;
            }

    /* B2: F = F_B + F_K with F_K = kappa rho grad(lap rho) (Eq. korteweg_force); Q(x) */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = cidx(s, x, y, z);
                double r = s->rho[k];
                for (int a = 0; a < 3; ++a) {
                    double Fa = 0.0;
                    if (a < D) {
                        int e[3] = {0, 0, 0};
                        e[a] = 1;
                        double gL = 0.5 * (nb_scalar(s, s->lap, x, y, z, e[0], e[1], e[2]) -
                                           nb_scalar(s, s->lap, x, y, z, -e[0], -e[1], -e[2]));
                        Fa = r * p->accel[a] + p->kappa * r * gL;
                        if (s->Ffield) Fa += s->Ffield[(long)a * N + k];
                    }
                    s->F[(long)a * N + k] = Fa;
                }
                int in_mask = (p->zhi <= 0) || (z >= p->zlo && z < p->zhi);
                s->Qs[k] = (in_mask ? p->q : 0.0) + (s->Qfield ? s->Qfield[k] : 0.0);
            }

    /* C: Eqs. def_u, def_E, T(rho,e), P, and the closure scalars */
    long caps = 0, nonpos = 0;
#pragma omp parallel for schedule(static) reduction(+ : caps, nonpos)
    for (long k = 0; k < N; ++k) {
        double r = s->rho[k];
        double uu[3] = {0, 0, 0}, uF = 0, u2 = 0;
        double Kphi = throttle_phi(p, k / ((long)p->nx * p->ny));
        if (p->friction > 0.0 || Kphi > 0.0) {
            /* duct resistance F_r = -rho (K phi + k |u|) u at the u it produces, and Q_r = -F_r.u */
            double w[3] = {0, 0, 0}, wn = 0, un = 0;
            for (int a = 0; a < D; ++a) {
                w[a] = (s->J[(long)a * N + k] + 0.5 * s->F[(long)a * N + k]) / r;
                wn += w[a] * w[a];
            }
            wn = sqrt(wn);
            double a0 = 1.0 + 0.5 * Kphi;
            double sc = 2.0 / (a0 + sqrt(a0 * a0 + 2.0 * p->friction * wn));
            for (int a = 0; a < D; ++a) un += (sc * w[a]) * (sc * w[a]);
            un = sqrt(un);
            double Qf = 0;
            for (int a = 0; a < D; ++a) {
                double Ff = -r * (Kphi + p->friction * un) * (sc * w[a]);
                s->F[(long)a * N + k] += Ff;
                Qf -= Ff * (sc * w[a]);
            }
            s->Qs[k] += Qf;
        }
        for (int a = 0; a < D; ++a) {
            uu[a] = (s->J[(long)a * N + k] + 0.5 * s->F[(long)a * N + k]) / r;
            uF += uu[a] * s->F[(long)a * N + k];
            u2 += uu[a] * uu[a];
        }
        for (int a = 0; a < 3; ++a) s->u[(long)a * N + k] = uu[a];
        double e, T, E;
        if (p->isothermal) {
            /* isothermal: T stays at its initial value; e follows from the EoS */
            T = s->T[k];
            e = orc_eos_e(p, r, T);
            E = e + 0.5 * u2;
        } else {
            double rhoE = s->G[k] + 0.5 * (uF + s->Qs[k]);
            E = rhoE / r;
            e = E - 0.5 * u2;
            int it;
            T = orc_eos_T(p, r, e, s->T[k], &it);
            if (p->eos == ORC_PR && it >= 50) caps++;
        }
        double P = orc_eos_P(p, r, T);
        double th = P / r;
        if (!(th > 0.0)) nonpos++;
        double cv = orc_eos_cv(p, r, T);
        double PT = orc_eos_dPdT(p, r, T);
        double Pr = orc_eos_dPdrho(p, r, T);
        double cs2 = Pr + T * PT * PT / (r * r * cv);
        s->E[k] = E;
        s->e[k] = e;
        s->T[k] = T;
        s->P[k] = P;
        s->theta[k] = th;
        s->h[k] = e + P / r;
        s->cvl[k] = cv;
        s->gam[k] = 1.0 + PT / (r * cv);
        s->athe[k] = ((double)(D + 2) / D - p->eta_over_mu) * th - cs2;
        for (int a = 0; a < 3; ++a)
            s->X[(long)a * N + k] = (a < D) ? r * uu[a] * uu[a] * uu[a] + 3.0 * r * uu[a] * (th - 1.0 / 3.0) : 0.0;
    }
    s->newton_cap_hits += caps;
    s->theta_nonpos += nonpos;
}

/* ------------------------------------------------------------------------- */
/* Non-equilibrium-extrapolation walls (zwalls = 2; App. B, thermal Couette): */
/* rebuild the boundary cells from the wall state and the non-equilibrium    */
/* part of their neighbours, after phases A-C.  pops = 0 rebuilds only the    */
/* macroscopic fields (for the reported moments).                             */
/* ------------------------------------------------------------------------- */
static void nee_walls(orc_state *s, int pops)
{
    const orc_params *p = &s->p;
    if (p->zwalls != 2) return;
    int D = p->dim, Q = s->Q;
    long N = s->N;
    for (int side = 0; side < 2; ++side) {
        int zb = side ? p->nz - 1 : 0, zn = side ? p->nz - 2 : 1;
        const double *uw = side ? p->uw_hi : p->uw_lo;
        double Tw;
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long kb = cidx(s, x, y, zb), kn = cidx(s, x, y, zn);
                double rn = s->rho[kn], un[3], uW[3] = {0, 0, 0}, xi[3], zeta[3];
                for (int a = 0; a < 3; ++a) un[a] = s->u[(long)a * N + kn];
                for (int a = 0; a < D; ++a) uW[a] = uw[a];
                /* boundary state: rho_B, u_B (uW), T_B (Tw) of the face's kind */
                int kind = p->face_kind[side];
                double Pt = -1.0; /* pressure that rho_B must meet at Tw, if any */
                Tw = side ? p->Tw_hi : p->Tw_lo;
                if (kind == ORC_FACE_WALL) {
                    if (p->wall_rho == 0) Pt = orc_eos_P(p, rn, s->T[kn]);
                    if (p->wall_rho == 2) { /* pressure extrapolated linearly from the two cells inside */
                        long knn = cidx(s, x, y, side ? p->nz - 3 : 2);
                        Pt = 2.0 * s->P[kn] - s->P[knn];
                    }
                } else if (kind == ORC_FACE_INLET_TOTAL) {
                    double cp = p->cv + p->R, n2 = 0;
                    for (int a = 0; a < D; ++a) { uW[a] = un[a]; n2 += un[a] * un[a]; }
                    double T0 = Tw;
                    Tw = T0 - 0.5 * n2 / cp;
                    Pt = p->face_P[side] * pow(Tw / T0, cp / p->R);
                } else if (kind == ORC_FACE_INLET_STATIC) {
                    Pt = p->face_P[side];
                } else if (kind == ORC_FACE_OUTLET_P) {
                    Tw = s->T[kn];
                    Pt = p->face_P[side];
                } else if (kind == ORC_FACE_INLET_PT) {
                    for (int a = 0; a < D; ++a) uW[a] = un[a];
                    Pt = p->face_P[side];
                } else {
                    for (int a = 0; a < D; ++a) uW[a] = un[a];
                    Tw = s->T[kn];
                }
                double rb = rn;
                if (Pt > 0.0) {
                    double r = rn;
                    for (int it = 0; it < 8; ++it) r -= (orc_eos_P(p, r, Tw) - Pt) / orc_eos_dPdrho(p, r, Tw);
                    if (isfinite(r) && r > 0.0) rb = r;
                }
                if (kind == ORC_FACE_OUTLET_P) /* the neighbour's mass flux */
                    for (int a = 0; a < D; ++a) uW[a] = un[a] * (rn / rb);
                double Pw = orc_eos_P(p, rb, Tw), thw = Pw / rb, ew = orc_eos_e(p, rb, Tw);
                if (pops) {
                    double feqB[27], geqB[27], feqN[27], geqN[27];
                    for (int a = 0; a < D; ++a) { xi[a] = uW[a]; zeta[a] = thw + uW[a] * uW[a]; }
                    orc_fprod(D, rb, xi, zeta, feqB);
                    orc_geq(D, rb, uW, ew, thw, geqB);
                    for (int a = 0; a < D; ++a) { xi[a] = un[a]; zeta[a] = s->theta[kn] + un[a] * un[a]; }
                    orc_fprod(D, rn, xi, zeta, feqN);
                    orc_geq(D, rn, un, s->e[kn], s->theta[kn], geqN);
                    for (int i = 0; i < Q; ++i) {
                        s->f[(long)i * N + kb] = feqB[i] + (s->f[(long)i * N + kn] - feqN[i]);
                        s->g[(long)i * N + kb] = geqB[i] + (s->g[(long)i * N + kn] - geqN[i]);
                    }
                }
                /* force and heat: non-friction part per unit mass kept, friction at (rho_B, u_B) */
                double ro = s->rho[kb], uo2 = 0, u2 = 0;
                for (int a = 0; a < D; ++a) { uo2 += s->u[(long)a * N + kb] * s->u[(long)a * N + kb]; u2 += uW[a] * uW[a]; }
                double uon = sqrt(uo2), ubn = sqrt(u2);
                double Kphi = throttle_phi(p, zb);
                for (int a = 0; a < 3; ++a) {
                    double Ffo = a < D ? -ro * (Kphi + p->friction * uon) * s->u[(long)a * N + kb] : 0.0;
                    double Ffb = a < D ? -rb * (Kphi + p->friction * ubn) * uW[a] : 0.0;
                    s->F[(long)a * N + kb] = (s->F[(long)a * N + kb] - Ffo) * (rb / ro) + Ffb;
                }
                s->Qs[kb] += rb * (Kphi + p->friction * ubn) * u2 - ro * (Kphi + p->friction * uon) * uo2;
                for (int a = 0; a < 3; ++a) s->u[(long)a * N + kb] = uW[a];
                double cv = orc_eos_cv(p, rb, Tw), PT = orc_eos_dPdT(p, rb, Tw), Pr = orc_eos_dPdrho(p, rb, Tw);
                double cs2 = Pr + Tw * PT * PT / (rb * rb * cv);
                s->rho[kb] = rb;
                s->T[kb] = Tw;
                s->e[kb] = ew;
                s->E[kb] = ew + 0.5 * u2;
                s->P[kb] = Pw;
                s->theta[kb] = thw;
                s->h[kb] = ew + Pw / rb;
                s->cvl[kb] = cv;
                s->gam[kb] = 1.0 + PT / (rb * cv);
                s->athe[kb] = ((double)(D + 2) / D - p->eta_over_mu) * thw - cs2;
                for (int a = 0; a < 3; ++a)
                    s->X[(long)a * N + kb] = (a < D) ? rb * uW[a] * uW[a] * uW[a] + 3.0 * rb * uW[a] * (thw - 1.0 / 3.0) : 0.0;
            }
    }
}

/* ------------------------------------------------------------------------- */
/* One time step                                                              */
/* ------------------------------------------------------------------------- */
static void one_step(orc_state *s)
{
    const orc_params *p = &s->p;
    int D = p->dim, Q = s->Q;
    long N = s->N;
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double beta_f = 1.0 / (2.0 * p->tau_f + 1.0);
    double beta_g = 1.0 / (2.0 * p->tau_g + 1.0);

    macro_fields(s);
    nee_walls(s, 1);

#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = cidx(s, x, y, z);
                double r = s->rho[k], T = s->T[k], P = s->P[k], th = s->theta[k];
                double cv = s->cvl[k], Qk = s->Qs[k];
                double uu[3], Fv[3];
                for (int a = 0; a < 3; ++a) { uu[a] = s->u[(long)a * N + k]; Fv[a] = s->F[(long)a * N + k]; }

                /* D: gradients (central) and the Galilean correction (upwind-biased) */
                double divu = 0, gh[3] = {0, 0, 0}, gT[3] = {0, 0, 0}, Phi[3] = {0, 0, 0};
                for (int a = 0; a < D; ++a) {
                    int e[3] = {0, 0, 0};
                    e[a] = 1;
                    divu += 0.5 * (nb_vector(s, s->u, a, x, y, z, e[0], e[1], e[2]) -
                                   nb_vector(s, s->u, a, x, y, z, -e[0], -e[1], -e[2]));
                    gh[a] = 0.5 * (nb_scalar(s, s->h, x, y, z, e[0], e[1], e[2]) -
                                   nb_scalar(s, s->h, x, y, z, -e[0], -e[1], -e[2]));
                    gT[a] = 0.5 * (nb_scalar(s, s->T, x, y, z, e[0], e[1], e[2]) -
                                   nb_scalar(s, s->T, x, y, z, -e[0], -e[1], -e[2]));
                    double X0 = s->X[(long)a * N + k], dX;
                    if (p->phi_central == 1) {
                        dX = 0.5 * (nb_vector(s, s->X, a, x, y, z, e[0], e[1], e[2]) -
                                    nb_vector(s, s->X, a, x, y, z, -e[0], -e[1], -e[2]));
                    } else {
                        /* Upwind-biased (phi_central = 0): the third-order stencil with two
                         * points on the side the local u_alpha comes from and one on the other,
                         * (2 X_{+1} + 3 X_0 - 6 X_{-1} + X_{-2}) / 6 for u_alpha >= 0 and its mirror
                         * image otherwise.  Other values are stencils kept for the stability
                         * analysis only: 2 second-order one-sided, 3 the same reversed, 4 the
                         * third-order stencil reversed, 5 first-order upwind. */
                        const int sch = p->phi_central;
                        const int up = (uu[a] >= 0.0) != (sch == 3 || sch == 4);
                        const int sg = up ? 1 : -1;  /* +1: the upwind side is the backward one */
                        double Xb1 = nb_vector(s, s->X, a, x, y, z, -sg * e[0], -sg * e[1], -sg * e[2]);
                        double Xb2 = nb_vector(s, s->X, a, x, y, z, -2 * sg * e[0], -2 * sg * e[1], -2 * sg * e[2]);
                        double Xf1 = nb_vector(s, s->X, a, x, y, z, sg * e[0], sg * e[1], sg * e[2]);
                        if (sch == 5) dX = sg * (X0 - Xb1);
                        else if (sch == 2 || sch == 3) dX = sg * 0.5 * (3.0 * X0 - 4.0 * Xb1 + Xb2);
                        else dX = sg * (2.0 * Xf1 + 3.0 * X0 - 6.0 * Xb1 + Xb2) / 6.0;
                    }
                    Phi[a] = -dX / r; /* Eq. correction */
                }

                /* shifted states, Eqs. sh_vel_1, sh_temp_1, sh_T_1, qc_1 */
                double us[3] = {0, 0, 0}, FF = 0, qc[3] = {0, 0, 0};
                for (int a = 0; a < D; ++a) {
                    us[a] = uu[a] + Fv[a] / r;
                    FF += Fv[a] * Fv[a];
                    qc[a] = P * (gh[a] - p->k_over_mu * gT[a]);
                }
                double ths = th + s->athe[k] * divu + (s->gam[k] - 1.0) * Qk / r;
                double Ts = T + Qk / (r * cv) - FF / (2.0 * r * r * cv);
                double es = orc_eos_e(p, r, Ts);

                /* E: equilibria in product form */
                double xi[3], zeta[3], feq[27], fst[27], geq[27], gst[27];
                for (int a = 0; a < D; ++a) { xi[a] = uu[a]; zeta[a] = th + uu[a] * uu[a]; }
                orc_fprod(D, r, xi, zeta, feq);                          /* Eq. LBMeq */
                for (int a = 0; a < D; ++a) { xi[a] = us[a]; zeta[a] = ths + us[a] * us[a] + Phi[a]; }
                orc_fprod(D, r, xi, zeta, fst);                          /* Eq. LBMstar */
                orc_geq(D, r, uu, s->e[k], th, geq);                      /* Eq. LBMeqG */
                orc_geq(D, r, us, es, ths, gst);                          /* Eq. LBMgstar, first term */
                for (int i = 0; i < Q; ++i) {
                    int c2 = 0;
                    double cq = 0;
                    for (int a = 0; a < D; ++a) { c2 += s->c[i][a] * s->c[i][a]; cq += s->c[i][a] * qc[a]; }
                    if (c2 == 1) gst[i] += 0.5 * cq;                      /* Eq. LBMgstar, correction */
                }

                /* beta (Eq. beta): constant, or from tau = mu / P of this cell */
                double bf = beta_f, bg = beta_g;
                if (p->mu > 0.0) {
                    double tau = p->mu / P;
                    bf = bg = 1.0 / (2.0 * tau + 1.0);
                }

                /* collide (Eqs. LBM_f, LBM_g with lambda = dt) and stream (push) */
                for (int i = 0; i < Q; ++i) {
                    double fi = s->f[(long)i * N + k], gi = s->g[(long)i * N + k];
                    double fo = fi + 2.0 * bf * (feq[i] - fi) + (1.0 - bf) * (fst[i] - feq[i]);
                    double go = gi + 2.0 * bg * (geq[i] - gi) + (1.0 - bg) * (gst[i] - geq[i]);
                    int zt = z + s->c[i][2];
                    if (p->zwalls && (zt < 0 || zt >= nz)) {
                        /* half-way bounce-back: returns to this cell reversed */
                        s->fn[(long)s->opp[i] * N + k] = fo;
                        if (!p->isothermal) s->gn[(long)s->opp[i] * N + k] = go;
                    } else {
                        long kt = cidx(s, wrap(x + s->c[i][0], nx), wrap(y + s->c[i][1], ny), wrap(zt, nz));
                        s->fn[(long)i * N + kt] = fo;
                        if (!p->isothermal) s->gn[(long)i * N + kt] = go;
                    }
                }
            }

    double *t;
    t = s->f; s->f = s->fn; s->fn = t;
    if (!p->isothermal) { t = s->g; s->g = s->gn; s->gn = t; }  /* isothermal: g is not evolved */
}

/* Replace the body acceleration (F_B = rho a, Eq. force_decomposition) from
 * the next step on: forcing that varies in time. */
/* Per-cell body force F_B(x) [dim][N] (added to rho a + F_K, Eq. force_decomposition)
 * and heat source Q(x) [N] (added to the uniform or masked Q), copied; NULL
 * removes them. */
void orc_set_fields(orc_state *s, const double *F, const double *Q)
{
    int D = s->p.dim;
    long N = s->N;
    free(s->Ffield);
    free(s->Qfield);
    s->Ffield = s->Qfield = NULL;
    if (F) {
        s->Ffield = zalloc(3 * N);
        for (int a = 0; a < D; ++a) memcpy(s->Ffield + (long)a * N, F + (long)a * N, (size_t)N * sizeof(double));
    }
    if (Q) {
        s->Qfield = zalloc(N);
        memcpy(s->Qfield, Q, (size_t)N * sizeof(double));
    }
}

void orc_set_accel(orc_state *s, const double *a)
{
    for (int k = 0; k < 3; ++k) s->p.accel[k] = a[k];
}

int orc_step(orc_state *s, int n)
{
    for (int it = 0; it < n; ++it) one_step(s);
    return 0;
}

/* Macroscopic fields of the current state: rho, u (Eq. def_u), T. */
int orc_moments(orc_state *s, double *rho, double *u /* [dim][N] */, double *T)
{
    macro_fields(s);
    nee_walls(s, 0);
    long N = s->N;
    for (long k = 0; k < N; ++k) {
        if (rho) rho[k] = s->rho[k];
        if (T) T[k] = s->T[k];
        if (u)
            for (int a = 0; a < s->p.dim; ++a) u[(long)a * N + k] = s->u[(long)a * N + k];
    }
    return 0;
}

/* Totals of the current state:
 *   out = [ sum rho, sum rho u (dim), sum rho E, sum F (dim), sum (u.F + Q) ]
 * with rho u and rho E from Eqs. def_u and def_E. */
int orc_invariants(orc_state *s, double *out)
{
    macro_fields(s);
    nee_walls(s, 0);
    int D = s->p.dim;
    long N = s->N;
    double m = 0, M[3] = {0, 0, 0}, En = 0, Fs[3] = {0, 0, 0}, S = 0;
    for (long k = 0; k < N; ++k) {
        double r = s->rho[k], uF = 0;
        m += r;
        for (int a = 0; a < D; ++a) {
            M[a] += r * s->u[(long)a * N + k];
            Fs[a] += s->F[(long)a * N + k];
            uF += s->u[(long)a * N + k] * s->F[(long)a * N + k];
        }
        En += r * s->E[k];
        S += uF + s->Qs[k];
    }
    int o = 0;
    out[o++] = m;
    for (int a = 0; a < D; ++a) out[o++] = M[a];
    out[o++] = En;
    for (int a = 0; a < D; ++a) out[o++] = Fs[a];
    out[o++] = S;
    return o;
}

/* Copies of the populations [Q][N]. */
int orc_populations(const orc_state *s, double *f, double *g)
{
    size_t n = (size_t)s->Q * (size_t)s->N * sizeof(double);
    if (f) memcpy(f, s->f, n);
    if (g) memcpy(g, s->g, n);
    return 0;
}

/* Overwrite the populations (used by tests that start from a given state). */
int orc_set_populations(orc_state *s, const double *f, const double *g, const double *T_guess)
{
    size_t n = (size_t)s->Q * (size_t)s->N * sizeof(double);
    memcpy(s->f, f, n);
    memcpy(s->g, g, n);
    if (T_guess) memcpy(s->T, T_guess, (size_t)s->N * sizeof(double));
    return 0;
}

long orc_newton_cap_hits(const orc_state *s) { return s->newton_cap_hits; }
long orc_theta_nonpositive(const orc_state *s) { return s->theta_nonpos; }
