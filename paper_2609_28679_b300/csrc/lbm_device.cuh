// Device building blocks of one time step of the consistent DDF lattice
// Boltzmann scheme (arxiv 2609.28679, Sec. II): lattice, population storage
// codecs, equations of state, per-cell macroscopic state and the collision.
// Shared by the split (three-pass) and fused (one-pass) step kernels.
#pragma once

#include <cstddef>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// ---------------------------------------------------------------------------
// Lattice (Eq. D3Q27c; D2Q9 is its restriction to two axes).  Direction i has
// base-3 digits (d0, d1, d2); digit 0, 1, 2 means c = 0, +1, -1, which is also
// the index into the per-axis factor triples below.
// ---------------------------------------------------------------------------
template <int D> struct Lat { static constexpr int Q = (D == 2) ? 9 : 27; };

__host__ __device__ constexpr int dig(int i, int a) { return a == 0 ? i % 3 : (a == 1 ? (i / 3) % 3 : (i / 9) % 3); }
__host__ __device__ constexpr int cval(int d) { return d == 0 ? 0 : (d == 1 ? 1 : -1); }
__host__ __device__ constexpr int cc(int i, int a) { return cval(dig(i, a)); }
__host__ __device__ constexpr int odig(int d) { return d == 0 ? 0 : 3 - d; }
__host__ __device__ constexpr int opp(int i) { return odig(i % 3) + 3 * odig((i / 3) % 3) + 9 * odig((i / 9) % 3); }
__host__ __device__ constexpr int cnorm2(int i) { return cc(i, 0) * cc(i, 0) + cc(i, 1) * cc(i, 1) + cc(i, 2) * cc(i, 2); }

enum { EOS_IDEAL = 0, EOS_VDW = 1, EOS_PR = 2 };

// Per-simulation constants, resident in device memory.
struct SimDev {
    int nx, ny, nz, zwalls;
    long long N;         // cells
    long long pop_off;   // element offset of this simulation's f block; g follows at +Q*N
    long long cell_off;  // element offset of its cells in per-cell arrays
    int eos, phi_central, t_solver, zlo, zhi;
    int iso;                      // 1: isothermal, g not evolved, T kept at its initial value
    double R, cv, a, b, Tc, kw;   // kw: Soave kappa(omega) for Peng-Robinson
    double kappa, eta_mu, k_mu;   // Korteweg coefficient, eta/mu, k/mu
    double beta_f, beta_g;        // 1/(2 tau + 1)
    double acc[3], q;             // body acceleration, heat source
    double inv_cv, inv_Tc, lam_c; // 1/cv, 1/Tc, 1/(2 sqrt2 b) (Peng-Robinson)
    double athe_c;                // (D+2)/D - eta/mu
    double mu;                    // > 0: tau = mu / P per cell (beta per cell); 0: beta_f, beta_g
    float fref[27], gref[27];     // storage offsets (16-bit storage only; zero otherwise)
    const float* mlp;             // learned T(rho, e) parameters (t_solver == LBM_T_MLP), or null
    double uw[2][3], Tw[2];       // zwalls == 2: velocity and temperature of the walls at z = 0 and z = nz - 1
    int wall_rho;                 // zwalls == 2: 0 rho_B from the neighbour's pressure, 1 rho_B = rho_N
    int face_kind[2];             // zwalls == 2: 0 wall, else LBM_FACE_* (open duct end)
    int face_set[2];              // zwalls == 2: the face has its data (lbm_set_walls / lbm_set_face)
    double face_P[2];             // pressure datum of an open face (total for INLET_TOTAL)
    double friction;              // duct friction k: F_f = -k rho |u| u, Q_f = -F_f.u (split kernels)
    double throttle_K, throttle_sigma;  // Darcy throttle F_t = -K phi(z) rho u, Q_t = -F_t.u (split kernels)
    const double* ffield;         // optional per-cell body force [D][N] (device, caller's), split kernels
    const double* qfield;         // optional per-cell heat source [N] (device, caller's), split kernels
};

// The same constants in the arithmetic type R (built once per tile on the
// device, so that float32 kernels never convert from float64 on the way).
template <typename F> struct SimC {
    int nx, ny, nz, zwalls;
    long long N, pop_off, cell_off;
    int eos, phi_central, t_solver, zlo, zhi, iso;
    F R, cv, a, b, Tc, kw, kappa, eta_mu, k_mu, beta_f, beta_g, acc[3], q, inv_cv, inv_Tc, lam_c, athe_c, mu;
    F fref[27], gref[27];
    const float* mlp;
};

template <typename R> __device__ inline void simc_from(SimC<R>& d, const SimDev& s)
{
    d.nx = s.nx; d.ny = s.ny; d.nz = s.nz; d.zwalls = s.zwalls;
    d.N = s.N; d.pop_off = s.pop_off; d.cell_off = s.cell_off;
    d.eos = s.eos; d.phi_central = s.phi_central; d.t_solver = s.t_solver; d.zlo = s.zlo; d.zhi = s.zhi;
    d.iso = s.iso;
    d.R = (R)s.R; d.cv = (R)s.cv; d.a = (R)s.a; d.b = (R)s.b; d.Tc = (R)s.Tc; d.kw = (R)s.kw;
    d.kappa = (R)s.kappa; d.eta_mu = (R)s.eta_mu; d.k_mu = (R)s.k_mu; d.beta_f = (R)s.beta_f; d.beta_g = (R)s.beta_g;
    for (int a = 0; a < 3; ++a) d.acc[a] = (R)s.acc[a];
    d.q = (R)s.q; d.inv_cv = (R)s.inv_cv; d.inv_Tc = (R)s.inv_Tc; d.lam_c = (R)s.lam_c; d.athe_c = (R)s.athe_c;
    d.mu = (R)s.mu;
    for (int i = 0; i < 27; ++i) { d.fref[i] = (R)s.fref[i]; d.gref[i] = (R)s.gref[i]; }
    d.mlp = s.mlp;
}

// The same conversion shared out over a block's threads (one field each):
// the twenty float64 scalars from R to mu are consecutive members in both
// structures, as are the two offset tables.  The caller synchronises after.
template <typename R> __device__ inline void simc_from_coop(SimC<R>& d, const SimDev& s, int tid)
{
    static_assert(offsetof(SimDev, mu) - offsetof(SimDev, R) == 19 * sizeof(double), "SimDev scalar layout");
    static_assert(offsetof(SimC<R>, mu) - offsetof(SimC<R>, R) == 19 * sizeof(R), "SimC scalar layout");
    static_assert(offsetof(SimDev, gref) - offsetof(SimDev, fref) == 27 * sizeof(float), "SimDev table layout");
    static_assert(offsetof(SimC<R>, gref) - offsetof(SimC<R>, fref) == 27 * sizeof(R), "SimC table layout");
    if (tid < 20) {
        (&d.R)[tid] = (R)(&s.R)[tid];
    } else if (tid < 74) {
        (&d.fref[0])[tid - 20] = (R)(&s.fref[0])[tid - 20];
    } else if (tid == 74) {
        d.nx = s.nx; d.ny = s.ny; d.nz = s.nz; d.zwalls = s.zwalls;
        d.N = s.N; d.pop_off = s.pop_off; d.cell_off = s.cell_off;
        d.eos = s.eos; d.phi_central = s.phi_central; d.t_solver = s.t_solver; d.zlo = s.zlo; d.zhi = s.zhi;
    d.iso = s.iso;
        d.mlp = s.mlp;
    }
}

// ---------------------------------------------------------------------------
// Storage codecs: populations are stored as S, computed in R.
// ---------------------------------------------------------------------------
template <typename S, typename R> struct Codec;
template <> struct Codec<double, double> {
    static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
    static constexpr bool offset = false;
};
template <> struct Codec<float, float> {
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
    static constexpr bool offset = false;
};
template <> struct Codec<__nv_bfloat16, float> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    static constexpr bool offset = true;
};
template <> struct Codec<__half, float> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
    static constexpr bool offset = true;
};

// ---------------------------------------------------------------------------
// Equations of state.  Per cell, the density-only parts are evaluated once
// (RhoPart, with the reciprocals the T-dependent parts need), then P, e and
// the derivatives as functions of T.
// ---------------------------------------------------------------------------
template <typename R> struct RhoPart {
    R rho, id1, iden, lam;  // 1/(1 - b rho); 1/(1 + 2 b rho - b^2 rho^2); Lambda(rho) (Peng-Robinson)
};

template <typename R, typename C> __host__ __device__ __forceinline__ RhoPart<R> rho_part(const C& s, R rho)
{
    RhoPart<R> p;
    p.rho = rho;
    p.id1 = R(1);
    p.iden = R(1);
    p.lam = R(0);
    if (s.eos == EOS_IDEAL) return p;
    const R b = (R)s.b;
    p.id1 = R(1) / (R(1) - b * rho);
    if (s.eos == EOS_PR) {
        const R r2 = (R)1.4142135623730951;
        const R br = b * rho;
        p.iden = R(1) / (R(1) + R(2) * br - br * br);
        // Lambda = int_0^rho dr/(1 + 2 b r - b^2 r^2) = ln[(1 + (1+sqrt2) b rho)/(1 + (1-sqrt2) b rho)] / (2 sqrt2 b)
        p.lam = log((R(1) + (R(1) + r2) * br) / (R(1) + (R(1) - r2) * br)) * (R)s.lam_c;
    }
    return p;
}

template <typename R, typename C> __host__ __device__ __forceinline__ R pr_sq(const C& s, R T) { return sqrt(T * (R)s.inv_Tc); }

template <typename R, typename C> __host__ __device__ __forceinline__ R eos_P(const C& s, const RhoPart<R>& p, R T)
{
    const R rho = p.rho;
    if (s.eos == EOS_IDEAL) return rho * (R)s.R * T;
    if (s.eos == EOS_VDW) return rho * (R)s.R * T * p.id1 - (R)s.a * rho * rho;
    const R m = R(1) + (R)s.kw * (R(1) - pr_sq<R>(s, T));
    return rho * (R)s.R * T * p.id1 - (R)s.a * m * m * rho * rho * p.iden;
}

template <typename R, typename C> __host__ __device__ __forceinline__ R eos_e(const C& s, const RhoPart<R>& p, R T)
{
    if (s.eos == EOS_IDEAL) return (R)s.cv * T;
    if (s.eos == EOS_VDW) return (R)s.cv * T - (R)s.a * p.rho;
    const R k = (R)s.kw;
    return (R)s.cv * T - (R)s.a * (R(1) + k) * (R(1) + k - k * pr_sq<R>(s, T)) * p.lam;
}

// c_v = (de/dT)_rho
template <typename R, typename C> __host__ __device__ __forceinline__ R eos_cv(const C& s, const RhoPart<R>& p, R T)
{
    if (s.eos != EOS_PR) return (R)s.cv;
    const R k = (R)s.kw;
    return (R)s.cv + (R)s.a * (R(1) + k) * k * p.lam * R(0.5) * (R)s.inv_Tc / pr_sq<R>(s, T);
}

// P, (dP/dT)_rho, (dP/drho)_T and c_v at (rho, T) with shared subexpressions
template <typename R> struct Thermo {
    R P, PT, Pr, cv;
};

template <typename R, typename C> __host__ __device__ __forceinline__ Thermo<R> thermo(const C& s, const RhoPart<R>& p, R T)
{
    Thermo<R> t;
    const R rho = p.rho, Rg = (R)s.R;
    if (s.eos == EOS_IDEAL) {
        t.PT = rho * Rg;
        t.P = t.PT * T;
        t.Pr = Rg * T;
        t.cv = (R)s.cv;
    } else if (s.eos == EOS_VDW) {
        t.PT = rho * Rg * p.id1;
        t.P = t.PT * T - (R)s.a * rho * rho;
        t.Pr = Rg * T * p.id1 * p.id1 - R(2) * (R)s.a * rho;
        t.cv = (R)s.cv;
    } else {
        const R k = (R)s.kw, b = (R)s.b, a = (R)s.a;
        const R sq = pr_sq<R>(s, T), isq = R(1) / sq;
        const R m = R(1) + k * (R(1) - sq);
        const R q = rho * rho * p.iden;                       // rho^2 / den
        const R dq = (R(2) * rho - q * (R(2) * b - R(2) * b * b * rho)) * p.iden;  // d(rho^2/den)/drho
        const R dal = -m * k * isq * (R)s.inv_Tc;             // d alpha / dT
        t.P = rho * Rg * T * p.id1 - a * m * m * q;
        t.PT = rho * Rg * p.id1 - a * dal * q;
        t.Pr = Rg * T * p.id1 * p.id1 - a * m * m * dq;
        t.cv = (R)s.cv + a * (R(1) + k) * k * p.lam * R(0.5) * (R)s.inv_Tc * isq;
    }
    return t;
}

template <typename R, typename C> __device__ __forceinline__ R eos_dPdT(const C& s, const RhoPart<R>& p, R T)
{
    return thermo<R>(s, p, T).PT;
}

template <typename R, typename C> __device__ __forceinline__ R eos_dPdrho(const C& s, const RhoPart<R>& p, R T)
{
    return thermo<R>(s, p, T).Pr;
}

// Newton's method on e(rho, T) - e = 0 for Peng-Robinson, in precision W.
// Returns the iteration count (cap + 1 when the cap was hit).
template <typename W, typename C>
__device__ __forceinline__ int pr_newton(const C& s, const RhoPart<W>& p, W e, W& T, W tol, int cap)
{
    for (int it = 1; it <= cap; ++it) {
        W r = eos_e<W>(s, p, T) - e;
        W dT = -r / eos_cv<W>(s, p, T);
        T += dT;
        if (fabs(dT) <= tol * fabs(T)) return it;
    }
    return cap + 1;
}

// T(rho, e): explicit for ideal gas and van der Waals (Eqs. idealgasT,
// lbm_temp); Peng-Robinson by Newton from Tguess -- in float64 for the
// float64 path; in float32 with a float64 fallback for the float32 path.
template <typename R, typename C>
__device__ __forceinline__ R eos_T(const C& s, const RhoPart<R>& p, R e, R Tguess, bool& capped, int& iters)
{
    capped = false;
    iters = 0;
    if (s.eos == EOS_IDEAL) return e * (R)s.inv_cv;
    if (s.eos == EOS_VDW) return (e + (R)s.a * p.rho) * (R)s.inv_cv;
    // without a previous T (Tguess <= 0) start from the critical temperature
    R T = Tguess > R(0) ? Tguess : (R)s.Tc;
    if (sizeof(R) == 8) {
        int it = pr_newton<R>(s, p, e, T, (R)1e-14, 50);
        capped = it > 50;
        iters = it;
        return T;
    }
    int it = pr_newton<R>(s, p, e, T, (R)1e-6, 8);
    iters = it;
    if (it <= 8 && T > R(0)) return T;
    RhoPart<double> pd = rho_part<double>(s, (double)p.rho);
    double Td = (Tguess > R(0)) ? (double)Tguess : (double)s.Tc;
    int itd = pr_newton<double>(s, pd, (double)e, Td, 1e-12, 50);
    capped = itd > 50;
    iters = 8 + itd;
    return (R)Td;
}

// ---------------------------------------------------------------------------
// Macroscopic state of one cell (flowchart boxes 2-3): from the moments
// rho, j = sum c f, G = sum g, the force F and source Q.
// ---------------------------------------------------------------------------
template <typename R> struct Macro {
    R rho, ir, u[3], F[3], Q, T, P, theta, h, cv, icv, gam, athe, e;
};

template <int D, typename R, typename C>
__device__ __forceinline__ Macro<R> macro_cell(const C& s, R rho, const R* j, R G, const R* F, R Q, R Tguess,
                                               unsigned& flags)
{
    Macro<R> m;
    m.rho = rho;
    m.ir = R(1) / rho;
    m.Q = Q;
    R uF = 0, u2 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.F[a] = a < D ? F[a] : R(0);
        m.u[a] = a < D ? (j[a] + R(0.5) * F[a]) * m.ir : R(0);  // Eq. def_u
        uF += m.u[a] * m.F[a];
        u2 += m.u[a] * m.u[a];
    }
    const RhoPart<R> p = rho_part<R>(s, rho);
    bool capped = false;
    int iters = 0;
    R e, T;
    if (s.iso) {
        // isothermal (g not evolved): the carried temperature is the cell's initial one
        T = Tguess;
        e = eos_e<R>(s, p, T);
    } else {
        const R rhoE = G + R(0.5) * (uF + Q);  // Eq. def_E
        e = rhoE * m.ir - R(0.5) * u2;
        T = eos_T<R>(s, p, e, Tguess, capped, iters);
    }
    const Thermo<R> t = thermo<R>(s, p, T);
    const R th = t.P * m.ir;  // Eq. theta
    m.icv = s.eos == EOS_PR ? R(1) / t.cv : (R)s.inv_cv;
    const R cs2 = t.Pr + T * t.PT * t.PT * m.ir * m.ir * m.icv;
    m.T = T;
    m.P = t.P;
    m.theta = th;
    m.h = e + th;  // Eq. enthalpy: h = e + P/rho
    m.cv = t.cv;
    m.gam = R(1) + t.PT * m.ir * m.icv;  // Eq. corr_heat_source
    m.athe = (R)s.athe_c * th - cs2;     // alpha theta, Eq. corr_bulk: ((D+2)/D - eta/mu) theta - c_s^2
    m.e = e;
    if (capped) flags |= 4u;
    // learned start: accepted when the first Newton correction meets the tolerance
    if (s.eos == EOS_PR && s.t_solver == 1 && s.mlp != nullptr && iters > 1) flags |= 8u;
    if (!(th > R(0))) flags |= 2u;
    if (!isfinite(rho) || !isfinite(T) || !isfinite(u2)) flags |= 1u;
    return m;
}

// Specific internal energy e of a cell (Eqs. def_u, def_E): the input of the
// learned temperature inversion, evaluated ahead of macro_cell.
template <int D, typename R>
__device__ __forceinline__ R macro_energy(R rho, const R* j, R G, const R* F, R Q)
{
    const R ir = R(1) / rho;
    R uF = 0, u2 = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const R u = (j[a] + R(0.5) * F[a]) * ir;
        uF += u * F[a];
        u2 += u * u;
    }
    return (G + R(0.5) * (uF + Q)) * ir - R(0.5) * u2;
}

// X_alpha = rho u_alpha^3 + 3 rho u_alpha (theta - 1/3), the flux whose
// derivative is the Galilean correction Phi (Eq. correction).
template <typename R> __device__ __forceinline__ R xflux(R rho, R u, R th)
{
    return rho * u * (u * u + R(3) * th - R(1));
}

// The upwind-biased first derivative of X in Eq. correction (Sec. II.E): the
// third-order difference with two points on the side u comes from and one on
// the other, (2 X_{+1} + 3 X_0 - 6 X_{-1} + X_{-2}) / 6 for u >= 0 and its
// mirror image for u < 0.
template <typename R> __host__ __device__ __forceinline__ R upwind_biased(R u, R x2, R xm1, R x0, R xp1)
{
    // x2: X_{-2} when u >= 0, X_{+2} otherwise
    return u >= R(0) ? (R(2) * xp1 + R(3) * x0 - R(6) * xm1 + x2) * R(1.0 / 6.0)
                     : -(R(2) * xm1 + R(3) * x0 - R(6) * xp1 + x2) * R(1.0 / 6.0);
}

// beta of a cell (Eq. beta, dt = 1) under the paper's tau = mu / P (Sec. II.C)
template <typename R, typename C> __device__ __forceinline__ R relax_beta(const C& s, R P)
{
    const R tau = (R)s.mu / P;
    return R(1) / (R(2) * tau + R(1));
}

// ---------------------------------------------------------------------------
// Collision of one cell (Eqs. LBMeq, LBMstar, LBMeqG, LBMgstar, LBM_f, LBM_g).
// f, g: pre-collision populations in, post-collision out.
// ---------------------------------------------------------------------------
template <typename R> __host__ __device__ __forceinline__ void psi3(R xi, R zeta, R* o)
{
    // Eq. phi at c = 0, +1, -1
    o[0] = R(1) - zeta;
    o[1] = R(0.5) * (zeta + xi);
    o[2] = R(0.5) * (zeta - xi);
}

// Psi(c; O, O^2) applied to u^2/2, with O = theta d/du + u (Eq. Oa):
// O(u^2/2) = theta u + u^3/2, O^2(u^2/2) = theta^2 + 5/2 theta u^2 + u^4/2.
template <typename R> __host__ __device__ __forceinline__ void hpsi3(R u, R th, R* o)
{
    R u2 = u * u;
    R o1 = th * u + R(0.5) * u2 * u;
    R o2 = th * th + R(2.5) * th * u2 + R(0.5) * u2 * u2;
    o[0] = R(0.5) * u2 - o2;
    o[1] = R(0.5) * (o2 + o1);
    o[2] = R(0.5) * (o2 - o1);
}

// psi3 and hpsi3 for two axes at once (two-wide float32 operations)
__device__ __forceinline__ void psi3_x2(float2 xi, float2 zeta, float2* o)
{
    const float2 one = make_float2(1.f, 1.f), half = make_float2(0.5f, 0.5f), mone = make_float2(-1.f, -1.f);
    o[0] = __ffma2_rn(mone, zeta, one);
    o[1] = __fmul2_rn(half, __fadd2_rn(zeta, xi));
    o[2] = __fmul2_rn(half, __ffma2_rn(mone, xi, zeta));
}
__device__ __forceinline__ void hpsi3_x2(float2 u, float2 th, float2* o)
{
    const float2 half = make_float2(0.5f, 0.5f), f25 = make_float2(2.5f, 2.5f), mone = make_float2(-1.f, -1.f);
    const float2 u2 = __fmul2_rn(u, u);
    const float2 hu2 = __fmul2_rn(half, u2);
    const float2 o1 = __ffma2_rn(th, u, __fmul2_rn(hu2, u));
    const float2 o2 = __ffma2_rn(th, th, __ffma2_rn(__fmul2_rn(f25, th), u2, __fmul2_rn(hu2, u2)));
    o[0] = __ffma2_rn(mone, o2, hu2);
    o[1] = __fmul2_rn(half, __fadd2_rn(o2, o1));
    o[2] = __fmul2_rn(half, __ffma2_rn(mone, o1, o2));
}

// In the isothermal mode g is relaxed here all the same and never read: f's
// collision takes nothing from g, and skipping it under a runtime test cost
// the fused kernel more than the work it saved.
template <int D, typename R, typename C>
__device__ __forceinline__ void collide_cell(const C& s, const Macro<R>& m, R divu, const R* gh, const R* gT,
                                             const R* Phi, R* f, R* g)
{
    constexpr int Q = Lat<D>::Q;
    const R rho = m.rho;
    // shifted states (Eqs. sh_vel_1, sh_temp_1, sh_T_1, qc_1), lambda = dt = 1
    R us[3], qc[3], FF = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        us[a] = a < D ? m.u[a] + m.F[a] * m.ir : R(0);
        FF += m.F[a] * m.F[a];
        qc[a] = a < D ? m.P * (gh[a] - (R)s.k_mu * gT[a]) : R(0);
    }
    R ths = m.theta + m.athe * divu + (m.gam - R(1)) * m.Q * m.ir;
    R Ts = m.T + (m.Q * m.ir - R(0.5) * FF * m.ir * m.ir) * m.icv;
    RhoPart<R> p = rho_part<R>(s, rho);
    R es = eos_e<R>(s, p, Ts);

    // per-axis factors
    R A0[3][3], As[3][3], B0[3][3], H0[3][3], Hs[3][3];
    if constexpr (D == 2 && std::is_same<R, float>::value) {
        // the x and y factors side by side in two-wide float32 operations
        const float2 u2v = make_float2(m.u[0], m.u[1]), usv = make_float2(us[0], us[1]);
        const float2 thv = make_float2(m.theta, m.theta), tsv = make_float2(ths, ths);
        const float2 phv = make_float2(Phi[0], Phi[1]);
        float2 a0[3], as[3], b0[3], h0[3], hs[3];
        const float2 zs = __ffma2_rn(usv, usv, tsv);
        psi3_x2(u2v, __ffma2_rn(u2v, u2v, thv), a0);
        psi3_x2(usv, __fadd2_rn(zs, phv), as);
        psi3_x2(usv, zs, b0);
        hpsi3_x2(u2v, thv, h0);
        hpsi3_x2(usv, tsv, hs);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            A0[0][d] = a0[d].x; A0[1][d] = a0[d].y;
            As[0][d] = as[d].x; As[1][d] = as[d].y;
            B0[0][d] = b0[d].x; B0[1][d] = b0[d].y;
            H0[0][d] = h0[d].x; H0[1][d] = h0[d].y;
            Hs[0][d] = hs[d].x; Hs[1][d] = hs[d].y;
        }
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            psi3<R>(m.u[a], m.theta + m.u[a] * m.u[a], A0[a]);              // f^eq, g^eq
            psi3<R>(us[a], ths + us[a] * us[a] + Phi[a], As[a]);            // f*
            psi3<R>(us[a], ths + us[a] * us[a], B0[a]);                     // g* (no Phi)
            hpsi3<R>(m.u[a], m.theta, H0[a]);
            hpsi3<R>(us[a], ths, Hs[a]);
        }
    }
    R bf = (R)s.beta_f, bg = (R)s.beta_g;
    if (s.mu > 0) bf = bg = relax_beta<R>(s, m.P);
    const R cf0 = R(1) - R(2) * bf, cf1 = R(3) * bf - R(1), cf2 = R(1) - bf;
    const R cg0 = R(1) - R(2) * bg, cg1 = R(3) * bg - R(1), cg2 = R(1) - bg;
    //   f'_i = cf0 f_i + cf1 f^eq_i + cf2 f*_i,  g'_i = cg0 g_i + cg1 g^eq_i + cg2 g*_i
    if constexpr (D == 2) {
        // The relaxation is linear in the equilibria, so rho and its weights are
        // folded into the x factors once: g^eq = rho [(e A0x + H0x) A0y + A0x H0y],
        // g* likewise from B0, Hs, e*, plus 1/2 c.q^c for |c|^2 = 1.
        const R r1 = cf1 * rho, r2 = cf2 * rho, s1 = cg1 * rho, s2 = cg2 * rho;
        R hq[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) hq[a] = cg2 * R(0.5) * qc[a];
        R fa[3], fs[3], ga[3], gh0[3], gb[3], gk[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            fa[d] = r1 * A0[0][d];
            fs[d] = r2 * As[0][d];
            ga[d] = s1 * (m.e * A0[0][d] + H0[0][d]);
            gh0[d] = s1 * A0[0][d];
            gb[d] = s2 * (es * B0[0][d] + Hs[0][d]);
            gk[d] = s2 * B0[0][d];
        }
        if constexpr (std::is_same<R, float>::value) {
            // f_i and g_i side by side in two-wide float32 multiply-adds (the
            // same products, sums and rounding as the scalar lines below)
            const float2 c0 = make_float2(cf0, cg0);
            float2 P1[3], P2[3], Q1[3], Q2[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                P1[d] = make_float2(fa[d], ga[d]);
                P2[d] = make_float2(fs[d], gh0[d]);
                Q1[d] = make_float2(A0[1][d], A0[1][d]);
                Q2[d] = make_float2(As[1][d], H0[1][d]);
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int d0 = dig(i, 0), d1 = dig(i, 1);
                float2 w = __fmul2_rn(c0, make_float2(f[i], g[i]));
                w = __ffma2_rn(P1[d0], Q1[d1], w);
                w = __ffma2_rn(P2[d0], Q2[d1], w);
                f[i] = w.x;
                R gi = w.y + gb[d0] * B0[1][d1] + gk[d0] * Hs[1][d1];
                if (cnorm2(i) == 1) gi += cc(i, 0) != 0 ? R(cc(i, 0)) * hq[0] : R(cc(i, 1)) * hq[1];
                g[i] = gi;
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int d0 = dig(i, 0), d1 = dig(i, 1);
                f[i] = cf0 * f[i] + fa[d0] * A0[1][d1] + fs[d0] * As[1][d1];
                R gi = cg0 * g[i] + ga[d0] * A0[1][d1] + gh0[d0] * H0[1][d1] + gb[d0] * B0[1][d1] + gk[d0] * Hs[1][d1];
                if (cnorm2(i) == 1) gi += cc(i, 0) != 0 ? R(cc(i, 0)) * hq[0] : R(cc(i, 1)) * hq[1];
                g[i] = gi;
            }
        }
    } else {
        // 3-D: per population (folding the xy products costs registers that the
        // 3-D kernels do not have to spare; measured slower)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int d0 = dig(i, 0), d1 = dig(i, 1), d2 = dig(i, 2);
            const R a01 = A0[0][d0] * A0[1][d1];
            const R feq = rho * a01 * A0[2][d2];
            const R fst = rho * As[0][d0] * As[1][d1] * As[2][d2];
            const R geq = rho * ((m.e * a01 + H0[0][d0] * A0[1][d1] + A0[0][d0] * H0[1][d1]) * A0[2][d2] + a01 * H0[2][d2]);
            const R b01 = B0[0][d0] * B0[1][d1];
            R gst = rho * ((es * b01 + Hs[0][d0] * B0[1][d1] + B0[0][d0] * Hs[1][d1]) * B0[2][d2] + b01 * Hs[2][d2]);
            if (cnorm2(i) == 1) {
                R cq = R(0);
#pragma unroll
                for (int a = 0; a < D; ++a) cq += R(cc(i, a)) * qc[a];
                gst += R(0.5) * cq;
            }
            f[i] = cf0 * f[i] + cf1 * feq + cf2 * fst;
            g[i] = cg0 * g[i] + cg1 * geq + cg2 * gst;
        }
    }
}

// The same collision split per population, so that a kernel can stream f
// and then g through the registers: make() forms the per-axis factors of
// f^eq and f* (and keeps the few scalars g needs), f<I>() relaxes f_I;
// prepare_g() forms the factors of g^eq and g*, and g<I>() relaxes g_I.
template <int D, typename R> struct Coll {
    R rho, e, es, qc[3];
    R u[3], th, us[3], ths;
    R A0[3][3], As[3][3], B0[3][3], H0[3][3], Hs[3][3];
    R cf0, cf1, cf2, cg0, cg1, cg2;

    // ES_FROM_CV: e(rho, T*) from e(rho, T) and the local c_v instead of the
    // equation of state.  e is linear in T for the ideal and van der Waals
    // gases; for Peng-Robinson e(T) = cv0 T - A(rho) (1 + k - k sqrt(T/Tc))
    // and c_v(T) = cv0 + A k / (2 sqrt(T Tc)) give
    //   e(T*) = e(T) + cv0 (T* - T) + 2 (c_v(T) - cv0)(sqrt(T T*) - T)
    // exactly (one square root; no logarithm or division).
    template <bool ES_FROM_CV = false, typename C>
    __device__ __forceinline__ static Coll make(const C& s, const Macro<R>& m, R divu, const R* gh, const R* gT,
                                                const R* Phi)
    {
        Coll c;
        c.rho = m.rho;
        c.e = m.e;
        c.th = m.theta;
        R FF = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c.u[a] = m.u[a];
            c.us[a] = a < D ? m.u[a] + m.F[a] * m.ir : R(0);
            FF += m.F[a] * m.F[a];
            c.qc[a] = a < D ? m.P * (gh[a] - (R)s.k_mu * gT[a]) : R(0);
        }
        c.ths = m.theta + m.athe * divu + (m.gam - R(1)) * m.Q * m.ir;
        const R Ts = m.T + (m.Q * m.ir - R(0.5) * FF * m.ir * m.ir) * m.icv;
        if constexpr (ES_FROM_CV) {
            c.es = m.e + (R)s.cv * (Ts - m.T);
            if (s.eos == EOS_PR) c.es += R(2) * (m.cv - (R)s.cv) * (sqrt(m.T * Ts) - m.T);
        } else {
            const RhoPart<R> p = rho_part<R>(s, m.rho);
            c.es = eos_e<R>(s, p, Ts);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            psi3<R>(m.u[a], m.theta + m.u[a] * m.u[a], c.A0[a]);
            psi3<R>(c.us[a], c.ths + c.us[a] * c.us[a] + Phi[a], c.As[a]);
        }
        R bf = (R)s.beta_f, bg = (R)s.beta_g;
        if (s.mu > 0) bf = bg = relax_beta<R>(s, m.P);
        c.cf0 = R(1) - R(2) * bf;
        c.cf1 = R(3) * bf - R(1);
        c.cf2 = R(1) - bf;
        c.cg0 = R(1) - R(2) * bg;
        c.cg1 = R(3) * bg - R(1);
        c.cg2 = R(1) - bg;
        return c;
    }

    __device__ __forceinline__ void prepare_g()
    {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            psi3<R>(us[a], ths + us[a] * us[a], B0[a]);
            hpsi3<R>(u[a], th, H0[a]);
            hpsi3<R>(us[a], ths, Hs[a]);
        }
    }

    // post-collision f_i from pre-collision f_i
    template <int I> __device__ __forceinline__ R f(R fi) const
    {
        constexpr int d0 = dig(I, 0), d1 = dig(I, 1), d2 = dig(I, 2);
        R feq, fst;
        if (D == 2) {
            feq = rho * A0[0][d0] * A0[1][d1];
            fst = rho * As[0][d0] * As[1][d1];
        } else {
            feq = rho * A0[0][d0] * A0[1][d1] * A0[2][d2];
            fst = rho * As[0][d0] * As[1][d1] * As[2][d2];
        }
        return cf0 * fi + cf1 * feq + cf2 * fst;
    }

    // post-collision g_i from pre-collision g_i (after prepare_g)
    template <int I> __device__ __forceinline__ R g(R gi) const
    {
        constexpr int d0 = dig(I, 0), d1 = dig(I, 1), d2 = dig(I, 2);
        R geq, gst;
        if (D == 2) {
            geq = rho * (e * A0[0][d0] * A0[1][d1] + H0[0][d0] * A0[1][d1] + A0[0][d0] * H0[1][d1]);
            gst = rho * (es * B0[0][d0] * B0[1][d1] + Hs[0][d0] * B0[1][d1] + B0[0][d0] * Hs[1][d1]);
        } else {
            const R a01 = A0[0][d0] * A0[1][d1];
            geq = rho * ((e * a01 + H0[0][d0] * A0[1][d1] + A0[0][d0] * H0[1][d1]) * A0[2][d2] + a01 * H0[2][d2]);
            const R b01 = B0[0][d0] * B0[1][d1];
            gst = rho * ((es * b01 + Hs[0][d0] * B0[1][d1] + B0[0][d0] * Hs[1][d1]) * B0[2][d2] + b01 * Hs[2][d2]);
        }
        if (cnorm2(I) == 1) {
            R cq = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) cq += R(cc(I, a)) * qc[a];
            gst += R(0.5) * cq;
        }
        return cg0 * gi + cg1 * geq + cg2 * gst;
    }
};

// compile-time loop over the populations
template <int I, int N, typename F> __device__ __forceinline__ void static_for(F&& fn)
{
    if constexpr (I < N) {
        fn(std::integral_constant<int, I>{});
        static_for<I + 1, N>(fn);
    }
}

// Rest equilibria (used for initialisation and the 16-bit storage offsets).
template <int D, typename R>
__host__ __device__ __forceinline__ void equilibria(R rho, const R* u, R theta, R e, R* f, R* g)
{
    constexpr int Q = Lat<D>::Q;
    R A0[3][3], H0[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        psi3<R>(u[a], theta + u[a] * u[a], A0[a]);
        hpsi3<R>(u[a], theta, H0[a]);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int d0 = dig(i, 0), d1 = dig(i, 1), d2 = dig(i, 2);
        if (D == 2) {
            f[i] = rho * A0[0][d0] * A0[1][d1];
            g[i] = rho * (e * A0[0][d0] * A0[1][d1] + H0[0][d0] * A0[1][d1] + A0[0][d0] * H0[1][d1]);
        } else {
            R a01 = A0[0][d0] * A0[1][d1];
            f[i] = rho * a01 * A0[2][d2];
            g[i] = rho * ((e * a01 + H0[0][d0] * A0[1][d1] + A0[0][d0] * H0[1][d1]) * A0[2][d2] + a01 * H0[2][d2]);
        }
    }
}

// ---------------------------------------------------------------------------
// Addressing: periodic wrap in x, y (and z without walls); for macroscopic
// stencils a cell beyond a z wall stands for its mirror image about the wall
// (sign flips the velocity).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ int mirror_z(int z, int nz, bool& flip)
{
    flip = false;
#pragma unroll 1
    for (int k = 0; k < 4 && (z < 0 || z >= nz); ++k) {
        z = z < 0 ? -1 - z : 2 * nz - 1 - z;
        flip = !flip;
    }
    return z;
}

// cell index of the stencil neighbour, with the mirror flag
template <typename C>
__device__ __forceinline__ long long nb_index(const C& s, int x, int y, int z, bool& flip)
{
    x = wrapi(x, s.nx);
    y = wrapi(y, s.ny);
    if (s.zwalls) {
        z = mirror_z(z, s.nz, flip);
    } else {
        flip = false;
        z = wrapi(z, s.nz);
    }
    return (long long)x + (long long)s.nx * ((long long)y + (long long)s.ny * (long long)z);
}

// Pull streaming: the pre-collision f_i(x) is f'_i(x - c_i); across a z wall
// (half-way bounce-back) it is f'_opp(i)(x).  Returns the storage element
// index within one distribution block and the direction whose offset applies.
template <int D, typename C>
__device__ __forceinline__ long long pull_index(const C& s, int i, int x, int y, int z, int& isrc)
{
    int sx = wrapi(x - cc(i, 0), s.nx);
    int sy = wrapi(y - cc(i, 1), s.ny);
    int sz = z - (D == 3 ? cc(i, 2) : 0);
    isrc = i;
    if (D == 3) {
        if (s.zwalls && (sz < 0 || sz >= s.nz)) {
            sx = x;
            sy = y;
            sz = z;
            isrc = opp(i);
        } else {
            sz = wrapi(sz, s.nz);
        }
    } else {
        sz = 0;
    }
    long long k = (long long)sx + (long long)s.nx * ((long long)sy + (long long)s.ny * (long long)sz);
    return (long long)isrc * s.N + k;
}

}  // namespace lbm
