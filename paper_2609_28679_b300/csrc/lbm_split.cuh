// Per-cell kernels: initialisation, the three-pass ("split") time step,
// export of fields/populations and the float64 conservation reduction.
//
// Work arrays W are [NF][Ntot] in the arithmetic type R; field f of global
// cell (cell_off + k) sits at W[f * Ntot + cell_off + k].  Kernels run over a
// block table: block b handles cells [start, start + 256) of simulation sim.
#pragma once

#include "lbm_device.cuh"
#include "lbm_mlp.cuh"

namespace lbm {

enum Field {
    W_RHO = 0, W_J = 1, W_G = 4, W_U = 5, W_T = 8, W_H = 9, W_X = 10, W_F = 13,
    W_P = 16, W_TH = 17, W_CV = 18, W_GAM = 19, W_ATHE = 20, W_E = 21, W_NF = 22
};

// carried per-cell values of the one-pass and z-march paths: rho, j (3), G, T (Newton guess)
enum MField { M_RHO = 0, M_J = 1, M_G = 4, M_T = 5, M_NF = 6 };

constexpr int kBlockCells = 256;

// device diagnostic counters: slots 0-3 are the ones lbm_diagnostics reports
// (non-finite state, theta <= 0, Newton cap, learned-T fallback); slot 4
// counts the cells lbm_init rejected (rho <= 0 or T <= 0, or NaN)
constexpr int kDiagInitBad = 4;
constexpr int kDiagSlots = 8;

struct BlockEntry {
    int sim;
    int start;
};

// Copy the simulation's constants to shared memory (one block = one simulation).
__device__ __forceinline__ void load_sim(SimDev& dst, const SimDev* sims, int sim)
{
    const int n = (int)(sizeof(SimDev) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(sims + sim);
    int* d = reinterpret_cast<int*>(&dst);
    for (int t = threadIdx.x; t < n; t += blockDim.x) d[t] = src[t];
    __syncthreads();
}

template <typename C>
__device__ __forceinline__ void cell_xyz(const C& s, long long k, int& x, int& y, int& z)
{
    // k < N, and lbm_create keeps Q N below 2^32 per simulation: 32-bit division
    const unsigned ku = (unsigned)k, nx = (unsigned)s.nx, ny = (unsigned)s.ny;
    const unsigned r = ku / nx;
    x = (int)(ku - r * nx);
    z = (int)(r / ny);
    y = (int)(r - (unsigned)z * ny);
}

template <typename C>
__device__ __forceinline__ double heat_at(const C& s, int z)
{
    return (s.zhi <= 0 || (z >= s.zlo && z < s.zhi)) ? (double)s.q : 0.0;
}

// heat source of a cell in the arithmetic type
template <typename R, typename C>
__device__ __forceinline__ R heat_q(const C& s, int z)
{
    return (s.zhi <= 0 || (z >= s.zlo && z < s.zhi)) ? (R)s.q : R(0);
}

// Warp-aggregated diagnostic counters (bit 0: non-finite, 1: theta <= 0,
// 2: Newton cap, 3: learned temperature not accepted by the residual test).
__device__ __forceinline__ void count_flags(unsigned flags, unsigned long long* diag)
{
    if (!__any_sync(0xffffffffu, flags != 0u)) return;  // the usual case: nothing to count in this warp
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        unsigned m = __ballot_sync(0xffffffffu, (flags >> b) & 1u);
        if (lane == 0 && m) atomicAdd(diag + b, (unsigned long long)__popc(m));
    }
}

// ---------------------------------------------------------------------------
// Initial state: f = f^eq(rho, u, theta), g = g^eq (flowchart, first box),
// written where the first pull reads them.
// ---------------------------------------------------------------------------
template <int D, typename R, typename S, typename H = double>
__global__ void __launch_bounds__(kBlockCells) k_init(const SimDev* __restrict__ sims, const BlockEntry* __restrict__ table,
                                                      const H* __restrict__ rho_in, const H* __restrict__ u_in,
                                                      const H* __restrict__ T_in, S* __restrict__ pop,
                                                      R* __restrict__ W, long long Ntot,
                                                      unsigned long long* __restrict__ bad)
{
    constexpr int Q = Lat<D>::Q;
    __shared__ SimDev s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long k = (long long)be.start + threadIdx.x;
    if (k >= s.N) return;
    int x, y, z;
    cell_xyz(s, k, x, y, z);
    const long long gk = s.cell_off + k;
    const double rho_d = rho_in[gk], T_d = T_in[gk];
    if (!(rho_d > 0.0) || !(T_d > 0.0)) atomicAdd(bad, 1ull);
    R rho = (R)rho_d, T = (R)T_d, u[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = (R)u_in[(long long)D * s.cell_off + (long long)a * s.N + k];
    RhoPart<R> p = rho_part<R>(s, rho);
    R th = eos_P<R>(s, p, T) / rho;
    R e = eos_e<R>(s, p, T);
    R f[Q], g[Q];
    equilibria<D, R>(rho, u, th, e, f, g);
    S* fb = pop + s.pop_off;
    S* gb = fb + (long long)Q * s.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // slot read by the pull of (x, i): (i, x - c_i), or (opp(i), x) across a wall
        int sx = wrapi(x - cc(i, 0), s.nx), sy = wrapi(y - cc(i, 1), s.ny), sz = z - (D == 3 ? cc(i, 2) : 0);
        int j = i;
        if (D == 3 && s.zwalls && (sz < 0 || sz >= s.nz)) {
            sx = x; sy = y; sz = z; j = opp(i);
        } else if (D == 3) {
            sz = wrapi(sz, s.nz);
        } else {
            sz = 0;
        }
        long long kk = (long long)sx + (long long)s.nx * ((long long)sy + (long long)s.ny * (long long)sz);
        R fo = Codec<S, R>::offset ? (R)s.fref[j] : R(0);
        R go = Codec<S, R>::offset ? (R)s.gref[j] : R(0);
        Codec<S, R>::st(fb + (long long)j * s.N + kk, f[i] - fo);
        Codec<S, R>::st(gb + (long long)j * s.N + kk, g[i] - go);
    }
    W[W_T * Ntot + gk] = T;
}

// Pre-collision populations of cell (x,y,z), decoded to R.
template <int D, typename R, typename S>
__device__ __forceinline__ void pull_cell(const SimDev& s, const S* __restrict__ pop, int x, int y, int z, R* f, R* g)
{
    constexpr int Q = Lat<D>::Q;
    const S* fb = pop + s.pop_off;
    const S* gb = fb + (long long)Q * s.N;
    if (x >= 1 && x < s.nx - 1 && y >= 1 && y < s.ny - 1 && (D == 2 || (z >= 1 && z < s.nz - 1))) {
        // every source cell x - c_i lies inside the lattice: the same elements at
        // fixed offsets c_x + c_y nx + c_z nx ny from the cell
        const long long k = (long long)x + (long long)s.nx * ((long long)y + (long long)s.ny * (long long)z);
        const long long NX = s.nx, NP = (long long)s.nx * s.ny;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const long long idx = (long long)i * s.N + k - (cc(i, 0) + cc(i, 1) * NX + (D == 3 ? cc(i, 2) * NP : 0));
            f[i] = Codec<S, R>::ld(fb + idx);
            g[i] = Codec<S, R>::ld(gb + idx);
            if (Codec<S, R>::offset) {
                f[i] += (R)s.fref[i];
                g[i] += (R)s.gref[i];
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int j;
        long long idx = pull_index<D>(s, i, x, y, z, j);
        f[i] = Codec<S, R>::ld(fb + idx);
        g[i] = Codec<S, R>::ld(gb + idx);
        if (Codec<S, R>::offset) {
            f[i] += (R)s.fref[j];
            g[i] += (R)s.gref[j];
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 1: moments rho = sum f (Eq. def_h), j = sum c f, G = sum g.
// ---------------------------------------------------------------------------
template <int D, typename R, typename S>
__global__ void __launch_bounds__(kBlockCells) k_moments(const SimDev* __restrict__ sims, const BlockEntry* __restrict__ table,
                                                         const S* __restrict__ pop, R* __restrict__ W, long long Ntot)
{
    constexpr int Q = Lat<D>::Q;
    __shared__ SimDev s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long k = (long long)be.start + threadIdx.x;
    if (k >= s.N) return;
    int x, y, z;
    cell_xyz(s, k, x, y, z);
    R f[Q], g[Q];
    pull_cell<D, R, S>(s, pop, x, y, z, f, g);
    R rho = 0, j[3] = {0, 0, 0}, G = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
#pragma unroll
        for (int a = 0; a < D; ++a) j[a] += R(cc(i, a)) * f[i];
        G += g[i];
    }
    const long long gk = s.cell_off + k;
    W[W_RHO * Ntot + gk] = rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) W[(W_J + a) * Ntot + gk] = j[a];
    W[W_G * Ntot + gk] = G;
}

// Coordinate v + o (|o| small) of an in-domain coordinate v: periodic, or,
// with mirror set, the image about the walls of a cell beyond them.
__device__ __forceinline__ int nb_coord(int v, int o, int n, bool mirror)
{
    int w = v + o;
    if (mirror) {
        if (w < 0) w = -1 - w;
        else if (w >= n) w = 2 * n - 1 - w;
        if ((unsigned)w >= (unsigned)n) {
            bool fl;
            w = mirror_z(v + o, n, fl);
        }
    } else {
        if (w < 0) w += n;
        else if (w >= n) w -= n;
        if ((unsigned)w >= (unsigned)n) w = wrapi(v + o, n);
    }
    return w;
}

// Value of field v at (x, y, z) between non-equilibrium-extrapolation walls
// on the boundary cells z_B = 0 and nz - 1: v itself inside, the linear
// extrapolation 2 v(z_B) - v(2 z_B - z) through the boundary cell past it
// (x, y in the domain, z at most nz - 1 cells past a face).
template <typename R, typename V>
__device__ __forceinline__ R zval(const V& v, int x, int y, int z, int nz, int walls)
{
    if (z < 0 || z >= nz) {
        const int zb = z < 0 ? 0 : nz - 1;
        return R(2) * v(x, y, zb) - v(x, y, 2 * zb - z);
    }
    return v(x, y, z);
}

// lap rho at the in-domain cell (ix, iy, iz): (2D+1)-point stencil, with
// neighbours past a z wall as zval gives them
template <int D, typename R>
__device__ __forceinline__ R lap_img(const R* __restrict__ rho, int ix, int iy, int iz, int nx, int ny, int nz,
                                     int walls)
{
    auto at = [&](int x, int y, int z) {
        return rho[(long long)x + (long long)nx * ((long long)y + (long long)ny * (long long)z)];
    };
    const R c = at(ix, iy, iz);
    R L = 0;
    L += at(nb_coord(ix, 1, nx, false), iy, iz) - R(2) * c + at(nb_coord(ix, -1, nx, false), iy, iz);
    L += at(ix, nb_coord(iy, 1, ny, false), iz) - R(2) * c + at(ix, nb_coord(iy, -1, ny, false), iz);
    if (D == 3) {
        if (walls == 2)
            L += zval<R>(at, ix, iy, iz + 1, nz, 2) - R(2) * c + zval<R>(at, ix, iy, iz - 1, nz, 2);
        else
            L += at(ix, iy, nb_coord(iz, 1, nz, walls == 1)) - R(2) * c + at(ix, iy, nb_coord(iz, -1, nz, walls == 1));
    }
    return L;
}

// Korteweg gradient of lap rho at (x, y, z) (central difference of lap rho
// between the images of the two neighbours along each axis; past a
// non-equilibrium-extrapolation wall lap rho is extrapolated like any field)
template <int D, typename R>
__device__ __forceinline__ void grad_lap(const R* __restrict__ rho, int x, int y, int z, int nx, int ny, int nz,
                                         int walls, R* gl)
{
    gl[0] = R(0.5) * (lap_img<D, R>(rho, nb_coord(x, 1, nx, false), y, z, nx, ny, nz, walls) -
                      lap_img<D, R>(rho, nb_coord(x, -1, nx, false), y, z, nx, ny, nz, walls));
    gl[1] = R(0.5) * (lap_img<D, R>(rho, x, nb_coord(y, 1, ny, false), z, nx, ny, nz, walls) -
                      lap_img<D, R>(rho, x, nb_coord(y, -1, ny, false), z, nx, ny, nz, walls));
    if (D == 3 && walls == 2) {
        auto lap = [&](int xx, int yy, int zz) { return lap_img<D, R>(rho, xx, yy, zz, nx, ny, nz, 2); };
        gl[2] = R(0.5) * (zval<R>(lap, x, y, z + 1, nz, 2) - zval<R>(lap, x, y, z - 1, nz, 2));
    } else {
        gl[2] = D == 3 ? R(0.5) * (lap_img<D, R>(rho, x, y, nb_coord(z, 1, nz, walls == 1), nx, ny, nz, walls) -
                                   lap_img<D, R>(rho, x, y, nb_coord(z, -1, nz, walls == 1), nx, ny, nz, walls))
                       : R(0);
    }
}

// K phi(z) of the Darcy throttle at layer z (0 without one)
__device__ __forceinline__ double throttle_phi(const SimDev& s, int z)
{
    if (!(s.throttle_K > 0.0)) return 0.0;
    const double d = ((double)z - 0.5 * (double)(s.nz - 1)) / s.throttle_sigma;
    return s.throttle_K * exp(-d * d);
}

// Duct resistance: friction (Fanno flow) and throttle (throttling process),
// F_r = -rho (K phi + k |u|) u joins F and Q gains Q_r = -F_r.u, with
// u = (j + F/2)/rho solved exactly: for w the velocity without F_r and
// a = 1 + K phi/2, |u| (a + k |u|/2) = |w|, so u = 2 w / (a + sqrt(a^2 + 2 k |w|)).
template <int D, typename R>
__device__ __forceinline__ void apply_friction(const SimDev& s, int z, R r, const R* j, R* F, R& Q)
{
    const R Kphi = (R)throttle_phi(s, z);
    if (!(s.friction > 0.0) && !(Kphi > R(0))) return;
    const R k = (R)s.friction;
    R w[3] = {0, 0, 0}, wn = 0, un = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        w[a] = (j[a] + R(0.5) * F[a]) / r;
        wn += w[a] * w[a];
    }
    wn = sqrt(wn);
    const R a0 = R(1) + R(0.5) * Kphi;
    const R sc = R(2) / (a0 + sqrt(a0 * a0 + R(2) * k * wn));
#pragma unroll
    for (int a = 0; a < D; ++a) un += (sc * w[a]) * (sc * w[a]);
    un = sqrt(un);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const R Ff = -r * (Kphi + k * un) * (sc * w[a]);
        F[a] += Ff;
        Q -= Ff * (sc * w[a]);
    }
}

// heat source of cell k (layer z): the uniform or masked Q, the caller's per-cell Q, and the resistance
// heat rho (K phi + k |u|) |u|^2 at its velocity
template <int D, typename R>
__device__ __forceinline__ R cell_heat(const SimDev& s, int z, long long k, R r, const R* u)
{
    R Q = (R)(heat_at(s, z) + (s.qfield ? s.qfield[k] : 0.0));
    const R Kphi = (R)throttle_phi(s, z);
    if (s.friction > 0.0 || Kphi > R(0)) {
        R u2 = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) u2 += u[a] * u[a];
        Q += r * (Kphi + (R)s.friction * sqrt(u2)) * u2;
    }
    return Q;
}

// ---------------------------------------------------------------------------
// Pass 2: force, velocity, energy, temperature and closure scalars per cell.
// ---------------------------------------------------------------------------
// FROM_M: rho, j, G come from the carried moments M (z-march path) and rho is
// copied into W; otherwise from W (written by k_moments).
template <int D, typename R, bool FROM_M = false>
__global__ void __launch_bounds__(kBlockCells) k_macro(const SimDev* __restrict__ sims, const BlockEntry* __restrict__ table,
                                                       R* __restrict__ W, long long Ntot, unsigned long long* diag,
                                                       const R* __restrict__ M = nullptr)
{
    __shared__ SimDev s;
    __shared__ MlpSmem mlp_s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const bool use_mlp = s.eos == EOS_PR && s.t_solver == 1 && s.mlp != nullptr;  // block-uniform
    if (use_mlp) {
        mlp_load(mlp_s, s.mlp);
        __syncthreads();
    }
    const long long k = (long long)be.start + threadIdx.x;
    const bool valid = k < s.N;
    unsigned flags = 0;
    R Tml = R(0);
    if (use_mlp) {
        // learned start of the temperature inversion, one warp per 32 cells
        float rr = 1.f, ee = 0.f;
        if (valid) {
            int x, y, z;
            cell_xyz(s, k, x, y, z);
            const long long gk = s.cell_off + k;
            const R* rho = (FROM_M ? M + M_RHO * Ntot : W + W_RHO * Ntot) + s.cell_off;
            const R r = rho[k];
            R F[3] = {0, 0, 0}, j[3], gl[3];
            grad_lap<D, R>(rho, x, y, z, s.nx, s.ny, s.nz, s.zwalls, gl);
#pragma unroll
            for (int a = 0; a < D; ++a)
                F[a] = r * (R)s.acc[a] + (R)s.kappa * r * gl[a] + (s.ffield ? (R)s.ffield[(long long)a * s.N + k] : R(0));
#pragma unroll
            for (int a = 0; a < 3; ++a) j[a] = FROM_M ? M[(M_J + a) * Ntot + gk] : W[(W_J + a) * Ntot + gk];
            R Qc = (R)(heat_at(s, z) + (s.qfield ? s.qfield[k] : 0.0));
            apply_friction<D, R>(s, z, r, j, F, Qc);
            rr = (float)r;
            ee = (float)macro_energy<D, R>(r, j, FROM_M ? M[M_G * Ntot + gk] : W[W_G * Ntot + gk], F, Qc);
        }
        Tml = (R)mlp_T_warp(mlp_s, rr, ee);
    }
    if (valid) {
        int x, y, z;
        cell_xyz(s, k, x, y, z);
        const long long gk = s.cell_off + k;
        const R* rho = (FROM_M ? M + M_RHO * Ntot : W + W_RHO * Ntot) + s.cell_off;
        R r = rho[k];
        R F[3] = {0, 0, 0}, j[3], gl[3];
        grad_lap<D, R>(rho, x, y, z, s.nx, s.ny, s.nz, s.zwalls, gl);
#pragma unroll
        for (int a = 0; a < D; ++a)  // Eqs. force_decomposition, korteweg_force; the caller's F_B(x)
            F[a] = r * (R)s.acc[a] + (R)s.kappa * r * gl[a] + (s.ffield ? (R)s.ffield[(long long)a * s.N + k] : R(0));
#pragma unroll
        for (int a = 0; a < 3; ++a) j[a] = FROM_M ? M[(M_J + a) * Ntot + gk] : W[(W_J + a) * Ntot + gk];
        R Q = (R)(heat_at(s, z) + (s.qfield ? s.qfield[k] : 0.0));
        apply_friction<D, R>(s, z, r, j, F, Q);
        Macro<R> m = macro_cell<D, R>(s, r, j, FROM_M ? M[M_G * Ntot + gk] : W[W_G * Ntot + gk], F, Q,
                                      use_mlp ? Tml : W[W_T * Ntot + gk], flags);
        if (FROM_M) W[W_RHO * Ntot + gk] = r;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            W[(W_U + a) * Ntot + gk] = m.u[a];
            W[(W_F + a) * Ntot + gk] = m.F[a];
            W[(W_X + a) * Ntot + gk] = a < D ? xflux<R>(r, m.u[a], m.theta) : R(0);
        }
        W[W_T * Ntot + gk] = m.T;
        W[W_H * Ntot + gk] = m.h;
        W[W_P * Ntot + gk] = m.P;
        W[W_TH * Ntot + gk] = m.theta;
        W[W_CV * Ntot + gk] = m.cv;
        W[W_GAM * Ntot + gk] = m.gam;
        W[W_ATHE * Ntot + gk] = m.athe;
        W[W_E * Ntot + gk] = m.e;
    }
    if (diag) count_flags(flags, diag);
}

template <typename R>
__device__ __forceinline__ R wget(const SimDev& s, const R* __restrict__ fld, int x, int y, int z, bool odd)
{
    if (s.zwalls == 2 && (z < 0 || z >= s.nz)) {
        // past a non-equilibrium-extrapolation wall: linear extrapolation through the boundary cell
        const int zb = z < 0 ? 0 : s.nz - 1;
        const long long xy = (long long)wrapi(x, s.nx) + (long long)s.nx * wrapi(y, s.ny);
        const long long plane = (long long)s.nx * s.ny;
        return R(2) * fld[xy + plane * zb] - fld[xy + plane * (2 * zb - z)];
    }
    bool fl;
    long long kk = nb_index(s, x, y, z, fl);
    R v = fld[kk];
    return (odd && fl) ? -v : v;
}

// Stencil quantities of cell (x,y,z): div u, grad h, grad T (central) and
// Phi (Eq. correction; upwind-biased or central derivative of X).
template <int D, typename R>
__device__ __forceinline__ void stencils(const SimDev& s, const R* __restrict__ W, long long Ntot, int x, int y, int z,
                                         R rho, const R* u, R& divu, R* gh, R* gT, R* Phi)
{
    const long long off = s.cell_off;
    divu = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) { gh[a] = 0; gT[a] = 0; Phi[a] = 0; }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int e0 = a == 0, e1 = a == 1, e2 = a == 2;
        const R* ua = W + (W_U + a) * Ntot + off;
        const R* h = W + W_H * Ntot + off;
        const R* T = W + W_T * Ntot + off;
        const R* X = W + (W_X + a) * Ntot + off;
        divu += R(0.5) * (wget(s, ua, x + e0, y + e1, z + e2, true) - wget(s, ua, x - e0, y - e1, z - e2, true));
        gh[a] = R(0.5) * (wget(s, h, x + e0, y + e1, z + e2, false) - wget(s, h, x - e0, y - e1, z - e2, false));
        gT[a] = R(0.5) * (wget(s, T, x + e0, y + e1, z + e2, false) - wget(s, T, x - e0, y - e1, z - e2, false));
        R dX;
        if (s.phi_central) {
            dX = R(0.5) * (wget(s, X, x + e0, y + e1, z + e2, true) - wget(s, X, x - e0, y - e1, z - e2, true));
        } else {
            const R X0 = wget(s, X, x, y, z, true);
            const R Xm1 = wget(s, X, x - e0, y - e1, z - e2, true), Xp1 = wget(s, X, x + e0, y + e1, z + e2, true);
            const int sg = u[a] >= R(0) ? -2 : 2;  // the second neighbour on the upwind side
            dX = upwind_biased<R>(u[a], wget(s, X, x + sg * e0, y + sg * e1, z + sg * e2, true), Xm1, X0, Xp1);
        }
        Phi[a] = -dX / rho;
    }
}

// ---------------------------------------------------------------------------
// Non-equilibrium-extrapolation walls (zwalls == 2; the wall treatment of the
// thermal Couette flow, App. B), between the macroscopic pass and the
// collision.  Each boundary cell z_B in {0, nz - 1} takes the wall velocity
// and temperature, the density rho_N of its neighbour z_N in {1, nz - 2}
// (wall_rho 1) or the density whose pressure at T_W is the neighbour's
// (wall_rho 0) or the linear extrapolation 2 P_N - P_NN from two cells
// inside (wall_rho 2) (eight Newton steps from rho_N, rho_N again if they
// end non-finite or non-positive); an open face (the duct ends of Sec. III.A)
// takes the boundary state of its kind instead (LBM_FACE_* in lbm.h).  The
// populations are
//   f_B = f^eq(rho_B, u_W, theta_W) + f_N - f^eq(rho_N, u_N, theta_N), g alike,
// written to the storage slots its pull reads (no other cell reads those).
// Its macroscopic fields become the wall state; its force keeps the
// per-mass value of the macroscopic pass.  pops = 0 rebuilds the fields
// only (for the reported moments and totals).
// ---------------------------------------------------------------------------
// face_table: blocks of (simulation, first face cell), the face cells of a
// simulation numbered z = 0 layer first, then z = nz - 1.
template <int D, typename R, typename S>
__global__ void __launch_bounds__(kBlockCells) k_nee(const SimDev* __restrict__ sims,
                                                     const BlockEntry* __restrict__ face_table, S* pop,
                                                     R* __restrict__ W, long long Ntot, int pops)
{
    constexpr int Q = Lat<D>::Q;
    __shared__ SimDev s;
    const BlockEntry be = face_table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long plane = (long long)s.nx * s.ny;
    const long long idx = (long long)be.start + threadIdx.x;
    if (D != 3 || s.zwalls != 2 || idx >= 2 * plane) return;
    const int side = idx >= plane ? 1 : 0;
    const long long k = side ? (long long)(s.nz - 1) * plane + (idx - plane) : idx;
    int x, y, z;
    cell_xyz(s, k, x, y, z);
    const long long gb = s.cell_off + k, gn = s.cell_off + (side ? k - plane : k + plane);
    const R rn = W[W_RHO * Ntot + gn];
    const int kind = s.face_kind[side];
    R uw[3], un[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        uw[a] = a < D ? (R)s.uw[side][a] : R(0);
        un[a] = W[(W_U + a) * Ntot + gn];
    }
    // boundary state (rho_B, u_B = uw, T_B = Tw) of the face's kind; Pt: the pressure rho_B must meet at Tw
    R Tw = (R)s.Tw[side], Pt = R(-1);
    if (kind == 0) {
        if (s.wall_rho == 0) Pt = W[W_P * Ntot + gn];  // P(rho_N, T_N)
        if (s.wall_rho == 2) {                        // 2 P_N - P_NN, NN two cells inside (nz >= 4)
            const long long gnn = s.cell_off + (side ? k - 2 * plane : k + 2 * plane);
            Pt = R(2) * W[W_P * Ntot + gn] - W[W_P * Ntot + gnn];
        }
    } else if (kind == 1) {  // subsonic inlet from the total state (ideal gas)
        const R cp = (R)s.cv + (R)s.R;
        R n2 = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) { uw[a] = un[a]; n2 += un[a] * un[a]; }
        const R T0 = Tw;
        Tw = T0 - R(0.5) * n2 / cp;
        Pt = (R)s.face_P[side] * pow(Tw / T0, cp / (R)s.R);
    } else if (kind == 2) {  // static inlet
        Pt = (R)s.face_P[side];
    } else if (kind == 3) {  // pressure outlet
        Tw = W[W_T * Ntot + gn];
        Pt = (R)s.face_P[side];
    } else if (kind == 5) {  // inlet at fixed static P and T
#pragma unroll
        for (int a = 0; a < D; ++a) uw[a] = un[a];
        Pt = (R)s.face_P[side];
    } else {  // extrapolated outlet
#pragma unroll
        for (int a = 0; a < D; ++a) uw[a] = un[a];
        Tw = W[W_T * Ntot + gn];
    }
    R rb = rn;
    if (Pt > R(0)) {
        R r = rn;
#pragma unroll 1
        for (int it = 0; it < 8; ++it) {
            const Thermo<R> t = thermo<R>(s, rho_part<R>(s, r), Tw);
            r -= (t.P - Pt) / t.Pr;
        }
        if (isfinite(r) && r > R(0)) rb = r;
    }
    if (kind == 3) {  // the neighbour's mass flux
#pragma unroll
        for (int a = 0; a < D; ++a) uw[a] = un[a] * (rn / rb);
    }
    const RhoPart<R> pb = rho_part<R>(s, rb);
    const Thermo<R> t = thermo<R>(s, pb, Tw);
    const R ib = R(1) / rb;
    const R thw = t.P * ib, ew = eos_e<R>(s, pb, Tw);
    if (pops) {
        R feqB[Q], geqB[Q], feqN[Q], geqN[Q], fN[Q], gN[Q];
        equilibria<D, R>(rb, uw, thw, ew, feqB, geqB);
        equilibria<D, R>(rn, un, W[W_TH * Ntot + gn], W[W_E * Ntot + gn], feqN, geqN);
        pull_cell<D, R, S>(s, pop, x, y, side ? z - 1 : z + 1, fN, gN);
        S* fb = pop + s.pop_off;
        S* gbuf = fb + (long long)Q * s.N;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int j;
            const long long idx = pull_index<D>(s, i, x, y, z, j);
            const R fo = Codec<S, R>::offset ? (R)s.fref[j] : R(0);
            const R go = Codec<S, R>::offset ? (R)s.gref[j] : R(0);
            Codec<S, R>::st(fb + idx, feqB[i] + (fN[i] - feqN[i]) - fo);
            Codec<S, R>::st(gbuf + idx, geqB[i] + (gN[i] - geqN[i]) - go);
        }
    }
    // force and heat: the non-friction part per unit mass kept, friction at (rho_B, u_B)
    const R ro = W[W_RHO * Ntot + gb], kf = (R)s.friction, Kphi = (R)throttle_phi(s, z);
    R uo[3], uo2 = 0, u2 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        uo[a] = W[(W_U + a) * Ntot + gb];
        if (a < D) { uo2 += uo[a] * uo[a]; u2 += uw[a] * uw[a]; }
    }
    const R uon = sqrt(uo2), ubn = sqrt(u2);
    const R Qh = cell_heat<D, R>(s, z, k, rb, uw);
    R uF = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R Ffo = a < D ? -ro * (Kphi + kf * uon) * uo[a] : R(0);
        const R Ffb = a < D ? -rb * (Kphi + kf * ubn) * uw[a] : R(0);
        const R Fa = (W[(W_F + a) * Ntot + gb] - Ffo) * (rb / ro) + Ffb;
        W[(W_F + a) * Ntot + gb] = Fa;
        W[(W_U + a) * Ntot + gb] = uw[a];
        W[(W_J + a) * Ntot + gb] = rb * uw[a] - R(0.5) * Fa;  // so that J + F/2 = rho_B u_B (Eq. def_u)
        W[(W_X + a) * Ntot + gb] = a < D ? xflux<R>(rb, uw[a], thw) : R(0);
        uF += uw[a] * Fa;
    }
    const R icv = s.eos == EOS_PR ? R(1) / t.cv : (R)s.inv_cv;
    const R cs2 = t.Pr + Tw * t.PT * t.PT * ib * ib * icv;
    W[W_RHO * Ntot + gb] = rb;
    W[W_G * Ntot + gb] = rb * (ew + R(0.5) * u2) - R(0.5) * (uF + Qh);  // rho E at the wall state (Eq. def_E)
    W[W_T * Ntot + gb] = Tw;
    W[W_E * Ntot + gb] = ew;
    W[W_P * Ntot + gb] = t.P;
    W[W_TH * Ntot + gb] = thw;
    W[W_H * Ntot + gb] = ew + thw;
    W[W_CV * Ntot + gb] = t.cv;
    W[W_GAM * Ntot + gb] = R(1) + t.PT * ib * icv;
    W[W_ATHE * Ntot + gb] = (R)s.athe_c * thw - cs2;
}

// ---------------------------------------------------------------------------
// Pass 3: shifted states, equilibria, collision and pull streaming.
// ---------------------------------------------------------------------------
template <int D, typename R, typename S>
__global__ void __launch_bounds__(kBlockCells) k_collide(const SimDev* __restrict__ sims, const BlockEntry* __restrict__ table,
                                                         const S* __restrict__ src, S* __restrict__ dst,
                                                         const R* __restrict__ W, long long Ntot)
{
    constexpr int Q = Lat<D>::Q;
    __shared__ SimDev s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long k = (long long)be.start + threadIdx.x;
    if (k >= s.N) return;
    int x, y, z;
    cell_xyz(s, k, x, y, z);
    const long long gk = s.cell_off + k;
    Macro<R> m;
    m.rho = W[W_RHO * Ntot + gk];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.u[a] = W[(W_U + a) * Ntot + gk];
        m.F[a] = W[(W_F + a) * Ntot + gk];
    }
    m.Q = cell_heat<D, R>(s, z, k, m.rho, m.u);
    m.T = W[W_T * Ntot + gk];
    m.P = W[W_P * Ntot + gk];
    m.theta = W[W_TH * Ntot + gk];
    m.h = W[W_H * Ntot + gk];
    m.cv = W[W_CV * Ntot + gk];
    m.gam = W[W_GAM * Ntot + gk];
    m.athe = W[W_ATHE * Ntot + gk];
    m.e = W[W_E * Ntot + gk];
    m.ir = R(1) / m.rho;
    m.icv = R(1) / m.cv;
    R divu, gh[3], gT[3], Phi[3];
    stencils<D, R>(s, W, Ntot, x, y, z, m.rho, m.u, divu, gh, gT, Phi);
    R f[Q], g[Q];
    pull_cell<D, R, S>(s, src, x, y, z, f, g);
    collide_cell<D, R>(s, m, divu, gh, gT, Phi, f, g);
    S* fb = dst + s.pop_off;
    S* gb = fb + (long long)Q * s.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        R fo = Codec<S, R>::offset ? (R)s.fref[i] : R(0);
        R go = Codec<S, R>::offset ? (R)s.gref[i] : R(0);
        Codec<S, R>::st(fb + (long long)i * s.N + k, f[i] - fo);
        Codec<S, R>::st(gb + (long long)i * s.N + k, g[i] - go);
    }
}

// ---------------------------------------------------------------------------
// Float64 totals per block (after k_moments + k_macro of the current state):
// [rho, rho u (D), rho E, F (D), u.F + Q].  Warp shuffles, then shared memory.
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void __launch_bounds__(kBlockCells) k_invariants(const SimDev* __restrict__ sims, const BlockEntry* __restrict__ table,
                                                            const R* __restrict__ W, long long Ntot, double* __restrict__ partials)
{
    constexpr int NV = 2 * D + 3;
    __shared__ SimDev s;
    __shared__ double red[kBlockCells / 32][NV];
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long k = (long long)be.start + threadIdx.x;
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = 0.0;
    if (k < s.N) {
        int x, y, z;
        cell_xyz(s, k, x, y, z);
        const long long gk = s.cell_off + k;
        double r = (double)W[W_RHO * Ntot + gk], uF = 0.0;
        v[0] = r;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double Fa = (double)W[(W_F + a) * Ntot + gk];
            double ua = (double)W[(W_U + a) * Ntot + gk];
            v[1 + a] = (double)W[(W_J + a) * Ntot + gk] + 0.5 * Fa;  // Eq. def_u
            v[D + 2 + a] = Fa;
            uF += ua * Fa;
        }
        R ur[3] = {W[(W_U + 0) * Ntot + gk], W[(W_U + 1) * Ntot + gk], W[(W_U + 2) * Ntot + gk]};
        double Q = (double)cell_heat<D, R>(s, z, k, W[W_RHO * Ntot + gk], ur);
        v[D + 1] = (double)W[W_G * Ntot + gk] + 0.5 * (uF + Q);  // Eq. def_E
        v[2 * D + 2] = uF + Q;
    }
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        double t = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < kBlockCells / 32; ++w) t += red[w][threadIdx.x];
        partials[(long long)blockIdx.x * NV + threadIdx.x] = t;
    }
}

// Fixed-order sum of the block partials of each simulation.
static __global__ void k_invariants_final(const double* __restrict__ partials, const int* __restrict__ sim_block_start, int nsim,
                                   int nv, double* __restrict__ out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsim * nv) return;
    int sim = t / nv, c = t % nv;
    double acc = 0.0;
    for (int b = sim_block_start[sim]; b < sim_block_start[sim + 1]; ++b) acc += partials[(long long)b * nv + c];
    out[t] = acc;
}

// Export rho, u, T (float64 or float32 H, per-simulation field layout of the ABI).
template <int D, typename R, typename H = double>
__global__ void __launch_bounds__(kBlockCells) k_export_moments(const SimDev* __restrict__ sims, const BlockEntry* __restrict__ table,
                                                                const R* __restrict__ W, long long Ntot, H* rho,
                                                                H* u, H* T)
{
    __shared__ SimDev s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long k = (long long)be.start + threadIdx.x;
    if (k >= s.N) return;
    const long long gk = s.cell_off + k;
    if (rho) rho[gk] = (H)W[W_RHO * Ntot + gk];
    if (T) T[gk] = (H)W[W_T * Ntot + gk];
    if (u) {
#pragma unroll
        for (int a = 0; a < D; ++a) u[(long long)D * s.cell_off + (long long)a * s.N + k] = (H)W[(W_U + a) * Ntot + gk];
    }
}

// Export the pre-collision populations (pulled, decoded) as float64 [Q][N].
template <int D, typename R, typename S>
__global__ void __launch_bounds__(kBlockCells) k_export_pops(const SimDev* __restrict__ sims, const BlockEntry* __restrict__ table,
                                                             const S* __restrict__ pop, double* f_out, double* g_out)
{
    constexpr int Q = Lat<D>::Q;
    __shared__ SimDev s;
    const BlockEntry be = table[blockIdx.x];
    load_sim(s, sims, be.sim);
    const long long k = (long long)be.start + threadIdx.x;
    if (k >= s.N) return;
    int x, y, z;
    cell_xyz(s, k, x, y, z);
    R f[Q], g[Q];
    pull_cell<D, R, S>(s, pop, x, y, z, f, g);
    const long long base = (long long)Q * s.cell_off;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (f_out) f_out[base + (long long)i * s.N + k] = (double)f[i];
        if (g_out) g_out[base + (long long)i * s.N + k] = (double)g[i];
    }
}

}  // namespace lbm
