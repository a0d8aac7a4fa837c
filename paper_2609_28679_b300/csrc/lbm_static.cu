// lbm_step_static: one float64 time step on caller-owned populations that
// allocates nothing.
//
// Some callers cannot allocate device memory at the point where they step a
// simulation: code running while a framework captures a CUDA graph (where an
// allocation would be recorded into, or break, the capture), embedded or
// plugin hosts that hand out a fixed device-memory budget and forbid further
// allocation, and callers whose allocator is not PyTorch's.  For them the
// work arrays of the three-pass step (moments, macroscopic fields, the
// simulation constants and the block table) live in one file-scope
// __device__ array of fixed size, so the call needs no cudaMalloc, no
// cudaFree and no allocating library routine.
//
// The array holds room for kStaticMaxCells cells.  Every process that loads
// the library keeps it on every GPU it uses until exit.  All calls share it:
// two calls whose kernels overlap on the GPU (different streams, different
// host threads) race on it and produce garbage; serialise them.  Each call
// rewrites all of the array it reads, so no state carries from one call to
// the next.
#include <cmath>
#include <cstring>
#include <string>

#include "lbm.h"
#include "lbm_split.cuh"

void lbm_set_global_error(const std::string& msg);  // lbm_abi.cu

namespace {

using namespace lbm;

constexpr long long kStaticMaxCells = 65536;  // e.g. 256 x 256 (D2Q9) or 40 x 40 x 40 (D3Q27)
constexpr long long kStaticBlocks = kStaticMaxCells / kBlockCells;
constexpr size_t kSimBytes = (sizeof(SimDev) + 255) / 256 * 256;
constexpr size_t kTableBytes = (kStaticBlocks * sizeof(BlockEntry) + 255) / 256 * 256;
constexpr size_t kWorkBytes = (size_t)W_NF * kStaticMaxCells * sizeof(double);
constexpr size_t kScratchBytes = kSimBytes + kTableBytes + kWorkBytes;

// [SimDev][BlockEntry table][W: W_NF x kStaticMaxCells doubles]
static __device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

// device address of g_step_scratch per device, taken once per device
constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {nullptr};

int fail(int code, const std::string& msg)
{
    lbm_set_global_error(msg);  // reported by lbm_last_error(NULL)
    return code;
}

// moments of pre-collision populations held at their own cell: rho, j, G;
// the Newton guess slot is cleared (Newton then starts from e / c_v)
template <int D>
__global__ void __launch_bounds__(kBlockCells) k_static_moments(const SimDev* __restrict__ sims,
                                                                const double* __restrict__ f,
                                                                const double* __restrict__ g, double* __restrict__ W,
                                                                long long Ntot)
{
    constexpr int Q = Lat<D>::Q;
    const long long N = sims[0].N;
    const long long k = (long long)blockIdx.x * kBlockCells + threadIdx.x;
    if (k >= N) return;
    double rho = 0, j[3] = {0, 0, 0}, G = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double fi = f[(long long)i * N + k];
        rho += fi;
#pragma unroll
        for (int a = 0; a < D; ++a) j[a] += (double)cc(i, a) * fi;
        G += g[(long long)i * N + k];
    }
    W[W_RHO * Ntot + k] = rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) W[(W_J + a) * Ntot + k] = j[a];
    W[W_G * Ntot + k] = G;
    W[W_T * Ntot + k] = 0.0;
}

// collide at x and push f'_i to x + c_i (across a z wall: back to x as opp(i))
template <int D>
__global__ void __launch_bounds__(kBlockCells) k_static_collide(const SimDev* __restrict__ sims,
                                                                const double* __restrict__ f_in,
                                                                const double* __restrict__ g_in,
                                                                double* __restrict__ f_out, double* __restrict__ g_out,
                                                                const double* __restrict__ W, long long Ntot)
{
    constexpr int Q = Lat<D>::Q;
    __shared__ SimDev s;
    load_sim(s, sims, 0);
    const long long k = (long long)blockIdx.x * kBlockCells + threadIdx.x;
    if (k >= s.N) return;
    int x, y, z;
    cell_xyz(s, k, x, y, z);
    Macro<double> m;
    m.rho = W[W_RHO * Ntot + k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.u[a] = W[(W_U + a) * Ntot + k];
        m.F[a] = W[(W_F + a) * Ntot + k];
    }
    m.Q = heat_at(s, z);
    m.T = W[W_T * Ntot + k];
    m.P = W[W_P * Ntot + k];
    m.theta = W[W_TH * Ntot + k];
    m.h = W[W_H * Ntot + k];
    m.cv = W[W_CV * Ntot + k];
    m.gam = W[W_GAM * Ntot + k];
    m.athe = W[W_ATHE * Ntot + k];
    m.e = W[W_E * Ntot + k];
    m.ir = 1.0 / m.rho;
    m.icv = 1.0 / m.cv;
    double divu, gh[3], gT[3], Phi[3];
    stencils<D, double>(s, W, Ntot, x, y, z, m.rho, m.u, divu, gh, gT, Phi);
    double f[Q], g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        f[i] = f_in[(long long)i * s.N + k];
        g[i] = g_in[(long long)i * s.N + k];
    }
    collide_cell<D, double>(s, m, divu, gh, gT, Phi, f, g);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int zt = z + (D == 3 ? cc(i, 2) : 0);
        long long dst;
        int j = i;
        if (D == 3 && s.zwalls && (zt < 0 || zt >= s.nz)) {
            dst = k;
            j = opp(i);
        } else {
            const int xt = wrapi(x + cc(i, 0), s.nx), yt = wrapi(y + cc(i, 1), s.ny);
            const int zz = D == 3 ? wrapi(zt, s.nz) : 0;
            dst = (long long)xt + (long long)s.nx * ((long long)yt + (long long)s.ny * (long long)zz);
        }
        f_out[(long long)j * s.N + dst] = f[i];
        g_out[(long long)j * s.N + dst] = g[i];
    }
}

// The scratch's device address on the current device (set-up on first use).
int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_E_UNSUPPORTED, "device index beyond the static table");
    if (g_scratch_dev[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(LBM_E_CUDA, std::string("cudaGetSymbolAddress(g_step_scratch): ") + cudaGetErrorString(e));
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_step_static(const lbm_lattice* lattice, const lbm_eos* eos, double tau_f, double tau_g,
                    const lbm_force* force, const lbm_heat* heat, const double* f_in, const double* g_in,
                    double* f_out, double* g_out, void* stream)
{
    if (!lattice || !eos || !f_in || !g_in || !f_out || !g_out) return fail(LBM_E_INVALID, "NULL argument");
    const lbm_lattice& L = *lattice;
    if (L.dim != 2 && L.dim != 3) return fail(LBM_E_INVALID, "dim must be 2 or 3");
    if (L.nx < 1 || L.ny < 1 || L.nz < 1 || (L.dim == 2 && (L.nz != 1 || L.zwalls)))
        return fail(LBM_E_INVALID, "bad lattice sizes");
    if (L.storage != LBM_F64) return fail(LBM_E_UNSUPPORTED, "lbm_step_static works on float64 populations only");
    if (L.zwalls == 2) return fail(LBM_E_UNSUPPORTED, "non-equilibrium-extrapolation walls need a handle (lbm_set_walls)");
    if (force && (force->friction != 0.0 || force->throttle_K != 0.0 || force->field))
        return fail(LBM_E_UNSUPPORTED, "duct friction, throttles and force fields run on the split kernels of a handle");
    if (heat && heat->field) return fail(LBM_E_UNSUPPORTED, "heat fields run on the split kernels of a handle");
    if (L.zwalls != 0 && L.zwalls != 1) return fail(LBM_E_INVALID, "zwalls must be 0, 1 or 2");
    if (L.phi_scheme != LBM_PHI_UPWIND && L.phi_scheme != LBM_PHI_CENTRAL) return fail(LBM_E_INVALID, "unknown phi_scheme");
    const long long N = (long long)L.nx * L.ny * L.nz;
    if (N > kStaticMaxCells)
        return fail(LBM_E_INVALID, "lbm_step_static: " + std::to_string(N) + " cells exceed the static maximum of " +
                                       std::to_string(kStaticMaxCells));
    if (f_in == f_out || g_in == g_out) return fail(LBM_E_INVALID, "input and output populations must not alias");
    if (eos->kind < LBM_IDEAL || eos->kind > LBM_PR || !(eos->R > 0) || !(eos->cv > 0) || !(tau_f > 0) || !(tau_g > 0))
        return fail(LBM_E_INVALID, "bad equation of state or relaxation time");
    if (eos->kind == LBM_PR && !(eos->Tc > 0)) return fail(LBM_E_INVALID, "Peng-Robinson needs Tc > 0");

    SimDev s;
    std::memset(&s, 0, sizeof(s));
    s.nx = L.nx; s.ny = L.ny; s.nz = L.nz; s.zwalls = L.zwalls;
    s.N = N;
    s.eos = eos->kind;
    s.phi_central = L.phi_scheme == LBM_PHI_CENTRAL;
    s.R = eos->R; s.cv = eos->cv; s.a = eos->a; s.b = eos->b; s.Tc = eos->Tc;
    if (eos->kind == LBM_PR) {
        if (eos->a == 0.0) {
            if (!(eos->Pc > 0)) return fail(LBM_E_INVALID, "Peng-Robinson needs a, b or Pc > 0");
            s.a = 0.45724 * eos->R * eos->R * eos->Tc * eos->Tc / eos->Pc;
            s.b = 0.07780 * eos->R * eos->Tc / eos->Pc;
        }
        s.kw = 0.37464 + 1.54226 * eos->omega - 0.26992 * eos->omega * eos->omega;
    }
    if (!(eos->mu >= 0) || !std::isfinite(eos->mu)) return fail(LBM_E_INVALID, "mu must be finite and >= 0");
    if (eos->isothermal) return fail(LBM_E_UNSUPPORTED, "the isothermal mode needs the temperature a handle carries");
    s.kappa = eos->kappa; s.eta_mu = eos->eta_over_mu; s.k_mu = eos->k_over_mu;
    s.mu = eos->mu;
    s.beta_f = 1.0 / (2.0 * tau_f + 1.0);
    s.beta_g = 1.0 / (2.0 * tau_g + 1.0);
    if (force) { s.acc[0] = force->accel[0]; s.acc[1] = force->accel[1]; s.acc[2] = L.dim == 3 ? force->accel[2] : 0.0; }
    if (heat) { s.q = heat->q; s.zlo = heat->zmask_lo; s.zhi = heat->zmask_hi; }
    s.inv_cv = 1.0 / s.cv;
    s.inv_Tc = s.Tc > 0 ? 1.0 / s.Tc : 0.0;
    s.lam_c = s.b > 0 ? 1.0 / (2.0 * 1.4142135623730951 * s.b) : 0.0;
    s.athe_c = (double)(L.dim + 2) / (double)L.dim - s.eta_mu;

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    SimDev* d_sim = reinterpret_cast<SimDev*>(base);
    BlockEntry* d_table = reinterpret_cast<BlockEntry*>(static_cast<unsigned char*>(base) + kSimBytes);
    double* W = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kSimBytes + kTableBytes);
    const int nb = (int)((N + kBlockCells - 1) / kBlockCells);
    BlockEntry table[kStaticBlocks];
    for (int b = 0; b < nb; ++b) table[b] = BlockEntry{0, b * kBlockCells};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(d_sim, &s, sizeof(SimDev), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_table, table, nb * sizeof(BlockEntry), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(LBM_E_CUDA, std::string("lbm_step_static upload: ") + cudaGetErrorString(e));
    // the work arrays are laid out as [W_NF][N] for this call
    if (L.dim == 2) {
        k_static_moments<2><<<nb, kBlockCells, 0, st>>>(d_sim, f_in, g_in, W, N);
        k_macro<2, double><<<nb, kBlockCells, 0, st>>>(d_sim, d_table, W, N, nullptr);
        k_static_collide<2><<<nb, kBlockCells, 0, st>>>(d_sim, f_in, g_in, f_out, g_out, W, N);
    } else {
        k_static_moments<3><<<nb, kBlockCells, 0, st>>>(d_sim, f_in, g_in, W, N);
        k_macro<3, double><<<nb, kBlockCells, 0, st>>>(d_sim, d_table, W, N, nullptr);
        k_static_collide<3><<<nb, kBlockCells, 0, st>>>(d_sim, f_in, g_in, f_out, g_out, W, N);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_E_CUDA, std::string("lbm_step_static launch: ") + cudaGetErrorString(e));
    // the host copies of s and table above must not be released before the
    // stream consumed them (pageable source: the copy is staged before return)
    return LBM_OK;
}

}  // extern "C"
