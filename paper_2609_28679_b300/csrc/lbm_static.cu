// lbm_step_static: one float64 time step on caller-owned populations that
// allocates nothing.
//
// The handle-based entry points take their device memory (populations,
// moments, macroscopic fields, tables) from PyTorch's caching allocator when
// a simulation is created.  Some callers cannot allocate device memory at
// all, or not at the point where they step:
//   - host programs that hand every library a fixed device-memory budget up
//     front and refuse later requests (plugin hosts, embedded solvers that
//     pre-plan their memory);
//   - C or C++ programs that link liblbm.so without PyTorch, so there is no
//     caching allocator behind the handle path;
//   - time-critical loops that must not call cudaFree, which waits for the
//     whole device, or cudaMalloc, whose latency is unbounded.
// For them the work arrays of the three-pass step (the simulation constants,
// the block table and the macroscopic fields) live in one file-scope
// __device__ array of fixed size: the call makes no cudaMalloc, no cudaFree
// and no allocating library call, and copies nothing from host memory (the
// constants reach the device as a kernel argument).
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
int lbm_check_and_fill_sim(lbm::SimDev& s, const lbm_lattice* L, const lbm_eos* E, double tau_f, double tau_g,
                           const lbm_force* F, const lbm_heat* H, std::string& why);  // lbm_abi.cu

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

// The constants of this call (a kernel argument, copied by the launch) and
// the block table {0, b * kBlockCells} written into the scratch's head.
__global__ void __launch_bounds__(kBlockCells) k_static_setup(SimDev s, SimDev* __restrict__ d_sim,
                                                              BlockEntry* __restrict__ d_table, int nb)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_sim = s;
    for (int b = blockIdx.x * kBlockCells + threadIdx.x; b < nb; b += gridDim.x * kBlockCells)
        d_table[b] = BlockEntry{0, b * kBlockCells};
}

// moments of pre-collision populations held at their own cell: rho, j, G;
// the Newton guess slot is cleared (Newton then starts from the critical
// temperature, as on a handle's first step)
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
    // what this entry point leaves to the handle path
    if (L.storage != LBM_F64) return fail(LBM_E_UNSUPPORTED, "lbm_step_static works on float64 populations only");
    if (L.zwalls == 2) return fail(LBM_E_UNSUPPORTED, "non-equilibrium-extrapolation walls need a handle (lbm_set_walls)");
    if (force && (force->friction != 0.0 || force->throttle_K != 0.0 || force->field))
        return fail(LBM_E_UNSUPPORTED, "duct friction, throttles and force fields run on the split kernels of a handle");
    if (heat && heat->field) return fail(LBM_E_UNSUPPORTED, "heat fields run on the split kernels of a handle");
    if (eos->t_solver != LBM_T_NEWTON)
        return fail(LBM_E_UNSUPPORTED, "lbm_step_static inverts the temperature by Newton only (t_solver = LBM_T_NEWTON)");
    if (eos->isothermal) return fail(LBM_E_UNSUPPORTED, "the isothermal mode needs the temperature a handle carries");
    // the checks of lbm_create
    SimDev s;
    std::string why;
    int rc = lbm_check_and_fill_sim(s, lattice, eos, tau_f, tau_g, force, heat, why);
    if (rc) return fail(rc, "lbm_step_static: " + why);
    const long long N = s.N;
    if (N > kStaticMaxCells)
        return fail(LBM_E_INVALID, "lbm_step_static: " + std::to_string(N) + " cells exceed the static maximum of " +
                                       std::to_string(kStaticMaxCells));
    const int Q = L.dim == 2 ? 9 : 27;
    const double* in_lo[2] = {f_in, g_in};
    const double* out_lo[2] = {f_out, g_out};
    for (int a = 0; a < 2; ++a)  // [Q][N] ranges of the inputs and outputs must not overlap
        for (int b = 0; b < 2; ++b)
            if (in_lo[a] < out_lo[b] + (size_t)Q * N && out_lo[b] < in_lo[a] + (size_t)Q * N)
                return fail(LBM_E_INVALID, "input and output populations must not alias");

    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    SimDev* d_sim = reinterpret_cast<SimDev*>(base);
    BlockEntry* d_table = reinterpret_cast<BlockEntry*>(static_cast<unsigned char*>(base) + kSimBytes);
    double* W = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kSimBytes + kTableBytes);
    const int nb = (int)((N + kBlockCells - 1) / kBlockCells);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_static_setup<<<1, kBlockCells, 0, st>>>(s, d_sim, d_table, nb);
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
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_E_CUDA, std::string("lbm_step_static launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}

}  // extern "C"
