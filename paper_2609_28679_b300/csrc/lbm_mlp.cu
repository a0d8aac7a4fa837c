// Training, prediction and sample generation of the learned temperature
// inversion (network layout in lbm_mlp.cuh), and its C ABI.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_mlp.cuh"

extern "C" void* lbm_glue_alloc(size_t nbytes, void* stream);
extern "C" void lbm_glue_free(void* ptr);
void lbm_set_global_error(const std::string& msg);  // lbm_abi.cu

namespace {

using namespace lbm;

constexpr int kTrainWarps = 4;
constexpr int kStageLd = 24;  // bfloat16 pitch of the warp-private transposed staging tiles [64][16]

int fail(int code, const std::string& msg)
{
    lbm_set_global_error(msg);
    return code;
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long idx)
{
    return (double)(splitmix64(seed ^ idx) >> 11) * (1.0 / 9007199254740992.0);
}

// Samples: rho log-uniform over [rho_lo, rho_hi], T uniform over [Tr_lo, Tr_hi] Tc;
// e = e(rho, T) and the target temperature re-solved from (rho, e) by float64 Newton.
__global__ void k_mlp_samples(SimDev s, double rho_lo, double rho_hi, double tr_lo, double tr_hi,
                              unsigned long long seed, long long n, double* rho_o, double* e_o, double* T_o,
                              unsigned long long* capped)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double u1 = u01(seed, 2 * (unsigned long long)i), u2 = u01(seed, 2 * (unsigned long long)i + 1);
    const double rho = exp(log(rho_lo) + u1 * (log(rho_hi) - log(rho_lo)));
    const double T = (tr_lo + u2 * (tr_hi - tr_lo)) * s.Tc;
    const RhoPart<double> p = rho_part<double>(s, rho);
    const double e = eos_e<double>(s, p, T);
    double Tn = s.Tc;
    const int it = pr_newton<double>(s, p, e, Tn, 1e-14, 50);
    if (it > 50) atomicAdd(capped, 1ull);
    rho_o[i] = rho;
    e_o[i] = e;
    T_o[i] = Tn;
}

// Prediction through the warp routine used inside the time step.
__global__ void __launch_bounds__(128) k_mlp_predict(const float* __restrict__ params, const double* __restrict__ rho,
                                                     const double* __restrict__ e, long long n, double* T_out)
{
    __shared__ MlpSmem m;
    mlp_load(m, params);
    __syncthreads();
    const long long nwarp = (long long)gridDim.x * (blockDim.x / 32);
    const long long w0 = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    for (long long base = w0 * 32; base < n; base += nwarp * 32) {
        const long long i = base + (threadIdx.x & 31);
        const bool ok = i < n;
        const float r = ok ? (float)rho[i] : 1.f, ee = ok ? (float)e[i] : 0.f;
        const float T = mlp_T_warp(m, r, ee);
        if (ok) T_out[i] = (double)T;
    }
}

struct GradSmem {
    MlpSmem m;
    __nv_bfloat16 w2t[kMlpH * kW2Ld];
    __nv_bfloat16 h1t[kTrainWarps][kMlpH * kStageLd];
    __nv_bfloat16 d2t[kTrainWarps][kMlpH * kStageLd];
    float gs[kMlpParams];
    float lsum;
};

// Forward and backward of minibatches with accumulation of the loss
// gradient into g (float32, kMlpParams, zeroed by the caller).  Sample k of
// the batch is sample k itself when n < 0, else splitmix64(seed ^ (step*B + k)) mod n.
// Loss = (1/B) sum (y - t)^2 / 2 over the B samples of the batch.
__global__ void __launch_bounds__(kTrainWarps * 32)
    k_mlp_grad(const float* __restrict__ params, const double* __restrict__ rho, const double* __restrict__ e,
               const double* __restrict__ T, long long n, int B, unsigned long long seed, long long step,
               float* __restrict__ g, double* __restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem& sm = *reinterpret_cast<GradSmem*>(smem_raw);
    MlpSmem& m = sm.m;
    __nv_bfloat16* w2t = sm.w2t;  // W2^T [in][out]: B operand of delta2 . W2
    float* gs = sm.gs;            // block gradient
    auto& h1t = sm.h1t;           // h1^T [in][row] per warp
    auto& d2t = sm.d2t;           // delta2^T [out][row] per warp
    float& lsum = sm.lsum;
    mlp_load(m, params);
    for (int k = threadIdx.x; k < kMlpH * kMlpH; k += blockDim.x)
        w2t[(k % kMlpH) * kW2Ld + (k / kMlpH)] = __float2bfloat16_rn(params[MP_W2 + k]);
    for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) gs[k] = 0.f;
    if (threadIdx.x == 0) lsum = 0.f;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g8 = lane >> 2, c = lane & 3;
    const float invB = 1.f / (float)B;
    const int nchunks = (B + 15) / 16;
    for (int ch = blockIdx.x * kTrainWarps + warp; ch < nchunks; ch += gridDim.x * kTrainWarps) {
        // lanes 0..15 hold the samples (rows) of this chunk
        const int row = lane & 15;
        const int k = ch * 16 + row;
        const bool valid_me = k < B;
        long long si = 0;
        if (valid_me)
            si = n < 0 ? (long long)k  // samples in order
                       : (long long)(splitmix64(seed ^ (unsigned long long)(step * (long long)B + k)) % (unsigned long long)n);
        const float x0 = valid_me ? (logf((float)rho[si]) - m.norm[0]) / m.norm[1] : 0.f;
        const float x1 = valid_me ? ((float)e[si] - m.norm[2]) / m.norm[3] : 0.f;
        const float tt = valid_me ? ((float)T[si] - m.norm[4]) / m.norm[5] : 0.f;
        const float xa0 = __shfl_sync(0xffffffffu, x0, g8), xa1 = __shfl_sync(0xffffffffu, x1, g8);
        const float xb0 = __shfl_sync(0xffffffffu, x0, g8 + 8), xb1 = __shfl_sync(0xffffffffu, x1, g8 + 8);
        const float ta = __shfl_sync(0xffffffffu, tt, g8), tb = __shfl_sync(0xffffffffu, tt, g8 + 8);
        const bool va = ch * 16 + g8 < B, vb = ch * 16 + g8 + 8 < B;

        // forward; keep h1^T for the weight gradient of the second layer
        float acc[8][4];
        mlp_layer2<true>(m, xa0, xa1, xb0, xb1, acc);
        __nv_bfloat16* H1 = h1t[warp];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const int k0 = 16 * ks + 2 * c;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = k0 + (q & 1) + (q >> 1) * 8;
                H1[kk * kStageLd + g8] = __float2bfloat16_rn(mlp_h1<true>(m, xa0, xa1, kk));
                H1[kk * kStageLd + g8 + 8] = __float2bfloat16_rn(mlp_h1<true>(m, xb0, xb1, kk));
            }
        }
        float h2[8][4];
        float ya = 0.f, yb = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n0 = 8 * nt + 2 * c;
            h2[nt][0] = mlp_tanh<true>(acc[nt][0] + m.b2[n0]);
            h2[nt][1] = mlp_tanh<true>(acc[nt][1] + m.b2[n0 + 1]);
            h2[nt][2] = mlp_tanh<true>(acc[nt][2] + m.b2[n0]);
            h2[nt][3] = mlp_tanh<true>(acc[nt][3] + m.b2[n0 + 1]);
            ya = fmaf(m.w3[n0], h2[nt][0], fmaf(m.w3[n0 + 1], h2[nt][1], ya));
            yb = fmaf(m.w3[n0], h2[nt][2], fmaf(m.w3[n0 + 1], h2[nt][3], yb));
        }
        ya += __shfl_xor_sync(0xffffffffu, ya, 1);
        ya += __shfl_xor_sync(0xffffffffu, ya, 2);
        yb += __shfl_xor_sync(0xffffffffu, yb, 1);
        yb += __shfl_xor_sync(0xffffffffu, yb, 2);
        ya += m.b3;
        yb += m.b3;
        const float da = va ? (ya - ta) * invB : 0.f, db = vb ? (yb - tb) * invB : 0.f;  // dL/dy
        if (c == 0) {
            float l = (va ? 0.5f * (ya - ta) * (ya - ta) : 0.f) + (vb ? 0.5f * (yb - tb) * (yb - tb) : 0.f);
            atomicAdd(&lsum, l * invB);
        }

        // output layer gradients and delta2 = dy W3 (1 - h2^2)
        float d2[8][4];
        float gw3[16], gb2[16];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n0 = 8 * nt + 2 * c;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float w = m.w3[n0 + q];
                d2[nt][q] = da * w * (1.f - h2[nt][q] * h2[nt][q]);
                d2[nt][2 + q] = db * w * (1.f - h2[nt][2 + q] * h2[nt][2 + q]);
                gw3[2 * nt + q] = da * h2[nt][q] + db * h2[nt][2 + q];
                gb2[2 * nt + q] = d2[nt][q] + d2[nt][2 + q];
            }
        }
        // sum over the 8 row groups (lanes with the same c)
#pragma unroll
        for (int q = 0; q < 16; ++q) {
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                gw3[q] += __shfl_xor_sync(0xffffffffu, gw3[q], o);
                gb2[q] += __shfl_xor_sync(0xffffffffu, gb2[q], o);
            }
        }
        if (g8 == 0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int nidx = 8 * (q >> 1) + 2 * c + (q & 1);
                atomicAdd(&gs[MP_W3 + nidx], gw3[q]);
                atomicAdd(&gs[MP_B2 + nidx], gb2[q]);
            }
        }
        float gb3 = (c == 0) ? da + db : 0.f;
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
        if (lane == 0) atomicAdd(&gs[MP_B3], gb3);

        // delta2^T staging for the W2 gradient
        __nv_bfloat16* D2 = d2t[warp];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n0 = 8 * nt + 2 * c;
            D2[n0 * kStageLd + g8] = __float2bfloat16_rn(d2[nt][0]);
            D2[(n0 + 1) * kStageLd + g8] = __float2bfloat16_rn(d2[nt][1]);
            D2[n0 * kStageLd + g8 + 8] = __float2bfloat16_rn(d2[nt][2]);
            D2[(n0 + 1) * kStageLd + g8 + 8] = __float2bfloat16_rn(d2[nt][3]);
        }

        // delta1 = (delta2 . W2) (1 - h1^2): delta2's accumulator tiles are the A operand
        float a1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) a1[nt][0] = a1[nt][1] = a1[nt][2] = a1[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a[4];
            a[0] = pack_bf16(d2[2 * ks][0], d2[2 * ks][1]);
            a[1] = pack_bf16(d2[2 * ks][2], d2[2 * ks][3]);
            a[2] = pack_bf16(d2[2 * ks + 1][0], d2[2 * ks + 1][1]);
            a[3] = pack_bf16(d2[2 * ks + 1][2], d2[2 * ks + 1][3]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint32_t* w = reinterpret_cast<const uint32_t*>(w2t + (8 * nt + g8) * kW2Ld + 16 * ks + 2 * c);
                mma_bf16(a1[nt], a, w[0], w[4]);
            }
        }
        float gw1[16][2], gb1[16];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n0 = 8 * nt + 2 * c;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float ha = mlp_h1<true>(m, xa0, xa1, n0 + q), hb = mlp_h1<true>(m, xb0, xb1, n0 + q);
                const float d1a = a1[nt][q] * (1.f - ha * ha), d1b = a1[nt][2 + q] * (1.f - hb * hb);
                gb1[2 * nt + q] = d1a + d1b;
                gw1[2 * nt + q][0] = d1a * xa0 + d1b * xb0;
                gw1[2 * nt + q][1] = d1a * xa1 + d1b * xb1;
            }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                gb1[q] += __shfl_xor_sync(0xffffffffu, gb1[q], o);
                gw1[q][0] += __shfl_xor_sync(0xffffffffu, gw1[q][0], o);
                gw1[q][1] += __shfl_xor_sync(0xffffffffu, gw1[q][1], o);
            }
        }
        if (g8 == 0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int kidx = 8 * (q >> 1) + 2 * c + (q & 1);
                atomicAdd(&gs[MP_B1 + kidx], gb1[q]);
                atomicAdd(&gs[MP_W1 + 2 * kidx], gw1[q][0]);
                atomicAdd(&gs[MP_W1 + 2 * kidx + 1], gw1[q][1]);
            }
        }

        // grad W2 [out][in] += delta2^T (64 x 16) . h1 (16 x 64): one k-step per tile
        __syncwarp();
#pragma unroll 1
        for (int mt = 0; mt < 4; ++mt) {
            uint32_t a[4];
            const uint32_t* ar = reinterpret_cast<const uint32_t*>(D2 + (16 * mt + g8) * kStageLd + 2 * c);
            const uint32_t* br = reinterpret_cast<const uint32_t*>(D2 + (16 * mt + g8 + 8) * kStageLd + 2 * c);
            a[0] = ar[0];
            a[1] = br[0];
            a[2] = ar[4];
            a[3] = br[4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint32_t* w = reinterpret_cast<const uint32_t*>(H1 + (8 * nt + g8) * kStageLd + 2 * c);
                float cc4[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(cc4, a, w[0], w[4]);
                const int out = 16 * mt + g8, in = 8 * nt + 2 * c;
                atomicAdd(&gs[MP_W2 + out * kMlpH + in], cc4[0]);
                atomicAdd(&gs[MP_W2 + out * kMlpH + in + 1], cc4[1]);
                atomicAdd(&gs[MP_W2 + (out + 8) * kMlpH + in], cc4[2]);
                atomicAdd(&gs[MP_W2 + (out + 8) * kMlpH + in + 1], cc4[3]);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x)
        if (k >= 6 && gs[k] != 0.f) atomicAdd(&g[k], gs[k]);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, (double)lsum);
}

// Adam on the trainable entries (beta1 0.9, beta2 0.999, eps 1e-8); zeroes g.
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ mo,
                           float* __restrict__ ve, float lr, float bc1, float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 6 || k >= kMlpParams) return;
    const float gr = g[k];
    const float m = 0.9f * mo[k] + 0.1f * gr;
    const float v = 0.999f * ve[k] + 0.001f * gr * gr;
    mo[k] = m;
    ve[k] = v;
    p[k] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
    g[k] = 0.f;
}

cudaError_t grad_smem_setup()
{
    return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem));
}

int sim_from_eos(const lbm_eos* eos, SimDev& s)
{
    std::memset(&s, 0, sizeof(s));
    if (!eos || eos->kind != LBM_PR) return fail(LBM_E_INVALID, "the learned inversion is built for Peng-Robinson");
    if (!(eos->Tc > 0) || !(eos->R > 0) || !(eos->cv > 0)) return fail(LBM_E_INVALID, "bad Peng-Robinson constants");
    s.eos = EOS_PR;
    s.R = eos->R; s.cv = eos->cv; s.Tc = eos->Tc; s.a = eos->a; s.b = eos->b;
    if (eos->a == 0.0) {
        if (!(eos->Pc > 0)) return fail(LBM_E_INVALID, "Peng-Robinson needs a, b or Pc > 0");
        s.a = 0.45724 * eos->R * eos->R * eos->Tc * eos->Tc / eos->Pc;
        s.b = 0.07780 * eos->R * eos->Tc / eos->Pc;
    }
    s.kw = 0.37464 + 1.54226 * eos->omega - 0.26992 * eos->omega * eos->omega;
    s.inv_cv = 1.0 / s.cv;
    s.inv_Tc = 1.0 / s.Tc;
    s.lam_c = 1.0 / (2.0 * std::sqrt(2.0) * s.b);
    return LBM_OK;
}

struct DevBuf {
    void* p = nullptr;
    explicit DevBuf(size_t n, cudaStream_t st) : p(lbm_glue_alloc(n, (void*)st)) {}
    ~DevBuf() { lbm_glue_free(p); }
    template <typename T> T* as() { return static_cast<T*>(p); }
};

}  // namespace

extern "C" {

int lbm_mlp_train(const lbm_eos* eos, const double box[4], long long nsamples, int steps, int batch, double lr,
                  unsigned long long seed, int init, float* params, double* loss_hist, void* stream)
{
    SimDev s;
    int rc = sim_from_eos(eos, s);
    if (rc) return rc;
    if (!box || !params || nsamples < 16 || steps < 0 || batch < 16 || !(lr > 0))
        return fail(LBM_E_INVALID, "lbm_mlp_train: bad arguments");
    if (!(box[0] > 0) || !(box[1] > box[0]) || !(box[2] > 0) || !(box[3] > box[2]))
        return fail(LBM_E_INVALID, "lbm_mlp_train: bad sample box");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf samp((size_t)nsamples * 3 * sizeof(double), st), state((size_t)4 * kMlpParams * sizeof(float), st),
        acc(64, st);
    if (!samp.p || !state.p || !acc.p) return fail(LBM_E_NOMEM, "lbm_mlp_train: allocation failed");
    double* rho = samp.as<double>();
    double* e = rho + nsamples;
    double* T = e + nsamples;
    float* p = state.as<float>();
    float* g = p + kMlpParams;
    float* mo = g + kMlpParams;
    float* ve = mo + kMlpParams;
    unsigned long long* capped = acc.as<unsigned long long>();
    double* dloss = reinterpret_cast<double*>(capped + 1);
    cudaMemsetAsync(acc.p, 0, 64, st);
    cudaMemsetAsync(g, 0, 3 * kMlpParams * sizeof(float), st);
    k_mlp_samples<<<(int)((nsamples + 255) / 256), 256, 0, st>>>(s, box[0], box[1], box[2], box[3], seed, nsamples,
                                                               rho, e, T, capped);
    std::vector<float> hp(params, params + kMlpParams);
    if (init) {
        // normalisation from the sample box; weights uniform in +-1/sqrt(fan_in)
        std::vector<double> he(nsamples);
        cudaMemcpyAsync(he.data(), e, nsamples * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(LBM_E_CUDA, "lbm_mlp_train: sample generation failed");
        double emin = he[0], emax = he[0];
        for (double v : he) { emin = std::fmin(emin, v); emax = std::fmax(emax, v); }
        const double l0 = std::log(box[0]), l1 = std::log(box[1]);
        hp[0] = (float)(0.5 * (l0 + l1)); hp[1] = (float)(0.5 * (l1 - l0));
        hp[2] = (float)(0.5 * (emin + emax)); hp[3] = (float)(0.5 * (emax - emin));
        hp[4] = (float)(0.5 * (box[2] + box[3]) * s.Tc); hp[5] = (float)(0.5 * (box[3] - box[2]) * s.Tc);
        unsigned long long z = seed * 0x9E3779B97F4A7C15ull + 12345;
        auto urand = [&]() {
            z += 0x9E3779B97F4A7C15ull;
            unsigned long long q = z;
            q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ull;
            q = (q ^ (q >> 27)) * 0x94D049BB133111EBull;
            q ^= q >> 31;
            return (double)(q >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        };
        for (int k = 0; k < 2 * kMlpH; ++k) hp[MP_W1 + k] = (float)(urand() / std::sqrt(2.0));
        for (int k = 0; k < kMlpH * kMlpH; ++k) hp[MP_W2 + k] = (float)(urand() / 8.0);
        for (int k = 0; k < kMlpH; ++k) {
            hp[MP_B1 + k] = 0.f;
            hp[MP_B2 + k] = 0.f;
            hp[MP_W3 + k] = (float)(urand() / 8.0);
        }
        hp[MP_B3] = 0.f;
    }
    cudaMemcpyAsync(p, hp.data(), kMlpParams * sizeof(float), cudaMemcpyHostToDevice, st);
    const int nchunks = (batch + 15) / 16;
    const int grid = (nchunks + kTrainWarps - 1) / kTrainWarps;
    if (grad_smem_setup() != cudaSuccess) return fail(LBM_E_CUDA, "lbm_mlp_train: shared-memory attribute");
    for (int t = 1; t <= steps; ++t) {
        cudaMemsetAsync(dloss, 0, sizeof(double), st);
        k_mlp_grad<<<grid, kTrainWarps * 32, sizeof(GradSmem), st>>>(p, rho, e, T, nsamples, batch, seed + 7, t, g,
                                                                      dloss);
        k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p, g, mo, ve, (float)lr,
                                                               (float)(1.0 - std::pow(0.9, t)),
                                                               (float)(1.0 - std::pow(0.999, t)));
        if (loss_hist) cudaMemcpyAsync(loss_hist + (t - 1), dloss, sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    cudaMemcpyAsync(params, p, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaError_t err = cudaStreamSynchronize(st);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) return fail(LBM_E_CUDA, std::string("lbm_mlp_train: ") + cudaGetErrorString(err));
    return LBM_OK;
}

int lbm_mlp_grad(const float* params, const double* rho, const double* e, const double* T, long long n,
                 float* grad, double* loss)
{
    if (!params || !rho || !e || !T || n < 1 || n > (1LL << 30) || !grad)
        return fail(LBM_E_INVALID, "lbm_mlp_grad: bad arguments");
    cudaStream_t st = nullptr;
    // layout: [loss (double, 16 B)][rho][e][T (doubles)][params][grad (floats)]
    DevBuf buf(16 + (size_t)n * 3 * sizeof(double) + 2 * kMlpParams * sizeof(float), st);
    if (!buf.p) return fail(LBM_E_NOMEM, "lbm_mlp_grad: allocation failed");
    double* dl = buf.as<double>();
    double* dr = dl + 2;
    double* de = dr + n;
    double* dT = de + n;
    float* dp = reinterpret_cast<float*>(dT + n);
    float* dg = dp + kMlpParams;
    cudaMemcpy(dr, rho, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(de, e, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(dT, T, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(dp, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(dg, 0, kMlpParams * sizeof(float));
    cudaMemset(dl, 0, sizeof(double));
    // seed 0 / step 0 are not used: indices are taken in order (idx = k for k < n == B)
    const int B = (int)n;
    const int grid = ((B + 15) / 16 + kTrainWarps - 1) / kTrainWarps;
    if (grad_smem_setup() != cudaSuccess) return fail(LBM_E_CUDA, "lbm_mlp_grad: shared-memory attribute");
    k_mlp_grad<<<grid, kTrainWarps * 32, sizeof(GradSmem)>>>(dp, dr, de, dT, -1, B, 0, 0, dg, dl);
    cudaMemcpy(grad, dg, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost);
    if (loss) cudaMemcpy(loss, dl, sizeof(double), cudaMemcpyDeviceToHost);
    cudaError_t err = cudaDeviceSynchronize();
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) return fail(LBM_E_CUDA, std::string("lbm_mlp_grad: ") + cudaGetErrorString(err));
    return LBM_OK;
}

int lbm_mlp_predict(const float* params, const double* rho, const double* e, long long n, double* T_out)
{
    if (!params || !rho || !e || !T_out || n < 1) return fail(LBM_E_INVALID, "lbm_mlp_predict: bad arguments");
    DevBuf buf((size_t)n * 3 * sizeof(double) + kMlpParams * sizeof(float), nullptr);
    if (!buf.p) return fail(LBM_E_NOMEM, "lbm_mlp_predict: allocation failed");
    double* dr = buf.as<double>();
    double* de = dr + n;
    double* dT = de + n;
    float* dp = reinterpret_cast<float*>(dT + n);
    cudaMemcpy(dr, rho, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(de, e, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(dp, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
    const long long warps = (n + 31) / 32;
    const int grid = (int)std::min<long long>((warps + 3) / 4, 4096);
    k_mlp_predict<<<grid, 128>>>(dp, dr, de, n, dT);
    cudaMemcpy(T_out, dT, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaError_t err = cudaDeviceSynchronize();
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) return fail(LBM_E_CUDA, std::string("lbm_mlp_predict: ") + cudaGetErrorString(err));
    return LBM_OK;
}

int lbm_mlp_nparams(void) { return kMlpParams; }

}  // extern "C"
