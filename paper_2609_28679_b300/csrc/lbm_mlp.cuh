// Learned temperature inversion T(rho, e): a 2 -> 64 -> 64 -> 1 tanh network
// whose 64 x 64 layer runs on the tensor cores (mma.sync m16n8k16, bfloat16
// operands, float32 accumulation), one warp per 16 cells or samples.
//
// Parameter array (float32, kMlpParams entries):
//   [c_rho, s_rho, c_e, s_e, c_T, s_T | W1 (64x2) | b1 (64) | W2 (64x64, [out][in]) | b2 | W3 (64) | b3]
// x0 = (log rho - c_rho)/s_rho, x1 = (e - c_e)/s_e, h1 = tanh(W1 x + b1),
// h2 = tanh(W2 h1 + b2), y = W3 . h2 + b3, T_hat = c_T + s_T y.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {

constexpr int kMlpH = 64;
constexpr int MP_NORM = 0, MP_W1 = 6, MP_B1 = MP_W1 + 2 * kMlpH, MP_W2 = MP_B1 + kMlpH, MP_B2 = MP_W2 + kMlpH * kMlpH,
              MP_W3 = MP_B2 + kMlpH, MP_B3 = MP_W3 + kMlpH, kMlpParams = MP_B3 + 1;
constexpr int kW2Ld = 72;  // bfloat16 row pitch of the shared copies (bank-conflict-free fragment loads)

// Shared-memory image of the network for the tensor-core routines.
struct MlpSmem {
    __nv_bfloat16 w2[kMlpH * kW2Ld];   // W2 [out][in]: B operand of h1 . W2^T
    float w1[2 * kMlpH], b1[kMlpH], b2[kMlpH], w3[kMlpH], norm[6], b3;
};

// cooperative load by the whole block (the caller synchronises afterwards)
__device__ inline void mlp_load(MlpSmem& m, const float* __restrict__ p)
{
    for (int k = threadIdx.x; k < kMlpH * kMlpH; k += blockDim.x)
        m.w2[(k / kMlpH) * kW2Ld + (k % kMlpH)] = __float2bfloat16_rn(p[MP_W2 + k]);
    for (int k = threadIdx.x; k < 2 * kMlpH; k += blockDim.x) m.w1[k] = p[MP_W1 + k];
    for (int k = threadIdx.x; k < kMlpH; k += blockDim.x) {
        m.b1[k] = p[MP_B1 + k];
        m.b2[k] = p[MP_B2 + k];
        m.w3[k] = p[MP_W3 + k];
    }
    if (threadIdx.x < 6) m.norm[threadIdx.x] = p[MP_NORM + threadIdx.x];
    if (threadIdx.x == 0) m.b3 = p[MP_B3];
}

__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// c += a . b for one m16n8k16 tile (row-major A, column-major B, fp32 C)
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// tanh for the network: the one-instruction approximation (in-step
// inference) or the correctly rounded-to-a-few-ulp library tanhf (training,
// whose gradients are checked against a float64 reference).
template <bool EXACT> __device__ __forceinline__ float mlp_tanh(float x)
{
    if constexpr (EXACT) return tanhf(x);
    else return tanh_fast(x);
}

// First layer at (row, k): tanh(W1[k] . x_row + b1[k])
template <bool EXACT = false>
__device__ __forceinline__ float mlp_h1(const MlpSmem& m, float x0, float x1, int k)
{
    return mlp_tanh<EXACT>(fmaf(m.w1[2 * k], x0, fmaf(m.w1[2 * k + 1], x1, m.b1[k])));
}

// Second layer for one 16-row tile whose rows g and g+8 (g = lane/4) have
// inputs (xa0, xa1), (xb0, xb1): acc[nt][0..1] -> row g, cols 8nt + 2c + {0,1};
// acc[nt][2..3] -> row g + 8 (pre-activation, before b2).
template <bool EXACT = false>
__device__ __forceinline__ void mlp_layer2(const MlpSmem& m, float xa0, float xa1, float xb0, float xb1,
                                           float acc[8][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        const int k0 = 16 * ks + 2 * c;
        uint32_t a[4];
        a[0] = pack_bf16(mlp_h1<EXACT>(m, xa0, xa1, k0), mlp_h1<EXACT>(m, xa0, xa1, k0 + 1));
        a[1] = pack_bf16(mlp_h1<EXACT>(m, xb0, xb1, k0), mlp_h1<EXACT>(m, xb0, xb1, k0 + 1));
        a[2] = pack_bf16(mlp_h1<EXACT>(m, xa0, xa1, k0 + 8), mlp_h1<EXACT>(m, xa0, xa1, k0 + 9));
        a[3] = pack_bf16(mlp_h1<EXACT>(m, xb0, xb1, k0 + 8), mlp_h1<EXACT>(m, xb0, xb1, k0 + 9));
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint32_t* w = reinterpret_cast<const uint32_t*>(m.w2 + (8 * nt + g) * kW2Ld + k0);
            mma_bf16(acc[nt], a, w[0], w[4]);
        }
    }
}

// Warp-collective inference: each lane passes the (rho, e) of its own cell and
// receives T_hat for it.  All 32 lanes must be active.
__device__ __forceinline__ float mlp_T_warp(const MlpSmem& m, float rho, float e)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const float x0 = (__logf(rho) - m.norm[0]) / m.norm[1];
    const float x1 = (e - m.norm[2]) / m.norm[3];
    float yout = 0.f;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int ra = 16 * mt + g, rb = ra + 8;
        const float xa0 = __shfl_sync(0xffffffffu, x0, ra), xa1 = __shfl_sync(0xffffffffu, x1, ra);
        const float xb0 = __shfl_sync(0xffffffffu, x0, rb), xb1 = __shfl_sync(0xffffffffu, x1, rb);
        float acc[8][4];
        mlp_layer2(m, xa0, xa1, xb0, xb1, acc);
        float ya = 0.f, yb = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n0 = 8 * nt + 2 * c;
            ya = fmaf(m.w3[n0], tanh_fast(acc[nt][0] + m.b2[n0]), ya);
            ya = fmaf(m.w3[n0 + 1], tanh_fast(acc[nt][1] + m.b2[n0 + 1]), ya);
            yb = fmaf(m.w3[n0], tanh_fast(acc[nt][2] + m.b2[n0]), yb);
            yb = fmaf(m.w3[n0 + 1], tanh_fast(acc[nt][3] + m.b2[n0 + 1]), yb);
        }
        ya += __shfl_xor_sync(0xffffffffu, ya, 1);
        ya += __shfl_xor_sync(0xffffffffu, ya, 2);
        yb += __shfl_xor_sync(0xffffffffu, yb, 1);
        yb += __shfl_xor_sync(0xffffffffu, yb, 2);
        const int rr = lane & 15;  // row of this lane's cell within its tile
        const int src = 4 * (rr & 7);
        const float va = __shfl_sync(0xffffffffu, ya, src), vb = __shfl_sync(0xffffffffu, yb, src);
        if ((lane >> 4) == mt) yout = (rr < 8 ? va : vb) + m.b3;
    }
    return m.norm[4] + m.norm[5] * yout;
}

}  // namespace lbm
