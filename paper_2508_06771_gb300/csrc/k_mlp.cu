// k_mlp.cu -- rate-coefficient surrogate: a 66 -> 128 -> 128 -> 2 perceptron
// with GELU, BF16 weights and activations, FP32 accumulation, trained with Adam.
//
// The paper motivates it: rate terms C_kc = int sigma_kc |v| f (Eq. 1) feed the
// fluid equations, and resolving the high-energy tail can take tens of
// thousands of particles per cell (Sec. 1).  The network maps a cell's binned
// energy distribution (64 log bins) plus its density and mean energy to the
// ionization and elastic rate coefficients; the exact particle reduction of the
// cell kernel is both its training target and the reference for its error.
//
// Kernels: feature extraction from the per-cell moments, one fused kernel per
// 64-row tile for the forward pass and (when training) the backward pass with
// bfloat16 tensor-core MMAs (mma.sync m16n8k16, FP32 accumulate), a fixed-
// order reduction of the per-tile gradients, and Adam.  BF16 rounding happens
// at exactly the points the FP64 reference (oracle/mlp_oracle.c) rounds.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <new>
#include <vector>

#include "../../include/ltpc.h"
#include "ltpc_launch.h"
#include "philox.cuh"

namespace ltpc {
namespace mlp {

constexpr int DIN = 66, DINP = 80, H = 128, DOUT = 2;
constexpr int ROWS = 64;               // rows per CTA tile
constexpr int NTH = 256;               // threads per CTA (8 warps)
constexpr int LDX = DINP + 8;          // padded bf16 strides (conflict-free fragment loads)
constexpr int LDH = H + 8;
// packed parameter vector: W1 [H][DINP], b1 [H], W2 [H][H], b2 [H], W3 [DOUT][H], b3 [DOUT]
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * DINP, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + DOUT * H, NPARAM = OFF_B3 + DOUT;
constexpr int NPARAM_PAD = (NPARAM + 63) / 64 * 64;

struct Smem {
    __nv_bfloat16 w1[H * LDX];
    __nv_bfloat16 w2[H * LDH];
    float w3[DOUT * H];
    float b1[H], b2[H], b3[DOUT];
    __nv_bfloat16 x[ROWS * LDX];
    __nv_bfloat16 a1[ROWS * LDH];
    __nv_bfloat16 a2[ROWS * LDH];
    __nv_bfloat16 d[ROWS * LDH];      // dz2, then dz1
    float z1[ROWS * H];
    float z2[ROWS * H];
    float y[ROWS * DOUT];
    float g[ROWS * DOUT];
    float red[NTH / 32];
};

__device__ __forceinline__ uint16_t bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Warp tile of MT x NT8 MMA tiles: acc += A[m0.., 0..K) * B[0..K, n0..], with
// element accessors returning bfloat16 bits.  Fragment layout of m16n8k16:
// lane = 4 g + t; A rows g, g+8 and columns 2t, 2t+1, 2t+8, 2t+9; B columns g,
// rows 2t, 2t+1, 2t+8, 2t+9; C rows g, g+8, columns 2t, 2t+1.
template <int MT, int NT8, class FA, class FB>
__device__ __forceinline__ void warp_gemm(float (&acc)[MT][NT8][4], int m0, int n0, int K, FA ga, FB gb)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[MT][4];
#pragma unroll
        for (int mi = 0; mi < MT; ++mi) {
            const int r = m0 + mi * 16 + g;
            a[mi][0] = pack2(ga(r, k0 + 2 * t), ga(r, k0 + 2 * t + 1));
            a[mi][1] = pack2(ga(r + 8, k0 + 2 * t), ga(r + 8, k0 + 2 * t + 1));
            a[mi][2] = pack2(ga(r, k0 + 2 * t + 8), ga(r, k0 + 2 * t + 9));
            a[mi][3] = pack2(ga(r + 8, k0 + 2 * t + 8), ga(r + 8, k0 + 2 * t + 9));
        }
#pragma unroll
        for (int ni = 0; ni < NT8; ++ni) {
            const int c = n0 + ni * 8 + g;
            const uint32_t b0 = pack2(gb(k0 + 2 * t, c), gb(k0 + 2 * t + 1, c));
            const uint32_t b1 = pack2(gb(k0 + 2 * t + 8, c), gb(k0 + 2 * t + 9, c));
#pragma unroll
            for (int mi = 0; mi < MT; ++mi) mma_bf16(acc[mi][ni], a[mi], b0, b1);
        }
    }
}

// Visit the accumulator elements of a warp tile: f(row, col, value&).
template <int MT, int NT8, class F>
__device__ __forceinline__ void for_acc(float (&acc)[MT][NT8][4], int m0, int n0, F f)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int ni = 0; ni < NT8; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                f(m0 + mi * 16 + g + (e >= 2 ? 8 : 0), n0 + ni * 8 + 2 * t + (e & 1), acc[mi][ni][e]);
}

template <int MT, int NT8>
__device__ __forceinline__ void zero(float (&acc)[MT][NT8][4])
{
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int ni = 0; ni < NT8; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct Weights {
    const float* params;               // FP32 master parameters (biases and W3 used directly)
    const __nv_bfloat16* w1b;          // bf16 copies of W1, W2
    const __nv_bfloat16* w2b;
};

// One 64-row tile: forward; with `train`, also the backward pass, writing this
// tile's parameter-gradient partial sums and loss partial sum.
__global__ void __launch_bounds__(NTH) k_mlp_tile(Weights W, const float* __restrict__ X, const float* __restrict__ T,
                                                   int B, float* __restrict__ Y, int train,
                                                   float* __restrict__ gpart, float* __restrict__ lpart)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * ROWS;
    const int rows = min(ROWS, B - row0);

    // ---- stage weights and inputs (inputs rounded to bf16, padding zero).  The
    // bf16 weight rows move 16 bytes (8 values) at a time: every row of W1, W2
    // and of their padded shared-memory copies starts on a 16-byte boundary.
    constexpr int V1 = DINP / 8, V2 = H / 8;          // 16-byte vectors per row
    static_assert(DINP % 8 == 0 && H % 8 == 0 && LDX % 8 == 0 && LDH % 8 == 0, "16-byte rows");
    for (int i = tid; i < H * V1; i += NTH) {
        const int r = i / V1, c = (i % V1) * 8;
        *reinterpret_cast<uint4*>(&S.w1[r * LDX + c]) = *reinterpret_cast<const uint4*>(W.w1b + r * DINP + c);
    }
    for (int i = tid; i < H * V2; i += NTH) {
        const int r = i / V2, c = (i % V2) * 8;
        *reinterpret_cast<uint4*>(&S.w2[r * LDH + c]) = *reinterpret_cast<const uint4*>(W.w2b + r * H + c);
    }
    for (int i = tid; i < DOUT * H; i += NTH) S.w3[i] = W.params[OFF_W3 + i];
    for (int i = tid; i < H; i += NTH) { S.b1[i] = W.params[OFF_B1 + i]; S.b2[i] = W.params[OFF_B2 + i]; }
    if (tid < DOUT) S.b3[tid] = W.params[OFF_B3 + tid];
    for (int i = tid; i < ROWS * DINP; i += NTH) {
        const int r = i / DINP, c = i % DINP;
        const float v = (r < rows && c < DIN) ? X[(size_t)(row0 + r) * DIN + c] : 0.f;
        S.x[r * LDX + c] = __float2bfloat16_rn(v);
    }
    __syncthreads();

    // warp tiles for 64 x 128 outputs: 4 row blocks x 2 column halves
    const int wm = (warp & 3) * 16, wn = (warp >> 2) * 64;
    // ---- layer 1: z1 = x W1^T + b1, a1 = bf16(GELU(z1))
    {
        float acc[1][8][4];
        zero(acc);
        warp_gemm<1, 8>(acc, wm, wn, DINP, [&](int m, int k) { return bits(S.x[m * LDX + k]); },
                        [&](int k, int n) { return bits(S.w1[n * LDX + k]); });
        for_acc(acc, wm, wn, [&](int r, int c, float& v) {
            const float z = v + S.b1[c];
            S.z1[r * H + c] = z;
            S.a1[r * LDH + c] = __float2bfloat16_rn(gelu(z));
        });
    }
    __syncthreads();
    // ---- layer 2: z2 = a1 W2^T + b2, a2 = bf16(GELU(z2))
    {
        float acc[1][8][4];
        zero(acc);
        warp_gemm<1, 8>(acc, wm, wn, H, [&](int m, int k) { return bits(S.a1[m * LDH + k]); },
                        [&](int k, int n) { return bits(S.w2[n * LDH + k]); });
        for_acc(acc, wm, wn, [&](int r, int c, float& v) {
            const float z = v + S.b2[c];
            S.z2[r * H + c] = z;
            S.a2[r * LDH + c] = __float2bfloat16_rn(gelu(z));
        });
    }
    __syncthreads();
    // ---- layer 3 on CUDA cores: y = a2 W3^T + b3 (one warp per output column pair of rows)
    for (int i = tid; i < ROWS * DOUT; i += NTH) {
        const int r = i / DOUT, o = i % DOUT;
        float s = 0.f;
        for (int k = 0; k < H; ++k) s += __bfloat162float(S.a2[r * LDH + k]) * __bfloat162float(__float2bfloat16_rn(S.w3[o * H + k]));
        s += S.b3[o];
        S.y[i] = s;
        if (r < rows) Y[(size_t)(row0 + r) * DOUT + o] = s;
    }
    if (!train) return;
    __syncthreads();

    // ---- loss and dL/dy = 2 (y - t) / (B DOUT)
    {
        const float scale = 2.f / ((float)B * DOUT);
        float l = 0.f;
        for (int i = tid; i < ROWS * DOUT; i += NTH) {
            const int r = i / DOUT;
            float gv = 0.f;
            if (r < rows) {
                const float e = S.y[i] - T[(size_t)(row0 + r) * DOUT + i % DOUT];
                l += e * e;
                gv = scale * e;
            }
            S.g[i] = gv;
        }
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
        if (lane == 0) S.red[warp] = l;
    }
    __syncthreads();
    float* gp = gpart + (size_t)blockIdx.x * NPARAM_PAD;
    if (tid == 0) {
        float l = 0.f;
        for (int w = 0; w < NTH / 32; ++w) l += S.red[w];
        lpart[blockIdx.x] = l;
    }
    // ---- layer 3 gradients: gW3 = g^T a2, gb3 = sum g
    for (int i = tid; i < DOUT * H; i += NTH) {
        const int o = i / H, k = i % H;
        float s = 0.f;
        for (int r = 0; r < ROWS; ++r) s += S.g[r * DOUT + o] * __bfloat162float(S.a2[r * LDH + k]);
        gp[OFF_W3 + i] = s;
    }
    if (tid < DOUT) {
        float s = 0.f;
        for (int r = 0; r < ROWS; ++r) s += S.g[r * DOUT + tid];
        gp[OFF_B3 + tid] = s;
    }
    // ---- dz2 = bf16((g W3) * GELU'(z2))   (W3 used as bf16 like the forward pass)
    for (int i = tid; i < ROWS * H; i += NTH) {
        const int r = i / H, k = i % H;
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < DOUT; ++o) s += S.g[r * DOUT + o] * __bfloat162float(__float2bfloat16_rn(S.w3[o * H + k]));
        S.d[r * LDH + k] = __float2bfloat16_rn(s * gelu_grad(S.z2[r * H + k]));
    }
    __syncthreads();
    // ---- gb2 = sum over rows of dz2
    for (int c = tid; c < H; c += NTH) {
        float s = 0.f;
        for (int r = 0; r < ROWS; ++r) s += __bfloat162float(S.d[r * LDH + c]);
        gp[OFF_B2 + c] = s;
    }
    // ---- gW2 = dz2^T a1 (M = 128 outputs, N = 128 inputs, K = 64 rows): warp w owns outputs 16 w ..
    {
        float acc[1][16][4];
        zero(acc);
        warp_gemm<1, 16>(acc, warp * 16, 0, ROWS, [&](int m, int k) { return bits(S.d[k * LDH + m]); },
                         [&](int k, int n) { return bits(S.a1[k * LDH + n]); });
        for_acc(acc, warp * 16, 0, [&](int r, int c, float& v) { gp[OFF_W2 + r * H + c] = v; });
    }
    // ---- da1 = dz2 W2 (64 x 128), dz1 = bf16(da1 * GELU'(z1)) -> S.d after all uses of dz2
    float acc1[1][8][4];
    zero(acc1);
    warp_gemm<1, 8>(acc1, wm, wn, H, [&](int m, int k) { return bits(S.d[m * LDH + k]); },
                    [&](int k, int n) { return bits(S.w2[k * LDH + n]); });
    __syncthreads();
    for_acc(acc1, wm, wn, [&](int r, int c, float& v) {
        S.d[r * LDH + c] = __float2bfloat16_rn(v * gelu_grad(S.z1[r * H + c]));
    });
    __syncthreads();
    // ---- gb1 = sum dz1; gW1 = dz1^T x (M = 128, N = 80, K = 64)
    for (int c = tid; c < H; c += NTH) {
        float s = 0.f;
        for (int r = 0; r < ROWS; ++r) s += __bfloat162float(S.d[r * LDH + c]);
        gp[OFF_B1 + c] = s;
    }
    {
        float acc[1][10][4];
        zero(acc);
        warp_gemm<1, 10>(acc, warp * 16, 0, ROWS, [&](int m, int k) { return bits(S.d[k * LDH + m]); },
                         [&](int k, int n) { return bits(S.x[k * LDX + n]); });
        for_acc(acc, warp * 16, 0, [&](int r, int c, float& v) { gp[OFF_W1 + r * DINP + c] = v; });
    }
}

// Fixed-order sum of the per-tile partials (deterministic).
__global__ void k_mlp_reduce(const float* __restrict__ gpart, int tiles, float* __restrict__ grad,
                             const float* __restrict__ lpart, float* __restrict__ loss, float inv_count)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) {
        float s = 0.f;
        for (int c = 0; c < tiles; ++c) s += gpart[(size_t)c * NPARAM_PAD + p];
        grad[p] = s;
    }
    if (p == 0 && loss) {
        float s = 0.f;
        for (int c = 0; c < tiles; ++c) s += lpart[c];
        *loss = s * inv_count;
    }
}

// Adam update of the FP32 master parameters, then refresh of the bf16 copies.
__global__ void k_mlp_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, __nv_bfloat16* __restrict__ w1b, __nv_bfloat16* __restrict__ w2b,
                           float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float wp = w[p];
    if (lr != 0.f) {
        const float gv = g[p];
        const float mm = b1 * m[p] + (1.f - b1) * gv;
        const float vv = b2 * v[p] + (1.f - b2) * gv * gv;
        m[p] = mm;
        v[p] = vv;
        wp -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        if (p >= OFF_W1 && p < OFF_B1 && (p - OFF_W1) % DINP >= DIN) wp = 0.f;   // padding columns stay zero
        w[p] = wp;
    }
    if (p >= OFF_W1 && p < OFF_B1) w1b[p - OFF_W1] = __float2bfloat16_rn(wp);
    if (p >= OFF_W2 && p < OFF_B2) w2b[p - OFF_W2] = __float2bfloat16_rn(wp);
}

// Deterministic initialisation: uniform in +-1/sqrt(fan_in) from Philox, biases zero.
__global__ void k_mlp_init(float* __restrict__ w, uint64_t seed)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float bound = 0.f;
    if (p < OFF_B1) bound = ((p - OFF_W1) % DINP < DIN) ? rsqrtf((float)DIN) : 0.f;
    else if (p >= OFF_W2 && p < OFF_B2) bound = rsqrtf((float)H);
    else if (p >= OFF_W3 && p < OFF_B3) bound = rsqrtf((float)H);
    const uint4 r = draw((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)p, 0u, 7u);
    w[p] = bound * (2.f * unif<float>(r.x) - 1.f);
}

// Features of every cell from its moments (10 sums + 64-bin histogram):
// 64 bin fractions, log10 n_e, mean energy [eV]; normalised with (x - mean)/std.
// Targets: k_ion = sum sigma_ion|v| / N, k_el = sum sigma_el|v| / N [m^3/s].
// One warp per cell (lane l: bins l and l + 32; lanes 0 and 1 the last two
// features and the targets).  The features are binary32, so they are formed
// in binary32 from one reciprocal of N (binary64 divisions per feature ran on
// this GPU's narrow FP64 pipe).
constexpr int FEAT_WARPS = 4;
__global__ void __launch_bounds__(32 * FEAT_WARPS)
k_mlp_features(int M, const double* __restrict__ mom, const uint32_t* __restrict__ hist,
               const double* __restrict__ mom_dens, const double* __restrict__ inv_vol, double weight,
               double half_m_over_e,
               const float* __restrict__ fmean, const float* __restrict__ fistd, int normalize,
               float* __restrict__ Xo, float* __restrict__ To)
{
    const int j = blockIdx.x * FEAT_WARPS + (int)(threadIdx.x >> 5);
    const int lane = (int)(threadIdx.x & 31u);
    if (j >= M) return;
    const double* m = mom + (size_t)j * NMOM;
    const double N = m[0];
    const float iN = N > 0.0 ? 1.0f / (float)N : 0.0f;
    float* X = Xo + (size_t)j * DIN;
    auto put = [&](int c, float x) {
        if (normalize) x = (x - fmean[c]) * fistd[c];
        X[c] = x;
    };
    const uint32_t* hj = hist + (size_t)j * NBIN;
    put(lane, (float)hj[lane] * iN);
    put(lane + 32, (float)hj[lane + 32] * iN);
    if (lane == 0) {
        const double Nd = mom_dens ? mom_dens[(size_t)j * NMOM] : N;   // density from the whole cell
        put(NBIN, Nd > 0 ? log10f((float)(weight * Nd * inv_vol[j])) : 0.0f);
        if (To) To[(size_t)j * DOUT + 0] = (float)m[9] * iN;
    } else if (lane == 1) {
        put(NBIN + 1, (float)(half_m_over_e * (m[5] + m[6] + m[7])) * iN);
        if (To) To[(size_t)j * DOUT + 1] = (float)m[8] * iN;
    }
}

// Features of a random subsample of each cell: particle l of cell j is kept
// with probability per_cell / N_j (decided from a Philox word of (l, salt)).
// Accumulates a 64-bin histogram and the sample's count, sum of v^2 and rate
// sums with integer / float atomics into `sub` [M][NMOM] and `subh` [M][NBIN].
template <class T>
__global__ void k_subsample(const T* __restrict__ vx, const T* __restrict__ vy, const T* __restrict__ vz,
                            const int32_t* __restrict__ cell, const uint32_t* __restrict__ counts,
                            unsigned long long n, uint32_t per_cell, uint32_t salt, uint64_t seed,
                            double half_m_over_e, double sigma_el, double sigma_ion, double e_ion, XsArgs xs,
                            float* __restrict__ sub, uint32_t* __restrict__ subh)
{
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t c = cell[l];
        if (c < 0) continue;                              // removed (wall, recombination)
        const uint32_t N = counts[c];
        if (N == 0) continue;
        const uint4 r = draw((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)l, salt, 9u);
        if ((double)r.x >= (double)per_cell / (double)N * 4294967296.0) continue;
        const double x = vx[l], y = vy[l], z = vz[l];
        const double v2 = x * x + y * y + z * z, v = sqrt(v2), E = v2 * half_m_over_e;
        float* s = sub + (size_t)c * NMOM;
        atomicAdd(&s[0], 1.f);
        atomicAdd(&s[5], (float)v2);
        atomicAdd(&s[8], (float)(xs_el<double>(xs, E, sigma_el) * v));
        atomicAdd(&s[9], (float)(xs_ion<double>(xs, E, sigma_ion, e_ion) * v));
        int b = 0;
        if (E > 0.0) {
            const double t = (log10(E) + 2.0) * 12.8;
            b = t < 0.0 ? 0 : (t >= 63.0 ? 63 : (int)t);
        }
        atomicAdd(&subh[(size_t)c * NBIN + b], 1u);
    }
}

__global__ void k_sub_to_moments(int M, const float* __restrict__ sub, double* __restrict__ momd)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    for (int k = 0; k < NMOM; ++k) momd[(size_t)j * NMOM + k] = 0.0;
    momd[(size_t)j * NMOM + 0] = sub[(size_t)j * NMOM + 0];
    momd[(size_t)j * NMOM + 5] = sub[(size_t)j * NMOM + 5];
    momd[(size_t)j * NMOM + 8] = sub[(size_t)j * NMOM + 8];
    momd[(size_t)j * NMOM + 9] = sub[(size_t)j * NMOM + 9];
}

}  // namespace mlp
}  // namespace ltpc

using namespace ltpc;
using namespace ltpc::mlp;

struct ltpc_mlp {
    unsigned char* buf;
    int32_t batch_max, tiles_max;
    cudaStream_t stream;
    float *params, *m, *v, *grad, *gpart, *lpart, *loss, *fmean, *fistd, *tscale, *xbuf, *ybuf;
    float *sub;
    uint32_t* subh;
    double* subm;
    __nv_bfloat16 *w1b, *w2b;
    int32_t M_max;
    int adam_t;
};

namespace {

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

struct MlpLayout {
    size_t params, m, v, grad, gpart, lpart, loss, fmean, fistd, tscale, w1b, w2b, xbuf, ybuf, sub, subh, subm, total;
};

bool mlp_layout(int32_t batch_max, int32_t m_max, MlpLayout* L)
{
    if (batch_max < 1 || m_max < 0) return false;
    const size_t tiles = (size_t)(batch_max + ROWS - 1) / ROWS;
    const size_t rows = (size_t)(batch_max > m_max ? batch_max : m_max);
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o = up(o + b); return r; };
    L->params = take(NPARAM_PAD * 4);
    L->m = take(NPARAM_PAD * 4);
    L->v = take(NPARAM_PAD * 4);
    L->grad = take(NPARAM_PAD * 4);
    L->gpart = take(tiles * NPARAM_PAD * 4);
    L->lpart = take(tiles * 4);
    L->loss = take(4);
    L->fmean = take(DIN * 4);
    L->fistd = take(DIN * 4);
    L->tscale = take(DOUT * 4);
    L->w1b = take(H * DINP * 2);
    L->w2b = take(H * H * 2);
    L->xbuf = take(rows * DIN * 4);
    L->ybuf = take(rows * DOUT * 4);
    L->sub = take((size_t)(m_max > 0 ? m_max : 1) * NMOM * 4);
    L->subh = take((size_t)(m_max > 0 ? m_max : 1) * NBIN * 4);
    L->subm = take((size_t)(m_max > 0 ? m_max : 1) * NMOM * 8);
    L->total = o;
    return true;
}

cudaError_t tile_smem_attr()
{
    static cudaError_t once = cudaFuncSetAttribute(k_mlp_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(Smem));
    return once;
}

int run_tiles(ltpc_mlp* p, const float* X, const float* T, int B, float* Y, int train)
{
    if (B < 1 || B > p->batch_max) return LTPC_EINVAL;
    if (tile_smem_attr() != cudaSuccess) return LTPC_ECUDA;
    const int tiles = (B + ROWS - 1) / ROWS;
    Weights W{p->params, p->w1b, p->w2b};
    k_mlp_tile<<<tiles, NTH, sizeof(Smem), p->stream>>>(W, X, T, B, Y, train, p->gpart, p->lpart);
    if (cudaGetLastError() != cudaSuccess) return LTPC_ECUDA;
    if (train) {
        k_mlp_reduce<<<(NPARAM + 255) / 256, 256, 0, p->stream>>>(p->gpart, tiles, p->grad, p->lpart, p->loss,
                                                                  1.f / ((float)B * DOUT));
        if (cudaGetLastError() != cudaSuccess) return LTPC_ECUDA;
    }
    return LTPC_OK;
}

int refresh_bf16(ltpc_mlp* p)
{
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, p->stream>>>(p->params, p->grad, p->m, p->v, p->w1b, p->w2b, 0.f, 0.f,
                                                           0.f, 0.f, 1.f, 1.f);
    return cudaGetLastError() == cudaSuccess ? LTPC_OK : LTPC_ECUDA;
}

}  // namespace

extern "C" {

int ltpc_mlp_param_count(void) { return NPARAM; }

int ltpc_mlp_required_bytes(int32_t batch_max, int32_t n_cells_max, size_t* bytes)
{
    MlpLayout L;
    if (!bytes || !mlp_layout(batch_max, n_cells_max, &L)) return LTPC_EINVAL;
    *bytes = L.total;
    return LTPC_OK;
}

int ltpc_mlp_create(ltpc_mlp** out, void* d_buf, int32_t batch_max, int32_t n_cells_max, uint64_t seed,
                    void* cuda_stream)
{
    MlpLayout L;
    if (!out || !d_buf || ((uintptr_t)d_buf & 255) || !mlp_layout(batch_max, n_cells_max, &L)) return LTPC_EINVAL;
    ltpc_mlp* p = new (std::nothrow) ltpc_mlp();
    if (!p) return LTPC_EINVAL;
    unsigned char* b = (unsigned char*)d_buf;
    p->buf = b;
    p->batch_max = batch_max;
    p->M_max = n_cells_max;
    p->tiles_max = (batch_max + ROWS - 1) / ROWS;
    p->stream = (cudaStream_t)cuda_stream;
    p->params = (float*)(b + L.params); p->m = (float*)(b + L.m); p->v = (float*)(b + L.v);
    p->grad = (float*)(b + L.grad); p->gpart = (float*)(b + L.gpart); p->lpart = (float*)(b + L.lpart);
    p->loss = (float*)(b + L.loss); p->fmean = (float*)(b + L.fmean); p->fistd = (float*)(b + L.fistd);
    p->tscale = (float*)(b + L.tscale); p->w1b = (__nv_bfloat16*)(b + L.w1b); p->w2b = (__nv_bfloat16*)(b + L.w2b);
    p->xbuf = (float*)(b + L.xbuf); p->ybuf = (float*)(b + L.ybuf);
    p->sub = (float*)(b + L.sub); p->subh = (uint32_t*)(b + L.subh); p->subm = (double*)(b + L.subm);
    p->adam_t = 0;
    std::vector<float> ones(DIN, 1.f), zeros(DIN, 0.f);
    if (cudaMemsetAsync(b, 0, L.total, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(p->fistd, ones.data(), DIN * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(p->tscale, ones.data(), DOUT * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess) {
        delete p;
        return LTPC_ECUDA;
    }
    k_mlp_init<<<(NPARAM + 255) / 256, 256, 0, p->stream>>>(p->params, seed);
    if (cudaGetLastError() != cudaSuccess || refresh_bf16(p) != LTPC_OK ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
        delete p;
        return LTPC_ECUDA;
    }
    *out = p;
    return LTPC_OK;
}

void ltpc_mlp_destroy(ltpc_mlp* p) { delete p; }

int ltpc_mlp_set_params(ltpc_mlp* p, const float* params, int src_is_device)
{
    if (!p || !params) return LTPC_EINVAL;
    if (cudaMemcpyAsync(p->params, params, NPARAM * 4, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        p->stream) != cudaSuccess)
        return LTPC_ECUDA;
    if (refresh_bf16(p) != LTPC_OK) return LTPC_ECUDA;
    return cudaStreamSynchronize(p->stream) == cudaSuccess ? LTPC_OK : LTPC_ECUDA;
}

int ltpc_mlp_get_params(ltpc_mlp* p, float* params, int dst_is_device)
{
    if (!p || !params) return LTPC_EINVAL;
    if (cudaMemcpyAsync(params, p->params, NPARAM * 4, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        p->stream) != cudaSuccess)
        return LTPC_ECUDA;
    return cudaStreamSynchronize(p->stream) == cudaSuccess ? LTPC_OK : LTPC_ECUDA;
}

int ltpc_mlp_set_norm(ltpc_mlp* p, const float* feat_mean, const float* feat_std, const float* target_scale)
{
    if (!p || !feat_mean || !feat_std || !target_scale) return LTPC_EINVAL;
    float istd[DIN];
    for (int i = 0; i < DIN; ++i) istd[i] = feat_std[i] > 0.f ? 1.f / feat_std[i] : 1.f;
    if (cudaMemcpyAsync(p->fmean, feat_mean, DIN * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(p->fistd, istd, DIN * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(p->tscale, target_scale, DOUT * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
        return LTPC_ECUDA;
    return cudaStreamSynchronize(p->stream) == cudaSuccess ? LTPC_OK : LTPC_ECUDA;
}

int ltpc_mlp_forward(ltpc_mlp* p, const float* d_X, int32_t B, float* d_Y)
{
    if (!p || !d_X || !d_Y) return LTPC_EINVAL;
    return run_tiles(p, d_X, nullptr, B, d_Y, 0);
}

int ltpc_mlp_gradients(ltpc_mlp* p, const float* d_X, const float* d_T, int32_t B, float* d_grad, float* d_loss)
{
    if (!p || !d_X || !d_T) return LTPC_EINVAL;
    int rc = run_tiles(p, d_X, d_T, B, p->ybuf, 1);
    if (rc) return rc;
    if (d_grad && cudaMemcpyAsync(d_grad, p->grad, NPARAM * 4, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
        return LTPC_ECUDA;
    if (d_loss && cudaMemcpyAsync(d_loss, p->loss, 4, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
        return LTPC_ECUDA;
    return LTPC_OK;
}

int ltpc_mlp_train_step(ltpc_mlp* p, const float* d_X, const float* d_T, int32_t B, float lr, float* d_loss)
{
    if (!p || !d_X || !d_T || !(lr > 0.f)) return LTPC_EINVAL;
    int rc = run_tiles(p, d_X, d_T, B, p->ybuf, 1);
    if (rc) return rc;
    p->adam_t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, p->adam_t)), c2 = (float)(1.0 - std::pow(b2, p->adam_t));
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, p->stream>>>(p->params, p->grad, p->m, p->v, p->w1b, p->w2b, lr,
                                                           (float)b1, (float)b2, 1e-8f, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return LTPC_ECUDA;
    if (d_loss && cudaMemcpyAsync(d_loss, p->loss, 4, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
        return LTPC_ECUDA;
    return LTPC_OK;
}

}  // extern "C"

// ---- coupling with a collision context (defined here, declared in ltpc.h)
extern "C" int ltpc_internal_moments_view(ltpc_ctx* ctx, const double** mom, const uint32_t** hist,
                                          const double** inv_vol, int32_t* M, double* weight, double* half_m_over_e,
                                          cudaStream_t* stream);
extern "C" int ltpc_internal_particles_view(ltpc_ctx* ctx, const void** vx, const void** vy, const void** vz,
                                            const int32_t** cell, const uint32_t** counts, unsigned long long* n,
                                            int* precision, uint64_t* seed, double* sig_el, double* sig_ion,
                                            double* e_ion);
extern "C" int ltpc_internal_xs_view(ltpc_ctx* ctx, XsArgs* xs);

extern "C" int ltpc_mlp_features(ltpc_ctx* ctx, ltpc_mlp* p, float* d_X, float* d_T, int normalize)
{
    if (!ctx || !p || !d_X) return LTPC_EINVAL;
    const double *mom, *inv;
    const uint32_t* hist;
    int32_t M;
    double w, hme;
    cudaStream_t s;
    int rc = ltpc_internal_moments_view(ctx, &mom, &hist, &inv, &M, &w, &hme, &s);
    if (rc) return rc;
    k_mlp_features<<<(M + FEAT_WARPS - 1) / FEAT_WARPS, 32 * FEAT_WARPS, 0, s>>>(M, mom, hist, nullptr, inv, w, hme, p->fmean, p->fistd, normalize, d_X, d_T);
    return cudaGetLastError() == cudaSuccess ? LTPC_OK : LTPC_ECUDA;
}

__global__ void k_mlp_rates(int M, const float* __restrict__ Y, const float* __restrict__ tscale, float* __restrict__ R)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M * DOUT) R[i] = Y[i] * tscale[i % DOUT];
}

extern "C" int ltpc_mlp_infer(ltpc_ctx* ctx, ltpc_mlp* p, float* d_rates)
{
    if (!ctx || !p || !d_rates) return LTPC_EINVAL;
    const double *mom, *inv;
    const uint32_t* hist;
    int32_t M;
    double w, hme;
    cudaStream_t s;
    int rc = ltpc_internal_moments_view(ctx, &mom, &hist, &inv, &M, &w, &hme, &s);
    if (rc) return rc;
    if (M > p->batch_max && M > p->M_max) return LTPC_EINVAL;
    k_mlp_features<<<(M + FEAT_WARPS - 1) / FEAT_WARPS, 32 * FEAT_WARPS, 0, s>>>(M, mom, hist, nullptr, inv, w, hme, p->fmean, p->fistd, 1, p->xbuf, nullptr);
    if (cudaGetLastError() != cudaSuccess) return LTPC_ECUDA;
    // forward in batches of batch_max rows
    cudaStream_t keep = p->stream;
    p->stream = s;
    for (int32_t r0 = 0; r0 < M && rc == LTPC_OK; r0 += p->batch_max) {
        const int32_t B = M - r0 < p->batch_max ? M - r0 : p->batch_max;
        rc = run_tiles(p, p->xbuf + (size_t)r0 * DIN, nullptr, B, p->ybuf + (size_t)r0 * DOUT, 0);
    }
    p->stream = keep;
    if (rc) return rc;
    k_mlp_rates<<<(M * DOUT + 255) / 256, 256, 0, s>>>(M, p->ybuf, p->tscale, d_rates);
    return cudaGetLastError() == cudaSuccess ? LTPC_OK : LTPC_ECUDA;
}

extern "C" int ltpc_mlp_subsample_features(ltpc_ctx* ctx, ltpc_mlp* p, int32_t per_cell, uint32_t salt, float* d_X,
                                           float* d_rates_direct)
{
    if (!ctx || !p || !d_X || per_cell < 1) return LTPC_EINVAL;
    const double *mom, *inv;
    const uint32_t* hist;
    int32_t M;
    double w, hme;
    cudaStream_t s;
    int rc = ltpc_internal_moments_view(ctx, &mom, &hist, &inv, &M, &w, &hme, &s);
    if (rc) return rc;
    if (M > p->M_max) return LTPC_EINVAL;
    const void *vx, *vy, *vz;
    const int32_t* cell;
    const uint32_t* counts;
    unsigned long long n;
    int prec;
    uint64_t seed;
    double se, si, ei;
    rc = ltpc_internal_particles_view(ctx, &vx, &vy, &vz, &cell, &counts, &n, &prec, &seed, &se, &si, &ei);
    if (rc) return rc;
    XsArgs xs;
    rc = ltpc_internal_xs_view(ctx, &xs);
    if (rc) return rc;
    if (cudaMemsetAsync(p->sub, 0, (size_t)M * NMOM * 4, s) != cudaSuccess ||
        cudaMemsetAsync(p->subh, 0, (size_t)M * NBIN * 4, s) != cudaSuccess)
        return LTPC_ECUDA;
    if (prec == LTPC_F32)
        k_subsample<float><<<1024, 256, 0, s>>>((const float*)vx, (const float*)vy, (const float*)vz, cell, counts, n,
                                                (uint32_t)per_cell, salt, seed, hme, se, si, ei, xs, p->sub, p->subh);
    else
        k_subsample<double><<<1024, 256, 0, s>>>((const double*)vx, (const double*)vy, (const double*)vz, cell, counts,
                                                 n, (uint32_t)per_cell, salt, seed, hme, se, si, ei, xs, p->sub, p->subh);
    k_sub_to_moments<<<(M + 255) / 256, 256, 0, s>>>(M, p->sub, p->subm);
    // the distribution features and the direct rate estimate come from the sample only; the
    // density feature is the cell's density (known exactly from its count)
    k_mlp_features<<<(M + FEAT_WARPS - 1) / FEAT_WARPS, 32 * FEAT_WARPS, 0, s>>>(M, p->subm, p->subh, mom, inv, w, hme, p->fmean, p->fistd, 1, d_X, d_rates_direct);
    return cudaGetLastError() == cudaSuccess ? LTPC_OK : LTPC_ECUDA;
}
