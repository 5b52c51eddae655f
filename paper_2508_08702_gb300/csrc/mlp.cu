// mlp.cu -- the subtree scorer: a 3-layer MLP (32 -> 64 -> 64 -> 8) whose
// output orders the subtree queue of the first-solution mode.  It never
// changes the pruning, so the set of solutions of the all-solutions mode is
// unaffected.  Not part of the paper.
//
// All products run on the tensor cores: mma.sync m16n8k16 with bfloat16
// operands and float32 accumulation.  A warp owns 16 rows; the float32
// accumulator fragment of one layer (two adjacent 16x8 tiles) is exactly the
// bfloat16 A fragment of the next layer, so activations stay in registers.
// Weight gradients are contractions over the rows of a mini-batch, computed
// with the same instruction from bfloat16 copies of the activations staged
// in shared memory.
//
// Parameter vector (float32): W1[32][64] b1[64] W2[64][64] b2[64] W3[64][8] b3[8]
// (row = input).  Outputs: y0 = logit of P(the subtree holds a solution),
// y1 = predicted log(1 + nodes).  Loss per row: w BCE(y0, found) +
// 0.1 (y1 - log1p(nodes))^2, w = pos_weight for found rows; mean over rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace msp {

constexpr int kIn = 32, kHid = 64, kOut = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kOut, kParams = kOffB3 + kOut;   // 6792
constexpr float kNodeWeight = 0.1f;
constexpr int kRowsPerBlock = 128;   // 8 warps x 16 rows
constexpr int kWarps = kRowsPerBlock / 16;

struct __align__(16) MlpSmem {
    __nv_bfloat16 W1T[kHid][kIn + 8];    // [hid][in]   forward layer 1
    __nv_bfloat16 W2T[kHid][kHid + 8];   // [out][in]   forward layer 2
    __nv_bfloat16 W2[kHid][kHid + 8];    // [in][out]   backward through layer 2
    __nv_bfloat16 W3T[kOut][kHid + 8];   // [out][hid]  forward layer 3
    __nv_bfloat16 W3[kHid][kOut];        // [hid][out]  backward through layer 3
    float b1[kHid], b2[kHid], b3[kOut];
};

// bfloat16 copies of the mini-batch activations and gradients (training)
struct __align__(16) MlpStage {
    __nv_bfloat16 X[kRowsPerBlock][kIn];
    __nv_bfloat16 H1[kRowsPerBlock][kHid];
    __nv_bfloat16 H2[kRowsPerBlock][kHid];
    __nv_bfloat16 G1[kRowsPerBlock][kHid];   // dL/d(pre-activation 1)
    __nv_bfloat16 G2[kRowsPerBlock][kHid];   // dL/d(pre-activation 2)
    __nv_bfloat16 GY[kRowsPerBlock][kOut];   // dL/dy
    // per-warp partial bias gradients and losses, summed in warp order so
    // that training is deterministic
    float gb1w[kWarps][kHid], gb2w[kWarps][kHid], gb3w[kWarps][kOut];
    float lossw[kWarps];
    float loss;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {   // two adjacent bf16
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ uint32_t pair_of(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ void load_weights(MlpSmem& S, const float* __restrict__ th) {
    for (int e = threadIdx.x; e < kIn * kHid; e += blockDim.x) {
        const int i = e / kHid, h = e % kHid;
        S.W1T[h][i] = __float2bfloat16_rn(th[kOffW1 + e]);
    }
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
        const int i = e / kHid, o = e % kHid;
        const __nv_bfloat16 v = __float2bfloat16_rn(th[kOffW2 + e]);
        S.W2T[o][i] = v;
        S.W2[i][o] = v;
    }
    for (int e = threadIdx.x; e < kHid * kOut; e += blockDim.x) {
        const int h = e / kOut, o = e % kOut;
        const __nv_bfloat16 v = __float2bfloat16_rn(th[kOffW3 + e]);
        S.W3T[o][h] = v;
        S.W3[h][o] = v;
    }
    for (int e = threadIdx.x; e < kHid; e += blockDim.x) {
        S.b1[e] = th[kOffB1 + e];
        S.b2[e] = th[kOffB2 + e];
    }
    if (threadIdx.x < kOut) S.b3[threadIdx.x] = th[kOffB3 + threadIdx.x];
}

// Forward pass of the warp's 16 rows.  x(r, c) returns input feature c of
// local row r (0 for rows past the end).  On return C1, C2 hold the layer
// pre-activations (float32, accumulator layout) and C3 the outputs.
template <class XAt>
__device__ __forceinline__ void forward16(const MlpSmem& S, XAt x, float (&C1)[8][4], float (&C2)[8][4],
                                          float (&C3)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t a[4][4];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        a[s][0] = pack_bf16(x(g, 16 * s + 2 * t), x(g, 16 * s + 2 * t + 1));
        a[s][1] = pack_bf16(x(g + 8, 16 * s + 2 * t), x(g + 8, 16 * s + 2 * t + 1));
        a[s][2] = pack_bf16(x(g, 16 * s + 8 + 2 * t), x(g, 16 * s + 9 + 2 * t));
        a[s][3] = pack_bf16(x(g + 8, 16 * s + 8 + 2 * t), x(g + 8, 16 * s + 9 + 2 * t));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float bl = S.b1[8 * j + 2 * t], bh = S.b1[8 * j + 2 * t + 1];
        C1[j][0] = bl; C1[j][1] = bh; C1[j][2] = bl; C1[j][3] = bh;
#pragma unroll
        for (int s = 0; s < 2; ++s)
            mma_bf16(C1[j], a[s], ld_pair(&S.W1T[8 * j + g][16 * s + 2 * t]), ld_pair(&S.W1T[8 * j + g][16 * s + 8 + 2 * t]));
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a[s][0] = pack_bf16(fmaxf(C1[2 * s][0], 0.f), fmaxf(C1[2 * s][1], 0.f));
        a[s][1] = pack_bf16(fmaxf(C1[2 * s][2], 0.f), fmaxf(C1[2 * s][3], 0.f));
        a[s][2] = pack_bf16(fmaxf(C1[2 * s + 1][0], 0.f), fmaxf(C1[2 * s + 1][1], 0.f));
        a[s][3] = pack_bf16(fmaxf(C1[2 * s + 1][2], 0.f), fmaxf(C1[2 * s + 1][3], 0.f));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float bl = S.b2[8 * j + 2 * t], bh = S.b2[8 * j + 2 * t + 1];
        C2[j][0] = bl; C2[j][1] = bh; C2[j][2] = bl; C2[j][3] = bh;
#pragma unroll
        for (int s = 0; s < 4; ++s)
            mma_bf16(C2[j], a[s], ld_pair(&S.W2T[8 * j + g][16 * s + 2 * t]), ld_pair(&S.W2T[8 * j + g][16 * s + 8 + 2 * t]));
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a[s][0] = pack_bf16(fmaxf(C2[2 * s][0], 0.f), fmaxf(C2[2 * s][1], 0.f));
        a[s][1] = pack_bf16(fmaxf(C2[2 * s][2], 0.f), fmaxf(C2[2 * s][3], 0.f));
        a[s][2] = pack_bf16(fmaxf(C2[2 * s + 1][0], 0.f), fmaxf(C2[2 * s + 1][1], 0.f));
        a[s][3] = pack_bf16(fmaxf(C2[2 * s + 1][2], 0.f), fmaxf(C2[2 * s + 1][3], 0.f));
    }
    {
        const float bl = S.b3[2 * t], bh = S.b3[2 * t + 1];
        C3[0] = bl; C3[1] = bh; C3[2] = bl; C3[3] = bh;
#pragma unroll
        for (int s = 0; s < 4; ++s)
            mma_bf16(C3, a[s], ld_pair(&S.W3T[g][16 * s + 2 * t]), ld_pair(&S.W3T[g][16 * s + 8 + 2 * t]));
    }
}

// y = mlp(x) for n rows (x: n x 32 float32, y: n x 8 float32)
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* __restrict__ theta, const float* __restrict__ X,
                                                          int64_t n, float* __restrict__ Y) {
    __shared__ MlpSmem S;   // 26 KB
    load_weights(S, theta);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * 16; r0 < n; r0 += warps * 16) {
        auto x = [&](int r, int c) { return (r0 + r < n) ? X[(r0 + r) * kIn + c] : 0.f; };
        float C1[8][4], C2[8][4], C3[4];
        forward16(S, x, C1, C2, C3);
        if (r0 + g < n) { Y[(r0 + g) * kOut + 2 * t] = C3[0]; Y[(r0 + g) * kOut + 2 * t + 1] = C3[1]; }
        if (r0 + g + 8 < n) { Y[(r0 + g + 8) * kOut + 2 * t] = C3[2]; Y[(r0 + g + 8) * kOut + 2 * t + 1] = C3[3]; }
    }
}

// Sum over the 8 row groups g of a warp (lanes 4g + t): every lane gets the
// column totals of its t, combined in a fixed order.
__device__ __forceinline__ float2 rows_sum(float a, float b) {
#pragma unroll
    for (int off = 4; off <= 16; off <<= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    return make_float2(a, b);
}

// One block: loss and gradient (summed, already divided by `denom`) over the
// 128 rows rows[0..127] (row index < 0: padding).  Writes the gradient into
// grad (kParams floats, accumulated with +=) and adds the loss to *loss.
__device__ void block_grad(const MlpSmem& S, MlpStage& T, const float* __restrict__ X, const float* __restrict__ target,
                           const int64_t* rows, float denom, float pos_weight, float* grad) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int base = warp * 16;
    auto x = [&](int r, int c) { const int64_t i = rows[base + r]; return i >= 0 ? X[i * kIn + c] : 0.f; };
    float C1[8][4], C2[8][4], C3[4];
    forward16(S, x, C1, C2, C3);
    // stage bf16 inputs and activations (the values the forward pass multiplied)
    for (int e = lane; e < 16 * kIn; e += 32) {
        const int r = e / kIn, c = e % kIn;
        T.X[base + r][c] = __float2bfloat16_rn(x(r, c));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        T.H1[base + g][c] = __float2bfloat16_rn(fmaxf(C1[j][0], 0.f));
        T.H1[base + g][c + 1] = __float2bfloat16_rn(fmaxf(C1[j][1], 0.f));
        T.H1[base + g + 8][c] = __float2bfloat16_rn(fmaxf(C1[j][2], 0.f));
        T.H1[base + g + 8][c + 1] = __float2bfloat16_rn(fmaxf(C1[j][3], 0.f));
        T.H2[base + g][c] = __float2bfloat16_rn(fmaxf(C2[j][0], 0.f));
        T.H2[base + g][c + 1] = __float2bfloat16_rn(fmaxf(C2[j][1], 0.f));
        T.H2[base + g + 8][c] = __float2bfloat16_rn(fmaxf(C2[j][2], 0.f));
        T.H2[base + g + 8][c + 1] = __float2bfloat16_rn(fmaxf(C2[j][3], 0.f));
    }
    // dL/dy in the accumulator layout (only columns 0 and 1 are trained)
    float dY[4] = {0.f, 0.f, 0.f, 0.f};
    float lsum = 0.f;
    if (t == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = g + 8 * h;
            const int64_t i = rows[base + r];
            if (i < 0) continue;
            const float z = C3[2 * h], f = target[i * 2], ln = target[i * 2 + 1];
            const float w = f > 0.5f ? pos_weight : 1.f;
            const float p = 1.f / (1.f + __expf(-z));
            const float diff = C3[2 * h + 1] - ln;
            lsum += w * (fmaxf(z, 0.f) - z * f + log1pf(__expf(-fabsf(z)))) + kNodeWeight * diff * diff;
            dY[2 * h] = w * (p - f) / denom;
            dY[2 * h + 1] = 2.f * kNodeWeight * diff / denom;
        }
    }
    for (int off = 16; off >= 1; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0) T.lossw[warp] = lsum;
    T.GY[base + g][2 * t] = __float2bfloat16_rn(dY[0]);
    T.GY[base + g][2 * t + 1] = __float2bfloat16_rn(dY[1]);
    T.GY[base + g + 8][2 * t] = __float2bfloat16_rn(dY[2]);
    T.GY[base + g + 8][2 * t + 1] = __float2bfloat16_rn(dY[3]);
    {
        const float2 v = rows_sum(dY[0] + dY[2], dY[1] + dY[3]);
        if (g == 0) { T.gb3w[warp][2 * t] = v.x; T.gb3w[warp][2 * t + 1] = v.y; }
    }
    // dH2 = (dY W3^T) * [a2 > 0]   (K = 8 outputs, zero-padded to 16)
    uint32_t ay[4] = {pack_bf16(dY[0], dY[1]), pack_bf16(dY[2], dY[3]), 0u, 0u};
    float D2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        D2[j][0] = D2[j][1] = D2[j][2] = D2[j][3] = 0.f;
        mma_bf16(D2[j], ay, ld_pair(&S.W3[8 * j + g][2 * t]), 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) D2[j][q] = C2[j][q] > 0.f ? D2[j][q] : 0.f;
        const int c = 8 * j + 2 * t;
        const float2 v = rows_sum(D2[j][0] + D2[j][2], D2[j][1] + D2[j][3]);
        if (g == 0) { T.gb2w[warp][c] = v.x; T.gb2w[warp][c + 1] = v.y; }
        T.G2[base + g][c] = __float2bfloat16_rn(D2[j][0]);
        T.G2[base + g][c + 1] = __float2bfloat16_rn(D2[j][1]);
        T.G2[base + g + 8][c] = __float2bfloat16_rn(D2[j][2]);
        T.G2[base + g + 8][c + 1] = __float2bfloat16_rn(D2[j][3]);
    }
    // dH1 = (dH2 W2^T) * [a1 > 0]
    uint32_t a2[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a2[s][0] = pack_bf16(D2[2 * s][0], D2[2 * s][1]);
        a2[s][1] = pack_bf16(D2[2 * s][2], D2[2 * s][3]);
        a2[s][2] = pack_bf16(D2[2 * s + 1][0], D2[2 * s + 1][1]);
        a2[s][3] = pack_bf16(D2[2 * s + 1][2], D2[2 * s + 1][3]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float D1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int s = 0; s < 4; ++s)
            mma_bf16(D1, a2[s], ld_pair(&S.W2[8 * j + g][16 * s + 2 * t]), ld_pair(&S.W2[8 * j + g][16 * s + 8 + 2 * t]));
#pragma unroll
        for (int q = 0; q < 4; ++q) D1[q] = C1[j][q] > 0.f ? D1[q] : 0.f;
        const int c = 8 * j + 2 * t;
        const float2 v = rows_sum(D1[0] + D1[2], D1[1] + D1[3]);
        if (g == 0) { T.gb1w[warp][c] = v.x; T.gb1w[warp][c + 1] = v.y; }
        T.G1[base + g][c] = __float2bfloat16_rn(D1[0]);
        T.G1[base + g][c + 1] = __float2bfloat16_rn(D1[1]);
        T.G1[base + g + 8][c] = __float2bfloat16_rn(D1[2]);
        T.G1[base + g + 8][c + 1] = __float2bfloat16_rn(D1[3]);
    }
    __syncthreads();
    // weight gradients: dW = A^T G over the 128 rows; tiles of 16 x 8 spread over the warps
    //   dW1 = X^T G1  (32 x 64: 2 x 8 tiles)   dW2 = H1^T G2  (64 x 64: 4 x 8)   dW3 = H2^T GY (64 x 8: 4 x 1)
    for (int tile = warp; tile < 16 + 32 + 4; tile += blockDim.x / 32) {
        const __nv_bfloat16* Am;
        const __nv_bfloat16* Gm;
        int lda, ldg, mt, nt, off, ncol;
        if (tile < 16) { Am = &T.X[0][0]; lda = kIn; Gm = &T.G1[0][0]; ldg = kHid; mt = tile / 8; nt = tile % 8; off = kOffW1; ncol = kHid; }
        else if (tile < 48) { Am = &T.H1[0][0]; lda = kHid; Gm = &T.G2[0][0]; ldg = kHid; mt = (tile - 16) / 8; nt = (tile - 16) % 8; off = kOffW2; ncol = kHid; }
        else { Am = &T.H2[0][0]; lda = kHid; Gm = &T.GY[0][0]; ldg = kOut; mt = tile - 48; nt = 0; off = kOffW3; ncol = kOut; }
        float D[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < kRowsPerBlock; k0 += 16) {
            // A(m, k) = Act[k0 + k][16 mt + m];  B(k, n) = Grad[k0 + k][8 nt + n]
            uint32_t a[4];
            const int m0 = 16 * mt + g, kk = k0 + 2 * t;
            a[0] = pair_of(Am[(kk) * lda + m0], Am[(kk + 1) * lda + m0]);
            a[1] = pair_of(Am[(kk) * lda + m0 + 8], Am[(kk + 1) * lda + m0 + 8]);
            a[2] = pair_of(Am[(kk + 8) * lda + m0], Am[(kk + 9) * lda + m0]);
            a[3] = pair_of(Am[(kk + 8) * lda + m0 + 8], Am[(kk + 9) * lda + m0 + 8]);
            const int n0 = 8 * nt + g;
            const uint32_t b0 = pair_of(Gm[(kk) * ldg + n0], Gm[(kk + 1) * ldg + n0]);
            const uint32_t b1 = pair_of(Gm[(kk + 8) * ldg + n0], Gm[(kk + 9) * ldg + n0]);
            mma_bf16(D, a, b0, b1);
        }
        const int r = 16 * mt + g, c = 8 * nt + 2 * t;
        atomicAdd(&grad[off + r * ncol + c], D[0]);
        atomicAdd(&grad[off + r * ncol + c + 1], D[1]);
        atomicAdd(&grad[off + (r + 8) * ncol + c], D[2]);
        atomicAdd(&grad[off + (r + 8) * ncol + c + 1], D[3]);
    }
    for (int e = threadIdx.x; e < kHid; e += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kWarps; ++w) { a += T.gb1w[w][e]; b += T.gb2w[w][e]; }
        atomicAdd(&grad[kOffB1 + e], a);
        atomicAdd(&grad[kOffB2 + e], b);
    }
    if (threadIdx.x < kOut) {
        float a = 0.f;
        for (int w = 0; w < kWarps; ++w) a += T.gb3w[w][threadIdx.x];
        atomicAdd(&grad[kOffB3 + threadIdx.x], a);
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int w = 0; w < kWarps; ++w) l += T.lossw[w];
        T.loss = l;
    }
    __syncthreads();
}

// Gradient of the mean loss over n rows; one block per 128 rows.
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float* __restrict__ theta, const float* __restrict__ X,
                                                       const float* __restrict__ target, int64_t n, float pos_weight,
                                                       float* __restrict__ grad, float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char dsm[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(dsm);
    MlpStage& T = *reinterpret_cast<MlpStage*>(dsm + sizeof(MlpSmem));
    int64_t* rows = reinterpret_cast<int64_t*>(dsm + sizeof(MlpSmem) + sizeof(MlpStage));
    load_weights(S, theta);
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
    for (int r = threadIdx.x; r < kRowsPerBlock; r += blockDim.x) rows[r] = (r0 + r < n) ? r0 + r : -1;
    __syncthreads();
    block_grad(S, T, X, target, rows, (float)n, pos_weight, grad);
    if (threadIdx.x == 0) atomicAdd(loss, T.loss / (float)n);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {   // splitmix64 finaliser
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Adam on mini-batches of 128 rows drawn uniformly with replacement (one
// block; the gradient buffer `work` holds kParams floats, m and v follow).
__global__ void __launch_bounds__(256) mlp_train_kernel(float* __restrict__ theta, const float* __restrict__ X,
                                                        const float* __restrict__ target, int64_t n, int steps,
                                                        float lr, float pos_weight, uint64_t seed,
                                                        float* __restrict__ work, float* __restrict__ losses) {
    extern __shared__ __align__(16) unsigned char dsm[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(dsm);
    MlpStage& T = *reinterpret_cast<MlpStage*>(dsm + sizeof(MlpSmem));
    int64_t* rows = reinterpret_cast<int64_t*>(dsm + sizeof(MlpSmem) + sizeof(MlpStage));
    float* grad = work;
    float* m1 = work + kParams;
    float* m2 = work + 2 * kParams;
    for (int e = threadIdx.x; e < 3 * kParams; e += blockDim.x) work[e] = 0.f;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float p1 = 1.f, p2 = 1.f;
    for (int step = 0; step < steps; ++step) {
        __syncthreads();
        load_weights(S, theta);
        for (int r = threadIdx.x; r < kRowsPerBlock; r += blockDim.x)
            rows[r] = (int64_t)(mix64(seed ^ ((uint64_t)step << 20) ^ (uint64_t)r) % (uint64_t)n);
        for (int e = threadIdx.x; e < kParams; e += blockDim.x) grad[e] = 0.f;
        __syncthreads();
        block_grad(S, T, X, target, rows, (float)kRowsPerBlock, pos_weight, grad);
        __syncthreads();
        p1 *= b1;
        p2 *= b2;
        for (int e = threadIdx.x; e < kParams; e += blockDim.x) {
            const float gr = grad[e];
            const float a = m1[e] = b1 * m1[e] + (1.f - b1) * gr;
            const float b = m2[e] = b2 * m2[e] + (1.f - b2) * gr * gr;
            theta[e] -= lr * (a / (1.f - p1)) / (sqrtf(b / (1.f - p2)) + eps);
        }
        if (threadIdx.x == 0 && losses) losses[step] = T.loss / (float)kRowsPerBlock;
    }
}

constexpr size_t kTrainSmem = sizeof(MlpSmem) + sizeof(MlpStage) + sizeof(int64_t) * kRowsPerBlock;

cudaError_t mlp_forward(const float* theta, const float* X, int64_t n, float* Y, int sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + kRowsPerBlock - 1) / kRowsPerBlock;
    mlp_forward_kernel<<<(int)(blocks < 4 * sms ? blocks : 4 * sms), 256, 0, st>>>(theta, X, n, Y);
    return cudaGetLastError();
}

cudaError_t mlp_grad(const float* theta, const float* X, const float* target, int64_t n, float pos_weight,
                     float* grad, float* loss, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kParams, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess || n <= 0) return e;
    const int64_t blocks = (n + kRowsPerBlock - 1) / kRowsPerBlock;
    e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    if (e != cudaSuccess) return e;
    mlp_grad_kernel<<<(int)blocks, 256, kTrainSmem, st>>>(theta, X, target, n, pos_weight, grad, loss);
    return cudaGetLastError();
}

cudaError_t mlp_train(float* theta, const float* X, const float* target, int64_t n, int steps, float lr,
                      float pos_weight, uint64_t seed, float* work, float* losses, cudaStream_t st) {
    if (n <= 0 || steps <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    if (e != cudaSuccess) return e;
    mlp_train_kernel<<<1, 256, kTrainSmem, st>>>(theta, X, target, n, steps, lr, pos_weight, seed, work, losses);
    return cudaGetLastError();
}

int mlp_param_count() { return kParams; }

}  // namespace msp
