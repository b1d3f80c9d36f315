// Warm-start MLP with H = 64 hidden units on the tensor cores: bfloat16
// operands, tcgen05.mma kind::f16 with float32 accumulation in tensor memory.
//
// Model (F = 8 features, two tanh layers of 64, one output), per point p:
//   z1 = W1 x + b1, h1 = tanh z1, z2 = W2 bf16(h1) + b2, h2 = tanh z2,
//   y = W3 . h2 + b3,
// with x, W1, W2, W3 in bfloat16 (rounded from the float64 master weights),
// b1, b2, b3 and every activation in float32; the input of the second layer
// is rounded to bfloat16 as the tensor cores take it.  Gradient of
// L = sum_p wt_p (y_p - t_p)^2:
//   dy = 2 wt (y - t), dz2 = dy W3 (1 - h2^2), dz1 = (bf16(dz2) W2)(1 - h1^2),
//   dW2 = sum bf16(dz2) bf16(h1)^T, db2 = sum bf16(dz2),
//   dW1 = sum bf16(dz1) x^T,        db1 = sum bf16(dz1),
//   dW3 = sum bf16(dy) bf16(h2),    db3 = sum bf16(dy).
//
// One CTA of four warpgroups (512 threads) per SM, persistent over 128-point
// tiles.  Point p of a tile is TMEM lane p of the per-point products, and
// warpgroup g handles hidden units [16 g, 16 g + 16) of every point (a warp
// reads its own 32-lane quarter of TMEM, so thread 128 g + p owns point p's
// units of block g).  Four warps per scheduler hide the latency of the
// activation work (tanh, rounding, operand stores), which is what bounds a
// tile; the products are:
//   Z1 = X W1^T           (M 128 points, N 64, K 16: features padded)
//   Z2 = H1 W2^T          (M 128, N 64, K 64)
//   dH1 = dZ2 W2          (M 128, N 64, K 64)
// and the weight gradients are contractions over the tile's points,
// accumulated in TMEM over up to kFold tiles:
//   D1 = [dZ2^T; dZ1^T] [H1^T; X^T; 1]^T   (M 128 = 64 + 64, N 80, K 128)
//   D2 = [H2^T; 1] [dy]^T                  (M 128, N 16, K 128)
// then added to the CTA's float64 partial row in global memory (each entry
// is one TMEM lane and column, read by one thread: one writer).  All operand tiles are
// K-major with the 128-byte swizzle (64 bf16 per row); an operand with K =
// 128 points is two such tiles.  Every wait is bounded; one that gives up
// sets *err and the CTA returns after a bounded wait for its MMAs.
#include <cuda_runtime.h>

#include "tagi_internal.cuh"
#include "tc.cuh"

namespace tagi {

namespace {

constexpr int kF = 8;
constexpr int kH = 64;
constexpr int oW1 = 0, oB1 = kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kP64 = oB3 + 1;  // 4801 parameters
constexpr int kT = 128;        // points per tile
constexpr int kWG = 4;         // warpgroups per CTA
constexpr int kCB = 64 / kWG;  // hidden units per warpgroup
constexpr int kThreads = kT * kWG;
constexpr int kFold = 8;       // tiles accumulated in tensor memory between float64 folds
constexpr long long kWait = 2000000000LL;
constexpr uint32_t kCols = 512;

// byte layout of the shared memory (every tile 1024-aligned)
constexpr int sX = 0;                    // 128 rows (points) x 128 B: features 0..7, zeros
constexpr int sW1 = sX + 128 * 128;      // 64 rows (units) x 128 B: W1 row, zeros
constexpr int sW2 = sW1 + 64 * 128;      // 64 rows (out j) x 64 (in i)
constexpr int sW2T = sW2 + 64 * 128;     // 64 rows (in i) x 64 (out j)
constexpr int sH1 = sW2T + 64 * 128;     // 128 rows (points) x 64 (i): bf16(h1)
constexpr int sDZ2 = sH1 + 128 * 128;    // 128 rows (points) x 64 (j): bf16(dz2)
constexpr int sAT = sDZ2 + 128 * 128;    // 2 tiles of 128 rows ([dz2 j; dz1 i]) x 64 points
constexpr int sBT = sAT + 2 * 128 * 128; // 2 tiles of 80 rows ([h1 i; x f; 1; 0]) x 64 points
constexpr int sA2 = sBT + 2 * 80 * 128;  // 2 tiles of 128 rows ([h2 k; 1; 0]) x 64 points
constexpr int sB2 = sA2 + 2 * 128 * 128; // 2 tiles of 16 rows ([dy; 0]) x 64 points
constexpr int kSmem = sB2 + 2 * 16 * 128;
constexpr int kSmemAlloc = kSmem + 1024;
// TMEM columns
constexpr uint32_t cZ1 = 0, cZ2 = 64, cDH1 = 128, cD1 = 192, cD2 = 272;

__device__ __forceinline__ uint32_t swz2(int r, int k)  // bf16 element k of row r, 128B swizzle
{
    return r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint16_t bf16_rn(float x)  // nearest, ties to even (finite x)
{
    const uint32_t u = __float_as_uint(x);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

__device__ __forceinline__ float bf16_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// nearest bfloat16 of a float64 value, ties to even, as the H = 32 kernels round
__device__ __forceinline__ uint16_t bf16_of_double(double x)
{
    if (x == 0.0) return signbit(x) ? 0x8000 : 0;
    int e;
    frexp(x, &e);
    const double q = ldexp(1.0, max(e - 8, -133));
    return (uint16_t)(__float_as_uint((float)(rint(x / q) * q)) >> 16);
}

__device__ __forceinline__ void st16(uint8_t* sm, uint32_t off, uint16_t v) { *reinterpret_cast<uint16_t*>(sm + off) = v; }

struct Bias {
    float b1[kH], b2[kH], w3[kH], b3;
};

// MMAs of one stage, issued by thread 0, then all threads wait for them
struct Sync {
    uint64_t* bar;
    uint32_t phase;
    bool ok;
    __device__ void wait()
    {
        if (ok && !tc::mbar_wait(bar, phase, kWait)) ok = false;
        phase ^= 1;
        tc::fence_after_sync();
    }
};

__device__ __forceinline__ void mma_chain(uint32_t d, uint32_t a, uint32_t b, int ksteps, uint32_t idesc, bool acc0)
{
    const uint64_t da = tc::sdesc_sw128(a), db = tc::sdesc_sw128(b);
    for (int k = 0; k < ksteps; k++) tc::mma_bf16(d, da + 2 * k, db + 2 * k, idesc, (k > 0 || acc0) ? 1u : 0u);
}

// the thread's place: point (TMEM lane) pl of the tile, hidden units
// [c0, c0 + kCB) of warpgroup g
struct Who {
    int t, pl, g, c0;
    uint32_t lane_base;
    __device__ explicit Who(uint32_t tmem)
    {
        t = threadIdx.x;
        pl = t & (kT - 1);
        g = t / kT;
        c0 = g * kCB;
        lane_base = tmem + ((uint32_t)((pl >> 5) * 32) << 16);
    }
};

// Weights (bf16 operand tiles) and float32 biases from the float64 master
// weights; zero every operand tile; the constant rows of the transposed tiles.
__device__ void setup(uint8_t* sm, Bias* B, const double* __restrict__ master)
{
    for (int e = threadIdx.x; e < kSmem / 16; e += kThreads) reinterpret_cast<uint4*>(sm)[e] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int e = threadIdx.x; e < kH * kF; e += kThreads)
        st16(sm, sW1 + swz2(e / kF, e % kF), bf16_of_double(master[oW1 + e]));
    for (int e = threadIdx.x; e < kH * kH; e += kThreads) {
        const int j = e / kH, i = e % kH;
        const uint16_t v = bf16_of_double(master[oW2 + e]);
        st16(sm, sW2 + swz2(j, i), v);
        st16(sm, sW2T + swz2(i, j), v);
    }
    for (int e = threadIdx.x; e < kH; e += kThreads) {
        B->b1[e] = (float)master[oB1 + e];
        B->b2[e] = (float)master[oB2 + e];
        B->w3[e] = bf16_f(bf16_of_double(master[oW3 + e]));
    }
    if (threadIdx.x == 0) B->b3 = (float)master[oB3];
    // ones rows: BT row 72 (bias of the first layer's gradient), A2 row 64
    for (int e = threadIdx.x; e < 2 * 64; e += kThreads) {
        const int t = e / 64, p = e % 64;
        st16(sm, sBT + t * 80 * 128 + swz2(72, p), 0x3F80);
        st16(sm, sA2 + t * 128 * 128 + swz2(64, p), 0x3F80);
    }
}

// Forward pass of point p (lane pl) for this warpgroup's units; returns y.
// h1, h2: this warpgroup's activations of the point (float32), xb: the
// point's features (warpgroup 0 only).  ypart: [kWG][kT] shared partial
// sums of W3 . h2, one per warpgroup, added in warpgroup order.
__device__ float forward_tile(uint8_t* sm, const Bias& B, const uint16_t* __restrict__ feat, int64_t p, bool valid,
                              const Who& w, uint32_t tmem, Sync& sy, float* ypart, float h1[kCB], float h2[kCB],
                              uint16_t xb[kF])
{
    if (w.g == 0) {
        uint4 xv = make_uint4(0, 0, 0, 0);
        if (valid) xv = *reinterpret_cast<const uint4*>(feat + p * kF);
        const uint32_t xu[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            xb[2 * k] = (uint16_t)(xu[k] & 0xFFFFu);
            xb[2 * k + 1] = (uint16_t)(xu[k] >> 16);
        }
#pragma unroll
        for (int f = 0; f < kF; f++) st16(sm, sX + swz2(w.pl, f), xb[f]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (w.t == 0) {
        tc::fence_after_sync();
        mma_chain(tmem + cZ1, tc::smem_u32(sm + sX), tc::smem_u32(sm + sW1), 1, tc::idesc_bf16(128, 64), false);
        tc::commit(sy.bar);
    }
    sy.wait();
    // h1 = tanh(z1 + b1) -> bf16 into the second layer's A tile
#pragma unroll
    for (int c = 0; c < kCB; c += 8) {
        float v[8];
        tc::tmem_ld8(w.lane_base + cZ1 + w.c0 + c, v);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            h1[c + i] = tanhf(v[i] + B.b1[w.c0 + c + i]);
            st16(sm, sH1 + swz2(w.pl, w.c0 + c + i), bf16_rn(h1[c + i]));
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (w.t == 0) {
        tc::fence_after_sync();
        mma_chain(tmem + cZ2, tc::smem_u32(sm + sH1), tc::smem_u32(sm + sW2), 4, tc::idesc_bf16(128, 64), false);
        tc::commit(sy.bar);
    }
    sy.wait();
    float yp = 0.0f;
#pragma unroll
    for (int c = 0; c < kCB; c += 8) {
        float v[8];
        tc::tmem_ld8(w.lane_base + cZ2 + w.c0 + c, v);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            h2[c + i] = tanhf(v[i] + B.b2[w.c0 + c + i]);
            yp = fmaf(B.w3[w.c0 + c + i], h2[c + i], yp);
        }
    }
    ypart[w.g * kT + w.pl] = yp;
    __syncthreads();
    float y = B.b3;
#pragma unroll
    for (int q = 0; q < kWG; q++) y += ypart[q * kT + w.pl];
    return y;
}

__global__ void __launch_bounds__(kThreads, 1) k_mlp64_fwd(const uint16_t* __restrict__ feat, int64_t n,
                                                           const double* __restrict__ master, float* __restrict__ y,
                                                           int* __restrict__ err)
{
    extern __shared__ uint8_t raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    __shared__ Bias B;
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    __shared__ float ypart[kWG * kT];
    const int t = threadIdx.x;
    setup(sm, &B, master);
    if ((t >> 5) == 0) tc::tmem_alloc(&slot, kCols);
    if (t == 0) tc::mbar_init(&bar, 1);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = slot;
    const Who w(tmem);
    Sync sy{&bar, 0, true};
    const int64_t ntiles = (n + kT - 1) / kT;
    for (int64_t tile = blockIdx.x; tile < ntiles && __syncthreads_and(sy.ok); tile += gridDim.x) {
        const int64_t p = tile * kT + w.pl;
        float h1[kCB], h2[kCB];
        uint16_t xb[kF];
        const float out = forward_tile(sm, B, feat, p, p < n, w, tmem, sy, ypart, h1, h2, xb);
        if (w.g == 0 && p < n && sy.ok) y[p] = out;
    }
    if (!__syncthreads_and(sy.ok) && t == 0) {
        atomicOr(err, 1);
        tc::mbar_wait(&bar, sy.phase ^ 1, kWait);  // the MMAs of the last commit, bounded
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((t >> 5) == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kCols);
    }
}

// partial[blockIdx.x][kP64 + 1] (the loss last): this CTA's gradient sums
__global__ void __launch_bounds__(kThreads, 1) k_mlp64_grad(const uint16_t* __restrict__ feat,
                                                            const float* __restrict__ target,
                                                            const float* __restrict__ wt, int64_t n,
                                                            const double* __restrict__ master,
                                                            double* __restrict__ partial, int* __restrict__ err)
{
    extern __shared__ uint8_t raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    __shared__ Bias B;
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    __shared__ float ypart[kWG * kT];
    __shared__ double lsum[kT];
    const int t = threadIdx.x;
    double* out = partial + (size_t)blockIdx.x * (kP64 + 1);
    for (int e = t; e <= kP64; e += kThreads) out[e] = 0.0;
    setup(sm, &B, master);
    if ((t >> 5) == 0) tc::tmem_alloc(&slot, kCols);
    if (t == 0) tc::mbar_init(&bar, 1);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = slot;
    const Who w(tmem);
    Sync sy{&bar, 0, true};
    double loss = 0.0;
    const int64_t ntiles = (n + kT - 1) / kT;
    // the tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int64_t mine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int tp = w.pl & 63, tt = w.pl >> 6;  // column of this point in the transposed tiles, and which tile

    // TMEM lane r of D1 and D2 into the parameters: D1's 8-column chunks go
    // round-robin over the warpgroups, D2 (one column) to warpgroup 0; every
    // entry has one writer
    auto fold = [&]() {
        const int r = w.pl;
#pragma unroll 1
        for (int q = w.g; q < 10; q += kWG) {
            const int c8 = q * 8;
            float v[8];
            tc::tmem_ld8(w.lane_base + cD1 + c8, v);
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int c = c8 + i;
                int e = -1;
                if (r < 64) {
                    if (c < 64) e = oW2 + r * kH + c;
                    else if (c == 72) e = oB2 + r;
                } else {
                    if (c >= 64 && c < 72) e = oW1 + (r - 64) * kF + (c - 64);
                    else if (c == 72) e = oB1 + (r - 64);
                }
                if (e >= 0) out[e] += (double)v[i];
            }
        }
        if (w.g == 0) {
            float v[8];
            tc::tmem_ld8(w.lane_base + cD2, v);
            if (r < 64) out[oW3 + r] += (double)v[0];
            if (r == 64) out[oB3] += (double)v[0];
        }
    };

    for (int64_t k = 0; k < mine && __syncthreads_and(sy.ok); k++) {
        const int64_t tile = blockIdx.x + k * gridDim.x;
        const int64_t p = tile * kT + w.pl;
        const bool valid = p < n;
        float h1[kCB], h2[kCB];
        uint16_t xb[kF];
        const float yv = forward_tile(sm, B, feat, p, valid, w, tmem, sy, ypart, h1, h2, xb);
        const float r = valid ? yv - target[p] : 0.0f;
        const float wv = valid ? wt[p] : 0.0f;
        if (w.g == 0) loss += (double)wv * (double)r * (double)r;
        const float dy = 2.0f * wv * r;
        // dz2 (A of dH1, and rows j of D1's A), h2 (rows j of D2's A) and
        // bf16(h1) (rows i of D1's B) for this warpgroup's units
#pragma unroll
        for (int j = 0; j < kCB; j++) {
            const int jj = w.c0 + j;
            const uint16_t d = bf16_rn(dy * B.w3[jj] * (1.0f - h2[j] * h2[j]));
            st16(sm, sDZ2 + swz2(w.pl, jj), d);
            st16(sm, sAT + tt * 128 * 128 + swz2(jj, tp), d);
            st16(sm, sA2 + tt * 128 * 128 + swz2(jj, tp), bf16_rn(h2[j]));
            st16(sm, sBT + tt * 80 * 128 + swz2(jj, tp), bf16_rn(h1[j]));
        }
        if (w.g == 0) {
            // dy (D2's B) and x (rows 64..71 of D1's B)
            st16(sm, sB2 + tt * 16 * 128 + swz2(0, tp), bf16_rn(dy));
#pragma unroll
            for (int f = 0; f < kF; f++) st16(sm, sBT + tt * 80 * 128 + swz2(64 + f, tp), xb[f]);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (w.t == 0) {
            tc::fence_after_sync();
            mma_chain(tmem + cDH1, tc::smem_u32(sm + sDZ2), tc::smem_u32(sm + sW2T), 4, tc::idesc_bf16(128, 64), false);
            tc::commit(sy.bar);
        }
        sy.wait();
        // dz1 = dh1 (1 - h1^2) (rows 64 + i of D1's A)
#pragma unroll
        for (int c = 0; c < kCB; c += 8) {
            float a[8];
            tc::tmem_ld8(w.lane_base + cDH1 + w.c0 + c, a);
#pragma unroll
            for (int i = 0; i < 8; i++)
                st16(sm, sAT + tt * 128 * 128 + swz2(64 + w.c0 + c + i, tp), bf16_rn(a[i] * (1.0f - h1[c + i] * h1[c + i])));
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (w.t == 0) {
            tc::fence_after_sync();
            const bool acc = (k % kFold) != 0;
            const uint32_t aT = tc::smem_u32(sm + sAT), bT = tc::smem_u32(sm + sBT);
            const uint32_t a2 = tc::smem_u32(sm + sA2), b2 = tc::smem_u32(sm + sB2);
            // K = 128 points: two 64-point tiles of each operand
            mma_chain(tmem + cD1, aT, bT, 4, tc::idesc_bf16(128, 80), acc);
            mma_chain(tmem + cD1, aT + 128 * 128, bT + 80 * 128, 4, tc::idesc_bf16(128, 80), true);
            mma_chain(tmem + cD2, a2, b2, 4, tc::idesc_bf16(128, 16), acc);
            mma_chain(tmem + cD2, a2 + 128 * 128, b2 + 16 * 128, 4, tc::idesc_bf16(128, 16), true);
            tc::commit(sy.bar);
        }
        // the next tile rewrites these operand tiles: wait here
        sy.wait();
        if ((k % kFold) == kFold - 1 || k == mine - 1) fold();
        tc::fence_before_sync();
    }
    if (w.g == 0) lsum[w.pl] = loss;
    const bool ok = __syncthreads_and(sy.ok);
    if (!ok && t == 0) {
        atomicOr(err, 1);
        tc::mbar_wait(&bar, sy.phase ^ 1, kWait);  // the MMAs of the last commit, bounded
    }
    if (ok && t == 0) {
        double s = 0.0;
        for (int q = 0; q < kT; q++) s += lsum[q];
        out[kP64] = s;
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((t >> 5) == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kCols);
    }
}

}  // namespace

int mlp64_params() { return kP64; }

// Launchers (one CTA per SM, persistent over the tiles): y[n] of the network,
// and the per-CTA gradient partials [grid][kP64 + 1].  err: device int.
void mlp64_forward(const uint16_t* feat, int64_t n, const double* master, float* y, int* err, int sms, cudaStream_t s)
{
    static bool set[64] = {};
    int dev = 0;
    TAGI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !set[dev]) {
        TAGI_CUDA(cudaFuncSetAttribute(k_mlp64_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAlloc));
        if (dev >= 0 && dev < 64) set[dev] = true;
    }
    const int64_t tiles = (n + kT - 1) / kT;
    const int grid = (int)(tiles < sms ? tiles : sms);
    launch(k_mlp64_fwd, grid, kThreads, kSmemAlloc, s, feat, n, master, y, err);
    TAGI_LAUNCH_CHECK();
}

int mlp64_grad_grid(int64_t n, int sms)
{
    // one CTA per SM; the float32 tensor-memory sums span at most kFold
    // tiles before they are added to the CTA's float64 row
    const int64_t tiles = (n + kT - 1) / kT;
    return (int)(tiles < sms ? tiles : sms);
}

void mlp64_gradient(const uint16_t* feat, const float* target, const float* wt, int64_t n, const double* master,
                    double* partial, int grid, int* err, cudaStream_t s)
{
    static bool set[64] = {};
    int dev = 0;
    TAGI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !set[dev]) {
        TAGI_CUDA(cudaFuncSetAttribute(k_mlp64_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAlloc));
        if (dev >= 0 && dev < 64) set[dev] = true;
    }
    launch(k_mlp64_grad, grid, kThreads, kSmemAlloc, s, feat, target, wt, n, master, partial, err);
    TAGI_LAUNCH_CHECK();
}

}  // namespace tagi
