// Anterpolation: proxy weights of Eq. particle-cluster-approx-rearranged,
//   qh_k = sum_{j in C} L_k1(x_j) L_k2(y_j) L_k3(z_j) q_j,
// with the barycentric basis of Eq. Lagrange_polynomials and the weights of
// Eq. barycentric_weights on Chebyshev points of the second kind mapped to the
// cluster box (Section 5.2).
//
// Two kernels, both over work items (a chunk of at most kAntChunk points of
// one cluster), with chunk partials summed in a fixed order afterwards, so
// results are reproducible run to run:
//   k_ant (SIMT): each thread owns up to four proxies; the points stream
//     through shared memory 64 at a time with their 3 (n+1) basis values, so a
//     proxy weight costs 2 multiplies plus one FMA per charge column per point.
//     Float64 (the plain form) and the float32 anterpolation of the quadrature
//     weights w^, whose rounding the singularity subtraction amplifies.
//   k_ant_tc (tensor cores, the fields of the FP32C form): the contraction
//     over points is split along the tensor-product basis,
//       qh[(k1,k2), (k3,c)] = sum_j A[(k1,k2), j] B[(k3,c), j],
//       A = L_k1(x_j) L_k2(y_j),  B = L_k3(z_j) q_c(j),
//     a (n+1)^2 x N_S by N_S x (n+1) C product (M = 128 rows, N <= 80
//     columns) issued as tcgen05.mma kind::tf32 with three-term split
//     precision (3xTF32: A_hi B_hi + A_hi B_lo + A_lo B_hi, each operand split
//     into a tf32 value and its tf32 remainder), accumulated in tensor memory
//     and folded into two-float registers every kTcFold point tiles.  Forming
//     the operands costs (n+1)^2 + (n+1) C products per point instead of the
//     (n+1)^3 (2 + C) operations of the SIMT kernel.
#include <cuda_runtime.h>

#include "tagi_internal.cuh"
#include "tc.cuh"

namespace tagi {

namespace {

constexpr int kAntThreads = 256;
constexpr int kAntTile = 64;
constexpr int kMaxPPT = 4;  // proxies per thread: (9+1)^3 = 1000 <= 4 * 256

// Lagrange basis at t in [-1, 1] on the nodes cos(pi k / n) (Eq. Lagrange_polynomials).
// Division-free (first barycentric form):
//   L_k(t) = prod_{j != k} (t - s_j) * inv_k,  inv_k = 1 / prod_{j != k} (s_k - s_j),
// with prefix and suffix products; exact zeros at the other nodes.  float64
// divisions are slow on this GPU, and this form needs none per point.
__device__ __forceinline__ void basis_prod(double t, bool degenerate, int n, const double* s, const double* inv,
                                           double* L)
{
    if (degenerate) {
        for (int k = 0; k <= n; k++) L[k] = k == 0 ? 1.0 : 0.0;
        return;
    }
    double pre = 1.0;
    for (int k = 0; k <= n; k++) {
        L[k] = pre;
        pre *= t - s[k];
    }
    double suf = 1.0;
    for (int k = n; k >= 0; k--) {
        L[k] *= suf * inv[k];
        suf *= t - s[k];
    }
}

// Double-float arithmetic for the basis cache: a value is an unevaluated
// sum h + l of two float32 with |l| <= ulp(h) / 2 (about 48 significant
// bits).  The error-free sum is Knuth's TwoSum, the product uses the FMA for
// the exact error of h * h; every step is an explicit round-to-nearest
// intrinsic so that no contraction changes it.
struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 two_sum_f(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return F2{s, e};
}

__device__ __forceinline__ F2 df_mul(F2 a, F2 b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);  // exact: a.h * b.h = p + e
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return two_sum_f(p, e);
}

// (t - s) for a double-float t and a float32 node s
__device__ __forceinline__ F2 df_sub(F2 t, float s)
{
    const F2 d = two_sum_f(t.h, -s);
    return two_sum_f(d.h, __fadd_rn(d.l, t.l));
}

__device__ __forceinline__ F2 df_of(double x)
{
    const float h = (float)x;
    return F2{h, (float)(x - (double)h)};
}

// basis_prod in double-float arithmetic: the same products, with t given as
// a double-float and the nodes s exact in float32; L[k] is the float32
// rounding of the result.  float64 runs at about 1/70 of the float32 rate on
// this GPU; this form costs about a twelfth of the float64 one.
template <int N>
__device__ __forceinline__ void basis_df_n(F2 t, const float* s, const F2* inv, float* L)
{
    F2 d[N + 1], P[N + 1];
    F2 pre{1.0f, 0.0f};
#pragma unroll
    for (int k = 0; k <= N; k++) {
        d[k] = df_sub(t, s[k]);
        P[k] = pre;
        pre = df_mul(pre, d[k]);
    }
    F2 suf{1.0f, 0.0f};
#pragma unroll
    for (int k = N; k >= 0; k--) {
        const F2 v = df_mul(P[k], df_mul(suf, inv[k]));
        L[k] = __fadd_rn(v.h, v.l);
        suf = df_mul(suf, d[k]);
    }
}

__device__ __forceinline__ void basis_df(F2 t, bool degenerate, int n, const float* s, const F2* inv,
                                         float (&L)[kMaxDegree + 1])
{
    if (degenerate) {
#pragma unroll
        for (int k = 0; k <= kMaxDegree; k++) L[k] = k == 0 ? 1.0f : 0.0f;
        return;
    }
    switch (n) {  // unrolled per degree, so the products stay in registers
        case 1: basis_df_n<1>(t, s, inv, L); break;
        case 2: basis_df_n<2>(t, s, inv, L); break;
        case 3: basis_df_n<3>(t, s, inv, L); break;
        case 4: basis_df_n<4>(t, s, inv, L); break;
        case 5: basis_df_n<5>(t, s, inv, L); break;
        case 6: basis_df_n<6>(t, s, inv, L); break;
        case 7: basis_df_n<7>(t, s, inv, L); break;
        case 8: basis_df_n<8>(t, s, inv, L); break;
        default: basis_df_n<kMaxDegree>(t, s, inv, L); break;
    }
}

constexpr int kAntLP = 12;  // padded basis row of the cache (degree <= 11)
static_assert(kMaxDegree + 1 <= kAntLP, "basis row fits");

constexpr int kTcK = 32;                             // points per tensor-core tile
constexpr int kTilesPerItem = kAntChunk / kTcK;      // 64
constexpr int kTileFloats = 3 * kAntLP * kTcK;       // basis floats of one tile (4608 bytes)
static_assert(kAntChunk % kTcK == 0, "whole tiles per item");

// index of basis value k of dimension d of point j (0 <= j < kAntChunk) of
// item `item` in the basis cache: tiles of 32 points, each [3][kAntLP][32]
__host__ __device__ inline size_t antl_index(size_t item, int j, int d, int k)
{
    return ((item * kTilesPerItem + (j >> 5)) * 3 + d) * (size_t)(kAntLP * kTcK) + k * kTcK + (j & 31);
}

// Basis cache of the float32 path: for every point of every anterpolation
// item and each dimension, the basis of Eq. Lagrange_polynomials on the
// float32-rounded nodes at the float64 scaled coordinate, evaluated in
// double-float arithmetic (basis_df) and rounded to float32 (the float32
// rounding of the float64 basis except where a value lies within about
// 1e-13 of a rounding boundary), in the tile layout of antl_index; the
// points of the last tile beyond the item's end hold zeros.
__global__ void __launch_bounds__(kAntThreads) k_ant_basis(const AntItem* __restrict__ items,
                                                           const double* __restrict__ px,
                                                           const double* __restrict__ py,
                                                           const double* __restrict__ pz,
                                                           const double* __restrict__ lo,
                                                           const double* __restrict__ hi, int degree,
                                                           float* __restrict__ antL)
{
    __shared__ double dnodes[kMaxDegree + 1], inv[kMaxDegree + 1];
    __shared__ float fnodes[kMaxDegree + 1];
    __shared__ F2 finv[kMaxDegree + 1];
    const AntItem it = items[blockIdx.x];
    const int c = it.cluster;
    double cc[3], hh[3], ih[3];
    for (int d = 0; d < 3; d++) {
        cc[d] = (lo[3 * c + d] + hi[3 * c + d]) * 0.5;
        hh[d] = (hi[3 * c + d] - lo[3 * c + d]) * 0.5;
        ih[d] = hh[d] == 0.0 ? 0.0 : 1.0 / hh[d];
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k <= degree; k++) dnodes[k] = (double)(float)cos(M_PI * k / degree);
        for (int k = 0; k <= degree; k++) {
            double d = 1.0;
            for (int j = 0; j <= degree; j++)
                if (j != k) d *= dnodes[k] - dnodes[j];
            inv[k] = 1.0 / d;
            fnodes[k] = (float)dnodes[k];
            finv[k] = df_of(inv[k]);
        }
    }
    __syncthreads();
    const int np = it.p1 - it.p0;
    const int ntile = (np + kTcK - 1) / kTcK;
    // thread e: point j = 32 * tile + (e % 32) of dimension d, so a warp
    // writes 32 consecutive floats per basis index
    for (int e = threadIdx.x; e < ntile * 3 * kTcK; e += blockDim.x) {
        const int jj = e & 31, rest = e >> 5, d = rest % 3, j = (rest / 3) * kTcK + jj;
        const double* x = d == 0 ? px : (d == 1 ? py : pz);
        // (select, not index: a runtime index would put the arrays in local memory)
        const double ccd = d == 0 ? cc[0] : (d == 1 ? cc[1] : cc[2]);
        const double hhd = d == 0 ? hh[0] : (d == 1 ? hh[1] : hh[2]);
        const double ihd = d == 0 ? ih[0] : (d == 1 ? ih[1] : ih[2]);
        const bool deg = hhd == 0.0;
        float Lf[kMaxDegree + 1];
        if (j < np) basis_df(df_of(deg ? 0.0 : (x[it.p0 + j] - ccd) * ihd), deg, degree, fnodes, finv, Lf);
#pragma unroll
        for (int k = 0; k < kAntLP; k++)
            antL[antl_index(blockIdx.x, j, d, k)] = (j < np && k <= degree && k <= kMaxDegree) ? Lf[k] : 0.0f;
    }
}

// R: arithmetic type of the basis and per-tile sums; A: accumulator type.
// antL: the basis rows of every point of every item (k_ant_basis), or null
// to evaluate them here.
template <class R, class A, int NQ>
__global__ void __launch_bounds__(kAntThreads) k_ant(const AntItem* __restrict__ items, const double* __restrict__ px,
                                                     const double* __restrict__ py, const double* __restrict__ pz,
                                                     const double* __restrict__ lo, const double* __restrict__ hi,
                                                     int degree, int f32nodes, const R* __restrict__ q,
                                                     int64_t ldq, double* __restrict__ part,
                                                     const float* __restrict__ antL)
{
    __shared__ R Ls[kAntTile][3][kMaxDegree + 1];
    __shared__ R qs[NQ][kAntTile];
    __shared__ R nodes[kMaxDegree + 1];
    const AntItem it = items[blockIdx.x];
    const int m = degree + 1, P = m * m * m;
    const int c = it.cluster;
    double cc[3], hh[3], ih[3];
    for (int d = 0; d < 3; d++) {
        cc[d] = (lo[3 * c + d] + hi[3 * c + d]) * 0.5;
        hh[d] = (hi[3 * c + d] - lo[3 * c + d]) * 0.5;
        ih[d] = hh[d] == 0.0 ? 0.0 : 1.0 / hh[d];
    }
    __shared__ double dnodes[kMaxDegree + 1], inv[kMaxDegree + 1];
    if (threadIdx.x == 0) {
        // FP32C proxies sit on the float32-rounded nodes; interpolate there
        for (int k = 0; k <= degree; k++) {
            const double sk = cos(M_PI * k / degree);
            nodes[k] = f32nodes ? (R)(float)sk : (R)sk;
            dnodes[k] = (double)nodes[k];
        }
        for (int k = 0; k <= degree; k++) {
            double d = 1.0;
            for (int j = 0; j <= degree; j++)
                if (j != k) d *= dnodes[k] - dnodes[j];
            inv[k] = 1.0 / d;
        }
    }
    int k1[kMaxPPT], k2[kMaxPPT], k3[kMaxPPT];
    A acc[kMaxPPT][NQ];
#pragma unroll
    for (int i = 0; i < kMaxPPT; i++) {
        int k = threadIdx.x + i * kAntThreads;
        k1[i] = k < P ? k / (m * m) : 0;
        k2[i] = k < P ? (k / m) % m : 0;
        k3[i] = k < P ? k % m : 0;
#pragma unroll
        for (int j = 0; j < NQ; j++) acc[i][j] = 0;
    }
    for (int p0 = it.p0; p0 < it.p1; p0 += kAntTile) {
        const int nt = min(kAntTile, it.p1 - p0);
        __syncthreads();
        if (threadIdx.x < 3 * kAntTile) {
            int j = threadIdx.x / 3, d = threadIdx.x % 3;
            R L[kMaxDegree + 1];
            if (j < nt && antL) {
                for (int k = 0; k <= degree; k++) L[k] = (R)antL[antl_index(blockIdx.x, (p0 - it.p0) + j, d, k)];
            } else if (j < nt) {
                const double* x = d == 0 ? px : (d == 1 ? py : pz);
                bool deg = hh[d] == 0.0;
                // the basis on [-1, 1], evaluated in
                // float64 for both paths (a float32 evaluation is biased at
                // the 1e-8 level, which the singularity subtraction would
                // amplify); the float32 path interpolates on the float32
                // nodes, where its proxies sit
                double Ld[kMaxDegree + 1];
                const double td = deg ? 0.0 : (x[p0 + j] - cc[d]) * ih[d];
                basis_prod(td, deg, degree, dnodes, inv, Ld);
                for (int q = 0; q <= degree; q++) L[q] = (R)Ld[q];
            } else {
                for (int k = 0; k <= degree; k++) L[k] = R(0);
            }
            for (int k = 0; k <= degree; k++) Ls[j][d][k] = L[k];
        }
        for (int e = threadIdx.x; e < NQ * kAntTile; e += kAntThreads) {
            int col = e / kAntTile, j = e % kAntTile;
            qs[col][j] = j < nt ? q[col * ldq + p0 + j] : R(0);
        }
        __syncthreads();
        R tacc[kMaxPPT][NQ];
#pragma unroll
        for (int i = 0; i < kMaxPPT; i++)
#pragma unroll
            for (int j = 0; j < NQ; j++) tacc[i][j] = 0;
        for (int j = 0; j < nt; j++) {
#pragma unroll
            for (int i = 0; i < kMaxPPT; i++) {
                R L = Ls[j][0][k1[i]] * Ls[j][1][k2[i]] * Ls[j][2][k3[i]];
#pragma unroll
                for (int col = 0; col < NQ; col++) tacc[i][col] += L * qs[col][j];
            }
        }
#pragma unroll
        for (int i = 0; i < kMaxPPT; i++)
#pragma unroll
            for (int col = 0; col < NQ; col++) acc[i][col] += (A)tacc[i][col];
    }
    double* out = part + (size_t)blockIdx.x * NQ * P;
#pragma unroll
    for (int i = 0; i < kMaxPPT; i++) {
        int k = threadIdx.x + i * kAntThreads;
        if (k < P)
#pragma unroll
            for (int col = 0; col < NQ; col++) out[col * P + k] = (double)acc[i][col];
    }
}

// w^ of the FP32C tree from the two-float weight columns (w_hi, w_lo) and
// the basis cache, in proxy pencils: thread t < M^2 owns the M proxies
// (k1, k2, k3 = 0 .. M-1) with k1 = t / M, k2 = t % M.  L1 L2 is formed once
// per point and pencil and the k3 values are broadcast from shared memory,
// so a point costs 2 + M + 2 shared loads per pencil instead of 5 per proxy
// (k_ant is bound by its shared loads).  The products, (L1 L2) L3 times each
// column, and the summation order (float sums over 64-point tiles in point
// order, float64 across tiles) are those of k_ant, so w^ is bit-identical.
template <int M>
struct Pencil {
    static constexpr int threads = (M * M + 31) / 32 * 32;
};

template <int M>
__global__ void __launch_bounds__(Pencil<M>::threads) k_ant_pencil(const AntItem* __restrict__ items,
                                                                   const float* __restrict__ q, int64_t ldq,
                                                                   double* __restrict__ part,
                                                                   const float* __restrict__ antL)
{
    constexpr int P = M * M * M;
    __shared__ float Ls[kAntTile][3][M];
    __shared__ float qs[2][kAntTile];
    const AntItem it = items[blockIdx.x];
    const int t = threadIdx.x;
    const bool own = t < M * M;
    const int k1 = own ? t / M : 0, k2 = own ? t % M : 0;
    double acc[M][2];
#pragma unroll
    for (int k = 0; k < M; k++) acc[k][0] = acc[k][1] = 0.0;
    for (int p0 = it.p0; p0 < it.p1; p0 += kAntTile) {
        const int nt = min(kAntTile, it.p1 - p0);
        __syncthreads();
        for (int e = t; e < kAntTile * 3 * M; e += Pencil<M>::threads) {
            const int j = e / (3 * M), d = (e / M) % 3, k = e % M;
            Ls[j][d][k] = j < nt ? antL[antl_index(blockIdx.x, (p0 - it.p0) + j, d, k)] : 0.0f;
        }
        for (int e = t; e < 2 * kAntTile; e += Pencil<M>::threads) {
            const int col = e / kAntTile, j = e % kAntTile;
            qs[col][j] = j < nt ? q[col * ldq + p0 + j] : 0.0f;
        }
        __syncthreads();
        float tacc[M][2];
#pragma unroll
        for (int k = 0; k < M; k++) tacc[k][0] = tacc[k][1] = 0.0f;
        for (int j = 0; j < nt; j++) {
            const float l12 = Ls[j][0][k1] * Ls[j][1][k2];
            const float q0 = qs[0][j], q1 = qs[1][j];
#pragma unroll
            for (int k = 0; k < M; k++) {
                const float L = l12 * Ls[j][2][k];
                tacc[k][0] += L * q0;
                tacc[k][1] += L * q1;
            }
        }
#pragma unroll
        for (int k = 0; k < M; k++) {
            acc[k][0] += (double)tacc[k][0];
            acc[k][1] += (double)tacc[k][1];
        }
    }
    if (!own) return;
    double* out = part + (size_t)blockIdx.x * 2 * P;
#pragma unroll
    for (int k = 0; k < M; k++) {
        const int pk = (k1 * M + k2) * M + k;
        out[pk] = acc[k][0];
        out[P + pk] = acc[k][1];
    }
}

// ---------------------------------------------------------------- tensor cores
constexpr int kTcFormWarps = 8;                      // warps that form operands and fold
constexpr int kTcThreads = 32 * (kTcFormWarps + 1);  // + one warp that issues MMAs and bulk copies
constexpr int kTcFold = 1;             // tiles accumulated in tensor memory between two-float folds
constexpr int kTcSlots = 3;            // load slots: bulk copies run up to 2 tiles ahead
constexpr uint32_t kTcCols = 256;      // TMEM columns per CTA: two accumulators at columns 0 and 128
constexpr long long kTcWait = 2000000000LL;  // SM clocks before a wait gives up (about 1 s)
constexpr int kTcSmemFloor = 76 * 1024;      // dynamic shared memory asked per CTA, at least: three
                                             // CTAs never fit an SM's 228 KB, so at most two CTAs
                                             // (2 x 256 = 512 TMEM columns) share an SM

// Operand stage: A hi, A lo (ra rows each), B hi, B lo (npad rows each),
// 128-byte rows.  The MMA reads 128 rows of A; rows ra .. 127 fall on the
// next operand tiles or the basis tiles, all inside the CTA's shared memory,
// and only change accumulator lanes >= (n+1)^2, which are never read.
__host__ __device__ constexpr int tc_stage_bytes(int ra, int npad) { return 2 * ra * 128 + 2 * npad * 128; }
__host__ __device__ constexpr int tc_smem_bytes(int ra, int npad)
{
    // two operand stages, the load slots (basis tile and charges), 1024 alignment slack
    return 2 * tc_stage_bytes(ra, npad) + kTcSlots * (kTileFloats + 8 * kTcK) * 4 + 1024;
}

// nearest tf32 value, ties away from zero (as cvt.rna.tf32.f32): add half a
// tf32 unit in the last place to the magnitude bits and clear the 13 low bits
__device__ __forceinline__ float tf32_round(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// (hi, lo) += x with an error-free TwoSum of hi and x
__device__ __forceinline__ void fold2(float& hi, float& lo, float x)
{
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16) that completes its bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

// One CTA per item (at most 2048 points of one cluster): 8 warps form the
// operands and fold the accumulators, one more warp (its lane 0) issues the
// MMAs and the bulk copies.  The basis rows of the item's points (basis
// cache, tile layout) and its charges (charge tiles of k_qtiles, columns q0
// .. q0 + nq of nqt) arrive through bulk copies up to two tiles ahead.
// Per tile t of 32 points:
//   forming warps: wait for the tile's copies and for the MMAs of tile t - 2
//     (operand stage t % 2 free), write A (rows k1 (n+1) + k2 < (n+1)^2 of
//     128) and B (rows k3 nq + c < (n+1) nq of N = 2 NH) as tf32 hi/lo pairs
//     in 128B-swizzled K-major tiles (padding rows stay zero), and arrive on
//     the stage's full barrier;
//   issuing lane: waits for it (and, at the start of a fold group, for the
//     fold of the group two before it), issues 4 K-steps x 3 tf32 MMAs into
//     the accumulator of the tile's fold group (TMEM columns 0 or 128,
//     alternating per group), commits them to the stage's barrier, and
//     starts the copies of tile t + 3 into the load slot tile t used;
//   when tile t - 1 closed a group of kTcFold tiles, the forming warps wait
//     for its MMAs, read that accumulator (warp w: lanes 32 (w % 4) ..,
//     columns (w / 4) NH ..), fold it into float two-sums and release it.
// Every wait is bounded: one that gives up raises the CTA's abort flag, the
// others then stop at their next wait, the issuing lane waits (bounded) for
// its MMAs and copies in flight, *err is set and no output is written.
template <int NH>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_ant_tc(const float* __restrict__ antL, const float* __restrict__ qT, int nqt, int q0, int nq,
             const AntItem* __restrict__ items, int degree, double* __restrict__ part, int* __restrict__ err)
{
    constexpr int NPAD = 2 * NH;
    constexpr uint32_t idesc = tc::idesc_tf32(128, NPAD);
    constexpr int kSlot = kTileFloats + 8 * kTcK;  // basis tile [3][kAntLP][32] then charges [8][32]
    // accumulators per fold buffer (one per K-step while they fit the 128
    // columns of a buffer): each takes its K-steps' cross terms and then
    // their hi x hi products, so a large partial sum sees few float32
    // additions, which the tensor cores may round toward zero
    constexpr int NACC = NPAD <= 32 ? 4 : (NPAD <= 64 ? 2 : 1);
    constexpr int KPA = (kTcK / 8) / NACC;  // K-steps per accumulator
    const int ra = ((degree + 1) * (degree + 1) + 7) / 8 * 8;
    const int SB = tc_stage_bytes(ra, NPAD), SA = ra * 128;
    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    float* Lb = reinterpret_cast<float*>(sm + 2 * SB);
    // row table: factor offsets within a load slot (floats), byte offset of
    // the hi row in the stage, and the hi -> lo distance, for rows [0, mm) of
    // A and then rows [0, ncol) of B
    __shared__ int4 rowtab[128 + NPAD];
    __shared__ uint8_t ck3[NPAD], cq[NPAD];
    __shared__ uint64_t ld_full[kTcSlots], op_full[2], op_free[2], acc_free[2];
    __shared__ uint32_t tslot;
    __shared__ volatile int abort_flag;

    const AntItem it = items[blockIdx.x];
    const int m = degree + 1, mm = m * m, P = mm * m, ncol = m * nq;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (it.p1 - it.p0 + kTcK - 1) / kTcK;
    const int ngroups = (ntiles + kTcFold - 1) / kTcFold;
    const int nrows = mm + ncol;
    const uint32_t qbytes = (uint32_t)nq * kTcK * 4;

    for (int e = tid; e < 2 * SB / 16; e += kTcThreads) reinterpret_cast<uint4*>(sm)[e] = make_uint4(0, 0, 0, 0);
    for (int rho = tid; rho < nrows; rho += kTcThreads) {
        if (rho < mm) {
            const int k1 = rho / m, k2 = rho - k1 * m;
            rowtab[rho] = make_int4(k1 * kTcK, (kAntLP + k2) * kTcK, rho * 128, SA);
        } else {
            const int c = rho - mm, k3 = c / nq, col = c - k3 * nq;
            rowtab[rho] = make_int4((2 * kAntLP + k3) * kTcK, kTileFloats + col * kTcK, 2 * SA + c * 128, NPAD * 128);
        }
    }
    if (tid < NPAD) {
        ck3[tid] = tid < ncol ? tid / nq : 0;
        cq[tid] = tid < ncol ? tid % nq : 0;
    }
    if (warp == kTcFormWarps) tc::tmem_alloc(&tslot, kTcCols);
    if (tid == 0) {
        abort_flag = 0;
        for (int u = 0; u < kTcSlots; u++) tc::mbar_init(&ld_full[u], 1);
        for (int u = 0; u < 2; u++) {
            tc::mbar_init(&op_full[u], 32 * kTcFormWarps);
            tc::mbar_init(&op_free[u], 1);
            tc::mbar_init(&acc_free[u], 32 * kTcFormWarps);
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;

    // bounded waits: a wait that gives up raises the abort flag; once it is
    // up every later wait returns false at once
    auto wait1 = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (abort_flag) return false;
        if (tc::mbar_wait(bar, parity, kTcWait)) return true;
        abort_flag = 1;
        return false;
    };
    // the same, with one answer for the whole warp
    auto wait32 = [&](uint64_t* bar, uint32_t parity) -> bool {
        const bool r = __all_sync(0xffffffffu, !abort_flag && tc::mbar_wait(bar, parity, kTcWait));
        if (!r) abort_flag = 1;
        return r;
    };

    float ah[NH], al[NH];  // the forming warps' two-float accumulators
#pragma unroll
    for (int i = 0; i < NH; i++) ah[i] = al[i] = 0.0f;

    if (warp == kTcFormWarps) {
        // ------------------------------------------------ issuing warp
        if (lane == 0) {
            auto load_tile = [&](int t) {
                const int u = t % kTcSlots;
                const size_t tile = (size_t)blockIdx.x * kTilesPerItem + t;
                float* dst = Lb + u * kSlot;
                tc::fence_async_smem();
                mbar_expect_tx(&ld_full[u], (uint32_t)kTileFloats * 4 + qbytes);
                bulk_g2s(dst, antL + tile * kTileFloats, kTileFloats * 4, &ld_full[u]);
                bulk_g2s(dst + kTileFloats, qT + (tile * nqt + q0) * kTcK, qbytes, &ld_full[u]);
            };
            int loaded = -1, issued = -1;
            for (int t = 0; t < kTcSlots && t < ntiles; t++) load_tile(loaded = t);
            for (int t = 0; t < ntiles; t++) {
                const int s = t & 1, grp = t / kTcFold;
                if (!wait1(&op_full[s], (t >> 1) & 1)) break;
                if (t % kTcFold == 0 && grp >= 2 && !wait1(&acc_free[grp & 1], ((grp - 2) >> 1) & 1)) break;
                tc::fence_after_sync();
                const uint32_t b = tc::smem_u32(sm + s * SB);
                const uint64_t dah = tc::sdesc_sw128(b), dal = tc::sdesc_sw128(b + SA);
                const uint64_t dbh = tc::sdesc_sw128(b + 2 * SA), dbl = tc::sdesc_sw128(b + 2 * SA + NPAD * 128);
                const uint32_t first = (t % kTcFold) == 0;
#pragma unroll
                for (int a = 0; a < NACC; a++) {
                    const uint32_t acc = tmem + (uint32_t)((grp & 1) * 128 + a * NPAD);
                    // the small cross terms first, then the hi x hi products
#pragma unroll
                    for (int j = 0; j < KPA; j++) {
                        const int ks = a * KPA + j;
                        tc::mma_tf32(acc, dah + 2 * ks, dbl + 2 * ks, idesc, !(first && j == 0));
                        tc::mma_tf32(acc, dal + 2 * ks, dbh + 2 * ks, idesc, 1);
                    }
#pragma unroll
                    for (int j = 0; j < KPA; j++) {
                        const int ks = a * KPA + j;
                        tc::mma_tf32(acc, dah + 2 * ks, dbh + 2 * ks, idesc, 1);
                    }
                }
                tc::commit(&op_free[s]);
                issued = t;
                // the forming warps are done with tile t's load slot
                if (t + kTcSlots < ntiles) load_tile(loaded = t + kTcSlots);
            }
            if (abort_flag) {
                // nothing may still write this CTA's shared or tensor memory when it exits
                if (issued >= 0) tc::mbar_wait(&op_free[issued & 1], (issued >> 1) & 1, kTcWait);
                for (int u = loaded; u > issued && u >= 0; u--)
                    tc::mbar_wait(&ld_full[u % kTcSlots], (u / kTcSlots) & 1, kTcWait);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ forming warps
        // rows a warp forms are all congruent to it mod 8, so the 128B swizzle
        // of this thread's point is one constant for its A rows, one for its B rows
        const uint32_t swzA = ((((uint32_t)lane >> 2) ^ (uint32_t)warp) << 4) | (((uint32_t)lane & 3) << 2);
        const uint32_t swzB =
            ((((uint32_t)lane >> 2) ^ ((uint32_t)(warp - mm) & 7)) << 4) | (((uint32_t)lane & 3) << 2);
        auto fold_group = [&](int g) -> bool {
            const int tl = min(g * kTcFold + kTcFold - 1, ntiles - 1);
            if (!wait32(&op_free[tl & 1], (tl >> 1) & 1)) return false;
            tc::fence_after_sync();
            const uint32_t base =
                tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((g & 1) * 128 + (warp >> 2) * NH);
#pragma unroll
            for (int c8 = 0; c8 < NH; c8 += 8) {
                float v[8], x[8];
                tc::tmem_ld8(base + c8, v);
#pragma unroll
                for (int a = 1; a < NACC; a++) {
                    tc::tmem_ld8(base + a * NPAD + c8, x);
#pragma unroll
                    for (int i = 0; i < 8; i++) v[i] = __fadd_rn(v[i], x[i]);
                }
#pragma unroll
                for (int i = 0; i < 8; i++) fold2(ah[c8 + i], al[c8 + i], v[i]);
            }
            tc::fence_before_sync();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&acc_free[g & 1])) : "memory");
            return true;
        };
        bool ok = true;
        for (int t = 0; t < ntiles && ok; t++) {
            const int s = t & 1, u = t % kTcSlots;
            if (!wait32(&ld_full[u], (t / kTcSlots) & 1)) break;
            if (t >= 2 && !wait32(&op_free[s], ((t >> 1) + 1) & 1)) break;
            const float* S = Lb + u * kSlot;
            uint8_t* st = sm + s * SB;
            // four rows at a time, every load before any store, so that the
            // four chains overlap
            for (int r0 = warp; r0 < nrows; r0 += 4 * kTcFormWarps) {
                int4 R[4];
                float a[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int rho = r0 + q * kTcFormWarps;
                    R[q] = rowtab[rho < nrows ? rho : 0];
                }
#pragma unroll
                for (int q = 0; q < 4; q++) a[q] = S[R[q].x + lane] * S[R[q].y + lane];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int rho = r0 + q * kTcFormWarps;
                    if (rho < nrows) {
                        const float h = tf32_round(a[q]), l = tf32_round(a[q] - h);
                        const uint32_t o = R[q].z + (rho < mm ? swzA : swzB);
                        *reinterpret_cast<float*>(st + o) = h;
                        *reinterpret_cast<float*>(st + o + R[q].w) = l;
                    }
                }
            }
            tc::fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&op_full[s])) : "memory");
            if (t >= 1 && ((t - 1) % kTcFold) == kTcFold - 1) ok = fold_group((t - 1) / kTcFold);
        }
        // the group holding the last tile is not folded yet
        if (ok && ntiles > 0) fold_group(ngroups - 1);
    }
    __syncthreads();
    if (abort_flag) {
        if (tid == 0) atomicOr(err, 1);
    } else if (warp < kTcFormWarps) {
        const int r = (warp & 3) * 32 + lane;
        if (r < mm) {
            double* out = part + (size_t)blockIdx.x * nq * P;
#pragma unroll
            for (int i = 0; i < NH; i++) {
                const int c = (warp >> 2) * NH + i;
                if (c < ncol) out[(size_t)cq[c] * P + r * m + ck3[c]] = (double)ah[i] + (double)al[i];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kTcFormWarps) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTcCols);
    }
}

// Charge tiles of the tensor-core anterpolation: qT[(item * 64 + tile) * nf +
// col][32] = q[col][p0 + 32 tile + j] (zero beyond the item's end).
__global__ void k_qtiles(const AntItem* __restrict__ items, int64_t nitems, const float* __restrict__ q, int nf,
                         int64_t ldq, float* __restrict__ qT)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nitems * kAntChunk * nf) return;
    const int jj = (int)(e & 31);
    const int64_t rest = e >> 5;
    const int col = (int)(rest % nf);
    const int64_t tile = rest / nf;
    const int64_t item = tile / kTilesPerItem;
    const AntItem it = items[item];
    const int j = (int)(tile % kTilesPerItem) * kTcK + jj;
    qT[e] = it.p0 + j < it.p1 ? q[col * ldq + it.p0 + j] : 0.0f;
}

// Sum the partials of every item of far cluster f (fixed order) and store.
// mode 0: float rows dst32[(col0+col) * ldd + n + f P + k];
// mode 1: double rows dst64[...].
__global__ void k_ant_reduce(int nfar, const int* far_ant0, const double* part, int nq, int P, int64_t n,
                             int mode, float* dst32, double* dst64, int col0, int64_t ldd)
{
    const int f = blockIdx.x;
    const int a0 = far_ant0[f], a1 = far_ant0[f + 1];
    for (int e = threadIdx.x; e < nq * P; e += blockDim.x) {
        int col = e / P, k = e % P;
        double s = 0.0;
        for (int a = a0; a < a1; a++) s += part[((size_t)a * nq + col) * P + k];
        int64_t r = n + (int64_t)f * P + k;
        if (mode == 0)
            dst32[(col0 + col) * ldd + r] = (float)s;
        else
            dst64[(col0 + col) * ldd + r] = s;
    }
}

// w^ of far cluster f from the two columns (w_hi, w_lo) of a two-float weight:
// rec4[n + f P + k].w = sum over items and both columns.
__global__ void k_ant_reduce_w(const int* far_ant0, const double* part, int P, int64_t n, float4* rec4)
{
    const int f = blockIdx.x;
    const int a0 = far_ant0[f], a1 = far_ant0[f + 1];
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double s = 0.0;
        for (int a = a0; a < a1; a++) s += part[((size_t)a * 2 + 0) * P + k] + part[((size_t)a * 2 + 1) * P + k];
        rec4[n + (int64_t)f * P + k].w = (float)s;
    }
}

__global__ void k_split_w(const double* w, int64_t n, float* out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = (float)w[i];
    out[i] = h;
    out[n + i] = (float)(w[i] - (double)h);
}


template <class R, class A>
void launch_ant(int nq, int nitems, const AntItem* items, Tree& T, const R* q, int64_t ldq, double* part,
                cudaStream_t s, const float* antL = nullptr)
{
#define TAGI_ANT_CASE(NQ)                                                                                   \
    case NQ:                                                                                                \
        launch(k_ant<R, A, NQ>, nitems, kAntThreads, 0, s, items, T.px.as<double>(), T.py.as<double>(),         \
                                                       T.pz.as<double>(), T.cl_lo.as<double>(),             \
                                                       T.cl_hi.as<double>(), T.degree, T.prec == TAGI_FP32C, q, ldq, part, antL); \
        break;
    switch (nq) {
        TAGI_ANT_CASE(1)
        TAGI_ANT_CASE(2)
        TAGI_ANT_CASE(3)
        TAGI_ANT_CASE(4)
        TAGI_ANT_CASE(5)
        TAGI_ANT_CASE(6)
        TAGI_ANT_CASE(7)
        TAGI_ANT_CASE(8)
        default:
            throw Error(TAGI_ERR_INVALID_ARG, "anterpolation column group larger than 8");
    }
#undef TAGI_ANT_CASE
    TAGI_LAUNCH_CHECK();
}


template <int NH>
void launch_ant_tc_nh(int nq, int nitems, const AntItem* items, int degree, const float* antL, const float* qT,
                      int nqt, int q0, double* part, int* err, cudaStream_t s)
{
    const int ra = ((degree + 1) * (degree + 1) + 7) / 8 * 8;
    const int need = tc_smem_bytes(ra, 2 * NH);
    const int smem = need > kTcSmemFloor ? need : kTcSmemFloor;
    constexpr int kMaxSmem = tc_smem_bytes(104, 2 * NH) > kTcSmemFloor ? tc_smem_bytes(104, 2 * NH) : kTcSmemFloor;
    static bool attr_set[64] = {};
    int dev = 0;
    TAGI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        TAGI_CUDA(cudaFuncSetAttribute(k_ant_tc<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    launch(k_ant_tc<NH>, nitems, kTcThreads, smem, s, antL, qT, nqt, q0, nq, items, degree, part, err);
    TAGI_LAUNCH_CHECK();
}

// Tensor-core anterpolation (the FP32C form) of nq <= 8 charge columns
// [q0, q0 + nq) of the charge tiles qT (nqt columns, k_qtiles) with the basis
// cache antL of the same items: part[item][col][P] in float64.  err: device
// int, set to nonzero if a bounded wait of the kernel gave up.
void launch_ant_tc(int nq, int nitems, const AntItem* items, int degree, const float* antL, const float* qT, int nqt,
                   int q0, double* part, int* err, cudaStream_t s)
{
    TAGI_REQUIRE(nq >= 1 && nq <= 8, "anterpolation column group must hold 1..8 columns");
    const int npad = ((degree + 1) * nq + 15) / 16 * 16;
    switch (npad / 2) {
        case 8: launch_ant_tc_nh<8>(nq, nitems, items, degree, antL, qT, nqt, q0, part, err, s); break;
        case 16: launch_ant_tc_nh<16>(nq, nitems, items, degree, antL, qT, nqt, q0, part, err, s); break;
        case 24: launch_ant_tc_nh<24>(nq, nitems, items, degree, antL, qT, nqt, q0, part, err, s); break;
        case 32: launch_ant_tc_nh<32>(nq, nitems, items, degree, antL, qT, nqt, q0, part, err, s); break;
        case 40: launch_ant_tc_nh<40>(nq, nitems, items, degree, antL, qT, nqt, q0, part, err, s); break;
        default: throw Error(TAGI_ERR_INVALID_ARG, "tensor-core anterpolation: (degree+1) * columns exceeds 80");
    }
}

void fill_basis_cache(Tree& T, int nitems, const AntItem* items, DevBuf& cache)
{
    cache.ensure(sizeof(float) * (size_t)nitems * kTilesPerItem * kTileFloats);
    launch(k_ant_basis, nitems, kAntThreads, 0, T.stream, items, T.px.as<double>(), T.py.as<double>(),
           T.pz.as<double>(), T.cl_lo.as<double>(), T.cl_hi.as<double>(), T.degree, cache.as<float>());
    TAGI_LAUNCH_CHECK();
}

void fill_charge_tiles(Tree& T, int64_t nitems, const AntItem* items, const float* q, int nf, int64_t ldq,
                       DevBuf& qT)
{
    const int64_t total = nitems * kAntChunk * nf;
    qT.ensure(sizeof(float) * (size_t)total);
    launch(k_qtiles, (int)((total + 255) / 256), 256, 0, T.stream, items, nitems, q, nf, ldq, qT.as<float>());
    TAGI_LAUNCH_CHECK();
}

}  // namespace

void anterpolate_weights(Tree& T)
{
    if (T.nfar == 0) return;
    cudaStream_t s = T.stream;
    if (T.prec == TAGI_FP32C) {
        // basis cache (kept with the tree while it fits the budget below)
        fill_basis_cache(T, (int)T.nant, T.ant_items.as<AntItem>(), T.antL);
        const float* antL = T.antL.p ? T.antL.as<float>() : nullptr;
        // w^ from the two-float weights (w_hi, w_lo), on the float32 nodes
        // where the proxies sit
        T.antpart.ensure(sizeof(double) * (size_t)T.nant * T.P * 2);
        DevBuf w2;
        w2.ensure(sizeof(float) * 2 * (size_t)T.n);
        launch(k_split_w, (int)((T.n + 255) / 256), 256, 0, s, T.pw.as<double>(), T.n, w2.as<float>());
        if (antL && T.degree == 8)
            launch(k_ant_pencil<9>, (int)T.nant, Pencil<9>::threads, 0, s, T.ant_items.as<AntItem>(), w2.as<float>(),
                   T.n, T.antpart.as<double>(), antL);
        else if (antL && T.degree == 6)
            launch(k_ant_pencil<7>, (int)T.nant, Pencil<7>::threads, 0, s, T.ant_items.as<AntItem>(), w2.as<float>(),
                   T.n, T.antpart.as<double>(), antL);
        else
            launch_ant<float, double>(2, (int)T.nant, T.ant_items.as<AntItem>(), T, w2.as<float>(), T.n,
                                      T.antpart.as<double>(), s, antL);
        launch(k_ant_reduce_w, T.nfar, 256, 0, s, T.far_ant0.as<int>(), T.antpart.as<double>(), T.P, T.n,
               T.rec4.as<float4>());
        TAGI_LAUNCH_CHECK();
        TAGI_CUDA(cudaStreamSynchronize(s));
    } else {
        T.antpart.ensure(sizeof(double) * (size_t)T.nant * T.P);
        launch_ant<double, double>(1, (int)T.nant, T.ant_items.as<AntItem>(), T, T.pw.as<double>(), T.n,
                                   T.antpart.as<double>(), s);
        launch(k_ant_reduce, T.nfar, 256, 0, s, T.nfar, T.far_ant0.as<int>(), T.antpart.as<double>(), 1, T.P, T.n,
               1, nullptr, T.rw.as<double>(), 0, 0);
        TAGI_LAUNCH_CHECK();
    }
}

void anterpolate_fields32(Tree& T, int nf)
{
    if (T.nfar == 0) return;
    cudaStream_t s = T.stream;
    fill_charge_tiles(T, T.nant, T.ant_items.as<AntItem>(), T.qant.as<float>(), nf, T.n, T.qtiles);
    for (int g0 = 0; g0 < nf; g0 += 8) {
        int g = nf - g0 < 8 ? nf - g0 : 8;
        T.antpart.ensure(sizeof(double) * (size_t)T.nant * T.P * g);
        launch_ant_tc(g, (int)T.nant, T.ant_items.as<AntItem>(), T.degree, T.antL.as<float>(), T.qtiles.as<float>(),
                      nf, g0, T.antpart.as<double>(), T.errflag.as<int>() + 1, s);
        launch(k_ant_reduce, T.nfar, 256, 0, s, T.nfar, T.far_ant0.as<int>(), T.antpart.as<double>(), g, T.P, T.n, 0,
                                            T.fa.as<float>(), nullptr, g0, T.nrec);
        TAGI_LAUNCH_CHECK();
    }
}

void anterpolate_fields64(Tree& T, int nf)
{
    if (T.nfar == 0) return;
    cudaStream_t s = T.stream;
    for (int g0 = 0; g0 < nf; g0 += 8) {
        int g = nf - g0 < 8 ? nf - g0 : 8;
        T.antpart.ensure(sizeof(double) * (size_t)T.nant * T.P * g);
        launch_ant<double, double>(g, (int)T.nant, T.ant_items.as<AntItem>(), T, T.q64.as<double>() + g0 * T.nrec,
                                   T.nrec, T.antpart.as<double>(), s);
        launch(k_ant_reduce, T.nfar, 256, 0, s, T.nfar, T.far_ant0.as<int>(), T.antpart.as<double>(), g, T.P, T.n, 1,
                                            nullptr, T.q64.as<double>(), g0, T.nrec);
        TAGI_LAUNCH_CHECK();
    }
}

namespace {
__global__ void k_all_items(int nc, const int* begin, const int* end, const int64_t* off, AntItem* items)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int64_t o = off[c];
    for (int p = begin[c]; p < end[c]; p += kAntChunk) items[o++] = AntItem{p, min(end[c], p + kAntChunk), c, c};
}
__global__ void k_all_counts(int nc, const int* begin, const int* end, int64_t* cnt)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) cnt[c] = (end[c] - begin[c] + kAntChunk - 1) / kAntChunk;
}
__global__ void k_gather_rows(const double* q, int nq, int64_t n, const int* perm, double* out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nq) return;
    int64_t row = i / n, p = i % n;
    out[i] = q[row * n + perm[p]];
}
// qh[c][col][k] = sum over items of cluster c (items are grouped by cluster)
__global__ void k_all_reduce(const int64_t* off, const double* part, int nq, int P, int col0, int nqt, double* qh)
{
    const int c = blockIdx.x;
    for (int e = threadIdx.x; e < nq * P; e += blockDim.x) {
        int col = e / P, k = e % P;
        double s = 0.0;
        for (int64_t a = off[c]; a < off[c + 1]; a++) s += part[((size_t)a * nq + col) * P + k];
        qh[((size_t)c * nqt + col0 + col) * P + k] = s;
    }
}
}  // namespace

namespace {
__global__ void k_gather_rows32(const double* q, int nq, int64_t n, const int* perm, float* out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nq) return;
    int64_t row = i / n, p = i % n;
    out[i] = (float)q[row * n + perm[p]];
}
}  // namespace

// Every cluster's proxy weights by the FP32C form's anterpolation (charges
// rounded to float32, the float64-evaluated basis on the float32 nodes,
// 3xTF32 tensor-core products); partials folded in float64 per cluster.
void anterpolate_all_clusters32(Tree& T, const double* q, int nq, double* qh)
{
    cudaStream_t s = T.stream;
    const int nc = T.nc;
    DevBuf cnt, off, items, qt, part;
    cnt.ensure(8 * (size_t)nc);
    off.ensure(8 * ((size_t)nc + 1));
    launch(k_all_counts, (nc + 255) / 256, 256, 0, s, nc, T.cl_begin.as<int>(), T.cl_end.as<int>(), cnt.as<int64_t>());
    exclusive_scan_i64(cnt.as<int64_t>(), off.as<int64_t>(), nc, s);
    int64_t ni = 0;
    TAGI_CUDA(cudaMemcpyAsync(&ni, off.as<int64_t>() + nc, 8, cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaStreamSynchronize(s));
    items.ensure(sizeof(AntItem) * (size_t)ni);
    launch(k_all_items, (nc + 255) / 256, 256, 0, s, nc, T.cl_begin.as<int>(), T.cl_end.as<int>(), off.as<int64_t>(),
           items.as<AntItem>());
    qt.ensure(4 * (size_t)T.n * nq);
    launch(k_gather_rows32, (int)((T.n * nq + 255) / 256), 256, 0, s, q, nq, T.n, T.perm.as<int>(), qt.as<float>());
    TAGI_LAUNCH_CHECK();
    DevBuf basis, qtiles;
    fill_basis_cache(T, (int)ni, items.as<AntItem>(), basis);
    fill_charge_tiles(T, ni, items.as<AntItem>(), qt.as<float>(), nq, T.n, qtiles);
    for (int g0 = 0; g0 < nq; g0 += 8) {
        int g = nq - g0 < 8 ? nq - g0 : 8;
        part.ensure(sizeof(double) * (size_t)ni * T.P * g);
        launch_ant_tc(g, (int)ni, items.as<AntItem>(), T.degree, basis.as<float>(), qtiles.as<float>(), nq, g0,
                      part.as<double>(), T.errflag.as<int>() + 1, s);
        launch(k_all_reduce, nc, 256, 0, s, off.as<int64_t>(), part.as<double>(), g, T.P, g0, nq, qh);
        TAGI_LAUNCH_CHECK();
    }
    TAGI_CUDA(cudaStreamSynchronize(s));
}

void anterpolate_all_clusters64(Tree& T, const double* q, int nq, double* qh)
{
    cudaStream_t s = T.stream;
    const int nc = T.nc;
    DevBuf cnt, off, items, qt, part;
    cnt.ensure(8 * (size_t)nc);
    off.ensure(8 * ((size_t)nc + 1));
    launch(k_all_counts, (nc + 255) / 256, 256, 0, s, nc, T.cl_begin.as<int>(), T.cl_end.as<int>(), cnt.as<int64_t>());
    exclusive_scan_i64(cnt.as<int64_t>(), off.as<int64_t>(), nc, s);
    int64_t ni = 0;
    TAGI_CUDA(cudaMemcpyAsync(&ni, off.as<int64_t>() + nc, 8, cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaStreamSynchronize(s));
    items.ensure(sizeof(AntItem) * (size_t)ni);
    launch(k_all_items, (nc + 255) / 256, 256, 0, s, nc, T.cl_begin.as<int>(), T.cl_end.as<int>(), off.as<int64_t>(),
                                                 items.as<AntItem>());
    qt.ensure(8 * (size_t)T.n * nq);
    launch(k_gather_rows, (int)((T.n * nq + 255) / 256), 256, 0, s, q, nq, T.n, T.perm.as<int>(), qt.as<double>());
    TAGI_LAUNCH_CHECK();
    for (int g0 = 0; g0 < nq; g0 += 8) {
        int g = nq - g0 < 8 ? nq - g0 : 8;
        part.ensure(sizeof(double) * (size_t)ni * T.P * g);
        launch_ant<double, double>(g, (int)ni, items.as<AntItem>(), T, qt.as<double>() + (size_t)g0 * T.n, T.n,
                                   part.as<double>(), s);
        launch(k_all_reduce, nc, 256, 0, s, off.as<int64_t>(), part.as<double>(), g, T.P, g0, nq, qh);
        TAGI_LAUNCH_CHECK();
    }
    TAGI_CUDA(cudaStreamSynchronize(s));
}

}  // namespace tagi
