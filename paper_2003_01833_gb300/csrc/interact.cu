// Batch-cluster interactions: the near field (Eq. direct-sum_2, r = 0 skipped)
// and the far field (Eq. particle-cluster-approx-rearranged) in one kernel.
//
// Both have the same direct-sum structure, so the kernel sees only "source
// records": mesh points for direct entries and proxy points for approximated
// ones.  A record carries a position, a weight omega and one charge q per
// field: omega = w_j, q = f_j w_j for points; omega = w^_k, q = q^_k for
// proxies.  With the singularity subtraction of Section 3.3 (far-field form
// reading: two anterpolated charge sets) every field accumulates
//   Yukawa:   sum_s exp(-k r) / r * (q_s - c_i omega_s)
//   Coulomb:  sum_s (q_s - c_i omega_s exp(-r^2 / alpha^2)) / r
// where c_i = f(x_i); the constant terms c_i/k^2 and 2 pi alpha^2 c_i and the
// 1/(4 pi) of G_k are added by the epilogue.
//
// FP32C kernel: all fields of a call (each Yukawa field with its own k, plus
// the Hartree field) share one pass over the geometry.  Each thread holds a
// pair of targets, and the near field and the tensor-grid far field run on
// both with the packed f32x2 FMA/add/multiply (same rounding per lane as
// scalar code).  Each CTA owns up to 256 targets of one batch (128 threads x
// 2 targets) and a contiguous segment
// of the batch's interaction list; source tiles of 256 records are staged in
// shared memory with positions shifted from the record's frame (its leaf or
// cluster center) to the batch center in float64 and rounded once.  Near-field
// values and weights are two-float (see tile_near); proxies are single float.
// rsqrt and exp2 use the MUFU unit (rsqrt.approx, ex2.approx); their mean
// bias is measured once per device (fp32_bias) and compensated in the SS
// epilogue.  Quadrature weights of mesh points are two-float too: adaptive
// octree cells scale by powers of two, so a float32 rounding of w repeats the
// same few relative errors everywhere and would bias sum_j G w_j, which the
// singularity subtraction amplifies.  Every 16 sources (every row of proxies
// on the tensor far path) the float32 partial sums are folded into a
// per-target two-float (hi, lo) accumulator with an error-free TwoSum.  The SS constant c_i is the float32 high part of f_i, the same value
// the epilogue uses, so the subtraction telescopes exactly.
//
// Approximated clusters of degree 6 or 8 take the tensor-grid far path
// (tile_far_tensor): proxies sit on a product grid, so the squared distance
// costs one subtraction and one FMA per pair.  Entries whose boxes are at
// least sqrt(42) alpha apart (list flag bit2) leave out the Gaussian of the
// Coulomb SS, which is below 2^-60 there.
//
// FP64 kernel (plain form): one field per launch, float64 throughout,
// absolute coordinates, libm exp and sqrt.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "tagi_internal.cuh"

namespace tagi {

namespace {

constexpr int kTile = 256;
// targets per thread: 2 (one f32x2 pair), 128 threads per CTA.  Measured
// against 4 targets per thread (64 threads, 122-128 registers): more warps
// per SM hide the MUFU latency better than the extra reuse of staged values
// per thread buys.  The CTA always owns kTargetsPerItem targets.
template <int NF>
struct Tpt {
    static constexpr int value = 2;
    static constexpr int threads = kTargetsPerItem / value;
};
constexpr int kThreads64 = 256;
constexpr int kTile64 = 128;

static_assert(kThreads64 == kTargetsPerItem, "item size");

struct KParams {
    float ky[8];  // -k_o * log2(e) for the Yukawa fields
    float ga;     // -log2(e) / alpha^2 for the Hartree field
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Error-free transformation: s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Every kFold sources (record paths; every row of M proxies on the tensor
// far path), each target's float32 partial sums are folded into its
// two-float (hi, lo) accumulator by an error-free TwoSum.  Short folds keep
// the float32 summation error small against the large subtracted term
// c_i sum_j G w_j, which cancels against the analytic SS term.
constexpr int kFold = 16;
template <int NF, int TPT>
__device__ __forceinline__ void fold(float (&acc)[TPT][NF], float (&hi)[TPT][NF], float (&lo)[TPT][NF])
{
#pragma unroll
    for (int j = 0; j < TPT; j++)
#pragma unroll
        for (int o = 0; o < NF; o++) {
            float sum, er;
            two_sum(hi[j][o], acc[j][o], sum, er);
            hi[j][o] = sum;
            lo[j][o] += er;
        }
}

// Shared-memory layout of a staged tile: per source one float4 of position
// (relative to the batch center) and weight (high part), and the values
// packed four to a float4: components [0, NF) hold fh (points) or qh
// (proxies), components [NF, 2 NF) hold fl and component 2 NF the low part of
// the weight (points only).
template <int NF>
struct TileLayout {
    static constexpr int G = (2 * NF + 4) / 4;  // float4 groups of values per source
};

template <int NF>
__device__ __forceinline__ void load_values(const float4* __restrict__ sv, int k, float (&v)[4 * TileLayout<NF>::G])
{
    constexpr int G = TileLayout<NF>::G;
#pragma unroll
    for (int g = 0; g < G; g++) {
        const float4 t = sv[g * kTile + k];
        v[4 * g] = t.x;
        v[4 * g + 1] = t.y;
        v[4 * g + 2] = t.z;
        v[4 * g + 3] = t.w;
    }
}

// Targets live in pairs: target 2i is lane x and target 2i+1 lane y of pair i,
// with the coordinates stored negated (s - t is computed as s + (-t), the same
// IEEE result).  Scalar code reads one lane; j is a compile-time index once
// the target loops are unrolled.
__device__ __forceinline__ float lane(const float2& v, int j) { return (j & 1) ? v.y : v.x; }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Far field: proxies, single-float positions relative to the batch center;
//   Yukawa term  e^{-k r} / r * (qh - c w^),  Coulomb term (qh - c w^ e^{-r^2/a^2}) / r.
// GZ: the entry's Gaussian of the Coulomb SS is below float32 resolution for
// every pair (list flag bit2), so the Hartree term is q / r alone.
template <int NY, bool HH, bool SS, int TPT, bool GZ>
__device__ __forceinline__ void tile_far(const float4* __restrict__ srec, const float4* __restrict__ sv, int nk,
                                         const float2 (&ntx)[TPT / 2], const float2 (&nty)[TPT / 2],
                                         const float2 (&ntz)[TPT / 2], const float2 (&nc)[TPT / 2][NY + HH],
                                         float (&hi)[TPT][NY + HH], float (&lo)[TPT][NY + HH], const KParams& kp)
{
    constexpr int NF = NY + HH;
    constexpr int G = TileLayout<NF>::G;
    for (int k0 = 0; k0 < nk; k0 += kFold) {
        float acc[TPT][NF];
#pragma unroll
        for (int j = 0; j < TPT; j++)
#pragma unroll
            for (int o = 0; o < NF; o++) acc[j][o] = 0.0f;
#pragma unroll 2
        for (int k = k0; k < k0 + kFold; k++) {
            const float4 s = srec[k];
            float qv[4 * G];
            load_values<NF>(sv, k, qv);
#pragma unroll
            for (int j = 0; j < TPT; j++) {
                const float dx = s.x + lane(ntx[j >> 1], j), dy = s.y + lane(nty[j >> 1], j),
                            dz = s.z + lane(ntz[j >> 1], j);
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float ri = rsqrt_approx(r2);
                const float r = r2 * ri;
#pragma unroll
                for (int o = 0; o < NY; o++) {
                    const float e = ex2_approx(kp.ky[o] * r);
                    const float d = SS ? fmaf(lane(nc[j >> 1][o], j), s.w, qv[o]) : qv[o];
                    acc[j][o] = fmaf(e * ri, d, acc[j][o]);
                }
                if (HH) {
                    float d;
                    if (SS && !GZ) {
                        const float g = ex2_approx(kp.ga * r2);
                        d = fmaf(lane(nc[j >> 1][NY], j) * s.w, g, qv[NY]);
                    } else {
                        d = qv[NY];
                    }
                    acc[j][NY] = fmaf(ri, d, acc[j][NY]);
                }
            }
        }
        fold<NF, TPT>(acc, hi, lo);
    }
}

// Shared layout of a staged near-field tile: per source the float2 values
// x, y, z, w_hi, w_lo, fh[NF], fl[NF], each duplicated into both lanes, packed
// two to a float4.
template <int NF>
struct NearLayout {
    static constexpr int NV2 = 5 + 2 * NF;
    static constexpr int NV4 = (NV2 + 1) / 2;
};

// The fields' exponent factors duplicated into both lanes.
struct KParams2 {
    float2 ky[8];
    float2 ga;
};

// Fold of pair accumulators: lane x of pair i belongs to target 2i, lane y
// to target 2i+1.  The TwoSum of fold() on both lanes at once: each
// difference x - y is fma(y, -1, x), one rounding as in the scalar form, so
// the result is bit for bit that of two_sum.
template <int NF, int TPT>
__device__ __forceinline__ void fold2(float2 (&acc)[TPT / 2][NF], float (&hi)[TPT][NF], float (&lo)[TPT][NF])
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int i = 0; i < TPT / 2; i++)
#pragma unroll
        for (int o = 0; o < NF; o++) {
            const float2 a = make_float2(hi[2 * i][o], hi[2 * i + 1][o]);
            const float2 b = acc[i][o];
            const float2 s = add2(a, b);
            const float2 bp = fma2(a, m1, s);                        // s - a
            const float2 ap = fma2(bp, m1, s);                       // s - bp
            const float2 e = add2(fma2(ap, m1, a), fma2(bp, m1, b));  // (a - ap) + (b - bp)
            const float2 l = add2(make_float2(lo[2 * i][o], lo[2 * i + 1][o]), e);
            hi[2 * i][o] = s.x;
            hi[2 * i + 1][o] = s.y;
            lo[2 * i][o] = l.x;
            lo[2 * i + 1][o] = l.y;
        }
}

// Far field on the tensor grid of one cluster's proxies (M nodes per
// dimension): proxy (k1, k2, k3) sits at (X[k1], Y[k2], Z[k3]) relative to the
// batch center, each coordinate rounded once to float32 exactly as the record
// path rounds it, so r^2 = ((X - tx)^2 + (Y - ty)^2) + (Z - tz)^2 costs one
// subtraction and one FMA per pair once the (k1, k2) part is formed.  Two
// targets per instruction (f32x2, same rounding per lane as scalar code); the
// tile holds whole k1-planes, and per proxy the values q^ of the fields and w^
// (component NF) duplicated into both lanes, TensorLayout<NF>::GF2 float4
// each; sZ2 holds Z duplicated.  Every row of M proxies is folded into the
// two-float sums.
template <int NF>
struct TensorLayout {
    static constexpr int GF2 = (NF + 2) / 2;  // float4 per proxy: NF + 1 duplicated values
};

template <int NY, bool HH, bool SS, int TPT, int M, bool GZ>
__device__ __forceinline__ void tile_far_tensor(const float* __restrict__ sX, const float* __restrict__ sY,
                                                const float2* __restrict__ sZ2, const float4* __restrict__ st, int np,
                                                const float2 (&ntx)[TPT / 2], const float2 (&nty)[TPT / 2],
                                                const float2 (&ntz)[TPT / 2], const float2 (&nc)[TPT / 2][NY + HH],
                                                float (&hi)[TPT][NY + HH], float (&lo)[TPT][NY + HH],
                                                const KParams2& kp)
{
    constexpr int NF = NY + HH;
    constexpr int NP = TPT / 2;
    constexpr int GF2 = TensorLayout<NF>::GF2;
    for (int pl = 0; pl < np; pl++) {
        float2 dx2[NP];
        const float xk = sX[pl];
#pragma unroll
        for (int j = 0; j < NP; j++) {
            const float2 d = add2(make_float2(xk, xk), ntx[j]);
            dx2[j] = mul2(d, d);
        }
        for (int k2 = 0; k2 < M; k2++) {
            float2 a[NP];
            const float yk = sY[k2];
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const float2 d = add2(make_float2(yk, yk), nty[j]);
                a[j] = fma2(d, d, dx2[j]);
            }
            float2 acc[NP][NF];
#pragma unroll
            for (int j = 0; j < NP; j++)
#pragma unroll
                for (int o = 0; o < NF; o++) acc[j][o] = make_float2(0.0f, 0.0f);
            const float4* row = st + (pl * M + k2) * M;
#pragma unroll
            for (int k3 = 0; k3 < M; k3++) {
                float2 q[2 * GF2];  // q^ of the fields, then w^ at NF
#pragma unroll
                for (int g = 0; g < GF2; g++) {
                    const float4 t = row[g * kTile + k3];
                    q[2 * g] = make_float2(t.x, t.y);
                    q[2 * g + 1] = make_float2(t.z, t.w);
                }
                const float2 w = q[NF];
                const float2 z = sZ2[k3];
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const float2 dz = add2(z, ntz[j]);
                    const float2 r2 = fma2(dz, dz, a[j]);
                    const float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                    const float2 r = mul2(r2, ri);
#pragma unroll
                    for (int o = 0; o < NY; o++) {
                        const float2 t = mul2(kp.ky[o], r);
                        const float2 e = make_float2(ex2_approx(t.x), ex2_approx(t.y));
                        const float2 d = SS ? fma2(nc[j][o], w, q[o]) : q[o];
                        acc[j][o] = fma2(mul2(e, ri), d, acc[j][o]);
                    }
                    if (HH) {
                        float2 d;
                        if (SS && !GZ) {
                            const float2 t = mul2(kp.ga, r2);
                            const float2 g = make_float2(ex2_approx(t.x), ex2_approx(t.y));
                            d = fma2(mul2(nc[j][NY], w), g, q[NY]);
                        } else {
                            d = q[NY];
                        }
                        acc[j][NY] = fma2(ri, d, acc[j][NY]);
                    }
                }
            }
            fold2<NF, TPT>(acc, hi, lo);
        }
    }
}

// Near field: mesh points with positions relative to the batch center and
// two-float field values f = fh + fl and weights w = wh + wl.  The SS
// difference (fh_j - c_i) + fl_j, with c_i = fh_i, is exact up to one rounding
// for close pairs (Sterbenz), where f_j - f_i cancels.
//   Yukawa term  e^{-k r} / r * w_j (f_j - c_i),
//   Coulomb term (rho_j - c_i e^{-r^2/a^2}) w_j / r.
// Two targets per instruction (f32x2), each lane rounding exactly as the
// scalar form would.
template <int NY, bool HH, bool SS, bool SELF, int TPT, bool GZ>
__device__ __forceinline__ void tile_near(const float4* __restrict__ sn, int nk, const float2 (&ntx)[TPT / 2],
                                          const float2 (&nty)[TPT / 2], const float2 (&ntz)[TPT / 2],
                                          const float2 (&nc)[TPT / 2][NY + HH], float (&hi)[TPT][NY + HH],
                                          float (&lo)[TPT][NY + HH], const KParams2& kp)
{
    constexpr int NF = NY + HH;
    constexpr int NP = TPT / 2;
    constexpr int NV4 = NearLayout<NF>::NV4;
    for (int k0 = 0; k0 < nk; k0 += kFold) {
        float2 acc[NP][NF];
#pragma unroll
        for (int j = 0; j < NP; j++)
#pragma unroll
            for (int o = 0; o < NF; o++) acc[j][o] = make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int k = k0; k < k0 + kFold; k++) {
            float2 v[2 * NV4];  // 0 x, 1 y, 2 z, 3 w_hi, 4 w_lo, 5 + o fh, 5 + NF + o fl
#pragma unroll
            for (int g = 0; g < NV4; g++) {
                const float4 t = sn[g * kTile + k];
                v[2 * g] = make_float2(t.x, t.y);
                v[2 * g + 1] = make_float2(t.z, t.w);
            }
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const float2 dx = add2(v[0], ntx[j]), dy = add2(v[1], nty[j]), dz = add2(v[2], ntz[j]);
                const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                if (SELF) {
                    ri.x = r2.x > 0.0f ? ri.x : 0.0f;
                    ri.y = r2.y > 0.0f ? ri.y : 0.0f;
                }
                const float2 r = mul2(r2, ri);
                const float2 riw = fma2(ri, v[4], mul2(ri, v[3]));  // ri (w_hi + w_lo)
#pragma unroll
                for (int o = 0; o < NY; o++) {
                    const float2 t = mul2(kp.ky[o], r);
                    const float2 e = make_float2(ex2_approx(t.x), ex2_approx(t.y));
                    const float2 d = SS ? add2(add2(v[5 + o], nc[j][o]), v[5 + NF + o]) : add2(v[5 + o], v[5 + NF + o]);
                    acc[j][o] = fma2(mul2(e, riw), d, acc[j][o]);
                }
                if (HH) {
                    float2 d;
                    if (SS && !GZ) {
                        const float2 t = mul2(kp.ga, r2);
                        const float2 g = make_float2(ex2_approx(t.x), ex2_approx(t.y));
                        d = add2(fma2(nc[j][NY], g, v[5 + NY]), v[5 + NF + NY]);
                    } else {
                        d = add2(v[5 + NY], v[5 + NF + NY]);
                    }
                    acc[j][NY] = fma2(riw, d, acc[j][NY]);
                }
            }
        }
        fold2<NF, TPT>(acc, hi, lo);
    }
}

// Per-chunk sum of the item partials, in the kernel that writes them.  Each
// CTA stores its partial rows, fences them and counts itself in; the CTA
// that completes its target chunk's count sums the chunk's rows in item order
// (the fixed order, so the result does not depend on which CTA finishes
// last), stores the sum, resets the counter for the next launch, and drops
// the partial rows' lines from L2 without writing them back: the rows are
// dead, so they never reach DRAM while they fit in L2 together with the
// in-flight chunks.  Rows of fields [field0, field0 + nf) of each item are
// contiguous (nf x 2 KB), so they are whole 128-byte lines.
__device__ __forceinline__ void discard_line(const void* p)
{
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

template <int THREADS>
__device__ __forceinline__ void chunk_sum(const Item& it, double* __restrict__ part, double* __restrict__ tsum,
                                          int* __restrict__ cnt, int nf_tot, int field0, int nf)
{
    __shared__ int s_last;
    __threadfence();  // this CTA's partial rows before its count
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(cnt + it.tchunk, 1) == it.ni - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();  // the other CTAs' rows after their counts
    for (int q = threadIdx.x; q < nf * kTargetsPerItem; q += THREADS) {
        const int o = field0 + q / kTargetsPerItem, slot = q % kTargetsPerItem;
        const double* src = part + (size_t)o * kTargetsPerItem + slot;
        double S = 0.0;
        for (int i = it.i0; i < it.i0 + it.ni; i++) S += __ldcg(src + (size_t)i * nf_tot * kTargetsPerItem);
        tsum[((size_t)it.tchunk * nf_tot + o) * kTargetsPerItem + slot] = S;
    }
    __syncthreads();  // every read of the rows has returned
    constexpr int kLineDoubles = 128 / sizeof(double);
    const int lines = nf * kTargetsPerItem / kLineDoubles;  // per item
    for (int q = threadIdx.x; q < it.ni * lines; q += THREADS) {
        const int i = it.i0 + q / lines, l = q % lines;
        discard_line(part + ((size_t)i * nf_tot + field0) * kTargetsPerItem + (size_t)l * kLineDoubles);
    }
    if (threadIdx.x == 0) cnt[it.tchunk] = 0;
}

// M > 0: approximated clusters use the tensor-grid far path (degree M - 1);
// M == 0: every entry goes through the record path.
template <int NY, bool HH, bool SS, int M>
__global__ void __launch_bounds__(Tpt<NY + HH>::threads) k_interact32(const Item* __restrict__ items,
                                                           const Entry* __restrict__ ents,
                                                           const double* __restrict__ cen,
                                                           const float4* __restrict__ rec4,
                                                           const float4* __restrict__ rec4lo,
                                                           const float* __restrict__ fa, int64_t lda,
                                                           const float* __restrict__ fb, int64_t ldb,
                                                           const float* __restrict__ kyd,
                                                           double* __restrict__ part, double* __restrict__ tsum,
                                                           int* __restrict__ cnt, int nf_tot, int field0)
{
    constexpr int NF = NY + HH;
    constexpr int G = TileLayout<NF>::G;
    constexpr int NV4 = NearLayout<NF>::NV4;
    constexpr int TPT = Tpt<NF>::value;
    constexpr int NP = TPT / 2;
    constexpr int THREADS = Tpt<NF>::threads;
    constexpr int SB = NV4 > 1 + G ? NV4 : 1 + G;  // float4 per staged source, largest layout
    static_assert(TensorLayout<NF>::GF2 <= SB, "tensor layout fits");
    // exponent factors of this launch's fields, from device memory so that a
    // captured graph picks up the current eigenvalues on every replay
    KParams kp{};
    KParams2 kp2{};
#pragma unroll
    for (int o = 0; o < NY; o++) {
        kp.ky[o] = kyd[o];
        kp2.ky[o] = make_float2(kp.ky[o], kp.ky[o]);
    }
    if (HH) {
        kp.ga = kyd[NY];
        kp2.ga = make_float2(kp.ga, kp.ga);
    }
    __shared__ float4 sbuf[SB * kTile];
    float4* const srec = sbuf;         // record path: positions and w
    float4* const sv = sbuf + kTile;   // record path: values
    float4* const sn = sbuf;           // near field: duplicated float2 values
    float4* const st = sbuf;           // tensor far path: (q^, w^)

    const Item it = items[blockIdx.x];
    const int tid = threadIdx.x;
    float2 ntx[NP], nty[NP], ntz[NP];
    float2 nc[NP][NF];
    float hi[TPT][NF], lo[TPT][NF];
#pragma unroll
    for (int j = 0; j < TPT; j++) {
        const int p = it.t0 + tid + j * THREADS;
        const bool ok = p < it.t1;
        const float4 r = ok ? rec4[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 rl = ok ? rec4lo[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        // rounded exactly as a staged source of the batch's own leaf, so the
        // self pair gives r = 0 bit for bit
        const float x = -(float)(((double)r.x + (double)rl.x) + 0.0);
        const float y = -(float)(((double)r.y + (double)rl.y) + 0.0);
        const float z = -(float)(((double)r.z + (double)rl.z) + 0.0);
        if (j & 1) {
            ntx[j >> 1].y = x;
            nty[j >> 1].y = y;
            ntz[j >> 1].y = z;
        } else {
            ntx[j >> 1].x = x;
            nty[j >> 1].x = y;
            ntz[j >> 1].x = z;
        }
#pragma unroll
        for (int o = 0; o < NF; o++) {
            const float c = ok ? -fa[o * lda + p] : 0.0f;  // SS constant c_i = fh_i
            if (j & 1)
                nc[j >> 1][o].y = c;
            else
                nc[j >> 1][o].x = c;
            hi[j][o] = lo[j][o] = 0.0f;
        }
    }
    const double bx = cen[3 * it.batch], by = cen[3 * it.batch + 1], bz = cen[3 * it.batch + 2];
    constexpr bool GZOK = HH && SS;  // a Gaussian to leave out exists

    for (int e = it.e0; e < it.e1; e++) {
        const Entry en = ents[e];
        const int f = en.frame;
        const double ox = cen[3 * f] - bx, oy = cen[3 * f + 1] - by, oz = cen[3 * f + 2] - bz;
        const bool far = en.flags & 2;
        const bool self = en.flags & 1;
        const bool gz = en.flags & 4;
        if constexpr (M > 0) {
            if (far) {
                // proxies k = (k1 M + k2) M + k3 of this cluster: records src0 + k
                constexpr int PL = kTile / (M * M);  // k1-planes per tile
                constexpr int GF2 = TensorLayout<NF>::GF2;
                __shared__ float sX[M], sY[M];
                __shared__ float2 sZ2[M];
                __syncthreads();
                if (tid < M) {
                    const float4 rx = rec4[en.src0 + tid * M * M];
                    const float4 ry = rec4[en.src0 + tid * M];
                    const float4 rz = rec4[en.src0 + tid];
                    sX[tid] = (float)((double)rx.x + ox);
                    sY[tid] = (float)((double)ry.y + oy);
                    const float z = (float)((double)rz.z + oz);
                    sZ2[tid] = make_float2(z, z);
                }
                for (int p0 = 0; p0 < M; p0 += PL) {
                    const int np = min(PL, M - p0);
                    const int nk = np * M * M;
                    const int base = en.src0 + p0 * M * M;
                    __syncthreads();
#pragma unroll
                    for (int h = 0; h < kTile / THREADS; h++) {
                        const int k = tid + h * THREADS;
                        if (k < nk) {
                            float v[2 * GF2];
#pragma unroll
                            for (int m = 0; m < 2 * GF2; m++) v[m] = 0.0f;
#pragma unroll
                            for (int o = 0; o < NF; o++) v[o] = fa[o * lda + base + k];
                            v[NF] = rec4[base + k].w;
#pragma unroll
                            for (int g = 0; g < GF2; g++)
                                st[g * kTile + k] = make_float4(v[2 * g], v[2 * g], v[2 * g + 1], v[2 * g + 1]);
                        }
                    }
                    __syncthreads();
                    if (GZOK && gz)
                        tile_far_tensor<NY, HH, SS, TPT, M, GZOK>(sX + p0, sY, sZ2, st, np, ntx, nty, ntz, nc, hi, lo,
                                                                  kp2);
                    else
                        tile_far_tensor<NY, HH, SS, TPT, M, false>(sX + p0, sY, sZ2, st, np, ntx, nty, ntz, nc, hi, lo,
                                                                   kp2);
                }
                continue;
            }
        }
        for (int s0 = en.src0; s0 < en.src1; s0 += kTile) {
            const int ns = min(kTile, en.src1 - s0);
            const int nk = (ns + 15) & ~15;
            __syncthreads();
            if (far) {
#pragma unroll
                for (int h = 0; h < kTile / THREADS; h++) {
                    const int k = tid + h * THREADS;
                    float v[4 * G];
#pragma unroll
                    for (int m = 0; m < 4 * G; m++) v[m] = 0.0f;
                    if (k < ns) {
                        // proxy = cluster center + delta; one rounding to float32
                        float4 r = rec4[s0 + k];
                        r.x = (float)((double)r.x + ox);
                        r.y = (float)((double)r.y + oy);
                        r.z = (float)((double)r.z + oz);
                        srec[k] = r;
#pragma unroll
                        for (int o = 0; o < NF; o++) v[o] = fa[o * lda + s0 + k];
                    } else if (k < nk) {
                        // padding record: far away, zero weight and values -> contributes 0
                        srec[k] = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
                    }
                    if (k < nk)
#pragma unroll
                        for (int g = 0; g < G; g++)
                            sv[g * kTile + k] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                }
            } else {
#pragma unroll
                for (int h = 0; h < kTile / THREADS; h++) {
                    const int k = tid + h * THREADS;
                    float v[2 * NV4];  // x y z w_hi w_lo fh[NF] fl[NF], then padding
#pragma unroll
                    for (int m = 0; m < 2 * NV4; m++) v[m] = 0.0f;
                    if (k < ns) {
                        // point = leaf center + (delta_hi + delta_lo); one rounding
                        const float4 r = rec4[s0 + k];
                        const float4 rl = rec4lo[s0 + k];
                        v[0] = (float)(((double)r.x + (double)rl.x) + ox);
                        v[1] = (float)(((double)r.y + (double)rl.y) + oy);
                        v[2] = (float)(((double)r.z + (double)rl.z) + oz);
                        v[3] = r.w;   // weight, high part
                        v[4] = rl.w;  // weight, low part
#pragma unroll
                        for (int o = 0; o < NF; o++) {
                            v[5 + o] = fa[o * lda + s0 + k];
                            v[5 + NF + o] = fb[o * ldb + s0 + k];
                        }
                    } else if (k < nk) {
                        // padding record: far away, zero weight and values -> contributes 0
                        v[0] = v[1] = v[2] = 1e18f;
                    }
                    if (k < nk)
#pragma unroll
                        for (int g = 0; g < NV4; g++)
                            sn[g * kTile + k] = make_float4(v[2 * g], v[2 * g], v[2 * g + 1], v[2 * g + 1]);
                }
            }
            __syncthreads();
            if (far) {
                if (GZOK && gz)
                    tile_far<NY, HH, SS, TPT, GZOK>(srec, sv, nk, ntx, nty, ntz, nc, hi, lo, kp);
                else
                    tile_far<NY, HH, SS, TPT, false>(srec, sv, nk, ntx, nty, ntz, nc, hi, lo, kp);
            } else if (self) {
                tile_near<NY, HH, SS, true, TPT, false>(sn, nk, ntx, nty, ntz, nc, hi, lo, kp2);
            } else if (GZOK && gz) {
                tile_near<NY, HH, SS, false, TPT, GZOK>(sn, nk, ntx, nty, ntz, nc, hi, lo, kp2);
            } else {
                tile_near<NY, HH, SS, false, TPT, false>(sn, nk, ntx, nty, ntz, nc, hi, lo, kp2);
            }
        }
    }
    double* out = part + ((size_t)blockIdx.x * nf_tot + field0) * kTargetsPerItem;
#pragma unroll
    for (int j = 0; j < TPT; j++)
#pragma unroll
        for (int o = 0; o < NF; o++) out[o * kTargetsPerItem + tid + j * THREADS] = (double)hi[j][o] + (double)lo[j][o];
    chunk_sum<THREADS>(it, part, tsum, cnt, nf_tot, field0, NF);
}

// ---------------------------------------------------------------- bias calibration
// Mean relative error of the float32 kernel values evaluated exactly as in
// tile_near / tile_far, against float64, weighted as in the SS integrals:
//   mode 0: G~ = ex2(ky r) ri, weight r e^{-k r} (int G_k = 1/k^2, k-free in k r)
//   mode 1: H~ = ex2(ga r^2) ri, weight r e^{-r^2} (int e^{-r^2/a^2}/r = 2 pi a^2)
// on a deterministic sample of directions and radii.
constexpr int kCalBlocks = 256, kCalThreads = 256;
__global__ void k_calibrate(int mode, long long n, double* out)
{
    __shared__ double s0[kCalThreads], s1[kCalThreads];
    const double L2E = 1.4426950408889634;
    const float ky = (float)(-2.0 * L2E);
    const double kt = -(double)ky / L2E;
    const float ga = (float)(-L2E);
    const double rmax = mode == 0 ? 30.0 / kt : 6.0;
    double a = 0.0, b = 0.0;
    for (long long i = blockIdx.x * (long long)kCalThreads + threadIdx.x; i < n; i += (long long)kCalBlocks * kCalThreads) {
        const double rr = rmax * (i + 0.5) / n;
        const double th = 2.399963229728653 * i, fz = i * 0.6180339887498949;
        const double z = -1.0 + 2.0 * (fz - floor(fz));
        const double sn = sqrt(fmax(0.0, 1.0 - z * z));
        const float dx = (float)(rr * sn * cos(th)), dy = (float)(rr * sn * sin(th)), dz = (float)(rr * z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float ri = rsqrt_approx(r2);
        const double R = sqrt((double)r2);
        double e, w;
        if (mode == 0) {
            const float v = ex2_approx(ky * (r2 * ri)) * ri;
            const double ref = exp(-kt * R) / R;
            e = ((double)v - ref) / ref;
            w = R * exp(-kt * R);
        } else {
            const float v = ex2_approx(ga * r2) * ri;
            const double ref = exp((double)ga * (double)r2 / L2E) / R;  // alpha~ of the rounded ga
            e = ((double)v - ref) / ref;
            w = R * exp(-(double)r2);
        }
        a += e * w;
        b += w;
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int o = kCalThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s0[threadIdx.x] += s0[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = s0[0];
        out[2 * blockIdx.x + 1] = s1[0];
    }
}

// ---------------------------------------------------------------- FP64 plain form
template <int KIND, bool SS>
__global__ void __launch_bounds__(kThreads64) k_interact64(const Item* __restrict__ items,
                                                           const Entry* __restrict__ ents,
                                                           const double* __restrict__ rx, const double* __restrict__ ry,
                                                           const double* __restrict__ rz, const double* __restrict__ rw,
                                                           const double* __restrict__ q, const double* __restrict__ c,
                                                           const double* __restrict__ kvd, double* __restrict__ part,
                                                           double* __restrict__ tsum, int* __restrict__ cnt,
                                                           int nf_tot, int field)
{
    const double kval = kvd[field];
    __shared__ double sx[kTile64], sy[kTile64], sz[kTile64], sw[kTile64], sqv[kTile64];
    const Item it = items[blockIdx.x];
    const int tid = threadIdx.x;
    const int p = it.t0 + tid;
    const bool ok = p < it.t1;
    const double x = ok ? rx[p] : 0.0, y = ok ? ry[p] : 0.0, z = ok ? rz[p] : 0.0;
    const double ci = ok ? c[p] : 0.0;
    const double ia2 = KIND == 1 ? 1.0 / (kval * kval) : 0.0;
    double acc = 0.0;
    for (int e = it.e0; e < it.e1; e++) {
        const Entry en = ents[e];
        for (int s0 = en.src0; s0 < en.src1; s0 += kTile64) {
            const int ns = min(kTile64, en.src1 - s0);
            __syncthreads();
            if (tid < ns) {
                sx[tid] = rx[s0 + tid];
                sy[tid] = ry[s0 + tid];
                sz[tid] = rz[s0 + tid];
                sw[tid] = rw[s0 + tid];
                sqv[tid] = q[s0 + tid];
            }
            __syncthreads();
            for (int k = 0; k < ns; k++) {
                const double dx = x - sx[k], dy = y - sy[k], dz = z - sz[k];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0.0) continue;  // the singular r' = r term is skipped
                const double r = sqrt(r2);
                if (KIND == 0) {
                    const double d = SS ? sqv[k] - ci * sw[k] : sqv[k];
                    acc += exp(-kval * r) / r * d;
                } else {
                    const double d = SS ? sqv[k] - ci * sw[k] * exp(-r2 * ia2) : sqv[k];
                    acc += d / r;
                }
            }
        }
    }
    part[((size_t)blockIdx.x * nf_tot + field) * kTargetsPerItem + tid] = acc;
    chunk_sum<kThreads64>(it, part, tsum, cnt, nf_tot, field, 1);
}

template <int NY, bool HH, bool SS, int M>
void launch32_m(Tree& T, const float* kyd, const float* q, const float* c, double* part, double* tsum, int* cnt,
                int nf_tot, int field0)
{
    launch(k_interact32<NY, HH, SS, M>, (int)T.nitems, Tpt<NY + HH>::threads, 0, T.stream, T.items.as<Item>(),
           T.ent.as<Entry>(), T.cl_cen.as<double>(), T.rec4.as<float4>(), T.rec4lo.as<float4>(), q, T.nrec, c, T.n,
           kyd, part, tsum, cnt, nf_tot, field0);
}

template <int NY, bool HH>
void launch32_ss(Tree& T, bool ss, const float* kyd, const float* q, const float* c, double* part, double* tsum,
                 int* cnt, int nf_tot, int field0)
{
    // q: rows of fa (fh for points, qh for proxies), c: rows of fb (fl for points).
    // The tensor-grid far path serves degrees 6 and 8 with SS; others take
    // the record path.
    const int m = T.degree + 1;
    if (ss && m == 9)
        launch32_m<NY, HH, true, 9>(T, kyd, q, c, part, tsum, cnt, nf_tot, field0);
    else if (ss && m == 7)
        launch32_m<NY, HH, true, 7>(T, kyd, q, c, part, tsum, cnt, nf_tot, field0);
    else if (ss)
        launch32_m<NY, HH, true, 0>(T, kyd, q, c, part, tsum, cnt, nf_tot, field0);
    else
        launch32_m<NY, HH, false, 0>(T, kyd, q, c, part, tsum, cnt, nf_tot, field0);
    TAGI_LAUNCH_CHECK();
}

template <bool HH>
void launch32_ny(int ny, Tree& T, bool ss, const float* kyd, const float* q, const float* c, double* part,
                 double* tsum, int* cnt, int nf_tot, int field0)
{
    switch (ny) {
        case 0:
            if constexpr (HH) launch32_ss<0, true>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0);
            break;
        case 1: launch32_ss<1, HH>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0); break;
        case 2: launch32_ss<2, HH>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0); break;
        case 3: launch32_ss<3, HH>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0); break;
        case 4: launch32_ss<4, HH>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0); break;
        case 5: launch32_ss<5, HH>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0); break;
        case 6: launch32_ss<6, HH>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0); break;
        case 7: launch32_ss<7, HH>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0); break;
        case 8:
            if constexpr (!HH) launch32_ss<8, false>(T, ss, kyd, q, c, part, tsum, cnt, nf_tot, field0);
            break;
        default: throw Error(TAGI_ERR_INVALID_ARG, "field group too large");
    }
}

}  // namespace

void fp32_bias(cudaStream_t s, double* beta_y, double* beta_g)
{
    // measured once per device and process; deterministic
    static double cache[64][2];
    static bool done[64] = {false};
    int dev = 0;
    TAGI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) dev = 0;
    if (!done[dev]) {
        DevBuf buf;
        buf.ensure(sizeof(double) * 2 * kCalBlocks);
        std::vector<double> h(2 * kCalBlocks);
        for (int mode = 0; mode < 2; mode++) {
            launch(k_calibrate, kCalBlocks, kCalThreads, 0, s, mode, 1LL << 23, buf.as<double>());
            TAGI_LAUNCH_CHECK();
            TAGI_CUDA(cudaMemcpyAsync(h.data(), buf.p, sizeof(double) * 2 * kCalBlocks, cudaMemcpyDeviceToHost, s));
            TAGI_CUDA(cudaStreamSynchronize(s));
            double a = 0.0, b = 0.0;
            for (int i = 0; i < kCalBlocks; i++) {
                a += h[2 * i];
                b += h[2 * i + 1];
            }
            cache[dev][mode] = a / b;
        }
        done[dev] = true;
    }
    *beta_y = cache[dev][0];
    *beta_g = cache[dev][1];
}

// Float64 value of the decay rate the float32 kernel actually applies:
// ky = fl32(-k log2 e), k~ = -ky / log2 e.
double effective_k32(double k)
{
    const float ky = (float)(-k * 1.4426950408889634);
    return -(double)ky / 1.4426950408889634;
}

// Float64 Gaussian width the float32 kernel applies: ga = fl32(-log2 e / a^2).
double effective_alpha32(double a)
{
    const float ga = (float)(-1.4426950408889634 / (a * a));
    return sqrt(-1.4426950408889634 / (double)ga);
}

// Fields [0, nf) of T.fa / T.fb: Yukawa fields first (kinds[o] == 0), then
// at most one Coulomb field (kinds[o] == 1) last.  Groups of at most 8 fields
// share a launch; the Coulomb field joins the last group when it fits.
// kyd: device array of the fields' exponent factors (see make_rates).
void interact32(Tree& T, int nf, const int* kinds, const float* kyd, double* part, double* tsum, int* cnt)
{
    int ny = 0;
    while (ny < nf && kinds[ny] == 0) ny++;
    const bool hh = ny < nf;
    TAGI_REQUIRE(nf - ny <= 1, "at most one Coulomb field, after the Yukawa fields");
    int o = 0;
    while (o < nf) {
        int g_ny = ny - o < 8 ? ny - o : 8;
        if (g_ny < 0) g_ny = 0;
        bool g_hh = hh && (o + g_ny == ny) && g_ny < 8;
        const float* q = T.fa.as<float>() + (size_t)o * T.nrec;
        const float* c = T.fb.as<float>() + (size_t)o * T.n;
        if (g_hh)
            launch32_ny<true>(g_ny, T, T.ss != 0, kyd + o, q, c, part, tsum, cnt, nf, o);
        else
            launch32_ny<false>(g_ny, T, T.ss != 0, kyd + o, q, c, part, tsum, cnt, nf, o);
        o += g_ny + (g_hh ? 1 : 0);
    }
}

void interact64(Tree& T, int field, int nf_tot, int kind, const double* kvd, const double* q, const double* c,
                double* part, double* tsum, int* cnt)
{
    const int grid = (int)T.nitems;
    cudaStream_t s = T.stream;
    const Item* it = T.items.as<Item>();
    const Entry* en = T.ent.as<Entry>();
    const double *rx = T.rx.as<double>(), *ry = T.ry.as<double>(), *rz = T.rz.as<double>(), *rw = T.rw.as<double>();
    if (kind == 0) {
        if (T.ss)
            launch(k_interact64<0, true>, grid, kThreads64, 0, s, it, en, rx, ry, rz, rw, q, c, kvd, part, tsum, cnt, nf_tot, field);
        else
            launch(k_interact64<0, false>, grid, kThreads64, 0, s, it, en, rx, ry, rz, rw, q, c, kvd, part, tsum, cnt, nf_tot, field);
    } else {
        if (T.ss)
            launch(k_interact64<1, true>, grid, kThreads64, 0, s, it, en, rx, ry, rz, rw, q, c, kvd, part, tsum, cnt, nf_tot, field);
        else
            launch(k_interact64<1, false>, grid, kThreads64, 0, s, it, en, rx, ry, rz, rw, q, c, kvd, part, tsum, cnt, nf_tot, field);
    }
    TAGI_LAUNCH_CHECK();
}

}  // namespace tagi
