// Anterpolation: proxy weights of Eq. particle-cluster-approx-rearranged,
//   qh_k = sum_{j in C} L_k1(x_j) L_k2(y_j) L_k3(z_j) q_j,
// with the barycentric basis of Eq. Lagrange_polynomials and the weights of
// Eq. barycentric_weights on Chebyshev points of the second kind mapped to the
// cluster box (Section 5.2).
//
// One CTA per work item (a chunk of at most kAntChunk points of one cluster).
// Each thread owns up to four proxies; the points of the chunk stream through
// shared memory 64 at a time together with their 3 (n+1) basis values, so a
// proxy weight costs 2 multiplies plus one FMA per charge column per point.
// Per-tile sums are folded into float64 (FP32C) and chunk partials are summed
// in a fixed order, so results are reproducible run to run.
#include <cuda_runtime.h>

#include "tagi_internal.cuh"

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

constexpr int kAntLP = 12;  // padded basis row of the cache (degree <= 11)
static_assert(kMaxDegree + 1 <= kAntLP, "basis row fits");

// Basis cache of the float32 path: for every point of every anterpolation
// item and each dimension, the float64 basis of Eq. Lagrange_polynomials on
// the float32-rounded nodes, rounded to float32 (exactly the values k_ant
// evaluates), rows of kAntLP floats at ((item * kAntChunk + j) * 3 + d).
__global__ void __launch_bounds__(kAntThreads) k_ant_basis(const AntItem* __restrict__ items,
                                                           const double* __restrict__ px,
                                                           const double* __restrict__ py,
                                                           const double* __restrict__ pz,
                                                           const double* __restrict__ lo,
                                                           const double* __restrict__ hi, int degree,
                                                           float* __restrict__ antL)
{
    __shared__ double dnodes[kMaxDegree + 1], inv[kMaxDegree + 1];
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
        }
    }
    __syncthreads();
    const int np = it.p1 - it.p0;
    for (int e = threadIdx.x; e < 3 * np; e += blockDim.x) {
        const int j = e / 3, d = e % 3;
        const double* x = d == 0 ? px : (d == 1 ? py : pz);
        const bool deg = hh[d] == 0.0;
        double Ld[kMaxDegree + 1];
        const double td = deg ? 0.0 : (x[it.p0 + j] - cc[d]) * ih[d];
        basis_prod(td, deg, degree, dnodes, inv, Ld);
        float4* row = reinterpret_cast<float4*>(antL + (((size_t)blockIdx.x * kAntChunk + j) * 3 + d) * kAntLP);
#pragma unroll
        for (int g = 0; g < kAntLP / 4; g++) {
            float v[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int k = 4 * g + i;
                v[i] = k <= degree ? (float)Ld[k] : 0.0f;
            }
            row[g] = make_float4(v[0], v[1], v[2], v[3]);
        }
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
                const float4* row = reinterpret_cast<const float4*>(
                    antL + (((size_t)blockIdx.x * kAntChunk + (p0 - it.p0) + j) * 3 + d) * kAntLP);
#pragma unroll
                for (int g = 0; g < kAntLP / 4; g++) {
                    const float4 v = row[g];
                    if (4 * g <= degree) L[4 * g] = (R)v.x;
                    if (4 * g + 1 <= degree) L[4 * g + 1] = (R)v.y;
                    if (4 * g + 2 <= degree) L[4 * g + 2] = (R)v.z;
                    if (4 * g + 3 <= degree) L[4 * g + 3] = (R)v.w;
                }
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

}  // namespace

void anterpolate_weights(Tree& T)
{
    if (T.nfar == 0) return;
    cudaStream_t s = T.stream;
    if (T.prec == TAGI_FP32C) {
        // basis cache (kept with the tree while it fits the budget below)
        const size_t cache_bytes = sizeof(float) * (size_t)T.nant * kAntChunk * 3 * kAntLP;
        if (cache_bytes <= ((size_t)16 << 30)) {
            T.antL.ensure(cache_bytes);
            launch(k_ant_basis, (int)T.nant, kAntThreads, 0, s, T.ant_items.as<AntItem>(), T.px.as<double>(),
                   T.py.as<double>(), T.pz.as<double>(), T.cl_lo.as<double>(), T.cl_hi.as<double>(), T.degree,
                   T.antL.as<float>());
            TAGI_LAUNCH_CHECK();
        }
        const float* antL = T.antL.p ? T.antL.as<float>() : nullptr;
        // w^ from the two-float weights (w_hi, w_lo), on the float32 nodes
        // where the proxies sit
        T.antpart.ensure(sizeof(double) * (size_t)T.nant * T.P * 2);
        DevBuf w2;
        w2.ensure(sizeof(float) * 2 * (size_t)T.n);
        launch(k_split_w, (int)((T.n + 255) / 256), 256, 0, s, T.pw.as<double>(), T.n, w2.as<float>());
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
    for (int g0 = 0; g0 < nf; g0 += 8) {
        int g = nf - g0 < 8 ? nf - g0 : 8;
        T.antpart.ensure(sizeof(double) * (size_t)T.nant * T.P * g);
        launch_ant<float, double>(g, (int)T.nant, T.ant_items.as<AntItem>(), T, T.qant.as<float>() + g0 * T.n,
                                  T.n, T.antpart.as<double>(), s, T.antL.p ? T.antL.as<float>() : nullptr);
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
