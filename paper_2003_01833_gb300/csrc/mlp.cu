// Learned warm start for SCF runs of molecules: point features, a per-point
// MLP (F = 8 inputs, two tanh layers of H = 32 here, one output), its
// gradient and Adam.  The H = 64 network runs on the tensor cores
// (mlp64.cu); this file holds the entry points of both.  Weights enter the products rounded to bfloat16 and features are
// stored as bfloat16; the arithmetic of a point is float32, gradients are
// accumulated over points in float64 in a fixed order (deterministic for a
// given device), and Adam keeps float64 master weights.
//
// Not a method of the paper: its SCF runs start from superposed atomic data
// (Section 6).  The model predicts a relative correction y of the normalised
// superposition start s, psi = s (1 + y).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "tagi_internal.cuh"

namespace tagi {
namespace {

constexpr int kF = 8;
constexpr int kH = 32;
constexpr int oW1 = 0, oB1 = kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kP = oB3 + 1;  // 1377 parameters
constexpr int kPPad = 1380;  // float slots of the weights in shared memory (keeps the stash 16-byte aligned)
constexpr int kThreads = 128;
// Stash row of one point for the gradient reduction: x | h1 | h2 | dz1 | dz2 |
// dy | 1.  An odd stride keeps the rows of a warp's 32 points in 32 banks.
constexpr int cX = 0, cH1 = 8, cH2 = 40, cD1 = 72, cD2 = 104, cDy = 136, cOne = 137, kStride = 139;
// Gradient entries per thread: a 2 x 4 tile of W2 (rows j0, j0+1; columns
// i0..i0+3), 6 shared loads per point for its 8 products, and up to 3 of the
// other 353 entries (W1, b1, b2, W3, b3), 2 loads per product.
constexpr int kRest = kP - kH * kH;
constexpr int kRestPer = (kRest + kThreads - 1) / kThreads;
static_assert(kThreads == (kH / 2) * (kH / 4), "one 2 x 4 tile of W2 per thread");
constexpr int kMaxNuclei = 16;
constexpr size_t kGradSmem = sizeof(float) * (kPPad + (size_t)kThreads * kStride);

struct Nuclei {
    double x[kMaxNuclei], y[kMaxNuclei], z[kMaxNuclei];
    double zs[kMaxNuclei];  // decay rate of each nucleus's exponential features (1 by default)
    int m;
    int ordered;  // 1: two nuclei taken in list order (r1 to the first) instead of by distance
};

// Nearest bfloat16 value of x, ties to even, from the float64 value: x / q
// with q the spacing of bfloat16 values at x (a power of two, so exact),
// rounded to an integer half-to-even, scaled back.  The result has 8
// significant bits within float32's exponent range, so the float32
// conversion is exact and its high half is the bfloat16 encoding.
__device__ __forceinline__ uint16_t bf16_bits(double x)
{
    if (isnan(x)) return 0x7FC0;
    if (x == 0.0) return signbit(x) ? 0x8000 : 0;
    int e;
    frexp(x, &e);
    const double q = ldexp(1.0, max(e - 8, -133));
    const double r = rint(x / q) * q;
    return (uint16_t)(__float_as_uint((float)r) >> 16);
}

__device__ __forceinline__ float bf16_float(uint32_t b) { return __uint_as_float(b << 16); }

__device__ __forceinline__ bool is_weight(int e)
{
    return (e >= oW1 && e < oB1) || (e >= oW2 && e < oB2) || (e >= oW3 && e < oB3);
}

// Weights rounded to bfloat16, biases as float32, into shared memory.
__device__ __forceinline__ void load_params(float* sw, const double* __restrict__ master)
{
    for (int e = threadIdx.x; e < kP; e += blockDim.x)
        sw[e] = is_weight(e) ? bf16_float(bf16_bits(master[e])) : (float)master[e];
}

__device__ __forceinline__ void load_x(const uint16_t* __restrict__ feat, int64_t i, float x[kF])
{
    const uint4 v = *reinterpret_cast<const uint4*>(feat + i * kF);
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        x[2 * k] = bf16_float(u[k] & 0xFFFFu);
        x[2 * k + 1] = bf16_float(u[k] >> 16);
    }
}

__device__ __forceinline__ void layer1(const float* sw, const float x[kF], float h1[kH])
{
#pragma unroll
    for (int i = 0; i < kH; i++) {
        float z = sw[oB1 + i];
#pragma unroll
        for (int f = 0; f < kF; f++) z = fmaf(sw[oW1 + i * kF + f], x[f], z);
        h1[i] = tanhf(z);
    }
}

__device__ __forceinline__ float layer2_unit(const float* sw, const float h1[kH], int j)
{
    float z = sw[oB2 + j];
#pragma unroll
    for (int i = 0; i < kH; i++) z = fmaf(sw[oW2 + j * kH + i], h1[i], z);
    return tanhf(z);
}

// ------------------------------------------------------------------ kernels
// Features of a point (float64, rounded once to bfloat16): with r1 <= r2 the
// distances to the two nearest nuclei (the lower index first on ties), z1
// and z2 those nuclei's decay rates (1 unless given) and R their
// separation, [e^-(z1 r1), e^-(z2 r2), tanh r1, tanh r2, (r2 - r1)/R,
// tanh((r1 + r2)/R - 1), R - 1.5, e^-(r1 + r2 - R)].  Sums of squares are
// formed left to right without contraction.
__global__ void k_features(const double* __restrict__ xyz, int64_t n, Nuclei nuc, uint16_t* __restrict__ feat)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double px = xyz[i], py = xyz[n + i], pz = xyz[2 * n + i];
    double d1 = INFINITY, d2 = INFINITY;
    int a1 = 0, a2 = 1;
    for (int a = 0; a < (nuc.ordered ? 0 : nuc.m); a++) {
        const double dx = px - nuc.x[a], dy = py - nuc.y[a], dz = pz - nuc.z[a];
        const double d = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        if (d < d1) {
            d2 = d1;
            a2 = a1;
            d1 = d;
            a1 = a;
        } else if (d < d2) {
            d2 = d;
            a2 = a;
        }
    }
    if (nuc.ordered) {
        const double dx1 = px - nuc.x[0], dy1 = py - nuc.y[0], dz1 = pz - nuc.z[0];
        const double dx2 = px - nuc.x[1], dy2 = py - nuc.y[1], dz2 = pz - nuc.z[1];
        d1 = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx1, dx1), __dmul_rn(dy1, dy1)), __dmul_rn(dz1, dz1)));
        d2 = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx2, dx2), __dmul_rn(dy2, dy2)), __dmul_rn(dz2, dz2)));
    }
    const double ex = nuc.x[a1] - nuc.x[a2], ey = nuc.y[a1] - nuc.y[a2], ez = nuc.z[a1] - nuc.z[a2];
    const double R = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
    const double s12 = __dadd_rn(d1, d2);
    const double f[kF] = {exp(-__dmul_rn(nuc.zs[a1], d1)),
                          exp(-__dmul_rn(nuc.zs[a2], d2)),
                          tanh(d1),
                          tanh(d2),
                          __dsub_rn(d2, d1) / R,
                          tanh(__dsub_rn(s12 / R, 1.0)),
                          __dsub_rn(R, 1.5),
                          exp(-__dsub_rn(s12, R))};
    uint32_t u[4];
#pragma unroll
    for (int k = 0; k < 4; k++) u[k] = (uint32_t)bf16_bits(f[2 * k]) | ((uint32_t)bf16_bits(f[2 * k + 1]) << 16);
    *reinterpret_cast<uint4*>(feat + i * kF) = make_uint4(u[0], u[1], u[2], u[3]);
}

__global__ void __launch_bounds__(kThreads) k_mlp_forward(const uint16_t* __restrict__ feat, int64_t n,
                                                          const double* __restrict__ master, float* __restrict__ y)
{
    __shared__ float sw[kPPad];
    load_params(sw, master);
    __syncthreads();
#pragma unroll 1
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        // the weights are read from shared memory in every iteration rather
        // than all 1377 held in registers across the loop
        asm volatile("" ::: "memory");
        float x[kF], h1[kH];
        load_x(feat, i, x);
        layer1(sw, x, h1);
        float out = sw[oB3];
#pragma unroll 1
        for (int j = 0; j < kH; j++) out = fmaf(sw[oW3 + j], layer2_unit(sw, h1, j), out);
        y[i] = out;
    }
}

// Loss L = sum_p wt_p (y_p - t_p)^2 and its gradient: each thread runs the
// forward and backward pass of one point of a 128-point tile and stashes
// (x, h1, h2, dz1, dz2, dy) in shared memory; then each thread forms its own
// gradient entries (outer-product sums over the tile in point order, float32;
// a 2 x 4 register tile of W2 and up to 3 other entries) and adds them to
// float64 accumulators.  Tiles are strided over a fixed
// grid; per-block partials [grid][kP + 1] (the loss last) are reduced by
// k_mlp_adam in block order.
__global__ void __launch_bounds__(kThreads) k_mlp_grad(const uint16_t* __restrict__ feat,
                                                       const float* __restrict__ target, const float* __restrict__ wt,
                                                       int64_t n, const double* __restrict__ master,
                                                       double* __restrict__ partial)
{
    extern __shared__ float sm[];
    float* sw = sm;
    float* st = sm + kPPad;
    __shared__ double sl[kThreads];
    const int tid = threadIdx.x;
    load_params(sw, master);

    const int j0 = 2 * (tid >> 3), i0 = 4 * (tid & 7);
    double accw[8];
    int ca[kRestPer], cb[kRestPer], ce[kRestPer];
    double acc[kRestPer];
#pragma unroll
    for (int k = 0; k < 8; k++) accw[k] = 0.0;
#pragma unroll
    for (int k = 0; k < kRestPer; k++) {
        const int q = tid + k * kThreads;  // index among the entries outside W2
        int e = -1, a = cDy, b = cOne;     // q >= kRest: computed, never written
        if (q < oW2) {                     // W1 and b1 precede W2
            e = q;
            a = cD1 + (q < oB1 ? q / kF : q - oB1);
            b = q < oB1 ? cX + q % kF : cOne;
        } else if (q < oW2 + kH) {         // b2
            e = oB2 + (q - oW2);
            a = cD2 + (q - oW2);
        } else if (q < oW2 + 2 * kH) {     // W3
            e = oW3 + (q - oW2 - kH);
            b = cH2 + (q - oW2 - kH);
        } else if (q < kRest) {            // b3
            e = oB3;
        }
        ce[k] = e;
        ca[k] = a;
        cb[k] = b;
        acc[k] = 0.0;
    }
    double lsum = 0.0;
    __syncthreads();

    const int64_t ntiles = (n + kThreads - 1) / kThreads;
    float* row = st + tid * kStride;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * kThreads + tid;
        if (i < n) {
            float x[kF], h1[kH];
            load_x(feat, i, x);
            layer1(sw, x, h1);
            float y = sw[oB3];
            for (int j = 0; j < kH; j++) {
                const float a = layer2_unit(sw, h1, j);
                row[cH2 + j] = a;
                y = fmaf(sw[oW3 + j], a, y);
            }
            const float r = y - target[i];
            const float dy = 2.0f * wt[i] * r;
            lsum += (double)wt[i] * (double)r * (double)r;
            float g1[kH];
#pragma unroll
            for (int q = 0; q < kH; q++) g1[q] = 0.0f;
            for (int j = 0; j < kH; j++) {
                const float a = row[cH2 + j];
                const float d2 = dy * sw[oW3 + j] * (1.0f - a * a);
                row[cD2 + j] = d2;
#pragma unroll
                for (int q = 0; q < kH; q++) g1[q] = fmaf(sw[oW2 + j * kH + q], d2, g1[q]);
            }
#pragma unroll
            for (int q = 0; q < kH; q++) {
                row[cH1 + q] = h1[q];
                row[cD1 + q] = g1[q] * (1.0f - h1[q] * h1[q]);
            }
#pragma unroll
            for (int f = 0; f < kF; f++) row[cX + f] = x[f];
            row[cDy] = dy;
            row[cOne] = 1.0f;
        } else {
            for (int c = 0; c < kStride; c++) row[c] = 0.0f;
        }
        __syncthreads();
        {
            float s[8], r[kRestPer];
#pragma unroll
            for (int k = 0; k < 8; k++) s[k] = 0.0f;
#pragma unroll
            for (int k = 0; k < kRestPer; k++) r[k] = 0.0f;
            for (int p = 0; p < kThreads; p++) {
                const float* rp = st + p * kStride;
                const float d0 = rp[cD2 + j0], d1 = rp[cD2 + j0 + 1];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float h = rp[cH1 + i0 + c];
                    s[c] = fmaf(d0, h, s[c]);
                    s[4 + c] = fmaf(d1, h, s[4 + c]);
                }
#pragma unroll
                for (int k = 0; k < kRestPer; k++) r[k] = fmaf(rp[ca[k]], rp[cb[k]], r[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; k++) accw[k] += (double)s[k];
#pragma unroll
            for (int k = 0; k < kRestPer; k++) acc[k] += (double)r[k];
        }
        __syncthreads();
    }
    double* out = partial + (size_t)blockIdx.x * (kP + 1);
#pragma unroll
    for (int c = 0; c < 4; c++) {
        out[oW2 + j0 * kH + i0 + c] = accw[c];
        out[oW2 + (j0 + 1) * kH + i0 + c] = accw[4 + c];
    }
#pragma unroll
    for (int k = 0; k < kRestPer; k++)
        if (ce[k] >= 0) out[ce[k]] = acc[k];
    sl[tid] = lsum;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int t = 0; t < kThreads; t++) s += sl[t];
        out[kP] = s;
    }
}

// Gradient and loss from the per-block partials [nblk][np + 1] (block
// order), then, if apply, one Adam step on the float64 master weights
// (c1 = 1 - beta1^t, c2 = 1 - beta2^t).
__global__ void k_mlp_adam(const double* __restrict__ partial, int nblk, int np, double* __restrict__ master,
                           double* __restrict__ m, double* __restrict__ v, double lr, double beta1, double beta2,
                           double eps, double c1, double c2, int apply, double* __restrict__ grad_out,
                           double* __restrict__ loss_out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > np) return;
    double g = 0.0;
    for (int b = 0; b < nblk; b++) g += partial[(size_t)b * (np + 1) + e];
    if (e == np) {
        *loss_out = g;
        return;
    }
    grad_out[e] = g;
    if (!apply) return;
    const double mm = beta1 * m[e] + (1.0 - beta1) * g;
    const double vv = beta2 * v[e] + (1.0 - beta2) * g * g;
    m[e] = mm;
    v[e] = vv;
    master[e] -= (lr * (mm / c1)) / (sqrt(vv / c2) + eps);
}

// psi = s (1 + y) and per-block partial sums of psi^2 w (block order).
__global__ void __launch_bounds__(256) k_warm_apply(const float* __restrict__ y, const double* __restrict__ s,
                                                    const double* __restrict__ w, int64_t n,
                                                    double* __restrict__ psi, double* __restrict__ part)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double p = s[i] * (1.0 + (double)y[i]);
        psi[i] = p;
        acc += p * p * w[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// psi /= sqrt(sum of the partials): one thread of each block sums them in
// block order (every block gets the same value) and shares the factor.
__global__ void k_warm_scale(double* __restrict__ psi, int64_t n, const double* __restrict__ part, int nblk)
{
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += part[b];
        inv = 1.0 / sqrt(s);
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        psi[i] *= inv;
}

// ------------------------------------------------------------------ object
struct Mlp {
    int dev = 0;
    int sms = 0;
    int H = kH;     // 32: SIMT kernels of this file; 64: tensor-core kernels (mlp64.cu)
    int np = kP;    // parameters
    int64_t step = 0;
    DevBuf master, m, v, partial, grad, loss, part, errd;
    std::string err;
};

int grad_grid(const Mlp& M, int64_t n)
{
    const int64_t tiles = (n + kThreads - 1) / kThreads;
    return (int)std::min<int64_t>(tiles, 2LL * M.sms);
}

thread_local std::string g_mlp_err;

template <class F>
tagi_status guarded_mlp(F&& f)
{
    try {
        report_error(TAGI_OK, "");
        f();
        return TAGI_OK;
    } catch (const Error& e) {
        g_mlp_err = e.what();
        return report_error(e.status, g_mlp_err.c_str());
    } catch (const std::bad_alloc&) {
        return report_error(TAGI_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        g_mlp_err = e.what();
        return report_error(TAGI_ERR_CUDA, g_mlp_err.c_str());
    }
}

Mlp* as_mlp(const tagi_mlp* p)
{
    TAGI_REQUIRE(p != nullptr, "mlp is NULL");
    return reinterpret_cast<Mlp*>(const_cast<tagi_mlp*>(p));
}

void check_data(const void* feat, int64_t n)
{
    TAGI_REQUIRE(feat != nullptr, "feat is NULL");
    TAGI_REQUIRE(n >= 1, "n must be >= 1");
    TAGI_REQUIRE(((uintptr_t)feat & 15) == 0, "feat must be 16-byte aligned");
}

// Gradient (and loss) of the current master weights into M.grad / M.loss;
// with apply, one Adam step as well.
void grad_pass(Mlp& M, const uint16_t* feat, const float* target, const float* wt, int64_t n,
               const tagi_adam_params* a, bool apply, cudaStream_t s)
{
    const int grid = M.H == 64 ? mlp64_grad_grid(n, M.sms) : grad_grid(M, n);
    M.partial.ensure(sizeof(double) * (size_t)grid * (M.np + 1));
    if (M.H == 64)
        mlp64_gradient(feat, target, wt, n, M.master.as<double>(), M.partial.as<double>(), grid, M.errd.as<int>(), s);
    else
        launch(k_mlp_grad, grid, kThreads, kGradSmem, s, feat, target, wt, n, M.master.as<double>(),
               M.partial.as<double>());
    double c1 = 1.0, c2 = 1.0, lr = 0.0, b1 = 0.9, b2 = 0.999, eps = 1e-8;
    if (apply) {
        M.step += 1;
        lr = a->lr;
        b1 = a->beta1;
        b2 = a->beta2;
        eps = a->eps;
        c1 = 1.0 - std::pow(b1, (double)M.step);
        c2 = 1.0 - std::pow(b2, (double)M.step);
    }
    launch(k_mlp_adam, (M.np + 1 + 127) / 128, 128, 0, s, M.partial.as<double>(), grid, M.np, M.master.as<double>(),
           M.m.as<double>(), M.v.as<double>(), lr, b1, b2, eps, c1, c2, apply ? 1 : 0, M.grad.as<double>(),
           M.loss.as<double>());
    TAGI_LAUNCH_CHECK();
}

// y of the network for n points (the H = 32 or the H = 64 kernels)
void run_forward(Mlp& M, const uint16_t* feat, int64_t n, float* y, cudaStream_t s)
{
    if (M.H == 64) {
        mlp64_forward(feat, n, M.master.as<double>(), y, M.errd.as<int>(), M.sms, s);
    } else {
        const int64_t blocks = std::min<int64_t>((n + kThreads - 1) / kThreads, 8LL * M.sms);
        launch(k_mlp_forward, (unsigned)blocks, kThreads, 0, s, feat, n, M.master.as<double>(), y);
        TAGI_LAUNCH_CHECK();
    }
}

// after a synchronisation: a bounded wait of the tensor-core kernels gave up
void check_mlp_err(Mlp& M, cudaStream_t s)
{
    if (M.H != 64) return;
    int h = 0;
    TAGI_CUDA(cudaMemcpyAsync(&h, M.errd.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaStreamSynchronize(s));
    if (h) throw Error(TAGI_ERR_TIMEOUT, "a bounded wait of the tensor-core MLP kernels gave up");
}

}  // namespace
}  // namespace tagi

using namespace tagi;

extern "C" {

tagi_status tagi_mlp_create(int n_features, int hidden, const double* params, int64_t n_params, tagi_mlp** out)
{
    return guarded_mlp([&] {
        TAGI_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        TAGI_REQUIRE(n_features == kF && (hidden == kH || hidden == 64),
                     "the model has 8 features and 32 or 64 hidden units");
        const int np = hidden == 64 ? mlp64_params() : kP;
        TAGI_REQUIRE(params != nullptr && n_params == np, "params must hold 1377 (H = 32) or 4801 (H = 64) values");
        for (int64_t e = 0; e < n_params; e++) TAGI_REQUIRE(std::isfinite(params[e]), "params must be finite");
        TAGI_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem));
        auto* M = new Mlp();
        M->H = hidden;
        M->np = np;
        try {
            TAGI_CUDA(cudaGetDevice(&M->dev));
            TAGI_CUDA(cudaDeviceGetAttribute(&M->sms, cudaDevAttrMultiProcessorCount, M->dev));
            AllocStream as(nullptr);
            M->master.ensure(sizeof(double) * np);
            M->m.ensure(sizeof(double) * np);
            M->v.ensure(sizeof(double) * np);
            M->grad.ensure(sizeof(double) * np);
            M->loss.ensure(sizeof(double));
            M->errd.ensure(sizeof(int));
            TAGI_CUDA(cudaMemcpy(M->master.p, params, sizeof(double) * np, cudaMemcpyHostToDevice));
            TAGI_CUDA(cudaMemset(M->m.p, 0, sizeof(double) * np));
            TAGI_CUDA(cudaMemset(M->v.p, 0, sizeof(double) * np));
            TAGI_CUDA(cudaMemset(M->errd.p, 0, sizeof(int)));
        } catch (...) {
            delete M;
            throw;
        }
        *out = reinterpret_cast<tagi_mlp*>(M);
    });
}

tagi_status tagi_mlp_get_params(const tagi_mlp* mlp, double* params, int64_t n_params, void* stream)
{
    return guarded_mlp([&] {
        Mlp* M = as_mlp(mlp);
        TAGI_REQUIRE(params != nullptr && n_params == M->np, "params must hold the model's parameter count");
        cudaStream_t s = (cudaStream_t)stream;
        TAGI_CUDA(cudaMemcpyAsync(params, M->master.p, sizeof(double) * M->np, cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
        check_mlp_err(*M, s);
    });
}

static tagi_status features_call(const double* xyz, int64_t n, const double* nuclei, const double* scale,
                                 int n_nuclei, int ordered, uint16_t* feat, void* stream)
{
    return guarded_mlp([&] {
        TAGI_REQUIRE(xyz != nullptr && nuclei != nullptr, "xyz or nuclei is NULL");
        check_data(feat, n);
        TAGI_REQUIRE(n_nuclei >= 2 && n_nuclei <= kMaxNuclei, "need 2 to 16 nuclei");
        TAGI_REQUIRE(!ordered || n_nuclei == 2, "list order needs exactly two nuclei");
        Nuclei nu{};
        nu.m = n_nuclei;
        nu.ordered = ordered;
        for (int a = 0; a < n_nuclei; a++) {
            nu.x[a] = nuclei[3 * a];
            nu.y[a] = nuclei[3 * a + 1];
            nu.z[a] = nuclei[3 * a + 2];
            nu.zs[a] = scale ? scale[a] : 1.0;
            TAGI_REQUIRE(std::isfinite(nu.x[a]) && std::isfinite(nu.y[a]) && std::isfinite(nu.z[a]),
                         "nuclei must be finite");
            TAGI_REQUIRE(std::isfinite(nu.zs[a]) && nu.zs[a] > 0.0, "decay rates must be finite and positive");
        }
        for (int a = 0; a < n_nuclei; a++)
            for (int b = 0; b < a; b++)
                TAGI_REQUIRE(nu.x[a] != nu.x[b] || nu.y[a] != nu.y[b] || nu.z[a] != nu.z[b],
                             "nuclei must be distinct");
        launch(k_features, (unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream, xyz, n, nu, feat);
        TAGI_LAUNCH_CHECK();
    });
}

tagi_status tagi_mlp_features(const double* xyz, int64_t n, const double* nuclei, int n_nuclei, uint16_t* feat,
                              void* stream)
{
    return features_call(xyz, n, nuclei, nullptr, n_nuclei, 0, feat, stream);
}

tagi_status tagi_mlp_features_ordered(const double* xyz, int64_t n, const double* nuclei, uint16_t* feat,
                                      void* stream)
{
    return features_call(xyz, n, nuclei, nullptr, 2, 1, feat, stream);
}

tagi_status tagi_mlp_features_scaled(const double* xyz, int64_t n, const double* nuclei, const double* scale,
                                     int n_nuclei, int ordered, uint16_t* feat, void* stream)
{
    if (!scale) return report_error(TAGI_ERR_INVALID_ARG, "scale is NULL");
    return features_call(xyz, n, nuclei, scale, n_nuclei, ordered ? 1 : 0, feat, stream);
}

tagi_status tagi_mlp_forward(const tagi_mlp* mlp, const uint16_t* feat, int64_t n, float* y, void* stream)
{
    return guarded_mlp([&] {
        Mlp* M = as_mlp(mlp);
        check_data(feat, n);
        TAGI_REQUIRE(y != nullptr, "y is NULL");
        run_forward(*M, feat, n, y, (cudaStream_t)stream);
    });
}

tagi_status tagi_mlp_gradient(tagi_mlp* mlp, const uint16_t* feat, const float* target, const float* wt, int64_t n,
                              double* grad, double* loss, void* stream)
{
    return guarded_mlp([&] {
        Mlp* M = as_mlp(mlp);
        check_data(feat, n);
        TAGI_REQUIRE(target != nullptr && wt != nullptr, "target or wt is NULL");
        TAGI_REQUIRE(grad != nullptr && loss != nullptr, "grad or loss is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        AllocStream as(s);
        grad_pass(*M, feat, target, wt, n, nullptr, false, s);
        TAGI_CUDA(cudaMemcpyAsync(grad, M->grad.p, sizeof(double) * M->np, cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaMemcpyAsync(loss, M->loss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
        check_mlp_err(*M, s);
    });
}

tagi_status tagi_mlp_train_step(tagi_mlp* mlp, const uint16_t* feat, const float* target, const float* wt,
                                int64_t n, const tagi_adam_params* adam, double* loss, void* stream)
{
    return guarded_mlp([&] {
        Mlp* M = as_mlp(mlp);
        check_data(feat, n);
        TAGI_REQUIRE(target != nullptr && wt != nullptr && adam != nullptr, "target, wt or adam is NULL");
        TAGI_REQUIRE(std::isfinite(adam->lr) && adam->lr >= 0.0, "lr must be >= 0");
        TAGI_REQUIRE(adam->beta1 >= 0.0 && adam->beta1 < 1.0 && adam->beta2 >= 0.0 && adam->beta2 < 1.0,
                     "beta1 and beta2 must be in [0, 1)");
        TAGI_REQUIRE(adam->eps > 0.0, "eps must be > 0");
        cudaStream_t s = (cudaStream_t)stream;
        AllocStream as(s);
        grad_pass(*M, feat, target, wt, n, adam, true, s);
        if (loss) {
            TAGI_CUDA(cudaMemcpyAsync(loss, M->loss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            TAGI_CUDA(cudaStreamSynchronize(s));
            check_mlp_err(*M, s);
        }
    });
}

tagi_status tagi_mlp_warm_start(const tagi_mlp* mlp, const uint16_t* feat, const double* s0, const double* w,
                                int64_t n, double* psi, void* stream)
{
    return guarded_mlp([&] {
        Mlp* M = as_mlp(mlp);
        check_data(feat, n);
        TAGI_REQUIRE(s0 != nullptr && w != nullptr && psi != nullptr, "s, w or psi is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        AllocStream as(s);
        DevBuf y;
        y.ensure(sizeof(float) * (size_t)n);
        run_forward(*M, feat, n, y.as<float>(), s);
        const int nb = (int)std::min<int64_t>((n + 255) / 256, 4LL * M->sms);
        M->part.ensure(sizeof(double) * nb);
        launch(k_warm_apply, nb, 256, 0, s, (const float*)y.as<float>(), s0, w, n, psi, M->part.as<double>());
        launch(k_warm_scale, (unsigned)std::min<int64_t>((n + 255) / 256, 8LL * M->sms), 256, 0, s, psi, n,
               (const double*)M->part.as<double>(), nb);
        TAGI_LAUNCH_CHECK();
    });
}

tagi_status tagi_mlp_destroy(tagi_mlp* mlp)
{
    return guarded_mlp([&] {
        if (!mlp) return;
        Mlp* M = reinterpret_cast<Mlp*>(mlp);
        TAGI_CUDA(cudaDeviceSynchronize());
        delete M;
    });
}

}  // extern "C"
