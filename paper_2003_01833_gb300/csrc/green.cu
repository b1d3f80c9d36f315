// Field preparation, the singularity-subtraction epilogue and the float64
// reductions of the Green step (Algorithm 2 lines 3-6, Eq. gradient-free,
// Eq. quadrature-example).
//
// All reductions are two-stage with a fixed grid and a fixed summation order,
// so results are bitwise reproducible run to run.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "tagi_internal.cuh"

namespace tagi {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 608;  // 4 per SM on a 152-SM GB300
constexpr double kPi = 3.14159265358979323846;

inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Two-float split of each field value, f = fh + fl, and the rounded charge
// f w for the anterpolation.
__global__ void k_prepare32(const double* __restrict__ f, int nf, int64_t n, const int* __restrict__ perm,
                            const double* __restrict__ pw, float* fa, int64_t lda, float* fb, float* qa)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nf) return;
    int64_t o = i / n, p = i % n;
    double v = f[o * n + perm[p]];
    float h = (float)v;
    fa[o * lda + p] = h;
    fb[o * n + p] = (float)(v - (double)h);
    qa[o * n + p] = (float)(v * pw[p]);
}

__global__ void k_prepare64(const double* __restrict__ f, int nf, int64_t n, const int* __restrict__ perm,
                            const double* __restrict__ pw, double* q, int64_t ldq, double* c)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nf) return;
    int64_t o = i / n, p = i % n;
    double v = f[o * n + perm[p]];
    q[o * ldq + p] = v * pw[p];
    c[o * n + p] = v;
}

struct EpiField {
    double* out;
    double cfac;  // factor on the analytic SS term: 1 + the kernel's measured mean bias
    int kind;
    int pad;
};
constexpr int kEpiMax = 32;
struct EpiFields {
    EpiField f[kEpiMax];
};

// One CTA per target chunk: the chunk's sum of item partials (formed by the
// near/far kernel), plus the SS constant and the kernel normalisation,
// scattered to the caller's order.
__global__ void k_epilogue(EpiFields E, const double* __restrict__ kvd, int nf_g, int field0, int nf_tot,
                           const int* __restrict__ tc_t0, const int* __restrict__ tc_t1, const int* __restrict__ perm,
                           const double* __restrict__ tsum, const float* __restrict__ c32, int64_t ldc32,
                           const double* __restrict__ c64, int64_t n, int ss)
{
    const int tc = blockIdx.x;
    const int t = tc_t0[tc] + threadIdx.x;
    if (t >= tc_t1[tc]) return;
    const int dest = perm[t];
    for (int g = 0; g < nf_g; g++) {
        const int o = field0 + g;
        const double S = tsum[((size_t)tc * nf_tot + o) * kTargetsPerItem + threadIdx.x];
        const double c = c32 ? (double)c32[(size_t)o * ldc32 + t] : c64[(size_t)o * n + t];
        const EpiField F = E.f[g];
        const double kv = kvd[o];  // k (Yukawa) or alpha (Coulomb), as the kernel applied them
        double u;
        if (F.kind == 0)  // G_k = e^{-kr}/(4 pi r); SS constant 4 pi c / k^2 over 4 pi
            u = S / (4.0 * kPi) + (ss ? F.cfac * c / (kv * kv) : 0.0);
        else  // Coulomb; SS constant 2 pi alpha^2 c (Eq. correction_term)
            u = S + (ss ? F.cfac * 2.0 * kPi * kv * kv * c : 0.0);
        F.out[dest] = u;
    }
}

// ---------------------------------------------------------------- dots
constexpr int kDotMax = 16;
struct DotJobs {
    DotJob j[kDotMax];
};

// D_j = sum_i (x_j - zx_j)_i (y_j - zy_j)_i w_i ; zx / zy may be null.
__global__ void k_dot1(DotJobs J, int nj, const double* __restrict__ w, int64_t n, double* part)
{
    __shared__ double sm[kRedThreads];
    for (int j = 0; j < nj; j++) {
        const DotJob d = J.j[j];
        double s = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
            double a = d.x[i] - (d.zx ? d.zx[i] : 0.0);
            double b = d.y[i] - (d.zy ? d.zy[i] : 0.0);
            s += a * b * w[i];
        }
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int off = kRedThreads / 2; off > 0; off >>= 1) {
            if (threadIdx.x < off) sm[threadIdx.x] += sm[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = sm[0];
        __syncthreads();
    }
}

__global__ void k_dot2(const double* part, int nblk, double* out)
{
    __shared__ double sm[kRedThreads];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kRedThreads) s += part[(size_t)j * nblk + b];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int off = kRedThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sm[threadIdx.x] += sm[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = sm[0];
}

__global__ void k_form(const double* __restrict__ veff, double vshift, const double* __restrict__ psi, int nw,
                       int64_t n, double* f)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n * nw) f[i] = (veff[i % n] + vshift) * psi[i];
}

__global__ void k_scale(double* a, int64_t n, double s)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] *= s;
}

// y -= d[0] * x
__global__ void k_axpy_dev(const double* __restrict__ x, double* y, int64_t n, const double* d)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] -= d[0] * x[i];
}

// y /= sqrt(d[0])
__global__ void k_normalize(double* y, int64_t n, const double* d)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] /= sqrt(d[0]);
}

}  // namespace

void weighted_dots(Tree& T, const std::vector<DotJob>& jobs, double* out_dev)
{
    cudaStream_t s = T.stream;
    T.scratch.ensure(sizeof(double) * kDotMax * kRedBlocks);
    for (size_t j0 = 0; j0 < jobs.size(); j0 += kDotMax) {
        DotJobs J{};
        int nj = (int)std::min<size_t>(kDotMax, jobs.size() - j0);
        for (int j = 0; j < nj; j++) J.j[j] = jobs[j0 + j];
        launch(k_dot1, kRedBlocks, kRedThreads, 0, s, J, nj, T.wc.as<double>(), T.n, T.scratch.as<double>());
        launch(k_dot2, nj, kRedThreads, 0, s, T.scratch.as<double>(), kRedBlocks, out_dev + j0);
        TAGI_LAUNCH_CHECK();
    }
}

void prepare_points32(Tree& T, const double* f, int nf)
{
    T.fa.ensure(sizeof(float) * (size_t)nf * T.nrec);
    T.fb.ensure(sizeof(float) * (size_t)nf * T.n);
    T.qant.ensure(sizeof(float) * (size_t)nf * T.n);
    launch(k_prepare32, nblocks(T.n * nf, 256), 256, 0, T.stream, f, nf, T.n, T.perm.as<int>(), T.pw.as<double>(),
                                                             T.fa.as<float>(), T.nrec, T.fb.as<float>(),
                                                             T.qant.as<float>());
    TAGI_LAUNCH_CHECK();
}

void prepare_points64(Tree& T, const double* f, int nf)
{
    T.q64.ensure(sizeof(double) * (size_t)nf * T.nrec);
    T.c64.ensure(sizeof(double) * (size_t)nf * T.n);
    launch(k_prepare64, nblocks(T.n * nf, 256), 256, 0, T.stream, f, nf, T.n, T.perm.as<int>(), T.pw.as<double>(),
                                                             T.q64.as<double>(), T.nrec, T.c64.as<double>());
    TAGI_LAUNCH_CHECK();
}

// Decay rates of one call, on the device: kyd[o] = fl32(-k_o log2 e) for
// Yukawa fields and fl32(-log2 e / alpha^2) for the Coulomb field (the
// float32 kernel's exponent factors); kvd[o] = the k or alpha the kernel
// therefore applies (FP32C) or the exact one (FP64).  The first n_eps fields
// take k = sqrt(-2 (eps_o + vshift)) from device eigenvalues; a
// non-positive eps + vshift sets *err.
__global__ void k_make_rates(RateSrc R, const double* __restrict__ eps_dev, float* kyd, double* kvd, int* err)
{
    const int o = threadIdx.x + blockIdx.x * blockDim.x;
    if (o >= R.nf) return;
    const double L2E = 1.4426950408889634;
    double v;
    if (o < R.n_eps) {
        const double es = eps_dev[o] + R.vshift;
        if (!(es < 0.0)) atomicOr(err, 1);
        v = sqrt(-2.0 * es);
    } else {
        v = R.val[o];
    }
    if (R.kind[o] == 0) {
        const float ky = (float)(-v * L2E);
        kyd[o] = ky;
        kvd[o] = R.fp32 ? -(double)ky / L2E : v;
    } else {
        const float ga = (float)(-L2E / (v * v));
        kyd[o] = ga;
        kvd[o] = R.fp32 ? sqrt(-L2E / (double)ga) : v;
    }
}

void make_rates(Tree& T, const RateSrc& R, const double* eps_dev)
{
    T.rates32.ensure(sizeof(float) * kMaxCallFields);
    T.rates64.ensure(sizeof(double) * kMaxCallFields);
    launch(k_make_rates, 1, kMaxCallFields, 0, T.stream, R, eps_dev, T.rates32.as<float>(), T.rates64.as<double>(),
           T.errflag.as<int>());
    TAGI_LAUNCH_CHECK();
}

void reduce_epilogue(Tree& T, int nf, const int* kinds, const double* tsum, double* const* out)
{
    const bool fp32 = T.prec == TAGI_FP32C;
    // FP32C: the subtracted sum c_i sum_j G~ w_j carries the mean bias beta of
    // the float32 kernel values, and cancels against the analytic SS term; the
    // analytic term gets the same factor (1 + beta) and the decay rate the
    // kernel applied (make_rates), so the subtraction telescopes.
    double by = 0.0, bg = 0.0;
    if (fp32) fp32_bias(T.stream, &by, &bg);
    for (int g0 = 0; g0 < nf; g0 += kEpiMax) {
        int g = std::min(kEpiMax, nf - g0);
        EpiFields E{};
        for (int u = 0; u < g; u++) {
            const int kind = kinds[g0 + u];
            const double cf = fp32 ? 1.0 + (kind == 0 ? by : bg) : 1.0;
            E.f[u] = EpiField{out[g0 + u], cf, kind, 0};
        }
        launch(k_epilogue, (int)T.ntchunk, kTargetsPerItem, 0, T.stream, E, (const double*)T.rates64.as<double>(),
               g, g0, nf, T.tc_t0.as<int>(), T.tc_t1.as<int>(), T.perm.as<int>(), tsum,
               fp32 ? T.fa.as<float>() : nullptr, T.nrec, fp32 ? nullptr : T.c64.as<double>(), T.n, T.ss);
        TAGI_LAUNCH_CHECK();
    }
}

void form_fields(Tree& T, const double* veff, double vshift, const double* psi, int nw, double* f)
{
    launch(k_form, nblocks(T.n * nw, 256), 256, 0, T.stream, veff, vshift, psi, nw, T.n, f);
    TAGI_LAUNCH_CHECK();
}

namespace {
// eps_o -= a_o / b_o (Eq. gradient-free; the gauge shift cancels)
__global__ void k_eps_update_dev(double* eps, const double* dots, int nw)
{
    int o = threadIdx.x + blockIdx.x * blockDim.x;
    if (o < nw) eps[o] -= dots[2 * o] / dots[2 * o + 1];
}
__global__ void k_sqrt_copy(const double* a, double* out, int n)
{
    int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (i < n) out[i] = sqrt(a[i]);
}
__global__ void k_half(const double* a, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = 0.5 * a[0];
}
}  // namespace

// v <- v - <v, b_p>_w b_p for each basis vector in order (modified
// Gram-Schmidt), then v <- v / ||v||_w.  scalar: one device double.
void orthonormalize(Tree& T, double* v, const std::vector<const double*>& basis, double* scalar)
{
    cudaStream_t s = T.stream;
    const int64_t n = T.n;
    const int nb = nblocks(n, 256);
    for (const double* b : basis) {
        weighted_dots(T, {DotJob{v, nullptr, b, nullptr}}, scalar);
        launch(k_axpy_dev, nb, 256, 0, s, b, v, n, (const double*)scalar);
    }
    weighted_dots(T, {DotJob{v, nullptr, v, nullptr}}, scalar);
    launch(k_normalize, nb, 256, 0, s, v, n, (const double*)scalar);
    TAGI_LAUNCH_CHECK();
}

// Green step reductions, all on the device and without host synchronisation:
// eps_dev (unshifted) updated in place, resid_dev[o] = ||psi_new - psi_old||_w.
void green_reductions(Tree& T, const double* f, double* psi, double* u, int nw, double* eps_dev,
                      double* resid_dev)
{
    cudaStream_t s = T.stream;
    const int64_t n = T.n;
    // psi~ = -2 u (Eq. Yukawa)
    launch(k_scale, nblocks(n * nw, 256), 256, 0, s, u, n * nw, -2.0);
    TAGI_LAUNCH_CHECK();
    T.dots.ensure(sizeof(double) * (2 * (size_t)nw + 8));
    double* dots = T.dots.as<double>();  // 2 nw
    double* one = dots + 2 * nw;         // scalar
    // gradient-free update uses psi~ before orthogonalisation
    std::vector<DotJob> jobs;
    for (int o = 0; o < nw; o++) {
        jobs.push_back(DotJob{f + o * n, nullptr, psi + o * n, u + o * n});
        jobs.push_back(DotJob{u + o * n, nullptr, u + o * n, nullptr});
    }
    weighted_dots(T, jobs, dots);
    launch(k_eps_update_dev, 1, 64 * ((nw + 63) / 64), 0, s, eps_dev, (const double*)dots, nw);
    TAGI_LAUNCH_CHECK();
    // modified Gram-Schmidt in index order under <a, b>_w
    std::vector<const double*> basis;
    for (int o = 0; o < nw; o++) {
        orthonormalize(T, u + o * n, basis, one);
        basis.push_back(u + o * n);
    }
    // residual ||psi_new - psi_old||_w, then psi <- psi_new
    jobs.clear();
    for (int o = 0; o < nw; o++) jobs.push_back(DotJob{u + o * n, psi + o * n, u + o * n, psi + o * n});
    weighted_dots(T, jobs, dots);
    if (resid_dev) launch(k_sqrt_copy, 1, 64 * ((nw + 63) / 64), 0, s, (const double*)dots, resid_dev, nw);
    TAGI_CUDA(cudaMemcpyAsync(psi, u, sizeof(double) * n * nw, cudaMemcpyDeviceToDevice, s));
    TAGI_LAUNCH_CHECK();
}

// eh_dev = 1/2 <vh, rho>_w on the device
void hartree_energy(Tree& T, const double* vh, const double* rho, double* eh_dev)
{
    T.dots2.ensure(sizeof(double) * 8);
    weighted_dots(T, {DotJob{vh, nullptr, rho, nullptr}}, T.dots2.as<double>());
    launch(k_half, 1, 32, 0, T.stream, (const double*)T.dots2.as<double>(), eh_dev);
    TAGI_LAUNCH_CHECK();
}

}  // namespace tagi
