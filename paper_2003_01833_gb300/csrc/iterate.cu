// Green Iteration to convergence (Algorithm 2) for several orbitals at once,
// with Anderson mixing of the eigenpairs x = (eps, psi) (Section 4.3).
//
// Per step the host reads only the residuals and the device error flag, to
// decide which orbitals converged; eigenvalues stay on the device for the
// whole loop.  The Anderson normal equations are solved by one device thread
// (at most 8 unknowns); the Gram matrix comes from the library's weighted
// inner products, with the eps component added in the solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tagi_internal.cuh"

namespace tagi {

namespace {

constexpr int kMaxHist = 8;

inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

__global__ void k_gather_eps(const double* __restrict__ eps_all, const int* __restrict__ act, int na,
                             double* __restrict__ eps_a)
{
    int a = threadIdx.x + blockIdx.x * blockDim.x;
    if (a < na) eps_a[a] = eps_all[act[a]];
}

// eps' = eps - <f, psi - psi~> / <psi~, psi~> (Eq. gradient-free; the gauge shift cancels)
__global__ void k_eps_next(const double* __restrict__ eps_a, const double* __restrict__ dots, int na,
                           double* __restrict__ eps_new)
{
    int a = threadIdx.x + blockIdx.x * blockDim.x;
    if (a < na) eps_new[a] = eps_a[a] - dots[2 * a] / dots[2 * a + 1];
}

__global__ void k_sqrt_n(const double* __restrict__ a, double* __restrict__ out, int n)
{
    int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (i < n) out[i] = sqrt(a[i]);
}

__global__ void k_scale_n(double* a, int64_t n, double s)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] *= s;
}

__global__ void k_copy_scalar(double* dst, const double* src) { *dst = *src; }

// one history entry: psi part x = psi_in, F = psi_out - psi_in; eps part in
// the small ring arrays
__global__ void k_push(const double* __restrict__ pin, const double* __restrict__ pout, int64_t n,
                       double* __restrict__ hx, double* __restrict__ hf, const double* eps_in,
                       const double* eps_out, double* hxe, double* hfe)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const double x = pin[i];
        hx[i] = x;
        hf[i] = pout[i] - x;
    }
    if (i == 0) {
        *hxe = *eps_in;
        *hfe = *eps_out - *eps_in;
    }
}

struct MixArgs {
    int m;                     // differences D_1..D_m
    int slot[kMaxHist + 1];    // ring slots, newest first: slot[j] holds x_{n-j}
    double beta;
};

// Anderson normal equations of one orbital.  gram: the psi parts of
// <D_j, D_l> for j <= l (row-major upper triangle), then of <D_j, F_n>.
// Writes coef[j] (x_next = sum_j coef_j (x_{n-j} + beta F_{n-j})) and the
// mixed eigenvalue.  Gaussian elimination with partial pivoting; a pivot
// below 1e-13 of the largest diagonal entry gives theta = 0.
__global__ void k_anderson_solve(MixArgs M, const double* __restrict__ gram, const double* __restrict__ hxe,
                                 const double* __restrict__ hfe, double* __restrict__ coef, double* __restrict__ eps_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = M.m;
    double A[kMaxHist][kMaxHist + 1];
    double th[kMaxHist];
    const double fn = hfe[M.slot[0]];
    int g = 0;
    for (int j = 0; j < m; j++)
        for (int l = j; l < m; l++) {
            const double v = gram[g++] + (fn - hfe[M.slot[j + 1]]) * (fn - hfe[M.slot[l + 1]]);
            A[j][l] = v;
            A[l][j] = v;
        }
    for (int j = 0; j < m; j++) A[j][m] = gram[g++] + (fn - hfe[M.slot[j + 1]]) * fn;
    double dmax = 0.0;
    for (int j = 0; j < m; j++) dmax = fmax(dmax, fabs(A[j][j]));
    bool ok = dmax > 0.0 && isfinite(dmax);
    for (int c = 0; c < m && ok; c++) {
        int piv = c;
        for (int r = c + 1; r < m; r++)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (!(fabs(A[piv][c]) > 1e-13 * dmax)) {
            ok = false;
            break;
        }
        if (piv != c)
            for (int k = c; k <= m; k++) {
                const double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
        for (int r = c + 1; r < m; r++) {
            const double fct = A[r][c] / A[c][c];
            for (int k = c; k <= m; k++) A[r][k] -= fct * A[c][k];
        }
    }
    for (int j = m - 1; j >= 0; j--) {
        double v = ok ? A[j][m] : 0.0;
        if (ok) {
            for (int k = j + 1; k < m; k++) v -= A[j][k] * th[k];
            v /= A[j][j];
        }
        th[j] = v;
    }
    double c0 = 1.0;
    for (int j = 0; j < m; j++) {
        c0 -= th[j];
        coef[j + 1] = th[j];
    }
    coef[0] = c0;
    double e = 0.0;
    for (int j = 0; j <= m; j++) e += coef[j] * (hxe[M.slot[j]] + M.beta * hfe[M.slot[j]]);
    *eps_out = e;
}

struct Rows {
    const double* x[kMaxHist + 1];
    const double* f[kMaxHist + 1];
};

__global__ void k_anderson_combine(Rows R, int m, double beta, const double* __restrict__ coef, int64_t n,
                                   double* __restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int j = 0; j <= m; j++) s += coef[j] * (R.x[j][i] + beta * R.f[j][i]);
    out[i] = s;
}

// ---------------------------------------------------------------- SCF kernels
// Spin-unpolarised LDA (Section 2): Slater exchange
//   eps_x = -(3/4) (3 rho/pi)^(1/3), v_x = -(3 rho/pi)^(1/3),
// and the Perdew-Zunger fit of the Ceperley-Alder correlation in
// r_s = (3/(4 pi rho))^(1/3): for r_s >= 1
//   eps_c = g/(1 + b1 sqrt(r_s) + b2 r_s), v_c = eps_c (1 + 7/6 b1 sqrt(r_s) + 4/3 b2 r_s)/(1 + b1 sqrt(r_s) + b2 r_s),
// below it eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
//   v_c = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s + (2D - C)/3 r_s.
__global__ void k_lda(const double* __restrict__ rho, int64_t n, double* __restrict__ exc, double* __restrict__ vxc)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = rho[i];
    if (!(r > 1e-30)) {
        exc[i] = 0.0;
        vxc[i] = 0.0;
        return;
    }
    const double kPi = 3.14159265358979323846;
    const double t = cbrt(3.0 * r / kPi);
    double e = -0.75 * t, v = -t;
    const double rs = cbrt(3.0 / (4.0 * kPi * r));
    if (rs >= 1.0) {
        const double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
        const double sq = sqrt(rs), den = 1.0 + b1 * sq + b2 * rs;
        const double ec = g / den;
        e += ec;
        v += ec * (1.0 + 7.0 / 6.0 * b1 * sq + 4.0 / 3.0 * b2 * rs) / den;
    } else {
        const double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
        const double ln = log(rs);
        e += A * ln + B + C * rs * ln + D * rs;
        v += A * ln + (B - A / 3.0) + 2.0 / 3.0 * C * rs * ln + (2.0 * D - C) / 3.0 * rs;
    }
    exc[i] = e;
    vxc[i] = v;
}

__global__ void k_add3(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                       int64_t n, double* __restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i] + c[i];
}

// Fermi energy by bisection (one thread): 2 sum_i f(eps_i, mu) = N_e,
// f = 1/(1 + e^{(eps - mu)/kT}).  out: mu, band energy 2 sum f eps.
__global__ void k_fermi(const double* __restrict__ eps, int nw, double ne, double kT, double* __restrict__ f,
                        double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo = eps[0], hi = eps[0];
    for (int o = 1; o < nw; o++) {
        lo = fmin(lo, eps[o]);
        hi = fmax(hi, eps[o]);
    }
    lo -= 60.0 * kT;
    hi += 60.0 * kT;
    for (int it = 0; it < 400; it++) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double s = 0.0;
        for (int o = 0; o < nw; o++) s += 1.0 / (1.0 + exp((eps[o] - mid) / kT));
        if (2.0 * s < ne)
            lo = mid;
        else
            hi = mid;
    }
    const double mu = 0.5 * (lo + hi);
    double band = 0.0;
    for (int o = 0; o < nw; o++) {
        f[o] = 1.0 / (1.0 + exp((eps[o] - mu) / kT));
        band += 2.0 * f[o] * eps[o];
    }
    out[0] = mu;
    out[1] = band;
}

// rho_out = 2 sum_o f_o psi_o^2
__global__ void k_density(const double* __restrict__ psi, const double* __restrict__ f, int nw, int64_t n,
                          double* __restrict__ rho)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int o = 0; o < nw; o++) {
        const double p = psi[(size_t)o * n + i];
        s += f[o] * p * p;
    }
    rho[i] = 2.0 * s;
}

}  // namespace

void green_iterate(Tree& T, const double* veff, double vshift, double* psi, double* eps, int nw,
                   const tagi_gi_params& gp, double* resid_out, int* iters_out, tagi_gi_stats* stats)
{
    cudaStream_t s = T.stream;
    const int64_t n = T.n;
    const int H = gp.history;
    const int ring = H + 1;
    DevBuf pa, eps_all, eps_a, eps_new, dots, res_d, act_d, hist, hring, coef;
    pa.ensure(sizeof(double) * (size_t)nw * n);
    T.fbuf.ensure(sizeof(double) * (size_t)nw * n);
    T.ubuf.ensure(sizeof(double) * (size_t)nw * n);
    eps_all.ensure(sizeof(double) * nw);
    eps_a.ensure(sizeof(double) * nw);
    eps_new.ensure(sizeof(double) * nw);
    res_d.ensure(sizeof(double) * nw);
    act_d.ensure(sizeof(int) * nw);
    dots.ensure(sizeof(double) * (2 * (size_t)nw + 8));
    coef.ensure(sizeof(double) * (kMaxHist + 1) * 2);
    double* P = pa.as<double>();
    double* F = T.fbuf.as<double>();
    double* U = T.ubuf.as<double>();
    double* one = dots.as<double>() + 2 * nw;
    TAGI_CUDA(cudaMemcpyAsync(eps_all.p, eps, sizeof(double) * nw, cudaMemcpyHostToDevice, s));
    clear_err(T);

    std::vector<char> conv(nw, 0), mixing(nw, 0);
    std::vector<int> iters(nw, -1), count(nw, 0), head(nw, -1);
    std::vector<double> resid(nw, NAN);
    std::vector<int> act, idx(nw, -1);
    std::vector<double> r_host(nw);
    int steps = 0;
    int64_t field_steps = 0;
    const int nb = nblocks(n, 256);
    const int ne = 64 * ((nw + 63) / 64);

    for (int step = 0; step < gp.max_iter; step++) {
        act.clear();
        for (int o = 0; o < nw; o++)
            if (!conv[o]) {
                idx[o] = (int)act.size();
                act.push_back(o);
            } else {
                idx[o] = -1;
            }
        const int na = (int)act.size();
        if (na == 0) break;
        steps++;
        field_steps += na;
        // inputs of this step
        TAGI_CUDA(cudaMemcpyAsync(act_d.p, act.data(), sizeof(int) * na, cudaMemcpyHostToDevice, s));
        for (int a = 0; a < na; a++)
            TAGI_CUDA(cudaMemcpyAsync(P + (size_t)a * n, psi + (size_t)act[a] * n, sizeof(double) * n,
                                      cudaMemcpyDeviceToDevice, s));
        launch(k_gather_eps, 1, ne, 0, s, (const double*)eps_all.p, (const int*)act_d.p, na, eps_a.as<double>());
        TAGI_LAUNCH_CHECK();
        // line 3: psi~ = G(eps) psi
        form_fields(T, veff, vshift, P, na, F);
        RateSrc R = host_rates(T, na);
        R.n_eps = na;
        R.vshift = vshift;
        std::vector<double*> out(na);
        for (int a = 0; a < na; a++) out[a] = U + (size_t)a * n;
        run_convolution(T, F, R, eps_a.as<double>(), out.data());
        ProfScope ps(kProfReduce, s);
        launch(k_scale_n, nblocks(n * na, 256), 256, 0, s, U, n * na, -2.0);
        // line 4: gradient-free eigenvalue update
        std::vector<DotJob> jobs;
        for (int a = 0; a < na; a++) {
            jobs.push_back(DotJob{F + (size_t)a * n, nullptr, P + (size_t)a * n, U + (size_t)a * n});
            jobs.push_back(DotJob{U + (size_t)a * n, nullptr, U + (size_t)a * n, nullptr});
        }
        weighted_dots(T, jobs, dots.as<double>());
        launch(k_eps_next, 1, ne, 0, s, (const double*)eps_a.p, (const double*)dots.p, na, eps_new.as<double>());
        TAGI_LAUNCH_CHECK();
        // lines 5-6: orthogonalise in index order against every lower-index
        // orbital (new iterate if active, stored pair if converged), normalise
        for (int a = 0; a < na; a++) {
            std::vector<const double*> basis;
            for (int p = 0; p < act[a]; p++)
                basis.push_back(idx[p] >= 0 ? U + (size_t)idx[p] * n : psi + (size_t)p * n);
            orthonormalize(T, U + (size_t)a * n, basis, one);
        }
        // line 7: residual ||psi' - psi||_w
        jobs.clear();
        for (int a = 0; a < na; a++)
            jobs.push_back(DotJob{U + (size_t)a * n, P + (size_t)a * n, U + (size_t)a * n, P + (size_t)a * n});
        weighted_dots(T, jobs, dots.as<double>());
        launch(k_sqrt_n, 1, ne, 0, s, (const double*)dots.p, res_d.as<double>(), na);
        TAGI_LAUNCH_CHECK();
        TAGI_CUDA(cudaMemcpyAsync(r_host.data(), res_d.p, sizeof(double) * na, cudaMemcpyDeviceToHost, s));
        if (read_err(T) != 0) {
            // psi and eps keep the last completed step
            TAGI_CUDA(cudaMemcpyAsync(eps, eps_all.p, sizeof(double) * nw, cudaMemcpyDeviceToHost, s));
            TAGI_CUDA(cudaStreamSynchronize(s));
            throw Error(TAGI_ERR_INVALID_ARG, "eps + vshift became non-negative during Green Iteration (Section 3.3)");
        }

        for (int a = 0; a < na; a++) {
            const int o = act[a];
            const double r = r_host[a];
            resid[o] = r;
            if (r < gp.tol_gi) {
                conv[o] = 1;
                iters[o] = step + 1;
                if (gp.store_output) {
                    TAGI_CUDA(cudaMemcpyAsync(psi + (size_t)o * n, U + (size_t)a * n, sizeof(double) * n,
                                              cudaMemcpyDeviceToDevice, s));
                    launch(k_copy_scalar, 1, 1, 0, s, eps_all.as<double>() + o,
                           (const double*)(eps_new.as<double>() + a));
                    TAGI_LAUNCH_CHECK();
                }
                continue;
            }
            if (r < gp.mix_tol) mixing[o] = 1;
            double* dst = psi + (size_t)o * n;
            if (!mixing[o]) {
                TAGI_CUDA(cudaMemcpyAsync(dst, U + (size_t)a * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                launch(k_copy_scalar, 1, 1, 0, s, eps_all.as<double>() + o, (const double*)(eps_new.as<double>() + a));
                TAGI_LAUNCH_CHECK();
                continue;
            }
            if (!hist.p) {
                hist.ensure(sizeof(double) * (size_t)nw * ring * 2 * n);
                hring.ensure(sizeof(double) * (size_t)nw * ring * 2);
            }
            double* hx = hist.as<double>() + (size_t)o * ring * 2 * n;  // ring rows of x, then of F
            double* hf = hx + (size_t)ring * n;
            double* hxe = hring.as<double>() + (size_t)o * ring * 2;
            double* hfe = hxe + ring;
            head[o] = (head[o] + 1) % ring;
            count[o] = std::min(count[o] + 1, ring);
            const int h = head[o];
            launch(k_push, nb, 256, 0, s, (const double*)(P + (size_t)a * n), (const double*)(U + (size_t)a * n), n,
                   hx + (size_t)h * n, hf + (size_t)h * n, (const double*)(eps_a.as<double>() + a),
                   (const double*)(eps_new.as<double>() + a), hxe + h, hfe + h);
            MixArgs M{};
            M.m = count[o] - 1;
            M.beta = gp.beta;
            Rows rows{};
            for (int j = 0; j <= M.m; j++) {
                M.slot[j] = (h - j + ring) % ring;
                rows.x[j] = hx + (size_t)M.slot[j] * n;
                rows.f[j] = hf + (size_t)M.slot[j] * n;
            }
            jobs.clear();
            for (int j = 1; j <= M.m; j++)
                for (int l = j; l <= M.m; l++)
                    jobs.push_back(DotJob{rows.f[0], rows.f[j], rows.f[0], rows.f[l]});
            for (int j = 1; j <= M.m; j++) jobs.push_back(DotJob{rows.f[0], rows.f[j], rows.f[0], nullptr});
            T.dots2.ensure(sizeof(double) * (kMaxHist * (kMaxHist + 3) / 2 + 8));
            if (!jobs.empty()) weighted_dots(T, jobs, T.dots2.as<double>());
            launch(k_anderson_solve, 1, 32, 0, s, M, (const double*)T.dots2.p, (const double*)hxe, (const double*)hfe,
                   coef.as<double>(), eps_all.as<double>() + o);
            launch(k_anderson_combine, nb, 256, 0, s, rows, M.m, gp.beta, (const double*)coef.p, n, dst);
            TAGI_LAUNCH_CHECK();
        }
    }
    std::vector<double> e(nw);
    TAGI_CUDA(cudaMemcpyAsync(e.data(), eps_all.p, sizeof(double) * nw, cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaStreamSynchronize(s));
    int nconv = 0;
    for (int o = 0; o < nw; o++) {
        eps[o] = e[o];
        nconv += conv[o] ? 1 : 0;
        if (resid_out) resid_out[o] = resid[o];
        if (iters_out) iters_out[o] = iters[o];
    }
    if (stats) {
        stats->steps = steps;
        stats->n_converged = nconv;
        stats->field_steps = field_steps;
    }
}

// ---------------------------------------------------------------- SCF step
Scf::Scf(Tree* t, const tagi_scf_params& prm) : T(t), p(prm) {}

void scf_step(Scf& S, const double* vext, double vshift, double* rho, double* psi, double* eps, int nw,
              double* occ, double* rho_out_user, tagi_scf_report* rep)
{
    Tree& T = *S.T;
    cudaStream_t s = T.stream;
    const int64_t n = T.n;
    const int nb = nblocks(n, 256);
    const int ring = S.p.history + 1;
    DevBuf vh, exc, vxc, veff, rho_out, fo, scal, zero, coef;
    vh.ensure(sizeof(double) * n);
    exc.ensure(sizeof(double) * n);
    vxc.ensure(sizeof(double) * n);
    veff.ensure(sizeof(double) * n);
    rho_out.ensure(sizeof(double) * n);
    fo.ensure(sizeof(double) * (nw + 1));
    scal.ensure(sizeof(double) * 16);
    zero.ensure(sizeof(double) * 2);
    coef.ensure(sizeof(double) * (kMaxHist + 1) * 2);
    TAGI_CUDA(cudaMemsetAsync(zero.p, 0, sizeof(double) * 2, s));
    double* sc = scal.as<double>();  // [0] mu [1] band [2..4] E_H, E_xc, E_vxc [5] resid^2 [8] scratch

    // line 2: V_eff[rho_in]
    {
        RateSrc R = host_rates(T, 1);
        R.kind[0] = 1;
        R.val[0] = T.alpha;
        double* out = vh.as<double>();
        clear_err(T);
        run_convolution(T, rho, R, nullptr, &out);
    }
    launch(k_lda, nb, 256, 0, s, (const double*)rho, n, exc.as<double>(), vxc.as<double>());
    launch(k_add3, nb, 256, 0, s, vext, (const double*)vh.p, (const double*)vxc.p, n, veff.as<double>());
    TAGI_LAUNCH_CHECK();
    // double-counting terms of the energy, from rho_in
    weighted_dots(T, {DotJob{vh.as<double>(), nullptr, rho, nullptr}, DotJob{exc.as<double>(), nullptr, rho, nullptr},
                      DotJob{vxc.as<double>(), nullptr, rho, nullptr}},
                  sc + 2);

    // line 3: eigenpairs by Green Iteration
    const int k = S.step;
    double tol = S.p.tol_gi_final;
    if (k <= 0)
        tol = S.p.tol_gi_first;
    else if (k < S.p.tol_gi_ramp)
        tol = S.p.tol_gi_first * std::pow(S.p.tol_gi_final / S.p.tol_gi_first, (double)k / S.p.tol_gi_ramp);
    tagi_gi_params gp{tol, S.p.gi_max_iter, S.p.gi_beta, S.p.gi_history,
                      k == 0 ? S.p.gi_mix_tol_first : (double)INFINITY, S.p.gi_store_output};
    tagi_gi_stats gst{};
    green_iterate(T, veff.as<double>(), vshift, psi, eps, nw, gp, nullptr, nullptr, &gst);
    for (int o = 0; o < nw; o++) orthonormalize(T, psi + (size_t)o * n, {}, sc + 8);

    // line 4: occupations; line 5: density
    TAGI_CUDA(cudaMemcpyAsync(fo.p, eps, sizeof(double) * nw, cudaMemcpyHostToDevice, s));
    DevBuf fv;
    fv.ensure(sizeof(double) * nw);
    launch(k_fermi, 1, 32, 0, s, (const double*)fo.p, nw, S.p.n_electrons, S.p.kT, fv.as<double>(), sc);
    launch(k_density, nb, 256, 0, s, (const double*)psi, (const double*)fv.p, nw, n, rho_out.as<double>());
    TAGI_LAUNCH_CHECK();
    // line 6: residual
    weighted_dots(T, {DotJob{rho_out.as<double>(), rho, rho_out.as<double>(), rho}}, sc + 5);
    if (rho_out_user)
        TAGI_CUDA(cudaMemcpyAsync(rho_out_user, rho_out.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));

    // line 7: Anderson mixing of the density (no scalar component)
    if (!S.hist.p) {
        S.hist.ensure(sizeof(double) * (size_t)ring * 2 * n);
        S.hring.ensure(sizeof(double) * (size_t)ring * 2);
        TAGI_CUDA(cudaMemsetAsync(S.hring.p, 0, sizeof(double) * (size_t)ring * 2, s));
    }
    double* hx = S.hist.as<double>();
    double* hf = hx + (size_t)ring * n;
    double* hxe = S.hring.as<double>();
    double* hfe = hxe + ring;
    S.head = (S.head + 1) % ring;
    S.count = std::min(S.count + 1, ring);
    const int h = S.head;
    launch(k_push, nb, 256, 0, s, (const double*)rho, (const double*)rho_out.p, n, hx + (size_t)h * n,
           hf + (size_t)h * n, (const double*)zero.p, (const double*)zero.p, hxe + h, hfe + h);
    MixArgs M{};
    M.m = S.count - 1;
    M.beta = S.p.beta;
    Rows rows{};
    for (int j = 0; j <= M.m; j++) {
        M.slot[j] = (h - j + ring) % ring;
        rows.x[j] = hx + (size_t)M.slot[j] * n;
        rows.f[j] = hf + (size_t)M.slot[j] * n;
    }
    std::vector<DotJob> jobs;
    for (int j = 1; j <= M.m; j++)
        for (int l = j; l <= M.m; l++) jobs.push_back(DotJob{rows.f[0], rows.f[j], rows.f[0], rows.f[l]});
    for (int j = 1; j <= M.m; j++) jobs.push_back(DotJob{rows.f[0], rows.f[j], rows.f[0], nullptr});
    T.dots2.ensure(sizeof(double) * (kMaxHist * (kMaxHist + 3) / 2 + 8));
    if (!jobs.empty()) weighted_dots(T, jobs, T.dots2.as<double>());
    launch(k_anderson_solve, 1, 32, 0, s, M, (const double*)T.dots2.p, (const double*)hxe, (const double*)hfe,
           coef.as<double>(), sc + 9);
    launch(k_anderson_combine, nb, 256, 0, s, rows, M.m, S.p.beta, (const double*)coef.p, n, rho);
    TAGI_LAUNCH_CHECK();

    double hs[16];
    std::vector<double> fh(nw);
    TAGI_CUDA(cudaMemcpyAsync(hs, sc, sizeof(double) * 16, cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaMemcpyAsync(fh.data(), fv.p, sizeof(double) * nw, cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaStreamSynchronize(s));
    if (occ)
        for (int o = 0; o < nw; o++) occ[o] = fh[o];
    if (rep) {
        rep->step = k;
        rep->tol_gi = tol;
        rep->mu = hs[0];
        rep->residual = std::sqrt(hs[5]);
        rep->e_band = hs[1];
        rep->e_hartree = 0.5 * hs[2];
        rep->e_xc = hs[3];
        rep->e_vxc = hs[4];
        rep->e_zz = S.p.e_zz;
        rep->e_total = rep->e_band - rep->e_hartree + rep->e_xc - rep->e_vxc + rep->e_zz;
        rep->gi = gst;
    }
    S.step++;
}

}  // namespace tagi
