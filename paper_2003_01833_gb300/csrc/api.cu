// C ABI of libtagi: argument validation, object lifetime, error reporting,
// and the sequence of kernels behind each entry point.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "tagi_internal.cuh"

namespace tagi {


namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct ProfRec {
    cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof_pending[kProfN];
double g_prof_ms[kProfN];
int64_t g_prof_n[kProfN];
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(int g, cudaStream_t s) : group(g), stream(s)
{
    if (!g_prof_on.load()) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        a = b = nullptr;
        return;
    }
    cudaEventRecord(a, stream);
}

ProfScope::~ProfScope()
{
    if (!a) return;
    cudaEventRecord(b, stream);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending[group].push_back(ProfRec{a, b});
}

namespace {

thread_local std::string g_err;

tagi_status fail(const Error& e)
{
    g_err = e.what();
    return e.status;
}

}  // namespace

tagi_status report_error(tagi_status status, const char* msg)
{
    g_err = msg;
    return status;
}

namespace {

template <class F>
tagi_status guarded(F&& f)
{
    try {
        g_err.clear();
        f();
        return TAGI_OK;
    } catch (const Error& e) {
        return fail(e);
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return TAGI_ERR_OOM;
    } catch (const std::exception& e) {
        g_err = e.what();
        return TAGI_ERR_CUDA;
    } catch (...) {
        g_err = "unknown error";
        return TAGI_ERR_CUDA;
    }
}

Tree* as_tree(tagi_tree* t)
{
    TAGI_REQUIRE(t != nullptr, "tree is NULL");
    return reinterpret_cast<Tree*>(t);
}
const Tree* as_tree(const tagi_tree* t)
{
    TAGI_REQUIRE(t != nullptr, "tree is NULL");
    return reinterpret_cast<const Tree*>(t);
}

void ensure_part(Tree& T, int nf)
{
    T.part.ensure(sizeof(double) * (size_t)T.nitems * nf * kTargetsPerItem);
    T.tsum.ensure(sizeof(double) * (size_t)(T.ntchunk ? T.ntchunk : 1) * nf * kTargetsPerItem);
    // the chunk counters must start at zero; the kernels leave them at zero
    const size_t cb = sizeof(int) * (size_t)(T.ntchunk ? T.ntchunk : 1);
    const void* before = T.tc_cnt.p;
    T.tc_cnt.ensure(cb);
    if (T.tc_cnt.p != before) TAGI_CUDA(cudaMemsetAsync(T.tc_cnt.p, 0, T.tc_cnt.bytes, T.stream));
}

}  // namespace

// Convolutions of nf caller-order rows f (device): rates from R (and eps_dev
// for the first R.n_eps fields), outputs out[o].  Enqueued on T.stream, no
// host synchronisation.
void run_convolution(Tree& T, const double* f, const RateSrc& R, const double* eps_dev, double* const* out)
{
    const int nf = R.nf;
    ensure_part(T, nf);
    make_rates(T, R, eps_dev);
    if (T.prec == TAGI_FP32C) {
        {
            ProfScope ps(kProfAnterp, T.stream);
            prepare_points32(T, f, nf);
            anterpolate_fields32(T, nf);
        }
        ProfScope ps(kProfInteract, T.stream);
        interact32(T, nf, R.kind, T.rates32.as<float>(), T.part.as<double>(), T.tsum.as<double>(), T.tc_cnt.as<int>());
    } else {
        {
            ProfScope ps(kProfAnterp, T.stream);
            prepare_points64(T, f, nf);
            anterpolate_fields64(T, nf);
        }
        ProfScope ps(kProfInteract, T.stream);
        for (int o = 0; o < nf; o++)
            interact64(T, o, nf, R.kind[o], T.rates64.as<double>(), T.q64.as<double>() + (size_t)o * T.nrec,
                       T.c64.as<double>() + (size_t)o * T.n, T.part.as<double>(), T.tsum.as<double>(),
                       T.tc_cnt.as<int>());
    }
    ProfScope ps(kProfEpilogue, T.stream);
    reduce_epilogue(T, nf, R.kind, T.tsum.as<double>(), out);
}

RateSrc host_rates(const Tree& T, int nf)
{
    TAGI_REQUIRE(nf >= 1 && nf <= kMaxCallFields, "at most 128 fields per call");
    RateSrc R{};
    R.nf = nf;
    R.fp32 = T.prec == TAGI_FP32C;
    return R;
}

// errflag[0]: argument checks of the current call (cleared by every call);
// errflag[1]: sticky, set when a bounded device wait gave up (reported by the
// next call that reads the flags).
void clear_err(Tree& T)
{
    if (!T.errflag.p) {
        T.errflag.ensure(16);
        TAGI_CUDA(cudaMemsetAsync(T.errflag.p, 0, 16, T.stream));
    } else {
        TAGI_CUDA(cudaMemsetAsync(T.errflag.p, 0, 4, T.stream));
    }
}

int read_err(Tree& T)
{
    int h[2] = {0, 0};
    TAGI_CUDA(cudaMemcpyAsync(h, T.errflag.p, 8, cudaMemcpyDeviceToHost, T.stream));
    TAGI_CUDA(cudaStreamSynchronize(T.stream));
    if (h[1]) throw Error(TAGI_ERR_TIMEOUT, "a bounded wait of the tensor-core anterpolation gave up");
    return h[0];
}

namespace {

// One Green iteration with every per-iteration value on the device (eps_dev,
// resid_dev, eh_dev): the sequence a captured graph replays.
void green_step_device(Tree& T, const double* veff, double vshift, double* psi, double* eps_dev, int nw,
                       const double* rho, double* vh, double* resid_dev, double* eh_dev)
{
    const int64_t n = T.n;
    const int nf = nw + (rho ? 1 : 0);
    TAGI_REQUIRE(nf <= kMaxCallFields, "at most 127 orbitals per Green step");
    T.fbuf.ensure(sizeof(double) * (size_t)nf * n);
    T.ubuf.ensure(sizeof(double) * (size_t)nw * n);
    double* f = T.fbuf.as<double>();
    form_fields(T, veff, vshift, psi, nw, f);
    if (rho)
        TAGI_CUDA(cudaMemcpyAsync(f + (size_t)nw * n, rho, sizeof(double) * n, cudaMemcpyDeviceToDevice, T.stream));
    RateSrc R = host_rates(T, nf);
    R.n_eps = nw;
    R.vshift = vshift;
    std::vector<double*> out(nf);
    for (int o = 0; o < nw; o++) out[o] = T.ubuf.as<double>() + (size_t)o * n;
    if (rho) {
        R.kind[nw] = 1;
        R.val[nw] = T.alpha;
        out[nw] = vh;
    }
    run_convolution(T, f, R, eps_dev, out.data());
    ProfScope ps(kProfReduce, T.stream);
    green_reductions(T, f, psi, T.ubuf.as<double>(), nw, eps_dev, resid_dev);
    if (rho && eh_dev) hartree_energy(T, vh, rho, eh_dev);
}

struct GreenGraph {
    Tree* T = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
};

}  // namespace
}  // namespace tagi

using namespace tagi;

extern "C" {

const char* tagi_last_error(void) { return g_err.c_str(); }

const char* tagi_version(void) { return "tagi-gb300 0.1 (sm_103a)"; }

int64_t tagi_kernel_launches(void) { return g_launches.load(); }

tagi_status tagi_profile_enable(int on)
{
    return guarded([&] {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_on.store(on ? 1 : 0);
        for (int g = 0; g < kProfN; g++) {
            for (auto& r : g_prof_pending[g]) {
                cudaEventDestroy(r.a);
                cudaEventDestroy(r.b);
            }
            g_prof_pending[g].clear();
            g_prof_ms[g] = 0.0;
            g_prof_n[g] = 0;
        }
    });
}

tagi_status tagi_fp32_bias(double* beta_yukawa, double* beta_gauss, void* stream)
{
    return guarded([&] {
        AllocStream as((cudaStream_t)stream);
        double a = 0.0, b = 0.0;
        fp32_bias((cudaStream_t)stream, &a, &b);
        if (beta_yukawa) *beta_yukawa = a;
        if (beta_gauss) *beta_gauss = b;
    });
}

tagi_status tagi_profile_read(int group, double* ms, int64_t* count)
{
    return guarded([&] {
        TAGI_REQUIRE(group >= 0 && group < kProfN, "unknown profile group");
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto& r : g_prof_pending[group]) {
            float t = 0.0f;
            TAGI_CUDA(cudaEventSynchronize(r.b));
            TAGI_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
            g_prof_ms[group] += t;
            g_prof_n[group]++;
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        g_prof_pending[group].clear();
        if (ms) *ms = g_prof_ms[group];
        if (count) *count = g_prof_n[group];
    });
}

tagi_status tagi_tree_build(const double* xyz, const double* w, int64_t n, const tagi_params* params,
                            void* stream, tagi_tree** out)
{
    return guarded([&] {
        TAGI_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        TAGI_REQUIRE(params != nullptr, "params is NULL");
        TAGI_REQUIRE(xyz != nullptr && w != nullptr, "xyz or w is NULL");
        TAGI_REQUIRE(n >= 1, "n must be >= 1");
        const tagi_params& p = *params;
        TAGI_REQUIRE(std::isfinite(p.theta) && p.theta >= 0.0 && p.theta < 1.0, "theta must be in [0, 1)");
        TAGI_REQUIRE(p.degree >= 1 && p.degree <= kMaxDegree, "degree must be in [1, 9]");
        TAGI_REQUIRE(p.leaf_size >= 1, "leaf_size must be >= 1");
        TAGI_REQUIRE(p.batch_size == 0 || p.batch_size == p.leaf_size, "batch_size must equal leaf_size (or be 0)");
        TAGI_REQUIRE(p.prec == TAGI_FP64 || p.prec == TAGI_FP32C, "prec must be TAGI_FP64 or TAGI_FP32C");
        TAGI_REQUIRE(p.ss == 0 || p.ss == 1, "ss must be 0 or 1");
        TAGI_REQUIRE(std::isfinite(p.alpha) && p.alpha > 0.0, "alpha must be finite and > 0");
        TAGI_REQUIRE(p.segment == 0 || (p.segment >= 1024 && p.segment <= 65536), "segment must be 0 or in [1024, 65536]");
        std::unique_ptr<Tree> T(new Tree());
        T->segment = p.segment ? p.segment : 8192;
        T->n = n;
        T->theta = p.theta;
        T->degree = p.degree;
        T->leaf_size = p.leaf_size;
        T->prec = p.prec;
        T->ss = p.ss;
        T->alpha = p.alpha;
        T->P = (p.degree + 1) * (p.degree + 1) * (p.degree + 1);
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        ProfScope ps(kProfBuild, T->stream);
        build_tree(*T, xyz, w);
        T->wc.ensure(8 * (size_t)n);
        TAGI_CUDA(cudaMemcpyAsync(T->wc.p, w, 8 * (size_t)n, cudaMemcpyDeviceToDevice, T->stream));
        TAGI_CUDA(cudaStreamSynchronize(T->stream));
        *out = reinterpret_cast<tagi_tree*>(T.release());
    });
}

tagi_status tagi_tree_destroy(tagi_tree* tree)
{
    return guarded([&] {
        if (!tree) return;
        Tree* T = reinterpret_cast<Tree*>(tree);
        // the tree's buffers may have served calls on several streams; wait
        // for all of them before the blocks go back to the cache
        cudaDeviceSynchronize();
        delete T;
    });
}

tagi_status tagi_tree_info(const tagi_tree* tree, tagi_tree_stats* st)
{
    return guarded([&] {
        const Tree* T = as_tree(tree);
        TAGI_REQUIRE(st != nullptr, "stats is NULL");
        TAGI_CUDA(cudaStreamSynchronize(T->stream));
        st->n_points = T->n;
        st->n_clusters = T->nc;
        st->n_leaves = T->nleaf;
        st->depth = T->depth;
        st->n_far_clusters = T->nfar;
        st->n_list_entries = T->nent;
        st->n_items = T->nitems;
        st->near_pairs = T->near_pairs;
        st->far_pairs = T->far_pairs;
        st->degree = T->degree;
        st->n_proxies = T->P;
        st->near_pairs_nogauss = T->near_pairs_ng;
        st->far_pairs_nogauss = T->far_pairs_ng;
        st->ant_points = T->ant_points;
    });
}

tagi_status tagi_tree_export(const tagi_tree* tree, int32_t* perm, int32_t* begin, int32_t* end, double* lo,
                             double* hi, int32_t* parent, int32_t* nchild, int32_t* child)
{
    return guarded([&] {
        const Tree* T = as_tree(tree);
        cudaStream_t s = T->stream;
        const size_t nc = (size_t)T->nc;
        if (perm) TAGI_CUDA(cudaMemcpyAsync(perm, T->perm.p, 4 * (size_t)T->n, cudaMemcpyDeviceToHost, s));
        if (begin) TAGI_CUDA(cudaMemcpyAsync(begin, T->cl_begin.p, 4 * nc, cudaMemcpyDeviceToHost, s));
        if (end) TAGI_CUDA(cudaMemcpyAsync(end, T->cl_end.p, 4 * nc, cudaMemcpyDeviceToHost, s));
        if (lo) TAGI_CUDA(cudaMemcpyAsync(lo, T->cl_lo.p, 24 * nc, cudaMemcpyDeviceToHost, s));
        if (hi) TAGI_CUDA(cudaMemcpyAsync(hi, T->cl_hi.p, 24 * nc, cudaMemcpyDeviceToHost, s));
        if (parent) TAGI_CUDA(cudaMemcpyAsync(parent, T->cl_parent.p, 4 * nc, cudaMemcpyDeviceToHost, s));
        if (nchild) TAGI_CUDA(cudaMemcpyAsync(nchild, T->cl_nchild.p, 4 * nc, cudaMemcpyDeviceToHost, s));
        if (child) TAGI_CUDA(cudaMemcpyAsync(child, T->cl_child.p, 32 * nc, cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
    });
}

tagi_status tagi_tree_lists(const tagi_tree* tree, int64_t cap, int32_t* batch, int32_t* cluster, int32_t* kind,
                            int64_t* count)
{
    return guarded([&] {
        const Tree* T = as_tree(tree);
        TAGI_REQUIRE(count != nullptr, "count is NULL");
        *count = T->nent;
        const int64_t m = std::min(cap, T->nent);
        if (m <= 0) return;
        TAGI_REQUIRE(batch && cluster && kind, "output arrays are NULL");
        cudaStream_t s = T->stream;
        std::vector<Entry> e((size_t)m);
        TAGI_CUDA(cudaMemcpyAsync(batch, T->ent_batch.p, 4 * (size_t)m, cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaMemcpyAsync(cluster, T->ent_clus.p, 4 * (size_t)m, cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaMemcpyAsync(e.data(), T->ent.p, sizeof(Entry) * (size_t)m, cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < m; i++) kind[i] = (e[(size_t)i].flags & 2) ? 1 : 0;
    });
}

tagi_status tagi_anterpolate(tagi_tree* tree, const double* q, int nq, double* qh, void* stream)
{
    return guarded([&] {
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(q != nullptr && qh != nullptr, "q or qh is NULL");
        TAGI_REQUIRE(nq >= 1, "nq must be >= 1");
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        if (T->prec == TAGI_FP32C) {
            clear_err(*T);
            anterpolate_all_clusters32(*T, q, nq, qh);
            read_err(*T);
        } else {
            anterpolate_all_clusters64(*T, q, nq, qh);
        }
    });
}

tagi_status tagi_yukawa_conv(tagi_tree* tree, const double* f, const double* k, int nf, double* u, void* stream)
{
    return guarded([&] {
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(f != nullptr && k != nullptr && u != nullptr, "f, k or u is NULL");
        TAGI_REQUIRE(nf >= 1, "nf must be >= 1");
        for (int o = 0; o < nf; o++) TAGI_REQUIRE(std::isfinite(k[o]) && k[o] > 0.0, "every k must be finite and > 0");
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        RateSrc R = host_rates(*T, nf);
        for (int o = 0; o < nf; o++) R.val[o] = k[o];
        std::vector<double*> out(nf);
        for (int o = 0; o < nf; o++) out[o] = u + (size_t)o * T->n;
        clear_err(*T);
        run_convolution(*T, f, R, nullptr, out.data());
    });
}

tagi_status tagi_fields_conv(tagi_tree* tree, const double* f, const double* k, int nf_y, const double* rho,
                             double* u, double* vh, void* stream)
{
    return guarded([&] {
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(nf_y >= 0 && nf_y + (rho ? 1 : 0) >= 1, "no field to convolve");
        TAGI_REQUIRE(nf_y + (rho ? 1 : 0) <= kMaxCallFields, "at most 128 fields per call");
        TAGI_REQUIRE(nf_y == 0 || (f != nullptr && k != nullptr && u != nullptr), "f, k or u is NULL");
        TAGI_REQUIRE(rho == nullptr || vh != nullptr, "vh is required when rho is given");
        for (int o = 0; o < nf_y; o++) TAGI_REQUIRE(std::isfinite(k[o]) && k[o] > 0.0, "every k must be finite and > 0");
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        const int nf = nf_y + (rho ? 1 : 0);
        const size_t n = (size_t)T->n;
        T->fbuf.ensure(sizeof(double) * nf * n);
        double* fb = T->fbuf.as<double>();
        if (nf_y)
            TAGI_CUDA(cudaMemcpyAsync(fb, f, sizeof(double) * nf_y * n, cudaMemcpyDeviceToDevice, T->stream));
        if (rho) TAGI_CUDA(cudaMemcpyAsync(fb + nf_y * n, rho, sizeof(double) * n, cudaMemcpyDeviceToDevice, T->stream));
        RateSrc R = host_rates(*T, nf);
        std::vector<double*> out(nf);
        for (int o = 0; o < nf_y; o++) {
            R.val[o] = k[o];
            out[o] = u + o * n;
        }
        if (rho) {
            R.kind[nf_y] = 1;
            R.val[nf_y] = T->alpha;
            out[nf_y] = vh;
        }
        clear_err(*T);
        run_convolution(*T, fb, R, nullptr, out.data());
    });
}

tagi_status tagi_coulomb_conv(tagi_tree* tree, const double* rho, double* vh, void* stream)
{
    return guarded([&] {
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(rho != nullptr && vh != nullptr, "rho or vh is NULL");
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        RateSrc R = host_rates(*T, 1);
        R.kind[0] = 1;
        R.val[0] = T->alpha;
        double* out = vh;
        clear_err(*T);
        run_convolution(*T, rho, R, nullptr, &out);
    });
}

tagi_status tagi_green_step(tagi_tree* tree, const double* veff, double vshift, double* psi, double* eps, int nw,
                            const double* rho, double* vh, double* resid, double* eh, void* stream)
{
    return guarded([&] {
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(veff != nullptr && psi != nullptr && eps != nullptr, "veff, psi or eps is NULL");
        TAGI_REQUIRE(nw >= 1, "nw must be >= 1");
        TAGI_REQUIRE(std::isfinite(vshift), "vshift must be finite");
        TAGI_REQUIRE(rho == nullptr || vh != nullptr, "vh is required when rho is given");
        for (int o = 0; o < nw; o++) {
            const double es = eps[o] + vshift;
            TAGI_REQUIRE(std::isfinite(es) && es < 0.0, "eps + vshift must be negative (Section 3.3)");
        }
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        T->epsd.ensure(sizeof(double) * nw);
        T->residd.ensure(sizeof(double) * nw);
        T->ehd.ensure(sizeof(double) * 2);
        TAGI_CUDA(cudaMemcpyAsync(T->epsd.p, eps, sizeof(double) * nw, cudaMemcpyHostToDevice, T->stream));
        clear_err(*T);
        green_step_device(*T, veff, vshift, psi, T->epsd.as<double>(), nw, rho, vh, T->residd.as<double>(),
                          rho ? T->ehd.as<double>() : nullptr);
        std::vector<double> r(nw), e(nw);
        double h = 0.0;
        TAGI_CUDA(cudaMemcpyAsync(e.data(), T->epsd.p, sizeof(double) * nw, cudaMemcpyDeviceToHost, T->stream));
        TAGI_CUDA(cudaMemcpyAsync(r.data(), T->residd.p, sizeof(double) * nw, cudaMemcpyDeviceToHost, T->stream));
        if (rho) TAGI_CUDA(cudaMemcpyAsync(&h, T->ehd.p, sizeof(double), cudaMemcpyDeviceToHost, T->stream));
        TAGI_REQUIRE(read_err(*T) == 0, "eps + vshift must be negative (Section 3.3)");
        for (int o = 0; o < nw; o++) eps[o] = e[o];
        if (resid)
            for (int o = 0; o < nw; o++) resid[o] = r[o];
        if (rho && eh) *eh = h;
    });
}

tagi_status tagi_green_iterate(tagi_tree* tree, const double* veff, double vshift, double* psi, double* eps,
                               int nw, const tagi_gi_params* gp, double* resid, int* iters, tagi_gi_stats* stats,
                               void* stream)
{
    return guarded([&] {
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(veff != nullptr && psi != nullptr && eps != nullptr && gp != nullptr,
                     "veff, psi, eps or params is NULL");
        TAGI_REQUIRE(nw >= 1 && nw <= kMaxCallFields, "nw must be in [1, 128]");
        TAGI_REQUIRE(std::isfinite(vshift), "vshift must be finite");
        TAGI_REQUIRE(std::isfinite(gp->tol_gi) && gp->tol_gi >= 0.0, "tol_gi must be finite and >= 0");
        TAGI_REQUIRE(gp->max_iter >= 1, "max_iter must be >= 1");
        TAGI_REQUIRE(gp->beta > 0.0 && gp->beta <= 1.0, "beta must be in (0, 1]");
        TAGI_REQUIRE(gp->history >= 0 && gp->history <= 8, "history must be in [0, 8]");
        TAGI_REQUIRE(gp->mix_tol >= 0.0, "mix_tol must be >= 0 (INFINITY allowed)");
        TAGI_REQUIRE(gp->store_output == 0 || gp->store_output == 1, "store_output must be 0 or 1");
        for (int o = 0; o < nw; o++) {
            const double es = eps[o] + vshift;
            TAGI_REQUIRE(std::isfinite(es) && es < 0.0, "eps + vshift must be negative (Section 3.3)");
        }
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        green_iterate(*T, veff, vshift, psi, eps, nw, *gp, resid, iters, stats);
    });
}

tagi_status tagi_scf_create(tagi_tree* tree, const tagi_scf_params* p, tagi_scf** out)
{
    return guarded([&] {
        TAGI_REQUIRE(out != nullptr && p != nullptr, "params or out is NULL");
        *out = nullptr;
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(std::isfinite(p->n_electrons) && p->n_electrons > 0.0, "n_electrons must be > 0");
        TAGI_REQUIRE(std::isfinite(p->kT) && p->kT > 0.0, "kT must be > 0");
        TAGI_REQUIRE(std::isfinite(p->e_zz), "e_zz must be finite");
        TAGI_REQUIRE(p->beta > 0.0 && p->beta <= 1.0, "beta must be in (0, 1]");
        TAGI_REQUIRE(p->history >= 0 && p->history <= 8, "history must be in [0, 8]");
        TAGI_REQUIRE(std::isfinite(p->tol_gi_first) && p->tol_gi_first > 0.0 && std::isfinite(p->tol_gi_final) &&
                         p->tol_gi_final > 0.0 && p->tol_gi_ramp >= 0,
                     "tol_gi schedule must be positive");
        TAGI_REQUIRE(p->gi_max_iter >= 1, "gi_max_iter must be >= 1");
        TAGI_REQUIRE(p->gi_beta > 0.0 && p->gi_beta <= 1.0, "gi_beta must be in (0, 1]");
        TAGI_REQUIRE(p->gi_history >= 0 && p->gi_history <= 8, "gi_history must be in [0, 8]");
        TAGI_REQUIRE(p->gi_mix_tol_first >= 0.0, "gi_mix_tol_first must be >= 0");
        TAGI_REQUIRE(p->gi_store_output == 0 || p->gi_store_output == 1, "gi_store_output must be 0 or 1");
        *out = reinterpret_cast<tagi_scf*>(new Scf(T, *p));
    });
}

tagi_status tagi_scf_step(tagi_scf* scf, const double* vext, double vshift, double* rho, double* psi, double* eps,
                          int nw, double* occ, double* rho_out, tagi_scf_report* report, void* stream)
{
    return guarded([&] {
        TAGI_REQUIRE(scf != nullptr, "scf is NULL");
        Scf* S = reinterpret_cast<Scf*>(scf);
        TAGI_REQUIRE(vext != nullptr && rho != nullptr && psi != nullptr && eps != nullptr,
                     "vext, rho, psi or eps is NULL");
        TAGI_REQUIRE(nw >= 1 && nw <= kMaxCallFields, "nw must be in [1, 128]");
        TAGI_REQUIRE(S->p.n_electrons <= 2.0 * nw, "n_electrons must not exceed 2 nw");
        TAGI_REQUIRE(std::isfinite(vshift), "vshift must be finite");
        for (int o = 0; o < nw; o++) {
            const double es = eps[o] + vshift;
            TAGI_REQUIRE(std::isfinite(es) && es < 0.0, "eps + vshift must be negative (Section 3.3)");
        }
        S->T->stream = (cudaStream_t)stream;
        AllocStream as(S->T->stream);
        scf_step(*S, vext, vshift, rho, psi, eps, nw, occ, rho_out, report);
    });
}

tagi_status tagi_scf_destroy(tagi_scf* scf)
{
    return guarded([&] {
        if (!scf) return;
        Scf* S = reinterpret_cast<Scf*>(scf);
        TAGI_CUDA(cudaDeviceSynchronize());
        delete S;
    });
}

tagi_status tagi_green_graph_create(tagi_tree* tree, const double* veff, double vshift, double* psi, double* eps,
                                    int nw, const double* rho, double* vh, double* resid, double* eh, void* stream,
                                    tagi_green_graph** out)
{
    cudaStream_t s = (cudaStream_t)stream;
    bool capturing = false;
    cudaGraph_t g = nullptr;
    try {
        report_error(TAGI_OK, "");
        TAGI_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(T->prec == TAGI_FP32C, "graph capture serves the FP32C form (the plain form runs eagerly)");
        TAGI_REQUIRE(s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread,
                     "capture needs a created stream (the default streams cannot be captured)");
        TAGI_REQUIRE(veff && psi && eps && resid, "veff, psi, eps or resid is NULL");
        TAGI_REQUIRE(nw >= 1 && nw < kMaxCallFields, "need 1 <= nw < 128");
        TAGI_REQUIRE(std::isfinite(vshift), "vshift must be finite");
        TAGI_REQUIRE(rho == nullptr || (vh != nullptr && eh != nullptr), "vh and eh are required when rho is given");
        T->stream = s;
        AllocStream as(s);
        const int64_t n = T->n;
        {
            // one eager step on copies of psi and eps: sizes every buffer,
            // measures the float32 bias, and checks the eigenvalues
            DevBuf p2, e2, r2, h2;
            p2.ensure(sizeof(double) * (size_t)nw * n);
            e2.ensure(sizeof(double) * nw);
            r2.ensure(sizeof(double) * nw);
            h2.ensure(sizeof(double) * 2);
            TAGI_CUDA(cudaMemcpyAsync(p2.p, psi, sizeof(double) * nw * n, cudaMemcpyDeviceToDevice, s));
            TAGI_CUDA(cudaMemcpyAsync(e2.p, eps, sizeof(double) * nw, cudaMemcpyDeviceToDevice, s));
            clear_err(*T);
            green_step_device(*T, veff, vshift, p2.as<double>(), e2.as<double>(), nw, rho, vh, r2.as<double>(),
                              rho ? h2.as<double>() : nullptr);
            TAGI_REQUIRE(read_err(*T) == 0, "eps + vshift must be negative (Section 3.3)");
        }
        TAGI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        clear_err(*T);
        green_step_device(*T, veff, vshift, psi, eps, nw, rho, vh, resid, rho ? eh : nullptr);
        capturing = false;
        TAGI_CUDA(cudaStreamEndCapture(s, &g));
        std::unique_ptr<GreenGraph> G(new GreenGraph());
        G->T = T;
        TAGI_CUDA(cudaGraphInstantiate(&G->exec, g, 0));
        size_t nn = 0;
        TAGI_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        TAGI_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            TAGI_CUDA(cudaGraphNodeGetType(nd, &ty));
            if (ty == cudaGraphNodeTypeKernel) G->kernels++;
        }
        cudaGraphDestroy(g);
        *out = reinterpret_cast<tagi_green_graph*>(G.release());
        return TAGI_OK;
    } catch (const Error& e) {
        if (capturing) {
            cudaStreamEndCapture(s, &g);
            cudaGetLastError();
        }
        if (g) cudaGraphDestroy(g);
        return report_error(e.status, e.what());
    } catch (...) {
        if (g) cudaGraphDestroy(g);
        return report_error(TAGI_ERR_CUDA, "unknown error");
    }
}

tagi_status tagi_green_graph_launch(tagi_green_graph* graph, void* stream)
{
    return guarded([&] {
        TAGI_REQUIRE(graph != nullptr, "graph is NULL");
        GreenGraph* G = reinterpret_cast<GreenGraph*>(graph);
        TAGI_CUDA(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
        for (int64_t i = 0; i < G->kernels; i++) note_launch();
    });
}

tagi_status tagi_green_graph_check(tagi_green_graph* graph, void* stream)
{
    return guarded([&] {
        TAGI_REQUIRE(graph != nullptr, "graph is NULL");
        GreenGraph* G = reinterpret_cast<GreenGraph*>(graph);
        Tree* T = G->T;
        int h[2] = {0, 0};
        TAGI_CUDA(cudaMemcpyAsync(h, T->errflag.p, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
        TAGI_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        if (h[1]) throw Error(TAGI_ERR_TIMEOUT, "a bounded wait of the tensor-core anterpolation gave up");
        TAGI_REQUIRE(h[0] == 0, "eps + vshift became non-negative during a replay (Section 3.3)");
    });
}

tagi_status tagi_green_graph_destroy(tagi_green_graph* graph)
{
    return guarded([&] {
        if (!graph) return;
        GreenGraph* G = reinterpret_cast<GreenGraph*>(graph);
        cudaDeviceSynchronize();
        if (G->exec) cudaGraphExecDestroy(G->exec);
        delete G;
    });
}

}  // extern "C"
