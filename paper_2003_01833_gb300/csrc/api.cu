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

void form_fields(Tree& T, const double* veff, double vshift, const double* psi, int nw, double* f);

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
}

// Convolutions of nf caller-order rows f (device) with kinds/kval; outputs out[o].
void run_convolution(Tree& T, const double* f, int nf, const int* kinds, const double* kval, double* const* out)
{
    ensure_part(T, nf);
    if (T.prec == TAGI_FP32C) {
        {
            ProfScope ps(kProfAnterp, T.stream);
            prepare_points32(T, f, nf);
            anterpolate_fields32(T, nf);
        }
        ProfScope ps(kProfInteract, T.stream);
        interact32(T, nf, kinds, kval, T.part.as<double>());
    } else {
        {
            ProfScope ps(kProfAnterp, T.stream);
            prepare_points64(T, f, nf);
            anterpolate_fields64(T, nf);
        }
        ProfScope ps(kProfInteract, T.stream);
        for (int o = 0; o < nf; o++)
            interact64(T, o, nf, kinds[o], kval[o], T.q64.as<double>() + (size_t)o * T.nrec,
                       T.c64.as<double>() + (size_t)o * T.n, T.part.as<double>());
    }
    ProfScope ps(kProfEpilogue, T.stream);
    reduce_epilogue(T, nf, kinds, kval, T.part.as<double>(), out);
}

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
        std::unique_ptr<Tree> T(new Tree());
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
        anterpolate_all_clusters64(*T, q, nq, qh);
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
        std::vector<int> kinds(nf, 0);
        std::vector<double> kv(k, k + nf);
        std::vector<double*> out(nf);
        for (int o = 0; o < nf; o++) out[o] = u + (size_t)o * T->n;
        run_convolution(*T, f, nf, kinds.data(), kv.data(), out.data());
    });
}

tagi_status tagi_coulomb_conv(tagi_tree* tree, const double* rho, double* vh, void* stream)
{
    return guarded([&] {
        Tree* T = as_tree(tree);
        TAGI_REQUIRE(rho != nullptr && vh != nullptr, "rho or vh is NULL");
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        int kind = 1;
        double a = T->alpha;
        double* out = vh;
        run_convolution(*T, rho, 1, &kind, &a, &out);
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
        std::vector<double> es(nw);
        for (int o = 0; o < nw; o++) {
            es[o] = eps[o] + vshift;
            TAGI_REQUIRE(std::isfinite(es[o]) && es[o] < 0.0, "eps + vshift must be negative (Section 3.3)");
        }
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        const int64_t n = T->n;
        const int nf = nw + (rho ? 1 : 0);
        T->fbuf.ensure(sizeof(double) * (size_t)nf * n);
        T->ubuf.ensure(sizeof(double) * (size_t)nw * n);
        double* f = T->fbuf.as<double>();
        form_fields(*T, veff, vshift, psi, nw, f);
        if (rho)
            TAGI_CUDA(cudaMemcpyAsync(f + (size_t)nw * n, rho, sizeof(double) * n, cudaMemcpyDeviceToDevice, T->stream));
        std::vector<int> kinds(nf, 0);
        std::vector<double> kv(nf);
        std::vector<double*> out(nf);
        for (int o = 0; o < nw; o++) {
            kv[o] = std::sqrt(-2.0 * es[o]);
            out[o] = T->ubuf.as<double>() + (size_t)o * n;
        }
        if (rho) {
            kinds[nw] = 1;
            kv[nw] = T->alpha;
            out[nw] = vh;
        }
        run_convolution(*T, f, nf, kinds.data(), kv.data(), out.data());
        {
            ProfScope ps(kProfReduce, T->stream);
            green_reductions(*T, f, psi, T->ubuf.as<double>(), nw, es.data(), resid);
        }
        for (int o = 0; o < nw; o++) eps[o] = es[o] - vshift;
        if (rho && eh) *eh = 0.5 * weighted_dot(*T, vh, rho);
    });
}

}  // extern "C"
