// The Green step split over target batches, for one process per GPU
// (tagi_tree_batches, tagi_fields_conv_batches, tagi_green_conv_batches,
// tagi_green_reduce).
//
// Target batches are independent once the tree, the lists and the proxy
// weights exist (Section 5.5; the paper's multi-GPU runs give each GPU a
// share of the batches, Section 5.6).  Every process builds the same tree
// from the same inputs, forms and anterpolates all fields (replicated; about
// 1% of a step), and runs the near/far kernel and the epilogue only for the
// work items of its own batches, in the same item order as the whole step,
// so each target's sums are bit for bit those of tagi_green_step.  The
// caller exchanges the results (each target is written by exactly one
// process) and then applies the reductions of Algorithm 2 lines 4-6 with
// tagi_green_reduce on the full fields.
#include <cuda_runtime.h>

#include <cmath>
#include <utility>
#include <vector>

#include "tagi_internal.cuh"

namespace tagi {
namespace {

// dst[i] = src[idx[i]], renumbered into the subset's chunk tables: chunk
// tcn[i], whose items are [item0[tcn[i]], item0[tcn[i] + 1]).
__global__ void k_gather_items(const Item* __restrict__ src, const int* __restrict__ idx, const int* __restrict__ tcn,
                               const int* __restrict__ item0, int n, Item* dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Item it = src[idx[i]];
    const int c = tcn[i];
    it.tchunk = c;
    it.i0 = item0[c];
    it.ni = item0[c + 1] - item0[c];
    dst[i] = it;
}

template <class V>
std::vector<V> to_host(const DevBuf& b, size_t count, cudaStream_t s)
{
    std::vector<V> h(count);
    if (count) TAGI_CUDA(cudaMemcpyAsync(h.data(), b.p, sizeof(V) * count, cudaMemcpyDeviceToHost, s));
    return h;
}

// While alive, the tree's work items and target chunks are those of the
// given batches only (indices into the tree's batch order); the destructor
// puts the whole tables back.
struct BatchSubset {
    Tree& T;
    DevBuf items, tc_item0, tc_t0, tc_t1;
    int64_t nitems = 0, ntchunk = 0;

    BatchSubset(Tree& t, const int32_t* batches, int nb) : T(t)
    {
        cudaStream_t s = T.stream;
        auto leaves = to_host<int>(T.leaves, (size_t)T.nleaf, s);
        auto item0 = to_host<int>(T.tc_item0, (size_t)T.ntchunk + 1, s);
        auto t0 = to_host<int>(T.tc_t0, (size_t)T.ntchunk, s);
        auto t1 = to_host<int>(T.tc_t1, (size_t)T.ntchunk, s);
        auto tb = to_host<int>(T.tc_batch, (size_t)T.ntchunk, s);
        TAGI_CUDA(cudaStreamSynchronize(s));
        std::vector<char> mark((size_t)T.nleaf, 0);
        for (int i = 0; i < nb; i++) {
            TAGI_REQUIRE(batches[i] >= 0 && batches[i] < T.nleaf, "batch index out of range");
            TAGI_REQUIRE(!mark[(size_t)batches[i]], "batch listed twice");
            mark[(size_t)batches[i]] = 1;
        }
        std::vector<int> pos((size_t)T.nc, -1);
        for (int j = 0; j < T.nleaf; j++) pos[(size_t)leaves[(size_t)j]] = j;
        std::vector<int> idx, tcn, n0, n1, ni0;
        for (int64_t c = 0; c < T.ntchunk; c++) {
            if (!mark[(size_t)pos[(size_t)tb[(size_t)c]]]) continue;
            ni0.push_back((int)idx.size());
            n0.push_back(t0[(size_t)c]);
            n1.push_back(t1[(size_t)c]);
            for (int it = item0[(size_t)c]; it < item0[(size_t)c + 1]; it++) {
                idx.push_back(it);
                tcn.push_back((int)n0.size() - 1);
            }
        }
        ni0.push_back((int)idx.size());
        nitems = (int64_t)idx.size();
        ntchunk = (int64_t)n0.size();
        DevBuf didx, dtcn;
        items.ensure(sizeof(Item) * (size_t)(nitems ? nitems : 1));
        tc_item0.ensure(sizeof(int) * (size_t)(ntchunk + 1));
        tc_t0.ensure(sizeof(int) * (size_t)(ntchunk ? ntchunk : 1));
        tc_t1.ensure(sizeof(int) * (size_t)(ntchunk ? ntchunk : 1));
        didx.ensure(sizeof(int) * (size_t)(nitems ? nitems : 1));
        dtcn.ensure(sizeof(int) * (size_t)(nitems ? nitems : 1));
        if (nitems) {
            TAGI_CUDA(cudaMemcpyAsync(didx.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
            TAGI_CUDA(cudaMemcpyAsync(dtcn.p, tcn.data(), sizeof(int) * tcn.size(), cudaMemcpyHostToDevice, s));
        }
        TAGI_CUDA(cudaMemcpyAsync(tc_item0.p, ni0.data(), sizeof(int) * ni0.size(), cudaMemcpyHostToDevice, s));
        if (ntchunk) {
            TAGI_CUDA(cudaMemcpyAsync(tc_t0.p, n0.data(), sizeof(int) * n0.size(), cudaMemcpyHostToDevice, s));
            TAGI_CUDA(cudaMemcpyAsync(tc_t1.p, n1.data(), sizeof(int) * n1.size(), cudaMemcpyHostToDevice, s));
        }
        if (nitems) {
            launch(k_gather_items, (int)((nitems + 255) / 256), 256, 0, s, T.items.as<Item>(), didx.as<int>(),
                   dtcn.as<int>(), tc_item0.as<int>(), (int)nitems, items.as<Item>());
            TAGI_LAUNCH_CHECK();
        }
        // the host vectors above are pageable: the copies have completed when
        // cudaMemcpyAsync returns, but the gather must finish before didx and
        // dtcn go
        TAGI_CUDA(cudaStreamSynchronize(s));
        swap();
    }
    ~BatchSubset() { swap(); }
    void swap()
    {
        std::swap(T.items, items);
        std::swap(T.tc_item0, tc_item0);
        std::swap(T.tc_t0, tc_t0);
        std::swap(T.tc_t1, tc_t1);
        std::swap(T.nitems, nitems);
        std::swap(T.ntchunk, ntchunk);
    }
};

template <class F>
tagi_status guarded_call(F&& f)
{
    try {
        report_error(TAGI_OK, "");
        f();
        return TAGI_OK;
    } catch (const Error& e) {
        return report_error(e.status, e.what());
    } catch (const std::bad_alloc&) {
        return report_error(TAGI_ERR_OOM, "host allocation failed");
    } catch (...) {
        return report_error(TAGI_ERR_CUDA, "unknown error");
    }
}

Tree* tree_of(tagi_tree* t)
{
    TAGI_REQUIRE(t != nullptr, "tree is NULL");
    return reinterpret_cast<Tree*>(t);
}

}  // namespace
}  // namespace tagi

using namespace tagi;

extern "C" {

tagi_status tagi_tree_batches(const tagi_tree* tree, int32_t* size, int64_t* cost)
{
    return guarded_call([&] {
        TAGI_REQUIRE(tree != nullptr, "tree is NULL");
        const Tree* T = reinterpret_cast<const Tree*>(tree);
        cudaStream_t s = T->stream;
        auto leaves = to_host<int>(T->leaves, (size_t)T->nleaf, s);
        auto beg = to_host<int>(T->cl_begin, (size_t)T->nc, s);
        auto end = to_host<int>(T->cl_end, (size_t)T->nc, s);
        auto eoff = to_host<int64_t>(T->ent_off, (size_t)T->nleaf + 1, s);
        auto ent = to_host<Entry>(T->ent, (size_t)T->nent, s);
        TAGI_CUDA(cudaStreamSynchronize(s));
        for (int j = 0; j < T->nleaf; j++) {
            const int c = leaves[(size_t)j];
            const int nb = end[(size_t)c] - beg[(size_t)c];
            int64_t src = 0;
            for (int64_t e = eoff[(size_t)j]; e < eoff[(size_t)j + 1]; e++)
                src += ent[(size_t)e].src1 - ent[(size_t)e].src0;
            if (size) size[j] = nb;
            if (cost) cost[j] = (int64_t)nb * src;
        }
    });
}

tagi_status tagi_fields_conv_batches(tagi_tree* tree, const double* f, const double* k, int nf_y, const double* rho,
                                     double* u, double* vh, const int32_t* batches, int nb, void* stream)
{
    return guarded_call([&] {
        Tree* T = tree_of(tree);
        TAGI_REQUIRE(nf_y >= 0 && nf_y + (rho ? 1 : 0) >= 1, "no field to convolve");
        TAGI_REQUIRE(nf_y + (rho ? 1 : 0) <= kMaxCallFields, "at most 128 fields per call");
        TAGI_REQUIRE(nf_y == 0 || (f != nullptr && k != nullptr && u != nullptr), "f, k or u is NULL");
        TAGI_REQUIRE(rho == nullptr || vh != nullptr, "vh is required when rho is given");
        TAGI_REQUIRE(nb >= 0 && (nb == 0 || batches != nullptr), "batches is NULL");
        for (int o = 0; o < nf_y; o++) TAGI_REQUIRE(std::isfinite(k[o]) && k[o] > 0.0, "every k must be finite and > 0");
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        const int nf = nf_y + (rho ? 1 : 0);
        const size_t n = (size_t)T->n;
        T->fbuf.ensure(sizeof(double) * nf * n);
        double* fb = T->fbuf.as<double>();
        if (nf_y) TAGI_CUDA(cudaMemcpyAsync(fb, f, sizeof(double) * nf_y * n, cudaMemcpyDeviceToDevice, T->stream));
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
        if (nb == 0) return;  // no target of this caller
        clear_err(*T);
        BatchSubset sub(*T, batches, nb);
        run_convolution(*T, fb, R, nullptr, out.data());
        read_err(*T);
    });
}

tagi_status tagi_green_conv_batches(tagi_tree* tree, const double* veff, double vshift, const double* psi,
                                    const double* eps, int nw, const double* rho, double* u, double* vh,
                                    const int32_t* batches, int nb, void* stream)
{
    return guarded_call([&] {
        Tree* T = tree_of(tree);
        TAGI_REQUIRE(veff && psi && eps && u, "veff, psi, eps or u is NULL");
        TAGI_REQUIRE(nw >= 1 && nw + (rho ? 1 : 0) <= kMaxCallFields, "need 1 <= nw <= 127");
        TAGI_REQUIRE(rho == nullptr || vh != nullptr, "vh is required when rho is given");
        TAGI_REQUIRE(nb >= 0 && (nb == 0 || batches != nullptr), "batches is NULL");
        for (int o = 0; o < nw; o++)
            TAGI_REQUIRE(std::isfinite(eps[o]) && eps[o] + vshift < 0.0, "eps + vshift must be negative (Section 3.3)");
        if (nb == 0) return;  // no target of this caller
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        const int64_t n = T->n;
        const int nf = nw + (rho ? 1 : 0);
        T->epsd.ensure(sizeof(double) * (size_t)nw);
        TAGI_CUDA(cudaMemcpyAsync(T->epsd.p, eps, sizeof(double) * nw, cudaMemcpyHostToDevice, T->stream));
        T->fbuf.ensure(sizeof(double) * (size_t)nf * n);
        double* f = T->fbuf.as<double>();
        form_fields(*T, veff, vshift, psi, nw, f);
        if (rho)
            TAGI_CUDA(cudaMemcpyAsync(f + (size_t)nw * n, rho, sizeof(double) * n, cudaMemcpyDeviceToDevice, T->stream));
        RateSrc R = host_rates(*T, nf);
        R.n_eps = nw;
        R.vshift = vshift;
        std::vector<double*> out(nf);
        for (int o = 0; o < nw; o++) out[o] = u + (size_t)o * n;
        if (rho) {
            R.kind[nw] = 1;
            R.val[nw] = T->alpha;
            out[nw] = vh;
        }
        clear_err(*T);
        BatchSubset sub(*T, batches, nb);
        run_convolution(*T, f, R, T->epsd.as<double>(), out.data());
        TAGI_REQUIRE(read_err(*T) == 0, "eps + vshift must be negative (Section 3.3)");
    });
}

tagi_status tagi_green_reduce(tagi_tree* tree, const double* veff, double vshift, double* psi, double* eps, int nw,
                              const double* u, const double* rho, const double* vh, double* resid, double* eh,
                              void* stream)
{
    return guarded_call([&] {
        Tree* T = tree_of(tree);
        TAGI_REQUIRE(veff && psi && eps && u, "veff, psi, eps or u is NULL");
        TAGI_REQUIRE(nw >= 1 && nw <= kMaxCallFields, "need 1 <= nw <= 128");
        TAGI_REQUIRE(rho == nullptr || vh != nullptr, "vh is required when rho is given");
        T->stream = (cudaStream_t)stream;
        AllocStream as(T->stream);
        const int64_t n = T->n;
        T->fbuf.ensure(sizeof(double) * (size_t)nw * n);
        T->ubuf.ensure(sizeof(double) * (size_t)nw * n);
        T->epsd.ensure(sizeof(double) * (size_t)nw);
        T->residd.ensure(sizeof(double) * (size_t)nw);
        T->ehd.ensure(sizeof(double) * 2);
        TAGI_CUDA(cudaMemcpyAsync(T->epsd.p, eps, sizeof(double) * nw, cudaMemcpyHostToDevice, T->stream));
        TAGI_CUDA(cudaMemcpyAsync(T->ubuf.p, u, sizeof(double) * (size_t)nw * n, cudaMemcpyDeviceToDevice, T->stream));
        form_fields(*T, veff, vshift, psi, nw, T->fbuf.as<double>());
        {
            ProfScope ps(kProfReduce, T->stream);
            green_reductions(*T, T->fbuf.as<double>(), psi, T->ubuf.as<double>(), nw, T->epsd.as<double>(),
                             T->residd.as<double>());
            if (rho) hartree_energy(*T, vh, rho, T->ehd.as<double>());
        }
        std::vector<double> e((size_t)nw), r((size_t)nw);
        double h = 0.0;
        TAGI_CUDA(cudaMemcpyAsync(e.data(), T->epsd.p, sizeof(double) * nw, cudaMemcpyDeviceToHost, T->stream));
        TAGI_CUDA(cudaMemcpyAsync(r.data(), T->residd.p, sizeof(double) * nw, cudaMemcpyDeviceToHost, T->stream));
        if (rho) TAGI_CUDA(cudaMemcpyAsync(&h, T->ehd.p, sizeof(double), cudaMemcpyDeviceToHost, T->stream));
        TAGI_CUDA(cudaStreamSynchronize(T->stream));
        for (int o = 0; o < nw; o++) eps[o] = e[(size_t)o];
        if (resid)
            for (int o = 0; o < nw; o++) resid[o] = r[(size_t)o];
        if (rho && eh) *eh = h;
    });
}

}  // extern "C"
