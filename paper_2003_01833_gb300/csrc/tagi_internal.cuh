// Internal declarations shared by the translation units of libtagi.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tagi.h"

namespace tagi {

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
    tagi_status status;
    Error(tagi_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define TAGI_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw ::tagi::Error(e_ == cudaErrorMemoryAllocation ? TAGI_ERR_OOM : TAGI_ERR_CUDA, \
                                std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

#define TAGI_LAUNCH_CHECK() TAGI_CUDA(cudaGetLastError())

#define TAGI_REQUIRE(cond, msg)                                                   \
    do {                                                                          \
        if (!(cond)) throw ::tagi::Error(TAGI_ERR_INVALID_ARG, std::string(msg)); \
    } while (0)

// Device buffer from the caching allocator (alloc.cu); released to the cache
// of the stream it was allocated for when destroyed or regrown.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int dev = 0;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), dev(o.dev), stream(o.stream)
    {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf& operator=(DevBuf&& o) noexcept
    {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            dev = o.dev;
            stream = o.stream;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release();
    void ensure(size_t nbytes);  // grow (content not kept)
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Allocations made while an AllocStream is alive are ordered on its stream.
struct AllocStream {
    cudaStream_t prev;
    explicit AllocStream(cudaStream_t s);
    ~AllocStream();
};
void trim_cache();  // synchronises the device and frees every cached block

// Every kernel of the library is launched through launch(), which counts it
// (tagi_kernel_launches) before the <<<>>> launch.
void note_launch();
template <class... KArgs, class... Args>
inline void launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args)
{
    note_launch();
    k<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
}

// Optional CUDA-event timing of the phases of a call (tagi_profile_*).
enum ProfGroup { kProfBuild = 0, kProfAnterp = 1, kProfInteract = 2, kProfEpilogue = 3, kProfReduce = 4, kProfN = 5 };
struct ProfScope {
    int group;
    cudaStream_t stream;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(int g, cudaStream_t s);
    ~ProfScope();
};

// Limits
constexpr int kMaxDepth = 64;
constexpr int kMaxDegree = 9;
constexpr int kTargetsPerItem = 256;  // targets of one work item (one CTA)
constexpr int kAntChunk = 2048;       // points per anterpolation work item

// Decay rates of one call (make_rates): the first n_eps fields take
// k = sqrt(-2 (eps + vshift)) from device eigenvalues, the others val[o]
// (k for Yukawa, alpha for Coulomb).  kind[o]: 0 Yukawa, 1 Coulomb.
constexpr int kMaxCallFields = 128;
struct RateSrc {
    int nf, n_eps, fp32, pad;
    double vshift;
    double val[kMaxCallFields];
    int kind[kMaxCallFields];
};

// Interaction entry: a contiguous range of source records [src0, src1) seen
// from a batch.  frame: cluster whose center the records' local coordinates
// are relative to (FP32 path).  flags bit0: the range holds the batch's own
// points (self pair possible); bit1: proxies (far field).
struct Entry {
    int src0, src1, frame, flags;
};

// Work item of the near/far kernel: targets [t0, t1) of batch `batch`
// (tree positions), list entries [e0, e1); target chunk `tchunk` of the
// current chunk tables, whose items are [i0, i0 + ni) of the item array.
struct Item {
    int t0, t1, e0, e1;
    int batch, tchunk, i0, ni;
};

// Anterpolation work item: positions [p0, p1) of cluster `cluster`, whose
// proxies are record block `far` (index among approximated clusters).
struct AntItem {
    int p0, p1, cluster, far;
};

struct Tree {
    // parameters
    int64_t n = 0;
    double theta = 0.7;
    int degree = 6;
    int leaf_size = 2000;
    int prec = TAGI_FP32C;
    int ss = 1;
    double alpha = 1.0;
    int segment = 8192;  // sources per work item of the near/far kernel
    int P = 0;  // (degree+1)^3
    cudaStream_t stream = nullptr;

    // sizes
    int nc = 0, nleaf = 0, depth = 0, nfar = 0;
    int64_t nent = 0, nitems = 0, ntchunk = 0, nant = 0, nrec = 0;
    int64_t near_pairs = 0, far_pairs = 0;
    int64_t near_pairs_ng = 0, far_pairs_ng = 0;  // pairs of entries flagged bit2
    int64_t ant_points = 0;                        // sum of N_S over approximated clusters

    // points in tree order
    DevBuf perm;             // int[n] tree position -> caller index
    DevBuf px, py, pz, pw;   // double[n]
    DevBuf pt_leaf;          // int[n] leaf (batch) cluster owning each position

    // clusters
    DevBuf cl_begin, cl_end, cl_parent, cl_level, cl_nchild, cl_child;  // int
    DevBuf cl_lo, cl_hi, cl_cen;                                         // double[3*nc]
    DevBuf cl_rad;                                                       // double[nc]
    DevBuf cl_far;   // int[nc]: index among approximated clusters, or -1
    DevBuf leaves;   // int[nleaf]
    DevBuf far_cl;   // int[nfar]

    // lists (expanded): entries in batch order with CSR offsets by leaf index
    DevBuf ent;       // Entry[nent]
    DevBuf ent_off;   // int64 -> int[nleaf+1]
    DevBuf ent_batch; // int[nent] (leaf cluster id), for export
    DevBuf ent_clus;  // int[nent] (source cluster id: leaf for direct, cluster for far)

    // work items
    DevBuf items;       // Item[nitems]
    DevBuf tc_item0;    // int[ntchunk+1]: first item of each target chunk
    DevBuf tc_t0, tc_t1, tc_batch;  // int[ntchunk]
    DevBuf ant_items;   // AntItem[nant]
    DevBuf far_ant0;    // int[nfar+1]: first anterpolation item of each far cluster

    // source records (points then proxies), nrec = n + nfar * P
    DevBuf rec4;        // FP32C: float4 (dx, dy, dz, w) relative to frame center (high parts)
    DevBuf rec4lo;      // FP32C: float4 low parts of (dx, dy, dz) for the n mesh points
    DevBuf rx, ry, rz, rw;  // FP64: absolute coordinates and weight
    // per-call work buffers
    DevBuf fa;          // float [nf][nrec]: fh = f rounded (points), qh (proxies)
    DevBuf fb;          // float [nf][n]: fl = f - fh (points)
    DevBuf qant;        // float [nf][n]: f w rounded, the anterpolation input
    DevBuf q64;         // double [nf][nrec]
    DevBuf c64;         // double [nf][n] field values in tree order (FP64 SS constants)
    DevBuf wc;          // double [n] quadrature weights in the caller's order
    DevBuf part;        // double partial sums [nitems][nf][kTargetsPerItem]
    DevBuf tsum;        // double [ntchunk][nf][kTargetsPerItem]: partials summed per target chunk
    DevBuf tc_cnt;      // int [ntchunk]: items of the chunk finished in the current launch (0 between launches)
    DevBuf antpart;     // double anterpolation partials
    DevBuf antL;        // FP32C: float32 basis rows of every anterpolation point (anterp.cu)
    DevBuf qtiles;      // FP32C: charge tiles of the tensor-core anterpolation (anterp.cu)
    DevBuf scratch;     // general scratch (reductions)
    DevBuf rates32;     // float [kMaxCallFields] exponent factors of the current call
    DevBuf rates64;     // double [kMaxCallFields] k or alpha as applied by the kernels
    DevBuf errflag;     // int: set by device-side argument checks (make_rates)
    DevBuf dots, dots2; // double: Green-step inner products
    DevBuf epsd, residd, ehd;  // double: device copies for the host-value entry point
    DevBuf fbuf;        // double [nf][n] formed fields (Green step)
    DevBuf ubuf;        // double [nf][n] convolution results (Green step)

};

// tree.cu
void build_tree(Tree& T, const double* xyz, const double* w);
// anterp.cu
void anterpolate_weights(Tree& T);  // w^ for every approximated cluster (FP32C and FP64)
void anterpolate_fields32(Tree& T, int nf);  // q^ rows [0, nf) of T.fa from T.qant
void anterpolate_fields64(Tree& T, int nf);
void anterpolate_all_clusters64(Tree& T, const double* q, int nq, double* qh);
void anterpolate_all_clusters32(Tree& T, const double* q, int nq, double* qh);  // FP32C form (tensor cores)
// interact.cu
// kinds[o]: 0 = Yukawa with kval[o], 1 = Coulomb/Hartree
void interact32(Tree& T, int nf, const int* kinds, const float* kyd, double* part, double* tsum, int* cnt);
void interact64(Tree& T, int field, int nf_tot, int kind, const double* kvd, const double* q, const double* c,
                double* part, double* tsum, int* cnt);
// mean relative bias of the float32 Yukawa and Gaussian kernel values (measured)
void fp32_bias(cudaStream_t s, double* beta_y, double* beta_g);
double effective_k32(double k);
double effective_alpha32(double a);
// green.cu
void prepare_points32(Tree& T, const double* f, int nf);   // fa, fb, qant from caller-order fields
void prepare_points64(Tree& T, const double* f, int nf);   // q64 from caller-order fields
// rates of a call into T.rates32 / T.rates64 (see RateSrc)
void make_rates(Tree& T, const RateSrc& R, const double* eps_dev);
// u[o][caller i] for o in [0, nf): kinds[o] 0 = Yukawa, 1 = Coulomb, with the
// rates of the last make_rates.  out[o] points to the caller-order output row.
void reduce_epilogue(Tree& T, int nf, const int* kinds, const double* tsum, double* const* out);
void form_fields(Tree& T, const double* veff, double vshift, const double* psi, int nw, double* f);
// Green step reductions on caller-order rows, all on the device:
//   f (nw x n), psi (nw x n, in: old, out: new), u (nw x n, in: Yukawa
//   results, clobbered), eps_dev (nw, unshifted, updated), resid_dev (nw or null).
void green_reductions(Tree& T, const double* f, double* psi, double* u, int nw, double* eps_dev,
                      double* resid_dev);
void hartree_energy(Tree& T, const double* vh, const double* rho, double* eh_dev);
// Weighted inner products on the device, out[j] = sum_i (x - zx)_i (y - zy)_i w_i
// with the tree's quadrature weights in the caller's order (zx, zy may be null);
// a fixed two-stage summation order, so results are reproducible.
struct DotJob {
    const double *x, *zx, *y, *zy;
};
void weighted_dots(Tree& T, const std::vector<DotJob>& jobs, double* out_dev);
// modified Gram-Schmidt of v against basis (in order) and normalisation
void orthonormalize(Tree& T, double* v, const std::vector<const double*>& basis, double* scalar);
// api.cu: the convolution sequence (rates, fields, anterpolation, near/far,
// epilogue) of nf caller-order rows, enqueued on T.stream without host sync
void run_convolution(Tree& T, const double* f, const RateSrc& R, const double* eps_dev, double* const* out);
RateSrc host_rates(const Tree& T, int nf);
void clear_err(Tree& T);
int read_err(Tree& T);  // synchronises T.stream

// iterate.cu: Green Iteration with Anderson mixing (tagi_green_iterate);
// eps is host memory, psi device memory in the caller's order
void green_iterate(Tree& T, const double* veff, double vshift, double* psi, double* eps, int nw,
                   const tagi_gi_params& gp, double* resid, int* iters, tagi_gi_stats* stats);

// SCF state (tagi_scf): parameters, step count, density-mixing history
struct Scf {
    Tree* T;
    tagi_scf_params p;
    int step = 0, count = 0, head = -1;
    DevBuf hist, hring;
    Scf(Tree* t, const tagi_scf_params& prm);
};
void scf_step(Scf& S, const double* vext, double vshift, double* rho, double* psi, double* eps, int nw,
              double* occ, double* rho_out, tagi_scf_report* rep);

// mlp64.cu: the H = 64 warm-start network on the tensor cores
int mlp64_params();
void mlp64_forward(const uint16_t* feat, int64_t n, const double* master, float* y, int* err, int sms, cudaStream_t s);
int mlp64_grad_grid(int64_t n, int sms);
void mlp64_gradient(const uint16_t* feat, const float* target, const float* wt, int64_t n, const double* master,
                    double* partial, int grid, int* err, cudaStream_t s);

// sets the message tagi_last_error returns on this thread; returns status
tagi_status report_error(tagi_status status, const char* msg);

// scan helper (exclusive) on device, single CTA: out[i] = sum_{j<i} in[j], out[n] = total
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

}  // namespace tagi
