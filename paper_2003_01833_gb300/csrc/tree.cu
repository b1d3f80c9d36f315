// Source-cluster tree, target batches, interaction lists and work items
// (Section 5.1, Eq. MAC, Algorithm 3), built on the GPU level by level.
//
// Every level runs point-parallel passes over the positions of the clusters
// being split: bounding boxes (order-preserving 64-bit min/max), child codes,
// a stable partition by code (block counts + one global scan), and the child
// records.  Geometric decisions use explicitly rounded float64 operations
// (__dadd_rn and friends are never contracted into FMAs) so they round exactly
// as the formulas are written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "tagi_internal.cuh"

namespace tagi {

namespace {

constexpr double kSqrt2 = 1.4142135623730951;
constexpr int kScanThreads = 1024;
constexpr int kBlk = 1024;  // positions per block in the partition passes

__device__ __forceinline__ unsigned long long ord64(double v)
{
    v = v + 0.0;  // -0 -> +0
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord64(unsigned long long o)
{
    unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
    return __longlong_as_double((long long)b);
}

// ---------------------------------------------------------------- scans
__global__ void k_scan_i64(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n)
{
    __shared__ int64_t sm[kScanThreads];
    const int tid = threadIdx.x;
    const int64_t per = (n + kScanThreads - 1) / kScanThreads;
    const int64_t a = min(n, (int64_t)tid * per), b = min(n, a + per);
    int64_t s = 0;
    for (int64_t i = a; i < b; i++) s += in[i];
    sm[tid] = s;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {  // Hillis-Steele inclusive
        int64_t v = tid >= off ? sm[tid - off] : 0;
        __syncthreads();
        sm[tid] += v;
        __syncthreads();
    }
    int64_t run = sm[tid] - s;
    for (int64_t i = a; i < b; i++) {
        int64_t v = in[i];
        out[i] = run;
        run += v;
    }
    if (tid == kScanThreads - 1) out[n] = sm[tid];
}

// ---------------------------------------------------------------- level passes
__global__ void k_init(int* pos, int* seg, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        pos[i] = (int)i;
        seg[i] = 0;
    }
}

__global__ void k_init_clusters(int first, int last, unsigned long long* blo, unsigned long long* bhi)
{
    int c = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (c < last)
        for (int d = 0; d < 3; d++) {
            blo[3 * c + d] = ~0ull;
            bhi[3 * c + d] = 0ull;
        }
}

// Bounding boxes of the clusters owning seg[p] >= 0.
__global__ void k_bbox(const int* __restrict__ pos, const int* __restrict__ seg, const double* __restrict__ xyz,
                       int64_t n, unsigned long long* blo, unsigned long long* bhi)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int c = -1;
    unsigned long long v[3] = {0, 0, 0};
    if (p < n) {
        c = seg[p];
        if (c >= 0) {
            int i = pos[p];
            v[0] = ord64(xyz[i]);
            v[1] = ord64(xyz[n + i]);
            v[2] = ord64(xyz[2 * n + i]);
        }
    }
    const unsigned full = 0xffffffffu;
    int c0 = __shfl_sync(full, c, 0);
    bool uniform = __all_sync(full, c == c0);
    if (uniform) {
        if (c0 < 0) return;
        unsigned long long mn[3] = {v[0], v[1], v[2]}, mx[3] = {v[0], v[1], v[2]};
        for (int off = 16; off > 0; off >>= 1)
            for (int d = 0; d < 3; d++) {
                unsigned long long a = __shfl_down_sync(full, mn[d], off);
                unsigned long long b = __shfl_down_sync(full, mx[d], off);
                mn[d] = min(mn[d], a);
                mx[d] = max(mx[d], b);
            }
        if ((threadIdx.x & 31) == 0)
            for (int d = 0; d < 3; d++) {
                atomicMin(&blo[3 * c0 + d], mn[d]);
                atomicMax(&bhi[3 * c0 + d], mx[d]);
            }
    } else if (c >= 0) {
        for (int d = 0; d < 3; d++) {
            atomicMin(&blo[3 * c + d], v[d]);
            atomicMax(&bhi[3 * c + d], v[d]);
        }
    }
}

// Finish boxes of clusters [first, last): lo/hi, center, radius; decide the split.
__global__ void k_finalize(int first, int last, const unsigned long long* blo, const unsigned long long* bhi,
                           const int* begin, const int* end, int leaf_size, double* lo, double* hi,
                           double* cen, double* rad, double* mid, int* smask, int* nsplit)
{
    int c = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= last) return;
    double l[3], h[3], e[3], emax = 0.0;
    for (int d = 0; d < 3; d++) {
        l[d] = unord64(blo[3 * c + d]);
        h[d] = unord64(bhi[3 * c + d]);
        lo[3 * c + d] = l[d];
        hi[3 * c + d] = h[d];
        cen[3 * c + d] = __dmul_rn(__dadd_rn(l[d], h[d]), 0.5);
        e[d] = __dsub_rn(h[d], l[d]);
        if (e[d] > emax) emax = e[d];
    }
    rad[c] = __dmul_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])),
                                             __dmul_rn(e[2], e[2]))),
                       0.5);
    int m = 0;
    if (end[c] - begin[c] > leaf_size && emax > 0.0) {
        for (int d = 0; d < 3; d++)
            if (__dmul_rn(e[d], kSqrt2) >= emax) m |= 1 << d;
        atomicAdd(nsplit, 1);
    }
    smask[c] = m;
    for (int d = 0; d < 3; d++) mid[3 * c + d] = cen[3 * c + d];
}

__global__ void k_codes(const int* __restrict__ pos, const int* __restrict__ seg, const double* __restrict__ xyz,
                        int64_t n, const int* __restrict__ smask, const double* __restrict__ mid,
                        signed char* code)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c = seg[p];
    int k = -1;
    if (c >= 0) {
        int m = smask[c];
        if (m) {
            int i = pos[p];
            k = 0;
            for (int d = 0; d < 3; d++)
                if ((m >> d) & 1)
                    if (xyz[d * n + i] >= mid[3 * c + d]) k |= 1 << d;
        }
    }
    code[p] = (signed char)k;
}

// Per block of kBlk positions: number of positions with each code, stored
// bin-major: cnt[b * nblk + blk].
__global__ void k_blkcount(const signed char* __restrict__ code, int64_t n, int64_t nblk, int64_t* cnt)
{
    __shared__ int wc[kBlk / 32][8];
    int64_t p = blockIdx.x * (int64_t)kBlk + threadIdx.x;
    int k = p < n ? code[p] : -1;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = 0; b < 8; b++) {
        unsigned m = __ballot_sync(0xffffffffu, k == b);
        if (lane == 0) wc[warp][b] = __popc(m);
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        int s = 0;
        for (int w = 0; w < kBlk / 32; w++) s += wc[w][threadIdx.x];
        cnt[threadIdx.x * nblk + blockIdx.x] = s;
    }
}

// One warp per cluster of the level: per-bin counts between begin and end and
// the bin prefix at begin (block offsets plus a warp-parallel partial count).
__device__ void prefix8(const int64_t* off, const signed char* code, int64_t nblk, int64_t x, int lane, int64_t (&pf)[8])
{
    const int64_t blk = x / kBlk;
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t q = blk * kBlk + lane; q < x; q += 32) {
        const int k = code[q];
#pragma unroll
        for (int b = 0; b < 8; b++) cnt[b] += (k == b);
    }
#pragma unroll
    for (int b = 0; b < 8; b++) {
        int v = cnt[b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        pf[b] = off[b * nblk + blk] + v;
    }
}

__global__ void k_counts(int first, int last, const int* begin, const int* end, const int* smask,
                         const signed char* code, const int64_t* off, int64_t nblk, int* cnt, int64_t* pfx,
                         int64_t* nnz)
{
    const int c = first + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32);
    const int lane = threadIdx.x & 31;
    if (c >= last) return;  // uniform per warp
    const int j = c - first;
    int64_t pb[8], pe[8];
    if (smask[c]) {
        prefix8(off, code, nblk, begin[c], lane, pb);
        prefix8(off, code, nblk, end[c], lane, pe);
    } else {
        for (int b = 0; b < 8; b++) pb[b] = pe[b] = 0;
    }
    if (lane == 0) {
        int z = 0;
        for (int b = 0; b < 8; b++) {
            const int v = (int)(pe[b] - pb[b]);
            cnt[8 * j + b] = v;
            pfx[8 * j + b] = pb[b];
            z += v > 0;
        }
        nnz[j] = z;
    }
}

__global__ void k_children(int first, int last, int nc0, const int64_t* cbase, const int* begin, const int* cnt,
                           int lvl, int* cbeg, int* cend, int* cpar, int* clev, int* cnch, int* cchild,
                           int* bfirst, int* bid, unsigned long long* blo, unsigned long long* bhi)
{
    int c = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= last) return;
    int j = c - first;
    int id = nc0 + (int)cbase[j];
    int start = begin[c];
    int q = 0;
    for (int b = 0; b < 8; b++) {
        int v = cnt[8 * j + b];
        bfirst[8 * j + b] = start;
        bid[8 * j + b] = -1;
        if (v > 0) {
            cbeg[id] = start;
            cend[id] = start + v;
            cpar[id] = c;
            clev[id] = lvl + 1;
            cnch[id] = 0;
            for (int d = 0; d < 3; d++) {
                blo[3 * id + d] = ~0ull;
                bhi[3 * id + d] = 0ull;
            }
            cchild[8 * c + q] = id;
            bid[8 * j + b] = id;
            q++;
            id++;
        }
        start += v;
    }
    cnch[c] = q;
}

// Stable scatter of the positions of split clusters into their children.
__global__ void k_scatter(const int* __restrict__ posA, const int* __restrict__ segA,
                          const signed char* __restrict__ code, int64_t n, int64_t nblk, const int64_t* off,
                          int first, const int64_t* pfx, const int* bfirst, const int* bid, const int* cnt,
                          int* posB, int* segB, int* err)
{
    __shared__ int wc[kBlk / 32][8];
    int64_t p = blockIdx.x * (int64_t)kBlk + threadIdx.x;
    int k = p < n ? code[p] : -1;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned mine = 0;
    for (int b = 0; b < 8; b++) {
        unsigned m = __ballot_sync(0xffffffffu, k == b);
        if (lane == 0) wc[warp][b] = __popc(m);
        if (k == b) mine = m;
    }
    __syncthreads();
    if (p >= n) return;
    if (k < 0) {
        posB[p] = posA[p];
        segB[p] = -1;
        return;
    }
    int before = 0;
    for (int w = 0; w < warp; w++) before += wc[w][k];
    before += __popc(mine & ((1u << lane) - 1u));
    int c = segA[p];
    int j = c - first;
    int64_t rank = off[k * nblk + blockIdx.x] + before - pfx[8 * j + k];
    if (rank < 0 || rank >= cnt[8 * j + k]) {  // cannot happen; guards the write
        atomicOr(err, 2);
        return;
    }
    int64_t dest = bfirst[8 * j + k] + rank;
    posB[dest] = posA[p];
    segB[dest] = bid[8 * j + k];
}

__global__ void k_gather_points(const int* pos, const double* xyz, const double* w, int64_t n, double* px,
                                double* py, double* pz, double* pw)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int i = pos[p];
    px[p] = xyz[i];
    py[p] = xyz[n + i];
    pz[p] = xyz[2 * n + i];
    pw[p] = w[i];
}

__global__ void k_is_leaf(int nc, const int* nch, int64_t* flag)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) flag[c] = nch[c] == 0;
}

__global__ void k_compact(int nc, const int64_t* flag, const int64_t* off, int* out, int* idx_of)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    if (flag[c]) {
        out[off[c]] = c;
        if (idx_of) idx_of[c] = (int)off[c];
    } else if (idx_of) {
        idx_of[c] = -1;
    }
}

__global__ void k_fill_leaf(const int* leaves, const int* begin, const int* end, int* pt_leaf)
{
    int c = leaves[blockIdx.x];
    for (int p = begin[c] + threadIdx.x; p < end[c]; p += blockDim.x) pt_leaf[p] = c;
}

// ---------------------------------------------------------------- lists
struct ListArgs {
    const int *begin, *end, *nch, *child, *pt_leaf, *leaves;
    const double *cen, *rad;
    double theta;
    int P;
};

// Algorithm 3's ComputePotential for one batch, one warp per batch: the
// clusters to visit form a frontier (level by level from the root), each lane
// applies the MAC to one cluster, and warp prefix sums place the entries and
// the opened children in lane order, so the output order is deterministic.
// In count mode (FILL false) only counts are produced.  The MAC arithmetic is
// the float64 expression of the oracle, without contraction.
constexpr int kListWarps = 2;      // warps (batches) per CTA
constexpr int kFront = 1024;       // frontier capacity per warp and level

__device__ __forceinline__ int warp_excl(int v, int lane, int* total)
{
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

template <bool FILL>
__device__ void walk_warp(const ListArgs a, int batch, int limit, int* front, int* nent, int64_t* near_src,
                          int64_t* far_src, Entry* out, int* out_batch, int* out_clus, int* is_far, int* err)
{
    const int lane = threadIdx.x & 31;
    int* cur = front;
    int* nxt = front + kFront;
    if (lane == 0) cur[0] = 0;
    __syncwarp();
    int ncur = 1, cnt = 0;
    int64_t sn = 0, sf = 0;  // per lane
    const double bx = a.cen[3 * batch], by = a.cen[3 * batch + 1], bz = a.cen[3 * batch + 2];
    const double rb = a.rad[batch];
    while (ncur > 0) {
        int nnext = 0;
        for (int base = 0; base < ncur; base += 32) {
            const int i = base + lane;
            int c = -1, kind = 0, ne = 0, nch = 0;  // kind: 1 far, 2 open, 3 direct
            if (i < ncur) {
                c = cur[i];
                const double dx = __dsub_rn(bx, a.cen[3 * c]), dy = __dsub_rn(by, a.cen[3 * c + 1]),
                             dz = __dsub_rn(bz, a.cen[3 * c + 2]);
                const double R =
                    __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
                const bool theta_ok = __ddiv_rn(__dadd_rn(rb, a.rad[c]), R) < a.theta;
                const bool size_ok = a.P < a.end[c] - a.begin[c];
                if (theta_ok && size_ok) {
                    kind = 1;
                    ne = 1;
                } else if (!theta_ok && a.nch[c] > 0) {
                    kind = 2;
                    nch = a.nch[c];
                } else {
                    // direct sum with every point of c: one entry per leaf below it
                    kind = 3;
                    for (int p = a.begin[c]; p < a.end[c]; p = a.end[a.pt_leaf[p]]) ne++;
                }
            }
            int etot, ctot;
            const int eoff = warp_excl(ne, lane, &etot);
            const int coff = warp_excl(nch, lane, &ctot);
            if ((FILL && cnt + etot > limit) || nnext + ctot > kFront) {
                if (lane == 0) *err = 1;
                return;
            }
            if (kind == 2)
                for (int q = 0; q < nch; q++) nxt[nnext + coff + q] = a.child[8 * c + q];
            if (kind == 1) {
                sf += a.P;
                if (FILL) {
                    out[cnt + eoff] = Entry{0, 0, c, 2};
                    out_batch[cnt + eoff] = batch;
                    out_clus[cnt + eoff] = c;
                    is_far[c] = 1;
                }
            } else if (kind == 3) {
                int t = 0;
                for (int p = a.begin[c]; p < a.end[c];) {
                    const int leaf = a.pt_leaf[p];
                    const int e = a.end[leaf];
                    if (FILL) {
                        out[cnt + eoff + t] = Entry{a.begin[leaf], e, leaf, leaf == batch ? 1 : 0};
                        out_batch[cnt + eoff + t] = batch;
                        out_clus[cnt + eoff + t] = leaf;
                    }
                    sn += e - a.begin[leaf];
                    t++;
                    p = e;
                }
            }
            cnt += etot;
            nnext += ctot;
        }
        __syncwarp();
        int* t = cur;
        cur = nxt;
        nxt = t;
        ncur = nnext;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sn += __shfl_down_sync(0xffffffffu, sn, o);
        sf += __shfl_down_sync(0xffffffffu, sf, o);
    }
    *nent = cnt;
    *near_src = sn;  // lane 0 holds the sums
    *far_src = sf;
}

__global__ void __launch_bounds__(32 * kListWarps) k_list_count(ListArgs a, int nleaf, int64_t* cnt,
                                                                 int64_t* near_pairs, int64_t* far_pairs, int* err)
{
    __shared__ int front[kListWarps][2 * kFront];
    const int w = threadIdx.x >> 5;
    const int j = blockIdx.x * kListWarps + w;
    if (j >= nleaf) return;
    const int b = a.leaves[j];
    int ne = 0;
    int64_t sn = 0, sf = 0;
    walk_warp<false>(a, b, 0, front[w], &ne, &sn, &sf, nullptr, nullptr, nullptr, nullptr, err);
    if ((threadIdx.x & 31) == 0) {
        cnt[j] = ne;
        const int64_t nb = a.end[b] - a.begin[b];
        near_pairs[j] = nb * sn;
        far_pairs[j] = nb * sf;
    }
}

__global__ void __launch_bounds__(32 * kListWarps) k_list_fill(ListArgs a, int nleaf, const int64_t* off, Entry* ent,
                                                                int* eb, int* ec, int* is_far, int* err)
{
    __shared__ int front[kListWarps][2 * kFront];
    const int w = threadIdx.x >> 5;
    const int j = blockIdx.x * kListWarps + w;
    if (j >= nleaf) return;
    const int b = a.leaves[j];
    int ne;
    int64_t sn, sf;
    const int64_t o = off[j];
    walk_warp<true>(a, b, (int)(off[j + 1] - o), front[w], &ne, &sn, &sf, ent + o, eb + o, ec + o, is_far, err);
}

__global__ void k_far_ranges(int64_t nent, Entry* ent, const int* cl_far, int64_t n, int P)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nent) return;
    Entry x = ent[e];
    if (x.flags & 2) {
        int64_t s0 = n + (int64_t)cl_far[x.frame] * P;
        x.src0 = (int)s0;
        x.src1 = (int)(s0 + P);
        ent[e] = x;
    }
}

// flags bit2: the boxes of the batch and of the source cluster are at least
// sqrt(42) alpha apart, so exp(-r^2/alpha^2) <= 2^-60 for every pair of the
// entry and the Gaussian of the Coulomb SS is below float32 resolution there
// (the FP32C kernel leaves it out; the float64 kernel ignores the bit).
// pairs[0], pairs[1]: near and far pairs of the flagged entries.
__global__ void k_gauss_flags(int64_t nent, Entry* ent, const int* eb, const int* ec, const double* lo,
                              const double* hi, const int* begin, const int* end, double alpha,
                              unsigned long long* pairs)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nent) return;
    const int b = eb[e], c = ec[e];
    double d2 = 0.0;
    for (int k = 0; k < 3; k++) {
        const double g = fmax(0.0, fmax(lo[3 * c + k] - hi[3 * b + k], lo[3 * b + k] - hi[3 * c + k]));
        d2 += g * g;
    }
    if (d2 >= 42.0 * alpha * alpha) {
        Entry x = ent[e];
        x.flags |= 4;
        ent[e] = x;
        const unsigned long long np = (unsigned long long)(end[b] - begin[b]) * (unsigned long long)(x.src1 - x.src0);
        atomicAdd(pairs + ((x.flags & 2) ? 1 : 0), np);
    }
}

// ---------------------------------------------------------------- work items
__device__ __forceinline__ int padded(int v) { return (v + 7) & ~7; }

__global__ void k_item_counts(int nleaf, const int* leaves, const int* begin, const int* end, const int64_t* eoff,
                              const Entry* ent, int seg_src, int64_t* nchunk, int64_t* nitem)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nleaf) return;
    int b = leaves[j];
    int nb = end[b] - begin[b];
    int ch = (nb + kTargetsPerItem - 1) / kTargetsPerItem;
    int segs = 0, acc = 0;
    for (int64_t e = eoff[j]; e < eoff[j + 1]; e++) {
        acc += padded(ent[e].src1 - ent[e].src0);
        if (acc >= seg_src) {
            segs++;
            acc = 0;
        }
    }
    if (acc > 0 || segs == 0) segs++;
    nchunk[j] = ch;
    nitem[j] = (int64_t)ch * segs;
}

__global__ void k_item_fill(int nleaf, const int* leaves, const int* begin, const int* end, const int64_t* eoff,
                            const Entry* ent, int seg_src, const int64_t* chunk_off, const int64_t* item_off,
                            Item* items, int* tc_item0, int* tc_t0, int* tc_t1, int* tc_batch)
{
    // one block per leaf, one thread per target chunk of the leaf
    const int j = blockIdx.x;
    if (j >= nleaf) return;
    int b = leaves[j];
    int nb = end[b] - begin[b];
    int ch = (int)(chunk_off[j + 1] - chunk_off[j]);
    int segs = ch ? (int)((item_off[j + 1] - item_off[j]) / ch) : 0;
    for (int ci = threadIdx.x; ci < ch; ci += blockDim.x) {
        int64_t tc = chunk_off[j] + ci;
        int t0 = begin[b] + ci * kTargetsPerItem;
        int t1 = min(begin[b] + nb, t0 + kTargetsPerItem);
        int64_t first = item_off[j] + (int64_t)ci * segs;
        tc_item0[tc] = (int)first;
        tc_t0[tc] = t0;
        tc_t1[tc] = t1;
        tc_batch[tc] = b;
        int s = 0, acc = 0;
        int64_t e0 = eoff[j];
        for (int64_t e = eoff[j]; e < eoff[j + 1]; e++) {
            acc += padded(ent[e].src1 - ent[e].src0);
            bool last = e + 1 == eoff[j + 1];
            if (acc >= seg_src || last) {
                if (s < segs) items[first + s] = Item{t0, t1, (int)e0, (int)(e + 1), b, (int)tc, (int)first, segs};
                s++;
                acc = 0;
                e0 = e + 1;
            }
        }
        for (; s < segs; s++)
            items[first + s] = Item{t0, t1, (int)eoff[j + 1], (int)eoff[j + 1], b, (int)tc, (int)first, segs};
    }
}

__global__ void k_ant_counts(int nfar, const int* far_cl, const int* begin, const int* end, int64_t* cnt)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfar) return;
    int c = far_cl[f];
    cnt[f] = (end[c] - begin[c] + kAntChunk - 1) / kAntChunk;
}

__global__ void k_far_points(int nfar, const int* far_cl, const int* begin, const int* end, int64_t* cnt)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfar) return;
    int c = far_cl[f];
    cnt[f] = end[c] - begin[c];
}

__global__ void k_ant_fill(int nfar, const int* far_cl, const int* begin, const int* end, const int64_t* off,
                           AntItem* items, int* far_ant0)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f > nfar) return;
    far_ant0[f] = (int)off[f];
    if (f == nfar) return;
    int c = far_cl[f];
    int64_t o = off[f];
    for (int p = begin[c]; p < end[c]; p += kAntChunk) items[o++] = AntItem{p, min(end[c], p + kAntChunk), c, f};
}

// ---------------------------------------------------------------- records
// Mesh-point records: position relative to the center of the point's leaf
// and quadrature weight, each as a two-float (hi in rec4, lo in rec4lo).
__global__ void k_point_records(int64_t n, const double* px, const double* py, const double* pz, const double* pw,
                                const int* pt_leaf, const double* cen, float4* rec4, float4* rec4lo, double* rx,
                                double* ry, double* rz, double* rw)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (rec4) {
        int c = pt_leaf[p];
        double d[3] = {px[p] - cen[3 * c], py[p] - cen[3 * c + 1], pz[p] - cen[3 * c + 2]};
        float h[3], l[3];
        for (int k = 0; k < 3; k++) {
            h[k] = (float)d[k];
            l[k] = (float)(d[k] - (double)h[k]);
        }
        const float wh = (float)pw[p];
        rec4[p] = make_float4(h[0], h[1], h[2], wh);
        rec4lo[p] = make_float4(l[0], l[1], l[2], (float)(pw[p] - (double)wh));
    }
    if (rx) {
        rx[p] = px[p];
        ry[p] = py[p];
        rz[p] = pz[p];
        rw[p] = pw[p];
    }
}

// Proxy positions: Chebyshev points of the second kind cos(pi k / n) mapped
// to each approximated cluster's box (Section 5.2).  Index (k1 (n+1) + k2)(n+1) + k3.
__global__ void k_proxy_records(int nfar, const int* far_cl, int degree, int64_t n, const double* lo,
                                const double* hi, float4* rec4, double* rx, double* ry, double* rz)
{
    int f = blockIdx.x;
    int c = far_cl[f];
    int m = degree + 1, P = m * m * m;
    double cc[3], hh[3];
    for (int d = 0; d < 3; d++) {
        cc[d] = (lo[3 * c + d] + hi[3 * c + d]) * 0.5;
        hh[d] = (hi[3 * c + d] - lo[3 * c + d]) * 0.5;
    }
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        int k1 = k / (m * m), k2 = (k / m) % m, k3 = k % m;
        double s1 = cos(M_PI * k1 / degree), s2 = cos(M_PI * k2 / degree), s3 = cos(M_PI * k3 / degree);
        int64_t r = n + (int64_t)f * P + k;
        if (rec4) {
            // the float32 anterpolation interpolates on the float32-rounded
            // nodes; the proxies sit on exactly those nodes
            s1 = (double)(float)s1;
            s2 = (double)(float)s2;
            s3 = (double)(float)s3;
            rec4[r] = make_float4((float)(hh[0] * s1), (float)(hh[1] * s2), (float)(hh[2] * s3), 0.0f);
        }
        if (rx) {
            rx[r] = cc[0] + hh[0] * s1;
            ry[r] = cc[1] + hh[1] * s2;
            rz[r] = cc[2] + hh[2] * s3;
        }
    }
}

__global__ void k_check_finite(const double* a, int64_t n, int* bad)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(a[i])) atomicOr(bad, 1);
}

inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

struct Host1 {
    // pinned scalars for readbacks, allocated once per host thread
    int64_t* h = nullptr;
    Host1()
    {
        thread_local int64_t* buf = nullptr;
        if (!buf) TAGI_CUDA(cudaMallocHost(&buf, 8 * sizeof(int64_t)));
        h = buf;
    }
};

}  // namespace

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s)
{
    launch(k_scan_i64, 1, kScanThreads, 0, s, in, out, n);
    TAGI_LAUNCH_CHECK();
}

static int64_t read_i64(const int64_t* dev, cudaStream_t s, Host1& h)
{
    TAGI_CUDA(cudaMemcpyAsync(h.h, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaStreamSynchronize(s));
    return h.h[0];
}

static int read_i32(const int* dev, cudaStream_t s, Host1& h)
{
    TAGI_CUDA(cudaMemcpyAsync(h.h, dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    TAGI_CUDA(cudaStreamSynchronize(s));
    return (int)((int*)h.h)[0];
}

// Grow every per-cluster array to hold `cap` clusters, keeping contents.
static void grow_clusters(Tree& T, int cur, int cap, DevBuf& blo, DevBuf& bhi, cudaStream_t s)
{
    struct G {
        DevBuf* b;
        size_t per;
    } g[] = {{&T.cl_begin, 4},  {&T.cl_end, 4}, {&T.cl_parent, 4}, {&T.cl_level, 4}, {&T.cl_nchild, 4},
             {&T.cl_child, 32}, {&T.cl_lo, 24}, {&T.cl_hi, 24},     {&T.cl_cen, 24},  {&T.cl_rad, 8},
             {&blo, 24},        {&bhi, 24}};
    for (auto& x : g) {
        if (x.b->bytes >= x.per * (size_t)cap) continue;
        DevBuf nb;
        nb.ensure(x.per * (size_t)cap);
        if (x.b->p && cur > 0) TAGI_CUDA(cudaMemcpyAsync(nb.p, x.b->p, x.per * (size_t)cur, cudaMemcpyDeviceToDevice, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
        *x.b = std::move(nb);
    }
}

void build_tree(Tree& T, const double* xyz, const double* w)
{
    cudaStream_t s = T.stream;
    const int64_t n = T.n;
    TAGI_REQUIRE(n <= (int64_t)0x3fffffff, "n too large for 32-bit tree positions");
    Host1 H;
    // ---- input validation (non-finite coordinates or weights)
    DevBuf flag;
    flag.ensure(64);
    TAGI_CUDA(cudaMemsetAsync(flag.p, 0, 64, s));
    launch(k_check_finite, nblocks(3 * n, 256), 256, 0, s, xyz, 3 * n, flag.as<int>());
    launch(k_check_finite, nblocks(n, 256), 256, 0, s, w, n, flag.as<int>());
    TAGI_LAUNCH_CHECK();
    TAGI_REQUIRE(read_i32(flag.as<int>(), s, H) == 0, "xyz or w holds a non-finite value");

    DevBuf posA, posB, segA, segB, code, blo, bhi, mid, smask, nsplit;
    posA.ensure(4 * n);
    posB.ensure(4 * n);
    segA.ensure(4 * n);
    segB.ensure(4 * n);
    code.ensure(n);
    const int64_t nblk = (n + kBlk - 1) / kBlk;
    DevBuf bcnt, boff;
    bcnt.ensure(8 * 8 * nblk);
    boff.ensure(8 * (8 * nblk + 1));
    nsplit.ensure(16);

    int cap = 1024;
    grow_clusters(T, 0, cap, blo, bhi, s);
    mid.ensure(24 * (size_t)cap);
    smask.ensure(4 * (size_t)cap);

    launch(k_init, nblocks(n, 256), 256, 0, s, posA.as<int>(), segA.as<int>(), n);
    {
        int one_begin = 0, one_end = (int)n, minus1 = -1, zero = 0;
        TAGI_CUDA(cudaMemcpyAsync(T.cl_begin.p, &one_begin, 4, cudaMemcpyHostToDevice, s));
        TAGI_CUDA(cudaMemcpyAsync(T.cl_end.p, &one_end, 4, cudaMemcpyHostToDevice, s));
        TAGI_CUDA(cudaMemcpyAsync(T.cl_parent.p, &minus1, 4, cudaMemcpyHostToDevice, s));
        TAGI_CUDA(cudaMemcpyAsync(T.cl_level.p, &zero, 4, cudaMemcpyHostToDevice, s));
        TAGI_CUDA(cudaMemcpyAsync(T.cl_nchild.p, &zero, 4, cudaMemcpyHostToDevice, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
    }
    launch(k_init_clusters, 1, 32, 0, s, 0, 1, blo.as<unsigned long long>(), bhi.as<unsigned long long>());
    TAGI_LAUNCH_CHECK();

    int first = 0, last = 1, nc = 1, lvl = 0;
    DevBuf cnt, pfx, nnz, cbase, bfirst, bid;
    while (true) {
        const int nl = last - first;
        launch(k_bbox, nblocks(n, 256), 256, 0, s, posA.as<int>(), segA.as<int>(), xyz, n, blo.as<unsigned long long>(),
                                                bhi.as<unsigned long long>());
        TAGI_CUDA(cudaMemsetAsync(nsplit.p, 0, 4, s));
        launch(k_finalize, nblocks(nl, 128), 128, 0, s, first, last, blo.as<unsigned long long>(),
                                                     bhi.as<unsigned long long>(), T.cl_begin.as<int>(),
                                                     T.cl_end.as<int>(), T.leaf_size, T.cl_lo.as<double>(),
                                                     T.cl_hi.as<double>(), T.cl_cen.as<double>(),
                                                     T.cl_rad.as<double>(), mid.as<double>(), smask.as<int>(),
                                                     nsplit.as<int>());
        TAGI_LAUNCH_CHECK();
        int ns = read_i32(nsplit.as<int>(), s, H);
        if (ns == 0) {
            // the last level are all leaves
            TAGI_CUDA(cudaMemsetAsync(T.cl_nchild.as<int>() + first, 0, 4 * (size_t)nl, s));
            break;
        }
        TAGI_REQUIRE(lvl < kMaxDepth, "tree deeper than 64 levels (degenerate point set)");
        if (nc + 8 * ns > cap) {
            int ncap = std::max(2 * cap, nc + 8 * ns);
            grow_clusters(T, nc, ncap, blo, bhi, s);
            DevBuf m2, s2;
            m2.ensure(24 * (size_t)ncap);
            s2.ensure(4 * (size_t)ncap);
            TAGI_CUDA(cudaMemcpyAsync(m2.p, mid.p, 24 * (size_t)nc, cudaMemcpyDeviceToDevice, s));
            TAGI_CUDA(cudaMemcpyAsync(s2.p, smask.p, 4 * (size_t)nc, cudaMemcpyDeviceToDevice, s));
            TAGI_CUDA(cudaStreamSynchronize(s));
            mid = std::move(m2);
            smask = std::move(s2);
            cap = ncap;
        }
        launch(k_codes, nblocks(n, 256), 256, 0, s, posA.as<int>(), segA.as<int>(), xyz, n, smask.as<int>(),
                                                mid.as<double>(), code.as<signed char>());
        launch(k_blkcount, (int)nblk, kBlk, 0, s, code.as<signed char>(), n, nblk, bcnt.as<int64_t>());
        exclusive_scan_i64(bcnt.as<int64_t>(), boff.as<int64_t>(), 8 * nblk, s);
        cnt.ensure(32 * (size_t)nl);
        pfx.ensure(64 * (size_t)nl);
        nnz.ensure(8 * (size_t)nl);
        cbase.ensure(8 * ((size_t)nl + 1));
        bfirst.ensure(32 * (size_t)nl);
        bid.ensure(32 * (size_t)nl);
        launch(k_counts, nblocks(32 * (int64_t)nl, 128), 128, 0, s, first, last, T.cl_begin.as<int>(), T.cl_end.as<int>(),
                                                   smask.as<int>(), code.as<signed char>(), boff.as<int64_t>(), nblk,
                                                   cnt.as<int>(), pfx.as<int64_t>(), nnz.as<int64_t>());
        exclusive_scan_i64(nnz.as<int64_t>(), cbase.as<int64_t>(), nl, s);
        TAGI_LAUNCH_CHECK();
        int64_t nnew = read_i64(cbase.as<int64_t>() + nl, s, H);
        launch(k_children, nblocks(nl, 128), 128, 0, s, first, last, nc, cbase.as<int64_t>(), T.cl_begin.as<int>(),
                                                     cnt.as<int>(), lvl, T.cl_begin.as<int>(), T.cl_end.as<int>(),
                                                     T.cl_parent.as<int>(), T.cl_level.as<int>(),
                                                     T.cl_nchild.as<int>(), T.cl_child.as<int>(), bfirst.as<int>(),
                                                     bid.as<int>(), blo.as<unsigned long long>(),
                                                     bhi.as<unsigned long long>());
        launch(k_scatter, (int)nblk, kBlk, 0, s, posA.as<int>(), segA.as<int>(), code.as<signed char>(), n, nblk,
                                             boff.as<int64_t>(), first, pfx.as<int64_t>(), bfirst.as<int>(),
                                             bid.as<int>(), cnt.as<int>(), posB.as<int>(), segB.as<int>(),
                                             flag.as<int>());
        TAGI_LAUNCH_CHECK();
        std::swap(posA, posB);
        std::swap(segA, segB);
        first = nc;
        nc += (int)nnew;
        last = nc;
        lvl++;
    }
    T.nc = nc;
    T.depth = lvl;
    TAGI_REQUIRE(read_i32(flag.as<int>(), s, H) == 0, "tree partition consistency check failed");

    // ---- points in tree order
    T.perm.ensure(4 * n);
    TAGI_CUDA(cudaMemcpyAsync(T.perm.p, posA.p, 4 * n, cudaMemcpyDeviceToDevice, s));
    T.px.ensure(8 * n);
    T.py.ensure(8 * n);
    T.pz.ensure(8 * n);
    T.pw.ensure(8 * n);
    launch(k_gather_points, nblocks(n, 256), 256, 0, s, posA.as<int>(), xyz, w, n, T.px.as<double>(), T.py.as<double>(),
                                                    T.pz.as<double>(), T.pw.as<double>());
    TAGI_LAUNCH_CHECK();
    posA.release();
    posB.release();
    segA.release();
    segB.release();
    code.release();
    bcnt.release();
    boff.release();
    blo.release();
    bhi.release();

    // ---- leaves (batches)
    DevBuf fl, fo;
    fl.ensure(8 * (size_t)nc);
    fo.ensure(8 * ((size_t)nc + 1));
    launch(k_is_leaf, nblocks(nc, 256), 256, 0, s, nc, T.cl_nchild.as<int>(), fl.as<int64_t>());
    exclusive_scan_i64(fl.as<int64_t>(), fo.as<int64_t>(), nc, s);
    T.nleaf = (int)read_i64(fo.as<int64_t>() + nc, s, H);
    T.leaves.ensure(4 * (size_t)T.nleaf);
    launch(k_compact, nblocks(nc, 256), 256, 0, s, nc, fl.as<int64_t>(), fo.as<int64_t>(), T.leaves.as<int>(), nullptr);
    T.pt_leaf.ensure(4 * n);
    launch(k_fill_leaf, T.nleaf, 256, 0, s, T.leaves.as<int>(), T.cl_begin.as<int>(), T.cl_end.as<int>(),
                                        T.pt_leaf.as<int>());
    TAGI_LAUNCH_CHECK();

    // ---- interaction lists (Algorithm 3, MAC of Eq. MAC)
    ListArgs la{T.cl_begin.as<int>(), T.cl_end.as<int>(),  T.cl_nchild.as<int>(), T.cl_child.as<int>(),
                T.pt_leaf.as<int>(),  T.leaves.as<int>(),   T.cl_cen.as<double>(), T.cl_rad.as<double>(),
                T.theta,              T.P};
    const int nleaf = T.nleaf;
    DevBuf lc, lo_, npair, fpair, err;
    lc.ensure(8 * (size_t)nleaf);
    lo_.ensure(8 * ((size_t)nleaf + 1));
    npair.ensure(8 * ((size_t)nleaf + 1));
    fpair.ensure(8 * ((size_t)nleaf + 1));
    err.ensure(16);
    TAGI_CUDA(cudaMemsetAsync(err.p, 0, 16, s));
    launch(k_list_count, nblocks(nleaf, kListWarps), 32 * kListWarps, 0, s, la, nleaf, lc.as<int64_t>(), npair.as<int64_t>(),
                                                   fpair.as<int64_t>(), err.as<int>());
    exclusive_scan_i64(lc.as<int64_t>(), lo_.as<int64_t>(), nleaf, s);
    TAGI_LAUNCH_CHECK();
    TAGI_REQUIRE(read_i32(err.as<int>(), s, H) == 0, "interaction-list stack overflow");
    T.nent = read_i64(lo_.as<int64_t>() + nleaf, s, H);
    {
        DevBuf tmp;
        tmp.ensure(8 * ((size_t)nleaf + 1));
        exclusive_scan_i64(npair.as<int64_t>(), tmp.as<int64_t>(), nleaf, s);
        T.near_pairs = read_i64(tmp.as<int64_t>() + nleaf, s, H);
        exclusive_scan_i64(fpair.as<int64_t>(), tmp.as<int64_t>(), nleaf, s);
        T.far_pairs = read_i64(tmp.as<int64_t>() + nleaf, s, H);
    }
    TAGI_REQUIRE(T.nent < (int64_t)0x7fffffff, "too many interaction entries");
    T.ent.ensure(sizeof(Entry) * (size_t)std::max<int64_t>(T.nent, 1));
    T.ent_batch.ensure(4 * (size_t)std::max<int64_t>(T.nent, 1));
    T.ent_clus.ensure(4 * (size_t)std::max<int64_t>(T.nent, 1));
    T.ent_off.ensure(8 * ((size_t)nleaf + 1));
    TAGI_CUDA(cudaMemcpyAsync(T.ent_off.p, lo_.p, 8 * ((size_t)nleaf + 1), cudaMemcpyDeviceToDevice, s));
    DevBuf isfar;
    isfar.ensure(4 * (size_t)nc);
    TAGI_CUDA(cudaMemsetAsync(isfar.p, 0, 4 * (size_t)nc, s));
    launch(k_list_fill, nblocks(nleaf, kListWarps), 32 * kListWarps, 0, s, la, nleaf, lo_.as<int64_t>(), T.ent.as<Entry>(),
                                                  T.ent_batch.as<int>(), T.ent_clus.as<int>(), isfar.as<int>(),
                                                  err.as<int>());
    TAGI_LAUNCH_CHECK();
    TAGI_REQUIRE(read_i32(err.as<int>(), s, H) == 0, "interaction-list fill disagrees with its count");

    // ---- approximated clusters
    {
        DevBuf f64, o64;
        f64.ensure(8 * (size_t)nc);
        o64.ensure(8 * ((size_t)nc + 1));
        // widen flags to int64 for the scan
        std::vector<int> hf(nc);
        TAGI_CUDA(cudaMemcpyAsync(hf.data(), isfar.p, 4 * (size_t)nc, cudaMemcpyDeviceToHost, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> hf64(hf.begin(), hf.end());
        TAGI_CUDA(cudaMemcpyAsync(f64.p, hf64.data(), 8 * (size_t)nc, cudaMemcpyHostToDevice, s));
        exclusive_scan_i64(f64.as<int64_t>(), o64.as<int64_t>(), nc, s);
        T.nfar = (int)read_i64(o64.as<int64_t>() + nc, s, H);
        T.far_cl.ensure(4 * (size_t)std::max(T.nfar, 1));
        T.cl_far.ensure(4 * (size_t)nc);
        launch(k_compact, nblocks(nc, 256), 256, 0, s, nc, f64.as<int64_t>(), o64.as<int64_t>(), T.far_cl.as<int>(),
                                                   T.cl_far.as<int>());
        TAGI_LAUNCH_CHECK();
    }
    T.nrec = n + (int64_t)T.nfar * T.P;
    TAGI_REQUIRE(T.nrec < (int64_t)0x7fffffff, "too many source records");
    if (T.nent > 0)
        launch(k_far_ranges, nblocks(T.nent, 256), 256, 0, s, T.nent, T.ent.as<Entry>(), T.cl_far.as<int>(), n, T.P);
    T.near_pairs_ng = T.far_pairs_ng = 0;
    if (T.nent > 0) {
        DevBuf ng;
        ng.ensure(2 * sizeof(int64_t));
        TAGI_CUDA(cudaMemsetAsync(ng.p, 0, 2 * sizeof(int64_t), s));
        launch(k_gauss_flags, nblocks(T.nent, 256), 256, 0, s, T.nent, T.ent.as<Entry>(), T.ent_batch.as<int>(),
               T.ent_clus.as<int>(), T.cl_lo.as<double>(), T.cl_hi.as<double>(), T.cl_begin.as<int>(),
               T.cl_end.as<int>(), T.alpha, ng.as<unsigned long long>());
        TAGI_LAUNCH_CHECK();
        T.near_pairs_ng = read_i64(ng.as<int64_t>(), s, H);
        T.far_pairs_ng = read_i64(ng.as<int64_t>() + 1, s, H);
    }
    TAGI_LAUNCH_CHECK();

    // ---- work items of the near/far kernel
    const int seg_src = T.segment;
    DevBuf nch, nit, choff, itoff;
    nch.ensure(8 * (size_t)nleaf);
    nit.ensure(8 * (size_t)nleaf);
    choff.ensure(8 * ((size_t)nleaf + 1));
    itoff.ensure(8 * ((size_t)nleaf + 1));
    launch(k_item_counts, nblocks(nleaf, 128), 128, 0, s, nleaf, T.leaves.as<int>(), T.cl_begin.as<int>(),
                                                      T.cl_end.as<int>(), T.ent_off.as<int64_t>(), T.ent.as<Entry>(),
                                                      seg_src, nch.as<int64_t>(), nit.as<int64_t>());
    exclusive_scan_i64(nch.as<int64_t>(), choff.as<int64_t>(), nleaf, s);
    exclusive_scan_i64(nit.as<int64_t>(), itoff.as<int64_t>(), nleaf, s);
    TAGI_LAUNCH_CHECK();
    T.ntchunk = read_i64(choff.as<int64_t>() + nleaf, s, H);
    T.nitems = read_i64(itoff.as<int64_t>() + nleaf, s, H);
    T.items.ensure(sizeof(Item) * (size_t)std::max<int64_t>(T.nitems, 1));
    T.tc_item0.ensure(4 * ((size_t)T.ntchunk + 1));
    T.tc_t0.ensure(4 * (size_t)T.ntchunk);
    T.tc_t1.ensure(4 * (size_t)T.ntchunk);
    T.tc_batch.ensure(4 * (size_t)T.ntchunk);
    launch(k_item_fill, nleaf, 32, 0, s, nleaf, T.leaves.as<int>(), T.cl_begin.as<int>(),
                                                    T.cl_end.as<int>(), T.ent_off.as<int64_t>(), T.ent.as<Entry>(),
                                                    seg_src, choff.as<int64_t>(), itoff.as<int64_t>(),
                                                    T.items.as<Item>(), T.tc_item0.as<int>(), T.tc_t0.as<int>(),
                                                    T.tc_t1.as<int>(), T.tc_batch.as<int>());
    TAGI_LAUNCH_CHECK();
    {
        int tot = (int)T.nitems;
        TAGI_CUDA(cudaMemcpyAsync(T.tc_item0.as<int>() + T.ntchunk, &tot, 4, cudaMemcpyHostToDevice, s));
        TAGI_CUDA(cudaStreamSynchronize(s));
    }

    // ---- anterpolation items
    T.ant_points = 0;
    if (T.nfar > 0) {
        DevBuf ac, ao;
        ac.ensure(8 * (size_t)T.nfar);
        ao.ensure(8 * ((size_t)T.nfar + 1));
        launch(k_ant_counts, nblocks(T.nfar, 128), 128, 0, s, T.nfar, T.far_cl.as<int>(), T.cl_begin.as<int>(),
                                                          T.cl_end.as<int>(), ac.as<int64_t>());
        exclusive_scan_i64(ac.as<int64_t>(), ao.as<int64_t>(), T.nfar, s);
        TAGI_LAUNCH_CHECK();
        T.nant = read_i64(ao.as<int64_t>() + T.nfar, s, H);
        // sum of N_S over approximated clusters (anterpolation work, reported by tagi_tree_info)
        launch(k_far_points, nblocks(T.nfar, 128), 128, 0, s, T.nfar, T.far_cl.as<int>(), T.cl_begin.as<int>(),
               T.cl_end.as<int>(), ac.as<int64_t>());
        exclusive_scan_i64(ac.as<int64_t>(), ao.as<int64_t>(), T.nfar, s);
        TAGI_LAUNCH_CHECK();
        T.ant_points = read_i64(ao.as<int64_t>() + T.nfar, s, H);
        T.ant_items.ensure(sizeof(AntItem) * (size_t)T.nant);
        T.far_ant0.ensure(4 * ((size_t)T.nfar + 1));
        launch(k_ant_counts, nblocks(T.nfar, 128), 128, 0, s, T.nfar, T.far_cl.as<int>(), T.cl_begin.as<int>(),
                                                          T.cl_end.as<int>(), ac.as<int64_t>());
        exclusive_scan_i64(ac.as<int64_t>(), ao.as<int64_t>(), T.nfar, s);
        launch(k_ant_fill, nblocks(T.nfar + 1, 128), 128, 0, s, T.nfar, T.far_cl.as<int>(), T.cl_begin.as<int>(),
                                                            T.cl_end.as<int>(), ao.as<int64_t>(),
                                                            T.ant_items.as<AntItem>(), T.far_ant0.as<int>());
        TAGI_LAUNCH_CHECK();
    }

    // ---- source records
    const bool fp32 = T.prec == TAGI_FP32C;
    if (fp32) {
        T.rec4.ensure(16 * (size_t)T.nrec);
        T.rec4lo.ensure(16 * (size_t)n);
    } else {
        T.rx.ensure(8 * (size_t)T.nrec);
        T.ry.ensure(8 * (size_t)T.nrec);
        T.rz.ensure(8 * (size_t)T.nrec);
        T.rw.ensure(8 * (size_t)T.nrec);
    }
    launch(k_point_records, nblocks(n, 256), 256, 0, s, 
        n, T.px.as<double>(), T.py.as<double>(), T.pz.as<double>(), T.pw.as<double>(), T.pt_leaf.as<int>(),
        T.cl_cen.as<double>(), fp32 ? T.rec4.as<float4>() : nullptr, fp32 ? T.rec4lo.as<float4>() : nullptr,
        fp32 ? nullptr : T.rx.as<double>(),
        fp32 ? nullptr : T.ry.as<double>(), fp32 ? nullptr : T.rz.as<double>(), fp32 ? nullptr : T.rw.as<double>());
    if (T.nfar > 0)
        launch(k_proxy_records, T.nfar, 256, 0, s, T.nfar, T.far_cl.as<int>(), T.degree, n, T.cl_lo.as<double>(),
                                               T.cl_hi.as<double>(), fp32 ? T.rec4.as<float4>() : nullptr,
                                               fp32 ? nullptr : T.rx.as<double>(), fp32 ? nullptr : T.ry.as<double>(),
                                               fp32 ? nullptr : T.rz.as<double>());
    TAGI_LAUNCH_CHECK();
    anterpolate_weights(T);
    TAGI_CUDA(cudaStreamSynchronize(s));
}

}  // namespace tagi
