// An entry point that allocates no device memory: the float64 direct-sum
// Yukawa convolution with singularity subtraction, for callers that cannot
// let a library call cudaMalloc -- host frameworks that hand out every
// device byte from their own pool (a second allocator would fragment it or
// exceed its budget), and latency-critical loops in which an allocation's
// implicit device synchronisation would stall other streams.  The caller
// passes inputs and outputs; the only other device memory used is one
// file-scope scratch array of fixed size that the library's module carries on
// every GPU that loads it, until process exit.
//
// It is a variant of the float64 near/far interaction kernel (k_interact64)
// that needs no tree: every target sums over every source (the theta = 0 case
// of the treecode, i.e. the direct sum), with the source range split into a
// few slices whose partial sums go to the scratch array and are reduced in a
// fixed order.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "tagi_internal.cuh"

namespace tagi {
namespace {

// Scratch: 2^20 float64 values (8 MiB), 256-byte aligned.
constexpr int64_t kNoAllocScratch = 1 << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

constexpr int kNaThreads = 256;
constexpr int kNaTile = 128;
constexpr int kNaMaxSplits = 8;
constexpr int kNaMaxDevices = 64;
constexpr int kNaMaxFields = 16;

// decay rates by value, so no host-to-device copy is needed
struct NaRates {
    double k[kNaMaxFields];
};

// partial[(s * nf + o) * n + i] = sum over sources j in slice s, r_ij != 0, of
//   exp(-k_o r) / r * (f_o[j] - f_o[i]) w_j
__global__ void __launch_bounds__(kNaThreads) k_direct_noalloc(const double* __restrict__ xyz,
                                                               const double* __restrict__ w,
                                                               const double* __restrict__ f, NaRates rates,
                                                               int nf, int64_t n, int splits,
                                                               double* __restrict__ partial)
{
    __shared__ double sx[kNaTile], sy[kNaTile], sz[kNaTile], sw[kNaTile], sf[kNaTile];
    const int64_t i = blockIdx.x * (int64_t)kNaThreads + threadIdx.x;
    const int s = blockIdx.y, o = blockIdx.z;
    const int64_t per = (n + splits - 1) / splits;
    const int64_t j0 = s * per, j1 = min(n, j0 + per);
    const bool ok = i < n;
    const double x = ok ? xyz[i] : 0.0, y = ok ? xyz[n + i] : 0.0, z = ok ? xyz[2 * n + i] : 0.0;
    const double fi = ok ? f[o * n + i] : 0.0;
    const double k = rates.k[o];
    double acc = 0.0;
    for (int64_t t0 = j0; t0 < j1; t0 += kNaTile) {
        const int nt = (int)min((int64_t)kNaTile, j1 - t0);
        __syncthreads();
        if (threadIdx.x < nt) {
            const int64_t j = t0 + threadIdx.x;
            sx[threadIdx.x] = xyz[j];
            sy[threadIdx.x] = xyz[n + j];
            sz[threadIdx.x] = xyz[2 * n + j];
            sw[threadIdx.x] = w[j];
            sf[threadIdx.x] = f[o * n + j];
        }
        __syncthreads();
        for (int q = 0; q < nt; q++) {
            const double dx = x - sx[q], dy = y - sy[q], dz = z - sz[q];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;  // the singular r' = r term is skipped
            const double r = sqrt(r2);
            acc += exp(-k * r) / r * (sf[q] - fi) * sw[q];
        }
    }
    if (ok) partial[((int64_t)s * nf + o) * n + i] = acc;
}

// u[o][i] = sum_s partial / (4 pi) + f_o[i] / k_o^2 (the SS constant)
__global__ void k_direct_noalloc_reduce(const double* __restrict__ f, NaRates rates, int nf, int64_t n, int splits,
                                        const double* __restrict__ partial, double* u)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * nf) return;
    const int o = (int)(e / n);
    const int64_t i = e % n;
    double S = 0.0;
    for (int s = 0; s < splits; s++) S += partial[((int64_t)s * nf + o) * n + i];
    const double k = rates.k[o];
    u[e] = S / (4.0 * 3.14159265358979323846) + f[e] / (k * k);
}

// Device address of the scratch array, looked up at set-up: once per device
// and CUDA context (the first call with that device current).  Keying on the
// context means that a call after cudaDeviceReset, which unloads the module
// and may load it again elsewhere, repeats the set-up instead of using the
// old address.
using CtxGetCurrent = CUresult (*)(CUcontext*);
std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {nullptr};
CUcontext g_na_ctx[kNaMaxDevices] = {nullptr};
CtxGetCurrent g_ctx_get = nullptr;

double* scratch_address()
{
    int dev = 0;
    TAGI_CUDA(cudaGetDevice(&dev));
    TAGI_REQUIRE(dev >= 0 && dev < kNaMaxDevices, "device ordinal out of range for the no-alloc scratch table");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_ctx_get) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        TAGI_CUDA(cudaGetDriverEntryPoint("cuCtxGetCurrent", &fn, cudaEnableDefault, &q));
        TAGI_REQUIRE(fn != nullptr && q == cudaDriverEntryPointSuccess, "cuCtxGetCurrent is not available");
        g_ctx_get = reinterpret_cast<CtxGetCurrent>(fn);
    }
    // no context may be bound to this host thread yet; the set-up below binds
    // the device's primary context (cudaGetSymbolAddress initialises it)
    CUcontext ctx = nullptr;
    if (g_ctx_get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    if (!ctx || !g_na_ptr[dev] || g_na_ctx[dev] != ctx) {
        void* p = nullptr;
        TAGI_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        TAGI_REQUIRE(g_ctx_get(&ctx) == CUDA_SUCCESS && ctx != nullptr, "no current CUDA context");
        g_na_ptr[dev] = p;
        g_na_ctx[dev] = ctx;
    }
    return static_cast<double*>(g_na_ptr[dev]);
}

}  // namespace
}  // namespace tagi

using namespace tagi;

extern "C" tagi_status tagi_yukawa_direct_noalloc(const double* xyz, const double* w, const double* f,
                                                  const double* k, int nf, int64_t n, double* u, void* stream)
{
    try {
        report_error(TAGI_OK, "");
        TAGI_REQUIRE(xyz && w && f && k && u, "xyz, w, f, k or u is NULL");
        TAGI_REQUIRE(nf >= 1 && nf <= kNaMaxFields && n >= 1, "need 1 <= nf <= 16 and n >= 1");
        TAGI_REQUIRE(n * (int64_t)nf <= kNoAllocScratch,
                     "n * nf exceeds the no-alloc scratch capacity of 1048576 values");
        NaRates rates{};
        for (int o = 0; o < nf; o++) {
            TAGI_REQUIRE(std::isfinite(k[o]) && k[o] > 0.0, "every k must be finite and > 0");
            rates.k[o] = k[o];
        }
        cudaStream_t s = (cudaStream_t)stream;
        double* scratch = scratch_address();
        int splits = kNaMaxSplits;
        while (splits > 1 && (int64_t)splits * nf * n > kNoAllocScratch) splits--;
        // every partial the reduction reads is written by this call first, so
        // nothing left in the array by an earlier call is ever read
        const dim3 grid((unsigned)((n + kNaThreads - 1) / kNaThreads), (unsigned)splits, (unsigned)nf);
        launch(k_direct_noalloc, grid, kNaThreads, 0, s, xyz, w, f, rates, nf, n, splits, scratch);
        launch(k_direct_noalloc_reduce, (int)((n * nf + 255) / 256), 256, 0, s, f, rates, nf, n, splits,
               (const double*)scratch, u);
        TAGI_LAUNCH_CHECK();
        return TAGI_OK;
    } catch (const Error& e) {
        return report_error(e.status, e.what());
    } catch (...) {
        return report_error(TAGI_ERR_CUDA, "unknown error");
    }
}
