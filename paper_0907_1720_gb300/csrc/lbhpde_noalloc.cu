// Diagnostics reduction that allocates nothing: the variant of the two-pass FP64 reduction
// of lbhpde_diagnostics whose scratch (one record per 1024-node block, plus the result)
// lives in file-scope device arrays instead of memory the library allocates.
//
// Every GPU that loads the library holds these arrays (about 1 MiB) until the process exits.
// Host code must not hand the array names to a kernel: on the host they name a stand-in, not
// device memory.  Their device addresses are taken once per device with
// cudaGetSymbolAddress, on the first call made while that device is current, and kept for the
// life of the process: a cudaDeviceReset() of that device would leave them pointing into the
// destroyed context, so the header asks callers not to call the entry point after one.
#include <cuda_runtime.h>

#include <mutex>

#include "lbhpde.h"
#include "lbhpde_kernels.cuh"

namespace {

constexpr int kChunk = 1024;    // nodes per block, as in lbhpde_diagnostics
constexpr int kThreads = 256;
constexpr long kMaxNodes = LBHPDE_NOALLOC_MAX_NODES;
constexpr int kMaxBlocks = (int)((kMaxNodes + kChunk - 1) / kChunk);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) lbk::DiagPart g_part[kMaxBlocks];
static __device__ __align__(256) lbk::DiagPart g_result;

struct Scratch {
    lbk::DiagPart *part = nullptr;
    lbk::DiagPart *result = nullptr;
};
Scratch g_scratch[kMaxDevices];
std::mutex g_mu;

// Pass 1: block i reduces nodes [i * kChunk, (i + 1) * kChunk) of phi into part[i].
__global__ void k_phi_diag_partial(const double *__restrict__ phi, long long n, const double *__restrict__ phistar,
                                   lbk::DiagPart *__restrict__ part) {
    lbk::Seg s{};
    s.off = 0;
    s.N = (int)n;
    lbk::diag_block<double>(phi, s, blockIdx.x * kChunk, kChunk, phistar, part + blockIdx.x);
}

// Pass 2: one thread sums the block records in block order.
__global__ void k_phi_diag_final(const lbk::DiagPart *__restrict__ part, int nblocks,
                                 lbk::DiagPart *__restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    lbk::DiagPart r{};
    for (int i = 0; i < nblocks; ++i) {
        const lbk::DiagPart &p = part[i];
        r.sum += p.sum;
        r.maxabs = fmax(r.maxabs, p.maxabs);
        r.l1d += p.l1d;
        r.l1s += p.l1s;
        r.l2d += p.l2d;
        r.l2s += p.l2s;
        r.nonfinite += p.nonfinite;
    }
    *out = r;
}

// Device addresses of the scratch arrays for the current device (set up on first use).
int scratch_for_current_device(Scratch *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return LBHPDE_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Scratch &s = g_scratch[dev];
    if (!s.part) {
        void *p = nullptr, *r = nullptr;
        if (cudaGetSymbolAddress(&p, g_part) != cudaSuccess || cudaGetSymbolAddress(&r, g_result) != cudaSuccess) {
            (void)cudaGetLastError();
            return LBHPDE_ERR_CUDA;
        }
        s.part = (lbk::DiagPart *)p;
        s.result = (lbk::DiagPart *)r;
    }
    *out = s;
    return LBHPDE_OK;
}

}  // namespace

extern "C" int lbhpde_phi_diagnostics_noalloc(const double *phi_device, long N, const double *phistar_device,
                                              lbhpde_diag *out, void *cuda_stream) {
    if (!phi_device || !out || N <= 0) return LBHPDE_ERR_ARG;
    if (N > kMaxNodes) return LBHPDE_ERR_ARG;
    Scratch s;
    int rc = scratch_for_current_device(&s);
    if (rc != LBHPDE_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nblocks = (int)((N + kChunk - 1) / kChunk);
    k_phi_diag_partial<<<nblocks, kThreads, 0, st>>>(phi_device, N, phistar_device, s.part);
    k_phi_diag_final<<<1, 32, 0, st>>>(s.part, nblocks, s.result);
    lbk::DiagPart h{};
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, s.result, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return LBHPDE_ERR_CUDA;
    }
    out->sum_phi = h.sum;
    out->max_abs_phi = h.maxabs;
    out->nonfinite = (long)h.nonfinite;
    out->err_E = phistar_device ? h.l1d / h.l1s : 0.0;
    out->err_L2 = phistar_device ? sqrt(h.l2d / h.l2s) : 0.0;
    out->steps = 0;
    return h.nonfinite ? LBHPDE_ERR_DIVERGED : LBHPDE_OK;
}
