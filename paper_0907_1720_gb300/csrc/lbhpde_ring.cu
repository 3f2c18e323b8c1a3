// Launch of the 16-node resident kernel (k_ring, FP32 D1Q5), a translation unit of its own so it
// compiles in parallel with the other kernels.
#include <cuda_runtime.h>

#include "lbhpde.h"
#include "lbhpde_internal.h"
#include "lbhpde_ring.cuh"

namespace lbh {

namespace {

template <int MAXT, int DC>
int launch_ring_t(const Packed &p, const lbk::OnchipInst *insts, const int *first, const void *in, void *out,
                  const void *coefT, int nsteps, cudaStream_t st) {
    auto fn = lbk::k_ring<float, 5, kRingK, MAXT, DC>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return LBHPDE_ERR_CUDA;
    }
    fn<<<p.ncta(), p.nthreads, p.smem, st>>>((const float *)in, (float *)out, insts, first, (const float *)coefT,
                                             nsteps);
    if (cudaGetLastError() != cudaSuccess) return LBHPDE_ERR_CUDA;
    return LBHPDE_OK;
}

template <int MAXT>
int launch_ring_d(int dc, const Packed &p, const lbk::OnchipInst *insts, const int *first, const void *in, void *out,
                  const void *coefT, int nsteps, cudaStream_t st) {
    if (dc == 5) return launch_ring_t<MAXT, 5>(p, insts, first, in, out, coefT, nsteps, st);
    if (dc == 0) return launch_ring_t<MAXT, 0>(p, insts, first, in, out, coefT, nsteps, st);
    return LBHPDE_ERR_UNSUPPORTED;
}

}  // namespace

// The 16-node resident kernel (FP32 D1Q5) compiled for the plan's class: CTAs of up to 128, 256 or
// 512 threads, whose exchange rows have that stride.
int launch_ring_f32(int dc, const Packed &p, const lbk::OnchipInst *insts_d, const int *first_d, const void *in,
                    void *out, const void *coefT, int nsteps, cudaStream_t st) {
    if (p.nthreads > p.stride || p.nthreads % 32 != 0 || p.max_inst > lbk::kRingMaxInst) return LBHPDE_ERR_ARG;
    if (p.stride == 128) return launch_ring_d<128>(dc, p, insts_d, first_d, in, out, coefT, nsteps, st);
    if (p.stride == 256) return launch_ring_d<256>(dc, p, insts_d, first_d, in, out, coefT, nsteps, st);
    if (p.stride == 512) return launch_ring_d<512>(dc, p, insts_d, first_d, in, out, coefT, nsteps, st);
    return LBHPDE_ERR_UNSUPPORTED;
}

}  // namespace lbh
