// Launch of the on-chip kernel (k_onchip) for one precision: the variant for the lattice, nodes
// per thread, CTA size class and f^eq degree of a packed plan.  Included by
// lbhpde_onchip_f32.cu and lbhpde_onchip_f64.cu, which instantiate the kernels of one precision
// each and compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "lbhpde.h"
#include "lbhpde_internal.h"
#include "lbhpde_kernels.cuh"

namespace lbh {
namespace onchip_launch {

using lbk::OnchipInst;

#define LBH_OCK(call)                     \
    do {                                  \
        cudaError_t e_ = (call);          \
        if (e_ != cudaSuccess) {          \
            (void)cudaGetLastError();     \
            return LBHPDE_ERR_CUDA;       \
        }                                 \
    } while (0)

struct OnchipArgs {
    const Packed *p;
    const OnchipInst *insts;
    const int *first;
    const void *in;
    void *out;
    const void *coefT;
    int nsteps;
    cudaStream_t st;
};

template <typename T, int B, int K, int MAXT, bool HALO, int DC>
int launch_onchip_t(const OnchipArgs &a) {
    auto fn = lbk::k_onchip<T, B, K, MAXT, HALO, DC>;
    LBH_OCK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.p->smem));
    fn<<<a.p->ncta(), a.p->nthreads, a.p->smem, a.st>>>((const T *)a.in, (T *)a.out, a.insts, a.first,
                                                         (const T *)a.coefT, a.nsteps, a.p->max_inst);
    LBH_OCK(cudaGetLastError());
    return LBHPDE_OK;
}

// compile-time polynomial degree: D = 5 on D1Q5 and D = 7 on D1Q7 (the KdV/KS/KdV-Burgers and
// Kawahara families), run-time degree otherwise
template <typename T, int B, int K, int MAXT, bool HALO>
int launch_onchip_d(int dc, const OnchipArgs &a) {
    constexpr int DC = B == 5 ? 5 : 7;
    if (dc == DC) return launch_onchip_t<T, B, K, MAXT, HALO, DC>(a);
    if (dc < 0) {  // real exponents: evaluated four nodes at a time, so K >= 4
        if constexpr (K >= 4) return launch_onchip_t<T, B, K, MAXT, HALO, -1>(a);
        return LBHPDE_ERR_UNSUPPORTED;
    }
    return launch_onchip_t<T, B, K, MAXT, HALO, 0>(a);
}

template <typename T, int B, bool HALO>
int launch_onchip_b(int K, int dc, const OnchipArgs &a) {
    if constexpr (sizeof(T) == 4) {
        if constexpr (B == 5) {
            if (K == 8) {  // CTAs of 128, 256 (resident only) or 512 threads: the plan's size class
                if (a.p->nthreads <= 128) return launch_onchip_d<T, B, 8, 128, HALO>(dc, a);
                if constexpr (!HALO) {
                    if (a.p->nthreads <= 256) return launch_onchip_d<T, B, 8, 256, HALO>(dc, a);
                }
                return launch_onchip_d<T, B, 8, 512, HALO>(dc, a);
            }
            if (K == 4) return launch_onchip_d<T, B, 4, 1024, HALO>(dc, a);
            if (K == 2) return launch_onchip_d<T, B, 2, 1024, HALO>(dc, a);
        } else {
            if (K == 8) return launch_onchip_d<T, B, 8, 256, HALO>(dc, a);
            if (K == 4) return launch_onchip_d<T, B, 4, 512, HALO>(dc, a);
        }
    } else {
        if constexpr (B == 5) {
            if (K == 4) return launch_onchip_d<T, B, 4, 512, HALO>(dc, a);
            if (K == 2) return launch_onchip_d<T, B, 2, 1024, HALO>(dc, a);
        } else {
            if (K == 4) return launch_onchip_d<T, B, 4, 256, HALO>(dc, a);
        }
    }
    return LBHPDE_ERR_UNSUPPORTED;
}

template <typename T>
int launch_prec(int b, int K, int dc, bool halo, const OnchipArgs &a) {
    if (b == 5) return halo ? launch_onchip_b<T, 5, true>(K, dc, a) : launch_onchip_b<T, 5, false>(K, dc, a);
    return halo ? launch_onchip_b<T, 7, true>(K, dc, a) : launch_onchip_b<T, 7, false>(K, dc, a);
}

#undef LBH_OCK

}  // namespace onchip_launch
}  // namespace lbh
