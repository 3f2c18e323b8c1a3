// Launchers of the bounded-grid kernels (lbhpde_bounded.cuh): the resident kernel k_bounded,
// one instance per CTA, and the outer-node rebuild k_nee_fix that follows a streaming step.
#include <algorithm>

#include "lbhpde_bounded.cuh"
#include "lbhpde_internal.h"

namespace lbh {

namespace {

#define LBB_CK(call)                  \
    do {                              \
        cudaError_t e_ = (call);      \
        if (e_ != cudaSuccess) {      \
            (void)cudaGetLastError(); \
            return LBHPDE_ERR_CUDA;   \
        }                             \
    } while (0)

struct BoundedArgs {
    int ninst, nthreads;
    size_t smem;
    const lbk::BoundedInst *insts;
    const void *in;
    void *out;
    const void *coefT;
    const double *phib;
    long long stride, step0;
    int nsteps;
    cudaStream_t st;
};

template <typename T, int B, int DC>
int launch_bounded_t(const BoundedArgs &a) {
    auto fn = lbk::k_bounded<T, B, kBoundedK, kBoundedMaxT, DC>;
    LBB_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem));
    fn<<<a.ninst, a.nthreads, a.smem, a.st>>>((const T *)a.in, (T *)a.out, a.insts, (const T *)a.coefT, a.phib,
                                             a.stride, a.step0, a.nsteps);
    LBB_CK(cudaGetLastError());
    return LBHPDE_OK;
}

template <typename T, int B>
int launch_bounded_d(int dc, const BoundedArgs &a) {
    constexpr int DC = B == 5 ? 5 : 7;
    if (dc == DC) return launch_bounded_t<T, B, DC>(a);
    if (dc < 0) return launch_bounded_t<T, B, -1>(a);  // real-exponent members
    return launch_bounded_t<T, B, 0>(a);
}

}  // namespace

size_t bounded_smem(int b, size_t esz, int nthreads, int D, int nsteps) {
    const int W = lbk::wmax(b), NE = lbk::nedge(b), cs = lbk::crow(D);
    return (size_t(4) * NE * nthreads + size_t(2) * (b - 1) * cs + 16 + size_t(nsteps) * 2 * W * b) * esz;
}

int bounded_shift(int b, int N, int depth) {
    const int W = lbk::wmax(b), K = kBoundedK;
    const int kL = W - 1 + depth, kR = N - W - depth;
    for (int shift = 0; kL + shift < 32 * K; ++shift) {
        const bool right_in_one_warp = ((kR + shift) / K) / 32 == ((N - 1 + shift) / K) / 32;
        if (right_in_one_warp && N + shift <= K * kBoundedMaxT) return shift;
    }
    return -1;
}

int bounded_launch_steps(int b, size_t esz) {
    const int per_step = 2 * lbk::wmax(b) * b * (int)esz;  // bytes of staged boundary data per step
    return std::max(32, std::min(kBoundedMaxSteps, kBoundedStageBytes / per_step));
}

int launch_bounded(int b, size_t esz, int dc, int ninst, int nthreads, size_t smem, const lbk::BoundedInst *insts_d,
                   const void *in, void *out, const void *coefT, const double *phib, long long stride,
                   long long step0, int nsteps, cudaStream_t st) {
    if (ninst == 0 || nsteps <= 0) return LBHPDE_OK;
    if (nthreads <= 0 || nthreads > kBoundedMaxT || nthreads % 32) return LBHPDE_ERR_ARG;
    const BoundedArgs a{ninst, nthreads, smem, insts_d, in, out, coefT, phib, stride, step0, nsteps, st};
    if (esz == 4) return b == 5 ? launch_bounded_d<float, 5>(dc, a) : launch_bounded_d<float, 7>(dc, a);
    return b == 5 ? launch_bounded_d<double, 5>(dc, a) : launch_bounded_d<double, 7>(dc, a);
}

int launch_nee_fix(int b, size_t esz, void *st, const lbk::Seg *segs, const int *members, int nmem,
                   const void *coefT, const double *phib, long long stride, long long step, cudaStream_t stream) {
    if (nmem == 0) return LBHPDE_OK;
    if (esz == 4) {
        if (b == 5)
            lbk::k_nee_fix<float, 5><<<nmem, 32, 0, stream>>>((float *)st, segs, members, (const float *)coefT, phib,
                                                              stride, step);
        else
            lbk::k_nee_fix<float, 7><<<nmem, 32, 0, stream>>>((float *)st, segs, members, (const float *)coefT, phib,
                                                              stride, step);
    } else {
        if (b == 5)
            lbk::k_nee_fix<double, 5><<<nmem, 32, 0, stream>>>((double *)st, segs, members, (const double *)coefT,
                                                               phib, stride, step);
        else
            lbk::k_nee_fix<double, 7><<<nmem, 32, 0, stream>>>((double *)st, segs, members, (const double *)coefT,
                                                               phib, stride, step);
    }
    LBB_CK(cudaGetLastError());
    return LBHPDE_OK;
}

}  // namespace lbh
