// On-chip kernel variants in FP64 (a translation unit of its own, so the two precisions
// compile in parallel).
#include "lbhpde_onchip_launch.cuh"

namespace lbh {

int launch_onchip_f64(int b, int K, int dc, bool halo, const Packed &p, const lbk::OnchipInst *insts_d,
                      const int *first_d, const void *in, void *out, const void *coefT, int nsteps, cudaStream_t st) {
    const onchip_launch::OnchipArgs a{&p, insts_d, first_d, in, out, coefT, nsteps, st};
    return onchip_launch::launch_prec<double>(b, K, dc, halo, a);
}

}  // namespace lbh
