// Launch of the 16-node resident kernel (k_ring, FP32 D1Q5), a translation unit of its own so it
// compiles in parallel with the other kernels.
#include <cuda_runtime.h>

#include <algorithm>

#include "lbhpde.h"
#include "lbhpde_internal.h"
#include "lbhpde_ring.cuh"
#include "lbhpde_ring_nee.cuh"

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

namespace {

template <int MAXT, int DC, bool D2>
int launch_ring_nee_t(const PackedNee &p, const lbk::RingNeeInst *insts, const int *first, const void *in, void *out,
                      const void *coefT, const double *phib, long long stride, long long step0, int nsteps,
                      cudaStream_t st) {
    auto fn = lbk::k_ring_nee<float, 5, kRingK, MAXT, DC, D2>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return LBHPDE_ERR_CUDA;
    }
    fn<<<p.ncta(), p.nthreads, p.smem, st>>>((const float *)in, (float *)out, insts, first, (const float *)coefT, phib,
                                             stride, step0, nsteps);
    if (cudaGetLastError() != cudaSuccess) return LBHPDE_ERR_CUDA;
    return LBHPDE_OK;
}

template <int MAXT>
int launch_ring_nee_d(int dc, const PackedNee &p, const lbk::RingNeeInst *insts, const int *first, const void *in,
                      void *out, const void *coefT, const double *phib, long long stride, long long step0, int nsteps,
                      cudaStream_t st) {
    if (dc == 5 && p.d2)
        return launch_ring_nee_t<MAXT, 5, true>(p, insts, first, in, out, coefT, phib, stride, step0, nsteps, st);
    if (dc == 5) return launch_ring_nee_t<MAXT, 5, false>(p, insts, first, in, out, coefT, phib, stride, step0, nsteps, st);
    if (dc == 0 && p.d2)
        return launch_ring_nee_t<MAXT, 0, true>(p, insts, first, in, out, coefT, phib, stride, step0, nsteps, st);
    if (dc == 0) return launch_ring_nee_t<MAXT, 0, false>(p, insts, first, in, out, coefT, phib, stride, step0, nsteps, st);
    return LBHPDE_ERR_UNSUPPORTED;
}

}  // namespace

bool ring_nee_ok(size_t esz, int b, const lbk::Seg &s) {
    const int W = lbk::wmax(b);
    return esz == 4 && b == 5 && s.A == 0 && s.pad >= 1 && s.N - 2 * W <= 512 * kRingK && s.N >= 2 * (W + s.pad);
}

int pack_ring_nee(int b, int dc, const std::vector<NeeMember> &m, PackedNee &out, int threads) {
    out = PackedNee{};
    const int W = lbk::wmax(b), K = kRingK;
    // one helper thread per (instance, outer node, population j >= 1) must exist in the CTA
    const int hper = 2 * lbk::nedge(b);
    const int max_inst = std::min(lbk::kRingMaxInst, threads / hper);
    auto thr = [&](const NeeMember &x) { return (x.seg.N - 2 * W + K - 1) / K; };
    std::vector<int> order(m.size());
    for (size_t i = 0; i < m.size(); ++i) {
        if (thr(m[i]) > threads) return LBHPDE_ERR_UNSUPPORTED;
        order[i] = (int)i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return thr(m[a]) > thr(m[c]); });
    struct Cta {
        int used = 0;
        std::vector<int> inst;
    };
    std::vector<Cta> ctas;
    // depth 2 with x_f of the right end in the last thread (at least 2 nodes there) in every
    // member: the variant that rebuilds the inflow at fixed register positions
    out.d2 = true;
    for (const NeeMember &x : m) {
        const int last_nodes = x.seg.N - 2 * W - K * (thr(x) - 1);
        if (x.seg.pad != 2 || last_nodes < 2) out.d2 = false;
    }
    for (int i : order) {
        bool placed = false;
        for (auto &c : ctas)
            if (c.used + thr(m[i]) <= threads && (int)c.inst.size() < max_inst) {
                c.inst.push_back(i);
                c.used += thr(m[i]);
                placed = true;
                break;
            }
        if (!placed) ctas.push_back(Cta{thr(m[i]), {i}});
    }
    size_t coef_max = 0;
    for (auto &c : ctas) {
        out.first.push_back((int)out.insts.size());
        int tb = 0, sco = 0, il = 0;
        for (int i : c.inst) {
            const lbk::Seg &s = m[i].seg;
            lbk::RingNeeInst I{};
            I.off = s.off;
            I.off2 = s.off;
            I.ld = s.ld;
            I.N = s.N;
            I.D = s.D;
            I.gcoef = s.coef;
            I.scoef = sco;
            I.tbase = tb;
            I.nthr = thr(m[i]);
            I.mi = m[i].mi;
            I.depth = s.pad;
            I.il = il++;
            I.steps = m[i].steps;
            out.insts.push_back(I);
            sco += lbk::nee_cblock(b, dc > 0 ? dc : s.D);
            tb += I.nthr;
        }
        out.nthreads = std::max(out.nthreads, std::max(tb, il * hper));
        coef_max = std::max(coef_max, (size_t)sco);
    }
    out.first.push_back((int)out.insts.size());
    out.nthreads = (out.nthreads + 31) & ~31;
    out.stride = threads;
    out.smem = (size_t(lbk::nee_fixed_elems(b, threads)) + coef_max) * sizeof(float);
    if (out.smem > 227 * 1024) return LBHPDE_ERR_UNSUPPORTED;
    return LBHPDE_OK;
}

int launch_ring_nee_f32(int dc, const PackedNee &p, const lbk::RingNeeInst *insts_d, const int *first_d,
                        const void *in, void *out, const void *coefT, const double *phib, long long stride,
                        long long step0, int nsteps, cudaStream_t st) {
    if (p.ncta() == 0 || nsteps <= 0) return LBHPDE_OK;
    if (p.nthreads > p.stride || p.nthreads % 32 != 0) return LBHPDE_ERR_ARG;
    for (int c = 0; c < p.ncta(); ++c)  // every helper role has its thread
        if ((p.first[c + 1] - p.first[c]) * lbk::nee_roles(5) > p.nthreads) return LBHPDE_ERR_ARG;
    if (p.stride == 512)
        return launch_ring_nee_d<512>(dc, p, insts_d, first_d, in, out, coefT, phib, stride, step0, nsteps, st);
    return LBHPDE_ERR_UNSUPPORTED;
}

}  // namespace lbh
