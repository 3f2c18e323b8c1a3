// C ABI of the solver: batches of periodic instances (and the single-instance handle as a
// batch of one).  Host planning (arena layout, block maps, CTA packing), kernel launches,
// readout and diagnostics.  See include/lbhpde.h for the contract of each entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "lbhpde.h"
#include "lbhpde_internal.h"
#include "lbhpde_kernels.cuh"

using lbh::kChunk;
using lbh::kGenericThreads;
using lbk::DiagPart;
using lbk::OnchipInst;
using lbk::Seg;

namespace {

constexpr int kStreamThreads = kChunk / 4;  // k_stream: one group of 4 nodes per thread
constexpr int kGraphSteps = 64;             // one-step launches per captured graph (even)

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            (void)cudaGetLastError();                         \
            return LBHPDE_ERR_CUDA;                           \
        }                                                     \
    } while (0)

#define RC(call)                    \
    do {                            \
        int r_ = (call);            \
        if (r_ != LBHPDE_OK) return r_; \
    } while (0)

// One kernel group: the instances of one lattice (the kernels are compiled per b).
struct Group {
    int b = 0;
    std::vector<int> members;     // batch indices
    int maxD = 0;
    // node-parallel block map (segment, first node), kChunk nodes per block
    std::vector<int2> blocks_h;
    int2 *blocks = nullptr;
    long long *blk_off = nullptr;  // per block: offset of its member in a concatenated phi array
    // on-chip plans: whole instances resident for all steps (ring) and temporally blocked
    // windows for instances longer than one CTA holds (halo)
    bool onchip_ok = false;  // false: every member uses the streaming kernel
    struct Plan {
        lbh::Packed host;
        OnchipInst *insts = nullptr;
        int *cta_first = nullptr;
        int ncta() const { return host.ncta(); }
    } ring[lbh::kRingClasses], halo;  // resident instances by CTA size class; windows
    int K = 0, maxt = 0, tblk = 0;
    int Kr = 0;  // nodes per thread of the resident plans (lbh::kRingK: k_ring)
    int Kt = 0;  // nodes per thread of the tail of a plan in whole waves
    int dc = 0;  // compile-time degree of the on-chip kernel variant (0 = run time)
    bool uniform = false;  // every member has the same model (coefficients and omega)
    bool has_nu = false;   // a member has real-exponent terms: the real-exponent variants (on chip: degree code -1)
    bool waves = false;    // ring[2]: whole waves of full CTAs; ring[0]: the tail, launched after it
    // bounded groups (LBHPDE_NEE): resident members, one CTA each, and streaming members
    std::vector<lbk::BoundedInst> bnd_h;
    lbk::BoundedInst *bnd = nullptr;
    int bnd_threads = 0, bnd_dc = 0, bnd_D = 0;
    lbh::PackedNee rn_h;               // bounded members on the 16-node resident kernel
    lbk::RingNeeInst *rn_insts = nullptr;
    int *rn_first = nullptr;
    int rn_dc = 0;
    std::vector<int> smembers_h;       // streaming members
    int *smembers = nullptr;
    std::vector<int2> sblocks_h;       // their node blocks (kChunk nodes each)
    int2 *sblocks = nullptr;
};

}  // namespace

struct lbhpde_batch_s {
    int precision = LBHPDE_FP64;
    size_t esz = 8;
    int count = 0;
    cudaStream_t stream = nullptr;
    // resident instances run on `side`, forked from and joined back into `stream` with events,
    // so that the window launches fill the SMs the resident launch leaves idle
    cudaStream_t side[lbh::kRingClasses] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[lbh::kRingClasses] = {};
    // streaming path: kGraphSteps one-step launches captured once per buffer parity and replayed
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool has_alloc = false;
    lbhpde_allocator alloc{};
    std::vector<lbhpde_model_info> mi;
    std::vector<long long> N;
    std::vector<int> depth;          // per member: NEE extrapolation depth, 0 = periodic
    std::vector<long long> phi_off;  // prefix sums of N: concatenated host/device phi arrays
    long long total = 0;
    std::vector<Seg> segs_h;
    Seg *segs = nullptr;
    void *st[2] = {nullptr, nullptr};
    size_t st_bytes = 0;
    int cur = 0;
    void *coefT = nullptr;  // coefficient arena in the state type
    double *coefD = nullptr;  // FP64 batches: the table in double (coefT points to it)
    long long *phi_off_d = nullptr;  // per block of the combined map: offset into a concatenated array
    std::vector<int2> all_blocks_h;  // combined block map over all members (segment order)
    std::vector<int> part_first_h;
    int2 *all_blocks = nullptr;
    long long *blk_off = nullptr;
    int *part_first = nullptr;
    DiagPart *part = nullptr;      // scratch: one record per block of the combined map
    DiagPart *diag_out = nullptr;  // one record per member
    double *phi_buf = nullptr;     // device staging of phi in double (host transfers)
    int *nonfinite = nullptr;      // readout flag: a non-finite phi was copied
    Group groups[2];               // periodic members: b = 5, b = 7
    Group bgroups[2];              // bounded members: b = 5, b = 7
    int nbounded = 0;
    double *phib_buf = nullptr;    // device copy of host boundary values
    size_t phib_cap = 0;           // its capacity in doubles
    int kernel = LBHPDE_KERNEL_AUTO;
    int K_req = 0, spl_req = 0;
    long long launches = 0;          // kernels launched (a graph replay counts its kernels)
    long long graph_launches[2] = {0, 0};  // kernels in each captured graph
    long steps = 0;
    bool initialised = false;
    std::vector<std::pair<void *, size_t>> allocations;

    int dev_alloc(void **p, size_t bytes) {
        bytes = std::max<size_t>(bytes, 256);
        void *q = nullptr;
        if (has_alloc) {
            q = alloc.alloc(bytes, (void *)stream, alloc.user);
            if (!q) return LBHPDE_ERR_OOM;
        } else {
            cudaError_t e = cudaMalloc(&q, bytes);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return e == cudaErrorMemoryAllocation ? LBHPDE_ERR_OOM : LBHPDE_ERR_CUDA;
            }
        }
        allocations.emplace_back(q, bytes);
        *p = q;
        return LBHPDE_OK;
    }
    // Release one allocation made by dev_alloc (waits for the stream first: kernels in flight may
    // still read it).  nullptr is ignored.
    void dev_free(void *p) {
        if (!p) return;
        for (size_t i = 0; i < allocations.size(); ++i)
            if (allocations[i].first == p) {
                cudaStreamSynchronize(stream);
                if (has_alloc)
                    alloc.release(p, allocations[i].second, (void *)stream, alloc.user);
                else
                    cudaFree(p);
                allocations.erase(allocations.begin() + i);
                return;
            }
    }
    template <typename X>
    int upload(X **dst, const std::vector<X> &src) {
        RC(dev_alloc((void **)dst, sizeof(X) * std::max<size_t>(src.size(), 1)));
        if (!src.empty())
            CK(cudaMemcpyAsync(*dst, src.data(), sizeof(X) * src.size(), cudaMemcpyHostToDevice, stream));
        return LBHPDE_OK;
    }
    void free_all() {
        cudaStreamSynchronize(stream);
        for (auto &a : allocations) {
            if (has_alloc)
                alloc.release(a.first, a.second, (void *)stream, alloc.user);
            else
                cudaFree(a.first);
        }
        allocations.clear();
        for (auto &gx : graph)
            if (gx) cudaGraphExecDestroy(gx);
        graph[0] = graph[1] = nullptr;
        for (int c = 0; c < lbh::kRingClasses; ++c) {
            if (side[c]) cudaStreamDestroy(side[c]);
            if (ev_join[c]) cudaEventDestroy(ev_join[c]);
            side[c] = nullptr;
            ev_join[c] = nullptr;
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        ev_fork = nullptr;
        stream = nullptr;
    }
};

struct lbhpde_ctx {
    lbhpde_batch_s *b = nullptr;
};

// ===================================================== shared on-chip planning and launch

namespace lbh {

int onchip_maxt(size_t esz, int b, int K) {
    if (esz == 4) {
        if (b == 5) return K == kRingK ? 512 : (K == 8 ? 512 : (K == 4 ? 1024 : (K == 2 ? 1024 : 0)));  // resident CTAs
        return K == 8 ? 256 : (K == 4 ? 512 : 0);
    }
    if (b == 5) return K == 4 ? 512 : (K == 2 ? 1024 : 0);
    return K == 4 ? 256 : 0;
}

// Threads of a window CTA.  FP32 D1Q5 windows with K = 8 take 128 threads (96 registers), so
// five CTAs share an SM: some load or write back their windows while others compute, and their
// per-step barriers fall at different times.  (Measured on GB300: 5.92e11 node-updates/s on the
// ensemble against 5.80e11 with 256 threads and 5.61e11 with 512; the D1Q7 and FP64 windows
// were slower with 128 threads than with their resident CTA size.)
int onchip_maxt_halo(size_t esz, int b, int K) {
    if (K == kRingK) return 0;  // the 16-node variant holds resident instances only
    if (esz == 4 && b == 5 && K == 8) return kHaloThreadsF32Q5;
    return onchip_maxt(esz, b, K);
}

bool ring_split_ok(size_t esz, int b, int dc) { return esz == 4 && b == 5 && dc >= 0; }

int default_K(size_t esz, int b) { return esz == 4 && b == 5 ? 8 : 4; }

// Resident size classes.  FP32 D1Q5 with K = 8 puts an instance in the smallest of 128-, 256- and
// 512-thread CTAs that holds it (classes 0, 1, 2): small CTAs share an SM (128 registers a
// thread) and step on their own barriers.  (GB300, 1000 steps: 1024-node instances 6.77e11
// node-updates/s in 128-thread CTAs against 5.73e11 packed four to a 512-thread CTA; 2048-node
// ones 6.52e11 against 6.24e11.)  Other configurations have class 2 only.
int ring_class(size_t esz, int b, int K, long long N) {
    if (esz == 4 && b == 5 && (K == 8 || K == kRingK)) return N <= 128 * K ? 0 : (N <= 256 * K ? 1 : 2);
    return 2;
}
int ring_class_threads(size_t esz, int b, int K, int cls) {
    if (esz == 4 && b == 5 && (K == 8 || K == kRingK)) return cls == 0 ? 128 : (cls == 1 ? 256 : 512);
    return onchip_maxt(esz, b, K);
}
// Threads an instance's run is rounded up to: whole warps for k_onchip, single threads for
// k_ring (its instances may share a warp)
int ring_granule(int K) { return K == kRingK ? 1 : 32; }

void split_ring_classes(size_t esz, int b, int K, const std::vector<Member> &m, std::vector<Member> (&out)[kRingClasses]) {
    for (auto &v : out) v.clear();
    const int gr = ring_granule(K);
    auto pad = [&](long long n) { return (int)(((n + K - 1) / K + gr - 1) / gr * gr); };
    std::vector<int> order(m.size());
    for (size_t i = 0; i < m.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return pad(m[a].seg.N) > pad(m[c].seg.N); });
    // the largest class first, first fit, as pack_ring will place it; then a smaller instance
    // joins it where it fills a gap (an idle warp costs as much as a busy one) and takes a CTA
    // of its own class otherwise
    const int top = kRingClasses - 1, cap = ring_class_threads(esz, b, K, top);
    struct Gap {
        int free, n;
    };
    std::vector<Gap> ctas;
    for (int i : order) {
        const int c = ring_class(esz, b, K, m[i].seg.N), t = pad(m[i].seg.N);
        bool placed = false;
        for (auto &g : ctas)
            if (g.free >= t && g.n < kRingMaxInstances) {
                g.free -= t;
                ++g.n;
                placed = true;
                break;
            }
        if (!placed && c == top) {
            ctas.push_back(Gap{cap - t, 1});
            placed = true;
        }
        out[placed ? top : c].push_back(m[i]);
    }
}

int default_tblk(int capacity, int W, int valid_eighths) {
    int t = 64;
    while (t > 1 && capacity - 2 * t * W < capacity * valid_eighths / 8) t /= 2;
    return t;
}

int onchip_dc(int b, int maxD) { return maxD == (b == 5 ? 5 : 7) ? maxD : 0; }

bool split_ring_waves(int b, int K, int sms, const std::vector<Member> &m, std::vector<Member> &full,
                      std::vector<Member> &tail) {
    full.clear();
    tail.clear();
    if (K != kRingK || sms <= 0) return false;
    const int cap = ring_class_threads(4, b, K, kRingClasses - 1);
    auto thr = [&](int i) { return (int)((m[i].seg.N + K - 1) / K); };
    std::vector<int> order(m.size());
    long long total = 0;
    for (size_t i = 0; i < m.size(); ++i) {
        order[i] = (int)i;
        total += thr((int)i);
    }
    const long long limit = total / ((long long)sms * cap) * sms;  // CTAs of the whole waves
    if (limit == 0) return false;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return thr(a) > thr(c); });
    // first fit, largest first, into at most `limit` CTAs; then each member that fitted nowhere
    // takes the CTA where evicting the fewest smaller members makes room, and the evicted members
    // (the smallest at hand) form the tail
    struct Cta {
        int used = 0;
        std::vector<int> inst;
    };
    std::vector<Cta> ctas;
    std::vector<int> deferred, evicted;
    for (int i : order) {
        const int t = thr(i);
        bool placed = false;
        for (auto &c : ctas)
            if (c.used + t <= cap && (int)c.inst.size() < kRingMaxInstances) {
                c.inst.push_back(i);
                c.used += t;
                placed = true;
                break;
            }
        if (placed) continue;
        if ((long long)ctas.size() < limit)
            ctas.push_back(Cta{t, {i}});
        else
            deferred.push_back(i);
    }
    for (int i : deferred) {
        const int t = thr(i);
        int best = -1, best_n = 1 << 30;
        for (size_t c = 0; c < ctas.size(); ++c) {
            std::vector<int> small;
            for (int q : ctas[c].inst)
                if (thr(q) < t) small.push_back(thr(q));
            std::sort(small.begin(), small.end());
            int room = cap - ctas[c].used, n = 0;
            for (int x : small) {
                if (room >= t) break;
                room += x;
                ++n;
            }
            if (room >= t && n < best_n) {
                best = (int)c;
                best_n = n;
                if (n <= 1) break;
            }
        }
        if (best < 0) {
            evicted.push_back(i);
            continue;
        }
        Cta &c = ctas[best];
        std::stable_sort(c.inst.begin(), c.inst.end(), [&](int a, int d) { return thr(a) < thr(d); });
        while (cap - c.used < t) {
            size_t k = 0;
            while (thr(c.inst[k]) >= t) ++k;  // the smallest member below t (one exists: room >= t)
            c.used -= thr(c.inst[k]);
            evicted.push_back(c.inst[k]);
            c.inst.erase(c.inst.begin() + (long)k);
        }
        c.inst.push_back(i);
        c.used += t;
    }
    if (evicted.empty()) return false;
    for (auto &c : ctas)
        for (int q : c.inst) full.push_back(m[q]);
    for (int q : evicted) tail.push_back(m[q]);
    return true;
}

int pack_ring(int b, size_t esz, int K, int dc, const std::vector<Member> &m, Packed &out, int threads) {
    out = Packed{};
    const int maxt = threads > 0 ? threads : onchip_maxt(esz, b, K);
    if (maxt == 0) return LBHPDE_ERR_UNSUPPORTED;
    auto thr = [&](long long n) { return (int)((n + K - 1) / K); };
    const int gr = ring_granule(K);
    auto pad = [&](long long n) { return (thr(n) + gr - 1) / gr * gr; };
    std::vector<int> order(m.size());
    for (size_t i = 0; i < m.size(); ++i) {
        if ((long long)m[i].seg.N > (long long)maxt * K) return LBHPDE_ERR_UNSUPPORTED;
        order[i] = (int)i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return pad(m[a].seg.N) > pad(m[c].seg.N); });
    struct Cta {
        int used = 0;
        std::vector<int> inst;
    };
    std::vector<Cta> ctas;
    for (int i : order) {
        bool placed = false;
        for (auto &c : ctas) {
            if (c.used + pad(m[i].seg.N) <= maxt && (int)c.inst.size() < kRingMaxInstances) {
                c.inst.push_back(i);
                c.used += pad(m[i].seg.N);
                placed = true;
                break;
            }
        }
        if (!placed) {
            Cta c;
            c.inst.push_back(i);
            c.used = pad(m[i].seg.N);
            ctas.push_back(c);
        }
    }
    size_t coef_max = 0;
    for (auto &c : ctas) {
        out.first.push_back((int)out.insts.size());
        int tb = 0, sco = 0, il = 0;
        for (int i : c.inst) {
            const Seg &s = m[i].seg;
            OnchipInst I{};
            I.off = s.off;
            I.off2 = m[i].off2;
            I.ld = s.ld;
            I.N = s.N;
            I.D = s.D;
            I.gcoef = s.coef;
            I.scoef = sco;
            I.tbase = tb;
            I.nthr = thr(s.N);
            I.il = il++;
            I.x0 = 0;
            I.npos = s.N;
            I.vlo = 0;
            I.vhi = s.N;
            I.steps = m[i].steps;
            I.A = s.A;
            I.Dg = s.Dg;
            I.nu = s.nu;
            out.insts.push_back(I);
            sco += lbk::cblock(b, dc > 0 ? dc : s.D);
            tb += pad(s.N);
        }
        out.nthreads = std::max(out.nthreads, tb);
        out.max_inst = std::max(out.max_inst, (int)c.inst.size());
        coef_max = std::max(coef_max, (size_t)sco);
    }
    out.first.push_back((int)out.insts.size());
    out.nthreads = (out.nthreads + 31) & ~31;
    out.max_inst = (out.max_inst + 3) & ~3;  // keeps the shared-memory coefficient rows 16-byte aligned
    const int ne = lbk::nedge(b);
    if (K == kRingK) {  // exchange rows and tails at the class's CTA size
        out.stride = maxt;
        out.smem = (size_t(lbk::ring_xchg_elems(b, maxt)) + coef_max) * esz;
    } else {
        out.smem = (size_t(4) * ne * out.nthreads + size_t(2) * ne * out.max_inst + coef_max) * esz;
    }
    if (out.smem > 227 * 1024) return LBHPDE_ERR_UNSUPPORTED;
    return LBHPDE_OK;
}

int pack_halo(int b, size_t esz, int K, int dc, int H, const std::vector<Member> &m, Packed &out, bool wide) {
    out = Packed{};
    const int maxt = wide ? onchip_maxt(esz, b, K) : onchip_maxt_halo(esz, b, K);
    if (maxt == 0) return LBHPDE_ERR_UNSUPPORTED;
    const int valid = maxt * K - 2 * H;
    if (valid < 32) return LBHPDE_ERR_UNSUPPORTED;
    size_t coef_max = 0;
    for (const Member &mb : m) {
        const Seg &s = mb.seg;
        for (long long x = 0; x < s.N; x += valid) {
            const int v = (int)std::min<long long>(valid, s.N - x);
            OnchipInst I{};
            I.off = s.off;
            I.off2 = mb.off2;
            I.ld = s.ld;
            I.N = s.N;
            I.D = s.D;
            I.gcoef = s.coef;
            I.scoef = 0;
            I.tbase = 0;
            I.npos = v + 2 * H;
            I.nthr = (I.npos + K - 1) / K;
            I.il = 0;
            I.x0 = (int)(x - H);
            I.vlo = H;
            I.vhi = H + v;
            I.steps = mb.steps;
            I.A = s.A;
            I.Dg = s.Dg;
            I.nu = s.nu;
            out.first.push_back((int)out.insts.size());
            out.insts.push_back(I);
            coef_max = std::max(coef_max, (size_t)lbk::cblock(b, dc > 0 ? dc : s.D));
        }
    }
    out.first.push_back((int)out.insts.size());
    out.nthreads = maxt;
    out.max_inst = 1;
    out.smem = (size_t(4) * lbk::nedge(b) * maxt + coef_max) * esz;
    return LBHPDE_OK;
}

namespace {

#define LBH_CK(call)                      \
    do {                                  \
        cudaError_t e_ = (call);          \
        if (e_ != cudaSuccess) {          \
            (void)cudaGetLastError();     \
            return LBHPDE_ERR_CUDA;       \
        }                                 \
    } while (0)

}  // namespace

int launch_onchip(int b, size_t esz, int K, int dc, bool halo, const Packed &p, const OnchipInst *insts_d,
                  const int *first_d, const void *in, void *out, const void *coefT, int nsteps, cudaStream_t st) {
    if (p.ncta() == 0 || nsteps <= 0) return LBHPDE_OK;
    if (K == kRingK) {
        if (halo || esz != 4 || b != 5) return LBHPDE_ERR_UNSUPPORTED;
        return launch_ring_f32(dc, p, insts_d, first_d, in, out, coefT, nsteps, st);
    }
    return esz == 4 ? launch_onchip_f32(b, K, dc, halo, p, insts_d, first_d, in, out, coefT, nsteps, st)
                    : launch_onchip_f64(b, K, dc, halo, p, insts_d, first_d, in, out, coefT, nsteps, st);
}

int launch_init(int b, size_t esz, void *st, const Seg *segs, const int2 *blocks, int nb, const void *coefT,
                const double *phi0, const long long *blk_off, cudaStream_t stream) {
    if (nb == 0) return LBHPDE_OK;
    if (esz == 4) {
        const float *cf = (const float *)coefT;
        if (b == 5)
            lbk::k_init<float, 5><<<nb, kGenericThreads, 0, stream>>>((float *)st, segs, blocks, cf, phi0, blk_off,
                                                                       kChunk);
        else
            lbk::k_init<float, 7><<<nb, kGenericThreads, 0, stream>>>((float *)st, segs, blocks, cf, phi0, blk_off,
                                                                       kChunk);
    } else {
        const double *cd = (const double *)coefT;
        if (b == 5)
            lbk::k_init<double, 5><<<nb, kGenericThreads, 0, stream>>>((double *)st, segs, blocks, cd, phi0,
                                                                        blk_off, kChunk);
        else
            lbk::k_init<double, 7><<<nb, kGenericThreads, 0, stream>>>((double *)st, segs, blocks, cd, phi0,
                                                                        blk_off, kChunk);
    }
    LBH_CK(cudaGetLastError());
    return LBHPDE_OK;
}

}  // namespace lbh

// ============================================================================= autotuner

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tuned;  // (esz, b, dc) -> (K, tblk)

bool tuned_choice(size_t esz, int b, int dc, int *K, int *tblk) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple((int)esz, b, dc));
    if (it == g_tuned.end()) return false;
    *K = it->second.first;
    *tblk = it->second.second;
    return true;
}

// Time one (K, tblk) candidate: temporally blocked windows over a synthetic periodic grid of
// n nodes (zero state, zero polynomial; the kernel's work does not depend on the values).
int time_candidate(size_t esz, int b, int dc, int K, int tblk, long long n, void *buf0, void *buf1, void *coef,
                   cudaStream_t st, double *rate) {
    const int W = lbk::wmax(b);
    lbh::Member m{};
    m.seg.off = 0;
    m.seg.ld = n;
    m.seg.N = (int)n;
    m.seg.D = dc > 0 ? dc : 5;
    m.seg.coef = 0;
    m.off2 = 0;
    m.steps = tblk;
    lbh::Packed p;
    RC(lbh::pack_halo(b, esz, K, dc, tblk * W, {m}, p));
    lbk::OnchipInst *insts = nullptr;
    int *first = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBHPDE_OK;
    if (cudaMalloc(&insts, sizeof(lbk::OnchipInst) * p.insts.size()) != cudaSuccess ||
        cudaMalloc(&first, sizeof(int) * p.first.size()) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = LBHPDE_ERR_CUDA;
    if (rc == LBHPDE_OK) {
        cudaMemcpyAsync(insts, p.insts.data(), sizeof(lbk::OnchipInst) * p.insts.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(first, p.first.data(), sizeof(int) * p.first.size(), cudaMemcpyHostToDevice, st);
        rc = lbh::launch_onchip(b, esz, K, dc, true, p, insts, first, buf0, buf1, coef, tblk, st);  // warm-up
        const int reps = std::max(2, 512 / tblk);
        if (rc == LBHPDE_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = LBHPDE_ERR_CUDA;
        for (int r = 0; r < reps && rc == LBHPDE_OK; ++r)
            rc = lbh::launch_onchip(b, esz, K, dc, true, p, insts, first, (r & 1) ? buf1 : buf0, (r & 1) ? buf0 : buf1,
                                    coef, tblk, st);
        float ms = 0.f;
        if (rc == LBHPDE_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = LBHPDE_ERR_CUDA;
        if (rc == LBHPDE_OK) *rate = (double)n * tblk * reps / (ms * 1e-3);
    }
    (void)cudaGetLastError();
    if (insts) cudaFree(insts);
    if (first) cudaFree(first);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int lbhpde_autotune(int precision, int lattice, int degree, int *nodes_per_thread, int *steps_per_launch,
                               double *node_updates_per_s) {
    if ((precision != LBHPDE_FP64 && precision != LBHPDE_FP32_DEV) || (lattice != 5 && lattice != 7) || degree < 1 ||
        degree > LBHPDE_MAX_DEG)
        return LBHPDE_ERR_ARG;
    const size_t esz = precision == LBHPDE_FP64 ? 8 : 4;
    const int b = lattice, dc = lbh::onchip_dc(b, degree);
    const long long n = esz == 4 ? (1LL << 22) : (1LL << 21);
    void *buf0 = nullptr, *buf1 = nullptr, *coef = nullptr;
    cudaStream_t st = nullptr;
    int rc = LBHPDE_OK;
    if (cudaMalloc(&buf0, esz * b * n) != cudaSuccess || cudaMalloc(&buf1, esz * b * n) != cudaSuccess ||
        cudaMalloc(&coef, esz * lbk::cblock(b, lbk::kMaxDeg) * 2) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        rc = LBHPDE_ERR_OOM;
    if (rc == LBHPDE_OK) {
        cudaMemsetAsync(buf0, 0, esz * b * n, st);
        cudaMemsetAsync(buf1, 0, esz * b * n, st);
        cudaMemsetAsync(coef, 0, esz * lbk::cblock(b, lbk::kMaxDeg) * 2, st);
    }
    int bestK = 0, bestT = 0;
    double best = 0.0;
    for (int K : {2, 4, 8}) {
        if (rc != LBHPDE_OK) break;
        const int maxt = lbh::onchip_maxt_halo(esz, b, K);
        if (maxt == 0 || K < lbk::wmax(b)) continue;
        for (int tblk : {16, 32, 64, 96, 128}) {
            if (maxt * K - 2 * tblk * lbk::wmax(b) < maxt * K / 2) continue;
            double r = 0.0;
            rc = time_candidate(esz, b, dc, K, tblk, n, buf0, buf1, coef, st, &r);
            if (rc != LBHPDE_OK) break;
            if (r > best) {
                best = r;
                bestK = K;
                bestT = tblk;
            }
        }
    }
    (void)cudaGetLastError();
    if (st) cudaStreamSynchronize(st);
    if (buf0) cudaFree(buf0);
    if (buf1) cudaFree(buf1);
    if (coef) cudaFree(coef);
    if (st) cudaStreamDestroy(st);
    if (rc != LBHPDE_OK) return rc;
    if (bestK == 0) return LBHPDE_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[std::make_tuple((int)esz, b, dc)] = std::make_pair(bestK, bestT);
    }
    if (nodes_per_thread) *nodes_per_thread = bestK;
    if (steps_per_launch) *steps_per_launch = bestT;
    if (node_updates_per_s) *node_updates_per_s = best;
    return LBHPDE_OK;
}

extern "C" int lbhpde_set_tuning(int precision, int lattice, int degree, int nodes_per_thread, int steps_per_launch) {
    if ((precision != LBHPDE_FP64 && precision != LBHPDE_FP32_DEV) || (lattice != 5 && lattice != 7) || degree < 1 ||
        degree > LBHPDE_MAX_DEG || steps_per_launch < 1)
        return LBHPDE_ERR_ARG;
    const size_t esz = precision == LBHPDE_FP64 ? 8 : 4;
    const int b = lattice, K = nodes_per_thread;
    const int maxt = lbh::onchip_maxt_halo(esz, b, K);
    if (maxt == 0 || K < lbk::wmax(b)) return LBHPDE_ERR_UNSUPPORTED;
    // the same bound as the autotuner's candidates: the halo leaves at least half the window valid
    if ((long long)maxt * K - 2LL * steps_per_launch * lbk::wmax(b) < (long long)maxt * K / 2)
        return LBHPDE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple((int)esz, b, lbh::onchip_dc(b, degree))] = std::make_pair(K, steps_per_launch);
    return LBHPDE_OK;
}

// ============================================================================= batches

namespace {

template <typename T, int B, int DC, bool PARAMC>
int launch_stream_t(lbhpde_batch_s *bt, Group &g, const int2 *blocks, int nb, const void *in_, void *out_) {
    if (nb == 0) return LBHPDE_OK;
    const T *in = (const T *)in_;
    T *out = (T *)out_;
    lbk::StreamCoef<T, B, (DC > 0 ? DC : 1)> pc{};
    if constexpr (PARAMC) {
        // one model for the whole launch: its coefficients (zero-padded to degree DC)
        const lbhpde_model_info &M = bt->mi[g.members[0]];
        for (int j = 1; j < B; ++j)
            for (int p = 0; p <= DC; ++p) pc.c[(j - 1) * (DC + 1) + p] = p <= M.D ? (T)M.coef[j][p] : T(0);
        pc.omw = (T)(1.0 - M.omega);
    }
    if constexpr (DC == 0)
        lbk::k_stream_rt<T, B, kStreamThreads><<<nb, kStreamThreads, 0, bt->stream>>>(in, out, bt->segs, blocks,
                                                                                    (const T *)bt->coefT);
    else
        lbk::k_stream<T, B, DC, kStreamThreads, PARAMC><<<nb, kStreamThreads, 0, bt->stream>>>(
            in, out, bt->segs, blocks, (const T *)bt->coefT, pc);
    CK(cudaGetLastError());
    ++bt->launches;
    return LBHPDE_OK;
}

template <typename T, int B>
int launch_stream_b(lbhpde_batch_s *bt, Group &g, const int2 *blocks, int nb, const void *in, void *out) {
    constexpr int DC = B == 5 ? 5 : 7;
    if (g.maxD <= DC && g.uniform && !g.has_nu) return launch_stream_t<T, B, DC, true>(bt, g, blocks, nb, in, out);
    if (g.maxD <= DC && !g.has_nu) return launch_stream_t<T, B, DC, false>(bt, g, blocks, nb, in, out);
    return launch_stream_t<T, B, 0, false>(bt, g, blocks, nb, in, out);
}

// One streaming step of the node blocks `blocks` of group g from buffer `in` to `out`.
int launch_stream(lbhpde_batch_s *bt, Group &g, const int2 *blocks, int nb, const void *in, void *out) {
    if (bt->esz == 4)
        return g.b == 5 ? launch_stream_b<float, 5>(bt, g, blocks, nb, in, out)
                        : launch_stream_b<float, 7>(bt, g, blocks, nb, in, out);
    return g.b == 5 ? launch_stream_b<double, 5>(bt, g, blocks, nb, in, out)
                    : launch_stream_b<double, 7>(bt, g, blocks, nb, in, out);
}

int upload_plan(lbhpde_batch_s *bt, Group::Plan &pl) {
    if (pl.host.ncta() == 0) return LBHPDE_OK;
    RC(bt->upload(&pl.insts, pl.host.insts));
    RC(bt->upload(&pl.cta_first, pl.host.first));
    return LBHPDE_OK;
}

// Members that fit one CTA become resident instances; longer members (or all, with
// force_halo) are cut into temporally blocked windows of tblk steps.
// Kr: nodes per thread of the resident instances (K, or lbh::kRingK for the 16-node kernel, whose
// instances hold up to 8192 nodes; the windows then keep K).
// Nodes a thread of the tail of a plan in whole waves (members that fit it; the others keep 16)
constexpr int kTailK = 8;

int plan_onchip(lbhpde_batch_s *bt, Group &g, int K, int Kr, int tblk, bool force_halo) {
    g.onchip_ok = false;
    const int maxt = lbh::onchip_maxt(bt->esz, g.b, Kr);
    if (maxt == 0 || K < lbk::wmax(g.b) || lbh::onchip_maxt(bt->esz, g.b, K) == 0) return LBHPDE_ERR_UNSUPPORTED;
    const int W = lbk::wmax(g.b);
    const int cap = maxt * Kr, cap_h = lbh::onchip_maxt_halo(bt->esz, g.b, K) * K;
    g.dc = g.has_nu ? -1 : lbh::onchip_dc(g.b, g.maxD);  // real exponents: their own variant
    if (Kr == lbh::kRingK && !lbh::ring_split_ok(bt->esz, g.b, g.dc)) return LBHPDE_ERR_UNSUPPORTED;
    if (tblk <= 0) tblk = lbh::default_tblk(cap_h, W);
    const int H = tblk * W;
    std::vector<lbh::Member> resident, ring[lbh::kRingClasses], halo;
    for (int i : g.members) {
        const lbh::Member mb{bt->segs_h[i], bt->segs_h[i].off, 1 << 30};
        (bt->N[i] <= cap && !force_halo ? resident : halo).push_back(mb);
    }
    // the 16-node kernel: whole waves of full CTAs and a tail of small ones when the members fill a
    // wave; otherwise (and for the other kernels) CTA size classes
    std::vector<lbh::Member> full, tail;
    int sms = 0;
    if (Kr == lbh::kRingK) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    g.waves = Kr == lbh::kRingK && lbh::split_ring_waves(g.b, Kr, sms, resident, full, tail);
    g.Kt = 0;
    if (g.waves) {
        for (auto &v : ring) v.clear();
        ring[lbh::kRingClasses - 1] = full;
        ring[0] = tail;
    } else {
        lbh::split_ring_classes(bt->esz, g.b, Kr, resident, ring);
    }
    // windows must keep some valid nodes; resident members only chunk their launches by tblk
    if (!halo.empty() && cap_h - 2 * H < 32) return LBHPDE_ERR_UNSUPPORTED;
    // the previous plan's device tables (a re-plan after lbhpde_batch_set_kernel)
    for (auto &pl : g.ring) {
        bt->dev_free(pl.insts);
        bt->dev_free(pl.cta_first);
        pl = Group::Plan{};
    }
    bt->dev_free(g.halo.insts);
    bt->dev_free(g.halo.cta_first);
    g.halo = Group::Plan{};
    for (int c = 0; c < lbh::kRingClasses; ++c) {
        if (ring[c].empty()) continue;
        int threads = lbh::ring_class_threads(bt->esz, g.b, Kr, c);
        int Kc = Kr;
        if (g.waves && c == 0) {
            // the tail runs after the waves with an SM to itself per CTA: fewer nodes a thread
            // (more warps) when its members fit, in the smallest class that holds the largest
            long long nmax = 0;
            for (const auto &mb : ring[c]) nmax = std::max<long long>(nmax, mb.seg.N);
            if (nmax <= (long long)lbh::onchip_maxt(bt->esz, g.b, kTailK) * kTailK) Kc = kTailK;
            int cl = 0;
            while (cl < lbh::kRingClasses - 1 && nmax > (long long)lbh::ring_class_threads(bt->esz, g.b, Kc, cl) * Kc) ++cl;
            threads = lbh::ring_class_threads(bt->esz, g.b, Kc, cl);
            g.Kt = Kc;
        }
        RC(lbh::pack_ring(g.b, bt->esz, Kc, g.dc, ring[c], g.ring[c].host, threads));
        RC(upload_plan(bt, g.ring[c]));
    }
    if (!halo.empty()) RC(lbh::pack_halo(g.b, bt->esz, K, g.dc, H, halo, g.halo.host));
    RC(upload_plan(bt, g.halo));
    g.K = K;
    g.Kr = Kr;
    g.maxt = maxt;
    g.tblk = tblk;
    g.onchip_ok = true;
    return LBHPDE_OK;
}

int launch_group(lbhpde_batch_s *bt, Group &g, bool halo, const void *in, void *out, int nsteps, cudaStream_t st,
                 int cls = lbh::kRingClasses - 1) {
    Group::Plan &pl = halo ? g.halo : g.ring[cls];
    if (pl.ncta() > 0 && nsteps > 0) ++bt->launches;
    const int Kx = halo ? g.K : (g.waves && cls == 0 && g.Kt ? g.Kt : g.Kr);
    return lbh::launch_onchip(g.b, bt->esz, Kx, g.dc, halo, pl.host, pl.insts, pl.cta_first, in, out, bt->coefT,
                              nsteps, st);
}

int batch_build(lbhpde_batch_s *bt, int count, const lbhpde_instance *m) {
    bt->count = count;
    bt->depth.assign(count, 0);
    bt->mi.resize(count);
    bt->N.resize(count);
    bt->phi_off.resize(count + 1);
    long long off = 0;
    for (int i = 0; i < count; ++i) {
        const lbhpde_instance &I = m[i];
        RC(lbhpde_model(I.m, I.alpha, I.pi, I.dx, I.dt, I.tau, I.lattice, I.scheme, &bt->mi[i]));
        const int W = (bt->mi[i].b - 1) / 2;
        if (I.N < 2 * W || I.N > (1LL << 30)) return LBHPDE_ERR_ARG;
        // boundary: LBHPDE_PERIODIC, or LBHPDE_NEE with the depth in the bits above the kind
        if (I.boundary < 0) return LBHPDE_ERR_ARG;
        const int kind = I.boundary & 0xff, dcode = I.boundary >> 8;
        if (kind != LBHPDE_PERIODIC && kind != LBHPDE_NEE) return LBHPDE_ERR_UNSUPPORTED;
        int depth = 0;
        if (kind == LBHPDE_PERIODIC) {
            if (dcode != 0) return LBHPDE_ERR_ARG;
        } else {
            depth = dcode == 0 ? 2 : dcode;
            if (depth > 4096 || I.N < 2LL * (W + depth)) return LBHPDE_ERR_ARG;
            ++bt->nbounded;
        }
        bt->depth[i] = depth;
        bt->N[i] = I.N;
        bt->phi_off[i] = off;
        off += I.N;
    }
    bt->phi_off[count] = off;
    bt->total = off;

    // arena: per member b rows of ld elements; coefficient blocks
    std::vector<Seg> segs(count);
    long long st_elems = 0;
    std::vector<double> coefd;
    for (int i = 0; i < count; ++i) {
        const lbhpde_model_info &M = bt->mi[i];
        Seg s{};
        s.off = st_elems;
        s.ld = (bt->N[i] + 31) / 32 * 32;
        s.N = (int)bt->N[i];
        s.D = M.D;
        s.pad = bt->depth[i];  // extrapolation depth of a bounded member, 0 when periodic
        s.A = M.nu_rows - 1;
        s.Dg = M.nu_deg;
        s.nu = M.nu;
        s.coef = (int)coefd.size();
        st_elems += s.ld * M.b;
        // rows of the generalised tables: for an ordinary polynomial model they are the degree-D
        // coefficients; with real exponents, the flattened (A + 1)(Dg + 1) = D + 1 entries
        for (int j = 1; j < M.b; ++j)
            for (int p = 0; p <= M.D; ++p) coefd.push_back(M.gcoef[j][p]);
        for (int j = 1; j < M.b; ++j)
            for (int p = 0; p <= M.D; ++p) coefd.push_back(M.gfeq[j][p]);
        coefd.push_back(1.0 - M.omega);
        segs[i] = s;
    }
    bt->segs_h = segs;
    bt->st_bytes = size_t(st_elems) * bt->esz;
    RC(bt->dev_alloc(&bt->st[0], bt->st_bytes));
    RC(bt->dev_alloc(&bt->st[1], bt->st_bytes));
    RC(bt->upload(&bt->segs, segs));
    if (bt->esz == 4) {
        std::vector<float> cf(coefd.begin(), coefd.end());
        RC(bt->upload((float **)&bt->coefT, cf));
    } else {
        RC(bt->upload(&bt->coefD, coefd));
        bt->coefT = bt->coefD;
    }

    // block maps
    std::vector<int2> all;
    std::vector<long long> blk_off;
    std::vector<int> part_first;
    for (int i = 0; i < count; ++i) {
        part_first.push_back((int)all.size());
        for (long long x = 0; x < bt->N[i]; x += kChunk) {
            all.push_back(make_int2(i, (int)x));
            blk_off.push_back(bt->phi_off[i]);
        }
    }
    part_first.push_back((int)all.size());
    bt->all_blocks_h = all;
    bt->part_first_h = part_first;
    RC(bt->upload(&bt->all_blocks, all));
    RC(bt->upload(&bt->blk_off, blk_off));
    RC(bt->upload(&bt->part_first, part_first));
    RC(bt->dev_alloc((void **)&bt->part, sizeof(DiagPart) * all.size()));
    RC(bt->dev_alloc((void **)&bt->diag_out, sizeof(DiagPart) * count));
    RC(bt->dev_alloc((void **)&bt->phi_buf, sizeof(double) * bt->total));
    RC(bt->dev_alloc((void **)&bt->nonfinite, sizeof(int)));

    for (int gi = 0; gi < 4; ++gi) {
        const bool bounded = gi >= 2;
        Group &g = bounded ? bt->bgroups[gi - 2] : bt->groups[gi];
        g.b = gi % 2 == 0 ? 5 : 7;
        for (int i = 0; i < count; ++i)
            if (bt->mi[i].b == g.b && (bt->depth[i] > 0) == bounded) {
                g.members.push_back(i);
                g.maxD = std::max(g.maxD, bt->mi[i].D);
                if (bt->mi[i].nu_rows > 1) g.has_nu = true;
                for (long long x = 0; x < bt->N[i]; x += kChunk) g.blocks_h.push_back(make_int2(i, (int)x));
            }
        g.uniform = !g.members.empty();
        for (int i : g.members) {
            const lbhpde_model_info &A = bt->mi[g.members[0]], &Bm = bt->mi[i];
            if (A.D != Bm.D || A.omega != Bm.omega ||
                std::memcmp(A.coef, Bm.coef, sizeof(A.coef)) != 0)
                g.uniform = false;
        }
        if (!g.members.empty()) {
            std::vector<long long> off(g.blocks_h.size());
            for (size_t q = 0; q < off.size(); ++q) off[q] = bt->phi_off[g.blocks_h[q].x];
            RC(bt->upload(&g.blocks, g.blocks_h));
            RC(bt->upload(&g.blk_off, off));
        }
    }
    return LBHPDE_OK;
}

// Bounded members of up to kBoundedK * kBoundedMaxT nodes stay resident in one CTA each
// (unless the streaming kernel was requested); longer ones stream and are rebuilt each step.
int plan_bounded(lbhpde_batch_s *bt, Group &g) {
    g.bnd_h.clear();
    g.smembers_h.clear();
    g.sblocks_h.clear();
    const int K = lbh::kBoundedK;
    int maxthr = 0, maxD = 0, maxDn = 0;
    bool real = false;
    // FP32 D1Q5 polynomial members take the 16-node resident kernel (unless a kernel or 4 nodes
    // a thread was asked for), the others one CTA each (real-exponent members on its variant
    // with the generalised f^eq) or the streaming step
    std::vector<lbh::NeeMember> nee;
    const bool nee_auto = bt->kernel == LBHPDE_KERNEL_AUTO || (bt->kernel == LBHPDE_KERNEL_ONCHIP && bt->K_req != K);
    for (int i : g.members) {
        const Seg &sg = bt->segs_h[i];
        if (nee_auto && lbh::ring_nee_ok(bt->esz, g.b, sg)) {
            nee.push_back(lbh::NeeMember{sg, i, 1 << 30});
            maxDn = std::max(maxDn, sg.D);
            continue;
        }
        const int shift =
            bt->N[i] <= (long long)K * lbh::kBoundedMaxT ? lbh::bounded_shift(g.b, sg.N, sg.pad) : -1;
        if (bt->kernel != LBHPDE_KERNEL_STREAM && shift >= 0) {
            lbk::BoundedInst I{};
            I.off = sg.off;
            I.ld = sg.ld;
            I.mi = i;
            I.N = sg.N;
            I.D = sg.D;
            I.gcoef = sg.coef;
            I.depth = sg.pad;
            I.shift = shift;
            I.nthr = (sg.N + shift + K - 1) / K;
            I.A = sg.A;
            I.Dg = sg.Dg;
            I.nu = sg.nu;
            real = real || sg.A > 0;
            g.bnd_h.push_back(I);
            maxthr = std::max(maxthr, I.nthr);
            maxD = std::max(maxD, sg.D);
        } else {
            g.smembers_h.push_back(i);
            for (long long x = 0; x < bt->N[i]; x += kChunk) g.sblocks_h.push_back(make_int2(i, (int)x));
        }
    }
    g.bnd_threads = (maxthr + 31) / 32 * 32;
    g.bnd_dc = real ? -1 : lbh::onchip_dc(g.b, maxD);
    g.bnd_D = g.bnd_dc > 0 ? g.bnd_dc : maxD;
    bt->dev_free(g.bnd);
    bt->dev_free(g.smembers);
    bt->dev_free(g.sblocks);
    bt->dev_free(g.rn_insts);
    bt->dev_free(g.rn_first);
    g.bnd = nullptr;
    g.smembers = nullptr;
    g.sblocks = nullptr;
    g.rn_insts = nullptr;
    g.rn_first = nullptr;
    g.rn_h = lbh::PackedNee{};
    if (!nee.empty()) {
        g.rn_dc = lbh::onchip_dc(g.b, maxDn);
        RC(lbh::pack_ring_nee(g.b, g.rn_dc, nee, g.rn_h, 512));
        RC(bt->upload(&g.rn_insts, g.rn_h.insts));
        RC(bt->upload(&g.rn_first, g.rn_h.first));
    }
    if (!g.bnd_h.empty()) RC(bt->upload(&g.bnd, g.bnd_h));
    if (!g.smembers_h.empty()) {
        RC(bt->upload(&g.smembers, g.smembers_h));
        RC(bt->upload(&g.sblocks, g.sblocks_h));
    }
    return LBHPDE_OK;
}

int choose_kernels(lbhpde_batch_s *bt) {
    // captured streaming graphs hold the launches of the groups that streamed when they were
    // captured: a new plan may change that set, so they are rebuilt on the next long run
    if (bt->graph[0] || bt->graph[1]) {
        cudaStreamSynchronize(bt->stream);
        for (auto &gx : bt->graph)
            if (gx) cudaGraphExecDestroy(gx);
        bt->graph[0] = bt->graph[1] = nullptr;
    }
    for (auto &g : bt->groups) {
        if (g.members.empty()) continue;
        g.onchip_ok = false;
        if (bt->kernel == LBHPDE_KERNEL_STREAM) continue;
        // K_req = kRingK asks for the 16-node resident kernel, whose windows keep the default (or
        // tuned) K; automatic choice: that kernel wherever it applies
        const int dcg = g.has_nu ? -1 : lbh::onchip_dc(g.b, g.maxD);
        // a group too small to give every SM a warp at 16 nodes a thread is latency-bound: it
        // takes the fewest nodes a thread (the most threads) whose CTA still holds its largest
        // member (GB300, 100 000 steps: KdV on 400 nodes 0.29 us a step at 2 nodes a thread
        // against 0.43 at 8 and 0.71 at 16; FP64 3.9 against 4.6)
        long long thr16 = 0, nmax = 0;
        for (int i : g.members) {
            thr16 += (bt->N[i] + lbh::kRingK - 1) / lbh::kRingK;
            nmax = std::max<long long>(nmax, bt->N[i]);
        }
        int sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            sms = 0;
        }
        const bool small = bt->K_req == 0 && bt->kernel != LBHPDE_KERNEL_HALO && thr16 < 32LL * sms;
        int K_small = 0;
        if (small)
            for (int Kc : {2, 4, 8})
                if (Kc >= lbk::wmax(g.b) && (!g.has_nu || Kc >= 4) && lbh::onchip_maxt(bt->esz, g.b, Kc) > 0 &&
                    nmax <= (long long)lbh::onchip_maxt(bt->esz, g.b, Kc) * Kc) {
                    K_small = Kc;
                    break;
                }
        const bool ring16 = bt->kernel != LBHPDE_KERNEL_HALO && lbh::ring_split_ok(bt->esz, g.b, dcg) &&
                            (bt->K_req == 0 || bt->K_req == lbh::kRingK) && !small;
        if (bt->K_req == lbh::kRingK && !ring16) return LBHPDE_ERR_UNSUPPORTED;
        int K = bt->K_req > 0 && bt->K_req != lbh::kRingK ? bt->K_req : (K_small ? K_small : lbh::default_K(bt->esz, g.b));
        int tblk = bt->spl_req;
        int tk = 0, tt = 0;
        if (!K_small && tuned_choice(bt->esz, g.b, dcg, &tk, &tt)) {
            if (bt->K_req == 0 || bt->K_req == lbh::kRingK) K = tk;
            if (bt->spl_req == 0) tblk = tt;
        }
        if (g.has_nu && K < 4) continue;  // the real-exponent on-chip variants hold 4 or more nodes a thread
        // FP64 real exponents: the FP64 pow binds both kernels, and streaming was faster on GB300
        // (3.88e9 node-updates/s against 3.62e9 in windows on a 2^24-node gKdV grid)
        if (g.has_nu && bt->esz == 8 && bt->kernel == LBHPDE_KERNEL_AUTO) continue;
        int rc = plan_onchip(bt, g, K, ring16 ? lbh::kRingK : K, tblk, bt->kernel == LBHPDE_KERNEL_HALO);
        if (rc != LBHPDE_OK) return rc;
    }
    for (auto &g : bt->bgroups)
        if (!g.members.empty()) RC(plan_bounded(bt, g));
    return LBHPDE_OK;
}

// nsteps steps of the periodic members (groups); bt->cur ends on the buffer that holds them.
int step_periodic(lbhpde_batch_s *bt, long nsteps) {
    bool any_stream = false, any_halo = false;
    for (auto &g : bt->groups) {
        if (g.members.empty()) continue;
        if (!g.onchip_ok) any_stream = true;
        else if (g.halo.ncta()) any_halo = true;
    }
    if (any_stream) {
        // one fused collide+stream launch per step, ping-pong buffers
        auto one_step = [&]() -> int {
            for (auto &g : bt->groups) {
                if (g.members.empty()) continue;
                RC(launch_stream(bt, g, g.blocks, (int)g.blocks_h.size(), bt->st[bt->cur], bt->st[bt->cur ^ 1]));
            }
            bt->cur ^= 1;
            return LBHPDE_OK;
        };
        long left = nsteps;
        // long runs replay a captured graph of kGraphSteps launches (even, so the buffer parity
        // after a replay is the parity before it); not on the legacy stream, and not while the
        // caller is capturing the stream itself
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        const bool graphs = bt->stream != nullptr && left >= 2 * kGraphSteps &&
                            cudaStreamIsCapturing(bt->stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
        (void)cudaGetLastError();
        if (graphs) {
            const int par = bt->cur;
            if (!bt->graph[par]) {
                cudaGraph_t gr = nullptr;
                CK(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal));
                int rc = LBHPDE_OK;
                const long long before = bt->launches;
                for (int s = 0; s < kGraphSteps && rc == LBHPDE_OK; ++s) rc = one_step();
                const cudaError_t ec = cudaStreamEndCapture(bt->stream, &gr);
                bt->cur = par;  // capture launched nothing
                bt->graph_launches[par] = bt->launches - before;
                bt->launches = before;
                RC(rc);
                if (ec != cudaSuccess) {
                    (void)cudaGetLastError();
                    return LBHPDE_ERR_CUDA;
                }
                const cudaError_t ei = cudaGraphInstantiate(&bt->graph[par], gr, 0);
                cudaGraphDestroy(gr);
                if (ei != cudaSuccess) {
                    (void)cudaGetLastError();
                    bt->graph[par] = nullptr;
                    return LBHPDE_ERR_CUDA;
                }
            }
            while (left >= kGraphSteps) {
                CK(cudaGraphLaunch(bt->graph[par], bt->stream));
                bt->launches += bt->graph_launches[par];
                left -= kGraphSteps;
            }
        }
        for (; left > 0; --left) RC(one_step());
        return LBHPDE_OK;
    }
    // halo windows advance tblk steps per launch through the ping-pong buffers; ring instances
    // read the current buffer once and write the buffer the halo launches end in
    int tb = 1 << 30;
    for (auto &g : bt->groups)
        if (!g.members.empty() && g.halo.ncta()) tb = std::min(tb, g.tblk);
    const long nchunks = any_halo ? (nsteps + tb - 1) / tb : 0;
    const int cur0 = bt->cur, cur1 = bt->cur ^ (int)(nchunks & 1);
    // resident instances (each size class) and windows touch disjoint rows: when there is more
    // than one kind, they run concurrently, the resident classes on streams of their own
    // (a group planned in whole waves launches its tail (class 0) after its full CTAs (class 2), on
    // the same stream)
    bool used[lbh::kRingClasses] = {};
    int kinds = any_halo ? 1 : 0;
    for (int c = 0; c < lbh::kRingClasses; ++c) {
        for (auto &g : bt->groups)
            if (!g.members.empty() && (g.ring[c].ncta() || (c == lbh::kRingClasses - 1 && g.waves && g.ring[0].ncta())))
                if (!(g.waves && c == 0)) used[c] = true;
        kinds += used[c] ? 1 : 0;
    }
    const bool fork = kinds > 1;
    if (fork) {
        if (!bt->ev_fork) CK(cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming));
        CK(cudaEventRecord(bt->ev_fork, bt->stream));
    }
    for (int c = 0; c < lbh::kRingClasses; ++c) {
        if (!used[c]) continue;
        cudaStream_t rs = bt->stream;
        if (fork) {
            if (!bt->side[c]) {
                CK(cudaStreamCreateWithFlags(&bt->side[c], cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&bt->ev_join[c], cudaEventDisableTiming));
            }
            CK(cudaStreamWaitEvent(bt->side[c], bt->ev_fork, 0));
            rs = bt->side[c];
        }
        for (auto &g : bt->groups) {
            if (g.members.empty() || (g.waves && c == 0)) continue;
            const bool tail = g.waves && c == lbh::kRingClasses - 1 && g.ring[0].ncta();
            if (!g.ring[c].ncta() && !tail) continue;
            const long spl = bt->spl_req > 0 ? bt->spl_req : (1L << 30);
            long left = nsteps;
            bool firstl = true;
            while (left > 0) {
                const int n = (int)std::min(left, spl);
                RC(launch_group(bt, g, false, bt->st[firstl ? cur0 : cur1], bt->st[cur1], n, rs, c));
                if (tail) RC(launch_group(bt, g, false, bt->st[firstl ? cur0 : cur1], bt->st[cur1], n, rs, 0));
                firstl = false;
                left -= n;
            }
        }
        if (fork) CK(cudaEventRecord(bt->ev_join[c], bt->side[c]));
    }
    long left = nsteps;
    for (long c = 0; c < nchunks; ++c) {
        const int n = (int)std::min<long>(left, tb);
        for (auto &g : bt->groups)
            if (!g.members.empty() && g.halo.ncta())
                RC(launch_group(bt, g, true, bt->st[bt->cur], bt->st[bt->cur ^ 1], n, bt->stream));
        bt->cur ^= 1;
        left -= n;
    }
    if (fork)
        for (int c = 0; c < lbh::kRingClasses; ++c)
            if (used[c]) CK(cudaStreamWaitEvent(bt->stream, bt->ev_join[c], 0));
    bt->cur = cur1;
    return LBHPDE_OK;
}

// Device pointer to the boundary values of this call (copied from the host when needed),
// after checking the layout: member i's [nsteps][2W_i] block at phib + i * stride.
int stage_boundary(lbhpde_batch_s *bt, long nsteps, const double *phib, long long stride, int on_device,
                   const double **out) {
    if (stride < 0) return LBHPDE_ERR_ARG;
    long long need = 0, w2_shared = -1;
    for (int i = 0; i < bt->count; ++i) {
        if (bt->depth[i] == 0) continue;
        const long long w2 = 2LL * lbk::wmax(bt->mi[i].b);
        if (stride == 0) {
            if (w2_shared >= 0 && w2_shared != w2) return LBHPDE_ERR_ARG;
            w2_shared = w2;
        } else if (stride < nsteps * w2) {
            return LBHPDE_ERR_ARG;
        }
        need = std::max(need, (long long)i * stride + nsteps * w2);
    }
    if (on_device) {
        *out = phib;
        return LBHPDE_OK;
    }
    if ((size_t)need > bt->phib_cap) {
        if (bt->phib_buf) bt->dev_free(bt->phib_buf);
        bt->phib_buf = nullptr;
        bt->phib_cap = 0;
        RC(bt->dev_alloc((void **)&bt->phib_buf, sizeof(double) * (size_t)need));
        bt->phib_cap = (size_t)need;
    }
    CK(cudaMemcpyAsync(bt->phib_buf, phib, sizeof(double) * (size_t)need, cudaMemcpyHostToDevice, bt->stream));
    *out = bt->phib_buf;
    return LBHPDE_OK;
}

// nsteps steps of the bounded members.  Resident members read buffer cur0 once and write the
// buffer the periodic members end in (fixed), else the one the streaming members end in;
// streaming members ping-pong from cur0 and are copied over if they end in the other buffer.
int step_bounded(lbhpde_batch_s *bt, long nsteps, const double *pbd, long long stride, int cur0, bool fixed) {
    bool any_stream = false, any_res = false;
    for (auto &g : bt->bgroups) {
        if (!g.smembers_h.empty()) any_stream = true;
        if (!g.bnd_h.empty() || g.rn_h.ncta()) any_res = true;
    }
    int a = cur0;
    if (any_stream) {
        for (long s = 0; s < nsteps; ++s) {
            for (auto &g : bt->bgroups) {
                if (g.smembers_h.empty()) continue;
                RC(launch_stream(bt, g, g.sblocks, (int)g.sblocks_h.size(), bt->st[a], bt->st[a ^ 1]));
                RC(lbh::launch_nee_fix(g.b, bt->esz, bt->st[a ^ 1], bt->segs, g.smembers, (int)g.smembers_h.size(),
                                       bt->coefT, pbd, stride, s, bt->stream));
                ++bt->launches;
            }
            a ^= 1;
        }
    }
    const int target = fixed ? bt->cur : (any_stream ? a : cur0);
    if (any_res) {
        for (auto &g : bt->bgroups) {
            for (long done = 0; g.rn_h.ncta() && done < nsteps;) {
                const int n = (int)std::min<long>(nsteps - done, 1L << 30);
                RC(lbh::launch_ring_nee_f32(g.rn_dc, g.rn_h, g.rn_insts, g.rn_first, bt->st[done == 0 ? cur0 : target],
                                            bt->st[target], bt->coefT, pbd, stride, done, n, bt->stream));
                ++bt->launches;
                done += n;
            }
            if (g.bnd_h.empty()) continue;
            for (long done = 0; done < nsteps;) {
                const int n = (int)std::min<long>(nsteps - done, lbh::bounded_launch_steps(g.b, bt->esz));
                const size_t smem = lbh::bounded_smem(g.b, bt->esz, g.bnd_threads, g.bnd_D, n);
                RC(lbh::launch_bounded(g.b, bt->esz, g.bnd_dc, (int)g.bnd_h.size(), g.bnd_threads, smem, g.bnd,
                                       bt->st[done == 0 ? cur0 : target], bt->st[target], bt->coefT, pbd, stride,
                                       done, n, bt->stream));
                ++bt->launches;
                done += n;
            }
        }
    }
    if (any_stream && a != target) {
        for (auto &g : bt->bgroups)
            for (int i : g.smembers_h) {
                const Seg &sg = bt->segs_h[i];
                const size_t off = size_t(sg.off) * bt->esz, bytes = size_t(sg.ld) * g.b * bt->esz;
                CK(cudaMemcpyAsync((char *)bt->st[target] + off, (const char *)bt->st[a] + off, bytes,
                                   cudaMemcpyDeviceToDevice, bt->stream));
            }
    }
    bt->cur = target;
    return LBHPDE_OK;
}

int batch_step(lbhpde_batch_s *bt, long nsteps, const double *phib = nullptr, long long stride = 0,
               int on_device = 0) {
    lbh::TraceRange trace("lbhpde.step");
    if (nsteps < 0) return LBHPDE_ERR_ARG;
    if (!bt->initialised) return LBHPDE_ERR_ARG;
    if (bt->nbounded && !phib) return LBHPDE_ERR_ARG;
    if (nsteps == 0) return LBHPDE_OK;
    const double *pbd = nullptr;
    if (bt->nbounded) RC(stage_boundary(bt, nsteps, phib, stride, on_device, &pbd));
    const int cur0 = bt->cur;
    bool any_periodic = false;
    for (auto &g : bt->groups)
        if (!g.members.empty()) any_periodic = true;
    if (any_periodic) RC(step_periodic(bt, nsteps));
    if (bt->nbounded) RC(step_bounded(bt, nsteps, pbd, stride, cur0, any_periodic));
    bt->steps += nsteps;
    return LBHPDE_OK;
}

int batch_set_phi(lbhpde_batch_s *bt, const double *phi0, int on_device) {
    lbh::TraceRange trace("lbhpde.set_phi");
    if (!phi0) return LBHPDE_ERR_ARG;
    const double *src = phi0;
    if (!on_device) {
        CK(cudaMemcpyAsync(bt->phi_buf, phi0, sizeof(double) * bt->total, cudaMemcpyHostToDevice, bt->stream));
        src = bt->phi_buf;
    }
    bt->cur = 0;
    for (int gi = 0; gi < 4; ++gi) {
        Group &g = gi < 2 ? bt->groups[gi] : bt->bgroups[gi - 2];
        if (g.members.empty()) continue;
        RC(lbh::launch_init(g.b, bt->esz, bt->st[0], bt->segs, g.blocks, (int)g.blocks_h.size(), bt->coefT, src,
                            g.blk_off, bt->stream));
        if (!g.blocks_h.empty()) ++bt->launches;
    }
    bt->steps = 0;
    bt->initialised = true;
    return LBHPDE_OK;
}

int batch_read_phi(lbhpde_batch_s *bt, double *out, int on_device) {
    lbh::TraceRange trace("lbhpde.read_phi");
    if (!out) return LBHPDE_ERR_ARG;
    if (!bt->initialised) return LBHPDE_ERR_ARG;
    double *dst = on_device ? out : bt->phi_buf;
    const int nb = (int)bt->all_blocks_h.size();
    int *flag = bt->nonfinite;
    CK(cudaMemsetAsync(flag, 0, sizeof(int), bt->stream));
    if (bt->esz == 4)
        lbk::k_read_phi<float><<<nb, kGenericThreads, 0, bt->stream>>>((const float *)bt->st[bt->cur], bt->segs,
                                                                       bt->all_blocks, dst, bt->blk_off, kChunk, flag);
    else
        lbk::k_read_phi<double><<<nb, kGenericThreads, 0, bt->stream>>>((const double *)bt->st[bt->cur], bt->segs,
                                                                        bt->all_blocks, dst, bt->blk_off, kChunk, flag);
    CK(cudaGetLastError());
    ++bt->launches;
    // device or host output alike: the non-finite flag is read back, so the call synchronises
    int bad = 0;
    if (!on_device)
        CK(cudaMemcpyAsync(out, bt->phi_buf, sizeof(double) * bt->total, cudaMemcpyDeviceToHost, bt->stream));
    CK(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
    CK(cudaStreamSynchronize(bt->stream));
    if (bad) return LBHPDE_ERR_DIVERGED;
    return LBHPDE_OK;
}

int batch_diag(lbhpde_batch_s *bt, const double *phistar, lbhpde_diag *out) {
    lbh::TraceRange trace("lbhpde.diagnostics");
    if (!out) return LBHPDE_ERR_ARG;
    if (!bt->initialised) return LBHPDE_ERR_ARG;
    const int nb = (int)bt->all_blocks_h.size();
    if (bt->esz == 4)
        lbk::k_diag_partial<float><<<nb, kGenericThreads, 0, bt->stream>>>(
            (const float *)bt->st[bt->cur], bt->segs, bt->all_blocks, phistar, bt->blk_off, kChunk, bt->part);
    else
        lbk::k_diag_partial<double><<<nb, kGenericThreads, 0, bt->stream>>>(
            (const double *)bt->st[bt->cur], bt->segs, bt->all_blocks, phistar, bt->blk_off, kChunk, bt->part);
    CK(cudaGetLastError());
    lbk::k_diag_final<<<(bt->count + 127) / 128, 128, 0, bt->stream>>>(bt->part, bt->part_first, bt->count,
                                                                      bt->diag_out);
    CK(cudaGetLastError());
    bt->launches += 2;
    std::vector<DiagPart> h(bt->count);
    CK(cudaMemcpyAsync(h.data(), bt->diag_out, sizeof(DiagPart) * bt->count, cudaMemcpyDeviceToHost, bt->stream));
    CK(cudaStreamSynchronize(bt->stream));
    int rc = LBHPDE_OK;
    for (int i = 0; i < bt->count; ++i) {
        lbhpde_diag &d = out[i];
        d.sum_phi = h[i].sum;
        d.max_abs_phi = h[i].maxabs;
        d.nonfinite = (long)h[i].nonfinite;
        d.err_E = phistar ? h[i].l1d / h[i].l1s : 0.0;
        d.err_L2 = phistar ? std::sqrt(h[i].l2d / h[i].l2s) : 0.0;
        d.steps = bt->steps;
        if (h[i].nonfinite) rc = LBHPDE_ERR_DIVERGED;
    }
    return rc;
}

int batch_create(lbhpde_batch_s **out, int count, const lbhpde_instance *members, int precision, void *stream,
                 const lbhpde_allocator *alloc) {
    if (!out || count <= 0 || !members) return LBHPDE_ERR_ARG;
    if (precision != LBHPDE_FP64 && precision != LBHPDE_FP32_DEV) return LBHPDE_ERR_ARG;
    if (alloc && (!alloc->alloc || !alloc->release)) return LBHPDE_ERR_ARG;
    *out = nullptr;
    auto *bt = new (std::nothrow) lbhpde_batch_s();
    if (!bt) return LBHPDE_ERR_OOM;
    bt->precision = precision;
    bt->esz = precision == LBHPDE_FP64 ? 8 : 4;
    if (alloc) {
        bt->has_alloc = true;
        bt->alloc = *alloc;
    }
    bt->stream = (cudaStream_t)stream;  // NULL: the legacy default stream
    int rc = batch_build(bt, count, members);
    if (rc == LBHPDE_OK) rc = choose_kernels(bt);
    if (rc == LBHPDE_OK && cudaStreamSynchronize(bt->stream) != cudaSuccess) rc = LBHPDE_ERR_CUDA;
    if (rc != LBHPDE_OK) {
        bt->free_all();
        delete bt;
        return rc;
    }
    *out = bt;
    return LBHPDE_OK;
}

void fill_instance(lbhpde_instance &I, int m, const double *alpha, const lbhpde_pi *pi, long N, double dx, double dt,
                   double tau, int lattice, int scheme, int boundary) {
    std::memset(&I, 0, sizeof(I));
    I.m = m;
    for (int k = 0; k < m && k < 6; ++k) {
        I.alpha[k] = alpha[k];
        I.pi[k] = pi[k];
    }
    I.N = N;
    I.dx = dx;
    I.dt = dt;
    I.tau = tau;
    I.lattice = lattice;
    I.scheme = scheme;
    I.boundary = boundary;
}

}  // namespace

// ============================================================================ C ABI

extern "C" int lbhpde_batch_create(lbhpde_batch_t *out, int count, const lbhpde_instance *members, int precision,
                                   void *cuda_stream, const lbhpde_allocator *alloc) {
    return batch_create(out, count, members, precision, cuda_stream, alloc);
}
extern "C" int lbhpde_batch_set_phi(lbhpde_batch_t b, const double *phi0, int on_device) {
    return b ? batch_set_phi(b, phi0, on_device) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_batch_step(lbhpde_batch_t b, long nsteps) { return b ? batch_step(b, nsteps) : LBHPDE_ERR_ARG; }
extern "C" int lbhpde_batch_step_nee(lbhpde_batch_t b, long nsteps, const double *phib, long member_stride,
                                     int phib_on_device) {
    return b ? batch_step(b, nsteps, phib, member_stride, phib_on_device) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_batch_read_phi(lbhpde_batch_t b, double *out, int on_device) {
    return b ? batch_read_phi(b, out, on_device) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_batch_diagnostics(lbhpde_batch_t b, const double *phistar, lbhpde_diag *out) {
    return b ? batch_diag(b, phistar, out) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_batch_kernel_launches(lbhpde_batch_t b, long long *count) {
    if (!b || !count) return LBHPDE_ERR_ARG;
    *count = b->launches;
    return LBHPDE_OK;
}
extern "C" int lbhpde_batch_set_kernel(lbhpde_batch_t b, int kernel, int nodes_per_thread, int steps_per_launch) {
    if (!b || kernel < LBHPDE_KERNEL_AUTO || kernel > LBHPDE_KERNEL_HALO || nodes_per_thread < 0 ||
        steps_per_launch < 0)
        return LBHPDE_ERR_ARG;
    const int old_k = b->kernel, old_K = b->K_req, old_s = b->spl_req;
    b->kernel = kernel;
    b->K_req = nodes_per_thread;
    b->spl_req = steps_per_launch;
    int rc = choose_kernels(b);
    if (rc != LBHPDE_OK) {
        b->kernel = old_k;
        b->K_req = old_K;
        b->spl_req = old_s;
        choose_kernels(b);
    }
    return rc;
}
extern "C" int lbhpde_batch_size(lbhpde_batch_t b, long *total_nodes, size_t *device_bytes) {
    if (!b) return LBHPDE_ERR_ARG;
    if (total_nodes) *total_nodes = (long)b->total;
    if (device_bytes) {
        size_t s = 0;
        for (auto &a : b->allocations) s += a.second;
        *device_bytes = s;
    }
    return LBHPDE_OK;
}
// ------------------------------------------------------------------ checkpoint / resume
// A checkpoint is a header (format, layout fingerprint, state bytes, steps taken, precision,
// member count) followed by the batch's state arena as it is on the device (every member's phi
// row and stored populations, in the state's type).  Loading it into a batch of the same layout
// continues bit for bit where the saved batch stood.
namespace {
constexpr uint64_t kCkptMagic = 0x314b43504448424cull;  // "LBHDPCK1" read as little-endian bytes
struct CkptHeader {
    uint64_t magic, layout, state_bytes;
    int64_t steps;
    int32_t precision, count;
};
uint64_t layout_fingerprint(const lbhpde_batch_s *bt) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the layout of every member
    auto mix = [&](long long v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (uint64_t)((v >> (8 * i)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    mix(bt->count);
    mix((long long)bt->esz);
    for (int i = 0; i < bt->count; ++i) {
        mix(bt->N[i]);
        mix(bt->mi[i].b);
        mix(bt->segs_h[i].off);
        mix(bt->segs_h[i].ld);
        mix(bt->depth[i]);
    }
    return h;
}
}  // namespace

extern "C" int lbhpde_batch_checkpoint_size(lbhpde_batch_t b, size_t *bytes) {
    if (!b || !bytes) return LBHPDE_ERR_ARG;
    *bytes = sizeof(CkptHeader) + b->st_bytes;
    return LBHPDE_OK;
}
extern "C" int lbhpde_batch_save(lbhpde_batch_t b, void *buf, size_t bytes) {
    if (!b || !buf || !b->initialised || bytes < sizeof(CkptHeader) + b->st_bytes) return LBHPDE_ERR_ARG;
    CkptHeader h{kCkptMagic, layout_fingerprint(b), b->st_bytes, b->steps, b->precision, b->count};
    std::memcpy(buf, &h, sizeof h);
    CK(cudaMemcpyAsync((char *)buf + sizeof h, b->st[b->cur], b->st_bytes, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return LBHPDE_OK;
}
extern "C" int lbhpde_batch_load(lbhpde_batch_t b, const void *buf, size_t bytes) {
    if (!b || !buf || bytes < sizeof(CkptHeader)) return LBHPDE_ERR_ARG;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != kCkptMagic || h.layout != layout_fingerprint(b) || h.state_bytes != b->st_bytes ||
        h.precision != b->precision || h.count != b->count || h.steps < 0 || bytes < sizeof h + b->st_bytes)
        return LBHPDE_ERR_ARG;
    CK(cudaMemcpyAsync(b->st[0], (const char *)buf + sizeof h, b->st_bytes, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));  // the caller may free buf once the call returns
    b->cur = 0;
    b->steps = (long)h.steps;
    b->initialised = true;
    return LBHPDE_OK;
}
extern "C" int lbhpde_checkpoint_size(lbhpde_t h, size_t *bytes) {
    return h ? lbhpde_batch_checkpoint_size(h->b, bytes) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_save(lbhpde_t h, void *buf, size_t bytes) { return h ? lbhpde_batch_save(h->b, buf, bytes) : LBHPDE_ERR_ARG; }
extern "C" int lbhpde_load(lbhpde_t h, const void *buf, size_t bytes) {
    return h ? lbhpde_batch_load(h->b, buf, bytes) : LBHPDE_ERR_ARG;
}

extern "C" int lbhpde_batch_destroy(lbhpde_batch_t b) {
    if (!b) return LBHPDE_ERR_ARG;
    b->free_all();
    delete b;
    return LBHPDE_OK;
}

extern "C" int lbhpde_create(lbhpde_t *out, int m, const double *alpha, const lbhpde_pi *pi, long N, double dx,
                             double dt, double tau, int lattice, int scheme, int precision, int boundary,
                             void *cuda_stream, const lbhpde_allocator *alloc) {
    if (!out || !alpha || !pi || m < 1 || m > 6) return LBHPDE_ERR_ARG;
    *out = nullptr;
    lbhpde_instance I;
    fill_instance(I, m, alpha, pi, N, dx, dt, tau, lattice, scheme, boundary);
    auto *h = new (std::nothrow) lbhpde_ctx();
    if (!h) return LBHPDE_ERR_OOM;
    int rc = batch_create(&h->b, 1, &I, precision, cuda_stream, alloc);
    if (rc != LBHPDE_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return LBHPDE_OK;
}
extern "C" int lbhpde_set_phi(lbhpde_t h, const double *phi0, int on_device) {
    return h ? batch_set_phi(h->b, phi0, on_device) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_step(lbhpde_t h, long nsteps) { return h ? batch_step(h->b, nsteps) : LBHPDE_ERR_ARG; }
extern "C" int lbhpde_step_nee(lbhpde_t h, long nsteps, const double *phib, int phib_on_device) {
    if (!h) return LBHPDE_ERR_ARG;
    if (h->b->nbounded == 0) return batch_step(h->b, nsteps);
    return batch_step(h->b, nsteps, phib, 0, phib_on_device);
}
extern "C" int lbhpde_read_phi(lbhpde_t h, double *out, int on_device) {
    return h ? batch_read_phi(h->b, out, on_device) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_diagnostics(lbhpde_t h, const double *phistar, lbhpde_diag *out) {
    return h ? batch_diag(h->b, phistar, out) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_kernel_launches(lbhpde_t h, long long *count) {
    return h ? lbhpde_batch_kernel_launches(h->b, count) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_set_kernel(lbhpde_t h, int kernel, int nodes_per_thread, int steps_per_launch) {
    return h ? lbhpde_batch_set_kernel(h->b, kernel, nodes_per_thread, steps_per_launch) : LBHPDE_ERR_ARG;
}
extern "C" int lbhpde_get_model(lbhpde_t h, lbhpde_model_info *out) {
    if (!h || !out) return LBHPDE_ERR_ARG;
    *out = h->b->mi[0];
    return LBHPDE_OK;
}
extern "C" int lbhpde_destroy(lbhpde_t h) {
    if (!h) return LBHPDE_ERR_ARG;
    lbhpde_batch_destroy(h->b);
    delete h;
    return LBHPDE_OK;
}
