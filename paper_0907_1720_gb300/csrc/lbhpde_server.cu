// Request server: continuous batching of independent solves on one GPU.
//
// Requests (an equation, a grid, an initial profile and a step count) are submitted from any
// host thread.  A scheduler thread admits them as device memory and slots allow, keeps their
// distributions resident in one device arena, and advances every admitted request in step
// blocks on the on-chip kernel -- whole instances resident in registers when they fit one CTA,
// temporally blocked windows otherwise.  Requests that arrive while others run are admitted at
// the next block boundary; each finished request is read back and released, freeing memory
// for the queue.  Work per request is identical to a single-instance solve, so each result is
// the same alone and in the mix.
//
// Bounded requests (the non-equilibrium extrapolation boundary of Sec. IV, submitted with their
// boundary values for every step) stay resident one CTA each on the bounded kernel; a step
// block gathers the boundary rows its requests need into one table per lattice and class.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lbhpde.h"
#include "lbhpde_internal.h"

using lbk::Seg;

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kGrain = 256;        // arena allocation granularity (bytes)
constexpr int kCoefStride = 772;      // coefficient slot: 2 (b-1)(D+1) + 1 <= 769 values (D+1 <= 64), padded
constexpr int kLookahead = 64;        // queued requests examined per admission pass
constexpr int kClasses = 6;           // (D1Q5, D1Q7) x (compiled degree, run-time degree, real exponents)

size_t round_up(size_t n, size_t g) { return (n + g - 1) / g * g; }

// First-fit free list over [0, size) with neighbour coalescing.
class Arena {
  public:
    void reset(size_t n) {
        free_.clear();
        if (n) free_[0] = n;
        size_ = n;
        used_ = 0;
    }
    bool alloc(size_t n, size_t *off) {
        n = round_up(n, kGrain);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, o = it->first + n;
            free_.erase(it);
            if (rest) free_[o] = rest;
            used_ += n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round_up(n, kGrain);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

struct Req {
    uint64_t id = 0;
    lbhpde_model_info mi{};
    long long N = 0;
    long nsteps = 0, done = 0;        // steps to take; steps planned into step blocks so far
    long done_gpu = 0;                // steps of blocks that have completed on the GPU
    long long final_block = -1;       // the block that holds its last steps (-1: none)
    std::vector<double> phi0, phi;
    int status = LBHPDE_PENDING;
    long nonfinite = 0;
    double t_submit = 0, t_admit = -1, t_finish = -1, sum_phi = 0;
    size_t bytes = 0, dev_off = 0;   // placement in the arena
    long long ld = 0, off[2] = {0, 0};  // element offsets of the two state buffers
    int cur = 0;                     // buffer holding the state
    int slot = -1;                   // coefficient slot
    int depth = 0;                   // bounded: extrapolation depth (0: periodic)
    std::vector<double> phib;        // bounded: [nsteps][2W] boundary values
    Seg seg() const {
        Seg s{};
        s.off = off[cur];
        s.ld = ld;
        s.N = (int)N;
        s.D = mi.D;
        s.A = mi.nu_rows - 1;  // real-exponent rows (0: an ordinary polynomial)
        s.Dg = mi.nu_deg;
        s.nu = mi.nu;
        s.coef = slot * kCoefStride;
        s.pad = depth;
        return s;
    }
};

template <typename X>
struct DevBuf {  // growable device array (capacity only grows)
    X *p = nullptr;
    size_t cap = 0;
    int ensure(size_t n) {
        if (n <= cap) return LBHPDE_OK;
        const size_t c = std::max<size_t>(n, 2 * cap + 64);
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        if (cudaMalloc(&p, sizeof(X) * c) != cudaSuccess) {
            (void)cudaGetLastError();
            return LBHPDE_ERR_OOM;
        }
        cap = c;
        return LBHPDE_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

}  // namespace

struct lbhpde_server_s {
    int precision = LBHPDE_FP32_DEV;
    size_t esz = 4;
    int device = 0, max_active = 0, block = 256;
    cudaStream_t stream = nullptr;
    // set-up of admitted requests (uploads, initialisation) runs on `up`, beside a block in
    // flight on `stream`; `stream` waits for it through ev_setup
    cudaStream_t up = nullptr;
    cudaEvent_t ev_setup = nullptr;
    // A step block's independent launch chains (per lattice and degree class: one resident launch
    // per CTA size class, and the window launches, which follow each other) run on lanes of
    // their own, after the table uploads on `stream`, and join it before the block's one
    // synchronisation.
    // (and one lane per lattice and class for the bounded requests)
    static constexpr int kLanes = 4 * 6 + 6;  // 4 per (lattice, class), then the bounded lanes
    cudaStream_t lane[kLanes] = {};
    cudaEvent_t ev_up = nullptr, ev_done[kLanes] = {};
    cudaEvent_t ev_t0[2] = {}, ev_t1[2] = {};  // timing of the step blocks (by block parity)
    long long next_block = 0;                  // id of the next block to plan
    double gpu_busy = 0.0;
    // host time of the scheduler thread by phase (written by that thread, under mu)
    double t_admit = 0.0, t_setup = 0.0, t_plan = 0.0, t_launch = 0.0, t_wait = 0.0, t_retire = 0.0;
    void *arena_d = nullptr;
    Arena arena;
    void *coefT_d = nullptr;
    double *coefD_d = nullptr;
    std::vector<int> free_slots;
    DevBuf<lbk::OnchipInst> insts_d;
    DevBuf<lbk::BoundedInst> binsts_d;
    DevBuf<double> phibt_d;
    DevBuf<int> first_d;
    DevBuf<Seg> segs_d;
    DevBuf<int2> blocks_d;
    DevBuf<long long> boff_d;
    DevBuf<double> phi0_d;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::vector<Req *> active;  // touched by the worker only
    std::atomic<uint64_t> next_id{1};
    std::thread worker;
    bool stop = false;
    int error = LBHPDE_OK;  // sticky CUDA failure of the worker
    Clock::time_point t0;
    long completed = 0, launches = 0;
    double node_updates = 0;
    size_t bytes_used = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

#define SCK(call)                         \
    do {                                  \
        if ((call) != cudaSuccess) {      \
            (void)cudaGetLastError();     \
            return LBHPDE_ERR_CUDA;       \
        }                                 \
    } while (0)
#define SRC(call)                       \
    do {                                \
        int r_ = (call);                \
        if (r_ != LBHPDE_OK) return r_; \
    } while (0)

size_t state_bytes(const Req &r, size_t esz) { return 2 * (size_t)r.mi.b * (size_t)r.ld * esz; }

// Upload a request's coefficients to its slot and initialise its state (step a1).
int setup_admitted(lbhpde_server_s *S, std::vector<Req *> &adm) {
    if (adm.empty()) return LBHPDE_OK;
    std::vector<double> cd((size_t)adm.size() * kCoefStride, 0.0);
    long long phi_total = 0;
    for (size_t q = 0; q < adm.size(); ++q) {
        const Req &r = *adm[q];
        double *c = cd.data() + q * kCoefStride;
        int k = 0;
        // the generalised tables: the degree-D coefficients of an ordinary polynomial model, the
        // flattened (A + 1)(Dg + 1) = D + 1 entries of a real-exponent one
        for (int j = 1; j < r.mi.b; ++j)
            for (int p = 0; p <= r.mi.D; ++p) c[k++] = r.mi.gcoef[j][p];
        for (int j = 1; j < r.mi.b; ++j)
            for (int p = 0; p <= r.mi.D; ++p) c[k++] = r.mi.gfeq[j][p];
        c[k] = 1.0 - r.mi.omega;
        phi_total += r.N;
    }
    for (size_t q = 0; q < adm.size(); ++q) {
        const Req &r = *adm[q];
        const double *c = cd.data() + q * kCoefStride;
        SCK(cudaMemcpyAsync(S->coefD_d + (size_t)r.slot * kCoefStride, c, sizeof(double) * kCoefStride,
                            cudaMemcpyHostToDevice, S->up));
        if (S->esz == 4) {
            std::vector<float> cf(c, c + kCoefStride);
            SCK(cudaMemcpyAsync((float *)S->coefT_d + (size_t)r.slot * kCoefStride, cf.data(),
                                sizeof(float) * kCoefStride, cudaMemcpyHostToDevice, S->up));
        }
    }
    SRC(S->phi0_d.ensure(phi_total));
    std::vector<Seg> segs;
    long long o = 0;
    for (Req *r : adm) {
        SCK(cudaMemcpyAsync(S->phi0_d.p + o, r->phi0.data(), sizeof(double) * r->N, cudaMemcpyHostToDevice,
                            S->up));
        segs.push_back(r->seg());
        o += r->N;
    }
    for (int b : {5, 7}) {
        std::vector<int2> blocks;
        std::vector<long long> boff;
        long long po = 0;
        for (size_t q = 0; q < adm.size(); ++q) {
            if (adm[q]->mi.b == b)
                for (long long x = 0; x < adm[q]->N; x += lbh::kChunk) {
                    blocks.push_back(make_int2((int)q, (int)x));
                    boff.push_back(po);
                }
            po += adm[q]->N;
        }
        if (blocks.empty()) continue;
        SRC(S->segs_d.ensure(segs.size()));
        SRC(S->blocks_d.ensure(blocks.size()));
        SRC(S->boff_d.ensure(boff.size()));
        SCK(cudaMemcpyAsync(S->segs_d.p, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice, S->up));
        SCK(cudaMemcpyAsync(S->blocks_d.p, blocks.data(), sizeof(int2) * blocks.size(), cudaMemcpyHostToDevice,
                            S->up));
        SCK(cudaMemcpyAsync(S->boff_d.p, boff.data(), sizeof(long long) * boff.size(), cudaMemcpyHostToDevice,
                            S->up));
        SRC(lbh::launch_init(b, S->esz, S->arena_d, S->segs_d.p, S->blocks_d.p, (int)blocks.size(), S->coefT_d,
                             S->phi0_d.p, S->boff_d.p, S->up));
        // the next lattice reuses the tables: order the copies after this launch (the set-up
        // stream holds only set-up work, so this does not wait for a block in flight)
        SCK(cudaStreamSynchronize(S->up));
    }
    // the next block (and the wait before retiring) come after the new requests' initialisation
    SCK(cudaEventRecord(S->ev_setup, S->up));
    SCK(cudaStreamWaitEvent(S->stream, S->ev_setup, 0));
    return LBHPDE_OK;
}

// One on-chip launch of a step block, planned on the host.
struct Planned {
    int b, K, dc;
    bool halo;
    int lane;    // stream lane: 4 * (lattice, class) + (windows ? 3 : resident size class)
    int nsteps;
    lbh::Packed p;
    size_t ioff = 0, foff = 0;  // offsets of its tables in the block's device arrays
};

// One bounded launch of a step block: instances of one lattice and class for steps
// [step0, step0 + nsteps) of the block, reading their boundary rows from the block's table of
// that lattice and class (rows of instance mi at table + mi * stride).
struct PlannedBnd {
    int b, dc, lane, nthreads, nsteps;
    long long step0, stride;
    size_t smem;
    std::vector<lbk::BoundedInst> insts;
    size_t ioff = 0, toff = 0;  // offsets of its instances and of its table in the block's arrays
};

// A planned step block: its launches and, per request, the steps it advances.
struct Block {
    long long id = -1;
    std::vector<Planned> plan;
    std::vector<PlannedBnd> bplan;
    std::vector<double> phibt;  // the bounded requests' boundary rows, one table per lattice and class
    std::vector<std::pair<Req *, int>> members;
};

// The bounded requests of one lattice and polynomial class in a step block: each advances by
// up to S->block steps on the bounded kernel (one CTA an instance, in place).  Their boundary
// rows for the block go into a table of their own; the launches cover the block in spans that
// end where a request's steps end or the kernel's staged-row limit falls, so that every launch
// has one step count.
int plan_bounded(lbhpde_server_s *S, Block &blk, int b, int kind, int maxD, std::vector<Req *> &bnd) {
    const int W = (b - 1) / 2, K = lbh::kBoundedK;
    const long long stride = (long long)S->block * 2 * W;
    const size_t toff = blk.phibt.size();
    blk.phibt.resize(toff + bnd.size() * (size_t)stride, 0.0);
    std::vector<int> st(bnd.size());
    for (size_t q = 0; q < bnd.size(); ++q) {
        Req *r = bnd[q];
        st[q] = (int)std::min<long>(S->block, r->nsteps - r->done);
        std::memcpy(blk.phibt.data() + toff + q * stride, r->phib.data() + (size_t)r->done * 2 * W,
                    sizeof(double) * (size_t)st[q] * 2 * W);
        blk.members.emplace_back(r, st[q]);
    }
    const int dc = kind == 2 ? -1 : (kind == 1 ? 0 : lbh::onchip_dc(b, maxD));
    const int D = dc > 0 ? dc : maxD;
    const int span = lbh::bounded_launch_steps(b, S->esz);
    for (int c0 = 0;;) {
        int c1 = c0 + span;
        PlannedBnd pl{b, dc, 4 * kClasses + 3 * (b == 7) + kind, 32, 0, c0, stride, 0, {}};
        for (size_t q = 0; q < bnd.size(); ++q)
            if (st[q] > c0) c1 = std::min(c1, st[q]);
        for (size_t q = 0; q < bnd.size(); ++q) {
            if (st[q] <= c0) continue;
            const Seg sg = bnd[q]->seg();
            lbk::BoundedInst I{};
            I.off = sg.off;
            I.ld = sg.ld;
            I.mi = (int)q;
            I.N = sg.N;
            I.D = sg.D;
            I.gcoef = sg.coef;
            I.depth = sg.pad;
            I.shift = lbh::bounded_shift(b, sg.N, sg.pad);
            I.nthr = (sg.N + I.shift + K - 1) / K;
            I.A = sg.A;
            I.Dg = sg.Dg;
            I.nu = sg.nu;
            pl.nthreads = std::max(pl.nthreads, (I.nthr + 31) / 32 * 32);
            pl.insts.push_back(I);
        }
        if (pl.insts.empty()) break;
        pl.nsteps = c1 - c0;
        pl.smem = lbh::bounded_smem(b, S->esz, pl.nthreads, D, pl.nsteps);
        pl.toff = toff;
        blk.bplan.push_back(std::move(pl));
        c0 = c1;
    }
    for (Req *r : bnd) r->done += std::min<long>(S->block, r->nsteps - r->done);
    return LBHPDE_OK;
}

// Plan the next step block on the host: every active request advances by up to S->block steps
// (resident instances once per lattice and class, windows in chunks of tblk steps).  Requests'
// planned step counts and buffers advance here; the block runs when launch_block issues it.
int plan_block(lbhpde_server_s *S, Block &blk) {
    const auto t_enter = Clock::now();
    blk = Block{};
    blk.id = S->next_block;
    std::vector<Planned> &plan = blk.plan;
    // per lattice, three classes: requests whose f^eq degree the compiled variant covers (D <= 5
    // on D1Q5, <= 7 on D1Q7), higher-degree polynomials, and real-exponent models, each with its
    // own launches, so that one high-degree or real-exponent request does not send the whole
    // lattice to a slower variant
    for (int cls = 0; cls < kClasses; ++cls) {
        const int b = cls < kClasses / 2 ? 5 : 7;
        const int kind = cls % 3;  // 0: compiled degree, 1: run-time degree, 2: real exponents
        const int dcmax = b == 5 ? 5 : 7;
        const int K = lbh::default_K(S->esz, b);
        const int maxt = lbh::onchip_maxt(S->esz, b, K);
        const int cap = maxt * K, W = (b - 1) / 2;
        const int tblk = lbh::default_tblk(cap, W, 6);  // windows as wide as a resident CTA
        // resident requests keep the windows' K: a request's latency is set by its own CTA, and
        // more threads an instance hold its steps shorter when the GPU is not full (the 16-node
        // kernel gave the same throughput at 2000 requests/s on GB300, and 0.35 s against
        // 0.20 s p99 latency at 500/s)
        const int Kr = K;
        const int capr = lbh::onchip_maxt(S->esz, b, Kr) * Kr;
        std::vector<Req *> ring, halo, bnd;
        int maxD = 0, maxDb = 0;
        for (Req *r : S->active)
            if (r->mi.b == b && r->done < r->nsteps &&
                (r->mi.nu_rows > 1 ? 2 : (r->mi.D > dcmax ? 1 : 0)) == kind) {
                if (r->depth > 0) {
                    bnd.push_back(r);
                    maxDb = std::max(maxDb, r->mi.D);
                    continue;
                }
                (r->N <= capr ? ring : halo).push_back(r);
                maxD = std::max(maxD, r->mi.D);
            }
        if (!bnd.empty()) SRC(plan_bounded(S, blk, b, kind, maxDb, bnd));
        if (ring.empty() && halo.empty()) continue;
        const int dc = kind == 2 ? -1 : lbh::onchip_dc(b, maxD);
        if (!ring.empty()) {
            std::vector<lbh::Member> m;
            int n = 0;
            for (Req *r : ring) {
                const int st = (int)std::min<long>(S->block, r->nsteps - r->done);
                m.push_back(lbh::Member{r->seg(), r->off[r->cur], st});
                n = std::max(n, st);
                r->done += st;
                blk.members.emplace_back(r, st);
            }
            // one launch per resident size class, each on a lane of its own
            std::vector<lbh::Member> mc[lbh::kRingClasses];
            lbh::split_ring_classes(S->esz, b, Kr, m, mc);
            for (int c = 0; c < lbh::kRingClasses; ++c) {
                if (mc[c].empty()) continue;
                Planned pl{b, Kr, dc, false, 4 * cls + c, n, {}};
                SRC(lbh::pack_ring(b, S->esz, Kr, dc, mc[c], pl.p, lbh::ring_class_threads(S->esz, b, Kr, c)));
                plan.push_back(std::move(pl));
            }
        }
        if (!halo.empty()) {
            std::vector<long> left(halo.size());
            for (size_t q = 0; q < halo.size(); ++q) left[q] = std::min<long>(S->block, halo[q]->nsteps - halo[q]->done);
            for (;;) {
                std::vector<lbh::Member> m;
                int n = 0;
                for (size_t q = 0; q < halo.size(); ++q) {
                    if (left[q] <= 0) continue;
                    const int st = (int)std::min<long>(tblk, left[q]);
                    Req *r = halo[q];
                    m.push_back(lbh::Member{r->seg(), r->off[r->cur ^ 1], st});
                    n = std::max(n, st);
                    blk.members.emplace_back(r, st);
                    r->cur ^= 1;  // the launch writes the other buffer
                    r->done += st;
                    left[q] -= st;
                }
                if (m.empty()) break;
                Planned pl{b, K, dc, true, 4 * cls + 3, n, {}};
                SRC(lbh::pack_halo(b, S->esz, K, dc, tblk * W, m, pl.p, true));
                plan.push_back(std::move(pl));
            }
        }
    }
    if (plan.empty() && blk.bplan.empty()) {
        blk.id = -1;
        return LBHPDE_OK;
    }
    ++S->next_block;
    for (auto &mr : blk.members)
        if (mr.first->done >= mr.first->nsteps) mr.first->final_block = blk.id;
    std::lock_guard<std::mutex> lk(S->mu);
    S->t_plan += std::chrono::duration<double>(Clock::now() - t_enter).count();
    return LBHPDE_OK;
}

// Issue a planned block: its tables in one upload each, then its launches on the stream lanes,
// joined back into `stream` (no wait).  The next block's tables are uploaded on `stream` after
// this block's join, so one set of table buffers serves every block.
int launch_block(lbhpde_server_s *S, Block &blk) {
    const auto t_enter = Clock::now();
    std::vector<Planned> &plan = blk.plan;
    const int par = (int)(blk.id & 1);
    std::vector<lbk::OnchipInst> insts;
    std::vector<int> first;
    for (Planned &pl : plan) {
        pl.ioff = insts.size();
        pl.foff = first.size();
        insts.insert(insts.end(), pl.p.insts.begin(), pl.p.insts.end());
        first.insert(first.end(), pl.p.first.begin(), pl.p.first.end());
    }
    std::vector<lbk::BoundedInst> binsts;
    for (PlannedBnd &pl : blk.bplan) {
        pl.ioff = binsts.size();
        binsts.insert(binsts.end(), pl.insts.begin(), pl.insts.end());
    }
    SRC(S->insts_d.ensure(insts.size()));
    SRC(S->first_d.ensure(first.size()));
    SRC(S->binsts_d.ensure(binsts.size()));
    SRC(S->phibt_d.ensure(blk.phibt.size()));
    SCK(cudaEventRecord(S->ev_t0[par], S->stream));
    if (!insts.empty()) {
        SCK(cudaMemcpyAsync(S->insts_d.p, insts.data(), sizeof(lbk::OnchipInst) * insts.size(),
                            cudaMemcpyHostToDevice, S->stream));
        SCK(cudaMemcpyAsync(S->first_d.p, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice,
                            S->stream));
    }
    if (!binsts.empty()) {
        SCK(cudaMemcpyAsync(S->binsts_d.p, binsts.data(), sizeof(lbk::BoundedInst) * binsts.size(),
                            cudaMemcpyHostToDevice, S->stream));
        SCK(cudaMemcpyAsync(S->phibt_d.p, blk.phibt.data(), sizeof(double) * blk.phibt.size(),
                            cudaMemcpyHostToDevice, S->stream));
    }
    // the lanes start after the uploads; different lanes touch disjoint requests
    SCK(cudaEventRecord(S->ev_up, S->stream));
    bool used[lbhpde_server_s::kLanes] = {};
    for (const Planned &pl : plan) {
        if (!used[pl.lane]) SCK(cudaStreamWaitEvent(S->lane[pl.lane], S->ev_up, 0));
        used[pl.lane] = true;
        SRC(lbh::launch_onchip(pl.b, S->esz, pl.K, pl.dc, pl.halo, pl.p, S->insts_d.p + pl.ioff,
                               S->first_d.p + pl.foff, S->arena_d, S->arena_d, S->coefT_d, pl.nsteps,
                               S->lane[pl.lane]));
        ++S->launches;
    }
    // bounded launches of one lattice and class follow each other on their lane (in place)
    for (const PlannedBnd &pl : blk.bplan) {
        if (!used[pl.lane]) SCK(cudaStreamWaitEvent(S->lane[pl.lane], S->ev_up, 0));
        used[pl.lane] = true;
        SRC(lbh::launch_bounded(pl.b, S->esz, pl.dc, (int)pl.insts.size(), pl.nthreads, pl.smem,
                                S->binsts_d.p + pl.ioff, S->arena_d, S->arena_d, S->coefT_d, S->phibt_d.p + pl.toff,
                                pl.stride, pl.step0, pl.nsteps, S->lane[pl.lane]));
        ++S->launches;
    }
    for (int i = 0; i < lbhpde_server_s::kLanes; ++i)
        if (used[i]) {
            SCK(cudaEventRecord(S->ev_done[i], S->lane[i]));
            SCK(cudaStreamWaitEvent(S->stream, S->ev_done[i], 0));
        }
    SCK(cudaEventRecord(S->ev_t1[par], S->stream));
    std::lock_guard<std::mutex> lk(S->mu);
    S->t_launch += std::chrono::duration<double>(Clock::now() - t_enter).count();
    return LBHPDE_OK;
}

// After `stream` has drained: a launched block's GPU time, and its steps as done.
int complete_block(lbhpde_server_s *S, Block &blk) {
    if (blk.id < 0) return LBHPDE_OK;
    const int par = (int)(blk.id & 1);
    float ms = 0.0f;
    SCK(cudaEventElapsedTime(&ms, S->ev_t0[par], S->ev_t1[par]));
    for (auto &mr : blk.members) mr.first->done_gpu += mr.second;
    std::lock_guard<std::mutex> lk(S->mu);
    S->gpu_busy += ms * 1e-3;
    return LBHPDE_OK;
}

// Copy a finished request's phi to the host and release its device resources.  The copy runs on
// the set-up stream, beside the block in flight (which does not touch the request).
int retire(lbhpde_server_s *S, Req *r) {
    r->phi.resize(r->N);
    if (S->esz == 4) {
        std::vector<float> tmp(r->N);
        SCK(cudaMemcpyAsync(tmp.data(), (float *)S->arena_d + r->off[r->cur], sizeof(float) * r->N,
                            cudaMemcpyDeviceToHost, S->up));
        SCK(cudaStreamSynchronize(S->up));
        for (long long i = 0; i < r->N; ++i) r->phi[i] = tmp[i];
    } else {
        SCK(cudaMemcpyAsync(r->phi.data(), (double *)S->arena_d + r->off[r->cur], sizeof(double) * r->N,
                            cudaMemcpyDeviceToHost, S->up));
        SCK(cudaStreamSynchronize(S->up));
    }
    double sum = 0.0;
    long nf = 0;
    for (double v : r->phi) {
        if (std::isfinite(v))
            sum += v;
        else
            ++nf;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    r->sum_phi = sum;
    r->nonfinite = nf;
    r->status = nf ? LBHPDE_ERR_DIVERGED : LBHPDE_OK;
    r->t_finish = S->now();
    S->arena.release(r->dev_off, r->bytes);
    S->free_slots.push_back(r->slot);
    S->bytes_used = S->arena.used();
    ++S->completed;
    r->phi0.clear();
    r->phi0.shrink_to_fit();
    return LBHPDE_OK;
}

void worker_main(lbhpde_server_s *S) {
    if (cudaSetDevice(S->device) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->error = LBHPDE_ERR_CUDA;
        S->cv_done.notify_all();
        return;
    }
    Block inflight;  // launched and not yet waited for (id -1: none)
    for (;;) {
        std::vector<Req *> adm;
        const auto ta = Clock::now();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            // admission: FIFO, looking past requests that do not fit yet
            int looked = 0;
            for (auto it = S->queue.begin(); it != S->queue.end() && looked < kLookahead;) {
                ++looked;
                if ((int)(S->active.size() + adm.size()) >= S->max_active || S->free_slots.empty()) break;
                Req *r = *it;
                size_t off;
                if (!S->arena.alloc(r->bytes, &off)) {
                    ++it;
                    continue;
                }
                r->dev_off = off;
                r->off[0] = (long long)(off / S->esz);
                r->off[1] = r->off[0] + (long long)r->mi.b * r->ld;
                r->cur = 0;
                r->slot = S->free_slots.back();
                S->free_slots.pop_back();
                r->t_admit = S->now();
                S->bytes_used = S->arena.used();
                adm.push_back(r);
                it = S->queue.erase(it);
            }
            if (S->active.empty() && adm.empty() && inflight.id < 0) {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        // admission, set-up and the plan of the next block run while the block in flight runs
        const auto ts = Clock::now();
        int rc;
        {
            lbh::TraceRange trace("lbhpde.server.setup");
            rc = setup_admitted(S, adm);
        }
        for (Req *r : adm) S->active.push_back(r);
        const auto tv = Clock::now();
        Block next;
        if (rc == LBHPDE_OK) {
            lbh::TraceRange trace("lbhpde.server.plan");
            rc = plan_block(S, next);
        }
        // the next block is queued behind the one in flight, so the GPU goes from one to the other
        // without waiting for the host; then the host waits for the block in flight only (the
        // next one touches no request that the block in flight finishes)
        Block launched;
        if (rc == LBHPDE_OK && next.id >= 0) {
            lbh::TraceRange trace("lbhpde.server.launch");
            rc = launch_block(S, next);
            if (rc == LBHPDE_OK) launched = std::move(next);
        }
        const auto tw = Clock::now();
        if (rc == LBHPDE_OK && inflight.id >= 0) {
            lbh::TraceRange trace("lbhpde.server.wait");
            rc = cudaEventSynchronize(S->ev_t1[inflight.id & 1]) == cudaSuccess ? LBHPDE_OK : LBHPDE_ERR_CUDA;
        }
        const auto tr = Clock::now();
        if (rc == LBHPDE_OK) rc = complete_block(S, inflight);
        const long long done_id = inflight.id;
        inflight = std::move(launched);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->t_admit += std::chrono::duration<double>(ts - ta).count();
            S->t_setup += std::chrono::duration<double>(tv - ts).count();
            S->t_wait += std::chrono::duration<double>(tr - tw).count();
        }
        // the requests whose last block has completed (and those that take no steps) are retired
        // while the next block runs (their copies on the set-up stream); the ones that finish in
        // a block still queued or running stay until it has run
        const auto tt = Clock::now();
        std::vector<Req *> still;
        for (Req *r : S->active) {
            if (rc == LBHPDE_OK && r->done >= r->nsteps && r->final_block <= done_id) {
                S->node_updates += (double)r->N * (double)r->nsteps;
                rc = retire(S, r);
            } else {
                still.push_back(r);
            }
        }
        S->active.swap(still);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->t_retire += std::chrono::duration<double>(Clock::now() - tt).count();
        }
        if (rc != LBHPDE_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->error = rc;
            for (Req *r : S->active) {
                r->status = rc;
                r->t_finish = S->now();
            }
            for (Req *r : S->queue) {
                r->status = rc;
                r->t_finish = S->now();
            }
            S->queue.clear();
            S->active.clear();
            S->cv_done.notify_all();
            break;
        }
        S->cv_done.notify_all();
    }
}

void fill_result(const Req *r, lbhpde_result *info) {
    if (!info) return;
    info->status = r->status;
    info->steps_done = r->done_gpu;
    info->submit_s = r->t_submit;
    info->admit_s = r->t_admit;
    info->finish_s = r->t_finish;
    info->sum_phi = r->sum_phi;
    info->nonfinite = r->nonfinite;
}

}  // namespace

// ============================================================================ C ABI

extern "C" int lbhpde_server_create(lbhpde_server_t *out, int precision, size_t device_bytes, int max_active,
                                    int steps_per_block, int device) {
    if (!out || (precision != LBHPDE_FP64 && precision != LBHPDE_FP32_DEV) || device_bytes < (1u << 20) ||
        max_active < 1 || max_active > 65536 || steps_per_block < 0 || device < 0)
        return LBHPDE_ERR_ARG;
    *out = nullptr;
    auto *S = new (std::nothrow) lbhpde_server_s();
    if (!S) return LBHPDE_ERR_OOM;
    S->precision = precision;
    S->esz = precision == LBHPDE_FP64 ? 8 : 4;
    S->device = device;
    S->max_active = max_active;
    S->block = steps_per_block > 0 ? steps_per_block : 256;
    S->t0 = Clock::now();
    int prev = 0;
    bool ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&S->ev_setup, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&S->ev_up, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&S->ev_t0[0]) == cudaSuccess && cudaEventCreate(&S->ev_t1[0]) == cudaSuccess &&
              cudaEventCreate(&S->ev_t0[1]) == cudaSuccess && cudaEventCreate(&S->ev_t1[1]) == cudaSuccess &&
              cudaMalloc(&S->arena_d, device_bytes) == cudaSuccess &&
              cudaMalloc((void **)&S->coefD_d, sizeof(double) * (size_t)max_active * kCoefStride) == cudaSuccess;
    for (int i = 0; ok && i < lbhpde_server_s::kLanes; ++i)
        ok = cudaStreamCreateWithFlags(&S->lane[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->ev_done[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok && S->esz == 4)
        ok = cudaMalloc(&S->coefT_d, sizeof(float) * (size_t)max_active * kCoefStride) == cudaSuccess;
    else if (ok)
        S->coefT_d = S->coefD_d;
    cudaSetDevice(prev);
    if (!ok) {
        const cudaError_t e = cudaGetLastError();
        if (S->arena_d) cudaFree(S->arena_d);
        if (S->coefD_d) cudaFree(S->coefD_d);
        if (S->coefT_d && S->coefT_d != S->coefD_d) cudaFree(S->coefT_d);
        if (S->stream) cudaStreamDestroy(S->stream);
        if (S->up) cudaStreamDestroy(S->up);
        if (S->ev_setup) cudaEventDestroy(S->ev_setup);
        for (int i = 0; i < lbhpde_server_s::kLanes; ++i) {
            if (S->lane[i]) cudaStreamDestroy(S->lane[i]);
            if (S->ev_done[i]) cudaEventDestroy(S->ev_done[i]);
        }
        if (S->ev_up) cudaEventDestroy(S->ev_up);
        for (int i = 0; i < 2; ++i) {
            if (S->ev_t0[i]) cudaEventDestroy(S->ev_t0[i]);
            if (S->ev_t1[i]) cudaEventDestroy(S->ev_t1[i]);
        }
        delete S;
        return e == cudaErrorMemoryAllocation ? LBHPDE_ERR_OOM : LBHPDE_ERR_CUDA;
    }
    S->arena.reset(device_bytes / kGrain * kGrain);
    for (int i = max_active - 1; i >= 0; --i) S->free_slots.push_back(i);
    S->worker = std::thread(worker_main, S);
    *out = S;
    return LBHPDE_OK;
}

static int submit_common(lbhpde_server_t S, const lbhpde_request *q, int boundary, const double *phib,
                         uint64_t *id) {
    if (!S || !q || !id || !q->phi0 || q->nsteps < 0) return LBHPDE_ERR_ARG;
    auto *r = new (std::nothrow) Req();
    if (!r) return LBHPDE_ERR_OOM;
    int rc = lbhpde_model(q->m, q->alpha, q->pi, q->dx, q->dt, q->tau, q->lattice, q->scheme, &r->mi);
    const int W = (r->mi.b - 1) / 2;
    if (rc == LBHPDE_OK && (q->N < 2 * W || q->N > (1L << 26))) rc = LBHPDE_ERR_ARG;
    // real-exponent models take the on-chip variant that evaluates four or more nodes a thread
    if (rc == LBHPDE_OK && r->mi.nu_rows > 1 && lbh::default_K(S->esz, r->mi.b) < 4) rc = LBHPDE_ERR_UNSUPPORTED;
    if (rc == LBHPDE_OK && boundary != LBHPDE_PERIODIC) {
        // LBHPDE_NEE with the depth in the bits above the kind (0: depth 2)
        const int kind = boundary & 0xff, dcode = boundary >> 8;
        r->depth = dcode == 0 ? 2 : dcode;
        if (boundary < 0 || kind != LBHPDE_NEE || r->depth > 4096 || q->N < 2L * (W + r->depth) ||
            (q->nsteps > 0 && !phib))
            rc = LBHPDE_ERR_ARG;
        // the bounded kernel: instances of up to kBoundedK * kBoundedMaxT nodes
        else if (q->N > (long)lbh::kBoundedK * lbh::kBoundedMaxT ||
                 lbh::bounded_shift(r->mi.b, (int)q->N, r->depth) < 0)
            rc = LBHPDE_ERR_UNSUPPORTED;
    }
    if (rc != LBHPDE_OK) {
        delete r;
        return rc;
    }
    if (r->depth > 0) r->phib.assign(phib, phib + (size_t)q->nsteps * 2 * W);
    r->N = q->N;
    r->ld = (q->N + 31) / 32 * 32;
    r->nsteps = q->nsteps;
    r->bytes = round_up(state_bytes(*r, S->esz), kGrain);
    if (r->bytes > S->arena.size()) {
        delete r;
        return LBHPDE_ERR_OOM;
    }
    r->phi0.assign(q->phi0, q->phi0 + q->N);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error != LBHPDE_OK) {
        delete r;
        return S->error;
    }
    r->id = S->next_id++;
    r->t_submit = S->now();
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    *id = r->id;
    S->cv_work.notify_one();
    return LBHPDE_OK;
}

extern "C" int lbhpde_submit(lbhpde_server_t S, const lbhpde_request *q, uint64_t *id) {
    return submit_common(S, q, LBHPDE_PERIODIC, nullptr, id);
}

extern "C" int lbhpde_submit_nee(lbhpde_server_t S, const lbhpde_request *q, int boundary, const double *phib,
                                 uint64_t *id) {
    if (boundary == LBHPDE_PERIODIC) return LBHPDE_ERR_ARG;
    return submit_common(S, q, boundary, phib, id);
}

static int take_result(lbhpde_server_t S, std::unordered_map<uint64_t, Req *>::iterator it, double *phi_out,
                       lbhpde_result *info) {
    Req *r = it->second;
    fill_result(r, info);
    const int st = r->status;
    if (st == LBHPDE_PENDING) return st;
    if (phi_out && !r->phi.empty()) std::memcpy(phi_out, r->phi.data(), sizeof(double) * r->phi.size());
    S->reqs.erase(it);
    delete r;
    return st;
}

extern "C" int lbhpde_poll(lbhpde_server_t S, uint64_t id, double *phi_out, lbhpde_result *info) {
    if (!S) return LBHPDE_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LBHPDE_ERR_NOT_FOUND;
    return take_result(S, it, phi_out, info);
}

extern "C" int lbhpde_wait(lbhpde_server_t S, uint64_t id, double timeout_s, double *phi_out, lbhpde_result *info) {
    if (!S || !(timeout_s >= 0.0)) return LBHPDE_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LBHPDE_ERR_NOT_FOUND;
    Req *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration<double>(std::min(timeout_s, 1e6));
    if (!S->cv_done.wait_until(lk, deadline, [&] { return r->status != LBHPDE_PENDING; })) {
        fill_result(r, info);
        return LBHPDE_ERR_TIMEOUT;
    }
    return take_result(S, S->reqs.find(id), phi_out, info);
}

extern "C" int lbhpde_server_stats(lbhpde_server_t S, lbhpde_server_info *out) {
    if (!S || !out) return LBHPDE_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (long)S->queue.size();
    out->in_flight = (long)(S->reqs.size() - S->queue.size());
    out->completed = S->completed;
    out->node_updates = S->node_updates;
    out->bytes_in_use = S->bytes_used;
    out->bytes_total = S->arena.size();
    out->launches = S->launches;
    out->error = S->error;
    out->gpu_busy_s = S->gpu_busy;
    out->host_admit_s = S->t_admit;
    out->host_setup_s = S->t_setup;
    out->host_plan_s = S->t_plan;
    out->host_launch_s = S->t_launch;
    out->host_wait_s = S->t_wait;
    out->host_retire_s = S->t_retire;
    return LBHPDE_OK;
}

extern "C" int lbhpde_server_destroy(lbhpde_server_t S) {
    if (!S) return LBHPDE_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    cudaStreamSynchronize(S->stream);
    for (auto &kv : S->reqs) delete kv.second;
    S->reqs.clear();
    S->insts_d.release();
    S->binsts_d.release();
    S->phibt_d.release();
    S->first_d.release();
    S->segs_d.release();
    S->blocks_d.release();
    S->boff_d.release();
    S->phi0_d.release();
    cudaFree(S->arena_d);
    if (S->coefT_d != S->coefD_d) cudaFree(S->coefT_d);
    cudaFree(S->coefD_d);
    cudaStreamSynchronize(S->up);
    cudaStreamDestroy(S->stream);
    cudaStreamDestroy(S->up);
    cudaEventDestroy(S->ev_setup);
    for (int i = 0; i < lbhpde_server_s::kLanes; ++i) {
        cudaStreamDestroy(S->lane[i]);
        cudaEventDestroy(S->ev_done[i]);
    }
    cudaEventDestroy(S->ev_up);
    for (int i = 0; i < 2; ++i) {
        cudaEventDestroy(S->ev_t0[i]);
        cudaEventDestroy(S->ev_t1[i]);
    }
    cudaSetDevice(prev);
    delete S;
    return LBHPDE_OK;
}
