// Host-side pieces shared by the batch API (lbhpde_api.cu) and the request server
// (lbhpde_server.cu): packing of instances onto CTAs for the on-chip kernel and the typed
// kernel launchers.  Implemented in lbhpde_api.cu, so each kernel is compiled once.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "lbhpde.h"
#include "lbhpde_bounded.cuh"
#include "lbhpde_kernels.cuh"
#include "lbhpde_ring.cuh"
#include "lbhpde_ring_nee.cuh"

namespace lbh {

// A named NVTX range for the scope (tracing: host phases of the API and of the server show in
// Nsight timelines and can filter ncu captures; without a tool attached it costs a branch).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

constexpr int kChunk = 1024;          // nodes per block of the node-parallel kernels
constexpr int kGenericThreads = 256;  // init / readout / diagnostics threads per block

// One instance to place on the on-chip kernel.
struct Member {
    lbk::Seg seg;      // placement of the current state (and its coefficient block)
    long long off2;    // where the kernel writes the result (== seg.off for in-place)
    int steps;         // steps this instance takes in the launch
};

// A packed on-chip launch: CTA c holds insts[first[c] .. first[c + 1]).
struct Packed {
    std::vector<lbk::OnchipInst> insts;
    std::vector<int> first;
    int nthreads = 32;  // threads per CTA
    int max_inst = 1;   // instances per CTA (resident mode: rounded up to a multiple of 4)
    size_t smem = 0;    // dynamic shared memory per CTA, bytes
    int stride = 0;     // k_ring: the class's CTA size, the row stride of its exchange buffers
    int ncta() const { return first.empty() ? 0 : (int)first.size() - 1; }
};

// Threads per CTA of the on-chip kernels for (element size, lattice, nodes per thread), 0 when
// no variant exists: resident instances (capacity = threads * K nodes) and temporally blocked
// windows (FP32 D1Q5 with K = 8 uses smaller window CTAs).
constexpr int kHaloThreadsF32Q5 = 128;
// Nodes a thread of the 16-node resident kernel (k_ring, FP32 D1Q5) holds: an instance of up to
// 16 * 512 = 8192 nodes stays in one CTA.  Planned with K == kRingK, resident instances only.
constexpr int kRingK = 16;
// Whether members of (element size, lattice, on-chip degree code) can take k_ring.
bool ring_split_ok(size_t esz, int b, int dc);
int onchip_maxt(size_t esz, int b, int K);
int onchip_maxt_halo(size_t esz, int b, int K);
int default_K(size_t esz, int b);
// Steps per halo window (a power of two up to 64) such that the halo (steps * max|e| on each
// side) leaves at least valid_eighths / 8 of a window of `capacity` nodes valid.  Batches take
// 7/8 (the autotuner's picks on GB300: 32 for FP32 windows, 16 for FP64 D1Q7); the server takes
// 6/8, since each window chunk of a step block is another launch.
int default_tblk(int capacity, int W, int valid_eighths = 7);
// Compile-time degree variant the on-chip kernel uses for a set of members of maximum degree D.
int onchip_dc(int b, int maxD);

// Resident instances (N <= capacity): first fit, largest first, <= 32 per CTA, in CTAs of `threads`
// threads (0: the configuration's resident CTA size).  Runs of threads are warp-aligned for
// k_onchip and thread-granular for k_ring (K == kRingK).
int pack_ring(int b, size_t esz, int K, int dc, const std::vector<Member> &m, Packed &out, int threads = 0);
// Resident size class of an instance of N nodes (0, 1, 2) and the CTA size of a class.
constexpr int kRingClasses = 3;
int ring_class(size_t esz, int b, int K, long long N);
int ring_class_threads(size_t esz, int b, int K, int cls);
// Threads an instance's run is rounded up to (32 for k_onchip, 1 for k_ring).
int ring_granule(int K);
// Instances a CTA holds at most (the tail buffer rows of the on-chip kernels).
constexpr int kRingMaxInstances = 32;
// Wave-aware split of the 16-node resident members (K == kRingK) for a GPU of `sms` SMs: `full`
// packs (first fit, largest first) into whole waves of full-SM CTAs, one CTA per SM at a time;
// `tail` holds the members that do not fit there (or were evicted from a CTA to make room for a
// larger one).  The tail runs afterwards in CTAs of its own size class spread over the SMs, so the
// last, partial wave costs the time of its members' own work instead of a whole wave of full
// CTAs.  False (both empty) when the members do not fill one wave or all fit.
bool split_ring_waves(int b, int K, int sms, const std::vector<Member> &m, std::vector<Member> &full,
                      std::vector<Member> &tail);
// Resident members by the CTA size class they take: their own class, or the largest one where
// they fill a gap left by larger instances.
void split_ring_classes(size_t esz, int b, int K, const std::vector<Member> &m, std::vector<Member> (&out)[kRingClasses]);
// Temporally blocked windows with halo H: one window per CTA.
// wide: windows as large as a resident CTA (fewer, longer windows: the server, whose step
// blocks fix the steps per window) instead of the smaller window CTAs.
int pack_halo(int b, size_t esz, int K, int dc, int H, const std::vector<Member> &m, Packed &out,
              bool wide = false);

// K == kRingK launches k_ring (resident plans only).
int launch_onchip(int b, size_t esz, int K, int dc, bool halo, const Packed &p, const lbk::OnchipInst *insts_d,
                  const int *first_d, const void *in, void *out, const void *coefT, int nsteps, cudaStream_t st);
int launch_ring_f32(int dc, const Packed &p, const lbk::OnchipInst *insts_d, const int *first_d, const void *in,
                    void *out, const void *coefT, int nsteps, cudaStream_t st);
// the same for one precision (lbhpde_onchip_f32.cu, lbhpde_onchip_f64.cu)
int launch_onchip_f32(int b, int K, int dc, bool halo, const Packed &p, const lbk::OnchipInst *insts_d,
                      const int *first_d, const void *in, void *out, const void *coefT, int nsteps, cudaStream_t st);
int launch_onchip_f64(int b, int K, int dc, bool halo, const Packed &p, const lbk::OnchipInst *insts_d,
                      const int *first_d, const void *in, void *out, const void *coefT, int nsteps, cudaStream_t st);
// coefT: the coefficient table in the state's type (f^eq rows after the P_j rows, as lbk::Seg::coef).
int launch_init(int b, size_t esz, void *st, const lbk::Seg *segs, const int2 *blocks, int nb, const void *coefT,
                const double *phi0, const long long *blk_off, cudaStream_t stream);

// Bounded grids (lbhpde_bounded.cu): instances of up to kBoundedK * kBoundedMaxT nodes stay
// resident in one CTA each; longer ones take the streaming step plus the outer-node rebuild.
constexpr int kBoundedK = 4;
constexpr int kBoundedMaxT = 512;
constexpr int kBoundedMaxSteps = 1024;     // steps per resident launch, at most
constexpr int kBoundedStageBytes = 16384;  // shared memory for the launch's boundary data
// Dynamic shared memory of k_bounded for a launch of nsteps steps.
size_t bounded_smem(int b, size_t esz, int nthreads, int D, int nsteps);
// Steps per resident launch: as many as kBoundedStageBytes of staged boundary data hold.
int bounded_launch_steps(int b, size_t esz);
// Smallest position shift that puts each end's outer nodes and extrapolation node in one warp of
// the resident kernel (and keeps the instance within one CTA); -1 if there is none.
int bounded_shift(int b, int N, int depth);
// dc: the compiled degree (5 on D1Q5, 7 on D1Q7), 0 for a run-time degree, -1 for the variant
// that also evaluates real-exponent instances (A > 0).
int launch_bounded(int b, size_t esz, int dc, int ninst, int nthreads, size_t smem, const lbk::BoundedInst *insts_d,
                   const void *in, void *out, const void *coefT, const double *phib, long long stride,
                   long long step0, int nsteps, cudaStream_t st);
int launch_nee_fix(int b, size_t esz, void *st, const lbk::Seg *segs, const int *members, int nmem,
                   const void *coefT, const double *phib, long long stride, long long step, cudaStream_t stream);

// Bounded members on the 16-node resident kernel (k_ring_nee, FP32 D1Q5 polynomial models): the
// interior nodes W..N-W-1 in thread-granular runs of ceil((N - 2W) / 16) threads, first fit,
// largest first, at most 32 instances per CTA of `threads` threads.
struct PackedNee {
    std::vector<lbk::RingNeeInst> insts;
    std::vector<int> first;
    int nthreads = 32, stride = 0;
    bool d2 = false;  // every member of depth 2 with at least 2 interior nodes in its last thread
    size_t smem = 0;
    int ncta() const { return first.empty() ? 0 : (int)first.size() - 1; }
};
struct NeeMember {
    lbk::Seg seg;
    int mi;     // batch member index (its boundary rows)
    int steps;  // steps in the launch
};
// Whether a bounded member can take k_ring_nee: FP32 D1Q5 polynomial, its interior within one
// 512-thread CTA, depth within the first and last 16 interior nodes' reach.
bool ring_nee_ok(size_t esz, int b, const lbk::Seg &s);
int pack_ring_nee(int b, int dc, const std::vector<NeeMember> &m, PackedNee &out, int threads);
int launch_ring_nee_f32(int dc, const PackedNee &p, const lbk::RingNeeInst *insts_d, const int *first_d,
                        const void *in, void *out, const void *coefT, const double *phib, long long stride,
                        long long step0, int nsteps, cudaStream_t st);

}  // namespace lbh
