// Host-side check of the on-chip planning (no GPU): size classes, resident packing and window
// cutting on random member sets, the position shift of bounded resident instances, and the
// packing of bounded members on the 16-node kernel, called through the library's exported
// functions.  Prints
// "ok" and exits 0 when every invariant holds; otherwise prints the first violation and exits 1.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <set>
#include <vector>

#include "lbhpde_internal.h"

static int fails = 0;
#define CHECK(c, ...)                                  \
    do {                                               \
        if (!(c) && fails++ == 0) {                    \
            std::printf("FAIL %s:%d: ", __FILE__, __LINE__); \
            std::printf(__VA_ARGS__);                  \
            std::printf("\n");                         \
        }                                              \
    } while (0)

static std::vector<lbh::Member> members(std::mt19937 &g, int count, long long nmin, long long nmax, int D) {
    std::vector<lbh::Member> m;
    long long off = 0;
    std::uniform_int_distribution<long long> dn(nmin, nmax);
    for (int i = 0; i < count; ++i) {
        lbh::Member mb{};
        mb.seg.N = (int)dn(g);
        mb.seg.ld = (mb.seg.N + 31) / 32 * 32;
        mb.seg.off = off;
        mb.seg.D = D;
        mb.off2 = off;
        mb.steps = 1 + i % 7;
        off += mb.seg.ld * 7;
        m.push_back(mb);
    }
    return m;
}

static void check_ring(const lbh::Packed &p, const std::vector<lbh::Member> &m, int b, int K, int threads, int dc) {
    std::map<long long, int> seen;
    int maxn = 0;
    for (int c = 0; c < p.ncta(); ++c) {
        const int i0 = p.first[c], i1 = p.first[c + 1];
        CHECK(i1 > i0 && i1 - i0 <= 32, "cta %d holds %d instances", c, i1 - i0);
        maxn = std::max(maxn, i1 - i0);
        int tb = 0, sco = 0;
        const int gr = lbh::ring_granule(K);
        for (int i = i0; i < i1; ++i) {
            const lbk::OnchipInst &I = p.insts[i];
            CHECK(I.tbase == tb && I.tbase % gr == 0, "instance %d: thread base %d, expected %d", i, I.tbase, tb);
            CHECK(I.nthr == (I.N + K - 1) / K, "instance %d: %d threads for N = %d", i, I.nthr, I.N);
            CHECK(I.npos == I.N && I.vlo == 0 && I.vhi == I.N && I.x0 == 0, "instance %d: ring window", i);
            CHECK(I.il == i - i0, "instance %d: tail slot %d", i, I.il);
            CHECK(I.scoef == sco && I.scoef % 4 == 0, "instance %d: coefficient offset %d", i, I.scoef);
            sco += lbk::cblock(b, dc > 0 ? dc : I.D);
            tb += (I.nthr + gr - 1) / gr * gr;
            ++seen[I.off];
        }
        CHECK(tb <= threads && tb <= p.nthreads, "cta %d uses %d threads of %d (plan %d)", c, tb, threads, p.nthreads);
    }
    CHECK(p.nthreads <= threads && p.nthreads % 32 == 0, "plan threads %d, CTA size %d", p.nthreads, threads);
    if (K == lbh::kRingK) {  // exchange rows and tails at the class stride
        const size_t xchg = size_t(4) * lbk::ring_xchg_elems(b, threads);
        CHECK(p.stride == threads && p.max_inst <= lbk::kRingMaxInst && p.smem > xchg && p.smem <= 227 * 1024,
              "k_ring plan: stride %d (class %d), %d instances, shared memory %zu (exchange %zu)", p.stride, threads,
              p.max_inst, p.smem, xchg);
    }
    CHECK(p.max_inst % 4 == 0 && p.max_inst >= maxn, "max_inst %d for %d", p.max_inst, maxn);
    CHECK(seen.size() == m.size(), "%zu of %zu members placed", seen.size(), m.size());
    for (auto &kv : seen) CHECK(kv.second == 1, "member at %lld placed %d times", kv.first, kv.second);
}

static void check_halo(const lbh::Packed &p, const std::vector<lbh::Member> &m, int K, int H, int maxt) {
    std::map<long long, std::vector<int>> cover;  // member offset -> coverage count per node
    for (const lbh::Member &mb : m) cover[mb.seg.off].assign(mb.seg.N, 0);
    for (int c = 0; c < p.ncta(); ++c) {
        CHECK(p.first[c + 1] - p.first[c] == 1, "window cta %d holds %d windows", c, p.first[c + 1] - p.first[c]);
        const lbk::OnchipInst &I = p.insts[p.first[c]];
        CHECK(I.vlo == H && I.npos == I.vhi + H && I.vhi > I.vlo, "window %d: [%d, %d) of %d", c, I.vlo, I.vhi, I.npos);
        CHECK(I.nthr == (I.npos + K - 1) / K && I.nthr <= maxt, "window %d: %d threads", c, I.nthr);
        auto &cv = cover[I.off];
        for (int q = I.vlo; q < I.vhi; ++q) {
            long long x = ((long long)I.x0 + q) % I.N;
            x += x < 0 ? I.N : 0;
            ++cv[(size_t)x];
        }
    }
    CHECK(p.nthreads == maxt, "window threads %d, expected %d", p.nthreads, maxt);
    for (auto &kv : cover)
        for (size_t x = 0; x < kv.second.size(); ++x)
            if (kv.second[x] != 1) {
                CHECK(false, "member at %lld: node %zu covered %d times", kv.first, x, kv.second[x]);
                break;
            }
}

int main() {
    std::mt19937 g(20260907);
    struct Cfg {
        size_t esz;
        int b, K;
    };
    const Cfg cfgs[] = {{4, 5, lbh::kRingK}, {4, 5, 8}, {4, 5, 4}, {4, 5, 2}, {4, 7, 8},
                        {4, 7, 4},           {8, 5, 4}, {8, 5, 2}, {8, 7, 4}};
    for (const Cfg &cf : cfgs) {
        const int W = (cf.b - 1) / 2;
        const int cap = lbh::onchip_maxt(cf.esz, cf.b, cf.K) * cf.K;
        for (int trial = 0; trial < 20; ++trial) {
            const int D = trial % 2 ? 5 : 9, dc = lbh::onchip_dc(cf.b, D);
            // resident members: size classes, then each class packed
            auto m = members(g, 1 + trial * 9, 2 * W, cap, D);
            std::vector<lbh::Member> cls[lbh::kRingClasses];
            lbh::split_ring_classes(cf.esz, cf.b, cf.K, m, cls);
            size_t total = 0;
            for (int c = 0; c < lbh::kRingClasses; ++c) {
                total += cls[c].size();
                for (const lbh::Member &mb : cls[c])
                    CHECK(lbh::ring_class(cf.esz, cf.b, cf.K, mb.seg.N) == c || c == lbh::kRingClasses - 1,
                          "N = %d in class %d", mb.seg.N, c);
                if (cls[c].empty()) continue;
                const int thr = lbh::ring_class_threads(cf.esz, cf.b, cf.K, c);
                lbh::Packed p;
                CHECK(lbh::pack_ring(cf.b, cf.esz, cf.K, dc, cls[c], p, thr) == LBHPDE_OK, "pack_ring failed");
                check_ring(p, cls[c], cf.b, cf.K, thr, dc);
                // the gap fillers of the largest class do not open CTAs of their own
                if (c == lbh::kRingClasses - 1) {
                    int own = 0;
                    for (const lbh::Member &mb : cls[c]) own += lbh::ring_class(cf.esz, cf.b, cf.K, mb.seg.N) == c;
                    CHECK(own == 0 ? p.ncta() == 0 : p.ncta() <= own, "%d CTAs for %d own members", p.ncta(), own);
                }
            }
            CHECK(total == m.size(), "%zu of %zu members classified", total, m.size());
            // windows: batch-sized and server-wide, several depths (the 16-node variant is resident only)
            for (bool wide : {false, true}) {
                if (cf.K == lbh::kRingK) {
                    CHECK(lbh::onchip_maxt_halo(cf.esz, cf.b, cf.K) == 0, "windows offered for K = %d", cf.K);
                    break;
                }
                const int maxt = wide ? lbh::onchip_maxt(cf.esz, cf.b, cf.K) : lbh::onchip_maxt_halo(cf.esz, cf.b, cf.K);
                for (int eighths : {6, 7}) {
                    const int T = lbh::default_tblk(maxt * cf.K, W, eighths), H = T * W;
                    CHECK(maxt * cf.K - 2 * H >= maxt * cf.K * eighths / 8 && (T & (T - 1)) == 0 && T >= 1,
                          "default depth %d for %d nodes", T, maxt * cf.K);
                    auto mh = members(g, 1 + trial % 5, 2 * W, 3 * cap + 17, D);
                    lbh::Packed p;
                    CHECK(lbh::pack_halo(cf.b, cf.esz, cf.K, dc, H, mh, p, wide) == LBHPDE_OK, "pack_halo failed");
                    check_halo(p, mh, cf.K, H, maxt);
                }
            }
        }
    }
    // whole waves of full CTAs plus a tail (16-node kernel): every member placed once and the full
    // members pack into the whole waves' CTAs
    for (int trial = 0; trial < 24; ++trial) {
        const int sms = trial % 3 == 0 ? 4 : (trial % 3 == 1 ? 19 : 152);
        auto m = members(g, 50 + trial * 37, 4, 8192, 5);
        std::vector<lbh::Member> full, tail;
        const bool split = lbh::split_ring_waves(5, lbh::kRingK, sms, m, full, tail);
        long long total = 0;
        for (auto &mb : m) total += (mb.seg.N + lbh::kRingK - 1) / lbh::kRingK;
        const long long limit = total / (512LL * sms) * sms;
        if (!split) {
            CHECK(full.empty() && tail.empty(), "no split, yet members assigned");
            continue;
        }
        CHECK(limit > 0 && full.size() + tail.size() == m.size(), "split of %zu members: %zu + %zu", m.size(),
              full.size(), tail.size());
        std::set<long long> seen;
        for (auto &mb : full) seen.insert(mb.seg.off);
        for (auto &mb : tail) seen.insert(mb.seg.off);
        CHECK(seen.size() == m.size(), "%zu distinct members of %zu after the split", seen.size(), m.size());
        lbh::Packed p;
        CHECK(lbh::pack_ring(5, 4, lbh::kRingK, 5, full, p, 512) == LBHPDE_OK, "pack of the full members failed");
        CHECK(p.ncta() <= limit, "%d full CTAs for %lld in the whole waves", p.ncta(), limit);
        check_ring(p, full, 5, lbh::kRingK, 512, 5);
    }
    // bounded resident instances: the host's position shift puts each end's outer nodes and its
    // extrapolation node in one warp of live threads, inside the CTA
    const int KB = lbh::kBoundedK, wpos = 32 * KB;  // positions per warp
    long long shifted = 0;
    for (int b : {5, 7}) {
        const int W = (b - 1) / 2;
        for (int depth = 1; depth <= 4; ++depth)
            for (int N = 2 * (W + depth); N <= KB * lbh::kBoundedMaxT; ++N) {
                const int sh = lbh::bounded_shift(b, N, depth);
                if (sh < 0) {
                    // only when the shifted grid would not fit the CTA
                    CHECK(N + wpos > KB * lbh::kBoundedMaxT, "no shift for N = %d, depth %d, b = %d", N, depth, b);
                    continue;
                }
                ++shifted;
                const int kL = W - 1 + depth, kR = N - W - depth;
                CHECK(N + sh <= KB * lbh::kBoundedMaxT, "N = %d + shift %d exceeds the CTA", N, sh);
                CHECK((0 + sh) / wpos == (kL + sh) / wpos, "left end split, N = %d, depth %d", N, depth);
                CHECK((kR + sh) / wpos == (N - 1 + sh) / wpos, "right end split, N = %d, depth %d", N, depth);
            }
    }
    CHECK(shifted > 10000, "only %lld bounded cases placed", shifted);

    // bounded members on the 16-node kernel (pack_ring_nee, FP32 D1Q5): every member once, thread
    // runs of ceil((N - 2W) / 16) threads one after the other, at most 32 instances a CTA and at
    // least one thread per helper role (2 nedge(B) an instance) in the launch, coefficient blocks
    // of nee_cblock at 16-byte aligned offsets, shared memory within 227 KB, and the depth-2
    // variant chosen exactly when every member has depth 2 and 2 or more nodes in its last thread
    for (int trial = 0; trial < 60; ++trial) {
        const int b = 5, W = 2, K = lbh::kRingK, dc = trial % 3 ? 5 : 0;
        std::uniform_int_distribution<int> dcount(1, 400), ddepth(1, 4);
        const bool only2 = trial % 2 == 0;
        const long long nmax = trial % 5 == 0 ? 40 : 512LL * K + 2 * W;
        std::vector<lbh::NeeMember> m;
        const int count = dcount(g);
        long long off = 0;
        bool d2 = true;
        for (int i = 0; i < count; ++i) {
            lbh::NeeMember x{};
            x.seg.pad = only2 ? 2 : ddepth(g);
            std::uniform_int_distribution<long long> dn(2 * (W + x.seg.pad), nmax);
            x.seg.N = (int)dn(g);
            x.seg.ld = (x.seg.N + 31) / 32 * 32;
            x.seg.off = off;
            x.seg.D = 5;
            x.mi = i;
            x.steps = 1 << 30;
            off += x.seg.ld * b;
            const int thr = (x.seg.N - 2 * W + K - 1) / K;
            if (x.seg.pad != 2 || x.seg.N - 2 * W - K * (thr - 1) < 2) d2 = false;
            CHECK(lbh::ring_nee_ok(4, b, x.seg), "ring_nee_ok refused N = %d depth %d", x.seg.N, x.seg.pad);
            m.push_back(x);
        }
        lbh::PackedNee p;
        CHECK(lbh::pack_ring_nee(b, dc, m, p, 512) == LBHPDE_OK, "pack_ring_nee failed (trial %d)", trial);
        CHECK(p.d2 == d2, "depth-2 variant %d, expected %d (trial %d)", (int)p.d2, (int)d2, trial);
        CHECK(p.nthreads % 32 == 0 && p.nthreads <= 512 && p.stride == 512, "launch of %d threads", p.nthreads);
        CHECK(p.smem <= 227 * 1024, "shared memory %zu", p.smem);
        std::set<int> seen;
        for (int c = 0; c < p.ncta(); ++c) {
            const int i0 = p.first[c], i1 = p.first[c + 1];
            CHECK(i1 > i0 && i1 - i0 <= lbk::kRingMaxInst, "cta %d holds %d instances", c, i1 - i0);
            CHECK((i1 - i0) * lbk::nee_roles(b) <= p.nthreads, "cta %d: %d helper roles, %d threads", c,
                  (i1 - i0) * lbk::nee_roles(b), p.nthreads);
            int tb = 0, sco = 0;
            for (int i = i0; i < i1; ++i) {
                const lbk::RingNeeInst &I = p.insts[i];
                CHECK(I.tbase == tb, "instance %d: thread base %d, expected %d", i, I.tbase, tb);
                CHECK(I.nthr == (I.N - 2 * W + K - 1) / K, "instance %d: %d threads for N = %d", i, I.nthr, I.N);
                CHECK(I.il == i - i0, "instance %d: block %d", i, I.il);
                CHECK(I.scoef == sco && I.scoef % 4 == 0, "instance %d: coefficient offset %d", i, I.scoef);
                CHECK(I.depth == m[I.mi].seg.pad && I.N == m[I.mi].seg.N && I.off == m[I.mi].seg.off,
                      "instance %d: member %d", i, I.mi);
                sco += lbk::nee_cblock(b, dc > 0 ? dc : I.D);
                tb += I.nthr;
                CHECK(seen.insert(I.mi).second, "member %d placed twice", I.mi);
            }
            CHECK(tb <= p.nthreads, "cta %d: %d threads of runs, launch of %d", c, tb, p.nthreads);
        }
        CHECK((int)seen.size() == count, "%zu of %d members placed", seen.size(), count);
    }
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
