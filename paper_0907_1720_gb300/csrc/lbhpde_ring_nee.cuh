// Bounded instances (non-equilibrium extrapolation boundary) resident at 16 nodes a thread.
//
// The step of k_ring (Eq. (LBE) in pull form, flux-difference update of phi, relaxation with
// P_j = omega f^eq_j of Eqs. (EDF5)/(EDF7)) on the interior nodes W..N-W-1, and the rebuild of
// the W = max|e| outer nodes at each end that the paper applies to its bounded test problems
// (Sec. IV, after Guo et al.; the rule and its depth are this library's reading):
//   phi(x_b) = phi_b,   s_j(x_b) = f^eq_j(phi_b) + [s_j(x_f) - f^eq_j(phi(x_f))],
// x_f = W - 1 + depth on the left and N - W - depth on the right.  Collision scales the
// non-equilibrium part of every node by (1 - omega) and leaves f^eq unchanged, so rebuilding
// from the post-collision state equals rebuilding before the collision (as in k_bounded).
//
// Layout: the interior nodes of an instance sit in registers, 16 a thread in a thread-granular
// run (interior node W + 16 t + k at position k of thread t).  The 2W outer nodes live in shared
// memory, one block per instance and step parity, since their own collision and streaming would
// be overwritten by the rebuild anyway:
//   * the first thread's right-moving inflow from nodes below W reads the left outer nodes
//     (fixed addresses);
//   * the last thread's left-moving inflow from nodes past N-W-1 reads the right outer nodes:
//     the registers of its first positions past the last interior node take them by a jump on
//     the remainder, and neighbour reads past it take their address (as the wrap-around of
//     k_ring);
//   * after the relaxation, the thread that holds x_f of an end copies x_f's phi and s_j to its
//     column of shared memory (a jump on the position that only reads registers), and writes the
//     end's rebuilt outer nodes into the block of the next step's parity.  The next step's
//     barrier orders that write before every read of it.
// The interior reads only the inflow populations of the outer nodes (at the left end those with
// e_j > 0 at nodes W - e_j .. W - 1, at the right end those with e_j < 0 at nodes N - W ..
// N - W - 1 - e_j: 2 nedge(B) values an instance), so every step but the last rebuilds only those;
// the last rebuilds every population and phi_b, the state written back.  The state-free term of
// an inflow value, f^eq_j(phi_b), is ready before the rebuild needs it: during step s - 1 one
// helper thread per (instance, inflow value) evaluates it for the rebuild of step s into a block
// of parity s & 1 (the barrier of step s orders it before the rebuild; the block is rewritten only
// after the next barrier), from a boundary value that it copied into shared memory by cp.async
// a step before (row step0 + s of the member's block, phib + mi * stride), so neither the global
// load nor that polynomial lies on the rebuild's path.  After the last step the first thread of
// each instance writes the outer nodes back.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbhpde_ring.cuh"

namespace lbk {

// One bounded instance of the 16-node resident kernel.
struct RingNeeInst {
    long long off, ld;  // state placement (as Seg) in st_in
    long long off2;     // placement of the result in st_out
    int N, D;
    int gcoef;          // coefficient block in global memory (as Seg::coef)
    int scoef;          // this instance's P_j rows, f^eq_j rows and 1 - omega in shared memory
    int tbase, nthr;    // first CTA thread, threads: ceil((N - 2W) / 16)
    int mi;             // batch member index: its boundary rows start at phib + mi * stride
    int depth;          // extrapolation depth
    int il;             // index among the CTA's instances (outer-node block)
    int steps;          // steps this instance takes in the launch (capped at nsteps)
};

// Shared coefficient block of one bounded instance: P_j rows, f^eq_j rows (stride crow(D)),
// 1 - omega, padded to a multiple of 4.
__host__ __device__ constexpr int nee_cblock(int B, int D) { return 2 * (B - 1) * crow(D) + 4; }
// Helper threads of an instance: one per inflow value of its outer nodes (nedge(B) an end).
__host__ __device__ constexpr int nee_roles(int B) { return 2 * nedge(B); }
// Helper threads of a CTA at most.
__host__ __device__ constexpr int nee_helpers(int B) { return kRingMaxInst * nee_roles(B); }
// Shared elements (4-byte) of a k_ring_nee CTA of MAXT threads, without the coefficient blocks:
// the exchange rows, the x_f column, the outer-node blocks and the boundary terms
// [2 parities][kRingMaxInst][2W][B] (f^eq_j(phi_b) of the inflow values), the helpers' copied
// boundary values [2 parities][helpers] doubles, and each helper's source address (8 bytes) and
// its int4 (coefficient row, steps, destination, -) in shared memory rather than in registers.
__host__ __device__ constexpr int nee_fixed_elems(int B, int MAXT) {
    return 4 * nedge(B) * MAXT + B * MAXT + 2 * 2 * kRingMaxInst * 2 * wmax(B) * B + 2 * 2 * nee_helpers(B) +
           2 * nee_helpers(B) + 4 * nee_helpers(B);
}

// Asynchronous 8-byte copy global -> shared (visible to this thread after cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Horner of one coefficient row (degree DC at compile time, else D).
template <typename T, int DC>
__device__ __forceinline__ T nee_row(const T *c, int D, T x) {
    if constexpr (DC > 0) {
        T acc = c[DC];
#pragma unroll
        for (int p = DC - 1; p >= 0; --p) acc = fma_t(acc, x, c[p]);
        return acc;
    } else {
        T acc = c[D];
        for (int p = D - 1; p >= 0; --p) acc = fma_t(acc, x, c[p]);
        return acc;
    }
}

template <typename T, int B, int K, int MAXT, int DC, bool D2>
__global__ void __launch_bounds__(MAXT, ring_minb(MAXT))
    k_ring_nee(const T *__restrict__ st_in, T *__restrict__ st_out, const RingNeeInst *__restrict__ insts,
               const int *__restrict__ cta_first, const T *__restrict__ coefs, const double *__restrict__ phib,
               long long stride, long long step0, int nsteps) {
    constexpr int W = wmax(B);
    constexpr int NE = nedge(B);
    constexpr int PS = NE * MAXT;                 // one parity of R (or L)
    constexpr int OS = kRingMaxInst * 2 * W * B;  // one parity of the outer-node blocks
    constexpr int RCH = 8;                        // Horner chunk, as in k_ring
    static_assert(K >= 2 * W + 1 && K <= 16, "nodes a thread");
    static_assert(std::is_same<T, float>::value, "the bounded 16-node kernel is FP32 (packed pairs)");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *R = reinterpret_cast<T *>(smem_raw);  // [2][NE][MAXT]
    T *L = R + 2 * PS;                        // [2][NE][MAXT]
    T *X = L + 2 * PS;                        // [B][MAXT]: x_f values of the rebuilding threads
    T *OB = X + B * MAXT;                     // [2][kRingMaxInst][2W][B] outer nodes
    T *GB = OB + 2 * OS;                      // [2][kRingMaxInst][2W][B] f^eq_j(phi_b), inflow
    constexpr int NH = nee_helpers(B);
    double *PBs = reinterpret_cast<double *>(GB + 2 * OS);  // [2][NH] helpers' boundary values
    const double **HSrc = reinterpret_cast<const double **>(PBs + 2 * NH);  // [NH] helper's next row
    int4 *HMeta = reinterpret_cast<int4 *>(HSrc + NH);  // [NH] row of f^eq_j, steps, destination
    T *scoef = reinterpret_cast<T *>(HMeta + NH);

    const int nt = blockDim.x;
    const int first = cta_first[blockIdx.x], last = cta_first[blockIdx.x + 1];
    const int tid = threadIdx.x;
    for (int i = first; i < last; ++i) {
        const RingNeeInst I = insts[i];
        const int Dk = DC > 0 ? DC : I.D;
        const int cs = crow(Dk), n = (B - 1) * (I.D + 1);
        for (int q = tid; q < 2 * (B - 1) * cs; q += nt) {
            const int h = q / ((B - 1) * cs), r = q % ((B - 1) * cs);  // h = 0: P_j, 1: f^eq_j
            const int j = r / cs, pp = r % cs;
            scoef[I.scoef + q] = pp <= I.D ? coefs[I.gcoef + h * n + j * (I.D + 1) + pp] : T(0);
        }
        if (tid == 0) scoef[I.scoef + 2 * (B - 1) * cs] = coefs[I.gcoef + 2 * n];
        // the outer nodes' initial state (parity 0): row j of node o (o < W: node o; else node
        // N - 2W + o)
        for (int q = tid; q < 2 * W * B; q += nt) {
            const int o = q / B, j = q % B;
            const long long x = o < W ? o : I.N - 2 * W + o;
            OB[(I.il * 2 * W + o) * B + j] = st_in[I.off + (long long)j * I.ld + x];
        }
    }
    // helper role: instance hi of the CTA, inflow value of outer node ho (ho < W: left end) and
    // population hj (|e| = ha, the ha - 1 - hk-th node from the interior at the left end, the
    // hk-th at the right); it copies the boundary value of rebuild r (row step0 + r) two
    // rebuilds ahead
    constexpr int HP = nee_roles(B);
    const int h_n = (last - first) * HP;
    const bool helper = tid < h_n;
    const int hi = tid / HP, hr = tid % HP, hside = hr / NE, hrr = hr % NE;
    int ha = 1;
    while (ha < W && hrr >= eslot(ha + 1)) ++ha;
    const int hk = hrr - eslot(ha);
    const int ho = hside == 0 ? W - ha + hk : W + hk, hj = hside == 0 ? 2 * ha - 1 : 2 * ha;
    if (helper) {
        const RingNeeInst &H = insts[first + hi];
        const double *hsrc = phib + (long long)H.mi * stride + step0 * (2 * W) + ho;
        const int hsteps = H.steps < nsteps ? H.steps : nsteps;
        const int hD = DC > 0 ? DC : H.D;
        HSrc[tid] = hsrc + 2 * (2 * W);
        HMeta[tid] = make_int4(H.scoef + (B - 1) * crow(hD) + (hj - 1) * crow(hD), hsteps,
                               (hi * 2 * W + ho) * B + hj, hD);
        if (hsteps > 0) cp_async8(PBs + tid, hsrc);
        if (hsteps > 1) cp_async8(PBs + NH + tid, hsrc + 2 * W);
    }
    // f^eq_j(phi_b) of rebuild r into its parity, and the copy of row r + 2 into the freed slot
    // (the helper's state comes from shared memory each step: no registers held across steps)
    auto help = [&](int r) {
        if (!helper) return;
        const int4 m = HMeta[tid];
        if (r >= m.y) return;
        cp_async_wait_all();
        const T pb = (T)PBs[(r & 1) * NH + tid];
        GB[(r & 1) * OS + m.z] = nee_row<T, DC>(scoef + m.x, m.w, pb);
        if (r + 2 < m.y) {
            const double *src = HSrc[tid];
            cp_async8(PBs + (r & 1) * NH + tid, src);
            HSrc[tid] = src + 2 * W;
        }
    };
    int me = -1;
    for (int i = first; i < last; ++i) {
        const int tb = insts[i].tbase;
        if (tid >= tb && tid < tb + insts[i].nthr) me = i;
    }
    RingNeeInst I{};
    if (me >= 0) I = insts[me];
    const int t = tid - I.tbase;
    const bool has = me >= 0;
    const int N = I.N;
    const int xb = W + t * K;    // node of this thread's first position
    const int rem = N - W - xb;  // positions k >= rem lie past the last interior node
    T phi[K], v[B][K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const bool ok = has && k < rem;
        phi[k] = ok ? st_in[I.off + xb + k] : T(0);
#pragma unroll
        for (int j = 1; j < B; ++j) v[j][k] = ok ? st_in[I.off + (long long)j * I.ld + xb + k] : T(0);
    }
    __syncthreads();  // coefficients and outer nodes staged
    if constexpr (!D2) help(0);  // ordered before the rebuild of step 0 by the barrier of step 0
    const T *sc = scoef + I.scoef;
    const int D = DC > 0 ? DC : I.D;
    const int cs = crow(D);
    const T *Q = sc + (B - 1) * cs;  // f^eq_j rows
    const T omw = has ? sc[2 * (B - 1) * cs] : T(0);
    const int steps = has ? (I.steps < nsteps ? I.steps : nsteps) : 0;
    T *const Rme = R + tid;
    T *const Lme = L + tid;
    T *const Xme = X + tid;
    const bool has_right = has && t + 1 < I.nthr;
    const T *const Lrt = L + (has_right ? tid + 1 : tid);
    T *const OBi = OB + (has ? I.il : 0) * 2 * W * B;  // this instance's outer block, parity 0
    // x_f of each end, as interior indices: its thread rebuilds that end
    // (packed: bit 0 left end, bit 1 right end, then x_f's position in this thread for each end)
    int rbk = 0;
    {
        const int fL = has ? I.depth - 1 : -K, fR = has ? N - 2 * W - I.depth : -K;
        if (fL >= t * K && fL < t * K + K) rbk |= 1 | (fL - t * K) << 2;
        if (fR >= t * K && fR < t * K + K) rbk |= 2 | (fR - t * K) << 6;
    }

    // x_f's phi and s_j into this thread's column of X (a jump on its position pf)
    auto extract = [&](int pf) {
        auto get = [&](auto pc) {
            constexpr int Pv = decltype(pc)::value;
            Xme[0] = phi[Pv];
#pragma unroll
            for (int j = 1; j < B; ++j) Xme[j * MAXT] = v[j][Pv];
        };
        switch (pf) {
#define LBK_NEE_XF(Pv)                          \
    case Pv:                                    \
        get(std::integral_constant<int, Pv>{}); \
        break;
            LBK_NEE_XF(0) LBK_NEE_XF(1) LBK_NEE_XF(2) LBK_NEE_XF(3) LBK_NEE_XF(4) LBK_NEE_XF(5)
            LBK_NEE_XF(6) LBK_NEE_XF(7) LBK_NEE_XF(8) LBK_NEE_XF(9) LBK_NEE_XF(10) LBK_NEE_XF(11)
            LBK_NEE_XF(12) LBK_NEE_XF(13) LBK_NEE_XF(14) LBK_NEE_XF(15)
#undef LBK_NEE_XF
            default:
                break;
        }
    };
    // the inflow values of one end after step s (of parity P) into the block of parity P ^ 1
    auto rebuild_inflow = [&](int P, int pf, auto sidec) {
        constexpr int side = decltype(sidec)::value;
        extract(pf);
        const T phf = Xme[0];
        const int blk = (OBi - OB) + side * W * B;  // this end's outer nodes in a block
        T *const nob = OB + (P ^ 1) * OS + blk;
        const T *const g = GB + P * OS + blk;  // f^eq_j(phi_b), from the helpers
#pragma unroll
        for (int a = 1; a <= W; ++a) {
            const int j = side == 0 ? 2 * a - 1 : 2 * a;
            const T fn = Xme[j * MAXT] - nee_row<T, DC>(Q + (j - 1) * cs, D, phf);
#pragma unroll
            for (int k = 0; k < a; ++k) {
                const int o = side == 0 ? W - a + k : k;
                nob[o * B + j] = g[o * B + j] + fn;
            }
        }
    };
    // every population and phi_b of one end after the last step (the state written back), into
    // the block of parity steps & 1
    auto rebuild_all = [&](int pf, int side) {
        extract(pf);
        const T phf = Xme[0];
        T *const nob = OB + (steps & 1) * OS + (OBi - OB) + side * W * B;
        const double *row = phib + (long long)I.mi * stride + (step0 + steps - 1) * (2 * W) + side * W;
        for (int x = 0; x < W; ++x) {
            const T pb = (T)row[x];
            for (int j = 1; j < B; ++j) {
                const T *q = Q + (j - 1) * cs;
                nob[x * B + j] = nee_row<T, DC>(q, D, pb) + (Xme[j * MAXT] - nee_row<T, DC>(q, D, phf));
            }
            nob[x * B] = pb;
        }
    };
    auto step = [&](auto parc, int s) {
        constexpr int P = decltype(parc)::value;
        const bool live = s < steps;
        if (live) {
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const int e = vel(j);
                if (e > 0) {
#pragma unroll
                    for (int i = 0; i < e; ++i) Rme[P * PS + (eslot(e) + i) * MAXT] = v[j][K - e + i];
                } else {
#pragma unroll
                    for (int i = 0; i < -e; ++i) Lme[P * PS + (eslot(-e) + i) * MAXT] = v[j][i];
                }
            }
        }
        __syncthreads();
        if constexpr (D2)
            help(s);  // read at the start of step s + 1
        else
            help(s + 1);
        if (!live) return;
        const T *ob = OBi + P * OS;  // the outer nodes of this step
        // depth 2 (every instance of the launch, x_f of each end in its end thread): the inflow of
        // step s is rebuilt at its start by the thread that reads it, from x_f's state after step
        // s - 1 at a fixed register position (position 1 of the first thread; position rem - 2 of
        // the last, in the jump on the remainder), with f^eq_j(phi_b) of rebuild s - 1 from the
        // helpers (block of parity s - 1)
        T inL[NE] = {};
        if constexpr (D2) {
            if (t == 0) {
                if (s == 0) {
#pragma unroll
                    for (int e = 1; e <= W; ++e)
#pragma unroll
                        for (int k = 0; k < e; ++k) inL[eslot(e) + k] = ob[(W - e + k) * B + 2 * e - 1];
                } else {
                    const T *const g = GB + (P ^ 1) * OS + (OBi - OB);
#pragma unroll
                    for (int e = 1; e <= W; ++e) {
                        const int j = 2 * e - 1;
                        const T fn = v[j][1] - nee_row<T, DC>(Q + (j - 1) * cs, D, phi[1]);
#pragma unroll
                        for (int k = 0; k < e; ++k) inL[eslot(e) + k] = g[(W - e + k) * B + j] + fn;
                    }
                }
            }
        }
        // the last thread: its first positions past the last interior node take the right outer
        // nodes' left-moving populations (named registers, a jump on the remainder)
        auto put = [&](auto rc) {
            constexpr int Rr = decltype(rc)::value;
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const int a = -vel(j);
#pragma unroll
                for (int i = 0; i < a; ++i)
                    if (Rr + i < K) v[j][Rr + i] = ob[(W + i) * B + j];
            }
        };
        if constexpr (D2) {
            // the last thread (rem >= 2): the right end's inflow values into this step's block
            // (read back by the jump below and by the neighbour reads past the last node)
            auto fixput = [&](auto rc) {
                constexpr int Rr = decltype(rc)::value, pf = Rr - 2;
                if (s > 0) {
                    T *const o = OBi + P * OS + W * B;
                    const T *const g = GB + (P ^ 1) * OS + (OBi - OB) + W * B;
#pragma unroll
                    for (int a = 1; a <= W; ++a) {
                        const int j = 2 * a;
                        const T fn = v[j][pf] - nee_row<T, DC>(Q + (j - 1) * cs, D, phi[pf]);
#pragma unroll
                        for (int i = 0; i < a; ++i) o[i * B + j] = g[i * B + j] + fn;
                    }
                }
                put(rc);
            };
            if (has && !has_right) {
                switch (rem < K ? rem : K) {
#define LBK_NEE_FIX(Rv)                            \
    case Rv:                                       \
        fixput(std::integral_constant<int, Rv>{}); \
        break;
                    LBK_NEE_FIX(2) LBK_NEE_FIX(3) LBK_NEE_FIX(4) LBK_NEE_FIX(5) LBK_NEE_FIX(6) LBK_NEE_FIX(7)
                    LBK_NEE_FIX(8) LBK_NEE_FIX(9) LBK_NEE_FIX(10) LBK_NEE_FIX(11) LBK_NEE_FIX(12) LBK_NEE_FIX(13)
                    LBK_NEE_FIX(14) LBK_NEE_FIX(15) LBK_NEE_FIX(16)
#undef LBK_NEE_FIX
                    default:
                        break;
                }
            }
        } else if (rem < K) {
            switch (rem) {
#define LBK_NEE_REM(Rv)                         \
    case Rv:                                    \
        put(std::integral_constant<int, Rv>{}); \
        break;
                LBK_NEE_REM(1) LBK_NEE_REM(2) LBK_NEE_REM(3) LBK_NEE_REM(4) LBK_NEE_REM(5)
                LBK_NEE_REM(6) LBK_NEE_REM(7) LBK_NEE_REM(8) LBK_NEE_REM(9) LBK_NEE_REM(10)
                LBK_NEE_REM(11) LBK_NEE_REM(12) LBK_NEE_REM(13) LBK_NEE_REM(14) LBK_NEE_REM(15)
#undef LBK_NEE_REM
                default:
                    break;
            }
        }
        T d[K];
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = T(-0.0);
        // sources in this thread's registers first, then the neighbours' or the outer nodes'
#pragma unroll
        for (int j = 1; j < B; ++j) {
            const int e = vel(j);
            if (e == 2 && K % 2 == 0) {
                // |e| = 2: pairs of nodes in one packed operation each (as in k_ring)
#pragma unroll
                for (int k = K - 2; k >= 2; k -= 2) {
                    const float2 nv = make_float2(v[j][k - 2], v[j][k - 1]);
                    const float2 df = __ffma2_rn(make_float2(v[j][k], v[j][k + 1]), make_float2(-1.f, -1.f), nv);
                    const float2 dd = __fadd2_rn(make_float2(d[k], d[k + 1]), df);
                    d[k] = dd.x;
                    d[k + 1] = dd.y;
                    v[j][k] = nv.x;
                    v[j][k + 1] = nv.y;
                }
            } else if (e == -2 && K % 2 == 0) {
#pragma unroll
                for (int k = 0; k + 2 < K; k += 2) {
                    const float2 nv = make_float2(v[j][k + 2], v[j][k + 3]);
                    const float2 df = __ffma2_rn(make_float2(v[j][k], v[j][k + 1]), make_float2(-1.f, -1.f), nv);
                    const float2 dd = __fadd2_rn(make_float2(d[k], d[k + 1]), df);
                    d[k] = dd.x;
                    d[k + 1] = dd.y;
                    v[j][k] = nv.x;
                    v[j][k + 1] = nv.y;
                }
            } else if (e > 0) {
#pragma unroll
                for (int k = K - 1; k >= e; --k) {
                    const T nv = v[j][k - e];
                    d[k] += nv - v[j][k];
                    v[j][k] = nv;
                }
            } else {
                const int a = -e;
#pragma unroll
                for (int k = 0; k + a < K; ++k) {
                    const T nv = v[j][k + a];
                    d[k] += nv - v[j][k];
                    v[j][k] = nv;
                }
            }
        }
#pragma unroll
        for (int j = 1; j < B; ++j) {
            const int e = vel(j);
            if (e > 0) {
#pragma unroll
                for (int k = 0; k < e; ++k) {
                    const T nv = t > 0 ? Rme[P * PS + (eslot(e) + k) * MAXT - 1]
                                       : (D2 ? inL[eslot(e) + k] : ob[(W + k - e) * B + j]);
                    d[k] += nv - v[j][k];
                    v[j][k] = nv;
                }
            } else {
                const int a = -e;
#pragma unroll
                for (int k = K - a; k < K; ++k) {
                    // right outer node index, clamped so that the address not taken stays in bounds
                    int q = k + a - rem;
                    q = q < 0 ? 0 : (q < W - 1 ? q : W - 1);
                    const T *src = k + a >= rem ? ob + (W + q) * B + j : Lrt + P * PS + (eslot(a) + k + a - K) * MAXT;
                    const T nv = *src;
                    d[k] += nv - v[j][k];
                    v[j][k] = nv;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; k += 2) {  // two nodes per packed add
            const float2 p2 = __fadd2_rn(make_float2(phi[k], phi[k + 1]), make_float2(d[k], d[k + 1]));
            phi[k] = p2.x;
            phi[k + 1] = p2.y;
        }
        ring_relax<T, B, K, DC, RCH, 0, K>(sc, cs, D, omw, phi, v);
        // the rebuild of the inflow values (population j with |e_j| = a at its a nodes next to
        // the interior) from x_f's phi and s_j, which pass through this thread's column of X
        if (!D2 && rbk && s + 1 < steps) {
            if (rbk & 1) rebuild_inflow(P, (rbk >> 2) & 15, std::integral_constant<int, 0>{});
            if (rbk & 2) rebuild_inflow(P, (rbk >> 6) & 15, std::integral_constant<int, 1>{});
        }
    };
    for (int s = 0; s < nsteps; s += 2) {
        step(std::integral_constant<int, 0>{}, s);
        if (s + 1 < nsteps) step(std::integral_constant<int, 1>{}, s + 1);
    }
    // (parity steps & 1 was last read in step steps - 2, before the barrier of step steps - 1)
    if (has) I = insts[me];  // reloaded: nothing of it stays in registers across the steps
    if (steps > 0 && (rbk & 1)) rebuild_all((rbk >> 2) & 15, 0);
    if (steps > 0 && (rbk & 2)) rebuild_all((rbk >> 6) & 15, 1);
    __syncthreads();  // the outer nodes after the last step are in the block of parity steps & 1
    if (has && t == 0) {
        const T *ob = OBi + (steps & 1) * OS;
        for (int o = 0; o < 2 * W; ++o) {
            const long long x = o < W ? o : N - 2 * W + o;
#pragma unroll
            for (int j = 0; j < B; ++j) st_out[I.off2 + (long long)j * I.ld + x] = ob[o * B + j];
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (has && k < rem) {
            st_out[I.off2 + xb + k] = phi[k];
#pragma unroll
            for (int j = 1; j < B; ++j) st_out[I.off2 + (long long)j * I.ld + xb + k] = v[j][k];
        }
    }
}

}  // namespace lbk
