// Resident periodic instances, 16 nodes a thread (a2-a6, many steps per launch).
//
// Same state, placement and update as the ring mode of k_onchip (Eq. (LBE) in pull form with
// the flux-difference update of phi, coefficients P_j = omega f^eq_j of Eqs. (EDF5)/(EDF7)),
// with two differences that keep the FP32 D1Q5 lanes busy:
//   * 16 nodes a thread, so an instance of up to 8192 nodes stays in the registers of one
//     512-thread CTA for every step, and the per-step exchange and barrier are spread over
//     twice as many node-updates;
//   * instances take runs of consecutive threads that need not start on a warp boundary
//     (no idle lanes between instances).
// Every thread runs the same step: publish its edge populations, one CTA barrier, then the
// pulls from its own registers, the pulls from its neighbours' slots and the relaxation of all
// 16 nodes.  The wrap-around of an instance is folded into the pulls: the registers of the
// last thread's first positions past node N-1 take the head values (thread 0's published first
// values) before the pulls, and a neighbour read past node N-1 reads the head slot instead.
// (A split barrier that relaxed the interior nodes while the edge values were in flight, with an
// mbarrier per step parity, was slower on GB300: 6.0e11 against 6.9e11 node-updates/s on the
// ensemble.)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbhpde_kernels.cuh"

namespace lbk {

// The first NC coefficients of a 16-byte aligned shared-memory row, by the widest loads that fit.
template <typename T, int NC>
__device__ __forceinline__ void load_coefs(const T *c, T (&cr)[NC]) {
    constexpr int V = 16 / (int)sizeof(T);
    int q = 0;
#pragma unroll
    for (; q + V <= NC; q += V) {
        if constexpr (sizeof(T) == 4) {
            const float4 w = *reinterpret_cast<const float4 *>(c + q);
            cr[q] = w.x, cr[q + 1] = w.y, cr[q + 2] = w.z, cr[q + 3] = w.w;
        } else {
            const double2 w = *reinterpret_cast<const double2 *>(c + q);
            cr[q] = w.x, cr[q + 1] = w.y;
        }
    }
    if constexpr (sizeof(T) == 4 && NC % 4 >= 2) {
        const float2 w = *reinterpret_cast<const float2 *>(c + (NC & ~3));
        cr[NC & ~3] = w.x, cr[(NC & ~3) + 1] = w.y;
    }
    if constexpr (NC % V % 2 == 1) cr[NC - 1] = c[NC - 1];
}

// Relax the nodes [K0, K1) and [K2, K3) of a thread: s'_j = (1 - omega) f_j + P_j(phi'), Horner in
// phi with the coefficient rows of P_j in shared memory (stride cs; DC > 0: degree DC at compile
// time).  The nodes go through the recursion in chunks of CH (fewer live registers than one
// chain per node at once).  In FP32 with a compile-time degree, two neighbouring nodes take one
// packed multiply-add (__ffma2_rn: each half rounds as one fmaf, so the result is bit for bit
// that of one node at a time), which halves the issue slots of the recursion.  (Measured on
// GB300: 4% faster on the ensemble; pairing two populations of one node instead, or loading
// duplicated coefficient pairs by 8-byte loads, was slower than the unpaired recursion.)
template <typename T, int B, int K, int DC, int CH, int K0, int K1, int K2 = K1, int K3 = K1>
__device__ __forceinline__ void ring_relax(const T *sc, int cs, int D, T omw, const T (&phi)[K], T (&v)[B][K]) {
    constexpr int NA = K1 - K0, NN = NA + (K3 - K2);
    if constexpr (NN > 0) {
        auto node = [](int i) { return i < NA ? K0 + i : K2 + i - NA; };
#pragma unroll
        for (int j = 1; j < B; ++j) {
            const T *c = sc + (j - 1) * cs;
            if constexpr (DC > 0 && std::is_same<T, float>::value && CH % 2 == 0 && NN % CH == 0) {
                // two nodes per packed FP32 multiply-add (the same roundings as one at a time)
#pragma unroll
                for (int i0 = 0; i0 < NN; i0 += CH) {
                    float2 acc[CH / 2];
                    const float cD = c[DC];
#pragma unroll
                    for (int i = 0; i < CH / 2; ++i) acc[i] = make_float2(cD, cD);
#pragma unroll
                    for (int p = DC - 1; p >= 0; --p) {
                        const float cp = c[p];
                        const float2 cp2 = make_float2(cp, cp);
#pragma unroll
                        for (int i = 0; i < CH / 2; ++i)
                            acc[i] = __ffma2_rn(acc[i], make_float2(phi[node(i0 + 2 * i)], phi[node(i0 + 2 * i + 1)]), cp2);
                    }
#pragma unroll
                    for (int i = 0; i < CH / 2; ++i) {
                        v[j][node(i0 + 2 * i)] = fma_t(omw, v[j][node(i0 + 2 * i)], acc[i].x);
                        v[j][node(i0 + 2 * i + 1)] = fma_t(omw, v[j][node(i0 + 2 * i + 1)], acc[i].y);
                    }
                }
            } else if constexpr (DC > 0) {
#pragma unroll
                for (int i0 = 0; i0 < NN; i0 += CH) {
                    T acc[CH];
                    const T cD = c[DC];
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        if (i0 + i < NN) acc[i] = cD;
#pragma unroll
                    for (int p = DC - 1; p >= 0; --p) {
                        const T cp = c[p];
#pragma unroll
                        for (int i = 0; i < CH; ++i)
                            if (i0 + i < NN) acc[i] = fma_t(acc[i], phi[node(i0 + i)], cp);
                    }
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        if (i0 + i < NN) v[j][node(i0 + i)] = fma_t(omw, v[j][node(i0 + i)], acc[i]);
                }
            } else {
#pragma unroll
                for (int i0 = 0; i0 < NN; i0 += CH) {
                    T acc[CH];
                    const T cD = c[D];
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        if (i0 + i < NN) acc[i] = cD;
                    for (int p = D - 1; p >= 0; --p) {
                        const T cp = c[p];
#pragma unroll
                        for (int i = 0; i < CH; ++i)
                            if (i0 + i < NN) acc[i] = fma_t(acc[i], phi[node(i0 + i)], cp);
                    }
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        if (i0 + i < NN) v[j][node(i0 + i)] = fma_t(omw, v[j][node(i0 + i)], acc[i]);
                }
            }
        }
    }
}

// CTA budget of k_ring: FP32 D1Q5 with 16 nodes a thread holds 512 threads an SM (128
// registers); a smaller CTA asks for the registers of 512 / MAXT CTAs per SM.
__host__ __device__ constexpr int ring_minb(int MAXT) { return 512 / MAXT > 1 ? 512 / MAXT : 1; }

// Shared memory of a k_ring launch: the exchange buffers R and L and the wrap-around tails (two
// step parities each, row stride MAXT, the CTA size of the plan's class; an instance's tail sits
// in the column of its first thread) and the coefficient rows.  Compile-time strides keep every
// exchange address an immediate offset from one per-thread base.
constexpr int kRingMaxInst = 32;  // instances per CTA (the packer's limit)
__host__ __device__ constexpr int ring_xchg_elems(int B, int MAXT) { return 6 * nedge(B) * MAXT; }

template <typename T, int B, int K, int MAXT, int DC>
__global__ void __launch_bounds__(MAXT, ring_minb(MAXT))
    k_ring(const T *__restrict__ st_in, T *__restrict__ st_out, const OnchipInst *__restrict__ insts,
           const int *__restrict__ cta_first, const T *__restrict__ coefs, int nsteps) {
    constexpr int W = wmax(B);
    constexpr int NE = nedge(B);
    constexpr int PS = NE * MAXT;          // one parity of R, L or the tails
    constexpr int RCH = 8;                 // Horner chunk (12 and 16 were slower on GB300; no spills)
    static_assert(K >= 2 * W + 1, "a thread must own interior nodes");
    static_assert(std::is_same<T, float>::value, "the 16-node kernel is FP32 (packed pairs)");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *R = reinterpret_cast<T *>(smem_raw);                   // [2][NE][MAXT]
    T *L = R + 2 * PS;                                        // [2][NE][MAXT]
    T *tail = L + 2 * PS;                                     // [2][NE][MAXT]
    T *scoef = tail + 2 * PS;

    const int nt = blockDim.x;  // <= MAXT
    const int first = cta_first[blockIdx.x], last = cta_first[blockIdx.x + 1];
    const int tid = threadIdx.x;
    for (int i = first; i < last; ++i) {
        const OnchipInst I = insts[i];
        const int Dk = DC > 0 ? DC : I.D;
        const int cs = crow(Dk), n = (B - 1) * (I.D + 1);
        for (int q = tid; q < (B - 1) * cs; q += nt) {
            const int j = q / cs, pp = q % cs;
            scoef[I.scoef + q] = pp <= I.D ? coefs[I.gcoef + j * (I.D + 1) + pp] : T(0);
        }
        if (tid == 0) scoef[I.scoef + (B - 1) * cs] = coefs[I.gcoef + 2 * n];
    }
    int me = -1;
    for (int i = first; i < last; ++i) {
        const int tb = insts[i].tbase;
        if (tid >= tb && tid < tb + insts[i].nthr) me = i;
    }
    OnchipInst I{};
    if (me >= 0) I = insts[me];
    const int t = tid - I.tbase;
    const bool has = me >= 0;
    const int N = I.N;
    const int xb = t * K;
    const bool near_end = has && (t + 1) * K + W > N;  // threads nthr-2, nthr-1 at most

    constexpr int VW = 16 / (int)sizeof(T);
    auto vec_ok = [&](const T *base) {
        return K % VW == 0 && xb + K <= N && ((uintptr_t)(base + xb) & 15) == 0 &&
               ((I.ld * (long long)sizeof(T)) & 15) == 0;
    };
    T phi[K], v[B][K];
    if (has && vec_ok(st_in + I.off)) {
        const T *src = st_in + I.off + xb;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            T *dst = j == 0 ? phi : v[j];
#pragma unroll
            for (int q = 0; q < K / VW; ++q) {
                if constexpr (sizeof(T) == 4) {
                    const float4 w = reinterpret_cast<const float4 *>(src + (long long)j * I.ld)[q];
                    dst[4 * q] = w.x;
                    dst[4 * q + 1] = w.y;
                    dst[4 * q + 2] = w.z;
                    dst[4 * q + 3] = w.w;
                } else {
                    const double2 w = reinterpret_cast<const double2 *>(src + (long long)j * I.ld)[q];
                    dst[2 * q] = w.x;
                    dst[2 * q + 1] = w.y;
                }
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int x = xb + k;
            const bool ok = has && x < N;
            phi[k] = ok ? st_in[I.off + x] : T(0);
#pragma unroll
            for (int j = 1; j < B; ++j) v[j][k] = ok ? st_in[I.off + (long long)j * I.ld + x] : T(0);
        }
    }
    __syncthreads();  // coefficients staged
    const T *sc = scoef + I.scoef;
    const int D = DC > 0 ? DC : I.D;
    const int cs = crow(D);
    const T omw = has ? sc[(B - 1) * cs] : T(0);
    const int steps = has ? I.steps : 0;
    // per-thread exchange bases: this thread's slot column, the column its left-moving pulls read
    // (the next thread's, or its own for the instance's last thread, whose reads there are all
    // replaced by head slots), the instance's head column and its tail column
    T *const Rme = R + tid;
    T *const Lme = L + tid;
    const T *const Lrt = L + ((t + 1 >= I.nthr) ? tid : tid + 1);
    const T *const Lhd = L + I.tbase;
    T *const Thd = tail + I.tbase;  // the instance's tail column
    // right-moving pulls: the previous thread's slots, or the tail for the instance's first thread
    const T *const Rsrc = t > 0 ? Rme - 1 : tail + tid;
    const int rem = N - xb;  // positions k >= rem lie past node N-1 (near-end threads only)

    // one step with the parity of its exchange buffers known at compile time
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
            if (near_end) {
                // tail slot i of a right-moving population holds node N - e + i, at the position
                // k = rem - e + i of this thread: one compile-time case of rem (1 .. K + W - 1)
                auto tput = [&](auto rc) {
                    constexpr int R = decltype(rc)::value;
#pragma unroll
                    for (int j = 1; j < B; ++j) {
                        const int e = vel(j);
                        if (e > 0) {
#pragma unroll
                            for (int i = 0; i < e; ++i)
                                if (R - e + i >= 0 && R - e + i < K)
                                    Thd[P * PS + (eslot(e) + i) * MAXT] = v[j][R - e + i];
                        }
                    }
                };
                static_assert(K + W - 1 <= 18, "tail cases");
                switch (rem) {
#define LBK_RING_TAIL(R)                        \
    case R:                                     \
        tput(std::integral_constant<int, R>{}); \
        break;
                    LBK_RING_TAIL(1) LBK_RING_TAIL(2) LBK_RING_TAIL(3) LBK_RING_TAIL(4) LBK_RING_TAIL(5)
                    LBK_RING_TAIL(6) LBK_RING_TAIL(7) LBK_RING_TAIL(8) LBK_RING_TAIL(9) LBK_RING_TAIL(10)
                    LBK_RING_TAIL(11) LBK_RING_TAIL(12) LBK_RING_TAIL(13) LBK_RING_TAIL(14) LBK_RING_TAIL(15)
                    LBK_RING_TAIL(16) LBK_RING_TAIL(17) LBK_RING_TAIL(18)
#undef LBK_RING_TAIL
                    default:
                        break;
                }
            }
        }
        __syncthreads();
        if (live) {
            // sources in this thread's registers first, then the neighbours'.  Every left-moving
            // source past node N-1 is a head slot (thread 0's published first values): in the
            // last thread the registers of the first positions past node N-1 (padding, never
            // written back) take the head values first, and in the last two threads a neighbour
            // read past node N-1 takes the head address.  The remainder rem picks one
            // compile-time case, so the registers are named, not indexed; positions further out
            // are read only by padding.
            // the flux differences of a node add up apart from phi (they are of the size of the
            // deviations, O(phi / c)), and phi takes their sum once: one rounding of phi a step.
            // The sums start at -0, the identity of IEEE addition, so the first add folds away.
            T d[K];
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = T(-0.0);
            if (near_end && rem < K) {
                auto put = [&](auto rc) {
                    constexpr int R = decltype(rc)::value;
#pragma unroll
                    for (int j = 1; j < B; ++j) {
                        const int a = -vel(j);
#pragma unroll
                        for (int i = 0; i < a; ++i)
                            if (R + i < K) v[j][R + i] = Lhd[P * PS + (eslot(a) + i) * MAXT];
                    }
                };
                static_assert(K <= 16, "remainder cases");
                switch (rem) {
#define LBK_RING_REM(R)                        \
    case R:                                    \
        put(std::integral_constant<int, R>{}); \
        break;
                    LBK_RING_REM(1) LBK_RING_REM(2) LBK_RING_REM(3) LBK_RING_REM(4) LBK_RING_REM(5)
                    LBK_RING_REM(6) LBK_RING_REM(7) LBK_RING_REM(8) LBK_RING_REM(9) LBK_RING_REM(10)
                    LBK_RING_REM(11) LBK_RING_REM(12) LBK_RING_REM(13) LBK_RING_REM(14) LBK_RING_REM(15)
#undef LBK_RING_REM
                    default:
                        break;
                }
            }
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const int e = vel(j);
                if (e == 2 && K % 2 == 0) {
                    // |e| = 2: a pair of nodes (k, k + 1) pulls from the pair (k - 2, k - 1), so
                    // the difference and its sum into d take one packed operation each (a
                    // multiply-add by -1 rounds as the subtraction; each half as one operation)
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
                        const T nv = Rsrc[P * PS + (eslot(e) + k) * MAXT];
                        d[k] += nv - v[j][k];
                        v[j][k] = nv;
                    }
                } else if (near_end) {
                    // near-end threads only (a branch, not a select in every thread)
                    const int a = -e;
#pragma unroll
                    for (int k = K - a; k < K; ++k) {
                        // head slot q = k + a - rem in [0, a - 1] (clamped both ways, so the
                        // address not taken stays in bounds too)
                        int q = k + a - rem;
                        q = q < 0 ? 0 : (q < a - 1 ? q : a - 1);
                        const T *src = k + a >= rem ? Lhd + P * PS + (eslot(a) + q) * MAXT
                                                    : Lrt + P * PS + (eslot(a) + k + a - K) * MAXT;
                        const T nv = *src;
                        d[k] += nv - v[j][k];
                        v[j][k] = nv;
                    }
                } else {
                    // the other threads (rem >= K + W): every source is the next thread's
                    const int a = -e;
#pragma unroll
                    for (int k = K - a; k < K; ++k) {
                        const T nv = Lrt[P * PS + (eslot(a) + k + a - K) * MAXT];
                        d[k] += nv - v[j][k];
                        v[j][k] = nv;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < K; k += 2) {  // phi takes the sums once, two nodes per packed add
                const float2 p2 = __fadd2_rn(make_float2(phi[k], phi[k + 1]), make_float2(d[k], d[k + 1]));
                phi[k] = p2.x;
                phi[k + 1] = p2.y;
            }
            ring_relax<T, B, K, DC, RCH, 0, K>(sc, cs, D, omw, phi, v);
        }
    };
    // two steps per iteration, one of each parity
    for (int s = 0; s < nsteps; s += 2) {
        step(std::integral_constant<int, 0>{}, s);
        if (s + 1 < nsteps) step(std::integral_constant<int, 1>{}, s + 1);
    }
    // the placement again (not kept in registers through the steps)
    if (has) I = insts[me];
    if (has && vec_ok(st_out + I.off2)) {
        T *dst = st_out + I.off2 + xb;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const T *src = j == 0 ? phi : v[j];
#pragma unroll
            for (int q = 0; q < K / VW; ++q) {
                if constexpr (sizeof(T) == 4)
                    reinterpret_cast<float4 *>(dst + (long long)j * I.ld)[q] =
                        make_float4(src[4 * q], src[4 * q + 1], src[4 * q + 2], src[4 * q + 3]);
                else
                    reinterpret_cast<double2 *>(dst + (long long)j * I.ld)[q] = make_double2(src[2 * q], src[2 * q + 1]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int x = xb + k;
            if (has && x < N) {
                st_out[I.off2 + x] = phi[k];
#pragma unroll
                for (int j = 1; j < B; ++j) st_out[I.off2 + (long long)j * I.ld + x] = v[j][k];
            }
        }
    }
}

}  // namespace lbk
