// CUDA kernels of the collide-and-stream hot path (Eq. (LBE)) for sm_103a.
//
// State of one instance in HBM (structure of arrays, rows of stride ld):
//   row 0      phi(x)
//   row j>=1   s_j(x) = f*_j(x), the post-collision population of velocity e_j,
//              e = {_, 1, -1, 2, -2, 3, -3} (Sec. III A/B).
// The rest population is not stored: collision keeps sum_j f*_j = phi (first relation of
// Eq. (moments)), so f*_0 = phi - sum_{j>=1} s_j.  In FP32 this makes every stored
// population a deviation from the rest equilibrium (phi, 0, ..., 0), whose magnitude is
// O(phi / c): the "deviation storage" of the FP32 path.
//
// One time step at node x (pull form of Eq. (LBE)):
//   f_j(x)   = s_j(x - e_j)                       stream                 (a2)
//   phi'(x)  = phi(x) + sum_{j>=1} [f_j(x) - s_j(x)]                      (a3)
//   s'_j(x)  = (1 - omega) f_j(x) + P_j(phi'(x))  relax, P_j = omega f^eq_j (a4, a5)
// where f^eq_j is the polynomial of Eqs. (EDF5)/(EDF7) built on the host.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbk {

constexpr int kMaxDeg = 31;
constexpr int kMaxRow = 64;  // longest coefficient row (real-exponent models: (A + 1)(Dg + 1))

// compile-time flag passed to generic lambdas
template <bool V> struct BoolC { static constexpr bool value = V; };

// e_j for j = 0..6: {0, 1, -1, 2, -2, 3, -3}
__host__ __device__ constexpr int vel(int j) { return j == 0 ? 0 : ((j & 1) ? (j + 1) / 2 : -(j / 2)); }
// Largest |e_j| of the lattice
__host__ __device__ constexpr int wmax(int B) { return (B - 1) / 2; }
// Number of edge values a thread publishes for the populations moving one way:
// 1 + 2 (+ 3) = 3 on D1Q5, 6 on D1Q7.
__host__ __device__ constexpr int nedge(int B) { return wmax(B) * (wmax(B) + 1) / 2; }
// First edge slot of the population with |e| = a (a = 1, 2, 3): 0, 1, 3.
__host__ __device__ constexpr int eslot(int a) { return (a - 1) * a / 2; }

// Shared-memory coefficient rows of the on-chip kernel: P_j for j = 1..B-1 at stride
// crow(D) (a multiple of 4, so rows start on 16-byte boundaries), then 1 - omega.
__host__ __device__ constexpr int crow(int D) { return (D + 1 + 3) & ~3; }
__host__ __device__ constexpr int cblock(int B, int D) { return (B - 1) * crow(D) + 4; }

// One instance's place in the state and coefficient arenas.
struct Seg {
    long long off;  // element offset of row 0 (phi)
    long long ld;   // row stride in elements (multiple of 32)
    int N;          // nodes
    int D;          // degree of the f^eq polynomials (A > 0: row length - 1, (A + 1)(Dg + 1) - 1)
    int coef;       // element offset of the coefficient block:
                    //   [(B-1)(D+1)]  P_j = omega f^eq_j, j = 1..B-1 (row j-1)
                    //   [(B-1)(D+1)]  f^eq_j (unscaled, for initialisation)
                    //   [1]           1 - omega
    int pad;        // bounded grids: extrapolation depth (0: periodic)
    int A, Dg;      // real-exponent models: f^eq_j = sum_{a<=A} (phi^nu)^a sum_{i<=Dg} c[a(Dg+1)+i] phi^i
    double nu;      //   (A = 0: an ordinary polynomial of degree D = Dg)
};

// Load NCR consecutive coefficients from a 16-byte aligned shared-memory row.
template <typename T, int NCR>
__device__ __forceinline__ void load_row(const T *c, T (&cr)[NCR]) {
    if constexpr (sizeof(T) == 4) {
        static_assert(NCR % 4 == 0, "row length");
#pragma unroll
        for (int q = 0; q < NCR / 4; ++q) {
            const float4 w = reinterpret_cast<const float4 *>(c)[q];
            cr[4 * q] = w.x;
            cr[4 * q + 1] = w.y;
            cr[4 * q + 2] = w.z;
            cr[4 * q + 3] = w.w;
        }
    } else {
        static_assert(NCR % 2 == 0, "row length");
#pragma unroll
        for (int q = 0; q < NCR / 2; ++q) {
            const double2 w = reinterpret_cast<const double2 *>(c)[q];
            cr[2 * q] = w.x;
            cr[2 * q + 1] = w.y;
        }
    }
}

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// phi^nu for the real-exponent terms, zero where phi <= 0 (the continuous extension).  FP32 takes
// the fast intrinsic (relative error ~1e-6, far below the FP32 path's discretisation error).
template <typename T>
__device__ __forceinline__ T nu_pow(T phi, double nu) {
    if constexpr (sizeof(T) == 4)
        return phi > 0.0f ? __powf(phi, (float)nu) : 0.0f;
    else
        return phi > 0.0 ? pow(phi, nu) : 0.0;
}

// sum_{a<=A} w^a sum_{i<=Dg} c[a(Dg+1)+i] phi^i: Horner in phi within a row, in w across rows.
template <typename T>
__device__ __forceinline__ T gen_eval(const T *c, int A, int Dg, T phi, T w) {
    T acc = T(0);
    for (int a = A; a >= 0; --a) {
        const T *r = c + a * (Dg + 1);
        T h = r[Dg];
        for (int p = Dg - 1; p >= 0; --p) h = fma_t(h, phi, r[p]);
        acc = a == A ? h : fma_t(acc, w, h);
    }
    return acc;
}

// gen_eval for NN nodes at once (a k_stream group of four, an on-chip thread's K): each
// coefficient is loaded once and feeds NN independent accumulators.  DG: the row degree at
// compile time (the rows unroll); DG < 0: run time.
template <typename T, int DG, int NN, int AA = -1>
__device__ __forceinline__ void gen_evalN(const T *c, int A_, int Dg, const T (&phi)[NN], const T (&w)[NN],
                                          T (&out)[NN]) {
    const int dg = DG >= 0 ? DG : Dg;
    const int A = AA >= 0 ? AA : A_;  // AA >= 0: the row count at compile time (the rows unroll)
    if constexpr (std::is_same<T, float>::value && DG >= 0 && AA >= 0 && NN % 2 == 0) {
        // pairs of nodes through packed multiply-adds (each half rounds as one fmaf)
        float2 o2[NN / 2];
        auto row2 = [&](int a, float2 (&h)[NN / 2]) {
            const T *r = c + a * (DG + 1);
            T cr[DG + 1];
#pragma unroll
            for (int p = 0; p <= DG; ++p) cr[p] = r[p];
#pragma unroll
            for (int n = 0; n < NN / 2; ++n) h[n] = make_float2(cr[DG], cr[DG]);
#pragma unroll
            for (int p = DG - 1; p >= 0; --p)
#pragma unroll
                for (int n = 0; n < NN / 2; ++n)
                    h[n] = __ffma2_rn(h[n], make_float2(phi[2 * n], phi[2 * n + 1]), make_float2(cr[p], cr[p]));
        };
        row2(AA, o2);
#pragma unroll
        for (int a = AA - 1; a >= 0; --a) {
            float2 h[NN / 2];
            row2(a, h);
#pragma unroll
            for (int n = 0; n < NN / 2; ++n) o2[n] = __ffma2_rn(o2[n], make_float2(w[2 * n], w[2 * n + 1]), h[n]);
        }
#pragma unroll
        for (int n = 0; n < NN / 2; ++n) {
            out[2 * n] = o2[n].x;
            out[2 * n + 1] = o2[n].y;
        }
        return;
    }
    auto row = [&](int a, T (&h)[NN]) {  // Q_a(phi) for every node
        const T *r = c + a * (dg + 1);
        if constexpr (DG >= 0) {
            T cr[DG + 1];
#pragma unroll
            for (int p = 0; p <= DG; ++p) cr[p] = r[p];
#pragma unroll
            for (int n = 0; n < NN; ++n) h[n] = cr[DG];
#pragma unroll
            for (int p = DG - 1; p >= 0; --p)
#pragma unroll
                for (int n = 0; n < NN; ++n) h[n] = fma_t(h[n], phi[n], cr[p]);
        } else {
            const T cD = r[dg];
#pragma unroll
            for (int n = 0; n < NN; ++n) h[n] = cD;
            for (int p = dg - 1; p >= 0; --p) {
                const T cp = r[p];
#pragma unroll
                for (int n = 0; n < NN; ++n) h[n] = fma_t(h[n], phi[n], cp);
            }
        }
    };
    row(A, out);  // the top row starts the Horner recursion in w
    if constexpr (AA >= 0) {
#pragma unroll
        for (int a = AA - 1; a >= 0; --a) {
            T h[NN];
            row(a, h);
#pragma unroll
            for (int n = 0; n < NN; ++n) out[n] = fma_t(out[n], w[n], h[n]);
        }
    } else {
#pragma unroll 2
        for (int a = A - 1; a >= 0; --a) {
            T h[NN];
            row(a, h);
#pragma unroll
            for (int n = 0; n < NN; ++n) out[n] = fma_t(out[n], w[n], h[n]);
        }
    }
}

// gen_evalN with the row degree dispatched to a compile-time variant (0..7 in FP32, 0..3 in FP64,
// where more would spill), else run time.
template <typename T, int NN = 4>
__device__ __forceinline__ void gen_eval4_any(const T *c, int A, int Dg, const T (&phi)[NN], const T (&w)[NN],
                                              T (&out)[NN]) {
    if constexpr (sizeof(T) == 8) {
        switch (Dg) {
        case 0: gen_evalN<T, 0, NN>(c, A, Dg, phi, w, out); break;
        case 1: gen_evalN<T, 1, NN>(c, A, Dg, phi, w, out); break;
        case 2: gen_evalN<T, 2, NN>(c, A, Dg, phi, w, out); break;
        case 3: gen_evalN<T, 3, NN>(c, A, Dg, phi, w, out); break;
        default: gen_evalN<T, -1, NN>(c, A, Dg, phi, w, out); break;
        }
    } else {
        switch (Dg) {
        case 0: gen_evalN<T, 0, NN>(c, A, Dg, phi, w, out); break;
        case 1: gen_evalN<T, 1, NN>(c, A, Dg, phi, w, out); break;
        case 2: gen_evalN<T, 2, NN>(c, A, Dg, phi, w, out); break;
        case 3: gen_evalN<T, 3, NN>(c, A, Dg, phi, w, out); break;
        case 4: gen_evalN<T, 4, NN>(c, A, Dg, phi, w, out); break;
        case 5: gen_evalN<T, 5, NN>(c, A, Dg, phi, w, out); break;
        case 6: gen_evalN<T, 6, NN>(c, A, Dg, phi, w, out); break;
        case 7: gen_evalN<T, 7, NN>(c, A, Dg, phi, w, out); break;
        default: gen_evalN<T, -1, NN>(c, A, Dg, phi, w, out); break;
        }
    }
}

// ---------------------------------------------------------------------------- a1: init
// s_j(x) = f^eq_j(phi0(x)) (post-collision state of an equilibrium, collision leaves it
// unchanged), phi(x) = phi0(x).  f^eq is evaluated in the state's type T from the coefficient
// table of that type (FP32 deviation storage: FP32 arithmetic, as every later step; FP64: double).
// Grid: blocks[i] = (segment, first node); each block covers `chunk` nodes; phi0_off[i] is
// the offset of block i's segment in the concatenated phi0 array.
template <typename T, int B>
__global__ void k_init(T *__restrict__ st, const Seg *__restrict__ segs, const int2 *__restrict__ blocks,
                       const T *__restrict__ coef, const double *__restrict__ phi0,
                       const long long *__restrict__ phi0_off, int chunk) {
    const int2 bl = blocks[blockIdx.x];
    const Seg s = segs[bl.x];
    const T *__restrict__ fe = coef + s.coef + (B - 1) * (s.D + 1);
    const double *__restrict__ p0 = phi0 + phi0_off[blockIdx.x];
    const int xend = min(bl.y + chunk, s.N);
    for (int x = bl.y + threadIdx.x; x < xend; x += blockDim.x) {
        const T ph = (T)p0[x];
        st[s.off + x] = ph;
        const T w = s.A > 0 ? nu_pow<T>(ph, s.nu) : T(0);
#pragma unroll
        for (int j = 1; j < B; ++j) {
            const T *c = fe + (j - 1) * (s.D + 1);
            T acc;
            if (s.A > 0) {
                acc = gen_eval<T>(c, s.A, s.Dg, ph, w);
            } else {
                acc = c[s.D];
                for (int p = s.D - 1; p >= 0; --p) acc = fma_t(acc, ph, c[p]);
            }
            st[s.off + (long long)j * s.ld + x] = acc;
        }
    }
}

// ------------------------------------------------------------- a2-a6: streaming step
// One fused collide+stream step through HBM.  A thread owns one group of 4 consecutive nodes
// (16 bytes per row in FP32, 32 in FP64), consecutive lanes own consecutive groups, so every
// row is read and written with coalesced vector accesses.  The shifted sources s_j(x - e_j)
// at a group's edges come from the neighbouring lane by warp shuffle (the lanes at a warp
// edge load the neighbouring group themselves; it is in L1/L2).  Groups within max|e| of
// either end of the grid take a scalar path with periodic indices.
// DC > 0: compile-time polynomial degree (lower-degree segments are zero-padded); the
// coefficients are kernel parameters when the whole launch shares one model (PARAMC), else
// registers loaded per block.  DC == 0: degree read at run time from shared memory.
template <typename T>
__device__ __forceinline__ void load4(const T *p, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 w = *reinterpret_cast<const float4 *>(p);
        v[0] = w.x, v[1] = w.y, v[2] = w.z, v[3] = w.w;
    } else {
        const double2 w0 = reinterpret_cast<const double2 *>(p)[0], w1 = reinterpret_cast<const double2 *>(p)[1];
        v[0] = w0.x, v[1] = w0.y, v[2] = w1.x, v[3] = w1.y;
    }
}
template <typename T>
__device__ __forceinline__ void store4(T *p, const T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
}

// Coefficients of one model passed by value: every thread of the launch reads them as
// uniform constant-bank operands (no registers, no loads).  Used when all segments of a launch
// share one model.
template <typename T, int B, int DC>
struct StreamCoef {
    T c[(B - 1) * (DC + 1)];  // P_j(phi) = omega f^eq_j(phi), row j - 1, degree DC
    T omw;                    // 1 - omega
};

template <typename T, int B, int DC, int NT, bool PARAMC>
__device__ __forceinline__ void stream_body(const T *__restrict__ in, T *__restrict__ out,
                                            const Seg *__restrict__ segs, const int2 *__restrict__ blocks,
                                            const T *__restrict__ coefs,
                                            const StreamCoef<T, B, (DC > 0 ? DC : 1)> &pc) {
    static_assert(!PARAMC || DC > 0, "parameter coefficients need a compile-time degree");
    constexpr int W = wmax(B);
    constexpr int NC = DC > 0 ? DC + 1 : kMaxRow;
    __shared__ T sc[PARAMC ? 1 : (B - 1) * NC + 1];
    const int2 bl = blocks[blockIdx.x];
    const Seg s = segs[bl.x];
    if constexpr (!PARAMC) {
        for (int i = threadIdx.x; i < (B - 1) * NC; i += blockDim.x) {
            const int j = i / NC, p = i % NC;
            sc[i] = p <= s.D ? coefs[s.coef + j * (s.D + 1) + p] : T(0);
        }
        if (threadIdx.x == 0) sc[(B - 1) * NC] = coefs[s.coef + 2 * (B - 1) * (s.D + 1)];
        __syncthreads();
    }
    const int D = DC > 0 ? DC : s.D;
    const T omw = PARAMC ? pc.omw : sc[PARAMC ? 0 : (B - 1) * NC];
    T creg[(DC > 0 && !PARAMC) ? (B - 1) * (DC + 1) : 1];
    if constexpr (DC > 0 && !PARAMC) {
#pragma unroll
        for (int j = 0; j < B - 1; ++j)
#pragma unroll
            for (int p = 0; p <= DC; ++p) creg[j * (DC + 1) + p] = sc[j * NC + p];
    }
    auto coef = [&](int j, int p) -> T {  // coefficient p of P_j, compile-time indices
        if constexpr (PARAMC)
            return pc.c[(j - 1) * (DC + 1) + p];
        else if constexpr (DC > 0)
            return creg[(j - 1) * (DC + 1) + p];
        else
            return T(0);  // run-time degree: the coefficients come from shared memory instead
    };
    // real-exponent models (run-time degree path only): w = phi^nu once per node
    const int A = DC > 0 ? 0 : s.A;
    auto wpow = [&](T ph) -> T {
        if constexpr (DC > 0)
            return T(0);
        else
            return A > 0 ? nu_pow<T>(ph, s.nu) : T(0);
    };
    auto poly = [&](int j, T ph, T w) -> T {  // P_j(phi), Horner
        T acc;
        if constexpr (DC > 0) {
            acc = coef(j, DC);
#pragma unroll
            for (int p = DC - 1; p >= 0; --p) acc = fma_t(acc, ph, coef(j, p));
        } else {
            const T *c = sc + (j - 1) * NC;
            if (A > 0) return gen_eval<T>(c, A, s.Dg, ph, w);
            acc = c[D];
            for (int p = D - 1; p >= 0; --p) acc = fma_t(acc, ph, c[p]);
        }
        return acc;
    };
    const T *__restrict__ src = in + s.off;
    T *__restrict__ dst = out + s.off;
    const long long ld = s.ld;
    const int N = s.N;
    const int lane = threadIdx.x & 31;
    const int x = bl.y + (int)threadIdx.x * 4;  // first node of this thread's group
    const bool active = x < N;
    const int xa = active ? x : 0;  // an in-bounds address for lanes past the end
    T a[B][4];
    T ed[B][W];  // edge sources: the last e nodes of the previous group (e > 0) or the first
                 // |e| nodes of the next group (e < 0)
#pragma unroll
    for (int j = 0; j < B; ++j) load4(src + j * ld + xa, a[j]);
#pragma unroll
    for (int j = 1; j < B; ++j) {
        const int e = vel(j);
        if (e > 0) {
#pragma unroll
            for (int i = 0; i < e; ++i) ed[j][i] = __shfl_up_sync(0xffffffffu, a[j][4 - e + i], 1);
            if (lane == 0 && xa >= 4)
#pragma unroll
                for (int i = 0; i < e; ++i) ed[j][i] = src[j * ld + xa - e + i];
        } else {
#pragma unroll
            for (int i = 0; i < -e; ++i) ed[j][i] = __shfl_down_sync(0xffffffffu, a[j][i], 1);
            if (lane == 31 && xa + 4 - e <= N)
#pragma unroll
                for (int i = 0; i < -e; ++i) ed[j][i] = src[j * ld + xa + 4 + i];
        }
    }
    if (!active) return;
    if (DC == 0 && A > 0 && x >= W && x + 4 + W <= N) {
        // real-exponent model: pull and phi' for the whole group first, then every P_j for the
        // four nodes together
        T o[B][4], w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T d = T(0);
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const int e = vel(j);
                const int q = i - e;
                const T sj = q < 0 ? ed[j][e + q] : (q >= 4 ? ed[j][q - 4] : a[j][q]);
                d += sj - a[j][i];
                o[j][i] = sj;
            }
            o[0][i] = a[0][i] + d;
            w[i] = wpow(o[0][i]);
        }
#pragma unroll
        for (int j = 1; j < B; ++j) {
            T acc[4];
            gen_eval4_any<T>(sc + (j - 1) * NC, A, s.Dg, o[0], w, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[j][i] = fma_t(omw, o[j][i], acc[i]);
        }
#pragma unroll
        for (int j = 0; j < B; ++j) store4(dst + j * ld + x, o[j]);
    } else if (x >= W && x + 4 + W <= N) {
        T o[B][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T f[B];
            T d = T(0);
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const int e = vel(j);
                const int q = i - e;  // source index within the group
                const T sj = q < 0 ? ed[j][e + q] : (q >= 4 ? ed[j][q - 4] : a[j][q]);
                d += sj - a[j][i];
                f[j] = sj;
            }
            const T ph = a[0][i] + d;
            o[0][i] = ph;
            const T w = wpow(ph);
#pragma unroll
            for (int j = 1; j < B; ++j) o[j][i] = fma_t(omw, f[j], poly(j, ph, w));
        }
#pragma unroll
        for (int j = 0; j < B; ++j) store4(dst + j * ld + x, o[j]);
    } else {
        // within max|e| of a grid end: periodic indices, scalar accesses
        for (int i = 0; i < 4 && x + i < N; ++i) {
            const int xi = x + i;
            T f[B];
            T d = T(0);
#pragma unroll
            for (int j = 1; j < B; ++j) {
                int xs = xi - vel(j);
                xs += xs < 0 ? N : 0;
                xs -= xs >= N ? N : 0;
                const T sj = src[j * ld + xs];
                d += sj - src[j * ld + xi];
                f[j] = sj;
            }
            const T ph = src[xi] + d;
            dst[xi] = ph;
            const T w = wpow(ph);
#pragma unroll
            for (int j = 1; j < B; ++j) dst[j * ld + xi] = fma_t(omw, f[j], poly(j, ph, w));
        }
    }
}

template <typename T, int B, int DC, int NT, bool PARAMC>
__global__ void __launch_bounds__(NT) k_stream(const T *__restrict__ in, T *__restrict__ out,
                                               const Seg *__restrict__ segs, const int2 *__restrict__ blocks,
                                               const T *__restrict__ coefs,
                                               const __grid_constant__ StreamCoef<T, B, (DC > 0 ? DC : 1)> pc) {
    stream_body<T, B, DC, NT, PARAMC>(in, out, segs, blocks, coefs, pc);
}

// The run-time-degree variant (high degrees and real exponents): its general evaluation needs
// more registers than the compile-time variants, so it may take up to 255 (no spills), except
// FP32 D1Q5, which fits 64 and so keeps four CTAs per SM for more loads in flight.
template <typename T, int B, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && B == 5) ? 4 : 1) k_stream_rt(const T *__restrict__ in, T *__restrict__ out,
                                                     const Seg *__restrict__ segs, const int2 *__restrict__ blocks,
                                                     const T *__restrict__ coefs) {
    const StreamCoef<T, B, 1> unused{};
    stream_body<T, B, 0, NT, false>(in, out, segs, blocks, coefs, unused);
}

// ------------------------------------------------------ a2-a6: on-chip, many steps
// A run of a CTA's threads holds a window of one instance in registers for many steps.
// Thread t of the run owns window positions tK .. tK+K-1 (the last thread may own fewer).
// Each step the populations that cross a thread boundary are exchanged through
// double-buffered shared memory (one __syncthreads per step):
//   R: the last |e| values of every right-moving population (read by thread t+1),
//   L: the first |e| values of every left-moving population (read by thread t-1).
// Two modes:
//   ring (HALO = false): the window is the whole periodic instance and stays resident for
//     all nsteps; the wrap-around uses
//       tail: the last |e| nodes of the instance (read by thread 0),
//       head = thread 0's L window (read by the threads at the end of the instance: a
//             left-moving source past node N-1 is replaced by its head slot, a run-time
//             select taken only in the warps that hold such a thread).
//     Several instances may share a CTA (warp-aligned thread runs).
//   halo (HALO = true): temporal blocking.  The window is npos = valid + 2H consecutive
//     nodes (global index taken modulo N) with H = nsteps * max|e|; the window edges read
//     stale values, whose influence moves inward max|e| nodes per step and stays inside the
//     H-wide borders.  After nsteps steps the middle `valid` nodes are exact and are written
//     to the output buffer.  One window per CTA.
struct OnchipInst {
    long long off, ld;  // state placement (as Seg) in st_in
    long long off2;     // placement of the result in st_out
    int N, D;
    int gcoef;          // coefficient block in global memory (as Seg::coef)
    int scoef;          // this instance's copy of P_j and 1 - omega in shared memory
    int tbase;          // first CTA thread
    int nthr;           // threads that own positions: ceil(npos / K)
    int il;             // index among the CTA's instances (tail buffer slot)
    int x0;             // global node of window position 0 (halo: may be negative)
    int npos;           // window positions (ring: N)
    int vlo, vhi;       // positions written back: [vlo, vhi)
    int steps;          // steps this instance takes in the launch (<= nsteps; the state is
                        // frozen after them while the CTA's barriers continue)
    int A, Dg;          // real-exponent models (run-time degree variant only): P_j =
    double nu;          //   sum_{a<=A} (phi^nu)^a sum_{i<=Dg} c[a(Dg+1)+i] phi^i; A = 0: polynomial
};

// gen_eval for the K nodes of a thread, every coefficient loaded once for all K
template <typename T, int K>
__device__ __forceinline__ void gen_evalK(const T *c, int A, int Dg, const T (&phi)[K], const T (&w)[K], T (&out)[K]) {
    gen_eval4_any<T, K>(c, A, Dg, phi, w, out);
}

// The relaxation of every moving population of a thread's K nodes for a real-exponent model
// whose row count (AA + 1) and row degree DG are known at compile time: one dispatch per step
// instead of one per population.  Rows of P_j start at sc + (j - 1) cs.
template <typename T, int B, int K, int AA, int DG>
__device__ __forceinline__ void relax_rows(const T *sc, int cs, const T (&phi)[K], const T (&w)[K], T (&v)[B][K],
                                           T omw) {
#pragma unroll
    for (int j = 1; j < B; ++j) {
        T acc[K];
        gen_evalN<T, DG, K, AA>(sc + (j - 1) * cs, AA, DG, phi, w, acc);
#pragma unroll
        for (int k = 0; k < K; ++k) v[j][k] = fma_t(omw, v[j][k], acc[k]);
    }
}
template <typename T, int B, int K, int AA>
__device__ __forceinline__ bool relax_rows_dg(int Dg, const T *sc, int cs, const T (&phi)[K], const T (&w)[K],
                                              T (&v)[B][K], T omw) {
    switch (Dg) {
    case 0: relax_rows<T, B, K, AA, 0>(sc, cs, phi, w, v, omw); return true;
    case 1: relax_rows<T, B, K, AA, 1>(sc, cs, phi, w, v, omw); return true;
    case 2: relax_rows<T, B, K, AA, 2>(sc, cs, phi, w, v, omw); return true;
    case 3: relax_rows<T, B, K, AA, 3>(sc, cs, phi, w, v, omw); return true;
    default: return false;
    }
}
// the common shapes (2..5 rows, degree 0..3); false for the others
template <typename T, int B, int K>
__device__ __forceinline__ bool relax_rows_fixed(int A, int Dg, const T *sc, int cs, const T (&phi)[K],
                                                 const T (&w)[K], T (&v)[B][K], T omw) {
    switch (A) {
    case 1: return relax_rows_dg<T, B, K, 1>(Dg, sc, cs, phi, w, v, omw);
    case 2: return relax_rows_dg<T, B, K, 2>(Dg, sc, cs, phi, w, v, omw);
    case 3: return relax_rows_dg<T, B, K, 3>(Dg, sc, cs, phi, w, v, omw);
    case 4: return relax_rows_dg<T, B, K, 4>(Dg, sc, cs, phi, w, v, omw);
    default: return false;
    }
}

// threads per SM at each configuration's register budget (FP32 D1Q5 with K = 8: 128 registers);
// a CTA smaller than that asks for the registers of budget / MAXT CTAs per SM
__host__ __device__ constexpr int onchip_budget(int esz, int B, int K) {
    return esz == 4 ? (B == 5 ? (K == 8 ? 512 : 1024) : (K == 8 ? 256 : 512)) : (B == 5 ? (K == 4 ? 512 : 1024) : 256);
}
__host__ __device__ constexpr int onchip_minb(int esz, int B, int K, int MAXT) {
    return onchip_budget(esz, B, K) / MAXT > 1 ? onchip_budget(esz, B, K) / MAXT : 1;
}

// DC: the f^eq degree at compile time; 0: run time; -1: run time with real-exponent terms
// (P_j evaluated in phi and w = phi^nu for the instances with A > 0).
template <typename T, int B, int K, int MAXT, bool HALO, int DC>
__global__ void __launch_bounds__(MAXT, onchip_minb(sizeof(T), B, K, MAXT))
    k_onchip(const T *__restrict__ st_in, T *__restrict__ st_out, const OnchipInst *__restrict__ insts,
             const int *__restrict__ cta_first, const T *__restrict__ coefs, int nsteps, int max_inst) {
    static_assert(K >= wmax(B), "a thread must own at least max|e| nodes");
    constexpr int NE = nedge(B);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int nt = blockDim.x;
    T *R = smem;                        // [2][NE][nt]
    T *L = R + 2 * NE * nt;             // [2][NE][nt]
    T *tail = L + 2 * NE * nt;          // [2][NE][max_inst]                (ring; max_inst % 4 == 0)
    T *scoef = HALO ? tail : tail + 2 * NE * max_inst;

    const int first = cta_first[blockIdx.x], last = cta_first[blockIdx.x + 1];
    const int tid = threadIdx.x;
    // stage every instance's coefficients into shared memory: P_j rows at stride crow(Dk)
    // (zero-padded up to the compile-time degree DC when DC > 0), then 1 - omega
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
    // which instance does this thread serve?
    int me = -1;
    for (int i = first; i < last; ++i) {
        const int tb = insts[i].tbase;
        if (tid >= tb && tid < tb + ((insts[i].nthr + 31) & ~31)) me = i;
    }
    OnchipInst I{};
    if (me >= 0) I = insts[me];
    const int t = tid - I.tbase;
    const bool has = me >= 0 && t < I.nthr;
    const int N = I.N;
    const int npos = I.npos;
    const bool near_end = !HALO && has && (t + 1) * K + wmax(B) > N;  // ring: threads nthr-2, nthr-1
    const int xb = t * K;
    // ring: the warps that hold a near-end thread take the gather with the wrap-around select
    const bool wrap_warp = !HALO && __any_sync(0xffffffffu, near_end);
    // the outermost threads have no neighbour on that side (halo: window edge; ring: the
    // last thread, whose reads past node N-1 are replaced by the head); they read their own
    // edge slot (in bounds, stale) instead
    const int left_nb = (HALO && t == 0) ? tid : tid - 1;
    const int right_nb = (t + 1 >= I.nthr) ? tid : tid + 1;

    // global node of window position p (halo: taken modulo N)
    auto gnode = [&](int p) -> long long {
        long long x = p;
        if (HALO) {
            x = (long long)I.x0 + p;
            x %= N;
            x += x < 0 ? N : 0;
        }
        return x;
    };
    // a thread whose K positions are consecutive global nodes on 16-byte boundaries moves
    // them with vector loads and stores (VW elements each)
    constexpr int VW = 16 / (int)sizeof(T);
    auto vec_ok = [&](const T *base, long long x) {
        return K % VW == 0 && x + K <= N && ((uintptr_t)(base + x) & 15) == 0 && ((I.ld * (long long)sizeof(T)) & 15) == 0;
    };
    T phi[K], v[B][K];
    const long long xv = has ? gnode(xb) : 0;
    if (has && xb + K <= npos && vec_ok(st_in + I.off, xv)) {
        const T *src = st_in + I.off + xv;
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
            const int p = xb + k;
            const bool ok = has && p < npos;
            const long long x = gnode(p);
            phi[k] = ok ? st_in[I.off + x] : T(0);
#pragma unroll
            for (int j = 1; j < B; ++j) v[j][k] = ok ? st_in[I.off + (long long)j * I.ld + x] : T(0);
        }
    }
    __syncthreads();
    const T *sc = scoef + I.scoef;
    const int D = DC > 0 ? DC : I.D;
    const int cs = crow(D);
    const T omw = has ? sc[(B - 1) * cs] : T(0);

    for (int s = 0; s < nsteps; ++s) {
        T *Rb = R + (s & 1) * NE * nt;
        T *Lb = L + (s & 1) * NE * nt;
        T *Tb = tail + (s & 1) * NE * max_inst;
        const bool live = has && s < I.steps;
        if (live) {
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const int e = vel(j);
                if (e > 0) {
#pragma unroll
                    for (int i = 0; i < e; ++i) Rb[(eslot(e) + i) * nt + tid] = v[j][K - e + i];
                } else {
#pragma unroll
                    for (int i = 0; i < -e; ++i) Lb[(eslot(-e) + i) * nt + tid] = v[j][i];
                }
            }
            if (!HALO && near_end) {  // near_end implies has
#pragma unroll
                for (int j = 1; j < B; ++j) {
                    const int e = vel(j);
                    if (e > 0) {
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const int x = xb + k;
                            if (x >= N - e && x < N) Tb[(eslot(e) + x - (N - e)) * max_inst + I.il] = v[j][k];
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (live) {
            T d[K];
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = T(0);
            // f_j(x) = s_j(x - e_j) from own registers or a neighbour's published edge
            // (ring: thread 0 takes its right-moving inflow from the tail buffer, and a
            // left-moving source past node N-1 wraps to thread 0's head window)
            auto pull = [&](auto wrapc) {
                constexpr bool WRAP = decltype(wrapc)::value;
#pragma unroll
                for (int j = 1; j < B; ++j) {
                    const int e = vel(j);
                    if (e > 0) {
#pragma unroll
                        for (int k = K - 1; k >= 0; --k) {  // descending: v[j][k - e] still old
                            T nv;
                            if (k >= e) {
                                nv = v[j][k - e];
                            } else if (HALO) {
                                nv = Rb[(eslot(e) + k) * nt + left_nb];
                            } else {
                                const T *p = t > 0 ? &Rb[(eslot(e) + k) * nt + tid - 1]
                                                   : &Tb[(eslot(e) + k) * max_inst + I.il];
                                nv = *p;
                            }
                            d[k] += nv - v[j][k];
                            v[j][k] = nv;
                        }
                    } else {
                        const int a = -e;
#pragma unroll
                        for (int k = 0; k < K; ++k) {  // ascending: v[j][k + a] still old
                            T nv = (k + a < K) ? v[j][k + a] : Lb[(eslot(a) + k + a - K) * nt + right_nb];
                            if constexpr (WRAP) {
                                // positions past N-1 (last thread's padding) clamp to the
                                // last head slot: in bounds, never written back
                                const int src = xb + k + a;
                                if (src >= N) nv = Lb[(eslot(a) + min(src - N, a - 1)) * nt + I.tbase];
                            }
                            d[k] += nv - v[j][k];
                            v[j][k] = nv;
                        }
                    }
                }
            };
            if (wrap_warp)
                pull(BoolC<true>{});
            else
                pull(BoolC<false>{});
#pragma unroll
            for (int k = 0; k < K; ++k) phi[k] += d[k];
            // relax: s'_j = (1 - omega) f_j + P_j(phi'), Horner with coefficients from shared memory
            // (real exponents: w = phi^nu once per node, then the rows in phi and w)
            T w[K];
            bool relaxed = false;
            if constexpr (DC < 0) {
                if (I.A > 0) {
#pragma unroll
                    for (int k = 0; k < K; ++k) w[k] = nu_pow<T>(phi[k], I.nu);
                    if constexpr (sizeof(T) == 4) relaxed = relax_rows_fixed<T, B, K>(I.A, I.Dg, sc, cs, phi, w, v, omw);
                }
            }
#pragma unroll
            for (int j = 1; j < B && !relaxed; ++j) {
                const T *c = sc + (j - 1) * cs;
                T acc[K];
                if constexpr (DC > 0 && std::is_same<T, float>::value && K % 2 == 0) {
                    // two nodes per packed multiply-add (each half rounds as one fmaf)
                    T cr[crow(DC)];
                    load_row<T, crow(DC)>(c, cr);
                    float2 a2[K / 2];
#pragma unroll
                    for (int k = 0; k < K / 2; ++k) a2[k] = make_float2(cr[DC], cr[DC]);
#pragma unroll
                    for (int p = DC - 1; p >= 0; --p)
#pragma unroll
                        for (int k = 0; k < K / 2; ++k)
                            a2[k] = __ffma2_rn(a2[k], make_float2(phi[2 * k], phi[2 * k + 1]), make_float2(cr[p], cr[p]));
#pragma unroll
                    for (int k = 0; k < K / 2; ++k) {
                        acc[2 * k] = a2[k].x;
                        acc[2 * k + 1] = a2[k].y;
                    }
                } else if constexpr (DC > 0) {
                    T cr[crow(DC)];
                    load_row<T, crow(DC)>(c, cr);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc[k] = cr[DC];
#pragma unroll
                    for (int p = DC - 1; p >= 0; --p)
#pragma unroll
                        for (int k = 0; k < K; ++k) acc[k] = fma_t(acc[k], phi[k], cr[p]);
                } else {
                    auto horner = [&] {
                        const T cD = c[D];
#pragma unroll
                        for (int k = 0; k < K; ++k) acc[k] = cD;
                        for (int p = D - 1; p >= 0; --p) {
                            const T cp = c[p];
#pragma unroll
                            for (int k = 0; k < K; ++k) acc[k] = fma_t(acc[k], phi[k], cp);
                        }
                    };
                    if constexpr (DC < 0) {
                        if (I.A > 0)
                            gen_evalK<T, K>(c, I.A, I.Dg, phi, w, acc);
                        else
                            horner();
                    } else {
                        horner();
                    }
                }
#pragma unroll
                for (int k = 0; k < K; ++k) v[j][k] = fma_t(omw, v[j][k], acc[k]);
            }
        }
    }
    if (has && xb >= I.vlo && xb + K <= I.vhi && vec_ok(st_out + I.off2, xv)) {
        T *dst = st_out + I.off2 + xv;
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
            const int p = xb + k;
            if (has && p >= I.vlo && p < I.vhi) {
                const long long x = gnode(p);
                st_out[I.off2 + x] = phi[k];
#pragma unroll
                for (int j = 1; j < B; ++j) st_out[I.off2 + (long long)j * I.ld + x] = v[j][k];
            }
        }
    }
}

// ------------------------------------------------------------------- a7: readout
// phi (row 0, type T) of every segment into a concatenated double array; any non-finite value
// sets *nonfinite (when given), so the host need not scan the copy.
template <typename T>
__global__ void k_read_phi(const T *__restrict__ st, const Seg *__restrict__ segs, const int2 *__restrict__ blocks,
                           double *__restrict__ out, const long long *__restrict__ out_off, int chunk,
                           int *__restrict__ nonfinite) {
    const int2 bl = blocks[blockIdx.x];
    const Seg s = segs[bl.x];
    const int xend = min(bl.y + chunk, s.N);
    double *o = out + out_off[blockIdx.x];
    bool bad = false;
    for (int x = bl.y + threadIdx.x; x < xend; x += blockDim.x) {
        const double v = (double)st[s.off + x];
        o[x] = v;
        bad |= !isfinite(v);
    }
    if (bad && nonfinite) atomicOr(nonfinite, 1);
}

// ------------------------------------------------------------ a7: diagnostics
// Deterministic two-pass FP64 reduction per segment.  Pass 1 writes one record per block
// into the scratch array `part`; pass 2 (one thread block per segment) sums its blocks'
// records in block order.
struct DiagPart {
    double sum, maxabs, l1d, l1s, l2d, l2s;
    long long nonfinite;
    long long pad;
};

// Error-free sum in float pairs (Knuth's TwoSum): hi + lo carries the running sum of float values
// to about 2^-48 relative, with FP32 operations only (FP64 ones are scarce on this part).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = hi + x, bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// Sum, max|phi| and non-finite count of FP32 phi without a reference solution: float-pair sums
// per thread and across the warp, FP64 only for the warps' partial sums.
static __device__ void diag_block_f32(const float *__restrict__ st, const Seg &s, int x0, int chunk,
                               DiagPart *__restrict__ dst) {
    float hi = 0.f, lo = 0.f, mx = 0.f;
    int nf = 0;
    const int xend = min(x0 + chunk, s.N);
    for (int x = x0 + threadIdx.x; x < xend; x += blockDim.x) {
        const float ph = st[s.off + x];
        if (!isfinite(ph)) {
            ++nf;
            continue;
        }
        two_sum_acc(hi, lo, ph);
        mx = fmaxf(mx, fabsf(ph));
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
        two_sum_acc(hi, lo, h2);
        lo += l2;
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        nf += __shfl_down_sync(0xffffffffu, nf, o);
    }
    __shared__ double rs[32];
    __shared__ float rm[32];
    __shared__ int rn[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        rs[w] = (double)hi + (double)lo;
        rm[w] = mx;
        rn[w] = nf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DiagPart r{};
        float m = 0.f;
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) {
            r.sum += rs[i];
            m = fmaxf(m, rm[i]);
            r.nonfinite += rn[i];
        }
        r.maxabs = m;
        *dst = r;
    }
}

template <typename T>
__device__ void diag_block(const T *__restrict__ st, const Seg &s, int x0, int chunk, const double *__restrict__ ps,
                           DiagPart *__restrict__ dst) {
    if constexpr (sizeof(T) == 4) {
        if (!ps) {
            diag_block_f32(st, s, x0, chunk, dst);
            return;
        }
    }
    double a[6] = {0, 0, 0, 0, 0, 0};
    long long nf = 0;
    const int xend = min(x0 + chunk, s.N);
    for (int x = x0 + threadIdx.x; x < xend; x += blockDim.x) {
        const double ph = (double)st[s.off + x];
        if (!isfinite(ph)) {
            ++nf;
            continue;
        }
        a[0] += ph;
        a[1] = fmax(a[1], fabs(ph));
        if (ps) {
            const double q = ps[x], dd = ph - q;
            a[2] += fabs(dd);
            a[3] += fabs(q);
            a[4] += dd * dd;
            a[5] += q * q;
        }
    }
    __shared__ double red[6][32];
    __shared__ long long rnf[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        double v = a[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_down_sync(0xffffffffu, v, o);
            v = q == 1 ? fmax(v, u) : v + u;
        }
        if (lane == 0) red[q][w] = v;
    }
    for (int o = 16; o > 0; o >>= 1) nf += __shfl_down_sync(0xffffffffu, nf, o);
    if (lane == 0) rnf[w] = nf;
    __syncthreads();
    if (threadIdx.x == 0) {
        DiagPart r{};
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) {
            r.sum += red[0][i];
            r.maxabs = fmax(r.maxabs, red[1][i]);
            r.l1d += red[2][i];
            r.l1s += red[3][i];
            r.l2d += red[4][i];
            r.l2s += red[5][i];
            r.nonfinite += rnf[i];
        }
        *dst = r;
    }
}

template <typename T>
__global__ void k_diag_partial(const T *__restrict__ st, const Seg *__restrict__ segs, const int2 *__restrict__ blocks,
                               const double *__restrict__ phistar, const long long *__restrict__ ps_off, int chunk,
                               DiagPart *__restrict__ part) {
    const int2 bl = blocks[blockIdx.x];
    const Seg s = segs[bl.x];
    diag_block<T>(st, s, bl.y, chunk, phistar ? phistar + ps_off[blockIdx.x] : nullptr, part + blockIdx.x);
}

// part_first[seg] .. part_first[seg + 1]: the pass-1 records of segment seg.
static __global__ void k_diag_final(const DiagPart *__restrict__ part, const int *__restrict__ part_first, int nseg,
                             DiagPart *__restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg) return;
    DiagPart r{};
    for (int i = part_first[g]; i < part_first[g + 1]; ++i) {
        const DiagPart &p = part[i];
        r.sum += p.sum;
        r.maxabs = fmax(r.maxabs, p.maxabs);
        r.l1d += p.l1d;
        r.l1s += p.l1s;
        r.l2d += p.l2d;
        r.l2s += p.l2s;
        r.nonfinite += p.nonfinite;
    }
    out[g] = r;
}

}  // namespace lbk
