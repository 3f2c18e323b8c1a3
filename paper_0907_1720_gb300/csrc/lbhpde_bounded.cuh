// Bounded grids: the non-equilibrium extrapolation boundary that Sec. IV applies to its test
// problems (after Guo et al.; the paper gives no formula).  Each step is the collide+stream of
// Eq. (LBE) on nodes 0..N-1 followed by a rebuild of the W = max|e| outer nodes at each end:
//   f_j(x_b) = f^eq_j(phi_b) + [f_j(x_f) - f^eq_j(phi(x_f))],
// phi_b the prescribed value at x_b and x_f the node `depth` places inside the outer layer
// (x_f = W - 1 + depth on the left, N - W - depth on the right).
//
// In the state of this library (phi and the post-collision populations s_j, j >= 1) the rule
// reads s_j(x_b) = f^eq_j(phi_b) + [s_j(x_f) - f^eq_j(phi(x_f))], phi(x_b) = phi_b: collision
// scales the non-equilibrium part of every node by (1 - omega) and leaves f^eq unchanged, so
// rebuilding after the relaxation equals rebuilding before it.  Interior nodes pull only from
// nodes 0..N-1, so the periodic step of the other kernels is exact for them; the outer nodes'
// pulls (which wrap) are discarded by the rebuild.
#pragma once
#include "lbhpde_kernels.cuh"

namespace lbk {

// One bounded instance resident in one CTA.
struct BoundedInst {
    long long off, ld;  // state placement (as Seg)
    int mi;             // batch member index: its boundary data start at phib + mi * stride
    int N, D;
    int gcoef;          // coefficient block in global memory (as Seg::coef)
    int depth;          // extrapolation depth (>= 1)
    int shift;          // node x sits at position x + shift
    int nthr;           // threads that own positions: ceil((N + shift) / K)
    int pad;
    int A, Dg;          // real-exponent models (variant DC < 0 only): f^eq_j and P_j =
    double nu;          //   sum_{a<=A} (phi^nu)^a sum_{i<=Dg} c[a(Dg+1)+i] phi^i; A = 0: polynomial
};

// Horner evaluation of one 16-byte aligned coefficient row of degree DC (DC > 0) or D (DC == 0).
template <typename T, int DC>
__device__ __forceinline__ T row_eval(const T *c, int D, T x) {
    if constexpr (DC > 0) {
        T cr[crow(DC)];
        load_row<T, crow(DC)>(c, cr);
        T acc = cr[DC];
#pragma unroll
        for (int p = DC - 1; p >= 0; --p) acc = fma_t(acc, x, cr[p]);
        return acc;
    } else {
        T acc = c[D];
        for (int p = D - 1; p >= 0; --p) acc = fma_t(acc, x, c[p]);
        return acc;
    }
}

// f^eq_j or P_j at x: the row of degree DC or D, or (variant DC < 0, instances with A > 0) the
// real-exponent form in x and w = x^nu.
template <typename T, int DC>
__device__ __forceinline__ T feq_eval(const T *c, int D, const BoundedInst &I, T x) {
    if constexpr (DC < 0) {
        if (I.A > 0) return gen_eval<T>(c, I.A, I.Dg, x, nu_pow<T>(x, I.nu));
    }
    return row_eval<T, DC>(c, D, x);
}

// nsteps steps of every bounded instance, one instance per CTA, the state in registers for the
// whole launch.  Node x sits at position x + shift; thread t owns positions tK .. tK+K-1, and
// positions that hold no node stay zero.  The host picks the shift so that each end's outer
// nodes and its extrapolation node x_f fall in one warp.  Per step:
//   1. publish the populations that cross a thread boundary (shared memory R/L, one buffer per
//      step parity), barrier;
//   2. pull, phi' = phi + sum_j (f_j - s_j), relax;
//   3. in the warp of each end: the lane owning x_f computes s_j(x_f) - f^eq_j(phi(x_f)), the
//      warp shares it by shuffle, and the lanes owning outer nodes rebuild them.
// One barrier per step is race free: a buffer written at step s + 2 was last read at step s,
// before every thread passed the barrier of step s + 1.  The launch's boundary data,
// phib[(step0 + s) * 2W + l] for member mi, and their equilibria f^eq_j(phi_b) are evaluated by
// all threads before the first step.  Dynamic shared memory (elements of T):
//   R, L [2][NE][nt] | P, Q [(B-1) cs]: omega f^eq_j and f^eq_j, rows of stride cs = crow(D) |
//   X [16]: 1 - omega | PB [nsteps][2W][B]: phi_b, f^eq_1(phi_b) .. f^eq_{B-1}(phi_b)
template <typename T, int B, int K, int MAXT, int DC>
__global__ void __launch_bounds__(MAXT, 1)
    k_bounded(const T *__restrict__ st_in, T *__restrict__ st_out, const BoundedInst *__restrict__ insts,
              const T *__restrict__ coefs, const double *__restrict__ phib, long long stride, long long step0,
              int nsteps) {
    static_assert(K >= wmax(B), "a thread must own at least max|e| nodes");
    constexpr int W = wmax(B);
    constexpr int NE = nedge(B);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nt = blockDim.x;
    const BoundedInst I = insts[blockIdx.x];
    const int D = DC > 0 ? DC : I.D;
    const int cs = crow(D);
    T *R = reinterpret_cast<T *>(smem_raw);
    T *L = R + 2 * NE * nt;
    T *P = L + 2 * NE * nt;
    T *Q = P + (B - 1) * cs;
    T *X = Q + (B - 1) * cs;
    T *PB = X + 16;

    const int tid = threadIdx.x;
    const int n = (B - 1) * (I.D + 1);
    for (int q = tid; q < (B - 1) * cs; q += nt) {
        const int j = q / cs, pp = q % cs;
        P[q] = pp <= I.D ? coefs[I.gcoef + j * (I.D + 1) + pp] : T(0);
        Q[q] = pp <= I.D ? coefs[I.gcoef + n + j * (I.D + 1) + pp] : T(0);
    }
    if (tid == 0) X[0] = coefs[I.gcoef + 2 * n];
    __syncthreads();
    const double *pb = phib + (long long)I.mi * stride + step0 * (2 * W);
    for (int q = tid; q < nsteps * 2 * W; q += nt) {
        const T pbv = (T)pb[q];
        PB[q * B] = pbv;
#pragma unroll
        for (int j = 1; j < B; ++j) PB[q * B + j] = feq_eval<T, DC>(Q + (j - 1) * cs, D, I, pbv);
    }

    const bool has = tid < I.nthr;
    const int N = I.N;
    const int x0 = tid * K - I.shift;  // node of this thread's first position
    const int kL = W - 1 + I.depth, kR = N - W - I.depth;
    const int warp = tid >> 5;
    // the warps and lanes of the two ends (fixed for the launch)
    const int wL = ((kL + I.shift) / K) >> 5, wR = ((N - 1 + I.shift) / K) >> 5;
    const int srcL = ((kL + I.shift) / K) & 31, srcR = ((kR + I.shift) / K) & 31;
    const bool dead = has && (x0 < 0 || x0 + K > N);  // owns positions without a node
    T phi[K], v[B][K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int x = x0 + k;
        const bool ok = has && x >= 0 && x < N;
        phi[k] = ok ? st_in[I.off + x] : T(0);
#pragma unroll
        for (int j = 1; j < B; ++j) v[j][k] = ok ? st_in[I.off + (long long)j * I.ld + x] : T(0);
    }
    __syncthreads();
    const T omw = X[0];

    for (int s = 0; s < nsteps; ++s) {
        T *Rb = R + (s & 1) * NE * nt;
        T *Lb = L + (s & 1) * NE * nt;
        if (has) {
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
        }
        __syncthreads();
        if (has) {
            // pull f_j(x) = s_j(x - e_j); sources outside 0..N-1 only feed outer nodes, which the
            // rebuild overwrites: thread 0 and the last thread take their own (finite) values there
            T d[K];
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] = T(0);
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const int e = vel(j);
                if (e > 0) {
#pragma unroll
                    for (int k = K - 1; k >= 0; --k) {  // descending: v[j][k - e] still old
                        const T nv = k >= e ? v[j][k - e] : (tid > 0 ? Rb[(eslot(e) + k) * nt + tid - 1] : v[j][k]);
                        d[k] += nv - v[j][k];
                        v[j][k] = nv;
                    }
                } else {
                    const int a = -e;
#pragma unroll
                    for (int k = 0; k < K; ++k) {  // ascending: v[j][k + a] still old
                        const T nv = k + a < K ? v[j][k + a]
                                               : (tid + 1 < I.nthr ? Lb[(eslot(a) + k + a - K) * nt + tid + 1] : v[j][k]);
                        d[k] += nv - v[j][k];
                        v[j][k] = nv;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) phi[k] += d[k];
            // relax: s'_j = (1 - omega) f_j + P_j(phi') (real exponents: w = phi^nu once per
            // node, then the rows in phi and w)
            T w[K];
            bool relaxed = false;
            if constexpr (DC < 0) {
                if (I.A > 0) {
#pragma unroll
                    for (int k = 0; k < K; ++k) w[k] = nu_pow<T>(phi[k], I.nu);
                    if constexpr (sizeof(T) == 4) relaxed = relax_rows_fixed<T, B, K>(I.A, I.Dg, P, cs, phi, w, v, omw);
                }
            }
#pragma unroll
            for (int j = 1; j < B && !relaxed; ++j) {
                const T *c = P + (j - 1) * cs;
                T acc[K];
                if constexpr (DC < 0) {
                    if (I.A > 0) {
                        gen_evalK<T, K>(c, I.A, I.Dg, phi, w, acc);
                    } else {
                        const T cD = c[D];
#pragma unroll
                        for (int k = 0; k < K; ++k) acc[k] = cD;
                        for (int p = D - 1; p >= 0; --p) {
                            const T cp = c[p];
#pragma unroll
                            for (int k = 0; k < K; ++k) acc[k] = fma_t(acc[k], phi[k], cp);
                        }
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
                    const T cD = c[D];
#pragma unroll
                    for (int k = 0; k < K; ++k) acc[k] = cD;
                    for (int p = D - 1; p >= 0; --p) {
                        const T cp = c[p];
#pragma unroll
                        for (int k = 0; k < K; ++k) acc[k] = fma_t(acc[k], phi[k], cp);
                    }
                }
#pragma unroll
                for (int k = 0; k < K; ++k) v[j][k] = fma_t(omw, v[j][k], acc[k]);
            }
            if (dead) {
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (x0 + k < 0 || x0 + k >= N) {
                        phi[k] = T(0);
#pragma unroll
                        for (int j = 1; j < B; ++j) v[j][k] = T(0);
                    }
            }
        }
        // the ends: warp-uniform branches, every lane of the warp takes part in the shuffles
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            if (warp != (side == 0 ? wL : wR)) continue;
            const int kf = side == 0 ? kL : kR;
            T fneq[B];
#pragma unroll
            for (int j = 0; j < B; ++j) fneq[j] = T(0);
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (has && x0 + k == kf) {
#pragma unroll
                    for (int j = 1; j < B; ++j) fneq[j] = v[j][k] - feq_eval<T, DC>(Q + (j - 1) * cs, D, I, phi[k]);
                }
#pragma unroll
            for (int j = 1; j < B; ++j) fneq[j] = __shfl_sync(0xffffffffu, fneq[j], side == 0 ? srcL : srcR);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int x = x0 + k;
                const bool mine = has && (side == 0 ? (x >= 0 && x < W) : (x >= N - W && x < N));
                if (mine) {
                    const T *e = PB + (s * 2 * W + (side == 0 ? x : W + x - (N - W))) * B;
                    phi[k] = e[0];
#pragma unroll
                    for (int j = 1; j < B; ++j) v[j][k] = e[j] + fneq[j];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int x = x0 + k;
        if (has && x >= 0 && x < N) {
            st_out[I.off + x] = phi[k];
#pragma unroll
            for (int j = 1; j < B; ++j) st_out[I.off + (long long)j * I.ld + x] = v[j][k];
        }
    }
}

// Rebuild of the outer nodes after a streaming step (k_stream) of bounded segments, for
// instances longer than one CTA holds.  One block per member, thread l < 2W rebuilds outer node
// l (left nodes 0..W-1, then right nodes N-W..N-1); the extrapolation nodes are never outer
// nodes, so reads and writes do not overlap.  Seg::pad holds the depth.
template <typename T, int B>
__global__ void k_nee_fix(T *__restrict__ st, const Seg *__restrict__ segs, const int *__restrict__ members,
                          const T *__restrict__ coefs, const double *__restrict__ phib, long long stride,
                          long long step) {
    constexpr int W = wmax(B);
    const int l = threadIdx.x;
    if (l >= 2 * W) return;
    const int mi = members[blockIdx.x];
    const Seg s = segs[mi];
    const int side = l / W, li = l % W;
    const long long i = side ? s.N - W + li : li;
    const long long k = side ? s.N - W - s.pad : W - 1 + s.pad;
    const T phik = st[s.off + k];
    const T pbv = (T)phib[(long long)mi * stride + step * (2 * W) + l];
    const T *fe = coefs + s.coef + (B - 1) * (s.D + 1);
    const T wk = s.A > 0 ? nu_pow<T>(phik, s.nu) : T(0), wb = s.A > 0 ? nu_pow<T>(pbv, s.nu) : T(0);
#pragma unroll
    for (int j = 1; j < B; ++j) {
        const T *c = fe + (j - 1) * (s.D + 1);
        T ak, ab;
        if (s.A > 0) {
            ak = gen_eval<T>(c, s.A, s.Dg, phik, wk);
            ab = gen_eval<T>(c, s.A, s.Dg, pbv, wb);
        } else {
            ak = c[s.D], ab = c[s.D];
            for (int p = s.D - 1; p >= 0; --p) {
                ak = fma_t(ak, phik, c[p]);
                ab = fma_t(ab, pbv, c[p]);
            }
        }
        st[s.off + (long long)j * s.ld + i] = ab + (st[s.off + (long long)j * s.ld + k] - ak);
    }
    st[s.off + i] = pbv;
}

}  // namespace lbk
