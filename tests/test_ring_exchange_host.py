"""CPU emulation of the 16-node resident kernel's exchange (k_ring in
paper_0907_1720_gb300/csrc/lbhpde_ring.cuh), no GPU.

The emulation restates the kernel's index arithmetic for one CTA holding several periodic
instances in thread-granular runs of 16 nodes a thread (instances may share a warp):
publication of the edge populations (R, L) and of the wrap-around tail (one case of the
remainder N - xb in the last threads), the pull from own registers, from the neighbours' slots
and, past an instance's last node, from its head slots (a branch taken by the last two threads
of an instance only).  Checked against the exact periodic shift f_j(x) = s_j((x - e_j) mod N) of Eq. (LBE) for
every node, D1Q5, many instance sizes, including N = 4 (the minimum, 2 max|e|), N = 16 r + 1 and
every remainder mod 16.  Every shared-memory index is checked to stay inside its buffer.

The buffers are laid out as in the kernel: rows of stride MAXT (the CTA size class, 512 here)
for the R and L slots and for the tails, an instance's tail in the column of its first thread.

A second check replays the step protocol under random warp interleavings: publish into the
buffers of the step's parity, one CTA barrier, then the reads.  Every read must see the value
published for its own step (the double buffering by step parity is what lets a fast warp
publish step s + 1 while a slow one still reads step s).
"""
import math
import random

import numpy as np

K = 16
B = 5
W = 2
VEL = [0, 1, -1, 2, -2]


def eslot(a):
    return (a - 1) * a // 2


NE = W * (W + 1) // 2
MAXT = 512
MAXI = 32  # kRingMaxInst (instances a CTA)


def plan(sizes):
    """Thread-granular runs as the packer makes them: (tbase, nthr, il) per instance."""
    out, tb = [], 0
    for il, n in enumerate(sizes):
        nthr = -(-n // K)
        out.append((tb, nthr, il))
        tb += nthr
    return out, (tb + 31) // 32 * 32


def emulate_pull(sizes, rng):
    runs, nt = plan(sizes)
    assert nt <= MAXT and len(sizes) <= MAXI
    s_true = [rng.standard_normal((B, n)) for n in sizes]
    # per-thread registers
    v = np.full((nt, B, K), np.nan)
    owner = [-1] * nt
    for i, (tb, nthr, il) in enumerate(runs):
        for t in range(nthr):
            owner[tb + t] = i
            for k in range(K):
                x = t * K + k
                if x < sizes[i]:
                    v[tb + t, :, k] = s_true[i][:, x]
                else:
                    v[tb + t, :, k] = 1e300  # padding: must never reach a real node
    R = np.full(NE * MAXT, np.nan)  # one parity: slot row q at q * MAXT
    L = np.full(NE * MAXT, np.nan)
    T = np.full(NE * MAXT, np.nan)

    def info(tid):
        i = owner[tid]
        tb, nthr, il = runs[i]
        t = tid - tb
        N = sizes[i]
        near_end = (t + 1) * K + W > N
        return i, tb, nthr, il, t, N, near_end

    # publish
    for tid in range(nt):
        if owner[tid] < 0:
            continue
        i, tb, nthr, il, t, N, near_end = info(tid)
        for j in range(1, B):
            e = VEL[j]
            if e > 0:
                for q in range(e):
                    R[(eslot(e) + q) * MAXT + tid] = v[tid, j, K - e + q]
            else:
                for q in range(-e):
                    L[(eslot(-e) + q) * MAXT + tid] = v[tid, j, q]
        if near_end:
            # one case of the remainder R = N - xb (1 .. K + W - 1): tail slot q of a right-moving
            # population takes position R - e + q, node N - e + q, where this thread holds it
            R_ = N - t * K
            assert 1 <= R_ <= K + W - 1
            for j in range(1, B):
                e = VEL[j]
                if e > 0:
                    for q in range(e):
                        k = R_ - e + q
                        if 0 <= k < K:
                            assert t * K + k == N - e + q
                            assert 0 <= eslot(e) + q < NE and 0 <= tb < MAXT
                            T[(eslot(e) + q) * MAXT + tb] = v[tid, j, k]
    new = np.full((nt, B, K), np.nan)
    for tid in range(nt):
        if owner[tid] < 0:
            continue
        i, tb, nthr, il, t, N, near_end = info(tid)
        rt = tid if t + 1 >= nthr else tid + 1  # column of the left-moving neighbour reads
        rem = N - t * K
        assert 0 <= rt < nt
        w = v[tid].copy()
        if near_end and rem < K:
            # the last thread: positions rem .. rem + a - 1 take the head slots; positions further
            # out keep their padding, which must never reach a real node
            for j in range(1, B):
                a = -VEL[j]
                for q in range(max(a, 0)):
                    if rem + q < K:
                        w[j, rem + q] = L[(eslot(a) + q) * MAXT + tb]
        for j in range(1, B):
            e = VEL[j]
            for k in range(K):
                if e > 0:
                    if k >= e:
                        nv = w[j, k - e]
                    elif t > 0:
                        assert 0 <= tid - 1 < nt
                        nv = R[(eslot(e) + k) * MAXT + tid - 1]
                    else:
                        assert tid == tb
                        nv = T[(eslot(e) + k) * MAXT + tid]
                else:
                    a = -e
                    if k + a < K:
                        nv = w[j, k + a]
                    elif not near_end:
                        # the branch of the other threads: never a source past node N - 1
                        assert k + a < rem and rt == tid + 1
                        nv = L[(eslot(a) + k + a - K) * MAXT + rt]
                    elif k + a >= rem:
                        nv = L[(eslot(a) + min(k + a - rem, a - 1)) * MAXT + tb]
                    else:
                        assert 0 <= eslot(a) + k + a - K < NE
                        nv = L[(eslot(a) + k + a - K) * MAXT + rt]
                new[tid, j, k] = nv
    # compare with the exact periodic shift at every real node
    for i, (tb, nthr, il) in enumerate(runs):
        N = sizes[i]
        for x in range(N):
            tid, k = tb + x // K, x % K
            for j in range(1, B):
                want = s_true[i][j, (x - VEL[j]) % N]
                assert new[tid, j, k] == want, (sizes, i, x, j)
    return True


def test_ring_pull_matches_periodic_shift():
    rng = np.random.default_rng(20090717)
    cases = [[4], [5], [16], [17], [31], [32], [33], [8192], [8191], [4, 4, 4], [17, 5, 300, 16, 33]]
    cases += [[16 * r + q for q in range(16)] for r in (0, 1, 3)]  # every remainder, many per warp
    cases[-3] = [n for n in cases[-3] if n >= 4]
    for _ in range(30):
        cnt = int(rng.integers(1, 12))
        sizes = [int(rng.integers(4, 1200)) for _ in range(cnt)]
        while sum(-(-n // K) for n in sizes) > 512:
            sizes.pop()
        cases.append(sizes)
    for sizes in cases:
        assert sum(-(-n // K) for n in sizes) <= 512
        emulate_pull(sizes, rng)


def _protocol(nwarps, wrap, steps, rnd):
    """Random interleaving of the per-warp step protocol; returns the number of events."""
    PUB, BAR, READ = range(3)
    pc = [(0, PUB)] * nwarps          # (step, phase) of each warp
    arrived = {}                      # step -> warps at the barrier
    slot_step = [[-1] * nwarps for _ in range(2)]  # parity -> writer warp -> step of the value
    events = 0
    while True:
        ready = []
        for w in range(nwarps):
            s, ph = pc[w]
            if s >= steps:
                continue
            if ph == BAR and arrived.get(s, 0) < nwarps:
                continue
            ready.append(w)
        if not ready:
            break
        w = rnd.choice(ready)
        s, ph = pc[w]
        events += 1
        par = s & 1
        if ph == PUB:
            slot_step[par][w] = s
            arrived[s] = arrived.get(s, 0) + 1
            pc[w] = (s, BAR)
        elif ph == BAR:
            pc[w] = (s, READ)
        else:
            # reads: the neighbours' slots (and, for an instance's end, every warp's head slots)
            readers = range(nwarps) if wrap[w] else [max(w - 1, 0), w, min(w + 1, nwarps - 1)]
            for r in readers:
                assert slot_step[par][r] == s, (w, r, s, slot_step[par][r])
            pc[w] = (s + 1, PUB)
    assert all(p == (steps, PUB) for p in pc)
    return events


def test_step_protocol_random_interleavings():
    rnd = random.Random(7)
    for trial in range(300):
        nwarps = rnd.choice([1, 2, 3, 4, 8, 16])
        wrap = [rnd.random() < 0.3 for _ in range(nwarps)]
        assert _protocol(nwarps, wrap, 9, rnd) == 3 * 9 * nwarps


def emulate_bounded_pull(cases, rng):
    """The bounded variant (k_ring_nee in paper_0907_1720_gb300/csrc/lbhpde_ring_nee.cuh): the
    interior nodes W..N-W-1 of each instance in thread-granular runs, the 2W outer nodes in a
    shared block [instance][2W][B]; the first thread's right-moving inflow below node W reads
    the left outer nodes, the last thread's left-moving inflow past node N-W-1 reads the right
    outer nodes (registers by the jump on the remainder, neighbour reads by address).  Only the
    inflow values of the outer nodes (e_j > 0 at the left end, e_j < 0 at the right, within |e_j|
    of the interior) hold data; the others are NaN and must never reach a real node."""
    runs, tb = [], 0
    for il, N in enumerate(cases):
        nthr = -(-(N - 2 * W) // K)
        runs.append((tb, nthr, il))
        tb += nthr
    nt = (tb + 31) // 32 * 32
    assert nt <= MAXT and len(cases) <= MAXI
    s_true = [rng.standard_normal((B, N)) for N in cases]
    OB = np.full((MAXI, 2 * W, B), np.nan)
    v = np.full((nt, B, K), np.nan)
    owner = [-1] * nt
    for i, (tb, nthr, il) in enumerate(runs):
        N = cases[i]
        for o in range(2 * W):
            x = o if o < W else N - 2 * W + o
            OB[il, o, :] = s_true[i][:, x]
            # only the inflow values are rebuilt between steps: the rest must never be read
            for j in range(1, B):
                e = VEL[j]
                inflow = (e > 0 and o >= W - e) if o < W else (e < 0 and o - W < -e)
                if not inflow:
                    OB[il, o, j] = np.nan
        for t in range(nthr):
            owner[tb + t] = i
            for k in range(K):
                x = W + t * K + k
                v[tb + t, :, k] = s_true[i][:, x] if x < N - W else 0.0  # padding starts at zero
    R = np.full(NE * MAXT, np.nan)
    L = np.full(NE * MAXT, np.nan)
    for tid in range(nt):
        if owner[tid] < 0:
            continue
        for j in range(1, B):
            e = VEL[j]
            if e > 0:
                for q in range(e):
                    R[(eslot(e) + q) * MAXT + tid] = v[tid, j, K - e + q]
            else:
                for q in range(-e):
                    L[(eslot(-e) + q) * MAXT + tid] = v[tid, j, q]
    for tid in range(nt):
        if owner[tid] < 0:
            continue
        i = owner[tid]
        tb, nthr, il = runs[i]
        t, N = tid - tb, cases[i]
        xb = W + t * K
        rem = N - W - xb
        rt = tid + 1 if t + 1 < nthr else tid
        w = v[tid].copy()
        if rem < K:
            for j in range(1, B):
                a = -VEL[j]
                for q in range(max(a, 0)):
                    if rem + q < K:
                        w[j, rem + q] = OB[il, W + q, j]
        for j in range(1, B):
            e = VEL[j]
            for k in range(K):
                if xb + k >= N - W:
                    continue  # padding: not checked
                if e > 0:
                    if k >= e:
                        nv = w[j, k - e]
                    elif t > 0:
                        nv = R[(eslot(e) + k) * MAXT + tid - 1]
                    else:
                        nv = OB[il, W + k - e, j]
                else:
                    a = -e
                    if k + a < K:
                        nv = w[j, k + a]
                    elif k + a >= rem:
                        q = min(max(k + a - rem, 0), W - 1)
                        nv = OB[il, W + q, j]
                    else:
                        nv = L[(eslot(a) + k + a - K) * MAXT + rt]
                x = xb + k
                assert nv == s_true[i][j, x - e], (cases, i, x, j)


def test_bounded_pull_matches_exact_shift():
    rng = np.random.default_rng(601)
    cases = [[2 * (W + 1)], [2 * (W + 4)], [601], [601] * 13, [20, 21, 22, 36, 37, 38, 100], [8196], [8195]]
    cases += [[2 * W + 16 * r + q for q in range(1, 17)] for r in (0, 1)]
    for _ in range(20):
        sizes = [int(rng.integers(6, 1500)) for _ in range(int(rng.integers(1, 10)))]
        while sum(-(-(n - 2 * W) // K) for n in sizes) > 512:
            sizes.pop()
        cases.append(sizes)
    for c in cases:
        emulate_bounded_pull(c, rng)
