"""CPU re-statements of the schedules the CUDA kernels use, checked against
the oracle's plain definitions (no GPU): the chunked ranking for migration
(bitonic network split into register, shuffle and shared-memory steps, then
binary-search merge), the order crossover placed in 16-byte blocks with a
warp prefix sum, and the assignment decoder's merge of machine streams.
These pin the kernels' reformulations; the GPU tests pin the kernels."""
import numpy as np

import oracle as orc

U64 = np.iinfo(np.uint64).max


def _chunk_sort(keys, C=2048, P=8):
    """k_rank_chunks: C keys, P per thread; steps of distance >= 32 P in
    shared memory, P <= j < 32 P by shuffles, j < P in registers."""
    a = np.full(C, U64, dtype=np.uint64)
    a[:len(keys)] = keys
    nt, k = C // P, 2
    while k <= C:
        j = k >> 1
        while j >= 32 * P:
            e = np.arange(C)
            o = e ^ j
            m = o > e
            ee, oo = e[m], o[m]
            x, y = a[ee].copy(), a[oo].copy()
            sw = (x > y) == ((ee & k) == 0)
            a[ee], a[oo] = np.where(sw, y, x), np.where(sw, x, y)
            j >>= 1
        X = a.reshape(nt, P).copy()
        t = np.arange(nt)[:, None]
        e = P * t + np.arange(P)[None, :]
        while j >= P:
            lm = j // P
            Y = X[np.arange(nt) ^ lm, :]
            keep_min = ((np.arange(nt) & lm) == 0)[:, None] == ((e & k) == 0)
            X = np.where(keep_min, np.minimum(X, Y), np.maximum(X, Y))
            j >>= 1
        for J in (4, 2, 1):
            if J > j and J != 1:
                continue
            for r in range(P):
                if r & J == 0:
                    A, B = X[:, r].copy(), X[:, r | J].copy()
                    sw = (A > B) == (((P * np.arange(nt) + r) & k) == 0)
                    X[:, r], X[:, r | J] = np.where(sw, B, A), np.where(sw, A, B)
        a = X.reshape(-1)
        k <<= 1
    return a[:len(keys)]


def test_chunked_ranking_equals_the_plain_order():
    rng = np.random.default_rng(2)
    for N in [1, 5, 64, 2047, 2048, 2049, 5000, 16384]:
        ms = rng.integers(0, 30 if N > 100 else 5, N)
        keys = (ms.astype(np.uint64) << np.uint64(32)) | np.arange(N, dtype=np.uint64)
        srt = np.concatenate([_chunk_sort(keys[c:c + 2048]) for c in range(0, N, 2048)])
        order = np.full(N, -1)
        for e in range(N):   # k_rank_merge: position in the chunk + lower bounds in the others
            c0 = e // 2048 * 2048
            rank = e - c0 + sum(int(np.searchsorted(srt[c2:c2 + 2048], srt[e])) for c2 in range(0, N, 2048) if c2 != c0)
            assert order[rank] == -1
            order[rank] = int(srt[e]) & 0xFFFFFFFF
        assert np.array_equal(order, orc.rank_island(ms.astype(np.int64))), N


def _ox_blocks(p1, p2, l, r):
    """warp_build_children: the segment, then p2 in 16-byte blocks from block
    (r+1)/8 cyclically, each lane's kept genes placed after a prefix sum."""
    n = len(p1)
    ld = (n + 7) // 8 * 8
    P2 = np.zeros(ld, dtype=np.int64)
    P2[:n] = p2
    child = [None] * n
    for k in range(l, r + 1):
        child[k] = p1[k]
    seg = set(p1[l:r + 1])
    start = 0 if r + 1 == n else r + 1
    nb, b0, placed = (n + 7) >> 3, start >> 3, 0
    for t0 in range(0, nb + 1, 32):
        takes, cnt = [], []
        for lane in range(32):
            t = t0 + lane
            q = b0 + t - (nb if b0 + t >= nb else 0)
            lo, hi = (start if t == 0 else 0), (start if t == nb else n)
            if t > nb:   # lanes past the last pass load nothing
                tk = [(False, 0)] * 8
            else:
                tk = [(lo <= 8 * q + u < hi and int(P2[8 * q + u]) not in seg, int(P2[8 * q + u])) for u in range(8)]
            takes.append(tk)
            cnt.append(sum(x for x, _ in tk))
        incl = np.cumsum(cnt)
        for lane in range(32):
            pos = start + placed + incl[lane] - cnt[lane]
            for take, g in takes[lane]:
                if take:
                    child[pos - n if pos >= n else pos] = g
                    pos += 1
        placed += int(incl[31])
    return np.array(child, dtype=np.int16)


def test_block_crossover_equals_the_oracle_ox():
    rng = np.random.default_rng(3)
    for trial in range(600):
        n = int(rng.integers(1, 700)) if trial % 3 else int(rng.integers(1, 20))
        p1, p2 = rng.permutation(n).astype(np.int16), rng.permutation(n).astype(np.int16)
        u, v = rng.integers(0, n, 2)
        l, r = int(min(u, v)), int(max(u, v))
        assert np.array_equal(_ox_blocks(p1, p2, l, r), orc.order_crossover(p1, p2, l, r)), (n, l, r)


def test_stream_merge_equals_the_sorted_arrival_order():
    """k_eval_assign: a stage's arrivals are the previous stage's machine
    streams merged by smallest head; every stream is in (completion, job)
    order because a machine's completions increase (times >= 1).  Decoding
    by that merge gives the oracle's objective."""
    rng = np.random.default_rng(4)
    for trial in range(40):
        n, S = int(rng.integers(1, 40)), int(rng.integers(1, 6))
        M = rng.integers(1, 5, size=S)
        p_u = rng.integers(1, 30, size=(n, int(M.sum())))
        R = rng.integers(0, 50, size=n)
        genes = np.array([rng.integers(0, M[s]) for j in range(n) for s in range(S)], dtype=np.int16)
        off = np.concatenate([[0], np.cumsum(M)[:-1]])
        runs = [sorted((int(R[j]), j) for j in range(n))]
        cmax = 0
        for s in range(S):
            streams = [[] for _ in range(M[s])]
            free = [0] * M[s]
            heads = [0] * len(runs)
            for _ in range(n):
                q = min((i for i in range(len(runs)) if heads[i] < len(runs[i])), key=lambda i: runs[i][heads[i]])
                ready, j = runs[q][heads[q]]
                heads[q] += 1
                m = genes[j * S + s]
                c = max(free[m], ready) + int(p_u[j, off[s] + m])
                free[m] = c
                streams[m].append((c, j))
                cmax = max(cmax, c)
            assert all(st == sorted(st) for st in streams)
            runs = streams
        inst = orc.AssignInstance(n, S, M, p_u, release=R)
        assert orc.decode_assign(inst, genes) == max(c for st in runs for c, _ in st)


def _single(f, key, p, SH):
    """One dispatch on the sorted key array f: pop f[0], insert the new key."""
    low = (1 << SH) - 1
    f0 = f[0]
    x = p * (1 << SH) + max((f0 & ~low) | (key & low), key)
    return f0, sorted(f[1:] + [x])


def _pair(f, k1, p1, k2, p2, SH):
    """The decoder's two-job dispatch: pop f[0], x1; q = min(f[1], x1) popped
    second; x2; the sorted pair (lo, hi) of {max(f[1], x1), x2} merged into
    f[2..]: slot k = max(min(f[k+2], lo), min(f[k+1], hi), f[k])."""
    low = (1 << SH) - 1
    M = len(f)
    f0 = f[0]
    x1 = p1 * (1 << SH) + max((f0 & ~low) | (k1 & low), k1)
    if M == 1:
        return f0, x1, [p2 * (1 << SH) + max((x1 & ~low) | (k2 & low), k2)]
    q, y = min(f[1], x1), max(f[1], x1)
    x2 = p2 * (1 << SH) + max((q & ~low) | (k2 & low), k2)
    lo, hi = min(y, x2), max(y, x2)
    g = []
    for k in range(M):
        t0 = min(f[k + 2], lo) if k + 2 < M else lo
        if k == 0:
            g.append(t0)
        else:
            t1 = min(f[k + 1], hi) if k + 1 < M else hi
            g.append(max(t0, t1) if k == 1 else max(t0, t1, f[k]))
    return f0, q, g


def test_two_job_dispatch_equals_two_single_dispatches():
    """Same pops and same heap as two single dispatches, for every heap size
    the decoder instantiates, with ties in time (keys differ in the job bits)."""
    rng = np.random.default_rng(7)
    SH = 10
    for trial in range(4000):
        M = int(rng.integers(1, 33))
        times = sorted(int(x) for x in rng.integers(0, 60, size=M))
        f = sorted(t << SH | (int(rng.integers(1, 500)) << 1) for t in times)
        k1 = int(rng.integers(0, 60)) << SH | (int(rng.integers(1, 500)) << 1)
        k2 = int(rng.integers(0, 60)) << SH | (int(rng.integers(1, 500)) << 1)
        p1, p2 = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        a1, fa = _single(f, k1, p1, SH)
        a2, fb = _single(fa, k2, p2, SH)
        b1, b2, g = _pair(f, k1, p1, k2, p2, SH)
        assert (a1, a2, fb) == (b1, b2, g), (M, trial)


def test_completion_key_carries_the_job_and_the_later_start():
    """x = p 2^SH + max((f & ~low) | (in & low), in): time max(time(f), time(in)) + p,
    the incoming job's bits."""
    rng = np.random.default_rng(8)
    SH = 11
    low = (1 << SH) - 1
    for _ in range(2000):
        tf, ti, p = (int(v) for v in rng.integers(0, 1 << 15, size=3))
        jf, ji = (int(v) for v in rng.integers(1, 1000, size=2))
        f, key = tf << SH | jf << 1, ti << SH | ji << 1
        x = p * (1 << SH) + max((f & ~low) | (key & low), key)
        assert x >> SH == max(tf, ti) + p and x & low == ji << 1


def _lane_pipeline(n, S, M, p, genes, release=None, due=None, wt=0):
    """The stage-parallel decoder's schedule, step by step as the warp runs
    it: lane s owns stage s's sorted machine keys; each step every lane
    takes the key its predecessor emitted the step before (lane 0: the next
    gene), dispatches a key that carries a job (pop, complete, insert), or,
    once all n jobs are dispatched, drains one key (inserting +inf); a popped
    key is emitted to the next lane, which ignores keys without a job (the
    initial machines).  The last lane adds each completion's tardiness and
    keeps the largest completion.  Returns (objective, steps)."""
    SH = int(n + 1).bit_length() + 1
    INF = (1 << 62)
    Meff = [min(int(m), n) for m in M]
    f = [[0] * Meff[s] for s in range(S)]
    d = [0] * S
    drained = [0] * S
    emit = [0] * S
    done = [False] * S
    mk = tard = 0
    bad = False
    steps = 0
    while not all(done):
        recv = [0] + emit[:-1]          # shuffle up: what the predecessor emitted last step
        emit = [0] * S
        for s in range(S):
            if done[s]:
                continue
            if s == 0:
                g = int(genes[d[0]]) if d[0] < n else None
                key = 0
                if g is not None:
                    if not 0 <= g < n:
                        bad, g = True, 0
                    key = (g + 1) << 1
                    if release is not None:
                        key |= int(release[g]) << SH
            else:
                key = recv[s]
            job_bits = key & ((1 << SH) - 2)
            if job_bits:
                j = (job_bits >> 1) - 1
                f0 = f[s][0]
                low = (1 << SH) - 1
                start_key = max((f0 & ~low) | (key & low), key)
                x = int(p[j][s]) * (1 << SH) + start_key
                f[s] = sorted(f[s][1:] + [x])
                emit[s] = f0
                d[s] += 1
                if s == S - 1:
                    mk = max(mk, x)
                    if due is not None:
                        tard += max(0, (x >> SH) - int(due[j]))
            elif d[s] == n and s < S - 1 and drained[s] < Meff[s]:
                emit[s] = f[s][0]
                f[s] = f[s][1:] + [INF]
                drained[s] += 1
            done[s] = d[s] == n if s == S - 1 else (d[s] == n and drained[s] == Meff[s])
        steps += 1
    return (-1 if bad else (mk >> SH) + wt * tard), steps


def _lane_static(n, S, M, p, genes, release=None, due=None, wt=0):
    """The same schedule as the kernel runs it, with the windows fixed in
    advance: at step t lane s dispatches the key its predecessor emitted at
    t - 1 if t - start_s is in [0, n) (lane 0: gene t), drains if it is in
    [n, n + M_s) (all lanes but the last), and is idle otherwise; no test
    of the keys' job bits."""
    SH = int(n + 1).bit_length() + 1
    INF = (1 << 62)
    low = (1 << SH) - 1
    Meff = [min(int(m), n) for m in M]
    start = [sum(Meff[j] + 1 for j in range(s)) for s in range(S)]
    total = start[S - 1] + n
    f = [[0] * Meff[s] for s in range(S)]
    emit = [0] * S
    mk = tard = 0
    bad = False
    for t in range(total):
        recv = [0] + emit[:-1]
        emit = [0] * S
        for s in range(S):
            r = t - start[s]
            if 0 <= r < n:
                if s == 0:
                    g = int(genes[r])
                    if not 0 <= g < n:
                        bad, g = True, 0
                    key = (g + 1) << 1 | ((int(release[g]) << SH) if release is not None else 0)
                else:
                    key = recv[s]
                j = ((key & (low - 1)) >> 1) - 1
                assert j >= 0                       # a real job arrives in every dispatch step
                f0 = f[s][0]
                x = int(p[j][s]) * (1 << SH) + max((f0 & ~low) | (key & low), key)
                f[s] = sorted(f[s][1:] + [x])
                emit[s] = f0
                if s == S - 1:
                    mk = max(mk, x)
                    if due is not None:
                        tard += max(0, (x >> SH) - int(due[j]))
            elif s < S - 1 and n <= r < n + Meff[s]:
                emit[s] = f[s][0]
                f[s] = f[s][1:] + [INF]
    return -1 if bad else (mk >> SH) + wt * tard


def test_stage_parallel_lanes_equal_the_oracle():
    """The lane pipeline gives the oracle's objective on random instances
    (ties in time included, M_s >= n, M_s = 1, releases and due times,
    invalid genes) in about n + sum M_s + S steps instead of n * S."""
    rng = np.random.default_rng(12)
    for trial in range(300):
        n = int(rng.integers(1, 40))
        S = int(rng.integers(1, 9))
        M = rng.integers(1, 7, size=S).astype(np.int32)
        p = rng.integers(1, 6 if trial % 2 else 60, size=(n, S)).astype(np.int32)
        genes = rng.permutation(n).astype(np.int16)
        rel = due = None
        wt = 0
        if trial % 3 == 0:
            rel = rng.integers(0, 40, size=n).astype(np.int32)
            due = (rel + rng.integers(0, 80, size=n)).astype(np.int32)
            wt = 100
        o = orc.Instance(n, S, M, p, release=rel, due=due, wt=wt)
        want = orc.decode(o, genes)
        got, steps = _lane_pipeline(n, S, M, p, genes, rel, due, wt)
        assert got == want, (trial, n, S, M.tolist())
        # the schedule is static: lane s receives its n jobs in the steps
        # [start_s, start_s + n), start_s = sum_{j<s} (M_j + 1), so the last
        # lane ends after start_{S-1} + n steps whatever the data
        Meff = np.minimum(M, n)
        assert steps == n + int((Meff[:-1] + 1).sum())
        got_static = _lane_static(n, S, M, p, genes, rel, due, wt)
        assert got_static == want, (trial, n, S, M.tolist())
    # an invalid gene
    M = np.array([2, 3], dtype=np.int32)
    p = np.ones((5, 2), dtype=np.int32)
    assert _lane_pipeline(5, 2, M, p, np.array([0, 1, 7, 3, 4]))[0] == -1
