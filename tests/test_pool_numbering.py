"""Host replica of the job numbering of the persistent schedule's shooting
pool and noise pool (csrc/mc_closedloop.cuh: pool_shoot, pool_noise), run
over random warp states: every job is taken exactly once, every index stays
within its array, and a fully pending warp maps job t of pool round r to
lane t, interval r (the coalesced joint loop).  A lane whose line search
backtracks speculatively has nc line-search candidates pending, N nc trial
jobs at positions q N + k (candidate q, interval k)."""
import random

MAX_HORIZON = 64
LS_CAND = 4   # kLsCand: candidates a backtracking line search may shoot in one round


def shoot_jobs(n_jobs, modes, Ns):
    """(owner lane, candidate, interval, pool round, lane) per job, as pool_shoot
    numbers them: interval-major, binary search over the prefix counts, n-th
    set bit, and a trial job's position split into candidate and interval."""
    max_jobs = max(n_jobs)
    assert max_jobs <= MAX_HORIZON * LS_CAND   # the table's size
    mask, pref, total = [], [], 0
    for i in range(max_jobs):
        mi = sum(1 << lane for lane in range(32) if n_jobs[lane] > i)
        mask.append(mi)
        pref.append(total)
        total += bin(mi).count("1")
    out = []
    for lane in range(32):
        for q in range(lane, total, 32):
            lo, hi = 0, max_jobs
            while hi - lo > 1:
                mid = (lo + hi) >> 1
                if pref[mid] <= q:
                    lo = mid
                else:
                    hi = mid
            mo = mask[lo]
            for _ in range(q - pref[lo]):
                mo &= mo - 1
            assert mo
            o = (mo & -mo).bit_length() - 1
            trial = modes[o] == 0
            cq = lo // Ns[o] if trial else 0
            k = Ns[o] - 1 if (modes[o] == 1 and lo == 1) else lo - cq * Ns[o]
            out.append((o, cq, k, q // 32, lane))
    return out


def noise_jobs(sm, n_em):
    """(owner lane, substep, tag) per job, as pool_noise numbers them."""
    P = bin(sm).count("1")
    out = []
    for lane in range(32):
        for q in range(lane, P * 2 * n_em, 32):
            e = q // P
            mo = sm
            for _ in range(q - e * P):
                mo &= mo - 1
            assert mo
            out.append(((mo & -mo).bit_length() - 1, e >> 1, e & 1))
    return out


def test_every_interval_is_shot_once():
    rng = random.Random(1)
    for _ in range(4000):
        Ns, modes, n_jobs, ncs = [], [], [], []
        for _lane in range(32):
            state = rng.choice(["trial", "trial", "ends", "all", "done"])
            N = rng.randint(1, MAX_HORIZON)
            nc = rng.choice([1, 1, 2, LS_CAND]) if state == "trial" else 1
            Ns.append(N)
            ncs.append(nc)
            modes.append({"trial": 0, "ends": 1, "all": 2, "done": 0}[state])
            n_jobs.append({"trial": N * nc, "ends": 2 if N > 1 else 1, "all": N,
                           "done": 0}[state])
        if max(n_jobs) == 0:
            continue
        got = shoot_jobs(n_jobs, modes, Ns)
        for o, cq, k, _, _ in got:
            assert 0 <= o < 32 and 0 <= k < Ns[o] and 0 <= cq < ncs[o]
        want = set()
        for o in range(32):
            if n_jobs[o]:
                if modes[o] == 1:
                    want |= {(o, 0, 0), (o, 0, Ns[o] - 1)}
                else:
                    want |= {(o, c, k) for c in range(ncs[o]) for k in range(Ns[o])}
        triples = [(o, cq, k) for o, cq, k, _, _ in got]
        assert len(triples) == len(set(triples)) and set(triples) == want


def test_full_warp_shoots_like_the_joint_loop():
    got = shoot_jobs([20] * 32, [0] * 32, [20] * 32)
    assert len(got) == 640
    assert all(o == lane and cq == 0 and k == r for o, cq, k, r, lane in got)


def test_every_noise_pair_is_drawn_once():
    rng = random.Random(2)
    for _ in range(2000):
        sm = rng.getrandbits(32) or 1
        n_em = rng.randint(1, 40)
        got = noise_jobs(sm, n_em)
        assert len(got) == len(set(got))
        assert set(got) == {(o, s, g) for o in range(32) if (sm >> o) & 1
                            for s in range(n_em) for g in (0, 1)}


def test_replica_constants_match_the_kernel():
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "paper_2212_02197_gb300", "csrc", "mc_qp.cuh")).read()
    assert int(re.search(r"constexpr int kLsCand = (\d+);", src).group(1)) == LS_CAND
    hdr = open(os.path.join(root, "include", "mc.h")).read()
    assert int(re.search(r"#define MC_MAX_HORIZON (\d+)", hdr).group(1)) == MAX_HORIZON
