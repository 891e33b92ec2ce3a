"""Host replica of the job numbering of the persistent schedule's shooting
pool and noise pool (csrc/mc_closedloop.cuh: pool_shoot, pool_noise), run
over random warp states: every job is taken exactly once, every index stays
within its array, and a fully pending warp maps job t of pool round r to
lane t, interval r (the coalesced joint loop)."""
import random

MAX_HORIZON = 64


def shoot_jobs(n_jobs, modes, Ns):
    """(owner lane, interval, pool round, lane) per job, as pool_shoot numbers
    them: interval-major, binary search over the prefix counts, n-th set bit."""
    max_jobs = max(n_jobs)
    assert max_jobs <= MAX_HORIZON
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
            k = Ns[o] - 1 if (modes[o] == 1 and lo == 1) else lo
            out.append((o, k, q // 32, lane))
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
        Ns, modes, n_jobs = [], [], []
        for _lane in range(32):
            state = rng.choice(["trial", "ends", "all", "done"])
            N = rng.randint(1, MAX_HORIZON)
            Ns.append(N)
            modes.append({"trial": 0, "ends": 1, "all": 2, "done": 0}[state])
            n_jobs.append({"trial": N, "ends": 2 if N > 1 else 1, "all": N, "done": 0}[state])
        if max(n_jobs) == 0:
            continue
        got = shoot_jobs(n_jobs, modes, Ns)
        for o, k, _, _ in got:
            assert 0 <= o < 32 and 0 <= k < Ns[o] and k + 1 <= Ns[o]
        want = set()
        for o in range(32):
            if n_jobs[o]:
                if modes[o] == 1:
                    want |= {(o, 0), (o, Ns[o] - 1)}
                else:
                    want |= {(o, k) for k in range(Ns[o])}
        pairs = [(o, k) for o, k, _, _ in got]
        assert len(pairs) == len(set(pairs)) and set(pairs) == want


def test_full_warp_shoots_like_the_joint_loop():
    got = shoot_jobs([20] * 32, [0] * 32, [20] * 32)
    assert len(got) == 640
    assert all(o == lane and k == r for o, k, r, lane in got)


def test_every_noise_pair_is_drawn_once():
    rng = random.Random(2)
    for _ in range(2000):
        sm = rng.getrandbits(32) or 1
        n_em = rng.randint(1, 40)
        got = noise_jobs(sm, n_em)
        assert len(got) == len(set(got))
        assert set(got) == {(o, s, g) for o in range(32) if (sm >> o) & 1
                            for s in range(n_em) for g in (0, 1)}
