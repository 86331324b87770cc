"""CPU mirrors of two kernel invariants of the CUDA-core block-Toeplitz
product (no GPU needed).

1. Generator stages: the 32 rows of a source sit in shared memory as one
   contiguous run of 32 (4N+1) values between 8 zero guards before and 16
   after.  A thread of mode block m0 .. m0 + KB - 1 and lane (target row) r
   reads positions 8 + r L + 2N - m0 + t for t in [-(KB - 1), npad - 1].
   Every read must stay inside the stage, and every read outside its own row
   must meet a padded source mode (x_n = 0) or a padded target mode (result
   discarded), so that the product is the one of the section 4.2 blocks.
2. The barrier-free single-column kernel's two stages: a producer refills a
   stage after every warp released it (empty mbarrier, one arrival per warp)
   and warps consume a stage after its copy landed (full mbarrier).  A
   randomised schedule of warps and copy completions must never let a warp
   read a stage that does not hold its source, and must never deadlock.
"""
import random

import pytest

MSD_MAX_N = 55
FRONT, BACK = 8, 16


def test_stage_window_reads_stay_in_bounds_and_meet_only_padding():
    for N in range(1, MSD_MAX_N + 1):
        n, L = 2 * N + 1, 4 * N + 1
        size = 32 * L + FRONT + BACK
        for KB in range(4, 10):
            I = -(-n // KB)
            npad = I * KB
            for blk in range(I):
                m0 = blk * KB
                for lane in (0, 31):
                    base = FRONT + lane * L + 2 * N - m0
                    assert base - (KB - 1) >= 0 and base + npad - 1 < size, (N, KB, m0, lane)
                for b in range(KB):
                    m = m0 + b
                    for nn in range(npad):
                        l = nn - m + 2 * N
                        if not 0 <= l < L:  # outside the thread's own row
                            assert nn >= n or m >= n, (N, KB, m, nn)


class _Barrier:
    """mbarrier phase semantics: try_wait.parity(p) succeeds once the phase
    with parity p has completed."""

    def __init__(self, count):
        self.count = self.pending = count
        self.phase = 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.phase ^= 1
            self.pending = self.count

    def test(self, parity):
        return self.phase != parity


def _run_pipeline(nq, nwarps, seed):
    rnd = random.Random(seed)
    full, empty = [_Barrier(1), _Barrier(1)], [_Barrier(nwarps), _Barrier(nwarps)]
    stage = [None, None]           # (source, landed)
    inflight = [0]
    stage[0] = (0, False)
    it = [0] * nwarps
    produced = [False] * nwarps    # warp 0 runs the producer step first
    consumed = 0
    for _ in range(200000):
        if all(i >= nq for i in it) and not inflight:
            return consumed
        if inflight and rnd.random() < 0.3:
            s = inflight.pop(0)
            stage[s] = (stage[s][0], True)
            full[s].arrive()
            continue
        w = rnd.randrange(nwarps)
        i = it[w]
        if i >= nq:
            continue
        sb = i & 1
        if w == 0 and not produced[w]:
            if i + 1 < nq:
                if i >= 1 and not empty[sb ^ 1].test(((i - 1) >> 1) & 1):
                    continue
                stage[sb ^ 1] = (i + 1, False)
                inflight.append(sb ^ 1)
            produced[w] = True
            continue
        if not full[sb].test((i >> 1) & 1):
            continue
        assert stage[sb] == (i, True), (stage[sb], i)
        consumed += 1
        empty[sb].arrive()
        it[w] += 1
        produced[w] = False
    raise AssertionError("deadlock")


@pytest.mark.parametrize("nq", [1, 2, 3, 8])
@pytest.mark.parametrize("nwarps", [1, 3, 7, 16])
def test_two_stage_release_protocol(nq, nwarps):
    for seed in range(60):
        assert _run_pipeline(nq, nwarps, seed) == nq * nwarps
