"""A step-level model of the speculative kernel's rounds, run under random
interleavings on the CPU (no GPU; the kernel itself is checked against the
oracle by the GPU tests).

W teams run a GVNS loop whose iteration `it` accepts or not as a fixed
function of (it, incumbent): the incumbent is the last accepted iteration,
so an iteration computed from an incumbent that a committed acceptance has
since replaced is wrong, as in the real search.  Each team, per round r:
takes a ticket once all W tickets of round r - 1 are out (its position), skips
its iteration when the round is already decided for an earlier position,
else runs it over several sweeps (giving up at a sweep boundary once the
round is decided for an earlier position), publishes a done word
(2 r + accepted) into the slot of its position and round parity, scans the
done words and writes the decision (tag r + 1, first accepting position or
the active count) once a finished prefix holds it, waits for the decision,
reads the slots up to it and commits.  Every shared-memory access is one
step; the scheduler picks a random runnable team at each step.

Checked: every team commits the sequential run's trajectory; every schedule
ends (no team waits forever); no slot is rewritten while a team of an
earlier round may still read it.  With the done word made visible only
after its writer's scan (the missing fence), some schedule leaves every
team waiting for a decision nobody writes."""
import random

import pytest

TAG = 1 << 23


def accepts(it, incumbent):
    """Whether iteration `it` from incumbent `incumbent` is accepted (about
    one in five, like the benchmark's run)."""
    return (it * 2654435761 ^ (incumbent + 7) * 40503) % 97 < 19


def sequential(n):
    inc, out = -1, []
    for it in range(n):
        a = accepts(it, inc)
        out.append((it, a))
        if a:
            inc = it
    return out


class Shared:
    def __init__(self, W):
        self.W = W
        self.tickets = 0
        self.dec = [0, 0]
        self.done = [[-1] * W for _ in range(2)]
        self.inc = [[None] * W for _ in range(2)]  # incumbent a slot's iteration used
        self.slot_round = [[-1] * W for _ in range(2)]
        self.readers = {}  # (par, pos) -> rounds whose commit may still read it


def team(sh, n, rng, fence, log):
    """One team as a generator: yields None between shared-memory steps, or
    a condition (a callable) that must hold before it continues."""
    W = sh.W
    it0, inc, rnd = 0, -1, 0
    committed = []
    while it0 < n:
        par, tag = rnd & 1, (rnd + 1) % TAG
        nact = min(W, n - it0)
        base = W * rnd
        yield lambda: sh.tickets >= base  # every team holds a ticket of round rnd - 1
        pos = sh.tickets - W * rnd
        sh.tickets += 1
        assert 0 <= pos < W
        yield None
        v = sh.dec[par]
        moot = (v >> 8) == tag and (v & 0xff) < pos
        yield None
        if pos < nact and not moot:
            it = it0 + pos
            quit_early = False
            for _ in range(rng.randint(1, 4)):  # sweeps
                yield None
                v = sh.dec[par]
                if (v >> 8) == tag and (v & 0xff) < pos:
                    quit_early = True
                    break
            if not quit_early:
                # slot (par, pos) is rewritten: no commit of round rnd - 2 may
                # still read it
                assert not any(r < rnd for r in sh.readers.get((par, pos), ())), \
                    "slot overwritten while an earlier round reads it"
                a = accepts(it, inc)
                sh.inc[par][pos] = inc
                sh.slot_round[par][pos] = rnd
                pending = 2 * rnd + (1 if a else 0)
                if fence:
                    sh.done[par][pos] = pending
                    yield None
                d = None
                for i in range(nact):  # the scan, one word per step
                    vi = sh.done[par][i]
                    yield None
                    if (vi >> 1) != rnd:
                        break  # an unfinished position precedes any acceptance
                    if vi & 1:
                        d = i
                        break
                else:
                    d = nact
                if not fence:
                    sh.done[par][pos] = pending  # visible only now
                    yield None
                if d is not None:
                    sh.dec[par] = (tag << 8) | d
                    yield None
        yield lambda: (sh.dec[par] >> 8) == tag
        d = sh.dec[par] & 0xff
        a_pos = d if d < nact else -1
        ncommit = a_pos + 1 if a_pos >= 0 else nact
        for i in range(ncommit):
            sh.readers.setdefault((par, i), set()).add(rnd)
        for i in range(ncommit):
            assert sh.slot_round[par][i] == rnd and sh.inc[par][i] == inc
            assert (sh.done[par][i] >> 1) == rnd
            committed.append((it0 + i, i == a_pos))
            yield None
        for i in range(ncommit):
            sh.readers[(par, i)].discard(rnd)
        if a_pos >= 0:
            inc = it0 + a_pos
        it0 += ncommit
        rnd += 1
    log.append(committed)


def run(W, n, seed, fence=True, max_steps=200000):
    """Run W teams under a random schedule; their committed trajectories, or
    None when every unfinished team waits on a condition that cannot change."""
    rng = random.Random(seed)
    sh = Shared(W)
    log = []
    teams = {t: team(sh, n, random.Random(seed * 31 + t), fence, log) for t in range(W)}
    cond = {t: None for t in teams}
    for _ in range(max_steps):
        if not teams:
            return log
        ready = [t for t in teams if cond[t] is None or cond[t]()]
        if not ready:
            return None  # deadlock
        t = rng.choice(ready)
        try:
            cond[t] = next(teams[t])
        except StopIteration:
            del teams[t]
    raise RuntimeError("too many steps")


@pytest.mark.parametrize("W", [2, 3, 5, 8])
def test_every_schedule_commits_the_sequential_trajectory(W):
    ref = sequential(60)
    for seed in range(40):
        log = run(W, 60, seed)
        assert log is not None, f"deadlock (W={W}, seed={seed})"
        assert len(log) == W
        for committed in log:
            assert committed == ref


def test_without_the_fence_a_schedule_can_stall():
    """The done word published only after its writer's scan: two teams that
    finish together can each miss the other, and then nobody decides."""
    stalled = 0
    for seed in range(300):
        if run(4, 40, seed, fence=False) is None:
            stalled += 1
    assert stalled > 0
