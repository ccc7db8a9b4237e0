"""Host model of the one-launch batched-uneven exec (k_fft_uneven_one): the
scheduling protocol step by step, with CTAs run in random order and fewer
resident slots than CTAs, as when other work shares the GPU.

Each CTA follows the kernel's loop:
  * claim two tickets; look up the first tile's job; poll its dependency;
  * per tile: if its inputs were not ready when it was claimed, publish the
    pending count, then wait for them and load; claim the ticket after next;
    poll the next tile's dependency (load it if ready); run the first stage;
    publish the previous column tile's count; run the other stages; the
    finished tile, if a column tile, becomes the pending count;
  * after the last tile: publish the pending count, count the CTA out; the
    last one out zeroes the counters.
The model checks that every launch ends (no CTA waits forever), that no row
tile loads before all column tiles of its chunk are counted, that every
column tile is counted once, and that the counters end at zero.  A planted
change -- a pending count not published before a wait -- must deadlock."""
import random

import pytest


def make_table(rng, njobs):
    """Jobs in table order: single passes and four-step columns (phase 0),
    then four-step rows (phase 1).  Returns (tiles per job, dep_post, dep,
    dep_need), slots numbered from 1."""
    p0, p1 = [], []
    slot = 0
    for _ in range(njobs):
        if rng.random() < 0.5:
            p0.append((rng.randint(1, 6), 0, 0, 0))  # single pass
        else:
            slot += 1
            cols = rng.randint(1, 8)
            p0.append((cols, slot, 0, 0))
            p1.append((rng.randint(1, 8), 0, slot, cols))
    return p0 + p1, slot


class Launch:
    def __init__(self, jobs, nslots, grid, resident, rng, flush_before_wait=True, static=False):
        self.jobs = jobs
        self.start = [0]
        for j in jobs:
            self.start.append(self.start[-1] + j[0])
        self.total = self.start[-1]
        self.sync = [0] * (2 + nslots)  # [0] tickets, [1] CTAs out, [1 + s] counted tiles of slot s
        self.grid, self.resident, self.rng = grid, resident, rng
        self.flush_before_wait = flush_before_wait
        self.static = static  # planted: tiles b, b + grid, ... instead of claims
        self.counted = [0] * len(jobs)
        self.loaded_rows = 0
        self.reset_seen = False

    def job_of(self, t):
        j = 0
        while t >= self.start[j + 1]:
            j += 1
        return j

    def ready(self, j, seen):
        """The kernel's udeps_ready: a slot found complete is remembered."""
        dep, need = self.jobs[j][2], self.jobs[j][3]
        if dep == 0 or dep == seen[0]:
            return True
        if self.sync[1 + dep] < need:
            return False
        seen[0] = dep
        return True

    def cta(self, b):
        """CTA b as a generator: yields after every step, and yields 'wait'
        while it waits for a dependency."""
        s = self.sync
        seen = [0]
        pend = 0
        mine = iter(range(b, 1 << 30, self.grid))

        def ticket():
            if self.static:
                return next(mine)
            t = s[0]
            s[0] += 1
            return t

        def publish():
            nonlocal pend
            if pend:
                s[1 + pend] += 1
                pend = 0

        g = ticket()
        yield
        gn = ticket()
        yield
        cur_loaded = False
        jg = 0
        if g < self.total:
            jg = self.job_of(g)
            cur_loaded = self.ready(jg, seen)
            if cur_loaded:
                self.on_load(jg)
            yield
        while g < self.total:
            if not cur_loaded:
                if self.flush_before_wait:
                    publish()
                while not self.ready(jg, seen):
                    yield "wait"
                self.on_load(jg)
                yield
            claim = ticket()
            next_loaded = False
            jn = jg
            if gn < self.total:
                jn = self.job_of(gn)
                next_loaded = self.ready(jn, seen)
                if next_loaded:
                    self.on_load(jn)
            yield
            # first stage, then the previous column tile's count
            publish()
            yield
            # the other stages and the stores; a column tile is pending now
            pend = self.jobs[jg][1]
            if pend:
                self.counted[jg] += 1
            yield
            g, jg, gn, cur_loaded = gn, jn, claim, next_loaded
        publish()
        s[1] += 1
        if s[1] == self.grid and not self.static:
            # last out: every other CTA has finished, every count is final
            for j, (tiles, post, dep, need) in enumerate(self.jobs):
                if post:
                    assert s[1 + post] == tiles and self.counted[j] == tiles
            self.reset_seen = True
            for k in range(len(s)):
                s[k] = 0
        yield

    def on_load(self, j):
        dep, need = self.jobs[j][2], self.jobs[j][3]
        if dep:
            assert self.sync[1 + dep] >= need, "a row tile loaded before its chunk's columns were counted"
            self.loaded_rows += 1

    def run(self, max_steps=200000):
        waiting = list(range(self.grid))
        self.rng.shuffle(waiting)  # CTAs become resident in any order
        active = {}
        steps = 0
        while waiting or active:
            while waiting and len(active) < self.resident:
                b = waiting.pop()
                active[b] = self.cta(b)
            progressed = False
            for b in self.rng.sample(list(active), len(active)):
                try:
                    r = next(active[b])
                except StopIteration:
                    del active[b]
                    progressed = True
                    break
                if r != "wait":
                    progressed = True
                    break
            steps += 1
            if not progressed or steps > max_steps:
                return False  # every resident CTA is waiting: deadlock
        return True


@pytest.mark.parametrize("seed", range(40))
def test_one_launch_protocol_ends_and_orders_rows_after_columns(seed):
    rng = random.Random(seed)
    jobs, nslots = make_table(rng, rng.randint(1, 12))
    grid = rng.randint(1, 12)
    resident = rng.randint(1, grid)
    L = Launch(jobs, nslots, grid, resident, rng)
    assert L.run(), f"deadlock: grid {grid}, resident {resident}, jobs {jobs}"
    assert L.reset_seen and all(v == 0 for v in L.sync)
    assert L.loaded_rows == sum(j[0] for j in jobs if j[2])


def test_the_model_catches_a_pending_count_kept_across_a_wait():
    """Planted mistake: a CTA that waits for a row tile's inputs while it still
    holds the count of that chunk's last column tile waits forever."""
    jobs = [(1, 1, 0, 0), (1, 0, 1, 1)]  # one column tile, then its row tile
    deadlocks = 0
    for seed in range(20):
        L = Launch(jobs, 1, grid=1, resident=1, rng=random.Random(seed), flush_before_wait=False)
        deadlocks += not L.run(max_steps=2000)
    assert deadlocks == 20
    L = Launch(jobs, 1, grid=1, resident=1, rng=random.Random(0))
    assert L.run()


def test_the_model_catches_static_tile_assignment_with_few_resident_ctas():
    """Planted mistake: tiles assigned round robin (CTA b takes b, b + grid,
    ...) instead of claimed.  With fewer resident CTAs than the grid, a
    resident CTA can wait for a column tile that belongs to a CTA not yet
    resident, while every resident CTA waits: the claims are what make the
    one launch safe on a shared GPU."""
    jobs = [(4, 1, 0, 0), (4, 0, 1, 4)]  # four column tiles, then four row tiles
    assert not Launch(jobs, 1, grid=4, resident=1, rng=random.Random(3), static=True).run(max_steps=5000)
    assert Launch(jobs, 1, grid=4, resident=1, rng=random.Random(3)).run()
    assert Launch(jobs, 1, grid=4, resident=4, rng=random.Random(3), static=True).run()
