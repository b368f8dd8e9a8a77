"""Host model of the hand-off protocol of the persistent set-operation kernel
(setop_keys_kernel): a stager warp, NT walker threads and a look-back warp
pass each tile through a ring of three shared-memory buffers with four
mbarriers per buffer (full, walked, placed, freed).  The model keeps the
kernel's arrival counts and its phase-parity formulas (tile k uses buffer
k % 3; a wait for the j-th use of a buffer tests parity (j / 3) & 1), runs the
roles under random interleavings with the copies completing at random times,
and checks that no role waits forever, that no buffer is staged while a tile
in it is unplaced, that every tile is placed once with its own prefix, and
that a wrong parity in any role is caught.  An mbarrier phase completes when
its pending arrivals reach zero (and, for full, the copy has landed); a wait
for parity q succeeds once the current phase's parity differs from q."""
import random

import pytest

NB = 3  # buffers in the ring


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        assert self.pending > 0, "arrival on a completed phase"
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        return self.phase % 2 != parity


def run_pipeline(ntiles, seed, walkers=3, stager_parity=None, walker_parity=None):
    rnd = random.Random(seed)
    full = [Bar(2) for _ in range(NB)]      # stager lanes + the copy (modelled as one arrival each)
    walked = [Bar(1) for _ in range(NB)]    # walker 0 with the tile's kept count
    placed = [Bar(1) for _ in range(NB)]    # look-back lane 0 with the prefix
    freed = [Bar(walkers) for _ in range(NB)]  # every walker after its store
    stager_parity = stager_parity or (lambda k: ((k - NB) // NB) & 1)
    walker_parity = walker_parity or (lambda k: (k // NB) & 1)
    counter = [0]
    info = [None] * NB
    slot = [dict() for _ in range(NB)]
    unplaced = [None] * NB  # the tile staged in each buffer until it is placed
    copies = []
    placed_tiles = []
    barrier = {"n": 0, "gen": 0}

    def walker_sync():
        gen = barrier["gen"]
        barrier["n"] += 1
        if barrier["n"] == walkers:
            barrier["n"], barrier["gen"] = 0, gen + 1
        while barrier["gen"] == gen:
            yield

    def stager():
        k = 0
        while True:
            b = k % NB
            tile = counter[0]
            counter[0] += 1
            yield
            if k >= NB:
                while not freed[b].done(stager_parity(k)):
                    yield
            assert unplaced[b] is None, f"buffer {b} staged while tile {unplaced[b]} is unplaced"
            if tile >= ntiles:
                info[b] = -1
                full[b].arrive()
                full[b].arrive()
                return
            info[b] = tile
            unplaced[b] = tile
            copies.append(b)
            full[b].arrive()
            k += 1
            yield

    def place(j, wid):
        b = j % NB
        while not placed[b].done((j // NB) & 1):
            yield
        yield from walker_sync()
        assert slot[b].get("tile") == j and slot[b].get("prefix") == ("prefix of", j), (j, slot[b])
        if wid == 0:
            placed_tiles.append(j)
        yield
        freed[b].arrive()
        if freed[b].pending == freed[b].count:  # the last walker's arrival completed the phase
            unplaced[b] = None

    def walker(wid):
        k = 0
        while True:
            b = k % NB
            while not full[b].done(walker_parity(k)):
                yield
            yield from walker_sync()
            tile = info[b]
            if tile == -1:
                break
            assert unplaced[b] == tile
            yield from walker_sync()
            if wid == 0:
                slot[b] = {"tile": tile}
                walked[b].arrive()
            yield
            if k > 0:
                yield from place(k - 1, wid)
            k += 1
        if wid == 0:
            slot[k % NB] = {"tile": -1}
            walked[k % NB].arrive()
        if k > 0:
            yield from place(k - 1, wid)

    def lookback():
        k = 0
        while True:
            b = k % NB
            while not walked[b].done((k // NB) & 1):
                yield
            tile = slot[b]["tile"]
            if tile == -1:
                return
            yield
            slot[b]["prefix"] = ("prefix of", tile)
            placed[b].arrive()
            k += 1
            yield

    actors = {"stager": stager(), "lookback": lookback()}
    for w in range(walkers):
        actors[f"walker{w}"] = walker(w)
    for _ in range(200_000):
        if not actors and not copies:
            break
        choice = rnd.choice(list(actors) + (["copy"] if copies else []))
        if choice == "copy":
            full[copies.pop(0)].arrive()
            continue
        try:
            next(actors[choice])
        except StopIteration:
            del actors[choice]
    else:
        raise AssertionError("a role waits forever")
    assert placed_tiles == list(range(ntiles))


@pytest.mark.parametrize("ntiles", [0, 1, 2, 3, 4, 5, 7, 11, 20])
def test_pipeline_places_every_tile_once_under_random_interleavings(ntiles):
    for seed in range(150):
        run_pipeline(ntiles, seed)


def test_pipeline_model_catches_a_wrong_parity():
    # The stager reusing a buffer one phase early, or walkers waiting for the
    # wrong phase of a full buffer, must trip the model.
    with pytest.raises(AssertionError):
        for seed in range(200):
            run_pipeline(9, seed, stager_parity=lambda k: (k // NB) & 1)
    with pytest.raises(AssertionError):
        for seed in range(200):
            run_pipeline(9, seed, walker_parity=lambda k: ((k // NB) + 1) & 1)
