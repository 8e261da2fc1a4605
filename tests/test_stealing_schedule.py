"""Schedule simulation of Section 5.2's task-stealing example (three thread
blocks, nine intervals; makespan 10 without stealing, 7 with inter-interval
stealing, 6 with intra-interval stealing as well) and of the evaluation
kernel's replacement for both: a shared queue of equal tiles claimed in
order (the kernel's atomic tile counter), which reaches the balanced
makespan up to one tile.

The paper gives the example's totals (block 1: 10 time units, block 3: 3)
and the stealing moves (block 3 takes interval 4, block 2 interval 7, then
block 3 halves block 2's rest of interval 7), not every interval's time; the
times below are one assignment consistent with all of them.  The intra-
interval split uses the midpoint of the victim's remaining range (the formula
printed in the paper overshoots it, shown below) and leaves work below one
time unit unsplit, as pairs are indivisible."""
import heapq

# interval -> time units; round-robin assignment: block b gets intervals b, b + 3, b + 6
TIMES = {1: 5.5, 2: 1.5, 3: 1.0, 4: 2.0, 5: 1.5, 6: 1.0, 7: 2.5, 8: 1.5, 9: 1.0}
MIN_SPLIT = 1.0   # work below which a running interval is not split (pairs are indivisible)
ASSIGNED = {1: [1, 4, 7], 2: [2, 5, 8], 3: [3, 6, 9]}


def static_makespan():
    return max(sum(TIMES[i] for i in ivs) for ivs in ASSIGNED.values())


def stealing_makespan(intra: bool):
    """Each block walks its own intervals, skipping those already taken (the
    bitmap), then steals the lowest-numbered untaken interval; with intra
    stealing an idle block with nothing left to take halves the remaining
    work of a running interval (the midpoint of its remaining range)."""
    taken = set()
    done_at = {}
    # event queue of (time block becomes free, block); ties go to the higher-numbered block, which
    # finished its (shorter) own work first in the example
    free = [(0.0, -b, b) for b in ASSIGNED]
    heapq.heapify(free)
    running = {}          # block -> (interval, start, end)
    pos = {b: 0 for b in ASSIGNED}
    while free:
        t, _, b = heapq.heappop(free)
        nxt = None
        while pos[b] < len(ASSIGNED[b]):
            i = ASSIGNED[b][pos[b]]
            pos[b] += 1
            if i not in taken:
                nxt = i
                break
        if nxt is None:
            rest = [i for i in sorted(TIMES) if i not in taken]
            nxt = rest[0] if rest else None
        if nxt is not None:
            taken.add(nxt)
            running[b] = (nxt, t, t + TIMES[nxt])
            heapq.heappush(free, (t + TIMES[nxt], -b, b))
            continue
        if intra:
            victims = [(end, v) for v, (i, s, end) in running.items() if v != b and end - t > MIN_SPLIT]
            if victims:
                end, v = max(victims)
                half = t + (end - t) / 2          # midpoint of the victim's remaining work
                i, s, _ = running[v]
                running[v] = (i, s, half)
                running[b] = (i, t, half)
                # the victim's queued finish event moves to the midpoint
                free = [(half if x == v else ft, nb, x) for ft, nb, x in free]
                heapq.heapify(free)
                heapq.heappush(free, (half, -b, b))
                continue
        done_at[b] = t
    return max(done_at.values())


def queue_makespan(tile: float):
    """The evaluation kernel's scheme: every interval cut into tiles of equal
    work, tiles in order in one queue, each block claiming the next tile when
    it becomes free."""
    tiles = []
    for i in sorted(TIMES):
        n = round(TIMES[i] / tile)
        tiles += [tile] * n
    free = [0.0, 0.0, 0.0]
    for w in tiles:
        k = min(range(3), key=lambda x: free[x])
        free[k] += w
    return max(free)


def test_paper_example_10_7_6():
    assert static_makespan() == 10.0
    assert stealing_makespan(intra=False) == 7.0
    assert stealing_makespan(intra=True) == 6.0


def test_shared_tile_queue_reaches_the_balanced_makespan():
    total = sum(TIMES.values())
    for tile in (0.5, 0.25):
        m = queue_makespan(tile)
        assert total / 3 <= m <= total / 3 + tile
        assert m <= stealing_makespan(intra=True)


def test_midpoint_reading_of_intra_interval_split():
    # the victim keeps [start_b, mid), the thief takes [mid, end_b): an exact split of the rest
    for start_b, end_b in [(0, 10), (10, 20), (7, 8), (3, 100)]:
        mid = start_b + (end_b - start_b) // 2
        assert start_b <= mid <= end_b
        assert (mid - start_b) + (end_b - mid) == end_b - start_b
        # the printed formula start_a = start_b + (start_b + end_b) / 2 leaves the range once start_b > 0
        printed = start_b + (start_b + end_b) // 2
        if start_b > 0:
            assert printed > end_b or printed > mid
