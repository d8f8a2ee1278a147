"""CPU test of bench.py's enqueue gates (host logic only): timed steps come in
blocks behind a fixed-length spin; a block whose host enqueue outlasted the
spin is enqueued again (its step times replace the late attempt's), up to the
retry limit, and the summary counts the re-runs and the blocks still late.
The CUDA calls are stubs: nothing here needs a GPU."""
import contextlib
import os
import sys
import time
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Event:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 1.0  # ms: the calibration spin of 2M cycles "took" 1 ms


def _fake_torch(log):
    cuda = types.SimpleNamespace(
        Event=_Event,
        synchronize=lambda: log.append("sync"),
        stream=lambda s: contextlib.nullcontext(),
        _sleep=lambda cycles: log.append(("spin", cycles)),
    )
    return types.SimpleNamespace(cuda=cuda)


def test_blocks_cover_the_steps_in_order_behind_a_spin():
    log = []
    g = bench.Gate(_fake_torch(log), stream=None, block=4, ms=50.0)
    assert g.cycles == 2_000_000 * 50  # calibrated: 2M cycles per ms
    seen = [list(b) for b in g.blocks(10)]
    assert seen == [[0, 1, 2, 3], [4, 5, 6, 7], [8, 9]]
    spins = [x for x in log if isinstance(x, tuple)]
    assert len(spins) == 1 + 3  # the calibration, then one spin per block
    s = g.summary()
    assert s["blocks"] == 3 and s["redone"] == 0 and s["late"] == 0 and s["block_steps"] == 4


def test_a_late_block_is_timed_again_and_a_block_late_every_time_is_counted():
    g = bench.Gate(_fake_torch([]), stream=None, block=3, ms=5.0, retries=2)
    attempts = {}
    seen = []
    for blk in g.blocks(9):
        k = blk.start
        attempts[k] = attempts.get(k, 0) + 1
        seen.append(k)
        if (k == 3 and attempts[k] == 1) or k == 6:  # a host pause while enqueuing
            time.sleep(0.02)
    # block 3 once late then on time; block 6 late on all 1 + 2 attempts
    assert seen == [0, 3, 3, 6, 6, 6]
    s = g.summary()
    assert s["redone"] == 3 and s["late"] == 1 and s["blocks"] == 3
    assert s["host_enqueue_ms_max"] >= 20.0
