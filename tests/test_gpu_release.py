"""Releasing library objects in stream order.

A roadmap, monitor, session or batch freed right after work was enqueued with
it (no synchronisation in between) keeps its memory until that work has run:
the labels come out right.  And freeing one roadmap does not wait for work of
others: with several milliseconds of labeling queued on another stream,
lbl_roadmap_free of an unrelated roadmap returns long before that work ends."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


def test_objects_freed_right_after_enqueued_work_keep_their_memory_until_it_ran():
    wl = synth.make("driving", seed=41, edges=30_000)
    m = synth.random_monitor(np.random.default_rng(5), 6, 3, wl.P)
    s = torch.cuda.Stream()
    O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
    L.lbl_frame_transform(wl.world, torch.from_numpy(wl.planes).cuda(), wl.P, wl.pose, wl.agent, O)
    torch.cuda.synchronize()
    want = oracle.label(wl.rowptr, wl.colidx, O.cpu().numpy(), wl.P, threads=8)
    wn, wv = oracle.monitor(m.n_states, m.m, m.relbits, m.delta, m.reject, want)
    for algo in (L.LBL_ALGO_QUAD, L.LBL_ALGO_CSR):
        rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
        mon = L.lbl_monitor_create(m.n_states, m.m, m.relbits, m.delta, m.reject)
        out = torch.zeros(wl.n_edges, dtype=torch.uint64, device="cuda")
        nxt = torch.zeros(wl.n_edges, dtype=torch.uint64, device="cuda")
        vio = torch.zeros(wl.n_edges, dtype=torch.uint16, device="cuda")
        with torch.cuda.stream(s):
            for _ in range(5):
                L.lbl_label(rm, O, wl.P, out, mon, nxt, vio, cfg=dict(algo=algo), stream=s)
        L.lbl_monitor_free(mon)  # no synchronisation before the frees
        L.lbl_roadmap_free(rm)
        s.synchronize()
        assert np.array_equal(out.cpu().numpy(), want), algo
        assert np.array_equal(nxt.cpu().numpy(), wn) and np.array_equal(vio.cpu().numpy(), wv), algo
    # a session freed right after its frame was enqueued
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    ss = L.lbl_session_create(rm, wl.world, wl.P)
    h_L = torch.zeros(wl.n_edges, dtype=torch.uint64).pin_memory()
    L.lbl_session_run(ss, torch.from_numpy(wl.planes).pin_memory(), wl.pose, h_L, stream=s)
    L.lbl_session_free(ss)
    L.lbl_roadmap_free(rm)
    s.synchronize()
    assert np.array_equal(h_L.numpy(), want)


def test_freeing_one_roadmap_does_not_wait_for_another_streams_work():
    big = synth.make("large", seed=42, edges=400_000)
    small = synth.make("plain", seed=43, edges=500)
    rm_big = L.lbl_roadmap_upload(big.agent, big.rowptr, big.colidx, flags=L.LBL_UPLOAD_QUAD)
    try:
        O = torch.zeros(big.agent.cells, dtype=torch.uint64, device="cuda")
        out = torch.empty(big.n_edges, dtype=torch.uint64, device="cuda")
        a = torch.cuda.Stream()
        L.lbl_label(rm_big, O, big.P, out, cfg=dict(algo=L.LBL_ALGO_CSR), stream=a)  # warm
        a.synchronize()
        t_one = time.perf_counter()
        L.lbl_label(rm_big, O, big.P, out, cfg=dict(algo=L.LBL_ALGO_CSR), stream=a)
        a.synchronize()
        t_one = time.perf_counter() - t_one
        reps = max(10, int(0.02 / max(t_one, 1e-5)))  # about 20 ms of queued work on stream a
        rm_small = L.lbl_roadmap_upload(small.agent, small.rowptr, small.colidx)
        for _ in range(reps):
            L.lbl_label(rm_big, O, big.P, out, cfg=dict(algo=L.LBL_ALGO_CSR), stream=a)
        t = time.perf_counter()
        L.lbl_roadmap_free(rm_small)
        t_free = time.perf_counter() - t
        queued = a.query() is False
        a.synchronize()
        assert queued, "the queued work ended before the free returned"
        assert t_free < 0.25 * reps * t_one, (t_free, reps * t_one)
    finally:
        L.lbl_roadmap_free(rm_big)
