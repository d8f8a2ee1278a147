"""Parity at full size, in the configuration bench.py times: the 1M-edge,
64-proposition workload with the fused monitor through the quadtree form (and
the CSR form), the 2^21-cell 2-D and (x, y, tau) workloads, the 100k-edge
driving workload and the 64-frame batch, all with the bench's seeds.

The oracle cannot label 1.2e9 nonzeros per case in a test, so it checks the
whole frame transform and a seeded sample of rows (label, next states and
violations); over all edges the forms must agree with each other, labels have
no bits at or above P, and next states follow from the labels through the
monitor table."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402

SAMPLE = 20_000


def _label(rm, O, P, algo, mon=None, E=None):
    out = torch.empty(E, dtype=torch.uint64, device="cuda")
    nxt = torch.empty(E, dtype=torch.uint64, device="cuda") if mon else None
    viol = torch.empty(E, dtype=torch.uint16, device="cuda") if mon else None
    L.lbl_label(rm, O, P, out, mon, nxt, viol, dict(algo=algo))
    torch.cuda.synchronize()
    if mon:
        return out.cpu().numpy(), nxt.cpu().numpy(), viol.cpu().numpy()
    return out.cpu().numpy()


def _check_workload(wl, algos, seed):
    E, P = wl.n_edges, wl.P
    flags = L.LBL_UPLOAD_QUAD | (L.LBL_UPLOAD_BITTILE if L.LBL_ALGO_BITTILE in algos else 0)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=flags)
    mh = None
    try:
        O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        planes = torch.from_numpy(wl.planes).cuda()
        if wl.agent.d > 1:
            L.lbl_frame_transform(wl.world, planes, P, wl.pose, wl.agent, O)
            want_O = oracle.frame_transform3(wl.world, wl.planes, wl.pose, wl.agent)
        else:
            L.lbl_frame_transform(wl.world, planes, P, wl.pose[:3], wl.agent, O)
            want_O = oracle.frame_transform(wl.world, wl.planes, wl.pose[:3], wl.agent)
        torch.cuda.synchronize()
        O_h = O.cpu().numpy()
        assert np.array_equal(O_h, want_O)
        rows = np.sort(np.random.default_rng(seed).choice(E, size=min(SAMPLE, E), replace=False))
        want = oracle.label_rows(rows, wl.rowptr, wl.colidx, O_h, P)
        mon = wl.monitor
        if mon is not None:
            mh = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject)
            want_n, want_v = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want)
        first = None
        for algo in algos:
            got = _label(rm, O, P, algo, mh, E)
            labels = got[0] if mh else got
            assert np.array_equal(labels[rows], want), algo
            if P < 64:
                assert not (labels >> np.uint64(P)).any(), algo
            if mh:
                assert np.array_equal(got[1][rows], want_n) and np.array_equal(got[2][rows], want_v), algo
            if first is None:
                first = got
                if mh:  # next states of every edge follow from its label through the table
                    n_all, v_all = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, labels)
                    assert np.array_equal(got[1], n_all) and np.array_equal(got[2], v_all)
            else:  # every form gives every edge the same label
                for a, b in zip(first if mh else (first,), got if mh else (got,)):
                    assert np.array_equal(a, b), algo
        L.lbl_roadmap_status(rm)
    finally:
        if mh:
            L.lbl_monitor_free(mh)
        L.lbl_roadmap_free(rm)


def test_large_1m_edges_64_props_with_monitor():
    wl = synth.make("large", seed=0, threads=0)
    assert wl.n_edges == 1_000_000 and wl.P == 64 and wl.monitor is not None
    _check_workload(wl, [L.LBL_ALGO_QUAD, L.LBL_ALGO_CSR], seed=1)


def test_driving_100k_edges_all_rows():
    wl = synth.make("driving", seed=0, threads=0)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    try:
        O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        L.lbl_frame_transform(wl.world, torch.from_numpy(wl.planes).cuda(), wl.P, wl.pose, wl.agent, O)
        O_h = O.cpu().numpy()
        want = oracle.label(wl.rowptr, wl.colidx, O_h, wl.P, threads=8)
        for algo in (L.LBL_ALGO_QUAD, L.LBL_ALGO_CSR):
            assert np.array_equal(_label(rm, O, wl.P, algo, E=wl.n_edges), want), algo
    finally:
        L.lbl_roadmap_free(rm)


def test_paper_2d_2pow21_cells():
    wl = synth.make("paper", seed=0, threads=0)
    assert wl.agent.cells == 1 << 21
    _check_workload(wl, [L.LBL_ALGO_QUAD, L.LBL_ALGO_CSR, L.LBL_ALGO_BITTILE], seed=2)


def test_paper_time_augmented_2pow21_cells():
    wl = synth.make_paper3d(seed=0, threads=0)
    assert wl.agent.cells == 1 << 21 and wl.agent.d == 128
    _check_workload(wl, [L.LBL_ALGO_QUAD, L.LBL_ALGO_CSR, L.LBL_ALGO_BITTILE], seed=3)


def test_batched_64_frames_sampled():
    frames = synth.make_batch(seed=0, threads=0)
    rms = [L.lbl_roadmap_upload(f.agent, f.rowptr, f.colidx, flags=L.LBL_UPLOAD_QUAD) for f in frames]
    b = None
    try:
        fr = []
        for f in frames:
            fr.append(dict(world=f.world, d_planes=torch.from_numpy(np.ascontiguousarray(f.planes)).cuda(),
                           pose=f.pose, d_O=torch.empty(f.agent.cells, dtype=torch.uint64, device="cuda"),
                           d_L=torch.empty(f.n_edges, dtype=torch.uint64, device="cuda")))
        b = L.lbl_batch_create(rms, [f.P for f in frames])
        L.lbl_batch_set_frames(b, fr)
        L.lbl_batch_launch(b)
        torch.cuda.synchronize()
        rng = np.random.default_rng(4)
        for k, (f, d) in enumerate(zip(frames, fr)):
            O_h = d["d_O"].cpu().numpy()
            if k % 8 == 0:
                assert np.array_equal(O_h, oracle.frame_transform(f.world, f.planes, f.pose, f.agent)), k
            rows = np.sort(rng.choice(f.n_edges, size=min(500, f.n_edges), replace=False))
            got = d["d_L"].cpu().numpy()
            assert np.array_equal(got[rows], oracle.label_rows(rows, f.rowptr, f.colidx, O_h, f.P)), k
    finally:
        if b is not None:
            L.lbl_batch_free(b)
        for r in rms:
            L.lbl_roadmap_free(r)
