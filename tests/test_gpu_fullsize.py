"""Parity at full size, in the configuration bench.py times: the 1M-edge,
64-proposition workload with the fused monitor through the quadtree form (the
transform building the pyramid and the labels from it, as timed, and through
lbl_label; and the CSR form), the 2^21-cell 2-D and (x, y, tau) workloads, the 100k-edge
driving workload and the 64-frame batch, all with the bench's seeds.

Every edge of every case is compared with the oracle, element by element: the
whole frame transform, every label, and with a monitor every edge's next
states and violation mask.  Labels also have no bits at or above P."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402

THREADS = os.cpu_count() or 1


def _label(rm, O, P, cfg, mon=None, E=None):
    out = torch.empty(E, dtype=torch.uint64, device="cuda")
    nxt = torch.empty(E, dtype=torch.uint64, device="cuda") if mon else None
    viol = torch.empty(E, dtype=torch.uint16, device="cuda") if mon else None
    L.lbl_label(rm, O, P, out, mon, nxt, viol, cfg)
    torch.cuda.synchronize()
    if mon:
        return out.cpu().numpy(), nxt.cpu().numpy(), viol.cpu().numpy()
    return out.cpu().numpy()


# the labeling configurations bench.py can time on these workloads
QUAD_CFGS = [dict(algo=L.LBL_ALGO_QUAD), dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT),
             dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_REGISTERS)]


def _check_workload(wl, cfgs):
    E, P = wl.n_edges, wl.P
    flags = (L.LBL_UPLOAD_QUAD | (L.LBL_UPLOAD_BITTILE if any(c["algo"] == L.LBL_ALGO_BITTILE for c in cfgs) else 0)
             | (L.LBL_UPLOAD_MMA if any(c["algo"] == L.LBL_ALGO_MMA for c in cfgs) else 0))
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
        want = oracle.label(wl.rowptr, wl.colidx, O_h, P, threads=THREADS)
        mon = wl.monitor
        if mon is not None:
            mh = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject)
            want_n, want_v = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want)
        for cfg in cfgs:
            got = _label(rm, O, P, cfg, mh, E)
            labels = got[0] if mh else got
            assert np.array_equal(labels, want), cfg
            if P < 64:
                assert not (labels >> np.uint64(P)).any(), cfg
            if mh:
                assert np.array_equal(got[1], want_n) and np.array_equal(got[2], want_v), cfg
        L.lbl_roadmap_status(rm)
    finally:
        if mh:
            L.lbl_monitor_free(mh)
        L.lbl_roadmap_free(rm)


def test_large_1m_edges_64_props_with_monitor():
    wl = synth.make("large", seed=0, threads=0)
    assert wl.n_edges == 1_000_000 and wl.P == 64 and wl.monitor is not None
    _check_workload(wl, QUAD_CFGS + [dict(algo=L.LBL_ALGO_CSR), dict(algo=L.LBL_ALGO_MMA)])


def test_large_1m_edges_transform_building_the_pyramid():
    """The step bench.py times on this workload: packed planes, the frame
    transform that builds the quadtree pyramid, and the moving front gathering
    from it with the fused monitor, at two poses; the transform's O and every
    edge's label, next states and violations equal the oracle."""
    wl = synth.make("large", seed=0, threads=0)
    m = wl.monitor
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    hm = L.lbl_monitor_create(m.n_states, m.m, m.relbits, m.delta, m.reject)
    try:
        words = torch.empty(wl.world.cells, dtype=getattr(torch, L.packed_word_dtype(wl.P)), device="cuda")
        L.lbl_pack_planes(wl.world, torch.from_numpy(wl.planes).cuda(), wl.P, words)
        O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        out = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
        nxt = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
        viol = torch.empty(wl.n_edges, dtype=torch.uint16, device="cuda")
        for pose in (wl.pose, synth.random_pose(np.random.default_rng(72), wl.world)):
            L.lbl_frame_transform_pyramid(rm, wl.world, words, wl.P, pose, O)
            L.lbl_label_pyramid(rm, wl.P, out, hm, nxt, viol)
            torch.cuda.synchronize()
            want_O = oracle.frame_transform(wl.world, wl.planes, pose, wl.agent)
            assert np.array_equal(O.cpu().numpy(), want_O)
            want = oracle.label(wl.rowptr, wl.colidx, want_O, wl.P, threads=THREADS)
            wn, wv = oracle.monitor(m.n_states, m.m, m.relbits, m.delta, m.reject, want)
            assert np.array_equal(out.cpu().numpy(), want)
            assert np.array_equal(nxt.cpu().numpy(), wn) and np.array_equal(viol.cpu().numpy(), wv)
    finally:
        L.lbl_monitor_free(hm)
        L.lbl_roadmap_free(rm)


def test_large_1m_edges_session_frames_back_to_back():
    """The e2e path of bench.py: 1M-edge frames from pinned host memory through
    lbl_session_run (one moving-front launch per frame at this size), two frames
    at different poses enqueued back to back; every edge's label, next states
    and violations equal the oracle."""
    wl = synth.make("large", seed=0, threads=0)
    m = wl.monitor
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    hm = L.lbl_monitor_create(m.n_states, m.m, m.relbits, m.delta, m.reject)
    ss = L.lbl_session_create(rm, wl.world, wl.P, hm)
    try:
        planes = torch.from_numpy(wl.planes).pin_memory()
        rng = np.random.default_rng(71)
        poses = [wl.pose] + [synth.random_pose(rng, wl.world)]
        outs = [(torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory(),
                 torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory(),
                 torch.empty(wl.n_edges, dtype=torch.uint16).pin_memory()) for _ in poses]
        s = torch.cuda.Stream()
        for pose, (oL, oN, oV) in zip(poses, outs):
            L.lbl_session_run(ss, planes, pose, oL, oN, oV, stream=s)
        s.synchronize()
        for pose, (oL, oN, oV) in zip(poses, outs):
            O = oracle.frame_transform(wl.world, wl.planes, pose[:3], wl.agent)
            want = oracle.label(wl.rowptr, wl.colidx, O, wl.P, threads=THREADS)
            wn, wv = oracle.monitor(m.n_states, m.m, m.relbits, m.delta, m.reject, want)
            assert np.array_equal(oL.numpy(), want)
            assert np.array_equal(oN.numpy(), wn) and np.array_equal(oV.numpy(), wv)
    finally:
        L.lbl_session_free(ss)
        L.lbl_monitor_free(hm)
        L.lbl_roadmap_free(rm)


def test_driving_100k_edges_all_rows():
    wl = synth.make("driving", seed=0, threads=0)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    try:
        O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        L.lbl_frame_transform(wl.world, torch.from_numpy(wl.planes).cuda(), wl.P, wl.pose, wl.agent, O)
        O_h = O.cpu().numpy()
        want = oracle.label(wl.rowptr, wl.colidx, O_h, wl.P, threads=THREADS)
        for cfg in QUAD_CFGS + [dict(algo=L.LBL_ALGO_CSR)]:
            assert np.array_equal(_label(rm, O, wl.P, cfg, E=wl.n_edges), want), cfg
    finally:
        L.lbl_roadmap_free(rm)


def test_paper_2d_2pow21_cells():
    wl = synth.make("paper", seed=0, threads=0)
    assert wl.agent.cells == 1 << 21
    _check_workload(wl, QUAD_CFGS + [dict(algo=L.LBL_ALGO_CSR), dict(algo=L.LBL_ALGO_BITTILE),
                                     dict(algo=L.LBL_ALGO_MMA)])


def test_paper_2d_transform_pyramid_and_session_frames():
    """The paper frame's quadtree rows are in the tiled order (2048 x 1024 is
    whole 16 x 16 tiles): the transform building the pyramid with the labels
    from it, as bench.py times them, and host-buffer session frames back to
    back (which take the same kernels), at two poses; the transform's O and
    every edge's label equal the oracle."""
    wl = synth.make("paper", seed=0, threads=0)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    ss = L.lbl_session_create(rm, wl.world, wl.P)
    try:
        poses = [wl.pose, synth.random_pose(np.random.default_rng(73), wl.world)]
        wants = [oracle.frame_transform(wl.world, wl.planes, pose, wl.agent) for pose in poses]
        words = torch.empty(wl.world.cells, dtype=getattr(torch, L.packed_word_dtype(wl.P)), device="cuda")
        L.lbl_pack_planes(wl.world, torch.from_numpy(wl.planes).cuda(), wl.P, words)
        O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        out = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
        labels = []
        for pose, want_O in zip(poses, wants):
            L.lbl_frame_transform_pyramid(rm, wl.world, words, wl.P, pose, O)
            L.lbl_label_pyramid(rm, wl.P, out)
            torch.cuda.synchronize()
            assert np.array_equal(O.cpu().numpy(), want_O)
            labels.append(oracle.label(wl.rowptr, wl.colidx, want_O, wl.P, threads=THREADS))
            assert np.array_equal(out.cpu().numpy(), labels[-1])
        planes = torch.from_numpy(wl.planes).pin_memory()
        outs = [torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory() for _ in poses]
        s = torch.cuda.Stream()
        for pose, o in zip(poses, outs):
            L.lbl_session_run(ss, planes, pose, o, stream=s)
        s.synchronize()
        for o, want in zip(outs, labels):
            assert np.array_equal(o.numpy(), want)
    finally:
        L.lbl_session_free(ss)
        L.lbl_roadmap_free(rm)


def test_paper_time_augmented_2pow21_cells():
    wl = synth.make_paper3d(seed=0, threads=0)
    assert wl.agent.cells == 1 << 21 and wl.agent.d == 128
    _check_workload(wl, QUAD_CFGS + [dict(algo=L.LBL_ALGO_CSR), dict(algo=L.LBL_ALGO_BITTILE)])


def test_batched_64_frames_every_row():
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
        for k, (f, d) in enumerate(zip(frames, fr)):
            O_h = d["d_O"].cpu().numpy()
            assert np.array_equal(O_h, oracle.frame_transform(f.world, f.planes, f.pose, f.agent)), k
            got = d["d_L"].cpu().numpy()
            assert np.array_equal(got, oracle.label(f.rowptr, f.colidx, O_h, f.P, threads=THREADS)), k
    finally:
        if b is not None:
            L.lbl_batch_free(b)
        for r in rms:
            L.lbl_roadmap_free(r)
