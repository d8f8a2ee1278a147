"""Batched frames: one plan over roadmaps of uneven size, grid order, proposition
count, monitor and form (CSR or quadtree, the same roadmap twice), frames
packed or transformed from their planes (a world of more than 4x the agent's
cells; an odd world with planes off alignment); every item's outputs equal the
per-frame entry points' and the oracle's, also when the launch is captured in
a CUDA graph and replayed."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


def _items():
    rng = np.random.default_rng(5)
    specs = [("driving", dict(edges=9000)), ("plain", dict(edges=700)), ("large", dict(edges=5000)),
             ("paper", dict(edges=6000)), ("driving", dict(edges=1)), ("plain", dict(edges=2500, order=synth.ROWMAJOR))]
    items = []
    for k, (name, kw) in enumerate(specs):
        wl = synth.make(name, seed=30 + k, **kw)
        P = int(rng.integers(1, wl.P + 1))
        mon = synth.random_monitor(rng, 6, 3, P) if k % 2 == 0 else None
        items.append((wl, P, mon))
    # an edgeless roadmap
    wl0 = synth.make("plain", seed=99, edges=3)
    wl0.rowptr = np.zeros(1, np.int64)
    wl0.colidx = np.zeros(0, np.int32)
    items.append((wl0, 4, None))
    # a world of more than 4x the agent's cells: the batch transforms it from the planes
    wl1 = synth.make("plain", seed=41, edges=800)
    wl1.world = synth.world_grid(160, 120, 0.5)
    wl1.planes = (rng.random((wl1.P, 120, 160)) < 0.2).astype(np.uint8)
    items.append((wl1, wl1.P, None))
    # an odd world cell count and planes one byte past alignment: the batch packs with byte loads
    wl2 = synth.make("plain", seed=42, edges=600)
    wl2.world = synth.world_grid(61, 37, 0.6)
    wl2.planes = (rng.random((wl2.P, 37, 61)) < 0.3).astype(np.uint8) * 7
    wl2.misalign = 1
    items.append((wl2, 3, synth.random_monitor(rng, 5, 2, 3)))
    items.append((items[0][0], 9, None))  # the first roadmap again
    return items


def _run_batch(items, graph, tune=False):
    rms, mons, frames, outs = [], [], [], []
    rng = np.random.default_rng(8)
    for k, (wl, P, mon) in enumerate(items):
        if k == len(items) - 1 and wl is items[0][0]:
            rms.append(rms[0])  # the same roadmap again, in its own frame
        else:
            rms.append(L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=0 if k % 3 == 1 else L.LBL_UPLOAD_QUAD))
        mons.append(L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject) if mon else None)
    b = L.lbl_batch_create(rms, [P for _, P, _ in items], mons)
    try:
        for (wl, P, mon) in items:
            E = wl.rowptr.shape[0] - 1
            off = getattr(wl, "misalign", 0)
            flat = torch.from_numpy(np.ascontiguousarray(wl.planes[:P]).reshape(-1))
            buf = torch.zeros(flat.numel() + off, dtype=torch.uint8, device="cuda")
            buf[off:].copy_(flat.cuda())
            o = dict(world=wl.world, d_planes=buf[off:],
                     pose=synth.random_pose(rng, wl.world),
                     d_O=torch.zeros(wl.agent.cells, dtype=torch.uint64, device="cuda"),
                     d_L=torch.zeros(max(E, 1), dtype=torch.uint64, device="cuda"))
            if mon:
                o["d_next"] = torch.zeros(max(E, 1), dtype=torch.uint64, device="cuda")
                o["d_viol"] = torch.zeros(max(E, 1), dtype=torch.uint16, device="cuda")
            frames.append(o)
        L.lbl_batch_set_frames(b, frames)
        torch.cuda.synchronize()  # the frames' buffers were filled on the default stream
        s = torch.cuda.Stream()
        L.lbl_batch_launch(b, stream=s)  # first launch outside any capture
        s.synchronize()
        if tune:  # measured plan per word-width class, adopted by the launches below
            res = L.lbl_batch_autotune(b, reps=2, stream=s)
            used = [r for r in res if r["items"] > 0]
            assert used and sum(r["items"] for r in used) == len(items)
            for r in used:
                assert r["depth"] in (8, 12) and r["ctas_per_sm"] >= 1 and r["units_per_warp"] in (2, 4, 8, 16, 32)
                assert 0 < r["ms"] <= r["ms_default"]
        if graph:
            for f in frames:
                f["d_L"].zero_()
                f["d_O"].zero_()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                L.lbl_batch_launch(b, stream=torch.cuda.current_stream())
            g.replay()
            g.replay()
        else:
            for f in frames:  # the two stages on their own give the same outputs
                f["d_L"].zero_()
                f["d_O"].zero_()
            torch.cuda.synchronize()
            L.lbl_batch_launch(b, L.LBL_STAGE_TRANSFORM, stream=s)
            L.lbl_batch_launch(b, L.LBL_STAGE_LABEL, stream=s)
        torch.cuda.synchronize()
        return rms, mons, frames, b
    except Exception:
        L.lbl_batch_free(b)
        raise


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("tune", [False, True])
def test_batch_matches_per_frame_calls_and_oracle(graph, tune):
    items = _items()
    rms, mons, frames, b = _run_batch(items, graph, tune)
    try:
        for k, ((wl, P, mon), f, rm, mh) in enumerate(zip(items, frames, rms, mons)):
            E = wl.rowptr.shape[0] - 1
            O = f["d_O"].cpu().numpy()
            want_O = oracle.frame_transform(wl.world, np.ascontiguousarray(wl.planes[:P]), f["pose"], wl.agent)
            assert np.array_equal(O, want_O), k
            want_L = oracle.label(wl.rowptr, wl.colidx, want_O, P, threads=8)
            got_L = f["d_L"].cpu().numpy()[:E]
            assert np.array_equal(got_L, want_L), k
            # the single-frame entry point on the same frame
            one = torch.zeros(max(E, 1), dtype=torch.uint64, device="cuda")
            L.lbl_label(rm, f["d_O"], P, one[:E] if E else one)
            torch.cuda.synchronize()
            assert np.array_equal(one.cpu().numpy()[:E], got_L), k
            if mon:
                wn, wv = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want_L)
                assert np.array_equal(f["d_next"].cpu().numpy()[:E], wn), k
                assert np.array_equal(f["d_viol"].cpu().numpy()[:E], wv), k
    finally:
        L.lbl_batch_free(b)
        for m in mons:
            if m:
                L.lbl_monitor_free(m)
        for rm in {id(r): r for r in rms}.values():
            L.lbl_roadmap_free(rm)


def test_batch_argument_checks():
    wl = synth.make("plain", seed=1, edges=50)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx)
    try:
        with pytest.raises(L.LblError):
            L.lbl_batch_create([rm] * 129, [4] * 129)
        with pytest.raises(L.LblError):
            L.lbl_batch_create([rm], [65])
        b = L.lbl_batch_create([rm], [4])
        with pytest.raises(L.LblError):
            L.lbl_batch_launch(b)  # no frames set yet
        with pytest.raises(L.LblError):
            L.lbl_batch_set_frames(b, [dict(world=wl.world, d_planes=None, pose=wl.pose,
                                            d_O=torch.zeros(64 * 64, dtype=torch.uint64, device="cuda"),
                                            d_L=torch.zeros(50, dtype=torch.uint64, device="cuda"))])
        L.lbl_batch_free(b)
    finally:
        L.lbl_roadmap_free(rm)


def test_batch_words_buffer_grows_and_old_graphs_stay_valid():
    """Frames with a larger world replace the batch's packed-word buffer; a
    graph captured with the earlier frames still runs on them afterwards."""
    wl = synth.make("plain", seed=51, edges=400)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    b = L.lbl_batch_create([rm], [wl.P])
    rng = np.random.default_rng(3)
    E = wl.n_edges

    def frame(world):
        planes = (rng.random((wl.P, world.h, world.w)) < 0.3).astype(np.uint8)
        return planes, dict(world=world, d_planes=torch.from_numpy(planes.reshape(-1)).cuda(),
                            pose=synth.random_pose(rng, world),
                            d_O=torch.zeros(wl.agent.cells, dtype=torch.uint64, device="cuda"),
                            d_L=torch.zeros(E, dtype=torch.uint64, device="cuda"))

    try:
        p1, f1 = frame(synth.world_grid(32, 32, 0.5))     # packed (1,024 world cells)
        p2, f2 = frame(synth.world_grid(120, 100, 0.5))   # packed, a larger buffer (12,000 cells)
        s = torch.cuda.Stream()
        L.lbl_batch_set_frames(b, [f1])
        torch.cuda.synchronize()
        L.lbl_batch_launch(b, stream=s)  # first launch outside any capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            L.lbl_batch_launch(b, stream=torch.cuda.current_stream())
        L.lbl_batch_set_frames(b, [f2])
        f1["d_O"].zero_()
        f1["d_L"].zero_()
        torch.cuda.synchronize()
        g.replay()
        L.lbl_batch_launch(b, stream=s)
        torch.cuda.synchronize()
        for planes, f in ((p1, f1), (p2, f2)):
            want_O = oracle.frame_transform(f["world"], planes, f["pose"], wl.agent)
            assert np.array_equal(f["d_O"].cpu().numpy(), want_O)
            assert np.array_equal(f["d_L"].cpu().numpy(), oracle.label(wl.rowptr, wl.colidx, want_O, wl.P))
    finally:
        L.lbl_batch_free(b)
        L.lbl_roadmap_free(rm)


def test_graph_captured_before_tuning_stays_valid():
    """lbl_batch_autotune replaces the label plans; a graph captured before
    keeps its own plan, whose memory stays allocated, and still labels right;
    the launches after tuning use the tuned plan and label the same."""
    items = _items()[:4]
    rms, mons, frames, b = _run_batch(items, graph=False)
    try:
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            L.lbl_batch_launch(b, stream=torch.cuda.current_stream())
        L.lbl_batch_autotune(b, reps=2, stream=s)
        for f in frames:
            f["d_L"].zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        before = [f["d_L"].cpu().numpy().copy() for f in frames]
        for f in frames:
            f["d_L"].zero_()
        torch.cuda.synchronize()
        L.lbl_batch_launch(b, stream=s)
        torch.cuda.synchronize()
        for k, ((wl, P, mon), f, old) in enumerate(zip(items, frames, before)):
            E = wl.rowptr.shape[0] - 1
            want = oracle.label(wl.rowptr, wl.colidx, f["d_O"].cpu().numpy(), P, threads=8)
            assert np.array_equal(old[:E], want) and np.array_equal(f["d_L"].cpu().numpy()[:E], want), k
    finally:
        L.lbl_batch_free(b)
        for m in mons:
            if m:
                L.lbl_monitor_free(m)
        for rm in {id(r): r for r in rms}.values():
            L.lbl_roadmap_free(rm)
