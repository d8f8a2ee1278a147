"""Batched frames: one plan over roadmaps of uneven size, grid order, proposition
count, monitor and form (CSR or quadtree, the same roadmap twice); every
item's outputs equal the per-frame entry points' and the oracle's, also when
the launch is captured in a CUDA graph and replayed."""
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
    items.append((items[0][0], 9, None))  # the first roadmap again
    return items


def _run_batch(items, graph):
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
            o = dict(world=wl.world, d_planes=torch.from_numpy(np.ascontiguousarray(wl.planes[:P])).cuda(),
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
def test_batch_matches_per_frame_calls_and_oracle(graph):
    items = _items()
    rms, mons, frames, b = _run_batch(items, graph)
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
