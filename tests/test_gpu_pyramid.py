"""GPU parity of the one-launch transform + pyramid (lbl_frame_transform_pyramid)
and of labels gathered from that pyramid (lbl_label_pyramid): the agent words,
the labels and the fused monitor's outputs equal the oracle bit for bit
(eq. 13, eq. 10, Sec. 3.2).  Covers every pyramid word width, z-order grids
whose cell count is below one 256-cell block or not a whole number of blocks
per level, row-major grids in the tiled order and the row-major fallback,
(x, y, tau) z-order grids, the moving front
and the per-warp stream, and the calls' refusals."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def packed_words(wl, P):
    words = torch.empty(wl.world.cells, dtype=getattr(torch, L.packed_word_dtype(P)), device="cuda")
    L.lbl_pack_planes(wl.world, cuda(wl.planes), P, words)
    return words


def check_frame(wl, P, rm, mon=None, monitor=None, cfg=None, with_O=True):
    E = wl.n_edges
    words = packed_words(wl, P)
    O = (torch.full((wl.agent.cells,), 0x5A5A5A5A5A5A5A5A, dtype=torch.int64, device="cuda").view(torch.uint64)
         if with_O else None)
    L.lbl_frame_transform_pyramid(rm, wl.world, words, P, wl.pose, O)
    out = torch.full((E,), 0xFFFF, dtype=torch.int64, device="cuda").view(torch.uint64)
    nxt = torch.zeros(E, dtype=torch.uint64, device="cuda") if mon else None
    viol = torch.zeros(E, dtype=torch.uint16, device="cuda") if mon else None
    L.lbl_label_pyramid(rm, P, out, mon, nxt, viol, cfg)
    want_O = (oracle.frame_transform3(wl.world, wl.planes, wl.pose, wl.agent) if wl.agent.d > 1
              else oracle.frame_transform(wl.world, wl.planes, wl.pose, wl.agent))
    if with_O:
        assert np.array_equal(host(O), want_O)
    want_L = oracle.label(wl.rowptr, wl.colidx, want_O, P)
    assert np.array_equal(host(out), want_L), cfg
    if mon:
        m = monitor
        want_n, want_v = oracle.monitor(m.n_states, m.m, m.relbits, m.delta, m.reject, want_L)
        assert np.array_equal(host(nxt), want_n) and np.array_equal(host(viol), want_v), cfg


@pytest.mark.parametrize("P", [1, 3, 8, 9, 16, 20, 32, 33, 64])
def test_pyramid_path_every_word_width_with_monitor(P):
    """z-order 64 x 64 grid (16 whole top-level blocks), P over the four
    pyramid word widths, the fused monitor, the default and both pipelines,
    O written or left out."""
    wl = synth.make("plain", seed=30 + P, edges=900, P=P)
    m = synth.random_monitor(np.random.default_rng(P), 6, min(P, 8), P)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    mon = L.lbl_monitor_create(m.n_states, m.m, m.relbits, m.delta, m.reject)
    try:
        for cfg in (None, dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT),
                    dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_REGISTERS)):
            check_frame(wl, P, rm, mon, m, cfg)
        check_frame(wl, P, rm, with_O=False)
    finally:
        L.lbl_monitor_free(mon)
        L.lbl_roadmap_free(rm)


@pytest.mark.parametrize("n", [2, 8, 16, 32])
def test_pyramid_path_grids_below_and_around_one_block(n):
    """z-order grids of 4, 64, 256 and 1,024 cells: the top level is partial
    or absent, and the transform's last CTA is the only one."""
    wl = synth.make("plain", seed=40 + n, edges=300, n=n, res=2.0, P=5)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    try:
        check_frame(wl, 5, rm)
        check_frame(wl, 5, rm, cfg=dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT))
    finally:
        L.lbl_roadmap_free(rm)


def test_pyramid_path_row_major_grid_and_larger_roadmap():
    """Row-major agent grids of whole 16 x 16 tiles (the tiled order: one
    launch, also without O) and of partial tiles (transform and pyramid as two
    launches), and a z-order 256 x 256 roadmap of 20k edges (many chunks of
    the front)."""
    tiled = synth.make("plain", seed=56, edges=700, order=synth.ROWMAJOR, n=80, h=48, P=12)
    rm = L.lbl_roadmap_upload(tiled.agent, tiled.rowptr, tiled.colidx, flags=L.LBL_UPLOAD_QUAD)
    try:
        check_frame(tiled, 12, rm, with_O=False)
    finally:
        L.lbl_roadmap_free(rm)
    for wl, P in ((synth.make("plain", seed=50, edges=700, order=synth.ROWMAJOR, P=12), 12),
                  (synth.make("plain", seed=57, edges=700, order=synth.ROWMAJOR, n=72, h=40, P=12), 12),
                  (synth.make("driving", seed=51, edges=20_000), 32)):
        rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
        try:
            check_frame(wl, P, rm)
            check_frame(wl, P, rm, cfg=dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT))
        finally:
            L.lbl_roadmap_free(rm)


def test_pyramid_path_time_augmented_grid():
    """(x, y, tau) z-order grid of 16^3 cells: 256-cell blocks of the 3-D order."""
    wl = synth.make_paper3d(seed=52, edges=400, n=16, d=16)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    try:
        check_frame(wl, wl.P, rm)
    finally:
        L.lbl_roadmap_free(rm)


def test_labels_follow_the_latest_pyramid():
    """Two frames in a row on one roadmap, and a quadtree lbl_label in
    between: lbl_label_pyramid always labels the frame built last."""
    wl = synth.make("plain", seed=53, edges=600, P=10)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    try:
        rng = np.random.default_rng(5)
        words = packed_words(wl, 10)
        out = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
        for _ in range(3):
            pose = synth.random_pose(rng, wl.world)
            L.lbl_frame_transform_pyramid(rm, wl.world, words, 10, pose)
            L.lbl_label_pyramid(rm, 10, out)
            want_O = oracle.frame_transform(wl.world, wl.planes, pose, wl.agent)
            assert np.array_equal(host(out), oracle.label(wl.rowptr, wl.colidx, want_O, 10))
        pose = synth.random_pose(rng, wl.world)
        want_O = oracle.frame_transform(wl.world, wl.planes, pose, wl.agent)
        L.lbl_label(rm, cuda(want_O), 10, out, cfg=dict(algo=L.LBL_ALGO_QUAD))  # rebuilds the pyramid from O
        L.lbl_label_pyramid(rm, 10, out)
        assert np.array_equal(host(out), oracle.label(wl.rowptr, wl.colidx, want_O, 10))
    finally:
        L.lbl_roadmap_free(rm)


def test_pyramid_calls_refuse_what_they_cannot_do():
    wl = synth.make("plain", seed=54, edges=200, P=6)
    words = packed_words(wl, 6)
    out = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    plain = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=0)
    try:
        with pytest.raises(L.LblError, match="no pyramid"):
            L.lbl_label_pyramid(rm, 6, out)  # nothing built yet
        L.lbl_frame_transform_pyramid(rm, wl.world, words, 6, wl.pose)
        with pytest.raises(L.LblError, match="no pyramid"):
            L.lbl_label_pyramid(rm, 20, out)  # 2-byte words asked, 1-byte words built
        with pytest.raises(L.LblError, match="quadtree form"):
            L.lbl_label_pyramid(rm, 6, out, cfg=dict(algo=L.LBL_ALGO_CSR))
        with pytest.raises(L.LblError, match="LBL_UPLOAD_QUAD"):
            L.lbl_frame_transform_pyramid(plain, wl.world, words, 6, wl.pose)
        row = synth.make("plain", seed=55, edges=50, order=synth.ROWMAJOR, n=72, h=40, P=6)  # not whole tiles
        rrm = L.lbl_roadmap_upload(row.agent, row.rowptr, row.colidx, flags=L.LBL_UPLOAD_QUAD)
        try:
            with pytest.raises(L.LblError, match="row-major agent grids need O"):
                L.lbl_frame_transform_pyramid(rrm, row.world, packed_words(row, 6), 6, row.pose)
        finally:
            L.lbl_roadmap_free(rrm)
    finally:
        L.lbl_roadmap_free(plain)
        L.lbl_roadmap_free(rm)
