"""lbl_label_blocks_noalloc: block-form labels for callers that cannot allocate
device memory (a planning loop that may not allocate once it runs, or a host
framework that owns every allocation).  Its output must equal lbl_label's
block-form output bit for bit, call after call, although its working memory is
a fixed array that every call reuses.

Kept in a file of its own, collected last."""
import numpy as np
import pytest

import oracle
import synth

import paper_1810_02612_gb300 as L


def block_form(rowptr, colidx):
    """(block rowptr, block ids, cell masks) of CSR rows: one entry per
    distinct 64-cell block of a row, the layout lbl_roadmap_upload derives."""
    E = rowptr.shape[0] - 1
    row_of = np.repeat(np.arange(E), np.diff(rowptr))
    blk = colidx.astype(np.int64) >> 6
    start = np.ones(colidx.shape[0], bool)
    start[1:] = (blk[1:] != blk[:-1]) | (row_of[1:] != row_of[:-1])
    entry = np.cumsum(start) - 1
    n = int(start.sum())
    ids = blk[start].astype(np.uint32)
    masks = np.zeros(n, np.uint64)
    np.bitwise_or.at(masks, entry, np.left_shift(np.uint64(1), (colidx & 63).astype(np.uint64)))
    counts = np.bincount(row_of[start], minlength=E)
    brow = np.zeros(E + 1, np.int64)
    brow[1:] = np.cumsum(counts)
    return brow, ids, masks


def test_noalloc_rejects_sizes_beyond_its_fixed_array():
    n_cells = 1 << 20  # 16384 blocks x 64 propositions = 2^20 words > the fixed 2^19
    with pytest.raises(L.LblError) as ei:
        L.lbl_label_blocks_noalloc(0, 0, 0, 10, 0, n_cells, 64, 0, stream=0)
    assert ei.value.code == L.LBL_EINVAL
    assert "LBL_NOALLOC_MAX_PLANE_WORDS" in L.lbl_last_error()


@pytest.mark.gpu
def test_noalloc_matches_lbl_label_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    wl = synth.make("driving", seed=12, edges=20_000)
    E, cells = wl.n_edges, wl.agent.cells
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_BITTILE)
    try:
        brow, ids, masks = block_form(wl.rowptr, wl.colidx)
        assert L.lbl_roadmap_info(rm)[2] == ids.shape[0]
        d_brow = torch.from_numpy(brow).cuda()
        d_ids = torch.from_numpy(ids.view(np.int32)).cuda().view(torch.uint32)
        d_masks = torch.from_numpy(masks).cuda()
        d_planes = torch.from_numpy(wl.planes).cuda()
        rng = np.random.default_rng(3)
        # two calls in a row with different poses and proposition counts: the
        # second must not see anything the first left in the shared array
        for P in (wl.P, 20):
            pose = synth.random_pose(rng, wl.world)
            O = torch.empty(cells, dtype=torch.uint64, device="cuda")
            L.lbl_frame_transform(wl.world, d_planes[:P].contiguous(), P, pose, wl.agent, O)
            want = torch.empty(E, dtype=torch.uint64, device="cuda")
            L.lbl_label(rm, O, P, want, cfg=dict(algo=L.LBL_ALGO_BITTILE))
            got = torch.full((E,), 0x5A5A, dtype=torch.int64, device="cuda").view(torch.uint64)
            L.lbl_label_blocks_noalloc(d_brow, d_ids, d_masks, E, O, cells, P, got)
            torch.cuda.synchronize()
            got_h, want_h = got.cpu().numpy(), want.cpu().numpy()
            assert np.array_equal(got_h, want_h), P
            assert np.array_equal(got_h, oracle.label(wl.rowptr, wl.colidx, O.cpu().numpy(), P, threads=8))
    finally:
        L.lbl_roadmap_free(rm)


@pytest.mark.gpu
@pytest.mark.parametrize("P", [3, 64])
def test_noalloc_partial_last_block_and_word_widths(P):
    """A row-major grid of 203 x 157 cells (not a multiple of 64, so the last
    64-cell block is partial), P = 3 (few propositions) and P = 64 (every lane
    of the block kernel owns two propositions): two calls in a row equal the
    block form of lbl_label and the oracle."""
    torch = pytest.importorskip("torch")
    agent = synth.Grid(203, 157, 0.3, 0.0, 0.0, synth.ROWMAJOR)
    cells = agent.cells
    assert cells % 64 != 0 and ((cells + 63) // 64) * 64 <= L.LBL_NOALLOC_MAX_PLANE_WORDS
    rng = np.random.default_rng(40 + P)
    rows = []
    for e in range(3000):
        r = rng.random()
        if e == 0:
            rows.append(np.arange(cells - 70, cells))  # ends at the grid's last cell
        elif r < 0.05:
            rows.append(np.zeros(0, np.int64))
        elif r < 0.5:
            a = int(rng.integers(0, cells))
            rows.append(np.arange(a, min(cells, a + int(rng.integers(1, 500)))))
        else:
            rows.append(np.sort(rng.choice(cells, size=int(rng.integers(1, 300)), replace=False)))
    rowptr = np.zeros(len(rows) + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colidx = np.concatenate(rows).astype(np.int32)
    E = len(rows)
    rm = L.lbl_roadmap_upload(agent, rowptr, colidx, flags=L.LBL_UPLOAD_BITTILE)
    try:
        brow, ids, masks = block_form(rowptr, colidx)
        d_brow = torch.from_numpy(brow).cuda()
        d_ids = torch.from_numpy(ids.view(np.int32)).cuda().view(torch.uint32)
        d_masks = torch.from_numpy(masks).cuda()
        for call in range(2):
            O_h = rng.integers(0, 2**63, size=cells, dtype=np.uint64) | np.uint64(1 << 63)
            O_h[rng.random(cells) < 0.8 + 0.1 * call] = 0
            O = torch.from_numpy(O_h).cuda()
            want = torch.empty(E, dtype=torch.uint64, device="cuda")
            L.lbl_label(rm, O, P, want, cfg=dict(algo=L.LBL_ALGO_BITTILE))
            got = torch.full((E,), 0x5A5A, dtype=torch.int64, device="cuda").view(torch.uint64)
            L.lbl_label_blocks_noalloc(d_brow, d_ids, d_masks, E, O, cells, P, got)
            torch.cuda.synchronize()
            got_h = got.cpu().numpy()
            assert np.array_equal(got_h, want.cpu().numpy()), (P, call)
            assert np.array_equal(got_h, oracle.label(rowptr, colidx, O_h, P, threads=8)), (P, call)
    finally:
        L.lbl_roadmap_free(rm)
