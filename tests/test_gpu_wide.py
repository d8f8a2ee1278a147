"""Roadmaps of 2^31 nonzeros or more: the streaming kernels keep warp-range
positions in 64-bit registers there (the int32 fast path covers everything
smaller).  524,288 rows of 4,096 consecutive cells (2^31 nonzeros, 8.6 GB of
indices) on a 512x512 grid: every row of the CSR, sector and quadtree forms
equals the oracle (computed in slices of 65,536 rows), and so does the batched
kernel's 64-bit path."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


def test_rows_beyond_32_bit_positions():
    agent = synth.agent_grid(512, 0.2, synth.MORTON)
    cells = agent.cells
    E, run = 1 << 19, 4096
    rng = np.random.default_rng(23)
    starts = rng.integers(0, cells - run + 1, size=E).astype(np.int64)
    rowptr = np.arange(E + 1, dtype=np.int64) * run
    assert rowptr[-1] >= (1 << 31) - 4096  # past the 32-bit fast path
    d_starts = torch.from_numpy(starts).cuda()
    d_col = _cols(d_starts, run)
    d_rowptr = torch.from_numpy(rowptr).cuda()
    rm = L.lbl_roadmap_upload(agent, d_rowptr, d_col, flags=L.LBL_UPLOAD_SECTOR | L.LBL_UPLOAD_QUAD)
    del d_col
    torch.cuda.empty_cache()
    try:
        O_h = np.zeros(cells, np.uint64)
        hit = rng.random(cells) < 0.0005
        O_h[hit] = rng.integers(1, 2**63, size=hit.sum(), dtype=np.uint64)
        O = torch.from_numpy(O_h).cuda()
        outs = {}
        for algo in (L.LBL_ALGO_CSR, L.LBL_ALGO_SECTOR, L.LBL_ALGO_QUAD):
            out = torch.empty(E, dtype=torch.uint64, device="cuda")
            L.lbl_label(rm, O, 64, out, cfg=dict(algo=algo))
            torch.cuda.synchronize()
            outs[algo] = out.cpu().numpy()
        want = np.empty(E, np.uint64)
        step = 1 << 16
        for a in range(0, E, step):  # the oracle over every row, a slice of rows at a time
            n = min(step, E - a)
            cols = (starts[a:a + n, None] + np.arange(run, dtype=np.int64)[None, :]).astype(np.int32).ravel()
            want[a:a + n] = oracle.label(np.arange(n + 1, dtype=np.int64) * run, cols, O_h, 64,
                                         threads=os.cpu_count() or 1)
        for algo, got in outs.items():
            assert np.array_equal(got, want), algo
        assert (want != 0).any() and (want == 0).any()
        L.lbl_roadmap_status(rm)
        # the batched kernel's 64-bit path: one item with these CSR rows
        d_col = _cols(d_starts, run)
        rm_csr = L.lbl_roadmap_upload(agent, d_rowptr, d_col)  # CSR only: the batch streams it as is
        del d_col
        torch.cuda.empty_cache()
        b = None
        try:
            b = L.lbl_batch_create([rm_csr], [64])
            outb = torch.zeros(E, dtype=torch.uint64, device="cuda")
            world = synth.world_grid(512, 512, 0.2)
            planes = torch.zeros(64 * cells, dtype=torch.uint8, device="cuda")
            L.lbl_batch_set_frames(b, [dict(world=world, d_planes=planes, pose=(51.2, 51.2, 0.0), d_O=O, d_L=outb)])
            L.lbl_batch_launch(b, L.LBL_STAGE_LABEL)
            torch.cuda.synchronize()
            assert np.array_equal(outb.cpu().numpy(), want)
        finally:
            if b is not None:
                L.lbl_batch_free(b)
            L.lbl_roadmap_free(rm_csr)
    finally:
        L.lbl_roadmap_free(rm)


def _cols(d_starts, run):
    return (d_starts[:, None] + torch.arange(run, device="cuda")[None, :]).to(torch.int32).reshape(-1)
