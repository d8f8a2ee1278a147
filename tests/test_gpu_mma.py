"""The tensor-core form (LBL_ALGO_MMA, tcgen05.mma kind::f8f6f4): dense tiles
whose counts accumulate over many 128-cell blocks (whole-grid rows, rows of
half the cells), every proposition-count width (N = 16, 32, 64), a partial last
tile and a grid whose cell count is not a multiple of 128; and the rate probe,
whose accumulated counts must be exact."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


@pytest.mark.parametrize("P", [1, 16, 17, 33, 64])
def test_dense_tiles_match_the_oracle(P):
    rng = np.random.default_rng(60 + P)
    agent = synth.Grid(70, 61, 0.3, 0.0, 0.0, synth.ROWMAJOR)  # 4,270 cells: the last 128-cell block is partial
    cells = agent.cells
    rows = [np.arange(cells)] * 40                                             # whole-grid rows
    rows += [np.sort(rng.choice(cells, size=cells // 2, replace=False)) for _ in range(150)]  # half the cells
    rows += [np.arange(a, min(cells, a + int(rng.integers(1, 900)))) for a in rng.integers(0, cells, 200)]
    rows += [np.zeros(0, np.int64)] * 7
    rows = [rows[i] for i in rng.permutation(len(rows))]
    rowptr = np.zeros(len(rows) + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colidx = np.concatenate(rows).astype(np.int32)
    O_h = rng.integers(0, 2**63, size=cells, dtype=np.uint64)
    O_h[rng.random(cells) < 0.97] = 0  # sparse occupancy: labels differ between rows
    want = oracle.label(rowptr, colidx, O_h, P)
    rm = L.lbl_roadmap_upload(agent, rowptr, colidx, flags=L.LBL_UPLOAD_MMA)
    try:
        n_mma, tiles = L.lbl_roadmap_form_info(rm, L.LBL_ALGO_MMA)
        assert tiles == (len(rows) + 127) // 128 and n_mma >= tiles
        out = torch.full((len(rows),), 7, dtype=torch.int64, device="cuda").view(torch.uint64)
        L.lbl_label(rm, torch.from_numpy(O_h).cuda(), P, out, cfg=dict(algo=L.LBL_ALGO_MMA))
        torch.cuda.synchronize()
        L.lbl_roadmap_status(rm)
        assert np.array_equal(out.cpu().numpy(), want)
    finally:
        L.lbl_roadmap_free(rm)


@pytest.mark.parametrize("kind,n", [(0, 16), (0, 64), (0, 128), (1, 64)])
def test_mma_probe_counts_are_exact(kind, n):
    r = L.lbl_mma_probe(kind, n, reps=500, ctas_per_sm=2)
    assert r["exact"] and r["tflops"] > 50.0, r


def test_mma_probe_rejects_bad_arguments():
    for args in ((2, 64, 10, 1), (0, 48, 10, 1), (1, 128, 10, 1), (0, 64, 0, 1), (0, 64, 10, 5)):
        with pytest.raises(L.LblError):
            L.lbl_mma_probe(*args)
