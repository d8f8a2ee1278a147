"""Bounded waits inside the labeling kernels, made to run out on purpose.

The bulk-copy index stream (LBL_PIPE_BULK) waits on an mbarrier for each
copied chunk of column indices, and the tensor-core form waits on an mbarrier
for each group of MMAs.  With the roadmap's wait limit set to 0 a kernel tests
the awaited phase once and gives up when the data has not arrived yet (the
first copy of a warp's stream never has: it is issued just before): the kernel
records the failure, lets what it has in flight land, frees its tensor memory
and returns.  lbl_roadmap_status then reports LBL_ETIMEOUT once; with the limit
back at its default the same roadmap labels exactly like the oracle again, so
the context stayed usable."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


@pytest.mark.parametrize("cfg", [dict(algo=L.LBL_ALGO_CSR, pipeline=L.LBL_PIPE_BULK), dict(algo=L.LBL_ALGO_MMA)],
                         ids=["bulk-copy index stream", "tensor cores"])
def test_a_wait_that_runs_out_reports_timeout_and_the_roadmap_recovers(cfg):
    wl = synth.make("driving", seed=31, edges=20_000)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_MMA)
    try:
        O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        L.lbl_frame_transform(wl.world, torch.from_numpy(wl.planes).cuda(), wl.P, wl.pose, wl.agent, O)
        torch.cuda.synchronize()
        want = oracle.label(wl.rowptr, wl.colidx, O.cpu().numpy(), wl.P, threads=8)
        out = torch.zeros(wl.n_edges, dtype=torch.uint64, device="cuda")
        L.lbl_roadmap_set_wait_limit(rm, 0)
        L.lbl_label(rm, O, wl.P, out, cfg=cfg)
        with pytest.raises(L.LblError) as ei:
            L.lbl_roadmap_status(rm)
        assert ei.value.code == L.LBL_ETIMEOUT
        L.lbl_roadmap_status(rm)  # the flag was cleared
        L.lbl_roadmap_set_wait_limit(rm, 2_000_000_000)
        out.zero_()
        L.lbl_label(rm, O, wl.P, out, cfg=cfg)
        L.lbl_roadmap_status(rm)
        assert np.array_equal(out.cpu().numpy(), want)
        with pytest.raises(L.LblError):
            L.lbl_roadmap_set_wait_limit(rm, -1)
    finally:
        L.lbl_roadmap_free(rm)
