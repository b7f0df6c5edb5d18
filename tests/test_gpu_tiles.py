"""Tile widths of the fused split3 SGEMM (128, 192, 256 columns of C per
tile), chosen per task by the manager: every width gives each element of C
the same sum in the same order, so the results at all widths are bitwise
equal, and each is within the SGEMM rule against the binary64 oracle. Shapes
cover ragged row and column tails, n below, between and above the widths,
and k not a multiple of the 32-wide k-step."""
import numpy as np
import pytest
import torch

import oracle
import synth
from sgemm_bounds import check_sgemm

pytestmark = pytest.mark.gpu

SHAPES = [(128, 128, 512), (200, 192, 96), (130, 320, 64), (257, 384, 200), (64, 700, 33),
          (300, 1000, 160), (128, 64, 128), (1, 257, 31)]


@pytest.fixture(scope="module")
def gvm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    return g


def run(gvm, tile_n, inputs):
    outs = []
    with gvm.Manager(2, ring_depth=16, mode="barrier", sgemm_path="split3", slice_bytes=64 << 20,
                     sgemm_tile_n=tile_n) as mgr:
        ranks = [mgr.attach(r) for r in range(2)]
        seqs = []
        for i, (A, B) in enumerate(inputs):
            tA = torch.from_numpy(A).pin_memory()
            tB = torch.from_numpy(B).pin_memory()
            tC = torch.full((A.shape[0], B.shape[1]), float("nan")).pin_memory()
            seqs.append((ranks[i % 2], ranks[i % 2].submit_sgemm(tA, tB, tC), (tA, tB), tC))
        mgr.flush()
        for rk, seq, _, tC in seqs:
            rk.sync(seq)
            outs.append(tC.numpy().copy())
        assert mgr.stats()["device_status"] == 0
    return outs


def test_tile_widths_bitwise_equal_and_within_rule(gvm):
    inputs = [synth.sgemm_inputs(synth.task_seed(11, i), m, n, k) for i, (m, n, k) in enumerate(SHAPES)]
    by_width = {w: run(gvm, w, inputs) for w in (128, 192, 256)}
    for i, (A, B) in enumerate(inputs):
        check_sgemm(by_width[256][i], A, B, oracle.sgemm64(A, B))
        for w in (128, 192):
            assert np.array_equal(by_width[w][i].view(np.uint32), by_width[256][i].view(np.uint32)), (w, SHAPES[i])


def test_tile_width_from_cost_table(gvm, monkeypatch):
    # A cost table that makes narrow tiles cheap: every task is cut into
    # 128- or 192-wide tiles by the library's rule; results stay the oracle's
    # and equal the fixed-width ones.
    import paper_1511_07658_gb300.manager as mgr_mod

    inputs = [synth.sgemm_inputs(synth.task_seed(12, i), m, n, k) for i, (m, n, k) in enumerate(SHAPES)]
    fixed = run(gvm, 256, inputs)
    monkeypatch.setattr(mgr_mod, "tuning", lambda: {"sgemm_tile_cost": {"128": 0.3, "192": 0.5, "256": 1.0}})
    tuned = run(gvm, None, inputs)
    for i in range(len(inputs)):
        assert np.array_equal(tuned[i].view(np.uint32), fixed[i].view(np.uint32)), SHAPES[i]
