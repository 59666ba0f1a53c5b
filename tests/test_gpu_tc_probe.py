"""The tensor-core contraction probe (probe/tc_contract.cu): tcgen05.mma
kind::tf32 with the 3-term split on the cross evaluation's contraction tiles
must match FP64 products to FP32 accuracy and finish without an mbarrier
timeout, at both tile widths it times."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


@pytest.mark.gpu
def test_tc_contraction_probe_matches_fp64():
    import bench

    lines = [json.loads(l) for l in bench.tc_contract().splitlines() if l.strip()]
    assert {d["N"] for d in lines} == {16, 64}
    for d in lines:
        assert d["tc_timeout"] == 0
        # error relative to sum |a b| over K = 32 terms: the 3-term TF32 split keeps
        # about 2^-21 per product, FP32 accumulation adds K 2^-24 at most
        assert d["tc_rel_err"] < 2e-6, d
        assert d["simt_rel_err"] < 2e-6, d
        print("tile %dx%dx%d: tensor cores %.1f ns, FMA pipe %.1f ns per tile, errors %.1e / %.1e"
              % (d["M"], d["N"], d["K"], d["tc_ns_per_tile"], d["simt_ns_per_tile"], d["tc_rel_err"],
                 d["simt_rel_err"]))
