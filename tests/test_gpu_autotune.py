"""The window autotuner measures on the GPU, installs its table, and results stay exact."""
import pytest
import torch

from oracle import g1
from tests.util import closed_form_limbs, msm_inputs

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")
from paper_2502_11660_gb300 import autotune  # noqa: E402


def test_tune_install_and_use():
    res = autotune.tune(log2_sizes=[10, 12], reps=1)
    try:
        autotune.install(res["table"])
        for k in (10, 12):
            assert pkg.msm_g1_default_c(1 << k) == res["table"][k]
            assert res["table"][k] in res["timings"][k]
        n = 3000
        a, s, pts = msm_inputs(n, tag=61)
        out = pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), scalar_bits=253)   # c = 0: the table
        torch.cuda.synchronize()
        assert g1.from_limbs(pkg.to_host(out)) == closed_form_limbs(s, a)
    finally:
        autotune.clear()


def test_schedule_tuner_installs_and_results_stay_exact():
    """tune_schedule measures c, the chunk size, the sort, the reduction threads and the
    window groups per size, installs them, and calls with c = 0 use them (exact results)."""
    try:
        res = autotune.tune_schedule(log2_sizes=[12, 17], reps=1, edwards=True, glv=True)
        for k in (12, 17):
            c, chunk, sort, rlog2, groups = res["schedule"][k]
            sch = pkg.msm_g1_schedule(1 << k, scalar_bits=253, edwards=True, glv=True)
            assert sch["c"] == c
            if chunk:
                assert sch["chunk"] == chunk
            assert sch["sort"] == ("radix" if sort == 2 else "counting")
            assert set(res["ms"][k]) == {"c", "chunk", "sort", "reduce_log2", "groups"}
        for n in (1 << 12, (1 << 17) + 5):
            a, s, pts = msm_inputs(n, tag=62)
            out = pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), scalar_bits=253, edwards=True, glv=True)
            torch.cuda.synchronize()
            assert g1.from_limbs(pkg.to_host(out)) == closed_form_limbs(s, a)
    finally:
        autotune.clear_schedule(edwards=True, glv=True)
