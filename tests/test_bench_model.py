"""The bench's algorithmic-work model and roofline arithmetic (host logic, no GPU).

The bench reports, for the dominant kernel class of a solve, achieved = algorithmic
bytes (or FP64 operations) over the class's summed CUDA-event time; these tests fix
that arithmetic on hand-made inputs, so that the fraction printed in the JSON line
can be recomputed from the line's own fields.
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2502_04217_gb300 import binding  # noqa: E402


def _opt(**kw):
    return binding.default_options(precision=binding.IPM_MIXED, **kw)


def _res(cg=20, exact=2, it=6):
    return {"cg_iters_total": cg, "kkt_products": cg + exact, "ipm_iters": it, "refinements": 0}


def test_class_model_bytes_and_operations():
    dims = (64, 64, 64)
    H = 64 * 64 * 33
    m = bench._class_model(dims, "mixed", _res(), _opt())
    work, flops, nbytes, ops = m["prepare"]
    # predictor-corrector: two kernels per IPM iteration, bytes per slot as documented
    assert work == 12
    assert nbytes == 6 * ((128 + 176) * H + (144 + 128) * H + 16 * H)
    assert ops == 6 * 2 * H * (bench.FP64_OPS_PREDICTOR + bench.FP64_OPS_PREPARE_PC)
    # pcg_update: 272 bytes per slot, 48 more for the carried G x
    assert m["pcg_update"] == (20, 0.0, 20 * (272 * H + 48 * H))
    # step_length + step_update with the predictor-corrector's direction, G beta carried
    # (G beta and G x read, G beta written) and c read for the certificate's sums
    assert m["step"] == (12, 0.0, 6 * ((160 + 160 + 96) * H + (48 + 16) * H + 96 * H))
    # every other class is (work, flops, bytes)
    assert all(len(v) == 3 for k, v in m.items() if k != "prepare")


def test_certificate_counts_only_its_reducing_launches():
    """With G beta carried the certificate reads beta, G beta and c at the first point and
    after each exact product only; its other launches decide from step_update's sums."""
    dims = (64, 64, 64)
    H = 64 * 64 * 33
    res = _res(cg=20, exact=2, it=6)
    r = bench._roofline_line(dims, "mixed", res, _breakdown(10.0, 2.0), 1, "none", _opt())
    assert r["classes"]["certificate"]["algorithmic_bytes"] == 3 * 48 * H
    r = bench._roofline_line(dims, "mixed", dict(res, warm_start=True), _breakdown(10.0, 2.0), 1, "none", _opt())
    assert r["classes"]["certificate"]["algorithmic_bytes"] == 2 * 48 * H
    r = bench._roofline_line(dims, "mixed", res, _breakdown(10.0, 2.0), 1, "none", _opt(exact_residual=1))
    assert r["classes"]["certificate"]["algorithmic_bytes"] == 8 * 48 * H


def test_prepare_without_predictor_counts_its_own_operations():
    m = bench._class_model((32, 32), "mixed", _res(), _opt(sigma_rule=1))
    work, _, _, ops = m["prepare"]
    assert work == 6 and ops == 6 * 2 * 32 * 17 * bench.FP64_OPS_PREPARE


def _breakdown(prepare_ms, row_ms):
    return {"fft_row": {"launches": 44, "ms": row_ms}, "fft_col": {"launches": 44, "ms": 1.0},
            "fft_middle": {"launches": 22, "ms": 1.0}, "pcg_update": {"launches": 20, "ms": 1.0},
            "prepare": {"launches": 12, "ms": prepare_ms}, "step": {"launches": 12, "ms": 1.0},
            "certificate": {"launches": 8, "ms": 1.0}}


def test_fp64_bound_class_is_reported_against_the_fp64_pipe():
    dims = (64, 64, 64)
    r = bench._roofline_line(dims, "mixed", _res(), _breakdown(10.0, 2.0), 1, "none", _opt())
    assert r["kernel"] == "prepare" and r["bound"] == "alu"
    c = r["classes"]["prepare"]
    assert r["achieved"] == pytest.approx(c["fp64_ops"] / 10e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PIPE_TOPS)
    assert c["frac_of_hbm"] == pytest.approx(c["algorithmic_bytes"] / 10e-3 / 1e9 / bench._peaks().get("hbm_gbs", 6800.0))
    assert c["frac_of_fp64_pipe"] > c["frac_of_hbm"]


def test_hbm_bound_class_is_reported_against_hbm():
    dims = (64, 64, 64)
    r = bench._roofline_line(dims, "mixed", _res(), _breakdown(0.5, 30.0), 1, "none", _opt())
    assert r["kernel"] == "fft_row" and r["bound"] == "hbm"
    c = r["classes"]["fft_row"]
    peak = bench._peaks().get("hbm_gbs", 6800.0)
    assert r["achieved"] == pytest.approx(c["algorithmic_bytes"] / 30e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
