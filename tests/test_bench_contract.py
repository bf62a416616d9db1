"""The benchmark's host side (CPU only): the algorithmic flops and bytes per cell-apply that the
roofline divides by, derived here by hand for the benchmark workload, and the JSON line of the
reference arm (the FP64 oracle on the host cores), whose keys the benchmark contract fixes."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2402_02116_gb300 import inputs  # noqa: E402


def test_column_kernel_units_on_the_benchmark_workload():
    """256 x 256 cells, 512 x 512 FFT grid, 32 sources x 8 frequencies (256 problems):
    flops: 2 components x (forward + inverse) x 512 columns x 5 * 512 * log2(512) = 47,185,920,
    plus 28 flops at each of the 512 x 512 wavenumbers = 7,340,032; per cell: 832.
    bytes: T read and written, 2 x 2 x 256 x 512 x 8 = 4,194,304, plus the 3 x 512 x 512 x 8
    spectrum of each frequency over its 32 sources = 196,608; per cell: 67.0."""
    w = inputs.config2_batched_forward()
    assert (w.nz, w.nx, w.lz, w.lx, w.nf, w.n_problems) == (256, 256, 512, 512, 8, 256)
    assert bench.cols_flops_per_cell_apply(w) == pytest.approx(832.0, rel=1e-12)
    assert bench.cols_bytes_per_cell_apply(w) == pytest.approx(4_390_912 / 65_536, rel=1e-12)


def test_form_k_column_kernel_units():
    """Seven FFT lines per column (five sources forward, two outputs inverse) and the 2 x 5
    kernel's 80 flops per wavenumber; five sources read and two outputs written, nine tables per
    frequency."""
    w = inputs.config2_batched_forward()
    fft = 7 * 512 * 5 * 512 * 9
    assert bench.formk_cols_flops_per_cell_apply(w) == pytest.approx((fft + 80 * 512 * 512) / 65_536, rel=1e-12)
    byt = 7 * 256 * 512 * 8 + 9 * 512 * 512 * 8 * 8 / 256
    assert bench.formk_cols_bytes_per_cell_apply(w) == pytest.approx(byt / 65_536, rel=1e-12)
    assert math.isclose(bench.formk_cols_flops_per_cell_apply(w) / bench.cols_flops_per_cell_apply(w),
                        (fft + 80 * 512 * 512) / (4 * 512 * 5 * 512 * 9 + 28 * 512 * 512))


def test_reference_arm_json_line():
    """`bench.py --impl reference` prints one JSON line with the contract's keys: the metric of
    the GPU arm on its workload, the oracle as the CPU baseline (kind, cores, sample) and an e2e
    object with no host-device traffic."""
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "vti256x256_32src_8f"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("kind", ["formk", "gmres", "3d"])
def test_oracle_samples_of_the_other_workloads(kind):
    """The CPU baselines beside the form-K, GMRES and 3D lines: the oracle's own operator passes,
    counted and timed on one problem (small cases here)."""
    if kind == "3d":
        w = inputs.small_case_3d(nz=4, ny=3, nx=5, freqs=(6.0,))
        r = bench.oracle_3d_sample(w, 1, passes=2)
        assert "2 3D operator passes" in r["sample"]
    elif kind == "formk":
        w = inputs.small_case(nz=8, nx=7)
        r = bench.oracle_formk_sample(w, 1, passes=3)
        assert "3 paper-literal operator passes" in r["sample"]
    else:
        w = inputs.small_case(nz=8, nx=7)
        r = bench.oracle_gmres_sample(w, 1, restart=5)
        steps = int(r["sample"].split("Arnoldi steps")[0].split(",")[-1])
        passes = int(r["sample"].split("operator passes")[0].split(",")[-1])
        assert passes >= steps + 2  # at least one residual pass per cycle and the final check
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["unit"] == bench.UNIT
    assert r["value"] > 0 and r["seconds"] > 0


def test_oracle_sample_of_the_uneven_batch():
    """One oracle pass per distinct grid size, weighted by each size's cells in the batch."""
    ws = [inputs.small_case(nz=8, nx=7), inputs.small_case(nz=12, nx=10), inputs.small_case(nz=8, nx=7, seed=3)]
    r = bench.oracle_uneven_sample(ws)
    assert r["sample"].count("x") >= 2 and "8x7" in r["sample"] and "12x10" in r["sample"]
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0
