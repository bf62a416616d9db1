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
    the GPU arm on its workload (the 512 x 512 gradient batch), the oracle as the CPU baseline on
    every host core (kind, cores, sample) and an e2e object with no host-device traffic."""
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "vti512x512_64src_6f_misfit"
    assert (d["config"]["nz"], d["config"]["lz"], d["config"]["problems_per_gpu"]) == (512, 1024, 384)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["sample"]
    assert cb["value"] == d["value"]
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


def test_column_kernel_units_on_the_512_workload():
    """512 x 512 cells, 1024 x 1024 FFT grid, 64 sources x 6 frequencies (384 problems):
    flops: 2 x 2 x 1024 columns x 5 * 1024 * 10 = 209,715,200 plus 28 x 1024^2 = 29,360,128, per
    cell 912; bytes: T read and written 2 x 2 x 512 x 1024 x 8 = 16,777,216 plus 3 x 1024^2 x 8 of
    each frequency over its 64 sources = 393,216, per cell 65.5."""
    w = bench.workload("vti512")
    assert (w.nz, w.nx, w.lz, w.lx, w.nf, w.n_problems) == (512, 512, 1024, 1024, 6, 384)
    assert bench.cols_flops_per_cell_apply(w) == pytest.approx(239_075_328 / 262_144, rel=1e-12)
    assert bench.cols_bytes_per_cell_apply(w) == pytest.approx(17_170_432 / 262_144, rel=1e-12)


def test_accuracy_block():
    """The accuracy block's relative errors on stand-in values: a wavefield off by 1e-6 relative
    gives 1e-6, and the gradient error is per parameter."""
    import numpy as np
    w = inputs.small_case(nz=6, nx=5, n_src=2, freqs=(5.0, 9.0))
    rng = np.random.default_rng(0)
    u = rng.normal(size=(2, 2, 6, 5)) + 1j * rng.normal(size=(2, 2, 6, 5))
    d_obs = (rng.normal(size=(w.n_problems, 3, 2)) * (1 + 1j)).astype(np.complex64)
    rr = rng.normal(size=(2, 3, 2)) + 0j
    g = rng.normal(size=(5, 6, 5))
    res = [{"b": b, "u": u[k], "d": rr[k] + d_obs[b], "r": rr[k], "passes": 7, "relres": (1e-13, 1e-13),
            "seconds": 1.0, "freq_hz": 5.0, "source": 0} for k, b in enumerate((0, 3))]
    gpu = {"u": u * (1 + 1e-6), "r": rr.copy(), "g": g * (1 + np.array([0, 0, 2e-5, 0, 0]))[:, None, None]}
    acc = bench.accuracy_block(w, gpu, res, g, d_obs)
    assert acc["wavefield_max"] == pytest.approx(1e-6, rel=1e-6)
    assert acc["residual_max"] == 0.0 and acc["data_max"] < 1e-15
    assert acc["gradient_subbatch"]["C13"] == pytest.approx(2e-5, rel=1e-6)
    assert acc["gradient_subbatch"]["rho"] == 0.0 and acc["gradient_max"] == acc["gradient_subbatch"]["C13"]


def test_cpp_oracle_legs_on_a_small_workload():
    """The C++ oracle legs of the benchmark on a small workload: the accuracy reference returns each
    sampled problem's wavefield, data and residual and the sub-batch gradient, and the baseline
    reports its rate on the cores it used."""
    import numpy as np
    w = inputs.small_case(nz=10, nx=9, n_src=3, freqs=(6.0, 11.0), vti=True, seed=4)
    d_obs = bench.synthetic_data(w)
    acc, base = bench.run_cpp_oracle(w, d_obs, [0, w.n_problems - 1], True, cores=3)
    res, g = acc
    assert [r["b"] for r in res] == [0, w.n_problems - 1] and g.shape == (5, w.nz, w.nx)
    assert all(np.allclose(r["d"] - r["r"], d_obs[r["b"]], rtol=0, atol=1e-16) for r in res)
    assert base["cores"] == 1 and base["value"] > 0 and base["kind"] == "oracle" and "C++17" in base["sample"]


def test_operator_stage_bytes():
    """Algorithmic bytes per cell-apply of the ls_apply stages: 512^2 on L = 1024 (split rows: the
    source field out and back in), 256^2 on L = 512."""
    b = bench.operator_stage_bytes(bench.workload("vti512"))
    assert b == {"rows_forward": 80.0, "cols": 64.0 + 96 * 6 / 384, "rows_inverse": 64.0}
    b = bench.operator_stage_bytes(bench.workload("vti256"))
    assert b == {"rows_forward": 48.0, "cols": 64.0 + 96 * 8 / 256, "rows_inverse": 64.0}


def test_path_roofline_units_and_bound():
    """The path's own roofline on the 512^2 workload (L = 1024, 384 problems, 6 frequencies), by hand:
    rows forward and inverse over 512 rows, 2 components, 5 * 1024 * 10 flops each = 400 per cell;
    the columns 912 (as for the column kernel); compulsory bytes u 16 + out 16 + the Green's spectra
    3 * 1024^2 * 8 * 6 / (384 * 512^2) = 1.5 + the contrast 20 / 384."""
    w = bench.workload("vti512")
    assert bench.pass_flops_per_cell_apply(w) == pytest.approx(1312.0, rel=1e-12)
    assert bench.compulsory_bytes_per_cell_apply(w) == pytest.approx(33.5 + 20 / 384, rel=1e-12)
    # 1312 flops at 65.6 TFLOP/s: 5e10 cell-applies/s; 33.55 B at 6710 GB/s: 2e11, so the ALU bounds it
    r = bench.path_roofline(w, 262_144 / 2.5e10 * 1e6, 1.0e10, 65.6, 6710.0)
    assert r["bound"] == "alu" and r["alu_bound"] == pytest.approx(5e10, rel=1e-12)
    assert r["pass_achieved"] == pytest.approx(2.5e10, rel=1e-12)
    assert r["pass_frac"] == pytest.approx(0.5, rel=1e-12) and r["step_frac"] == pytest.approx(0.2, rel=1e-12)
    # with a slow memory the HBM side bounds it
    r = bench.path_roofline(w, 10.0, 1.0e9, 65.6, 100.0)
    assert r["bound"] == "hbm" and r["hbm_bound"] == pytest.approx(100e9 / (33.5 + 20 / 384), rel=1e-12)
