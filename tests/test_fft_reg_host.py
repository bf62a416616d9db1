"""The register-resident FFT plans of the CUDA kernels, run on the CPU (no GPU needed).

`tests/native/fft_reg_host.cu` compiles the kernels' __host__ __device__ plan code for the host
and runs every line with one std::thread per GPU lane and a std::barrier for the line's exchange
barrier. The outputs must equal numpy's FFT (the definition of the DFT: exp(-2 pi i jk/L) forward,
exp(+2 pi i jk/L) inverse, unnormalised) to the rounding of the precision, for every supported
length, both radix orders, the zero-half first pass and the inverse, with one line per thread
group and with two, three and four lines sharing the group's twiddle powers (as the column passes
transform a column's components, and at FFT length 1024 both parities of both, together); two
runs must agree bit for bit (a missing barrier between the lanes' stores and loads shows up as a
run-to-run difference); and the guard slots around each line must stay untouched (the harness
checks them)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "fft_reg_host.cu")


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cc = _nvcc()
    if cc is None:
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("fft_reg_host")
    exe = str(out / "fft_reg_host")
    cmd = [cc, "-std=c++20", "-O0", "--expt-relaxed-constexpr", "-diag-suppress", "20014",
           "-gencode", "arch=compute_103a,code=sm_103a", SRC, "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe, out


def _run(exe, path):
    res = subprocess.run([exe, str(path)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    return open(path, "rb").read()


def _cases(blob):
    off, cases = 0, []
    while off < len(blob):
        cb, L, V, inv, hin, nlt = (int(v) for v in np.frombuffer(blob[off:off + 24], dtype=np.int32))
        off += 24
        x = np.frombuffer(blob[off:off + 16 * L], dtype=np.complex128)
        off += 16 * L
        y = np.frombuffer(blob[off:off + 16 * L], dtype=np.complex128)
        off += 16 * L
        cases.append((cb, L, V, bool(inv), bool(hin), nlt, x, y))
    return cases


def test_register_plans_equal_the_dft(harness):
    exe, out = harness
    cases = _cases(_run(exe, out / "a.bin"))
    lengths = (16, 32, 64, 128, 256, 512, 1024)
    assert len(cases) == 2 * len(lengths) * (6 + 2 * 2 + 2 * 3 + 2 * 4)
    seen = set()
    for cb, L, V, inv, hin, nlt, x, y in cases:
        seen.add((cb, L, V, inv, hin, nlt))
        if hin:
            assert not np.any(x[L // 2:]), (L, V)
        want = L * np.fft.ifft(x) if inv else np.fft.fft(x)
        err = np.linalg.norm(y - want) / np.linalg.norm(want)
        assert err <= (1e-6 if cb == 8 else 1e-14), (cb, L, V, inv, hin, err)
    single = {(cb, L, V, inv, hin, 1) for cb in (8, 16) for L in lengths for V in (0, 1)
              for inv, hin in ((False, False), (False, True), (True, False))}
    grouped = {(cb, L, V, inv, hin, n) for cb in (8, 16) for L in lengths
               for V, inv, hin, n in ((0, False, True, 2), (1, True, False, 2), (0, False, True, 3), (0, True, False, 3),
                                   (0, False, False, 4), (0, True, False, 4))}
    assert seen == single | grouped


def test_register_plans_are_deterministic(harness):
    exe, out = harness
    assert _run(exe, out / "b.bin") == _run(exe, out / "c.bin")
