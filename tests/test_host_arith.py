"""The device arithmetic helpers that compile for the host too (fixed-point
rounding of the cell sums and the dispersion, the 2-byte weight rounding,
the register FFTs) against their plain definitions, in a small host program
built with nvcc (no GPU needed)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("arith") / "arith_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "host", "arith_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        name, cases, fails, *rest = line.split()
        res[name] = (int(cases), int(fails), float(rest[0]) if rest else 0.0)
    return res


@pytest.mark.parametrize("name", ["fix24", "sq_fix32", "round_half_even"])
def test_integer_rounding_matches_definition(results, name):
    cases, fails, _ = results[name]
    assert cases > 1_000_000 and fails == 0


@pytest.mark.parametrize("name", ["fft_dit", "rfft32"])
def test_register_ffts_match_the_dft(results, name):
    _, _, err = results[name]
    assert err < 1e-6, err
