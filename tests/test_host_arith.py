"""Device code that compiles for the host too, checked without a GPU in small
host programs built with nvcc:

- the arithmetic helpers (fixed-point rounding of the cell sums and the
  dispersion, the 2-byte weight rounding, the Eq. 3/4 velocity encoder, the
  register FFTs) against their plain definitions (host/arith_check.cu);
- the tile kernel's index arithmetic (shared-memory swizzles, the tiling of
  the coarse mesh, own and halo cells, the carving of shared memory) and its
  prologue and deposit phases run thread by thread on host arrays: the staged
  halo table and long-range force window against a plain periodic CIC
  gather, the fine density bit for bit against a plain integer CIC deposit
  of a clustered box, the force on the output nodes against a plain
  float64 DFT convolution with a packed symmetric table, and the
  interpolation, kick, drift and fused new-cell sums against a plain gather,
  and the low-memory tile pass against the default pass (host/tile_check.cu)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _run_host_check(tmp_path_factory, name):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp(name) / name)
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "host", name + ".cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        key, cases, fails, *rest = line.split()
        res[key] = (int(cases), int(fails), float(rest[0]) if rest else 0.0)
    return res


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    return _run_host_check(tmp_path_factory, "arith_check")


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    return _run_host_check(tmp_path_factory, "tile_check")


@pytest.mark.parametrize("name", ["fix24", "moments", "round_half_even"])
def test_integer_rounding_matches_definition(results, name):
    cases, fails, _ = results[name]
    assert cases > 1_000_000 and fails == 0


def test_encode_matches_definition(results):
    # Eq. 4 guess + one edge comparison each side = the bin count of Eq. 3,
    # at every edge and its float neighbours, specials and random floats
    cases, fails, _ = results["encode"]
    assert cases > 1_000_000 and fails == 0


@pytest.mark.parametrize("name", ["fft_dit", "rfft32"])
def test_register_ffts_match_the_dft(results, name):
    _, _, err = results[name]
    assert err < 1e-6, err


@pytest.mark.parametrize("name", ["swizzles", "tiling", "no_alias", "own_cells", "smem_layout"])
def test_tile_index_arithmetic(layout, name):
    cases, fails, _ = layout[name]
    assert cases > 0 and fails == 0, (cases, fails)


def test_tile_prologue_stages_halo_and_force_window(layout):
    # float32 CIC gather of values in [-1, 1] against the float64 gather
    cases, fails, err = layout["prologue"]
    assert cases > 1_000_000 and fails == 0 and err < 2e-6, (cases, fails, err)


def test_tile_deposit_matches_plain_cic(layout):
    # fine density bit-exact (1- and 2-byte positions, crowded cells past
    # both particle maps); parked long-range force within float32 rounding
    cases, fails, err = layout["deposit"]
    assert cases > 100_000 and fails == 0 and err < 2e-6, (cases, fails, err)


def test_tile_transforms_match_dft_convolution(layout):
    # forward transforms, packed Green multiply (including the kx = 0 / 16
    # pencil) and pruned inverse transforms, three force components, tiles of
    # 16 and 20 fine cells; error relative to the largest force value
    cases, fails, err = layout["spectral"]
    assert cases > 40_000 and fails == 0 and err < 1e-5, (cases, fails, err)


@pytest.mark.parametrize("mode", [0, 1])
def test_tile_interpolation_kick_drift(layout, mode):
    # mode 0: gathered force; mode 1: kicked momentum, drifted code (exact)
    # and the fused counts and momentum sums (exact); errors relative to the
    # field scale
    cases, fails, err = layout["interp_mode%d" % mode]
    assert cases > 50_000 and fails == 0 and err < 1e-6, (cases, fails, err)


def test_tile_lowmem_pass_matches_default_pass(layout):
    # new momenta bit for bit, counts and momentum sums, the 128-bit
    # dispersion sum (past 2^64), and the codes the low-memory re-encode
    # derives from the old store and the momenta: all exact
    cases, fails, _ = layout["lowmem"]
    assert cases > 100_000 and fails == 0, (cases, fails)


def test_tile_error_paths_flag_and_stay_in_bounds(layout):
    # a fine node past 2^32 units flags the overflow; every own particle's
    # long-range force is parked in its slot and no other slot is written
    cases, fails, _ = layout["error_paths"]
    assert cases > 1000 and fails == 0, (cases, fails)
