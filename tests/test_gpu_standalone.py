"""Standalone checks of two kernels outside the engine, on synthetic data of the sampling
job's shapes (tests/standalone/*.cu, built here with nvcc for sm_103a):

* tc_stacked: the tensor-core batch step with its A operand read in place from stored
  blocks (Sec. I.C: the batch's closed legs select a block of a batch-independent
  tensor), stacked and unstacked tiles, C laid out with n or m lowest; six outputs per
  run against FP64 sums of the split planes (relative to sqrt(sum |a|^2 |b|^2), 1e-3).
* long_k: the long-K kernel (64 x 8 outputs, K = 2048, complex64) in its three warp
  layouts; one output against an FP64 host sum (1e-5).

The same programs time full-size launches and serve the small-case profiler captures.
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def binaries(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = tmp_path_factory.mktemp("standalone")
    built = {}
    procs = {}
    for name in ("tc_stacked", "long_k"):
        exe = str(out / name)
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
               os.path.join(HERE, "standalone", name + ".cu"), "-I" + os.path.join(ROOT, "include"), "-lcuda"]
        procs[name] = (subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True), exe)
    for name, (p, exe) in procs.items():
        log, _ = p.communicate(timeout=600)
        assert p.returncode == 0, "nvcc failed for %s:\n%s" % (name, log[-3000:])
        built[name] = exe
    return built


def run(exe, *args):
    r = subprocess.run([exe] + [str(a) for a in args], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout.splitlines()[-1]
    return r.stdout


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("layout", [0, 1])
def test_tc_batch_step_with_in_place_operand(binaries, variant, layout):
    # 256 rows, 4 x 1024 batches, 2^10 stored blocks (about four batches per block)
    out = run(binaries["tc_stacked"], 2, 8, variant, layout, 10, 8)
    if variant < 2:
        stacks = int(out.split("stacks ")[1].split(",")[0])
        # every block's batches in runs of S = 4 (variant 0) or 2 (variant 1)
        assert 1024 // (4 if variant == 0 else 2) <= stacks <= 1024


def test_tc_batch_step_every_batch_bit_a_batch_index(binaries):
    # no non-index batch bits (the 40-qubit job's (12,11,5,8) step): 1024 batches of 2048 rows
    out = run(binaries["tc_stacked"], 2, 11, 0, 1, 10, 8, 0)
    assert 1024 // 4 <= int(out.split("stacks ")[1].split(",")[0]) <= 1024


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_long_k_kernel_warp_layouts(binaries, variant):
    run(binaries["long_k"], 2, 8, variant)
