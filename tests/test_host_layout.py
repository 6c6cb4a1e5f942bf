"""Host-only consistency of the kernel's shared-memory layout and launch shapes.

`host_layout_check.cu` is compiled with nvcc and run on the host (it makes no
CUDA calls): the kernel's carve of dynamic shared memory must end exactly where
the host's size formula says, with every region aligned for its type and large
enough for the indices the kernel uses, for both samplers (the N -> infinity
sampler adds per-term clocks), both precisions, rings and chains, and every
launch variant the host can pick must fit 227 KB per CTA and hold the SVD
working matrix it promises."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_shared_memory_carve_and_launch_shapes(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "host_layout_check")
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "host_layout_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    assert int(r.stdout.split()[1]) > 1000
