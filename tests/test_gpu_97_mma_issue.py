"""The tensor core's issue rate for the product kernel's instruction shapes, a measurement the
kernel's design notes rest on: tests/probe_mma_issue.cu, built with nvcc for sm_103a and run once
with one CTA per SM.  It checks that an A operand copied into TMEM (tcgen05.cp) gives the same
product as one read from shared memory, and that two issuing warps reach a higher MMA rate than
one (one thread issues one 128x128x16 MMA about every 117 cycles; the tensor core takes 64)."""
import os
import re
import subprocess
import tempfile

import pytest

from gpu_helpers import cuda_or_fail, torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def test_mma_issue_rate_and_tmem_operand():
    cuda_or_fail()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "probe_mma_issue")
        subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-std=c++17", "-o", exe, os.path.join(HERE, "probe_mma_issue.cu")],
                       check=True, capture_output=True)
        run = subprocess.run([exe, str(sms)], capture_output=True, text=True, timeout=300)
    print(run.stdout)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "16384 of 16384 elements bitwise equal" in run.stdout
    cyc = {name.strip(): float(c) for name, c in
           re.findall(r"^(.*?)\s+grid \d+: ([\d.]+) cycles per MMA", run.stdout, re.M)}
    one, two = cyc["A,B smem N=128"], cyc["N=128, 2 issuing warps"]
    assert two < 0.75 * one, cyc
