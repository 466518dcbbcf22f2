"""Register budgets of the step kernels (CPU: nvcc -Xptxas -v, no GPU needed).

The real-field step keeps four r2c / five c2r plane blocks and two k-space
blocks per SM, the row-fused k-space pass four blocks; a kernel that grows past
its register budget loses a resident block and the step slows by a third, so
the budgets are checked at build time.
"""
import os
import re
import shutil
import subprocess

import pytest

from paper_2010_00409_gb300 import build

CSRC = os.path.join(os.path.dirname(build.__file__), "csrc")

# (source, kernel-name pattern, max registers[, max spill bytes])
BUDGETS = [
    ("plane_rc.cu", r"plane_r2c_kernel", 64),
    ("plane_rc.cu", r"plane_c2r_kernel", 48),
    ("kspace_tma.cu", r"kspace_tma_kernelIfLi16ELi16ELi8ELi2ELb0ELb1ELb0E", 128),   # real-field step
    ("kspace_tma.cu", r"kspace_tma_kernelIfLi16ELi16ELi8ELi2ELb0ELb0ELb0E", 128),   # complex step
    ("gemm.cu", r"gemm_tma_kernel", 64),
    ("kspace_rows.cu", r"kspace_rows_kernelIfLi32ELi32E", 80, 8),                  # 1024-point rows, four blocks per SM
]


def ptxas_report(src):
    if not shutil.which(build.nvcc()) and not os.path.exists(build.nvcc()):
        pytest.skip("nvcc not found")
    cmd = [build.nvcc()] + build.ARCH + build.NVCC_FLAGS + ["-Xptxas", "-v", "-c", os.path.join(CSRC, src),
                                                            "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    entries, cur = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
            entries[cur] = {}
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and cur:
            entries[cur]["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            entries[cur]["regs"] = int(m.group(1))
    return entries


@pytest.mark.parametrize("src", sorted({b[0] for b in BUDGETS}))
def test_step_kernels_keep_their_register_budgets(src):
    entries = ptxas_report(src)
    for b in BUDGETS:
        s, pat, cap = b[:3]
        max_spill = b[3] if len(b) > 3 else 0
        if s != src:
            continue
        hits = {k: v for k, v in entries.items() if re.search(pat, k)}
        assert hits, pat
        for name, v in hits.items():
            assert v.get("regs", 0) <= cap, (pat, v)
            assert v.get("spill", 0) <= max_spill, (pat, v)
