"""Resource check of the hot kernels on the CPU: the sm_103a build's ptxas
report (-Xptxas -v, registers and spills as the assembler prints them) must
show no register spills in the kernels the default solve spends its time in,
so that a change that makes them spill fails here before any GPU run."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# mangled-name prefixes of the kernels of the default 2D and 3D solves
HOT = {
    "kernels2d.cu": ["_ZN4hjbp9k_value2dIfLi8ELb0ELb0E",   # value sweep, FP32, 8-class pair form
                     "_ZN4hjbp7k_phi2dILi4ELb0E",          # colour transport, bulk
                     "_ZN4hjbp9k_reach2d", "_ZN4hjbp10k_polish2d", "_ZN4hjbp12k_feedback2d",
                     "_ZN4hjbp12k_schedule2d"],
    "kernels3d.cu": ["_ZN4hjbp9k_value3dIf", "_ZN4hjbp7k_phi3d", "_ZN4hjbp9k_reach3d",
                     "_ZN4hjbp10k_polish3d", "_ZN4hjbp12k_feedback3d"],
}


def _report(src, out):
    from paper_1109_3577_gb300 import build as b

    cmd = [b.nvcc(), *b.ARCH, *b.FLAGS, "-Xptxas", "-v", "-c", os.path.join(b.CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    kernels, name = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and name:
            kernels.setdefault(name, {})["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            kernels.setdefault(name, {})["regs"] = int(m.group(1))
    return kernels


@pytest.mark.parametrize("src", sorted(HOT))
def test_hot_kernels_do_not_spill(src, tmp_path):
    try:
        from paper_1109_3577_gb300 import build as b
        b.nvcc()
    except Exception as e:   # pragma: no cover
        pytest.skip(f"no nvcc: {e}")
    kernels = _report(src, str(tmp_path / "k.o"))
    for prefix in HOT[src]:
        hits = {k: v for k, v in kernels.items() if k.startswith(prefix)}
        assert hits, f"{prefix}: not in the ptxas report"
        for k, v in hits.items():
            assert v.get("spill", 0) == 0, f"{k} spills {v['spill']} bytes"
            assert 0 < v.get("regs", 0) <= 255, (k, v)
