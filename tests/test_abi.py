"""The C-ABI library loads and exports every entry point declared in
include/hjbp.h (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hjbp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hjbp_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1109_3577_gb300 import build as b

    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("hjbp_create", "hjbp_solve", "hjbp_get_values", "hjbp_get_labels", "hjbp_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_calls_need_no_gpu(lib):
    import paper_1109_3577_gb300 as pkg

    assert pkg.hjbp_version() >= 100
    assert isinstance(pkg.hjbp_last_error(), str)


def test_create_rejects_bad_descriptors(lib):
    """Validation happens before any device work, so it runs on CPU."""
    import numpy as np

    import paper_1109_3577_gb300 as pkg
    import workloads as W

    p = W.sincos2d(0, n=65, n_coarse=17)
    bad = [
        p.with_(dim=4),
        p.with_(n=(2, 65, 1)),
        p.with_(controls=np.zeros((0, 2))),
        p.with_(controls=p.controls * 2.0),
        p.with_(targets=np.zeros((0, 3))),
        p.with_(tol=0.0),
        p.with_(hi=(2.0, 3.0, 0.0)),
        p.with_(n_coarse=(129, 129, 1)),
    ]
    for q in bad:
        d, keep = pkg.desc_from_problem(q)
        with pytest.raises(pkg.HjbpError) as ei:
            pkg.hjbp_create(d, 0, None)
        assert ei.value.status == 1, q
    # patch-boundary options and control cones need a patchy solve; cones need
    # r >= 1 and at most 64 controls in 2D
    g = p.with_(n_coarse=None)
    bad_opts = [
        (g, {"flags": pkg.HJBP_FLAG_DIRICHLET}),
        (g, {"flags": pkg.HJBP_FLAG_WARM_START}),
        (g, {"reduce_r": 4.0}),
        (p, {"reduce_r": 0.5}),
        (p, {"reduce_r": float("nan")}),
        (p.with_(controls=W.controls_2d(128)), {"reduce_r": 4.0}),
        # cones are defined on unit controls
        (W.brockett3d(n=17, n_coarse=9), {"reduce_r": 4.0}),
        # s = 2 against the wind w = (2, 0): the control (-1, 0) cannot move
        (W.zermelo(n=33, n_coarse=9, n_c=8, parts=4, s=2.0), {}),
    ]
    for q, kw in bad_opts:
        d, keep = pkg.desc_from_problem(q, **kw)
        with pytest.raises(pkg.HjbpError) as ei:
            pkg.hjbp_create(d, 0, None)
        assert ei.value.status == 1, kw


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1109_3577_gb300 import _binding

    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "_LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _binding.library()


def test_autotune_reads_its_cache_file_without_a_gpu(lib, tmp_path):
    """A problem class already in the cache file is answered from it, with no
    solve (so no GPU): the class key is (dim, round(log2(cells per side)),
    round(log2(controls)), patchy, options)."""
    import math

    import paper_1109_3577_gb300 as pkg
    import workloads as W

    p = W.sincos2d(0, n=513, n_coarse=33, n_c=48)
    d, keep = pkg.desc_from_problem(p, flags=pkg.HJBP_FLAG_WARM_START)
    key = (2, round(math.log2(512)), round(math.log2(48)), 1, pkg.HJBP_FLAG_WARM_START)
    path = tmp_path / "tune.txt"
    path.write_text("%d %d %d %d %d 3 4 0 0\n" % key)
    tune, cached = pkg.hjbp_autotune(d, 0, str(path))
    assert cached and tune == [3, 4, 0, 0]
    # a NULL descriptor or output is EINVAL (1), not a crash
    fn = lib.hjbp_autotune
    fn.argtypes = [ctypes.c_void_p] * 5
    fn.restype = ctypes.c_int
    assert fn(None, None, None, None, None) == 1


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "hjbp.h"
int main(void) {
    hjbp_problem_desc d;
    hjbp_plan *plan = (hjbp_plan *)&d;
    hjbp_status s;
    printf("version %d\n", hjbp_version());
    memset(&d, 0, sizeof d);
    d.dim = 4;
    s = hjbp_create(&d, NULL, NULL, &plan);
    printf("create %d null_out %d msg %s\n", (int)s, plan == NULL, hjbp_last_error());
    s = hjbp_create(NULL, NULL, NULL, &plan);
    printf("null_desc %d\n", (int)s);
    return 0;
}
"""


def test_plain_c_program_uses_the_abi(lib, tmp_path):
    """The header is plain C11 (compiles with -Wall -Wextra -pedantic -Werror)
    and a C program links the library and gets statuses and messages back
    without Python or a GPU."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.join(root, "paper_1109_3577_gb300")
    src, exe = tmp_path / "abi.c", tmp_path / "abi"
    src.write_text(C_PROGRAM)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I" + os.path.join(root, "include"), str(src), "-L" + libdir, "-lhjbp",
                           "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.splitlines()
    assert out[0] == "version 100"
    assert out[1] == "create 1 null_out 1 msg dim must be 2 or 3"
    assert out[2] == "null_desc 1"
