"""Host-side checks of the C library that need no GPU: it builds, loads,
exports every function include/tcm.h declares, and rejects bad arguments
(including the CFL bound of Eq. 4) before touching a device."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1702_00216_gb300 import build as B
from paper_1702_00216_gb300 import tcm
from paper_1702_00216_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return tcm.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tcm_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(tcm.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", tcm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (tcm_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    for name in declared_functions():
        assert hasattr(lib, name)


def test_slot_bytes(lib):
    assert tcm.tcm_slot_bytes((8, 8, 8)) == 2 * 512 * 4
    # every supported shape, every storage (two halves per box)
    for brick, n in (((4, 4, 4), 64), ((8, 8, 8), 512), ((16, 8, 8), 1024)):
        assert tcm.tcm_slot_bytes(brick, tcm.TCM_STORAGE_F32) == 2 * n * 4
        # 16-bit: two field halves plus the velocity array
        assert tcm.tcm_slot_bytes(brick, tcm.TCM_STORAGE_BF16) == 3 * n * 2
        assert tcm.tcm_slot_bytes(brick, tcm.TCM_STORAGE_F16) == 3 * n * 2
    for bad in ((8, 8, 16), (4, 4, 8), (2, 2, 2)):
        with pytest.raises(tcm.TCMError):
            tcm.tcm_slot_bytes(bad)
        # a batch of mixed storages: boxes sized for binary32
        assert tcm.tcm_slot_bytes(brick, tcm.TCM_STORAGE_MIXED) == 2 * n * 4
    with pytest.raises(tcm.TCMError):
        tcm.tcm_slot_bytes((8, 8, 8), 4)
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_slot_bytes((8, 8, 4))
    assert e.value.status == tcm.TCM_EINVAL


def _opts(**kw):
    o = tcm.tcm_options()
    o.pool_bytes = kw.get("pool_bytes", 1 << 20)
    o.decay_alpha = 1.0
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("courant,expect", [(0.58, tcm.TCM_ECFL), (0.6, tcm.TCM_ECFL)])
def test_create_rejects_cfl_violation(lib, courant, expect):
    """Eq. 4: c dt / dx <= 1/sqrt(3), checked on the largest velocity."""
    media = W.Media(kind="rules", c_background=1.0, spheres=[(4, 4, 4, 2.0, 2.0)])
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_create((16, 16, 16), media, 1.0, courant / 2.0, 0.0, (8, 8, 8), _opts())
    assert e.value.status == expect
    dense = W.dense_media(np.full((8, 8, 8), 1.0, np.float32))
    dense.c[3, 3, 3] = 3.0
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_create((8, 8, 8), dense, 1.0, courant / 3.0, 0.0, (8, 8, 8), _opts())
    assert e.value.status == expect


@pytest.mark.parametrize("where", [0, 4_000_000, 16 * 1024 * 1024 - 1])
def test_dense_model_scan_split_over_threads(lib, where):
    """A dense model of 2^24 nodes is scanned in chunks on several host
    threads: one bad value or one too-fast node anywhere (first, middle,
    last chunk) is still found."""
    shape = (256, 256, 256)
    c = np.full(shape, 1.0, np.float32)
    flat = c.reshape(-1)
    for value, expect in ((np.nan, tcm.TCM_EINVAL), (np.inf, tcm.TCM_EINVAL), (-0.5, tcm.TCM_EINVAL),
                          (1.2, tcm.TCM_ECFL)):
        flat[where] = value
        with pytest.raises(tcm.TCMError) as e:
            tcm.tcm_create(shape, W.dense_media(c), 1.0, 0.5, 0.0, (8, 8, 8), _opts())
        assert e.value.status == expect, (value, where)
        flat[where] = 1.0


@pytest.mark.parametrize("where", [0, 3, 7, 1_000_003, 107 * 103 * 101 - 1])
def test_dense_model_scan_any_lane_and_the_tail(lib, where):
    """The scan keeps eight running maxima: a bad value or a too-fast node in
    any of them, or in the last nodes of a count that is not a multiple of
    eight, is still found."""
    shape = (101, 103, 107)
    c = np.full(shape, 1.0, np.float32)
    flat = c.reshape(-1)
    for value, expect in ((np.nan, tcm.TCM_EINVAL), (-0.5, tcm.TCM_EINVAL), (1.2, tcm.TCM_ECFL)):
        flat[where] = value
        with pytest.raises(tcm.TCMError) as e:
            tcm.tcm_create(shape, W.dense_media(c), 1.0, 0.5, 0.0, (8, 8, 8), _opts())
        assert e.value.status == expect, (value, where)
        flat[where] = 1.0


@pytest.mark.parametrize("bad", ["shape", "dx", "dt", "thr", "brick", "decay", "mode", "cneg",
                                 "pool"])
def test_create_rejects_bad_arguments(lib, bad):
    shape, dx, dt, thr, brick = (16, 16, 16), 1.0, 0.5, 0.0, (8, 8, 8)
    media = W.homogeneous(1.0)
    kw = {}
    if bad == "shape":
        shape = (0, 16, 16)
    elif bad == "dx":
        dx = 0.0
    elif bad == "dt":
        dt = -1.0
    elif bad == "thr":
        thr = -1.0
    elif bad == "brick":
        brick = (8, 8, 7)
    elif bad == "decay":
        kw["decay_steps"] = -1
    elif bad == "mode":
        kw["threshold_mode"] = 7
    elif bad == "cneg":
        media = W.homogeneous(-1.0)
    elif bad == "pool":
        kw["pool_bytes"] = 100
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_create(shape, media, dx, dt, thr, brick, _opts(**kw))
    assert e.value.status == tcm.TCM_EINVAL


def test_status_strings(lib):
    assert tcm.tcm_status_string(tcm.TCM_OK) == "ok"
    assert "CFL" in tcm.tcm_status_string(tcm.TCM_ECFL)
    assert tcm.tcm_status_string(99) == "unknown status"


def test_no_cpu_fallback_without_gpu(lib):
    """A valid simulation needs the GPU: without one, create fails loudly."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tcm.TCMError) as e:
        tcm.tcm_create((16, 16, 16), W.homogeneous(1.0), 1.0, 0.5, 0.0, (8, 8, 8), _opts())
    assert e.value.status == tcm.TCM_EDEVICE


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1702_00216_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "tcm_oracle" not in txt, f


def test_option_struct_layout_matches_header(tmp_path):
    """The binding's ctypes mirrors of tcm_options and tcm_batch_options have
    the C layout of include/tcm.h (sizes and every field offset, read from a
    C program compiled against the header)."""
    import ctypes
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tcm.h"', "int main(void) {"]
    for ct, c_name in ((tcm.tcm_options, "tcm_options"), (tcm.tcm_batch_options, "tcm_batch_options")):
        lines.append(f'printf("{c_name} size %zu\\n", sizeof({c_name}));')
        for f, _ in ct._fields_:
            lines.append(f'printf("{c_name} {f} %zu\\n", offsetof({c_name}, {f}));')
    lines.append("return 0; }")
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            name, field, val = ln.split()
            got[(name, field)] = int(val)
    for ct, c_name in ((tcm.tcm_options, "tcm_options"), (tcm.tcm_batch_options, "tcm_batch_options")):
        assert got[(c_name, "size")] == ctypes.sizeof(ct)
        for f, _ in ct._fields_:
            assert got[(c_name, f)] == getattr(ct, f).offset, (c_name, f)


def test_barrier_selftest_rejects_bad_arguments(lib):
    """Argument checks of the barrier self-test come before any device call."""
    for kw in ({"skew": 2}, {"skew": -1}, {"timeout_s": 0.0}, {"timeout_s": 2.0}):
        args = {"skew": 0, "timeout_s": 0.05}
        args.update(kw)
        assert tcm.tcm_barrier_selftest(0, **args)[0] == tcm.TCM_EINVAL
